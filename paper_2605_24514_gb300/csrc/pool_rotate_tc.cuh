// Tensor-core rotations of the batched appends (Section 2.2 Step 3: U' = blkdiag(U, 1) U_K,
// V' = [V z_hat] V_K, and the transposed roles for column appends) for rank buckets 16 and 32.
//
// A row of U or V costs 2 k^2 FLOP for 8 k bytes of HBM traffic (read and write, FP32), k / 4
// FLOP per byte: at k = 32 streaming at HBM rate needs most of the FP32 pipes' peak, so the row
// tile times the k x k core factor runs as a dense contraction on tcgen05 with the accumulators
// in TMEM.
//
// Exact-accumulation split. FP32 accuracy from 16-bit tensor-core inputs is obtained by writing
// each operand in block fixed point and cutting it into three 8-bit digits (the splitting behind
// Ozaki's error-free matrix products): a row a of the tile with max |a| < 2^e is
//   a = 2^(e-8) (d0 + d1 / 2^8 + d2 / 2^16),   d0 in [-256, 256], d1, d2 in [-128, 128],
// the 24-bit fixed-point value of a rounded to nearest; likewise each column b of the core factor
// with its own exponent. Digits are exact in BF16, products of two digits are integers below
// 2^16, and the three digit-product levels
//   D0 = sum d0 b0,   D1 = sum (d0 b1 + d1 b0),   D2 = sum (d0 b2 + d1 b1 + d2 b0)
// are integers below 2^23 for K <= 32 terms: every partial sum the tensor core forms is exactly
// representable in its FP32 accumulator, so its internal rounding never acts. The row of the
// product is 2^(e_a + e_b - 16) ((D0 + D1 / 2^8) + D2 / 2^16), rounded to nearest in FP32 once; the
// dropped levels (D3, D4) and the fixed-point rounding are below 2^-24 relative to the inputs'
// magnitudes, as for an FP32 dot product, and unbiased.
//
// Work split. A rotation block is 128 rows of one side of one update (the warp kernel's block ->
// update tables, 128 rows per block for these buckets). Persistent CTAs of 128 threads (a few per
// SM) each take a contiguous range of blocks, so consecutive blocks mostly share their update and
// side and the core factor's digit planes are cut once per run of blocks. Per block:
//   1. the block's rows (the 32-row boxes of the stream's U or V that hold them, through the
//      pool's tensor map of that matrix: TMA loads, swizzled so that a thread reading its row
//      meets no bank conflicts) were brought into one of two shared-memory stages one block
//      ahead; the next block's loads are issued now;
//   2. if the update or side changed: the core factor (V_K or U_K; rows >= r and columns >= k_out
//      zeroed) is cut into digit planes (B operands, K-major) with per-column scales, four threads
//      per column;
//   3. each thread takes one row: z_hat = (z1_row - row . p2) / rho when the projection side gains
//      the new direction (z1 = x - P p1, the warp kernel's first-pass residual, computed there in
//      float-float; p2 its small second-pass correction), then the row's scale and digit planes;
//   4. thread 0 issues the six digit-product MMAs per K step of 16 (M = 128, N = KB, BF16, FP32
//      accumulation) into the three level accumulators (TMEM, allocated once per CTA) and commits
//      them to an mbarrier;
//   5. each warp loads its 32 lanes of the three accumulators (one row per thread), combines them,
//      adds z_hat times the core factor's last row, and stores the row to global memory (a warp's
//      stores fill its 32 rows' lines).
// Every wait is bounded in wall time; on a timeout the stream's sticky status gets kStTimeout and
// the CTA stops, waits (bounded) for its copies, frees its TMEM and returns.
#pragma once

#include "pool_rotate_tma.cuh"

namespace isvd {

constexpr int kTcRotRows = 128;                        // rows per CTA (one per thread)
constexpr int kTcRotThreads = kTcRotRows;

template <int KB>
struct TcRotLayout {
  static constexpr uint32_t kTile = kTcRotRows * KB * 4;      // FP32 staging tile (one stage)
  static constexpr uint32_t kAplane = kTcRotRows * KB * 2;    // one BF16 digit plane of the tile
  static constexpr uint32_t kBplane = KB * KB * 2;            // one BF16 digit plane of the core factor
  static constexpr uint32_t kOffA = 2 * kTile;                // two stages, then three A planes
  static constexpr uint32_t kOffB = kOffA + 3 * kAplane;      // three B planes
  static constexpr uint32_t kOffVec = kOffB + 3 * kBplane;    // z row, p hi, p lo, column scales
  static constexpr uint32_t kOffBar = kOffVec + 4 * KB * 4;   // mbarriers: two stages, MMA
  static constexpr uint32_t kOffTmem = kOffBar + 32;
  static constexpr uint32_t kBytes = kOffTmem + 16 + 1024;  // + room to align the base to 1 KiB
  static constexpr uint32_t kTmemCols = 3 * KB <= 32 ? 32 : 3 * KB <= 64 ? 64 : 128;  // three levels
  static constexpr uint32_t kSbo = 8 * KB * 2;                // bytes per 8-row group (16-bit elements)
};
constexpr int kTcCtasPerSm = 3;  // persistent CTAs per SM (shared memory allows three at KB = 32)

// Block fixed point: the exponent e with max |v| < 2^e, from the FP32 exponent field (max |v| in
// [2^(E-127), 2^(E-126)) for a normal value with biased exponent E), clamped below at -100 so that
// the scales 2^(24 - e) and 2^(e - 8) stay normal FP32 values; sets below 2^-100 (all-zero ones
// included) get digits that are zero or carry their values at an absolute 2^-124.
__device__ __forceinline__ int fixed_exponent(float amax) {
  const int E = (int)((__float_as_uint(amax) >> 23) & 0xFFu);
  return max(E - 126, -100);
}

// 2^(24 - e) as an FP32 value (a power of two; e is at most 128 for finite inputs).
__device__ __forceinline__ float fixed_scale(int e) { return __int_as_float((127 + 24 - e) << 23); }

// Round to the nearest integer (ties to even) for |x| < 2^22: adding and removing 1.5 * 2^23 puts
// the sum where the FP32 spacing is 1. Explicit round-to-nearest intrinsics keep the compiler from
// folding the pair.
__device__ __forceinline__ float round_int(float x) {
  return __fsub_rn(__fadd_rn(x, 12582912.f), 12582912.f);
}

// The three digits of v in units of 2^(e - 24), x = v 2^(24 - e) = sc * v (exact, |x| < 2^24):
// q0 = round(x / 2^16), q1 = round((x - q0 2^16) / 2^8), q2 = round(x - q0 2^16 - q1 2^8), so that
// q0 2^16 + q1 2^8 + q2 is x rounded to the nearest integer; every step is exact in FP32 except the
// intended roundings, and each digit is a small integer (|q0| <= 256, |q1|, |q2| <= 128).
__device__ __forceinline__ void digits3(float v, float sc, float& d0, float& d1, float& d2) {
  const float x = v * sc;
  d0 = round_int(x * (1.f / 65536.f));
  const float r1 = fmaf(-d0, 65536.f, x);
  d1 = round_int(r1 * (1.f / 256.f));
  d2 = round_int(fmaf(-d1, 256.f, r1));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  // The digits are small integers: exactly representable in BF16, so the upper halves of the FP32
  // bit patterns are their BF16 encodings (one byte permute).
  return __byte_perm(__float_as_uint(lo), __float_as_uint(hi), 0x7632);
}

// Thread 0: the TMA loads of block bk's rows (32-row boxes, only those holding live rows) into
// stage buffer dst, completing on bar.
template <int KB>
__device__ __forceinline__ void tc_issue_rows(const RotBlock<KB, kTcRotRows>& bk, const PoolOp* ops,
                                              const RowTensorMap* maps, float* dst, uint64_t* bar) {
  const int nbox = (bk.rows + kRowBoxRows - 1) / kRowBoxRows;
  tc::mbar_arrive_expect_tx(bar, (uint32_t)nbox * (kRowBoxRows * KB * 4));
  const void* tm = bk.tmap(ops, maps);
  tc::fence_tensormap_acquire(tm);
  for (int b = 0; b < nbox; ++b)
    tc::tma_load_2d(dst + b * kRowBoxRows * KB, tm, 0, (int)bk.base + b * kRowBoxRows, bar);
}

template <int KB>
__global__ void __launch_bounds__(kTcRotThreads)
    k_pool_rotate_tc(const PoolOp* __restrict__ ops, const RotScratch<KB>* __restrict__ scratch,
                     const int* __restrict__ chunk_start, const int* __restrict__ block_op, int nblocks,
                     const RowTensorMap* __restrict__ maps) {
  static_assert(KB == 16 || KB == 32, "tensor-core rotation buckets");
  using L = TcRotLayout<KB>;
  constexpr int C4 = KB / 4;  // float4 chunks per row
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // The swizzled TMA boxes need a 1 KiB aligned destination.
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  auto stage_buf = [&](int st_) { return reinterpret_cast<float*>(smem + (uint32_t)st_ * L::kTile); };
  unsigned char* Ad = smem + L::kOffA;
  unsigned char* Bd = smem + L::kOffB;
  float* zrow = reinterpret_cast<float*>(smem + L::kOffVec);
  float* p2 = zrow + KB;  // the second-pass projection p2 (z_hat = (z1 - row . p2) / rho)
  float* bscale = p2 + 2 * KB;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kOffBar);  // tile landed in stage 0 / 1
  uint64_t* mmab = full + 2;                                          // MMAs of a block completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmem);
  const int tid = threadIdx.x, warp = tid >> 5;

  const int per = (nblocks + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b1 = min(nblocks, ((int)blockIdx.x + 1) * per);
  int cur = rot_next_live<KB>(scratch, block_op, (int)blockIdx.x * per, b1);
  if (cur >= b1) return;  // uniform: nothing to rotate in this range

  if (tid == 0) {
    tc::mbar_init(&full[0], 1);
    tc::mbar_init(&full[1], 1);
    tc::mbar_init(mmab, 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::kTmemCols);
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;

  RotBlock<KB, kTcRotRows> blk;
  blk.locate(ops, scratch, chunk_start, block_op, cur);
  uint32_t use0 = 0u, use1 = 0u;              // completed loads per stage (mbarrier parity)
  bool inflight0 = false, inflight1 = false;  // a load issued into the stage and not yet waited for
  uint32_t mma_uses = 0;
  bool mma_inflight = false;
  if (tid == 0) tc_issue_rows<KB>(blk, ops, maps, stage_buf(0), &full[0]);
  inflight0 = true;
  int stage = 0, prev_e = -1;
  bool prev_side = false, failed = false;
  while (cur < b1) {
    const int nxt = rot_next_live<KB>(scratch, block_op, cur + 1, b1);
    RotBlock<KB, kTcRotRows> nb;
    if (nxt < b1) {
      nb.locate(ops, scratch, chunk_start, block_op, nxt);
      if (tid == 0) {
        // The other stage was last read by the previous block's row loads, before barriers since.
        tc::fence_proxy_async_smem();
        tc_issue_rows<KB>(nb, ops, maps, stage_buf(stage ^ 1), &full[stage ^ 1]);
      }
      if (stage) inflight0 = true;
      else inflight1 = true;
    }
    const RotScratch<KB>& sc = scratch[blk.e];
    const PoolOp& op = ops[blk.e];
    const int r = sc.r, k_out = sc.k_out;
    if (blk.e != prev_e || blk.pside != prev_side) {
      // The core factor's digit planes, B[n = jj][kk = c] from R[c][jj] (c < r, jj < k_out), four
      // threads per output column jj (rows split four ways), the column's exponent by shuffles.
      // The previous block's MMAs, the last readers of these planes, have completed.
      const float* src = blk.pside ? sc.RP : sc.RQ;
      constexpr int RPT = KB / 4;
      if (tid < 4 * KB) {
        const int jj = tid >> 2, sub = tid & 3;
        float v[RPT];
        float amax = 0.f;
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int c = sub * RPT + q;
          v[q] = (c < r && jj < k_out) ? src[c * KB + jj] : 0.f;
          amax = fmaxf(amax, fabsf(v[q]));
        }
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 2));
        const int eb = fixed_exponent(amax);
        if (sub == 0) bscale[jj] = __int_as_float((127 + eb - 8) << 23);
        const float scb = fixed_scale(eb);
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          float d0, d1, d2;
          digits3(v[q], scb, d0, d1, d2);
          const uint32_t o = tc::kmajor_offset16(jj, sub * RPT + q, KB);
          *reinterpret_cast<uint16_t*>(Bd + o) = (uint16_t)(__float_as_uint(d0) >> 16);
          *reinterpret_cast<uint16_t*>(Bd + L::kBplane + o) = (uint16_t)(__float_as_uint(d1) >> 16);
          *reinterpret_cast<uint16_t*>(Bd + 2 * L::kBplane + o) = (uint16_t)(__float_as_uint(d2) >> 16);
        }
      }
      if (tid < KB) {
        zrow[tid] = (blk.pside && tid < k_out) ? src[r * KB + tid] : 0.f;
        p2[tid] = tid < r ? sc.p2[tid] : 0.f;
      }
      prev_e = blk.e;
      prev_side = blk.pside;
    }
    const bool got = tc::mbar_wait_bounded(&full[stage], (stage ? use1 : use0) & 1u, kRotWaitNs);
    if (__syncthreads_or(!got)) {  // also: the B planes, scales, z row and p are complete
      failed = true;
      break;
    }
    if (stage) {
      use1++;
      inflight1 = false;
    } else {
      use0++;
      inflight0 = false;
    }

    // This thread's row (columns >= r are stale and count as zero).
    float* T = stage_buf(stage);
    const int row = tid;
    const bool live = row < blk.rows;
    const float4* T4 = reinterpret_cast<const float4*>(T);
    float xv[KB];
#pragma unroll
    for (int q = 0; q < C4; ++q) {
      // the swizzle spreads a warp's reads of chunk q over all banks
      const float4 a = live ? T4[row * C4 + rows_swz<KB>(row, q)] : make_float4(0.f, 0.f, 0.f, 0.f);
      xv[4 * q] = a.x;
      xv[4 * q + 1] = a.y;
      xv[4 * q + 2] = a.z;
      xv[4 * q + 3] = a.w;
    }
    float amax = 0.f;
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      if (c >= r) xv[c] = 0.f;
      amax = fmaxf(amax, fabsf(xv[c]));
    }
    float zh = 0.f;
    if (blk.withz && live) {
      float corr = 0.f;  // the row's entries beyond r are zero
#pragma unroll
      for (int c = 0; c < KB; ++c) corr = fmaf(xv[c], p2[c], corr);
      zh = (op.z1[blk.base + row] - corr) * sc.inv_rho;
    }
    const int ea = fixed_exponent(amax);
    const float ascale = __int_as_float((127 + ea - 8) << 23);
    const float sca = fixed_scale(ea);
#pragma unroll
    for (int g = 0; g < KB / 8; ++g) {  // one 16-byte core-matrix row per digit plane
      uint32_t w0[4], w1[4], w2[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float a0, a1, a2, c0, c1, c2;
        digits3(xv[8 * g + 2 * h], sca, a0, a1, a2);
        digits3(xv[8 * g + 2 * h + 1], sca, c0, c1, c2);
        w0[h] = pack_bf16x2(a0, c0);
        w1[h] = pack_bf16x2(a1, c1);
        w2[h] = pack_bf16x2(a2, c2);
      }
      const uint32_t o = tc::kmajor_offset16(row, 8 * g, KB);
      *reinterpret_cast<uint4*>(Ad + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
      *reinterpret_cast<uint4*>(Ad + L::kAplane + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
      *reinterpret_cast<uint4*>(Ad + 2 * L::kAplane + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    }
    tc::fence_proxy_async_smem();
    __syncthreads();

    // Level l accumulator at TMEM columns l * KB; per K step of 16 the digit pairs (i, j), i + j = l.
    if (tid == 0) {
      tc::tc_fence_after_sync();
      constexpr uint32_t idesc = tc::idesc_bf16(128, KB);
      const uint32_t a0 = tc::smem_u32(Ad), bb0 = tc::smem_u32(Bd);
#pragma unroll
      for (int sk = 0; sk < KB / 16; ++sk) {
        const uint32_t ko = (uint32_t)sk * 256u;  // two core matrices along K
        uint64_t da[3], db[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          da[i] = tc::smem_desc_kmajor(a0 + i * L::kAplane + ko, 128, L::kSbo);
          db[i] = tc::smem_desc_kmajor(bb0 + i * L::kBplane + ko, 128, L::kSbo);
        }
        const uint32_t acc = sk > 0 ? 1u : 0u;
        tc::mma_bf16(tmem, da[0], db[0], idesc, acc);
        tc::mma_bf16(tmem + KB, da[0], db[1], idesc, acc);
        tc::mma_bf16(tmem + KB, da[1], db[0], idesc, 1u);
        tc::mma_bf16(tmem + 2 * KB, da[0], db[2], idesc, acc);
        tc::mma_bf16(tmem + 2 * KB, da[1], db[1], idesc, 1u);
        tc::mma_bf16(tmem + 2 * KB, da[2], db[0], idesc, 1u);
      }
      tc::mma_commit(mmab);
    }
    mma_inflight = true;
    const bool done = tc::mbar_wait_bounded(mmab, mma_uses & 1u, kRotWaitNs);
    if (__syncthreads_or(!done)) {
      failed = true;
      break;
    }
    mma_uses++;
    mma_inflight = false;
    tc::tc_fence_after_sync();

    // Warp w reads TMEM lanes 32 w .. 32 w + 31: rows 32 w .. 32 w + 31 of the tile, its own rows.
    {
      const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
      float acc[KB], lv[KB];
      if constexpr (KB == 32) {
        tc::tmem_ld32(lane_addr + 2 * KB, acc);
        tc::tmem_ld32(lane_addr + KB, lv);
      } else {
        tc::tmem_ld16(lane_addr + 2 * KB, acc);
        tc::tmem_ld16(lane_addr + KB, lv);
      }
      // D1 + D2 / 2^8, rounded once: that rounding is scaled down by 2^-8 in the result below
#pragma unroll
      for (int j = 0; j < KB; ++j) acc[j] = fmaf(acc[j], 1.f / 256.f, lv[j]);
      if constexpr (KB == 32) tc::tmem_ld32(lane_addr, lv);
      else tc::tmem_ld16(lane_addr, lv);
#pragma unroll
      for (int j = 0; j < KB; ++j) {
        float y = fmaf(acc[j], 1.f / 256.f, lv[j]) * (ascale * bscale[j]);
        if (blk.withz) y = fmaf(zh, zrow[j], y);
        acc[j] = y;
      }
      if (live) {
        // straight to global memory: a warp's stores cover its 32 rows' 128-byte lines in C4 steps
        float4* W4 = reinterpret_cast<float4*>(blk.tile(ops) + (int64_t)row * KB);
#pragma unroll
        for (int q = 0; q < C4; ++q) W4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      }
    }
    tc::tc_fence_before_sync();
    __syncthreads();  // every warp is done with the accumulators
    stage ^= 1;
    cur = nxt;
    if (cur < b1) blk = nb;
  }
  if (failed && tid == 0) {
    atomicOr(&ops[blk.e].st->status, kStTimeout);
    // let the copies and MMAs in flight finish (bounded) before the CTA's memory goes away
    if (inflight0) tc::mbar_wait_bounded(&full[0], use0 & 1u, kRotWaitNs);
    if (inflight1) tc::mbar_wait_bounded(&full[1], use1 & 1u, kRotWaitNs);
    if (mma_inflight) tc::mbar_wait_bounded(mmab, mma_uses & 1u, kRotWaitNs);
  }
  tc::tc_fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after_sync();
    tc::tmem_dealloc(tmem, L::kTmemCols);
  }
}

}  // namespace isvd
