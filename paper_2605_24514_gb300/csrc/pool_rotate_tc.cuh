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
// One CTA of 128 threads handles 128 rows of one side of one update (the rotation block -> update
// tables of the warp kernel, with 128 rows per block for these buckets):
//   1. thread 0 starts one bulk copy (TMA) of the contiguous row tile (rows x KB FP32) into
//      shared memory; meanwhile the CTA cuts the core factor (V_K or U_K; rows >= r and columns
//      >= k_out zeroed) into digit planes (B operands, K-major) and per-column scales;
//   2. each thread takes one row: z_hat = (x_row - row . p) / rho in float-float when the
//      projection side gains the new direction, then the row's scale and digit planes (A operands);
//   3. thread 0 issues the six digit-product MMAs per K step of 16 (M = 128, N = KB, BF16, FP32
//      accumulation) into the three level accumulators and commits them to an mbarrier;
//   4. each warp loads its 32 lanes of the three accumulators (one row per thread), combines them,
//      adds z_hat times the core factor's last row, writes the row back into the staging tile, and
//      thread 0 stores the tile with one bulk copy.
// Every wait is bounded in wall time; on a timeout the stream's sticky status gets kStTimeout,
// the CTA waits (bounded) for its copies, frees its TMEM and returns.
#pragma once

#include "pool_warp.cuh"
#include "tc_ptx.cuh"

namespace isvd {

constexpr int kTcRotRows = 128;                        // rows per CTA (one per thread)
constexpr int kTcRotThreads = kTcRotRows;
constexpr uint64_t kTcWaitNs = 2000ull * 1000 * 1000;  // 2 s

template <int KB>
struct TcRotLayout {
  static constexpr uint32_t kTile = kTcRotRows * KB * 4;      // FP32 staging tile
  static constexpr uint32_t kAplane = kTcRotRows * KB * 2;    // one BF16 digit plane of the tile
  static constexpr uint32_t kBplane = KB * KB * 2;            // one BF16 digit plane of the core factor
  static constexpr uint32_t kOffA = kTile;                    // three A planes
  static constexpr uint32_t kOffB = kOffA + 3 * kAplane;      // three B planes
  static constexpr uint32_t kOffVec = kOffB + 3 * kBplane;    // z row, p hi, p lo, column scales
  static constexpr uint32_t kOffBar = kOffVec + 4 * KB * 4;   // two mbarriers
  static constexpr uint32_t kOffTmem = kOffBar + 16;
  static constexpr uint32_t kBytes = kOffTmem + 16;
  static constexpr uint32_t kTmemCols = 3 * KB <= 32 ? 32 : 3 * KB <= 64 ? 64 : 128;  // three levels
  static constexpr uint32_t kSbo = 8 * KB * 2;                // bytes per 8-row group (16-bit elements)
};

// Block fixed point: the exponent e with max |v| < 2^e (0 for an all-zero set).
__device__ __forceinline__ int fixed_exponent(float amax) {
  int e = 0;
  if (amax > 0.f) frexpf(amax, &e);
  return e;
}

// The three digits of v in units of 2^(e - 24): v 2^(24 - e) rounded to nearest, then cut.
__device__ __forceinline__ void digits3(float v, int e, float& d0, float& d1, float& d2) {
  const int si = __float2int_rn(ldexpf(v, 24 - e));  // |si| <= 2^24
  const int q0 = (si + (1 << 15)) >> 16;              // in [-256, 256]
  const int r1 = si - (q0 << 16);                     // in [-2^15, 2^15)
  const int q1 = (r1 + (1 << 7)) >> 8;                // in [-128, 128]
  const int q2 = r1 - (q1 << 8);                      // in [-128, 128)
  d0 = (float)q0;
  d1 = (float)q1;
  d2 = (float)q2;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  // The digits are small integers: exactly representable in BF16, so truncating the FP32 bit
  // pattern to its upper half is exact.
  return (__float_as_uint(lo) >> 16) | (__float_as_uint(hi) & 0xFFFF0000u);
}

template <int KB>
__global__ void __launch_bounds__(kTcRotThreads)
    k_pool_rotate_tc(const PoolOp* __restrict__ ops, const RotScratch<KB>* __restrict__ scratch,
                     const int* __restrict__ chunk_start, const int* __restrict__ block_op) {
  static_assert(KB == 16 || KB == 32, "tensor-core rotation buckets");
  using L = TcRotLayout<KB>;
  constexpr int C4 = KB / 4;  // float4 chunks per row
  extern __shared__ __align__(1024) unsigned char smem[];
  float* T = reinterpret_cast<float*>(smem);
  unsigned char* Ad = smem + L::kOffA;
  unsigned char* Bd = smem + L::kOffB;
  float* zrow = reinterpret_cast<float*>(smem + L::kOffVec);
  float* ph = zrow + KB;
  float* pl = ph + KB;
  float* bscale = pl + KB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kOffBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + L::kOffTmem);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int e = block_op[blockIdx.x];
  const RotScratch<KB>& sc = scratch[e];
  const int k_out = sc.k_out;
  if (k_out < 0) return;  // handed to the CTA kernel (uniform over the block)
  const PoolOp& op = ops[e];
  const bool is_row = op.kind == kRow;
  const int64_t nP = is_row ? op.n : op.m;
  const int64_t nQ = is_row ? op.m : op.n;
  const int cP = (int)((nP + kTcRotRows - 1) / kTcRotRows);
  const int ci = blockIdx.x - chunk_start[e];
  const bool pside = ci < cP;
  const int r = sc.r;
  const bool withz = pside && sc.grew;
  const int64_t nrows = pside ? nP : nQ;
  const int64_t base = (int64_t)(pside ? ci : ci - cP) * kTcRotRows;
  const int rows = (int)(nrows - base < kTcRotRows ? nrows - base : kTcRotRows);
  float* X = (pside ? (is_row ? op.V : op.U) : (is_row ? op.U : op.V)) + base * KB;
  const float* src = pside ? sc.RP : sc.RQ;
  const uint32_t tile_bytes = (uint32_t)rows * KB * 4;

  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, L::kTmemCols);
  tc::tc_fence_before_sync();
  __syncthreads();
  tc::tc_fence_after_sync();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bars[0], tile_bytes);
    tc::bulk_g2s(T, X, tile_bytes, &bars[0]);
  }
  // Step 1: the core factor's digit planes, B[n = jj][kk = c] from R[c][jj] (c < r, jj < k_out),
  // one output column per thread, with its own exponent.
  if (tid < KB) {
    const int jj = tid;
    float amax = 0.f;
    for (int c = 0; c < r; ++c) amax = fmaxf(amax, jj < k_out ? fabsf(src[c * KB + jj]) : 0.f);
    const int eb = fixed_exponent(amax);
    bscale[jj] = ldexpf(1.f, eb - 8);
    for (int c = 0; c < KB; ++c) {
      const float v = (c < r && jj < k_out) ? src[c * KB + jj] : 0.f;
      float d0, d1, d2;
      digits3(v, eb, d0, d1, d2);
      const uint32_t o = tc::kmajor_offset16(jj, c, KB);
      *reinterpret_cast<uint16_t*>(Bd + o) = (uint16_t)(__float_as_uint(d0) >> 16);
      *reinterpret_cast<uint16_t*>(Bd + L::kBplane + o) = (uint16_t)(__float_as_uint(d1) >> 16);
      *reinterpret_cast<uint16_t*>(Bd + 2 * L::kBplane + o) = (uint16_t)(__float_as_uint(d2) >> 16);
    }
  } else if (withz && tid < 2 * KB) {
    const int c = tid - KB;
    zrow[c] = c < k_out ? src[r * KB + c] : 0.f;
    ph[c] = c < r ? sc.ph[c] : 0.f;
    pl[c] = c < r ? sc.pl[c] : 0.f;
  }
  const bool got = tc::mbar_wait_bounded(&bars[0], 0, kTcWaitNs);
  const int late = __syncthreads_or(!got);  // also: B planes, scales, z row and p complete
  if (late) {
    if (tid == 0) {
      atomicOr(&op.st->status, kStTimeout);
      tc::mbar_wait_bounded(&bars[0], 0, kTcWaitNs);  // let the copy in flight finish
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::kTmemCols);
    return;
  }

  // Step 2: this thread's row (columns >= r are stale and count as zero).
  const int row = tid;
  const bool live = row < rows;
  const float4* T4 = reinterpret_cast<const float4*>(T);
  float xv[KB];
#pragma unroll
  for (int q = 0; q < C4; ++q) {
    // chunk (q + row) mod C4 first: conflict-free across the warp; registers stay static-indexed
    // because the chunk order is undone below with a barrel shift
    const int qq = (q + row) % C4;
    const float4 a = live ? T4[row * C4 + qq] : make_float4(0.f, 0.f, 0.f, 0.f);
    xv[4 * q] = a.x;
    xv[4 * q + 1] = a.y;
    xv[4 * q + 2] = a.z;
    xv[4 * q + 3] = a.w;
  }
  {
    // undo the rotation: xv chunk q holds row chunk (q + sh) mod C4
    const int sh = row % C4;
#pragma unroll
    for (int b = 1; b < C4; b <<= 1) {
      if (sh & b) {
        float tmp[KB];
#pragma unroll
        for (int i = 0; i < KB; ++i) tmp[i] = xv[(i - 4 * b + KB) % KB];
#pragma unroll
        for (int i = 0; i < KB; ++i) xv[i] = tmp[i];
      }
    }
  }
  float amax = 0.f;
#pragma unroll
  for (int c = 0; c < KB; ++c) {
    if (c >= r) xv[c] = 0.f;
    amax = fmaxf(amax, fabsf(xv[c]));
  }
  float zh = 0.f;
  if (withz && live) {
    ff s{op.x[base + row], 0.f};
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      if (c < r) {
        ff pr = two_prod(xv[c], ph[c]);
        pr.lo = fmaf(xv[c], pl[c], pr.lo);
        s = ff_add(s, ff{-pr.hi, -pr.lo});
      }
    }
    zh = (s.hi + s.lo) * sc.inv_rho;
  }
  const int ea = fixed_exponent(amax);
  const float ascale = ldexpf(1.f, ea - 8);
#pragma unroll
  for (int g = 0; g < KB / 8; ++g) {  // one 16-byte core-matrix row per digit plane
    uint32_t w0[4], w1[4], w2[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      float a0, a1, a2, b0, b1, b2;
      digits3(xv[8 * g + 2 * h], ea, a0, a1, a2);
      digits3(xv[8 * g + 2 * h + 1], ea, b0, b1, b2);
      w0[h] = pack_bf16x2(a0, b0);
      w1[h] = pack_bf16x2(a1, b1);
      w2[h] = pack_bf16x2(a2, b2);
    }
    const uint32_t o = tc::kmajor_offset16(row, 8 * g, KB);
    *reinterpret_cast<uint4*>(Ad + o) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
    *reinterpret_cast<uint4*>(Ad + L::kAplane + o) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4*>(Ad + 2 * L::kAplane + o) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
  }
  tc::fence_proxy_async_smem();
  __syncthreads();

  // Step 3: level l accumulator at TMEM columns l * KB; per K step of 16 the digit pairs (i, j)
  // with i + j = l.
  if (tid == 0) {
    tc::tc_fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_bf16(128, KB);
    const uint32_t a0 = tc::smem_u32(Ad), b0 = tc::smem_u32(Bd);
#pragma unroll
    for (int s = 0; s < KB / 16; ++s) {
      const uint32_t ko = (uint32_t)s * 256u;  // two core matrices along K
      uint64_t da[3], db[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        da[i] = tc::smem_desc_kmajor(a0 + i * L::kAplane + ko, 128, L::kSbo);
        db[i] = tc::smem_desc_kmajor(b0 + i * L::kBplane + ko, 128, L::kSbo);
      }
      const uint32_t acc = s > 0 ? 1u : 0u;
      tc::mma_bf16(tmem, da[0], db[0], idesc, acc);
      tc::mma_bf16(tmem + KB, da[0], db[1], idesc, acc);
      tc::mma_bf16(tmem + KB, da[1], db[0], idesc, 1u);
      tc::mma_bf16(tmem + 2 * KB, da[0], db[2], idesc, acc);
      tc::mma_bf16(tmem + 2 * KB, da[1], db[1], idesc, 1u);
      tc::mma_bf16(tmem + 2 * KB, da[2], db[0], idesc, 1u);
    }
    tc::mma_commit(&bars[1]);
  }
  const bool done = tc::mbar_wait_bounded(&bars[1], 0, kTcWaitNs);
  const int late2 = __syncthreads_or(!done);
  if (late2) {
    if (tid == 0) {
      atomicOr(&op.st->status, kStTimeout);
      tc::mbar_wait_bounded(&bars[1], 0, kTcWaitNs);
    }
    tc::tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
      tc::tc_fence_after_sync();
      tc::tmem_dealloc(tmem, L::kTmemCols);
    }
    return;
  }
  tc::tc_fence_after_sync();

  // Step 4: warp w reads TMEM lanes 32 w .. 32 w + 31, i.e. rows 32 w .. 32 w + 31 of the tile.
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
#pragma unroll
    // D1 + D2 / 2^8, rounded once: that rounding is scaled down by 2^-8 in the result below
    for (int j = 0; j < KB; ++j) acc[j] = fmaf(acc[j], 1.f / 256.f, lv[j]);
    if constexpr (KB == 32) tc::tmem_ld32(lane_addr, lv);
    else tc::tmem_ld16(lane_addr, lv);
#pragma unroll
    for (int j = 0; j < KB; ++j) {
      float y = fmaf(acc[j], 1.f / 256.f, lv[j]) * (ascale * bscale[j]);
      if (withz) y = fmaf(zh, zrow[j], y);
      acc[j] = y;
    }
    if (live) {
      // Write step q stores chunk (q + row) mod C4 (conflict-free across the warp); rotate the
      // registers first so that every register index is static.
      const int sh = row % C4;
#pragma unroll
      for (int b = 1; b < C4; b <<= 1) {
        if (sh & b) {
          float tmp[KB];
#pragma unroll
          for (int i = 0; i < KB; ++i) tmp[i] = acc[(i + 4 * b) % KB];
#pragma unroll
          for (int i = 0; i < KB; ++i) acc[i] = tmp[i];
        }
      }
      float4* W4 = reinterpret_cast<float4*>(T);
#pragma unroll
      for (int q = 0; q < C4; ++q)
        W4[row * C4 + (q + sh) % C4] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
  }
  tc::fence_proxy_async_smem();
  tc::tc_fence_before_sync();
  __syncthreads();
  if (tid == 0) {
    tc::bulk_s2g(X, T, tile_bytes);
    tc::bulk_commit();
    tc::bulk_wait_all();
  }
  if (warp == 0) {
    tc::tc_fence_after_sync();
    tc::tmem_dealloc(tmem, L::kTmemCols);
  }
}

}  // namespace isvd
