// Tensor-core rotations of the batched appends (Section 2.2 Step 3: U' = blkdiag(U, 1) U_K,
// V' = [V z_hat] V_K, and the transposed roles for column appends) for rank buckets 16 and 32.
//
// A row of U or V costs 2 k^2 FLOP for 8 k bytes of HBM traffic (read and write, FP32), k / 4
// FLOP per byte: at k = 32 streaming at HBM rate needs most of the FP32 pipes' peak, so the row
// tile times the k x k core factor is a dense contraction and runs on tcgen05 with the
// accumulator in TMEM. To keep FP32 accuracy with TF32 inputs each operand is split into two
// TF32 parts, a = a_hi + a_lo (both rounded to nearest), and the product is accumulated as
// a_hi b_hi + a_hi b_lo + a_lo b_hi (three MMAs per K step, FP32 accumulation); the dropped
// a_lo b_lo term and the rounding of the parts are below 2^-21 relative.
//
// One CTA of 256 threads handles 256 rows of one side of one update (the same block -> update
// tables as the SIMT kernel k_pool_rotate):
//   1. thread 0 starts one bulk copy (TMA) of the contiguous row tile (rows x KB FP32) into
//      shared memory; meanwhile the CTA splits the core factor (V_K or U_K, rows >= r and columns
//      >= k_out zeroed) into TF32 hi / lo operands in the K-major core-matrix layout;
//   2. each thread takes one row: z_hat = (x_row - row . p) / rho in float-float when the
//      projection side gains the new direction, and the row's hi / lo split (columns >= r zeroed);
//   3. thread 0 issues the MMAs (M = 128 rows per accumulator, N = KB, K = 8 per instruction)
//      into two TMEM accumulators and commits them to an mbarrier;
//   4. each warp loads its 32 accumulator lanes (one row per thread), adds z_hat times the core
//      factor's last row, writes the row back into the staging tile, and thread 0 stores the tile
//      with one bulk copy.
// Every wait is bounded in wall time; on a timeout the stream's sticky status gets kStTimeout,
// the CTA waits (bounded) for its copies, frees its TMEM and returns.
#pragma once

#include "pool_warp.cuh"
#include "tc_ptx.cuh"

namespace isvd {

constexpr int kTcRotThreads = 256;                     // one row per thread
constexpr uint64_t kTcWaitNs = 2000ull * 1000 * 1000;  // 2 s

template <int KB>
struct TcRotLayout {
  static constexpr int kRows = kPoolRotRows;                  // 256
  static constexpr uint32_t kTile = kRows * KB * 4;           // FP32 staging tile
  static constexpr uint32_t kAop = kRows * KB * 4;            // one TF32 operand of the row tile
  static constexpr uint32_t kBop = KB * KB * 4;               // one TF32 operand of the core factor
  static constexpr uint32_t kOffA_hi = kTile;
  static constexpr uint32_t kOffA_lo = kOffA_hi + kAop;
  static constexpr uint32_t kOffB_hi = kOffA_lo + kAop;
  static constexpr uint32_t kOffB_lo = kOffB_hi + kBop;
  static constexpr uint32_t kOffVec = kOffB_lo + kBop;        // z row, p hi, p lo (KB floats each)
  static constexpr uint32_t kOffBar = kOffVec + 3 * KB * 4;   // two mbarriers
  static constexpr uint32_t kOffTmem = kOffBar + 16;
  static constexpr uint32_t kBytes = kOffTmem + 16;
  static constexpr uint32_t kTmemCols = 2 * KB < 32 ? 32 : 2 * KB;  // two M = 128 accumulators
  static constexpr uint32_t kSbo = 8 * KB * 4;                // bytes per 8-row group
};

template <int KB>
__global__ void __launch_bounds__(kTcRotThreads, 1)
    k_pool_rotate_tc(const PoolOp* __restrict__ ops, const RotScratch<KB>* __restrict__ scratch,
                     const int* __restrict__ chunk_start, const int* __restrict__ block_op) {
  static_assert(KB == 16 || KB == 32, "tensor-core rotation buckets");
  using L = TcRotLayout<KB>;
  constexpr int C4 = KB / 4;  // float4 chunks per row
  extern __shared__ __align__(1024) unsigned char smem[];
  float* T = reinterpret_cast<float*>(smem);
  unsigned char* Ahi = smem + L::kOffA_hi;
  unsigned char* Alo = smem + L::kOffA_lo;
  unsigned char* Bhi = smem + L::kOffB_hi;
  unsigned char* Blo = smem + L::kOffB_lo;
  float* zrow = reinterpret_cast<float*>(smem + L::kOffVec);
  float* ph = zrow + KB;
  float* pl = ph + KB;
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
  const int cP = (int)((nP + L::kRows - 1) / L::kRows);
  const int ci = blockIdx.x - chunk_start[e];
  const bool pside = ci < cP;
  const int r = sc.r;
  const bool withz = pside && sc.grew;
  const int64_t nrows = pside ? nP : nQ;
  const int64_t base = (int64_t)(pside ? ci : ci - cP) * L::kRows;
  const int rows = (int)(nrows - base < L::kRows ? nrows - base : L::kRows);
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
  // Core factor as TF32 hi / lo B operands: B[n = jj][kk = c] = R[c][jj] for c < r, jj < k_out.
  for (int idx = tid; idx < KB * KB; idx += kTcRotThreads) {
    const int c = idx / KB, jj = idx - c * KB;
    const float v = (c < r && jj < k_out) ? src[c * KB + jj] : 0.f;
    const float hi = tc::to_tf32(v);
    const float lo = tc::to_tf32(v - hi);
    const uint32_t o = tc::kmajor_offset(jj, c, KB);
    *reinterpret_cast<float*>(Bhi + o) = hi;
    *reinterpret_cast<float*>(Blo + o) = lo;
  }
  if (withz && tid < KB) {
    zrow[tid] = tid < k_out ? src[r * KB + tid] : 0.f;
    ph[tid] = tid < r ? sc.ph[tid] : 0.f;
    pl[tid] = tid < r ? sc.pl[tid] : 0.f;
  }
  const bool got = tc::mbar_wait_bounded(&bars[0], 0, kTcWaitNs);
  __syncthreads();  // B operand, z row and p complete; the tile has landed (or timed out)
  const int late = __syncthreads_or(!got);
  if (late) {
    if (tid == 0) {
      atomicOr(&op.st->status, kStTimeout);
      tc::mbar_wait_bounded(&bars[0], 0, kTcWaitNs);  // let the copy in flight finish
    }
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, L::kTmemCols);
    return;
  }

  // Step 2: this thread's row.
  const int row = tid;
  const bool live = row < rows;
  const float4* T4 = reinterpret_cast<const float4*>(T);
  float zh = 0.f;
  if (withz && live) {
    ff s{op.x[base + row], 0.f};
#pragma unroll
    for (int q = 0; q < C4; ++q) {
      const int qq = (q + row) % C4;  // rotated chunk order: conflict-free across the warp
      const float4 a = T4[row * C4 + qq];
      const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 4 * qq + j;
        if (c < r) {
          ff pr = two_prod(av[j], ph[c]);
          pr.lo = fmaf(av[j], pl[c], pr.lo);
          s = ff_add(s, ff{-pr.hi, -pr.lo});
        }
      }
    }
    zh = (s.hi + s.lo) * sc.inv_rho;
  }
#pragma unroll
  for (int q = 0; q < C4; ++q) {
    const int qq = (q + row) % C4;
    float4 a = live ? T4[row * C4 + qq] : make_float4(0.f, 0.f, 0.f, 0.f);
    float av[4] = {a.x, a.y, a.z, a.w};
    float hv[4], lv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float v = 4 * qq + j < r ? av[j] : 0.f;  // columns >= r are stale
      hv[j] = tc::to_tf32(v);
      lv[j] = tc::to_tf32(v - hv[j]);
    }
    const uint32_t o = tc::kmajor_offset(row, 4 * qq, KB);
    *reinterpret_cast<float4*>(Ahi + o) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *reinterpret_cast<float4*>(Alo + o) = make_float4(lv[0], lv[1], lv[2], lv[3]);
  }
  tc::fence_proxy_async_smem();
  __syncthreads();

  // Step 3: two M = 128 accumulators, K = KB in steps of 8, three MMAs per step.
  if (tid == 0) {
    tc::tc_fence_after_sync();
    constexpr uint32_t idesc = tc::idesc_tf32(128, KB);
    const uint32_t a_hi = tc::smem_u32(Ahi), a_lo = tc::smem_u32(Alo);
    const uint32_t b_hi = tc::smem_u32(Bhi), b_lo = tc::smem_u32(Blo);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t d = tmem + (uint32_t)(h * KB);
      const uint32_t aoff = (uint32_t)h * 16u * L::kSbo;  // 128 rows = 16 row groups
#pragma unroll
      for (int s = 0; s < KB / 8; ++s) {
        const uint32_t ko = (uint32_t)s * 256u;  // two core matrices along K
        const uint64_t dah = tc::smem_desc_kmajor(a_hi + aoff + ko, 128, L::kSbo);
        const uint64_t dal = tc::smem_desc_kmajor(a_lo + aoff + ko, 128, L::kSbo);
        const uint64_t dbh = tc::smem_desc_kmajor(b_hi + ko, 128, L::kSbo);
        const uint64_t dbl = tc::smem_desc_kmajor(b_lo + ko, 128, L::kSbo);
        tc::mma_tf32(d, dah, dbh, idesc, s > 0 ? 1u : 0u);
        tc::mma_tf32(d, dah, dbl, idesc, 1u);
        tc::mma_tf32(d, dal, dbh, idesc, 1u);
      }
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

  // Step 4: warp w reads accumulator lanes 32 (w % 4) .. + 31 of half w / 4, i.e. rows 32 w ..
  // 32 w + 31 of the tile: its own rows.
  {
    const int h = warp >> 2;
    const uint32_t taddr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(h * KB);
    float acc[KB];
    if constexpr (KB == 32) tc::tmem_ld32(taddr, acc);
    else tc::tmem_ld16(taddr, acc);
    if (withz) {
#pragma unroll
      for (int j = 0; j < KB; ++j) acc[j] = fmaf(zh, zrow[j], acc[j]);
    }
    if (live) {
      // Write step q stores chunk (q + row) mod C4 (conflict-free across the warp); the chunks are
      // first rotated in registers by a barrel shifter so that every register index is static.
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
