// Rotations of the batched appends on the FP32 pipes (Section 2.2 Step 3: U' = blkdiag(U, 1) U_K,
// V' = [V z_hat] V_K, and the transposed roles for column appends), for rank buckets 8, 16, 32.
//
// A row of U or V costs 2 k^2 FLOP for 8 k bytes of HBM traffic (read and write, FP32): k / 4 FLOP
// per byte, an HBM-bound stream at these ranks. The kernel is built to keep HBM busy:
//   - persistent CTAs (as many as fit on the SMs), each over a contiguous range of the rotation
//     blocks (256 rows of one side of one update; the warp kernel's block -> update tables);
//   - a producer warp per CTA brings every block's rows by TMA through the stream's tensor map of
//     U or V (32-row boxes, swizzled so that a thread reading its own row meets no bank
//     conflicts), together with the update's core factor (V_K or U_K) and p2 by bulk copies, on one
//     mbarrier per stage; three stages keep the next two blocks in flight while one is rotated;
//   - four rotating warps take two rows per thread, rotated in place in shared memory (every
//     core-factor value read feeds both rows), then write the block back with coalesced 16-byte
//     stores and free the stage.
// The arithmetic per row is fixed: y_j = sum_c x_c R[c][j] over the row's r entries (FMAs in c
// order), then + z_hat R[r][j], with z_hat = (z1_row - row . p2) / rho: z1 = x - P p1 is the warp
// kernel's first-pass residual (formed there in float-float, which carries the cancellation) and
// p2 = P^T z1 its small second-pass correction, so z = x - P (p1 + p2) needs only FP32 here.
// Results do not depend on the tiling. Waits are bounded in wall time; on a timeout the stream's status
// gets kStTimeout and the CTA stops after its copies in flight have landed (bounded).
#pragma once

#include "pool_warp.cuh"
#include "tc_ptx.cuh"

namespace isvd {

// A CUtensorMap (128 bytes, 64-byte aligned) as the kernels see it: opaque.
struct alignas(64) RowTensorMap {
  unsigned char bytes[128];
};

constexpr uint64_t kRotWaitNs = 2000ull * 1000 * 1000;  // 2 s

// The 16-byte chunk where logical chunk q of staged row `row` lands under the tensor maps'
// swizzle: 128-byte swizzle for 128-byte rows (KB = 32), 64-byte for 64-byte rows, 32-byte for
// 32-byte rows. A stage starts on a 1 KiB boundary and boxes are whole multiples of the pattern.
template <int KB>
__device__ __forceinline__ int rows_swz(int row, int q) {
  return KB == 32 ? (q ^ (row & 7)) : KB == 16 ? (q ^ ((row >> 1) & 3)) : (q ^ ((row >> 2) & 1));
}

// Where rotation block b (ROWS rows per block) sits: its update, side, first row and row count.
template <int KB, int ROWS>
struct RotBlock {
  int e, rows;
  bool pside, withz;
  int64_t base;
  __device__ __forceinline__ void locate(const PoolOp* ops, const RotScratch<KB>* scratch, const int* chunk_start,
                                         const int* block_op, int b) {
    e = block_op[b];
    const PoolOp& op = ops[e];
    const bool is_row = op.kind == kRow;
    const int64_t nP = is_row ? op.n : op.m, nQ = is_row ? op.m : op.n;
    const int cP = (int)((nP + ROWS - 1) / ROWS);
    const int ci = b - chunk_start[e];
    pside = ci < cP;
    withz = pside && scratch[e].grew;
    const int64_t nrows = pside ? nP : nQ;
    base = (int64_t)(pside ? ci : ci - cP) * ROWS;
    rows = (int)(nrows - base < ROWS ? nrows - base : ROWS);
  }
  __device__ __forceinline__ float* tile(const PoolOp* ops) const {
    const PoolOp& op = ops[e];
    const bool is_row = op.kind == kRow;
    return (pside ? (is_row ? op.V : op.U) : (is_row ? op.U : op.V)) + base * KB;
  }
  // The tensor map of the matrix the block rotates: maps[2 * stream + 0] covers U, [.. + 1] V.
  __device__ __forceinline__ const void* tmap(const PoolOp* ops, const RowTensorMap* maps) const {
    const PoolOp& op = ops[e];
    const bool is_v = pside == (op.kind == kRow);
    return &maps[2 * op.sid + (is_v ? 1 : 0)];
  }
};

// First block at or after b (below b1) whose update has work (k_out >= 0), or b1. A table entry
// outside [0, nops) stops the scan (the caller's checks reject that block).
template <int KB>
__device__ __forceinline__ int rot_next_live(const RotScratch<KB>* scratch, const int* block_op, int b, int b1,
                                             int nops = 0x7fffffff) {
  while (b < b1) {
    const int e = block_op[b];
    if (e < 0 || e >= nops || scratch[e].k_out >= 0) break;
    ++b;
  }
  return b;
}

// What the producer warp tells the rotating warps about the block in a stage.
struct RotMeta {
  float* X;        // the block's first row in global memory
  int rows, r, k_out, withz;
  float inv_rho;
  int e;           // the update; < 0: no more blocks
  int pad[2];
};

template <int KB>
struct RotTmaLayout {
  static constexpr int kStages = 3;
  static constexpr uint32_t kTile = kPoolRotRows * KB * 4;     // one stage of rows
  static constexpr uint32_t kFactor = (KB + 1) * KB * 4;       // V_K or U_K (row stride KB)
  static constexpr uint32_t kPvec = KB * 4;                    // p2
  static constexpr uint32_t kXvec = kPoolRotRows * 4;          // the rows' first-pass residuals z1
  static constexpr uint32_t kOffF = kStages * kTile;
  static constexpr uint32_t kOffP = kOffF + kStages * kFactor;
  static constexpr uint32_t kOffX = kOffP + kStages * kPvec;
  static constexpr uint32_t kOffMeta = kOffX + kStages * kXvec;
  static constexpr uint32_t kOffBar = kOffMeta + kStages * sizeof(RotMeta);
  static constexpr uint32_t kUsed = kOffBar + 16 * kStages;
  // + room to align the base to 1 KiB, as far as two CTAs per SM still fit at KB = 32 (the
  // kernel checks that the aligned layout fits what the launch gave it)
  static constexpr uint32_t kBytes = kUsed + (KB == 32 ? 512 : 1024);
  static constexpr int kMinBlocks = KB == 32 ? 2 : KB == 16 ? 4 : 6;
  static_assert(kFactor % 16 == 0 && kPvec % 16 == 0 && kTile % 1024 == 0, "bulk copy granularity");
  static_assert(kOffMeta % 8 == 0 && kOffBar % 8 == 0, "alignment of the stage records and barriers");
};
constexpr int kRotConsumers = kPoolRotThreads;          // rotating threads (four warps, two rows each)
constexpr int kRotThreadsAll = kRotConsumers + 32;      // + one producer warp

// The r leading entries of staged row `row`, zero beyond.
template <int KB>
__device__ __forceinline__ void rot_load_row(const float* T, int row, int r, float (&v)[KB]) {
  const float4* T4 = reinterpret_cast<const float4*>(T) + row * (KB / 4);
#pragma unroll
  for (int q = 0; q < KB / 4; ++q) {
    const int c4 = 4 * q;
    if (c4 < r) {
      const float4 a = T4[rows_swz<KB>(row, q)];
      v[c4] = a.x;
      v[c4 + 1] = c4 + 1 < r ? a.y : 0.f;
      v[c4 + 2] = c4 + 2 < r ? a.z : 0.f;
      v[c4 + 3] = c4 + 3 < r ? a.w : 0.f;
    } else {
      v[c4] = v[c4 + 1] = v[c4 + 2] = v[c4 + 3] = 0.f;
    }
  }
}

// Rows a and b (b only when has1) times the core factor R, written back in place for columns
// < k_out, eight output columns per pass; every R value read feeds both rows. The row entries
// beyond r are zero and R's rows beyond r are zero (the warp kernel writes them so), so the sum
// runs over all KB rows without branches; the z_hat term (R's row r) is added last.
template <int KB>
__device__ __forceinline__ void rot_two_rows(float* T, int a, int b, const float (&x0)[KB], const float (&x1)[KB],
                                             int r, const float* R, int k_out, float z0, float z1, bool withz,
                                             bool has1) {
  float4* T4 = reinterpret_cast<float4*>(T);
  const float4* R4 = reinterpret_cast<const float4*>(R);
#pragma unroll 1
  for (int h0 = 0; h0 < k_out; h0 += 8) {
    const int q = h0 >> 2;
    float o0[8], o1[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) o0[jj] = o1[jj] = 0.f;
#pragma unroll
    for (int c = 0; c < KB; ++c) {
      const float4 ra = R4[c * (KB / 4) + q], rb = R4[c * (KB / 4) + q + 1];
      const float u0 = x0[c], u1 = x1[c];
      o0[0] = fmaf(u0, ra.x, o0[0]);
      o0[1] = fmaf(u0, ra.y, o0[1]);
      o0[2] = fmaf(u0, ra.z, o0[2]);
      o0[3] = fmaf(u0, ra.w, o0[3]);
      o0[4] = fmaf(u0, rb.x, o0[4]);
      o0[5] = fmaf(u0, rb.y, o0[5]);
      o0[6] = fmaf(u0, rb.z, o0[6]);
      o0[7] = fmaf(u0, rb.w, o0[7]);
      o1[0] = fmaf(u1, ra.x, o1[0]);
      o1[1] = fmaf(u1, ra.y, o1[1]);
      o1[2] = fmaf(u1, ra.z, o1[2]);
      o1[3] = fmaf(u1, ra.w, o1[3]);
      o1[4] = fmaf(u1, rb.x, o1[4]);
      o1[5] = fmaf(u1, rb.y, o1[5]);
      o1[6] = fmaf(u1, rb.z, o1[6]);
      o1[7] = fmaf(u1, rb.w, o1[7]);
    }
    if (withz) {
      const float4 ra = R4[r * (KB / 4) + q], rb = R4[r * (KB / 4) + q + 1];
      const float zr[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        o0[jj] = fmaf(z0, zr[jj], o0[jj]);
        o1[jj] = fmaf(z1, zr[jj], o1[jj]);
      }
    }
    if (h0 + 7 < k_out) {
      T4[a * (KB / 4) + rows_swz<KB>(a, q)] = make_float4(o0[0], o0[1], o0[2], o0[3]);
      T4[a * (KB / 4) + rows_swz<KB>(a, q + 1)] = make_float4(o0[4], o0[5], o0[6], o0[7]);
      if (has1) {
        T4[b * (KB / 4) + rows_swz<KB>(b, q)] = make_float4(o1[0], o1[1], o1[2], o1[3]);
        T4[b * (KB / 4) + rows_swz<KB>(b, q + 1)] = make_float4(o1[4], o1[5], o1[6], o1[7]);
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (h0 + jj < k_out) {
          const int col = h0 + jj;
          T[a * KB + 4 * rows_swz<KB>(a, col >> 2) + (col & 3)] = o0[jj];
          if (has1) T[b * KB + 4 * rows_swz<KB>(b, col >> 2) + (col & 3)] = o1[jj];
        }
    }
  }
}

// Self-check codes recorded in the pool's check word (first failure wins; the block is skipped).
constexpr int kChkBlockOp = 1;   // block -> update entry outside the run's updates
constexpr int kChkChunk = 2;     // block outside its update's blocks
constexpr int kChkRows = 3;      // block rows outside (0, 256] or past the side's rows
constexpr int kChkMap = 4;       // stream id outside the tensor-map table, or a zeroed map
constexpr int kChkRank = 5;      // r or k_out of the update outside [0, KB]
constexpr int kChkWarpTable = 6; // the warp kernel's block table write past the run's table

__device__ __forceinline__ void kcheck_record(int* kcheck, int code, int detail) {
  if (atomicCAS(&kcheck[0], 0, code) == 0) kcheck[1] = detail;
}

// Producer-side validation of block b before any of its loads is issued.
template <int KB>
__device__ __forceinline__ bool rot_block_ok(const RotBlock<KB, kPoolRotRows>& bk, const PoolOp* ops,
                                             const RotScratch<KB>* scratch, const int* chunk_start, int b,
                                             int nops, int nmaps, const RowTensorMap* maps, int* kcheck) {
  if (bk.e < 0 || bk.e >= nops) return kcheck_record(kcheck, kChkBlockOp, b), false;
  if (b < chunk_start[bk.e]) return kcheck_record(kcheck, kChkChunk, b), false;
  const PoolOp& op = ops[bk.e];
  const int64_t nrows = bk.pside ? (op.kind == kRow ? op.n : op.m) : (op.kind == kRow ? op.m : op.n);
  if (bk.rows <= 0 || bk.rows > kPoolRotRows || bk.base + bk.rows > nrows) return kcheck_record(kcheck, kChkRows, b), false;
  if (op.sid < 0 || 2 * op.sid + 1 >= nmaps) return kcheck_record(kcheck, kChkMap, b), false;
  const RotScratch<KB>& sc = scratch[bk.e];
  if (sc.r < 0 || sc.r > KB || sc.k_out > KB) return kcheck_record(kcheck, kChkRank, b), false;
  const uint64_t* mw = reinterpret_cast<const uint64_t*>(bk.tmap(ops, maps));
  uint64_t any = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) any |= mw[i];
  if (!any) return kcheck_record(kcheck, kChkMap, b), false;
  return true;
}

// nblocks rotation blocks of one rank bucket's updates (tables from the warp kernel, 256 rows per
// block); persistent CTAs, block range [blockIdx.x * per, (blockIdx.x + 1) * per). nops: the run's
// updates; nmaps: entries of the tensor-map table; kcheck: the pool's self-check word.
// Warp specialisation: warp 4 is the producer (for each live block of the range: wait until the
// stage is free, describe the block in the stage's RotMeta, stage the payload entries of the
// rows, issue the TMA and bulk loads); warps 0-3 rotate (wait for the stage, rotate two rows per
// thread in place, store the block with coalesced 16-byte stores, free the stage). A RotMeta
// with e < 0 ends the range.
template <int KB>
__global__ void __launch_bounds__(kRotThreadsAll, RotTmaLayout<KB>::kMinBlocks)
    k_pool_rotate(const PoolOp* __restrict__ ops, const RotScratch<KB>* __restrict__ scratch,
                  const int* __restrict__ chunk_start, const int* __restrict__ block_op, int nblocks,
                  const RowTensorMap* __restrict__ maps, int nops, int nmaps, int* __restrict__ kcheck) {
  using L = RotTmaLayout<KB>;
  constexpr int S = L::kStages;
  constexpr int C4 = KB / 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  RotMeta* meta = reinterpret_cast<RotMeta*>(smem + L::kOffMeta);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::kOffBar);  // stage loaded (producer arrival + bytes)
  uint64_t* empty = full + S;                                         // stage free (one arrival per rotating warp)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  const int per = (nblocks + (int)gridDim.x - 1) / (int)gridDim.x;
  const int b1 = min(nblocks, ((int)blockIdx.x + 1) * per);
  const int b0 = rot_next_live<KB>(scratch, block_op, (int)blockIdx.x * per, b1, nops);
  if (b0 >= b1) return;  // uniform: nothing to rotate in this range
  const int e0 = block_op[b0];
  DevState* st0 = e0 >= 0 && e0 < nops ? ops[e0].st : nullptr;  // where a failure of this CTA is reported
  if ((uint32_t)(smem - smem_raw) + L::kUsed > tc::dynamic_smem_bytes()) {  // uniform
    if (tid == 0) {
      if (st0) atomicOr(&st0->status, kStLayout);
      else kcheck_record(kcheck, kChkBlockOp, b0);
    }
    return;
  }

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], kRotConsumers / 32);
    }
    tc::fence_mbar_init();
  }
  __syncthreads();

  if (warp == kRotConsumers / 32) {
    // ---- producer warp ----
    int b = b0, it = 0, issued = 0;
    bool failed = false;
    for (;; ++it) {
      const int s = it % S;
      if (it >= S && !tc::mbar_wait_bounded(&empty[s], (uint32_t)(it / S - 1) & 1u, kRotWaitNs)) {
        failed = true;
        break;
      }
      if (b >= b1) {
        if (lane == 0) {
          meta[s].e = -1;
          tc::mbar_arrive(&full[s]);
        }
        break;
      }
      RotBlock<KB, kPoolRotRows> bk;
      bk.e = block_op[b];
      if (bk.e < 0 || bk.e >= nops) {
        if (lane == 0) kcheck_record(kcheck, kChkBlockOp, b);
        b = rot_next_live<KB>(scratch, block_op, b + 1, b1, nops);
        --it;  // the stage stays free for the next block
        continue;
      }
      bk.locate(ops, scratch, chunk_start, block_op, b);
      if (!rot_block_ok<KB>(bk, ops, scratch, chunk_start, b, nops, nmaps, maps, kcheck)) {
        b = rot_next_live<KB>(scratch, block_op, b + 1, b1, nops);
        --it;
        continue;
      }
      const RotScratch<KB>& sc = scratch[bk.e];
      if (bk.withz) {
        const float* z1 = ops[bk.e].z1 + bk.base;
        float* zs = reinterpret_cast<float*>(smem + L::kOffX + (uint32_t)s * L::kXvec);
        for (int i = lane; i < bk.rows; i += 32) zs[i] = z1[i];
      }
      __syncwarp();
      if (lane == 0) {
        RotMeta& M = meta[s];
        M.X = bk.tile(ops);
        M.rows = bk.rows;
        M.r = sc.r;
        M.k_out = sc.k_out;
        M.withz = bk.withz ? 1 : 0;
        M.inv_rho = sc.inv_rho;
        M.e = bk.e;
        tc::fence_proxy_async_smem();
        const int nbox = (bk.rows + kRowBoxRows - 1) / kRowBoxRows;
        tc::mbar_arrive_expect_tx(&full[s], (uint32_t)nbox * (kRowBoxRows * KB * 4) + L::kFactor +
                                                (bk.withz ? L::kPvec : 0u));
        const void* tm = bk.tmap(ops, maps);
        tc::fence_tensormap_acquire(tm);
        float* dst = reinterpret_cast<float*>(smem + (uint32_t)s * L::kTile);
        for (int q = 0; q < nbox; ++q)
          tc::tma_load_2d(dst + q * kRowBoxRows * KB, tm, 0, (int)bk.base + q * kRowBoxRows, &full[s]);
        tc::bulk_g2s(smem + L::kOffF + (uint32_t)s * L::kFactor, bk.pside ? sc.RP : sc.RQ, L::kFactor, &full[s]);
        if (bk.withz) tc::bulk_g2s(smem + L::kOffP + (uint32_t)s * L::kPvec, sc.p2, L::kPvec, &full[s]);
      }
      ++issued;
      b = rot_next_live<KB>(scratch, block_op, b + 1, b1, nops);
    }
    if (failed && lane == 0) {
      if (st0) atomicOr(&st0->status, kStTimeout);
      // the loads of stages not yet consumed land (bounded) before the CTA's shared memory goes away
      for (int j = max(0, issued - S); j < issued; ++j)
        tc::mbar_wait_bounded(&full[j % S], (uint32_t)(j / S) & 1u, kRotWaitNs);
    }
    return;
  }

  // ---- rotating warps ----
  for (int it = 0;; ++it) {
    const int s = it % S;
    const bool got = tc::mbar_wait_bounded(&full[s], (uint32_t)(it / S) & 1u, kRotWaitNs);
    if (tc::named_bar_or(1, kRotConsumers, !got)) {
      if (tid == 0 && st0) atomicOr(&st0->status, kStTimeout);
      return;
    }
    const RotMeta M = meta[s];
    if (M.e < 0) return;
    float* T = reinterpret_cast<float*>(smem + (uint32_t)s * L::kTile);
    const float* R = reinterpret_cast<const float*>(smem + L::kOffF + (uint32_t)s * L::kFactor);
    const int t0 = tid, t1 = tid + kRotConsumers;
    const bool has0 = t0 < M.rows, has1 = t1 < M.rows;
    if (has0) {
      const int u1 = has1 ? t1 : t0;
      float x0[KB], x1[KB];
      rot_load_row<KB>(T, t0, M.r, x0);
      rot_load_row<KB>(T, u1, M.r, x1);
      float z0 = 0.f, z1 = 0.f;
      if (M.withz) {
        // the rows' entries beyond r are zero, and so is p2 beyond r
        const float* p2 = reinterpret_cast<const float*>(smem + L::kOffP + (uint32_t)s * L::kPvec);
        const float* zs = reinterpret_cast<const float*>(smem + L::kOffX + (uint32_t)s * L::kXvec);
        float c0 = 0.f, c1 = 0.f;
#pragma unroll
        for (int c = 0; c < KB; ++c) {
          c0 = fmaf(x0[c], p2[c], c0);
          c1 = fmaf(x1[c], p2[c], c1);
        }
        z0 = (zs[t0] - c0) * M.inv_rho;
        z1 = (zs[u1] - c1) * M.inv_rho;
      }
      rot_two_rows<KB>(T, t0, u1, x0, x1, M.r, R, M.k_out, z0, z1, M.withz != 0, has1);
    }
    tc::named_bar_sync(1, kRotConsumers);
    // Columns >= k_out keep what the tile held (stale, never read: the working rank is k_out).
    float4* X4 = reinterpret_cast<float4*>(M.X);
    const float4* T4 = reinterpret_cast<const float4*>(T);
    for (int f = tid; f < M.rows * C4; f += kRotConsumers) {
      const int rr = f / C4, q = f - rr * C4;
      X4[f] = T4[rr * C4 + rows_swz<KB>(rr, q)];
    }
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(&empty[s]);
  }
}

}  // namespace isvd
