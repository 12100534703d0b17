// Host-side launchers of the heavy kernel families, each compiled in a translation unit of its own
// (core_f32.cu, core_f64.cu, pool_tick8/16/32/64.cu, pool_retry.cu, pool_warp.cu) so that the
// library builds in parallel. The templates are defined in those units and explicitly instantiated
// there. Every launcher enqueues one launch on stream s and returns cudaGetLastError(); the
// set_attr(s) functions raise the dynamic shared-memory limit of the kernels they name.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "isvd_common.cuh"

namespace isvd {

struct PoolOp;

// Core SVD kernel k_core<T, T, kb> (one CTA; kb = rank bucket 16/32/64/128). px and tol_rel serve
// the rank-increasing entry update (kind kEntryX); RU, RV (row stride ldr; nullptr: none) are the
// deferred rotations an entry update's gathers go through; gq: (kKmaxLimit + 1)^2 floats of global
// scratch for the fast core of the 128 bucket.
template <typename T>
cudaError_t core_launch(int kb, int threads, size_t smem, cudaStream_t s, int kind, DevState* st, double* sig,
                        const double* p, const T* U, const T* V, int ld, int64_t ei, int64_t ej, double delta, T* A,
                        int64_t lda, T* UK, T* VKo, int ldo, double* px, double tol_rel, const T* RU, const T* RV,
                        int ldr, float* gq);
// smem[b] = dynamic shared memory of bucket 16 << b (b = 0..3).
template <typename T>
cudaError_t core_set_attrs(const size_t smem[4]);

// Pool CTA kernels k_pool_tick<KB> (KB = 8/16/32/64, one translation unit each) and
// k_pool_retry<32> (its own unit).
template <int KB>
cudaError_t pool_tick_launch(int count, cudaStream_t s, const PoolOp* ops);
template <int KB>
cudaError_t pool_tick_set_attr();
cudaError_t pool_retry_launch(int blocks, cudaStream_t s, const PoolOp* ops, const int* retry, const int* retry_n);
cudaError_t pool_retry_set_attr();

// Pool warp-per-update kernels k_pool_warp<kb> and row-parallel rotations k_pool_rotate<kb>
// (kb = 8/16/32); scratch is the bucket run's first RotScratch<kb> record.
// nblocks: entries of the run's block table; kcheck: the pool's self-check word (code, detail).
cudaError_t pool_warp_launch(int kb, int count, cudaStream_t s, const PoolOp* ops, int base, int* retry, int* retry_n,
                             void* scratch, const int* chunks, int* block_op, int rot_rows, int nblocks, int* kcheck);
// Rows of one side per rotation block for rank bucket kb (the warp kernel's block tables).
int pool_rot_rows(int kb, bool use_tc);
// Both rotations load their row tiles through the pool's tensor maps (two per stream slot: U, V;
// nmaps entries); use_tc selects the tensor-core one (k_pool_rotate_tc, buckets 16 and 32). nops:
// the run's updates; kcheck: the pool's self-check word.
cudaError_t pool_rotate_launch(int kb, int nblocks, cudaStream_t s, const PoolOp* ops, const void* scratch,
                               const int* chunks, const int* block_op, bool use_tc, const void* tmaps, int nops,
                               int nmaps, int* kcheck);
cudaError_t pool_warp_set_attrs();

// Batched loss-of-orthogonality monitor / re-orthogonalisation (k_pool_reorth), one CTA per
// listed stream.
struct PoolReorthOp;
cudaError_t pool_reorth_launch(int count, cudaStream_t s, const PoolReorthOp* list, double tol);

// Completion records of ops[0 .. count) (the state each op left behind, after its tick), and
// the gather of many streams' singular values into one array (out[s * ld + c], zero-padded).
struct PoolCompletion;
struct PoolRankOp;
// k <- min(k + 1, kcap) for every listed stream whose EVR = sum sigma^2 / N_t is below tau.
cudaError_t pool_rank_launch(int count, cudaStream_t s, const PoolRankOp* list, double tau, double tau_shrink);
cudaError_t pool_complete_launch(int count, cudaStream_t s, const PoolOp* ops, PoolCompletion* out);
// out[s] = the status word of slot s's device state, s < n.
cudaError_t pool_gather_status_launch(int64_t n, cudaStream_t s, const DevState* const* st, int* out);
cudaError_t pool_gather_sigma_launch(int64_t n, cudaStream_t s, const double* const* sig, const DevState* const* st,
                                     int ld, double* out);

}  // namespace isvd
