// Launch wrappers of the sm_103a kernels (host-callable, plain types).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "lq_device.h"

namespace lq {
// Dynamic shared memory of one CTA, global workspace per CTA (nonzero only
// when M > LQ_NS_SMALL: then every launch needs grid x workspace_bytes of
// 256-byte aligned device memory in ws), and the staging buffer size the
// plan wants for M particles per spin and Nmax sites.
size_t smem_bytes(int M, int Nmax, int buf_bytes);
size_t workspace_bytes(int M, int Nmax, int buf_bytes);
// prop_cols: panel columns the propagation stages at once (1 for the
// checkerboard, 2 when a chain uses the exact kinetic propagator)
int staging_bytes(int M, int Nmax, int prop_cols = 1);
int staging_min_bytes(int M, int Nmax, int prop_cols = 1);  // the smallest staging buffer a plan can run with
cudaError_t launch_sweep(int prec, LqChainDev* chains, const int* order, int n_order, int* queue, int n_sweeps,
                         int do_measure, int M, int Nmax, int buf_bytes, int grid, cudaStream_t st, void* ws,
                         size_t ws_bytes, const int* caps = nullptr, long long budget_ns = 0,
                         int threads = LQ_THREADS);
cudaError_t launch_build(int prec, LqChainDev* chains, const int* order, int n_order, int M, int Nmax, int buf_bytes,
                         int grid, cudaStream_t st, void* ws, size_t ws_bytes);
cudaError_t launch_clear_records(LqChainDev* chains, int n, cudaStream_t st);
cudaError_t launch_init(LqChainDev* chains, const int* order, int n_order, int grid, cudaStream_t st);
cudaError_t launch_field_ratio(int prec, LqChainDev* chains, int c, int l, int i, int M, int Nmax, int buf_bytes,
                               cudaStream_t st, void* ws, size_t ws_bytes);
cudaError_t launch_swap_ratio(int prec, LqChainDev* chains, int c, int sg, int k, int j, int M, int Nmax,
                              int buf_bytes, cudaStream_t st, void* ws, size_t ws_bytes);
// threads: LQ_THREADS, or LQ_THREADS / 2 for plans of at most LQ_NS_SMALL
// particles per spin (anything else, and every big plan, runs LQ_THREADS)
int max_active_sweep_ctas(int prec, int M, size_t smem, int threads = LQ_THREADS);
// the flip loop's FP64 quotient d/r and the IEEE one, elementwise (device arrays of n)
cudaError_t launch_quotient(const double* d, const double* r, int n, double* q_ours, double* q_ieee, cudaStream_t st);
}  // namespace lq
