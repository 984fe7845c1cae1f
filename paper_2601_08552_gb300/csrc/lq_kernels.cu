// lq_kernels.cu -- host side of the sm_103a kernels: the shared-memory plan
// sizes, the chain build, initial-state and test-hook kernels, and the launch
// wrappers.  The sweep kernel's four instances (panel type x plan class) live
// in their own translation units (lq_sweep_*.cu) so that they compile in
// parallel.
#include "lq_sweep.cuh"

namespace lq {
size_t smem_bytes(int M, int Nmax, int buf_bytes) { return plan_smem(M, Nmax, buf_bytes).total; }
size_t workspace_bytes(int M, int Nmax, int buf_bytes) { return plan_smem(M, Nmax, buf_bytes).ws_cta; }
int staging_min_bytes(int M, int Nmax, int prop_cols) {
  // prop_cols panel columns (N values each: 1 for the checkerboard, 2 for the
  // exact propagator's Horner buffers) for the propagation; for big plans one
  // window of sites for the flip staging
  const int MP = (M < 1 ? 1 : M) | 1;
  size_t b = (size_t)Nmax * 8 * (prop_cols < 1 ? 1 : prop_cols);
  if (b < 16 * 1024) b = 16 * 1024;
  if (M > LQ_NS_SMALL) {
    const size_t w = (size_t)LQ_WIN * (4 * (size_t)MP * 8 + 32);
    if (b < w) b = w;
  }
  return (int)b;
}
int staging_bytes(int M, int Nmax, int prop_cols) {
  // propagation needs prop_cols panel columns (N values each); the flip
  // staging of the big path needs at least one window of sites (four rows of
  // MP per site)
  const int MP = (M < 1 ? 1 : M) | 1;
  size_t b = (size_t)Nmax * 8 * (prop_cols < 1 ? 1 : prop_cols);
  if (b < 48 * 1024) b = 48 * 1024;
  if (M > LQ_NS_SMALL) {
    const size_t w = (size_t)LQ_WIN * (4 * (size_t)MP * 8 + 32);
    if (b < w) b = w;
  }
  return (int)b;
}


__global__ void clear_records_kernel(LqChainDev* chains, int n) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) chains[c].nrec = 0;
}

// Fields uniform +-1 and occupations by Fisher-Yates from Philox (tags 4, 5).
__global__ void init_kernel(LqChainDev* chains, const int* order, int n_order) {
  for (int q = blockIdx.x; q < n_order; q += gridDim.x) {
    LqChainDev* C = chains + order[q];
    const int N = C->N, L = C->L;
    for (int idx = TID; idx < L * N; idx += blockDim.x) {
      const int l = idx / N, i = idx - l * N;
      uint32_t w[4];
      philox(C->chain_id, 0xFFFFFFFFu, (4u << 24) | (uint32_t)l, (uint32_t)i, C->key0, C->key1, w);
      C->s[idx] = (w[0] & 1u) ? 1 : -1;
    }
    if (TID < 2) {
      const int sg = TID, m = C->ns[sg];
      int* occ = C->occ[sg];
      // partial Fisher-Yates on an implicit identity permutation, kept in occ
      // (positions >= m that were swapped are remembered through a small map)
      // N may be large, so the permutation lives in C->vec reinterpreted as ints
      int* perm = (int*)(C->vec) + sg * N;
      for (int i = 0; i < N; ++i) perm[i] = i;
      for (int t = 0; t < m; ++t) {
        uint32_t w[4];
        philox(C->chain_id, 0xFFFFFFFFu, (5u << 24) | (uint32_t)sg, (uint32_t)t, C->key0, C->key1, w);
        const int r = t + (int)(u53(w[0], w[1]) * (double)(N - t));
        const int tmp = perm[t]; perm[t] = perm[r]; perm[r] = tmp;
      }
      for (int a = 0; a < m; ++a) occ[a] = perm[a];
      for (int a = 1; a < m; ++a) {
        int v = occ[a], b = a - 1;
        while (b >= 0 && occ[b] > v) { occ[b + 1] = occ[b]; --b; }
        occ[b + 1] = v;
      }
    }
  }
}

// Ratio of flipping s at (l, i) on freshly built chains (test hook).
template <class R>
__global__ void __launch_bounds__(LQ_THREADS, 2) field_ratio_kernel(LqChainDev* chains, int c, int l, int i, SmemPlan plan) {
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm = carve(plan, smem_raw);
  LqChainDev* g = chains + c;
  load_chain(g, sm);
  LqChainDev& C = *sm.C;
  const int N = C.N, MP = sm.MP;
  int j = 1;
  while (bnd(C, j) <= l) ++j;
  const int lo = bnd(C, j - 1), hi = bnd(C, j);
  double r = 1.0;
  const int s = C.s[(size_t)l * N + i];
  for (int sg = 0; sg < 2; ++sg) {
    const int m = C.ns[sg];
    R* X = (R*)C.live[sg];
    R* Z = (R*)C.stored[sg];
    prop<R, R>(C, sg, X, qr_panel<R>(C, sg, C.cur[sg], j - 1), m, m, lo, 0, -1, sm);
    for (int ll = lo; ll < l; ++ll) prop<R, R>(C, sg, X, X, m, m, -1, 1, ll + 1, sm);
    prop<R, R>(C, sg, Z, ql_panel<R>(C, sg, j), m, m, -1, 2, -1, sm);
    for (int ll = hi - 1; ll > l; --ll) prop<R, R>(C, sg, Z, Z, m, m, ll, 2, -1, sm);
    gram<double>((const R*)Z, m, m, (const R*)X, m, m, N, sm.W, MP);
    double la;
    int s1;
    inverse(sm.W, MP, sm.T[sg], MP, m, sm, &la, &s1);
    double part = 0.0;
    for (int b = TID; b < m; b += LQ_THREADS) {
      double x = 0.0;
      for (int a = 0; a < m; ++a) x += (double)X[(size_t)i * m + a] * sm.T[sg][a * MP + b];
      part += x * (double)Z[(size_t)i * m + b];
    }
    const double gg = cta_sum(part, sm);
    r *= 1.0 + delta_of(C, sg, s) * gg;
  }
  if (C.charge) r *= (s > 0) ? C.cfac_p : C.cfac_m;
  if (TID == 0) C.hook[0] = r;
  store_chain(g, sm);
}

// Swap ratio (remove column k, add site j) on the current right chain (test hook).
template <class R>
__global__ void __launch_bounds__(LQ_THREADS, 2) swap_ratio_kernel(LqChainDev* chains, int c, int sg, int k, int j, SmemPlan plan) {
  extern __shared__ __align__(16) char smem_raw[];
  Smem sm = carve(plan, smem_raw);
  LqChainDev* g = chains + c;
  load_chain(g, sm);
  LqChainDev& C = *sm.C;
  swap_setup<R>(C, sg, sm);
  swap_attempt<R>(C, sg, k, j, 0.0, 0, sm);
  store_chain(g, sm);
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------
template <class R> static cudaError_t set_attr(const void* fn, size_t smem) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// the four sweep-kernel instances, each defined in its own translation unit
LQ_SWEEP_INSTANCE_DECL(d_small)
LQ_SWEEP_INSTANCE_DECL(d_big)
LQ_SWEEP_INSTANCE_DECL(f_small)
LQ_SWEEP_INSTANCE_DECL(f_big)

static const void* sweep_fn(int prec, int big) {
  if (prec == 0) return big ? sweep_fn_d_big() : sweep_fn_d_small();
  return big ? sweep_fn_f_big() : sweep_fn_f_small();
}

// Big plans keep their m x m matrices in the caller's workspace: grid slabs of ws_cta bytes.
static cudaError_t bind_ws(SmemPlan& p, void* ws, size_t ws_bytes, int grid) {
  if (!p.big) return cudaSuccess;
  if (!ws || (size_t)grid * p.ws_cta > ws_bytes || ((uintptr_t)ws & 255)) return cudaErrorInvalidValue;
  p.ws = (char*)ws;
  return cudaSuccess;
}

cudaError_t launch_sweep(int prec, LqChainDev* chains, const int* order, int n_order, int* queue, int n_sweeps,
                         int do_measure, int M, int Nmax, int buf_bytes, int grid, cudaStream_t st, void* ws,
                         size_t ws_bytes, const int* caps, long long budget_ns, int threads) {
  SmemPlan p = plan_smem(M, Nmax, buf_bytes);
  cudaError_t e = bind_ws(p, ws, ws_bytes, grid);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(queue, 0, sizeof(int) * (1 + 1024), st);
  if (e != cudaSuccess) return e;
  const void* fn = sweep_fn(prec, p.big);
  if ((e = set_attr<double>(fn, p.total)) != cudaSuccess) return e;
  // big plans flip with four-warp groups per spin: always a full CTA
  const int nt = (p.big || threads != LQ_THREADS / 2) ? LQ_THREADS : LQ_THREADS / 2;
  if (prec == 0 && !p.big)
    return sweep_launch_d_small(grid, nt, st, chains, order, n_order, queue, n_sweeps, caps, budget_ns, do_measure, p);
  if (prec == 0)
    return sweep_launch_d_big(grid, nt, st, chains, order, n_order, queue, n_sweeps, caps, budget_ns, do_measure, p);
  if (!p.big)
    return sweep_launch_f_small(grid, nt, st, chains, order, n_order, queue, n_sweeps, caps, budget_ns, do_measure, p);
  return sweep_launch_f_big(grid, nt, st, chains, order, n_order, queue, n_sweeps, caps, budget_ns, do_measure, p);
}

cudaError_t launch_build(int prec, LqChainDev* chains, const int* order, int n_order, int M, int Nmax, int buf_bytes,
                         int grid, cudaStream_t st, void* ws, size_t ws_bytes) {
  SmemPlan p = plan_smem(M, Nmax, buf_bytes);
  cudaError_t e = bind_ws(p, ws, ws_bytes, grid);
  if (e != cudaSuccess) return e;
  if (prec == 0) {
    if ((e = set_attr<double>((const void*)build_kernel<double>, p.total)) != cudaSuccess) return e;
    build_kernel<double><<<grid, LQ_THREADS, p.total, st>>>(chains, order, n_order, p);
  } else {
    if ((e = set_attr<float>((const void*)build_kernel<float>, p.total)) != cudaSuccess) return e;
    build_kernel<float><<<grid, LQ_THREADS, p.total, st>>>(chains, order, n_order, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_clear_records(LqChainDev* chains, int n, cudaStream_t st) {
  clear_records_kernel<<<(n + 255) / 256, 256, 0, st>>>(chains, n);
  return cudaGetLastError();
}

cudaError_t launch_init(LqChainDev* chains, const int* order, int n_order, int grid, cudaStream_t st) {
  init_kernel<<<grid, LQ_THREADS, 0, st>>>(chains, order, n_order);
  return cudaGetLastError();
}

cudaError_t launch_field_ratio(int prec, LqChainDev* chains, int c, int l, int i, int M, int Nmax, int buf_bytes,
                               cudaStream_t st, void* ws, size_t ws_bytes) {
  SmemPlan p = plan_smem(M, Nmax, buf_bytes);
  cudaError_t e = bind_ws(p, ws, ws_bytes, 1);
  if (e != cudaSuccess) return e;
  if (prec == 0) {
    if ((e = set_attr<double>((const void*)field_ratio_kernel<double>, p.total)) != cudaSuccess) return e;
    field_ratio_kernel<double><<<1, LQ_THREADS, p.total, st>>>(chains, c, l, i, p);
  } else {
    if ((e = set_attr<float>((const void*)field_ratio_kernel<float>, p.total)) != cudaSuccess) return e;
    field_ratio_kernel<float><<<1, LQ_THREADS, p.total, st>>>(chains, c, l, i, p);
  }
  return cudaGetLastError();
}

cudaError_t launch_swap_ratio(int prec, LqChainDev* chains, int c, int sg, int k, int j, int M, int Nmax,
                              int buf_bytes, cudaStream_t st, void* ws, size_t ws_bytes) {
  SmemPlan p = plan_smem(M, Nmax, buf_bytes);
  cudaError_t e = bind_ws(p, ws, ws_bytes, 1);
  if (e != cudaSuccess) return e;
  if (prec == 0) {
    if ((e = set_attr<double>((const void*)swap_ratio_kernel<double>, p.total)) != cudaSuccess) return e;
    swap_ratio_kernel<double><<<1, LQ_THREADS, p.total, st>>>(chains, c, sg, k, j, p);
  } else {
    if ((e = set_attr<float>((const void*)swap_ratio_kernel<float>, p.total)) != cudaSuccess) return e;
    swap_ratio_kernel<float><<<1, LQ_THREADS, p.total, st>>>(chains, c, sg, k, j, p);
  }
  return cudaGetLastError();
}

}  // namespace lq

namespace lq {
// The flip loop's FP64 quotient beside the IEEE one (test hook).
__global__ void quotient_kernel(const double* d, const double* r, int n, double* q_ours, double* q_ieee) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    q_ours[k] = OpsF64<double>::div(d[k], r[k]);
    q_ieee[k] = d[k] / r[k];
  }
}
cudaError_t launch_quotient(const double* d, const double* r, int n, double* q_ours, double* q_ieee, cudaStream_t st) {
  quotient_kernel<<<(n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024, 256, 0, st>>>(d, r, n, q_ours, q_ieee);
  return cudaGetLastError();
}

int max_active_sweep_ctas(int prec, int M, size_t smem, int threads) {
  int n = 0;
  const bool big = M > LQ_NS_SMALL;
  const void* fn = sweep_fn(prec, big);
  const int nt = (big || threads != LQ_THREADS / 2) ? LQ_THREADS : LQ_THREADS / 2;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, nt, smem) != cudaSuccess) return 0;
  return n;
}
}  // namespace lq
