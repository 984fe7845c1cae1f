// lq_gram_probe.cu -- the Gram contractions of the sweep (W = A^T B for two
// N x m panels: the block Green's function L~^T R~ and the CholeskyQR2 Grams)
// on the CUDA cores and on the tensor cores, timed side by side.
//
// GB300's tensor cores reach FP64 only through DMMA (mma.sync m8n8k4 .f64),
// and FP32 panels through TF32 products; a TF32 product alone carries 2^-11
// relative error, so the FP32-panel variant splits each operand x = hi + lo
// into two TF32 parts and sums hi*hi + hi*lo + lo*hi (three products, FP32
// accumulation).  Each CTA owns one pair of panels, as a chain does in the
// sweep; the panels stream through shared memory in chunks of rows.  The
// probe reports the time per Gram and the largest error against the FP64
// CUDA-core Gram of the same panels, so that the sweep can use whichever is
// faster at its tolerance.
#include "lq_sweep.cuh"

#include <string>
#include <vector>

#include "lq_lattice.h"

namespace {

constexpr int kChunk = 32;  // panel rows staged per step

// W = A^T B with the sweep's own CUDA-core routine (FP64 accumulation).
template <class R>
__global__ void __launch_bounds__(LQ_THREADS, 1) gram_cuda_core(const R* A, const R* B, double* W, int N, int m) {
  const size_t pn = (size_t)N * m;
  lq::gram<double>(A + blockIdx.x * pn, m, m, B + blockIdx.x * pn, m, m, N, W + (size_t)blockIdx.x * m * m, m);
}

// W = A^T B on the FP64 tensor cores: each warp owns 8 x 8 output tiles; per
// chunk of kChunk rows, mma.sync m8n8k4 with A^T (8 x 4, row-major) and B
// (4 x 8, column-major) fragments read from the staged rows.  Lane layout of
// m8n8k4 .f64: A element (lane / 4, lane % 4), B element (lane % 4, lane / 4),
// C elements (lane / 4, 2 (lane % 4) + {0, 1}).
__global__ void __launch_bounds__(LQ_THREADS, 1) gram_dmma(const double* A, const double* B, double* W, int N, int m) {
  extern __shared__ __align__(16) char smem_raw[];
  double* sa = (double*)smem_raw;          // kChunk x m
  double* sb = sa + (size_t)kChunk * m;    // kChunk x m
  const size_t pn = (size_t)N * m;
  A += blockIdx.x * pn;
  B += blockIdx.x * pn;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tiles = (m / 8) * (m / 8);
  const int g = lane >> 2, t = lane & 3;
  constexpr int kMaxTiles = 32;  // per warp (m <= 128 with 8 warps)
  double acc[kMaxTiles][2];
  for (int q = 0; q < kMaxTiles; ++q) acc[q][0] = acc[q][1] = 0.0;
  for (int i0 = 0; i0 < N; i0 += kChunk) {
    const int rows = min(kChunk, N - i0);
    for (int idx = threadIdx.x; idx < kChunk * m; idx += blockDim.x) {
      const int r = idx / m;
      sa[idx] = r < rows ? A[(size_t)i0 * m + idx] : 0.0;
      sb[idx] = r < rows ? B[(size_t)i0 * m + idx] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxTiles; ++q) {
      const int tile = warp + q * 8;
      if (tile >= tiles) continue;
      const int a0 = (tile / (m / 8)) * 8, b0 = (tile % (m / 8)) * 8;
#pragma unroll
      for (int k = 0; k < kChunk; k += 4) {
        const double fa = sa[(size_t)(k + t) * m + a0 + g];  // (A^T)[a0 + g][k + t]
        const double fb = sb[(size_t)(k + t) * m + b0 + g];  // B[k + t][b0 + g]
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                     : "+d"(acc[q][0]), "+d"(acc[q][1])
                     : "d"(fa), "d"(fb));
      }
    }
    __syncthreads();
  }
  double* Wc = W + (size_t)blockIdx.x * m * m;
#pragma unroll
  for (int q = 0; q < kMaxTiles; ++q) {
    const int tile = warp + q * 8;
    if (tile >= tiles) continue;
    const int a0 = (tile / (m / 8)) * 8, b0 = (tile % (m / 8)) * 8;
    Wc[(size_t)(a0 + g) * m + b0 + 2 * t] = acc[q][0];
    Wc[(size_t)(a0 + g) * m + b0 + 2 * t + 1] = acc[q][1];
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// W = A^T B for FP32 panels on the TF32 tensor cores with the three-product
// split: mma.sync m16n8k8 (A^T tile 16 x 8 row-major, B tile 8 x 8 column-
// major, FP32 accumulators).  Lane layout, g = lane / 4, t = lane % 4:
// A regs (g, t), (g + 8, t), (g, t + 4), (g + 8, t + 4); B regs (t, g),
// (t + 4, g); C regs (g, 2t), (g, 2t + 1), (g + 8, 2t), (g + 8, 2t + 1).
__global__ void __launch_bounds__(LQ_THREADS, 1) gram_3xtf32(const float* A, const float* B, double* W, int N, int m) {
  extern __shared__ __align__(16) char smem_raw[];
  float* sa = (float*)smem_raw;
  float* sb = sa + (size_t)kChunk * m;
  const size_t pn = (size_t)N * m;
  A += blockIdx.x * pn;
  B += blockIdx.x * pn;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ta = m / 16, tb = m / 8, tiles = ta * tb;
  const int g = lane >> 2, t = lane & 3;
  constexpr int kMaxTiles = 16;  // per warp (m <= 128 with 8 warps)
  float acc[kMaxTiles][4];
  for (int q = 0; q < kMaxTiles; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
  for (int i0 = 0; i0 < N; i0 += kChunk) {
    const int rows = min(kChunk, N - i0);
    for (int idx = threadIdx.x; idx < kChunk * m; idx += blockDim.x) {
      const int r = idx / m;
      sa[idx] = r < rows ? A[(size_t)i0 * m + idx] : 0.f;
      sb[idx] = r < rows ? B[(size_t)i0 * m + idx] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxTiles; ++q) {
      const int tile = warp + q * 8;
      if (tile >= tiles) continue;
      const int a0 = (tile / tb) * 16, b0 = (tile % tb) * 8;
#pragma unroll
      for (int k = 0; k < kChunk; k += 8) {
        const float xa[4] = {sa[(size_t)(k + t) * m + a0 + g], sa[(size_t)(k + t) * m + a0 + g + 8],
                             sa[(size_t)(k + t + 4) * m + a0 + g], sa[(size_t)(k + t + 4) * m + a0 + g + 8]};
        const float xb[2] = {sb[(size_t)(k + t) * m + b0 + g], sb[(size_t)(k + t + 4) * m + b0 + g]};
        uint32_t ah[4], al[4], bh[2], bl[2];
        for (int r = 0; r < 4; ++r) {
          ah[r] = to_tf32(xa[r]);
          al[r] = to_tf32(xa[r] - __uint_as_float(ah[r]));
        }
        for (int r = 0; r < 2; ++r) {
          bh[r] = to_tf32(xb[r]);
          bl[r] = to_tf32(xb[r] - __uint_as_float(bh[r]));
        }
#define LQ_MMA_TF32(AR, BR)                                                                                    \
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "     \
               "{%8, %9}, {%0, %1, %2, %3};"                                                                  \
               : "+f"(acc[q][0]), "+f"(acc[q][1]), "+f"(acc[q][2]), "+f"(acc[q][3])                           \
               : "r"(AR[0]), "r"(AR[1]), "r"(AR[2]), "r"(AR[3]), "r"(BR[0]), "r"(BR[1]))
        LQ_MMA_TF32(al, bh);
        LQ_MMA_TF32(ah, bl);
        LQ_MMA_TF32(ah, bh);
#undef LQ_MMA_TF32
      }
    }
    __syncthreads();
  }
  double* Wc = W + (size_t)blockIdx.x * m * m;
#pragma unroll
  for (int q = 0; q < kMaxTiles; ++q) {
    const int tile = warp + q * 8;
    if (tile >= tiles) continue;
    const int a0 = (tile / tb) * 16, b0 = (tile % tb) * 8;
    Wc[(size_t)(a0 + g) * m + b0 + 2 * t] = acc[q][0];
    Wc[(size_t)(a0 + g) * m + b0 + 2 * t + 1] = acc[q][1];
    Wc[(size_t)(a0 + g + 8) * m + b0 + 2 * t] = acc[q][2];
    Wc[(size_t)(a0 + g + 8) * m + b0 + 2 * t + 1] = acc[q][3];
  }
}

// Panel entries uniform in [-0.025, 0.025) from a fixed integer hash of the
// index, so every variant sees the same numbers.
template <class R>
__global__ void fill_panels(R* A, R* B, size_t n) {
  for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)k * 2654435761u ^ 0x9E3779B9u;
    h ^= h >> 15; h *= 0x85EBCA6Bu; h ^= h >> 13;
    A[k] = (R)(((double)(h & 0xFFFFFF) / 16777216.0 - 0.5) * 0.05);
    h *= 0xC2B2AE35u; h ^= h >> 16;
    B[k] = (R)(((double)(h & 0xFFFFFF) / 16777216.0 - 0.5) * 0.05);
  }
}

lq_status gp_fail(cudaError_t e, const char* where) {
  return lq_internal_fail(LQ_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" lq_status lq_probe_gram(int32_t N, int32_t m, int32_t variant, int32_t n_panels, double* host_us,
                                   double* host_max_rel_err) {
  if (N < 8 || m < 8 || m > 128 || (m % 16) || n_panels < 1 || n_panels > 4096 || variant < 0 || variant > 3 ||
      !host_us || !host_max_rel_err)
    return lq_internal_fail(LQ_EINVAL, "lq_probe_gram: N >= 8, m a multiple of 16 in [16, 128], variant 0..3");
  const size_t n = (size_t)n_panels * N * m;
  const bool fp32 = variant >= 2;
  void *A = nullptr, *B = nullptr, *A64 = nullptr, *B64 = nullptr;
  double *W = nullptr, *Wref = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&A64, n * 8);
  if (e == cudaSuccess) e = cudaMalloc(&B64, n * 8);
  if (e == cudaSuccess && fp32) e = cudaMalloc(&A, n * 4);
  if (e == cudaSuccess && fp32) e = cudaMalloc(&B, n * 4);
  if (e == cudaSuccess) e = cudaMalloc((void**)&W, (size_t)n_panels * m * m * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&Wref, (size_t)n_panels * m * m * 8);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const size_t smem = (size_t)2 * kChunk * m * (fp32 ? 4 : 8);
  if (e == cudaSuccess) {
    fill_panels<double><<<1024, 256>>>((double*)A64, (double*)B64, n);
    if (fp32) fill_panels<float><<<1024, 256>>>((float*)A, (float*)B, n);
    e = cudaGetLastError();
  }
  // the reference: FP64 CUDA-core Gram of the same values (FP32 values widened)
  if (e == cudaSuccess) {
    if (fp32) gram_cuda_core<float><<<n_panels, LQ_THREADS>>>((float*)A, (float*)B, Wref, N, m);
    else gram_cuda_core<double><<<n_panels, LQ_THREADS>>>((double*)A64, (double*)B64, Wref, N, m);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && variant == 1)
    e = cudaFuncSetAttribute((const void*)gram_dmma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && variant == 3)
    e = cudaFuncSetAttribute((const void*)gram_3xtf32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  auto launch = [&]() {
    switch (variant) {
      case 0: gram_cuda_core<double><<<n_panels, LQ_THREADS>>>((double*)A64, (double*)B64, W, N, m); break;
      case 1: gram_dmma<<<n_panels, LQ_THREADS, smem>>>((double*)A64, (double*)B64, W, N, m); break;
      case 2: gram_cuda_core<float><<<n_panels, LQ_THREADS>>>((float*)A, (float*)B, W, N, m); break;
      default: gram_3xtf32<<<n_panels, LQ_THREADS, smem>>>((float*)A, (float*)B, W, N, m); break;
    }
    return cudaGetLastError();
  };
  float ms = 0.f;
  const int reps = 5;
  if (e == cudaSuccess) e = launch();  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
  if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  std::vector<double> w((size_t)n_panels * m * m), wr(w.size());
  if (e == cudaSuccess) e = cudaMemcpy(w.data(), W, w.size() * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(wr.data(), Wref, wr.size() * 8, cudaMemcpyDeviceToHost);
  cudaFree(A); cudaFree(B); cudaFree(A64); cudaFree(B64); cudaFree(W); cudaFree(Wref);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return gp_fail(e, "lq_probe_gram");
  // error relative to each Gram's largest entry
  double worst = 0.0;
  for (int p = 0; p < n_panels; ++p) {
    double scale = 0.0, err = 0.0;
    for (size_t k = (size_t)p * m * m; k < (size_t)(p + 1) * m * m; ++k) {
      scale = std::max(scale, std::fabs(wr[k]));
      err = std::max(err, std::fabs(w[k] - wr[k]));
    }
    worst = std::max(worst, err / (scale > 0 ? scale : 1.0));
  }
  *host_us = 1e3 * ms / reps;
  *host_max_rel_err = worst;
  return LQ_OK;
}
