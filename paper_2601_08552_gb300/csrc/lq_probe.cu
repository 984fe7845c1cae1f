// lq_probe.cu -- measured FP64 throughput of the current device, the ALU roof
// that the sweep kernel's FP64 flops are reported against.
//
// GB300 runs FP64 on its CUDA cores at a fraction of the FP32 rate: one FP64
// FMA warp instruction occupies a sub-partition for many cycles whatever the
// number of active lanes.  The probe measures both the aggregate rate (every
// SM busy with independent FMA chains, timed with CUDA events) and the issue
// cost of single warp instructions (one warp, clock64), so that the roof is a
// number taken on the device rather than a constant.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lecqmc.h"
#include "lq_kernels.h"
#include "lq_lattice.h"

namespace {

// Eight independent FMA chains per thread keep every FP64 pipe fed.
__global__ void fma_rate_kernel(double* out, long long iters, double a, double b) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  double x0 = tid * 1e-9, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  for (long long it = 0; it < iters; ++it) {
    x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
    x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
  }
  out[tid] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

// Cycles per warp instruction on one sub-partition: one warp, `active` lanes
// run eight independent FMA chains of ITERS steps between two clock reads.
constexpr int kIters = 4096;
template <class T>
__global__ void fma_issue_kernel(T* out, long long* cyc, int active, T a, T b) {
  const int lane = threadIdx.x & 31;
  T x0 = lane, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  __syncwarp();
  const long long t0 = clock64();
  if (lane < active)
    for (int it = 0; it < kIters; ++it) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  __syncwarp();
  const long long t1 = clock64();
  out[threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (lane == 0) *cyc = t1 - t0;
}

// Latency of one instruction that depends on the previous one: one warp, one
// chain of kIters steps.  op 0: FP64 FMA, 1: FP64 multiply, 2: the FP64
// reciprocal seed rcp.approx.ftz.f64, 3: an FP32 -> FP64 -> FP32 conversion
// pair, 4: a 64-bit warp shuffle, 5: a shared-memory load whose address
// depends on the previous load.
__global__ void op_latency_kernel(int op, double* out, long long* cyc, double a, double b) {
  __shared__ int ring[64];
  ring[threadIdx.x] = (threadIdx.x + 1) & 31;
  ring[threadIdx.x + 32] = 0;
  double x = 0.5 + threadIdx.x * 1e-3;
  float f = 0.5f + threadIdx.x * 1e-3f;
  int k = threadIdx.x;
  __syncwarp();
  const long long t0 = clock64();
  switch (op) {
    case 0:
      for (int it = 0; it < kIters; ++it) x = fma(x, a, b);
      break;
    case 1:
      for (int it = 0; it < kIters; ++it) x = x * a;
      break;
    case 2:
      for (int it = 0; it < kIters; ++it) asm volatile("rcp.approx.ftz.f64 %0, %0;" : "+d"(x));
      break;
    case 3:
      for (int it = 0; it < kIters; ++it) {
        double d;
        asm volatile("cvt.f64.f32 %0, %1;" : "=d"(d) : "f"(f));
        asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(d));
      }
      x = f;
      break;
    case 4:
      for (int it = 0; it < kIters; ++it) x = __shfl_xor_sync(0xffffffffu, x, 1);
      break;
    default:
      for (int it = 0; it < kIters; ++it) k = ring[k];
      x = k;
      break;
  }
  __syncwarp();
  const long long t1 = clock64();
  out[threadIdx.x] = x;
  if (threadIdx.x == 0) *cyc = t1 - t0;
}

cudaError_t latency_cycles(void* scratch, int op, double* out) {
  double* o = (double*)scratch;
  long long* cyc = (long long*)((char*)scratch + 32 * sizeof(double));
  long long h = 0;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    op_latency_kernel<<<1, 32>>>(op, o, cyc, 0.999, 0.001);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
  *out = (double)h / kIters;
  return e;
}

template <class T>
cudaError_t issue_cycles(void* scratch, int active, double* out) {
  T* o = (T*)scratch;
  long long* cyc = (long long*)((char*)scratch + 32 * sizeof(double));
  long long h = 0;
  cudaError_t e = cudaSuccess;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
    fma_issue_kernel<T><<<1, 32>>>(o, cyc, active, (T)0.999, (T)0.001);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
  }
  if (e == cudaSuccess) e = cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
  *out = (double)h / (8.0 * kIters);
  return e;
}

lq_status probe_fail(cudaError_t e, const char* where) {
  return lq_internal_fail(LQ_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" lq_status lq_device_fp64_rate(double ms, double* host_tflops, double* host_cycles9) {
  if (!(ms > 0) || ms > 60000 || !host_tflops) return lq_internal_fail(LQ_EINVAL, "bad arguments to lq_device_fp64_rate");
  int dev = 0, sms = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return probe_fail(e, "device query");
  const int threads = 256, blocks = sms * 8;
  double* out = nullptr;
  e = cudaMalloc((void**)&out, sizeof(double) * threads * blocks);
  if (e != cudaSuccess) return probe_fail(e, "probe buffer");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  long long iters = 1024;
  float t = 0.f;
  // grow the loop until one launch takes about the requested time
  for (int round = 0; round < 12 && e == cudaSuccess; ++round) {
    e = cudaEventRecord(e0, 0);
    if (e == cudaSuccess) {
      fma_rate_kernel<<<blocks, threads>>>(out, iters, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e != cudaSuccess || t >= 0.5 * ms) break;
    const double grow = t > 0.f ? ms / t : 16.0;
    iters = (long long)(iters * (grow < 16.0 ? grow : 16.0)) + 1;
  }
  if (e == cudaSuccess && t > 0.f)
    *host_tflops = 2.0 * 8.0 * (double)iters * threads * blocks / (t * 1e-3) / 1e12;
  if (e == cudaSuccess && host_cycles9) {
    e = issue_cycles<double>(out, 1, &host_cycles9[0]);
    if (e == cudaSuccess) e = issue_cycles<double>(out, 32, &host_cycles9[1]);
    if (e == cudaSuccess) e = issue_cycles<float>(out, 32, &host_cycles9[2]);
    for (int op = 0; op < 6 && e == cudaSuccess; ++op) e = latency_cycles(out, op, &host_cycles9[3 + op]);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  if (e != cudaSuccess) return probe_fail(e, "fp64 rate probe");
  return LQ_OK;
}

extern "C" lq_status lq_test_quotient(int32_t n, const double* host_d, const double* host_r, double* host_q,
                                      double* host_q_ieee) {
  if (n < 0 || (n > 0 && (!host_d || !host_r || !host_q || !host_q_ieee)))
    return lq_internal_fail(LQ_EINVAL, "bad arguments to lq_test_quotient");
  if (n == 0) return LQ_OK;
  double* buf = nullptr;
  const size_t b = sizeof(double) * (size_t)n;
  cudaError_t e = cudaMalloc((void**)&buf, 4 * b);
  if (e != cudaSuccess) return probe_fail(e, "quotient buffers");
  e = cudaMemcpy(buf, host_d, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(buf + n, host_r, b, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = lq::launch_quotient(buf, buf + n, n, buf + 2 * (size_t)n, buf + 3 * (size_t)n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(host_q, buf + 2 * (size_t)n, b, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(host_q_ieee, buf + 3 * (size_t)n, b, cudaMemcpyDeviceToHost);
  cudaFree(buf);
  if (e != cudaSuccess) return probe_fail(e, "quotient test");
  return LQ_OK;
}
