// Cost of one warp instruction on one SM sub-partition: DFMA with 1 and 32
// active lanes, and FFMA.  One block of one warp; every thread writes only
// out[threadIdx.x]; no waits.  Prints "name cycles_per_instruction".
#include <cstdio>
#include <cuda_runtime.h>

#define ITERS 4096

template <class T>
__global__ void chain8(T* out, long long* cyc, int active, T a, T b) {
  const int lane = threadIdx.x & 31;
  T x0 = lane, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
  __syncwarp();
  const long long t0 = clock64();
  if (lane < active)
    for (int it = 0; it < ITERS; ++it) {
      x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
      x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
  __syncwarp();
  const long long t1 = clock64();
  out[threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
  if (lane == 0) *cyc = t1 - t0;
}

template <class T>
static double run(int active) {
  T* out;
  long long* cyc;
  cudaMalloc(&out, 32 * sizeof(T));
  cudaMalloc(&cyc, sizeof(long long));
  long long h = 0;
  for (int rep = 0; rep < 2; ++rep) {
    chain8<T><<<1, 32>>>(out, cyc, active, (T)0.999, (T)0.001);
    cudaDeviceSynchronize();
  }
  cudaMemcpy(&h, cyc, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(out);
  cudaFree(cyc);
  return (double)h / (8.0 * ITERS);
}

int main() {
  printf("dfma_1lane %.2f\n", run<double>(1));
  printf("dfma_32lanes %.2f\n", run<double>(32));
  printf("ffma_32lanes %.2f\n", run<float>(32));
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
