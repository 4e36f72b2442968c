// Test probe (not part of the library): applies the library's f2d_exact to an
// array on the GPU so tests can compare it with an exact host widening.
#include <cuda_runtime.h>
#include "../../paper_1603_04570_gb300/csrc/ok_internal.cuh"

namespace okg {
std::atomic<long long> g_launch_count{0};
thread_local bool g_pdl = false;
}

__global__ void k_widen(const float* in, double* out, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = okg::f2d_exact(in[i]);
}

extern "C" int widen_probe(const float* h_in, double* h_out, int n) {
  float* d_in = nullptr;
  double* d_out = nullptr;
  if (cudaMalloc(&d_in, n * sizeof(float)) != cudaSuccess) return 1;
  if (cudaMalloc(&d_out, n * sizeof(double)) != cudaSuccess) return 1;
  cudaMemcpy(d_in, h_in, n * sizeof(float), cudaMemcpyHostToDevice);
  k_widen<<<(n + 127) / 128, 128>>>(d_in, d_out, n);
  cudaMemcpy(h_out, d_out, n * sizeof(double), cudaMemcpyDeviceToHost);
  const cudaError_t e = cudaGetLastError();
  cudaFree(d_in);
  cudaFree(d_out);
  return e == cudaSuccess ? 0 : 2;
}
