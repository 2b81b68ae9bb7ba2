// Test fixture of tests/test_df_reduction_gpu.py: runs the FP64-accurate kernel's phase reduction
// (paper_1910_10391_gb300/csrc/rad_df_reduce.cuh) on the GPU for an array of phases and returns
// j and the float-pair remainder (xh, xl) of each.
#include <cuda_runtime.h>

#include "../paper_1910_10391_gb300/csrc/rad_df_reduce.cuh"

__global__ void k_reduce_probe(const double *phi, int n, int *j, float *xh, float *xl) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float h, l;
  j[i] = rad::dfr::reduce_phase(phi[i], h, l);
  xh[i] = h;
  xl[i] = l;
}

// Host arrays in and out; returns 0 or the CUDA error code.
extern "C" int reduce_probe(const double *h_phi, int n, int *h_j, float *h_xh, float *h_xl) {
  double *d_phi = nullptr;
  int *d_j = nullptr;
  float *d_xh = nullptr, *d_xl = nullptr;
  const size_t nn = static_cast<size_t>(n);
  cudaError_t e = cudaMalloc(&d_phi, nn * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_j, nn * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&d_xh, nn * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_xl, nn * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(d_phi, h_phi, nn * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && n > 0) {
    k_reduce_probe<<<(n + 255) / 256, 256>>>(d_phi, n, d_j, d_xh, d_xl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h_j, d_j, nn * sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_xh, d_xh, nn * sizeof(float), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(h_xl, d_xl, nn * sizeof(float), cudaMemcpyDeviceToHost);
  cudaFree(d_phi);
  cudaFree(d_j);
  cudaFree(d_xh);
  cudaFree(d_xl);
  return static_cast<int>(e);
}
