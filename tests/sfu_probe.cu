// Test kernel: SFU sin/cos (the __sincosf intrinsic) of FP32 arguments, for tests/test_sfu.py.
#include <cuda_runtime.h>
__global__ void k_sfu(const float* x, float* s, float* c, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { float a, b; __sincosf(x[i], &a, &b); s[i] = a; c[i] = b; }
}
extern "C" int sfu_eval(const float* hx, float* hs, float* hc, int n) {
  float *x, *s, *c;
  if (cudaMalloc(&x, n * 4) || cudaMalloc(&s, n * 4) || cudaMalloc(&c, n * 4)) return 1;
  cudaMemcpy(x, hx, n * 4, cudaMemcpyHostToDevice);
  k_sfu<<<(n + 255) / 256, 256>>>(x, s, c, n);
  cudaMemcpy(hs, s, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(hc, c, n * 4, cudaMemcpyDeviceToHost);
  cudaFree(x); cudaFree(s); cudaFree(c);
  return (int)cudaGetLastError();
}
