// Pipe throughput probe for the rooflines of the warp-level tensor kernels:
// peaks of mma.sync m8n8k4 f64 (DMMA), of scalar DFMA, and of mma.sync
// m16n8k16 BF16 with FP32 accumulation (the instruction of the sliced
// products) on this device.  Register-only loops; every thread writes one
// value to its own slot.  Prints one JSON line.
// Build: nvcc -gencode arch=compute_103a,code=sm_103a -O3
#include <cstdio>
#include <cuda_runtime.h>

#define ITERS 2048

__global__ void k_dmma(double *out, double a) {
  double A = a + threadIdx.x * 1e-12, B = a - threadIdx.x * 1e-12;
  double c[8][2] = {};
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[q][0]), "+d"(c[q][1]) : "d"(A), "d"(B));
  }
  double s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += c[q][0] + c[q][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_dfma(double *out, double a, double b) {
  double x[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) x[q] = threadIdx.x * 1e-9 + q;
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q) x[q] = fma(x[q], a, b);
  }
  double s = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += x[q];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void k_hmma_bf16(float *out, unsigned a) {
  const unsigned A0 = a, A1 = a ^ (threadIdx.x & 1u), B0 = a;
  float c[8][4] = {};
  for (int i = 0; i < ITERS; ++i) {
#pragma unroll
    for (int q = 0; q < 8; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
          : "r"(A0), "r"(A1), "r"(A0), "r"(A1), "r"(B0), "r"(B0));
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += c[q][0] + c[q][1] + c[q][2] + c[q][3];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int main() {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, 0) != cudaSuccess) return 1;
  const int blocks = p.multiProcessorCount * 8, threads = 256;
  const size_t n = (size_t)blocks * threads;
  double *d = nullptr;
  if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms;
  double best_mma = 0, best_fma = 0, best_bf16 = 0;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0);
    k_dmma<<<blocks, threads>>>(d, 0.5);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    // per warp and iteration: 8 mma of 8x8x4 multiply-adds
    double fl = 2.0 * 8 * 8 * 4 * 8.0 * ITERS * (double)(n / 32);
    if (fl / ms / 1e9 > best_mma) best_mma = fl / ms / 1e9;
    cudaEventRecord(e0);
    k_dfma<<<blocks, threads>>>(d, 0.999999, 1e-7);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    fl = 2.0 * 8 * ITERS * (double)n;
    if (fl / ms / 1e9 > best_fma) best_fma = fl / ms / 1e9;
    cudaEventRecord(e0);
    k_hmma_bf16<<<blocks, threads>>>(reinterpret_cast<float *>(d), 0x3f803f80u);  // bf16 pairs (1, 1)
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    // per warp and iteration: 8 mma of 16x8x16 multiply-adds
    fl = 2.0 * 16 * 8 * 16 * 8.0 * ITERS * (double)(n / 32);
    if (fl / ms / 1e9 > best_bf16) best_bf16 = fl / ms / 1e9;
  }
  cudaError_t err = cudaGetLastError();
  printf("{\"fp64_dmma_tflops\": %.4f, \"fp64_dfma_tflops\": %.4f, \"mma_sync_bf16_tflops\": %.1f, \"sms\": %d, "
         "\"ok\": %s}\n",
         best_mma, best_fma, best_bf16, p.multiProcessorCount, err == cudaSuccess ? "true" : "false");
  cudaFree(d);
  return err == cudaSuccess ? 0 : 1;
}
