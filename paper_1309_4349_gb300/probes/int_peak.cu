// int_peak.cu -- measures the integer issue rate that bounds the sweep kernel:
// LOP3 (3-input logic, the bit-sliced adder tree), IMAD.WIDE.U32 (the 32x32->64
// products of Philox) and whole Philox4x32-10 evaluations, over a full-GPU grid.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o int_peak int_peak.cu && ./int_peak
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d; asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); return d; }
__global__ void k_lop3(uint32_t* out, int iters) {
  uint32_t r[8]; for (int i = 0; i < 8; ++i) r[i] = threadIdx.x * (i + 3) + blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) r[i] = lop3(r[i], r[(i + 1) & 7], r[(i + 3) & 7]);
  }
  uint32_t x = 0; for (int i = 0; i < 8; ++i) x ^= r[i];
  if (x == 0x12345678u) out[0] = x;
}
__global__ void k_imadw(uint32_t* out, int iters) {
  uint32_t r[8]; for (int i = 0; i < 8; ++i) r[i] = threadIdx.x * (i + 3) + blockIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      unsigned long long p; asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(r[i]), "r"(0xD2511F53u));
      r[i] = (uint32_t)p; r[i + 1] ^= (uint32_t)(p >> 32);
    }
  }
  uint32_t x = 0; for (int i = 0; i < 8; ++i) x ^= r[i];
  if (x == 0x12345678u) out[0] = x;
}
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53ull, p1 = (unsigned long long)c2 * 0xCD9E8D57ull;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1; c3 = (uint32_t)p0; c0 = n0; c2 = n2; k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return c0;
}
__global__ void k_philox(uint32_t* out, int iters, uint32_t k0, uint32_t k1) {
  uint32_t acc = 0, base = blockIdx.x * blockDim.x + threadIdx.x;
  for (int it = 0; it < iters; ++it) acc ^= philox_w0(base + it * 7919u, 3u, (uint32_t)it, 0u, k0, k1);
  if (acc == 0x12345678u) out[0] = acc;
}
int main() {
  cudaDeviceProp p; cudaGetDeviceProperties(&p, 0);
  int sms = p.multiProcessorCount; printf("SMs %d\n", sms);
  uint32_t* out; cudaMalloc(&out, 4);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  int blocks = sms * 8, threads = 256, iters = 20000;
  for (int rep = 0; rep < 2; ++rep) {
    float ms;
    cudaEventRecord(a); k_lop3<<<blocks, threads>>>(out, iters); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    double ops = (double)blocks * threads * iters * 8;
    printf("lop3: %.3f Tops/s lane, %.1f lane-ops/clk/SM at 2070 MHz, ms=%.3f\n", ops / ms / 1e9, ops / (ms * 1e-3) / sms / 2.07e9, ms);
    cudaEventRecord(a); k_imadw<<<blocks, threads>>>(out, iters); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    ops = (double)blocks * threads * iters * 4;  // 4 mul.wide per iter (each with an xor too)
    printf("imad.wide(+xor): %.3f T mul.wide/s lane, %.1f per clk/SM @2.07GHz ms=%.3f\n", ops / ms / 1e9, ops / (ms * 1e-3) / sms / 2.07e9, ms);
    int pit = 2000;
    cudaEventRecord(a); k_philox<<<blocks, threads>>>(out, pit, 1u, 2u); cudaEventRecord(b); cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    double n = (double)blocks * threads * pit;
    printf("philox4x32-10 (w0): %.3f G draws/s, %.2f ns per draw-lane, %.1f clk/draw/SM-lane-group @2.07GHz ms=%.3f\n", n / ms / 1e6, ms * 1e6 / n, (ms*1e-3) * sms * 2.07e9 * 128 / n, ms);
  }
  return 0;
}
