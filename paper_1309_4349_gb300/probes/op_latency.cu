// op_latency.cu -- single-warp and 8-warp latencies of the operations on the sweep
// kernel's critical path: one Philox4x32-10 evaluation (one, two and four
// independent chains), shared-memory XOR reductions, dependent shared loads, warp
// shuffles, LOP3 and 32x32->64 multiplies; clock64 overhead for reference.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o op_latency op_latency.cu && ./op_latency
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
__device__ __forceinline__ uint32_t philox_w0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53ull, p1 = (unsigned long long)c2 * 0xCD9E8D57ull;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    c1 = (uint32_t)p1; c3 = (uint32_t)p0; c0 = n0; c2 = n2; k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return c0;
}
__global__ void k(unsigned long long* out, uint32_t seed) {
  __shared__ uint32_t sm[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) sm[i] = i;
  __syncthreads();
  uint32_t x = seed + threadIdx.x;
  long long t0, t1;
  // 1. clock64 overhead
  t0 = clock64(); t1 = clock64(); out[0] = t1 - t0;
  // 2. single philox, dependent chain of 8
  t0 = clock64();
  for (int i = 0; i < 8; ++i) x = philox_w0(x, 3u, 7u, 0u, 11u, 13u);
  t1 = clock64(); out[1] = (t1 - t0) / 8;
  // 3. two independent chains of 8 (interleaved)
  uint32_t y = x ^ 0x55u;
  t0 = clock64();
  for (int i = 0; i < 8; ++i) { x = philox_w0(x, 3u, 7u, 0u, 11u, 13u); y = philox_w0(y, 3u, 7u, 0u, 11u, 13u); }
  t1 = clock64(); out[2] = (t1 - t0) / 8;
  // 4. four independent chains
  uint32_t z = x ^ 0x77u, w = y ^ 0x99u;
  t0 = clock64();
  for (int i = 0; i < 8; ++i) { x = philox_w0(x, 3u, 7u, 0u, 11u, 13u); y = philox_w0(y, 3u, 7u, 0u, 11u, 13u); z = philox_w0(z, 3u, 7u, 0u, 11u, 13u); w = philox_w0(w, 3u, 7u, 0u, 11u, 13u); }
  t1 = clock64(); out[3] = (t1 - t0) / 8;
  // 5. 16 red.shared.xor to distinct words per lane (fire and forget), then a dependent load
  uint32_t base = (uint32_t)__cvta_generic_to_shared(sm);
  t0 = clock64();
  for (int i = 0; i < 16; ++i) asm volatile("red.shared.xor.b32 [%0], %1;" :: "r"(base + 4u * ((threadIdx.x + 32 * i) & 1023)), "r"(x) : "memory");
  t1 = clock64(); out[4] = (t1 - t0) / 16;
  // 6. atomicXor (returning) chain
  t0 = clock64();
  uint32_t v = x;
  for (int i = 0; i < 16; ++i) v = atomicXor(&sm[(threadIdx.x + 32 * i + (v & 1)) & 1023], v);
  t1 = clock64(); out[5] = (t1 - t0) / 16;
  // 7. dependent LDS chain
  t0 = clock64();
  uint32_t idx = threadIdx.x;
  for (int i = 0; i < 16; ++i) idx = sm[idx & 1023] + 1;
  t1 = clock64(); out[6] = (t1 - t0) / 16;
  // 8. dependent shfl chain
  t0 = clock64();
  uint32_t s = x;
  for (int i = 0; i < 16; ++i) s = __shfl_xor_sync(0xFFFFFFFFu, s, 1) + 1;
  t1 = clock64(); out[7] = (t1 - t0) / 16;
  // 9. dependent LOP3 chain
  t0 = clock64();
  uint32_t a = x, b = y, c = z;
  for (int i = 0; i < 32; ++i) { uint32_t d; asm volatile("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c)); a = d; }
  t1 = clock64(); out[8] = (t1 - t0) / 32;
  // 10. dependent mul.wide chain
  t0 = clock64();
  uint32_t m = x;
  for (int i = 0; i < 32; ++i) { unsigned long long p; asm volatile("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(m), "r"(0xD2511F53u)); m = (uint32_t)(p >> 32) ^ (uint32_t)p; }
  t1 = clock64(); out[9] = (t1 - t0) / 32;
  out[10] = x ^ y ^ z ^ w ^ v ^ idx ^ s ^ a ^ m;
}
int main() {
  unsigned long long* d; cudaMalloc(&d, 16 * 8);
  const char* names[] = {"clock64 pair", "philox (1 chain) per eval", "philox x2 chains per pair", "philox x4 chains per quad", "red.shared.xor issue per op", "atomicXor dependent per op", "LDS dependent", "SHFL dependent", "LOP3 dependent", "mul.wide+xor dependent"};
  for (int threads : {32, 256}) {
    k<<<1, threads>>>(d, 1u); cudaDeviceSynchronize();
    k<<<1, threads>>>(d, 2u); cudaDeviceSynchronize();
    unsigned long long h[16]; cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    printf("threads=%d\n", threads);
    for (int i = 0; i < 10; ++i) printf("  %-32s %llu cycles\n", names[i], h[i]);
  }
  printf("%s\n", cudaGetErrorString(cudaGetLastError()));
}
