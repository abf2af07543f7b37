// cluster_barrier.cu -- measures the per-phase synchronisation cost options of the
// resident sweep: __syncthreads at 1024 threads, and a thread-block-cluster barrier
// (sizes 2..16, 256..1024 threads) together with 32 remote distributed-shared-memory
// atomics per iteration.
// Build and run: nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o cluster_barrier cluster_barrier.cu && ./cluster_barrier
#include <cstdio>
#include <cstdint>
#include <cooperative_groups.h>
#include <cuda_runtime.h>
namespace cg = cooperative_groups;
__global__ void k_sync(uint32_t* out, int iters) {
  __shared__ uint32_t s[1024];
  uint32_t v = threadIdx.x;
  for (int i = 0; i < iters; ++i) { s[threadIdx.x] = v; __syncthreads(); v += s[(threadIdx.x + 1) & 1023]; __syncthreads(); }
  if (v == 0x12345678u) out[0] = v;
}
__global__ void k_cluster(uint32_t* out, int iters) {
  __shared__ uint32_t s[1024];
  cg::cluster_group cl = cg::this_cluster();
  uint32_t v = threadIdx.x;
  unsigned rank = cl.block_rank(), n = cl.num_blocks();
  uint32_t* peer = cl.map_shared_rank(s, (rank + 1) % n);
  s[threadIdx.x] = 0;
  cl.sync();
  for (int i = 0; i < iters; ++i) {
    if (threadIdx.x < 32) atomicXor(peer + threadIdx.x, v);   // remote DSMEM atomics
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    v += s[threadIdx.x & 31];
  }
  cl.sync();
  if (v == 0x12345678u) out[0] = v;
}
int main() {
  uint32_t* out; cudaMalloc(&out, 4);
  cudaEvent_t a, b; cudaEventCreate(&a); cudaEventCreate(&b);
  float ms; int iters = 20000;
  k_sync<<<1, 1024>>>(out, 100); cudaDeviceSynchronize();
  cudaEventRecord(a); k_sync<<<1, 1024>>>(out, iters); cudaEventRecord(b); cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b); printf("__syncthreads x2 per iter, 1024 thr: %.1f ns per barrier\n", ms * 1e6 / iters / 2);
  cudaEventRecord(a); k_sync<<<152, 1024>>>(out, iters); cudaEventRecord(b); cudaEventSynchronize(b);
  cudaEventElapsedTime(&ms, a, b); printf("same, 152 CTAs: %.1f ns per barrier\n", ms * 1e6 / iters / 2);
  cudaError_t e = cudaFuncSetAttribute(k_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  printf("nonportable attr: %s\n", cudaGetErrorString(e));
  int threads_list[3] = {1024, 512, 256};
  for (int ti = 0; ti < 3; ++ti) {
    for (int cs = 2; cs <= 16; cs *= 2) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs * 5); cfg.blockDim = dim3(threads_list[ti]); cfg.dynamicSmemBytes = 0;
      cudaLaunchAttribute attr[1]; attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = cs; attr[0].val.clusterDim.y = 1; attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr; cfg.numAttrs = 1;
      int ncl = 0; cudaOccupancyMaxActiveClusters(&ncl, (void*)k_cluster, &cfg);
      e = cudaLaunchKernelEx(&cfg, k_cluster, out, 100); cudaDeviceSynchronize();
      if (e != cudaSuccess) { printf("cluster %d launch failed: %s\n", cs, cudaGetErrorString(e)); cudaGetLastError(); continue; }
      cudaEventRecord(a); cudaLaunchKernelEx(&cfg, k_cluster, out, iters); cudaEventRecord(b); cudaEventSynchronize(b);
      cudaEventElapsedTime(&ms, a, b);
      printf("threads %d cluster %2d (x5 clusters, max active clusters %d): %.1f ns per iter (barrier + 32 remote atomics)\n", threads_list[ti], cs, ncl, ms * 1e6 / iters);
    }
  }
  printf("last error: %s\n", cudaGetErrorString(cudaGetLastError()));
  return 0;
}
