// clusters.cu -- cluster-size histogram of one lipid species (section "Cluster
// Analysis methods": clusters of like lipids over the six nearest neighbours, an
// O(n) labelling, the distribution of cluster sizes).
//
// Labelling is a concurrent union-find over the sites of the species: every
// bond (site, site + o) with both ends of the species unites the two trees by
// hooking the larger root under the smaller with an atomic compare-and-swap
// (lock-free union as in Jaiganesh & Burtscher, ECL-CC, 2018).  Parents always
// point to smaller indices, so every root is the smallest site index of its
// component and the final labelling is deterministic.  Then: component sizes at
// the roots, a dense histogram of sizes with a bitmap of occupied sizes, and a
// single-CTA compaction into an ascending sparse list.  The histogram and the
// bitmap are returned to zero by the compaction, so no clearing pass is needed.
#include "klmc_internal.h"

namespace klmc {
namespace {

constexpr int kBlock = 256;
constexpr int kCompactThreads = 1024;

__device__ __forceinline__ uint32_t site_at(const void *lat, int packing, int pitch, int x, int y)
{
    if (packing == kPackBit) {
        const uint32_t *row = (const uint32_t *)lat + (size_t)y * pitch;
        return (row[x >> 5] >> (x & 31)) & 1u;
    }
    return ((const uint8_t *)lat)[(size_t)y * pitch + x] ? 1u : 0u;
}

// Root of x, shortening the path on the way: every visited node is re-pointed to
// its grandparent (pointer jumping).  That write is always an ancestor, and only
// non-roots are written, so it is safe next to the compare-and-swap on roots.
__device__ __forceinline__ int find_root(volatile int32_t *parent, int x)
{
    int p = parent[x];
    if (p == x) return x;
    int prev = x;
    int next;
    while (p != (next = parent[p])) {
        parent[prev] = next;
        prev = p;
        p = next;
    }
    return p;
}

__device__ __forceinline__ void unite(int32_t *parent, int a, int b)
{
    while (true) {
        a = find_root((volatile int32_t *)parent, a);
        b = find_root((volatile int32_t *)parent, b);
        if (a == b) return;
        if (a < b) {
            const int t = a;
            a = b;
            b = t;
        }
        // a > b: hook root a under b; if a stopped being a root, retry from there.
        const int old = atomicCAS(parent + a, a, b);
        if (old == a) return;
        a = old;
    }
}

__global__ void cc_init_kernel(const void *lat, int packing, int Lx, int Ly, int pitch, int species,
                               int32_t *parent, int32_t *csize)
{
    const long long N = (long long)Lx * Ly;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
        parent[i] = site_at(lat, packing, pitch, x, y) == (uint32_t)species ? (int32_t)i : -1;
        csize[i] = 0;
    }
}

// Bonds {i, i+o}, o in (1,0), (0,1) and, for TRI6, (1,-1), with periodic wrap or
// (helical) the x wrap carrying into the next or previous row.
__global__ void cc_union_kernel(int Lx, int Ly, int geometry, int helical, int32_t *parent)
{
    const long long N = (long long)Lx * Ly;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        if (parent[i] < 0) continue;
        const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
        const bool xe = x + 1 == Lx;
        const int xp = xe ? 0 : x + 1;
        const int yp = y + 1 == Ly ? 0 : y + 1;
        const int ym = y == 0 ? Ly - 1 : y - 1;
        const int self = (int)i;
        const int j0 = (helical && xe ? yp : y) * Lx + xp;
        if (parent[j0] >= 0) unite(parent, self, j0);
        const int j1 = yp * Lx + x;
        if (parent[j1] >= 0) unite(parent, self, j1);
        if (geometry == kTRI6) {
            const int j2 = (helical && xe ? y : ym) * Lx + xp;
            if (parent[j2] >= 0) unite(parent, self, j2);
        }
    }
}

__global__ void cc_size_kernel(long long N, int32_t *parent, int32_t *csize)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        if (parent[i] < 0) continue;
        const int r = find_root((volatile int32_t *)parent, (int)i);
        parent[i] = r;  // an ancestor: concurrent finds stay valid
        atomicAdd(csize + r, 1);
    }
}

__global__ void cc_hist_kernel(long long N, const int32_t *parent, const int32_t *csize,
                               int32_t *hist, uint32_t *bitmap)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        if (parent[i] != (int32_t)i) continue;
        const int s = csize[i];
        if (atomicAdd(hist + s, 1) == 0) atomicOr(bitmap + (s >> 5), 1u << (s & 31));
    }
}

// Ascending (size, count) pairs from the occupied-size bitmap; clears what it reads.
__global__ void __launch_bounds__(kCompactThreads)
cc_compact_kernel(int32_t *hist, uint32_t *bitmap, long long nwords, long long *sizes,
                  long long *counts, long long capacity, long long *n_distinct)
{
    __shared__ int warp_tot[kCompactThreads / 32];
    __shared__ long long base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) base = 0;
    __syncthreads();
    for (long long w0 = 0; w0 < nwords; w0 += kCompactThreads) {
        const long long w = w0 + tid;
        uint32_t bits = w < nwords ? bitmap[w] : 0u;
        const int c = __popc(bits);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) warp_tot[warp] = incl;
        __syncthreads();
        int warp_off = 0, total = 0;
        for (int k = 0; k < kCompactThreads / 32; ++k) {
            if (k < warp) warp_off += warp_tot[k];
            total += warp_tot[k];
        }
        long long pos = base + warp_off + incl - c;
        if (bits) bitmap[w] = 0u;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const long long s = w * 32 + b;
            const int cnt = hist[s];
            hist[s] = 0;
            if (pos < capacity) {
                sizes[pos] = s;
                counts[pos] = cnt;
            }
            ++pos;
        }
        __syncthreads();
        if (tid == 0) base += total;
        __syncthreads();
    }
    if (tid == 0) *n_distinct = base;
}

int grid_for(long long work)
{
    long long g = (work + kBlock * 4 - 1) / (kBlock * 4);
    if (g < 1) g = 1;
    if (g > 152 * 8) g = 152 * 8;
    return (int)g;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

size_t cluster_scratch_bytes(long long N, long long n_species_max)
{
    const long long nwords = (n_species_max + 1 + 31) / 32;
    return align256((size_t)N * 4) * 2 + align256((size_t)(n_species_max + 1) * 4) +
           align256((size_t)nwords * 4);
}

void cluster_scratch_carve(void *base, long long N, long long n_species_max, ClusterScratch *s)
{
    const long long nwords = (n_species_max + 1 + 31) / 32;
    char *p = (char *)base;
    s->parent = (int32_t *)p;
    p += align256((size_t)N * 4);
    s->csize = (int32_t *)p;
    p += align256((size_t)N * 4);
    s->hist = (int32_t *)p;
    p += align256((size_t)(n_species_max + 1) * 4);
    s->bitmap = (uint32_t *)p;
    (void)nwords;
    s->n_species_max = n_species_max;
}

cudaError_t cluster_scratch_clear(const ClusterScratch &s, cudaStream_t stream)
{
    const long long nwords = (s.n_species_max + 1 + 31) / 32;
    cudaError_t e = cudaMemsetAsync(s.hist, 0, (size_t)(s.n_species_max + 1) * 4, stream);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(s.bitmap, 0, (size_t)nwords * 4, stream);
}

cudaError_t launch_cluster_histogram(const void *lat, int packing, int Lx, int Ly, int pitch,
                                     int geometry, int species, const ClusterScratch &s,
                                     long long *sizes, long long *counts, long long capacity,
                                     long long *n_distinct, cudaStream_t stream, int helical)
{
    const long long N = (long long)Lx * Ly;
    const int g = grid_for(N);
    cc_init_kernel<<<g, kBlock, 0, stream>>>(lat, packing, Lx, Ly, pitch, species, s.parent, s.csize);
    cc_union_kernel<<<g, kBlock, 0, stream>>>(Lx, Ly, geometry, helical, s.parent);
    cc_size_kernel<<<g, kBlock, 0, stream>>>(N, s.parent, s.csize);
    cc_hist_kernel<<<g, kBlock, 0, stream>>>(N, s.parent, s.csize, s.hist, s.bitmap);
    const long long nwords = (s.n_species_max + 1 + 31) / 32;
    cc_compact_kernel<<<1, kCompactThreads, 0, stream>>>(s.hist, s.bitmap, nwords, sizes, counts,
                                                         capacity, n_distinct);
    return cudaGetLastError();
}

}  // namespace klmc
