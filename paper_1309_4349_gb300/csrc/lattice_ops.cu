// lattice_ops.cu -- initial placement, energy recount, and lattice (un)packing.
//
// Initial placement (Fig. 2: lipids randomly distributed over the lattice, the
// number of each type fixed): every site i gets the 96-bit key (K64_i, i), K64_i a
// 64-bit Philox value; the n_A sites with the smallest keys are A.  The keys are
// distinct, so this is a uniformly random n_A-subset.  It is computed by a radix
// select over 8-bit digits, most significant first, recomputing the keys in every
// pass instead of storing them; it stops as soon as the selected bucket is taken
// whole.
#include <string.h>

#include "klmc_internal.h"
#include "philox.cuh"

namespace klmc {
namespace {

constexpr int kBlock = 256;


// Placement key of site i: Philox counter {i, 0xFFFFFFFF, 0, 0}, words w1:w0.
__device__ __forceinline__ unsigned long long site_key(uint32_t i, uint32_t k0, uint32_t k1)
{
    const Philox4 w = philox4(i, 0xFFFFFFFFu, 0u, 0u, k0, k1);
    return ((unsigned long long)w.v[1] << 32) | w.v[0];
}

struct SelectState {
    unsigned long long p_hi;  // fixed key bits, left-aligned in the 96-bit key
    unsigned int p_lo;
    int nbits;                // number of fixed bits
    long long k;              // rank (1-based) still to reach inside the prefix bucket
    int done;
    int pad;
    unsigned long long hist[256];
};

__device__ __forceinline__ void key_masks(int nbits, unsigned long long &mh, unsigned int &ml)
{
    mh = nbits >= 64 ? ~0ull : (nbits == 0 ? 0ull : (~0ull << (64 - nbits)));
    ml = nbits <= 64 ? 0u : (~0u << (96 - nbits));
}

__global__ void select_hist_kernel(long long N, uint32_t k0, uint32_t k1, SelectState *st)
{
    __shared__ unsigned int h[256];
    if (st->done) return;
    const int nbits = st->nbits;
    const unsigned long long p_hi = st->p_hi;
    const unsigned int p_lo = st->p_lo;
    unsigned long long mh;
    unsigned int ml;
    key_masks(nbits, mh, ml);
    for (int b = threadIdx.x; b < 256; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long kh = site_key((uint32_t)i, k0, k1);
        const unsigned int kl = (unsigned int)i;
        if ((kh & mh) != p_hi || (kl & ml) != p_lo) continue;
        const unsigned int digit =
            nbits < 64 ? (unsigned int)(kh >> (56 - nbits)) & 0xFFu : (kl >> (88 - nbits)) & 0xFFu;
        atomicAdd(&h[digit], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b]) atomicAdd(&st->hist[b], (unsigned long long)h[b]);
}

__global__ void select_pick_kernel(SelectState *st)
{
    if (threadIdx.x != 0 || st->done) return;
    unsigned long long before = 0;
    int b = 0;
    for (; b < 255; ++b) {
        if ((long long)(before + st->hist[b]) >= st->k) break;
        before += st->hist[b];
    }
    const unsigned long long cnt = st->hist[b];
    const int nbits = st->nbits;
    if (nbits < 64)
        st->p_hi |= (unsigned long long)b << (56 - nbits);
    else
        st->p_lo |= (unsigned int)b << (88 - nbits);
    st->k -= (long long)before;
    st->nbits = nbits + 8;
    if ((long long)cnt == st->k || st->nbits >= 96) st->done = 1;
    for (int i = 0; i < 256; ++i) st->hist[i] = 0ull;
}

// mode 0: none are A; 1: all are A; 2: A iff the key's fixed top bits <= prefix.
__device__ __forceinline__ uint32_t is_A(uint32_t i, uint32_t k0, uint32_t k1, int mode,
                                         const SelectState &st)
{
    if (mode != 2) return (uint32_t)mode;
    unsigned long long mh;
    unsigned int ml;
    key_masks(st.nbits, mh, ml);
    const unsigned long long kh = site_key(i, k0, k1) & mh;
    const unsigned int kl = i & ml;
    return (kh < st.p_hi || (kh == st.p_hi && kl <= st.p_lo)) ? 1u : 0u;
}

__global__ void mark_kernel(void *lat, int packing, int Lx, int Ly, int pitch, uint32_t k0,
                            uint32_t k1, int mode, const SelectState *st_ptr)
{
    SelectState st;
    st.p_hi = st_ptr->p_hi;
    st.p_lo = st_ptr->p_lo;
    st.nbits = st_ptr->nbits;
    if (packing == kPackBit) {
        const int W = (Lx + 31) / 32;
        const long long nwords = (long long)W * Ly;
        const int lane = threadIdx.x & 31;
        for (long long wi = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; wi < nwords;
             wi += ((long long)gridDim.x * blockDim.x) >> 5) {
            const int y = (int)(wi / W), w = (int)(wi - (long long)y * W);
            const int x = 32 * w + lane;
            uint32_t a = 0u;
            if (x < Lx) a = is_A((uint32_t)((long long)y * Lx + x), k0, k1, mode, st);
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, a != 0u);
            if (lane == 0) ((uint32_t *)lat)[(size_t)y * pitch + w] = word;
        }
    } else {
        const long long N = (long long)Lx * Ly;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
             i += (long long)gridDim.x * blockDim.x) {
            const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
            ((uint8_t *)lat)[(size_t)y * pitch + x] = (uint8_t)is_A((uint32_t)i, k0, k1, mode, st);
        }
    }
}

__device__ __forceinline__ uint32_t site_at(const void *lat, int packing, int pitch, int x, int y)
{
    if (packing == kPackBit) {
        const uint32_t *row = (const uint32_t *)lat + (size_t)y * pitch;
        return (row[x >> 5] >> (x & 31)) & 1u;
    }
    return ((const uint8_t *)lat)[(size_t)y * pitch + x] ? 1u : 0u;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ void block_add(long long v, long long *out)
{
    __shared__ long long part[32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        long long s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
        s = warp_sum(s);
        if (threadIdx.x == 0 && s != 0) atomicAdd((unsigned long long *)out, (unsigned long long)s);
    }
}

// Unlike bonds: every site with its forward orientations (TRI6: (1,0), (0,1),
// (1,-1); SQ4: (1,0), (0,1)), each bond once.
// Unlike bonds {i, i+o}, o in (1,0), (0,1) and, for TRI6, (1,-1): periodic wrap of x
// and y, or (helical) the x wrap carrying into the next or previous row.
__global__ void recount_kernel(const void *lat, int packing, int Lx, int Ly, int pitch, int geometry,
                               int helical, long long *out)
{
    long long n = 0;
    const long long N = (long long)Lx * Ly;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
        const bool xe = x + 1 == Lx;
        const int xp = xe ? 0 : x + 1;
        const int yp = y + 1 == Ly ? 0 : y + 1;
        const int ym = y == 0 ? Ly - 1 : y - 1;
        const uint32_t t = site_at(lat, packing, pitch, x, y);
        n += t != site_at(lat, packing, pitch, xp, helical && xe ? yp : y);
        n += t != site_at(lat, packing, pitch, x, yp);
        if (geometry == kTRI6) n += t != site_at(lat, packing, pitch, xp, helical && xe ? y : ym);
    }
    block_add(n, out);
}

// Fraction of first neighbours, random-neighbour estimator (sample m): the number
// of sites whose chosen nearest neighbour has the same type.  Site i's neighbour is
// direction floor(w z / 2^32) of (1,0), (-1,0), (0,1), (0,-1), (1,-1), (-1,1) (the
// first four for SQ4), w = word (i mod 4) of Philox(seed, {i div 4, 0xFFFFFFFE,
// m_lo, m_hi}); periodic wrap, or the helical wrap of x into the next row.
__constant__ int kNbX[6] = {1, -1, 0, 0, 1, -1};
__constant__ int kNbY[6] = {0, 0, 1, -1, -1, 1};

__global__ void ffn_kernel(const void *lat, int packing, int Lx, int Ly, int pitch, int geometry, int helical,
                           uint32_t k0, uint32_t k1, unsigned long long m, long long *out)
{
    const uint32_t z = geometry == kTRI6 ? 6u : 4u;
    const long long N = (long long)Lx * Ly;
    const long long G = (N + 3) / 4;
    long long n = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < G;
         q += (long long)gridDim.x * blockDim.x) {
        const Philox4 pw = philox4((uint32_t)q, 0xFFFFFFFEu, (uint32_t)m, (uint32_t)(m >> 32), k0, k1);
        const uint32_t *w = pw.v;
        const long long i0 = 4 * q;
        int y = (int)(i0 / Lx), x = (int)(i0 - (long long)y * Lx);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (i0 + r < N) {
                const int k = (int)__umulhi(w[r], z);
                int nx = x + kNbX[k], ny = y + kNbY[k];
                if (nx >= Lx) {
                    nx -= Lx;
                    if (helical) ny += 1;
                } else if (nx < 0) {
                    nx += Lx;
                    if (helical) ny -= 1;
                }
                if (ny >= Ly) ny -= Ly;
                if (ny < 0) ny += Ly;
                n += site_at(lat, packing, pitch, x, y) == site_at(lat, packing, pitch, nx, ny);
            }
            if (++x == Lx) {
                x = 0;
                ++y;
            }
        }
    }
    block_add(n, out);
}

__global__ void count_A_kernel(const void *lat, int packing, int Lx, int Ly, int pitch, long long *out)
{
    long long n = 0;
    const long long N = (long long)Lx * Ly;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
        n += site_at(lat, packing, pitch, x, y);
    }
    block_add(n, out);
}

__global__ void pack_kernel(const uint8_t *bytes, void *lat, int packing, int Lx, int Ly, int pitch)
{
    if (packing == kPackBit) {
        const int W = (Lx + 31) / 32;
        const long long nwords = (long long)W * Ly;
        const int lane = threadIdx.x & 31;
        for (long long wi = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; wi < nwords;
             wi += ((long long)gridDim.x * blockDim.x) >> 5) {
            const int y = (int)(wi / W), w = (int)(wi - (long long)y * W);
            const int x = 32 * w + lane;
            const bool a = x < Lx && bytes[(size_t)y * Lx + x] != 0;
            const uint32_t word = __ballot_sync(0xFFFFFFFFu, a);
            if (lane == 0) ((uint32_t *)lat)[(size_t)y * pitch + w] = word;
        }
    } else {
        const long long N = (long long)Lx * Ly;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
             i += (long long)gridDim.x * blockDim.x) {
            const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
            ((uint8_t *)lat)[(size_t)y * pitch + x] = bytes[i] ? 1 : 0;
        }
    }
}

__global__ void unpack_kernel(const void *lat, int packing, int Lx, int Ly, int pitch, uint8_t *bytes)
{
    const long long N = (long long)Lx * Ly;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / Lx), x = (int)(i - (long long)y * Lx);
        bytes[i] = (uint8_t)site_at(lat, packing, pitch, x, y);
    }
}

int grid_for(long long work, int per_block)
{
    long long g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

size_t init_scratch_bytes() { return sizeof(SelectState); }

cudaError_t launch_init_lattice(void *lat, int packing, int Lx, int Ly, int pitch, uint32_t key0,
                                uint32_t key1, long long nA, void *scratch, cudaStream_t stream)
{
    const long long N = (long long)Lx * Ly;
    SelectState *st = (SelectState *)scratch;
    int mode = 2;
    if (nA <= 0) mode = 0;
    else if (nA >= N) mode = 1;
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(SelectState), stream);
    if (e != cudaSuccess) return e;
    if (mode == 2) {
        // k = nA: the rank of the last A site among all keys.
        SelectState h;
        memset(&h, 0, sizeof(h));
        h.k = nA;
        // From pageable memory: the copy is staged before cudaMemcpyAsync returns.
        e = cudaMemcpyAsync(st, &h, sizeof(SelectState), cudaMemcpyHostToDevice, stream);
        if (e != cudaSuccess) return e;
        const int g = grid_for(N, kBlock * 8);
        for (int pass = 0; pass < 12; ++pass) {
            select_hist_kernel<<<g, kBlock, 0, stream>>>(N, key0, key1, st);
            select_pick_kernel<<<1, 32, 0, stream>>>(st);
        }
    }
    const int g = grid_for(N, kBlock);
    mark_kernel<<<g, kBlock, 0, stream>>>(lat, packing, Lx, Ly, pitch, key0, key1, mode, st);
    return cudaGetLastError();
}

cudaError_t launch_recount(const void *lat, int packing, int Lx, int Ly, int pitch, int geometry,
                           long long *out, cudaStream_t stream, int helical)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(long long), stream);
    if (e != cudaSuccess) return e;
    const long long N = (long long)Lx * Ly;
    recount_kernel<<<grid_for(N, kBlock * 4), kBlock, 0, stream>>>(lat, packing, Lx, Ly, pitch,
                                                                   geometry, helical, out);
    return cudaGetLastError();
}

cudaError_t launch_ffn(const void *lat, int packing, int Lx, int Ly, int pitch, int geometry, int helical,
                       uint32_t key0, uint32_t key1, long long sample, long long *out, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(long long), stream);
    if (e != cudaSuccess) return e;
    const long long G = ((long long)Lx * Ly + 3) / 4;
    ffn_kernel<<<grid_for(G, kBlock * 2), kBlock, 0, stream>>>(lat, packing, Lx, Ly, pitch, geometry, helical,
                                                              key0, key1, (unsigned long long)sample, out);
    return cudaGetLastError();
}

cudaError_t launch_count_A(const void *lat, int packing, int Lx, int Ly, int pitch, long long *out,
                           cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(long long), stream);
    if (e != cudaSuccess) return e;
    const long long N = (long long)Lx * Ly;
    count_A_kernel<<<grid_for(N, kBlock * 4), kBlock, 0, stream>>>(lat, packing, Lx, Ly, pitch, out);
    return cudaGetLastError();
}

cudaError_t launch_pack(const uint8_t *bytes, void *lat, int packing, int Lx, int Ly, int pitch,
                        cudaStream_t stream)
{
    const long long N = (long long)Lx * Ly;
    pack_kernel<<<grid_for(N, kBlock), kBlock, 0, stream>>>(bytes, lat, packing, Lx, Ly, pitch);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const void *lat, int packing, int Lx, int Ly, int pitch, uint8_t *bytes,
                          cudaStream_t stream)
{
    const long long N = (long long)Lx * Ly;
    unpack_kernel<<<grid_for(N, kBlock), kBlock, 0, stream>>>(lat, packing, Lx, Ly, pitch, bytes);
    return cudaGetLastError();
}

}  // namespace klmc
