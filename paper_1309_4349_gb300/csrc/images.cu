// images.cu -- snapshot images of the lattice and their fraction of first
// neighbours, computed on the device (section "Image analysis": each site a white
// (A) or black (B) pixel, the image sloped to keep the triangular geometry and
// scaled down with supersampling to gray levels; the fraction of first neighbours
// of a gray image compares a randomly chosen neighbour pixel within a gray-level
// threshold delta_col).
//
// Geometry: site (x, y) covers u in [2x + y, 2x + y + 2) half-sites and v in
// [y, y+1) rows; the image is U = 2 Lx + Ly - 1 half-sites wide.  Output pixel
// (i, j) of a W x H image averages an S x S grid of samples at
// u = (2(iS + a) + 1) U / (2WS), v = (2(jS + b) + 1) Ly / (2HS), evaluated in
// integers so that the image is exact: row y = floor(v), site x = floor((u - y)/2),
// inside iff 0 <= x < Lx.  A pixel belongs to the lattice iff at least half its
// samples are inside; its gray level is round(255 n_A / n_in), halves up.
//
// The image estimator: every lattice pixel p = jW + i takes one of its eight
// neighbours, direction floor(w * 8 / 2^32) of (1,0), (1,1), (0,1), (-1,1), (-1,0),
// (-1,-1), (0,-1), (1,-1), w = word (p mod 4) of Philox(seed, {p div 4, 0xFFFFFFFC,
// m_lo, m_hi}); it is similar iff that neighbour is a lattice pixel whose gray
// level differs by at most delta.
#include "klmc_internal.h"
#include "philox.cuh"

namespace klmc {
namespace {

constexpr int kImgBlock = 256;

__device__ __forceinline__ long long floor_div_ll(long long a, long long b)
{
    long long q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

__device__ __forceinline__ uint32_t lattice_site(const void *lat, int packing, int pitch, int x, int y)
{
    if (packing == kPackBit) return (((const uint32_t *)lat)[(size_t)y * pitch + (x >> 5)] >> (x & 31)) & 1u;
    return ((const uint8_t *)lat)[(size_t)y * pitch + x] ? 1u : 0u;
}

__global__ void snapshot_kernel(const void *lat, int packing, int pitch, int Lx, int Ly, int W, int H, int S,
                                uint8_t *image, uint8_t *mask)
{
    const long long P = (long long)W * H;
    const long long U = 2ll * Lx + Ly - 1, D = 2ll * W * S;
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(p / W), i = (int)(p - (long long)j * W);
        long long n_in = 0, n_A = 0;
        for (int b = 0; b < S; ++b) {
            const long long y = (2ll * ((long long)j * S + b) + 1) * Ly / (2ll * H * S);
            for (int a = 0; a < S; ++a) {
                const long long un = (2ll * ((long long)i * S + a) + 1) * U;
                const long long x = floor_div_ll(un - y * D, 2 * D);
                if (x < 0 || x >= Lx) continue;
                n_in += 1;
                n_A += lattice_site(lat, packing, pitch, (int)x, (int)y);
            }
        }
        mask[p] = (uint8_t)(2 * n_in >= (long long)S * S);
        image[p] = n_in > 0 ? (uint8_t)((510 * n_A + n_in) / (2 * n_in)) : (uint8_t)0;
    }
}


__constant__ int kMooreI[8] = {1, 1, 0, -1, -1, -1, 0, 1};
__constant__ int kMooreJ[8] = {0, 1, 1, 1, 0, -1, -1, -1};

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void image_ffn_kernel(const uint8_t *image, const uint8_t *mask, int W, int H, int delta, uint32_t k0,
                                 uint32_t k1, unsigned long long m, long long *out)
{
    __shared__ long long red[2][kImgBlock / 32];
    const long long P = (long long)W * H;
    const long long G = (P + 3) / 4;
    long long similar = 0, pixels = 0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < G;
         q += (long long)gridDim.x * blockDim.x) {
        const Philox4 pw = philox4((uint32_t)q, 0xFFFFFFFCu, (uint32_t)m, (uint32_t)(m >> 32), k0, k1);
        const uint32_t *w = pw.v;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const long long p = 4 * q + r;
            if (p >= P || !mask[p]) continue;
            pixels += 1;
            const int k = (int)__umulhi(w[r], 8u);
            const int j = (int)(p / W), i = (int)(p - (long long)j * W);
            const int a = i + kMooreI[k], b = j + kMooreJ[k];
            if (a < 0 || a >= W || b < 0 || b >= H) continue;
            const long long qq = (long long)b * W + a;
            if (!mask[qq]) continue;
            const int d = (int)image[p] - (int)image[qq];
            similar += (d <= delta && -d <= delta) ? 1 : 0;
        }
    }
    const long long s1 = warp_sum(similar), s2 = warp_sum(pixels);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = s1;
        red[1][threadIdx.x >> 5] = s2;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        long long sum = 0;
        for (int w = 0; w < kImgBlock / 32; ++w) sum += red[threadIdx.x][w];
        if (sum) atomicAdd((unsigned long long *)out + threadIdx.x, (unsigned long long)sum);
    }
}

int img_grid(long long work)
{
    long long g = (work + kImgBlock - 1) / kImgBlock;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_snapshot(const void *lat, int packing, int pitch, int Lx, int Ly, int W, int H, int S,
                            uint8_t *image, uint8_t *mask, cudaStream_t stream)
{
    snapshot_kernel<<<img_grid((long long)W * H), kImgBlock, 0, stream>>>(lat, packing, pitch, Lx, Ly, W, H, S,
                                                                          image, mask);
    return cudaGetLastError();
}

cudaError_t launch_image_ffn(const uint8_t *image, const uint8_t *mask, int W, int H, int delta, uint32_t key0,
                             uint32_t key1, long long sample, long long *out2, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(long long), stream);
    if (e != cudaSuccess) return e;
    image_ffn_kernel<<<img_grid(((long long)W * H + 3) / 4), kImgBlock, 0, stream>>>(
        image, mask, W, H, delta, key0, key1, (unsigned long long)sample, out2);
    return cudaGetLastError();
}

}  // namespace klmc
