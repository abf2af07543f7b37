// sweep_mpkk.cu -- Kawasaki exchange sweeps of the helical triangular lattice with
// the seven-colour schedule of the paper's MPKK loop (section "Massive Parallel
// Kawasaki Kinetics"; Fig. 4: seven-lipid domains covering the lattice under
// helical boundary conditions).
//
// Helical boundary: site i's neighbours are (i + d) mod N for the six axial steps
// d = dx + dy*Lx, so stepping past the end of a row continues in the next row.
// The domains of coverage k are the sites c with c mod 7 = k and their six
// neighbours; they tile the lattice when 7 | N and Lx mod 7 is 3 or 5.
//
// One launch per iteration (seven per Monte Carlo step), one thread per domain
// centre, as in the paper's one-domain-per-processing-unit design.  Iteration f of
// sweep s draws the coverage k and one direction d for all domains from Philox at
// {0xFFFFFFFF, f, s_lo, s_hi}; every centre c attempts the exchange with c + D[d]
// (Metropolis steps a-c, draw counter {c, f, s_lo, s_hi}).  Centres are three
// steps apart, so no site of one pair equals or neighbours a site of another: the
// threads read the device store and flip their own two sites without conflicts.
// The sweep index is read from device state, so a CUDA graph of K sweeps can be
// replayed.
#include "klmc_internal.h"
#include "philox.cuh"

namespace klmc {
namespace {

#include "sweep_common.cuh"

constexpr int kMpkkThreads = 256;

// The six axial steps of the triangular lattice, in the order of the direction
// index d: (1,0), (-1,0), (0,1), (0,-1), (1,-1), (-1,1).
__constant__ int kStepX[6] = {1, -1, 0, 0, 1, -1};
__constant__ int kStepY[6] = {0, 0, 1, -1, -1, 1};

// (x, y) + (dx, dy) on the helical lattice (|dx| <= 1): the x wrap carries into y.
__device__ __forceinline__ void helical_step(int Lx, int Ly, int x, int y, int dx, int dy, int &nx, int &ny)
{
    nx = x + dx;
    ny = y + dy;
    if (nx >= Lx) {
        nx -= Lx;
        ny += 1;
    } else if (nx < 0) {
        nx += Lx;
        ny -= 1;
    }
    if (ny >= Ly) ny -= Ly;
    if (ny < 0) ny += Ly;
}

__device__ __forceinline__ uint32_t store_site(const SweepJob &J, int x, int y)
{
    if (J.packing == kPackBit)
        return (((const uint32_t *)J.lat)[(size_t)y * J.pitch + (x >> 5)] >> (x & 31)) & 1u;
    return ((const uint8_t *)J.lat)[(size_t)y * J.pitch + x] ? 1u : 0u;
}

// Flip one site of the store.  Bit store: an atomic XOR (other threads flip other
// bits of the word); byte store: the byte belongs to this thread's pair alone.
__device__ __forceinline__ void flip_store_site(const SweepJob &J, int x, int y)
{
    if (J.packing == kPackBit) {
        atomicXor((uint32_t *)J.lat + (size_t)y * J.pitch + (x >> 5), 1u << (x & 31));
    } else {
        uint8_t *p = (uint8_t *)J.lat + (size_t)y * J.pitch + x;
        *p = (uint8_t)(*p ^ 1u);
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void __launch_bounds__(kMpkkThreads)
mpkk_phase_kernel(const SweepJob J, int k, int f)
{
    __shared__ int kc, dir;
    __shared__ uint64_t thr[16];
    __shared__ long long red[5][kMpkkThreads / 32];
    const int tid = threadIdx.x;
    const long long s = J.state[kSweepBase] + k;
    const uint32_t s_lo = (uint32_t)(unsigned long long)s;
    const uint32_t s_hi = (uint32_t)((unsigned long long)s >> 32);
    if (tid == 0) {
        const Philox4 w = philox4(0xFFFFFFFFu, (uint32_t)f, s_lo, s_hi, J.key0, J.key1);
        kc = (int)__umulhi(w.v[0], 7u);
        dir = (int)__umulhi(w.v[1], 6u);
    }
    if (tid < 16) thr[tid] = J.thr[tid];
    __syncthreads();

    const int Lx = J.Lx, Ly = J.Ly;
    const int ddx = kStepX[dir], ddy = kStepY[dir];
    // The host's draw range is [z, 2(z-1)] (omega > 0), [0, z-2] (omega < 0) or empty.
    const int sign = J.draw_lo > J.draw_hi ? 0 : (J.draw_lo == 0 ? -1 : 1);
    const DrawKey dk = draw_key((uint32_t)f, s_lo, s_hi, J.key0, J.key1);
    const long long n_centres = (long long)Lx * Ly / 7;
    long long att = 0, unl = 0, drw = 0, acc = 0, dn_sum = 0;
    for (long long q = blockIdx.x * (long long)kMpkkThreads + tid; q < n_centres;
         q += (long long)gridDim.x * kMpkkThreads) {
        const long long c = kc + 7 * q;
        const int cy = (int)(c / Lx), cx = (int)(c - (long long)cy * Lx);
        int bx, by;
        helical_step(Lx, Ly, cx, cy, ddx, ddy, bx, by);
        const uint32_t ta = store_site(J, cx, cy), tb = store_site(J, bx, by);
        att += 1;
        if (ta == tb) continue;
        unl += 1;
        // S: neighbours of c other than b equal to c, plus neighbours of b other
        // than c equal to b; the exchange changes n_unlike by 2 (S - 5).
        int S = 0;
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            int nx, ny;
            helical_step(Lx, Ly, cx, cy, kStepX[e], kStepY[e], nx, ny);
            if (nx != bx || ny != by) S += store_site(J, nx, ny) == ta;
            helical_step(Lx, Ly, bx, by, kStepX[e], kStepY[e], nx, ny);
            if (nx != cx || ny != cy) S += store_site(J, nx, ny) == tb;
        }
        const bool need = sign > 0 ? S > 5 : (sign < 0 ? S < 5 : false);
        bool accept = true;
        if (need) {
            drw += 1;
            uint32_t r, r2;
            philox2_w0_key((uint32_t)c, (uint32_t)c, dk, r, r2);
            accept = (uint64_t)r < thr[S];
        }
        if (accept) {
            acc += 1;
            dn_sum += 2 * (S - 5);
            flip_store_site(J, cx, cy);
            flip_store_site(J, bx, by);
        }
    }
    long long vals[5] = {att, unl, drw, acc, dn_sum};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const long long ws = warp_sum(vals[q]);
        if ((tid & 31) == 0) red[q][tid >> 5] = ws;
    }
    __syncthreads();
    if (tid < 5) {
        long long sum = 0;
        for (int w = 0; w < kMpkkThreads / 32; ++w) sum += red[tid][w];
        if (sum != 0) {
            const int slot = tid == 4 ? kNUnlike : kAttempts + tid;
            atomicAdd((unsigned long long *)&J.state[slot], (unsigned long long)sum);
        }
    }
}

}  // namespace

bool helical_tiles(int Lx, int Ly)
{
    const long long N = (long long)Lx * Ly;
    return Lx >= 4 && Ly >= 4 && N % 7 == 0 && (Lx % 7 == 3 || Lx % 7 == 5);
}

cudaError_t launch_mpkk_phases(const SweepJob &job, int k0, int n_sweeps, int sm_count, cudaStream_t stream)
{
    const long long n_centres = (long long)job.Lx * job.Ly / 7;
    long long grid = (n_centres + kMpkkThreads - 1) / kMpkkThreads;
    const long long cap = (long long)sm_count * 8;
    if (grid > cap) grid = cap;
    if (grid < 1) grid = 1;
    for (int k = 0; k < n_sweeps; ++k)
        for (int f = 0; f < 7; ++f)
            mpkk_phase_kernel<<<(unsigned)grid, kMpkkThreads, 0, stream>>>(job, k0 + k, f);
    return cudaGetLastError();
}

}  // namespace klmc
