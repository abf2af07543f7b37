// sweep_tiled.cu -- Kawasaki exchange sweeps of a lattice too large for shared
// memory: one kernel launch per phase over the device store.
//
// The grid splits the lattice into row bands of H rows, one CTA each.  A CTA stages
// its band plus two halo rows on each side into shared memory (the padded row
// layout of sweep_common.cuh), evaluates the phase's anchors of its band with the
// same bit-sliced code as the resident kernel, draws, and applies accepted
// exchanges to the device store with atomic XORs.  Within a phase no site of one
// pair neighbours a site of another (the schedule is conflict-free), so no bit a
// CTA reads is changed by another CTA during the phase; a word shared by two
// pairs is updated atomically.  The launch boundary orders the phases.
//
// The sweep index is read from device state so that a captured CUDA graph of K
// sweeps (8 K phase launches and one advance node) can be replayed.
#include <string.h>

#include "klmc_internal.h"
#include "philox.cuh"

namespace klmc {
namespace {

#include "sweep_common.cuh"

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct Acc {
    uint32_t att, unl, drw, acc;
    int32_t dn;
};

// XOR the sites x0 + i (bit i of m, x0 = 32 j, every site < Lx) of row y in the store.
__device__ __forceinline__ void flip_store(const SweepJob &J, int y, int j, unsigned long long m)
{
    if (J.packing == kPackBit) {
        uint32_t *row = (uint32_t *)J.lat + (size_t)y * J.pitch;
        const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
        if (lo) atomicXor(row + j, lo);
        if (hi) atomicXor(row + j + 1, hi);
        return;
    }
    uint8_t *row = (uint8_t *)J.lat + (size_t)y * J.pitch;
    while (m) {
        const int i = __ffsll((long long)m) - 1;
        m &= m - 1ull;
        const size_t off = (size_t)(row - (uint8_t *)J.lat) + (size_t)(32 * j + i);
        uint32_t *word = (uint32_t *)((uint8_t *)J.lat + (off & ~(size_t)3));
        atomicXor(word, 1u << (8 * (off & 3)));
    }
}

template <int G, int OI>
__device__ __forceinline__ void run_tiles(const uint32_t *tile, const SweepJob &J, const PhaseP &P,
                                          int Y0, int sign, int zm1, const uint64_t *thr, int f,
                                          uint32_t s_lo, uint32_t s_hi, Acc &A)
{
    constexpr int bdy = OI == 0 ? 0 : (OI == 1 ? 1 : -1);
    constexpr int bdx = OI == 1 ? 0 : 1;
    const DrawKey dk = draw_key((uint32_t)f, s_lo, s_hi, J.key0, J.key1);
    for (int t = threadIdx.x; t < P.ntask; t += kThreads) {
        const int mi = (int)(((unsigned long long)t * J.magicW) >> 32);
        const int j = t - mi * J.W;
        const int m = mi < P.n1 ? P.a1 + mi : P.a2 + (mi - P.n1);
        int y = P.ry + P.py * m;
        if (y >= J.Ly) y -= J.Ly;
        const int x0 = j << 5;
        const uint32_t am = anchor_mask(x0, P, J.Lx);
        if (am == 0u) continue;
        uint32_t ta, tb;
        Planes S;
        evaluate<G, OI>(tile + (size_t)(y - Y0 + 2) * J.RW, J.RW, j, ta, tb, S);
        const uint32_t unl = (ta ^ tb) & am;
        const uint32_t dmask = unl & draw_positions<G>(S, sign);
        uint32_t acc = unl & ~dmask;
        acc |= draw_accepts(dmask, S, (uint32_t)(y * J.Lx + x0), dk, thr);
        A.att += __popc(am);
        A.unl += __popc(unl);
        A.drw += __popc(dmask);
        if (acc) {
            const int na = __popc(acc);
            A.acc += na;
            const int sum_s = __popc(S.s0 & acc) + 2 * __popc(S.s1 & acc) +
                              4 * __popc(S.s2 & acc) + 8 * __popc(S.s3 & acc);
            A.dn += 2 * (sum_s - zm1 * na);
            unsigned long long mb = (unsigned long long)acc << bdx;
            bool wrap0 = false;  // the pair of anchor Lx-1 wraps to site 0
            if (bdx == 1) {
                const int wb = J.Lx - x0;
                if (wb <= 32 && ((mb >> wb) & 1ull)) {
                    mb &= ~(1ull << wb);
                    wrap0 = true;
                }
            }
            int yb = y + bdy;
            if (yb < 0) yb += J.Ly;
            if (yb >= J.Ly) yb -= J.Ly;
            if (bdy == 0) {
                flip_store(J, y, j, (unsigned long long)acc | mb);
            } else {
                flip_store(J, y, j, (unsigned long long)acc);
                flip_store(J, yb, j, mb);
            }
            if (wrap0) flip_store(J, yb, 0, 1ull);
        }
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void __launch_bounds__(kThreads, 2)
tiled_phase_kernel(const SweepJob J, int H, int k, int f)
{
    extern __shared__ __align__(16) uint32_t tile[];
    __shared__ PhaseP P;
    __shared__ uint64_t thr[16];
    __shared__ long long red[5][kWarps];

    const int tid = threadIdx.x;
    const int Y0 = (int)blockIdx.x * H;
    const int Y1 = min(Y0 + H, J.Ly);
    const long long s = J.state[kSweepBase] + k;
    const int NL = Y1 - Y0 + 4;
    for (int idx = tid; idx < NL * J.RW; idx += kThreads) {
        const int lr = idx / J.RW, w = idx - lr * J.RW;
        int y = Y0 - 2 + lr;
        if (y < 0) y += J.Ly;
        if (y >= J.Ly) y -= J.Ly;
        tile[idx] = padded_word(J.lat, J.packing, J.pitch, y, w, J.Lx, J.W);
    }
    if (tid == 0) phase_params(J.geometry, J.Lx, J.Ly, J.W, Y0, Y1, J.key0, J.key1, s, f, &P);
    if (tid < 16) thr[tid] = J.thr[tid];
    __syncthreads();

    const int zm1 = (J.geometry == kTRI6 ? 6 : 4) - 1;
    const int sign = J.draw_lo > J.draw_hi ? 0 : (J.draw_lo == 0 ? -1 : 1);
    const uint32_t s_lo = (uint32_t)(unsigned long long)s;
    const uint32_t s_hi = (uint32_t)((unsigned long long)s >> 32);
    Acc A = {0u, 0u, 0u, 0u, 0};
    if (J.geometry == kTRI6) {
        if (P.oi == 0) run_tiles<kTRI6, 0>(tile, J, P, Y0, sign, zm1, thr, f, s_lo, s_hi, A);
        else if (P.oi == 1) run_tiles<kTRI6, 1>(tile, J, P, Y0, sign, zm1, thr, f, s_lo, s_hi, A);
        else run_tiles<kTRI6, 2>(tile, J, P, Y0, sign, zm1, thr, f, s_lo, s_hi, A);
    } else {
        if (P.oi == 0) run_tiles<kSQ4, 0>(tile, J, P, Y0, sign, zm1, thr, f, s_lo, s_hi, A);
        else run_tiles<kSQ4, 1>(tile, J, P, Y0, sign, zm1, thr, f, s_lo, s_hi, A);
    }

    long long vals[5] = {(long long)A.att, (long long)A.unl, (long long)A.drw, (long long)A.acc,
                         (long long)A.dn};
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const long long ws = warp_sum(vals[q]);
        if ((tid & 31) == 0) red[q][tid >> 5] = ws;
    }
    __syncthreads();
    if (tid < 5) {
        long long sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += red[tid][w];
        if (sum != 0) {
            const int slot = tid == 4 ? kNUnlike : kAttempts + tid;
            atomicAdd((unsigned long long *)&J.state[slot], (unsigned long long)sum);
        }
    }
}

// state[kSweepBase] += n
__global__ void advance_kernel(long long *state, int n) { state[kSweepBase] += n; }

// trace[state[kTracePos]++] = state[kNUnlike], trace pointer in state[kTracePtr]
__global__ void trace_kernel(long long *state)
{
    long long *trace = (long long *)state[kTracePtr];
    trace[state[kTracePos]] = state[kNUnlike];
    state[kTracePos] += 1;
}

}  // namespace

cudaError_t configure_tiled()
{
    cudaError_t e = cudaFuncSetAttribute(tiled_phase_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(227 * 1024 - 2048));
    if (e == cudaSuccess) e = configure_band();
    return e;
}

TiledPlan tiled_plan(int Lx, int Ly, int sm_count)
{
    TiledPlan p = tiled_band_plan(Lx, Ly, sm_count);
    if (p.K >= 2) return p;
    int h = (Ly + 2 * sm_count - 1) / (2 * sm_count);
    p.H = h < 4 ? 4 : h;
    p.K = 1;
    p.threads = kThreads;
    p.smem = (size_t)((Lx + 95) / 32) * (size_t)(p.H + 4) * sizeof(uint32_t);
    return p;
}

cudaError_t launch_tiled_phases(const SweepJob &job, const TiledPlan &plan, void *alt, size_t lat_bytes,
                                int k0, int n_sweeps, cudaStream_t stream)
{
    const int grid = (job.Ly + plan.H - 1) / plan.H;
    if (plan.K < 2) {
        for (int k = 0; k < n_sweeps; ++k)
            for (int f = 0; f < 8; ++f)
                tiled_phase_kernel<<<grid, kThreads, plan.smem, stream>>>(job, plan.H, k0 + k, f);
        return cudaGetLastError();
    }
    const void *src = job.lat;
    void *dst = alt;
    int launches = 0;
    for (int k = 0; k < n_sweeps; ++k) {
        for (int f0 = 0; f0 < 8; f0 += plan.K) {
            cudaError_t e = launch_band_phases(job, plan, src, dst, k0 + k, f0, stream);
            if (e != cudaSuccess) return e;
            void *t = (void *)src;
            src = dst;
            dst = t;
            ++launches;
        }
    }
    if (launches & 1) return cudaMemcpyAsync(job.lat, alt, lat_bytes, cudaMemcpyDeviceToDevice, stream);
    return cudaSuccess;
}

cudaError_t launch_advance(long long *state, int n, cudaStream_t stream)
{
    advance_kernel<<<1, 1, 0, stream>>>(state, n);
    return cudaGetLastError();
}

cudaError_t launch_trace(long long *state, cudaStream_t stream)
{
    trace_kernel<<<1, 1, 0, stream>>>(state);
    return cudaGetLastError();
}

}  // namespace klmc
