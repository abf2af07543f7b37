// sweep_helical.cu -- Kawasaki exchange sweeps of the helical triangular lattice
// with the seven-colour schedule of the paper's MPKK loop (section "Massive
// Parallel Kawasaki Kinetics", Fig. 4), the lattice resident in the shared memory
// of a thread-block cluster for the whole launch and evaluated 32 sites per thread.
//
// Helical boundary: site i's neighbours are (i + d) mod N for the six axial steps
// d = dx + dy*Lx.  Read row by row, padded position p of row y holds site
// (y*Lx + p) mod N: position -1 is the last site of row y-1 and positions Lx,
// Lx+1 are the first two sites of row y+1.  With these pads in place the
// bit-sliced evaluation of the periodic kernels applies unchanged, and a flip of
// site 0, 1 or Lx-1 of a row also flips its copy in the pad of the row above or
// below.
//
// Iteration f of sweep s draws the coverage k and one direction d from Philox at
// {0xFFFFFFFF, f, s_lo, s_hi}; every centre c (c mod 7 = k) attempts the
// exchange with c + D[d].  Direction d is orientation o = d/2 of (1,0), (0,1),
// (1,-1), forward for even d and backward for odd d; a backward pair {c - o, c}
// is evaluated as the forward pair of its anchor a = c - o, whose residue mod 7 is
// k - step(o).  So every iteration is one orientation and one residue class of
// anchors, 4 to 5 per 32-site word in every row, and the draw of anchor a uses
// the counter of its centre, {c, f, s_lo, s_hi}.
//
// Work split as in the periodic resident kernel: CTA r of a C-CTA cluster owns
// rows [Y_r, Y_r+1) and holds D = 2K + 1 halo rows per side; it advances K
// iterations alone, evaluating in the j-th of them the anchors within
// 2 (K - 1 - j) + 1 rows of its band (a pair's evaluation and its flips reach two
// rows, and the pads only hold copies of sites in the adjacent rows), and only
// anchors of its own band are counted.  Then each CTA stores its D lowest and D
// highest band rows into its neighbours' mailboxes, a cluster barrier follows,
// the mailboxes fill the halo rows, and every row's pads are recomputed from the
// rows beside it.  Iterations run across sweep boundaries (seven per sweep).
#include <string.h>

#include "klmc_internal.h"
#include "philox.cuh"

namespace klmc {
namespace {

#include "sweep_common.cuh"

constexpr int kHelicalThreads = 512;
constexpr int kHelicalMaxSmem = 227 * 1024 - 6144;

__device__ __forceinline__ uint32_t hsmem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void hred_xor(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.xor.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t hcluster_nctarank()
{
    uint32_t v;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(v));
    return v;
}

__device__ __forceinline__ uint32_t hcluster_ctarank()
{
    uint32_t v;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(v));
    return v;
}

__device__ __forceinline__ void hcluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

template <typename T>
__device__ __forceinline__ T hwarp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Iterations per block for Lx x Ly over C CTAs: the largest K of 4, 2 whose halo
// D = 2K + 1 fits every band (twice for C = 2) and whose rows and mailboxes fit in
// shared memory; 0 when none does (the per-iteration kernel runs the lattice).
__host__ __device__ __forceinline__ int helical_block(int Lx, int Ly, int C)
{
    if (C < 2) return 0;
    const int hmin = Ly / C, hmax = (Ly + C - 1) / C;
    const long long RW = (Lx + 95) / 32;
    for (int K = 4; K >= 2; K >>= 1) {
        const int D = 2 * K + 1;
        if (D > hmin || (C == 2 && 2 * D > hmin)) continue;
        if (RW * (hmax + 6 * D) * 4 > kHelicalMaxSmem) continue;
        return K;
    }
    return 0;
}

struct HGeo {
    int Lx, Ly, W, RW, D, H, Y0, C, rank, sign, NL;
    long long N;
    unsigned long long magicW;
    uint32_t k0, k1, lat_addr;
};

// Word w of the padded row of global row y: positions [32 w - 32, 32 w); position
// p holds site (y Lx + p) mod N.  Only positions -1 .. Lx + 1 are ever read.
__device__ __forceinline__ uint32_t helical_word(const SweepJob &J, int y, int w)
{
    const int Lx = J.Lx, Ly = J.Ly, W = J.W;
    const int P0 = 32 * w - 32;
    uint32_t v = 0u;
    if (w >= 1 && w <= W) {
        v = store_word(J.lat, J.packing, J.pitch, y, w - 1, Lx);
        const int nvalid = Lx - P0;
        if (nvalid < 32) v &= (1u << nvalid) - 1u;
    }
    if (w == 0) {  // position -1: the last site of row y - 1
        const int yp = y == 0 ? Ly - 1 : y - 1;
        const int xl = Lx - 1;
        v |= ((store_word(J.lat, J.packing, J.pitch, yp, xl >> 5, Lx) >> (xl & 31)) & 1u) << 31;
    }
    const int q0 = Lx - P0;  // bit of position Lx in this word
    if (q0 >= -1 && q0 < 32) {
        const int yn = y + 1 == Ly ? 0 : y + 1;
        const uint32_t s01 = store_word(J.lat, J.packing, J.pitch, yn, 0, Lx) & 3u;  // sites 0, 1 of row y + 1
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = q0 + e;
            if (q >= 0 && q < 32) v |= ((s01 >> e) & 1u) << q;
        }
    }
    return v;
}

// Sets padded position pos of local row lr to bit b (plain store: one thread per row).
__device__ __forceinline__ void set_position(uint32_t *lat, int RW, int lr, int pos, uint32_t b)
{
    uint32_t *row = lat + (size_t)lr * RW;
    const int w = (pos + 32) >> 5, s = (pos + 32) & 31;
    row[w] = (row[w] & ~(1u << s)) | (b << s);
}

// Recomputes the pads of local rows [lo, hi) from the rows beside them.
__device__ __forceinline__ void helical_pads(uint32_t *lat, const HGeo &g, int lo, int hi)
{
    for (int lr = lo + (int)threadIdx.x; lr < hi; lr += kHelicalThreads) {
        if (lr >= 1) {
            const uint32_t *up = lat + (size_t)(lr - 1) * g.RW;
            const int xl = g.Lx - 1;
            set_position(lat, g.RW, lr, -1, (up[(xl >> 5) + 1] >> (xl & 31)) & 1u);
        }
        if (lr + 1 < g.NL) {
            const uint32_t s01 = lat[(size_t)(lr + 1) * g.RW + 1] & 3u;
            set_position(lat, g.RW, lr, g.Lx, s01 & 1u);
            set_position(lat, g.RW, lr, g.Lx + 1, s01 >> 1);
        }
    }
}

// XOR mask into padded positions q .. q+31 of the local row at shared address row.
__device__ __forceinline__ void hxor_at(uint32_t row, int RW, int q, uint32_t mask)
{
    if (mask == 0u) return;
    if (q < 0) {
        if (q <= -32) return;
        mask >>= -q;
        q = 0;
    }
    const int w = q >> 5, s = q & 31;
    if (w < RW) hred_xor(row + 4u * w, mask << s);
    if (s != 0 && w + 1 < RW) hred_xor(row + 4u * (w + 1), mask >> (32 - s));
}

// Flips, in local row lr, the sites x0 + i (bit i of m, x0 = 32 j, every site < Lx),
// and their copies in the pads of the rows above and below (when held).
__device__ __forceinline__ void helical_flip(const HGeo &g, int lr, int j, unsigned long long m)
{
    if (m == 0ull) return;
    const uint32_t rowbytes = 4u * (uint32_t)g.RW;
    const uint32_t row = g.lat_addr + rowbytes * (uint32_t)lr;
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
    if (lo) hred_xor(row + 4u * (uint32_t)(j + 1), lo);
    if (hi) hred_xor(row + 4u * (uint32_t)(j + 2), hi);
    if (j == 0 && (lo & 3u) && lr >= 1)  // sites 0, 1: positions Lx, Lx + 1 of the row above
        hxor_at(row - rowbytes, g.RW, g.Lx + 32, lo & 3u);
    const int b = g.Lx - 1 - 32 * j;  // site Lx - 1: position -1 of the row below
    if (b >= 0 && b < 64 && ((m >> b) & 1ull) && lr + 1 < g.NL) hred_xor(row + rowbytes, 0x80000000u);
}

struct HAcc {
    uint32_t att, unl, drw, acc;
    int32_t dn;
};

// Accept bits of the positions in dmask; the draw of position p uses the counter
// of site (base + p) mod N.  32-bit arithmetic: a lattice resident in one
// cluster's shared memory has far fewer than 2^30 sites, and base lies within
// [-Lx, N + Lx).
__device__ __forceinline__ uint32_t helical_draws(uint32_t dmask, const Planes &S, int base, int N,
                                                  const DrawKey &dk, const uint64_t *thr)
{
    uint32_t acc = 0u;
    uint32_t dm = dmask;
    while (dm != 0u) {
        const int p1 = __ffs(dm) - 1;
        dm &= dm - 1u;
        const int p2 = dm != 0u ? __ffs(dm) - 1 : p1;  // an odd last draw is repeated
        dm &= dm - 1u;
        int c1 = base + p1, c2 = base + p2;
        c1 += c1 >= N ? -N : (c1 < 0 ? N : 0);
        c2 += c2 >= N ? -N : (c2 < 0 ? N : 0);
        uint32_t r1, r2;
        philox2_w0_key((uint32_t)c1, (uint32_t)c2, dk, r1, r2);
        const uint32_t S1 = ((S.s0 >> p1) & 1u) | (((S.s1 >> p1) & 1u) << 1) | (((S.s2 >> p1) & 1u) << 2) |
                            (((S.s3 >> p1) & 1u) << 3);
        const uint32_t S2 = ((S.s0 >> p2) & 1u) | (((S.s1 >> p2) & 1u) << 1) | (((S.s2 >> p2) & 1u) << 2) |
                            (((S.s3 >> p2) & 1u) << 3);
        if ((uint64_t)r1 < thr[S1]) acc |= 1u << p1;
        if ((uint64_t)r2 < thr[S2]) acc |= 1u << p2;
    }
    return acc;
}

// One iteration: anchors of residue kr mod 7 in local rows [lr0, lr0 + nrows),
// orientation OI, draw counters shifted by delta (the centre of a backward pair).
template <int OI>
__device__ __forceinline__ void helical_iteration(const uint32_t *lat, const HGeo &g, int kr, int delta,
                                                  int lr0, int nrows, const DrawKey &dk, const uint64_t *thr,
                                                  HAcc &A)
{
    // b = a + o: (1,0) -> same row, +1; (0,1) -> next row; (1,-1) -> previous row, +1
    constexpr int bdy = OI == 0 ? 0 : (OI == 1 ? 1 : -1);
    constexpr int bdx = OI == 1 ? 0 : 1;
    const int ntask = nrows * g.W;
    for (int t = (int)threadIdx.x; t < ntask; t += kHelicalThreads) {
        const int mi = (int)(((unsigned long long)t * g.magicW) >> 32);
        const int j = t - mi * g.W;
        const int lr = lr0 + mi;
        int y = g.Y0 - g.D + lr;
        y = y < 0 ? y + g.Ly : (y >= g.Ly ? y - g.Ly : y);
        const int x0 = j << 5;
        const uint32_t a0 = (uint32_t)y * (uint32_t)g.Lx + (uint32_t)x0;  // site of position 0 (< N < 2^31)
        // anchors: positions p with (a0 + p) = kr mod 7, below Lx
        int o = kr - (int)(a0 % 7u);
        o += o < 0 ? 7 : 0;
        uint32_t am = 0x10204081u << o;  // bits o, o+7, o+14, o+21, o+28
        if (g.Lx - x0 < 32) am &= (1u << (g.Lx - x0)) - 1u;
        uint32_t ta, tb;
        Planes S;
        evaluate<kTRI6, OI>(lat + (size_t)lr * g.RW, g.RW, j, ta, tb, S);
        const uint32_t unl = (ta ^ tb) & am;
        const uint32_t dmask = unl & draw_positions<kTRI6>(S, g.sign);
        uint32_t acc = unl & ~dmask;
        acc |= helical_draws(dmask, S, (int)a0 + delta, (int)g.N, dk, thr);
        const bool own = (unsigned)(lr - g.D) < (unsigned)g.H;
        if (own) {
            A.att += __popc(am);
            A.unl += __popc(unl);
            A.drw += __popc(dmask);
        }
        if (acc == 0u) continue;
        if (own) {
            const int na = __popc(acc);
            A.acc += na;
            const int sum_s = __popc(S.s0 & acc) + 2 * __popc(S.s1 & acc) + 4 * __popc(S.s2 & acc) +
                              8 * __popc(S.s3 & acc);
            A.dn += 2 * (sum_s - 5 * na);
        }
        // b sites; with bdx = 1 the partner of anchor Lx-1 is position Lx, site 0 of
        // the next row of the b row.
        unsigned long long mb = (unsigned long long)acc << bdx;
        bool wrap0 = false;
        if (bdx == 1) {
            const int wb = g.Lx - x0;
            if (wb <= 32 && ((mb >> wb) & 1ull)) {
                mb &= ~(1ull << wb);
                wrap0 = true;
            }
        }
        if (bdy == 0) {
            helical_flip(g, lr, j, (unsigned long long)acc | mb);
        } else {
            helical_flip(g, lr, j, (unsigned long long)acc);
            helical_flip(g, lr + bdy, j, mb);
        }
        if (wrap0) helical_flip(g, lr + bdy + 1, 0, 1ull);
    }
}

// Iteration f of sweep s: the colour kc in [0, 7) and the direction draw d in [0, 6)
// (orientation d / 2, backward pair when d is odd), from the schedule's Philox block.
__device__ __forceinline__ uint2 helical_sched(const HGeo &g, unsigned long long s, int f)
{
    const Philox4 w = philox4(0xFFFFFFFFu, (uint32_t)f, (uint32_t)s, (uint32_t)(s >> 32), g.k0, g.k1);
    return make_uint2(__umulhi(w.v[0], 7u), __umulhi(w.v[1], 6u));
}

__global__ void __launch_bounds__(kHelicalThreads, 1)
helical_resident_kernel(const SweepJob J, const SweepCall Cl)
{
    constexpr int kWarps = kHelicalThreads / 32;
    extern __shared__ __align__(16) uint32_t lat[];
    __shared__ uint64_t thr[16];
    __shared__ long long red[5][kWarps];
    __shared__ uint2 sched[2];  // (colour, direction draw) of the current and the next iteration
    if (Cl.n_mcs <= 0) return;

    HGeo g;
    g.Lx = J.Lx; g.Ly = J.Ly; g.W = J.W; g.RW = J.RW; g.magicW = J.magicW;
    g.k0 = J.key0; g.k1 = J.key1;
    g.N = (long long)J.Lx * J.Ly;
    // The host's draw range is [z, 2(z-1)] (omega > 0), [0, z-2] (omega < 0) or empty.
    g.sign = J.draw_lo > J.draw_hi ? 0 : (J.draw_lo == 0 ? -1 : 1);
    g.C = (int)hcluster_nctarank();
    g.rank = (int)hcluster_ctarank();
    g.Y0 = (int)(((long long)g.rank * g.Ly) / g.C);
    const int Y1 = (int)(((long long)(g.rank + 1) * g.Ly) / g.C);
    g.H = Y1 - g.Y0;
    const int K = helical_block(g.Lx, g.Ly, g.C);  // >= 2: the host launches only such lattices
    g.D = 2 * K + 1;
    g.NL = g.H + 2 * g.D;
    g.lat_addr = hsmem_addr(lat);
    const int hmax = (g.Ly + g.C - 1) / g.C;
    const int tid = threadIdx.x;

    for (int idx = tid; idx < g.NL * g.RW; idx += kHelicalThreads) {
        const int lr = idx / g.RW, w = idx - lr * g.RW;
        int y = (g.Y0 - g.D + lr) % g.Ly;
        if (y < 0) y += g.Ly;
        lat[idx] = helical_word(J, y, w);
    }
    if (tid < 16) thr[tid] = J.thr[tid];
    // Iteration f of sweep s draws its colour and direction from one Philox block;
    // the last warp's lane 0 draws them one iteration ahead, off the tasks' path.
    const bool sched_lane = tid == kHelicalThreads - 32;
    if (sched_lane) sched[0] = helical_sched(g, (unsigned long long)Cl.sweep0, 0);
    const int lx7 = g.Lx % 7;
    hcluster_sync();  // every CTA of the cluster runs before any peer writes into it

    const long long n_unlike0 = (tid == 0 && g.rank == 0 && Cl.trace_every > 0) ? J.state[kNUnlike] : 0;
    unsigned long long t_att = 0, t_unl = 0, t_drw = 0, t_acc = 0;
    long long t_dn = 0;
    int jb = 0, pb = 0;  // iteration within the block; buffer of the current schedule entry
    int block = 0;
    for (long long it = 0; it < Cl.n_mcs; ++it) {
        const long long s = Cl.sweep0 + it;
        const uint32_t s_lo = (uint32_t)(unsigned long long)s;
        const uint32_t s_hi = (uint32_t)((unsigned long long)s >> 32);
        HAcc A = {0u, 0u, 0u, 0u, 0};
        for (int f = 0; f < 7; ++f) {
            const uint2 sc = sched[pb];
            const int kc = (int)sc.x;
            const int d = (int)sc.y;
            const int oi = d >> 1;
            const long long step = oi == 0 ? 1 : (oi == 1 ? g.Lx : 1 - g.Lx);
            const int delta = (d & 1) ? (int)step : 0;  // backward pair: its centre is anchor + o
            // kr = (kc - delta) mod 7, from delta mod 7 in {0, 1, Lx mod 7, 1 - Lx mod 7}
            const int dm7 = (d & 1) ? (oi == 0 ? 1 : (oi == 1 ? lx7 : (lx7 <= 1 ? 1 - lx7 : 8 - lx7))) : 0;
            int kr = kc - dm7;
            kr += kr < 0 ? 7 : 0;
            const int e = 2 * (K - 1 - jb) + 1;
            if (sched_lane && !(f == 6 && it + 1 == Cl.n_mcs))
                sched[pb ^ 1] = f == 6 ? helical_sched(g, (unsigned long long)(s + 1), 0)
                                       : helical_sched(g, (unsigned long long)s, f + 1);
            const DrawKey dk = draw_key((uint32_t)f, s_lo, s_hi, g.k0, g.k1);
            if (oi == 0) helical_iteration<0>(lat, g, kr, delta, g.D - e, g.H + 2 * e, dk, thr, A);
            else if (oi == 1) helical_iteration<1>(lat, g, kr, delta, g.D - e, g.H + 2 * e, dk, thr, A);
            else helical_iteration<2>(lat, g, kr, delta, g.D - e, g.H + 2 * e, dk, thr, A);
            __syncthreads();
            pb ^= 1;
            const bool last = f == 6 && it + 1 == Cl.n_mcs;
            const bool exch = jb == K - 1;
            jb = exch ? 0 : jb + 1;
            if (exch && !last) {
                // Exchange: the D lowest and D highest band rows to the neighbours'
                // mailboxes of parity block & 1, then this CTA's mailboxes into its
                // halo rows, then every row's pads from the rows beside it.
                const int rw = g.D * g.RW, p = block & 1;
                uint32_t *mbox = lat + (size_t)(hmax + 2 * g.D) * g.RW;
                const uint32_t prev = g.rank == 0 ? g.C - 1 : g.rank - 1;
                const uint32_t next = g.rank + 1 == g.C ? 0 : g.rank + 1;
                for (int idx = tid; idx < 2 * rw; idx += kHelicalThreads) {
                    const int side = idx >= rw ? 1 : 0;
                    const int k = idx - side * rw;
                    const uint32_t v = lat[(size_t)(side ? g.D : g.H) * g.RW + k];
                    const uint32_t local = hsmem_addr(mbox + (size_t)(2 * p + side) * rw + k);
                    uint32_t remote;
                    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                                 : "=r"(remote) : "r"(local), "r"(side ? prev : next));
                    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
                }
                hcluster_sync();
                for (int idx = tid; idx < 2 * rw; idx += kHelicalThreads) {
                    const int side = idx >= rw ? 1 : 0;
                    const int k = idx - side * rw;
                    lat[(size_t)(side ? g.D + g.H : 0) * g.RW + k] = mbox[(size_t)(2 * p + side) * rw + k];
                }
                __syncthreads();
                helical_pads(lat, g, 0, g.NL);
                __syncthreads();
                ++block;
            }
        }
        t_att += A.att; t_unl += A.unl; t_drw += A.drw; t_acc += A.acc;
        t_dn += A.dn;
        if (Cl.trace_every > 0 && (it + 1) % Cl.trace_every == 0) {
            const long long ws = hwarp_sum(t_dn);
            if ((tid & 31) == 0 && ws != 0)
                atomicAdd((unsigned long long *)&Cl.trace[(it + 1) / Cl.trace_every - 1], (unsigned long long)ws);
            if (tid == 0 && g.rank == 0)
                atomicAdd((unsigned long long *)&Cl.trace[(it + 1) / Cl.trace_every - 1],
                          (unsigned long long)n_unlike0);
        }
    }

    // Write the band back (sites only).
    for (int idx = tid; idx < g.H * g.W; idx += kHelicalThreads) {
        const int r = idx / g.W, w = idx - r * g.W;
        const int y = g.Y0 + r;
        const uint32_t v = lat[(size_t)(r + g.D) * g.RW + w + 1];
        const int pos0 = 32 * w;
        const int nvalid = min(32, g.Lx - pos0);
        if (J.packing == kPackBit) {
            const uint32_t valid = nvalid == 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
            ((uint32_t *)J.lat)[(size_t)y * J.pitch + w] = v & valid;
        } else {
            uint8_t *row = (uint8_t *)J.lat + (size_t)y * J.pitch;
            for (int b = 0; b < nvalid; ++b) row[pos0 + b] = (uint8_t)((v >> b) & 1u);
        }
    }

    long long vals[5] = {(long long)t_att, (long long)t_unl, (long long)t_drw, (long long)t_acc, t_dn};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const long long ws = hwarp_sum(vals[k]);
        if ((tid & 31) == 0) red[k][tid >> 5] = ws;
    }
    __syncthreads();
    if (tid < 5) {
        long long sum = 0;
        for (int w = 0; w < kWarps; ++w) sum += red[tid][w];
        const int slot = tid == 4 ? kNUnlike : kAttempts + tid;
        atomicAdd((unsigned long long *)&J.state[slot], (unsigned long long)sum);
    }
}

}  // namespace

int helical_resident_block(int Lx, int Ly, int cluster) { return helical_block(Lx, Ly, cluster); }

size_t helical_resident_smem_bytes(int Lx, int Ly, int cluster)
{
    const size_t RW = (size_t)(Lx + 95) / 32;
    const int C = cluster < 1 ? 1 : cluster;
    const size_t H = (size_t)((Ly + C - 1) / C);
    const int K = helical_block(Lx, Ly, C);
    return RW * (H + 6 * (size_t)(2 * (K > 0 ? K : 1) + 1)) * sizeof(uint32_t);
}

cudaError_t launch_helical_resident(const SweepJob &job, const SweepCall &call, int cluster, cudaStream_t stream)
{
    static thread_local int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device != dev) {
        e = cudaFuncSetAttribute(helical_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kHelicalMaxSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(helical_resident_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        configured_device = dev;
    }
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)cluster, 1, 1);
    cfg.blockDim = dim3(kHelicalThreads, 1, 1);
    cfg.dynamicSmemBytes = helical_resident_smem_bytes(job.Lx, job.Ly, cluster);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, helical_resident_kernel, job, call);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace klmc
