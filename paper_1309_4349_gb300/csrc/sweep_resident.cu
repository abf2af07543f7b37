// sweep_resident.cu -- Kawasaki exchange sweeps with the lattice resident in shared
// memory for the whole launch (section "Massive Parallel Kawasaki Kinetics": every
// iteration performs one exchange per domain of a random decomposition, all in
// parallel; here the decomposition is a conflict-free shifted sublattice phase).
//
// Work split.  One lattice per thread-block cluster of C CTAs (C = 1 is a plain
// CTA).  CTA c of the cluster owns the row band [Y_c, Y_c+1), Y_c = floor(c Ly / C),
// and keeps band rows plus two halo rows on each side in shared memory: local row
// lr holds global row (Y_c - 2 + lr) mod Ly.  A phase's anchor rows are split by
// band; every read of an anchor's neighbourhood (rows y-2 .. y+2) is local.  An
// accepted exchange flips its two sites in every copy of their rows: the local
// copy and, for rows within two of a band edge, the copies held by the
// neighbouring CTAs, through distributed shared memory.  Phases are separated by
// a cluster barrier (release/acquire), so the next phase sees every flip.
//
// Phase blocks.  When the bands are tall enough, a cluster of C > 1 CTAs instead
// advances K consecutive phases (K = 2, 4 or 8) between exchanges.  Each CTA
// keeps D = 2K + 1 halo rows on each side, and in the j-th phase of a block
// evaluates every anchor within 2 (K - 1 - j) + 1 rows of its band: a site's new
// value depends only on sites at most two rows away, so after K phases the band
// is exact although the outer halo rows are not.  The anchors outside the band
// are evaluated again by the CTA that owns them, with the same counter-based
// random numbers, hence identical results; only anchors of the own band are
// counted.  All flips are local.  At the end of a block each CTA stores its D
// lowest and D highest band rows into mailboxes in the neighbouring CTAs'
// shared memory (double-buffered by block parity), one cluster barrier follows,
// and each CTA copies its mailboxes into its halo rows.
//
// Row layout.  A shared-memory row is RW 32-bit words holding the padded bit
// positions pos in [-32, 32*RW - 32); when loaded, position pos holds site
// (pos mod Lx), so the 32-site window starting at any x in [-32, Lx + 32] is one
// funnel shift of two words.  The windows of anchors x < Lx read only positions
// -1 .. Lx+1, so flips keep exactly the copies at -1 (site Lx-1) and Lx, Lx+1
// (sites 0, 1) equal to their sites; other pad positions are never read.
//
// Evaluation.  One thread handles the anchors of one 32-site word of one anchor
// row.  Neighbour comparisons of all 32 positions are bitwise operations summed by
// a carry-save adder tree into bit planes of S = same_a + same_b (neighbours of a,
// other than b, equal to a, plus neighbours of b, other than a, equal to b).  An
// exchange changes the number of unlike contacts by dn = 2 (S - (z - 1)).  Unlike
// pairs whose S lies in the draw range draw a Philox number; the rest are accepted
// outright (Metropolis acceptance min{1, exp(-omega dn / kT)}, steps a-c).  A
// lane draws for its own anchors, two Philox evaluations interleaved at a time:
// a phase is short, so its cost is the latency of its slowest task.
#include <string.h>

#include "klmc_internal.h"
#include "philox.cuh"

namespace klmc {
namespace {

#include "sweep_common.cuh"

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// XOR v into the 32-bit word at shared address addr of CTA `rank` of the cluster.
__device__ __forceinline__ void xor_word(uint32_t addr, uint32_t rank, bool local, uint32_t v)
{
    if (v == 0u) return;
    if (local) {
        asm volatile("red.shared.xor.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
    } else {
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(addr), "r"(rank));
        asm volatile("red.shared::cluster.xor.b32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
    }
}

// XOR v into the 32-bit word at shared address addr of this CTA, unconditionally.
__device__ __forceinline__ void red_xor_local(uint32_t addr, uint32_t v)
{
    asm volatile("red.shared.xor.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// XOR mask into padded bit positions q .. q+31 of the row at shared address row (clipped).
__device__ __forceinline__ void xor_at(uint32_t row, int RW, int q, uint32_t mask, uint32_t rank,
                                       bool local)
{
    if (q < 0) {
        if (q <= -32) return;
        mask >>= -q;
        q = 0;
    }
    const int w = q >> 5, s = q & 31;
    if (w < RW) xor_word(row + 4u * w, rank, local, mask << s);
    if (s != 0 && w + 1 < RW) xor_word(row + 4u * (w + 1), rank, local, mask >> (32 - s));
}

struct Acc {
    uint32_t att, unl, drw, acc;
    int32_t dn;
};

struct Geo {
    int Lx, Ly, W, RW;
    unsigned long long magicW;
    uint32_t k0, k1;
    int sign;            // draw when the exchange raises (+1) / lowers (-1) E; 0: never
    int zm1;
    int C, rank, Y0, Y1;
    int prevY, prevH;    // band of CTA rank-1 (mod C)
    int nextY, nextH;    // band of CTA rank+1 (mod C)
    uint32_t lat_addr;   // shared address of local row 0
    int D;               // halo rows on each side: local row lr holds row (Y0 - D + lr) mod Ly
    int base;            // (Y0 - D) mod Ly
};

// Flip, in one copy of a row, the sites x0 + i (bit i of m, x0 = 32 j, every site
// < Lx), and the pad copies that windows read: position -1 (site Lx-1) and
// positions Lx, Lx+1 (sites 0, 1).
__device__ __forceinline__ void flip_row(const Geo &g, uint32_t row, int j, unsigned long long m,
                                         uint32_t rank, bool local)
{
    const uint32_t lo = (uint32_t)m, hi = (uint32_t)(m >> 32);
    xor_word(row + 4u * (uint32_t)(j + 1), rank, local, lo);
    xor_word(row + 4u * (uint32_t)(j + 2), rank, local, hi);
    if (j == 0 && (lo & 3u)) xor_at(row, g.RW, g.Lx + 32, lo & 3u, rank, local);
    const int b = g.Lx - 1 - 32 * j;
    if (b >= 0 && b < 64 && ((m >> b) & 1ull)) xor_word(row, rank, local, 0x80000000u);
}

// Flip sites of global row r (unwrapped, in [Y0 - 1, Y1]) in every CTA holding a copy.
__device__ __forceinline__ void flip_global_row(const Geo &g, int r, int j, unsigned long long m)
{
    const int lr_self = r - g.Y0 + 2;
    const uint32_t rowbytes = 4u * (uint32_t)g.RW;
    if (g.C > 1 && lr_self >= 4 && lr_self < g.Y1 - g.Y0) {  // interior row: local copy only
        flip_row(g, g.lat_addr + rowbytes * (uint32_t)lr_self, j, m, 0u, true);
        return;
    }
    const int gr = r < 0 ? r + g.Ly : (r >= g.Ly ? r - g.Ly : r);
    if (g.C == 1) {  // rows 0, 1 and Ly-2, Ly-1 also live in the opposite halo
        for (int lr = gr + 2 >= g.Ly ? gr + 2 - g.Ly : gr + 2; lr < g.Ly + 4; lr += g.Ly)
            flip_row(g, g.lat_addr + rowbytes * (uint32_t)lr, j, m, 0u, true);
        return;
    }
    for (int k = 0; k < 3; ++k) {
        if (k == 2 && g.C == 2) break;  // both neighbours are the same CTA
        const int d = k == 0 ? (g.rank == 0 ? g.C - 1 : g.rank - 1)
                             : (k == 1 ? g.rank : (g.rank + 1 == g.C ? 0 : g.rank + 1));
        const int Yd = k == 0 ? g.prevY : (k == 1 ? g.Y0 : g.nextY);
        const int Hd = k == 0 ? g.prevH : (k == 1 ? g.Y1 - g.Y0 : g.nextH);
        int lr = gr - Yd + 2;
        if (lr < 0) lr += g.Ly;
        if (lr >= g.Ly) lr -= g.Ly;
        for (; lr < Hd + 4; lr += g.Ly)
            flip_row(g, g.lat_addr + rowbytes * (uint32_t)lr, j, m, (uint32_t)d, d == g.rank);
    }
}

__device__ __forceinline__ void phase_barrier(int C)
{
    if (C == 1) {
        __syncthreads();
    } else {
        asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    }
}

// Per-phase task table: the anchor mask of every word and, per task row mi, the
// local row and the row's first site index, so that a task loads two entries
// instead of recomputing them.  The resident kernel keeps two (current and next
// phase) for bands of at most kTabW words per row and kTabRows anchor rows, built by
// the CTA's last warp while the other warps run the current phase; the band kernel
// builds one per phase of its block at launch.
constexpr int kTabW = 64;
constexpr int kTabRows = 128;

struct TaskTab {  // a table's storage and capacity
    uint32_t *am;
    int2 *row;   // (local row, y * Lx)
    int maxw, maxrows;
};

__device__ __forceinline__ bool table_fits(const Geo &g, const PhaseR &P, const TaskTab &T)
{
    return g.W <= T.maxw && P.c[3] <= T.maxrows;
}

// Fills the table entries with index = lane0 mod step (all of them for lane0 = 0,
// step = 1 per thread ... ), so that a warp (step 32) or a CTA (step THREADS)
// builds it together: the anchor masks (AM), the rows (ROWS) or both.
template <bool BLOCKED, bool AM = true, bool ROWS = true>
__device__ __forceinline__ void build_task_table(const PhaseR &P, const Geo &g, const TaskTab &T, int lane0,
                                                 int step)
{
    if (!table_fits(g, P, T)) return;
    if (AM)
        for (int j = lane0; j < g.W; j += step) T.am[j] = anchor_mask(j << 5, P, g.Lx);
    if (ROWS)
    for (int mi = lane0; mi < P.c[3]; mi += step) {
        const int m = mi < P.c[0] ? P.a[0] + mi
                    : (mi < P.c[1] ? P.a[1] + mi : (mi < P.c[2] ? P.a[2] + mi : P.a[3] + mi));
        int y = P.ry + P.py * m;
        if (y >= g.Ly) y -= g.Ly;
        int lr;
        if (BLOCKED) {
            lr = y - g.base;
            if (lr < 0) lr += g.Ly;
        } else {
            lr = y - g.Y0 + 2;
        }
        T.row[mi] = make_int2(lr, y * g.Lx);
    }
}

// One phase of one band.  Every task is (anchor row, word j).  BLOCKED: the
// anchors span the band and part of its halo, all flips are local, and only
// anchors of the band are counted; otherwise the anchors are those of the band
// and flips reach every copy of their rows.
template <int G, int OI, int THREADS, bool BLOCKED>
__device__ __forceinline__ void run_phase(const uint32_t *lat, const Geo &g, const PhaseR &P,
                                          const uint64_t *thr, int f,
                                          uint32_t s_lo, uint32_t s_hi, Acc &A, const TaskTab *tt = nullptr)
{
    // b = a + o: (1,0) -> same row, +1; (0,1) -> next row; (1,-1) -> previous row, +1
    constexpr int bdy = OI == 0 ? 0 : (OI == 1 ? 1 : -1);
    constexpr int bdx = OI == 1 ? 0 : 1;
    const int lane = threadIdx.x & 31;
    const int H = g.Y1 - g.Y0;
    // Split each word over 2^ls lanes when the phase has that few words: every lane
    // evaluates the word and keeps the anchors of its part, which divides the draws
    // (the longest step of a lane) among the lanes.
    // (At 512 threads the extra evaluations cost more issue slots than they save.)
    const int ls = THREADS > 256 ? 0 : (4 * P.ntask <= THREADS ? 2 : (2 * P.ntask <= THREADS ? 1 : 0));
    const int nlane = P.ntask << ls;
    const bool use_tab = tt != nullptr && table_fits(g, P, *tt);
    const DrawKey dk = draw_key((uint32_t)f, s_lo, s_hi, g.k0, g.k1);
    for (int t0 = threadIdx.x & ~31; t0 < nlane; t0 += THREADS) {
        const int tl = t0 + lane;
        uint32_t am = 0u, ta = 0u, tb = 0u;
        Planes S = {0u, 0u, 0u, 0u};
        int ybase = 0, x0 = 0, lr = 0;
        if (tl < nlane) {
            const int t = tl >> ls;
            const int mi = (int)(((unsigned long long)t * g.magicW) >> 32);
            const int j = t - mi * g.W;
            x0 = j << 5;
            if (use_tab) {
                const int2 r = tt->row[mi];
                lr = r.x;
                ybase = r.y;
                am = tt->am[j];
            } else {
                const int m = mi < P.c[0] ? P.a[0] + mi
                            : (mi < P.c[1] ? P.a[1] + mi : (mi < P.c[2] ? P.a[2] + mi : P.a[3] + mi));
                int y = P.ry + P.py * m;
                if (y >= g.Ly) y -= g.Ly;
                if (BLOCKED) {
                    lr = y - g.base;
                    if (lr < 0) lr += g.Ly;
                } else {
                    lr = y - g.Y0 + 2;  // y is a band row
                }
                ybase = y * g.Lx;
                am = anchor_mask(x0, P, g.Lx);
            }
            if (ls != 0) {
                const int part = tl & ((1 << ls) - 1), bits = 32 >> ls;
                am &= (0xFFFFFFFFu >> (32 - bits)) << (part * bits);
            }
            evaluate<G, OI>(lat + (size_t)lr * g.RW, g.RW, j, ta, tb, S);
        }
        const uint32_t unl = (ta ^ tb) & am;
        const uint32_t dmask = unl & draw_positions<G>(S, g.sign);
        uint32_t acc = unl & ~dmask;

        acc |= draw_accepts(dmask, S, (uint32_t)(ybase + x0), dk, thr);
        const bool own = !BLOCKED || (unsigned)(lr - g.D) < (unsigned)H;
        if (own) {
            A.att += __popc(am);
            A.unl += __popc(unl);
            A.drw += __popc(dmask);
        }
        if (acc) {
            if (own) {
                const int na = __popc(acc);
                A.acc += na;
                const int sum_s = __popc(S.s0 & acc) + 2 * __popc(S.s1 & acc) +
                                  4 * __popc(S.s2 & acc) + 8 * __popc(S.s3 & acc);
                A.dn += 2 * (sum_s - g.zm1 * na);
            }
            const int j = x0 >> 5;
            // b sites; with bdx = 1 the pair of anchor Lx-1 wraps to site 0.
            unsigned long long mb = (unsigned long long)acc << bdx;
            bool wrap0 = false;
            if (bdx == 1) {
                const int wb = g.Lx - x0;
                if (wb <= 32 && ((mb >> wb) & 1ull)) {
                    mb &= ~(1ull << wb);
                    wrap0 = true;
                }
            }
            if (BLOCKED) {
                const uint32_t rowbytes = 4u * (uint32_t)g.RW;
                const uint32_t ra = g.lat_addr + rowbytes * (uint32_t)lr;
                const uint32_t rb = g.lat_addr + rowbytes * (uint32_t)(lr + bdy);
                if (bdy == 0) {
                    flip_row(g, ra, j, (unsigned long long)acc | mb, 0u, true);
                } else {
                    flip_row(g, ra, j, (unsigned long long)acc, 0u, true);
                    flip_row(g, rb, j, mb, 0u, true);
                }
                if (wrap0) flip_row(g, rb, 0, 1ull, 0u, true);
            } else {
                const int yu = lr - g.D + g.Y0;  // unwrapped band row
                if (bdy == 0) {
                    flip_global_row(g, yu, j, (unsigned long long)acc | mb);
                } else {
                    flip_global_row(g, yu, j, (unsigned long long)acc);
                    flip_global_row(g, yu + bdy, j, mb);
                }
                if (wrap0) flip_global_row(g, yu + bdy, 0, 1ull);
            }
        }
    }
}

// Band kernel: one phase with two tasks per lane (t and t + THREADS) sharing one
// pass of the warp's draw queue.  Blocked (all flips local, only the band's anchors
// counted), with the phase's task table when it fits.
struct TaskPrep {
    uint32_t dmask, acc;  // positions that need a draw; accepted without one
    Planes S;
    uint32_t base;        // site index of position 0
    int lr, j;
    bool own;
};

template <int G, int OI>
__device__ __forceinline__ void band_task_prep(const uint32_t *lat, const Geo &g, const PhaseR &P, bool use_tab,
                                               const TaskTab *tt, int t, bool valid, TaskPrep &T, Acc &A)
{
    uint32_t am = 0u, ta = 0u, tb = 0u;
    Planes S = {0u, 0u, 0u, 0u};
    int ybase = 0, j = 0, lr = 0;
    if (valid) {
        const int mi = (int)(((unsigned long long)t * g.magicW) >> 32);
        j = t - mi * g.W;
        if (use_tab) {
            const int2 r = tt->row[mi];
            lr = r.x;
            ybase = r.y;
            am = tt->am[j];
        } else {
            const int m = mi < P.c[0] ? P.a[0] + mi
                        : (mi < P.c[1] ? P.a[1] + mi : (mi < P.c[2] ? P.a[2] + mi : P.a[3] + mi));
            int y = P.ry + P.py * m;
            if (y >= g.Ly) y -= g.Ly;
            lr = y - g.base;
            if (lr < 0) lr += g.Ly;
            ybase = y * g.Lx;
            am = anchor_mask(j << 5, P, g.Lx);
        }
        evaluate<G, OI>(lat + (size_t)lr * g.RW, g.RW, j, ta, tb, S);
    }
    const uint32_t unl = (ta ^ tb) & am;
    T.dmask = unl & draw_positions<G>(S, g.sign);
    T.acc = unl & ~T.dmask;
    T.S = S;
    T.base = (uint32_t)(ybase + (j << 5));
    T.lr = lr;
    T.j = j;
    T.own = (unsigned)(lr - g.D) < (unsigned)(g.Y1 - g.Y0);
    if (T.own) {
        A.att += __popc(am);
        A.unl += __popc(unl);
        A.drw += __popc(T.dmask);
    }
}

template <int OI>
__device__ __forceinline__ void band_task_finish(const Geo &g, const TaskPrep &T, uint32_t acc, Acc &A)
{
    constexpr int bdy = OI == 0 ? 0 : (OI == 1 ? 1 : -1);
    constexpr int bdx = OI == 1 ? 0 : 1;
    if (!acc) return;
    if (T.own) {
        const int na = __popc(acc);
        A.acc += na;
        const int sum_s = __popc(T.S.s0 & acc) + 2 * __popc(T.S.s1 & acc) + 4 * __popc(T.S.s2 & acc) +
                          8 * __popc(T.S.s3 & acc);
        A.dn += 2 * (sum_s - g.zm1 * na);
    }
    const int j = T.j, lr = T.lr, x0 = j << 5;
    unsigned long long mb = (unsigned long long)acc << bdx;
    bool wrap0 = false;
    if (bdx == 1) {
        const int wb = g.Lx - x0;
        if (wb <= 32 && ((mb >> wb) & 1ull)) {
            mb &= ~(1ull << wb);
            wrap0 = true;
        }
    }
    const uint32_t rowbytes = 4u * (uint32_t)g.RW;
    if (j != 0 && 32 * j + 65 <= g.Lx) {
        // a word clear of both row ends: no pad copies, no wrap, exact words
        const uint32_t wa = g.lat_addr + rowbytes * (uint32_t)lr + 4u * (uint32_t)(j + 1);
        const uint32_t wbw = wa + rowbytes * (uint32_t)bdy;
        const uint32_t lo = (uint32_t)mb, hi = (uint32_t)(mb >> 32);
        // every word is XORed, zero or not: an atomic of 0 costs less than a branch
        if (bdy == 0) {
            red_xor_local(wa, acc | lo);
        } else {
            red_xor_local(wa, acc);
            red_xor_local(wbw, lo);
        }
        red_xor_local(wbw + 4u, hi);
        return;
    }
    const uint32_t ra = g.lat_addr + rowbytes * (uint32_t)lr;
    const uint32_t rb = g.lat_addr + rowbytes * (uint32_t)(lr + bdy);
    if (bdy == 0) {
        flip_row(g, ra, j, (unsigned long long)acc | mb, 0u, true);
    } else {
        flip_row(g, ra, j, (unsigned long long)acc, 0u, true);
        flip_row(g, rb, j, mb, 0u, true);
    }
    if (wrap0) flip_row(g, rb, 0, 1ull, 0u, true);
}

template <int G, int OI, int THREADS, bool RK>
__device__ __forceinline__ void run_phase_pair(const uint32_t *lat, const Geo &g, const PhaseR &P,
                                               const uint64_t *thr, int f, uint32_t s_lo, uint32_t s_hi,
                                               Acc &A, uint32_t *q, const TaskTab *tt, const uint32_t (&rk)[2][8])
{
    const int lane = threadIdx.x & 31;
    const int ntask = P.ntask;
    const bool use_tab = tt != nullptr && table_fits(g, P, *tt);
    const DrawKey dk = draw_key((uint32_t)f, s_lo, s_hi, g.k0, g.k1);
    for (int t0 = threadIdx.x & ~31; t0 < ntask; t0 += 2 * THREADS) {
        const int ta = t0 + lane, tb = t0 + THREADS + lane;
        TaskPrep T0, T1;
        band_task_prep<G, OI>(lat, g, P, use_tab, tt, ta, ta < ntask, T0, A);
        band_task_prep<G, OI>(lat, g, P, use_tab, tt, tb, tb < ntask, T1, A);
        uint32_t a0, a1;
        draw_accepts_queue2<RK>(T0.dmask, T0.S, T0.base, T1.dmask, T1.S, T1.base, dk, rk, thr, q, a0, a1);
        band_task_finish<OI>(g, T0, T0.acc | a0, A);
        band_task_finish<OI>(g, T1, T1.acc | a1, A);
    }
}

template <int G, int THREADS, bool RK>
__device__ __forceinline__ void run_phase_pair_oi(const uint32_t *lat, const Geo &g, const PhaseR &P,
                                                  const uint64_t *thr, int f, uint32_t s_lo, uint32_t s_hi,
                                                  Acc &A, uint32_t *q, const TaskTab *tt, const uint32_t (&rk)[2][8])
{
    if (P.oi == 0) run_phase_pair<G, 0, THREADS, RK>(lat, g, P, thr, f, s_lo, s_hi, A, q, tt, rk);
    else if (G == kTRI6 && P.oi == 2) run_phase_pair<G, 2, THREADS, RK>(lat, g, P, thr, f, s_lo, s_hi, A, q, tt, rk);
    else run_phase_pair<G, 1, THREADS, RK>(lat, g, P, thr, f, s_lo, s_hi, A, q, tt, rk);
}

template <int G, int THREADS, bool BLOCKED>
__device__ __forceinline__ void run_phase_oi(const uint32_t *lat, const Geo &g, const PhaseR &P,
                                             const uint64_t *thr, int f, uint32_t s_lo,
                                             uint32_t s_hi, Acc &A, const TaskTab *tt = nullptr)
{
    if (P.oi == 0) run_phase<G, 0, THREADS, BLOCKED>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
    else if (G == kTRI6 && P.oi == 2) run_phase<G, 2, THREADS, BLOCKED>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
    else run_phase<G, 1, THREADS, BLOCKED>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__device__ __forceinline__ uint32_t cluster_nctarank()
{
    uint32_t v;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(v));
    return v;
}

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t v;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(v));
    return v;
}

// Dynamic shared memory a CTA may use (the kernels' static arrays take under 6 KB).
constexpr int kResidentMaxSmem = 227 * 1024 - 6144;

#ifndef KLMC_MAX_BLOCK
#define KLMC_MAX_BLOCK 4
#endif

// Phases per block for a lattice of Lx x Ly sites split over C CTAs: the largest K
// of 8, 4, 2 (at most KLMC_MAX_BLOCK) whose halo D = 2K + 1 fits in every band
// (twice, for C = 2, so that a CTA's rows never overlap themselves) and whose
// rows and mailboxes fit in shared memory; 1 (a cluster barrier per phase)
// otherwise.
__host__ __device__ __forceinline__ int block_phases(int Lx, int Ly, int C)
{
    if (C <= 1) return 1;
    const int hmin = Ly / C, hmax = (Ly + C - 1) / C;
    const long long RW = (Lx + 95) / 32;
    for (int K = KLMC_MAX_BLOCK; K >= 2; K >>= 1) {
        const int D = 2 * K + 1;
        if (D > hmin || (C == 2 && 2 * D > hmin)) continue;
        if (RW * (hmax + 6 * D) * 4 > kResidentMaxSmem) continue;
        return K;
    }
    return 1;
}

// Phase table of (sweep s, phase f): the band's anchors, widened for a block.
__device__ __forceinline__ void phase_table(const SweepJob &J, const Geo &g, int K, long long s, int f,
                                            PhaseR *P)
{
    const int e = K > 1 ? 2 * (K - 1 - f % K) + 1 : 0;
    phase_ranges(J.geometry, g.Lx, g.Ly, g.W, g.Y0 - e, g.Y1 + e, g.k0, g.k1, s, f, P);
}

// End of a block: the D lowest and D highest band rows go to the mailboxes of
// parity p in the neighbouring CTAs, a cluster barrier, then this CTA's own
// mailboxes of parity p fill its halo rows.
template <int THREADS>
__device__ __forceinline__ void exchange_halos(uint32_t *lat, const Geo &g, int hmax, int p)
{
    const int H = g.Y1 - g.Y0, D = g.D, rw = D * g.RW;
    uint32_t *mbox = lat + (size_t)(hmax + 2 * D) * g.RW;
    const uint32_t prev = g.rank == 0 ? g.C - 1 : g.rank - 1;
    const uint32_t next = g.rank + 1 == g.C ? 0 : g.rank + 1;
    for (int idx = threadIdx.x; idx < 2 * rw; idx += THREADS) {
        const int side = idx >= rw ? 1 : 0;
        const int k = idx - side * rw;
        const uint32_t v = lat[(size_t)(side ? D : H) * g.RW + k];
        const uint32_t local = smem_addr(mbox + (size_t)(2 * p + side) * rw + k);
        uint32_t remote;
        asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                     : "=r"(remote) : "r"(local), "r"(side ? prev : next));
        asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(remote), "r"(v) : "memory");
    }
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    for (int idx = threadIdx.x; idx < 2 * rw; idx += THREADS) {
        const int side = idx >= rw ? 1 : 0;
        const int k = idx - side * rw;
        lat[(size_t)(side ? D + H : 0) * g.RW + k] = mbox[(size_t)(2 * p + side) * rw + k];
    }
    __syncthreads();
}

template <int THREADS, int MINB>
__global__ void __launch_bounds__(THREADS, MINB)
resident_sweep_kernel(const SweepJob *__restrict__ jobs, const SweepCall *__restrict__ calls,
                      const int *__restrict__ job_map, const SweepJob job0, const SweepCall call0)
{
    constexpr int kWarps = THREADS / 32;
    extern __shared__ __align__(16) uint32_t lat[];
    __shared__ PhaseR pp[2][8];
    __shared__ uint64_t thr[16];
    __shared__ long long red[5][kWarps];
    __shared__ uint32_t tab_am[2][kTabW];   // tables of the current and the next phase
    __shared__ int2 tab_row[2][kTabRows];

    const int C = (int)cluster_nctarank();
    const int rank = (int)cluster_ctarank();
    const int job = job_map ? job_map[blockIdx.x / C] : (int)blockIdx.x / C;
    const SweepJob &J = jobs ? jobs[job] : job0;
    const SweepCall Cl = calls ? calls[job] : call0;
    if (Cl.n_mcs <= 0) return;  // uniform over the cluster

    Geo g;
    g.Lx = J.Lx; g.Ly = J.Ly; g.W = J.W; g.RW = J.RW; g.magicW = J.magicW;
    g.k0 = J.key0; g.k1 = J.key1;
    g.zm1 = (J.geometry == kTRI6 ? 6 : 4) - 1;
    // The host's draw range is [z, 2(z-1)] (omega > 0), [0, z-2] (omega < 0) or empty.
    g.sign = J.draw_lo > J.draw_hi ? 0 : (J.draw_lo == 0 ? -1 : 1);
    g.C = C;
    g.rank = rank;
    g.Y0 = (int)(((long long)rank * g.Ly) / C);
    g.Y1 = (int)(((long long)(rank + 1) * g.Ly) / C);
    {
        const int pr = rank == 0 ? C - 1 : rank - 1, nr = rank + 1 == C ? 0 : rank + 1;
        g.prevY = (int)(((long long)pr * g.Ly) / C);
        g.prevH = (int)(((long long)(pr + 1) * g.Ly) / C) - g.prevY;
        g.nextY = (int)(((long long)nr * g.Ly) / C);
        g.nextH = (int)(((long long)(nr + 1) * g.Ly) / C) - g.nextY;
    }
    g.lat_addr = smem_addr(lat);
    const int K = block_phases(g.Lx, g.Ly, C);
    const bool blocked = K > 1;
    g.D = blocked ? 2 * K + 1 : 2;
    g.base = g.Y0 - g.D < 0 ? g.Y0 - g.D + g.Ly : g.Y0 - g.D;
    const int hmax = (g.Ly + C - 1) / C;
    const int tid = threadIdx.x;
    const int H = g.Y1 - g.Y0;
    const int NL = H + 2 * g.D;

    // Load band and halo rows into padded shared-memory rows.
    for (int idx = tid; idx < NL * g.RW; idx += THREADS) {
        const int lr = idx / g.RW, w = idx - lr * g.RW;
        int y = g.Y0 - g.D + lr;
        y %= g.Ly;
        if (y < 0) y += g.Ly;
        lat[idx] = padded_word(J.lat, J.packing, J.pitch, y, w, g.Lx, g.W);
    }
    if (tid < 16) thr[tid] = J.thr[tid];
    // The last three warps prepare the next phase while the phase runs: its anchor
    // masks, its rows, and (lane 0) one schedule entry of the next sweep.
    const int warp = tid >> 5;
    const bool table_warp = warp == kWarps - 1;
    const bool row_warp = warp == kWarps - 2;
    const bool sched_warp = warp == kWarps - 3;
    if (table_warp) {
        if ((tid & 31) < 8) phase_table(J, g, K, Cl.sweep0, tid & 31, &pp[0][tid & 31]);
        __syncwarp();
        const TaskTab T0 = {tab_am[0], tab_row[0], kTabW, kTabRows};
        if (blocked) build_task_table<true>(pp[0][0], g, T0, tid & 31, 32);
        else build_task_table<false>(pp[0][0], g, T0, tid & 31, 32);
    }
    // Every CTA of the cluster must be running before any peer writes into it.
    if (C > 1) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    } else {
        __syncthreads();
    }

    // Start energy for the trace, read before any CTA of this lattice can finish.
    const long long n_unlike0 = (tid == 0 && rank == 0 && Cl.trace_every > 0) ? J.state[kNUnlike] : 0;
    unsigned long long t_att = 0, t_unl = 0, t_drw = 0, t_acc = 0;
    long long t_dn = 0;
    int block = 0;
    for (long long it = 0; it < Cl.n_mcs; ++it) {
        const long long s = Cl.sweep0 + it;
        const uint32_t s_lo = (uint32_t)(unsigned long long)s;
        const uint32_t s_hi = (uint32_t)((unsigned long long)s >> 32);
        const int buf = (int)(it & 1);
        Acc A = {0u, 0u, 0u, 0u, 0};
        for (int f = 0; f < 8; ++f) {
            const bool last = f == 7 && it + 1 == Cl.n_mcs;
            if ((table_warp || row_warp) && !last) {
                // the next phase's task table (phase 0 of the next sweep after phase 7)
                const PhaseR Pn = f == 7 ? pp[buf ^ 1][0] : pp[buf][f + 1];
                const TaskTab Tn = {tab_am[(f + 1) & 1], tab_row[(f + 1) & 1], kTabW, kTabRows};
                if (table_warp) {
                    if (blocked) build_task_table<true, true, false>(Pn, g, Tn, tid & 31, 32);
                    else build_task_table<false, true, false>(Pn, g, Tn, tid & 31, 32);
                } else {
                    if (blocked) build_task_table<true, false, true>(Pn, g, Tn, tid & 31, 32);
                    else build_task_table<false, false, true>(Pn, g, Tn, tid & 31, 32);
                }
            }
            // Phase f of the next sweep: one schedule entry per phase.  (Entry f of the
            // other buffer was last read in phase f of the previous sweep; phase 0's is
            // written here before phase 7 builds its task table from it.)
            if (sched_warp && (tid & 31) == 0 && it + 1 < Cl.n_mcs)
                phase_table(J, g, K, s + 1, f, &pp[buf ^ 1][f]);
            const PhaseR P = pp[buf][f];
            const TaskTab Tc = {tab_am[f & 1], tab_row[f & 1], kTabW, kTabRows};
            const TaskTab *tt = &Tc;
            if (blocked) {
                if (J.geometry == kTRI6)
                    run_phase_oi<kTRI6, THREADS, true>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
                else
                    run_phase_oi<kSQ4, THREADS, true>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
                __syncthreads();
                if (f % K == K - 1 && !(f == 7 && it + 1 == Cl.n_mcs)) {
                    exchange_halos<THREADS>(lat, g, hmax, block & 1);
                    ++block;
                }
            } else {
                if (J.geometry == kTRI6)
                    run_phase_oi<kTRI6, THREADS, false>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
                else
                    run_phase_oi<kSQ4, THREADS, false>(lat, g, P, thr, f, s_lo, s_hi, A, tt);
                phase_barrier(C);
            }
        }
        t_att += A.att; t_unl += A.unl; t_drw += A.drw; t_acc += A.acc;
        t_dn += A.dn;
        // Energy trace: each CTA adds its cumulative dn; CTA 0 adds the start value
        // (the launcher zeroes the trace buffer).
        if (Cl.trace_every > 0 && (it + 1) % Cl.trace_every == 0) {
            const long long ws = warp_sum(t_dn);
            if ((tid & 31) == 0 && ws != 0)
                atomicAdd((unsigned long long *)&Cl.trace[(it + 1) / Cl.trace_every - 1],
                          (unsigned long long)ws);
            if (tid == 0 && rank == 0)
                atomicAdd((unsigned long long *)&Cl.trace[(it + 1) / Cl.trace_every - 1],
                          (unsigned long long)n_unlike0);
        }
    }

    // Write the band back (main positions only).
    for (int idx = tid; idx < H * g.W; idx += THREADS) {
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

    // Counters and energy.
    long long vals[5] = {(long long)t_att, (long long)t_unl, (long long)t_drw, (long long)t_acc, t_dn};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const long long ws = warp_sum(vals[k]);
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

#ifndef KLMC_BAND_THREADS
#define KLMC_BAND_THREADS 1024
#endif
constexpr int kBandThreads = KLMC_BAND_THREADS;  // one CTA per SM

// Band kernel shared memory (32-bit words): rows (H + 2D) x RWb, the warps' draw
// queues, then (where they fit) K task tables of W words (rounded up to even) and
// 2 x rows words each.  A band row is the padded row of the resident kernel (word 0
// holds position -1, words 1..W the sites, W+1 the last pads) placed 3 words into
// RWb = W + 5 rounded up to 4 words, so that its sites start on a 16-byte boundary
// and a row of the bit store lands there by one bulk copy.
__host__ __device__ __forceinline__ int band_row_words(int W)
{
    return (W + 5 + 3) / 4 * 4;
}

__host__ __device__ __forceinline__ int band_table_rows(int H, int K)
{
    return (H + 4 * K) / 2 + 2;  // anchor rows of a phase over H + 2(2K - 1) rows, py >= 2
}

__host__ __device__ __forceinline__ long long band_table_offset(int H, int K, int RWb)
{
    return (long long)(H + 2 * (2 * K + 1)) * RWb + (long long)kBandThreads / 32 * kDrawQueue2Words;
}

// Waits for phase `parity` of the mbarrier at shared address mbar, giving up after
// `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

constexpr int kCopyWaitPolls = 1 << 20;
constexpr int kCopyWaitPollsShort = 1 << 12;  // under the test hook (SweepJob::copy_shortfall)

// Tiled path, blocked: bands of H rows of a lattice too large for a cluster's
// shared memory, one CTA each, K phases per launch.  A CTA loads its band and
// D = 2K + 1 halo rows per side from the store `src` as it was at the launch's
// start, advances K phases with the blocked phase code above (every flip local,
// only the band's anchors counted), and writes its band to `dst`.  Reading one
// buffer and writing the other keeps every CTA's halo at the launch's starting
// state while other CTAs finish; the launch boundary orders the blocks.
// Bit stores on 16-byte boundaries move their rows by bulk copies (the TMA unit:
// one copy per row in, one per band row out); other stores word by word.
template <int THREADS>
__global__ void __launch_bounds__(THREADS, 1)
band_phases_kernel(const SweepJob J, const void *__restrict__ src, void *__restrict__ dst, int H, int K,
                   int tables, int k, int f0)
{
    constexpr int kWarps = THREADS / 32;
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ PhaseR pp[8];
    __shared__ uint64_t thr[16];
    __shared__ long long red[5][kWarps];
    __shared__ __align__(8) unsigned long long copy_bar;
    // The next launch may be scheduled now; it waits for this one before it reads.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    Geo g;
    g.Lx = J.Lx; g.Ly = J.Ly; g.W = J.W; g.RW = band_row_words(J.W); g.magicW = J.magicW;
    g.k0 = J.key0; g.k1 = J.key1;
    g.zm1 = (J.geometry == kTRI6 ? 6 : 4) - 1;
    g.sign = J.draw_lo > J.draw_hi ? 0 : (J.draw_lo == 0 ? -1 : 1);
    g.C = (int)gridDim.x;
    g.rank = (int)blockIdx.x;
    g.Y0 = (int)blockIdx.x * H;
    g.Y1 = min(g.Y0 + H, g.Ly);
    g.prevY = g.prevH = g.nextY = g.nextH = 0;
    uint32_t *const lat = smem + 3;  // padded row lr, word w: lat[lr * RWb + w]
    g.lat_addr = smem_addr(lat);
    g.D = 2 * K + 1;
    g.base = g.Y0 - g.D < 0 ? g.Y0 - g.D + g.Ly : g.Y0 - g.D;
    const int tid = threadIdx.x;
    const int Hc = g.Y1 - g.Y0;
    const int NL = Hc + 2 * g.D;
    const int RWb = g.RW;
    const bool bulk = J.packing == kPackBit && ((((uintptr_t)src) | ((uintptr_t)dst)) & 15u) == 0u &&
                      (J.pitch & 3) == 0 && J.pitch + 4 <= RWb;
    const uint32_t row_bytes = 4u * (uint32_t)J.pitch;
    const uint32_t bar = smem_addr(&copy_bar);
    if (bulk && tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    // Everything below reads what earlier launches on the stream wrote.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (tid < 16) thr[tid] = J.thr[tid];
    const long long s = J.state[kSweepBase] + k;
    const uint32_t s_lo = (uint32_t)(unsigned long long)s;
    const uint32_t s_hi = (uint32_t)((unsigned long long)s >> 32);
    if (tid < K) phase_table(J, g, K, s, f0 + tid, &pp[tid]);

    if (bulk) {
        // One bulk copy per row (pitch words, 16-byte aligned at both ends) into the
        // row's site words, completing on one mbarrier whose expected byte count is
        // exactly theirs; then the pad words.  Under the test hook no copy is
        // issued and the barrier expects the hook's bytes instead, which nothing
        // delivers: the wait runs out with no copy in flight.
        __syncthreads();
        const bool hook = J.copy_shortfall != 0;
        if (tid < 32) {
            if (tid == 0) {
                unsigned long long st;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 %0, [%1], %2;"
                             : "=l"(st)
                             : "r"(bar), "r"(hook ? (uint32_t)J.copy_shortfall : row_bytes * (uint32_t)NL)
                             : "memory");
            }
            __syncwarp();
            for (int lr = tid; !hook && lr < NL; lr += 32) {
                int y = g.Y0 - g.D + lr;
                if (y < 0) y += g.Ly;
                if (y >= g.Ly) y -= g.Ly;
                const char *from = (const char *)src + (size_t)y * row_bytes;
                const uint32_t to = smem_addr(lat + (size_t)lr * RWb + 1);
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                    ::"r"(to), "l"(from), "r"(row_bytes), "r"(bar) : "memory");
            }
        }
        const int polls = hook ? kCopyWaitPollsShort : kCopyWaitPolls;
        const bool ok = mbar_wait(bar, 0u, polls);
        if (__syncthreads_or(!ok)) {
            // Give up on this launch: report it and leave the band unwritten.  Only a
            // copy that has not landed after the first bound can still be in flight
            // here (never under the hook); wait a second bound for it.
            if (tid == 0) atomicExch((unsigned long long *)&J.state[kFault], 1ull);
            mbar_wait(bar, 0u, polls);
            return;
        }
        for (int lr = tid; lr < NL; lr += THREADS) {
            uint32_t *row = lat + (size_t)lr * RWb;
            const int xl = g.Lx - 1;
            const uint32_t s01 = row[1] & 3u;
            const uint32_t last = (row[(xl >> 5) + 1] >> (xl & 31)) & 1u;
            const int nvalid = g.Lx - 32 * (g.W - 1);
            if (nvalid < 32) row[g.W] &= (1u << nvalid) - 1u;
            for (int w = g.W + 1; w <= J.pitch; ++w) row[w] = 0u;  // beyond the sites
            row[g.W + 1] = 0u;
            row[(g.Lx + 32) >> 5] |= (s01 & 1u) << (g.Lx & 31);       // position Lx: site 0
            row[(g.Lx + 33) >> 5] |= (s01 >> 1) << ((g.Lx + 1) & 31);  // position Lx + 1: site 1
            row[0] = last << 31;                                         // position -1: site Lx - 1
        }
    } else {
        for (int idx = tid; idx < NL * (g.W + 2); idx += THREADS) {
            const int lr = idx / (g.W + 2), w = idx - lr * (g.W + 2);
            int y = g.Y0 - g.D + lr;
            if (y < 0) y += g.Ly;
            if (y >= g.Ly) y -= g.Ly;
            lat[(size_t)lr * RWb + w] = padded_word(src, J.packing, J.pitch, y, w, g.Lx, g.W);
        }
    }
    __syncthreads();
    // The block's task tables follow the rows and the draw queues.
    const int tab_rows = band_table_rows(H, K);
    const int tab_w = (g.W + 1) & ~1;  // even, so that the int2 row entries stay aligned
    uint32_t *const tab_base = smem + band_table_offset(H, K, RWb);
    if (tables) {
        for (int q = 0; q < K; ++q) {
            uint32_t *const t = tab_base + (size_t)q * (tab_w + 2 * tab_rows);
            const TaskTab T = {t, (int2 *)(t + tab_w), g.W, tab_rows};
            build_task_table<true>(pp[q], g, T, tid, THREADS);
        }
        __syncthreads();
    }

    Acc A = {0u, 0u, 0u, 0u, 0};
    // the warps' draw queues follow the rows (H + 2D rows of the tallest band)
    uint32_t *const dq = smem + (size_t)(H + 2 * g.D) * RWb + (size_t)(tid >> 5) * kDrawQueue2Words;
    dq[2 * 32 * 4 + 2 * 32 + (tid & 31)] = 0u;       // the queue's accept words start at zero
    dq[2 * 32 * 4 + 2 * 32 + 32 + (tid & 31)] = 0u;
    for (int j = 0; j < K; ++j) {
        const PhaseR P = pp[j];
        uint32_t *const t = tab_base + (size_t)j * (tab_w + 2 * tab_rows);
        const TaskTab T = {t, (int2 *)(t + tab_w), g.W, tab_rows};
        const TaskTab *const tt = tables ? &T : nullptr;
        if (J.geometry == kTRI6)
            run_phase_pair_oi<kTRI6, THREADS, true>(lat, g, P, thr, f0 + j, s_lo, s_hi, A, dq, tt, J.rk);
        else
            run_phase_pair_oi<kSQ4, THREADS, true>(lat, g, P, thr, f0 + j, s_lo, s_hi, A, dq, tt, J.rk);
        __syncthreads();
    }

    if (bulk) {
        // The band's rows as stored: sites only, then one bulk copy per row.
        for (int r = tid; r < Hc; r += THREADS) {
            uint32_t *row = lat + (size_t)(r + g.D) * RWb;
            const int nvalid = g.Lx - 32 * (g.W - 1);
            if (nvalid < 32) row[g.W] &= (1u << nvalid) - 1u;
            for (int w = g.W + 1; w <= J.pitch; ++w) row[w] = 0u;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid < 32) {
            for (int r = tid; r < Hc; r += 32) {
                char *to = (char *)dst + (size_t)(g.Y0 + r) * row_bytes;
                const uint32_t from = smem_addr(lat + (size_t)(r + g.D) * RWb + 1);
                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                             ::"l"(to), "r"(from), "r"(row_bytes) : "memory");
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        }
    } else {
        for (int idx = tid; idx < Hc * g.W; idx += THREADS) {
            const int r = idx / g.W, w = idx - r * g.W;
            const int y = g.Y0 + r;
            const uint32_t v = lat[(size_t)(r + g.D) * RWb + w + 1];
            const int pos0 = 32 * w;
            const int nvalid = min(32, g.Lx - pos0);
            if (J.packing == kPackBit) {
                const uint32_t valid = nvalid == 32 ? 0xFFFFFFFFu : ((1u << nvalid) - 1u);
                ((uint32_t *)dst)[(size_t)y * J.pitch + w] = v & valid;
            } else {
                uint8_t *row = (uint8_t *)dst + (size_t)y * J.pitch;
                for (int b = 0; b < nvalid; ++b) row[pos0 + b] = (uint8_t)((v >> b) & 1u);
            }
        }
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

// Three variants: 512 threads (one CTA per SM; single lattices on one CTA), 256
// threads with at most 128 registers (two CTAs per SM) and 128 threads with at
// most 128 registers (four CTAs per SM; batches of many lattices).
template <int THREADS, int MINB>
cudaError_t configure_once()
{
    static thread_local int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(resident_sweep_kernel<THREADS, MINB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, resident_max_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(resident_sweep_kernel<THREADS, MINB>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) configured_device = dev;
    return e;
}

cudaError_t launch(const SweepJob *d_jobs, const SweepCall *d_calls, const int *d_map,
                   const SweepJob &job0, const SweepCall &call0, int n_jobs, int cluster,
                   int threads, size_t smem_bytes, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3((unsigned)(n_jobs * cluster), 1, 1);
    cfg.dynamicSmemBytes = smem_bytes;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (threads == 512) {
        e = configure_once<512, 1>();
        if (e != cudaSuccess) return e;
        cfg.blockDim = dim3(512, 1, 1);
        e = cudaLaunchKernelEx(&cfg, resident_sweep_kernel<512, 1>, d_jobs, d_calls, d_map, job0, call0);
    } else if (threads == 128) {
        e = configure_once<128, 4>();
        if (e != cudaSuccess) return e;
        cfg.blockDim = dim3(128, 1, 1);
        e = cudaLaunchKernelEx(&cfg, resident_sweep_kernel<128, 4>, d_jobs, d_calls, d_map, job0, call0);
    } else {
        e = configure_once<256, 2>();
        if (e != cudaSuccess) return e;
        cfg.blockDim = dim3(256, 1, 1);
        e = cudaLaunchKernelEx(&cfg, resident_sweep_kernel<256, 2>, d_jobs, d_calls, d_map, job0, call0);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace

size_t resident_smem_bytes(int Lx, int Ly, int cluster)
{
    const size_t RW = (size_t)(Lx + 95) / 32;  // ceil(Lx / 32) + 2
    const int C = cluster < 1 ? 1 : cluster;
    const size_t H = (size_t)((Ly + C - 1) / C);  // tallest band
    const int K = block_phases(Lx, Ly, C);
    if (K > 1) return RW * (H + 6 * (size_t)(2 * K + 1)) * sizeof(uint32_t);  // rows + mailboxes
    return RW * (H + 4) * sizeof(uint32_t);
}

int resident_max_smem_bytes() { return kResidentMaxSmem; }

int resident_block_phases(int Lx, int Ly, int cluster) { return block_phases(Lx, Ly, cluster); }

int resident_default_threads(int cluster) { return cluster == 1 ? 512 : 256; }

int resident_max_cluster(int Ly)
{
    int c = 16;
    while (c > 1 && Ly / c < 4) c >>= 1;
    return c;
}

cudaError_t launch_resident_sweep(const SweepJob *d_jobs, const SweepCall *d_calls,
                                  const int *d_map, int n_jobs, int cluster, int threads,
                                  size_t smem_bytes, cudaStream_t stream)
{
    if (n_jobs <= 0) return cudaSuccess;
    SweepJob none_job;
    SweepCall none_call;
    memset(&none_job, 0, sizeof(none_job));
    memset(&none_call, 0, sizeof(none_call));
    return launch(d_jobs, d_calls, d_map, none_job, none_call, n_jobs, cluster, threads, smem_bytes,
                  stream);
}

cudaError_t launch_resident_sweep_one(const SweepJob &job, const SweepCall &call, int cluster,
                                      int threads, size_t smem_bytes, cudaStream_t stream)
{
    return launch(nullptr, nullptr, nullptr, job, call, 1, cluster, threads, smem_bytes, stream);
}

#ifndef KLMC_TILED_BLOCK
#define KLMC_TILED_BLOCK 4
#endif


TiledPlan tiled_band_plan(int Lx, int Ly, int sm_count)
{
    TiledPlan p;
    const int RWb = band_row_words((Lx + 31) / 32);
    const long long W = (((Lx + 31) / 32) + 1) & ~1ll;
    for (int K = KLMC_TILED_BLOCK; K >= 2; K >>= 1) {
        const int D = 2 * K + 1;
        long long H = (Ly + sm_count - 1) / sm_count;  // one CTA per SM
        // rows and draw queues must fit: shrink the bands (more bands than SMs)
        // until they do
        while (H >= 1 && 4 * band_table_offset((int)H, K, RWb) > kResidentMaxSmem) --H;
        if (H < 1 || H + 2 * D > Ly) continue;  // a band's rows must not wrap onto themselves
        const long long rows = 4 * band_table_offset((int)H, K, RWb);
        const long long tabs = 4 * K * (W + 2 * band_table_rows((int)H, K));
        p.H = (int)H;
        p.K = K;
        p.threads = kBandThreads;
        p.tables = rows + tabs <= kResidentMaxSmem ? 1 : 0;  // the task tables where they fit
        p.smem = (size_t)(rows + (p.tables ? tabs : 0));
        return p;
    }
    p.H = 0;
    p.K = 1;
    p.threads = 0;
    p.tables = 0;
    p.smem = 0;
    return p;
}

cudaError_t configure_band()
{
    static thread_local int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(band_phases_kernel<kBandThreads>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kResidentMaxSmem);
    if (e == cudaSuccess) configured_device = dev;
    return e;
}

cudaError_t launch_band_phases(const SweepJob &job, const TiledPlan &plan, const void *src, void *dst,
                               int k, int f0, cudaStream_t stream)
{
    // Programmatic dependent launch: the CTAs of this launch may be scheduled while
    // the previous one drains, and wait for it in the kernel before reading.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((job.Ly + plan.H - 1) / plan.H), 1, 1);
    cfg.blockDim = dim3(kBandThreads, 1, 1);
    cfg.dynamicSmemBytes = plan.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, band_phases_kernel<kBandThreads>, job, src, dst, plan.H, plan.K,
                                       plan.tables, k, f0);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace klmc
