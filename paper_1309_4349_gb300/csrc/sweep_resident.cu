// sweep_resident.cu -- Kawasaki exchange sweeps with the whole lattice resident in
// shared memory, one CTA per lattice (section "Massive Parallel Kawasaki Kinetics":
// every iteration performs one exchange per domain of a random decomposition, all
// in parallel; here the decomposition is a conflict-free shifted sublattice phase).
//
// Shared-memory layout: row y is RW 32-bit words holding the padded bit positions
// pos in [-32, 32*RW - 32); position pos holds site (pos mod Lx, y).  Every copy of
// a site is kept equal, so the 32-site window starting at any x in [-32, Lx + 32]
// is one funnel shift of two words.
//
// One thread handles the anchors of one 32-site word of one anchor row.  The
// neighbour comparisons of all 32 positions are formed with bitwise operations
// and summed with a carry-save adder tree into bit planes of S = same_a + same_b,
// the number of neighbours of a (other than b) equal to a plus those of b (other
// than a) equal to b.  An exchange changes the unlike-contact count by
// dn = 2 (S - (z - 1)).  Only positions whose S lies in the draw range draw a
// Philox number; the rest of the unlike pairs are accepted outright (Metropolis
// acceptance min{1, exp(-omega dn / kT)}, Metropolis steps a-c).
#include <string.h>

#include "klmc_internal.h"

namespace klmc {
namespace {

constexpr int kThreads = 1024;
constexpr int kWarps = kThreads / 32;

struct PhaseP {
    int oi, rx, ry, px, py, Kx, My, ntask, umax;
};

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products,
// the high halves mixed into the other words with the round key; Weyl key bump.
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                           uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned long long p0 = (unsigned long long)c0 * 0xD2511F53ull;
        unsigned long long p1 = (unsigned long long)c2 * 0xCD9E8D57ull;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Philox4 out;
    out.v[0] = c0; out.v[1] = c1; out.v[2] = c2; out.v[3] = c3;
    return out;
}

// Phase parameters of (sweep s, phase f): orientation index, shift, sublattice
// periods and counts.  Orientation 1 is (0,1) in both geometries.
__device__ void phase_params(int geometry, int Lx, int Ly, int W, uint32_t k0, uint32_t k1,
                             long long s, int f, PhaseP *P)
{
    Philox4 w = philox4(0xFFFFFFFFu, (uint32_t)f, (uint32_t)(unsigned long long)s,
                        (uint32_t)((unsigned long long)s >> 32), k0, k1);
    int nO = geometry == kTRI6 ? 3 : 2;
    P->oi = (int)__umulhi(w.v[0], (uint32_t)nO);
    P->rx = (int)__umulhi(w.v[1], (uint32_t)Lx);
    P->ry = (int)__umulhi(w.v[2], (uint32_t)Ly);
    if (P->oi == 1) {
        P->px = 2; P->py = 4;
        P->Kx = (Lx - 2) / 2 + 1;
        P->My = (Ly - 3) / 4 + 1;
    } else {
        P->px = 4; P->py = 2;
        P->Kx = (Lx - 3) / 4 + 1;
        P->My = (Ly - 2) / 2 + 1;
    }
    P->ntask = P->My * W;
    P->umax = P->px * (P->Kx - 1);
}

// Bits p of the word at x0 with x0 + p in [lo, hi].
__device__ __forceinline__ uint32_t range_mask(int lo, int hi, int x0)
{
    int a = max(lo - x0, 0), b = min(hi - x0, 31);
    if (a > b) return 0u;
    return (0xFFFFFFFFu >> (31 - b)) & (0xFFFFFFFFu << a);
}

// Anchors of the phase in the word at x0: x = (rx + px k) mod Lx, k < Kx.
__device__ __forceinline__ uint32_t anchor_mask(int x0, const PhaseP &P, int Lx)
{
    const uint32_t rep = P.px == 4 ? 0x11111111u : 0x55555555u;
    const int pm = P.px - 1;
    uint32_t m = (rep << ((P.rx - x0) & pm)) & range_mask(P.rx, min(P.rx + P.umax, Lx - 1), x0);
    const int hi2 = min(P.rx - 1, P.rx + P.umax - Lx);  // wrapped part of the anchor row
    if (hi2 >= 0) m |= (rep << ((P.rx - Lx - x0) & pm)) & range_mask(0, hi2, x0);
    return m;
}

__device__ __forceinline__ uint32_t fsr(uint32_t lo, uint32_t hi, int s)
{
    return __funnelshift_r(lo, hi, s);
}

// Full adder on bit planes.
__device__ __forceinline__ void fa(uint32_t a, uint32_t b, uint32_t c, uint32_t &s, uint32_t &cy)
{
    s = a ^ b ^ c;
    cy = (a & b) | (c & (a ^ b));
}

struct Planes {
    uint32_t s0, s1, s2, s3;
};

// Bit-sliced sum of ten 1-bit inputs (0..10).
__device__ __forceinline__ Planes count10(uint32_t e0, uint32_t e1, uint32_t e2, uint32_t e3,
                                          uint32_t e4, uint32_t e5, uint32_t e6, uint32_t e7,
                                          uint32_t e8, uint32_t e9)
{
    uint32_t sa, ca, sb, cb, sc, cc, sd, cd;
    fa(e0, e1, e2, sa, ca);
    fa(e3, e4, e5, sb, cb);
    fa(e6, e7, e8, sc, cc);
    fa(sa, sb, sc, sd, cd);             // weight-1: sd; weight-2: cd
    Planes P;
    P.s0 = sd ^ e9;
    uint32_t ce = sd & e9;              // weight 2
    uint32_t s2a, c2a, s2b, c2b;
    fa(ca, cb, cc, s2a, c2a);           // weight 2 -> s2a (w2), c2a (w4)
    fa(cd, ce, s2a, s2b, c2b);          // weight 2 -> s2b (w2), c2b (w4)
    P.s1 = s2b;
    P.s2 = c2a ^ c2b;
    P.s3 = c2a & c2b;
    return P;
}

// Bit-sliced sum of six 1-bit inputs (0..6).
__device__ __forceinline__ Planes count6(uint32_t e0, uint32_t e1, uint32_t e2, uint32_t e3,
                                         uint32_t e4, uint32_t e5)
{
    uint32_t sa, ca, sb, cb, s2, c2;
    fa(e0, e1, e2, sa, ca);
    fa(e3, e4, e5, sb, cb);
    Planes P;
    P.s0 = sa ^ sb;
    fa(ca, cb, sa & sb, s2, c2);
    P.s1 = s2;
    P.s2 = c2;
    P.s3 = 0u;
    return P;
}

// Positions with S >= c (c uniform).
__device__ __forceinline__ uint32_t ge_const(const Planes &S, int c)
{
    if (c <= 0) return 0xFFFFFFFFu;
    if (c >= 16) return 0u;
    const uint32_t sb[4] = {S.s0, S.s1, S.s2, S.s3};
    uint32_t lt = 0u, eq = 0xFFFFFFFFu;
#pragma unroll
    for (int b = 3; b >= 0; --b) {
        if ((c >> b) & 1) {
            lt |= eq & ~sb[b];
            eq &= sb[b];
        } else {
            eq &= ~sb[b];
        }
    }
    return ~lt;
}

__device__ __forceinline__ uint32_t eqm(uint32_t v, uint32_t t) { return ~(v ^ t); }

// XOR mask into padded buffer bit positions q .. q+31 of one row (clipped).
__device__ __forceinline__ void xor_at(uint32_t *row, int RW, int q, uint32_t mask)
{
    if (q < 0) {
        if (q <= -32) return;
        mask >>= -q;
        q = 0;
    }
    const int w = q >> 5, s = q & 31;
    if (w < RW) atomicXor(row + w, mask << s);
    if (s != 0 && w + 1 < RW) atomicXor(row + w + 1, mask >> (32 - s));
}

// Flip the sites at positions pos + p (mask bit p) and every padded copy.
__device__ __forceinline__ void flip_sites(uint32_t *row, int RW, int Lx, int pos, uint32_t mask)
{
    const int q = pos + 32;
    for (int qq = q; qq > -32; qq -= Lx) xor_at(row, RW, qq, mask);
    for (int qq = q + Lx; qq < 32 * RW; qq += Lx) xor_at(row, RW, qq, mask);
}

struct Geo {
    int Lx, Ly, W, RW;
    unsigned long long magicW;
    uint32_t k0, k1;
    int draw_lo, draw_hi;
    int zm1;
};

struct Acc {
    uint32_t att, unl, drw, acc;
    int32_t dn;
};

__device__ __forceinline__ const uint32_t *row_ptr(const uint32_t *lat, const Geo &g, int y)
{
    if (y < 0) y += g.Ly;
    if (y >= g.Ly) y -= g.Ly;
    return lat + (size_t)y * g.RW;
}

// One phase of one lattice: every task is (anchor row m, word j).
template <int G, int OI>
__device__ __forceinline__ void run_phase(uint32_t *lat, const Geo &g, const PhaseP &P,
                                          const uint64_t *thr, int f, uint32_t s_lo,
                                          uint32_t s_hi, Acc &A)
{
    // b = a + o: (1,0) -> same row, +1; (0,1) -> next row; (1,-1) -> previous row, +1
    constexpr int bdy = OI == 0 ? 0 : (OI == 1 ? 1 : -1);
    constexpr int bdx = OI == 1 ? 0 : 1;
    for (int t = threadIdx.x; t < P.ntask; t += kThreads) {
        const int m = (int)(((unsigned long long)t * g.magicW) >> 32);
        const int j = t - m * g.W;
        int y = P.ry + P.py * m;
        if (y >= g.Ly) y -= g.Ly;
        const int x0 = j << 5;
        const uint32_t am = anchor_mask(x0, P, g.Lx);
        if (am == 0u) continue;

        uint32_t ta, tb;
        Planes S;
        const uint32_t *r0 = row_ptr(lat, g, y);
        const uint32_t a0 = r0[j], a1 = r0[j + 1], a2 = r0[j + 2];
        const uint32_t Am = fsr(a0, a1, 31), A0 = a1, A1 = fsr(a1, a2, 1);
        if (G == kTRI6 && OI == 0) {
            const uint32_t *rm = row_ptr(lat, g, y - 1), *rp = row_ptr(lat, g, y + 1);
            const uint32_t m1 = rm[j + 1], m2 = rm[j + 2];
            const uint32_t p0 = rp[j], p1 = rp[j + 1], p2 = rp[j + 2];
            const uint32_t M0 = m1, M1 = fsr(m1, m2, 1), M2 = fsr(m1, m2, 2);
            const uint32_t A2 = fsr(a1, a2, 2);
            const uint32_t Pm = fsr(p0, p1, 31), P0 = p1, P1 = fsr(p1, p2, 1);
            ta = A0; tb = A1;
            S = count10(eqm(Am, ta), eqm(P0, ta), eqm(M0, ta), eqm(M1, ta), eqm(Pm, ta),
                        eqm(A2, tb), eqm(P1, tb), eqm(M1, tb), eqm(M2, tb), eqm(P0, tb));
        } else if (G == kTRI6 && OI == 1) {
            const uint32_t *rm = row_ptr(lat, g, y - 1), *rp = row_ptr(lat, g, y + 1),
                           *rq = row_ptr(lat, g, y + 2);
            const uint32_t m1 = rm[j + 1], m2 = rm[j + 2];
            const uint32_t p0 = rp[j], p1 = rp[j + 1], p2 = rp[j + 2];
            const uint32_t q0 = rq[j], q1 = rq[j + 1];
            const uint32_t M0 = m1, M1 = fsr(m1, m2, 1);
            const uint32_t Pm = fsr(p0, p1, 31), P0 = p1, P1 = fsr(p1, p2, 1);
            const uint32_t Qm = fsr(q0, q1, 31), Q0 = q1;
            ta = A0; tb = P0;
            S = count10(eqm(A1, ta), eqm(Am, ta), eqm(M0, ta), eqm(M1, ta), eqm(Pm, ta),
                        eqm(P1, tb), eqm(Pm, tb), eqm(Q0, tb), eqm(A1, tb), eqm(Qm, tb));
        } else if (G == kTRI6 && OI == 2) {
            const uint32_t *rn = row_ptr(lat, g, y - 2), *rm = row_ptr(lat, g, y - 1),
                           *rp = row_ptr(lat, g, y + 1);
            const uint32_t n1 = rn[j + 1], n2 = rn[j + 2];
            const uint32_t m1 = rm[j + 1], m2 = rm[j + 2];
            const uint32_t p0 = rp[j], p1 = rp[j + 1];
            const uint32_t N1 = fsr(n1, n2, 1), N2 = fsr(n1, n2, 2);
            const uint32_t M0 = m1, M1 = fsr(m1, m2, 1), M2 = fsr(m1, m2, 2);
            const uint32_t Pm = fsr(p0, p1, 31), P0 = p1;
            ta = A0; tb = M1;
            S = count10(eqm(A1, ta), eqm(Am, ta), eqm(P0, ta), eqm(M0, ta), eqm(Pm, ta),
                        eqm(M2, tb), eqm(M0, tb), eqm(A1, tb), eqm(N1, tb), eqm(N2, tb));
        } else if (G == kSQ4 && OI == 0) {
            const uint32_t *rm = row_ptr(lat, g, y - 1), *rp = row_ptr(lat, g, y + 1);
            const uint32_t m1 = rm[j + 1], m2 = rm[j + 2];
            const uint32_t p1 = rp[j + 1], p2 = rp[j + 2];
            const uint32_t M0 = m1, M1 = fsr(m1, m2, 1);
            const uint32_t A2 = fsr(a1, a2, 2);
            const uint32_t P0 = p1, P1 = fsr(p1, p2, 1);
            ta = A0; tb = A1;
            S = count6(eqm(Am, ta), eqm(P0, ta), eqm(M0, ta), eqm(A2, tb), eqm(P1, tb),
                       eqm(M1, tb));
        } else {  // SQ4, (0,1)
            const uint32_t *rm = row_ptr(lat, g, y - 1), *rp = row_ptr(lat, g, y + 1),
                           *rq = row_ptr(lat, g, y + 2);
            const uint32_t m1 = rm[j + 1];
            const uint32_t p0 = rp[j], p1 = rp[j + 1], p2 = rp[j + 2];
            const uint32_t q1 = rq[j + 1];
            const uint32_t M0 = m1;
            const uint32_t Pm = fsr(p0, p1, 31), P0 = p1, P1 = fsr(p1, p2, 1);
            const uint32_t Q0 = q1;
            ta = A0; tb = P0;
            S = count6(eqm(A1, ta), eqm(Am, ta), eqm(M0, ta), eqm(P1, tb), eqm(Pm, tb),
                       eqm(Q0, tb));
        }

        const uint32_t unl = (ta ^ tb) & am;
        const uint32_t dmask = unl & ge_const(S, g.draw_lo) & ~ge_const(S, g.draw_hi + 1);
        uint32_t acc = unl & ~dmask;
        uint32_t dm = dmask;
        while (dm) {
            const int p = __ffs(dm) - 1;
            dm &= dm - 1;
            const uint32_t Sp = ((S.s0 >> p) & 1u) | (((S.s1 >> p) & 1u) << 1) |
                                (((S.s2 >> p) & 1u) << 2) | (((S.s3 >> p) & 1u) << 3);
            const uint32_t site = (uint32_t)(y * g.Lx + x0 + p);
            const Philox4 r = philox4(site, (uint32_t)f, s_lo, s_hi, g.k0, g.k1);
            if ((uint64_t)r.v[0] < thr[Sp]) acc |= 1u << p;
        }
        A.att += __popc(am);
        A.unl += __popc(unl);
        A.drw += __popc(dmask);
        if (acc) {
            const int na = __popc(acc);
            A.acc += na;
            const int sum_s = __popc(S.s0 & acc) + 2 * __popc(S.s1 & acc) +
                              4 * __popc(S.s2 & acc) + 8 * __popc(S.s3 & acc);
            A.dn += 2 * (sum_s - g.zm1 * na);
            flip_sites(lat + (size_t)y * g.RW, g.RW, g.Lx, x0, acc);
            int yb = y + bdy;
            if (yb < 0) yb += g.Ly;
            if (yb >= g.Ly) yb -= g.Ly;
            flip_sites(lat + (size_t)yb * g.RW, g.RW, g.Lx, x0 + bdx, acc);
        }
    }
}

__device__ __forceinline__ uint32_t load_site(const SweepJob &J, int x, int y)
{
    if (J.packing == kPackBit) {
        const uint32_t *row = (const uint32_t *)J.lat + (size_t)y * J.pitch;
        return (row[x >> 5] >> (x & 31)) & 1u;
    }
    return ((const uint8_t *)J.lat)[(size_t)y * J.pitch + x] ? 1u : 0u;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void __launch_bounds__(kThreads, 1)
resident_sweep_kernel(const SweepJob *__restrict__ jobs, const SweepCall *__restrict__ calls,
                      const SweepJob job0, const SweepCall call0)
{
    extern __shared__ __align__(16) uint32_t lat[];
    __shared__ PhaseP pp[2][8];
    __shared__ uint64_t thr[16];
    __shared__ long long red[5][kWarps];
    __shared__ long long running;

    const SweepJob &J = jobs ? jobs[blockIdx.x] : job0;
    const SweepCall C = calls ? calls[blockIdx.x] : call0;
    if (C.n_mcs <= 0) return;

    Geo g;
    g.Lx = J.Lx; g.Ly = J.Ly; g.W = J.W; g.RW = J.RW; g.magicW = J.magicW;
    g.k0 = J.key0; g.k1 = J.key1; g.draw_lo = J.draw_lo; g.draw_hi = J.draw_hi;
    g.zm1 = (J.geometry == kTRI6 ? 6 : 4) - 1;
    const int tid = threadIdx.x;

    // Load the lattice into padded shared-memory rows.
    for (int idx = tid; idx < g.Ly * g.RW; idx += kThreads) {
        const int y = idx / g.RW, w = idx - y * g.RW;
        const int pos0 = 32 * w - 32;
        uint32_t v = 0u;
        if (J.packing == kPackBit && pos0 >= 0 && pos0 + 32 <= g.Lx) {
            v = ((const uint32_t *)J.lat)[(size_t)y * J.pitch + (w - 1)];
        } else {
            for (int b = 0; b < 32; ++b) {
                int x = (pos0 + b) % g.Lx;
                if (x < 0) x += g.Lx;
                v |= load_site(J, x, y) << b;
            }
        }
        lat[idx] = v;
    }
    if (tid < 16) thr[tid] = J.thr[tid];
    if (tid < 8) phase_params(J.geometry, g.Lx, g.Ly, g.W, g.k0, g.k1, C.sweep0, tid, &pp[0][tid]);
    if (tid == 0) running = J.state[kNUnlike];
    __syncthreads();

    unsigned long long t_att = 0, t_unl = 0, t_drw = 0, t_acc = 0;
    long long t_dn = 0;
    int dn_trace = 0;
    for (long long it = 0; it < C.n_mcs; ++it) {
        const long long s = C.sweep0 + it;
        const uint32_t s_lo = (uint32_t)(unsigned long long)s;
        const uint32_t s_hi = (uint32_t)((unsigned long long)s >> 32);
        const int buf = (int)(it & 1);
        Acc A = {0u, 0u, 0u, 0u, 0};
        for (int f = 0; f < 8; ++f) {
            if (f == 7 && tid < 8 && it + 1 < C.n_mcs)
                phase_params(J.geometry, g.Lx, g.Ly, g.W, g.k0, g.k1, s + 1, tid, &pp[buf ^ 1][tid]);
            const PhaseP P = pp[buf][f];
            if (J.geometry == kTRI6) {
                if (P.oi == 0) run_phase<kTRI6, 0>(lat, g, P, thr, f, s_lo, s_hi, A);
                else if (P.oi == 1) run_phase<kTRI6, 1>(lat, g, P, thr, f, s_lo, s_hi, A);
                else run_phase<kTRI6, 2>(lat, g, P, thr, f, s_lo, s_hi, A);
            } else {
                if (P.oi == 0) run_phase<kSQ4, 0>(lat, g, P, thr, f, s_lo, s_hi, A);
                else run_phase<kSQ4, 1>(lat, g, P, thr, f, s_lo, s_hi, A);
            }
            __syncthreads();
        }
        t_att += A.att; t_unl += A.unl; t_drw += A.drw; t_acc += A.acc;
        t_dn += A.dn;
        dn_trace += A.dn;
        if (C.trace_every > 0 && C.trace != nullptr && (it + 1) % C.trace_every == 0) {
            const int ws = warp_sum(dn_trace);
            if ((tid & 31) == 0) red[0][tid >> 5] = ws;
            dn_trace = 0;
            __syncthreads();
            if (tid == 0) {
                long long sum = 0;
                for (int w = 0; w < kWarps; ++w) sum += red[0][w];
                running += sum;
                C.trace[(it + 1) / C.trace_every - 1] = running;
            }
            __syncthreads();
        }
    }

    // Write the lattice back (main positions only).
    for (int idx = tid; idx < g.Ly * g.W; idx += kThreads) {
        const int y = idx / g.W, w = idx - y * g.W;
        const uint32_t v = lat[(size_t)y * g.RW + w + 1];
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

}  // namespace

size_t resident_smem_bytes(int Lx, int Ly)
{
    const size_t RW = (size_t)(Lx + 127) / 32;
    return RW * (size_t)Ly * sizeof(uint32_t);
}

int resident_max_smem_bytes()
{
    // Dynamic shared memory left after the kernel's static arrays.
    return 227 * 1024 - 4096;
}

namespace {
cudaError_t configure_resident()
{
    // Once per process and device use; setting the attribute again is harmless.
    static thread_local int configured_device = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (configured_device == dev) return cudaSuccess;
    e = cudaFuncSetAttribute(resident_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             resident_max_smem_bytes());
    if (e == cudaSuccess) configured_device = dev;
    return e;
}
}  // namespace

cudaError_t launch_resident_sweep(const SweepJob *d_jobs, const SweepCall *d_calls, int n_jobs,
                                  size_t smem_bytes, cudaStream_t stream)
{
    if (n_jobs <= 0) return cudaSuccess;
    cudaError_t e = configure_resident();
    if (e != cudaSuccess) return e;
    SweepJob none_job;
    SweepCall none_call;
    memset(&none_job, 0, sizeof(none_job));
    memset(&none_call, 0, sizeof(none_call));
    resident_sweep_kernel<<<n_jobs, kThreads, smem_bytes, stream>>>(d_jobs, d_calls, none_job,
                                                                     none_call);
    return cudaGetLastError();
}

cudaError_t launch_resident_sweep_one(const SweepJob &job, const SweepCall &call, size_t smem_bytes,
                                      cudaStream_t stream)
{
    cudaError_t e = configure_resident();
    if (e != cudaSuccess) return e;
    resident_sweep_kernel<<<1, kThreads, smem_bytes, stream>>>(nullptr, nullptr, job, call);
    return cudaGetLastError();
}

}  // namespace klmc
