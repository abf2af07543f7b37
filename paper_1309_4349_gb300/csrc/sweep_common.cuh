// sweep_common.cuh -- device code shared by the resident and the tiled sweep
// kernels: the phase schedule, the anchor masks, the bit-sliced evaluation of one
// 32-site word and its draws (Philox4x32-10 from philox.cuh, which the including
// file includes at file scope).  Included inside namespace klmc.
#pragma once

struct PhaseP {
    int oi, rx, ry, px, py, umax;
    int a1, n1, a2, n2, M1;  // this band's anchor rows: m in [a1, a1+n1) u [a2, a2+n2)
    int ntask;
};

// floor(a / 2^sh) and ceil(a / 2^sh) for any sign of a (the row spacing py of an
// anchor sublattice is 2 or 4, so every division of the schedule is a shift).
__device__ __forceinline__ int floor_shr(int a, int sh) { return a >> sh; }
__device__ __forceinline__ int ceil_shr(int a, int sh) { return -((-a) >> sh); }

// Phase parameters of (sweep s, phase f) and this band's share of its anchor rows.
// Orientation 1 is (0,1) in both geometries.
__device__ void phase_params(int geometry, int Lx, int Ly, int W, int Y0, int Y1, uint32_t k0,
                             uint32_t k1, long long s, int f, PhaseP *P)
{
    Philox4 w = philox4(0xFFFFFFFFu, (uint32_t)f, (uint32_t)(unsigned long long)s,
                        (uint32_t)((unsigned long long)s >> 32), k0, k1);
    const int nO = geometry == kTRI6 ? 3 : 2;
    const int oi = (int)__umulhi(w.v[0], (uint32_t)nO);
    const int rx = (int)__umulhi(w.v[1], (uint32_t)Lx);
    const int ry = (int)__umulhi(w.v[2], (uint32_t)Ly);
    int px, py, Kx, My;
    if (oi == 1) {
        px = 2; py = 4;
        Kx = (Lx - 2) / 2 + 1;
        My = (Ly - 3) / 4 + 1;
    } else {
        px = 4; py = 2;
        Kx = (Lx - 3) / 4 + 1;
        My = (Ly - 2) / 2 + 1;
    }
    // Anchor rows y_m = (ry + py m) mod Ly, m < My: unwrapped for m < M1.
    const int sh = py == 4 ? 2 : 1;
    const int M1 = min(My, ceil_shr(Ly - ry, sh));
    const int a1 = max(ceil_shr(Y0 - ry, sh), 0);
    const int b1 = min(floor_shr(Y1 - 1 - ry, sh), M1 - 1);
    const int a2 = max(ceil_shr(Y0 + Ly - ry, sh), M1);
    const int b2 = min(floor_shr(Y1 - 1 + Ly - ry, sh), My - 1);
    P->oi = oi; P->rx = rx; P->ry = ry; P->px = px; P->py = py;
    P->umax = px * (Kx - 1);
    P->a1 = a1; P->n1 = max(0, b1 - a1 + 1);
    P->a2 = a2; P->n2 = max(0, b2 - a2 + 1);
    P->M1 = M1;
    P->ntask = (P->n1 + P->n2) * W;
}

// Phase parameters of (sweep s, phase f) and the anchor rows whose row lies in
// [lo, hi) modulo Ly (hi - lo <= Ly; lo may be negative and hi may exceed Ly).
// The anchor rows y_m = (ry + py m) mod Ly, m < My, come as up to four runs of
// consecutive m; task row mi (0 <= mi < c[3]) has m = a[i] + mi for the first run
// i with mi < c[i].
struct PhaseR {
    int oi, rx, ry, px, py, umax;
    int a[4], c[4];
    int ntask;
};

__device__ void phase_ranges(int geometry, int Lx, int Ly, int W, int lo, int hi, uint32_t k0,
                             uint32_t k1, long long s, int f, PhaseR *P)
{
    Philox4 w = philox4(0xFFFFFFFFu, (uint32_t)f, (uint32_t)(unsigned long long)s,
                        (uint32_t)((unsigned long long)s >> 32), k0, k1);
    const int nO = geometry == kTRI6 ? 3 : 2;
    const int oi = (int)__umulhi(w.v[0], (uint32_t)nO);
    const int rx = (int)__umulhi(w.v[1], (uint32_t)Lx);
    const int ry = (int)__umulhi(w.v[2], (uint32_t)Ly);
    int px, py, Kx, My;
    if (oi == 1) {
        px = 2; py = 4;
        Kx = (Lx - 2) / 2 + 1;
        My = (Ly - 3) / 4 + 1;
    } else {
        px = 4; py = 2;
        Kx = (Lx - 3) / 4 + 1;
        My = (Ly - 2) / 2 + 1;
    }
    const int sh = py == 4 ? 2 : 1;
    const int M1 = min(My, ceil_shr(Ly - ry, sh));  // m < M1: y_m = ry + py m (no wrap)
    // [lo, hi) as at most two intervals of [0, Ly)
    int u[2], v[2];
    if (lo < 0) {
        u[0] = lo + Ly; v[0] = Ly; u[1] = 0; v[1] = hi;
    } else if (hi > Ly) {
        u[0] = lo; v[0] = Ly; u[1] = 0; v[1] = hi - Ly;
    } else {
        u[0] = lo; v[0] = hi; u[1] = 0; v[1] = 0;
    }
    int total = 0;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int wr = 0; wr < 2; ++wr) {
            const int off = wr ? Ly : 0;
            int a = ceil_shr(u[q] + off - ry, sh);
            int b = floor_shr(v[q] - 1 + off - ry, sh);
            a = max(a, wr ? M1 : 0);
            b = min(b, wr ? My - 1 : M1 - 1);
            const int n = u[q] < v[q] ? max(0, b - a + 1) : 0;
            P->a[2 * q + wr] = a - total;
            total += n;
            P->c[2 * q + wr] = total;
        }
    }
    P->oi = oi; P->rx = rx; P->ry = ry; P->px = px; P->py = py;
    P->umax = px * (Kx - 1);
    P->ntask = total * W;
}

// Bits p of the word at x0 with x0 + p in [lo, hi].
__device__ __forceinline__ uint32_t range_mask(int lo, int hi, int x0)
{
    int a = max(lo - x0, 0), b = min(hi - x0, 31);
    if (a > b) return 0u;
    return (0xFFFFFFFFu >> (31 - b)) & (0xFFFFFFFFu << a);
}

// Anchors of the phase in the word at x0: x = (rx + px k) mod Lx, k < Kx.
template <typename PP>
__device__ __forceinline__ uint32_t anchor_mask(int x0, const PP &P, int Lx)
{
    const uint32_t rep = P.px == 4 ? 0x11111111u : 0x55555555u;
    const int pm = P.px - 1;
    const int hi1 = min(P.rx + P.umax, Lx - 1);
    if (x0 >= P.rx && x0 + 31 <= hi1) return rep << ((P.rx - x0) & pm);  // whole word in range
    uint32_t m = (rep << ((P.rx - x0) & pm)) & range_mask(P.rx, hi1, x0);
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

__device__ __forceinline__ uint32_t eqm(uint32_t v, uint32_t t) { return ~(v ^ t); }

// Positions that need a draw: the exchange raises the energy when omega > 0
// (sign > 0: S > z - 1) or lowers it when omega < 0 (sign < 0: S < z - 1).
template <int G>
__device__ __forceinline__ uint32_t draw_positions(const Planes &S, int sign)
{
    uint32_t up, down;
    if (G == kTRI6) {  // z - 1 = 5, S in 0..10
        up = S.s3 | (S.s2 & S.s1);                     // S >= 6
        down = ~(S.s3 | (S.s2 & (S.s1 | S.s0)));       // S <= 4
    } else {           // z - 1 = 3, S in 0..6
        up = S.s2;                                     // S >= 4
        down = ~(S.s2 | (S.s1 & S.s0));                // S <= 2
    }
    return sign > 0 ? up : (sign < 0 ? down : 0u);
}

// Bit-sliced evaluation of the word at x0 = 32 j of the anchor row whose padded
// shared-memory row is r0 (rows r0 - 2 RW .. r0 + 2 RW are its neighbours): the
// types ta, tb of a = (x, y) and b = a + o for all 32 positions x0 + p, and the bit
// planes of S = same_a + same_b.
template <int G, int OI>
__device__ __forceinline__ void evaluate(const uint32_t *r0, int RW, int j, uint32_t &ta,
                                         uint32_t &tb, Planes &S)
{
    const uint32_t *rm = r0 - RW, *rp = r0 + RW;
    const uint32_t a0 = r0[j], a1 = r0[j + 1], a2 = r0[j + 2];
    const uint32_t Am = fsr(a0, a1, 31), A0 = a1, A1 = fsr(a1, a2, 1);
    if (G == kTRI6 && OI == 0) {
        const uint32_t m1 = rm[j + 1], m2 = rm[j + 2];
        const uint32_t p0 = rp[j], p1 = rp[j + 1], p2 = rp[j + 2];
        const uint32_t M0 = m1, M1 = fsr(m1, m2, 1), M2 = fsr(m1, m2, 2);
        const uint32_t A2 = fsr(a1, a2, 2);
        const uint32_t Pm = fsr(p0, p1, 31), P0 = p1, P1 = fsr(p1, p2, 1);
        ta = A0; tb = A1;
        S = count10(eqm(Am, ta), eqm(P0, ta), eqm(M0, ta), eqm(M1, ta), eqm(Pm, ta),
                    eqm(A2, tb), eqm(P1, tb), eqm(M1, tb), eqm(M2, tb), eqm(P0, tb));
    } else if (G == kTRI6 && OI == 1) {
        const uint32_t *rq = rp + RW;
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
        const uint32_t *rn = rm - RW;
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
        const uint32_t m1 = rm[j + 1], m2 = rm[j + 2];
        const uint32_t p1 = rp[j + 1], p2 = rp[j + 2];
        const uint32_t M0 = m1, M1 = fsr(m1, m2, 1);
        const uint32_t A2 = fsr(a1, a2, 2);
        const uint32_t P0 = p1, P1 = fsr(p1, p2, 1);
        ta = A0; tb = A1;
        S = count6(eqm(Am, ta), eqm(P0, ta), eqm(M0, ta), eqm(A2, tb), eqm(P1, tb),
                   eqm(M1, tb));
    } else {  // SQ4, (0,1)
        const uint32_t *rq = rp + RW;
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
}

// Accept bits of the positions in dmask, each drawing Philox word 0 of counter
// {site_base + p, f, s_lo, s_hi}; two evaluations interleaved at a time.
__device__ __forceinline__ uint32_t draw_accepts(uint32_t dmask, const Planes &S,
                                                 uint32_t site_base, const DrawKey &dk,
                                                 const uint64_t *thr)
{
    uint32_t acc = 0u;
    uint32_t dm = dmask;
    while (dm != 0u) {
        const int p1 = __ffs(dm) - 1;
        dm &= dm - 1u;
        const int p2 = dm != 0u ? __ffs(dm) - 1 : p1;  // an odd last draw is repeated
        dm &= dm - 1u;
        uint32_t r1, r2;
        philox2_w0_key(site_base + (uint32_t)p1, site_base + (uint32_t)p2, dk, r1, r2);
        const uint32_t S1 = ((S.s0 >> p1) & 1u) | (((S.s1 >> p1) & 1u) << 1) |
                            (((S.s2 >> p1) & 1u) << 2) | (((S.s3 >> p1) & 1u) << 3);
        const uint32_t S2 = ((S.s0 >> p2) & 1u) | (((S.s1 >> p2) & 1u) << 1) |
                            (((S.s2 >> p2) & 1u) << 2) | (((S.s3 >> p2) & 1u) << 3);
        if ((uint64_t)r1 < thr[S1]) acc |= 1u << p1;
        if ((uint64_t)r2 < thr[S2]) acc |= 1u << p2;
    }
    return acc;
}

// Accept bits of two tasks per lane (t and t + THREADS) when the warp's draws are
// drawn by all its lanes.  Every lane stores each task's S planes and first site
// index once, and appends its draws (task, lane, bit) as 16-bit entries to the
// warp's queue at its prefix-sum offset; then lane i draws entries i and i + 32 of
// every 64 (two Philox chains interleaved), reading the entry's S and site from
// its record, and returns accepted bits through the warp's accept words with
// shared atomics.  One scan and one pass serve both tasks, so a pass drains about
// twice the draws of one task per lane.  When the warp has more than kDrawQueue2
// draws, each lane draws its own.  Every lane of the warp must call it.  Region q
// (16-byte aligned, kDrawQueue2Words words): planes uint4[2][32], sites
// uint32[2][32], accept words uint32[2][32] (zero on entry and on return),
// entries uint16[kDrawQueue2].
constexpr int kDrawQueue2 = 512;
constexpr int kDrawQueue2Words = 2 * 32 * 4 + 2 * 32 + 2 * 32 + kDrawQueue2 / 2;

template <bool RK>  // RK: the round keys from rk (kernel parameter space); else from dk
__device__ __forceinline__ void draw_accepts_queue2(uint32_t dmask0, const Planes &S0, uint32_t base0,
                                                    uint32_t dmask1, const Planes &S1, uint32_t base1,
                                                    const DrawKey &dk, const uint32_t (&rk)[2][8],
                                                    const uint64_t *thr, uint32_t *q, uint32_t &acc0,
                                                    uint32_t &acc1)
{
    acc0 = 0u;
    acc1 = 0u;
    if (!__any_sync(0xFFFFFFFFu, (dmask0 | dmask1) != 0u)) return;
    const int lane = (int)(threadIdx.x & 31);
    const int nd0 = __popc(dmask0), nd = nd0 + __popc(dmask1);
    int incl = nd;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    if (total > kDrawQueue2) {
        acc0 = draw_accepts(dmask0, S0, base0, dk, thr);
        acc1 = draw_accepts(dmask1, S1, base1, dk, thr);
        return;
    }
    uint4 *const planes = (uint4 *)q;                  // [2][32]
    uint32_t *const sites = (uint32_t *)(planes + 64);  // [2][32]
    uint32_t *const wacc = sites + 64;                  // [2][32]
    uint16_t *const ent = (uint16_t *)(wacc + 64);
    if (dmask0 != 0u) {
        planes[lane] = make_uint4(S0.s0, S0.s1, S0.s2, S0.s3);
        sites[lane] = base0;
    }
    if (dmask1 != 0u) {
        planes[32 + lane] = make_uint4(S1.s0, S1.s1, S1.s2, S1.s3);
        sites[32 + lane] = base1;
    }
    int slot = incl - nd;
    uint32_t dm = dmask0;
    while (dm != 0u) {
        const int p = __ffs(dm) - 1;
        dm &= dm - 1u;
        ent[slot++] = (uint16_t)(((uint32_t)lane << 5) | (uint32_t)p);
    }
    dm = dmask1;
    while (dm != 0u) {
        const int p = __ffs(dm) - 1;
        dm &= dm - 1u;
        ent[slot++] = (uint16_t)(1024u | ((uint32_t)lane << 5) | (uint32_t)p);
    }
    __syncwarp();
    // Rounds of 64 entries, lane i taking entries i and i + 32 (two Philox chains);
    // a last round of at most 32 entries takes one chain per lane.
    for (int k0 = 0; k0 < total; k0 += 64) {
        const int k = k0 + lane;
        if (total - k0 > 32) {
            const uint32_t e1 = ent[k];
            const bool two = k + 32 < total;
            const uint32_t e2 = two ? ent[k + 32] : e1;
            const uint32_t r1i = e1 >> 5, p1 = e1 & 31u, r2i = e2 >> 5, p2 = e2 & 31u;  // record = task*32 + lane
            uint32_t r1, r2;
            if (RK) philox2_w0_rk(sites[r1i] + p1, sites[r2i] + p2, dk, rk, r1, r2);
            else philox2_w0_key(sites[r1i] + p1, sites[r2i] + p2, dk, r1, r2);
            const uint4 a = planes[r1i], b = planes[r2i];
            const uint32_t Sa = ((a.x >> p1) & 1u) | (((a.y >> p1) & 1u) << 1) | (((a.z >> p1) & 1u) << 2) |
                                (((a.w >> p1) & 1u) << 3);
            const uint32_t Sb = ((b.x >> p2) & 1u) | (((b.y >> p2) & 1u) << 1) | (((b.z >> p2) & 1u) << 2) |
                                (((b.w >> p2) & 1u) << 3);
            if ((uint64_t)r1 < thr[Sa]) atomicOr(wacc + r1i, 1u << p1);
            if (two && (uint64_t)r2 < thr[Sb]) atomicOr(wacc + r2i, 1u << p2);
        } else if (k < total) {
            const uint32_t e1 = ent[k];
            const uint32_t r1i = e1 >> 5, p1 = e1 & 31u;
            const uint32_t r1 = RK ? philox_w0_rk(sites[r1i] + p1, dk, rk) : philox_w0_key(sites[r1i] + p1, dk);
            const uint4 a = planes[r1i];
            const uint32_t Sa = ((a.x >> p1) & 1u) | (((a.y >> p1) & 1u) << 1) | (((a.z >> p1) & 1u) << 2) |
                                (((a.w >> p1) & 1u) << 3);
            if ((uint64_t)r1 < thr[Sa]) atomicOr(wacc + r1i, 1u << p1);
        }
    }
    __syncwarp();
    acc0 = wacc[lane];
    acc1 = wacc[32 + lane];
    wacc[lane] = 0u;
    wacc[32 + lane] = 0u;
    __syncwarp();
}

// One padded shared-memory row from the device store (see the row layout above):
// word 0 holds position -1 (site Lx-1) in bit 31; words 1..W hold sites 0..Lx-1;
// positions Lx, Lx+1 hold sites 0, 1; every other pad bit is zero.
__device__ __forceinline__ uint32_t store_word(const void *lat, int packing, int pitch, int y, int w,
                                               int Lx)
{
    if (packing == kPackBit) return ((const uint32_t *)lat)[(size_t)y * pitch + w];
    const uint8_t *row = (const uint8_t *)lat + (size_t)y * pitch + 32 * w;
    const int n = min(32, Lx - 32 * w);
    uint32_t v = 0u;
    for (int b = 0; b < n; ++b) v |= (row[b] ? 1u : 0u) << b;
    return v;
}

__device__ __forceinline__ uint32_t padded_word(const void *lat, int packing, int pitch, int y,
                                                int w, int Lx, int W)
{
    const int P0 = 32 * w - 32;  // first position held by word w
    uint32_t v = 0u;
    if (w >= 1 && w <= W) {
        v = store_word(lat, packing, pitch, y, w - 1, Lx);
        const int nvalid = Lx - P0;
        if (nvalid < 32) v &= (1u << nvalid) - 1u;
    }
    if (w == 0) {
        const int xl = Lx - 1;
        v |= ((store_word(lat, packing, pitch, y, xl >> 5, Lx) >> (xl & 31)) & 1u) << 31;
    }
    const int q0 = Lx - P0;  // bit of position Lx in this word
    if (q0 >= -1 && q0 < 32) {
        const uint32_t s01 = store_word(lat, packing, pitch, y, 0, Lx) & 3u;  // sites 0, 1
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = q0 + e;
            if (q >= 0 && q < 32) v |= ((s01 >> e) & 1u) << q;
        }
    }
    return v;
}
