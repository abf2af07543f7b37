/*
 * klmc_oracle.c -- plain sequential CPU oracle for Kawasaki lattice Monte Carlo.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the CUDA
 * library is compared against, and the timed CPU baseline.  Only tests/, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code, header,
 * table or helper with the CUDA library (paper_1309_4349_gb300/csrc).
 *
 * Paper: M. Lis, L. Pintal, "GPU-Based Massive Parallel Kawasaki Kinetics in Monte
 * Carlo Modelling of Lipid Microdomains" (arXiv:1309.4349).
 *
 * What is computed, in the paper's order:
 *   - a binary A/B lipid lattice, one lipid per site, composition fixed
 *     (section "Monte Carlo model with Kawasaki based kinetics", Fig. 2);
 *   - energy omega_AB per unlike nearest-neighbour contact, the model's one
 *     parameter (same section, the omega_AB equation);
 *   - Metropolis-Hastings acceptance u < min{1, p(x*)/p(x)} with a symmetric
 *     Kawasaki nearest-neighbour exchange proposal (Metropolis steps a-c; Fig. 3A);
 *   - a parallel schedule in which each iteration picks a random decomposition and
 *     performs one exchange per domain (section "Massive Parallel Kawasaki
 *     Kinetics", MPKK loop), here as conflict-free shifted sublattice phases,
 *     eight per Monte Carlo step (one MCS = as many attempts as sites);
 *   - Hoshen-Kopelman style cluster statistics of one species
 *     (section "Cluster Analysis methods"), here by breadth-first search.
 *
 * Readings of the paper that this file fixes (each one is also listed in the
 * design notes of the repository):
 *   R1 geometry: triangular lattice with six neighbours (default) or square with
 *      four; periodic boundaries.
 *   R2 energy: E/kT = (omega/kT) * n_unlike.
 *   R3 acceptance: u = r / 2^32 with r a 32-bit Philox word; accept iff u < p,
 *      p = exp(-(omega/kT) * dn), i.e. r < ceil(p * 2^32).  Moves with
 *      (omega/kT)*dn <= 0 are accepted without a draw.
 *   R4 same-type pairs are attempts that change nothing and draw nothing.
 *   R5 initial placement: the n_A sites with the smallest (key_i, i), key_i a
 *      64-bit Philox value per site, are A (a uniformly random subset).
 *   R6 schedule: phase f of sweep s draws an orientation o and a shift (rx, ry);
 *      anchors form the (4,2) sublattice ((2,4) for o = (0,1)) shifted by
 *      (rx, ry); pairs {a, a+o}.  No site of one pair equals or neighbours a site
 *      of another pair of the same phase, so the phase result does not depend on
 *      the order of its anchors.
 *   R7 clusters: connected components under the lattice adjacency with the same
 *      periodic wrap; histogram of component sizes, sparse and ascending.
 *   R8 helical boundary (section "Massive Parallel Kawasaki Kinetics", Fig. 4
 *      and its caption on helical boundary conditions): site i's neighbours are
 *      (i + d) mod N for d in {+1, -1, +Lx, -Lx, -(Lx-1), +(Lx-1)} -- the axial
 *      offsets of R1 read as index steps, so the x wrap continues into the next
 *      row.  Triangular lattice only.
 *   R9 seven-colour schedule (the MPKK loop): coverage k has the domain centres
 *      i mod 7 = k; each centre with its six neighbours is one domain, and the
 *      domains tile the lattice iff 7 | N and Lx mod 7 is 3 or 5.  One MCS is
 *      seven iterations f = 0..6; iteration f of sweep s draws
 *      w = Philox(seed, {0xFFFFFFFF, f, s_lo, s_hi}), k = floor(w0 * 7 / 2^32)
 *      (with replacement, as the loop's k = rand%7) and one direction
 *      d = floor(w1 * 6 / 2^32) shared by all domains; every centre c attempts
 *      the exchange with c + D[d], draw counter {c, f, s_lo, s_hi}.  With one
 *      shared direction no pair touches another pair (centres are three steps
 *      apart), so the iteration does not depend on the order of its domains; a
 *      private direction per domain, as the loop's text allows, lets the pairs of
 *      adjacent domains neighbour each other.
 *   R12 fraction of first neighbours (section "Image analysis"): for every site
 *      one randomly chosen nearest neighbour; the count of sites whose chosen
 *      neighbour has the same type, divided by N.  In sample m the neighbour of
 *      site i is NB[floor(w * z / 2^32)], w = word (i mod 4) of
 *      Philox(seed, {i div 4, 0xFFFFFFFE, m_lo, m_hi}).  Its expectation is the
 *      all-bond fraction 1 - n_unlike / B, B = z N / 2.
 *   R13 snapshot images (section "Image analysis"): one pixel per site, row y
 *      shifted by half a site (the slope that keeps the triangular geometry):
 *      site (x, y) covers u in [2x + y, 2x + y + 2) half-sites and v in [y, y+1)
 *      rows, U = 2 Lx + Ly - 1 half-sites wide.  A W x H image samples each
 *      output pixel (i, j) on an S x S grid (supersampling): sample (a, b) sits
 *      at u = (2(iS + a) + 1) U / (2WS), v = (2(jS + b) + 1) Ly / (2HS), row
 *      y = floor(v), x = floor((u - y) / 2), inside iff 0 <= x < Lx; all in
 *      integers.  The pixel belongs to the lattice iff at least half its samples
 *      are inside; its gray level is round(255 nA / n_in) (A white, B black,
 *      halves up).  The image's fraction of first neighbours (sample m): every
 *      lattice pixel p = jW + i chooses one of its eight neighbours, direction
 *      floor(w * 8 / 2^32) of (1,0), (1,1), (0,1), (-1,1), (-1,0), (-1,-1),
 *      (0,-1), (1,-1), w = word (p mod 4) of Philox(seed, {p div 4, 0xFFFFFFFC,
 *      m_lo, m_hi}); it is similar iff that neighbour is a lattice pixel of the
 *      image whose gray level differs by at most delta (35 in the paper).
 *   R14 average cluster size (section "Cluster Analysis" results, which plot
 *      the average cluster size without naming the average): both the number
 *      average sum s c / sum c and the weight average sum s^2 c / sum s c of the
 *      sparse histogram, each one FP64 division of exact int64 sums; 0 when the
 *      species has no site.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_TRI6 0
#define ORC_SQ4 1

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator.                                     */
/* Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", */
/* SC'11: four 32-bit counter words, two key words, ten rounds; each round     */
/* multiplies two words by fixed constants, mixes the high halves with the     */
/* other words and the key, and the key is bumped by two Weyl constants.      */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(prod1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)prod1;
        uint32_t y2 = (uint32_t)(prod0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)prod0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void seed_key(uint64_t seed, uint32_t key[2])
{
    key[0] = (uint32_t)seed;
    key[1] = (uint32_t)(seed >> 32);
}

/* ------------------------------------------------------------------------- */
/* Geometry (R1).  Site (x, y) has index y*Lx + x.                            */
/* ------------------------------------------------------------------------- */
static const int TRI6_NB[6][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, -1}, {-1, 1}};
static const int SQ4_NB[4][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}};
/* Bond orientations: every bond is {i, i+o} for exactly one site i and o in O. */
static const int TRI6_O[3][2] = {{1, 0}, {0, 1}, {1, -1}};
static const int SQ4_O[2][2] = {{1, 0}, {0, 1}};

int orc_coordination(int geometry) { return geometry == ORC_TRI6 ? 6 : 4; }
int orc_n_orientations(int geometry) { return geometry == ORC_TRI6 ? 3 : 2; }

static const int (*nb_table(int geometry))[2] { return geometry == ORC_TRI6 ? TRI6_NB : SQ4_NB; }
static const int (*o_table(int geometry))[2] { return geometry == ORC_TRI6 ? TRI6_O : SQ4_O; }

static int64_t wrap(int64_t v, int64_t n)
{
    int64_t r = v % n;
    return r < 0 ? r + n : r;
}

static int64_t site_of(int Lx, int Ly, int64_t x, int64_t y)
{
    return wrap(y, Ly) * (int64_t)Lx + wrap(x, Lx);
}

#define ORC_PERIODIC 0
#define ORC_HELICAL 1

/* Index of the neighbour of site i in direction (dx, dy): periodic wrap of x and
 * y (R1), or the helical index step dx + dy*Lx modulo N (R8). */
static int64_t neighbour_b(int Lx, int Ly, int boundary, int64_t i, int dx, int dy)
{
    if (boundary == ORC_HELICAL) return wrap(i + dx + (int64_t)dy * Lx, (int64_t)Lx * Ly);
    int64_t x = i % Lx, y = i / Lx;
    return site_of(Lx, Ly, x + dx, y + dy);
}

static int64_t neighbour(int Lx, int Ly, int64_t i, int dx, int dy)
{
    return neighbour_b(Lx, Ly, ORC_PERIODIC, i, dx, dy);
}

/* ------------------------------------------------------------------------- */
/* Energy (R2): number of unlike nearest-neighbour bonds, every bond once.     */
/* ------------------------------------------------------------------------- */
int64_t orc_n_unlike_b(int Lx, int Ly, int geometry, int boundary, const uint8_t *t)
{
    const int (*O)[2] = o_table(geometry);
    int nO = orc_n_orientations(geometry);
    int64_t N = (int64_t)Lx * Ly, n = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int k = 0; k < nO; ++k)
            n += (t[i] != t[neighbour_b(Lx, Ly, boundary, i, O[k][0], O[k][1])]);
    return n;
}

int64_t orc_n_unlike(int Lx, int Ly, int geometry, const uint8_t *t)
{
    return orc_n_unlike_b(Lx, Ly, geometry, ORC_PERIODIC, t);
}

/* ------------------------------------------------------------------------- */
/* Acceptance threshold (R3), built once per run in FP64.                     */
/* For an energy change dn: always = 1 when (omega/kT)*dn <= 0 (no draw);     */
/* otherwise thr = ceil(exp(-(omega/kT)*dn) * 2^32) and a draw r is accepted  */
/* iff r < thr.                                                               */
/* ------------------------------------------------------------------------- */
void orc_threshold(double bw, int dn, int *always, uint64_t *thr)
{
    double x = bw * (double)dn;
    if (x <= 0.0) {
        *always = 1;
        *thr = (uint64_t)1 << 32;
        return;
    }
    double p = exp(-x);
    *always = 0;
    *thr = (uint64_t)ceil(ldexp(p, 32));
}

/* ------------------------------------------------------------------------- */
/* Initial placement (R5).                                                    */
/* ------------------------------------------------------------------------- */
int64_t orc_n_A(int Lx, int Ly, int64_t nA_param, double fraction)
{
    int64_t N = (int64_t)Lx * Ly;
    if (nA_param >= 0) return nA_param;
    return (int64_t)floor(fraction * (double)N + 0.5);
}

typedef struct {
    uint64_t key;
    int64_t site;
} orc_keyed_site;

static int cmp_keyed_site(const void *pa, const void *pb)
{
    const orc_keyed_site *a = (const orc_keyed_site *)pa, *b = (const orc_keyed_site *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->site != b->site) return a->site < b->site ? -1 : 1;
    return 0;
}

/* Placement key of site i: Philox(seed, {i, 0xFFFFFFFF, 0, 0}), words w1:w0. */
uint64_t orc_site_key(uint64_t seed, int64_t i)
{
    uint32_t key[2], ctr[4] = {(uint32_t)i, 0xFFFFFFFFu, 0u, 0u}, w[4];
    seed_key(seed, key);
    orc_philox4x32_10(ctr, key, w);
    return ((uint64_t)w[1] << 32) | (uint64_t)w[0];
}

/* t[i] = 1 (A) for the nA sites with the smallest (key_i, i), else 0 (B). */
int orc_init(int Lx, int Ly, int64_t nA, uint64_t seed, uint8_t *t)
{
    int64_t N = (int64_t)Lx * Ly;
    if (nA < 0 || nA > N) return -1;
    orc_keyed_site *ks = (orc_keyed_site *)malloc((size_t)N * sizeof(orc_keyed_site));
    if (!ks) return -2;
    for (int64_t i = 0; i < N; ++i) {
        ks[i].key = orc_site_key(seed, i);
        ks[i].site = i;
    }
    qsort(ks, (size_t)N, sizeof(orc_keyed_site), cmp_keyed_site);
    memset(t, 0, (size_t)N);
    for (int64_t r = 0; r < nA; ++r) t[ks[r].site] = 1;
    free(ks);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Phase schedule (R6).                                                       */
/* ------------------------------------------------------------------------- */
void orc_phase_params(int Lx, int Ly, int geometry, uint64_t seed, int64_t sweep, int phase,
                      int *o_index, int *rx, int *ry)
{
    uint32_t key[2], w[4];
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)phase, (uint32_t)(uint64_t)sweep,
                       (uint32_t)((uint64_t)sweep >> 32)};
    seed_key(seed, key);
    orc_philox4x32_10(ctr, key, w);
    *o_index = (int)(((uint64_t)w[0] * (uint64_t)orc_n_orientations(geometry)) >> 32);
    *rx = (int)(((uint64_t)w[1] * (uint64_t)Lx) >> 32);
    *ry = (int)(((uint64_t)w[2] * (uint64_t)Ly) >> 32);
}

/* Sublattice periods and counts for orientation (ox, oy). */
static void phase_grid(int Lx, int Ly, int ox, int oy, int *px, int *py, int *Kx, int *My)
{
    if (ox == 0 && oy == 1) {
        *px = 2; *py = 4;
        *Kx = (Lx - 2) / 2 + 1;
        *My = (Ly - 3) / 4 + 1;
    } else {
        *px = 4; *py = 2;
        *Kx = (Lx - 3) / 4 + 1;
        *My = (Ly - 2) / 2 + 1;
    }
}

/* Anchor sites of a phase, in schedule order (row-major over (m, k)).
 * Writes at most cap anchors; returns the number of anchors. */
int64_t orc_phase_anchors(int Lx, int Ly, int geometry, int o_index, int rx, int ry,
                          int64_t *anchors, int64_t cap)
{
    const int (*O)[2] = o_table(geometry);
    int px, py, Kx, My;
    phase_grid(Lx, Ly, O[o_index][0], O[o_index][1], &px, &py, &Kx, &My);
    int64_t n = 0;
    for (int m = 0; m < My; ++m)
        for (int k = 0; k < Kx; ++k) {
            if (n < cap) anchors[n] = site_of(Lx, Ly, (int64_t)rx + (int64_t)px * k,
                                              (int64_t)ry + (int64_t)py * m);
            ++n;
        }
    return n;
}

/* ------------------------------------------------------------------------- */
/* One Kawasaki exchange attempt (Metropolis steps a-c on one pair).          */
/* ------------------------------------------------------------------------- */

/* Unlike bonds incident to a or b; the bond a-b itself is counted once. */
static int local_unlike_b(int Lx, int Ly, int geometry, int boundary, const uint8_t *t, int64_t a,
                          int64_t b)
{
    const int (*NB)[2] = nb_table(geometry);
    int z = orc_coordination(geometry), n = 0;
    for (int k = 0; k < z; ++k) {
        int64_t c = neighbour_b(Lx, Ly, boundary, a, NB[k][0], NB[k][1]);
        n += (t[a] != t[c]);
    }
    for (int k = 0; k < z; ++k) {
        int64_t c = neighbour_b(Lx, Ly, boundary, b, NB[k][0], NB[k][1]);
        if (c == a) continue;
        n += (t[b] != t[c]);
    }
    return n;
}

static int local_unlike(int Lx, int Ly, int geometry, const uint8_t *t, int64_t a, int64_t b)
{
    return local_unlike_b(Lx, Ly, geometry, ORC_PERIODIC, t, a, b);
}

typedef struct {
    int64_t attempts, unlike, draws, accepts;
} orc_counters;

typedef struct {
    int always[32];
    uint64_t thr[32];
    int dn_offset;
} orc_table;

static void build_table(double bw, int geometry, orc_table *tab)
{
    int z = orc_coordination(geometry);
    tab->dn_offset = 2 * (z - 1);
    for (int dn = -2 * (z - 1); dn <= 2 * (z - 1); ++dn)
        orc_threshold(bw, dn, &tab->always[dn + tab->dn_offset], &tab->thr[dn + tab->dn_offset]);
}

static void exchange_attempt(int Lx, int Ly, int geometry, int boundary, const orc_table *tab,
                             const uint32_t key[2], int64_t sweep, int phase, uint8_t *t,
                             int64_t a, int64_t b, int64_t *n_unlike, orc_counters *cnt)
{
    cnt->attempts += 1;
    if (t[a] == t[b]) return; /* R4: the candidate state equals the current one */
    cnt->unlike += 1;
    /* a. candidate state x*: the lattice with a and b exchanged */
    int before = local_unlike_b(Lx, Ly, geometry, boundary, t, a, b);
    uint8_t ta = t[a];
    t[a] = t[b];
    t[b] = ta;
    int after = local_unlike_b(Lx, Ly, geometry, boundary, t, a, b);
    int dn = after - before;
    /* b.-c. u ~ U[0,1) from a 32-bit draw, accept iff u < min{1, exp(-bw*dn)} */
    int accept;
    if (tab->always[dn + tab->dn_offset]) {
        accept = 1;
    } else {
        uint32_t ctr[4] = {(uint32_t)a, (uint32_t)phase, (uint32_t)(uint64_t)sweep,
                           (uint32_t)((uint64_t)sweep >> 32)};
        uint32_t w[4];
        orc_philox4x32_10(ctr, key, w);
        cnt->draws += 1;
        accept = ((uint64_t)w[0] < tab->thr[dn + tab->dn_offset]);
    }
    if (accept) {
        cnt->accepts += 1;
        *n_unlike += dn;
    } else {
        t[b] = t[a];
        t[a] = ta;
    }
}

/* ------------------------------------------------------------------------- */
/* Sweeps.                                                                    */
/*   t        in/out lattice, one byte per site, 1 = A                         */
/*   sweep0   absolute index of the first sweep (RNG counter)                  */
/*   counters in/out [attempts, unlike, draws, accepts]                        */
/*   n_unlike in/out running energy                                            */
/*   trace    if trace_every > 0, n_unlike after every trace_every-th sweep     */
/*   flags    bit 0: recompute n_unlike from scratch after every phase;        */
/*            bit 1: visit each phase's anchors in reverse order (the result    */
/*            must not change, since the pairs of a phase do not interact)     */
/* Returns 0, or -1 when the incremental energy disagrees with a recount.     */
/* ------------------------------------------------------------------------- */
int orc_run(int Lx, int Ly, int geometry, double bw, uint64_t seed, uint8_t *t, int64_t sweep0,
            int64_t n_mcs, int64_t *n_unlike, int64_t counters[4], int64_t trace_every,
            int64_t *trace, int flags)
{
    const int (*O)[2] = o_table(geometry);
    orc_table tab;
    uint32_t key[2];
    orc_counters cnt = {counters[0], counters[1], counters[2], counters[3]};
    build_table(bw, geometry, &tab);
    seed_key(seed, key);
    for (int64_t s = sweep0; s < sweep0 + n_mcs; ++s) {
        for (int f = 0; f < 8; ++f) {
            int oi, rx, ry, px, py, Kx, My;
            orc_phase_params(Lx, Ly, geometry, seed, s, f, &oi, &rx, &ry);
            int ox = O[oi][0], oy = O[oi][1];
            phase_grid(Lx, Ly, ox, oy, &px, &py, &Kx, &My);
            for (int mm = 0; mm < My; ++mm)
                for (int kk = 0; kk < Kx; ++kk) {
                    int m = (flags & 2) ? My - 1 - mm : mm;
                    int k = (flags & 2) ? Kx - 1 - kk : kk;
                    int64_t ax = (int64_t)rx + (int64_t)px * k, ay = (int64_t)ry + (int64_t)py * m;
                    int64_t a = site_of(Lx, Ly, ax, ay);
                    int64_t b = site_of(Lx, Ly, ax + ox, ay + oy);
                    exchange_attempt(Lx, Ly, geometry, ORC_PERIODIC, &tab, key, s, f, t, a, b, n_unlike,
                                     &cnt);
                }
            if ((flags & 1) && *n_unlike != orc_n_unlike(Lx, Ly, geometry, t)) return -1;
        }
        int64_t done = s + 1 - sweep0;
        if (trace_every > 0 && done % trace_every == 0) trace[done / trace_every - 1] = *n_unlike;
    }
    counters[0] = cnt.attempts;
    counters[1] = cnt.unlike;
    counters[2] = cnt.draws;
    counters[3] = cnt.accepts;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Helical lattice with the seven-colour schedule (R8, R9).                   */
/* ------------------------------------------------------------------------- */

/* Whether the seven coverages tile the helical Lx x Ly lattice (R9). */
int orc_helical_valid(int Lx, int Ly)
{
    int64_t N = (int64_t)Lx * Ly;
    return Lx >= 4 && Ly >= 4 && N % 7 == 0 && (Lx % 7 == 3 || Lx % 7 == 5);
}

/* Coverage k and shared direction index d of iteration f of sweep s. */
void orc_mpkk_params(uint64_t seed, int64_t sweep, int phase, int *k, int *d)
{
    uint32_t key[2], w[4];
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)phase, (uint32_t)(uint64_t)sweep,
                       (uint32_t)((uint64_t)sweep >> 32)};
    seed_key(seed, key);
    orc_philox4x32_10(ctr, key, w);
    *k = (int)(((uint64_t)w[0] * 7u) >> 32);
    *d = (int)(((uint64_t)w[1] * 6u) >> 32);
}

/* Sweeps of the seven-colour schedule on the helical triangular lattice, same
 * arguments and flags as orc_run.  Returns -2 for a size the coverages do not
 * tile. */
int orc_run_mpkk(int Lx, int Ly, double bw, uint64_t seed, uint8_t *t, int64_t sweep0, int64_t n_mcs,
                 int64_t *n_unlike, int64_t counters[4], int64_t trace_every, int64_t *trace, int flags)
{
    if (!orc_helical_valid(Lx, Ly)) return -2;
    const int64_t N = (int64_t)Lx * Ly;
    orc_table tab;
    uint32_t key[2];
    orc_counters cnt = {counters[0], counters[1], counters[2], counters[3]};
    build_table(bw, ORC_TRI6, &tab);
    seed_key(seed, key);
    for (int64_t s = sweep0; s < sweep0 + n_mcs; ++s) {
        for (int f = 0; f < 7; ++f) {
            int k, d;
            orc_mpkk_params(seed, s, f, &k, &d);
            const int dx = TRI6_NB[d][0], dy = TRI6_NB[d][1];
            const int64_t n_centres = N / 7;
            for (int64_t q = 0; q < n_centres; ++q) {
                int64_t m = (flags & 2) ? n_centres - 1 - q : q;
                int64_t c = (int64_t)k + 7 * m;
                int64_t b = neighbour_b(Lx, Ly, ORC_HELICAL, c, dx, dy);
                exchange_attempt(Lx, Ly, ORC_TRI6, ORC_HELICAL, &tab, key, s, f, t, c, b, n_unlike, &cnt);
            }
            if ((flags & 1) && *n_unlike != orc_n_unlike_b(Lx, Ly, ORC_TRI6, ORC_HELICAL, t)) return -1;
        }
        int64_t done = s + 1 - sweep0;
        if (trace_every > 0 && done % trace_every == 0) trace[done / trace_every - 1] = *n_unlike;
    }
    counters[0] = cnt.attempts;
    counters[1] = cnt.unlike;
    counters[2] = cnt.draws;
    counters[3] = cnt.accepts;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Fraction of first neighbours (R12).                                        */
/* ------------------------------------------------------------------------- */

/* Number of sites whose randomly chosen nearest neighbour (sample m) has the same
 * type; the paper's fraction is this count divided by N. */
int64_t orc_ffn_count(int Lx, int Ly, int geometry, int boundary, const uint8_t *t, uint64_t seed,
                      int64_t sample)
{
    const int (*NB)[2] = nb_table(geometry);
    const int z = orc_coordination(geometry);
    const int64_t N = (int64_t)Lx * Ly;
    uint32_t key[2], w[4];
    seed_key(seed, key);
    int64_t similar = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (i % 4 == 0) {
            uint32_t ctr[4] = {(uint32_t)(i / 4), 0xFFFFFFFEu, (uint32_t)(uint64_t)sample,
                               (uint32_t)((uint64_t)sample >> 32)};
            orc_philox4x32_10(ctr, key, w);
        }
        int k = (int)(((uint64_t)w[i % 4] * (uint64_t)z) >> 32);
        int64_t j = neighbour_b(Lx, Ly, boundary, i, NB[k][0], NB[k][1]);
        similar += (t[i] == t[j]);
    }
    return similar;
}

/* ------------------------------------------------------------------------- */
/* Snapshot images and their fraction of first neighbours (R13).              */
/* ------------------------------------------------------------------------- */

static int64_t floor_div64(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

/* Gray level (0..255) and lattice membership (0/1) of every pixel, j-major. */
int orc_snapshot(int Lx, int Ly, const uint8_t *t, int W, int H, int S, uint8_t *image, uint8_t *mask)
{
    if (W < 1 || H < 1 || S < 1 || S > 64) return -1;
    const int64_t U = 2 * (int64_t)Lx + Ly - 1, D = 2 * (int64_t)W * S;
    if (2.0 * W * S * (U > Ly ? U : Ly) > 4.0e18 || 2.0 * H * S * (double)Ly > 4.0e18) return -1;
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            int64_t n_in = 0, n_A = 0;
            for (int b = 0; b < S; ++b) {
                const int64_t y = (2 * ((int64_t)j * S + b) + 1) * (int64_t)Ly / (2 * (int64_t)H * S);
                for (int a = 0; a < S; ++a) {
                    const int64_t un = (2 * ((int64_t)i * S + a) + 1) * U;  /* u = un / D */
                    const int64_t x = floor_div64(un - y * D, 2 * D);
                    if (x < 0 || x >= Lx) continue;
                    n_in += 1;
                    n_A += t[y * Lx + x];
                }
            }
            const int64_t p = (int64_t)j * W + i;
            mask[p] = (uint8_t)(2 * n_in >= (int64_t)S * S);
            image[p] = n_in > 0 ? (uint8_t)((510 * n_A + n_in) / (2 * n_in)) : 0;
        }
    return 0;
}

/* Similar pixels of sample m, and (pixels) the lattice pixels of the image. */
int64_t orc_image_ffn(const uint8_t *image, const uint8_t *mask, int W, int H, int delta, uint64_t seed,
                      int64_t sample, int64_t *pixels)
{
    static const int DI[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    static const int DJ[8] = {0, 1, 1, 1, 0, -1, -1, -1};
    uint32_t key[2], w[4];
    seed_key(seed, key);
    int64_t similar = 0, n = 0;
    const int64_t P = (int64_t)W * H;
    for (int64_t p = 0; p < P; ++p) {
        if (p % 4 == 0) {
            uint32_t ctr[4] = {(uint32_t)(p / 4), 0xFFFFFFFCu, (uint32_t)(uint64_t)sample,
                               (uint32_t)((uint64_t)sample >> 32)};
            orc_philox4x32_10(ctr, key, w);
        }
        if (!mask[p]) continue;
        n += 1;
        const int k = (int)(((uint64_t)w[p % 4] * 8u) >> 32);
        const int64_t i = p % W + DI[k], j = p / W + DJ[k];
        if (i < 0 || i >= W || j < 0 || j >= H) continue;
        const int64_t q = j * W + i;
        if (!mask[q]) continue;
        const int d = (int)image[p] - (int)image[q];
        similar += (d <= delta && -d <= delta);
    }
    if (pixels) *pixels = n;
    return similar;
}

/* ------------------------------------------------------------------------- */
/* Cluster statistics (R7).                                                   */
/* ------------------------------------------------------------------------- */

/* labels[i] = smallest site index of i's component if t[i] == species, else -1.
 * Breadth-first search started from sites in ascending order, so the first site
 * reached of every component is its smallest index.  Returns the number of
 * components. */
int64_t orc_cluster_labels_b(int Lx, int Ly, int geometry, int boundary, const uint8_t *t, int species,
                             int64_t *labels)
{
    const int (*NB)[2] = nb_table(geometry);
    int z = orc_coordination(geometry);
    int64_t N = (int64_t)Lx * Ly, n_comp = 0;
    int64_t *queue = (int64_t *)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    if (!queue) return -1;
    for (int64_t i = 0; i < N; ++i) labels[i] = -1;
    for (int64_t i = 0; i < N; ++i) {
        if (t[i] != species || labels[i] != -1) continue;
        int64_t head = 0, tail = 0;
        labels[i] = i;
        queue[tail++] = i;
        while (head < tail) {
            int64_t c = queue[head++];
            for (int k = 0; k < z; ++k) {
                int64_t d = neighbour_b(Lx, Ly, boundary, c, NB[k][0], NB[k][1]);
                if (t[d] == species && labels[d] == -1) {
                    labels[d] = i;
                    queue[tail++] = d;
                }
            }
        }
        ++n_comp;
    }
    free(queue);
    return n_comp;
}

int64_t orc_cluster_labels(int Lx, int Ly, int geometry, const uint8_t *t, int species, int64_t *labels)
{
    return orc_cluster_labels_b(Lx, Ly, geometry, ORC_PERIODIC, t, species, labels);
}

/* Sparse cluster-size histogram, ascending in size.  Writes at most capacity
 * (size, count) pairs and returns the number of distinct sizes (which may
 * exceed capacity), or -1 on allocation failure. */
int64_t orc_cluster_histogram_b(int Lx, int Ly, int geometry, int boundary, const uint8_t *t, int species,
                                int64_t *sizes, int64_t *counts, int64_t capacity)
{
    int64_t N = (int64_t)Lx * Ly;
    int64_t *labels = (int64_t *)malloc((size_t)N * sizeof(int64_t));
    int64_t *comp_size = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    int64_t *hist = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    if (!labels || !comp_size || !hist) {
        free(labels); free(comp_size); free(hist);
        return -1;
    }
    orc_cluster_labels_b(Lx, Ly, geometry, boundary, t, species, labels);
    for (int64_t i = 0; i < N; ++i)
        if (labels[i] >= 0) comp_size[labels[i]] += 1;
    for (int64_t i = 0; i < N; ++i)
        if (comp_size[i] > 0) hist[comp_size[i]] += 1;
    int64_t n = 0;
    for (int64_t s = 1; s <= N; ++s)
        if (hist[s] > 0) {
            if (n < capacity) {
                sizes[n] = s;
                counts[n] = hist[s];
            }
            ++n;
        }
    free(labels); free(comp_size); free(hist);
    return n;
}

int64_t orc_cluster_histogram(int Lx, int Ly, int geometry, const uint8_t *t, int species,
                              int64_t *sizes, int64_t *counts, int64_t capacity)
{
    return orc_cluster_histogram_b(Lx, Ly, geometry, ORC_PERIODIC, t, species, sizes, counts, capacity);
}

/* Average cluster size (section "Cluster Analysis" results: the average size of
 * the clusters over time) from a sparse histogram of n (size s_k, count c_k)
 * pairs.  The three sums are exact integers; each average is one FP64 division
 * of two of them:
 *   number average <s>_n = sum_k s_k c_k   / sum_k c_k
 *   weight average <s>_w = sum_k s_k^2 c_k / sum_k s_k c_k
 * R14: both are 0 for an empty histogram (no site of the species).  Returns 0,
 * -1 for a negative size or count, -2 when a sum would leave int64. */
int orc_cluster_averages(const int64_t *sizes, const int64_t *counts, int64_t n, double *number_avg,
                         double *weight_avg)
{
    int64_t n_clusters = 0, n_sites = 0, sum_sq = 0;
    for (int64_t k = 0; k < n; ++k) {
        int64_t s = sizes[k], c = counts[k];
        if (s < 0 || c < 0) return -1;
        if (s > 0 && c > INT64_MAX / s) return -2;
        int64_t sc = s * c;
        if (s > 0 && sc > INT64_MAX / s) return -2;
        int64_t ssc = sc * s;
        if (n_clusters > INT64_MAX - c || n_sites > INT64_MAX - sc || sum_sq > INT64_MAX - ssc) return -2;
        n_clusters += c;
        n_sites += sc;
        sum_sq += ssc;
    }
    *number_avg = n_clusters > 0 ? (double)n_sites / (double)n_clusters : 0.0;
    *weight_avg = n_sites > 0 ? (double)sum_sq / (double)n_sites : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Classical random-sequential Kawasaki (the paper's CPU comparison method,   */
/* Fig. 5B): per attempt a uniformly random site and a uniformly random one   */
/* of its neighbours, FP64 Metropolis acceptance with u = r / 2^32.  Used     */
/* only for statistical comparison; it draws from its own Philox stream       */
/* (counter word 2 = 0xFFFFFFFD) and shares nothing with the phase schedule.  */
/* ------------------------------------------------------------------------- */
int orc_run_random_sequential(int Lx, int Ly, int geometry, double bw, uint64_t seed,
                              uint8_t *t, int64_t attempt0, int64_t n_attempts,
                              int64_t *n_unlike, int64_t *accepts)
{
    const int (*NB)[2] = nb_table(geometry);
    int z = orc_coordination(geometry);
    int64_t N = (int64_t)Lx * Ly;
    uint32_t key[2];
    seed_key(seed, key);
    for (int64_t n = attempt0; n < attempt0 + n_attempts; ++n) {
        uint32_t ctr[4] = {(uint32_t)(uint64_t)n, (uint32_t)((uint64_t)n >> 32), 0xFFFFFFFDu, 0u},
                 w[4];
        orc_philox4x32_10(ctr, key, w);
        int64_t a = (int64_t)(((uint64_t)w[0] * (uint64_t)N) >> 32);
        int k = (int)(((uint64_t)w[1] * (uint64_t)z) >> 32);
        int64_t b = neighbour(Lx, Ly, a, NB[k][0], NB[k][1]);
        if (t[a] == t[b]) continue;
        int before = local_unlike(Lx, Ly, geometry, t, a, b);
        uint8_t ta = t[a];
        t[a] = t[b];
        t[b] = ta;
        int after = local_unlike(Lx, Ly, geometry, t, a, b);
        int dn = after - before;
        double p = exp(-bw * (double)dn);
        double u = ldexp((double)w[2], -32);
        if (u < p) {
            *n_unlike += dn;
            *accepts += 1;
        } else {
            t[b] = t[a];
            t[a] = ta;
        }
    }
    return 0;
}
