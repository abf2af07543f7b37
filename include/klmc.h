/*
 * klmc.h -- C ABI of the GB300 Kawasaki lattice Monte Carlo library (libklmc.so).
 *
 * The library simulates the paper's model: M. Lis, L. Pintal, "GPU-Based Massive
 * Parallel Kawasaki Kinetics in Monte Carlo Modelling of Lipid Microdomains"
 * (arXiv:1309.4349).  A two-component (A/B) lipid lattice, one lipid per site,
 * evolves by Metropolis-accepted nearest-neighbour exchanges (Kawasaki kinetics)
 * with energy omega per unlike contact, and is analysed by cluster-size
 * statistics of one lipid species.
 *
 * Conventions for every call:
 *  - Every call returns a klmc_status; nothing is thrown across the ABI.  On
 *    error, out-parameters are left untouched unless a call states otherwise,
 *    and klmc_last_error() returns a message for the calling thread.
 *  - Device memory is owned by the library and freed by klmc_destroy /
 *    klmc_batch_destroy.  Host buffers, device buffers passed in by the caller,
 *    the caller's allocator and the caller's stream stay owned by the caller.
 *  - Work is enqueued on the handle's CUDA stream.  Calls that return data in
 *    host memory synchronise that stream first; the others return after enqueue.
 *  - A handle is used by one host thread at a time.
 *  - Lattice layout seen by the caller: one byte per site, 1 = A, 0 = B,
 *    site (x, y) at index y*Lx + x.  Geometry: triangular (six neighbours
 *    (+-1,0), (0,+-1), (1,-1), (-1,1)) or square (four), periodic in x and y.
 */
#ifndef KLMC_H
#define KLMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum klmc_status {
    KLMC_OK = 0,
    KLMC_EINVAL = 1,   /* invalid argument                                   */
    KLMC_ENOMEM = 2,   /* device or host allocation failed                   */
    KLMC_ECUDA = 3,    /* a CUDA runtime call failed                         */
    KLMC_ETIMEOUT = 4, /* a bounded device-side wait gave up                 */
    KLMC_EBUSY = 5,    /* not admitted now, or a result is still pending     */
    KLMC_ETRUNC = 6,   /* output capacity too small; needed length reported  */
    KLMC_ESTATE = 7,   /* call not valid for this handle in its state        */
    KLMC_ENODEV = 8    /* no usable CUDA device of compute capability 10.3   */
} klmc_status;

enum { KLMC_TRI6 = 0, KLMC_SQ4 = 1 };                 /* geometry  */
enum { KLMC_PERIODIC = 0, KLMC_HELICAL = 1 };        /* boundary  */
enum { KLMC_PACK_AUTO = 0, KLMC_PACK_BIT = 1, KLMC_PACK_BYTE = 2 }; /* device store */

/* Caller-supplied device allocator (e.g. a framework's caching allocator).
 * alloc returns NULL on failure; free receives the size passed to alloc. */
typedef void *(*klmc_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*klmc_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Model and storage parameters (section "Monte Carlo model with Kawasaki based
 * kinetics": lattice, binary composition, the single parameter omega_AB). */
typedef struct klmc_params {
    int32_t Lx, Ly;        /* lattice sides, each >= 4; Lx*Ly <= 2^31 - 1        */
    int32_t geometry;      /* KLMC_TRI6 (the paper's lattice) or KLMC_SQ4        */
    int32_t boundary;      /* KLMC_PERIODIC (conflict-free shifted sublattice
                              phases, 8 per step), or KLMC_HELICAL: the paper's
                              helical triangular lattice (section "Massive
                              Parallel Kawasaki Kinetics", Fig. 4) with its
                              seven-colour MPKK schedule -- neighbours of site i
                              are (i + dx + dy*Lx) mod N for the six axial steps;
                              the domains (a site i with i mod 7 = k and its six
                              neighbours) tile the lattice, which requires TRI6,
                              7 | Lx*Ly and Lx mod 7 in {3, 5} (else EINVAL);
                              each step is 7 iterations, each drawing k in 0..6
                              and one direction for all domains.  Lattices whose
                              bands over a cluster of CTAs hold the halo rows of
                              blocks of iterations run resident in the cluster's
                              shared memory (512 threads per CTA; in handles,
                              batches and the server); smaller ones run one
                              launch per iteration over the device store (cluster
                              -1; handles only)                                   */
    int32_t packing;       /* device store: KLMC_PACK_BIT (1 bit/site), _BYTE, or
                              _AUTO (= BIT)                                       */
    int32_t cluster;       /* CTAs that share one lattice in the resident sweep
                              (a thread-block cluster, 1..16); -1 = tiled per-phase
                              path; 0 = automatic                                 */
    int32_t threads;       /* threads per CTA of the resident sweep: 128, 256 or
                              512; 0 = automatic                                  */
    int32_t reserved0;
    int64_t n_A;           /* number of A lipids; -1 = floor(fraction_A*N + 0.5)  */
    double fraction_A;     /* used when n_A < 0; in [0, 1]                        */
    double omega_over_kT;  /* omega_AB / kT, finite; E/kT = omega/kT * n_unlike   */
    uint64_t seed;         /* keys every random number of the run (Philox key)   */
    klmc_alloc_fn alloc;   /* NULL = stream-ordered cudaMallocAsync               */
    klmc_free_fn free;     /* required when alloc is set                          */
    void *user;            /* passed to alloc/free                                */
    void *stream;          /* cudaStream_t for all work; NULL = default stream    */
} klmc_params;

/* Exact integer counters since creation (or the last klmc_set_lattice).
 * attempts: pair proposals; unlike: proposals of an A-B pair; draws: random
 * numbers drawn (only for moves that raise the energy when omega > 0);
 * accepts: accepted exchanges.  sweeps is the absolute sweep index. */
typedef struct klmc_counters {
    int64_t sweeps, attempts, unlike, draws, accepts;
} klmc_counters;

typedef struct klmc_ctx klmc_ctx;
typedef struct klmc_batch klmc_batch;

/* Fills p with defaults: 64x64 TRI6 periodic, bit store, n_A = -1,
 * fraction 0.5, omega/kT 0, seed 1, library allocator, default stream. */
klmc_status klmc_params_default(klmc_params *p);

/* Creates an L x L triangular lattice with floor(composition_A*L*L + 0.5) A lipids
 * placed uniformly at random from seed (Fig. 2: randomly distributed lipids).
 * Equivalent to klmc_create_ex with defaults otherwise. */
klmc_status klmc_create(klmc_ctx **out, int32_t L, double composition_A, double omega_over_kT,
                        uint64_t seed);

/* Creates a lattice from full parameters.  The initial placement makes the
 * n_A sites with the smallest 64-bit Philox keys (ties by site index) A, which
 * is a uniformly random subset.  EINVAL on Lx or Ly < 4, N > 2^31 - 1, n_A
 * outside [0, N], fraction outside [0, 1], non-finite omega, or an unknown
 * geometry/boundary/packing; ENODEV without a compute-capability-10.3 GPU. */
klmc_status klmc_create_ex(klmc_ctx **out, const klmc_params *p);

/* Enqueues n_mcs Monte Carlo steps (n_mcs >= 0).  One step is eight conflict-free
 * phases of exchange attempts, N attempts when 4 | Lx and 4 | Ly (section
 * "Massive Parallel Kawasaki Kinetics": one MPKK step = as many attempts as
 * sites).  Deterministic: the result depends only on seed, the lattice and the
 * absolute sweep index, not on the cluster size.  With the automatic launch shape
 * (cluster = 0) a lattice of at least 786432 sites (where the tiled path measured
 * faster) or too large for one thread-block cluster's shared memory runs on the
 * tiled path (replicas of a batch and jobs of a server stay resident): bands of
 * rows, one CTA each, four phases per launch,
 * rows of a bit store on 16-byte boundaries moved by bulk copies.  With an explicit
 * cluster size, EINVAL when the lattice does not fit it (each CTA's band of padded
 * bit rows plus its halo rows must fit its shared memory). */
klmc_status klmc_sweep(klmc_ctx *c, int64_t n_mcs);

/* As klmc_sweep, and records n_unlike after every trace_every-th step into the
 * caller's device buffer dev_trace (int64, n_mcs / trace_every entries). */
klmc_status klmc_sweep_traced(klmc_ctx *c, int64_t n_mcs, int64_t trace_every,
                              int64_t *dev_trace);

/* Number of unlike contacts (kept exactly, updated by every accepted exchange)
 * and E/kT = omega/kT * n_unlike (energy model of the omega_AB equation).
 * Synchronises.  Either pointer may be NULL.  KLMC_ETIMEOUT if a tiled launch
 * of this handle gave up its bounded wait for its row copies: that launch left
 * its band unwritten, so the lattice is no longer a state of the chain. */
klmc_status klmc_energy(klmc_ctx *c, int64_t *n_unlike, double *energy_over_kT);

/* Recounts n_unlike from the lattice on the device (every bond once) without
 * changing the running value.  Synchronises. */
klmc_status klmc_energy_recount(klmc_ctx *c, int64_t *n_unlike);

/* Fraction of first neighbours (section "Image analysis"): *similar = the number
 * of sites whose randomly chosen nearest neighbour has the same type -- the
 * paper's fraction is *similar / N.  Sample m chooses site i's neighbour as
 * direction floor(w z / 2^32) of (1,0), (-1,0), (0,1), (0,-1), (1,-1), (-1,1)
 * (the first four for SQ4), w = word (i mod 4) of Philox4x32-10(seed,
 * {i div 4, 0xFFFFFFFE, m_lo, m_hi}), a stream of its own.  *exact = 1 - n_unlike
 * / B (B = z N / 2 bonds): the all-bond fraction, which the estimator's
 * expectation equals.  Synchronises.  Either output pointer may be NULL; EINVAL
 * for sample < 0. */
klmc_status klmc_ffn(klmc_ctx *c, int64_t sample, int64_t *similar, double *exact);

/* Device-side: enqueues sample m's count into *dev_similar (one int64 of device
 * memory) and returns without synchronising. */
klmc_status klmc_ffn_device(klmc_ctx *c, int64_t sample, int64_t *dev_similar);

/* Snapshot image of the lattice (section "Image analysis": one pixel per site,
 * white A and black B, sloped to keep the triangular geometry, scaled down with
 * supersampling).  Site (x, y) covers u in [2x + y, 2x + y + 2) half-sites and
 * v in [y, y+1) rows; the image spans U = 2 Lx + Ly - 1 half-sites by Ly rows.
 * Output pixel (i, j) averages an S x S grid of samples at
 * u = (2(iS + a) + 1) U / (2WS), v = (2(jS + b) + 1) Ly / (2HS) (integer
 * arithmetic: row floor(v), site floor((u - row) / 2), inside iff 0 <= x < Lx).
 * dev_image[jW + i] = round(255 n_A / n_in) (0 with no sample inside),
 * dev_mask[jW + i] = 1 iff at least half the samples are inside.  W = U, H =
 * round(sqrt(3) Ly) keeps the geometry at one pixel per half-site.  Both
 * buffers are W*H bytes of caller device memory.  1 <= S <= 64.  Enqueued. */
klmc_status klmc_snapshot(klmc_ctx *c, int32_t W, int32_t H, int32_t S, uint8_t *dev_image, uint8_t *dev_mask);

/* Fraction of first neighbours of a W x H gray image (section "Image analysis":
 * every lattice pixel takes one random neighbour pixel; similar when the gray
 * levels differ by at most delta, 35 in the paper).  Pixel p = jW + i takes
 * direction floor(w * 8 / 2^32) of (1,0), (1,1), (0,1), (-1,1), (-1,0), (-1,-1),
 * (0,-1), (1,-1), w = word (p mod 4) of Philox4x32-10(the handle's seed,
 * {p div 4, 0xFFFFFFFC, m_lo, m_hi}); neighbours outside the image or the mask
 * are not similar.  *similar / *pixels is the fraction.  Synchronises. */
klmc_status klmc_image_ffn(klmc_ctx *c, const uint8_t *dev_image, const uint8_t *dev_mask, int32_t W, int32_t H,
                           int32_t delta, int64_t sample, int64_t *similar, int64_t *pixels);

/* Sparse cluster-size histogram of the given species (1 = A, 0 = B): connected
 * components under the lattice adjacency with periodic wrap (section "Cluster
 * Analysis methods").  Writes (sizes[k], counts[k]) in ascending size to host
 * buffers and *n_distinct.  ETRUNC (with *n_distinct = needed length, other
 * outputs untouched) when capacity is too small.  Synchronises. */
klmc_status klmc_cluster_histogram(klmc_ctx *c, int32_t species, int64_t *sizes, int64_t *counts,
                                   int64_t capacity, int64_t *n_distinct);

/* Device-side variant: enqueues the same histogram into caller device buffers
 * (int64) and returns without synchronising.  *dev_n_distinct receives the
 * number of distinct sizes; only the first min(capacity, n) pairs are written. */
klmc_status klmc_cluster_histogram_device(klmc_ctx *c, int32_t species, int64_t *dev_sizes,
                                          int64_t *dev_counts, int64_t capacity,
                                          int64_t *dev_n_distinct);

/* Average cluster sizes of the given species (section "Cluster Analysis"
 * results: the average cluster size over time; the paper does not name the
 * average, so both are given).  From the histogram of klmc_cluster_histogram,
 * with exact int64 sums and one FP64 division each:
 *   *number_avg = sum s c / sum c        (mean size of a cluster)
 *   *weight_avg = sum s^2 c / sum s c    (mean size of the cluster holding a
 *                                         randomly chosen site of the species)
 * Both are 0 when the species has no site.  Synchronises.  Either output may be
 * NULL. */
klmc_status klmc_cluster_averages(klmc_ctx *c, int32_t species, double *number_avg, double *weight_avg);

/* The same two averages of any sparse histogram held in host memory: n pairs
 * (sizes[k], counts[k]), e.g. one copied back from
 * klmc_cluster_histogram_device or klmc_batch_cluster_histogram_device.  Host
 * arithmetic only; no device work.  EINVAL for n < 0, NULL arrays with n > 0, a
 * negative size or count, or sums beyond int64. */
klmc_status klmc_histogram_averages(const int64_t *sizes, const int64_t *counts, int64_t n,
                                    double *number_avg, double *weight_avg);

/* Largest lattice, in sites, accepted by klmc_cluster_histogram_noalloc. */
#define KLMC_NOALLOC_MAX_SITES (1 << 20)

/* The cluster-size histogram of klmc_cluster_histogram_device for a caller-owned
 * periodic lattice, without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call cudaMalloc,
 * such as a host framework that owns all device memory under a fixed budget with
 * no allocator hook, or a latency-bound loop that cannot accept cudaMalloc's
 * implicit device synchronisation.
 *  dev_lattice  device lattice, Ly rows of `pitch` 32-bit words (KLMC_PACK_BIT,
 *               site x is bit x%32 of word x/32) or `pitch` bytes (KLMC_PACK_BYTE,
 *               1 = A); owned by the caller, read only.  Boundaries are periodic
 *               (the paper's lattice model with periodic wrap); a helical lattice
 *               (KLMC_HELICAL) takes klmc_cluster_histogram_device instead.
 *  outputs      as klmc_cluster_histogram_device (caller device buffers).
 *  stream       cudaStream_t the work is enqueued on; returns without waiting.
 * Scratch comes from one fixed device array of the library (about 12.6 MB),
 * shared by all calls: calls whose work overlaps on the GPU race and must be
 * serialised by the caller.  The first call in a device's context loads the
 * library module that holds the array, which reserves the 12.6 MB on that device
 * until the process exits, may synchronise the device, and fails with
 * KLMC_ECUDA when that memory is not available; make that first call during
 * set-up, outside any latency-bound loop and before any stream capture.  Later
 * calls only look the array's address up.  EINVAL when Lx*Ly exceeds
 * KLMC_NOALLOC_MAX_SITES or an argument is invalid. */
klmc_status klmc_cluster_histogram_noalloc(const void *dev_lattice, int32_t packing, int32_t Lx,
                                           int32_t Ly, int32_t pitch, int32_t geometry,
                                           int32_t species, int64_t *dev_sizes,
                                           int64_t *dev_counts, int64_t capacity,
                                           int64_t *dev_n_distinct, void *stream);

/* Counters (see klmc_counters).  Synchronises.  KLMC_ETIMEOUT as klmc_energy. */
klmc_status klmc_get_counters(klmc_ctx *c, klmc_counters *out);

/* Test hook for the bounded waits (0 in normal use).  From the next sweep on, each
 * tiled launch of this handle that moves its rows by bulk copies issues no row
 * copy and waits instead for `bytes` that nothing delivers, so that its wait gives
 * up after a short bound with no copy in flight; the launch then leaves its band
 * unwritten and klmc_energy /
 * klmc_get_counters report KLMC_ETIMEOUT.  The handle's lattice is then no longer
 * a state of the chain; other handles are unaffected.  Synchronises.  EINVAL for
 * bytes < 0. */
klmc_status klmc_test_copy_shortfall(klmc_ctx *c, int32_t bytes);

/* Copies the lattice to host memory, one byte per site (n must equal Lx*Ly).
 * Synchronises. */
klmc_status klmc_get_lattice(klmc_ctx *c, uint8_t *host_out, int64_t n);

/* Replaces the lattice from host memory (n = Lx*Ly bytes, each 0 or 1), sets
 * the absolute sweep index, recounts n_unlike and n_A, and zeroes the counters.
 * Restoring a lattice saved with klmc_get_lattice at sweep s and continuing
 * reproduces the uninterrupted run exactly. */
klmc_status klmc_set_lattice(klmc_ctx *c, const uint8_t *host_in, int64_t n, int64_t sweep_index);

/* As klmc_set_lattice from a caller device buffer (n = Lx*Ly bytes, each 0 or
 * 1, not checked), enqueued without synchronising; n_A is recounted on the
 * device and reported by klmc_get_shape. */
klmc_status klmc_set_lattice_device(klmc_ctx *c, const uint8_t *dev_in, int64_t n,
                                    int64_t sweep_index);

/* Lattice sides, geometry and n_A of a handle.  Any pointer may be NULL.
 * Synchronises when n_A was last set on the device. */
klmc_status klmc_get_shape(klmc_ctx *c, int32_t *Lx, int32_t *Ly, int32_t *geometry, int64_t *n_A);

/* Autotuner: picks the fastest launch shape for this lattice's size by timing
 * every valid shape -- 1, 2, 4, 8 or 16 CTAs per lattice with 512, 256 or 128
 * threads per CTA, and the tiled per-phase path -- for probe_sweeps sweeps
 * on a scratch copy of the lattice at its current sweep index; for a handle
 * created with packing KLMC_PACK_AUTO, every shape with each store format (1 bit
 * and 1 byte per site), the handle's store then moved to the faster one (see
 * klmc_get_packing).  Every candidate's resulting sites and counters must equal
 * the first candidate's (exactness gate; a differing candidate is an error,
 * KLMC_ESTATE).  The choice is cached per (Lx, Ly, geometry, packing, with AUTO
 * its own key) for the process, applied to the handle and to handles of that
 * size created later with the automatic shape; the lattice, counters and
 * trajectory are unchanged.  Synchronises.  Either output pointer may be NULL.
 * ESTATE for a replica view; ENOMEM when the scratch copies cannot be allocated. */
klmc_status klmc_autotune(klmc_ctx *c, int32_t probe_sweeps, int32_t *cluster, int32_t *threads);

/* Moves the handle's lattice into a device store of the given format
 * (KLMC_PACK_BIT: 1 bit per site in 32-bit words; KLMC_PACK_BYTE: 1 byte per
 * site), leaving its sites, counters and sweep index as they are; the old store
 * is freed and a device pointer to it is no longer valid.  Enqueued on the
 * handle's stream (synchronises only with a caller's allocator, before freeing).
 * EINVAL for another value, ESTATE for a replica view, ENOMEM when the new store
 * cannot be allocated (the handle is then unchanged). */
klmc_status klmc_set_packing(klmc_ctx *c, int32_t packing);

/* Current store format of the handle: KLMC_PACK_BIT or KLMC_PACK_BYTE. */
klmc_status klmc_get_packing(klmc_ctx *c, int32_t *packing);

/* Launch shape of the handle's sweep: CTAs per lattice (thread-block cluster
 * size, -1 for the tiled per-phase path) and threads per CTA.  Either pointer may
 * be NULL. */
klmc_status klmc_get_launch(klmc_ctx *c, int32_t *cluster, int32_t *threads_per_cta);

/* Phases a CTA of this handle's sweep advances between exchanges of halo rows
 * with the CTAs of the neighbouring bands: for the resident sweep 2, 4 or 8 when
 * the bands are tall enough for a block (each CTA then re-evaluates 2K+1 halo
 * rows per side), 1 for a cluster barrier after every phase and for one CTA per
 * lattice; for the tiled path the phases per launch (2, 4 or 8 with halo rows read
 * from the store, 1 for one launch per phase with flips in place).  The
 * trajectory does not depend on it. */
klmc_status klmc_get_plan(klmc_ctx *c, int32_t *phases_per_exchange);

/* Waits for all work enqueued on the handle's stream. */
klmc_status klmc_synchronize(klmc_ctx *c);

/* Frees a handle created by klmc_create/klmc_create_ex.  NULL is accepted.
 * ESTATE for a replica view obtained from klmc_batch_replica. */
klmc_status klmc_destroy(klmc_ctx *c);

/* Batched form: n independent replicas (own sizes, compositions, omega, seeds)
 * advanced together by the resident kernel, one thread-block cluster per replica.
 * Each call chooses the launch shapes of the replicas it advances: a replica with
 * a fixed shape (params.cluster or params.threads set) keeps it; replicas with
 * automatic shapes keep theirs (tuned, else automatic) while the call's CTAs fit
 * the GPU's SMs, and otherwise run at half the CTAs per replica (where the band
 * still fits shared memory) with 128 threads per CTA, so that several CTAs share
 * an SM.  Replicas of one shape form one launch, larger lattices first; the
 * launches of different shapes run on internal streams forked from and joined
 * back to the stream of reps[0], which every replica uses.  The trajectory of a
 * replica does not depend on its launch shape.  Every replica must fit the
 * shared-memory resident sweep; a helical replica (KLMC_HELICAL) runs the resident
 * helical sweep, one launch of its own cluster on an internal stream, alongside
 * the others. */
klmc_status klmc_batch_create(klmc_batch **out, const klmc_params *reps, int32_t n);

/* Enqueues n_mcs[i] steps for replica i (entries may differ; 0 skips). */
klmc_status klmc_batch_sweep(klmc_batch *b, const int64_t *n_mcs);

/* Cluster-size histograms of the given species for every replica, as
 * klmc_cluster_histogram_device on each, enqueued on internal streams forked from
 * and joined back to the batch stream so that the replicas' histograms overlap.
 * Replica i writes dev_sizes[i*capacity ...], dev_counts[i*capacity ...] (device
 * int64 arrays of n*capacity) and dev_n_distinct[i] (device int64 array of n);
 * only the first min(capacity, n_distinct) pairs are written.  Does not
 * synchronise. */
klmc_status klmc_batch_cluster_histogram_device(klmc_batch *b, int32_t species, int64_t *dev_sizes,
                                                int64_t *dev_counts, int64_t capacity,
                                                int64_t *dev_n_distinct);

/* Launch shape (CTAs per replica, threads per CTA) replica i ran with in the last
 * klmc_batch_sweep that advanced it; before that, the replica's own shape.  Either
 * pointer may be NULL.  EINVAL for an index out of range. */
klmc_status klmc_batch_get_launch(klmc_batch *b, int32_t i, int32_t *cluster, int32_t *threads_per_cta);

/* Borrowed handle of replica i, usable with every per-lattice call except
 * klmc_destroy; valid until klmc_batch_destroy. */
klmc_status klmc_batch_replica(klmc_batch *b, int32_t i, klmc_ctx **view);

/* Frees the batch and its replicas.  NULL is accepted. */
klmc_status klmc_batch_destroy(klmc_batch *b);

/* ------------------------------------------------------------------------ */
/* Serving form: a job server with continuous batching.                      */
/* ------------------------------------------------------------------------ */
typedef struct klmc_server klmc_server;

enum { KLMC_JOB_KEEP_LATTICE = 1 }; /* submit flag: keep the final lattice on the host */

typedef struct klmc_job_result {
    int32_t status;        /* KLMC_OK, or the error that ended the job              */
    int32_t reserved;
    int64_t n_mcs;         /* Monte Carlo steps run                                 */
    int64_t n_unlike;      /* final number of unlike contacts                       */
    int64_t attempts, unlike, draws, accepts;  /* exact counters of the job          */
    double submit_s;       /* submission, admission and completion times, seconds   */
    double start_s;        /* since the server was created (host steady clock)      */
    double finish_s;
    int64_t n_histograms;  /* A-cluster histograms taken (hist_every cadence + end) */
} klmc_job_result;

typedef struct klmc_server_stats {
    int64_t submitted, finished, queued, resident, rounds, attempts;
    double busy_s, uptime_s;
    int64_t device_bytes, peak_device_bytes;
} klmc_server_stats;

/* Starts a server whose resident jobs may hold at most device_mem_budget bytes of
 * device memory.  stream: cudaStream_t for the server's work (NULL: a private
 * stream).  Jobs are admitted in arrival order while their memory fits both the
 * budget and the device's free memory; admitted lattices stay resident until their
 * job finishes.  Every round advances all resident jobs together (one
 * resident-kernel launch per launch shape, shapes chosen per round as for a batch
 * (klmc_batch_create), except that the jobs whose remaining steps take longest
 * keep their own shapes while their CTAs fit the SMs), each by a number of steps
 * sized to take about the same time; finished jobs leave and queued jobs join
 * between rounds.  A job's result does not depend on the other jobs. */
klmc_status klmc_server_create(klmc_server **out, size_t device_mem_budget, void *stream);

/* Queues a job: the lattice of p (p->stream is ignored; when p->alloc and p->free
 * are both set they serve the job's lattice memory and are called from the
 * server's worker thread, and a NULL from alloc fails the job with KLMC_ENOMEM), n_mcs
 * steps, an A-cluster histogram every hist_every steps and at the end
 * (0: none), flags (KLMC_JOB_KEEP_LATTICE).  Thread-safe; never blocks on GPU work.
 * Jobs too large for the budget, or too large for a cluster's shared memory, and
 * helical lattices too small for the resident helical sweep, finish with status
 * KLMC_EINVAL.  A helical job runs the resident helical sweep, one launch per round. */
klmc_status klmc_server_submit(klmc_server *s, const klmc_params *p, int64_t n_mcs,
                               int64_t hist_every, uint32_t flags, uint64_t *job_id);

/* Result of a job; KLMC_EBUSY while it is queued or running. */
klmc_status klmc_server_poll(klmc_server *s, uint64_t job_id, klmc_job_result *out);

/* Final lattice (one byte per site) of a finished job submitted with
 * KLMC_JOB_KEEP_LATTICE. */
klmc_status klmc_server_job_lattice(klmc_server *s, uint64_t job_id, uint8_t *host_out, int64_t n);

/* Last A-cluster histogram of a finished job (sparse, ascending); ETRUNC with
 * *n_distinct = needed length when capacity is too small. */
klmc_status klmc_server_job_histogram(klmc_server *s, uint64_t job_id, int64_t *sizes, int64_t *counts,
                                      int64_t capacity, int64_t *n_distinct);

/* Forgets a finished job's stored results. */
klmc_status klmc_server_release(klmc_server *s, uint64_t job_id);

/* Server counters (jobs, rounds, attempts of finished jobs, busy time, memory). */
klmc_status klmc_server_get_stats(klmc_server *s, klmc_server_stats *out);

/* Waits until every submitted job has finished; ETIMEOUT after timeout_s seconds. */
klmc_status klmc_server_drain(klmc_server *s, double timeout_s);

/* Finishes the queued and resident jobs, stops the worker and frees everything.
 * NULL is accepted. */
klmc_status klmc_server_destroy(klmc_server *s);

/* Human-readable name of a status. */
const char *klmc_status_str(klmc_status s);

/* Message describing the last error on the calling thread ("" if none). */
const char *klmc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KLMC_H */
