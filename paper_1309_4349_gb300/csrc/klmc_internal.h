// klmc_internal.h -- structures and launchers shared by the library's translation
// units.  Not part of the C ABI (see include/klmc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace klmc {

constexpr int kTRI6 = 0;
constexpr int kSQ4 = 1;
constexpr int kPackBit = 1;
constexpr int kPackByte = 2;

// Per-lattice device state, one int64 slot each.
enum StateSlot : int {
    kNUnlike = 0,   // running number of unlike contacts
    kAttempts = 1,
    kUnlike = 2,
    kDraws = 3,
    kAccepts = 4,
    kScratch0 = 5,  // recount result
    kNA = 6,        // A-site count after a device-side lattice load
    kSweepBase = 7, // absolute sweep index read by the tiled phase kernels
    kTracePos = 8,  // next entry of the energy trace (tiled path)
    kTracePtr = 9,  // device address of the energy trace (tiled path)
    kFfn = 10,      // random-neighbour count of klmc_ffn; with slot 11, klmc_image_ffn's counts
    kFault = 12,    // nonzero: a tiled launch gave up waiting for its row copies (band left unwritten)
    kStateSlots = 13
};

// Static description of one lattice for the sweep kernels.
struct SweepJob {
    void *lat;            // device store: packed bit rows (pitch in 32-bit words) or bytes
    int32_t Lx, Ly;
    int32_t pitch;        // row pitch: words (bit store) or bytes (byte store)
    int32_t packing;      // kPackBit / kPackByte
    int32_t geometry;     // kTRI6 / kSQ4
    int32_t W;            // 32-site words per row = ceil(Lx / 32)
    int32_t RW;           // padded shared-memory row length in words (W + 2)
    uint32_t key0, key1;  // Philox key = seed
    uint64_t magicW;      // ceil(2^32 / W): task t -> row (t * magicW) >> 32
    int32_t draw_lo;      // neighbour-agreement sums S in [draw_lo, draw_hi] need a draw
    int32_t draw_hi;
    int32_t copy_shortfall;  // test hook (0 in use): a band launch issues no row copy and waits for
                             // this many bytes instead, which nothing delivers, so its bounded wait runs out
    uint64_t thr[16];     // accept iff draw < thr[S] (S = same_a + same_b)
    long long *state;     // StateSlot array
    uint32_t rk[2][8];    // Philox round keys of rounds 2..9: key0 + r W0, key1 + r W1
};

// Per-call arguments of one lattice.
struct SweepCall {
    long long sweep0;      // absolute index of the first sweep
    long long n_mcs;       // sweeps to run (0 = skip)
    long long *trace;      // n_unlike after every trace_every-th sweep, or null
    long long trace_every;
};

// Dynamic shared memory per CTA for a lattice split over `cluster` CTAs (bytes),
// the per-CTA limit, and the largest cluster whose bands keep >= 4 rows.
size_t resident_smem_bytes(int Lx, int Ly, int cluster);
int resident_max_smem_bytes();
// Phases between halo exchanges of a lattice split over `cluster` CTAs (1: a
// cluster barrier after every phase).
int resident_block_phases(int Lx, int Ly, int cluster);
int resident_max_cluster(int Ly);
int resident_default_threads(int cluster);  // 512 for one CTA, else 256

// Batched launch: one cluster of `cluster` CTAs per job, tables in device memory;
// launched job i is d_jobs[d_map[i]] (d_map null: job i).  The trace buffers of
// the calls must be zeroed before the launch.
cudaError_t launch_resident_sweep(const SweepJob *d_jobs, const SweepCall *d_calls,
                                  const int *d_map, int n_jobs, int cluster, int threads,
                                  size_t smem_bytes, cudaStream_t stream);
// Single lattice: job and call passed by value as kernel parameters.  threads is
// 512 or 256.
cudaError_t launch_resident_sweep_one(const SweepJob &job, const SweepCall &call, int cluster,
                                      int threads, size_t smem_bytes, cudaStream_t stream);

// Tiled path for lattices too large for a cluster's shared memory.  Bands of H
// rows, one CTA each; sweep index read from state[kSweepBase].
//  K >= 2 (band plan): K phases per launch, each CTA with 2K+1 halo rows read
//    from one store buffer, its band written to the other (ping-pong).
//  K = 1: one launch per phase over the store in place, flips by atomics.
struct TiledPlan {
    int H, K, threads;
    int tables;  // 1: the band kernel keeps its K phases' task tables in shared memory
    size_t smem;
};
TiledPlan tiled_plan(int Lx, int Ly, int sm_count);
// The band plan alone (K = 1 when no block fits shared memory).
TiledPlan tiled_band_plan(int Lx, int Ly, int sm_count);
cudaError_t configure_tiled();
cudaError_t configure_band();
cudaError_t launch_band_phases(const SweepJob &job, const TiledPlan &plan, const void *src, void *dst,
                               int k, int f0, cudaStream_t stream);
// Sweeps k0 .. k0 + n_sweeps - 1 of the plan.  With K >= 2 the launches alternate
// between job.lat and alt (lat_bytes each) and end in job.lat (a copy back after
// an odd number of launches).
cudaError_t launch_tiled_phases(const SweepJob &job, const TiledPlan &plan, void *alt, size_t lat_bytes,
                                int k0, int n_sweeps, cudaStream_t stream);
cudaError_t launch_advance(long long *state, int n, cudaStream_t stream);
cudaError_t launch_trace(long long *state, cudaStream_t stream);

// Fraction of first neighbours, random-neighbour estimator of sample `sample`: the
// count of sites whose chosen neighbour is like them, into *out (overwritten).
cudaError_t launch_ffn(const void *lat, int packing, int Lx, int Ly, int pitch, int geometry, int helical,
                       uint32_t key0, uint32_t key1, long long sample, long long *out, cudaStream_t stream);

// Snapshot images (images.cu): W x H gray levels and lattice-pixel mask with S x S
// supersampling; and the image's (similar, lattice pixels) counts of sample `sample`
// into out2[0..1] (overwritten).
cudaError_t launch_snapshot(const void *lat, int packing, int pitch, int Lx, int Ly, int W, int H, int S,
                            uint8_t *image, uint8_t *mask, cudaStream_t stream);
cudaError_t launch_image_ffn(const uint8_t *image, const uint8_t *mask, int W, int H, int delta, uint32_t key0,
                             uint32_t key1, long long sample, long long *out2, cudaStream_t stream);

// Helical triangular lattice with the seven-colour schedule (sweep_mpkk.cu): whether
// the seven-site domains tile Lx x Ly (7 | N, Lx mod 7 in {3, 5}), and the seven
// iteration launches of each of n_sweeps sweeps k0 .. (sweep index from
// state[kSweepBase]).
bool helical_tiles(int Lx, int Ly);
// Resident helical sweep (sweep_helical.cu): iterations per block of a helical
// lattice over `cluster` CTAs (0: not resident), its dynamic shared memory, and one
// launch of n_mcs sweeps, one cluster of `cluster` CTAs of 512 threads.
int helical_resident_block(int Lx, int Ly, int cluster);
size_t helical_resident_smem_bytes(int Lx, int Ly, int cluster);
cudaError_t launch_helical_resident(const SweepJob &job, const SweepCall &call, int cluster, cudaStream_t stream);
cudaError_t launch_mpkk_phases(const SweepJob &job, int k0, int n_sweeps, int sm_count, cudaStream_t stream);

// Initial placement: the nA sites with the smallest (64-bit Philox key, index).
cudaError_t launch_init_lattice(void *lat, int packing, int Lx, int Ly, int pitch, uint32_t key0,
                                uint32_t key1, long long nA, void *scratch, cudaStream_t stream);
size_t init_scratch_bytes();

// n_unlike recount into *out (overwritten).
cudaError_t launch_recount(const void *lat, int packing, int Lx, int Ly, int pitch, int geometry,
                           long long *out, cudaStream_t stream,
                           int helical = 0);

// Pack one byte per site (0/1) into the device store, and back.
cudaError_t launch_pack(const uint8_t *bytes, void *lat, int packing, int Lx, int Ly, int pitch,
                        cudaStream_t stream);
cudaError_t launch_unpack(const void *lat, int packing, int Lx, int Ly, int pitch, uint8_t *bytes,
                          cudaStream_t stream);
// Count of A sites into *out (overwritten).
cudaError_t launch_count_A(const void *lat, int packing, int Lx, int Ly, int pitch, long long *out,
                           cudaStream_t stream);

// Cluster histogram scratch for n sites and up to n_species sites of one species.
struct ClusterScratch {
    int32_t *parent;      // [N]
    int32_t *csize;       // [N]
    int32_t *hist;        // [n_species + 1], zero between calls
    uint32_t *bitmap;     // [(n_species + 1 + 31) / 32], zero between calls
    long long n_species_max;
};
size_t cluster_scratch_bytes(long long N, long long n_species_max);
void cluster_scratch_carve(void *base, long long N, long long n_species_max, ClusterScratch *s);
// One-time zeroing of hist and bitmap (they are left zero by every histogram).
cudaError_t cluster_scratch_clear(const ClusterScratch &s, cudaStream_t stream);
cudaError_t launch_cluster_histogram(const void *lat, int packing, int Lx, int Ly, int pitch,
                                     int geometry, int species, const ClusterScratch &s,
                                     long long *sizes, long long *counts, long long capacity,
                                     long long *n_distinct, cudaStream_t stream,
                                     int helical = 0);

// Sets the message returned by klmc_last_error() on the calling thread.
void set_last_error(const char *msg);

}  // namespace klmc
