// klmc_host.h -- host-side handle structures shared by the C-ABI runtime
// (api.cu) and the job server (server.cu).  Not part of the C ABI.
#pragma once

#include <algorithm>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "klmc.h"
#include "klmc_internal.h"

struct klmc_ctx {
    klmc_params p;
    long long N = 0, nA = 0;
    bool nA_on_device = false;    // nA must be read back from state[kNA]
    int W = 0, pitch = 0;
    int cluster = 1;              // CTAs per lattice in the resident sweep (-1: tiled path)
    int threads = 512;            // threads per CTA of the resident sweep (128, 256 or 512)
    bool auto_shape = true;       // shape chosen by the library (params cluster = threads = 0)
    bool auto_packing = false;    // store format chosen by the library (params packing = AUTO)
    bool helical = false;         // helical boundary, seven-colour schedule (sweep_mpkk.cu)
    size_t lat_bytes = 0;
    void *lat = nullptr;
    long long *state = nullptr;   // StateSlot array
    void *init_scratch = nullptr;
    long long sweep = 0;
    klmc::SweepJob job;                 // host copy of the static job
    cudaStream_t stream = nullptr;
    void *cluster_mem = nullptr;  // lazily: klmc::ClusterScratch + host-API output
    klmc::ClusterScratch cs;
    long long *hist_out = nullptr;
    long long hist_cap = 0;
    uint8_t *dbytes = nullptr;    // lazily: one byte per site
    klmc_batch *owner = nullptr;  // non-null for replica views
    std::vector<std::pair<void *, size_t>> allocs;
    // tiled path: band height, capture stream, and instantiated graphs of K sweeps
    klmc::TiledPlan tiled{0, 0, 0, 0};  // tiled-path plan (H = 0: not yet chosen)
    void *tiled_alt = nullptr;          // second store buffer of the blocked tiled path
    int sm_count = 0;                   // SMs of the device (set with the tiled plan)
    cudaStream_t capture_stream = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
};

struct klmc_batch {
    std::vector<klmc_ctx *> reps;
    klmc::SweepJob *djobs = nullptr;
    klmc::SweepCall *dcalls = nullptr;
    int *dmap = nullptr;            // per call: active replicas grouped by launch shape
    std::vector<klmc::SweepCall> hcalls;
    cudaStream_t stream = nullptr;
    klmc_ctx *mem_owner = nullptr;  // holds the batch arrays' allocations
    // one internal stream and join event per launch shape (cluster, threads)
    std::map<std::pair<int, int>, std::pair<cudaStream_t, cudaEvent_t>> group_streams;
    cudaEvent_t fork = nullptr;
    int sm_count = 152;
    std::vector<std::pair<int, int>> last_shape;  // launch shape per replica, last call
    // internal streams and join events for the replicas' cluster histograms
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> hist_streams;
};

namespace klmc {
namespace host {

// Creates a lattice handle and enqueues its allocation, placement and energy
// count on p->stream without waiting for them.
klmc_status create_async(klmc_ctx **out, const klmc_params *p);
// Frees a handle created by create_async (synchronises its stream).
void destroy(klmc_ctx *c);
// Device bytes a handle with these parameters holds (lattice, state, placement
// scratch), for admission control.
size_t device_bytes(const klmc_params *p);

// Model of one step's time (8 phases) of the resident kernel at a launch shape:
// 1.3 us per phase plus 1 us per round of anchor words per thread.
inline double model_mcs_us(int Lx, int Ly, int cluster, int threads)
{
    const double words = (double)((Lx + 31) / 32);
    const double tasks = (Ly / 2.0) * words / (cluster > 0 ? cluster : 1);
    const double rounds = (double)(long long)((tasks + (threads > 0 ? threads : 256) - 1) /
                                              (threads > 0 ? threads : 256));
    return 8.0 * (1.3 + rounds);
}

// Launch shapes (cluster, threads) for one launch over several resident lattices,
// lattice i to advance by steps[i].  Lattices with fixed shapes keep them.  While
// the CTAs of all lattices at their own shapes fit the SMs, every lattice keeps its
// own (latency) shape.  Otherwise lattices with automatic shapes run with half as
// many CTAs (when the band still fits shared memory) and 128 threads per CTA, so
// that several CTAs share an SM: all of them when throughput is the goal (a batch
// call), or all but those whose remaining work takes longest, which keep their own
// shapes as long as their CTAs fit the SMs, when latency is (a server round).
void choose_shapes(const std::vector<klmc_ctx *> &cs, const std::vector<int64_t> &steps,
                   int sm_count, bool keep_longest, std::vector<std::pair<int, int>> *shapes);

}  // namespace host
}  // namespace klmc
