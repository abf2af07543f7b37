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
    int threads = 512;            // threads per CTA of the resident sweep (512 or 256)
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
    int tiled_H = 0;
    cudaStream_t capture_stream = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
};

struct klmc_batch {
    std::vector<klmc_ctx *> reps;
    klmc::SweepJob *djobs = nullptr;
    klmc::SweepCall *dcalls = nullptr;
    int *dmap = nullptr;            // replica indices grouped by cluster size, largest first
    std::vector<klmc::SweepCall> hcalls;
    cudaStream_t stream = nullptr;
    klmc_ctx *mem_owner = nullptr;  // holds the batch arrays' allocations
    // groups of replicas sharing a cluster size: (cluster, offset into dmap, count)
    struct Group {
        int cluster, threads, offset, count;
        size_t smem;
        cudaStream_t stream;
        cudaEvent_t done;
    };
    std::vector<Group> groups;
    std::vector<int> hmap;
    cudaEvent_t fork = nullptr;
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

}  // namespace host
}  // namespace klmc
