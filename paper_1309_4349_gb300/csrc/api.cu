// api.cu -- host runtime behind the C ABI in include/klmc.h: handle lifetime,
// device memory, the FP64 acceptance-threshold table, and the launches.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "klmc.h"
#include "klmc_internal.h"

using namespace klmc;

namespace {

thread_local std::string g_err;

klmc_status fail(klmc_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

// Concurrent streams for a batch's cluster histograms (each histogram is a chain
// of small launches, latency-bound for the lattice sizes batches hold).
constexpr int kHistStreams = 8;

#define KLMC_CUDA(expr)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(KLMC_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));           \
    } while (0)

bool device_ok(std::string *why)
{
    int dev = 0, n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        *why = "no CUDA device";
        return false;
    }
    if (cudaGetDevice(&dev) != cudaSuccess) {
        *why = "cudaGetDevice failed";
        return false;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
        *why = "cudaGetDeviceProperties failed";
        return false;
    }
    if (prop.major * 10 + prop.minor != 103) {
        *why = "library built for sm_103a; device is sm_" + std::to_string(prop.major * 10 + prop.minor);
        return false;
    }
    return true;
}

}  // namespace

void klmc::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

#include "klmc_host.h"

namespace {

void *dev_alloc(klmc_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    if (c->p.alloc) {
        p = c->p.alloc(bytes, c->p.stream, c->p.user);
    } else if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.push_back({p, bytes});
    return p;
}

void free_all(klmc_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
    c->graphs.clear();
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    c->capture_stream = nullptr;
    for (auto &a : c->allocs) {
        if (c->p.alloc && c->p.free) c->p.free(a.first, a.second, c->p.stream, c->p.user);
        else if (!c->p.alloc) cudaFreeAsync(a.first, c->stream);
    }
    c->allocs.clear();
    cudaStreamSynchronize(c->stream);
}

// Returns one allocation of dev_alloc; with a caller's allocator after the stream's
// work is done (its frees need not be stream-ordered).
void dev_free(klmc_ctx *c, void *p)
{
    for (size_t i = 0; i < c->allocs.size(); ++i) {
        if (c->allocs[i].first != p) continue;
        if (c->p.alloc && c->p.free) {
            cudaStreamSynchronize(c->stream);
            c->p.free(p, c->allocs[i].second, c->p.stream, c->p.user);
        } else if (!c->p.alloc) {
            cudaFreeAsync(p, c->stream);
        }
        c->allocs.erase(c->allocs.begin() + (long)i);
        return;
    }
}

// Row pitch and size of a device store: rows of 16 bytes, of 32-bit words (a bit
// per site) or of bytes (a byte per site).
void store_layout(int Lx, int Ly, int packing, int *pitch, size_t *bytes)
{
    if (packing == KLMC_PACK_BIT) {
        *pitch = ((Lx + 31) / 32 + 3) / 4 * 4;
        *bytes = (size_t)*pitch * 4 * (size_t)Ly;
    } else {
        *pitch = (Lx + 15) / 16 * 16;
        *bytes = (size_t)*pitch * (size_t)Ly;
    }
}

klmc_status validate(const klmc_params *p)
{
    if (!p) return fail(KLMC_EINVAL, "params is NULL");
    if (p->Lx < 4 || p->Ly < 4) return fail(KLMC_EINVAL, "Lx and Ly must be >= 4");
    const long long N = (long long)p->Lx * p->Ly;
    if (N > 2147483647LL) return fail(KLMC_EINVAL, "Lx*Ly must be <= 2^31 - 1");
    if (p->geometry != KLMC_TRI6 && p->geometry != KLMC_SQ4) return fail(KLMC_EINVAL, "unknown geometry");
    if (p->boundary != KLMC_PERIODIC && p->boundary != KLMC_HELICAL) return fail(KLMC_EINVAL, "unknown boundary");
    if (p->boundary == KLMC_HELICAL) {
        if (p->geometry != KLMC_TRI6)
            return fail(KLMC_EINVAL, "helical boundaries are for the triangular lattice (seven-site domains)");
        if (!helical_tiles(p->Lx, p->Ly))
            return fail(KLMC_EINVAL, "helical lattice: seven-site domains tile it only when 7 divides Lx*Ly "
                                     "and Lx mod 7 is 3 or 5");
        if (p->threads != 0 && p->threads != 512)
            return fail(KLMC_EINVAL, "helical lattices run at 512 threads per CTA (threads 0 or 512)");
        if (p->cluster > 0 && helical_resident_block(p->Lx, p->Ly, p->cluster) < 2)
            return fail(KLMC_EINVAL, "helical lattice: the resident sweep needs a cluster of at least 2 CTAs "
                                     "whose bands each hold 2K+1 halo rows for K >= 2 iterations per block "
                                     "(cluster 0 chooses, cluster -1 runs one launch per iteration)");
    }
    if (p->packing != KLMC_PACK_AUTO && p->packing != KLMC_PACK_BIT && p->packing != KLMC_PACK_BYTE)
        return fail(KLMC_EINVAL, "unknown packing");
    if (!isfinite(p->omega_over_kT)) return fail(KLMC_EINVAL, "omega_over_kT must be finite");
    if (p->n_A < 0 && !(p->fraction_A >= 0.0 && p->fraction_A <= 1.0))
        return fail(KLMC_EINVAL, "fraction_A must be in [0, 1]");
    if (p->n_A > N) return fail(KLMC_EINVAL, "n_A must be in [0, Lx*Ly]");
    if (p->alloc && !p->free) return fail(KLMC_EINVAL, "alloc given without free");
    if (p->cluster < -1 || p->cluster > 16) return fail(KLMC_EINVAL, "cluster must be in [-1, 16]");
    if (p->cluster > 1 && p->Ly / p->cluster < 4)
        return fail(KLMC_EINVAL, "cluster too large: every band needs >= 4 rows");
    if (p->threads != 0 && p->threads != 128 && p->threads != 256 && p->threads != 512)
        return fail(KLMC_EINVAL, "threads must be 0, 128, 256 or 512");
    return KLMC_OK;
}

// Automatic cluster size: the smallest power of two whose bands fit in shared
// memory, raised while every band keeps >= 24 rows (more CTAs shorten each phase;
// too-thin bands spend their time on halos and barriers).
int auto_cluster(int Lx, int Ly)
{
    const int cmax = resident_max_cluster(Ly);
    int c = 1;
    while (c < cmax && resident_smem_bytes(Lx, Ly, c) > (size_t)resident_max_smem_bytes()) c *= 2;
    while (c * 2 <= cmax && Ly / (c * 2) >= 24) c *= 2;
    return c;
}

// Acceptance table (Metropolis step c with u = r / 2^32): a pair whose
// neighbour-agreement sum is S changes n_unlike by dn = 2 (S - (z - 1)); it is
// accepted without a draw when (omega/kT) dn <= 0, otherwise iff a 32-bit draw
// r < ceil(exp(-(omega/kT) dn) 2^32).  Built once, in FP64, on the host.
klmc_status build_thresholds(double bw, int geometry, SweepJob *J)
{
    const int zm1 = (geometry == KLMC_TRI6 ? 6 : 4) - 1;
    int lo = 16, hi = -1;
    for (int S = 0; S < 16; ++S) J->thr[S] = 0;
    for (int S = 0; S <= 2 * zm1; ++S) {
        const int dn = 2 * (S - zm1);
        const double x = bw * (double)dn;
        if (x <= 0.0) continue;
        J->thr[S] = (uint64_t)ceil(ldexp(exp(-x), 32));
        if (S < lo) lo = S;
        if (S > hi) hi = S;
    }
    for (int S = lo; S <= hi; ++S) {
        const double x = bw * (double)(2 * (S - zm1));
        if (x <= 0.0) return fail(KLMC_EINVAL, "internal: draw set is not an interval");
    }
    if (hi < 0) {
        lo = 1;
        hi = 0;
    }
    J->draw_lo = lo;
    J->draw_hi = hi;
    return KLMC_OK;
}

klmc_status ensure_bytes(klmc_ctx *c)
{
    if (c->dbytes) return KLMC_OK;
    c->dbytes = (uint8_t *)dev_alloc(c, (size_t)c->N);
    if (!c->dbytes) return fail(KLMC_ENOMEM, "device allocation of the byte lattice failed");
    return KLMC_OK;
}

klmc_status ensure_clusters(klmc_ctx *c)
{
    if (c->cluster_mem) return KLMC_OK;
    const long long nsp = c->N;
    long long cap = (long long)floor(sqrt(2.0 * (double)c->N)) + 2;
    const size_t sbytes = cluster_scratch_bytes(c->N, nsp);
    const size_t obytes = (size_t)(2 * cap + 2) * sizeof(long long);
    void *mem = dev_alloc(c, sbytes + obytes);
    if (!mem) return fail(KLMC_ENOMEM, "device allocation of cluster scratch failed");
    cluster_scratch_carve(mem, c->N, nsp, &c->cs);
    KLMC_CUDA(cluster_scratch_clear(c->cs, c->stream));
    c->cluster_mem = mem;
    c->hist_out = (long long *)((char *)mem + sbytes);
    c->hist_cap = cap;
    return KLMC_OK;
}

bool tuned_shape(int Lx, int Ly, int geometry, int packing, int *cluster, int *threads, int *tuned_packing);

// Lattices of at least this many sites run faster on the tiled path, whose bands
// use every SM, than in one cluster's shared memory (GB300, 200 MCS of square TRI6
// lattices: 724^2 5.7 vs 4.8 ms resident, 1024^2 5.8 vs 7.1 ms, 2048^2 6.8 vs
// 20.1 ms); the automatic shape of a standalone handle takes it there.
constexpr long long kTiledAutoSites = 786432;

// standalone: a handle of its own (klmc_create, klmc_create_ex), which may take the
// tiled path automatically; batch replicas and server jobs stay resident.
klmc_status create_one(klmc_ctx **out, const klmc_params *p, klmc_batch *owner, bool sync = true,
                       bool standalone = false)
{
    klmc_status st = validate(p);
    if (st != KLMC_OK) return st;
    std::string why;
    if (!device_ok(&why)) return fail(KLMC_ENODEV, why);
    klmc_ctx *c = new (std::nothrow) klmc_ctx();
    if (!c) return fail(KLMC_ENOMEM, "host allocation failed");
    c->p = *p;
    c->auto_packing = p->packing == KLMC_PACK_AUTO && p->boundary != KLMC_HELICAL;
    if (c->p.packing == KLMC_PACK_AUTO) c->p.packing = KLMC_PACK_BIT;
    c->owner = owner;
    c->stream = (cudaStream_t)p->stream;
    c->N = (long long)p->Lx * p->Ly;
    c->nA = p->n_A >= 0 ? p->n_A : (long long)floor(p->fraction_A * (double)c->N + 0.5);
    c->W = (p->Lx + 31) / 32;
    c->helical = p->boundary == KLMC_HELICAL;
    if (c->helical) {
        // Resident in a cluster's shared memory when the bands are tall enough for
        // blocks of iterations; otherwise one launch per iteration over the store.
        c->cluster = p->cluster != 0 ? p->cluster : auto_cluster(p->Lx, p->Ly);
        if (c->cluster > 0 && helical_resident_block(p->Lx, p->Ly, c->cluster) < 2) c->cluster = -1;
        c->threads = c->cluster > 0 ? 512 : 256;
        c->auto_shape = false;
    } else {
        c->cluster = p->cluster != 0 ? p->cluster : auto_cluster(p->Lx, p->Ly);
        if (p->cluster == 0 &&
            resident_smem_bytes(p->Lx, p->Ly, c->cluster) > (size_t)resident_max_smem_bytes())
            c->cluster = -1;  // automatic choice, too large for shared memory: tiled path
        if (standalone && p->cluster == 0 && c->cluster > 0 && c->N >= kTiledAutoSites) {
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) == cudaSuccess &&
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                tiled_plan(p->Lx, p->Ly, sms).K >= 2)
                c->cluster = -1;  // automatic choice, large: bands over every SM
        }
        c->threads = resident_default_threads(c->cluster);
        int tuned_packing = c->p.packing;
        if (p->cluster == 0 && p->threads == 0 &&
            tuned_shape(p->Lx, p->Ly, p->geometry, c->auto_packing ? KLMC_PACK_AUTO : c->p.packing, &c->cluster,
                        &c->threads, &tuned_packing))
            c->p.packing = tuned_packing;  // the autotuner's store format for this size
        c->auto_shape = p->cluster == 0 && p->threads == 0;
        if (p->threads != 0) c->threads = p->threads;
    }
    store_layout(p->Lx, p->Ly, c->p.packing, &c->pitch, &c->lat_bytes);
    c->lat = dev_alloc(c, c->lat_bytes);
    c->state = (long long *)dev_alloc(c, kStateSlots * sizeof(long long));
    c->init_scratch = dev_alloc(c, init_scratch_bytes());
    if (!c->lat || !c->state || !c->init_scratch) {
        free_all(c);
        delete c;
        return fail(KLMC_ENOMEM, "device allocation failed");
    }
    SweepJob &J = c->job;
    memset(&J, 0, sizeof(J));
    J.lat = c->lat;
    J.Lx = p->Lx;
    J.Ly = p->Ly;
    J.pitch = c->pitch;
    J.packing = c->p.packing;
    J.geometry = p->geometry;
    J.W = c->W;
    J.RW = (p->Lx + 95) / 32;  // ceil(Lx / 32) + 2: windows read words j .. j+2
    J.magicW = (0x100000000ull + (unsigned long long)c->W - 1) / (unsigned long long)c->W;
    J.key0 = (uint32_t)p->seed;
    J.key1 = (uint32_t)(p->seed >> 32);
    for (int r = 2; r < 10; ++r) {  // Philox4x32-10 round keys (Weyl sequence of the key)
        J.rk[0][r - 2] = J.key0 + (uint32_t)r * 0x9E3779B9u;
        J.rk[1][r - 2] = J.key1 + (uint32_t)r * 0xBB67AE85u;
    }
    J.state = c->state;
    st = build_thresholds(p->omega_over_kT, p->geometry, &J);
    if (st != KLMC_OK) {
        free_all(c);
        delete c;
        return st;
    }
    cudaError_t e = cudaMemsetAsync(c->state, 0, kStateSlots * sizeof(long long), c->stream);
    // The store's row padding (words or bytes past the last site) stays zero: every
    // writer writes sites only, or whole rows with zero padding.
    if (e == cudaSuccess) e = cudaMemsetAsync(c->lat, 0, c->lat_bytes, c->stream);
    if (e == cudaSuccess)
        e = launch_init_lattice(c->lat, J.packing, p->Lx, p->Ly, c->pitch, J.key0, J.key1, c->nA,
                                c->init_scratch, c->stream);
    if (e == cudaSuccess)
        e = launch_recount(c->lat, J.packing, p->Lx, p->Ly, c->pitch, p->geometry,
                           c->state + kNUnlike, c->stream, c->helical);
    if (e == cudaSuccess && sync) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        free_all(c);
        delete c;
        return fail(KLMC_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    *out = c;
    return KLMC_OK;
}

klmc_status check_resident(const klmc_ctx *c, int cluster)
{
    const size_t need = resident_smem_bytes(c->p.Lx, c->p.Ly, cluster);
    if (need > (size_t)resident_max_smem_bytes())
        return fail(KLMC_EINVAL, "lattice too large for the shared-memory resident sweep (" +
                                     std::to_string(need) + " bytes of padded bit rows per CTA at " +
                                     std::to_string(cluster) + " CTAs per lattice)");
    return KLMC_OK;
}

// Plan of the handle's per-launch path (tiled bands, or the seven iteration launches
// of a helical lattice), and the second store buffer that band blocks need.
klmc_status ensure_tiled(klmc_ctx *c)
{
    if (c->tiled.H != 0) return KLMC_OK;
    int dev = 0, sms = 0;
    KLMC_CUDA(cudaGetDevice(&dev));
    KLMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    c->sm_count = sms;
    if (c->helical) {
        c->tiled = TiledPlan{1, 1, 256, 0, 0};
        return KLMC_OK;
    }
    KLMC_CUDA(configure_tiled());
    const TiledPlan plan = tiled_plan(c->p.Lx, c->p.Ly, sms);
    if (plan.K >= 2) {
        c->tiled_alt = dev_alloc(c, c->lat_bytes);
        if (!c->tiled_alt) return fail(KLMC_ENOMEM, "device allocation of the tiled path's second buffer failed");
        KLMC_CUDA(cudaMemsetAsync(c->tiled_alt, 0, c->lat_bytes, c->stream));
    }
    c->tiled = plan;
    return KLMC_OK;
}

// Sweeps k0 .. k0+n-1 of the handle's per-launch path on job J's store.
cudaError_t path_sweeps(klmc_ctx *c, const SweepJob &J, int k0, int n, cudaStream_t stream)
{
    if (c->helical) return launch_mpkk_phases(J, k0, n, c->sm_count, stream);
    return launch_tiled_phases(J, c->tiled, c->tiled_alt, c->lat_bytes, k0, n, stream);
}

// Instantiated graph of K sweeps on the tiled path (their phase launches, then
// state[kSweepBase] += K), built once per handle and K on a private capture stream.
klmc_status tiled_graph(klmc_ctx *c, int K, cudaGraphExec_t *out)
{
    auto it = c->graphs.find(K);
    if (it != c->graphs.end()) {
        *out = it->second;
        return KLMC_OK;
    }
    if (!c->capture_stream)
        KLMC_CUDA(cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    KLMC_CUDA(cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = path_sweeps(c, c->job, 0, K, c->capture_stream);
    if (e == cudaSuccess) e = launch_advance(c->state, K, c->capture_stream);
    cudaError_t e2 = cudaStreamEndCapture(c->capture_stream, &graph);
    if (e == cudaSuccess) e = e2;
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(KLMC_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    c->graphs[K] = exec;
    *out = exec;
    return KLMC_OK;
}

// n_mcs sweeps on the tiled path: graph replays of K sweeps, direct launches for
// the rest, the trace kernel after every trace_every-th sweep.
klmc_status sweep_tiled(klmc_ctx *c, int64_t n_mcs, int64_t trace_every, int64_t *dev_trace)
{
    klmc_status pst = ensure_tiled(c);
    if (pst != KLMC_OK) return pst;
    const long long init[3] = {c->sweep, 0, (long long)(intptr_t)dev_trace};
    KLMC_CUDA(cudaMemcpyAsync(c->state + kSweepBase, init, sizeof(init), cudaMemcpyHostToDevice,
                              c->stream));
    const int K = (trace_every > 0 && trace_every <= 64) ? (int)trace_every : 8;
    cudaGraphExec_t exec = nullptr;
    klmc_status st = tiled_graph(c, K, &exec);
    if (st != KLMC_OK) return st;
    int64_t done = 0;
    while (done < n_mcs) {
        const int64_t next = trace_every > 0 ? (done / trace_every + 1) * trace_every : n_mcs;
        const int64_t upto = next < n_mcs ? next : n_mcs;
        while (upto - done >= K) {
            KLMC_CUDA(cudaGraphLaunch(exec, c->stream));
            done += K;
        }
        if (upto > done) {
            const int r = (int)(upto - done);
            KLMC_CUDA(path_sweeps(c, c->job, 0, r, c->stream));
            KLMC_CUDA(launch_advance(c->state, r, c->stream));
            done = upto;
        }
        if (trace_every > 0 && done % trace_every == 0) KLMC_CUDA(launch_trace(c->state, c->stream));
    }
    c->sweep += n_mcs;
    return KLMC_OK;
}

klmc_status sweep_one(klmc_ctx *c, int64_t n_mcs, int64_t trace_every, int64_t *dev_trace)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (n_mcs < 0) return fail(KLMC_EINVAL, "n_mcs must be >= 0");
    if (trace_every < 0 || (trace_every > 0 && !dev_trace))
        return fail(KLMC_EINVAL, "trace_every > 0 needs a device trace buffer");
    if (n_mcs == 0) return KLMC_OK;
    if (c->cluster < 0) return sweep_tiled(c, n_mcs, trace_every, dev_trace);
    if (c->helical) {
        if (trace_every > 0 && n_mcs / trace_every > 0)
            KLMC_CUDA(cudaMemsetAsync(dev_trace, 0, (size_t)(n_mcs / trace_every) * sizeof(int64_t), c->stream));
        SweepCall call;
        call.sweep0 = c->sweep;
        call.n_mcs = n_mcs;
        call.trace = (long long *)dev_trace;
        call.trace_every = trace_every;
        KLMC_CUDA(launch_helical_resident(c->job, call, c->cluster, c->stream));
        c->sweep += n_mcs;
        return KLMC_OK;
    }
    klmc_status st = check_resident(c, c->cluster);
    if (st != KLMC_OK) return st;
    if (trace_every > 0 && n_mcs / trace_every > 0)
        KLMC_CUDA(cudaMemsetAsync(dev_trace, 0, (size_t)(n_mcs / trace_every) * sizeof(int64_t),
                                  c->stream));
    SweepCall call;
    call.sweep0 = c->sweep;
    call.n_mcs = n_mcs;
    call.trace = (long long *)dev_trace;
    call.trace_every = trace_every;
    KLMC_CUDA(launch_resident_sweep_one(c->job, call, c->cluster, c->threads,
                                        resident_smem_bytes(c->p.Lx, c->p.Ly, c->cluster),
                                        c->stream));
    c->sweep += n_mcs;
    return KLMC_OK;
}

// ---------------------------------------------------------------------------
// Autotuner: launch shape per lattice size, chosen by timing on a scratch copy,
// with every candidate's result required to be identical.
// ---------------------------------------------------------------------------
struct TuneKey {
    int Lx, Ly, geometry, packing;  // packing KLMC_PACK_AUTO: the tuner also picks the store format
    bool operator<(const TuneKey &o) const
    {
        if (Lx != o.Lx) return Lx < o.Lx;
        if (Ly != o.Ly) return Ly < o.Ly;
        if (geometry != o.geometry) return geometry < o.geometry;
        return packing < o.packing;
    }
};
struct Tuned {
    int cluster, threads, packing;
};
std::mutex g_tune_mutex;
std::map<TuneKey, Tuned> g_tune_cache;

bool tuned_shape(int Lx, int Ly, int geometry, int packing, int *cluster, int *threads, int *tuned_packing)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(TuneKey{Lx, Ly, geometry, packing});
    if (it == g_tune_cache.end()) return false;
    *cluster = it->second.cluster;
    *threads = it->second.threads;
    *tuned_packing = it->second.packing;
    return true;
}

// Moves the handle's lattice into a store of the other format (its sites, counters
// and sweep index unchanged).  Graphs and the tiled path's second buffer, which
// hold the old store's address or size, are dropped and rebuilt on next use.
klmc_status convert_store(klmc_ctx *c, int packing)
{
    if (packing == c->job.packing) return KLMC_OK;
    klmc_status st = ensure_bytes(c);
    if (st != KLMC_OK) return st;
    int pitch = 0;
    size_t bytes = 0;
    store_layout(c->p.Lx, c->p.Ly, packing, &pitch, &bytes);
    void *lat = dev_alloc(c, bytes);
    if (!lat) return fail(KLMC_ENOMEM, "device allocation of the new store failed");
    KLMC_CUDA(launch_unpack(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->dbytes, c->stream));
    KLMC_CUDA(cudaMemsetAsync(lat, 0, bytes, c->stream));  // row padding stays zero
    KLMC_CUDA(launch_pack(c->dbytes, lat, packing, c->p.Lx, c->p.Ly, pitch, c->stream));
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);
    c->graphs.clear();
    if (c->tiled_alt) dev_free(c, c->tiled_alt);
    c->tiled_alt = nullptr;
    c->tiled = TiledPlan{0, 0, 0, 0};
    dev_free(c, c->lat);
    c->lat = lat;
    c->lat_bytes = bytes;
    c->pitch = pitch;
    c->p.packing = packing;
    c->job.lat = lat;
    c->job.pitch = pitch;
    c->job.packing = packing;
    return KLMC_OK;
}

// A store for the probes: the lattice at its start, its format, and (for the tiled
// path's blocks) a second buffer of its size.
struct ProbeStore {
    const void *src;
    size_t bytes;
    int packing, pitch;
    void *alt;
};

struct ProbeResult {
    float ms;
    std::vector<uint8_t> sites;  // one byte per site after the probe
    long long state[kStateSlots];
};

// Runs n sweeps of the lattice in store `ps` with launch shape (cluster, threads) on
// the scratch lattice/state (copied from the store and the handle first).
klmc_status probe_shape(klmc_ctx *c, const ProbeStore &ps, void *scratch_lat, long long *scratch_state,
                        int cluster, int threads, int n, cudaEvent_t e0, cudaEvent_t e1, ProbeResult *out)
{
    SweepJob J = c->job;
    J.lat = scratch_lat;
    J.state = scratch_state;
    J.packing = ps.packing;
    J.pitch = ps.pitch;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up; the second is timed
        KLMC_CUDA(cudaMemcpyAsync(scratch_lat, ps.src, ps.bytes, cudaMemcpyDeviceToDevice, c->stream));
        KLMC_CUDA(cudaMemcpyAsync(scratch_state, c->state, kStateSlots * sizeof(long long),
                                  cudaMemcpyDeviceToDevice, c->stream));
        const long long base = c->sweep;
        KLMC_CUDA(cudaMemcpyAsync(scratch_state + kSweepBase, &base, sizeof(base),
                                  cudaMemcpyHostToDevice, c->stream));
        KLMC_CUDA(cudaEventRecord(e0, c->stream));
        if (cluster < 0) {
            KLMC_CUDA(launch_tiled_phases(J, c->tiled, ps.alt, ps.bytes, 0, n, c->stream));
            KLMC_CUDA(launch_advance(scratch_state, n, c->stream));
        } else {
            SweepCall call;
            call.sweep0 = c->sweep;
            call.n_mcs = n;
            call.trace = nullptr;
            call.trace_every = 0;
            KLMC_CUDA(launch_resident_sweep_one(J, call, cluster, threads,
                                                resident_smem_bytes(c->p.Lx, c->p.Ly, cluster),
                                                c->stream));
        }
        KLMC_CUDA(cudaEventRecord(e1, c->stream));
        KLMC_CUDA(cudaEventSynchronize(e1));
    }
    KLMC_CUDA(cudaEventElapsedTime(&out->ms, e0, e1));
    KLMC_CUDA(launch_unpack(scratch_lat, ps.packing, c->p.Lx, c->p.Ly, ps.pitch, c->dbytes, c->stream));
    out->sites.resize((size_t)c->N);
    KLMC_CUDA(cudaMemcpyAsync(out->sites.data(), c->dbytes, (size_t)c->N, cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaMemcpyAsync(out->state, scratch_state, sizeof(out->state), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    return KLMC_OK;
}

// Times every valid launch shape -- and, for a handle whose store format is the
// library's choice, both formats -- and keeps the fastest; every candidate must
// leave the same sites and counters as the first.
klmc_status autotune(klmc_ctx *c, int probe_sweeps)
{
    if (c->helical) return KLMC_OK;  // one launch shape: the iteration launches
    const TuneKey key{c->p.Lx, c->p.Ly, c->p.geometry, c->auto_packing ? (int)KLMC_PACK_AUTO : c->job.packing};
    {
        std::unique_lock<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            const Tuned t = it->second;
            lock.unlock();
            c->cluster = t.cluster;
            c->threads = t.threads;
            return convert_store(c, t.packing);
        }
    }
    std::vector<std::pair<int, int>> shapes;
    for (int C : {1, 2, 4, 8, 16}) {
        if (C > 1 && c->p.Ly / C < 4) continue;
        if (resident_smem_bytes(c->p.Lx, c->p.Ly, C) > (size_t)resident_max_smem_bytes()) continue;
        shapes.push_back({C, 512});
        shapes.push_back({C, 256});
        shapes.push_back({C, 128});
    }
    shapes.push_back({-1, 256});
    klmc_status st = ensure_bytes(c);
    if (st == KLMC_OK) st = ensure_tiled(c);
    if (st != KLMC_OK) return st;
    std::vector<ProbeStore> stores{{c->lat, c->lat_bytes, c->job.packing, c->pitch, c->tiled_alt}};
    std::vector<void *> scratch;  // freed on every return below
    auto release = [&]() {
        for (void *q : scratch) dev_free(c, q);
        scratch.clear();
    };
    size_t max_bytes = c->lat_bytes;
    if (c->auto_packing) {  // the other format's copy of the lattice
        ProbeStore o{};
        o.packing = c->job.packing == KLMC_PACK_BIT ? KLMC_PACK_BYTE : KLMC_PACK_BIT;
        store_layout(c->p.Lx, c->p.Ly, o.packing, &o.pitch, &o.bytes);
        void *lat = dev_alloc(c, o.bytes);
        if (lat) scratch.push_back(lat);
        void *alt = c->tiled.K >= 2 ? dev_alloc(c, o.bytes) : nullptr;
        if (alt) scratch.push_back(alt);
        if (!lat || (c->tiled.K >= 2 && !alt)) {
            release();
            return fail(KLMC_ENOMEM, "autotune scratch allocation failed");
        }
        cudaError_t e = launch_unpack(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->dbytes, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(lat, 0, o.bytes, c->stream);
        if (e == cudaSuccess) e = launch_pack(c->dbytes, lat, o.packing, c->p.Lx, c->p.Ly, o.pitch, c->stream);
        if (e != cudaSuccess) {
            release();
            return fail(KLMC_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
        }
        o.src = lat;
        o.alt = alt;
        stores.push_back(o);
        max_bytes = std::max(max_bytes, o.bytes);
    }
    void *slat = dev_alloc(c, max_bytes);
    if (slat) scratch.push_back(slat);
    long long *sstate = (long long *)dev_alloc(c, kStateSlots * sizeof(long long));
    if (sstate) scratch.push_back(sstate);
    if (!slat || !sstate) {
        release();
        return fail(KLMC_ENOMEM, "autotune scratch allocation failed");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        release();
        return fail(KLMC_ECUDA, "autotune: event creation failed");
    }
    ProbeResult ref, cur;
    float best_ms = 0.f;
    Tuned best{shapes.front().first, shapes.front().second, c->job.packing};
    bool first = true;
    for (const ProbeStore &ps : stores) {
        for (size_t i = 0; i < shapes.size() && st == KLMC_OK; ++i) {
            ProbeResult &r = first ? ref : cur;
            st = probe_shape(c, ps, slat, sstate, shapes[i].first, shapes[i].second, probe_sweeps, e0, e1, &r);
            if (st != KLMC_OK) break;
            if (!first) {
                bool same = r.sites == ref.sites;
                for (int k = kNUnlike; k <= kAccepts; ++k) same = same && r.state[k] == ref.state[k];
                if (!same) {
                    st = fail(KLMC_ESTATE, "autotune: launch shape (" + std::to_string(shapes[i].first) + ", " +
                                               std::to_string(shapes[i].second) + ") with store format " +
                                               std::to_string(ps.packing) + " changed the result; refusing it");
                    break;
                }
            }
            if (first || r.ms < best_ms) {
                best_ms = r.ms;
                best = Tuned{shapes[i].first, shapes[i].second, ps.packing};
            }
            first = false;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    if (st != KLMC_OK) return st;
    c->cluster = best.cluster;
    c->threads = best.threads;
    st = convert_store(c, best.packing);
    if (st != KLMC_OK) return st;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best;
    return KLMC_OK;
}

}  // namespace

void klmc::host::choose_shapes(const std::vector<klmc_ctx *> &cs, const std::vector<int64_t> &steps,
                               int sm_count, bool keep_longest, std::vector<std::pair<int, int>> *shapes)
{
    const size_t n = cs.size();
    shapes->resize(n);
    long long ctas = 0;
    for (size_t i = 0; i < n; ++i) {
        (*shapes)[i] = {cs[i]->cluster, cs[i]->threads};
        ctas += cs[i]->cluster > 0 ? cs[i]->cluster : 1;
    }
    if (ctas <= sm_count) return;
    std::vector<double> work(n);
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) {
        work[i] = (double)steps[i] * model_mcs_us(cs[i]->p.Lx, cs[i]->p.Ly, cs[i]->cluster, cs[i]->threads);
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
    long long left = keep_longest ? sm_count : 0;
    for (size_t i : order) {
        klmc_ctx *c = cs[i];
        const int own = c->cluster > 0 ? c->cluster : 1;
        if (own <= left || !c->auto_shape || c->cluster < 1) {
            if (own <= left) left -= own;
            continue;
        }
        int half = c->cluster > 1 ? c->cluster / 2 : 1;
        if (resident_smem_bytes(c->p.Lx, c->p.Ly, half) > (size_t)resident_max_smem_bytes())
            half = c->cluster;
        (*shapes)[i] = {half, 128};
    }
}

klmc_status klmc::host::create_async(klmc_ctx **out, const klmc_params *p)
{
    return create_one(out, p, nullptr, false);
}

void klmc::host::destroy(klmc_ctx *c)
{
    free_all(c);
    delete c;
}

size_t klmc::host::device_bytes(const klmc_params *p)
{
    const size_t W = (size_t)(p->Lx + 31) / 32;
    const size_t lat = p->packing == KLMC_PACK_BYTE ? (size_t)((p->Lx + 15) / 16 * 16) * (size_t)p->Ly
                                                    : (W + 3) / 4 * 16 * (size_t)p->Ly;
    return lat + kStateSlots * sizeof(long long) + init_scratch_bytes() + 3 * 256;
}

extern "C" {

klmc_status klmc_params_default(klmc_params *p)
{
    if (!p) return fail(KLMC_EINVAL, "params is NULL");
    memset(p, 0, sizeof(*p));
    p->Lx = p->Ly = 64;
    p->geometry = KLMC_TRI6;
    p->boundary = KLMC_PERIODIC;
    p->packing = KLMC_PACK_BIT;
    p->n_A = -1;
    p->fraction_A = 0.5;
    p->omega_over_kT = 0.0;
    p->seed = 1;
    return KLMC_OK;
}

klmc_status klmc_create(klmc_ctx **out, int32_t L, double composition_A, double omega_over_kT,
                        uint64_t seed)
{
    if (!out) return fail(KLMC_EINVAL, "out is NULL");
    klmc_params p;
    klmc_params_default(&p);
    p.Lx = p.Ly = L;
    p.fraction_A = composition_A;
    p.omega_over_kT = omega_over_kT;
    p.seed = seed;
    return create_one(out, &p, nullptr, true, true);
}

klmc_status klmc_create_ex(klmc_ctx **out, const klmc_params *p)
{
    if (!out) return fail(KLMC_EINVAL, "out is NULL");
    return create_one(out, p, nullptr, true, true);
}

klmc_status klmc_sweep(klmc_ctx *c, int64_t n_mcs) { return sweep_one(c, n_mcs, 0, nullptr); }

klmc_status klmc_sweep_traced(klmc_ctx *c, int64_t n_mcs, int64_t trace_every, int64_t *dev_trace)
{
    if (trace_every <= 0) return fail(KLMC_EINVAL, "trace_every must be > 0");
    return sweep_one(c, n_mcs, trace_every, dev_trace);
}

klmc_status klmc_energy(klmc_ctx *c, int64_t *n_unlike, double *energy_over_kT)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    long long v[kStateSlots];
    KLMC_CUDA(cudaMemcpyAsync(v, c->state, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    if (v[kFault]) return fail(KLMC_ETIMEOUT, "a tiled sweep launch gave up waiting for its row copies");
    if (n_unlike) *n_unlike = v[kNUnlike];
    if (energy_over_kT) *energy_over_kT = c->p.omega_over_kT * (double)v[kNUnlike];
    return KLMC_OK;
}

klmc_status klmc_ffn_device(klmc_ctx *c, int64_t sample, int64_t *dev_similar)
{
    if (!c || !dev_similar) return fail(KLMC_EINVAL, "NULL argument");
    if (sample < 0) return fail(KLMC_EINVAL, "sample must be >= 0");
    KLMC_CUDA(launch_ffn(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->p.geometry, c->helical,
                         c->job.key0, c->job.key1, sample, (long long *)dev_similar, c->stream));
    return KLMC_OK;
}

klmc_status klmc_ffn(klmc_ctx *c, int64_t sample, int64_t *similar, double *exact)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (sample < 0) return fail(KLMC_EINVAL, "sample must be >= 0");
    long long v[2] = {0, 0};  // n_unlike, similar
    if (similar) {
        klmc_status st = klmc_ffn_device(c, sample, (int64_t *)(c->state + kFfn));
        if (st != KLMC_OK) return st;
        KLMC_CUDA(cudaMemcpyAsync(&v[1], c->state + kFfn, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    }
    KLMC_CUDA(cudaMemcpyAsync(&v[0], c->state + kNUnlike, sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    if (similar) *similar = v[1];
    if (exact) {
        const double B = (double)(c->p.geometry == KLMC_TRI6 ? 3 : 2) * (double)c->N;
        *exact = 1.0 - (double)v[0] / B;
    }
    return KLMC_OK;
}

klmc_status klmc_snapshot(klmc_ctx *c, int32_t W, int32_t H, int32_t S, uint8_t *dev_image, uint8_t *dev_mask)
{
    if (!c || !dev_image || !dev_mask) return fail(KLMC_EINVAL, "NULL argument");
    if (W < 1 || H < 1 || S < 1 || S > 64) return fail(KLMC_EINVAL, "need W, H >= 1 and 1 <= S <= 64");
    if ((long long)W * H > 2147483647LL) return fail(KLMC_EINVAL, "W*H must be <= 2^31 - 1");
    {
        // sample positions are exact in 64-bit integers: (2WS) max(U, Ly) and (2HS) Ly stay below 2^62
        const double U = 2.0 * c->p.Lx + c->p.Ly - 1.0, m = U > c->p.Ly ? U : (double)c->p.Ly;
        if (2.0 * W * S * m > 4.0e18 || 2.0 * H * S * (double)c->p.Ly > 4.0e18)
            return fail(KLMC_EINVAL, "image too large for exact sample positions");
    }
    KLMC_CUDA(launch_snapshot(c->lat, c->job.packing, c->pitch, c->p.Lx, c->p.Ly, W, H, S, dev_image, dev_mask,
                              c->stream));
    return KLMC_OK;
}

klmc_status klmc_image_ffn(klmc_ctx *c, const uint8_t *dev_image, const uint8_t *dev_mask, int32_t W, int32_t H,
                           int32_t delta, int64_t sample, int64_t *similar, int64_t *pixels)
{
    if (!c || !dev_image || !dev_mask) return fail(KLMC_EINVAL, "NULL argument");
    if (W < 1 || H < 1 || (long long)W * H > 2147483647LL) return fail(KLMC_EINVAL, "bad image size");
    if (delta < 0 || sample < 0) return fail(KLMC_EINVAL, "delta and sample must be >= 0");
    KLMC_CUDA(launch_image_ffn(dev_image, dev_mask, W, H, delta, c->job.key0, c->job.key1, sample,
                               c->state + kFfn, c->stream));
    long long v[2];
    KLMC_CUDA(cudaMemcpyAsync(v, c->state + kFfn, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    if (similar) *similar = v[0];
    if (pixels) *pixels = v[1];
    return KLMC_OK;
}

klmc_status klmc_energy_recount(klmc_ctx *c, int64_t *n_unlike)
{
    if (!c || !n_unlike) return fail(KLMC_EINVAL, "NULL argument");
    KLMC_CUDA(launch_recount(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->p.geometry,
                             c->state + kScratch0, c->stream, c->helical));
    long long v = 0;
    KLMC_CUDA(cudaMemcpyAsync(&v, c->state + kScratch0, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    *n_unlike = v;
    return KLMC_OK;
}

klmc_status klmc_cluster_histogram_device(klmc_ctx *c, int32_t species, int64_t *dev_sizes,
                                          int64_t *dev_counts, int64_t capacity,
                                          int64_t *dev_n_distinct)
{
    if (!c || !dev_n_distinct) return fail(KLMC_EINVAL, "NULL argument");
    if (species != 0 && species != 1) return fail(KLMC_EINVAL, "species must be 0 (B) or 1 (A)");
    if (capacity < 0 || (capacity > 0 && (!dev_sizes || !dev_counts)))
        return fail(KLMC_EINVAL, "bad output buffers");
    klmc_status st = ensure_clusters(c);
    if (st != KLMC_OK) return st;
    KLMC_CUDA(launch_cluster_histogram(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch,
                                       c->p.geometry, species, c->cs, (long long *)dev_sizes,
                                       (long long *)dev_counts, capacity,
                                       (long long *)dev_n_distinct, c->stream, c->helical));
    return KLMC_OK;
}

klmc_status klmc_cluster_histogram(klmc_ctx *c, int32_t species, int64_t *sizes, int64_t *counts,
                                   int64_t capacity, int64_t *n_distinct)
{
    if (!c || !n_distinct) return fail(KLMC_EINVAL, "NULL argument");
    if (capacity < 0 || (capacity > 0 && (!sizes || !counts)))
        return fail(KLMC_EINVAL, "bad output buffers");
    klmc_status st = ensure_clusters(c);
    if (st != KLMC_OK) return st;
    long long *dsz = c->hist_out, *dct = c->hist_out + c->hist_cap, *dn = c->hist_out + 2 * c->hist_cap;
    st = klmc_cluster_histogram_device(c, species, (int64_t *)dsz, (int64_t *)dct, c->hist_cap,
                                       (int64_t *)dn);
    if (st != KLMC_OK) return st;
    long long n = 0;
    KLMC_CUDA(cudaMemcpyAsync(&n, dn, sizeof(n), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    if (n > c->hist_cap) return fail(KLMC_ECUDA, "internal: more distinct sizes than the bound");
    if (n > capacity) {
        *n_distinct = n;
        return fail(KLMC_ETRUNC, "capacity " + std::to_string(capacity) + " < " + std::to_string(n));
    }
    if (n > 0) {
        KLMC_CUDA(cudaMemcpyAsync(sizes, dsz, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
        KLMC_CUDA(cudaMemcpyAsync(counts, dct, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
        KLMC_CUDA(cudaStreamSynchronize(c->stream));
    }
    *n_distinct = n;
    return KLMC_OK;
}

// Average cluster sizes of a sparse histogram: the exact sums n_clusters = sum c,
// n_sites = sum s c and sum_sq = sum s^2 c in int64 (checked against overflow),
// then one FP64 division each.
klmc_status klmc_histogram_averages(const int64_t *sizes, const int64_t *counts, int64_t n,
                                    double *number_avg, double *weight_avg)
{
    if (n < 0 || (n > 0 && (!sizes || !counts))) return fail(KLMC_EINVAL, "bad histogram arrays");
    long long clusters = 0, sites = 0, sq = 0;
    for (int64_t k = 0; k < n; ++k) {
        const long long s = sizes[k], cnt = counts[k];
        if (s < 0 || cnt < 0) return fail(KLMC_EINVAL, "negative cluster size or count");
        long long sc = 0, ssc = 0;
        if (__builtin_mul_overflow(s, cnt, &sc) || __builtin_mul_overflow(sc, s, &ssc) ||
            __builtin_add_overflow(clusters, cnt, &clusters) || __builtin_add_overflow(sites, sc, &sites) ||
            __builtin_add_overflow(sq, ssc, &sq))
            return fail(KLMC_EINVAL, "histogram sums exceed int64");
    }
    const double na = clusters > 0 ? (double)sites / (double)clusters : 0.0;
    const double wa = sites > 0 ? (double)sq / (double)sites : 0.0;
    if (number_avg) *number_avg = na;
    if (weight_avg) *weight_avg = wa;
    return KLMC_OK;
}

klmc_status klmc_cluster_averages(klmc_ctx *c, int32_t species, double *number_avg, double *weight_avg)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (species != 0 && species != 1) return fail(KLMC_EINVAL, "species must be 0 (B) or 1 (A)");
    klmc_status st = ensure_clusters(c);
    if (st != KLMC_OK) return st;
    std::vector<int64_t> sizes((size_t)c->hist_cap), counts((size_t)c->hist_cap);
    int64_t n = 0;
    st = klmc_cluster_histogram(c, species, sizes.data(), counts.data(), c->hist_cap, &n);
    if (st != KLMC_OK) return st;
    return klmc_histogram_averages(sizes.data(), counts.data(), n, number_avg, weight_avg);
}

klmc_status klmc_test_copy_shortfall(klmc_ctx *c, int32_t bytes)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (bytes < 0) return fail(KLMC_EINVAL, "bytes must be >= 0");
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    c->job.copy_shortfall = bytes;
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.second);  // they hold the old value
    c->graphs.clear();
    return KLMC_OK;
}

klmc_status klmc_get_counters(klmc_ctx *c, klmc_counters *out)
{
    if (!c || !out) return fail(KLMC_EINVAL, "NULL argument");
    long long v[kStateSlots];
    KLMC_CUDA(cudaMemcpyAsync(v, c->state, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    if (v[kFault]) return fail(KLMC_ETIMEOUT, "a tiled sweep launch gave up waiting for its row copies");
    out->sweeps = c->sweep;
    out->attempts = v[kAttempts];
    out->unlike = v[kUnlike];
    out->draws = v[kDraws];
    out->accepts = v[kAccepts];
    return KLMC_OK;
}

klmc_status klmc_get_lattice(klmc_ctx *c, uint8_t *host_out, int64_t n)
{
    if (!c || !host_out) return fail(KLMC_EINVAL, "NULL argument");
    if (n != c->N) return fail(KLMC_EINVAL, "n must equal Lx*Ly");
    klmc_status st = ensure_bytes(c);
    if (st != KLMC_OK) return st;
    KLMC_CUDA(launch_unpack(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->dbytes, c->stream));
    KLMC_CUDA(cudaMemcpyAsync(host_out, c->dbytes, (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    return KLMC_OK;
}

klmc_status klmc_set_lattice(klmc_ctx *c, const uint8_t *host_in, int64_t n, int64_t sweep_index)
{
    if (!c || !host_in) return fail(KLMC_EINVAL, "NULL argument");
    if (n != c->N) return fail(KLMC_EINVAL, "n must equal Lx*Ly");
    if (sweep_index < 0) return fail(KLMC_EINVAL, "sweep_index must be >= 0");
    for (long long i = 0; i < n; ++i)
        if (host_in[i] > 1) return fail(KLMC_EINVAL, "lattice bytes must be 0 or 1");
    klmc_status st = ensure_bytes(c);
    if (st != KLMC_OK) return st;
    KLMC_CUDA(cudaMemcpyAsync(c->dbytes, host_in, (size_t)n, cudaMemcpyHostToDevice, c->stream));
    KLMC_CUDA(launch_pack(c->dbytes, c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->stream));
    KLMC_CUDA(cudaMemsetAsync(c->state, 0, kStateSlots * sizeof(long long), c->stream));
    KLMC_CUDA(launch_recount(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->p.geometry,
                             c->state + kNUnlike, c->stream, c->helical));
    KLMC_CUDA(launch_count_A(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->state + kScratch0,
                             c->stream));
    long long nA = 0;
    KLMC_CUDA(cudaMemcpyAsync(&nA, c->state + kScratch0, sizeof(nA), cudaMemcpyDeviceToHost, c->stream));
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    c->nA = nA;
    c->nA_on_device = false;
    c->sweep = sweep_index;
    return KLMC_OK;
}

klmc_status klmc_set_lattice_device(klmc_ctx *c, const uint8_t *dev_in, int64_t n,
                                    int64_t sweep_index)
{
    if (!c || !dev_in) return fail(KLMC_EINVAL, "NULL argument");
    if (n != c->N) return fail(KLMC_EINVAL, "n must equal Lx*Ly");
    if (sweep_index < 0) return fail(KLMC_EINVAL, "sweep_index must be >= 0");
    KLMC_CUDA(launch_pack(dev_in, c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->stream));
    KLMC_CUDA(cudaMemsetAsync(c->state, 0, kStateSlots * sizeof(long long), c->stream));
    KLMC_CUDA(launch_recount(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->p.geometry,
                             c->state + kNUnlike, c->stream, c->helical));
    KLMC_CUDA(launch_count_A(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->state + kNA,
                             c->stream));
    c->nA_on_device = true;
    c->sweep = sweep_index;
    return KLMC_OK;
}

klmc_status klmc_get_shape(klmc_ctx *c, int32_t *Lx, int32_t *Ly, int32_t *geometry, int64_t *n_A)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (n_A && c->nA_on_device) {
        long long v = 0;
        KLMC_CUDA(cudaMemcpyAsync(&v, c->state + kNA, sizeof(v), cudaMemcpyDeviceToHost, c->stream));
        KLMC_CUDA(cudaStreamSynchronize(c->stream));
        c->nA = v;
        c->nA_on_device = false;
    }
    if (Lx) *Lx = c->p.Lx;
    if (Ly) *Ly = c->p.Ly;
    if (geometry) *geometry = c->p.geometry;
    if (n_A) *n_A = c->nA;
    return KLMC_OK;
}

klmc_status klmc_autotune(klmc_ctx *c, int32_t probe_sweeps, int32_t *cluster, int32_t *threads)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (probe_sweeps < 1) return fail(KLMC_EINVAL, "probe_sweeps must be >= 1");
    if (c->owner) return fail(KLMC_ESTATE, "replica views are tuned with their batch");
    klmc_status st = autotune(c, probe_sweeps);
    if (st != KLMC_OK) return st;
    if (cluster) *cluster = c->cluster;
    if (threads) *threads = c->threads;
    return KLMC_OK;
}

klmc_status klmc_set_packing(klmc_ctx *c, int32_t packing)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (packing != KLMC_PACK_BIT && packing != KLMC_PACK_BYTE)
        return fail(KLMC_EINVAL, "packing must be KLMC_PACK_BIT or KLMC_PACK_BYTE");
    if (c->owner) return fail(KLMC_ESTATE, "a replica view's store belongs to its batch");
    return convert_store(c, packing);
}

klmc_status klmc_get_packing(klmc_ctx *c, int32_t *packing)
{
    if (!c || !packing) return fail(KLMC_EINVAL, "NULL argument");
    *packing = c->job.packing;
    return KLMC_OK;
}

klmc_status klmc_get_launch(klmc_ctx *c, int32_t *cluster, int32_t *threads_per_cta)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    if (cluster) *cluster = c->cluster;
    if (threads_per_cta) *threads_per_cta = c->threads;
    return KLMC_OK;
}

klmc_status klmc_get_plan(klmc_ctx *c, int32_t *phases_per_exchange)
{
    if (!c || !phases_per_exchange) return fail(KLMC_EINVAL, "NULL argument");
    if (c->cluster > 0) {
        *phases_per_exchange = c->helical ? helical_resident_block(c->p.Lx, c->p.Ly, c->cluster)
                                          : resident_block_phases(c->p.Lx, c->p.Ly, c->cluster);
        return KLMC_OK;
    }
    if (c->helical) {
        *phases_per_exchange = 1;
        return KLMC_OK;
    }
    int dev = 0, sms = 0;
    KLMC_CUDA(cudaGetDevice(&dev));
    KLMC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    *phases_per_exchange = tiled_plan(c->p.Lx, c->p.Ly, sms).K;
    return KLMC_OK;
}

klmc_status klmc_synchronize(klmc_ctx *c)
{
    if (!c) return fail(KLMC_EINVAL, "ctx is NULL");
    KLMC_CUDA(cudaStreamSynchronize(c->stream));
    return KLMC_OK;
}

klmc_status klmc_destroy(klmc_ctx *c)
{
    if (!c) return KLMC_OK;
    if (c->owner) return fail(KLMC_ESTATE, "replica views are freed by klmc_batch_destroy");
    free_all(c);
    delete c;
    return KLMC_OK;
}

klmc_status klmc_batch_create(klmc_batch **out, const klmc_params *reps, int32_t n)
{
    if (!out || !reps || n <= 0) return fail(KLMC_EINVAL, "bad batch arguments");
    klmc_batch *b = new (std::nothrow) klmc_batch();
    if (!b) return fail(KLMC_ENOMEM, "host allocation failed");
    b->stream = (cudaStream_t)reps[0].stream;
    for (int i = 0; i < n; ++i) {
        klmc_params p = reps[i];
        p.stream = reps[0].stream;
        klmc_ctx *c = nullptr;
        klmc_status st = create_one(&c, &p, b);
        if (st == KLMC_OK && c->helical && c->cluster < 0)
            st = fail(KLMC_EINVAL, "helical lattice whose bands are too thin for the resident sweep: it runs "
                                   "one launch per iteration, on its own handle");
        else if (st == KLMC_OK && c->cluster < 0)
            st = fail(KLMC_EINVAL, "lattice too large for a batched resident launch");
        if (st == KLMC_OK && !c->helical) st = check_resident(c, c->cluster);
        if (st != KLMC_OK) {
            std::string msg = "replica " + std::to_string(i) + ": " + g_err;
            if (c) {
                c->owner = nullptr;
                klmc_destroy(c);
            }
            klmc_batch_destroy(b);
            return fail(st, msg);
        }
        b->reps.push_back(c);
    }
    klmc_ctx *m = b->reps[0];
    b->mem_owner = m;
    b->djobs = (SweepJob *)dev_alloc(m, sizeof(SweepJob) * (size_t)n);
    b->dcalls = (SweepCall *)dev_alloc(m, sizeof(SweepCall) * (size_t)n);
    b->dmap = (int *)dev_alloc(m, sizeof(int) * (size_t)n);
    if (!b->djobs || !b->dcalls || !b->dmap) {
        klmc_batch_destroy(b);
        return fail(KLMC_ENOMEM, "device allocation of the batch tables failed");
    }
    std::vector<SweepJob> jobs(n);
    for (int i = 0; i < n; ++i) jobs[i] = b->reps[i]->job;
    cudaError_t e = cudaMemcpyAsync(b->djobs, jobs.data(), sizeof(SweepJob) * (size_t)n,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        klmc_batch_destroy(b);
        return fail(KLMC_ECUDA, std::string("batch upload: ") + cudaGetErrorString(e));
    }
    b->hcalls.resize(n);
    for (klmc_ctx *c : b->reps) b->last_shape.push_back({c->cluster, c->threads});
    e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    if (e != cudaSuccess) {
        klmc_batch_destroy(b);
        return fail(KLMC_ECUDA, std::string("batch events: ") + cudaGetErrorString(e));
    }
    *out = b;
    return KLMC_OK;
}

klmc_status klmc_batch_sweep(klmc_batch *b, const int64_t *n_mcs)
{
    if (!b || !n_mcs) return fail(KLMC_EINVAL, "NULL argument");
    const int n = (int)b->reps.size();
    std::vector<klmc_ctx *> active;
    std::vector<int64_t> active_steps;
    std::vector<int> index, helical;
    for (int i = 0; i < n; ++i) {
        if (n_mcs[i] < 0) return fail(KLMC_EINVAL, "n_mcs entries must be >= 0");
        klmc_ctx *c = b->reps[i];
        SweepCall &call = b->hcalls[i];
        call.sweep0 = c->sweep;
        call.n_mcs = n_mcs[i];
        call.trace = nullptr;
        call.trace_every = 0;
        if (n_mcs[i] > 0 && c->helical) {
            helical.push_back(i);
        } else if (n_mcs[i] > 0) {
            active.push_back(c);
            active_steps.push_back(n_mcs[i]);
            index.push_back(i);
        }
    }
    if (active.empty() && helical.empty()) return KLMC_OK;
    KLMC_CUDA(cudaEventRecord(b->fork, b->stream));
    // Helical replicas: the resident helical sweep, one launch each on a stream of its
    // own (key (-1 - i, 512) in the group-stream map), overlapping the others; joined
    // back to the batch stream after the other launches are enqueued.
    std::vector<cudaEvent_t> joins;
    for (int i : helical) {
        const std::pair<int, int> key(-1 - i, 512);
        auto it = b->group_streams.find(key);
        if (it == b->group_streams.end()) {
            cudaStream_t gs;
            cudaEvent_t ge;
            KLMC_CUDA(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
            KLMC_CUDA(cudaEventCreateWithFlags(&ge, cudaEventDisableTiming));
            it = b->group_streams.emplace(key, std::make_pair(gs, ge)).first;
        }
        klmc_ctx *c = b->reps[i];
        b->last_shape[i] = {c->cluster, 512};
        KLMC_CUDA(cudaStreamWaitEvent(it->second.first, b->fork, 0));
        KLMC_CUDA(launch_helical_resident(c->job, b->hcalls[i], c->cluster, it->second.first));
        KLMC_CUDA(cudaEventRecord(it->second.second, it->second.first));
        joins.push_back(it->second.second);
    }
    if (active.empty()) {
        for (cudaEvent_t ev : joins) KLMC_CUDA(cudaStreamWaitEvent(b->stream, ev, 0));
        for (int i = 0; i < n; ++i) b->reps[i]->sweep += n_mcs[i];
        return KLMC_OK;
    }
    // One launch per launch shape, each on its own stream (the launches overlap on
    // the GPU), larger lattices first inside a launch.
    std::vector<std::pair<int, int>> shapes;
    klmc::host::choose_shapes(active, active_steps, b->sm_count, false, &shapes);
    std::map<std::pair<int, int>, std::vector<int>> groups;
    for (size_t k = 0; k < active.size(); ++k) {
        groups[shapes[k]].push_back(index[k]);
        b->last_shape[index[k]] = shapes[k];
    }
    std::vector<int> hmap;
    hmap.reserve(active.size());
    for (auto &g : groups) {
        std::stable_sort(g.second.begin(), g.second.end(),
                         [&](int a, int c) { return b->reps[a]->N > b->reps[c]->N; });
        hmap.insert(hmap.end(), g.second.begin(), g.second.end());
    }
    KLMC_CUDA(cudaMemcpyAsync(b->dcalls, b->hcalls.data(), sizeof(SweepCall) * (size_t)n,
                              cudaMemcpyHostToDevice, b->stream));
    KLMC_CUDA(cudaMemcpyAsync(b->dmap, hmap.data(), sizeof(int) * hmap.size(), cudaMemcpyHostToDevice,
                              b->stream));
    KLMC_CUDA(cudaEventRecord(b->fork, b->stream));  // after the tables' upload
    int offset = 0;
    for (auto &g : groups) {
        auto it = b->group_streams.find(g.first);
        if (it == b->group_streams.end()) {
            cudaStream_t gs;
            cudaEvent_t ge;
            KLMC_CUDA(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
            KLMC_CUDA(cudaEventCreateWithFlags(&ge, cudaEventDisableTiming));
            it = b->group_streams.emplace(g.first, std::make_pair(gs, ge)).first;
        }
        size_t smem = 0;
        for (int i : g.second) {
            klmc_status st = check_resident(b->reps[i], g.first.first);
            if (st != KLMC_OK) return st;
            const size_t sm = resident_smem_bytes(b->reps[i]->p.Lx, b->reps[i]->p.Ly, g.first.first);
            if (sm > smem) smem = sm;
        }
        KLMC_CUDA(cudaStreamWaitEvent(it->second.first, b->fork, 0));
        KLMC_CUDA(launch_resident_sweep(b->djobs, b->dcalls, b->dmap + offset, (int)g.second.size(),
                                        g.first.first, g.first.second, smem, it->second.first));
        KLMC_CUDA(cudaEventRecord(it->second.second, it->second.first));
        KLMC_CUDA(cudaStreamWaitEvent(b->stream, it->second.second, 0));
        offset += (int)g.second.size();
    }
    for (cudaEvent_t ev : joins) KLMC_CUDA(cudaStreamWaitEvent(b->stream, ev, 0));
    for (int i = 0; i < n; ++i) b->reps[i]->sweep += n_mcs[i];
    return KLMC_OK;
}

klmc_status klmc_batch_get_launch(klmc_batch *b, int32_t i, int32_t *cluster, int32_t *threads_per_cta)
{
    if (!b) return fail(KLMC_EINVAL, "NULL batch");
    if (i < 0 || i >= (int)b->reps.size()) return fail(KLMC_EINVAL, "replica index out of range");
    if (cluster) *cluster = b->last_shape[i].first;
    if (threads_per_cta) *threads_per_cta = b->last_shape[i].second;
    return KLMC_OK;
}

klmc_status klmc_batch_replica(klmc_batch *b, int32_t i, klmc_ctx **view)
{
    if (!b || !view) return fail(KLMC_EINVAL, "NULL argument");
    if (i < 0 || i >= (int32_t)b->reps.size()) return fail(KLMC_EINVAL, "replica index out of range");
    *view = b->reps[i];
    return KLMC_OK;
}

klmc_status klmc_batch_cluster_histogram_device(klmc_batch *b, int32_t species, int64_t *dev_sizes,
                                                int64_t *dev_counts, int64_t capacity,
                                                int64_t *dev_n_distinct)
{
    if (!b || !dev_n_distinct) return fail(KLMC_EINVAL, "NULL argument");
    if (species != 0 && species != 1) return fail(KLMC_EINVAL, "species must be 0 (B) or 1 (A)");
    if (capacity < 0 || (capacity > 0 && (!dev_sizes || !dev_counts)))
        return fail(KLMC_EINVAL, "bad output buffers");
    const int n = (int)b->reps.size();
    for (int i = 0; i < n; ++i) {  // scratch first, on the batch stream
        klmc_status st = ensure_clusters(b->reps[i]);
        if (st != KLMC_OK) return st;
    }
    const int ns = n < kHistStreams ? n : kHistStreams;
    while ((int)b->hist_streams.size() < ns) {
        cudaStream_t hs;
        cudaEvent_t he;
        KLMC_CUDA(cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking));
        KLMC_CUDA(cudaEventCreateWithFlags(&he, cudaEventDisableTiming));
        b->hist_streams.push_back({hs, he});
    }
    KLMC_CUDA(cudaEventRecord(b->fork, b->stream));
    for (int k = 0; k < ns; ++k) KLMC_CUDA(cudaStreamWaitEvent(b->hist_streams[k].first, b->fork, 0));
    for (int i = 0; i < n; ++i) {
        klmc_ctx *c = b->reps[i];
        const size_t off = (size_t)i * (size_t)capacity;
        KLMC_CUDA(launch_cluster_histogram(c->lat, c->job.packing, c->p.Lx, c->p.Ly, c->pitch, c->p.geometry,
                                           species, c->cs, capacity ? (long long *)dev_sizes + off : nullptr,
                                           capacity ? (long long *)dev_counts + off : nullptr, capacity,
                                           (long long *)dev_n_distinct + i, b->hist_streams[i % ns].first,
                                           c->helical));
    }
    for (int k = 0; k < ns; ++k) {
        KLMC_CUDA(cudaEventRecord(b->hist_streams[k].second, b->hist_streams[k].first));
        KLMC_CUDA(cudaStreamWaitEvent(b->stream, b->hist_streams[k].second, 0));
    }
    return KLMC_OK;
}

klmc_status klmc_batch_destroy(klmc_batch *b)
{
    if (!b) return KLMC_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->group_streams) {
        cudaStreamSynchronize(g.second.first);
        cudaStreamDestroy(g.second.first);
        cudaEventDestroy(g.second.second);
    }
    for (auto &h : b->hist_streams) {
        cudaStreamSynchronize(h.first);
        cudaStreamDestroy(h.first);
        cudaEventDestroy(h.second);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    // The batch tables were allocated on reps[0]; free them with it, last.
    for (size_t i = b->reps.size(); i-- > 0;) {
        klmc_ctx *c = b->reps[i];
        free_all(c);
        delete c;
    }
    delete b;
    return KLMC_OK;
}

const char *klmc_status_str(klmc_status s)
{
    switch (s) {
    case KLMC_OK: return "KLMC_OK";
    case KLMC_EINVAL: return "KLMC_EINVAL";
    case KLMC_ENOMEM: return "KLMC_ENOMEM";
    case KLMC_ECUDA: return "KLMC_ECUDA";
    case KLMC_ETIMEOUT: return "KLMC_ETIMEOUT";
    case KLMC_EBUSY: return "KLMC_EBUSY";
    case KLMC_ETRUNC: return "KLMC_ETRUNC";
    case KLMC_ESTATE: return "KLMC_ESTATE";
    case KLMC_ENODEV: return "KLMC_ENODEV";
    }
    return "KLMC_UNKNOWN";
}

const char *klmc_last_error(void) { return g_err.c_str(); }

}  // extern "C"
