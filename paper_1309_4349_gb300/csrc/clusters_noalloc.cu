// clusters_noalloc.cu -- the cluster-size histogram for callers that cannot
// allocate device memory.
//
// Some callers have no way to call cudaMalloc: a host framework that owns every
// byte of device memory under a fixed budget and offers no allocator hook, or a
// latency-bound loop that shares the GPU with other streams and cannot accept the
// implicit device-wide synchronisation of cudaMalloc/cudaFree.  They pass their
// own lattice and output buffers; this entry point runs the same kernels as
// klmc_cluster_histogram_device, with the labelling scratch (parent and size
// arrays, size histogram, occupied-size bitmap) taken from a fixed array in this
// file instead of from an allocation.
//
// The array is a file-scope __device__ variable.  With lazy module loading (the
// CUDA default) a device holds it (about 12.6 MB) from the first call of this
// entry point in its context until the process exits; that first call loads the
// module, which may synchronise the device and may fail with KLMC_ECUDA when
// device memory is short, so callers make it during set-up, outside any
// latency-bound loop and outside stream capture.  Every call shares the array
// and it keeps the last call's contents; the parts that must start at zero are
// cleared by each call.  Two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array.  The lattice is read
// with periodic boundaries (the paper's lattice model); helical lattices take
// klmc_cluster_histogram_device.
#include <string>

#include "klmc.h"
#include "klmc_internal.h"

namespace {

constexpr long long kMaxSites = KLMC_NOALLOC_MAX_SITES;

constexpr unsigned long long align256(unsigned long long v) { return (v + 255ull) & ~255ull; }

// Same carve as cluster_scratch_carve for N = n_species_max = kMaxSites.
constexpr unsigned long long kScratchBytes =
    2 * align256(4ull * kMaxSites) + align256(4ull * (kMaxSites + 1)) +
    align256(4ull * ((kMaxSites + 1 + 31) / 32));

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

klmc_status fail(klmc_status s, const std::string &msg)
{
    klmc::set_last_error(msg.c_str());  // reported by klmc_last_error()
    return s;
}

// Device address of g_noalloc_scratch in the current device's context.  In host
// code the symbol itself is only a host-side stand-in, never a device address.
// It is resolved on every call instead of being cached: a cached address would
// be stale after cudaDeviceReset or in another context of the same device.  The
// first call in a context loads this file's module, which reserves the array.
klmc_status scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return fail(KLMC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = p;
    return KLMC_OK;
}

}  // namespace

extern "C" klmc_status klmc_cluster_histogram_noalloc(const void *dev_lattice, int32_t packing,
                                                      int32_t Lx, int32_t Ly, int32_t pitch,
                                                      int32_t geometry, int32_t species,
                                                      int64_t *dev_sizes, int64_t *dev_counts,
                                                      int64_t capacity, int64_t *dev_n_distinct,
                                                      void *stream)
{
    if (!dev_lattice || !dev_n_distinct) return fail(KLMC_EINVAL, "NULL lattice or count pointer");
    if (capacity < 0 || (capacity > 0 && (!dev_sizes || !dev_counts)))
        return fail(KLMC_EINVAL, "bad output buffers");
    if (packing != KLMC_PACK_BIT && packing != KLMC_PACK_BYTE)
        return fail(KLMC_EINVAL, "packing must be KLMC_PACK_BIT or KLMC_PACK_BYTE");
    if (geometry != KLMC_TRI6 && geometry != KLMC_SQ4) return fail(KLMC_EINVAL, "unknown geometry");
    if (species != 0 && species != 1) return fail(KLMC_EINVAL, "species must be 0 (B) or 1 (A)");
    if (Lx < 4 || Ly < 4) return fail(KLMC_EINVAL, "Lx and Ly must be >= 4");
    const long long N = (long long)Lx * Ly;
    if (N > kMaxSites)
        return fail(KLMC_EINVAL, "lattice of " + std::to_string(N) +
                                     " sites exceeds the fixed scratch of this entry point (" +
                                     std::to_string(kMaxSites) + " sites)");
    const int min_pitch = packing == KLMC_PACK_BIT ? (Lx + 31) / 32 : Lx;
    if (pitch < min_pitch) return fail(KLMC_EINVAL, "pitch smaller than one row");
    if (klmc::cluster_scratch_bytes(N, N) > kScratchBytes)
        return fail(KLMC_EINVAL, "internal: scratch layout exceeds the fixed array");

    void *base = nullptr;
    klmc_status st = scratch_address(&base);
    if (st != KLMC_OK) return st;
    klmc::ClusterScratch s;
    klmc::cluster_scratch_carve(base, N, N, &s);
    cudaStream_t cs = (cudaStream_t)stream;
    // The size histogram and occupied-size bitmap must start at zero.
    cudaError_t e = klmc::cluster_scratch_clear(s, cs);
    if (e == cudaSuccess)
        e = klmc::launch_cluster_histogram(dev_lattice, packing, Lx, Ly, pitch, geometry, species, s,
                                           (long long *)dev_sizes, (long long *)dev_counts,
                                           capacity, (long long *)dev_n_distinct, cs);
    if (e != cudaSuccess) return fail(KLMC_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return KLMC_OK;
}
