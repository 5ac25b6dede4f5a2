// burr_noalloc.cu -- the bucket sort of one layer without any device memory
// allocation, for callers that cannot allocate device memory themselves or let
// a library do it: a process whose device memory is all handed to its own pool
// allocator (so a cudaMalloc from a library would fail or fragment it), a
// latency-critical loop that cannot afford the implicit device synchronisation
// and unpredictable latency of cudaMalloc/cudaFree, or code that must not run
// out of memory half-way through a pipeline.
//
// The sort's scratch (the scatter buffer and the digit and group counters) lives
// in one file-scope device array of fixed size.  Every GPU that loads the
// library holds this array until the process exits.  All calls share it and
// it keeps the contents of the last call, so calls whose work overlaps on the
// GPU (different streams, or different host threads) race on it: the caller
// must order them, e.g. by issuing them on one stream.
#include <cstring>
#include <string>

#include "burr_internal.cuh"

namespace {

constexpr uint64_t kNoAllocMaxKeys = BURR_NOALLOC_MAX_KEYS;
constexpr uint64_t kNoAllocMaxSlots = BURR_NOALLOC_MAX_SLOTS;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// burr::sort_scratch_bytes(kNoAllocMaxKeys, kNoAllocMaxSlots, 4): the scatter
// buffer of the keys (8 B) and values (<= 4 B), three arrays of pass-1 digit
// counters, and three arrays of per-group counters (groups of 64 buckets of at
// least 64 slots).
constexpr size_t kDigits = 1024 + 1;
constexpr size_t kGroups = ((kNoAllocMaxSlots - 64 + 128) / 64 + 63) / 64 + 1 + 1;
constexpr size_t kScratchBytes = align256(kNoAllocMaxKeys * 8) + align256(kNoAllocMaxKeys * 4) +
                                 3 * align256(kDigits * 4) + 3 * align256(kGroups * 4);

static __device__ __align__(256) unsigned char g_sort_scratch[kScratchBytes];

// Device address of g_sort_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the kernels must be given this
// address instead.  It is looked up on every call (a table lookup that
// allocates nothing), so a context rebuilt after cudaDeviceReset gets its own
// array's address rather than a stale one; the first call on a device also
// loads the library's device code there.
int scratch_on_current_device(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return burr::set_error(BURR_ERR_CUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess || !p)
        return burr::set_error(BURR_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    *out = p;
    return BURR_OK;
}

}  // namespace

extern "C" {

int burr_stage_sort_noalloc(const uint64_t *d_keys, const void *d_values, uint64_t n, uint32_t r, uint64_t seed,
                            uint32_t layer_index, uint64_t m, uint64_t *d_sorted_keys, void *d_sorted_values,
                            uint32_t *d_bucket_start, void *stream) {
    using namespace burr;
    if (r < 1 || r > 32) return set_error(BURR_ERR_INVALID, "r outside [1,32]");
    if (n > kNoAllocMaxKeys)
        return set_error(BURR_ERR_INVALID, ("n = " + std::to_string(n) + " exceeds the allocation-free limit of " +
                                            std::to_string(kNoAllocMaxKeys) + " keys; use burr_stage_sort").c_str());
    if (m < kW || m % 64 || m > kNoAllocMaxSlots)
        return set_error(BURR_ERR_INVALID, ("m must be a multiple of 64 in [64, " +
                                            std::to_string(kNoAllocMaxSlots) + "] (allocation-free limit)").c_str());
    if (n && (!d_keys || !d_values || !d_sorted_keys || !d_sorted_values))
        return set_error(BURR_ERR_INVALID, "NULL argument");
    if (!d_bucket_start) return set_error(BURR_ERR_INVALID, "NULL bucket offsets");
    void *scratch = nullptr;
    int rc = scratch_on_current_device(&scratch);
    if (rc) return rc;
    const uint32_t vb = r <= 8 ? 1u : (r <= 16 ? 2u : 4u);
    if (sort_scratch_bytes(n, m, vb) > kScratchBytes)
        return set_error(BURR_ERR_INTERNAL, "sort scratch larger than the static array");
    LayerDesc L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    L.m = m;
    L.range = m - kW + 1;
    L.sigma = layer_seed(seed, layer_index);
    L.B = 128;
    L.nb = (m - kW + L.B) / L.B;
    L.r = r;
    // launch_sort zeroes the bin counters it accumulates into before use; every
    // other scratch word it reads was written earlier in the same call.
    cudaError_t e = launch_sort(L, vb, d_keys, d_values, d_sorted_keys, d_sorted_values, d_bucket_start, scratch,
                                nullptr, (cudaStream_t)stream, true);
    if (e != cudaSuccess) return set_error(BURR_ERR_CUDA, (std::string("sort: ") + cudaGetErrorString(e)).c_str());
    return BURR_OK;
}

}  // extern "C"
