// burr_internal.cuh -- device helpers and launch descriptors shared by the
// CUDA translation units of libburr.so (never included by the oracle).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include "burr.h"

namespace burr {

constexpr uint32_t kW = 64;                       // ribbon width (Sec. 2)
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// error bits written by kernels into the build's device error word
constexpr uint32_t kErrRingOverflow = 1u;         // a pivot left the on-chip window
constexpr uint32_t kErrUnsolvable = 2u;           // base case: an equation was dependent
constexpr uint32_t kErrSortSlack = 4u;            // a sort bin of fixed capacity overflowed (sort again exactly)

// SplitMix64 output function (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t layer_seed(uint64_t seed, uint64_t index) {
    return mix64(seed ^ ((index + 1) * kGolden));
}

// Start slot in [0, range): floor(h * range / 2^64), range = m - w + 1.
__device__ __forceinline__ uint32_t start_slot(uint64_t key, uint64_t sigma, uint64_t range) {
    return (uint32_t)__umul64hi(mix64(key ^ sigma), range);
}

// The equation of a key: start slot and 64-bit coefficient row (bit 0 set).
__device__ __forceinline__ void equation(uint64_t key, uint64_t sigma, uint64_t range,
                                         uint32_t &start, uint64_t &coeff) {
    const uint64_t h = mix64(key ^ sigma);
    start = (uint32_t)__umul64hi(h, range);
    coeff = mix64(h + sigma) | 1ull;
}

// The build's sorted records carry h = mix64(key ^ sigma), the first hash
// round of the key in its layer, instead of the key: the later passes then
// need one multiply-high for the start slot and one round for the
// coefficients, and the key itself only where a row is bumped to the next
// layer.  mix64 is a bijection (xor-shifts and multiplications by odd
// constants), so h determines the key.
__host__ __device__ __forceinline__ uint32_t start_of_h(uint64_t h, uint64_t range) {
#ifdef __CUDA_ARCH__
    return (uint32_t)__umul64hi(h, range);
#else
    return (uint32_t)(((unsigned __int128)h * range) >> 64);
#endif
}
__host__ __device__ __forceinline__ uint64_t coeff_of_h(uint64_t h, uint64_t sigma) { return mix64(h + sigma) | 1ull; }

// Inverse of an odd 64-bit multiplier modulo 2^64 (Newton's iteration
// x <- x (2 - c x), which doubles the number of correct low bits; x = c is
// right to 3 bits for odd c).
__host__ __device__ constexpr uint64_t inverse_mod64(uint64_t c) {
    uint64_t x = c;
    for (int i = 0; i < 5; ++i) x *= 2 - c * x;
    return x;
}
// Inverse of x ^= x >> s.
__host__ __device__ __forceinline__ uint64_t unxorshift(uint64_t y, int s) {
    uint64_t x = y;
    for (int k = s; k < 64; k += s) x ^= y >> k;
    return x;
}
// The key of record h in the layer with seed sigma: mix64 undone step by step.
__host__ __device__ __forceinline__ uint64_t key_of_h(uint64_t h, uint64_t sigma) {
    constexpr uint64_t i2 = inverse_mod64(0x94D049BB133111EBull), i1 = inverse_mod64(0xBF58476D1CE4E5B9ull);
    uint64_t z = unxorshift(h, 31) * i2;
    z = unxorshift(z, 27) * i1;
    return unxorshift(z, 30) ^ sigma;
}

// One layer as the kernels see it.
struct LayerDesc {
    uint64_t n;          // equations (keys) in the layer
    uint64_t m;          // slots, multiple of 64, < 2^32
    uint64_t range;      // start positions m - w + 1
    uint64_t sigma;      // hash seed of the layer
    uint64_t nb;         // buckets
    uint64_t P;          // partition slots
    uint32_t K;          // partitions
    uint32_t r;          // value bits
    uint32_t B;          // bucket slots
    uint32_t fallback;   // 1: base case (no thresholds, failure = unsolvable)
    uint32_t levels[4];
    uint32_t forced_code;
    uint32_t vmask;      // (1 << r) - 1
    uint32_t mode;       // BURR_THRESH_2BIT or BURR_THRESH_1PLUS
    uint32_t window;     // pivots at or past bucket start + window leave the band's window (0 = the whole ring)
    uint32_t test_slack; // 1: the fixed-capacity sort bins get half their expected size (testing the exact redo)
    uint32_t part_lo;    // band and back-substitution launches cover partitions [part_lo, part_hi)
    uint32_t part_hi;    // (0: up to K); a shard of a sharded build owns such a range
    const uint32_t *cuts;  // device: first bucket of each partition, [K] = nb; nullptr: partition j at j*P
};

// End of the partition range a launch covers.
__host__ __device__ inline uint64_t part_end(const LayerDesc &L) { return L.part_hi ? L.part_hi : L.K; }

// First bucket of partition j (j <= K) and the slots it owns.
__host__ __device__ inline uint64_t part_bucket(const LayerDesc &L, uint64_t j) {
    if (L.cuts) return L.cuts[j];
    return j >= L.K ? L.nb : j * L.P / L.B;
}
__host__ __device__ inline uint64_t part_own_lo(const LayerDesc &L, uint64_t j) {
    return j == 0 ? 0 : part_bucket(L, j) * L.B + 64;
}
__host__ __device__ inline uint64_t part_own_hi(const LayerDesc &L, uint64_t j) {
    return j + 1 >= L.K ? L.m : part_bucket(L, j + 1) * L.B + 64;
}

// One structure's layer inside a batched build: its layer descriptor and
// where its data sits in the layer-wide arrays shared by the batch.
struct StructDesc {
    LayerDesc L;            // the structure's layer (K partitions of P slots)
    uint64_t key_base;      // its keys in the layer's input buffer: [key_base, key_base + L.n)
    uint64_t out_base;      // its bumped keys in the next layer's buffer start here
    uint64_t bucket_base;   // first global bucket (index into the bucket offsets)
    uint64_t group_base;    // first global sort group (64 buckets)
    uint64_t slot_base;     // first slot in the layer-wide band arrays
    uint64_t tw_base;       // first threshold word
    uint64_t z_base;        // first table word
    uint32_t part_base;     // first global partition (band and back-substitution)
    uint32_t ngroups;       // sort groups of the structure
};

// Device tables of a batched layer (all device pointers).
struct BatchView {
    const StructDesc *sd = nullptr;     // per structure
    const uint32_t *part_struct = nullptr;  // global partition -> structure
    const uint32_t *part_order = nullptr;   // launch order -> global partition (longest first); null: identity
    const uint32_t *group_struct = nullptr; // global sort group -> structure
    const uint32_t *tile_struct = nullptr;  // sort tile -> structure
    const uint64_t *tile_lo = nullptr;      // sort tile -> first key index
    uint32_t *fail = nullptr;               // per structure: base case dependent
    uint32_t nstruct = 0, nparts = 0, ngroups = 0, ntiles = 0;
    uint64_t nbuckets = 0;                  // global buckets
    uint64_t nkeys = 0;                     // keys of the layer (sum over structures)
};

// Scratch bytes of launch_sort for n keys in a layer of m slots.
size_t sort_scratch_bytes(uint64_t n, uint64_t m, uint32_t vbytes);
// Kernels one launch_sort of this layer enqueues (n > 0).
uint32_t sort_kernel_count(const LayerDesc &L);

// Sort n (key, value) pairs of a layer into bucket order.  The output holds
// the records h = mix64(key ^ sigma) of the keys (what the band and the cut
// search read), or the keys themselves with out_keys.
// scratch: sort_scratch_bytes(n, m, vbytes) bytes of device memory.
cudaError_t launch_sort(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                        uint64_t *keys_out, void *vals_out, uint32_t *bucket_start, void *scratch,
                        uint32_t *err, cudaStream_t st, bool out_keys = false);

// The same sort without its counting passes, for layers sorted in two
// scatter passes (sort_slack_scratch_bytes is 0 for the others): bins of fixed
// capacity, sized from the binomial spread of the keys' uniform start slots.
// begin, then pass 1 over input ranges [lo, hi) that together cover [0, n)
// (in any order, each once), then end.  If a bin overflowed, *err gets
// kErrSortSlack and the output holds only part of the keys (each in its right
// place): the caller sorts again with launch_sort.
size_t sort_slack_scratch_bytes(const LayerDesc &L, uint32_t vbytes);
cudaError_t launch_sort_slack_begin(const LayerDesc &L, uint32_t vbytes, void *scratch, cudaStream_t st);
cudaError_t launch_sort_slack_pass1(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                                    uint64_t lo, uint64_t hi, void *scratch, uint32_t *err, cudaStream_t st);
cudaError_t launch_sort_slack_end(const LayerDesc &L, uint32_t vbytes, uint64_t *keys_out, void *vals_out,
                                  uint32_t *bucket_start, void *scratch, uint32_t *err, cudaStream_t st);

// Band + bump (or base case), writing the band of every partition to Cg/Yg.
// With a batch view (bv != nullptr) L is ignored: every partition of every
// structure of the view is processed, bumped_count is per structure.
cudaError_t launch_band(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                        const uint32_t *bucket_start, uint64_t *Cg, void *Yg, uint64_t *thresh, uint8_t *texact,
                        uint64_t *bumped_keys, void *bumped_vals, unsigned long long *bumped_count,
                        uint32_t *err, cudaStream_t st, const BatchView *bv = nullptr);

// Back-substitution of every partition: Z from the band.
// max_ctas_per_sm > 0 caps the grid at that many CTAs per SM (the warps then
// walk the partitions with the grid's stride), which leaves room beside the
// back-substitution for the kernels of the next layer.
cudaError_t launch_backsub(const LayerDesc &L, uint32_t vbytes, const uint64_t *Cg, const void *Yg,
                           uint64_t *Z, cudaStream_t st, const BatchView *bv = nullptr,
                           uint32_t max_ctas_per_sm = 0);

// Batched sort: every structure's keys of the layer grouped by global bucket
// (as records h of each structure's layer).
size_t sort_batch_scratch_bytes(uint64_t nkeys, uint64_t ngroups, uint32_t vbytes);
cudaError_t launch_sort_batch(const BatchView &bv, uint32_t vbytes, const uint64_t *keys, const void *vals,
                              uint64_t *keys_out, void *vals_out, uint32_t *bucket_start, void *scratch,
                              cudaStream_t st);
constexpr uint32_t kSortTile = 2048;      // keys per tile of the batched sort
constexpr uint32_t kMaxGroupsPerStruct = 1024;

// Query descriptor: every layer of a handle.
struct QueryDesc {
    uint32_t r;
    uint32_t B;
    uint32_t layers;          // bumping layers
    uint32_t levels[4];
    uint32_t mode;            // BURR_THRESH_2BIT or BURR_THRESH_1PLUS
    uint64_t m[BURR_MAX_LAYERS + 1];
    uint64_t sigma[BURR_MAX_LAYERS + 1];
    const uint64_t *thresh[BURR_MAX_LAYERS];   // 2-bit codes
    const uint64_t *flags[BURR_MAX_LAYERS];    // 1+-bit: bit per bucket
    const uint32_t *dir[BURR_MAX_LAYERS];      // 1+-bit: rank of each 512-bucket block
    const uint8_t *tbytes[BURR_MAX_LAYERS];    // 1+-bit: thresholds of flagged buckets (ranks index it)
    const uint64_t *z[BURR_MAX_LAYERS + 1];   // [layers] = base case
};

// Ask for the line holding p to be brought into L2 (no registers, no wait).
__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.L2 [%0];" ::"l"(p));
}

// Every build kernel asks for the largest shared-memory carve-out.  Kernels of
// different stages run side by side (back-substitution overlaps the next
// layer's sort and band), and an SM set up for a small shared-memory share
// must drain before a kernel that needs a larger one can start on it: with
// mixed carve-outs the next layer waited for the whole back-substitution.
// Kernel attributes are set once per (kernel, device, attribute, value): the
// calls cost host time between the per-layer synchronisations, while the GPU
// waits for the next layer's launches.
bool attr_is_set(const void *kernel, int attr, int value);
void attr_mark_set(const void *kernel, int attr, int value);

template <typename K>
inline cudaError_t func_attr(K *kernel, cudaFuncAttribute attr, int value) {
    if (attr_is_set((const void *)kernel, (int)attr, value)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kernel, attr, value);
    if (e == cudaSuccess) attr_mark_set((const void *)kernel, (int)attr, value);
    return e;
}

template <typename K>
inline cudaError_t prefer_shared(K *kernel) {
    return func_attr(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
}

// 1+-bit threshold storage of one structure layer inside a launch: its
// buckets in the band's exact-threshold array, its flag words and its
// directory blocks (512 buckets each) in the launch-wide arrays.
struct ThreshSeg {
    uint64_t bucket_base, nb, fw_base, dir_base;
};

// From the exact thresholds of every bucket: flag words and, per directory
// block, the count of flagged buckets (counts) and its exclusive prefix over
// the launch (dir, nblk + 1 entries, dir[nblk] = total).  blk_seg maps each of
// the nblk blocks to its segment.
cudaError_t launch_thresh_flags(const uint8_t *texact, const ThreshSeg *segs, const uint32_t *blk_seg, uint32_t nblk,
                                uint64_t *flags, uint32_t *counts, uint32_t *dir, cudaStream_t st);
// The thresholds of the flagged buckets, at bytes[dir[block] + rank in block].
cudaError_t launch_thresh_compact(const uint8_t *texact, const ThreshSeg *segs, const uint32_t *blk_seg,
                                  uint32_t nblk, const uint64_t *flags, const uint32_t *dir, uint8_t *bytes,
                                  cudaStream_t st);

cudaError_t launch_query(const QueryDesc &Q, uint32_t vbytes, const uint64_t *keys, void *out,
                         uint64_t n, cudaStream_t st);

cudaError_t launch_hash(const uint64_t *keys, uint64_t n, uint64_t sigma, uint64_t range,
                        uint32_t *start, uint64_t *coeff, cudaStream_t st);

// Cut-point search (BURR_CUT_*): the first bucket of every partition of the
// layer, cuts[0..K] (cuts[K] = nb), from the bucket-sorted keys.  With a
// batch view, every structure's table sits at its L.cuts.
// Sharded build: the owner rank of each of n keys in a layer (the rank whose
// partition range [part_first[g], part_first[g+1]) holds the key's start
// bucket; part_first has ranks+1 entries in device memory) and the keys and
// values grouped by owner.  cursor: ranks device words holding each rank's
// first output position, advanced by the call; rank_of: n words of scratch.
constexpr uint32_t kMaxShardRanks = 1024;
cudaError_t launch_route(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                         const uint32_t *part_first, uint32_t ranks, uint32_t *rank_of,
                         unsigned long long *counts, unsigned long long *cursor, uint64_t *keys_out,
                         void *vals_out, bool count_only, cudaStream_t st);

cudaError_t launch_cut_search(const LayerDesc &L, const uint64_t *sorted_keys, const uint32_t *bucket_start,
                              uint32_t mode, uint32_t range, uint32_t *cuts, cudaStream_t st,
                              const BatchView *bv = nullptr);

// Record a message for burr_last_error() and return `code`.
int set_error(int code, const char *msg);

// A named range on the host timeline for profilers (NVTX, header-only).
struct TraceRange {
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// Device memory of the library (the caller's allocator if set, else the
// device's stream-ordered pool): allocation usable in stream order on st,
// release after the work on st, and release of a handle's table (waits for
// the device first).
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t st);
void dev_free_async(void *p, cudaStream_t st);
void dev_free_sync(void *p);

inline unsigned grid_for(uint64_t work, unsigned per_block, unsigned cap) {
    uint64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (unsigned)g;
}

}  // namespace burr
