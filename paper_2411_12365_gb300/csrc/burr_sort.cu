// burr_sort.cu -- "sort the hashes by their insertion position" (Sec. 4; the
// paper uses the CPU sorter IPS2Ra).  The build only needs the equations
// grouped by bucket (start / B) in ascending bucket order: the order inside a
// bucket is free, because the band kernel inserts a bucket's rows as a set
// (any order inside a threshold band gives the same kept set and, with free
// slots fixed to 0, the same table).  So this is an MSD counting sort on the
// bucket id, shaped for HBM:
//
//   * groups of 64 buckets (about 8k keys) are the unit of the last pass;
//   * one or two scatter passes bring the keys into group order.  Each pass
//     works in tiles of 4096 keys (2048 in the batched sort): a shared-memory
//     histogram and scan order the tile by digit in shared memory, one global
//     atomic per (tile, digit) reserves the output range, and the tile is
//     written out as contiguous runs per digit (coalesced stores, not
//     scattered 8-byte writes).  The output ranges come from counting passes
//     over all keys, or, for layers sorted in two passes, from bins of fixed
//     capacity (see the fixed-capacity section below);
//   * the last pass sorts each group in shared memory (count, scan, place)
//     and writes it out in order, together with the bucket offsets.
//
// The first pass that writes turns each key into its record h = mix64(key ^
// sigma), the first hash round of the key in the layer (8 bytes, like the
// key, and a bijection of it).  Later passes and the band then find the start
// slot with one multiply-high and the coefficients with one more round,
// instead of hashing the key again in every pass; the band recovers the key
// only for the rows it bumps.  The stage entry points ask for keys instead.
#include <cmath>
#include <cstdio>

#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kGroupShift = 6;                  // 64 buckets per group
constexpr uint32_t kGroupBuckets = 1u << kGroupShift;
constexpr int kHistThreads = 256;
#ifndef BURR_SORT_TILE_THREADS
#define BURR_SORT_TILE_THREADS 256
#endif
#ifndef BURR_SORT_TILE_ITEMS
#define BURR_SORT_TILE_ITEMS 16
#endif
#ifndef BURR_SORT_TILE_CTAS
#define BURR_SORT_TILE_CTAS 2
#endif
constexpr int kTileThreads = BURR_SORT_TILE_THREADS;
constexpr int kTileItems = BURR_SORT_TILE_ITEMS;
constexpr int kTileCtas = BURR_SORT_TILE_CTAS;     // CTAs per SM the scatter is compiled for
// 4096 keys per tile, 2 CTAs per SM.  Longer tiles give longer runs per digit
// and so fewer, fuller sectors per write: layer-0 sort of 10^9 keys (GB300)
// 28.5 ms with 256 x 8 keys and 4 CTAs per SM, 24.8 with 256 x 16 and 2,
// 24.7 with 256 x 20 and 2, 24.9 with 512 x 10 and 2, 25.2 with 512 x 16 and 1,
// 27.8 with 256 x 12 and 3, 31.2 with 512 x 4 and 4.
constexpr int kTile = kTileThreads * kTileItems;
constexpr uint32_t kMaxDigits = 1024;           // digits of one scatter pass
static_assert(kTile >= (int)kSortTile, "a batched sort tile must fit one scatter tile");
static_assert(kMaxDigits % kTileThreads == 0, "the digit loops cover kMaxDigits in steps of the block");
#ifndef BURR_GROUP_THREADS
#define BURR_GROUP_THREADS 512
#endif
constexpr int kGroupThreads = BURR_GROUP_THREADS;
constexpr uint32_t kGroupCap = 12288;           // keys a group may hold to be sorted in shared memory
constexpr int kUnroll = 8;                      // keys in flight per thread in the counting loops

inline uint32_t ceil_log2(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

// Digits of the scatter passes.  group = start >> gshift.  One pass when the
// groups fit one pass's digits; otherwise pass 1 uses the top d1 bits of the
// group id and pass 2 the low d2 bits inside each pass-1 bin.
struct Plan {
    uint32_t log2B, gshift;
    uint64_t ngroups;
    int passes;          // 0 (one group), 1 or 2
    uint32_t d2;         // low group bits sorted by pass 2
    uint32_t D1, D2;     // digits of pass 1 and pass 2
};

Plan make_plan(const LayerDesc &L) {
    Plan p;
    p.log2B = ceil_log2(L.B);
    p.gshift = p.log2B + kGroupShift;
    p.ngroups = (L.nb + kGroupBuckets - 1) / kGroupBuckets;
    if (p.ngroups <= 1) {
        p.passes = 0;
        p.d2 = 0;
        p.D1 = p.D2 = 1;
    } else if (p.ngroups <= kMaxDigits) {
        p.passes = 1;
        p.d2 = 0;
        p.D1 = (uint32_t)p.ngroups;
        p.D2 = 1;
    } else {
        const uint32_t bits = ceil_log2(p.ngroups);
        p.passes = 2;
        p.d2 = bits / 2;
        p.D2 = 1u << p.d2;
        p.D1 = (uint32_t)((p.ngroups + p.D2 - 1) >> p.d2);
    }
    return p;
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Sort group of a key (input of the first pass) and of a record h (later passes).
__device__ __forceinline__ uint32_t group_of(uint64_t key, uint64_t sigma, uint64_t range, uint32_t gshift) {
    return start_slot(key, sigma, range) >> gshift;
}
__device__ __forceinline__ uint32_t group_of_h(uint64_t h, uint64_t range, uint32_t gshift) {
    return start_of_h(h, range) >> gshift;
}

// counts[digit] of every key, digit = group >> dshift.
__global__ void __launch_bounds__(kHistThreads)
k_hist(const uint64_t *__restrict__ keys, uint64_t n, uint64_t sigma, uint64_t range, uint32_t gshift,
       uint32_t dshift, uint32_t D, uint32_t *__restrict__ counts) {
    __shared__ uint32_t sh[kMaxDigits];
    for (uint32_t i = threadIdx.x; i < D; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (kUnroll - 1) * stride < n; i += kUnroll * stride) {
        uint64_t k[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; ++j) k[j] = keys[i + j * stride];
#pragma unroll
        for (int j = 0; j < kUnroll; ++j) atomicAdd(&sh[group_of(k[j], sigma, range, gshift) >> dshift], 1u);
    }
    for (; i < n; i += stride) atomicAdd(&sh[group_of(keys[i], sigma, range, gshift) >> dshift], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < D; i += blockDim.x)
        if (sh[i]) atomicAdd(&counts[i], sh[i]);
}

// Per pass-1 bin (segment), counts of its low group bits: counts[group]
// (from the records h the first pass wrote).
__global__ void __launch_bounds__(kHistThreads)
k_hist_seg(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ off1, uint32_t nseg_ctas,
           uint64_t sigma, uint64_t range, uint32_t gshift, uint32_t D2, uint32_t *__restrict__ counts) {
    __shared__ uint32_t sh[kMaxDigits];
    const uint32_t seg = blockIdx.x / nseg_ctas, part = blockIdx.x % nseg_ctas;
    for (uint32_t i = threadIdx.x; i < D2; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint32_t lo = off1[seg], hi = off1[seg + 1];
    const uint32_t stride = nseg_ctas * blockDim.x;
    uint32_t i = lo + part * blockDim.x + threadIdx.x;
    for (; (uint64_t)i + (kUnroll - 1) * (uint64_t)stride < hi; i += kUnroll * stride) {
        uint64_t k[kUnroll];
#pragma unroll
        for (int j = 0; j < kUnroll; ++j) k[j] = keys[i + j * stride];
#pragma unroll
        for (int j = 0; j < kUnroll; ++j) atomicAdd(&sh[group_of_h(k[j], range, gshift) & (D2 - 1)], 1u);
    }
    for (; i < hi; i += stride) atomicAdd(&sh[group_of_h(keys[i], range, gshift) & (D2 - 1)], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < D2; i += blockDim.x)
        if (sh[i]) atomicAdd(&counts[(uint64_t)seg * D2 + i], sh[i]);
}

// Exclusive scan of counts[0..len) into off[0..len] and cursor[0..len), one
// block.  The counts go through shared memory in tiles of kScanItems * 1024
// (coalesced loads, every thread then scans kScanItems consecutive entries),
// with the running total carried from tile to tile: the 120k group counts of a
// 10^9-key layer took 0.44 ms when each thread walked its own 117 entries in
// global memory.
constexpr int kScanItems = 8;
__global__ void __launch_bounds__(1024)
k_scan(const uint32_t *__restrict__ counts, uint32_t len, uint32_t *__restrict__ off, uint32_t *__restrict__ cursor) {
    __shared__ uint32_t tile[kScanItems * 1024];
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t T = (uint32_t)kScanItems * blockDim.x;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < len; base += T) {
        const uint32_t n = min(T, len - base);
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) tile[i] = counts[base + i];
        __syncthreads();
        const uint32_t lo = threadIdx.x * kScanItems;
        uint32_t v[kScanItems], local = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = lo + k < n ? tile[lo + k] : 0u;
            local += v[k];
        }
        uint32_t x = local;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_sums[warp] = x;
        __syncthreads();
        if (warp == 0) {
            uint32_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        uint32_t run = carry + x - local + (warp ? warp_sums[warp - 1] : 0);
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (lo + k < n) {
                off[base + lo + k] = run;
                cursor[base + lo + k] = run;
            }
            run += v[k];
        }
        carry += warp_sums[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) off[len] = carry;
}

// Block-wide exclusive scan of cnt[0..len) (len <= kMaxDigits) into out[].
__device__ void block_scan(const uint32_t *cnt, uint32_t *out, uint32_t len, uint32_t *warp_sums) {
    const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = threadIdx.x * per;
    uint32_t local = 0;
    for (uint32_t i = lo; i < lo + per && i < len; ++i) local += cnt[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t run = x - local + (warp ? warp_sums[warp - 1] : 0);
    for (uint32_t i = lo; i < lo + per && i < len; ++i) {
        out[i] = run;
        run += cnt[i];
    }
    __syncthreads();
}

// Asynchronous global -> shared copies (the tile loads of k_scatter).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared memory of k_scatter: the ordered tile (records, values) and the
// input buffer the next tile is copied into while this one is worked on.
template <typename V>
constexpr size_t scatter_smem_bytes() {
    return (((size_t)kTile * (8 + sizeof(V)) + 15) & ~(size_t)15) + (size_t)kTile * 8 + (size_t)kTile * sizeof(V) + 8;
}

// One scatter pass.  Tiles of kTile keys are ordered by digit in shared
// memory and written as contiguous runs.  Unsegmented (pass 1): digit =
// group >> dshift over all n keys, cursor[digit].  Segmented (pass 2): tiles
// stay inside pass-1 bin seg = blockIdx / nseg_ctas, digit = group & (D - 1),
// cursor[seg * D + digit] (= cursor[group]).
//
// A CTA copies its next tile into shared memory asynchronously (cp.async)
// while it orders and writes the current one, so the load latency overlaps
// the work.  Keys go in 8-byte copies.  Values go in 4-byte chunks from the
// aligned-down address, when the array starts on 4 bytes and the rounded-up
// end of the tile stays inside it; otherwise the tile's values are read
// directly when it is worked on.
//
// RAW: the input holds keys, and the pass writes records h = mix64(key ^
// sigma); otherwise the input already holds records.
//
// SLACK: output bin c (digit, or group for pass 2) is the fixed range
// [c * cap_out, (c + 1) * cap_out), its cursor starting at c * cap_out; a key
// that would land past its bin's end is dropped and kErrSortSlack is raised.
// Pass 2 then reads pass-1 bin seg from [seg * cap_in, min(off1[seg],
// (seg + 1) * cap_in)) (off1 = the pass-1 cursors).  n is the input array's
// length; pass 1 reads [in_lo, n).
template <typename V, bool SEG, bool RAW, bool SLACK = false>
__global__ void __launch_bounds__(kTileThreads, kTileCtas)
k_scatter(const uint64_t *__restrict__ keys, const V *__restrict__ vals, uint64_t n,
          const uint32_t *__restrict__ off1, uint32_t nseg_ctas, uint64_t sigma, uint64_t range, uint32_t gshift,
          uint32_t dshift, uint32_t D, uint32_t *__restrict__ cursor, uint64_t *__restrict__ keys_out,
          V *__restrict__ vals_out, uint64_t cap_in = 0, uint64_t cap_out = 0, uint32_t *__restrict__ err = nullptr,
          uint64_t in_lo = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem_raw);
    V *sval = reinterpret_cast<V *>(skey + kTile);
    uint64_t *ikey = reinterpret_cast<uint64_t *>(smem_raw + (((size_t)kTile * (8 + sizeof(V)) + 15) & ~(size_t)15));
    unsigned char *ival = reinterpret_cast<unsigned char *>(ikey + kTile);
    __shared__ uint32_t hist[kMaxDigits], excl[kMaxDigits], gbase[kMaxDigits], warp_sums[32];

    uint64_t lo = in_lo, hi = n;
    uint32_t seg = 0, part = blockIdx.x, nparts = gridDim.x;
    if (SEG) {
        seg = blockIdx.x / nseg_ctas;
        part = blockIdx.x % nseg_ctas;
        nparts = nseg_ctas;
        if (SLACK) {
            lo = (uint64_t)seg * cap_in;
            hi = min((uint64_t)off1[seg], lo + cap_in);
        } else {
            lo = off1[seg];
            hi = off1[seg + 1];
        }
    }
    const bool vals_aligned = ((uintptr_t)vals & 3u) == 0;
    // start the copy of tile t into the input buffer; returns whether its values are copied too
    auto issue = [&](uint64_t t) -> bool {
        const uint64_t base = lo + t * kTile;
        const uint32_t cnt = (uint32_t)min((uint64_t)kTile, hi - base);
        for (uint32_t i = threadIdx.x; i < cnt; i += kTileThreads) cp_async8(ikey + i, keys + base + i);
        const uint64_t b0 = base * sizeof(V), a0 = b0 & ~3ull, a1 = ((base + cnt) * sizeof(V) + 3) & ~3ull;
        const bool va = vals_aligned && a1 <= n * sizeof(V);
        if (va) {
            const unsigned char *src = reinterpret_cast<const unsigned char *>(vals) + a0;
            const uint32_t nchunks = (uint32_t)((a1 - a0) >> 2);
            for (uint32_t c = threadIdx.x; c < nchunks; c += kTileThreads) cp_async4(ival + 4 * c, src + 4 * c);
        }
        cp_async_commit();
        return va;
    };
    for (uint32_t i = threadIdx.x; i < D; i += blockDim.x) hist[i] = 0;
    const uint64_t ntiles = (hi - lo + kTile - 1) / kTile;
    bool va = part < ntiles ? issue(part) : false;
    __syncthreads();
    for (uint64_t t = part; t < ntiles; t += nparts) {
        const uint64_t base = lo + t * kTile;
        const uint32_t cnt = (uint32_t)min((uint64_t)kTile, hi - base);
        cp_async_wait_all();
        __syncthreads();
        uint64_t key[kTileItems];
        V val[kTileItems];
        uint32_t dig[kTileItems], rank[kTileItems];
        const uint32_t vshift = (uint32_t)((base * sizeof(V)) & 3u);
#pragma unroll
        for (int j = 0; j < kTileItems; ++j) {
            const uint32_t i = (uint32_t)j * kTileThreads + threadIdx.x;
            if (i < cnt) {
                key[j] = ikey[i];
                val[j] = va ? *reinterpret_cast<const V *>(ival + vshift + i * sizeof(V)) : vals[base + i];
            }
        }
        __syncthreads();   // the input buffer is free: copy the next tile while this one is worked on
        const bool va_next = t + nparts < ntiles ? issue(t + nparts) : false;
#pragma unroll
        for (int j = 0; j < kTileItems; ++j) {
            const uint32_t i = (uint32_t)j * kTileThreads + threadIdx.x;
            if (i < cnt) {
                if (RAW) key[j] = mix64(key[j] ^ sigma);
                const uint32_t g = group_of_h(key[j], range, gshift);
                dig[j] = SEG ? (g & (D - 1)) : (g >> dshift);
                rank[j] = atomicAdd(&hist[dig[j]], 1u);
            }
        }
        __syncthreads();
        // reserve the tile's output ranges first; the atomics' round trip overlaps the scan
        uint32_t res[kMaxDigits / kTileThreads];
#pragma unroll
        for (int k = 0; k < (int)(kMaxDigits / kTileThreads); ++k) {
            const uint32_t d = threadIdx.x + (uint32_t)k * kTileThreads;
            res[k] = 0;
            if (d < D && hist[d]) res[k] = atomicAdd(&cursor[(uint64_t)seg * (SEG ? D : 0) + d], hist[d]);
        }
        block_scan(hist, excl, D, warp_sums);
        // gbase[d] - excl[d]: the output of tile index i is gbase[d] + i, one shared read per key
#pragma unroll
        for (int k = 0; k < (int)(kMaxDigits / kTileThreads); ++k) {
            const uint32_t d = threadIdx.x + (uint32_t)k * kTileThreads;
            if (d < D) gbase[d] = res[k] - excl[d];
        }
#pragma unroll
        for (int j = 0; j < kTileItems; ++j) {
            const uint32_t i = (uint32_t)j * kTileThreads + threadIdx.x;
            if (i < cnt) {
                const uint32_t p = excl[dig[j]] + rank[j];
                skey[p] = key[j];
                sval[p] = val[j];
            }
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
            // the digit again from the record (one multiply-high) instead of a
            // third shared array written at random positions
            const uint64_t h = skey[i];
            const uint32_t g = group_of_h(h, range, gshift);
            const uint32_t d = SEG ? (g & (D - 1)) : (g >> dshift);
            const uint32_t dst = gbase[d] + i;
            if (SLACK && dst >= ((uint64_t)seg * (SEG ? D : 0) + d + 1) * cap_out) {
                atomicOr(err, kErrSortSlack);
                continue;
            }
            keys_out[dst] = h;
            vals_out[dst] = sval[i];
        }
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < D; d += blockDim.x) hist[d] = 0;
        va = va_next;
    }
    cp_async_wait_all();
}

// Last pass: one block per group of 64 buckets.  The group's keys are
// counted per bucket, placed into bucket order in shared memory and written
// out contiguously; the bucket offsets are written too.  A group larger than
// the shared-memory capacity is placed directly in global memory instead.
// RAW: the input holds keys (a layer of one group, sorted in this pass
// alone); otherwise records h.  OUT_KEYS: the output holds keys (the stage
// entry points); otherwise records h (the build).
template <bool RAW>
__device__ __forceinline__ uint32_t bucket_in_group(uint64_t x, uint64_t sigma, uint64_t range, uint32_t log2B,
                                                    uint64_t b_lo) {
    return ((RAW ? start_slot(x, sigma, range) : start_of_h(x, range)) >> log2B) - (uint32_t)b_lo;
}
template <bool RAW, bool OUT_KEYS>
__device__ __forceinline__ uint64_t group_out(uint64_t x, uint64_t sigma) {
    if (RAW) return OUT_KEYS ? x : mix64(x ^ sigma);
    return OUT_KEYS ? key_of_h(x, sigma) : x;
}
// SLACK: the input of group g starts at g * cap (the bins of a SLACK pass 2),
// and goff holds the packed offsets of the groups' counts.
template <typename V, bool RAW, bool OUT_KEYS, bool SLACK = false>
__global__ void __launch_bounds__(kGroupThreads)
k_group_sort(const uint64_t *__restrict__ keys, const V *__restrict__ vals, const uint32_t *__restrict__ goff,
             uint64_t sigma, uint64_t range, uint32_t log2B, uint64_t nb, uint64_t *__restrict__ keys_out,
             V *__restrict__ vals_out, uint32_t *__restrict__ bucket_start, uint64_t cap = 0) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem_raw);
    V *sval = reinterpret_cast<V *>(skey + kGroupCap);
    __shared__ uint32_t cnt[kGroupBuckets], cur[kGroupBuckets], warp_sums[32];
    const uint64_t g = blockIdx.x;
    const uint64_t b_lo = g << kGroupShift;
    const uint32_t nbk = (uint32_t)min((uint64_t)kGroupBuckets, nb - b_lo);
    const uint32_t lo = goff[g], hi = goff[g + 1], n = hi - lo;
    if (SLACK) {   // index i in [lo, hi) reads input g * cap + (i - lo)
        keys += g * cap - lo;
        vals += g * cap - lo;
    }
    if (threadIdx.x < kGroupBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    {
        uint32_t i = lo + threadIdx.x;
        for (; (uint64_t)i + (kUnroll - 1) * (uint64_t)blockDim.x < hi; i += kUnroll * blockDim.x) {
            uint64_t k[kUnroll];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) k[j] = keys[i + j * blockDim.x];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                atomicAdd(&cnt[bucket_in_group<RAW>(k[j], sigma, range, log2B, b_lo)], 1u);
        }
        for (; i < hi; i += blockDim.x)
            atomicAdd(&cnt[bucket_in_group<RAW>(keys[i], sigma, range, log2B, b_lo)], 1u);
    }
    __syncthreads();
    block_scan(cnt, cur, kGroupBuckets, warp_sums);
    if (threadIdx.x < nbk) bucket_start[b_lo + threadIdx.x] = lo + cur[threadIdx.x];
    if (g == gridDim.x - 1 && threadIdx.x == 0) bucket_start[nb] = hi;
    __syncthreads();
    if (n <= kGroupCap) {
        uint32_t i = lo + threadIdx.x;
        for (; (uint64_t)i + 3 * (uint64_t)blockDim.x < hi; i += 4 * blockDim.x) {
            uint64_t k[4];
            V v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                k[j] = keys[i + j * blockDim.x];
                v[j] = vals[i + j * blockDim.x];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t b = bucket_in_group<RAW>(k[j], sigma, range, log2B, b_lo);
                const uint32_t p = atomicAdd(&cur[b], 1u);
                skey[p] = group_out<RAW, OUT_KEYS>(k[j], sigma);
                sval[p] = v[j];
            }
        }
        for (; i < hi; i += blockDim.x) {
            const uint64_t key = keys[i];
            const uint32_t b = bucket_in_group<RAW>(key, sigma, range, log2B, b_lo);
            const uint32_t p = atomicAdd(&cur[b], 1u);
            skey[p] = group_out<RAW, OUT_KEYS>(key, sigma);
            sval[p] = vals[i];
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            keys_out[lo + i] = skey[i];
            vals_out[lo + i] = sval[i];
        }
    } else {
        for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const uint64_t key = keys[i];
            const uint32_t b = bucket_in_group<RAW>(key, sigma, range, log2B, b_lo);
            const uint32_t p = lo + atomicAdd(&cur[b], 1u);
            keys_out[p] = group_out<RAW, OUT_KEYS>(key, sigma);
            vals_out[p] = vals[i];
        }
    }
}

struct Scratch {
    uint64_t *keys;
    void *vals;
    uint32_t *c1, *o1, *u1;      // pass-1 counts, offsets, cursors (kMaxDigits + 1)
    uint32_t *c2, *o2, *u2;      // per-group counts, offsets (= group offsets), cursors
};

Scratch carve(void *scratch, uint64_t n, uint64_t ngroups, uint32_t vbytes) {
    Scratch s;
    char *p = (char *)scratch;
    s.keys = (uint64_t *)p;  p += align256(n * 8);
    s.vals = p;              p += align256(n * vbytes);
    s.c1 = (uint32_t *)p;    p += align256((kMaxDigits + 1) * 4);
    s.o1 = (uint32_t *)p;    p += align256((kMaxDigits + 1) * 4);
    s.u1 = (uint32_t *)p;    p += align256((kMaxDigits + 1) * 4);
    s.c2 = (uint32_t *)p;    p += align256((ngroups + 1) * 4);
    s.o2 = (uint32_t *)p;    p += align256((ngroups + 1) * 4);
    s.u2 = (uint32_t *)p;
    return s;
}

// The group pass of sort_impl: RAW when it reads the caller's keys (a layer
// of one group), OUT_KEYS when it writes keys instead of records; SLACK (with
// the bins' capacity cap) as k_group_sort.
template <typename V, bool RAW, bool OUT_KEYS, bool SLACK = false>
cudaError_t launch_group_sort(const Plan &P, const LayerDesc &L, const uint64_t *gk, const V *gv, const uint32_t *goff,
                              uint64_t *keys_out, V *vals_out, uint32_t *bucket_start, cudaStream_t st,
                              uint64_t cap = 0) {
    const size_t group_smem = (size_t)kGroupCap * (8 + sizeof(V));
    cudaError_t e = func_attr(k_group_sort<V, RAW, OUT_KEYS, SLACK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)group_smem);
    if (e != cudaSuccess) return e;
    if ((e = prefer_shared(k_group_sort<V, RAW, OUT_KEYS, SLACK>)) != cudaSuccess) return e;
    k_group_sort<V, RAW, OUT_KEYS, SLACK><<<(unsigned)P.ngroups, kGroupThreads, group_smem, st>>>(
        gk, gv, goff, L.sigma, L.range, P.log2B, L.nb, keys_out, vals_out, bucket_start, cap);
    return cudaGetLastError();
}

// CTAs per pass-1 bin in the second pass: enough for about eight waves of the
// resident CTAs, so that the last wave leaves few SMs idle (with one CTA per
// bin and more bins than resident CTAs, the second wave ran half empty).
uint32_t seg_ctas(const Plan &P) {
    const unsigned sms = (unsigned)num_sms();
    uint64_t per64 = (8ull * sms * (uint64_t)kTileCtas + P.D1 - 1) / P.D1;
    if (per64 > 64) per64 = 64;
    if (per64 < 1) per64 = 1;
    return (uint32_t)per64;
}

template <typename V>
cudaError_t sort_attrs_slack() {
    const int tile_smem = (int)scatter_smem_bytes<V>();
    cudaError_t e;
    if ((e = func_attr(k_scatter<V, false, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_smem)) !=
            cudaSuccess ||
        (e = func_attr(k_scatter<V, true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tile_smem)) !=
            cudaSuccess ||
        (e = prefer_shared(k_scatter<V, false, true, true>)) != cudaSuccess ||
        (e = prefer_shared(k_scatter<V, true, false, true>)) != cudaSuccess ||
        (e = prefer_shared(k_scan)) != cudaSuccess)
        return e;
    return cudaSuccess;
}

template <typename V>
cudaError_t sort_impl(const LayerDesc &L, const uint64_t *keys, const V *vals, uint64_t *keys_out, V *vals_out,
                      uint32_t *bucket_start, void *scratch, bool out_keys, cudaStream_t st) {
    const uint64_t n = L.n;
    const Plan P = make_plan(L);
    Scratch S = carve(scratch, n, P.ngroups, sizeof(V));
    const unsigned sms = (unsigned)num_sms();
    const size_t tile_smem = scatter_smem_bytes<V>();
    cudaError_t e;
    e = func_attr(k_scatter<V, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
    if (e != cudaSuccess) return e;
    e = func_attr(k_scatter<V, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
    if (e != cudaSuccess) return e;
    if ((e = prefer_shared(k_hist)) != cudaSuccess || (e = prefer_shared(k_scan)) != cudaSuccess ||
        (e = prefer_shared(k_scatter<V, false, true>)) != cudaSuccess ||
        (e = prefer_shared(k_scatter<V, true, false>)) != cudaSuccess || (e = prefer_shared(k_hist_seg)) != cudaSuccess)
        return e;

    if (P.passes == 0) {
        // one group: offsets [0, n]; the group pass reads the keys themselves
        const uint32_t h[2] = {0, (uint32_t)n};
        e = cudaMemcpyAsync(S.o2, h, sizeof(h), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        return out_keys ? launch_group_sort<V, true, true>(P, L, keys, vals, S.o2, keys_out, vals_out, bucket_start, st)
                        : launch_group_sort<V, true, false>(P, L, keys, vals, S.o2, keys_out, vals_out, bucket_start,
                                                            st);
    }
    const uint32_t *goff;
    if (P.passes == 1) {
        e = cudaMemsetAsync(S.c1, 0, (size_t)P.D1 * 4, st);
        if (e != cudaSuccess) return e;
        k_hist<<<grid_for(n, kHistThreads * 16, sms * 4), kHistThreads, 0, st>>>(keys, n, L.sigma, L.range,
                                                                                    P.gshift, 0, P.D1, S.c1);
        k_scan<<<1, 1024, 0, st>>>(S.c1, P.D1, S.o1, S.u1);
        k_scatter<V, false, true><<<grid_for(n, kTile, sms * kTileCtas), kTileThreads, tile_smem, st>>>(
            keys, vals, n, nullptr, 1, L.sigma, L.range, P.gshift, 0, P.D1, S.u1, S.keys, (V *)S.vals);
        goff = S.o1;
    } else {
        // pass 1 into the caller's output buffers, pass 2 into scratch
        e = cudaMemsetAsync(S.c1, 0, (size_t)P.D1 * 4, st);
        if (e != cudaSuccess) return e;
        e = cudaMemsetAsync(S.c2, 0, (size_t)P.ngroups * 4, st);
        if (e != cudaSuccess) return e;
        k_hist<<<grid_for(n, kHistThreads * 16, sms * 4), kHistThreads, 0, st>>>(keys, n, L.sigma, L.range,
                                                                                    P.gshift, P.d2, P.D1, S.c1);
        k_scan<<<1, 1024, 0, st>>>(S.c1, P.D1, S.o1, S.u1);
        k_scatter<V, false, true><<<grid_for(n, kTile, sms * kTileCtas), kTileThreads, tile_smem, st>>>(
            keys, vals, n, nullptr, 1, L.sigma, L.range, P.gshift, P.d2, P.D1, S.u1, keys_out, vals_out);
        const uint32_t per = seg_ctas(P);
        k_hist_seg<<<P.D1 * per, kHistThreads, 0, st>>>(keys_out, S.o1, per, L.sigma, L.range, P.gshift, P.D2,
                                                         S.c2);
        k_scan<<<1, 1024, 0, st>>>(S.c2, (uint32_t)P.ngroups, S.o2, S.u2);
        k_scatter<V, true, false><<<P.D1 * per, kTileThreads, tile_smem, st>>>(
            keys_out, vals_out, n, S.o1, per, L.sigma, L.range, P.gshift, 0, P.D2, S.u2, S.keys, (V *)S.vals);
        goff = S.o2;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return out_keys ? launch_group_sort<V, false, true>(P, L, S.keys, (const V *)S.vals, goff, keys_out, vals_out,
                                                        bucket_start, st)
                    : launch_group_sort<V, false, false>(P, L, S.keys, (const V *)S.vals, goff, keys_out, vals_out,
                                                         bucket_start, st);
}

// ---------------------------------------------------------------------------
// Two-pass layers without counting passes.  The start slots of a layer's keys
// are uniform over [0, range) (one multiply-high of a 64-bit hash), so the
// number of keys in a pass-1 bin or a sort group is binomial with a known
// mean mu.  Each bin and group gets a fixed range of mu + 8 sqrt(mu) + a
// margin slots in scratch, and the scatter passes reserve space in it with
// the same per-tile atomics as the exact sort: no histogram pass over the
// keys is needed before either scatter.  A key that would fall past its
// range's end (never seen with distinct keys: 8 standard deviations) is
// dropped and kErrSortSlack is raised; everything that is written is in its
// right bin, so the layer can go on, and the caller sorts it again exactly.
// The group pass packs the groups back to back (offsets from a scan of their
// counts), so the output is the exact sort's.
// ---------------------------------------------------------------------------

struct SlackPlan {
    Plan P;
    uint64_t cap1 = 0, cap2 = 0;   // slots of a pass-1 bin and of a group
    bool ok = false;
};

SlackPlan make_slack_plan(const LayerDesc &L) {
    SlackPlan S;
    S.P = make_plan(L);
    if (S.P.passes != 2 || L.range == 0 || L.n == 0) return S;
    const double mu1 = (double)L.n * (double)((uint64_t)S.P.D2 << S.P.gshift) / (double)L.range;
    const double mu2 = (double)L.n * (double)(1ull << S.P.gshift) / (double)L.range;
    S.cap1 = L.test_slack ? (uint64_t)(mu1 / 2) + 1 : (uint64_t)(mu1 + 8.0 * sqrt(mu1)) + 256;
    S.cap2 = L.test_slack ? (uint64_t)(mu2 / 2) + 1 : (uint64_t)(mu2 + 8.0 * sqrt(mu2)) + 64;
    // groups must fit the group pass's shared memory, positions 32 bits
    S.ok = S.cap2 <= kGroupCap && (double)S.P.D1 * (double)S.cap1 < 4.0e9 &&
           (double)S.P.ngroups * (double)S.cap2 < 4.0e9;
    return S;
}

struct SlackScratch {
    uint64_t *keys1, *keys2;
    void *vals1, *vals2;
    uint32_t *cur1, *cur2, *cnt, *off, *tmp;
};

size_t slack_bytes(const SlackPlan &S, uint32_t vbytes, SlackScratch *out) {
    const uint64_t n1 = (uint64_t)S.P.D1 * S.cap1, n2 = S.P.ngroups * S.cap2, G = S.P.ngroups;
    size_t o = 0;
    SlackScratch x;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o += align256(bytes);
        return at;
    };
    const size_t k1 = take(n1 * 8), v1 = take(n1 * vbytes), k2 = take(n2 * 8), v2 = take(n2 * vbytes),
                 c1 = take((size_t)S.P.D1 * 4), c2 = take(G * 4), cn = take((G + 1) * 4), of = take((G + 1) * 4),
                 tp = take((G + 1) * 4);
    if (out) {
        char *b = (char *)out->keys1;   // the scratch base, passed in keys1
        x.keys1 = (uint64_t *)(b + k1);
        x.vals1 = b + v1;
        x.keys2 = (uint64_t *)(b + k2);
        x.vals2 = b + v2;
        x.cur1 = (uint32_t *)(b + c1);
        x.cur2 = (uint32_t *)(b + c2);
        x.cnt = (uint32_t *)(b + cn);
        x.off = (uint32_t *)(b + of);
        x.tmp = (uint32_t *)(b + tp);
        *out = x;
    }
    return o;
}

SlackScratch slack_carve(const SlackPlan &S, uint32_t vbytes, void *scratch) {
    SlackScratch x;
    x.keys1 = (uint64_t *)scratch;
    slack_bytes(S, vbytes, &x);
    return x;
}

// cursor of pass-1 bin d = d * cap1, of group g = g * cap2
__global__ void k_slack_init(uint32_t *__restrict__ cur1, uint32_t D1, uint64_t cap1, uint32_t *__restrict__ cur2,
                             uint64_t G, uint64_t cap2) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D1 + G; i += stride) {
        if (i < D1) cur1[i] = (uint32_t)(i * cap1);
        else cur2[i - D1] = (uint32_t)((i - D1) * cap2);
    }
}

// keys each group holds (its cursor's advance, at most its capacity)
__global__ void k_slack_counts(const uint32_t *__restrict__ cur2, uint64_t G, uint64_t cap2, uint32_t *__restrict__ cnt,
                               uint32_t *__restrict__ err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += stride) {
        uint64_t c = cur2[g] - g * cap2;
        if (c > cap2) {
            c = cap2;
            atomicOr(err, kErrSortSlack);
        }
        cnt[g] = (uint32_t)c;
    }
}

template <typename V>
cudaError_t slack_begin_impl(const SlackPlan &S, const SlackScratch &X, cudaStream_t st) {
    cudaError_t e = sort_attrs_slack<V>();
    if (e != cudaSuccess) return e;
    k_slack_init<<<grid_for(S.P.D1 + S.P.ngroups, 256, 1024), 256, 0, st>>>(X.cur1, S.P.D1, S.cap1, X.cur2,
                                                                             S.P.ngroups, S.cap2);
    return cudaGetLastError();
}

template <typename V>
cudaError_t slack_pass1_impl(const LayerDesc &L, const SlackPlan &S, const SlackScratch &X, const uint64_t *keys,
                             const V *vals, uint64_t lo, uint64_t hi, uint32_t *err, cudaStream_t st) {
    if (hi <= lo) return cudaSuccess;
    const unsigned sms = (unsigned)num_sms();
    k_scatter<V, false, true, true><<<grid_for(hi - lo, kTile, sms * kTileCtas), kTileThreads, scatter_smem_bytes<V>(),
                                      st>>>(keys, vals, hi, nullptr, 1, L.sigma, L.range, S.P.gshift, S.P.d2, S.P.D1,
                                            X.cur1, X.keys1, (V *)X.vals1, 0, S.cap1, err, lo);
    return cudaGetLastError();
}

template <typename V>
cudaError_t slack_end_impl(const LayerDesc &L, const SlackPlan &S, const SlackScratch &X, uint64_t *keys_out,
                           V *vals_out, uint32_t *bucket_start, uint32_t *err, cudaStream_t st) {
    const Plan &P = S.P;
    const uint32_t per = seg_ctas(P);
    k_scatter<V, true, false, true><<<P.D1 * per, kTileThreads, scatter_smem_bytes<V>(), st>>>(
        X.keys1, (const V *)X.vals1, (uint64_t)P.D1 * S.cap1, X.cur1, per, L.sigma, L.range, P.gshift, 0, P.D2, X.cur2,
        X.keys2, (V *)X.vals2, S.cap1, S.cap2, err);
    k_slack_counts<<<grid_for(P.ngroups, 256, 1024), 256, 0, st>>>(X.cur2, P.ngroups, S.cap2, X.cnt, err);
    k_scan<<<1, 1024, 0, st>>>(X.cnt, (uint32_t)P.ngroups, X.off, X.tmp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_group_sort<V, false, false, true>(P, L, X.keys2, (const V *)X.vals2, X.off, keys_out, vals_out,
                                                    bucket_start, st, S.cap2);
}

// ---------------------------------------------------------------------------
// Batched layers: many structures at once.  Every structure's keys sit in its
// own range of the input buffer; global sort groups and global buckets are
// numbered structure by structure, so grouping by global group keeps each
// structure's keys contiguous and in bucket order.  One pass suffices per
// structure (at most kMaxGroupsPerStruct groups each): tiles never straddle
// structures (tile tables are built on the host).  The scatter turns each key
// into its record h = mix64(key ^ sigma) of its structure's layer.
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kHistThreads)
k_hist_batch(const uint64_t *__restrict__ keys, BatchView bv, uint32_t gshift, uint32_t *__restrict__ counts) {
    __shared__ uint32_t sh[kMaxDigits];
    const uint32_t t = blockIdx.x;
    const StructDesc &D = bv.sd[bv.tile_struct[t]];
    const uint64_t lo = bv.tile_lo[t];
    const uint64_t hi = min(lo + (uint64_t)kSortTile, D.key_base + D.L.n);
    const uint32_t G = D.ngroups;
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        atomicAdd(&sh[group_of(keys[i], D.L.sigma, D.L.range, gshift)], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x)
        if (sh[i]) atomicAdd(&counts[D.group_base + i], sh[i]);
}

template <typename V>
__global__ void __launch_bounds__(kTileThreads)
k_scatter_batch(const uint64_t *__restrict__ keys, const V *__restrict__ vals, BatchView bv, uint32_t gshift,
                uint32_t *__restrict__ cursor, uint64_t *__restrict__ keys_out, V *__restrict__ vals_out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem_raw);
    V *sval = reinterpret_cast<V *>(skey + kTile);
    __shared__ uint32_t hist[kMaxDigits], excl[kMaxDigits], gbase[kMaxDigits], warp_sums[32];
    const uint32_t t = blockIdx.x;
    const StructDesc &D = bv.sd[bv.tile_struct[t]];
    const uint64_t base = bv.tile_lo[t];
    const uint32_t cnt = (uint32_t)min((uint64_t)kSortTile, D.key_base + D.L.n - base);
    const uint32_t G = D.ngroups;
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    uint64_t key[kTileItems];
    V val[kTileItems];
    uint32_t dig[kTileItems], rank[kTileItems];
#pragma unroll
    for (int j = 0; j < kTileItems; ++j) {
        const uint32_t i = (uint32_t)j * kTileThreads + threadIdx.x;
        if (i < cnt) {
            key[j] = keys[base + i];
            val[j] = vals[base + i];
            key[j] = mix64(key[j] ^ D.L.sigma);          // the record h of the key
            dig[j] = group_of_h(key[j], D.L.range, gshift);
            rank[j] = atomicAdd(&hist[dig[j]], 1u);
        }
    }
    __syncthreads();
    block_scan(hist, excl, G, warp_sums);
    for (uint32_t d = threadIdx.x; d < G; d += blockDim.x)   // as in k_scatter: gbase[d] - excl[d]
        if (hist[d]) gbase[d] = atomicAdd(&cursor[D.group_base + d], hist[d]) - excl[d];
#pragma unroll
    for (int j = 0; j < kTileItems; ++j) {
        const uint32_t i = (uint32_t)j * kTileThreads + threadIdx.x;
        if (i < cnt) {
            const uint32_t p = excl[dig[j]] + rank[j];
            skey[p] = key[j];
            sval[p] = val[j];
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const uint32_t d = group_of_h(skey[i], D.L.range, gshift);   // skey holds records h
        const uint32_t dst = gbase[d] + i;
        keys_out[dst] = skey[i];
        vals_out[dst] = sval[i];
    }
}

// One block per global group: as k_group_sort (records h in and out), with
// the group's structure looked up in the batch tables.
template <typename V>
__global__ void __launch_bounds__(kGroupThreads)
k_group_sort_batch(const uint64_t *__restrict__ keys, const V *__restrict__ vals, const uint32_t *__restrict__ goff,
                   BatchView bv, uint32_t log2B, uint64_t *__restrict__ keys_out, V *__restrict__ vals_out,
                   uint32_t *__restrict__ bucket_start) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem_raw);
    V *sval = reinterpret_cast<V *>(skey + kGroupCap);
    __shared__ uint32_t cnt[kGroupBuckets], cur[kGroupBuckets], warp_sums[32];
    const uint64_t g = blockIdx.x;
    const StructDesc &D = bv.sd[bv.group_struct[g]];
    const uint64_t lg = g - D.group_base;
    const uint64_t b_lo = lg << kGroupShift;            // first local bucket of the group
    const uint32_t nbk = (uint32_t)min((uint64_t)kGroupBuckets, D.L.nb - b_lo);
    const uint64_t range = D.L.range;
    const uint32_t lo = goff[g], hi = goff[g + 1], n = hi - lo;
    if (threadIdx.x < kGroupBuckets) cnt[threadIdx.x] = 0;
    __syncthreads();
    {
        uint32_t i = lo + threadIdx.x;
        for (; (uint64_t)i + (kUnroll - 1) * (uint64_t)blockDim.x < hi; i += kUnroll * blockDim.x) {
            uint64_t k[kUnroll];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) k[j] = keys[i + j * blockDim.x];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                atomicAdd(&cnt[(start_of_h(k[j], range) >> log2B) - (uint32_t)b_lo], 1u);
        }
        for (; i < hi; i += blockDim.x)
            atomicAdd(&cnt[(start_of_h(keys[i], range) >> log2B) - (uint32_t)b_lo], 1u);
    }
    __syncthreads();
    block_scan(cnt, cur, kGroupBuckets, warp_sums);
    if (threadIdx.x < nbk) bucket_start[D.bucket_base + b_lo + threadIdx.x] = lo + cur[threadIdx.x];
    if (g == gridDim.x - 1 && threadIdx.x == 0) bucket_start[bv.nbuckets] = hi;
    __syncthreads();
    if (n <= kGroupCap) {
        uint32_t i = lo + threadIdx.x;
        for (; (uint64_t)i + 3 * (uint64_t)blockDim.x < hi; i += 4 * blockDim.x) {
            uint64_t k[4];
            V v[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                k[j] = keys[i + j * blockDim.x];
                v[j] = vals[i + j * blockDim.x];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint32_t b = (start_of_h(k[j], range) >> log2B) - (uint32_t)b_lo;
                const uint32_t p = atomicAdd(&cur[b], 1u);
                skey[p] = k[j];
                sval[p] = v[j];
            }
        }
        for (; i < hi; i += blockDim.x) {
            const uint64_t key = keys[i];
            const uint32_t b = (start_of_h(key, range) >> log2B) - (uint32_t)b_lo;
            const uint32_t p = atomicAdd(&cur[b], 1u);
            skey[p] = key;
            sval[p] = vals[i];
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
            keys_out[lo + i] = skey[i];
            vals_out[lo + i] = sval[i];
        }
    } else {
        for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const uint64_t key = keys[i];
            const uint32_t b = (start_of_h(key, range) >> log2B) - (uint32_t)b_lo;
            const uint32_t p = lo + atomicAdd(&cur[b], 1u);
            keys_out[p] = key;
            vals_out[p] = vals[i];
        }
    }
}

template <typename V>
cudaError_t sort_batch_impl(const BatchView &bv, const uint64_t *keys, const V *vals, uint64_t *keys_out,
                            V *vals_out, uint32_t *bucket_start, void *scratch, cudaStream_t st) {
    const uint32_t log2B = 7;   // bucket_slots = 128 for batched builds
    const uint32_t gshift = log2B + kGroupShift;
    char *p = (char *)scratch;
    uint64_t *tk = (uint64_t *)p;   p += align256(bv.nkeys * 8);
    V *tv = (V *)p;                 p += align256(bv.nkeys * sizeof(V));
    uint32_t *counts = (uint32_t *)p; p += align256(((uint64_t)bv.ngroups + 1) * 4);
    uint32_t *goff = (uint32_t *)p;   p += align256(((uint64_t)bv.ngroups + 1) * 4);
    uint32_t *cursor = (uint32_t *)p;
    const size_t tile_smem = (size_t)kTile * (8 + sizeof(V));
    const size_t group_smem = (size_t)kGroupCap * (8 + sizeof(V));
    cudaError_t e;
    e = func_attr(k_scatter_batch<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tile_smem);
    if (e != cudaSuccess) return e;
    e = func_attr(k_group_sort_batch<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)group_smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counts, 0, (size_t)bv.ngroups * 4, st);
    if (e != cudaSuccess) return e;
    if ((e = prefer_shared(k_hist_batch)) != cudaSuccess || (e = prefer_shared(k_scan)) != cudaSuccess ||
        (e = prefer_shared(k_scatter_batch<V>)) != cudaSuccess || (e = prefer_shared(k_group_sort_batch<V>)) != cudaSuccess)
        return e;
    k_hist_batch<<<bv.ntiles, kHistThreads, 0, st>>>(keys, bv, gshift, counts);
    k_scan<<<1, 1024, 0, st>>>(counts, bv.ngroups, goff, cursor);
    k_scatter_batch<V><<<bv.ntiles, kTileThreads, tile_smem, st>>>(keys, vals, bv, gshift, cursor, tk, tv);
    k_group_sort_batch<V><<<bv.ngroups, kGroupThreads, group_smem, st>>>(tk, tv, goff, bv, log2B, keys_out,
                                                                          vals_out, bucket_start);
    return cudaGetLastError();
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n, uint64_t m, uint32_t vbytes) {
    const uint64_t nb = m >= kW ? (m - kW + 128) / 64 : 1;   // buckets of >= 64 slots
    const uint64_t ngroups = (nb + kGroupBuckets - 1) / kGroupBuckets + 1;
    return align256(n * 8) + align256(n * vbytes) + 3 * align256((kMaxDigits + 1) * 4) +
           3 * align256((ngroups + 1) * 4);
}

size_t sort_batch_scratch_bytes(uint64_t nkeys, uint64_t ngroups, uint32_t vbytes) {
    return align256(nkeys * 8) + align256(nkeys * vbytes) + 3 * align256((ngroups + 1) * 4);
}

cudaError_t launch_sort_batch(const BatchView &bv, uint32_t vbytes, const uint64_t *keys, const void *vals,
                              uint64_t *keys_out, void *vals_out, uint32_t *bucket_start, void *scratch,
                              cudaStream_t st) {
    if (bv.nkeys == 0 || bv.ngroups == 0) return cudaSuccess;
    switch (vbytes) {
    case 1: return sort_batch_impl<uint8_t>(bv, keys, (const uint8_t *)vals, keys_out, (uint8_t *)vals_out,
                                            bucket_start, scratch, st);
    case 2: return sort_batch_impl<uint16_t>(bv, keys, (const uint16_t *)vals, keys_out, (uint16_t *)vals_out,
                                             bucket_start, scratch, st);
    default: return sort_batch_impl<uint32_t>(bv, keys, (const uint32_t *)vals, keys_out, (uint32_t *)vals_out,
                                              bucket_start, scratch, st);
    }
}

uint32_t sort_kernel_count(const LayerDesc &L) {
    const Plan P = make_plan(L);
    return P.passes == 0 ? 1u : (P.passes == 1 ? 4u : 7u);
}

size_t sort_slack_scratch_bytes(const LayerDesc &L, uint32_t vbytes) {
    const SlackPlan S = make_slack_plan(L);
    return S.ok ? slack_bytes(S, vbytes, nullptr) : 0;
}

cudaError_t launch_sort_slack_begin(const LayerDesc &L, uint32_t vbytes, void *scratch, cudaStream_t st) {
    const SlackPlan S = make_slack_plan(L);
    if (!S.ok) return cudaErrorInvalidValue;
    const SlackScratch X = slack_carve(S, vbytes, scratch);
    switch (vbytes) {
    case 1: return slack_begin_impl<uint8_t>(S, X, st);
    case 2: return slack_begin_impl<uint16_t>(S, X, st);
    default: return slack_begin_impl<uint32_t>(S, X, st);
    }
}

cudaError_t launch_sort_slack_pass1(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                                    uint64_t lo, uint64_t hi, void *scratch, uint32_t *err, cudaStream_t st) {
    const SlackPlan S = make_slack_plan(L);
    if (!S.ok || hi > L.n) return cudaErrorInvalidValue;
    const SlackScratch X = slack_carve(S, vbytes, scratch);
    switch (vbytes) {
    case 1: return slack_pass1_impl<uint8_t>(L, S, X, keys, (const uint8_t *)vals, lo, hi, err, st);
    case 2: return slack_pass1_impl<uint16_t>(L, S, X, keys, (const uint16_t *)vals, lo, hi, err, st);
    default: return slack_pass1_impl<uint32_t>(L, S, X, keys, (const uint32_t *)vals, lo, hi, err, st);
    }
}

cudaError_t launch_sort_slack_end(const LayerDesc &L, uint32_t vbytes, uint64_t *keys_out, void *vals_out,
                                  uint32_t *bucket_start, void *scratch, uint32_t *err, cudaStream_t st) {
    const SlackPlan S = make_slack_plan(L);
    if (!S.ok) return cudaErrorInvalidValue;
    const SlackScratch X = slack_carve(S, vbytes, scratch);
    switch (vbytes) {
    case 1: return slack_end_impl<uint8_t>(L, S, X, keys_out, (uint8_t *)vals_out, bucket_start, err, st);
    case 2: return slack_end_impl<uint16_t>(L, S, X, keys_out, (uint16_t *)vals_out, bucket_start, err, st);
    default: return slack_end_impl<uint32_t>(L, S, X, keys_out, (uint32_t *)vals_out, bucket_start, err, st);
    }
}

cudaError_t launch_sort(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                        uint64_t *keys_out, void *vals_out, uint32_t *bucket_start, void *scratch,
                        uint32_t * /*err*/, cudaStream_t st, bool out_keys) {
    if (L.n == 0) return cudaMemsetAsync(bucket_start, 0, (size_t)(L.nb + 1) * 4, st);
    switch (vbytes) {
    case 1: return sort_impl<uint8_t>(L, keys, (const uint8_t *)vals, keys_out, (uint8_t *)vals_out,
                                      bucket_start, scratch, out_keys, st);
    case 2: return sort_impl<uint16_t>(L, keys, (const uint16_t *)vals, keys_out, (uint16_t *)vals_out,
                                       bucket_start, scratch, out_keys, st);
    default: return sort_impl<uint32_t>(L, keys, (const uint32_t *)vals, keys_out, (uint32_t *)vals_out,
                                        bucket_start, scratch, out_keys, st);
    }
}

}  // namespace burr
