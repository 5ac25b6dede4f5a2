// burr_sort.cu -- "sort the hashes by their insertion position" (Sec. 4; the
// paper uses the CPU sorter IPS2Ra).  On the GPU the build only needs the
// equations grouped by bucket (start / B) in ascending bucket order: the order
// inside a bucket is free, because the band kernel inserts a bucket's rows as a
// set (any order inside a threshold band gives the same kept set and, with free
// slots fixed to 0, the same table).  So this is a two-pass MSD counting sort
// on the bucket id:
//   level 1: bins of 2^bshift1 buckets (<= 16384 bins), shared-memory
//            histograms per CTA, one global atomic per (tile, bin);
//   level 2: one CTA per level-1 bin counting-sorts its records by bucket in
//            shared memory and writes the bucket offsets.
// The equation is recomputed from the key in each pass (hash fused into the
// consumer) instead of materialising 16-byte records.
#include <cstdio>

#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kL1Threads = 256;
constexpr int kL1Items = 16;                       // tile = 4096 keys
constexpr int kL1Tile = kL1Threads * kL1Items;
constexpr uint32_t kMaxBins1 = 16384;
constexpr int kL2Threads = 512;
constexpr uint32_t kMaxBucketsPerBin = 4096;

inline uint32_t ceil_log2(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

inline uint32_t log2_exact(uint32_t x) {
    uint32_t l = 0;
    while ((1u << l) < x) ++l;
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

__global__ void __launch_bounds__(kL1Threads)
k_l1_hist(const uint64_t *__restrict__ keys, uint64_t n, uint64_t sigma, uint64_t range,
          uint32_t shift, uint32_t nbins, uint32_t *__restrict__ counts) {
    extern __shared__ uint32_t sh[];
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        atomicAdd(&sh[start_slot(keys[i], sigma, range) >> shift], 1u);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x)
        if (sh[i]) atomicAdd(&counts[i], sh[i]);
}

// Exclusive scan of nbins counts into off[0..nbins] and cursor[0..nbins).
__global__ void __launch_bounds__(1024)
k_scan_bins(const uint32_t *__restrict__ counts, uint32_t nbins, uint32_t *__restrict__ off,
            uint32_t *__restrict__ cursor) {
    __shared__ uint32_t warp_sums[32];
    const uint32_t per = (nbins + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = threadIdx.x * per;
    uint32_t local = 0;
    for (uint32_t i = lo; i < lo + per && i < nbins; ++i) local += counts[i];
    // block exclusive scan of `local`
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t run = x - local + (warp ? warp_sums[warp - 1] : 0);
    for (uint32_t i = lo; i < lo + per && i < nbins; ++i) {
        off[i] = run;
        cursor[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == blockDim.x - 1) off[nbins] = run;
}

template <typename V>
__global__ void __launch_bounds__(kL1Threads)
k_l1_scatter(const uint64_t *__restrict__ keys, const V *__restrict__ vals, uint64_t n,
             uint64_t sigma, uint64_t range, uint32_t shift, uint32_t nbins,
             uint32_t *__restrict__ cursor, uint64_t *__restrict__ keys_out, V *__restrict__ vals_out) {
    extern __shared__ uint32_t sh[];
    for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t ntiles = (n + kL1Tile - 1) / kL1Tile;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t base = tile * kL1Tile + threadIdx.x;
        uint64_t key[kL1Items];
        V val[kL1Items];
        uint32_t bin[kL1Items], rank[kL1Items];
#pragma unroll
        for (int j = 0; j < kL1Items; ++j) {
            const uint64_t i = base + (uint64_t)j * kL1Threads;
            if (i < n) {
                key[j] = keys[i];
                val[j] = vals[i];
                bin[j] = start_slot(key[j], sigma, range) >> shift;
                rank[j] = atomicAdd(&sh[bin[j]], 1u);
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kL1Items; ++j) {
            const uint64_t i = base + (uint64_t)j * kL1Threads;
            if (i < n && rank[j] == 0) {
                const uint32_t cnt = sh[bin[j]];
                sh[bin[j]] = atomicAdd(&cursor[bin[j]], cnt);
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kL1Items; ++j) {
            const uint64_t i = base + (uint64_t)j * kL1Threads;
            if (i < n) {
                const uint32_t pos = sh[bin[j]] + rank[j];
                keys_out[pos] = key[j];
                vals_out[pos] = val[j];
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kL1Items; ++j) {
            const uint64_t i = base + (uint64_t)j * kL1Threads;
            if (i < n) sh[bin[j]] = 0;
        }
        __syncthreads();
    }
}

// Block-wide exclusive scan over cnt[0..len) (len <= kMaxBucketsPerBin) in place.
__device__ void block_exclusive_scan(uint32_t *cnt, uint32_t len, uint32_t *warp_sums) {
    const uint32_t per = (len + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = threadIdx.x * per;
    uint32_t local = 0;
    for (uint32_t i = lo; i < lo + per && i < len; ++i) local += cnt[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = local;
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, d);
            if (lane >= d) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t run = x - local + (warp ? warp_sums[warp - 1] : 0);
    for (uint32_t i = lo; i < lo + per && i < len; ++i) {
        const uint32_t c = cnt[i];
        cnt[i] = run;
        run += c;
    }
    __syncthreads();
}

template <typename V>
__global__ void __launch_bounds__(kL2Threads)
k_l2_sort(const uint64_t *__restrict__ keys, const V *__restrict__ vals,
          const uint32_t *__restrict__ off1, uint64_t sigma, uint64_t range, uint32_t log2B,
          uint32_t bshift1, uint64_t nb, uint64_t *__restrict__ keys_out, V *__restrict__ vals_out,
          uint32_t *__restrict__ bucket_start) {
    __shared__ uint32_t hist[kMaxBucketsPerBin];
    __shared__ uint32_t warp_sums[32];
    const uint64_t b_lo = (uint64_t)blockIdx.x << bshift1;
    const uint32_t nbk = (uint32_t)min((uint64_t)1 << bshift1, nb - b_lo);
    const uint32_t lo = off1[blockIdx.x], hi = off1[blockIdx.x + 1];
    for (uint32_t i = threadIdx.x; i < nbk; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint32_t b = (start_slot(keys[i], sigma, range) >> log2B) - (uint32_t)b_lo;
        atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    block_exclusive_scan(hist, nbk, warp_sums);
    for (uint32_t i = threadIdx.x; i < nbk; i += blockDim.x) bucket_start[b_lo + i] = lo + hist[i];
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) bucket_start[nb] = hi;
    __syncthreads();
    for (uint32_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const uint64_t key = keys[i];
        const uint32_t b = (start_slot(key, sigma, range) >> log2B) - (uint32_t)b_lo;
        const uint32_t pos = lo + atomicAdd(&hist[b], 1u);
        keys_out[pos] = key;
        vals_out[pos] = vals[i];
    }
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <typename V>
cudaError_t sort_impl(const LayerDesc &L, const uint64_t *keys, const V *vals, uint64_t *keys_out,
                      V *vals_out, uint32_t *bucket_start, void *scratch, cudaStream_t st) {
    const uint64_t n = L.n;
    const uint32_t log2B = log2_exact(L.B);
    const uint32_t bshift1 = (uint32_t)max(9, (int)ceil_log2(L.nb) - 14);
    const uint32_t shift = log2B + bshift1;
    const uint32_t nbins = (uint32_t)((L.nb + (1ull << bshift1) - 1) >> bshift1);
    if (nbins > kMaxBins1 || (1u << bshift1) > kMaxBucketsPerBin) return cudaErrorInvalidValue;

    char *p = (char *)scratch;
    uint64_t *k1 = (uint64_t *)p;  p += align256(n * 8);
    V *v1 = (V *)p;                p += align256(n * sizeof(V));
    uint32_t *counts = (uint32_t *)p; p += align256((kMaxBins1 + 1) * 4);
    uint32_t *off1 = (uint32_t *)p;   p += align256((kMaxBins1 + 1) * 4);
    uint32_t *cursor = (uint32_t *)p;

    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)nbins * 4, st);
    if (e != cudaSuccess) return e;
    const size_t smem1 = (size_t)nbins * 4;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_l1_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins1 * 4);
        cudaFuncSetAttribute(k_l1_scatter<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins1 * 4);
        cudaFuncSetAttribute(k_l1_scatter<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins1 * 4);
        cudaFuncSetAttribute(k_l1_scatter<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxBins1 * 4);
        attr_set = true;
    }
    const unsigned sms = (unsigned)num_sms();
    k_l1_hist<<<grid_for(n, kL1Threads * 8, sms * 4), kL1Threads, smem1, st>>>(
        keys, n, L.sigma, L.range, shift, nbins, counts);
    k_scan_bins<<<1, 1024, 0, st>>>(counts, nbins, off1, cursor);
    k_l1_scatter<V><<<grid_for(n, kL1Tile, sms * 4), kL1Threads, smem1, st>>>(
        keys, vals, n, L.sigma, L.range, shift, nbins, cursor, k1, v1);
    k_l2_sort<V><<<nbins, kL2Threads, 0, st>>>(k1, v1, off1, L.sigma, L.range, log2B, bshift1, L.nb,
                                               keys_out, vals_out, bucket_start);
    return cudaGetLastError();
}

}  // namespace

size_t sort_scratch_bytes(uint64_t n, uint64_t /*m*/, uint32_t vbytes) {
    return align256(n * 8) + align256(n * vbytes) + 3 * align256((kMaxBins1 + 1) * 4);
}

cudaError_t launch_sort(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                        uint64_t *keys_out, void *vals_out, uint32_t *bucket_start, void *scratch,
                        uint32_t * /*err*/, cudaStream_t st) {
    if (L.n == 0) {
        // every bucket empty
        return cudaMemsetAsync(bucket_start, 0, (size_t)(L.nb + 1) * 4, st);
    }
    switch (vbytes) {
    case 1: return sort_impl<uint8_t>(L, keys, (const uint8_t *)vals, keys_out, (uint8_t *)vals_out,
                                      bucket_start, scratch, st);
    case 2: return sort_impl<uint16_t>(L, keys, (const uint16_t *)vals, keys_out, (uint16_t *)vals_out,
                                       bucket_start, scratch, st);
    default: return sort_impl<uint32_t>(L, keys, (const uint32_t *)vals, keys_out, (uint32_t *)vals_out,
                                        bucket_start, scratch, st);
    }
}

}  // namespace burr
