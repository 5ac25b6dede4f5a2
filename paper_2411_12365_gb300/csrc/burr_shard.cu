// burr_shard.cu -- routing of (key, value) records to the ranks of a sharded
// build (Sec. 3: once the cuts of a layer are placed its partitions are
// independent, so ranks that own disjoint, contiguous ranges of partitions can
// insert and back-substitute them without talking to each other; a key goes
// to the rank whose range holds its start bucket).
//
// Two launches: a count of the keys per rank (block histograms in shared
// memory, one global atomic per block and rank), then, after the host has
// turned the counts into each rank's first output position, a scatter in
// which every block reserves its run per rank with one atomic and places its
// keys inside it.  The order inside a rank's run is not fixed; nothing
// downstream depends on it (a layer's structure is a property of its key set).
#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kRouteThreads = 256;

// Owner rank of partition `part`: the g with part_first[g] <= part < part_first[g+1].
__device__ __forceinline__ uint32_t owner_of(uint32_t part, const uint32_t *part_first, uint32_t ranks) {
    uint32_t lo = 0, hi = ranks;          // part_first[lo] <= part < part_first[hi]
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (part_first[mid] <= part) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Partition of the key's start bucket: cuts at j*P, the last partition takes the rest.
__device__ __forceinline__ uint32_t partition_of(const LayerDesc &L, uint64_t key) {
    const uint64_t b = start_slot(key, L.sigma, L.range) / L.B;
    const uint64_t j = b / (L.P / L.B);
    return (uint32_t)(j < L.K ? j : L.K - 1);
}

template <typename V>
__global__ void __launch_bounds__(kRouteThreads)
k_route(LayerDesc L, const uint64_t *__restrict__ keys, const V *__restrict__ vals, const uint32_t *__restrict__ part_first,
        uint32_t ranks, uint32_t *__restrict__ rank_of, unsigned long long *__restrict__ counts,
        unsigned long long *__restrict__ cursor, uint64_t *__restrict__ keys_out, V *__restrict__ vals_out,
        bool count_only) {
    __shared__ unsigned int hist[kMaxShardRanks];
    __shared__ unsigned long long base[kMaxShardRanks];
    for (uint32_t g = threadIdx.x; g < ranks; g += blockDim.x) hist[g] = 0;
    __syncthreads();
    // each block covers one contiguous tile per pass, so that the scatter sees
    // the same tiles as the count
    const uint64_t tile = (uint64_t)blockDim.x * 8;
    for (uint64_t t0 = (uint64_t)blockIdx.x * tile; t0 < L.n; t0 += (uint64_t)gridDim.x * tile) {
        uint32_t own[8], slot[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            own[k] = 0xffffffffu;
            if (i < L.n) {
                own[k] = count_only ? owner_of(partition_of(L, keys[i]), part_first, ranks) : rank_of[i];
                slot[k] = atomicAdd(&hist[own[k]], 1u);
                if (count_only) rank_of[i] = own[k];
            }
        }
        if (count_only) continue;
        __syncthreads();
        // reserve this tile's run of every rank, then place the keys
        for (uint32_t g = threadIdx.x; g < ranks; g += blockDim.x) {
            base[g] = hist[g] ? atomicAdd(&cursor[g], (unsigned long long)hist[g]) : 0ull;
            hist[g] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint64_t i = t0 + threadIdx.x + (uint64_t)k * blockDim.x;
            if (own[k] != 0xffffffffu) {
                const unsigned long long o = base[own[k]] + slot[k];
                keys_out[o] = keys[i];
                vals_out[o] = vals[i];
            }
        }
        __syncthreads();
    }
    if (count_only) {
        __syncthreads();
        for (uint32_t g = threadIdx.x; g < ranks; g += blockDim.x)
            if (hist[g]) atomicAdd(&counts[g], (unsigned long long)hist[g]);
    }
}

template <typename V>
cudaError_t route_impl(const LayerDesc &L, const uint64_t *keys, const V *vals, const uint32_t *part_first,
                       uint32_t ranks, uint32_t *rank_of, unsigned long long *counts, unsigned long long *cursor,
                       uint64_t *keys_out, V *vals_out, bool count_only, cudaStream_t st) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = grid_for(L.n, kRouteThreads * 8, (unsigned)sms * 8);
    k_route<V><<<grid, kRouteThreads, 0, st>>>(L, keys, vals, part_first, ranks, rank_of, counts, cursor, keys_out,
                                               vals_out, count_only);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_route(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                         const uint32_t *part_first, uint32_t ranks, uint32_t *rank_of,
                         unsigned long long *counts, unsigned long long *cursor, uint64_t *keys_out,
                         void *vals_out, bool count_only, cudaStream_t st) {
    if (L.n == 0) return cudaSuccess;
    if (ranks == 0 || ranks > kMaxShardRanks) return cudaErrorInvalidValue;
    switch (vbytes) {
    case 1:
        return route_impl<uint8_t>(L, keys, (const uint8_t *)vals, part_first, ranks, rank_of, counts, cursor, keys_out,
                                   (uint8_t *)vals_out, count_only, st);
    case 2:
        return route_impl<uint16_t>(L, keys, (const uint16_t *)vals, part_first, ranks, rank_of, counts, cursor,
                                    keys_out, (uint16_t *)vals_out, count_only, st);
    default:
        return route_impl<uint32_t>(L, keys, (const uint32_t *)vals, part_first, ranks, rank_of, counts, cursor,
                                    keys_out, (uint32_t *)vals_out, count_only, st);
    }
}

}  // namespace burr
