// burr_thresh.cu -- storage of 1+-bit thresholds (Sec. 2: one bit per bucket
// says whether the bucket bumped anything; only those buckets keep their
// exact threshold).
//
// The band kernel leaves the exact threshold t of every bucket in a byte array.
// Here it becomes, per structure layer:
//   flags  one bit per bucket (bit b%64 of word b/64), set iff t > 0;
//   dir    per block of 512 buckets (8 flag words) the number of flagged
//          buckets before the block, counted over the whole launch;
//   bytes  the thresholds of the flagged buckets in bucket order.
// A query of bucket b reads its flag word; if the bit is set, its threshold is
// bytes[dir[b/512] + flagged buckets of the block before b].  The directory
// takes the place of the paper's small hash table: the same information
// (which buckets bump, and their exact thresholds), looked up by a rank
// instead of a probe.
#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kBlkBuckets = 512;   // buckets per directory entry
constexpr int kThreads = 256;      // 8 warps: one flag word each

__global__ void __launch_bounds__(kThreads)
k_tflags(const uint8_t *__restrict__ texact, const ThreshSeg *__restrict__ segs, const uint32_t *__restrict__ blk_seg,
         uint64_t *__restrict__ flags, uint32_t *__restrict__ counts) {
    __shared__ uint32_t wc[kThreads / 32];
    const uint32_t blk = blockIdx.x;
    const ThreshSeg g = segs[blk_seg[blk]];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t word = (uint64_t)(blk - g.dir_base) * (kBlkBuckets / 64) + warp;   // local flag word
    uint32_t cnt = 0;
    if (word * 64 < g.nb) {
        const uint64_t b = word * 64 + lane;
        const bool f0 = b < g.nb && texact[g.bucket_base + b] != 0;
        const bool f1 = b + 32 < g.nb && texact[g.bucket_base + b + 32] != 0;
        const unsigned lo = __ballot_sync(0xffffffffu, f0), hi = __ballot_sync(0xffffffffu, f1);
        if (lane == 0) flags[g.fw_base + word] = (uint64_t)lo | ((uint64_t)hi << 32);
        cnt = (uint32_t)(__popc(lo) + __popc(hi));
    }
    if (lane == 0) wc[warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += wc[w];
        counts[blk] = t;
    }
}

// Exclusive scan of counts[0..n) into dir[0..n], dir[n] = total (one block).
__global__ void __launch_bounds__(1024) k_tscan(const uint32_t *__restrict__ counts, uint32_t n, uint32_t *dir) {
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t base = 0; base < n; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < n ? counts[i] : 0u;
        uint32_t incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            uint32_t s = ws[lane], si = s;
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, si, d);
                if (lane >= d) si += t;
            }
            ws[lane] = si - s;   // exclusive warp offsets
        }
        __syncthreads();
        const uint32_t c = carry;
        if (i < n) dir[i] = c + ws[warp] + incl - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry = c + ws[warp] + incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) dir[n] = carry;
}

__global__ void __launch_bounds__(kThreads)
k_tcompact(const uint8_t *__restrict__ texact, const ThreshSeg *__restrict__ segs,
           const uint32_t *__restrict__ blk_seg, const uint64_t *__restrict__ flags, const uint32_t *__restrict__ dir,
           uint8_t *__restrict__ bytes) {
    __shared__ uint32_t wc[kThreads / 32];
    const uint32_t blk = blockIdx.x;
    const ThreshSeg g = segs[blk_seg[blk]];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t word = (uint64_t)(blk - g.dir_base) * (kBlkBuckets / 64) + warp;
    const bool valid = word * 64 < g.nb;
    const uint64_t f = valid ? flags[g.fw_base + word] : 0ull;
    if (lane == 0) wc[warp] = (uint32_t)__popcll(f);
    __syncthreads();
    uint32_t base = dir[blk];
    for (int w = 0; w < warp; ++w) base += wc[w];
    if (!valid) return;
    const uint32_t lo = (uint32_t)f, hi = (uint32_t)(f >> 32);
    const unsigned lt = (1u << lane) - 1u;
    if ((lo >> lane) & 1u) bytes[base + __popc(lo & lt)] = texact[g.bucket_base + word * 64 + lane];
    if ((hi >> lane) & 1u)
        bytes[base + __popc(lo) + __popc(hi & lt)] = texact[g.bucket_base + word * 64 + 32 + lane];
}

}  // namespace

cudaError_t launch_thresh_flags(const uint8_t *texact, const ThreshSeg *segs, const uint32_t *blk_seg, uint32_t nblk,
                                uint64_t *flags, uint32_t *counts, uint32_t *dir, cudaStream_t st) {
    if (nblk == 0) return cudaMemsetAsync(dir, 0, 4, st);
    cudaError_t e;
    if ((e = prefer_shared(k_tflags)) != cudaSuccess || (e = prefer_shared(k_tscan)) != cudaSuccess) return e;
    k_tflags<<<nblk, kThreads, 0, st>>>(texact, segs, blk_seg, flags, counts);
    k_tscan<<<1, 1024, 0, st>>>(counts, nblk, dir);
    return cudaGetLastError();
}

cudaError_t launch_thresh_compact(const uint8_t *texact, const ThreshSeg *segs, const uint32_t *blk_seg,
                                  uint32_t nblk, const uint64_t *flags, const uint32_t *dir, uint8_t *bytes,
                                  cudaStream_t st) {
    if (nblk == 0) return cudaSuccess;
    const cudaError_t e = prefer_shared(k_tcompact);
    if (e != cudaSuccess) return e;
    k_tcompact<<<nblk, kThreads, 0, st>>>(texact, segs, blk_seg, flags, dir, bytes);
    return cudaGetLastError();
}

}  // namespace burr
