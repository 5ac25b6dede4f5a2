// burr_cuts.cu -- cut-point search (Sec. 3, "Selecting Cut Points"): move each
// cut to a nearby bucket where the cut bumps fewer keys, or where more keys
// sit in the w-1 slots before it (they fill the gap the cut leaves).
//
// Cut j (1 <= j < K) is chosen among the buckets b0 .. b0+R-1, b0 = j*P/B,
// R = min(range, P/B).  For a cut at bucket b:
//   bumped(b) = keys of bucket b at offsets < w (cut away by the forced level)
//   prev(b)   = keys of bucket b-1 at offsets >= B - (w-1)
// minbump minimises bumped, maxprev maximises prev, diff minimises
// bumped - prev; the first best candidate wins.  One warp per partition j:
// j = 0 writes the table's ends, j >= 1 searches cut j.
#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kCutWarps = 4;

// Keys of global bucket g whose offset o satisfies lo <= o < hi (warp-wide).
__device__ __forceinline__ uint32_t count_offsets(const uint64_t *__restrict__ keys,
                                                  const uint32_t *__restrict__ bstart, const LayerDesc &L,
                                                  uint64_t g, uint64_t b, uint32_t lo, uint32_t hi, int lane) {
    uint32_t c = 0;
    const uint32_t e = bstart[g + 1];
    for (uint32_t i = bstart[g] + (uint32_t)lane; i < e; i += 32) {
        const uint32_t o = start_of_h(keys[i], L.range) - (uint32_t)(b * L.B);   // keys[] holds records h
        c += (o >= lo && o < hi) ? 1u : 0u;
    }
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    return c;
}

__global__ void __launch_bounds__(32 * kCutWarps)
k_cut_search(LayerDesc L0, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ bstart, uint32_t mode,
             uint32_t range, uint32_t *cuts0, BatchView bv) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t gp = (uint64_t)blockIdx.x * kCutWarps + warp;
    LayerDesc L;
    uint64_t j, bucket_base = 0;
    uint32_t *cuts = cuts0;
    if (bv.sd) {
        if (gp >= bv.nparts) return;
        const StructDesc &D = bv.sd[bv.part_struct[gp]];
        L = D.L;
        j = gp - D.part_base;
        bucket_base = D.bucket_base;
        cuts = const_cast<uint32_t *>(D.L.cuts);
    } else {
        if (gp >= L0.K) return;
        L = L0;
        j = gp;
    }
    if (!cuts) return;   // a structure layer without cuts to search
    if (j == 0) {
        if (lane == 0) {
            cuts[0] = 0;
            cuts[L.K] = (uint32_t)L.nb;
        }
        return;
    }
    const uint64_t b0 = j * L.P / L.B;
    const uint64_t R = min((uint64_t)range, L.P / L.B);
    uint64_t best_b = b0;
    int64_t best = 0;
    for (uint64_t b = b0; b < b0 + R && b < L.nb; ++b) {
        const int64_t bumped = count_offsets(keys, bstart, L, bucket_base + b, b, 0u, kW, lane);
        const int64_t prev =
            b > 0 ? count_offsets(keys, bstart, L, bucket_base + b - 1, b - 1, L.B - (kW - 1), L.B, lane) : 0;
        const int64_t score = mode == BURR_CUT_MINBUMP ? bumped : (mode == BURR_CUT_MAXPREV ? -prev : bumped - prev);
        if (b == b0 || score < best) {
            best = score;
            best_b = b;
        }
    }
    if (lane == 0) cuts[j] = (uint32_t)best_b;
}

}  // namespace

cudaError_t launch_cut_search(const LayerDesc &L, const uint64_t *sorted_keys, const uint32_t *bucket_start,
                              uint32_t mode, uint32_t range, uint32_t *cuts, cudaStream_t st, const BatchView *bv) {
    const uint64_t parts = bv ? bv->nparts : L.K;
    if (parts == 0) return cudaSuccess;
    const BatchView v = bv ? *bv : BatchView();
    const unsigned grid = (unsigned)((parts + kCutWarps - 1) / kCutWarps);
    const cudaError_t e = prefer_shared(k_cut_search);
    if (e != cudaSuccess) return e;
    k_cut_search<<<grid, 32 * kCutWarps, 0, st>>>(L, sorted_keys, bucket_start, mode, range, cuts, v);
    return cudaGetLastError();
}

}  // namespace burr
