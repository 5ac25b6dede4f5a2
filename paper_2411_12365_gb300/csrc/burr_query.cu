// burr_query.cu -- the layered query (Sec. 2: AND the key's coefficients with
// the table window, parity per value bit; a key below its bucket's threshold
// was bumped and is looked up in the next layer; the threshold is a 2-bit
// level code or, with 1+-bit thresholds, 0 unless the bucket's flag is set)
// and the standalone hash stage.
#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kQThreads = 256;

// Parity of a 64-bit word.
__device__ __forceinline__ uint32_t parity64q(uint64_t x) {
    return (uint32_t)__popc((uint32_t)x ^ (uint32_t)(x >> 32)) & 1u;
}

// Bit k of the value is the parity of c AND the 64 table bits of plane k from
// slot s on.  Those bits are bits o.. of block word w0 and bits ..o-1 of the
// next block's word w1 (o = s mod 64), so the parity is that of
// (w0 & (c << o)) ^ (w1 & (c >> (64 - o))): the row is shifted once per key
// instead of the window once per plane.
__device__ __forceinline__ void row_masks(uint64_t c, uint32_t o, uint64_t &cA, uint64_t &cB) {
    cA = c << o;
    cB = o ? c >> (64 - o) : 0ull;
}

// r-bit value of the window [s, s+63] selected by coefficient row c.
__device__ __forceinline__ uint32_t eval_window(const uint64_t *__restrict__ z, uint32_t r, uint32_t s,
                                                uint64_t c) {
    const uint64_t blk = s >> 6;
    const uint32_t o = s & 63u;
    const uint64_t *w0 = z + blk * r;
    uint64_t cA, cB;
    row_masks(c, o, cA, cB);
    uint32_t v = 0;
    if (o == 0) {
        for (uint32_t k = 0; k < r; ++k) v |= parity64q(__ldg(w0 + k) & cA) << k;
    } else {
        const uint64_t *w1 = w0 + r;
        for (uint32_t k = 0; k < r; ++k) v |= parity64q((__ldg(w0 + k) & cA) ^ (__ldg(w1 + k) & cB)) << k;
    }
    return v;
}

// The 2r table words around slot s (blocks s/64 and s/64 + 1), loaded before
// the threshold is known so that both reads are in flight together; R is the
// value width fixed at compile time.  The second block is needed only when the
// window is not block-aligned, and a window that starts at the last block
// (s = m - 64) has no second block inside the table: it is not read then.
template <int R>
struct Window {
    uint64_t w0[R], w1[R];
};

// 32-byte read-only global load (four table words).
__device__ __forceinline__ void ldg_v4(const uint64_t *p, uint64_t &a, uint64_t &b, uint64_t &c, uint64_t &d) {
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

// kWide: the table starts on 32 bytes and R is a multiple of 4, so each block
// of R words is read in R/4 32-byte loads (checked by the launcher).  Narrow
// reads of random windows cost one L1 wavefront per word and warp lane.
template <int R, bool kWide>
__device__ __forceinline__ void load_window(const uint64_t *__restrict__ z, uint32_t s, Window<R> &w) {
    const uint64_t *p = z + (uint64_t)(s >> 6) * R;
    const bool two = (s & 63u) != 0u;
    if constexpr (kWide) {
        static_assert(R % 4 == 0, "wide window loads need R % 4 == 0");
#pragma unroll
        for (int k = 0; k < R; k += 4) ldg_v4(p + k, w.w0[k], w.w0[k + 1], w.w0[k + 2], w.w0[k + 3]);
#pragma unroll
        for (int k = 0; k < R; ++k) w.w1[k] = 0;
        if (two) {
#pragma unroll
            for (int k = 0; k < R; k += 4) ldg_v4(p + R + k, w.w1[k], w.w1[k + 1], w.w1[k + 2], w.w1[k + 3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
            w.w0[k] = __ldg(p + k);
            w.w1[k] = two ? __ldg(p + R + k) : 0ull;
        }
    }
}

template <int R>
__device__ __forceinline__ uint32_t eval_loaded(const Window<R> &w, uint32_t s, uint64_t c) {
    uint64_t cA, cB;
    row_masks(c, s & 63u, cA, cB);   // w1 is zero when the window is block-aligned
    uint32_t v = 0;
#pragma unroll
    for (int k = 0; k < R; ++k) v |= parity64q((w.w0[k] & cA) ^ (w.w1[k] & cB)) << k;
    return v;
}

// Threshold t of bucket b of bumping layer l: keys with offset < t are bumped.
__device__ __forceinline__ uint32_t threshold_of(const QueryDesc &Q, uint32_t l, uint32_t b) {
    if (Q.mode == BURR_THRESH_1PLUS) {
        // flag bit; a flagged bucket's threshold sits at its rank
        const uint64_t *fl = Q.flags[l];
        const uint64_t w = __ldg(fl + (b >> 6));
        if (!((w >> (b & 63u)) & 1ull)) return 0;
        uint32_t rank = __ldg(Q.dir[l] + (b >> 9));
        for (uint32_t k = (b >> 9) << 3; k < (b >> 6); ++k) rank += (uint32_t)__popcll(__ldg(fl + k));
        rank += (uint32_t)__popcll(w & ((1ull << (b & 63u)) - 1ull));
        return __ldg(Q.tbytes[l] + rank);
    }
    return Q.levels[(uint32_t)(__ldg(Q.thresh[l] + (b >> 5)) >> (2 * (b & 31))) & 3u];
}

// Query kernel for a value width R known at compile time: the table window
// of a layer is loaded together with its threshold, and the thread's next key
// is read while this key's table reads are in flight.  Measured (ms per query
// of n keys, half members): 10^9 keys r = 8 72.5 either way, 10^8 keys r = 16
// 4.45 -> 4.20, r = 1 0.79 either way.  Two keys per thread (their layer-0
// reads in flight together, 98 registers) gave 70.7 at 10^9 but 4.69 and 0.89
// at 10^8 (r = 16, r = 1).
template <typename V, int R, bool kWide>
__global__ void __launch_bounds__(kQThreads)
k_query_r(QueryDesc Q, const uint64_t *__restrict__ keys, V *__restrict__ out, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t log2B = 31 - __clz(Q.B);
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t key_next = i < n ? keys[i] : 0ull;
    for (; i < n; i += stride) {
        const uint64_t key = key_next;
        if (i + stride < n) key_next = keys[i + stride];
        uint32_t v = 0;
        uint32_t l = 0;
        for (; l < Q.layers; ++l) {
            const uint64_t m = Q.m[l];
            if (m == 0) break;
            const uint64_t h = mix64(key ^ Q.sigma[l]);
            const uint32_t s = (uint32_t)__umul64hi(h, m - kW + 1);
            Window<R> w;
            load_window<R, kWide>(Q.z[l], s, w);
            if ((s & (Q.B - 1)) < threshold_of(Q, l, s >> log2B)) continue;   // bumped: next layer
            v = eval_loaded<R>(w, s, mix64(h + Q.sigma[l]) | 1ull);
            break;
        }
        if (l == Q.layers && Q.m[l] != 0) {                    // base case
            const uint64_t h = mix64(key ^ Q.sigma[l]);
            const uint32_t s = (uint32_t)__umul64hi(h, Q.m[l] - kW + 1);
            Window<R> w;
            load_window<R, kWide>(Q.z[l], s, w);
            v = eval_loaded<R>(w, s, mix64(h + Q.sigma[l]) | 1ull);
        }
        out[i] = (V)v;
    }
}

template <typename V>
__global__ void __launch_bounds__(kQThreads)
k_query(QueryDesc Q, const uint64_t *__restrict__ keys, V *__restrict__ out, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint32_t log2B = 31 - __clz(Q.B);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t key = keys[i];
        uint32_t v = 0;
        uint32_t l = 0;
        for (; l < Q.layers; ++l) {
            const uint64_t m = Q.m[l];
            if (m == 0) break;
            const uint64_t h = mix64(key ^ Q.sigma[l]);
            const uint32_t s = (uint32_t)__umul64hi(h, m - kW + 1);
            const uint32_t b = s >> log2B;
            const uint32_t off = s & (Q.B - 1);
            const uint32_t t = threshold_of(Q, l, b);
            if (off < t) continue;                             // bumped: next layer
            v = eval_window(Q.z[l], Q.r, s, mix64(h + Q.sigma[l]) | 1ull);
            break;
        }
        if (l == Q.layers && Q.m[l] != 0) {                    // base case
            const uint64_t h = mix64(key ^ Q.sigma[l]);
            const uint32_t s = (uint32_t)__umul64hi(h, Q.m[l] - kW + 1);
            v = eval_window(Q.z[l], Q.r, s, mix64(h + Q.sigma[l]) | 1ull);
        }
        out[i] = (V)v;
    }
}

__global__ void k_hash(const uint64_t *__restrict__ keys, uint64_t n, uint64_t sigma, uint64_t range,
                       uint32_t *__restrict__ start, uint64_t *__restrict__ coeff) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint32_t s;
        uint64_t c;
        equation(keys[i], sigma, range, s, c);
        start[i] = s;
        coeff[i] = c;
    }
}

}  // namespace

cudaError_t launch_query(const QueryDesc &Q, uint32_t vbytes, const uint64_t *keys, void *out, uint64_t n,
                         cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const unsigned grid = grid_for(n, kQThreads, 152u * 64u);
    // common widths: the window is loaded together with the threshold, in 32-byte reads when
    // every table of the structure starts on 32 bytes
    bool wide = true;
    for (uint32_t l = 0; l <= Q.layers; ++l)
        if (Q.m[l] != 0 && ((uintptr_t)Q.z[l] & 31u) != 0) wide = false;
    if (Q.r == 8 && vbytes == 1) {
        if (wide) k_query_r<uint8_t, 8, true><<<grid, kQThreads, 0, st>>>(Q, keys, (uint8_t *)out, n);
        else k_query_r<uint8_t, 8, false><<<grid, kQThreads, 0, st>>>(Q, keys, (uint8_t *)out, n);
        return cudaGetLastError();
    }
    if (Q.r == 1 && vbytes == 1) {
        k_query_r<uint8_t, 1, false><<<grid, kQThreads, 0, st>>>(Q, keys, (uint8_t *)out, n);
        return cudaGetLastError();
    }
    if (Q.r == 16 && vbytes == 2) {
        if (wide) k_query_r<uint16_t, 16, true><<<grid, kQThreads, 0, st>>>(Q, keys, (uint16_t *)out, n);
        else k_query_r<uint16_t, 16, false><<<grid, kQThreads, 0, st>>>(Q, keys, (uint16_t *)out, n);
        return cudaGetLastError();
    }
    switch (vbytes) {
    case 1: k_query<uint8_t><<<grid, kQThreads, 0, st>>>(Q, keys, (uint8_t *)out, n); break;
    case 2: k_query<uint16_t><<<grid, kQThreads, 0, st>>>(Q, keys, (uint16_t *)out, n); break;
    default: k_query<uint32_t><<<grid, kQThreads, 0, st>>>(Q, keys, (uint32_t *)out, n); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_hash(const uint64_t *keys, uint64_t n, uint64_t sigma, uint64_t range, uint32_t *start,
                        uint64_t *coeff, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_hash<<<grid_for(n, 256, 152u * 32u), 256, 0, st>>>(keys, n, sigma, range, start, coeff);
    return cudaGetLastError();
}

}  // namespace burr
