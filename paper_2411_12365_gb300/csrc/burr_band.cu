// burr_band.cu -- insertion with bumping ("Insertion" of Fig. 7; Sec. 2
// "Bumping" and Sec. 3 "Bumping at thread boundaries") and back-substitution
// ("Back Substitution" of Fig. 7).
//
// One warp per partition.  The paper gives one partition to one CPU thread,
// which eliminates the rows one by one.  Here the 32 lanes of a warp insert a
// whole bucket at once:
//
//   * The kept set of a bucket does not depend on the order of its rows
//     inside a threshold band: the threshold is the smallest level t such
//     that the rows kept so far plus the bucket's rows with offset >= t are
//     linearly independent, and independence is a property of the set.  The
//     table does not depend on it either (unique solution with free slots 0).
//   * So the warp first tries the whole bucket as one set.  Most buckets
//     insert without a dependency.  If the set is dependent it is rolled back
//     and the bands [l2,l3), [l1,l2), [l0,l1) are inserted from the top until
//     one is dependent, which fixes the threshold exactly as the row-by-row
//     elimination in descending offset order would.
//   * A set is inserted in rounds.  Every pending row is reduced against the
//     rows stored so far (read-only) until its leading coefficient sits on an
//     empty slot or the row vanishes (dependent).  Rows that landed on
//     distinct empty slots are then stored together (equivalent to inserting
//     them one after the other, because each one's elimination never touched
//     another's landing slot); rows that landed on an already claimed slot
//     continue in the next round.
//   * The live part of the band, [bucket start, bucket start + 512), sits in a
//     shared-memory ring per warp; slots left behind are final and are
//     written to the global band in coalesced runs.
#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kRing = 512;
constexpr uint32_t kRingMask = kRing - 1;
constexpr int kRPL = 6;                 // rows per lane in one chunk
constexpr uint32_t kChunk = 32 * kRPL;  // rows inserted per round set
constexpr int kBandWarps = 4;           // partitions per CTA
constexpr unsigned kFull = 0xffffffffu;

struct BandWarpSmem {
    uint64_t C[kRing];       // stored coefficient rows (bit 0 = pivot), 0 = empty
    uint32_t Y[kRing];       // stored right-hand sides
    uint16_t claim[kRing];   // landing-slot claims of one round
    uint16_t clist[kRing];   // ring indices stored in the current set (rollback)
};

template <typename V>
struct BandArgs {
    LayerDesc L;
    const uint64_t *keys;
    const V *vals;
    const uint32_t *bstart;
    uint64_t *Cg;
    V *Yg;
    uint64_t *thresh;
    uint64_t *bkeys;
    V *bvals;
    unsigned long long *bcount;
    uint32_t *err;
};

enum { kOk = 0, kDependent = 1, kOverflow = 2 };

__device__ __forceinline__ void rollback(BandWarpSmem &S, uint32_t ncommit, int lane) {
    __syncwarp();
    for (uint32_t i = lane; i < ncommit; i += 32) {
        const uint32_t ri = S.clist[i];
        S.C[ri] = 0;
        S.Y[ri] = 0;
    }
    __syncwarp();
}

// Insert rows [rs, re) of the bucket starting at slot bB whose offset lies in
// [lo, hi), as one set.  On a dependency (or a ring overflow) every row this
// call stored is removed again.
template <typename V>
__device__ int insert_set(BandWarpSmem &S, const BandArgs<V> &a, uint32_t rs, uint32_t re,
                          uint32_t bB, uint32_t lo, uint32_t hi, int lane) {
    const LayerDesc &L = a.L;
    uint32_t ncommit = 0;
    for (uint32_t base = rs; base < re; base += kChunk) {
        uint64_t cur[kRPL];
        uint32_t pos[kRPL], y[kRPL];
        uint32_t act = 0;
#pragma unroll
        for (int k = 0; k < kRPL; ++k) {
            const uint32_t idx = base + (uint32_t)k * 32u + (uint32_t)lane;
            cur[k] = 0;
            pos[k] = 0;
            y[k] = 0;
            if (idx < re) {
                uint32_t s;
                uint64_t c;
                equation(a.keys[idx], L.sigma, L.range, s, c);
                const uint32_t off = s - bB;
                if (off >= lo && off < hi) {
                    cur[k] = c;
                    pos[k] = s;
                    y[k] = (uint32_t)a.vals[idx] & L.vmask;
                    act |= 1u << k;
                }
            }
        }
        while (__any_sync(kFull, act)) {
            bool fail = false, ovf = false;
            uint32_t chase = act;
            while (chase) {
#pragma unroll
                for (int k = 0; k < kRPL; ++k) {
                    if (chase & (1u << k)) {
                        const uint32_t ri = pos[k] & kRingMask;
                        const uint64_t c = S.C[ri];
                        if (c == 0) {
                            chase &= ~(1u << k);           // leading bit on an empty slot
                        } else {
                            cur[k] ^= c;
                            y[k] ^= S.Y[ri];
                            if (cur[k] == 0) {
                                fail = true;               // the row vanished: dependent set
                                chase &= ~(1u << k);
                            } else {
                                const int tz = __ffsll((long long)cur[k]) - 1;
                                pos[k] += (uint32_t)tz;
                                cur[k] >>= tz;
                                if (pos[k] - bB >= (uint32_t)kRing) {
                                    ovf = true;
                                    chase &= ~(1u << k);
                                }
                            }
                        }
                    }
                }
            }
            const bool any_fail = __any_sync(kFull, fail);
            const bool any_ovf = __any_sync(kFull, ovf);
            if (any_fail || any_ovf) {
                rollback(S, ncommit, lane);
                if (any_ovf) {
                    if (lane == 0) atomicOr(a.err, kErrRingOverflow);
                    return kOverflow;
                }
                return kDependent;
            }
            // claim the landing slots; one claimant per slot wins
#pragma unroll
            for (int k = 0; k < kRPL; ++k)
                if (act & (1u << k)) S.claim[pos[k] & kRingMask] = (uint16_t)(lane * kRPL + k);
            __syncwarp();
            uint32_t win = 0;
#pragma unroll
            for (int k = 0; k < kRPL; ++k)
                if ((act & (1u << k)) && S.claim[pos[k] & kRingMask] == (uint16_t)(lane * kRPL + k))
                    win |= 1u << k;
            __syncwarp();
            const uint32_t nw = __popc(win);
            uint32_t incl = nw;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, incl, d);
                if (lane >= d) incl += t;
            }
            const uint32_t total = __shfl_sync(kFull, incl, 31);
            uint32_t o = ncommit + incl - nw;
#pragma unroll
            for (int k = 0; k < kRPL; ++k) {
                if (win & (1u << k)) {
                    const uint32_t ri = pos[k] & kRingMask;
                    S.C[ri] = cur[k];
                    S.Y[ri] = y[k];
                    S.clist[o++] = (uint16_t)ri;
                }
            }
            ncommit += total;
            act &= ~win;
            __syncwarp();
        }
    }
    return kOk;
}

// Rows of the bucket below threshold t leave for the next layer.
template <typename V>
__device__ void emit_bumped(const BandArgs<V> &a, uint32_t rs, uint32_t re, uint32_t bB, uint32_t t,
                            int lane) {
    for (uint32_t base = rs; base < re; base += 32) {
        const uint32_t idx = base + lane;
        bool bump = false;
        uint64_t key = 0;
        V val = 0;
        if (idx < re) {
            key = a.keys[idx];
            bump = (start_slot(key, a.L.sigma, a.L.range) - bB) < t;
            if (bump) val = a.vals[idx];
        }
        const uint32_t mask = __ballot_sync(kFull, bump);
        if (!mask) continue;
        unsigned long long ob = 0;
        if (lane == 0) ob = atomicAdd(a.bcount, (unsigned long long)__popc(mask));
        ob = __shfl_sync(kFull, ob, 0);
        if (bump) {
            const unsigned long long o = ob + __popc(mask & ((1u << lane) - 1u));
            a.bkeys[o] = key;
            a.bvals[o] = val;
        }
    }
}

// Write ring slots [from, to) to the global band and clear them.
template <typename V>
__device__ __forceinline__ void flush(BandWarpSmem &S, const BandArgs<V> &a, uint64_t from, uint64_t to,
                                      int lane) {
    __syncwarp();
    for (uint64_t s = from + lane; s < to; s += 32) {
        const uint32_t ri = (uint32_t)s & kRingMask;
        a.Cg[s] = S.C[ri];
        a.Yg[s] = (V)S.Y[ri];
        S.C[ri] = 0;
        S.Y[ri] = 0;
    }
    __syncwarp();
}

template <typename V>
__global__ void __launch_bounds__(32 * kBandWarps) k_band(BandArgs<V> a) {
    __shared__ BandWarpSmem smem[kBandWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const LayerDesc &L = a.L;
    const uint64_t part = (uint64_t)blockIdx.x * kBandWarps + warp;
    if (part >= L.K) return;
    BandWarpSmem &S = smem[warp];

    const uint64_t b0 = part * L.P / L.B;
    const uint64_t b1 = (part == L.K - 1) ? L.nb : (part + 1) * L.P / L.B;
    const uint64_t own_lo = part == 0 ? 0 : part * L.P + kW;
    const uint64_t own_hi = part == L.K - 1 ? L.m : (part + 1) * L.P + kW;

    for (int i = lane; i < kRing; i += 32) {
        S.C[i] = 0;
        S.Y[i] = 0;
    }
    __syncwarp();

    uint32_t lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) lv[i] = L.levels[i];
    const uint32_t fcode = L.forced_code;
    const uint32_t flevel = lv[fcode & 3];

    uint64_t flushed = own_lo;
    uint64_t tword = 0, twi = b0 >> 5;
    for (uint64_t b = b0; b < b1; ++b) {
        const uint64_t bB = b * L.B;
        if (bB > flushed) {
            flush(S, a, flushed, bB, lane);
            flushed = bB;
        }
        const bool cut = (part > 0 && b == b0 && !L.fallback);
        const uint32_t forced = cut ? flevel : 0;
        uint32_t code = cut ? fcode : 0;
        const uint32_t rs = a.bstart[b], re = a.bstart[b + 1];
        if (re > rs) {
            int rc = insert_set(S, a, rs, re, (uint32_t)bB, forced, L.B, lane);
            if (rc == kOverflow) return;
            if (rc == kDependent) {
                if (L.fallback) {
                    if (lane == 0) atomicOr(a.err, kErrUnsolvable);
                    return;
                }
                code = 3;
                for (int k = 2; k >= 0; --k) {
                    if (lv[k + 1] <= forced) break;
                    const uint32_t lo = max(lv[k], forced), hi = lv[k + 1];
                    const int rc2 = insert_set(S, a, rs, re, (uint32_t)bB, lo, hi, lane);
                    if (rc2 == kOverflow) return;
                    if (rc2 == kDependent) {
                        code = (uint32_t)k + 1;
                        break;
                    }
                    code = (lv[k] >= forced) ? (uint32_t)k : fcode;
                }
            }
            const uint32_t t = lv[code];
            if (!L.fallback && t > 0) emit_bumped(a, rs, re, (uint32_t)bB, t, lane);
        }
        if (!L.fallback) {
            if ((b >> 5) != twi) {
                if (lane == 0 && tword) atomicOr((unsigned long long *)&a.thresh[twi], (unsigned long long)tword);
                tword = 0;
                twi = b >> 5;
            }
            tword |= (uint64_t)code << (2 * (b & 31));
        }
    }
    if (!L.fallback && lane == 0 && tword)
        atomicOr((unsigned long long *)&a.thresh[twi], (unsigned long long)tword);
    flush(S, a, flushed, own_hi, lane);
}

// Back-substitution, right to left over the partition's owned slots, one
// lane per value bit: Z[i] = Y[i] ^ parity((C[i] >> 1) & Z[i+1 .. i+63]),
// Z[i] = 0 on empty slots (C = Y = 0 there).  The 64-bit register `st` holds
// Z of the 64 slots to the right of the current one; after a block of 64
// slots it is exactly that block's table word for this bit plane.
constexpr int kBsWarps = 4;

template <typename V>
__global__ void __launch_bounds__(32 * kBsWarps)
k_backsub(LayerDesc L, const uint64_t *__restrict__ Cg, const V *__restrict__ Yg, uint64_t *__restrict__ Z) {
    __shared__ uint64_t sc[kBsWarps][64];
    __shared__ uint32_t sy[kBsWarps][64];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t part = (uint64_t)blockIdx.x * kBsWarps + warp;
    if (part >= L.K) return;
    const uint64_t own_lo = part == 0 ? 0 : part * L.P + kW;
    const uint64_t own_hi = part == L.K - 1 ? L.m : (part + 1) * L.P + kW;
    const uint64_t blo = own_lo >> 6, bhi = own_hi >> 6;
    if (bhi <= blo) return;
    uint64_t st = 0;
    // software pipeline: registers hold the next block while this one is solved
    uint64_t nc0 = Cg[((bhi - 1) << 6) + lane], nc1 = Cg[((bhi - 1) << 6) + lane + 32];
    uint32_t ny0 = Yg[((bhi - 1) << 6) + lane], ny1 = Yg[((bhi - 1) << 6) + lane + 32];
    for (uint64_t blk = bhi; blk-- > blo;) {
        __syncwarp();
        sc[warp][lane] = nc0 >> 1;
        sc[warp][lane + 32] = nc1 >> 1;
        sy[warp][lane] = ny0;
        sy[warp][lane + 32] = ny1;
        __syncwarp();
        if (blk > blo) {
            const uint64_t s0 = (blk - 1) << 6;
            nc0 = Cg[s0 + lane];
            nc1 = Cg[s0 + lane + 32];
            ny0 = Yg[s0 + lane];
            ny1 = Yg[s0 + lane + 32];
        }
        if ((uint32_t)lane < L.r) {
#pragma unroll 16
            for (int i = 63; i >= 0; --i) {
                const uint64_t c = sc[warp][i];
                const uint32_t z = ((sy[warp][i] >> lane) & 1u) ^ (__popcll(c & st) & 1u);
                st = (st << 1) | z;
            }
            Z[blk * L.r + lane] = st;
        }
    }
}

template <typename V>
cudaError_t band_impl(const LayerDesc &L, const uint64_t *keys, const V *vals, const uint32_t *bstart,
                      uint64_t *Cg, V *Yg, uint64_t *thresh, uint64_t *bkeys, V *bvals,
                      unsigned long long *bcount, uint32_t *err, cudaStream_t st) {
    BandArgs<V> a;
    a.L = L;
    a.keys = keys;
    a.vals = vals;
    a.bstart = bstart;
    a.Cg = Cg;
    a.Yg = Yg;
    a.thresh = thresh;
    a.bkeys = bkeys;
    a.bvals = bvals;
    a.bcount = bcount;
    a.err = err;
    const unsigned grid = (unsigned)((L.K + kBandWarps - 1) / kBandWarps);
    k_band<V><<<grid, 32 * kBandWarps, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_band(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                        const uint32_t *bucket_start, uint64_t *Cg, void *Yg, uint64_t *thresh,
                        uint64_t *bumped_keys, void *bumped_vals, unsigned long long *bumped_count,
                        uint32_t *err, cudaStream_t st) {
    if (L.K == 0) return cudaSuccess;
    switch (vbytes) {
    case 1:
        return band_impl<uint8_t>(L, keys, (const uint8_t *)vals, bucket_start, Cg, (uint8_t *)Yg, thresh,
                                  bumped_keys, (uint8_t *)bumped_vals, bumped_count, err, st);
    case 2:
        return band_impl<uint16_t>(L, keys, (const uint16_t *)vals, bucket_start, Cg, (uint16_t *)Yg, thresh,
                                   bumped_keys, (uint16_t *)bumped_vals, bumped_count, err, st);
    default:
        return band_impl<uint32_t>(L, keys, (const uint32_t *)vals, bucket_start, Cg, (uint32_t *)Yg, thresh,
                                   bumped_keys, (uint32_t *)bumped_vals, bumped_count, err, st);
    }
}

cudaError_t launch_backsub(const LayerDesc &L, uint32_t vbytes, const uint64_t *Cg, const void *Yg,
                           uint64_t *Z, cudaStream_t st) {
    if (L.K == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((L.K + kBsWarps - 1) / kBsWarps);
    switch (vbytes) {
    case 1: k_backsub<uint8_t><<<grid, 32 * kBsWarps, 0, st>>>(L, Cg, (const uint8_t *)Yg, Z); break;
    case 2: k_backsub<uint16_t><<<grid, 32 * kBsWarps, 0, st>>>(L, Cg, (const uint16_t *)Yg, Z); break;
    default: k_backsub<uint32_t><<<grid, 32 * kBsWarps, 0, st>>>(L, Cg, (const uint32_t *)Yg, Z); break;
    }
    return cudaGetLastError();
}

}  // namespace burr
