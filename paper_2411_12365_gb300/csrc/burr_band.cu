// burr_band.cu -- insertion with bumping ("Insertion" of Fig. 7; Sec. 2
// "Bumping" and Sec. 3 "Bumping at thread boundaries") and back-substitution
// ("Back Substitution" of Fig. 7).
//
// One warp per partition.  The paper gives one partition to one CPU thread,
// which eliminates the rows one by one.  Here the 32 lanes of a warp insert a
// bucket together:
//
//   * The kept set of a bucket does not depend on the order of its rows
//     inside a threshold band: the threshold is the smallest level t such
//     that the rows kept so far plus the bucket's rows with offset >= t are
//     linearly independent, and independence is a property of the set.  The
//     table does not depend on it either (unique solution with free slots 0).
//   * So the warp first inserts the whole bucket as one set.  Most buckets
//     insert without a dependency.  If the set is dependent it is rolled back
//     and, with 2-bit thresholds, the rows [l1, B), then [l2, B), are tried as
//     one set each until one inserts, which fixes the threshold exactly as the
//     row-by-row elimination in descending offset order would.
//   * With 1+-bit thresholds (exact threshold t in [0, B]) t is the least
//     value for which the rows at offsets >= t insert.  The first pass over
//     the bucket carries row tags and drops dependent rows instead of
//     stopping.  The dropped rows' tags span the set's dependencies, and t
//     follows from them (insert_tagged).  The rows at offsets >= t are then
//     inserted again as one set.  Where the tags cannot place a dependency,
//     t is found by probes instead: a set of rows is independent whenever a
//     superset is, so each probe inserts the rows of [mid, t_ok) on top of
//     those already kept and either keeps them (t_ok = mid) or rolls them
//     back (t_fail = mid).
//   * A set is inserted as a stream: the 32 lanes eliminate one row each and
//     take their steps in lockstep.  A step is one 128-bit compare-and-swap
//     on the ring slot of the row's leading bit, which either claims the
//     slot if it is empty (row and right-hand side stored in one atomic
//     write) or returns the stored row and right-hand side to XOR with.  Plain
//     reads of the next two slots are in flight beside the swap, and the
//     elimination goes on through those that hold stored rows.  This
//     is a sequential insertion in claim order: every slot a row eliminated
//     against was occupied when read and stays so, and a row is stored only
//     on a slot that was still empty.  Lanes whose row was stored take the
//     next rows of the set, and the stored slots are listed for a rollback,
//     by ballot and prefix count; a dependent row ends the set at once.
//   * Rows are staged per bucket in shared memory in ascending offset order
//     (a counting sort on the 7-bit offset), so each threshold band is a
//     contiguous range and rows that run through the dense overflow of the
//     previous buckets start first.
//   * The live part of the band, [bucket start, bucket start + 512), sits in a
//     shared-memory ring per warp; slots left behind are final and are
//     written to the global band in coalesced runs.
#include "burr_internal.cuh"

namespace burr {

namespace {

constexpr int kRing = 512;
constexpr uint32_t kRingMask = kRing - 1;
constexpr int kStage = 256;             // rows of a bucket staged at once
constexpr int kStagePerLane = kStage / 32;
// Partitions (warps) per CTA.  Small CTAs spread partitions evenly over the
// SMs (1503 partitions at 10^8 keys fill ~10 of the 12 warp slots per SM) and
// give a finer tail; 2 measured best against 1 and 4.
#ifndef BURR_BAND_WARPS
#define BURR_BAND_WARPS 2
#endif
constexpr int kBandWarps = BURR_BAND_WARPS;
constexpr unsigned kFull = 0xffffffffu;

constexpr unsigned long long kYValid = 1ull << 32;   // marks a stored right-hand side

struct alignas(16) RingSlot {
    unsigned long long c;   // stored coefficient row (bit 0 = pivot), 0 = empty
    unsigned long long y;   // kYValid | right-hand side (low r bits); 0 = empty
};

// A staged equation: one 16-byte read hands it to a lane.
struct alignas(16) StagedRow {
    unsigned long long c;   // coefficient row (bit 0 = start slot)
    uint32_t y;             // right-hand side
    uint32_t o;             // offset of the start slot in its bucket
};

// Ring slots read ahead of the swap in each step (see stream_insert), per
// threshold mode: more read-ahead means fewer steps but more instructions per
// step, and with many warps per SM competing for issue slots two measured
// best in both modes (10^8 keys, r=8; 1+-bit: 1, 2, 3, 4 slots gave 27.2,
// 26.6, 27.5, 27.6 ms per build and query step; 2-bit, layer-0 band of 10^9
// keys: 68.2, 65.9, 69.0, 80.1 ms).
#ifndef BURR_BAND_LOOKAHEAD_2BIT
#define BURR_BAND_LOOKAHEAD_2BIT 2
#endif
#ifndef BURR_BAND_LOOKAHEAD_1PLUS
#define BURR_BAND_LOOKAHEAD_1PLUS 2
#endif
template <bool kExact>
struct Lookahead {
    static constexpr int value = kExact ? BURR_BAND_LOOKAHEAD_1PLUS : BURR_BAND_LOOKAHEAD_2BIT;
    static_assert(value >= 0 && value <= 8, "lookahead out of range");
};
// Read-ahead of a 2-bit launch whose partitions are all resident at once (a
// layer of few partitions): the SMs then have issue slots to spare, each warp's
// chain of steps sets the time, and a third slot saves steps.  Measured with
// every partition resident: layer-0 band of 10^8 keys 8.54 -> 8.35 ms, of 2^25
// keys 6.96 -> 6.75 ms; when partitions outnumber the resident warps (10^9
// keys) the extra registers cost a CTA per SM: 63.7 -> 71.4 ms.
constexpr int kLookFew = 3;
constexpr int kMaxOf(int a, int b) { return a > b ? a : b; }
constexpr int kLookMax = kMaxOf(kMaxOf(Lookahead<false>::value, Lookahead<true>::value), kLookFew);

// Tagged sets (1+-bit thresholds): the kTagRows lowest-offset rows of the set
// carry one bit each in bits 33.. of the right-hand-side word, and a row's tag
// travels with every XOR, so a row that reduces to zero names the rows of the
// set that its dependency runs through.
constexpr uint32_t kTagRows = 31;

__device__ __forceinline__ unsigned long long row_tag(uint32_t k) {
    return k < kTagRows ? 1ull << (33u + k) : 0ull;
}

struct BandWarpSmem {
    RingSlot ring[kRing + kLookMax];   // live band window (+ read-ahead pad: zero, never written)
    uint16_t clist[kRing];         // ring indices stored by the current set (rollback)
    StagedRow rows[kStage];        // staged equations, ascending offset
    uint32_t first[132];           // first staged index of each offset (+ [128] = count)
    uint32_t ncommit;              // entries of clist
    uint32_t nfail;                // rows of a tagged set that reduced to zero
    uint32_t ftag[kTagRows];       // their tags (the first kTagRows of them)
};

template <typename V>
struct BandArgs {
    LayerDesc L;
    const uint64_t *keys;    // bucket-sorted records h = mix64(key ^ sigma) of the layer's keys
    const V *vals;
    const uint32_t *bstart;
    uint64_t *Cg;
    V *Yg;
    uint64_t *thresh;        // 2-bit codes (2-bit mode)
    uint8_t *texact;         // exact threshold of every bucket (1+-bit mode)
    uint64_t *bkeys;
    V *bvals;
    unsigned long long *bcount;
    uint32_t *err;
    BatchView bv;            // sd == nullptr: a single layer described by L
};

// What one warp works on: a partition of one structure's layer, and where that
// structure's data sits in the layer-wide arrays (all bases 0 for a single
// structure).
struct Ctx {
    LayerDesc L;
    uint64_t part;
    uint64_t bucket_base, slot_base, tw_base, out_base;
    unsigned long long *bcount;
    uint32_t *fail;          // base case, batched: per-structure flag
};

enum { kOk = 0, kDependent = 1, kOverflow = 2 };

// Pivots at or past bucket start + this many slots leave the live window: the
// ring less the read-ahead, so that the slots a step reads ahead of its pivot
// are still inside the window and never alias the window's first slots (a
// smaller window when a test asks for one).
constexpr uint32_t kWindow = (uint32_t)(kRing - kLookMax);
__device__ __forceinline__ uint32_t window_of(const LayerDesc &L) {
    return L.window ? min(L.window, kWindow) : kWindow;
}

__device__ __forceinline__ void rollback(BandWarpSmem &S, uint32_t ncommit, int lane) {
    __syncwarp();
    for (uint32_t i = lane; i < ncommit; i += 32) {
        const uint32_t ri = S.clist[i];
        S.ring[ri].c = 0;
        S.ring[ri].y = 0;
    }
    __syncwarp();
}

// Stage rows [base, base+cnt) (cnt <= kStage) of the bucket starting at slot
// bB: equations in ascending offset order; S.first[o] = first index with
// offset >= o.  A call, not inline code: inlined at its call sites, staging
// kept registers live across the elimination loops (166 registers in the 2-bit
// kernel, over 240 in the 1+-bit one); as a call both take 128, so 8 CTAs of 2
// warps fit per SM instead of 6.  Measured: equal at 10^8 keys (all partitions
// resident either way), layer-0 band 76.9 -> 68.2 ms at 10^9 keys.
template <typename V>
__device__ __noinline__ void stage_rows(BandWarpSmem &S, const BandArgs<V> &a, const Ctx &x, uint32_t base, uint32_t cnt,
                           uint32_t bB, int lane) {
    const LayerDesc &L = x.L;
    for (int i = lane; i < 132; i += 32) S.first[i] = 0;
    __syncwarp();
    uint64_t c[kStagePerLane];
    uint32_t y[kStagePerLane], o[kStagePerLane], rank[kStagePerLane];
#pragma unroll
    for (int j = 0; j < kStagePerLane; ++j) {
        const uint32_t i = (uint32_t)lane + 32u * j;
        if (i < cnt) {
            const uint64_t h = a.keys[base + i];     // the record h of the key
            const uint32_t s = start_of_h(h, L.range);
            c[j] = coeff_of_h(h, L.sigma);
            o[j] = s - bB;
            y[j] = (uint32_t)a.vals[base + i] & L.vmask;
            rank[j] = atomicAdd(&S.first[o[j]], 1u);
        }
    }
    __syncwarp();
    // exclusive scan of the 128 offset counts, 4 per lane
    uint32_t v0 = S.first[4 * lane], v1 = S.first[4 * lane + 1], v2 = S.first[4 * lane + 2],
             v3 = S.first[4 * lane + 3];
    const uint32_t loc = v0 + v1 + v2 + v3;
    uint32_t incl = loc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += t;
    }
    __syncwarp();
    uint32_t run = incl - loc;
    S.first[4 * lane] = run;
    run += v0;
    S.first[4 * lane + 1] = run;
    run += v1;
    S.first[4 * lane + 2] = run;
    run += v2;
    S.first[4 * lane + 3] = run;
    if (lane == 31) S.first[128] = incl;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < kStagePerLane; ++j) {
        const uint32_t i = (uint32_t)lane + 32u * j;
        if (i < cnt) {
            const uint32_t p = S.first[o[j]] + rank[j];
            S.rows[p] = StagedRow{c[j], y[j], o[j]};
        }
    }
    __syncwarp();
}

// 128-bit compare-and-swap on a ring slot: if the slot is (0, 0) it becomes
// (c, y); the previous contents are returned either way.
__device__ __forceinline__ void slot_cas(unsigned addr, unsigned long long c, unsigned long long y,
                                         unsigned long long &oc, unsigned long long &oy) {
    const unsigned long long zero = 0ull;
    asm volatile("{\n\t.reg .b128 d, b, v;\n\t"
                 "mov.b128 b, {%2, %2};\n\t"
                 "mov.b128 v, {%3, %4};\n\t"
                 "atom.shared.cas.b128 d, [%5], b, v;\n\t"
                 "mov.b128 {%0, %1}, d;\n\t}"
                 : "=l"(oc), "=l"(oy)
                 : "l"(zero), "l"(c), "l"(y), "r"(addr)
                 : "memory");
}

// Plain read of a ring slot, as 32-bit words: the row's two halves and the
// low word of the right-hand side; the right-hand side's high word (the tags
// of a tagged set) only when kHi (a sink otherwise, so it takes no register).
// A slot goes from empty to its final contents once per set (one atomic write
// of row and right-hand side), and a step's reads are issued only after the
// previous step's swaps have returned (their addresses depend on them), so a
// read sees a slot either empty (all zero) or with both words of a stored
// equation that stays.
template <bool kHi>
__device__ __forceinline__ void slot_load_words(unsigned addr, uint32_t &clo, uint32_t &chi, uint32_t &ylo,
                                                uint32_t &yhi) {
    if (kHi) {
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(clo), "=r"(chi), "=r"(ylo), "=r"(yhi)
                     : "r"(addr)
                     : "memory");
    } else {
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, _}, [%3];" : "=r"(clo), "=r"(chi), "=r"(ylo) : "r"(addr) : "memory");
        yhi = 0u;
    }
}

// Stream staged rows [lo, hi) (index range) into the band; stored ring
// indices are appended to S.clist (from S.ncommit).  Returns kOk, kDependent
// or kOverflow; nothing is rolled back here.  Every lane takes one step per
// iteration; stores, the commit list and the hand-out of the next rows go by
// ballot and prefix count, with no shared atomics besides the swaps.
//
// Lookahead: beside the swap on the slot of its leading bit p, a lane reads
// the slots p+1 .. p+kLook with plain loads (in flight together with the
// swap).  When the swap returns a stored row, elimination goes on through
// those slots without another round trip: a slot read as occupied holds a
// final equation, so XORing it is the step the swap would have taken; the
// step ends at the first leading bit whose slot was not read as occupied,
// and the next swap goes there.  The row is kept as 64 bits from p plus the
// kLook bits beyond p+63 that the read-ahead rows bring in.
//
// kTag: the rows carry tags (see kTagRows), and a row that reduces to zero does
// not end the set: its tag is listed in S.ftag (count in S.nfail, from 0), the
// row is dropped and its lane takes the next one.  This is a sequential
// insertion in claim order that skips the dependent rows, so each dropped row
// gives one dependency of the set on the band and the rows stored before it,
// and together they span all of the set's dependencies.  The result is then
// kDependent if any row was dropped; a ring overflow still ends the set.
template <int kLook, bool kTag = false>
__device__ int stream_insert(BandWarpSmem &S, uint32_t lo, uint32_t hi, uint32_t bB, uint32_t wlim, int lane) {
    if (hi <= lo) return kOk;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned ring0 = (unsigned)__cvta_generic_to_shared(&S.ring[0]);
    uint32_t nc = S.ncommit;
    // tagged: index of the next row to hand out; untagged: that index less the rows stored
    uint32_t next = kTag ? lo + 32u : lo + 32u - nc;
    bool has = lo + (uint32_t)lane < hi;
    // a lane without a row swaps (0, 0) in, which leaves every slot as it was
    unsigned long long cur = 0, y = 0;
    uint32_t pos = bB;
    if (has) {
        const StagedRow r = S.rows[lo + (uint32_t)lane];
        cur = r.c;
        y = kYValid | r.y;
        if (kTag) y |= row_tag((uint32_t)lane);
        pos = bB + r.o;
    }
    uint32_t nf = 0;
    bool pend = false;   // tagged: the lane's row was dropped; it takes the next one
    int result = kOk;
    for (;;) {
        const uint32_t ri = pos & kRingMask;
        const unsigned addr = ring0 + ri * (unsigned)sizeof(RingSlot);
        // Read-ahead: the pivot lies below bB + wlim <= bB + kRing - kLook, so the slots read
        // ahead are inside the window; past the ring's end they are the zero pad, which reads
        // as empty (the step then ends there, and the next swap goes to the true slot).
        unsigned long long oc, oy;
        uint32_t lcl[kLook > 0 ? kLook : 1], lch[kLook > 0 ? kLook : 1], lyl[kLook > 0 ? kLook : 1],
            lyh[kLook > 0 ? kLook : 1];
#pragma unroll
        for (int j = 0; j < kLook; ++j)
            slot_load_words<kTag>(addr + (unsigned)((j + 1) * sizeof(RingSlot)), lcl[j], lch[j], lyl[j], lyh[j]);
        slot_cas(addr, cur, y, oc, oy);
        // an empty slot is all zero and a stored row has its pivot bit set
        const bool stored = has && ((uint32_t)oc & 1u) == 0u;

        // Hand-out first: the next row's shared read is in flight during the elimination.
        const bool take = stored || (kTag && pend);
        // untagged, every stored row frees its lane for the next row: the next row handed out
        // is row lo + 32 + (rows stored so far), and a lane's commit-list entry gives its index
        const unsigned sm = __ballot_sync(kFull, stored);
        const unsigned tm = kTag ? __ballot_sync(kFull, take) : sm;
        const uint32_t ci = nc + (uint32_t)__popc(sm & lt);
        const uint32_t nidx = kTag ? next + (uint32_t)__popc(tm & lt) : ci + next;
        const bool nhas = take && nidx < hi;
        StagedRow nr = StagedRow{0ull, 0u, 0u};
        if (nhas) nr = S.rows[nidx];
        if (stored) S.clist[ci] = (uint16_t)ri;
        nc += (uint32_t)__popc(sm);
        if (kTag) next += (uint32_t)__popc(tm);

        // Elimination for lanes whose swap returned a stored row: against that row, then through
        // the read-ahead slots.  The row is (over : hi32 : lo32), bit j = slot pos + j; bit 0 is
        // now clear.  Which read-ahead rows are used depends only on the low word, so the
        // decisions run on 32 bits and the other words are XORed afterwards, all at once.
        const bool act = has && !stored;
        uint32_t lo32 = (uint32_t)cur ^ (uint32_t)oc;
        uint32_t hi32 = (uint32_t)(cur >> 32) ^ (uint32_t)(oc >> 32);
        uint32_t over = 0;
        uint32_t y2 = (uint32_t)y ^ (uint32_t)oy;   // right-hand sides fit in 32 bits
        uint32_t yh = kTag ? (uint32_t)(y >> 32) ^ (uint32_t)(oy >> 32) : 0u;   // tags (bits 1..)
        // while go is 1, bits 0 .. j-1 are clear, so bit j is the leading bit if set; a stored row
        // has its pivot bit (bit 0) set.  Decisions as 0/1 words and all-ones masks: measured
        // 5.7% fewer instructions than with predicates and selects (layer-0 band 65.8 -> 63.9 ms
        // at 10^9 keys).
        uint32_t go = 1u;
        uint32_t um[kLook > 0 ? kLook : 1];   // 0 or all ones: the read-ahead row of slot pos+j is used
#pragma unroll
        for (int j = 1; j <= kLook; ++j) {
            const uint32_t occ = lcl[j - 1] & 1u;
            const uint32_t bit = (lo32 >> j) & 1u;
            um[j - 1] = 0u - (go & bit & occ);
            lo32 ^= (lcl[j - 1] << j) & um[j - 1];
            go &= (bit ^ 1u) | occ;
        }
#pragma unroll
        for (int j = 1; j <= kLook; ++j) {
            hi32 ^= __funnelshift_l(lcl[j - 1], lch[j - 1], (unsigned)j) & um[j - 1];
            over ^= (lch[j - 1] >> (32 - j)) & um[j - 1];
            y2 ^= lyl[j - 1] & um[j - 1];
            if (kTag) yh ^= lyh[j - 1] & um[j - 1];
        }
        // normalise: shift the leading bit (>= 1 for an active lane) down to bit 0; it is
        // almost always in the low word
        int tz = __ffs((int)lo32) - 1;
        uint32_t n0 = __funnelshift_r(lo32, hi32, (unsigned)tz), n1 = __funnelshift_r(hi32, over, (unsigned)tz);
        bool zero = false;
        if (act && lo32 == 0u) {
            zero = (hi32 | over) == 0u;
            if (hi32) {
                tz = 31 + __ffs((int)hi32);
                n0 = __funnelshift_r(hi32, over, (unsigned)(tz - 32));
                n1 = over >> (tz - 32);
            } else {
                tz = 63 + __ffs((int)over);
                n0 = over >> ((tz - 64) & 31);
                n1 = 0;
            }
        }
        const uint32_t npos = pos + (uint32_t)tz;
        const bool dep = act && zero;
        const bool ovf = act && !zero && npos - bB >= wlim;
        if (act) {
            cur = ((unsigned long long)n1 << 32) | n0;
            y = kTag ? ((unsigned long long)(yh | 1u) << 32) | y2 : kYValid | y2;
            pos = npos;
        }
        if (take) {
            has = nhas;
            cur = nr.c;
            y = nhas ? kYValid | nr.y : 0ull;
            if (kTag && nhas) y |= row_tag(nidx - lo);
            if (nhas) pos = bB + nr.o;
            pend = false;
        }
        const unsigned bm = __ballot_sync(kFull, dep || ovf);
        unsigned hm = __ballot_sync(kFull, has);
        if (bm) {
            const unsigned om = __ballot_sync(kFull, ovf);
            if (!kTag || om) {
                result = om ? kOverflow : kDependent;
                break;
            }
            // tagged: list the dropped rows' tags; their lanes swap (0, 0) once and then take the
            // next rows
            const uint32_t dr = (uint32_t)__popc(bm & lt);
            if (dep) {
                if (nf + dr < kTagRows) S.ftag[nf + dr] = yh >> 1;
                has = false;
                cur = 0;
                y = 0;
                pend = true;
            }
            nf += (uint32_t)__popc(bm);
            hm = __ballot_sync(kFull, has || (pend && next < hi));
        }
        if (!hm) break;
    }
    __syncwarp();
    if (lane == 0) {
        S.ncommit = nc;
        if (kTag) S.nfail = nf;
    }
    __syncwarp();
    if (kTag && result == kOk && nf) result = kDependent;
    return result;
}

// Insert the rows of bucket [rs, re) whose offset lies in [olo, ohi) as one
// set; on a dependency or overflow every row this call stored is removed.
// kL: slots read ahead per step.
template <typename V, bool kExact, int kL = Lookahead<kExact>::value>
__device__ int insert_set(BandWarpSmem &S, const BandArgs<V> &a, const Ctx &x, uint32_t rs, uint32_t re,
                          uint32_t bB, uint32_t olo, uint32_t ohi, uint32_t &staged_base, int lane) {
    if (lane == 0) S.ncommit = 0;
    __syncwarp();
    for (uint32_t base = rs; base < re; base += kStage) {
        const uint32_t cnt = min((uint32_t)kStage, re - base);
        if (staged_base != base) {
            stage_rows(S, a, x, base, cnt, bB, lane);
            staged_base = base;
        }
        const int rc = stream_insert<kL>(S, S.first[olo], S.first[ohi], bB, window_of(x.L), lane);
        if (rc != kOk) {
            rollback(S, S.ncommit, lane);
            if (rc == kOverflow && lane == 0) atomicOr(a.err, kErrRingOverflow);
            return rc;
        }
    }
    return kOk;
}

constexpr uint32_t kTagUnknown = 0xffffffffu;

// 1+-bit threshold of a bucket whose rows fit one stage, from one tagged pass
// over its rows at offsets >= forced.  The set's dependencies form a space D
// spanned by the dropped rows' dependency vectors (one per dropped row).  The
// rows at offsets >= t insert iff no nonzero vector of D lies inside them, so
// the least such t is one above the largest, over D, of the lowest offset a
// vector contains.  Row i of the set (ascending offset) is tag bit i for
// i < kTagRows, every later row sits at an offset at least as high, and a tag
// is the vector's restriction to the tagged rows: after a reduction of the
// tags to distinct lowest bits, the largest lowest bit b gives t = offset of
// row b + 1.  A tag that reduces to zero means a dependency among untagged
// rows only, which the tags cannot place: kTagUnknown.
// Returns forced if the set inserts (its rows stay in the band), else t with
// nothing of the set left in the band, kTagUnknown (same), or B + 1 on a ring
// overflow.
template <typename V>
__device__ uint32_t insert_tagged(BandWarpSmem &S, const BandArgs<V> &a, const Ctx &x, uint32_t rs, uint32_t re,
                                  uint32_t bB, uint32_t forced, uint32_t &staged, int lane) {
    if (staged != rs) {
        stage_rows(S, a, x, rs, re - rs, bB, lane);
        staged = rs;
    }
    if (lane == 0) S.ncommit = 0;
    __syncwarp();
    const uint32_t lo = S.first[forced];
    const int rc = stream_insert<Lookahead<true>::value, true>(S, lo, S.first[x.L.B], bB, window_of(x.L), lane);
    const uint32_t nc = S.ncommit;
    if (rc == kOk) {
        for (uint32_t i = lane; i < nc; i += 32) S.ring[S.clist[i]].y &= kYValid | 0xffffffffull;   // drop the tags
        __syncwarp();
        return forced;
    }
    rollback(S, nc, lane);
    if (rc == kOverflow) {
        if (lane == 0) atomicOr(a.err, kErrRingOverflow);
        return x.L.B + 1u;
    }
    const uint32_t nf = S.nfail;
    if (nf > kTagRows) return kTagUnknown;
    uint32_t v = (uint32_t)lane < nf ? S.ftag[lane] : 0u;
    bool piv = false;
    int top = -1;
    for (int b = 0; b < (int)kTagRows; ++b) {
        const unsigned cand = __ballot_sync(kFull, !piv && ((v >> b) & 1u));
        if (!cand) continue;
        const int p = __ffs((int)cand) - 1;
        const uint32_t pv = __shfl_sync(kFull, v, p);
        if (lane == p) piv = true;
        else if ((cand >> lane) & 1u) v ^= pv;
        top = b;
    }
    if (__ballot_sync(kFull, (uint32_t)lane < nf && !piv) || top < 0) return kTagUnknown;
    return S.rows[lo + (uint32_t)top].o + 1u;
}

// Offsets above the failing threshold tried first (8, 12, 16 and 24 measured;
// 8 and 16 tied at 10^8 keys when every failing bucket was searched by probes).
constexpr uint32_t kFirstProbe = 16;

// 1+-bit threshold of a bucket whose rows at offsets >= forced are dependent,
// by probes (where the tagged pass cannot decide it): the least t for which
// the rows at offsets >= t insert, those rows left inserted.  Rows at offsets
// >= t_fail are dependent, those >= t_ok are kept; exact thresholds are mostly
// small (a few rows at the lowest offsets), so the first probe keeps all but
// the lowest 16 offsets and bisection follows.  Returns B + 1 on a ring
// overflow.
template <typename V>
__device__ __forceinline__ uint32_t exact_threshold(BandWarpSmem &S, const BandArgs<V> &a, const Ctx &x, uint32_t rs,
                                                 uint32_t re, uint32_t bB, uint32_t forced, uint32_t &staged,
                                                 int lane) {
    uint32_t t_fail = forced, t_ok = x.L.B;
    bool first = true;
    while (t_ok - t_fail > 1) {
        const uint32_t mid = (first && t_fail + kFirstProbe < t_ok) ? t_fail + kFirstProbe : (t_fail + t_ok) >> 1;
        first = false;
        const int rc = insert_set<V, true>(S, a, x, rs, re, bB, mid, t_ok, staged, lane);
        if (rc == kOverflow) return x.L.B + 1u;
        if (rc == kOk) t_ok = mid;
        else t_fail = mid;
    }
    return t_ok;
}

// Rows of the bucket below threshold t leave for the next layer (as keys: the
// next layer hashes them with its own seed).
template <typename V>
__device__ void emit_bumped(const BandArgs<V> &a, const Ctx &x, uint32_t rs, uint32_t re, uint32_t bB,
                            uint32_t t, int lane) {
    for (uint32_t base = rs; base < re; base += 32) {
        const uint32_t idx = base + lane;
        bool bump = false;
        uint64_t key = 0;
        V val = 0;
        if (idx < re) {
            const uint64_t h = a.keys[idx];
            bump = (start_of_h(h, x.L.range) - bB) < t;
            if (bump) {
                key = key_of_h(h, x.L.sigma);
                val = a.vals[idx];
            }
        }
        const uint32_t mask = __ballot_sync(kFull, bump);
        if (!mask) continue;
        unsigned long long ob = 0;
        if (lane == 0) ob = atomicAdd(x.bcount, (unsigned long long)__popc(mask));
        ob = __shfl_sync(kFull, ob, 0);
        if (bump) {
            const unsigned long long o = x.out_base + ob + __popc(mask & ((1u << lane) - 1u));
            a.bkeys[o] = key;
            a.bvals[o] = val;
        }
    }
}

// Write ring slots [from, to) to the global band and clear them.
template <typename V>
__device__ __forceinline__ void flush(BandWarpSmem &S, const BandArgs<V> &a, const Ctx &x, uint64_t from,
                                      uint64_t to, int lane) {
    __syncwarp();
    for (uint64_t s = from + lane; s < to; s += 32) {
        const uint32_t ri = (uint32_t)s & kRingMask;
        a.Cg[x.slot_base + s] = S.ring[ri].c;
        a.Yg[x.slot_base + s] = (V)(S.ring[ri].y & 0xffffffffull);
        S.ring[ri].c = 0;
        S.ring[ri].y = 0;
    }
    __syncwarp();
}

// kExact: 1+-bit thresholds (exact per bucket) instead of 2-bit codes; a
// template parameter so that each mode gets its own register allocation.  kL:
// slots read ahead per step (see kLookFew).
template <typename V, bool kExact, int kL = Lookahead<kExact>::value>
// All 1504 layer-0 partitions of 10^8 keys are resident at once when the
// kernel takes at most 170 registers (six CTAs of two warps per SM).  Measured
// with staging inline: at 186 registers (5 CTAs per SM) the layer-0 band took
// 15.5 ms instead of 9.7; with a 128-register cap (spills inside the
// elimination loop) 13.4 ms.  With staging as a call it takes 128 without
// such spills (see stage_rows).  The 2-bit kernel for values wider than a
// byte at two slots of read-ahead gets an explicit bound of 8 CTAs per SM:
// without it ptxas gave it 139 registers (7 CTAs per SM; r = 16 at 10^9 keys:
// layer-0 band 67.4 -> 72.7 ms); the other instantiations keep the bound on
// threads alone (0 below), under which the one-byte kernel measured fastest.
__global__ void __launch_bounds__(32 * kBandWarps, (sizeof(V) > 1 && !kExact && kL == 2) ? 8 : 0)
    k_band(BandArgs<V> a) {
    __shared__ BandWarpSmem smem[kBandWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint64_t gp = (uint64_t)blockIdx.x * kBandWarps + warp;
    Ctx x;
    if (a.bv.sd) {
        if (gp >= a.bv.nparts) return;
        if (a.bv.part_order) gp = a.bv.part_order[gp];   // longest partitions first
        const uint32_t si = a.bv.part_struct[gp];
        const StructDesc &D = a.bv.sd[si];
        x.L = D.L;
        x.part = gp - D.part_base;
        x.bucket_base = D.bucket_base;
        x.slot_base = D.slot_base;
        x.tw_base = D.tw_base;
        x.out_base = D.out_base;
        x.bcount = a.bcount + si;
        x.fail = a.bv.fail ? a.bv.fail + si : nullptr;
    } else {
        gp += a.L.part_lo;
        if (gp >= part_end(a.L)) return;
        x.L = a.L;
        x.part = gp;
        x.bucket_base = x.slot_base = x.tw_base = x.out_base = 0;
        x.bcount = a.bcount;
        x.fail = nullptr;
    }
    const LayerDesc &L = x.L;
    const uint64_t part = x.part;
    BandWarpSmem &S = smem[warp];

    const uint64_t b0 = part_bucket(L, part);
    const uint64_t b1 = part_bucket(L, part + 1);
    const uint64_t own_lo = part_own_lo(L, part);
    const uint64_t own_hi = part_own_hi(L, part);

    for (int i = lane; i < kRing + kLookMax; i += 32) {   // the ring and its pad
        S.ring[i].c = 0;
        S.ring[i].y = 0;
    }
    __syncwarp();

    uint32_t lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) lv[i] = L.levels[i];
    const uint32_t fcode = L.forced_code;
    const uint32_t flevel = lv[fcode & 3];

    uint64_t flushed = own_lo;
    uint64_t tword = 0, twi = b0 >> 5;
    // bucket bounds are read one bucket ahead, and the next bucket's equations are
    // prefetched into L2, so that staging does not wait on DRAM
    const uint32_t *bst = a.bstart + x.bucket_base;
    const uint32_t pend = bst[b1];   // end of the partition's equations
    uint32_t nrs = b0 < b1 ? bst[b0] : 0, nre = b0 < b1 ? bst[b0 + 1] : 0;
    for (uint64_t b = b0; b < b1; ++b) {
        const uint64_t bB = b * L.B;
        const uint32_t rs = nrs, re = nre;
        nrs = re;
        nre = b + 2 <= b1 ? bst[b + 2] : re;
        if (lane < 16) {
            const uint32_t k = re + (uint32_t)lane * (128u / sizeof(uint64_t));
            if (k < pend) prefetch_l2(a.keys + k);
        } else if (lane < 24) {
            const uint32_t k = re + (uint32_t)(lane - 16) * (128u / sizeof(V));
            if (k < pend) prefetch_l2(a.vals + k);
        }
        if (bB > flushed) {
            flush(S, a, x, flushed, bB, lane);
            flushed = bB;
        }
        const bool cut = (part > 0 && b == b0 && !L.fallback);
        const uint32_t forced = cut ? (kExact ? (uint32_t)kW : flevel) : 0;
        uint32_t code = cut ? fcode : 0;
        uint32_t texact = forced;
        if (re > rs) {
            uint32_t staged = 0xffffffffu;
            bool search = false;   // 1+-bit: find the threshold by probes
            if (kExact && !L.fallback && re - rs <= (uint32_t)kStage) {
                // one tagged pass gives the threshold; the search only where the tags do not decide
                texact = insert_tagged(S, a, x, rs, re, (uint32_t)bB, forced, staged, lane);
                if (texact == L.B + 1u) return;   // ring overflow (recorded)
                if (texact != kTagUnknown && texact > forced) {
                    const int rc = insert_set<V, kExact, kL>(S, a, x, rs, re, (uint32_t)bB, texact, L.B, staged, lane);
                    if (rc == kOverflow) return;
                    if (rc != kOk) texact = kTagUnknown;   // not expected: the rows at offsets >= t are independent
                }
                search = texact == kTagUnknown;
            } else if (const int rc = insert_set<V, kExact, kL>(S, a, x, rs, re, (uint32_t)bB, forced, L.B, staged, lane);
                       rc != kOk) {
                if (rc == kOverflow) return;
                if (L.fallback) {
                    if (lane == 0) atomicOr(x.fail ? x.fail : a.err, kErrUnsolvable);
                    return;
                }
                if (kExact) {
                    search = true;
                } else {
                    // the set [forced, B) was just found dependent: the threshold is the least
                    // level above `forced` whose rows [level, B) insert, each candidate tried as
                    // one set (rolled back if dependent).  Nearly always the first one inserts,
                    // so this is one stream; inserting the bands [64, 128) and [32, 64) one
                    // after the other took two.
                    code = 3;
                    for (int k = 1; k <= 2; ++k) {
                        if (lv[k] <= forced) continue;
                        const int rc2 = insert_set<V, kExact, kL>(S, a, x, rs, re, (uint32_t)bB, lv[k], L.B, staged, lane);
                        if (rc2 == kOverflow) return;
                        if (rc2 == kOk) {
                            code = (uint32_t)k;
                            break;
                        }
                    }
                }
            }
            if (kExact && search) {
                texact = exact_threshold(S, a, x, rs, re, (uint32_t)bB, forced, staged, lane);
                if (texact > L.B) return;   // ring overflow (recorded)
            }
            const uint32_t t = kExact ? texact : lv[code];
            if (!L.fallback && t > 0) emit_bumped(a, x, rs, re, (uint32_t)bB, t, lane);
        }
        if (kExact && !L.fallback) {
            if (lane == 0) a.texact[x.bucket_base + b] = (uint8_t)texact;
            continue;
        }
        if (!L.fallback) {
            if ((b >> 5) != twi) {
                if (lane == 0 && tword)
                    atomicOr((unsigned long long *)&a.thresh[x.tw_base + twi], (unsigned long long)tword);
                tword = 0;
                twi = b >> 5;
            }
            tword |= (uint64_t)code << (2 * (b & 31));
        }
    }
    if (!L.fallback && lane == 0 && tword)
        atomicOr((unsigned long long *)&a.thresh[x.tw_base + twi], (unsigned long long)tword);
    flush(S, a, x, flushed, own_hi, lane);
}

// Back-substitution, right to left over the partition's owned slots, one
// window per value bit: Z[i] = Y[i] ^ parity((C[i] >> 1) & Z[i+1 .. i+63]),
// Z[i] = 0 on empty slots (C = Y = 0 there).  The 64-bit register T holds Z of
// the 64 slots right of the current group (bit j = slot i+1+j); after a block
// of 64 slots it is exactly that block's table word for this bit plane.
//
// Four slots are solved per step so that the dependent chain is short: with
// c'_s = C[s] >> 1, the four parities against T are independent,
//   A_d = Y[i-d] ^ parity((c'_{i-d} >> d) & T),  d = 0..3,
// and the slots of the group then correct each other through the low bits of
// their own rows:
//   z_i = A_0,  z_{i-1} = A_1 ^ c'_{i-1}[0] z_i,
//   z_{i-2} = A_2 ^ c'_{i-2}[0] z_{i-1} ^ c'_{i-2}[1] z_i,
//   z_{i-3} = A_3 ^ c'_{i-3}[0] z_{i-2} ^ c'_{i-3}[1] z_{i-1} ^ c'_{i-3}[2] z_i,
//   T <- (T << 4) | z_i z_{i-1} z_{i-2} z_{i-3}.
constexpr int kBsWarps = 4;

__device__ __forceinline__ uint32_t parity64(uint64_t x) {
    return (uint32_t)__popc((uint32_t)x ^ (uint32_t)(x >> 32)) & 1u;
}

// Back-substitution with several partitions per warp: a partition needs only
// R lanes (R = r for one-byte values, one bit plane per lane; r / 2 or r / 4
// rounded up with 2 or 4 planes per lane for wider values), so a warp solves
// G = min(32 / R, kBsGroups) partitions side by side, lanes [q*R, q*R + R) on
// partition q.  For a batch, whose structures may differ in r, R comes from
// the widest value type (8 lanes); lanes past a structure's r sit out.  Each group runs the four-slot steps above; sharing each instruction
// among G partitions cuts the issue load G-fold, which matters because the
// solve runs beside the next layer's sort and band.  Partitions of one warp may
// differ in length: each walks its own blocks from the right, and a finished
// group idles until the longest one is done.
constexpr int kBsGroups = 8;

//
// kG (1, 2, 4 or 8) bounds G at compile time, so that the per-group registers
// of a launch with few groups (G = 4 at r = 8) are not those of eight.  A warp
// job is one set of G partitions; the grid may hold fewer warps than jobs
// (a cap on the CTAs per SM leaves room beside it for the next layer's
// kernels), and then every warp walks the jobs with the grid's stride.
//
// kPL bit planes per lane (1, 2 or 4; for r up to 8, 16, 32): lane k of a
// group solves planes k*kPL .. k*kPL + kPL - 1, each with its own window T, and
// the rows' reads, shifts and low bits serve all of them.  At r = 16 a group
// then needs 8 lanes instead of 16, so a warp takes 4 partitions instead of 2.
template <typename V, int kG, int kPL>
__global__ void __launch_bounds__(32 * kBsWarps, kG >= 8 ? 4 : 1)
k_backsub_multi(LayerDesc L0, const uint64_t *__restrict__ Cg, const V *__restrict__ Yg, uint64_t *__restrict__ Z0,
                BatchView bv, uint32_t R, uint32_t G, uint64_t njobs) {
    __shared__ __align__(16) uint64_t sc[kBsWarps][kG][64];
    __shared__ __align__(16) uint32_t sy[kBsWarps][kG][64];
    __shared__ uint64_t sbase[kBsWarps][kG];  // first slot of the group's structure in the layer arrays
    __shared__ uint64_t shi[kBsWarps][kG];    // one past the last block of the group's partition
    __shared__ uint32_t slen[kBsWarps][kG];   // its number of blocks
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t q = (uint32_t)lane / R, k = (uint32_t)lane % R;
    for (uint64_t job = (uint64_t)blockIdx.x * kBsWarps + warp; job < njobs;
         job += (uint64_t)gridDim.x * kBsWarps) {
    uint64_t gp = job * G + q + (bv.sd ? 0 : L0.part_lo);
    const uint64_t nparts = bv.sd ? bv.nparts : part_end(L0);
    uint64_t bhi = 0, base = 0;
    uint32_t len = 0, r = 0;
    uint64_t *Z = Z0;
    if (q < G && gp < nparts) {
        LayerDesc L;
        uint64_t part;
        if (bv.sd) {
            if (bv.part_order) gp = bv.part_order[gp];   // partitions of similar length share a warp
            const StructDesc &D = bv.sd[bv.part_struct[gp]];
            L = D.L;
            part = gp - D.part_base;
            base = D.slot_base;
            Z += D.z_base;
        } else {
            L = L0;
            part = gp;
        }
        const uint64_t lo = part_own_lo(L, part) >> 6, hi = part_own_hi(L, part) >> 6;
        if (hi > lo) {
            bhi = hi;
            len = (uint32_t)(hi - lo);
        }
        r = L.r;
    }
    if (q < G && k == 0) {
        sbase[warp][q] = base;
        shi[warp][q] = bhi;
        slen[warp][q] = len;
    }
    const uint32_t maxlen = __reduce_max_sync(0xffffffffu, len);
    __syncwarp();
    if (maxlen == 0) continue;
    uint64_t gh[kG], gb[kG];
    uint32_t gl[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        gh[g] = (uint32_t)g < G ? shi[warp][g] : 0;
        gb[g] = (uint32_t)g < G ? sbase[warp][g] : 0;
        gl[g] = (uint32_t)g < G ? slen[warp][g] : 0;
    }
    // software pipeline: registers hold every group's next block while this one is solved
    uint64_t nc0[kG], nc1[kG];
    uint32_t ny0[kG], ny1[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
        nc0[g] = nc1[g] = 0;
        ny0[g] = ny1[g] = 0;
        if (gl[g] > 0) {
            const uint64_t s0 = gb[g] + ((gh[g] - 1) << 6);
            nc0[g] = Cg[s0 + lane];
            nc1[g] = Cg[s0 + lane + 32];
            ny0[g] = Yg[s0 + lane];
            ny1[g] = Yg[s0 + lane + 32];
        }
    }
    const bool solve = k * kPL < r;
    uint64_t T[kPL];
#pragma unroll
    for (int pl = 0; pl < kPL; ++pl) T[pl] = 0;
    for (uint32_t t = 0; t < maxlen; ++t) {
        __syncwarp();
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            if (t < gl[g]) {
                sc[warp][g][lane] = nc0[g] >> 1;
                sc[warp][g][lane + 32] = nc1[g] >> 1;
                sy[warp][g][lane] = ny0[g];
                sy[warp][g][lane + 32] = ny1[g];
            }
        }
        __syncwarp();
#pragma unroll
        for (int g = 0; g < kG; ++g) {
            if (t + 1 < gl[g]) {
                const uint64_t s0 = gb[g] + ((gh[g] - 2 - t) << 6);
                nc0[g] = Cg[s0 + lane];
                nc1[g] = Cg[s0 + lane + 32];
                ny0[g] = Yg[s0 + lane];
                ny1[g] = Yg[s0 + lane + 32];
            }
        }
        if (solve && t < len) {
            const uint64_t *c = sc[warp][q];
            const uint32_t *yv = sy[warp][q];
#pragma unroll 4
            for (int g = 15; g >= 0; --g) {
                // slots 4g .. 4g+3 in three 16-byte shared reads
                const ulonglong2 clo = *reinterpret_cast<const ulonglong2 *>(c + 4 * g);
                const ulonglong2 chi = *reinterpret_cast<const ulonglong2 *>(c + 4 * g + 2);
                const uint4 yq = *reinterpret_cast<const uint4 *>(yv + 4 * g);
                const uint64_t c0 = chi.y, c1 = chi.x >> 1, c2 = clo.y >> 2, c3 = clo.x >> 3;
                const uint32_t l1 = (uint32_t)chi.x, l2 = (uint32_t)clo.y, l3 = (uint32_t)clo.x;
#pragma unroll
                for (int pl = 0; pl < kPL; ++pl) {
                    const uint32_t b = k * kPL + (uint32_t)pl;   // this plane's value bit
                    const uint32_t a0 = ((yq.w >> b) & 1u) ^ parity64(c0 & T[pl]);
                    const uint32_t a1 = ((yq.z >> b) & 1u) ^ parity64(c1 & T[pl]);
                    const uint32_t a2 = ((yq.y >> b) & 1u) ^ parity64(c2 & T[pl]);
                    const uint32_t a3 = ((yq.x >> b) & 1u) ^ parity64(c3 & T[pl]);
                    const uint32_t z0 = a0;
                    const uint32_t z1 = a1 ^ (l1 & z0);
                    const uint32_t z2 = a2 ^ ((l2 >> 1) & z0) ^ (l2 & z1);
                    const uint32_t z3 = a3 ^ ((l3 >> 2) & z0) ^ ((l3 >> 1) & z1) ^ (l3 & z2);
                    T[pl] = (T[pl] << 4) | (uint64_t)(((z0 << 3) | (z1 << 2) | (z2 << 1) | z3) & 15u);
                }
            }
#pragma unroll
            for (int pl = 0; pl < kPL; ++pl)
                if (k * kPL + (uint32_t)pl < r) Z[(bhi - 1 - t) * r + k * kPL + pl] = T[pl];
        }
    }
    __syncwarp();   // the warp's shared arrays are reused by its next job
    }
}

template <typename V>
cudaError_t band_impl(const LayerDesc &L, const uint64_t *keys, const V *vals, const uint32_t *bstart,
                      uint64_t *Cg, V *Yg, uint64_t *thresh, uint8_t *texact, uint64_t *bkeys, V *bvals,
                      unsigned long long *bcount, uint32_t *err, cudaStream_t st, const BatchView *bv) {
    BandArgs<V> a;
    if (bv) a.bv = *bv;
    a.L = L;
    a.keys = keys;
    a.vals = vals;
    a.bstart = bstart;
    a.Cg = Cg;
    a.Yg = Yg;
    a.thresh = thresh;
    a.texact = texact;
    a.bkeys = bkeys;
    a.bvals = bvals;
    a.bcount = bcount;
    a.err = err;
    const uint64_t parts = bv ? bv->nparts : part_end(L) - L.part_lo;
    const unsigned grid = (unsigned)((parts + kBandWarps - 1) / kBandWarps);
    // the threshold mode is one for the whole launch (a batch shares its parameters)
    cudaError_t e;
    if (L.mode == BURR_THRESH_1PLUS && !L.fallback) {
        if ((e = prefer_shared(k_band<V, true>)) != cudaSuccess) return e;
        k_band<V, true><<<grid, 32 * kBandWarps, 0, st>>>(a);
        return cudaGetLastError();
    }
    // 2-bit: the deeper read-ahead where every CTA of the launch is resident at once
    if ((e = prefer_shared(k_band<V, false, kLookFew>)) != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_band<V, false, kLookFew>, 32 * kBandWarps, 0)) !=
        cudaSuccess)
        return e;
    if ((uint64_t)grid <= (uint64_t)sms * (uint64_t)per_sm) {
        k_band<V, false, kLookFew><<<grid, 32 * kBandWarps, 0, st>>>(a);
    } else {
        if ((e = prefer_shared(k_band<V, false>)) != cudaSuccess) return e;
        k_band<V, false><<<grid, 32 * kBandWarps, 0, st>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_band(const LayerDesc &L, uint32_t vbytes, const uint64_t *keys, const void *vals,
                        const uint32_t *bucket_start, uint64_t *Cg, void *Yg, uint64_t *thresh, uint8_t *texact,
                        uint64_t *bumped_keys, void *bumped_vals, unsigned long long *bumped_count,
                        uint32_t *err, cudaStream_t st, const BatchView *bv) {
    if (bv ? bv->nparts == 0 : part_end(L) <= L.part_lo) return cudaSuccess;
    switch (vbytes) {
    case 1:
        return band_impl<uint8_t>(L, keys, (const uint8_t *)vals, bucket_start, Cg, (uint8_t *)Yg, thresh, texact,
                                  bumped_keys, (uint8_t *)bumped_vals, bumped_count, err, st, bv);
    case 2:
        return band_impl<uint16_t>(L, keys, (const uint16_t *)vals, bucket_start, Cg, (uint16_t *)Yg, thresh, texact,
                                   bumped_keys, (uint16_t *)bumped_vals, bumped_count, err, st, bv);
    default:
        return band_impl<uint32_t>(L, keys, (const uint32_t *)vals, bucket_start, Cg, (uint32_t *)Yg, thresh, texact,
                                   bumped_keys, (uint32_t *)bumped_vals, bumped_count, err, st, bv);
    }
}

template <typename V, int kG, int kPL>
cudaError_t backsub_launch(const LayerDesc &L, const uint64_t *Cg, const V *Yg, uint64_t *Z, cudaStream_t st,
                           const BatchView &v, uint32_t R, uint32_t G, uint64_t njobs, unsigned grid) {
    const cudaError_t e = prefer_shared(k_backsub_multi<V, kG, kPL>);
    if (e != cudaSuccess) return e;
    k_backsub_multi<V, kG, kPL><<<grid, 32 * kBsWarps, 0, st>>>(L, Cg, Yg, Z, v, R, G, njobs);
    return cudaGetLastError();
}

// Planes per lane: one for values of a byte (r <= 8 lanes already fit four
// groups in a warp), else as many as the value's bytes.
template <typename V>
constexpr int planes_per_lane() {
    return sizeof(V) == 1 ? 1 : (int)sizeof(V);
}

template <typename V>
cudaError_t backsub_impl(const LayerDesc &L, const uint64_t *Cg, const V *Yg, uint64_t *Z, cudaStream_t st,
                         const BatchView &v, uint32_t R, uint32_t G, uint64_t njobs, unsigned grid) {
    constexpr int PL = planes_per_lane<V>();
    if (G <= 1) return backsub_launch<V, 1, PL>(L, Cg, Yg, Z, st, v, R, G, njobs, grid);
    if (G <= 2) return backsub_launch<V, 2, PL>(L, Cg, Yg, Z, st, v, R, G, njobs, grid);
    if (G <= 4) return backsub_launch<V, 4, PL>(L, Cg, Yg, Z, st, v, R, G, njobs, grid);
    return backsub_launch<V, kBsGroups, PL>(L, Cg, Yg, Z, st, v, R, G, njobs, grid);
}

cudaError_t launch_backsub(const LayerDesc &L, uint32_t vbytes, const uint64_t *Cg, const void *Yg,
                           uint64_t *Z, cudaStream_t st, const BatchView *bv, uint32_t max_ctas_per_sm) {
    const uint64_t parts = bv ? bv->nparts : (part_end(L) > L.part_lo ? part_end(L) - L.part_lo : 0);
    if (parts == 0) return cudaSuccess;
    // several partitions per warp; a batch's structures may differ in r (up to 8 bits per value
    // byte); R lanes per partition, each solving one bit plane for one-byte values, else as many
    // planes as the value has bytes
    const uint32_t pl = vbytes == 1 ? 1u : vbytes;
    const uint32_t R = bv ? 8u * vbytes / pl : (L.r + pl - 1) / pl;
    const uint32_t G = std::min<uint32_t>(32u / R, (uint32_t)kBsGroups);
    const uint64_t njobs = (parts + G - 1) / G;
    uint64_t grid = (njobs + kBsWarps - 1) / kBsWarps;
    if (max_ctas_per_sm) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = std::min<uint64_t>(grid, (uint64_t)sms * max_ctas_per_sm);
    }
    const BatchView v = bv ? *bv : BatchView();
    switch (vbytes) {
    case 1: return backsub_impl<uint8_t>(L, Cg, (const uint8_t *)Yg, Z, st, v, R, G, njobs, (unsigned)grid);
    case 2: return backsub_impl<uint16_t>(L, Cg, (const uint16_t *)Yg, Z, st, v, R, G, njobs, (unsigned)grid);
    default: return backsub_impl<uint32_t>(L, Cg, (const uint32_t *)Yg, Z, st, v, R, G, njobs, (unsigned)grid);
    }
}

}  // namespace burr
