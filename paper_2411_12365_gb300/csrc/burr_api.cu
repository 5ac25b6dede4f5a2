// burr_api.cu -- host side of libburr.so: parameter checks, the layer driver
// (Sec. 2 layers, Sec. 3 partitions and base case), handles, query dispatch,
// export and statistics.  Every step of the method runs in the kernels of
// burr_sort.cu, burr_band.cu and burr_query.cu; this file only sizes layers,
// allocates, launches and reads back one counter per layer.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <mutex>
#include <set>
#include <tuple>
#include <type_traits>
#include <vector>

#include "burr_internal.cuh"

using namespace burr;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(BURR_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(BURR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

uint32_t value_bytes(uint32_t r) { return r <= 8 ? 1u : (r <= 16 ? 2u : 4u); }
uint64_t align64(uint64_t x) { return (x + 63) & ~63ull; }

uint64_t layer_slots(uint64_t n, double alpha) {
    if (n == 0) return 0;
    return align64((uint64_t)std::ceil((double)n / alpha) + kW);
}

uint64_t fallback_slots(uint64_t n, double slack, uint32_t attempt) {
    if (n == 0) return 0;
    uint64_t m = align64((uint64_t)std::ceil((double)n * (1.0 + slack)) + kW);
    for (uint32_t a = 0; a < attempt; ++a) m = align64((uint64_t)std::ceil((double)m * 1.1));
    return m;
}

uint64_t num_buckets(uint64_t m, uint32_t B) { return m == 0 ? 0 : (m - kW + B) / B; }


// Partition size of bumping layer l: layer 0 is cut every partition_slots,
// deeper layers every lower_partition_slots (0: partition_slots).
uint64_t layer_partition_slots(const burr_params &p, uint32_t l) {
    return (l > 0 && p.lower_partition_slots) ? p.lower_partition_slots : p.partition_slots;
}

// Partitions of a layer of m slots (Sec. 3, minimum buckets per thread): one
// below minP slots or below P; else floor(m/P) partitions of P slots, plus one
// for the remainder m mod P when it is at least max(min(minP, P/2), 1024)
// slots (a smaller remainder joins the last partition).  No partition is then
// much longer than P; the longest partition sets the band kernel's time.
uint64_t num_partitions(uint64_t m, uint64_t P, uint64_t minP) {
    if (m == 0) return 0;
    if (m < minP || m < P) return 1;
    const uint64_t T = std::max<uint64_t>(std::min<uint64_t>(minP, P / 2), 1024);
    return m % P >= T ? m / P + 1 : m / P;
}

int forced_code(const uint32_t lv[4]) {
    for (int i = 0; i < 4; ++i)
        if (lv[i] >= kW) return i;
    return -1;
}

int validate(const burr_params &p, uint32_t r) {
    if (r < 1 || r > 32) return fail(BURR_ERR_INVALID, "r=%u outside [1,32]", r);
    if (p.ribbon_width != kW) return fail(BURR_ERR_INVALID, "ribbon_width must be 64");
    if (p.bucket_slots != 64 && p.bucket_slots != 128)
        return fail(BURR_ERR_INVALID, "bucket_slots must be 64 or 128");
    if (p.threshold_mode != BURR_THRESH_2BIT && p.threshold_mode != BURR_THRESH_1PLUS)
        return fail(BURR_ERR_INVALID, "threshold_mode must be BURR_THRESH_2BIT or BURR_THRESH_1PLUS");
    if (p.layers > BURR_MAX_LAYERS) return fail(BURR_ERR_INVALID, "layers > %d", BURR_MAX_LAYERS);
    if (!(p.levels[0] == 0 && p.levels[0] < p.levels[1] && p.levels[1] < p.levels[2] &&
          p.levels[2] < p.levels[3] && p.levels[3] == p.bucket_slots))
        return fail(BURR_ERR_INVALID, "levels must be 0 < l1 < l2 < bucket_slots");
    if (forced_code(p.levels) < 0) return fail(BURR_ERR_INVALID, "no level >= ribbon width");
    if (!(p.load_factor > 0.0) || !std::isfinite(p.load_factor))
        return fail(BURR_ERR_INVALID, "load_factor must be positive");
    if (p.partition_slots == 0 || p.partition_slots % p.bucket_slots != 0)
        return fail(BURR_ERR_INVALID, "partition_slots must be a positive multiple of bucket_slots");
    if (p.lower_partition_slots % p.bucket_slots != 0)
        return fail(BURR_ERR_INVALID, "lower_partition_slots must be a multiple of bucket_slots");
    if (p.cut_search > BURR_CUT_DIFF) return fail(BURR_ERR_INVALID, "cut_search must be a BURR_CUT_* value");
    if (!(p.fallback_slack >= 0.0) || !std::isfinite(p.fallback_slack))
        return fail(BURR_ERR_INVALID, "fallback_slack must be >= 0");
    return BURR_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Keep freed stream-ordered memory in the current device's pool (once per
// device; callers may be on several host threads).
void keep_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// Device memory of the library: the caller's allocator when one is set
// (burr_set_allocator), else the device's stream-ordered pool.  Every block
// the library holds is counted, so the allocator cannot change under it.
struct AllocHook {
    burr_alloc_fn alloc = nullptr;
    burr_free_fn free = nullptr;
    void *ctx = nullptr;
};
std::mutex g_alloc_mu;
AllocHook g_hook;
std::atomic<int64_t> g_live{0};

AllocHook current_hook() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_hook;
}

}  // namespace

// Stream-ordered allocation usable on `st`.
cudaError_t burr::dev_alloc(void **p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    const AllocHook h = current_hook();
    cudaError_t e;
    if (h.alloc) {
        *p = h.alloc((uint64_t)bytes, (void *)st, h.ctx);
        e = *p ? cudaSuccess : cudaErrorMemoryAllocation;
    } else {
        e = cudaMallocAsync(p, bytes, st);
    }
    if (e == cudaSuccess) g_live.fetch_add(1);
    return e;
}

// Release after the work enqueued on `st` (build scratch).
void burr::dev_free_async(void *p, cudaStream_t st) {
    if (!p) return;
    const AllocHook h = current_hook();
    if (h.free) h.free(p, (void *)st, h.ctx);
    else cudaFreeAsync(p, st);
    g_live.fetch_sub(1);
}

// Release a handle's table: work on any stream may still read it, so wait for
// the device first (as cudaFree does).
void burr::dev_free_sync(void *p) {
    if (!p) return;
    const AllocHook h = current_hook();
    if (h.free) {
        cudaDeviceSynchronize();
        h.free(p, nullptr, h.ctx);
    } else {
        cudaFree(p);
    }
    g_live.fetch_sub(1);
}

namespace {

// Device allocations released together, in stream order.
struct Arena {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Arena(cudaStream_t s) : st(s) {}
    cudaError_t alloc(void **p, size_t bytes) {
        if (bytes == 0) bytes = 256;
        cudaError_t e = dev_alloc(p, bytes, st);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) {
                dev_free_async(q, st);
                q = nullptr;
            }
    }
    ~Arena() {
        for (void *p : ptrs)
            if (p) dev_free_async(p, st);
    }
};

struct LayerStore {
    uint64_t n = 0, m = 0, nb = 0, K = 0, nbumped = 0, seed_index = 0, sigma = 0;
    uint64_t *thresh = nullptr;   // 2-bit: ceil(nb/32) words (bumping layers)
    uint64_t *flags = nullptr;    // 1+-bit: ceil(nb/64) flag words
    uint32_t *dir = nullptr;      // 1+-bit: ceil(nb/512) ranks (into tbytes)
    uint8_t *tbytes = nullptr;    // 1+-bit: thresholds of flagged buckets, from rank 0 of the launch
    uint64_t nflag = 0;           // 1+-bit: flagged buckets of this layer
    uint64_t tfirst = 0;          // 1+-bit: rank of this layer's first flagged bucket in tbytes
    uint64_t *z = nullptr;        // (m/64)*r words
};

uint64_t flag_words(uint64_t nb) { return (nb + 63) / 64; }
uint64_t dir_blocks(uint64_t nb) { return (nb + 511) / 512; }

// Device tables of a batched build, shared by the handles of its structures
// and released with the last of them.
struct BatchStorage {
    std::vector<void *> ptrs;
    ~BatchStorage() {
        for (void *p : ptrs) dev_free_sync(p);
    }
};

}  // namespace

int burr::set_error(int code, const char *msg) {
    g_err = msg ? msg : "";
    return code;
}

struct burr_handle {
    burr_params p;
    uint32_t r = 0, vbytes = 0;
    uint64_t n = 0;
    LayerStore L[BURR_MAX_LAYERS + 1];
    uint32_t fb_attempt = 0;
    float stage_ms[BURR_MAX_LAYERS + 1][3] = {};
    float total_ms = 0;
    uint64_t launches = 0;
    std::shared_ptr<BatchStorage> shared;   // set for a structure of a batched build
};

namespace {

void free_layers(burr_handle *h) {
    if (h->shared) {                        // tables belong to the batch
        for (auto &S : h->L) {
            S.thresh = S.z = S.flags = nullptr;
            S.dir = nullptr;
            S.tbytes = nullptr;
        }
        return;
    }
    for (auto &S : h->L) {
        dev_free_sync(S.thresh);
        dev_free_sync(S.flags);
        dev_free_sync(S.dir);
        dev_free_sync(S.tbytes);
        dev_free_sync(S.z);
        S.thresh = S.z = S.flags = nullptr;
        S.dir = nullptr;
        S.tbytes = nullptr;
    }
}

// Window of the band under BURR_FLAG_TEST_WINDOW: small enough that ordinary
// layers have pivots past it, so the overflow path can be driven by a test.
constexpr uint32_t kTestWindow = 136;

LayerDesc make_desc(const burr_params &p, uint32_t r, uint64_t n, uint64_t m, uint64_t sigma, uint64_t K,
                    bool fallback, uint64_t P) {
    LayerDesc L;
    memset(&L, 0, sizeof(L));
    L.n = n;
    L.m = m;
    L.range = m >= kW ? m - kW + 1 : 0;
    L.sigma = sigma;
    L.nb = num_buckets(m, p.bucket_slots);
    L.P = fallback ? (m ? m : 1) : P;
    L.K = (uint32_t)K;
    L.r = r;
    L.B = p.bucket_slots;
    L.fallback = fallback ? 1u : 0u;
    for (int i = 0; i < 4; ++i) L.levels[i] = p.levels[i];
    L.forced_code = (uint32_t)forced_code(p.levels);
    L.vmask = r >= 32 ? 0xffffffffu : ((1u << r) - 1u);
    L.mode = p.threshold_mode;
    L.window = (p.flags & BURR_FLAG_TEST_WINDOW) ? kTestWindow : 0u;
    L.test_slack = (p.flags & BURR_FLAG_TEST_SLACK) ? 1u : 0u;
    return L;
}

struct Timer {
    bool on;
    cudaStream_t st;
    std::vector<cudaEvent_t> ev;
    Timer(bool o, cudaStream_t s) : on(o), st(s) {}
    int mark() { return mark_on(st); }
    int mark_on(cudaStream_t s) {
        if (!on) return -1;
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, s);
        ev.push_back(e);
        return (int)ev.size() - 1;
    }
    float ms(int a, int b) {
        if (!on || a < 0 || b < 0) return 0.f;
        float t = 0;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    ~Timer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

// A second stream for back-substitution: layer l's back-substitution does not
// feed layer l+1 (only its bumped keys do), so it runs while layer l+1 sorts
// and bands.  The band buffers rotate over three sets (layer l uses set l % 3)
// so that neither layer l+1 nor layer l+2 overwrites the band layer l is still
// solving: with two sets, layer l+2 waited for layer l's back-substitution,
// which is the longest (layer 0's).  On destruction the build stream waits for
// the side stream, so every later free on the build stream is ordered after
// the side stream's reads.
constexpr int kBandSets = 3;
// CTAs per SM of a bumping layer's back-substitution (0: no cap).  It runs
// beside the next layers; capped, it leaves registers free for their kernels.
#ifndef BURR_BACKSUB_CTAS_PER_SM
#define BURR_BACKSUB_CTAS_PER_SM 0
#endif
constexpr uint32_t kBacksubCtasPerSm = BURR_BACKSUB_CTAS_PER_SM;
// Percent of a large layer's partitions (4096 or more) in its first band
// launch (0: one launch).  The rest go in a second launch on a stream of its
// own, started together with the first, and the first launch's
// back-substitution starts as soon as the first launch ends, in the SMs that
// the band's last partitions leave idle.  Measured at 10^9 keys (r = 8): one
// launch 96.1 ms per build; 70 / 80 / 90 / 95 percent 95.3 / 95.0 / 94.2 /
// 94.3 ms (the layer-0 band takes 1.2 ms longer, the back-substitution after
// it 3.1 ms less).
#ifndef BURR_BAND_SPLIT
#define BURR_BAND_SPLIT 90
#endif
constexpr uint32_t kBandSplitPct = BURR_BAND_SPLIT;
// Layers sorted in two scatter passes use fixed-capacity bins instead of
// counting passes (launch_sort_slack_*), with an exact sort again if a bin
// overflowed; 0 turns this off.
#ifndef BURR_SORT_SLACK
#define BURR_SORT_SLACK 1
#endif
constexpr bool kSortSlack = BURR_SORT_SLACK != 0;
constexpr int kOrderSlot = kBandSets;      // event slots after the per-set ones
constexpr int kJoinSlot = kBandSets + 1;
constexpr int kFinalSlot = kBandSets + 2;
constexpr int kSplitSlot = kBandSets + 3;
constexpr int kSplitEndSlot = kBandSets + 4;
constexpr int kCopySlot = kBandSets + 5;
// Keys per chunk of host input copied ahead of the sort's first pass.
constexpr uint64_t kStreamChunk = 1ull << 24;
struct SideStream {
    cudaStream_t main, side = nullptr, band2 = nullptr, copy = nullptr;
    cudaEvent_t ev[kBandSets + 6] = {};
    explicit SideStream(cudaStream_t m) : main(m) {}
    cudaError_t init() {
        cudaError_t e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess && kBandSplitPct) e = cudaStreamCreateWithFlags(&band2, cudaStreamNonBlocking);
        for (int i = 0; i < kBandSets + 6 && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
        return e;
    }
    cudaError_t copy_init() { return copy ? cudaSuccess : cudaStreamCreateWithFlags(&copy, cudaStreamNonBlocking); }
    // `to` waits for everything enqueued so far on `from`
    cudaError_t order(cudaStream_t from, cudaStream_t to, int slot) {
        cudaError_t e = cudaEventRecord(ev[slot], from);
        return e == cudaSuccess ? cudaStreamWaitEvent(to, ev[slot], 0) : e;
    }
    // mark the end of the back-substitution that read band set `set`
    cudaError_t solved(int set) { return cudaEventRecord(ev[set], side); }
    // the main stream waits until band set `set` is no longer read (no-op if never used)
    cudaError_t reuse(int set) { return cudaStreamWaitEvent(main, ev[set], 0); }
    ~SideStream() {
        if (copy) {
            if (ev[kFinalSlot] && cudaEventRecord(ev[kFinalSlot], copy) == cudaSuccess)
                cudaStreamWaitEvent(main, ev[kFinalSlot], 0);
            cudaStreamDestroy(copy);
        }
        if (band2) {
            if (ev[kFinalSlot] && cudaEventRecord(ev[kFinalSlot], band2) == cudaSuccess)
                cudaStreamWaitEvent(main, ev[kFinalSlot], 0);
            cudaStreamDestroy(band2);
        }
        if (side) {
            if (ev[kFinalSlot] && cudaEventRecord(ev[kFinalSlot], side) == cudaSuccess)
                cudaStreamWaitEvent(main, ev[kFinalSlot], 0);
            cudaStreamDestroy(side);
        }
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
};

int build_impl(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params &p,
               cudaStream_t st, burr_handle *h) {
    TraceRange trace("burr_build");
    const uint32_t vb = value_bytes(r);
    keep_pool_memory();
    Arena ar(st);
    Timer tm((p.flags & BURR_FLAG_TIMING) != 0, st);
    SideStream side(st);   // declared after the arena: destroyed first
    CK(side.init(), "side stream");
    const int t_begin = tm.mark();
    int tev[BURR_MAX_LAYERS + 1][7];   // [5], [6]: first back-substitution launch of a split band
    for (auto &row : tev)
        for (int &x : row) x = -1;

    // Inputs on the device.  Where layer 0 uses the fixed-capacity sort, host
    // inputs are copied in chunks on a stream of their own, and the sort's
    // first pass takes each chunk as it arrives (the copy, at the host link's
    // speed, takes several times the pass); otherwise they are copied here.
    const uint64_t m0 = layer_slots(n, p.load_factor);
    size_t slack0 = 0;
    if (kSortSlack && n > 0 && m0 < (1ull << 32)) {
        const uint64_t K0 = num_partitions(m0, layer_partition_slots(p, 0), p.min_partition_slots);
        const LayerDesc L0 = make_desc(p, r, n, m0, layer_seed(p.seed, 0), K0, false, layer_partition_slots(p, 0));
        slack0 = sort_slack_scratch_bytes(L0, vb);
    }
    const bool host_keys = !is_device_ptr(keys), host_vals = !is_device_ptr(values);
    const bool stream_in = (host_keys || host_vals) && slack0 != 0 && p.layers > 0;
    const uint64_t *dkeys = keys;
    const void *dvals = values;
    if (host_keys) {
        void *d;
        CK(ar.alloc(&d, n * 8), "alloc keys");
        if (!stream_in) CK(cudaMemcpyAsync(d, keys, n * 8, cudaMemcpyHostToDevice, st), "copy keys");
        dkeys = (const uint64_t *)d;
    }
    if (host_vals) {
        void *d;
        CK(ar.alloc(&d, n * vb), "alloc values");
        if (!stream_in) CK(cudaMemcpyAsync(d, values, n * vb, cudaMemcpyHostToDevice, st), "copy values");
        dvals = d;
    }

    // scratch sized for layer 0 (later layers and a normal base case are smaller)
    uint64_t cap_m = std::max<uint64_t>(m0, 64), cap_nb = num_buckets(cap_m, p.bucket_slots);
    void *sk, *sv, *bst, *ss, *cg, *yg, *bk[2], *bv[2], *ctr;
    CK(ar.alloc(&sk, n * 8), "alloc sorted keys");
    CK(ar.alloc(&sv, n * vb), "alloc sorted values");
    CK(ar.alloc(&bst, (cap_nb + 1) * 4), "alloc bucket offsets");
    // the exact sort's scratch, or the fixed-capacity sort's for layer 0 if larger
    size_t ss_bytes = std::max(sort_scratch_bytes(n, cap_m, vb), slack0);
    CK(ar.alloc(&ss, ss_bytes), "alloc sort scratch");
    void *cgs[kBandSets] = {}, *ygs[kBandSets] = {};
    uint64_t cgcap[kBandSets] = {};
    CK(ar.alloc(&cg, cap_m * 8), "alloc band");
    CK(ar.alloc(&yg, cap_m * vb), "alloc band values");
    cgs[0] = cg;
    ygs[0] = yg;
    cgcap[0] = cap_m;
    CK(ar.alloc(&bk[0], n * 8), "alloc bumped keys");
    CK(ar.alloc(&bv[0], n * vb), "alloc bumped values");
    bk[1] = bv[1] = nullptr;
    CK(ar.alloc(&ctr, 64), "alloc counters");
    unsigned long long *bcount = (unsigned long long *)ctr;
    uint32_t *err = (uint32_t *)((char *)ctr + 8);
    // 1+-bit thresholds: exact threshold per bucket, one segment covering
    // every directory block of the layer
    const bool onep = p.threshold_mode == BURR_THRESH_1PLUS;
    uint8_t *tex = nullptr;
    uint32_t *tcounts = nullptr, *blkseg = nullptr;
    ThreshSeg *dseg = nullptr;
    if (onep) {
        CK(ar.alloc((void **)&tex, cap_nb), "alloc exact thresholds");
        CK(ar.alloc((void **)&tcounts, dir_blocks(cap_nb) * 4), "alloc threshold counts");
        CK(ar.alloc((void **)&blkseg, dir_blocks(cap_nb) * 4), "alloc threshold blocks");
        CK(ar.alloc((void **)&dseg, sizeof(ThreshSeg)), "alloc threshold segment");
        CK(cudaMemsetAsync(blkseg, 0, dir_blocks(cap_nb) * 4, st), "clear threshold blocks");
    }

    // A bumping layer's back-substitution is queued on the side stream only
    // after the next layer's sort: it fills every SM for milliseconds, and the
    // sort, queued behind it, used to wait that long (layer 1 of a 10^9-key
    // build started 2.9 ms after layer 0's band ended).
    struct PendingBacksub {
        bool on;
        uint32_t l;
        int set;
        LayerDesc L;
        uint64_t *z;
    } pending{};
    auto start_backsub = [&]() -> cudaError_t {
        if (!pending.on) return cudaSuccess;
        pending.on = false;
        cudaError_t e = side.order(st, side.side, kOrderSlot);
        if (e != cudaSuccess) return e;
        tev[pending.l][3] = tm.mark_on(side.side);
        e = launch_backsub(pending.L, vb, (const uint64_t *)cgs[pending.set], ygs[pending.set], pending.z, side.side,
                           nullptr, kBacksubCtasPerSm);
        if (e != cudaSuccess) return e;
        tev[pending.l][4] = tm.mark_on(side.side);
        return side.solved(pending.set);
    };
    const uint64_t *cur_k = dkeys;
    const void *cur_v = dvals;
    uint64_t cur_n = n;
    int which = 0;
    static const char *kLayerNames[] = {"burr layer 0", "burr layer 1", "burr layer 2", "burr layer 3",
                                        "burr layer 4", "burr layer 5", "burr layer 6", "burr layer 7"};
    for (uint32_t l = 0; l < p.layers; ++l) {
        LayerStore &S = h->L[l];
        S.n = cur_n;
        S.seed_index = l;
        if (cur_n == 0) continue;
        TraceRange layer_trace(kLayerNames[l]);
        S.m = layer_slots(cur_n, p.load_factor);
        if (S.m >= (1ull << 32)) return fail(BURR_ERR_INVALID, "layer %u needs %llu slots (>= 2^32)", l,
                                             (unsigned long long)S.m);
        S.nb = num_buckets(S.m, p.bucket_slots);
        S.K = num_partitions(S.m, layer_partition_slots(p, l), p.min_partition_slots);
        S.sigma = layer_seed(p.seed, l);
        const uint64_t tw = (S.nb + 31) / 32, nd = dir_blocks(S.nb);
        if (onep) {
            CK(dev_alloc((void **)&S.flags, flag_words(S.nb) * 8, st), "alloc threshold flags");
            CK(dev_alloc((void **)&S.dir, (nd + 1) * 4, st), "alloc threshold directory");
            const ThreshSeg seg{0, S.nb, 0, 0};
            CK(cudaMemcpyAsync(dseg, &seg, sizeof(seg), cudaMemcpyHostToDevice, st), "copy threshold segment");
        } else {
            CK(dev_alloc((void **)&S.thresh, std::max<uint64_t>(tw, 1) * 8, st), "alloc thresholds");
            CK(cudaMemsetAsync(S.thresh, 0, tw * 8, st), "clear thresholds");
        }
        CK(dev_alloc((void **)&S.z, std::max<uint64_t>((S.m / 64) * r, 1) * 8, st), "alloc table");
        if (!bk[which]) {
            CK(ar.alloc(&bk[which], cur_n * 8), "alloc bumped keys");
            CK(ar.alloc(&bv[which], cur_n * vb), "alloc bumped values");
        }
        CK(cudaMemsetAsync(ctr, 0, 64, st), "clear counters");
        LayerDesc L = make_desc(p, r, cur_n, S.m, S.sigma, S.K, false, layer_partition_slots(p, l));
        const bool search = p.cut_search != BURR_CUT_NONE && S.K > 1;
        if (search) {
            uint32_t *dc;
            CK(ar.alloc((void **)&dc, (S.K + 1) * 4), "alloc cuts");
            L.cuts = dc;
        }
        const int set = (int)(l % kBandSets);
        if (cgcap[set] < S.m) {           // later band sets, sized by the first layer that uses them
            CK(ar.alloc(&cgs[set], S.m * 8), "alloc band");
            CK(ar.alloc(&ygs[set], S.m * vb), "alloc band values");
            cgcap[set] = S.m;
        }
        // the band of layer l overwrites the set that layer l-3 solved: wait for it
        CK(side.reuse(set), "order");
        // sorted with fixed-capacity bins where they fit the scratch; if a bin overflowed
        // (kErrSortSlack at the end of the layer), the layer is sorted and banded again exactly
        const size_t slack_bytes = kSortSlack ? sort_slack_scratch_bytes(L, vb) : 0;
        bool slack = slack_bytes != 0 && slack_bytes <= ss_bytes;
        bool streamed = false;   // layer 0: the host inputs have been copied in
        unsigned long long hc[2] = {0, 0};
        uint32_t nflag = 0;
        for (;;) {
            tev[l][0] = tm.mark();
            if (slack) {
                CK(launch_sort_slack_begin(L, vb, ss, st), "sort");
                if (l == 0 && stream_in && !streamed) {
                    // host inputs: copy chunk c, then pass 1 over it, while chunk c+1 is copied
                    CK(side.copy_init(), "copy stream");
                    CK(side.order(st, side.copy, kCopySlot), "order");   // after the allocations
                    for (uint64_t lo = 0; lo < n; lo += kStreamChunk) {
                        const uint64_t hi = std::min<uint64_t>(n, lo + kStreamChunk);
                        if (host_keys)
                            CK(cudaMemcpyAsync((uint64_t *)dkeys + lo, keys + lo, (hi - lo) * 8,
                                               cudaMemcpyHostToDevice, side.copy),
                               "copy keys");
                        if (host_vals)
                            CK(cudaMemcpyAsync((char *)dvals + lo * vb, (const char *)values + lo * vb,
                                               (hi - lo) * vb, cudaMemcpyHostToDevice, side.copy),
                               "copy values");
                        CK(side.order(side.copy, st, kCopySlot), "order");
                        CK(launch_sort_slack_pass1(L, vb, cur_k, cur_v, lo, hi, ss, err, st), "sort");
                        h->launches += 1;
                    }
                    h->launches -= 1;
                    streamed = true;
                } else {
                    CK(launch_sort_slack_pass1(L, vb, cur_k, cur_v, 0, cur_n, ss, err, st), "sort");
                }
                CK(launch_sort_slack_end(L, vb, (uint64_t *)sk, sv, (uint32_t *)bst, ss, err, st), "sort");
            } else {
                CK(launch_sort(L, vb, cur_k, cur_v, (uint64_t *)sk, sv, (uint32_t *)bst, ss, err, st), "sort");
            }
            CK(start_backsub(), "backsub");   // the previous layer's, now that this layer's sort is queued
            if (search) {
                CK(launch_cut_search(L, (const uint64_t *)sk, (const uint32_t *)bst, p.cut_search, p.cut_search_range,
                                     const_cast<uint32_t *>(L.cuts), st),
                   "cut search");
                h->launches += 1;
            }
            tev[l][1] = tm.mark();
            LayerDesc Lpend = L;
            const uint64_t K1 = kBandSplitPct && side.band2 && !search ? S.K * kBandSplitPct / 100 : 0;
            if (K1 > 0 && K1 < S.K && S.K >= 4096) {
                // first launch on the build stream, second on its own stream (started together, so
                // the second one's partitions fill the SMs the first one's last partitions leave);
                // the first launch's back-substitution follows it on the side stream
                LayerDesc La = L, Lb = L;
                La.part_hi = (uint32_t)K1;
                Lb.part_lo = (uint32_t)K1;
                CK(side.order(st, side.band2, kSplitSlot), "order");
                CK(launch_band(La, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cgs[set], ygs[set],
                               S.thresh, tex, (uint64_t *)bk[which], bv[which], bcount, err, st), "band");
                CK(launch_band(Lb, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cgs[set], ygs[set],
                               S.thresh, tex, (uint64_t *)bk[which], bv[which], bcount, err, side.band2), "band");
                CK(side.order(st, side.side, kOrderSlot), "order");
                tev[l][5] = tm.mark_on(side.side);
                CK(launch_backsub(La, vb, (const uint64_t *)cgs[set], ygs[set], S.z, side.side, nullptr,
                                  kBacksubCtasPerSm),
                   "backsub");
                tev[l][6] = tm.mark_on(side.side);
                CK(side.order(side.band2, st, kSplitEndSlot), "order");
                Lpend = Lb;
                h->launches += 2;
            } else {
                CK(launch_band(L, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cgs[set], ygs[set],
                               S.thresh, tex, (uint64_t *)bk[which], bv[which], bcount, err, st), "band");
            }
            tev[l][2] = tm.mark();
            if (onep) CK(launch_thresh_flags(tex, dseg, blkseg, (uint32_t)nd, S.flags, tcounts, S.dir, st), "flags");
            pending = PendingBacksub{true, l, set, Lpend, S.z};
            h->launches += (slack ? 6 : sort_kernel_count(L)) + 2 + (onep ? 2 : 0);
            CK(cudaMemcpyAsync(hc, ctr, 16, cudaMemcpyDeviceToHost, st), "read counters");
            if (onep) CK(cudaMemcpyAsync(&nflag, S.dir + nd, 4, cudaMemcpyDeviceToHost, st), "read threshold count");
            CK(cudaStreamSynchronize(st), "layer");
            if (!(hc[1] & kErrSortSlack)) break;
            // a bin overflowed: this layer's outputs are partial; sort and band it again exactly
            slack = false;
            pending.on = false;
            CK(cudaStreamSynchronize(side.side), "layer");   // a split band's first back-substitution
            if (!onep) CK(cudaMemsetAsync(S.thresh, 0, tw * 8, st), "clear thresholds");
            CK(cudaMemsetAsync(ctr, 0, 64, st), "clear counters");
        }
        const uint32_t e = (uint32_t)(hc[1] & 0xffffffffu);
        if (e & kErrRingOverflow) return fail(BURR_ERR_INTERNAL, "layer %u: pivot left the band window (509 slots)", l);
        if (e) return fail(BURR_ERR_INTERNAL, "layer %u: device error 0x%x", l, e);
        S.nbumped = hc[0];
        if (onep) {
            // exact thresholds of the flagged buckets (before the next layer's
            // band reuses the per-bucket array)
            S.nflag = nflag;
            S.tfirst = 0;
            CK(dev_alloc((void **)&S.tbytes, std::max<uint64_t>(nflag, 1), st), "alloc thresholds");
            CK(launch_thresh_compact(tex, dseg, blkseg, (uint32_t)nd, S.flags, S.dir, S.tbytes, st), "compact");
            h->launches += 1;
        }
        cur_k = (const uint64_t *)bk[which];
        cur_v = bv[which];
        cur_n = S.nbumped;
        which ^= 1;   // layer l+1 reads this list and bumps into the other one (n_{l+1} <= n_l)
    }

    CK(start_backsub(), "backsub");   // the last bumping layer's
    // base case: no bumping; grow by 10% and change the seed until it solves
    LayerStore &F = h->L[p.layers];
    F.n = cur_n;
    if (cur_n > 0) {
        TraceRange base_trace("burr base case");
        bool solved = false;
        for (uint32_t a = 0; a <= p.fallback_max_retries && !solved; ++a) {
            if (F.z) {
                dev_free_async(F.z, st);
                F.z = nullptr;
            }
            F.m = fallback_slots(cur_n, p.fallback_slack, a);
            if (F.m >= (1ull << 32)) return fail(BURR_ERR_INVALID, "base case needs >= 2^32 slots");
            F.nb = num_buckets(F.m, p.bucket_slots);
            F.K = 1;
            F.seed_index = p.layers + a;
            F.sigma = layer_seed(p.seed, F.seed_index);
            const int set = (int)(p.layers % kBandSets);
            if (cgcap[set] < F.m) {
                CK(ar.alloc(&cgs[set], F.m * 8), "alloc band");
                CK(ar.alloc(&ygs[set], F.m * vb), "alloc band values");
                cgcap[set] = F.m;
            }
            if (F.m > cap_m) {
                ar.release(bst);
                ar.release(ss);
                cap_m = F.m;
                cap_nb = num_buckets(cap_m, p.bucket_slots);
                CK(ar.alloc(&bst, (cap_nb + 1) * 4), "alloc bucket offsets");
                ss_bytes = sort_scratch_bytes(n, cap_m, vb);
                CK(ar.alloc(&ss, ss_bytes), "alloc sort scratch");
            }
            CK(side.reuse(set), "order");
            CK(dev_alloc((void **)&F.z, (F.m / 64) * r * 8, st), "alloc table");
            CK(cudaMemsetAsync(ctr, 0, 64, st), "clear counters");
            const LayerDesc L = make_desc(p, r, cur_n, F.m, F.sigma, 1, true, F.m);
            const int t0 = tm.mark();
            CK(launch_sort(L, vb, cur_k, cur_v, (uint64_t *)sk, sv, (uint32_t *)bst, ss, err, st), "sort");
            const int t1 = tm.mark();
            CK(launch_band(L, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cgs[set], ygs[set],
                           nullptr, nullptr, nullptr, nullptr, bcount, err, st), "band");
            h->launches += sort_kernel_count(L) + 1;
            uint32_t he = 0;
            CK(cudaMemcpyAsync(&he, err, 4, cudaMemcpyDeviceToHost, st), "read error word");
            CK(cudaStreamSynchronize(st), "base case");
            if (he & ~kErrUnsolvable) return fail(BURR_ERR_INTERNAL, "base case: device error 0x%x", he);
            if (he & kErrUnsolvable) continue;
            const int t2 = tm.mark();
            CK(launch_backsub(L, vb, (const uint64_t *)cgs[set], ygs[set], F.z, st), "backsub");
            h->launches += 1;
            const int t3 = tm.mark();
            solved = true;
            h->fb_attempt = a;
            tev[p.layers][0] = t0;
            tev[p.layers][1] = t1;
            tev[p.layers][2] = t2;
            tev[p.layers][3] = t3;
        }
        if (!solved)
            return fail(BURR_ERR_UNSOLVABLE, "base case unsolved after %u retries (duplicate keys?)",
                        p.fallback_max_retries);
    }
    CK(side.order(side.side, st, kJoinSlot), "order");
    const int t_end = tm.mark();
    CK(cudaStreamSynchronize(st), "build");
    for (uint32_t l = 0; l <= p.layers; ++l) {
        if (tev[l][0] < 0) continue;
        h->stage_ms[l][0] = tm.ms(tev[l][0], tev[l][1]);
        h->stage_ms[l][1] = tm.ms(tev[l][1], tev[l][2]);
        // back-substitution of a bumping layer runs on the side stream,
        // overlapped with the next layers; this is its span on that stream
        // (the sum of both launches' spans where the band was split)
        h->stage_ms[l][2] = l < p.layers ? tm.ms(tev[l][3], tev[l][4]) + tm.ms(tev[l][5], tev[l][6])
                                         : tm.ms(tev[l][2], tev[l][3]);
    }
    h->total_ms = tm.ms(t_begin, t_end);
    return BURR_OK;
}

// ---------------------------------------------------------------------------
// Batched build: S independent structures, one launch per stage per layer over
// all of them.  Each structure follows exactly the single-structure rules
// (sizes, seeds, cuts, thresholds), so its export equals its solo build with
// the same parameters; only the work is scheduled together.
// ---------------------------------------------------------------------------

// Partition size for a batch whose caller left it to the library: the largest
// of 2^16, 2^15, 2^14 slots that still gives every SM at least 8 partitions in
// the first layer (more partitions hide more latency; smaller ones bump more
// keys at the cuts).
uint64_t autotune_partition_slots(const std::vector<uint64_t> &n, double alpha) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (uint64_t P = 65536; P >= 16384; P /= 2) {
        uint64_t parts = 0;
        for (uint64_t x : n) parts += num_partitions(layer_slots(x, alpha), P, P);
        if (parts >= 8ull * (uint64_t)sms) return P;
    }
    return 16384;
}

struct BatchTables {
    std::vector<StructDesc> sd;
    std::vector<uint32_t> part_struct, group_struct, tile_struct;
    std::vector<uint32_t> part_order;   // partitions by decreasing length (the band's launch order)
    std::vector<uint64_t> tile_lo;
    std::vector<uint32_t> who;   // active index -> structure index
    uint64_t nbuckets = 0, ngroups = 0, nparts = 0, slots = 0, tw = 0, zw = 0, nkeys = 0;
};

// Descriptors of one layer for the structures in `who` with counts n[s].
// fb_attempt == nullptr: a bumping layer with index l; else the base case.
int batch_tables(const burr_params &p, const std::vector<uint32_t> &r, const std::vector<uint64_t> &offsets,
                 const std::vector<uint64_t> &n, const std::vector<uint32_t> &who, uint32_t l,
                 const std::vector<uint32_t> *fb_attempt, BatchTables &T) {
    T = BatchTables();
    T.who = who;
    const bool fb = fb_attempt != nullptr;
    const uint64_t Pl = layer_partition_slots(p, l);
    {
        // sizes of the tables first (for 10^4 structures they hold ~10^6 entries)
        uint64_t np = 0, ng = 0, nt = 0;
        for (const uint32_t s : who) {
            const uint64_t m = fb ? fallback_slots(n[s], p.fallback_slack, (*fb_attempt)[s])
                                  : layer_slots(n[s], p.load_factor);
            np += fb ? 1 : num_partitions(m, Pl, p.min_partition_slots);
            ng += (num_buckets(m, p.bucket_slots) + 63) / 64;
            nt += (n[s] + kSortTile - 1) / kSortTile;
        }
        T.sd.reserve(who.size());
        T.part_struct.reserve(np);
        T.group_struct.reserve(ng);
        T.tile_struct.reserve(nt);
        T.tile_lo.reserve(nt);
    }
    for (uint32_t i = 0; i < who.size(); ++i) {
        const uint32_t s = who[i];
        const uint64_t m = fb ? fallback_slots(n[s], p.fallback_slack, (*fb_attempt)[s])
                              : layer_slots(n[s], p.load_factor);
        if (m >= (1ull << 32)) return fail(BURR_ERR_INVALID, "structure %u needs >= 2^32 slots", s);
        const uint64_t K = fb ? 1 : num_partitions(m, Pl, p.min_partition_slots);
        const uint64_t sigma = layer_seed(p.seed, fb ? p.layers + (*fb_attempt)[s] : l);
        StructDesc D;
        memset(&D, 0, sizeof(D));
        D.L = make_desc(p, r[s], n[s], m, sigma, K, fb, fb ? m : Pl);
        const uint64_t ng = (D.L.nb + 63) / 64;
        if (ng > kMaxGroupsPerStruct)
            return fail(BURR_ERR_INVALID,
                        "structure %u (%llu keys) is too large for a batched build; build it with burr_build", s,
                        (unsigned long long)n[s]);
        D.key_base = offsets[s];
        D.out_base = offsets[s];
        D.bucket_base = T.nbuckets;
        D.group_base = T.ngroups;
        D.slot_base = T.slots;
        D.tw_base = T.tw;
        D.z_base = T.zw;
        D.part_base = (uint32_t)T.nparts;
        D.ngroups = (uint32_t)ng;
        T.sd.push_back(D);
        T.part_struct.insert(T.part_struct.end(), K, i);
        T.group_struct.insert(T.group_struct.end(), ng, i);
        T.tile_struct.insert(T.tile_struct.end(), (n[s] + kSortTile - 1) / kSortTile, i);
        for (uint64_t t = 0; t < n[s]; t += kSortTile) T.tile_lo.push_back(offsets[s] + t);
        T.nbuckets += D.L.nb;
        T.ngroups += ng;
        T.nparts += K;
        T.slots += m;
        T.tw += (D.L.nb + 31) / 32;
        T.zw += (m / 64) * r[s];
        T.zw = (T.zw + 3) & ~3ull;   // every structure's table starts on 32 bytes (wide query loads)
        T.nkeys += n[s];
    }
    // Longest partitions first: a warp's partition is one dependent chain, so
    // the launch ends with the short ones instead of a long one started late.
    // (A counting sort on the length in buckets, stable like the comparison
    // sort it replaces: most partitions share a handful of lengths.)
    std::vector<uint32_t> len(T.nparts);
    uint32_t lmax = 0;
    for (uint32_t i = 0; i < T.sd.size(); ++i)
        for (uint64_t k = 0; k < T.sd[i].L.K; ++k) {
            const uint32_t x = (uint32_t)(part_bucket(T.sd[i].L, k + 1) - part_bucket(T.sd[i].L, k));
            len[T.sd[i].part_base + k] = x;
            lmax = std::max(lmax, x);
        }
    std::vector<uint32_t> at(lmax + 2, 0);
    for (const uint32_t x : len) ++at[lmax - x + 1];   // decreasing length
    for (uint32_t x = 1; x <= lmax + 1; ++x) at[x] += at[x - 1];
    T.part_order.resize(T.nparts);
    for (uint32_t j = 0; j < T.nparts; ++j) T.part_order[at[lmax - len[j]]++] = j;
    return BURR_OK;
}

// Copy a host vector into a device buffer taken from the arena.
template <typename X>
cudaError_t upload(Arena &ar, const std::vector<X> &v, X **d, cudaStream_t st) {
    cudaError_t e = ar.alloc((void **)d, std::max<size_t>(v.size(), 1) * sizeof(X));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(*d, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice, st);
}

int build_batch_impl(const uint64_t *keys, const void *values, const std::vector<uint64_t> &offsets,
                     const std::vector<uint32_t> &r, const burr_params &p, cudaStream_t st,
                     std::vector<burr_handle *> &hs, const std::shared_ptr<BatchStorage> &store) {
    TraceRange trace("burr_build_batch");
    const uint32_t S = (uint32_t)r.size();
    uint32_t rmax = 1;
    for (uint32_t x : r) rmax = std::max(rmax, x);
    const uint32_t vb = value_bytes(rmax);
    const uint64_t N = offsets[S];
    keep_pool_memory();
    Arena ar(st);
    Timer tm((p.flags & BURR_FLAG_TIMING) != 0, st);
    SideStream side(st);   // back-substitution beside the next layer, as in build_impl
    CK(side.init(), "side stream");
    const int t_begin = tm.mark();

    const uint64_t *dkeys = keys;
    const void *dvals = values;
    if (!is_device_ptr(keys)) {
        void *d;
        CK(ar.alloc(&d, N * 8), "alloc keys");
        CK(cudaMemcpyAsync(d, keys, N * 8, cudaMemcpyHostToDevice, st), "copy keys");
        dkeys = (const uint64_t *)d;
    }
    if (!is_device_ptr(values)) {
        void *d;
        CK(ar.alloc(&d, N * vb), "alloc values");
        CK(cudaMemcpyAsync(d, values, N * vb, cudaMemcpyHostToDevice, st), "copy values");
        dvals = d;
    }
    void *bk[2], *bv2[2], *sk, *sv, *ctr;
    for (int i = 0; i < 2; ++i) {
        CK(ar.alloc(&bk[i], N * 8), "alloc bumped keys");
        CK(ar.alloc(&bv2[i], N * vb), "alloc bumped values");
    }
    CK(ar.alloc(&sk, N * 8), "alloc sorted keys");
    CK(ar.alloc(&sv, N * vb), "alloc sorted values");
    CK(ar.alloc(&ctr, (size_t)S * 12 + 64), "alloc counters");
    unsigned long long *bcount = (unsigned long long *)ctr;
    uint32_t *ffail = (uint32_t *)((char *)ctr + (size_t)S * 8);
    uint32_t *err = ffail + S;
    // buffers sized by the largest layer seen so far; the band arrays rotate over
    // kBandSets sets (a layer's back-substitution may still read its set while
    // the next layers band)
    void *scratch = nullptr, *bst = nullptr;
    void *cgs[kBandSets] = {}, *ygs[kBandSets] = {};
    uint64_t cap_scratch = 0, cap_nb = 0, cgcap[kBandSets] = {};
    auto ensure_band = [&](int set, uint64_t slots) -> int {
        if (slots > cgcap[set]) {
            CK(side.reuse(set), "order");   // its previous user's back-substitution is done
            if (cgs[set]) ar.release(cgs[set]);
            if (ygs[set]) ar.release(ygs[set]);
            CK(ar.alloc(&cgs[set], slots * 8), "alloc band");
            CK(ar.alloc(&ygs[set], slots * vb), "alloc band values");
            cgcap[set] = slots;
        }
        return BURR_OK;
    };
    auto ensure = [&](const BatchTables &T) -> int {
        const size_t need = sort_batch_scratch_bytes(T.nkeys, T.ngroups, vb);
        if (need > cap_scratch) {
            if (scratch) ar.release(scratch);
            CK(ar.alloc(&scratch, need), "alloc sort scratch");
            cap_scratch = need;
        }
        if (T.nbuckets + 1 > cap_nb) {
            if (bst) ar.release(bst);
            CK(ar.alloc(&bst, (T.nbuckets + 1) * 4), "alloc bucket offsets");
            cap_nb = T.nbuckets + 1;
        }
        return BURR_OK;
    };
    // a bumping layer's back-substitution, queued on the side stream after the next layer's sort;
    // bsm[l]: event marks of layer l's back-substitution launches (a split band's first one, the rest)
    struct PendingBatchBacksub {
        bool on = false;
        uint32_t l = 0;
        int set = 0;
        BatchView v;
        uint64_t *z = nullptr;
    } pending;
    std::vector<std::array<int, 4>> bsm(p.layers + 1, std::array<int, 4>{-1, -1, -1, -1});
    auto start_backsub = [&]() -> cudaError_t {
        if (!pending.on) return cudaSuccess;
        pending.on = false;
        cudaError_t e = side.order(st, side.side, kOrderSlot);
        if (e != cudaSuccess) return e;
        bsm[pending.l][2] = tm.mark_on(side.side);
        e = launch_backsub(LayerDesc(), vb, (const uint64_t *)cgs[pending.set], ygs[pending.set], pending.z, side.side,
                           &pending.v);
        if (e != cudaSuccess) return e;
        bsm[pending.l][3] = tm.mark_on(side.side);
        return side.solved(pending.set);
    };
    auto view = [&](const BatchTables &T, BatchView &v) -> int {
        StructDesc *dsd;
        uint32_t *dps, *dpo, *dgs, *dts;
        uint64_t *dtl;
        CK(upload(ar, T.sd, &dsd, st), "upload descriptors");
        CK(upload(ar, T.part_struct, &dps, st), "upload partitions");
        CK(upload(ar, T.part_order, &dpo, st), "upload partition order");
        CK(upload(ar, T.group_struct, &dgs, st), "upload groups");
        CK(upload(ar, T.tile_struct, &dts, st), "upload tiles");
        CK(upload(ar, T.tile_lo, &dtl, st), "upload tiles");
        v.sd = dsd;
        v.part_struct = dps;
        v.part_order = dpo;
        v.group_struct = dgs;
        v.tile_struct = dts;
        v.tile_lo = dtl;
        v.fail = ffail;
        v.nstruct = (uint32_t)T.sd.size();
        v.nparts = (uint32_t)T.nparts;
        v.ngroups = (uint32_t)T.ngroups;
        v.ntiles = (uint32_t)T.tile_struct.size();
        v.nbuckets = T.nbuckets;
        v.nkeys = T.nkeys;
        return BURR_OK;
    };
    auto table_alloc = [&](size_t bytes, auto **d) -> cudaError_t {
        void *q = nullptr;
        cudaError_t e = dev_alloc(&q, std::max<size_t>(bytes, 8), st);
        if (e == cudaSuccess) store->ptrs.push_back(q);
        *d = static_cast<std::remove_reference_t<decltype(**d)> *>(q);
        return e;
    };

    std::vector<uint64_t> n(S);
    for (uint32_t s = 0; s < S; ++s) n[s] = offsets[s + 1] - offsets[s];
    const LayerDesc none = make_desc(p, 1, 0, 64, 0, 0, false, p.partition_slots);
    const uint64_t *cur_k = dkeys;
    const void *cur_v = dvals;
    for (uint32_t l = 0; l < p.layers; ++l) {
        std::vector<uint32_t> who;
        for (uint32_t s = 0; s < S; ++s) {
            hs[s]->L[l].n = n[s];
            hs[s]->L[l].seed_index = l;
            if (n[s]) who.push_back(s);
        }
        if (who.empty()) break;
        BatchTables T;
        int rc = batch_tables(p, r, offsets, n, who, l, nullptr, T);
        if (rc) return rc;
        if ((rc = ensure(T))) return rc;
        // cut search: a table of partition starts per structure with cuts
        const bool search = p.cut_search != BURR_CUT_NONE;
        if (search) {
            uint64_t ncut = 0;
            for (const StructDesc &D : T.sd) ncut += D.L.K > 1 ? D.L.K + 1 : 0;
            uint32_t *dc = nullptr;
            CK(ar.alloc((void **)&dc, std::max<uint64_t>(ncut, 1) * 4), "alloc cuts");
            ncut = 0;
            for (StructDesc &D : T.sd) {
                if (D.L.K < 2) continue;
                D.L.cuts = dc + ncut;
                ncut += D.L.K + 1;
            }
        }
        BatchView v;
        if ((rc = view(T, v))) return rc;
        const int set = (int)(l % kBandSets);
        if ((rc = ensure_band(set, T.slots))) return rc;
        CK(side.reuse(set), "order");   // the set's last back-substitution is done
        void *cg = cgs[set], *yg = ygs[set];
        uint64_t *th = nullptr, *z, *tflags = nullptr;
        uint32_t *tdir = nullptr;
        uint8_t *tex = nullptr;
        // 1+-bit thresholds: one segment per structure (its flag words and
        // directory blocks) in launch-wide arrays
        const bool onep = p.threshold_mode == BURR_THRESH_1PLUS;
        std::vector<ThreshSeg> segs;
        std::vector<uint32_t> blkseg;
        uint64_t nfw = 0;
        if (onep) {
            for (uint32_t i = 0; i < who.size(); ++i) {
                const StructDesc &D = T.sd[i];
                segs.push_back(ThreshSeg{D.bucket_base, D.L.nb, nfw, (uint64_t)blkseg.size()});
                nfw += flag_words(D.L.nb);
                blkseg.insert(blkseg.end(), dir_blocks(D.L.nb), i);
            }
            CK(table_alloc(nfw * 8, &tflags), "alloc threshold flags");
            CK(table_alloc((blkseg.size() + 1) * 4, &tdir), "alloc threshold directory");
            CK(ar.alloc((void **)&tex, std::max<uint64_t>(T.nbuckets, 1)), "alloc exact thresholds");
        } else {
            CK(table_alloc(T.tw * 8, &th), "alloc thresholds");
            CK(cudaMemsetAsync(th, 0, std::max<uint64_t>(T.tw, 1) * 8, st), "clear thresholds");
        }
        CK(table_alloc(T.zw * 8, &z), "alloc tables");
        CK(cudaMemsetAsync(ctr, 0, (size_t)S * 12 + 64, st), "clear counters");
        const int w = (int)(l & 1);
        const int t0 = tm.mark();
        CK(launch_sort_batch(v, vb, cur_k, cur_v, (uint64_t *)sk, sv, (uint32_t *)bst, scratch, st), "sort");
        CK(start_backsub(), "backsub");   // the previous layer's, now that this layer's sort is queued
        if (search) {
            CK(launch_cut_search(none, (const uint64_t *)sk, (const uint32_t *)bst, p.cut_search,
                                 p.cut_search_range, nullptr, st, &v),
               "cut search");
            for (auto *h : hs) h->launches += 1;
        }
        const int t1 = tm.mark();
        // partitions in the order table (longest first): the first 90% in one launch, the rest in a
        // second launch on its own stream, and the first launch's back-substitution right after it
        const uint32_t K1 = kBandSplitPct && v.nparts >= 4096 ? (uint32_t)((uint64_t)v.nparts * kBandSplitPct / 100)
                                                              : 0;
        BatchView vrest = v;
        if (K1 > 0 && K1 < v.nparts && v.part_order) {
            BatchView va = v;
            va.nparts = K1;
            vrest.part_order = v.part_order + K1;
            vrest.nparts = v.nparts - K1;
            CK(side.order(st, side.band2, kSplitSlot), "order");
            CK(launch_band(none, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cg, yg, th, tex,
                           (uint64_t *)bk[w], bv2[w], bcount, err, st, &va), "band");
            CK(launch_band(none, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cg, yg, th, tex,
                           (uint64_t *)bk[w], bv2[w], bcount, err, side.band2, &vrest), "band");
            CK(side.order(st, side.side, kOrderSlot), "order");
            bsm[l][0] = tm.mark_on(side.side);
            CK(launch_backsub(none, vb, (const uint64_t *)cg, yg, z, side.side, &va), "backsub");
            bsm[l][1] = tm.mark_on(side.side);
            CK(side.order(side.band2, st, kSplitEndSlot), "order");
            for (auto *h : hs) h->launches += 2;
        } else {
            CK(launch_band(none, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cg, yg, th, tex,
                           (uint64_t *)bk[w], bv2[w], bcount, err, st, &v), "band");
        }
        const int t2 = tm.mark();
        ThreshSeg *dsegs = nullptr;
        uint32_t *dblk = nullptr, *tcounts = nullptr;
        if (onep) {
            CK(upload(ar, segs, &dsegs, st), "upload threshold segments");
            CK(upload(ar, blkseg, &dblk, st), "upload threshold blocks");
            CK(ar.alloc((void **)&tcounts, std::max<size_t>(blkseg.size(), 1) * 4), "alloc threshold counts");
            CK(launch_thresh_flags(tex, dsegs, dblk, (uint32_t)blkseg.size(), tflags, tcounts, tdir, st), "flags");
        }
        pending.on = true;
        pending.l = l;
        pending.set = set;
        pending.v = vrest;
        pending.z = z;
        for (auto *h : hs) h->launches += 6;
        std::vector<unsigned long long> cnt(who.size());
        std::vector<uint32_t> hdir(onep ? blkseg.size() + 1 : 0);
        uint32_t e = 0;
        CK(cudaMemcpyAsync(cnt.data(), bcount, cnt.size() * 8, cudaMemcpyDeviceToHost, st), "read counters");
        CK(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, st), "read error word");
        if (onep) CK(cudaMemcpyAsync(hdir.data(), tdir, hdir.size() * 4, cudaMemcpyDeviceToHost, st), "read ranks");
        CK(cudaStreamSynchronize(st), "layer");
        if (e & kErrRingOverflow) return fail(BURR_ERR_INTERNAL, "layer %u: pivot left the band window (509 slots)", l);
        if (e) return fail(BURR_ERR_INTERNAL, "layer %u: device error 0x%x", l, e);
        uint8_t *tbytes = nullptr;
        if (onep) {
            CK(table_alloc(std::max<uint64_t>(hdir.back(), 1), &tbytes), "alloc thresholds");
            CK(launch_thresh_compact(tex, dsegs, dblk, (uint32_t)blkseg.size(), tflags, tdir, tbytes, st),
               "compact");
            for (auto *h : hs) h->launches += 3;
        }
        for (uint32_t i = 0; i < who.size(); ++i) {
            const uint32_t s = who[i];
            const StructDesc &D = T.sd[i];
            LayerStore &Ls = hs[s]->L[l];
            Ls.m = D.L.m;
            Ls.nb = D.L.nb;
            Ls.K = D.L.K;
            Ls.sigma = D.L.sigma;
            Ls.nbumped = cnt[i];
            if (onep) {
                const ThreshSeg &g = segs[i];
                Ls.flags = tflags + g.fw_base;
                Ls.dir = tdir + g.dir_base;
                Ls.tbytes = tbytes;
                Ls.tfirst = hdir[g.dir_base];
                Ls.nflag = hdir[g.dir_base + dir_blocks(D.L.nb)] - hdir[g.dir_base];
            } else {
                Ls.thresh = th + D.tw_base;
            }
            Ls.z = z + D.z_base;
            hs[s]->stage_ms[l][0] = tm.ms(t0, t1);
            hs[s]->stage_ms[l][1] = tm.ms(t1, t2);   // [l][2] once the build's events are all recorded
            n[s] = cnt[i];
        }
        cur_k = (const uint64_t *)bk[w];
        cur_v = bv2[w];
    }
    CK(start_backsub(), "backsub");   // the last bumping layer's
    // base case of every structure with keys left; retries per structure
    std::vector<uint32_t> attempt(S, 0), left;
    for (uint32_t s = 0; s < S; ++s) {
        hs[s]->L[p.layers].n = n[s];
        hs[s]->L[p.layers].seed_index = p.layers;
        if (n[s]) left.push_back(s);
    }
    const int wfb = (int)(p.layers & 1);
    while (!left.empty()) {
        BatchTables T;
        int rc = batch_tables(p, r, offsets, n, left, p.layers, &attempt, T);
        if (rc) return rc;
        if ((rc = ensure(T))) return rc;
        BatchView v;
        if ((rc = view(T, v))) return rc;
        const int set = (int)(p.layers % kBandSets);
        if ((rc = ensure_band(set, T.slots))) return rc;
        CK(side.reuse(set), "order");
        void *cg = cgs[set], *yg = ygs[set];
        uint64_t *z;
        CK(table_alloc(T.zw * 8, &z), "alloc tables");
        CK(cudaMemsetAsync(ctr, 0, (size_t)S * 12 + 64, st), "clear counters");
        CK(launch_sort_batch(v, vb, cur_k, cur_v, (uint64_t *)sk, sv, (uint32_t *)bst, scratch, st), "sort");
        CK(launch_band(none, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cg, yg, nullptr, nullptr,
                       (uint64_t *)bk[wfb], bv2[wfb], bcount, err, st, &v), "band");
        CK(launch_backsub(none, vb, (const uint64_t *)cg, yg, z, st, &v), "backsub");
        for (auto *h : hs) h->launches += 6;
        std::vector<uint32_t> f(left.size());
        uint32_t e = 0;
        CK(cudaMemcpyAsync(f.data(), ffail, f.size() * 4, cudaMemcpyDeviceToHost, st), "read flags");
        CK(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, st), "read error word");
        CK(cudaStreamSynchronize(st), "base case");
        if (e) return fail(BURR_ERR_INTERNAL, "base case: device error 0x%x", e);
        std::vector<uint32_t> again;
        for (uint32_t i = 0; i < left.size(); ++i) {
            const uint32_t s = left[i];
            const StructDesc &D = T.sd[i];
            if (f[i] & kErrUnsolvable) {
                if (++attempt[s] > p.fallback_max_retries)
                    return fail(BURR_ERR_UNSOLVABLE, "structure %u: base case unsolved after %u retries", s,
                                p.fallback_max_retries);
                again.push_back(s);
                continue;
            }
            LayerStore &F = hs[s]->L[p.layers];
            F.m = D.L.m;
            F.nb = D.L.nb;
            F.K = 1;
            F.sigma = D.L.sigma;
            F.seed_index = p.layers + attempt[s];
            F.z = z + D.z_base;
            hs[s]->fb_attempt = attempt[s];
        }
        left.swap(again);
    }
    CK(side.order(side.side, st, kJoinSlot), "order");
    const int t_end = tm.mark();
    CK(cudaStreamSynchronize(st), "build");
    const float total = tm.ms(t_begin, t_end);
    for (auto *h : hs) {
        h->total_ms = total;
        for (uint32_t l = 0; l < p.layers; ++l)
            if (h->L[l].n)
                h->stage_ms[l][2] = tm.ms(bsm[l][0], bsm[l][1]) + tm.ms(bsm[l][2], bsm[l][3]);
    }
    return BURR_OK;
}

}  // namespace

extern "C" {

int burr_default_params(burr_params *p) {
    if (!p) return fail(BURR_ERR_INVALID, "params pointer is NULL");
    memset(p, 0, sizeof(*p));
    p->ribbon_width = 64;
    p->bucket_slots = 128;
    p->threshold_mode = BURR_THRESH_2BIT;
    p->layers = 4;
    p->levels[0] = 0;
    p->levels[1] = 32;
    p->levels[2] = 64;
    p->levels[3] = 128;
    p->load_factor = 1.015;
    p->partition_slots = 65536;
    p->min_partition_slots = 4096;
    p->lower_partition_slots = 4096;
    p->cut_search = BURR_CUT_NONE;
    p->cut_search_range = 50;
    p->seed = 0x5EED5EED5EED5EEDull;
    p->fallback_slack = 0.1;
    p->fallback_max_retries = 16;
    p->flags = 0;
    return BURR_OK;
}

int burr_build(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *pin,
               void *stream, burr_handle **out) {
    if (!out) return fail(BURR_ERR_INVALID, "out is NULL");
    *out = nullptr;
    burr_params p;
    if (pin) p = *pin;
    else burr_default_params(&p);
    int rc = validate(p, r);
    if (rc) return rc;
    if (n > 0 && (!keys || !values)) return fail(BURR_ERR_INVALID, "keys/values are NULL");
    if (n >= (1ull << 32)) return fail(BURR_ERR_INVALID, "n >= 2^32");
    burr_handle *h = new (std::nothrow) burr_handle();
    if (!h) return fail(BURR_ERR_OOM, "host allocation");
    h->p = p;
    h->r = r;
    h->vbytes = value_bytes(r);
    h->n = n;
    for (uint32_t l = 0; l <= p.layers; ++l) h->L[l].seed_index = l;
    if (n > 0) {
        rc = build_impl(keys, values, n, r, p, (cudaStream_t)stream, h);
        if (rc) {
            cudaStreamSynchronize((cudaStream_t)stream);
            free_layers(h);
            delete h;
            return rc;
        }
    }
    *out = h;
    return BURR_OK;
}

int burr_build_batch(const uint64_t *keys, const void *values, const uint64_t *offsets, const uint32_t *r,
                     uint32_t count, const burr_params *pin, void *stream, burr_handle **out) {
    if (!out || !offsets || !r || count == 0) return fail(BURR_ERR_INVALID, "NULL argument or empty batch");
    for (uint32_t s = 0; s < count; ++s) out[s] = nullptr;
    burr_params p;
    if (pin) p = *pin;
    else burr_default_params(&p);
    if (p.bucket_slots != 128) return fail(BURR_ERR_INVALID, "batched builds use bucket_slots = 128");
    std::vector<uint64_t> offs(offsets, offsets + count + 1);
    std::vector<uint32_t> rs(r, r + count);
    if (offs[0] != 0) return fail(BURR_ERR_INVALID, "offsets[0] must be 0");
    std::vector<uint64_t> n(count);
    for (uint32_t s = 0; s < count; ++s) {
        if (offs[s + 1] < offs[s]) return fail(BURR_ERR_INVALID, "offsets must not decrease");
        n[s] = offs[s + 1] - offs[s];
    }
    if (offs[count] >= (1ull << 32)) return fail(BURR_ERR_INVALID, "total keys >= 2^32");
    if (offs[count] > 0 && (!keys || !values)) return fail(BURR_ERR_INVALID, "keys/values are NULL");
    if (p.partition_slots == 0) {
        p.partition_slots = autotune_partition_slots(n, p.load_factor > 0 ? p.load_factor : 1.0);
        p.min_partition_slots = p.partition_slots;
    }
    for (uint32_t s = 0; s < count; ++s) {
        const int rc = validate(p, rs[s]);
        if (rc) return rc;
    }
    auto store = std::make_shared<BatchStorage>();
    std::vector<burr_handle *> hs(count);
    for (uint32_t s = 0; s < count; ++s) {
        hs[s] = new (std::nothrow) burr_handle();
        if (!hs[s]) {
            for (uint32_t q = 0; q < s; ++q) delete hs[q];
            return fail(BURR_ERR_OOM, "host allocation");
        }
        hs[s]->p = p;
        hs[s]->r = rs[s];
        hs[s]->vbytes = value_bytes(rs[s]);
        hs[s]->n = n[s];
        hs[s]->shared = store;
        for (uint32_t l = 0; l <= p.layers; ++l) hs[s]->L[l].seed_index = l;
    }
    int rc = BURR_OK;
    if (offs[count] > 0) {
        // values are passed in the value type of the widest r; per-structure
        // value types apply to queries (the handle's r)
        rc = build_batch_impl(keys, values, offs, rs, p, (cudaStream_t)stream, hs, store);
    }
    if (rc) {
        cudaStreamSynchronize((cudaStream_t)stream);
        for (auto *h : hs) delete h;
        return rc;
    }
    for (uint32_t s = 0; s < count; ++s) out[s] = hs[s];
    return BURR_OK;
}

int burr_query(const burr_handle *h, const uint64_t *keys, void *out, uint64_t n, void *stream) {
    TraceRange trace("burr_query");
    if (!h) return fail(BURR_ERR_INVALID, "handle is NULL");
    if (n == 0) return BURR_OK;
    if (!keys || !out) return fail(BURR_ERR_INVALID, "keys/out are NULL");
    cudaStream_t st = (cudaStream_t)stream;
    QueryDesc Q;
    memset(&Q, 0, sizeof(Q));
    Q.r = h->r;
    Q.B = h->p.bucket_slots;
    Q.layers = h->p.layers;
    Q.mode = h->p.threshold_mode;
    for (int i = 0; i < 4; ++i) Q.levels[i] = h->p.levels[i];
    for (uint32_t l = 0; l <= h->p.layers; ++l) {
        Q.m[l] = h->L[l].m;
        Q.sigma[l] = layer_seed(h->p.seed, h->L[l].seed_index);
        if (l < h->p.layers) {
            Q.thresh[l] = h->L[l].thresh;
            Q.flags[l] = h->L[l].flags;
            Q.dir[l] = h->L[l].dir;
            Q.tbytes[l] = h->L[l].tbytes;
        }
        Q.z[l] = h->L[l].z;
    }
    const uint32_t vb = h->vbytes;
    const bool dk = is_device_ptr(keys), dout = is_device_ptr(out);
    if (dk && dout) {
        CK(launch_query(Q, vb, keys, out, n, st), "query");
        return BURR_OK;
    }
    keep_pool_memory();
    Arena ar(st);
    constexpr uint64_t kChunk = 1ull << 22;   // keys per pipelined chunk
    if (n <= 2 * kChunk) {
        const uint64_t *k = keys;
        void *o = out;
        if (!dk) {
            void *d;
            CK(ar.alloc(&d, n * 8), "alloc query keys");
            CK(cudaMemcpyAsync(d, keys, n * 8, cudaMemcpyHostToDevice, st), "copy query keys");
            k = (const uint64_t *)d;
        }
        if (!dout) CK(ar.alloc(&o, n * vb), "alloc query output");
        CK(launch_query(Q, vb, k, o, n, st), "query");
        if (!dout) CK(cudaMemcpyAsync(out, o, n * vb, cudaMemcpyDeviceToHost, st), "copy query output");
        CK(cudaStreamSynchronize(st), "query");
        return BURR_OK;
    }
    // Large batches through host memory: chunks alternate between two streams,
    // so the copies of one chunk overlap the query kernel of the other (with
    // page-locked host memory; pageable copies are staged by the driver).
    SideStream side(st);
    CK(side.init(), "query stream");
    void *kb[2] = {nullptr, nullptr}, *ob[2] = {nullptr, nullptr};
    for (int i = 0; i < 2; ++i) {
        if (!dk) CK(ar.alloc(&kb[i], kChunk * 8), "alloc query keys");
        if (!dout) CK(ar.alloc(&ob[i], kChunk * vb), "alloc query output");
    }
    CK(side.order(st, side.side, kOrderSlot), "order");   // the second stream starts after the allocations
    for (uint64_t c = 0, i = 0; c < n; c += kChunk, ++i) {
        const uint64_t cnt = std::min(kChunk, n - c);
        const int b = (int)(i & 1);
        cudaStream_t s = b ? side.side : st;
        const uint64_t *k = keys + c;
        void *o = (uint8_t *)out + c * vb;
        if (!dk) {
            CK(cudaMemcpyAsync(kb[b], keys + c, cnt * 8, cudaMemcpyHostToDevice, s), "copy query keys");
            k = (const uint64_t *)kb[b];
        }
        if (!dout) o = ob[b];
        CK(launch_query(Q, vb, k, o, cnt, s), "query");
        if (!dout) CK(cudaMemcpyAsync((uint8_t *)out + c * vb, ob[b], cnt * vb, cudaMemcpyDeviceToHost, s),
                      "copy query output");
    }
    CK(side.order(side.side, st, kJoinSlot), "order");
    CK(cudaStreamSynchronize(st), "query");
    return BURR_OK;
}

int burr_set_allocator(burr_alloc_fn alloc, burr_free_fn free, void *ctx) {
    if ((alloc == nullptr) != (free == nullptr)) return fail(BURR_ERR_INVALID, "alloc and free must both be set or both NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (g_live.load() != 0)
        return fail(BURR_ERR_INVALID, "%lld device blocks of the current allocator are still held",
                    (long long)g_live.load());
    g_hook.alloc = alloc;
    g_hook.free = free;
    g_hook.ctx = alloc ? ctx : nullptr;
    return BURR_OK;
}

int burr_size_bytes(const burr_handle *h, uint64_t *bytes) {
    if (!h || !bytes) return fail(BURR_ERR_INVALID, "NULL argument");
    uint64_t b = 64;
    for (uint32_t l = 0; l <= h->p.layers; ++l) {
        const LayerStore &S = h->L[l];
        if (l < h->p.layers) {
            if (h->p.threshold_mode == BURR_THRESH_1PLUS)
                b += 8 * flag_words(S.nb) + 4 * dir_blocks(S.nb) + S.nflag;
            else
                b += 8 * ((S.nb + 31) / 32);
        }
        b += 8 * (S.m / 64) * h->r;
    }
    *bytes = b;
    return BURR_OK;
}

static uint8_t *put32(uint8_t *q, uint32_t v) {
    memcpy(q, &v, 4);
    return q + 4;
}
static uint8_t *put64(uint8_t *q, uint64_t v) {
    memcpy(q, &v, 8);
    return q + 8;
}

int burr_export(const burr_handle *h, void *host_buf, uint64_t *len) {
    if (!h || !len) return fail(BURR_ERR_INVALID, "NULL argument");
    const burr_params &p = h->p;
    const uint32_t r = h->r;
    const bool onep = p.threshold_mode == BURR_THRESH_1PLUS;
    // threshold section of a bumping layer: 2-bit code words, or (1+-bit) the
    // flag words, the count of flagged buckets and their thresholds as bytes
    // zero-padded to a multiple of 8
    auto tsection = [&](const LayerStore &S) -> uint64_t {
        return onep ? 8 * flag_words(S.nb) + 8 + 8 * ((S.nflag + 7) / 8) : 8 * ((S.nb + 31) / 32);
    };
    uint64_t need = 4 * 10 + 8 * 4 + (uint64_t)p.layers * 8 * 5 + 8 * 4;
    for (uint32_t l = 0; l < p.layers; ++l) need += tsection(h->L[l]) + 8 * (h->L[l].m / 64) * r;
    need += 8 * (h->L[p.layers].m / 64) * r;
    if (!host_buf || *len < need) {
        *len = need;
        return fail(BURR_ERR_INVALID, "export buffer too small (%llu bytes needed)", (unsigned long long)need);
    }
    uint8_t *q = (uint8_t *)host_buf;
    q = put32(q, 0x52525542u);
    q = put32(q, onep ? 2 : 1);
    q = put32(q, r);
    q = put32(q, p.ribbon_width);
    q = put32(q, p.bucket_slots);
    q = put32(q, p.layers);
    for (int i = 0; i < 4; ++i) q = put32(q, p.levels[i]);
    uint64_t abits;
    memcpy(&abits, &p.load_factor, 8);
    q = put64(q, p.seed);
    q = put64(q, abits);
    q = put64(q, h->n);
    q = put64(q, p.partition_slots);
    for (uint32_t l = 0; l < p.layers; ++l) {
        const LayerStore &S = h->L[l];
        q = put64(q, S.n);
        q = put64(q, S.m);
        q = put64(q, S.K);
        q = put64(q, S.nb);
        q = put64(q, S.nbumped);
    }
    const LayerStore &F = h->L[p.layers];
    q = put64(q, F.n);
    q = put64(q, F.m);
    q = put64(q, F.seed_index);
    q = put64(q, h->fb_attempt);
    for (uint32_t l = 0; l < p.layers; ++l) {
        const LayerStore &S = h->L[l];
        const uint64_t tw = (S.nb + 31) / 32, zw = (S.m / 64) * r;
        if (onep) {
            const uint64_t fw = flag_words(S.nb), padded = 8 * ((S.nflag + 7) / 8);
            if (fw) CK(cudaMemcpy(q, S.flags, fw * 8, cudaMemcpyDeviceToHost), "export threshold flags");
            q += fw * 8;
            q = put64(q, S.nflag);
            memset(q, 0, padded);
            if (S.nflag)
                CK(cudaMemcpy(q, S.tbytes + S.tfirst, S.nflag, cudaMemcpyDeviceToHost), "export thresholds");
            q += padded;
        } else {
            if (tw) CK(cudaMemcpy(q, S.thresh, tw * 8, cudaMemcpyDeviceToHost), "export thresholds");
            q += tw * 8;
        }
        if (zw) CK(cudaMemcpy(q, S.z, zw * 8, cudaMemcpyDeviceToHost), "export table");
        q += zw * 8;
    }
    const uint64_t zw = (F.m / 64) * r;
    if (zw) CK(cudaMemcpy(q, F.z, zw * 8, cudaMemcpyDeviceToHost), "export base case");
    q += zw * 8;
    *len = (uint64_t)(q - (uint8_t *)host_buf);
    return BURR_OK;
}

int burr_stats(const burr_handle *h, burr_stats_t *st) {
    if (!h || !st) return fail(BURR_ERR_INVALID, "NULL argument");
    memset(st, 0, sizeof(*st));
    st->n = h->n;
    st->r = h->r;
    st->layers = h->p.layers;
    for (uint32_t l = 0; l <= h->p.layers; ++l) {
        st->layer_n[l] = h->L[l].n;
        st->layer_m[l] = h->L[l].m;
        st->layer_parts[l] = h->L[l].K;
        st->layer_bumped[l] = h->L[l].nbumped;
        for (int s = 0; s < 3; ++s) st->stage_ms[l][s] = h->stage_ms[l][s];
    }
    st->fallback_attempt = h->fb_attempt;
    st->total_ms = h->total_ms;
    uint64_t b = 0;
    burr_size_bytes(h, &b);
    st->table_bytes = b;
    st->kernel_launches = h->launches;
    return BURR_OK;
}

namespace {

// Little-endian reader over the export buffer that refuses to run past its end.
struct Reader {
    const uint8_t *p, *end;
    bool ok = true;
    uint32_t u32() {
        uint32_t v = 0;
        if (end - p < 4) ok = false;
        else memcpy(&v, p, 4), p += 4;
        return v;
    }
    uint64_t u64() {
        uint64_t v = 0;
        if (end - p < 8) ok = false;
        else memcpy(&v, p, 8), p += 8;
        return v;
    }
    const uint8_t *bytes(uint64_t n) {
        if ((uint64_t)(end - p) < n) {
            ok = false;
            return nullptr;
        }
        const uint8_t *q = p;
        p += n;
        return q;
    }
};

int upload_table(void **d, const void *src, uint64_t bytes, cudaStream_t st) {
    CK(dev_alloc(d, std::max<uint64_t>(bytes, 8), st), "alloc imported table");
    if (bytes) CK(cudaMemcpyAsync(*d, src, bytes, cudaMemcpyHostToDevice, st), "copy imported table");
    return BURR_OK;
}

// Parse and check an export; with h == nullptr only the checks run.
int import_into(const uint8_t *buf, uint64_t len, cudaStream_t st, burr_handle *h) {
    Reader R{buf, buf + len};
    if (R.u32() != 0x52525542u) return fail(BURR_ERR_INVALID, "not a BuRR export (magic)");
    const uint32_t version = R.u32();
    if (version != 1 && version != 2) return fail(BURR_ERR_INVALID, "unknown export version %u", version);
    burr_params p;
    burr_default_params(&p);
    const uint32_t r = R.u32();
    p.ribbon_width = R.u32();
    p.bucket_slots = R.u32();
    p.layers = R.u32();
    for (int i = 0; i < 4; ++i) p.levels[i] = R.u32();
    p.seed = R.u64();
    const uint64_t abits = R.u64();
    memcpy(&p.load_factor, &abits, 8);
    const uint64_t n = R.u64();
    p.partition_slots = R.u64();
    p.threshold_mode = version == 2 ? BURR_THRESH_1PLUS : BURR_THRESH_2BIT;
    if (!R.ok) return fail(BURR_ERR_INVALID, "export header truncated");
    if (p.layers > BURR_MAX_LAYERS) return fail(BURR_ERR_INVALID, "export has %u layers", p.layers);
    if (int rc = validate(p, r)) return rc;
    uint64_t ln[BURR_MAX_LAYERS + 1], lm[BURR_MAX_LAYERS + 1], lk[BURR_MAX_LAYERS + 1], lb[BURR_MAX_LAYERS + 1],
        lbump[BURR_MAX_LAYERS + 1];
    for (uint32_t l = 0; l < p.layers; ++l) {
        ln[l] = R.u64();
        lm[l] = R.u64();
        lk[l] = R.u64();
        lb[l] = R.u64();
        lbump[l] = R.u64();
    }
    const uint64_t fn = R.u64(), fm = R.u64(), fseed = R.u64(), fatt = R.u64();
    if (!R.ok) return fail(BURR_ERR_INVALID, "export layer table truncated");
    uint64_t cur = n;
    for (uint32_t l = 0; l < p.layers; ++l) {
        if (ln[l] != cur || lm[l] % 64 || lm[l] >= (1ull << 32) || lb[l] != num_buckets(lm[l], p.bucket_slots) ||
            lbump[l] > ln[l] || (ln[l] == 0) != (lm[l] == 0) ||
            // partitions: none in an empty layer, otherwise at least one and at
            // most one per bucket (each partition starts at its own bucket)
            (lm[l] == 0 ? lk[l] != 0 : (lk[l] == 0 || lk[l] > lb[l])))
            return fail(BURR_ERR_INVALID, "export layer %u sizes are inconsistent", l);
        cur = lbump[l];
    }
    if (fn != cur || fm % 64 || fm >= (1ull << 32) || (fn == 0) != (fm == 0) || fseed != p.layers + fatt)
        return fail(BURR_ERR_INVALID, "export base-case sizes are inconsistent");
    if (h) {
        h->p = p;
        h->r = r;
        h->vbytes = value_bytes(r);
        h->n = n;
        h->fb_attempt = (uint32_t)fatt;
    }
    for (uint32_t l = 0; l < p.layers; ++l) {
        LayerStore *S = h ? &h->L[l] : nullptr;
        const uint64_t nb = lb[l];
        if (S) {
            S->n = ln[l];
            S->m = lm[l];
            S->nb = nb;
            S->K = lk[l];
            S->nbumped = lbump[l];
            S->seed_index = l;
            S->sigma = layer_seed(p.seed, l);
        }
        if (version == 2) {
            const uint64_t fw = flag_words(nb), nd = dir_blocks(nb);
            const uint8_t *fl = R.bytes(fw * 8);
            const uint64_t cnt = R.u64();
            const uint8_t *tb = R.bytes(8 * ((cnt + 7) / 8));
            if (!R.ok) return fail(BURR_ERR_INVALID, "export thresholds of layer %u truncated", l);
            // the rank directory is derived: flagged buckets before each 512-bucket block
            std::vector<uint64_t> words(fw);
            if (fw) memcpy(words.data(), fl, fw * 8);
            std::vector<uint32_t> dir(nd + 1, 0);
            uint64_t run = 0;
            for (uint64_t w = 0; w < fw; ++w) {
                if (w % 8 == 0) dir[w / 8] = (uint32_t)run;
                run += (uint64_t)__builtin_popcountll(words[w]);
            }
            dir[nd] = (uint32_t)run;
            if (run != cnt) return fail(BURR_ERR_INVALID, "export layer %u: %llu flags, %llu thresholds", l,
                                        (unsigned long long)run, (unsigned long long)cnt);
            if (fw && (nb % 64) && (words[fw - 1] >> (nb % 64)))
                return fail(BURR_ERR_INVALID, "export layer %u flags past the last bucket", l);
            for (uint64_t i = 0; i < cnt; ++i)
                if (tb[i] == 0 || tb[i] > p.bucket_slots)
                    return fail(BURR_ERR_INVALID, "export layer %u: threshold out of range", l);
            if (S) {
                if (int rc = upload_table((void **)&S->flags, words.data(), fw * 8, st)) return rc;
                if (int rc = upload_table((void **)&S->dir, dir.data(), (nd + 1) * 4, st)) return rc;
                if (int rc = upload_table((void **)&S->tbytes, tb, cnt, st)) return rc;
                S->nflag = cnt;
                S->tfirst = 0;
            }
        } else {
            const uint64_t tw = (nb + 31) / 32;
            const uint8_t *th = R.bytes(tw * 8);
            if (!R.ok) return fail(BURR_ERR_INVALID, "export thresholds of layer %u truncated", l);
            if (S)
                if (int rc = upload_table((void **)&S->thresh, th, tw * 8, st)) return rc;
        }
        const uint64_t zw = (lm[l] / 64) * r;
        const uint8_t *z = R.bytes(zw * 8);
        if (!R.ok) return fail(BURR_ERR_INVALID, "export table of layer %u truncated", l);
        if (S)
            if (int rc = upload_table((void **)&S->z, z, zw * 8, st)) return rc;
    }
    const uint64_t zw = (fm / 64) * r;
    const uint8_t *z = R.bytes(zw * 8);
    if (!R.ok) return fail(BURR_ERR_INVALID, "export base-case table truncated");
    if (R.p != R.end) return fail(BURR_ERR_INVALID, "export has %llu trailing bytes", (unsigned long long)(R.end - R.p));
    if (h) {
        LayerStore &F = h->L[p.layers];
        F.n = fn;
        F.m = fm;
        F.nb = num_buckets(fm, p.bucket_slots);
        F.K = fm ? 1 : 0;
        F.seed_index = fseed;
        F.sigma = layer_seed(p.seed, fseed);
        if (int rc = upload_table((void **)&F.z, z, zw * 8, st)) return rc;
    }
    return BURR_OK;
}

}  // namespace

int burr_import(const void *host_buf, uint64_t len, void *stream, burr_handle **out) {
    if (!host_buf || !out) return fail(BURR_ERR_INVALID, "NULL argument");
    *out = nullptr;
    // every check runs before anything is allocated
    if (int rc = import_into((const uint8_t *)host_buf, len, nullptr, nullptr)) return rc;
    auto *h = new (std::nothrow) burr_handle();
    if (!h) return fail(BURR_ERR_OOM, "host allocation");
    cudaStream_t st = (cudaStream_t)stream;
    TraceRange trace("burr_import");
    keep_pool_memory();
    int rc = import_into((const uint8_t *)host_buf, len, st, h);
    if (rc == BURR_OK) rc = cudaStreamSynchronize(st) == cudaSuccess ? BURR_OK : fail(BURR_ERR_CUDA, "import");
    if (rc) {
        free_layers(h);
        delete h;
        return rc;
    }
    *out = h;
    return BURR_OK;
}

void burr_free(burr_handle *h) {
    if (!h) return;
    free_layers(h);
    delete h;
}

void burr_free_many(burr_handle *const *handles, uint64_t count) {
    if (!handles) return;
    for (uint64_t i = 0; i < count; ++i) burr_free(handles[i]);
}

const char *burr_strerror(int code) {
    switch (code) {
    case BURR_OK: return "ok";
    case BURR_ERR_INVALID: return "invalid argument";
    case BURR_ERR_OOM: return "out of device memory";
    case BURR_ERR_UNSOLVABLE: return "unsolvable (base case retries exhausted)";
    case BURR_ERR_TIMEOUT: return "device wait timed out";
    case BURR_ERR_CUDA: return "CUDA error";
    case BURR_ERR_INTERNAL: return "internal capacity check failed";
    default: return "unknown error";
    }
}

const char *burr_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// Sharded construction (Sec. 3): the ranks of a build own contiguous ranges of
// each layer's partitions.  A key goes to the rank that owns its start bucket
// (burr_shard_route), each rank inserts and back-substitutes its partitions
// alone (burr_shard_build_layer), the bumped keys are routed again for the
// next layer, and one rank builds the base case (burr_shard_build_base).
// ---------------------------------------------------------------------------
namespace {

// The layer that n_layer keys (all ranks) form as bumping layer `layer`: the
// sizing, partition and seed rules of build_impl.
LayerDesc shard_layer_desc(const burr_params &p, uint32_t r, uint64_t n_layer, uint32_t layer) {
    const uint64_t m = layer_slots(n_layer, p.load_factor);
    const uint64_t P = layer_partition_slots(p, layer);
    return make_desc(p, r, n_layer, m, layer_seed(p.seed, layer), num_partitions(m, P, p.min_partition_slots), false,
                     P);
}

int shard_params(const burr_params *pin, uint32_t r, burr_params &p) {
    if (pin) p = *pin;
    else burr_default_params(&p);
    if (int rc = validate(p, r)) return rc;
    if (p.threshold_mode != BURR_THRESH_2BIT)
        return fail(BURR_ERR_INVALID, "sharded builds support 2-bit thresholds only");
    if (p.cut_search != BURR_CUT_NONE)
        return fail(BURR_ERR_INVALID, "sharded builds place cut j at j*P (no cut search)");
    return BURR_OK;
}

int shard_layer_args(const burr_params &p, uint32_t r, uint32_t layer, uint64_t n, uint64_t n_layer, LayerDesc &L) {
    if (layer >= p.layers) return fail(BURR_ERR_INVALID, "layer %u is not a bumping layer (layers = %u)", layer, p.layers);
    if (n > n_layer) return fail(BURR_ERR_INVALID, "n = %llu exceeds the layer's n_layer", (unsigned long long)n);
    if (n_layer >= (1ull << 32)) return fail(BURR_ERR_INVALID, "n_layer >= 2^32");
    L = shard_layer_desc(p, r, n_layer, layer);
    if (L.m >= (1ull << 32)) return fail(BURR_ERR_INVALID, "layer needs >= 2^32 slots");
    L.n = n;
    return BURR_OK;
}

}  // namespace

extern "C" {

int burr_layer_geometry(uint64_t n_layer, uint32_t layer, const burr_params *pin, burr_layer_geometry_t *out) {
    if (!out) return fail(BURR_ERR_INVALID, "out is NULL");
    burr_params p;
    if (int rc = shard_params(pin, 1, p)) return rc;
    LayerDesc L;
    if (int rc = shard_layer_args(p, 1, layer, 0, n_layer, L)) return rc;
    out->n = n_layer;
    out->m = L.m;
    out->buckets = L.nb;
    out->partitions = L.K;
    out->partition_slots = L.P;
    out->seed_index = layer;
    return BURR_OK;
}

int burr_shard_route(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *pin,
                     uint32_t layer, uint64_t n_layer, uint32_t ranks, const uint32_t *part_first, uint64_t *keys_out,
                     void *values_out, uint64_t *counts, void *stream) {
    burr_params p;
    if (int rc = shard_params(pin, r, p)) return rc;
    LayerDesc L;
    if (int rc = shard_layer_args(p, r, layer, n, n_layer, L)) return rc;
    if (!part_first || !counts) return fail(BURR_ERR_INVALID, "part_first/counts are NULL");
    if (ranks == 0 || ranks > kMaxShardRanks) return fail(BURR_ERR_INVALID, "ranks must be in [1, %u]", kMaxShardRanks);
    if (part_first[0] != 0 || part_first[ranks] != L.K)
        return fail(BURR_ERR_INVALID, "part_first must run from 0 to the layer's %llu partitions",
                    (unsigned long long)L.K);
    for (uint32_t g = 0; g < ranks; ++g)
        if (part_first[g] > part_first[g + 1]) return fail(BURR_ERR_INVALID, "part_first must not decrease");
    for (uint32_t g = 0; g < ranks; ++g) counts[g] = 0;
    if (n == 0) return BURR_OK;
    if (!keys || !values || !keys_out || !values_out) return fail(BURR_ERR_INVALID, "NULL key/value pointer");
    if (!is_device_ptr(keys) || !is_device_ptr(values) || !is_device_ptr(keys_out) || !is_device_ptr(values_out))
        return fail(BURR_ERR_INVALID, "burr_shard_route takes device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t vb = value_bytes(r);
    keep_pool_memory();
    Arena ar(st);
    uint32_t *d_pf, *rank_of;
    unsigned long long *d_counts, *d_cursor;
    CK(ar.alloc((void **)&d_pf, (ranks + 1) * 4ull), "alloc partition ranges");
    CK(ar.alloc((void **)&rank_of, n * 4), "alloc owners");
    CK(ar.alloc((void **)&d_counts, ranks * 8ull), "alloc counts");
    CK(ar.alloc((void **)&d_cursor, ranks * 8ull), "alloc cursors");
    CK(cudaMemcpyAsync(d_pf, part_first, (ranks + 1) * 4ull, cudaMemcpyHostToDevice, st), "copy partition ranges");
    CK(cudaMemsetAsync(d_counts, 0, ranks * 8ull, st), "clear counts");
    CK(launch_route(L, vb, keys, values, d_pf, ranks, rank_of, d_counts, nullptr, nullptr, nullptr, true, st), "route");
    std::vector<unsigned long long> hc(ranks), cur(ranks);
    CK(cudaMemcpyAsync(hc.data(), d_counts, ranks * 8ull, cudaMemcpyDeviceToHost, st), "read counts");
    CK(cudaStreamSynchronize(st), "route counts");
    unsigned long long run = 0;
    for (uint32_t g = 0; g < ranks; ++g) {
        cur[g] = run;
        run += hc[g];
        counts[g] = hc[g];
    }
    CK(cudaMemcpyAsync(d_cursor, cur.data(), ranks * 8ull, cudaMemcpyHostToDevice, st), "copy cursors");
    CK(launch_route(L, vb, keys, values, d_pf, ranks, rank_of, nullptr, d_cursor, keys_out, values_out, false, st),
       "route");
    CK(cudaStreamSynchronize(st), "route");
    return BURR_OK;
}

int burr_shard_build_layer(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *pin,
                           uint32_t layer, uint64_t n_layer, uint32_t part_lo, uint32_t part_hi, uint64_t *thresh,
                           uint64_t *z, uint64_t *bumped_keys, void *bumped_values, uint64_t *nbumped, void *stream) {
    burr_params p;
    if (int rc = shard_params(pin, r, p)) return rc;
    LayerDesc L;
    if (int rc = shard_layer_args(p, r, layer, n, n_layer, L)) return rc;
    if (!nbumped) return fail(BURR_ERR_INVALID, "nbumped is NULL");
    *nbumped = 0;
    if (part_lo > part_hi || part_hi > L.K) return fail(BURR_ERR_INVALID, "partition range outside [0, K]");
    if (n_layer == 0) return BURR_OK;
    if (!thresh || !z || (n && (!keys || !values || !bumped_keys || !bumped_values)))
        return fail(BURR_ERR_INVALID, "NULL pointer");
    if (!is_device_ptr(thresh) || !is_device_ptr(z) ||
        (n && (!is_device_ptr(keys) || !is_device_ptr(values) || !is_device_ptr(bumped_keys) ||
               !is_device_ptr(bumped_values))))
        return fail(BURR_ERR_INVALID, "burr_shard_build_layer takes device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t vb = value_bytes(r);
    CK(cudaMemsetAsync(thresh, 0, ((L.nb + 31) / 32) * 8, st), "clear thresholds");
    CK(cudaMemsetAsync(z, 0, (L.m / 64) * r * 8, st), "clear table");
    if (part_lo == part_hi) return BURR_OK;
    L.part_lo = part_lo;
    L.part_hi = part_hi;
    keep_pool_memory();
    Arena ar(st);
    void *sk, *sv, *bst, *ss, *cg, *yg, *ctr;
    CK(ar.alloc(&sk, std::max<uint64_t>(n, 1) * 8), "alloc sorted keys");
    CK(ar.alloc(&sv, std::max<uint64_t>(n, 1) * vb), "alloc sorted values");
    CK(ar.alloc(&bst, (L.nb + 1) * 4), "alloc bucket offsets");
    CK(ar.alloc(&ss, sort_scratch_bytes(n, L.m, vb)), "alloc sort scratch");
    CK(ar.alloc(&cg, L.m * 8), "alloc band");
    CK(ar.alloc(&yg, L.m * vb), "alloc band values");
    CK(ar.alloc(&ctr, 64), "alloc counters");
    CK(cudaMemsetAsync(ctr, 0, 64, st), "clear counters");
    unsigned long long *bcount = (unsigned long long *)ctr;
    uint32_t *err = (uint32_t *)((char *)ctr + 8);
    CK(launch_sort(L, vb, keys, values, (uint64_t *)sk, sv, (uint32_t *)bst, ss, err, st), "sort");
    CK(launch_band(L, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cg, yg, thresh, nullptr,
                   bumped_keys, bumped_values, bcount, err, st),
       "band");
    CK(launch_backsub(L, vb, (const uint64_t *)cg, yg, z, st), "backsub");
    unsigned long long hc[2] = {0, 0};
    CK(cudaMemcpyAsync(hc, ctr, 16, cudaMemcpyDeviceToHost, st), "read counters");
    CK(cudaStreamSynchronize(st), "shard layer");
    const uint32_t e = (uint32_t)(hc[1] & 0xffffffffu);
    if (e & kErrRingOverflow) return fail(BURR_ERR_INTERNAL, "layer %u: pivot left the band's window", layer);
    if (e) return fail(BURR_ERR_INTERNAL, "layer %u: device error 0x%x", layer, e);
    *nbumped = hc[0];
    return BURR_OK;
}

int burr_shard_build_base(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *pin,
                          uint64_t *z, uint64_t z_words, uint64_t *m_out, uint64_t *seed_index_out,
                          uint32_t *attempt_out, void *stream) {
    burr_params p;
    if (int rc = shard_params(pin, r, p)) return rc;
    if (!m_out || !seed_index_out || !attempt_out) return fail(BURR_ERR_INVALID, "NULL output");
    *m_out = 0;
    *seed_index_out = p.layers;
    *attempt_out = 0;
    if (n == 0) return BURR_OK;
    if (n >= (1ull << 32)) return fail(BURR_ERR_INVALID, "n >= 2^32");
    const uint64_t need = (fallback_slots(n, p.fallback_slack, p.fallback_max_retries) / 64) * r;
    if (!z || z_words < need) {
        *m_out = fallback_slots(n, p.fallback_slack, p.fallback_max_retries);
        return fail(BURR_ERR_INVALID, "z holds %llu words; the base case may need %llu", (unsigned long long)z_words,
                    (unsigned long long)need);
    }
    if (!keys || !values || !is_device_ptr(keys) || !is_device_ptr(values) || !is_device_ptr(z))
        return fail(BURR_ERR_INVALID, "burr_shard_build_base takes device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t vb = value_bytes(r);
    keep_pool_memory();
    Arena ar(st);
    const uint64_t mmax = fallback_slots(n, p.fallback_slack, p.fallback_max_retries);
    void *sk, *sv, *bst, *ss, *cg, *yg, *ctr;
    CK(ar.alloc(&sk, n * 8), "alloc sorted keys");
    CK(ar.alloc(&sv, n * vb), "alloc sorted values");
    CK(ar.alloc(&bst, (num_buckets(mmax, p.bucket_slots) + 1) * 4), "alloc bucket offsets");
    CK(ar.alloc(&ss, sort_scratch_bytes(n, mmax, vb)), "alloc sort scratch");
    CK(ar.alloc(&cg, mmax * 8), "alloc band");
    CK(ar.alloc(&yg, mmax * vb), "alloc band values");
    CK(ar.alloc(&ctr, 64), "alloc counters");
    uint32_t *err = (uint32_t *)((char *)ctr + 8);
    for (uint32_t a = 0; a <= p.fallback_max_retries; ++a) {
        const uint64_t m = fallback_slots(n, p.fallback_slack, a);
        const LayerDesc L = make_desc(p, r, n, m, layer_seed(p.seed, p.layers + a), 1, true, m);
        CK(cudaMemsetAsync(ctr, 0, 64, st), "clear counters");
        CK(launch_sort(L, vb, keys, values, (uint64_t *)sk, sv, (uint32_t *)bst, ss, err, st), "sort");
        CK(launch_band(L, vb, (const uint64_t *)sk, sv, (const uint32_t *)bst, (uint64_t *)cg, yg, nullptr, nullptr,
                       nullptr, nullptr, (unsigned long long *)ctr, err, st),
           "band");
        uint32_t he = 0;
        CK(cudaMemcpyAsync(&he, err, 4, cudaMemcpyDeviceToHost, st), "read error word");
        CK(cudaStreamSynchronize(st), "base case");
        if (he & ~kErrUnsolvable) return fail(BURR_ERR_INTERNAL, "base case: device error 0x%x", he);
        if (he & kErrUnsolvable) continue;
        CK(cudaMemsetAsync(z, 0, z_words * 8, st), "clear table");
        CK(launch_backsub(L, vb, (const uint64_t *)cg, yg, z, st), "backsub");
        CK(cudaStreamSynchronize(st), "base case");
        *m_out = m;
        *seed_index_out = p.layers + a;
        *attempt_out = a;
        return BURR_OK;
    }
    return fail(BURR_ERR_UNSOLVABLE, "base case unsolved after %u retries (duplicate keys?)", p.fallback_max_retries);
}

int burr_stage_hash(const uint64_t *d_keys, uint64_t n, uint64_t seed, uint32_t layer_index, uint64_t m,
                    uint32_t *d_start, uint64_t *d_coeff, void *stream) {
    if (m < kW || m % 64 || m >= (1ull << 32)) return fail(BURR_ERR_INVALID, "m must be a multiple of 64 in [64, 2^32)");
    if (n && (!d_keys || !d_start || !d_coeff)) return fail(BURR_ERR_INVALID, "NULL argument");
    CK(launch_hash(d_keys, n, layer_seed(seed, layer_index), m - kW + 1, d_start, d_coeff,
                   (cudaStream_t)stream), "hash");
    return BURR_OK;
}

int burr_stage_sort(const uint64_t *d_keys, const void *d_values, uint64_t n, uint32_t r, uint64_t seed,
                    uint32_t layer_index, uint64_t m, uint64_t *d_sorted_keys, void *d_sorted_values,
                    uint32_t *d_bucket_start, void *stream) {
    if (r < 1 || r > 32) return fail(BURR_ERR_INVALID, "r outside [1,32]");
    if (m < kW || m % 64 || m >= (1ull << 32)) return fail(BURR_ERR_INVALID, "m must be a multiple of 64 in [64, 2^32)");
    if (n >= (1ull << 32)) return fail(BURR_ERR_INVALID, "n >= 2^32");
    burr_params p;
    burr_default_params(&p);
    cudaStream_t st = (cudaStream_t)stream;
    const LayerDesc L = make_desc(p, r, n, m, layer_seed(seed, layer_index), 1, false, p.partition_slots);
    const uint32_t vb = value_bytes(r);
    keep_pool_memory();
    Arena ar(st);
    void *ss;
    CK(ar.alloc(&ss, sort_scratch_bytes(n, m, vb)), "alloc sort scratch");
    CK(launch_sort(L, vb, d_keys, d_values, d_sorted_keys, d_sorted_values, d_bucket_start, ss, nullptr, st, true),
       "sort");
    return BURR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Kernel attributes set once per (kernel, device, attribute, value).
// ---------------------------------------------------------------------------
namespace {
std::mutex g_attr_mu;
std::set<std::tuple<const void *, int, int, int>> g_attr_set;   // kernel, device, attribute, value
}  // namespace

bool burr::attr_is_set(const void *kernel, int attr, int value) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    return g_attr_set.count(std::make_tuple(kernel, dev, attr, value)) != 0;
}

void burr::attr_mark_set(const void *kernel, int attr, int value) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    g_attr_set.insert(std::make_tuple(kernel, dev, attr, value));
}
