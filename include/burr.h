/*
 * burr.h -- C ABI of libburr.so: GB300 (sm_103a) construction and query of
 * Bumped Ribbon Retrieval (BuRR) with partitioned parallel construction.
 *
 * The problem (Sec. 1 and the abstract of "Brief Announcement: Parallel
 * Construction of Bumped Ribbon Retrieval"): store a static function
 * f: S -> {0,1}^r for a set S of 64-bit keys so that a query of x in S returns
 * f(x); a query of x outside S returns an arbitrary (here: deterministic)
 * r-bit value.  The structure does not store S.
 *
 * Method (Sec. 2 and 3):
 *   - each key is one GF(2) equation: a 64-bit coefficient row starting at a
 *     hashed start slot of a layer of m slots (ribbon width w = 64);
 *   - equations are sorted by start slot and eliminated bucket by bucket
 *     (128 start slots per bucket); where elimination fails, a prefix of the
 *     bucket is bumped to the next layer and the bucket's 2-bit threshold
 *     (one of four levels) records it;
 *   - each layer is cut into independent partitions of P start slots; the
 *     first bucket of every partition after the first bumps its first 64
 *     offsets so that no kept equation overlaps a cut, which makes the
 *     partitions independent and the cuts invisible to queries;
 *   - back-substitution (free slots fixed to 0) gives the table Z;
 *   - bumped keys form the next layer; after `layers` layers a base case
 *     without bumping is retried with a new seed and 10% more slots until it
 *     solves.
 *
 * Conventions the paper leaves open (hash function, levels, load factor,
 * storage layout) are fixed here as the library's specification:
 *   mix(z)       SplitMix64 output function (Steele, Lea, Flood 2014)
 *   sigma_l      mix(seed ^ ((l+1) * 0x9E3779B97F4A7C15)), l = layer index
 *                (bumping layers 0..layers-1, base-case attempt a: layers+a)
 *   h            mix(key ^ sigma_l)
 *   start        floor(h * (m - 63) / 2^64)
 *   coefficients mix(h + sigma_l) | 1   (bit k <-> slot start+k)
 *   bucket       start / 128, offset = start % 128; keys with
 *                offset < levels[code] are bumped
 *   layer slots  m = align64(ceil(n / load_factor) + 64)
 *   partitions   P = partition_slots in layer 0, lower_partition_slots in
 *                deeper layers (the paper's minimum buckets per thread, Sec. 3:
 *                deep layers are small, so their partitions are short);
 *                K = 1 if m < max(P, min_partition_slots), else floor(m/P);
 *                cut j at start slot c_j = j*P, the last partition takes the
 *                rest; partition j owns slots [c_j + 64, c_{j+1} + 64)
 *   cut search   (Sec. 3, optional) c_j is the bucket among the first
 *                min(range, P/B) buckets from j*P that minimises: keys at its
 *                offsets < 64 (minbump), minus keys in the 63 slots before it
 *                (maxprev), or their difference (diff); first best wins
 *   table layout per 64-slot block, r 64-bit words; bit k of slot s is bit
 *                s%64 of word (s/64)*r + k
 *   thresholds   2-bit codes, 32 per 64-bit word, bucket b in bits
 *                [2(b%32), 2(b%32)+2) of word b/32; or 1+-bit (Sec. 2): the
 *                exact threshold t in [0, B] (rows with offset < t bumped,
 *                the least t for which the rest insert; t >= 64 after a
 *                cut), stored as a bit per bucket (t > 0) plus the t of the
 *                flagged buckets, found by their rank (a count per 512
 *                buckets) where the paper uses a small hash table
 *
 * Pointers: every key/value/output pointer may be host memory (pageable or
 * pinned) or device memory of the current device; the library detects which.
 * Values are unsigned integers of the smallest width holding r bits
 * (uint8 for r <= 8, uint16 for r <= 16, uint32 for r <= 32); bits at and
 * above r are ignored.  Queries write the same type.
 *
 * Errors: every call returns 0 or a negative BURR_ERR_* code; nothing throws
 * across the ABI.  burr_last_error() gives a message for the calling thread.
 */
#ifndef BURR_H
#define BURR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BURR_OK 0
#define BURR_ERR_INVALID (-1)     /* bad argument or parameter */
#define BURR_ERR_OOM (-2)         /* device allocation failed */
#define BURR_ERR_UNSOLVABLE (-3)  /* base case failed every retry (e.g. duplicate keys) */
#define BURR_ERR_TIMEOUT (-4)     /* a bounded device-side wait expired */
#define BURR_ERR_CUDA (-5)        /* a CUDA runtime call failed */
#define BURR_ERR_INTERNAL (-6)    /* a device-side capacity check tripped */

#define BURR_THRESH_2BIT 0u       /* four threshold levels, 2 bits per bucket */
#define BURR_THRESH_1PLUS 1u      /* 1+-bit: a bit per bucket, exact thresholds of bumping buckets */
#define BURR_CUT_NONE 0u          /* cut j of a layer at start slot j*P */
#define BURR_CUT_MINBUMP 1u       /* cut search: fewest keys bumped by the cut itself */
#define BURR_CUT_MAXPREV 2u       /* cut search: most keys in the w-1 slots before the cut */
#define BURR_CUT_DIFF 3u          /* cut search: least (bumped by the cut) - (keys before it) */
#define BURR_MAX_LAYERS 8
#define BURR_FLAG_TIMING 1u       /* record per-stage device times (burr_stats) */
#define BURR_FLAG_TEST_WINDOW 2u  /* testing only: the band treats a pivot 136 or more slots past
                                     its bucket's first slot as leaving the on-chip window (the
                                     BURR_ERR_INTERNAL path of a real window overflow, which needs
                                     a pivot 382 or more slots past its row's start) */
#define BURR_FLAG_TEST_SLACK 4u   /* testing only: a layer sorted in two scatter passes (more than
                                     2^16 buckets) sorts into bins of half their expected size, so
                                     that they overflow and the layer is sorted again exactly (the
                                     structure is the same either way) */

typedef struct burr_handle burr_handle;

/* Construction parameters (Sec. 2-4; defaults from burr_default_params). */
typedef struct {
    uint32_t ribbon_width;          /* w: must be 64 */
    uint32_t bucket_slots;          /* B: start slots per bucket, 64 or 128 (128) */
    uint32_t threshold_mode;        /* BURR_THRESH_2BIT or BURR_THRESH_1PLUS (2-bit) */
    uint32_t layers;                /* bumping layers before the base case, 0..8 (4) */
    uint32_t levels[4];             /* threshold levels in slots: 0 < l1 < l2 < B = l3 ({0,32,64,128});
                                       the smallest level >= w is the level forced after a cut */
    double load_factor;             /* keys per slot of a bumping layer (1.015) */
    uint64_t partition_slots;       /* P: start slots per partition of layer 0, a multiple of B (65536) */
    uint64_t min_partition_slots;   /* layers with fewer slots are one partition (4096) */
    uint64_t seed;                  /* hash seed */
    double fallback_slack;          /* base case m = align64(ceil(n (1+slack)) + 64) (0.1) */
    uint32_t fallback_max_retries;  /* base-case retries, each with 10% more slots (16) */
    uint32_t flags;                 /* BURR_FLAG_* */
    uint64_t lower_partition_slots; /* P of bumping layers >= 1, a multiple of B; 0 = partition_slots (4096) */
    uint32_t cut_search;            /* BURR_CUT_* (BURR_CUT_NONE) */
    uint32_t cut_search_range;      /* buckets searched from each nominal cut (50) */
} burr_params;

/* Per-build statistics. */
typedef struct {
    uint64_t n;                                 /* keys */
    uint32_t r;
    uint32_t layers;                            /* bumping layers configured */
    uint64_t layer_n[BURR_MAX_LAYERS + 1];      /* keys per layer; [layers] = base case */
    uint64_t layer_m[BURR_MAX_LAYERS + 1];      /* slots per layer */
    uint64_t layer_parts[BURR_MAX_LAYERS + 1];  /* partitions per layer */
    uint64_t layer_bumped[BURR_MAX_LAYERS + 1]; /* keys bumped out of each layer */
    uint32_t fallback_attempt;                  /* base-case attempt that solved */
    uint32_t pad;
    /* device milliseconds per layer and stage (BURR_FLAG_TIMING):
       [l][0] sort, [l][1] band+bump, [l][2] back-substitution */
    float stage_ms[BURR_MAX_LAYERS + 1][3];
    float total_ms;                             /* whole build, device time */
    float pad2;
    uint64_t table_bytes;                       /* Z + thresholds of all layers */
    uint64_t kernel_launches;                   /* CUDA kernels this build launched */
} burr_stats_t;

/*
 * Device memory.  By default the library takes its device memory (build
 * scratch, the tables of every handle, query staging, the server's batch
 * inputs) from the current device's stream-ordered pool.  burr_set_allocator
 * routes it through the caller's allocator instead, e.g. PyTorch's caching
 * allocator (an interface of this library; the paper has no counterpart):
 *   alloc(bytes, stream, ctx)  device memory usable in stream order on
 *                              `stream` (a cudaStream_t), or NULL (the call
 *                              that needed it fails with BURR_ERR_OOM);
 *   free(ptr, stream, ctx)     release after the work enqueued on `stream`;
 *                              stream NULL: no work uses it any more.
 * Both NULL restores the built-in pool.  Returns BURR_ERR_INVALID if exactly
 * one of alloc/free is NULL, or while blocks from the current allocator are
 * still held (handles not freed, a build running): set it before building.
 * The callbacks may be called from any thread that calls the library and
 * from the server's worker threads.
 */
typedef void *(*burr_alloc_fn)(uint64_t bytes, void *stream, void *ctx);
typedef void (*burr_free_fn)(void *ptr, void *stream, void *ctx);
int burr_set_allocator(burr_alloc_fn alloc, burr_free_fn free, void *ctx);

/* Fill *p with the defaults above.  Returns BURR_OK or BURR_ERR_INVALID (p NULL).
 * Defaults follow the paper's setup where it gives one: buckets of 128 and four
 * bumping layers plus a base case (Sec. 4), 2-bit thresholds (Sec. 2,
 * "Bumping"), partitions that bump at least w-1 slots after each cut (Sec. 3);
 * the rest (hash, levels, load factor, P) are this library's readings above. */
int burr_default_params(burr_params *p);

/*
 * Build the structure for n keys (distinct; S is a set) and their r-bit values.
 * Paper: the retrieval problem of Sec. 1 (store f: S -> {0,1}^r so that
 * x in S gives f(x)), built as in Sec. 2 (ribbon equations, bumping by
 * thresholds, overloading, back-substitution, layers) with the partitioned
 * parallel construction of Sec. 3 (cuts, w-1 slots bumped after each cut).
 *   keys    n uint64 keys, host or device, caller-owned, read only.
 *   values  n values of the r-bit value type, host or device, caller-owned.
 *   r       value bits, 1..32.
 *   p       parameters (NULL = defaults).
 *   stream  cudaStream_t the work is ordered on (NULL = legacy default stream).
 *   out     receives a handle owned by the library until burr_free.
 * The call returns when the handle is complete (it synchronises the stream
 * once per layer to size the next layer).  n = 0 gives a valid empty handle.
 * Errors: BURR_ERR_INVALID (bad arguments / parameters / m >= 2^32),
 * BURR_ERR_OOM, BURR_ERR_UNSOLVABLE, BURR_ERR_INTERNAL, BURR_ERR_CUDA.
 */
int burr_build(const uint64_t *keys, const void *values, uint64_t n, uint32_t r,
               const burr_params *p, void *stream, burr_handle **out);

/*
 * Build `count` independent structures together (the many-small-structures use
 * of retrieval, e.g. inside perfect hashing, Sec. 1 "Applications"): one
 * launch per stage and layer covers every structure, so thousands of small
 * builds share the GPU instead of running one after the other.
 *   keys, values  all structures' keys and values back to back (host or
 *                 device); structure s owns [offsets[s], offsets[s+1]).
 *                 Values use the value type of the largest r in the batch.
 *   offsets       host array of count+1 entries, offsets[0] = 0, non-decreasing.
 *   r             host array of count value widths (1..32).
 *   p             parameters shared by all structures (NULL = defaults); with
 *                 p->partition_slots == 0 the library picks P in {2^14, 2^15,
 *                 2^16} so that the first layer has at least 8 partitions per
 *                 SM, and records it in every structure's parameters.
 *   out           host array of count handles.
 * Each structure follows exactly the single-structure rules (its export equals
 * burr_build of its keys with the same parameters, including the chosen P).
 * Each handle is used and freed like any other; the device tables of the batch
 * are released with the last of its handles.  A structure must have at most
 * 64*1024 buckets (about 8.5M keys at the default load); larger ones go
 * through burr_build.  Bucket size must be 128.
 */
int burr_build_batch(const uint64_t *keys, const void *values, const uint64_t *offsets, const uint32_t *r,
                     uint32_t count, const burr_params *p, void *stream, burr_handle **out);

/*
 * Paper: the query of Sec. 2: per layer, a key below its bucket's threshold
 * continues in the next layer, else its value is the parity of its
 * coefficient row AND the table window at its start slot, one bit per value
 * bit; cuts are invisible to queries (Sec. 3, partitions change only which
 * keys are bumped).  Keys of S return f(x); other keys an arbitrary but
 * deterministic value (Sec. 1).
 * Query n keys (host or device), writing n values of the handle's value type
 * to out (host or device).  Stream-ordered: with device keys and output the
 * call only enqueues work on `stream`; with any host pointer it copies through
 * device buffers and returns after the results are in `out`.
 */
int burr_query(const burr_handle *h, const uint64_t *keys, void *out, uint64_t n, void *stream);

/* Bytes of the device tables (Z of every layer + thresholds + a 64-byte header):
 * the space the paper accounts as overhead over r*n bits (Sec. 4.1 and Fig. 3,
 * overhead per additional thread).  BURR_ERR_INVALID if h or bytes is NULL. */
int burr_size_bytes(const burr_handle *h, uint64_t *bytes);

/*
 * Canonical little-endian serialisation (checkpoint format and the form in
 * which results are compared bit for bit; the paper has no counterpart):
 *   u32 magic 0x52525542, u32 version (1: 2-bit, 2: 1+-bit thresholds),
 *   u32 r, u32 w, u32 B, u32 layers,
 *   u32 levels[4], u64 seed, u64 bits of load_factor, u64 n, u64 partition_slots,
 *   per bumping layer: u64 n, m, partitions, buckets, bumped;
 *   base case: u64 n, m, seed index, attempt;
 *   per bumping layer: thresholds, then table words ((m/64)*r u64);
 *   base-case table words.  Thresholds are ceil(buckets/32) u64 of 2-bit
 *   codes (version 1), or (version 2) ceil(buckets/64) u64 flag words (bit
 *   b%64 of word b/64 set iff bucket b bumps), a u64 count of flagged
 *   buckets and their thresholds as bytes in bucket order, zero-padded to a
 *   multiple of 8 bytes.
 * If host_buf is NULL or *len is too small, *len is set to the size needed and
 * BURR_ERR_INVALID is returned; otherwise *len = bytes written.
 */
int burr_export(const burr_handle *h, void *host_buf, uint64_t *len);

/*
 * Load a structure from the export format above (written by burr_export, or by
 * any writer of the same format): the device tables are allocated and filled
 * and the handle answers queries exactly as the exported structure did.
 * Checkpoint/resume of built structures (the paper has no counterpart).
 *   host_buf, len  the export bytes (host memory, read only);
 *   stream         cudaStream_t of the copies (the call returns when they are done);
 *   out            receives a handle owned by the library until burr_free.
 * The whole buffer is checked before anything is allocated: magic, version,
 * parameters, layer sizes (n, slots, buckets, bumped keys chaining from layer
 * to layer), flag and threshold counts, and the exact length.  Errors:
 * BURR_ERR_INVALID (malformed buffer), BURR_ERR_OOM, BURR_ERR_CUDA.  Build
 * statistics (stage times) of an imported handle are zero.
 */
int burr_import(const void *host_buf, uint64_t len, void *stream, burr_handle **out);

/* Sizes per layer (n, m, partitions, bumped keys: the quantities of Sec. 2-3),
 * device time per stage (the split of Fig. 7: sort, insertion with bumping,
 * back-substitution) and launch count of a build.  The call itself has no
 * counterpart in the paper.  BURR_ERR_INVALID if h or st is NULL. */
int burr_stats(const burr_handle *h, burr_stats_t *st);

/* Release the handle and its device memory (NULL is ignored).  The paper has
 * no counterpart (a library's resource management). */
void burr_free(burr_handle *h);

/* burr_free of handles[0 .. count) in one call (NULL entries are ignored),
 * e.g. for the handles of a batched build.  `handles` is a host array owned
 * by the caller; the handles must not be used afterwards. */
void burr_free_many(burr_handle *const *handles, uint64_t count);

/* Name of a BURR_* status code, and the message of the calling thread's last
 * failed call (both library conveniences with no counterpart in the paper;
 * the strings are owned by the library). */
const char *burr_strerror(int code);
const char *burr_last_error(void);

/*
 * Stage entry points, exposed so that each stage of the build can be checked
 * against an independent implementation.  All pointers are device memory.
 *
 * burr_stage_hash: step "hash each key to (start slot, coefficient row)" of
 * one layer (Sec. 2, Fig. 1): for i < n, start[i] and coeff[i] of keys[i] in a
 * layer of m slots with hash layer index `layer_index` and seed `seed`.
 */
int burr_stage_hash(const uint64_t *d_keys, uint64_t n, uint64_t seed, uint32_t layer_index,
                    uint64_t m, uint32_t *d_start, uint64_t *d_coeff, void *stream);

/*
 * burr_stage_sort: step "sort the equations by start slot" (Sec. 4, sorting by
 * insertion position) as the build does it: keys and values grouped by bucket
 * (start/128) in ascending bucket order, any order inside a bucket.
 * d_bucket_start receives buckets+1 offsets (buckets = (m - 64 + 128)/128).
 * Scratch is allocated on `stream` and released before return.
 */
int burr_stage_sort(const uint64_t *d_keys, const void *d_values, uint64_t n, uint32_t r,
                    uint64_t seed, uint32_t layer_index, uint64_t m,
                    uint64_t *d_sorted_keys, void *d_sorted_values, uint32_t *d_bucket_start,
                    void *stream);

/*
 * burr_stage_sort_noalloc: burr_stage_sort that allocates no device memory,
 * for callers that cannot allocate: a process whose device memory belongs to
 * its own pool allocator, a latency-critical loop that cannot take the
 * implicit synchronisation of cudaMalloc/cudaFree, or code that must not fail
 * with out-of-memory half-way through.  (The paper has no counterpart: it is
 * an interface convenience of this library.)
 *   Arguments, layout and result are those of burr_stage_sort; all pointers
 *   are device memory owned by the caller.
 *   n must be <= BURR_NOALLOC_MAX_KEYS and m <= BURR_NOALLOC_MAX_SLOTS, else
 *   BURR_ERR_INVALID with a message.
 *   The sort's scratch is one fixed file-scope device array of about 12.6 MB
 *   that every GPU which loads the library keeps until the process exits.
 *   Every call looks up that array's device address with the device current
 *   (a lookup that allocates nothing); the first call on a device also loads
 *   the library's device code there, so make that first call before any
 *   stream capture.  All calls share the array and it keeps the last call's
 *   contents: calls whose work overlaps on the GPU (other streams or host
 *   threads) race, so order them, e.g. on one stream.
 */
#define BURR_NOALLOC_MAX_KEYS (1u << 20)
#define BURR_NOALLOC_MAX_SLOTS (1u << 24)
int burr_stage_sort_noalloc(const uint64_t *d_keys, const void *d_values, uint64_t n, uint32_t r,
                            uint64_t seed, uint32_t layer_index, uint64_t m,
                            uint64_t *d_sorted_keys, void *d_sorted_values, uint32_t *d_bucket_start,
                            void *stream);

/*
 * Sharded construction of ONE structure over several ranks (processes, GPUs,
 * or shards sharing one GPU).  Paper: Sec. 3 ("Bumping" at thread
 * boundaries): once a layer's cuts are placed, the first bucket after every
 * cut bumps at least w-1 slots, so no kept equation crosses a cut and every
 * partition is inserted and back-substituted independently.  Rank g owns the
 * partitions [part_first[g], part_first[g+1]) of each bumping layer; a layer
 * is built as:
 *   1. n_layer = the layer's keys over all ranks (a sum the caller forms);
 *   2. burr_shard_route: each rank groups its keys by owner rank (the owner of
 *      the key's start bucket) -- the caller exchanges the groups (one
 *      all-to-all of (key, value) records per layer);
 *   3. burr_shard_build_layer: each rank sorts, bands and back-substitutes
 *      its partitions; its bumped keys are its input of the next layer.
 * After the last bumping layer one rank gathers the remaining keys and calls
 * burr_shard_build_base.  The thresholds of the buckets each rank owns, its
 * table words of the slots it owns ([c + 64, c' + 64) for its first cut c
 * and the first cut c' after its range; from 0 for partition 0, to m for the
 * last) and the base case together form the export of burr_build on the
 * union of the keys, byte for byte (2-bit thresholds, cut j at j*P; cut search
 * and 1+-bit thresholds are not supported here: BURR_ERR_INVALID).
 * All key/value/table pointers are device memory owned by the caller.
 */
typedef struct {
    uint64_t n;                 /* keys of the layer over all ranks */
    uint64_t m;                 /* slots */
    uint64_t buckets;
    uint64_t partitions;        /* K: partition j starts at bucket j*P/B */
    uint64_t partition_slots;   /* P */
    uint64_t seed_index;        /* hash layer index (= the layer) */
} burr_layer_geometry_t;

/* Geometry of bumping layer `layer` (0 .. p->layers-1) holding n_layer keys:
 * the sizing and partition rules of burr_build.  Host only. */
int burr_layer_geometry(uint64_t n_layer, uint32_t layer, const burr_params *p, burr_layer_geometry_t *out);

/* Group n (key, value) pairs by the rank that owns each key's start bucket in
 * layer `layer` of n_layer keys.  part_first: host array of ranks+1 entries,
 * from 0 to the layer's partitions, non-decreasing.  keys_out/values_out
 * (n entries) receive rank 0's pairs, then rank 1's, ...; counts (host,
 * ranks entries) their numbers.  The order inside a rank's run is not fixed.
 * ranks <= 1024.  Returns after the output is written. */
int burr_shard_route(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *p,
                     uint32_t layer, uint64_t n_layer, uint32_t ranks, const uint32_t *part_first,
                     uint64_t *keys_out, void *values_out, uint64_t *counts, void *stream);

/* Build partitions [part_lo, part_hi) of layer `layer` (n_layer keys over all
 * ranks) from their n keys -- exactly the keys whose start bucket lies in
 * those partitions.  thresh: ceil(buckets/32) words, z: (m/64)*r words; both
 * are cleared and then hold the codes of the range's buckets and the table
 * words of the slots it owns.  bumped_keys/values (capacity n) receive the
 * keys the range bumps, *nbumped (host) their number.  Returns after the
 * results are written; BURR_ERR_INTERNAL if a device check tripped. */
int burr_shard_build_layer(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *p,
                           uint32_t layer, uint64_t n_layer, uint32_t part_lo, uint32_t part_hi, uint64_t *thresh,
                           uint64_t *z, uint64_t *bumped_keys, void *bumped_values, uint64_t *nbumped,
                           void *stream);

/* The base case of n keys (all that the bumping layers bumped): no bumping,
 * retried with the next seed and 10% more slots until it solves (Sec. 3,
 * Sec. 4).  z must hold (m_max/64)*r words, m_max = the base-case slots of the
 * last retry; with z NULL or smaller the call returns BURR_ERR_INVALID and
 * sets *m_out = m_max.  Outputs: its slots, seed index (layers + attempt) and
 * attempt.  BURR_ERR_UNSOLVABLE after the last retry (duplicate keys). */
int burr_shard_build_base(const uint64_t *keys, const void *values, uint64_t n, uint32_t r, const burr_params *p,
                          uint64_t *z, uint64_t z_words, uint64_t *m_out, uint64_t *seed_index_out,
                          uint32_t *attempt_out, void *stream);

/*
 * Build/query server on one device: continuous batching of independent
 * builds with resident structures (the many-small-structures use of
 * retrieval, Sec. 1 "Applications"; the paper describes no server: the
 * request loop is an interface of this library around burr_build_batch).
 *
 * Each of cfg.build_workers build worker threads (one stream each)
 * repeatedly takes every queued build request whose device-memory estimate
 * fits the budget next to the resident structures and the builds in flight,
 * and builds them with one burr_build_batch call per value width (structures
 * larger than a batch allows get burr_build of their own).  A request
 * submitted while a batch runs is taken by an idle worker at once, so
 * batches overlap on the device (continuous batching); with every worker
 * busy it joins the next batch.
 * Payloads are copied at submission into a page-locked host region of
 * host_staging_bytes (so that the copies to the device are DMA at link
 * speed), or into pageable memory when the region has no room.  A query worker
 * thread runs queries on a second stream as soon as their structure is
 * resident, overlapping the builds.  The partition size is the server's
 * p->partition_slots (must be > 0), so a structure's export is the one
 * burr_build gives for its keys with the server's parameters, whatever else
 * shared its batch.
 */
typedef struct burr_server burr_server;

typedef struct {
    uint64_t memory_budget;          /* device bytes for resident structures plus builds in flight (> 0) */
    uint64_t host_staging_bytes;     /* page-locked host region for request payloads (0 = none) */
    uint32_t max_batch_structures;   /* most structures per batch (0 = 4096) */
    uint32_t build_workers;          /* build worker threads, one stream each: batches that
                                        overlap on the device (0 = 1, at most 8) */
} burr_server_config;

typedef struct {
    uint64_t bytes_resident;         /* table bytes of the resident structures */
    uint64_t bytes_inflight;         /* estimated bytes of the builds running now */
    uint64_t resident_structures;
    uint64_t queued_builds;          /* submitted, not yet admitted */
    uint64_t queued_queries;
    uint64_t batches;                /* burr_build_batch calls made */
    uint64_t batched_structures;     /* structures built by those calls */
    uint64_t staged_requests;        /* payloads copied into the page-locked region */
    uint64_t pageable_requests;      /* payloads that did not fit it (pageable memory) */
    uint64_t built_keys;             /* keys of the builds completed or failed */
    double build_busy_ms;            /* host time the build workers spent building (summed) */
    double query_busy_ms;            /* host time the query worker spent querying */
    uint64_t max_concurrent_batches; /* most admitted batches building at the same time */
} burr_server_stats_t;

/* Start a server on the current device.  p = NULL: defaults.  The server owns
 * two non-blocking streams and two threads until burr_server_destroy. */
int burr_server_create(const burr_server_config *cfg, const burr_params *p, burr_server **out);

/* Queue a build of n keys (distinct) with r-bit values (host memory, copied
 * before return).  *ticket names the structure.  The admission estimate of a
 * build is 4n(8+vb) + 2m(8+vb) + 8r(m/64) + 2^20 bytes, vb the value type's
 * bytes and m = align64(ceil(n / load_factor) + 64); BURR_ERR_OOM if it alone
 * exceeds the budget. */
int burr_server_submit_build(burr_server *s, const uint64_t *keys, const void *values, uint64_t n, uint32_t r,
                             uint64_t *ticket);

/* Queue a query of n host keys on the structure of build_ticket (which may
 * still be queued).  `out` (host, n values of the structure's value type)
 * must stay valid until burr_server_wait returns for *ticket. */
int burr_server_submit_query(burr_server *s, uint64_t build_ticket, const uint64_t *keys, uint64_t n, void *out,
                             uint64_t *ticket);

/* Block until the request is done; *latency_ms (if not NULL) = time from its
 * submission to its completion.  Returns the request's status (a failed
 * build's error, or a query on a structure that failed to build:
 * BURR_ERR_INVALID).  Waiting retires a query ticket; a build ticket stays
 * valid until burr_server_release. */
int burr_server_wait(burr_server *s, uint64_t ticket, double *latency_ms);

/* The resident structure of a completed build (owned by the server; valid
 * until burr_server_release of the ticket or burr_server_destroy). */
int burr_server_handle(burr_server *s, uint64_t build_ticket, const burr_handle **out);

/* Free a completed build's structure and return its memory to the budget.
 * BURR_ERR_INVALID while the build is pending or queries on it are queued;
 * a query running on it is waited for. */
int burr_server_release(burr_server *s, uint64_t build_ticket);

/* A snapshot of the counters above, taken under the server's lock.
 * BURR_ERR_INVALID if s or st is NULL. */
int burr_server_stats(burr_server *s, burr_server_stats_t *st);

/* Finish the running batch and queries, fail the builds still queued
 * (BURR_ERR_INVALID), free every structure and stop the threads.  No other
 * call on `s` may run concurrently or follow. */
void burr_server_destroy(burr_server *s);

#ifdef __cplusplus
}
#endif
#endif /* BURR_H */
