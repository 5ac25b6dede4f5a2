/*
 * burr_oracle.h -- serial CPU oracle of BuRR construction (test infrastructure
 * only; never linked into the CUDA library).
 */
#ifndef BURR_ORACLE_H
#define BURR_ORACLE_H
#include <stdint.h>

#define OR_MAX_LAYERS 8
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)
#define OR_UNSOLVABLE (-3)
#define OR_FAIL (-4)
#define OR_MAX_THREADS 256     /* host threads of the threaded variants */

#define OR_THRESH_2BIT 0u   /* four threshold levels, 2 bits per bucket */
#define OR_THRESH_1PLUS 1u  /* exact threshold; 1 bit per bucket + the bumping buckets' thresholds */

#define OR_CUT_NONE 0u      /* cut j at j*P */
#define OR_CUT_MINBUMP 1u   /* fewest keys bumped by the cut itself */
#define OR_CUT_MAXPREV 2u   /* most keys in the w-1 slots before the cut */
#define OR_CUT_DIFF 3u      /* least (bumped by the cut) - (keys in the w-1 slots before) */

typedef struct {
    uint32_t r;                     /* value bits, 1..32 */
    uint32_t w;                     /* ribbon width, 64 */
    uint32_t B;                     /* bucket size in slots, 128 */
    uint32_t levels[4];             /* 2-bit threshold levels in slots, {0,..,B} */
    double alpha;                   /* keys per slot (overload when > 1) */
    uint32_t layers;                /* bumping layers before the base case */
    uint32_t fb_max_retries;        /* base-case retries */
    uint64_t partition_slots;       /* P: cut every P start slots */
    uint64_t min_partition_slots;   /* layers below this are one partition */
    uint64_t seed;
    double fb_slack;                /* base case m = n(1+slack)+w, x1.1 per retry */
    uint64_t cut_P[OR_MAX_LAYERS];  /* per-layer override of P (0 = P) */
    uint32_t threshold_mode;        /* OR_THRESH_2BIT or OR_THRESH_1PLUS */
    uint32_t pad;
    uint64_t lower_partition_slots; /* P of layers >= 1 (0 = partition_slots) */
    uint32_t cut_search;            /* OR_CUT_* */
    uint32_t cut_search_range;      /* buckets searched from each nominal cut */
} or_params;

typedef struct {
    uint64_t n, m, seed_index, nbuckets, nparts, part_slots, nbumped;
    uint64_t *cuts;                 /* nparts-1 cut start slots used */
    uint64_t *thresh;               /* 2-bit mode: ceil(nbuckets/32) words of 2-bit codes */
    uint64_t *z;                    /* (m/64)*r words, interleaved bit planes */
    uint8_t *texact;                /* 1+-bit mode: exact threshold of every bucket, 0..B */
} or_layer;

typedef struct {
    or_params params;
    uint64_t n;
    uint64_t fb_attempt;
    or_layer layer[OR_MAX_LAYERS + 1];  /* [OR_MAX_LAYERS] is the base case */
} or_struct;

typedef struct {
    uint64_t xor_steps;             /* row XORs during elimination */
    uint64_t inserted;              /* insertion attempts */
    uint64_t max_drift;             /* max pivot - start */
    uint64_t bumped[OR_MAX_LAYERS];
} or_stats;

uint64_t or_mix64(uint64_t z);
uint64_t or_layer_seed(uint64_t seed, uint64_t index);
void or_hash(uint64_t key, uint64_t sigma, uint64_t m, uint32_t w,
             uint64_t *start, uint64_t *coeff);
void or_hash_batch(const uint64_t *keys, uint64_t n, uint64_t sigma, uint64_t m, uint32_t w,
                   uint64_t *starts, uint64_t *coeffs);
uint64_t or_layer_slots(uint64_t n, double alpha, uint32_t w);
uint64_t or_fallback_slots(uint64_t n, double slack, uint32_t w, uint32_t attempt);
uint64_t or_num_buckets(uint64_t m, uint32_t w, uint32_t B);
uint64_t or_num_partitions(uint64_t m, uint64_t P, uint64_t min_slots);
int or_forced_code(const uint32_t levels[4], uint32_t w);
int or_build_layer(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                   uint32_t r, uint64_t m, uint64_t sigma,
                   const uint32_t levels[4], uint32_t B, uint32_t w,
                   const uint64_t *cuts, uint64_t ncuts, int fallback,
                   uint64_t *thresh, uint64_t *z,
                   uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                   or_stats *st);
int or_build_layer_mode(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                        uint32_t r, uint64_t m, uint64_t sigma,
                        const uint32_t levels[4], uint32_t B, uint32_t w,
                        const uint64_t *cuts, uint64_t ncuts, int fallback,
                        uint32_t mode, uint64_t *thresh, uint8_t *texact, uint64_t *z,
                        uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                        or_stats *st);
int or_build_layer_mt(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                      uint32_t r, uint64_t m, uint64_t sigma,
                      const uint32_t levels[4], uint32_t B, uint32_t w,
                      const uint64_t *cuts, uint64_t ncuts, int fallback,
                      uint32_t mode, uint64_t *thresh, uint8_t *texact, uint64_t *z,
                      uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                      or_stats *st, unsigned nthreads);
int or_search_cuts(const uint64_t *keys, uint64_t n, uint64_t m, uint64_t sigma, uint32_t B, uint32_t w,
                   uint64_t P, uint64_t K, uint32_t mode, uint32_t range, uint64_t *cuts);
void or_default_params(or_params *p);
int or_build(const uint64_t *keys, const uint32_t *vals, uint64_t n,
             const or_params *p, or_struct *out, or_stats *st);
int or_build_mt(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                const or_params *p, or_struct *out, or_stats *st, unsigned nthreads);
void or_free(or_struct *s);
uint32_t or_query_one(const or_struct *s, uint64_t key);
void or_query(const or_struct *s, const uint64_t *keys, uint32_t *out, uint64_t n);
uint64_t or_export(const or_struct *s, uint8_t *buf, uint64_t cap);
double or_overhead(const or_struct *s);

#endif
