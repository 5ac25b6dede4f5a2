/*
 * burr_oracle.c -- serial CPU oracle for Bumped Ribbon Retrieval (BuRR)
 * construction with bumping at partition ("thread") boundaries.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the ground truth that the CUDA
 * library is checked against.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA path.
 *
 * It follows the method step by step, in the paper's order:
 *   - the retrieval problem f: S -> {0,1}^r                   (Sec. 1, abstract)
 *   - one GF(2) equation per key whose coefficients lie in a window of width
 *     w that starts at the key's hashed start slot ("spatial coupling")  (Sec. 2, Fig. 1)
 *   - sort the equations by start slot                       (Sec. 4, sort via IPS2Ra)
 *   - on-the-fly Gaussian elimination bucket by bucket, bumping a prefix of a
 *     bucket on failure, the prefix given by a 2-bit threshold (four levels,
 *     one bumping nothing and one bumping the whole bucket)     (Sec. 2, "Bumping")
 *     or by a 1+-bit threshold (one bit "anything bumped?" per bucket, the
 *     exact threshold stored only for the buckets that bump)    (Sec. 2, threshold storage)
 *   - overloading: more equations than slots per layer          (Sec. 2, last para.)
 *   - parallel construction: the equation system is cut into partitions and the
 *     first bucket after every cut bumps at least w-1 slots, so no kept equation
 *     overlaps a cut and partitions are independent             (Sec. 3, "Bumping")
 *   - optional cut-point search: move each cut to a nearby bucket where the
 *     cut bumps fewer keys or where more keys precede it     (Sec. 3, "Selecting Cut Points")
 *   - back-substitution                                         (Sec. 4, Fig. 7)
 *   - bumped keys go to the next layer; 4 layers, then a base case that cannot
 *     bump and is scaled up until it solves                     (Sec. 3, Sec. 4)
 *   - the query: AND the key's coefficients with the table window and take the
 *     parity, one bit per value bit                              (Sec. 2)
 *
 * Where the paper is silent (it defers to the SEA'22 BuRR paper) this oracle
 * takes one written reading; each reading is marked "READING" below.
 *
 * Parity pins: every function here is pinned by tests that do not reuse this
 * code (known-answer vectors of SplitMix64, an inverse of the mixer, a dense
 * GF(2) brute-force solver, the query invariant, permutation invariance).
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#include "burr_oracle.h"

/* ------------------------------------------------------------------------ */
/* Hashing (READING: the paper defers the hash to SEA'22).                   */
/* ------------------------------------------------------------------------ */

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014), a bijection
 * on 64-bit words. */
uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

#define OR_GOLDEN 0x9E3779B97F4A7C15ULL

/* Seed of hash layer `index` (bumping layers 0..L-1, base-case attempt a at
 * index L+a). */
uint64_t or_layer_seed(uint64_t seed, uint64_t index)
{
    return or_mix64(seed ^ ((index + 1) * OR_GOLDEN));
}

/* floor(a*b / 2^64): Lemire's multiply-shift range reduction. */
static uint64_t or_mulhi(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

/* The equation of one key in a layer with m slots: start slot s in
 * [0, m-w] and a w-bit coefficient row whose bit k stands for slot s+k;
 * bit 0 is always set. */
void or_hash(uint64_t key, uint64_t sigma, uint64_t m, uint32_t w,
             uint64_t *start, uint64_t *coeff)
{
    uint64_t h = or_mix64(key ^ sigma);
    *start = or_mulhi(h, m - w + 1);
    *coeff = or_mix64(h + sigma) | 1ULL;
}

/* or_hash over an array of keys. */
void or_hash_batch(const uint64_t *keys, uint64_t n, uint64_t sigma, uint64_t m, uint32_t w,
                   uint64_t *starts, uint64_t *coeffs)
{
    for (uint64_t i = 0; i < n; i++) or_hash(keys[i], sigma, m, w, &starts[i], &coeffs[i]);
}

/* ------------------------------------------------------------------------ */
/* Sizing and partitioning (READING: overload factor and cut placement).     */
/* ------------------------------------------------------------------------ */

static uint64_t or_align64(uint64_t x) { return (x + 63) & ~63ULL; }

/* Slots of a bumping layer holding n keys at load alpha (keys per slot). */
uint64_t or_layer_slots(uint64_t n, double alpha, uint32_t w)
{
    if (n == 0) return 0;
    return or_align64((uint64_t)ceil((double)n / alpha) + w);
}

/* Slots of the base case for n keys, attempt a: the first size leaves
 * `slack` spare rows, every retry grows it by 10%. */
uint64_t or_fallback_slots(uint64_t n, double slack, uint32_t w, uint32_t attempt)
{
    if (n == 0) return 0;
    uint64_t m = or_align64((uint64_t)ceil((double)n * (1.0 + slack)) + w);
    for (uint32_t a = 0; a < attempt; a++)
        m = or_align64((uint64_t)ceil((double)m * 1.1));
    return m;
}

/* Number of 128-slot (B-slot) buckets of start positions: starts are 0..m-w. */
uint64_t or_num_buckets(uint64_t m, uint32_t w, uint32_t B)
{
    if (m == 0) return 0;
    return (m - w + B) / B;
}

/* Number of partitions of a layer with m slots (minimum-buckets-per-thread
 * analogue, Sec. 3): layers below min_slots, or smaller than P, are one
 * partition.  Otherwise there are floor(m/P) partitions of P slots, plus one
 * more for the remainder m mod P when it is at least
 * T = max(min(min_slots, P/2), 1024) slots; a smaller remainder joins the
 * last partition.  So no partition is much longer than P (the paper gives the
 * threads near-equal shares).  Cut j (j >= 1) sits at start slot j*P. */
uint64_t or_num_partitions(uint64_t m, uint64_t P, uint64_t min_slots)
{
    if (m == 0) return 0;
    if (m < min_slots || m < P) return 1;
    uint64_t T = min_slots < P / 2 ? min_slots : P / 2;
    if (T < 1024) T = 1024;
    uint64_t K = m / P, rem = m % P;
    return rem >= T ? K + 1 : K;
}

/* ------------------------------------------------------------------------ */
/* One layer: sort, insert with bumping, back-substitute.                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t key;
    uint32_t val;
    uint64_t start;
    uint64_t coeff;
} or_row;

/* Equations ordered by bucket ascending, then offset descending (inside a
 * bucket the rows are inserted from the bucket's end towards its start, so
 * that a threshold bumps a prefix).  Ties are broken by key only to make the
 * oracle deterministic; the result does not depend on it. */
static uint32_t g_B;
static int or_row_cmp(const void *pa, const void *pb)
{
    const or_row *a = (const or_row *)pa, *b = (const or_row *)pb;
    uint64_t ba = a->start / g_B, bb = b->start / g_B;
    if (ba != bb) return ba < bb ? -1 : 1;
    uint64_t oa = a->start % g_B, ob = b->start % g_B;
    if (oa != ob) return oa > ob ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return 0;
}

/* On-the-fly Gaussian elimination of one equation into the band (C = stored
 * coefficient rows, C[p] has bit 0 = pivot p, 0 = empty slot; Y = stored
 * right-hand sides).  Returns the slot it was stored in, or -1 if the
 * coefficients vanished (READING: a vanishing row is a failure whatever its
 * right-hand side). */
static int64_t or_insert(uint64_t *C, uint32_t *Y, uint64_t start, uint64_t coeff,
                         uint32_t val, uint64_t *steps)
{
    uint64_t cur = coeff, p = start;
    uint32_t y = val;
    for (;;) {
        if (cur == 0) return -1;
        int tz = __builtin_ctzll(cur);
        p += (uint64_t)tz;
        cur >>= tz;
        if (C[p] == 0) {
            C[p] = cur;
            Y[p] = y;
            return (int64_t)p;
        }
        cur ^= C[p];
        y ^= Y[p];
        (*steps)++;
    }
}

/* Smallest level strictly above offset o. */
static uint32_t or_level_above(const uint32_t levels[4], uint32_t o)
{
    for (int i = 0; i < 4; i++)
        if (levels[i] > o) return (uint32_t)i;
    return 3;
}

/* Smallest level that bumps at least w-1 slots after a cut.  READING: we take
 * the smallest level >= w, which for w=64 and levels {0,32,64,128} is the
 * level 64 either way and places the ownership boundary between partitions at
 * cut + w, a multiple of 64. */
int or_forced_code(const uint32_t levels[4], uint32_t w)
{
    for (int i = 0; i < 4; i++)
        if (levels[i] >= w) return i;
    return -1;
}

/*
 * What the steps of one layer build share.  rows: the layer's equations, in
 * bucket order after step 2; C/Y: the band (C[p] = stored coefficient row,
 * bit 0 = pivot p, 0 = empty slot; Y[p] = its right-hand side); slot_of[k]:
 * slot of row k while it is stored, -1 otherwise; code_of / texact: the
 * threshold of every bucket (2-bit code / exact threshold); Zs: the solution,
 * one r-bit value per slot.
 */
typedef struct {
    or_row *rows;
    uint64_t n, m, nb;
    uint32_t r, B, w, mode;
    int fallback, forced;
    uint32_t t_forced;
    const uint32_t *levels;
    const uint64_t *cuts;
    uint64_t ncuts;
    uint64_t *C;
    uint32_t *Y;
    int64_t *slot_of;
    uint8_t *code_of;
    uint8_t *texact;
    uint32_t *Zs;
} or_work;

/*
 * Step 3 for rows [i0, i1), which hold whole buckets: insertion bucket by
 * bucket; on the first failure the bucket's threshold is set and every row of
 * the bucket below it is rolled back.  Bumped rows are appended to
 * bumped_keys/vals (count in *nbumped).  Returns 0, or OR_FAIL when a row of
 * the base case does not insert.
 */
static int or_insert_rows(or_work *W, uint64_t i0, uint64_t i1,
                          uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                          or_stats *st)
{
    const or_row *rows = W->rows;
    const uint64_t *cuts = W->cuts;
    const uint64_t ncuts = W->ncuts;
    const uint32_t B = W->B, mode = W->mode;
    const uint32_t *levels = W->levels;
    const int fallback = W->fallback, forced = W->forced;
    uint64_t *C = W->C;
    uint32_t *Y = W->Y;
    int64_t *slot_of = W->slot_of;
    uint8_t *texact = W->texact;
    uint64_t i = i0, cut_idx = 0;
    int status = 0;
    while (i < i1) {
        uint64_t b = rows[i].start / B;
        uint64_t j = i;
        while (j < i1 && rows[j].start / B == b) j++;
        /* rows[i..j) is bucket b in descending offset order */
        while (cut_idx < ncuts && cuts[cut_idx] < b * B) cut_idx++;
        int after_cut = (cut_idx < ncuts && cuts[cut_idx] == b * B);
        uint32_t t = (after_cut && !fallback) ? W->t_forced : 0;
        uint32_t code = (after_cut && !fallback && mode == OR_THRESH_2BIT) ? (uint32_t)forced : 0;
        for (uint64_t k = i; k < j; k++) slot_of[k] = -1;
        for (uint64_t k = i; k < j; k++) {
            uint32_t off = (uint32_t)(rows[k].start % B);
            if (off < t) break;              /* forced bump below the level */
            int64_t p = or_insert(C, Y, rows[k].start, rows[k].coeff, rows[k].val,
                                  st ? &st->xor_steps : &(uint64_t){0});
            if (st) st->inserted++;
            if (p >= 0) {
                slot_of[k] = p;
                if (st && (uint64_t)p - rows[k].start > st->max_drift)
                    st->max_drift = (uint64_t)p - rows[k].start;
                continue;
            }
            if (fallback) { status = OR_FAIL; break; }
            if (mode == OR_THRESH_1PLUS) {
                t = off + 1;                 /* rows at offsets >= t were all kept */
            } else {
                code = or_level_above(levels, off);
                if (after_cut && code < (uint32_t)forced) code = (uint32_t)forced;
                t = levels[code];
            }
            /* roll back every row of this bucket below the new threshold */
            for (uint64_t q = i; q < k; q++) {
                uint32_t oq = (uint32_t)(rows[q].start % B);
                if (oq < t && slot_of[q] >= 0) {
                    C[slot_of[q]] = 0;
                    Y[slot_of[q]] = 0;
                    slot_of[q] = -1;
                }
            }
            break;
        }
        if (status) break;
        if (!fallback) {
            if (mode == OR_THRESH_1PLUS)
                texact[b] = (uint8_t)t;
            else
                W->code_of[b] = (uint8_t)code;
            for (uint64_t k = i; k < j; k++) {
                if ((uint32_t)(rows[k].start % B) < t) {
                    bumped_keys[*nbumped] = rows[k].key;
                    bumped_vals[*nbumped] = rows[k].val;
                    (*nbumped)++;
                }
            }
        }
        i = j;
    }
    return status;
}

/* Step 4 for slots [s0, s1): back-substitution, right to left, free slots
 * fixed to 0 (READING: the paper is silent on free variables). */
static void or_backsub_slots(or_work *W, uint64_t s0, uint64_t s1)
{
    const uint64_t *C = W->C;
    const uint32_t *Y = W->Y;
    uint32_t *Zs = W->Zs;
    for (uint64_t s = s1; s-- > s0;) {
        if (C[s] == 0) { Zs[s] = 0; continue; }
        uint32_t v = Y[s];
        for (int k = 1; k < 64; k++)
            if ((C[s] >> k) & 1ULL) v ^= Zs[s + (uint64_t)k];
        Zs[s] = v;
    }
}

/* The solution of slots [s0, s1) (multiples of 64) as interleaved bit planes:
 * bit k of slot s is bit s%64 of z[(s/64)*r + k]. */
static void or_pack_planes(const or_work *W, uint64_t s0, uint64_t s1, uint64_t *z)
{
    const uint32_t r = W->r;
    memset(z + (s0 / 64) * r, 0, sizeof(uint64_t) * ((s1 - s0) / 64) * r);
    for (uint64_t s = s0; s < s1; s++)
        for (uint32_t k = 0; k < r; k++)
            if ((W->Zs[s] >> k) & 1u)
                z[(s / 64) * r + k] |= 1ULL << (s % 64);
}

/* ------------------------------------------------------------------------ */
/* The same steps with the partitions spread over host threads (the paper's  */
/* parallel construction, Sec. 3: once the cuts are placed, every partition  */
/* is inserted and back-substituted on its own).                             */
/* ------------------------------------------------------------------------ */

typedef struct or_mt or_mt;
typedef void (*or_task)(or_mt *M, unsigned tid);

struct or_mt {
    or_work *W;
    const uint64_t *keys;
    const uint32_t *vals;
    uint32_t mask;
    uint64_t sigma;
    unsigned nthreads;
    uint64_t K;                 /* partitions: K = ncuts + 1 */
    uint32_t *part_of_bucket;   /* bucket -> partition */
    or_row *hashed;             /* step 1 output, input order */
    uint64_t *cnt;              /* [tid][K]: rows of the thread's input chunk per partition */
    uint64_t *prow;             /* [K+1]: first row of each partition after step 2 */
    uint64_t *pbumped;          /* [K]: bumped rows of each partition (at bumped + prow[q]) */
    uint64_t *bumped_keys;
    uint32_t *bumped_vals;
    uint64_t *z;
    or_stats *tstats;           /* [tid] */
    int *tstatus;               /* [tid] */
    atomic_uint_fast64_t next;  /* next partition to take */
    or_task task;
};

typedef struct { or_mt *M; unsigned tid; } or_thread_arg;

static void *or_thread_main(void *p)
{
    or_thread_arg *a = (or_thread_arg *)p;
    a->M->task(a->M, a->tid);
    return NULL;
}

/* Run M->task on every thread id and wait for all of them (thread 0 runs on
 * the calling thread). */
static int or_run(or_mt *M, or_task task)
{
    pthread_t th[OR_MAX_THREADS];
    or_thread_arg arg[OR_MAX_THREADS];
    unsigned started = 1;
    M->task = task;
    atomic_store(&M->next, 0);
    for (unsigned t = 1; t < M->nthreads; t++) {
        arg[t].M = M;
        arg[t].tid = t;
        if (pthread_create(&th[t], NULL, or_thread_main, &arg[t]) != 0) break;
        started++;
    }
    task(M, 0);
    for (unsigned t = 1; t < started; t++) pthread_join(th[t], NULL);
    /* partitions left behind by threads that could not start */
    if (started < M->nthreads)
        for (unsigned t = started; t < M->nthreads; t++) task(M, t);
    return 0;
}

static void or_chunk(const or_mt *M, unsigned tid, uint64_t *lo, uint64_t *hi)
{
    uint64_t n = M->W->n, per = (n + M->nthreads - 1) / M->nthreads;
    *lo = per * tid < n ? per * tid : n;
    *hi = per * (tid + 1) < n ? per * (tid + 1) : n;
}

/* Step 1 on the thread's chunk of keys, counting rows per partition. */
static void or_task_hash(or_mt *M, unsigned tid)
{
    or_work *W = M->W;
    uint64_t lo, hi, *cnt = M->cnt + (uint64_t)tid * M->K;
    or_chunk(M, tid, &lo, &hi);
    for (uint64_t i = lo; i < hi; i++) {
        or_row *row = &M->hashed[i];
        row->key = M->keys[i];
        row->val = M->vals[i] & M->mask;
        or_hash(M->keys[i], M->sigma, W->m, W->w, &row->start, &row->coeff);
        cnt[M->part_of_bucket[row->start / W->B]]++;
    }
}

/* Step 2, first half: the rows of the thread's chunk to their partitions. */
static void or_task_scatter(or_mt *M, unsigned tid)
{
    uint64_t lo, hi, *pos = M->cnt + (uint64_t)tid * M->K;
    or_chunk(M, tid, &lo, &hi);
    for (uint64_t i = lo; i < hi; i++) {
        const or_row *row = &M->hashed[i];
        M->W->rows[pos[M->part_of_bucket[row->start / M->W->B]]++] = *row;
    }
}

/* Step 2, second half, then steps 3 and 4, one partition at a time. */
static void or_task_sort(or_mt *M, unsigned tid)
{
    (void)tid;
    for (uint64_t q; (q = atomic_fetch_add(&M->next, 1)) < M->K;)
        qsort(M->W->rows + M->prow[q], M->prow[q + 1] - M->prow[q], sizeof(or_row), or_row_cmp);
}

static void or_task_insert(or_mt *M, unsigned tid)
{
    for (uint64_t q; (q = atomic_fetch_add(&M->next, 1)) < M->K;) {
        uint64_t nb = 0;
        int rc = or_insert_rows(M->W, M->prow[q], M->prow[q + 1], M->bumped_keys + M->prow[q],
                                M->bumped_vals + M->prow[q], &nb, &M->tstats[tid]);
        M->pbumped[q] = nb;
        if (rc) M->tstatus[tid] = rc;
    }
}

static void or_task_backsub(or_mt *M, unsigned tid)
{
    (void)tid;
    const or_work *W = M->W;
    for (uint64_t q; (q = atomic_fetch_add(&M->next, 1)) < M->K;) {
        /* partition q owns [cut_{q} + w, cut_{q+1} + w): its kept rows start
         * at or after the forced level of its first bucket (>= w) and before
         * the next cut, so their supports stay inside */
        uint64_t s0 = q == 0 ? 0 : W->cuts[q - 1] + W->w;
        uint64_t s1 = q + 1 == M->K ? W->m : W->cuts[q] + W->w;
        if (s1 <= s0) continue;
        if (M->prow[q] == M->prow[q + 1]) {
            /* no rows: every slot it owns is free, so its table words are 0 */
            memset(M->z + (s0 / 64) * W->r, 0, sizeof(uint64_t) * ((s1 - s0) / 64) * W->r);
            continue;
        }
        or_backsub_slots(M->W, s0, s1);
        or_pack_planes(W, s0, s1, M->z);
    }
}

/* Steps 1-4 of a layer with nthreads threads (W set up, rows allocated). */
static int or_layer_steps_mt(or_work *W, const uint64_t *keys, const uint32_t *vals, uint32_t mask,
                             uint64_t sigma, unsigned nthreads, uint64_t *z,
                             uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                             or_stats *st)
{
    or_mt M;
    memset(&M, 0, sizeof(M));
    M.W = W; M.keys = keys; M.vals = vals; M.mask = mask; M.sigma = sigma;
    M.nthreads = nthreads; M.K = W->ncuts + 1; M.z = z;
    M.bumped_keys = bumped_keys; M.bumped_vals = bumped_vals;
    M.part_of_bucket = (uint32_t *)malloc(sizeof(uint32_t) * (W->nb ? W->nb : 1));
    M.hashed = (or_row *)malloc(sizeof(or_row) * W->n);
    M.cnt = (uint64_t *)calloc((uint64_t)nthreads * M.K, sizeof(uint64_t));
    M.prow = (uint64_t *)calloc(M.K + 1, sizeof(uint64_t));
    M.pbumped = (uint64_t *)calloc(M.K, sizeof(uint64_t));
    M.tstats = (or_stats *)calloc(nthreads, sizeof(or_stats));
    M.tstatus = (int *)calloc(nthreads, sizeof(int));
    int status = 0;
    if (!M.part_of_bucket || !M.hashed || !M.cnt || !M.prow || !M.pbumped || !M.tstats || !M.tstatus)
        status = OR_ENOMEM;
    if (status == 0) {
        for (uint64_t b = 0, q = 0; b < W->nb; b++) {
            while (q < W->ncuts && W->cuts[q] <= b * W->B) q++;
            M.part_of_bucket[b] = (uint32_t)q;
        }
        or_run(&M, or_task_hash);
        /* write offsets: partition q's rows of thread t follow those of threads < t */
        uint64_t pos = 0;
        for (uint64_t q = 0; q < M.K; q++) {
            M.prow[q] = pos;
            for (unsigned t = 0; t < nthreads; t++) {
                uint64_t c = M.cnt[(uint64_t)t * M.K + q];
                M.cnt[(uint64_t)t * M.K + q] = pos;
                pos += c;
            }
        }
        M.prow[M.K] = pos;
        or_run(&M, or_task_scatter);
        g_B = W->B;
        or_run(&M, or_task_sort);
        or_run(&M, or_task_insert);
        for (unsigned t = 0; t < nthreads; t++) {
            if (M.tstatus[t]) status = M.tstatus[t];
            if (st) {
                st->xor_steps += M.tstats[t].xor_steps;
                st->inserted += M.tstats[t].inserted;
                if (M.tstats[t].max_drift > st->max_drift) st->max_drift = M.tstats[t].max_drift;
            }
        }
        /* bumped rows in partition order, as the serial insertion emits them */
        for (uint64_t q = 0; q < M.K; q++) {
            memmove(bumped_keys + *nbumped, bumped_keys + M.prow[q], sizeof(uint64_t) * M.pbumped[q]);
            memmove(bumped_vals + *nbumped, bumped_vals + M.prow[q], sizeof(uint32_t) * M.pbumped[q]);
            *nbumped += M.pbumped[q];
        }
        if (status == 0) or_run(&M, or_task_backsub);
    }
    free(M.part_of_bucket); free(M.hashed); free(M.cnt); free(M.prow); free(M.pbumped);
    free(M.tstats); free(M.tstatus);
    return status;
}

/*
 * Build one layer.  keys/vals: n input pairs (vals masked to r bits).
 * m slots, hash seed sigma, cuts[0..ncuts) strictly increasing multiples of B
 * (start slots where a new partition begins; empty = one partition).
 * fallback != 0: base case -- no thresholds, every row must insert.
 * Outputs: thresh[ceil(nb/32)] packed 2-bit codes (ignored for fallback),
 * z[(m/64)*r] interleaved bit planes, bumped keys/vals (capacity n).
 * Returns 0, OR_FAIL (fallback could not solve) or OR_EINVAL.
 */
int or_build_layer(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                   uint32_t r, uint64_t m, uint64_t sigma,
                   const uint32_t levels[4], uint32_t B, uint32_t w,
                   const uint64_t *cuts, uint64_t ncuts, int fallback,
                   uint64_t *thresh, uint64_t *z,
                   uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                   or_stats *st)
{
    return or_build_layer_mode(keys, vals, n, r, m, sigma, levels, B, w, cuts, ncuts, fallback,
                               OR_THRESH_2BIT, thresh, NULL, z, bumped_keys, bumped_vals, nbumped, st);
}

/*
 * One layer in either threshold mode.  2-bit: on the first failure at offset
 * o the bucket's threshold becomes the smallest level above o.  1+-bit: it
 * becomes o + 1 exactly (every row at offsets <= o is bumped, the rows above
 * stay), so the threshold is the least t for which the bucket's rows at
 * offsets >= t can be kept.  The first bucket after a cut starts from the
 * forced threshold: the smallest level >= w (2-bit), exactly w (1+-bit).
 */
int or_build_layer_mode(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                        uint32_t r, uint64_t m, uint64_t sigma,
                        const uint32_t levels[4], uint32_t B, uint32_t w,
                        const uint64_t *cuts, uint64_t ncuts, int fallback,
                        uint32_t mode, uint64_t *thresh, uint8_t *texact, uint64_t *z,
                        uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                        or_stats *st)
{
    return or_build_layer_mt(keys, vals, n, r, m, sigma, levels, B, w, cuts, ncuts, fallback, mode,
                             thresh, texact, z, bumped_keys, bumped_vals, nbumped, st, 1);
}

/* or_build_layer_mode with the partitions spread over nthreads host threads
 * (1 = serial).  The result is the same for every nthreads. */
int or_build_layer_mt(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                      uint32_t r, uint64_t m, uint64_t sigma,
                      const uint32_t levels[4], uint32_t B, uint32_t w,
                      const uint64_t *cuts, uint64_t ncuts, int fallback,
                      uint32_t mode, uint64_t *thresh, uint8_t *texact, uint64_t *z,
                      uint64_t *bumped_keys, uint32_t *bumped_vals, uint64_t *nbumped,
                      or_stats *st, unsigned nthreads)
{
    *nbumped = 0;
    if (n == 0 || m == 0) return 0;
    if (w != 64 || m % 64 != 0 || m < w) return OR_EINVAL;
    uint32_t mask = (r >= 32) ? 0xFFFFFFFFu : ((1u << r) - 1u);
    uint64_t nb = or_num_buckets(m, w, B);
    int forced = or_forced_code(levels, w);
    if (mode == OR_THRESH_2BIT && forced < 0 && ncuts > 0) return OR_EINVAL;
    if (mode != OR_THRESH_2BIT && mode != OR_THRESH_1PLUS) return OR_EINVAL;
    if (mode == OR_THRESH_1PLUS && (B > 255 || (!fallback && !texact))) return OR_EINVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > OR_MAX_THREADS) nthreads = OR_MAX_THREADS;
    const uint32_t t_forced = mode == OR_THRESH_1PLUS ? w : (forced >= 0 ? levels[forced] : 0);

    or_work W;
    memset(&W, 0, sizeof(W));
    W.n = n; W.m = m; W.nb = nb; W.r = r; W.B = B; W.w = w; W.mode = mode;
    W.fallback = fallback; W.forced = forced; W.t_forced = t_forced; W.levels = levels;
    W.cuts = cuts; W.ncuts = fallback ? 0 : ncuts;
    W.rows = (or_row *)malloc(sizeof(or_row) * n);
    W.C = (uint64_t *)calloc(m, sizeof(uint64_t));
    W.Y = (uint32_t *)calloc(m, sizeof(uint32_t));
    W.slot_of = (int64_t *)malloc(sizeof(int64_t) * n);
    W.code_of = (uint8_t *)calloc(nb + 1, 1);
    W.texact = mode == OR_THRESH_1PLUS && !fallback ? texact : NULL;
    W.Zs = (uint32_t *)calloc(m + 64, sizeof(uint32_t));
    int status = 0;
    if (!W.rows || !W.C || !W.Y || !W.slot_of || !W.code_of || !W.Zs) status = OR_ENOMEM;

    /* every bucket that starts a partition j >= 1 carries the forced
     * threshold, also when no key falls into it */
    if (status == 0 && !fallback) {
        if (W.texact) memset(W.texact, 0, nb);
        for (uint64_t q = 0; q < ncuts; q++) {
            uint64_t b = cuts[q] / B;
            if (b >= nb) continue;
            if (W.texact) W.texact[b] = (uint8_t)w;
            else W.code_of[b] = (uint8_t)forced;
        }
    }
    if (status == 0 && nthreads == 1) {
        /* 1. hash every key to its equation */
        for (uint64_t i = 0; i < n; i++) {
            W.rows[i].key = keys[i];
            W.rows[i].val = vals[i] & mask;
            or_hash(keys[i], sigma, m, w, &W.rows[i].start, &W.rows[i].coeff);
        }
        /* 2. sort by start slot (bucket asc, offset desc) */
        g_B = B;
        qsort(W.rows, n, sizeof(or_row), or_row_cmp);
        /* 3. insertion, bucket by bucket */
        status = or_insert_rows(&W, 0, n, bumped_keys, bumped_vals, nbumped, st);
        /* 4. back-substitution, then the table's bit planes */
        if (status == 0) {
            or_backsub_slots(&W, 0, m);
            or_pack_planes(&W, 0, m, z);
        }
    } else if (status == 0) {
        status = or_layer_steps_mt(&W, keys, vals, mask, sigma, nthreads, z, bumped_keys, bumped_vals,
                                   nbumped, st);
    }
    /* 2-bit codes, 32 per word: bucket b in bits [2(b%32), 2(b%32)+2) of word b/32 */
    if (status == 0 && !fallback && mode == OR_THRESH_2BIT) {
        memset(thresh, 0, sizeof(uint64_t) * ((nb + 31) / 32));
        for (uint64_t b = 0; b < nb; b++)
            thresh[b / 32] |= (uint64_t)W.code_of[b] << (2 * (b % 32));
    }
    free(W.rows); free(W.C); free(W.Y); free(W.slot_of); free(W.code_of); free(W.Zs);
    return status;
}

/* Value stored for slot s, plane k, in the interleaved layout. */
static uint32_t or_zbit(const uint64_t *z, uint32_t r, uint64_t s, uint32_t k)
{
    return (uint32_t)((z[(s / 64) * r + k] >> (s % 64)) & 1ULL);
}

/* Query one key against one layer's table: XOR of the r-bit slot values
 * selected by the coefficient bits. */
static uint32_t or_layer_eval(const uint64_t *z, uint32_t r, uint64_t s, uint64_t c)
{
    uint32_t v = 0;
    for (int k = 0; k < 64; k++) {
        if (!((c >> k) & 1ULL)) continue;
        for (uint32_t q = 0; q < r; q++)
            v ^= or_zbit(z, r, s + (uint64_t)k, q) << q;
    }
    return v;
}

/* ------------------------------------------------------------------------ */
/* Cut-point search (Sec. 3, "Selecting Cut Points").                        */
/* ------------------------------------------------------------------------ */

/*
 * Cut j (1 <= j < K) is searched among the buckets b0, b0+1, ..., b0+R-1 with
 * b0 = j*P/B and R = min(range, P/B) (READING: the paper gives only "the
 * number of buckets to be searched"; searching forward from the nominal cut
 * and never a whole partition keeps the cuts increasing).  For a cut at
 * bucket b (slot c = b*B):
 *   bumped(b) = keys with start in [c, c + w)   (cut away by the forced level)
 *   prev(b)   = keys with start in [c - (w-1), c) (the w-1 slots before)
 * minbump minimises bumped(b), maxprev maximises prev(b), diff minimises
 * bumped(b) - prev(b); the first best candidate wins.  OR_CUT_NONE or
 * range <= 1 gives c = j*P.
 */
int or_search_cuts(const uint64_t *keys, uint64_t n, uint64_t m, uint64_t sigma, uint32_t B, uint32_t w,
                   uint64_t P, uint64_t K, uint32_t mode, uint32_t range, uint64_t *cuts)
{
    if (K < 2) return 0;
    for (uint64_t j = 1; j < K; j++) cuts[j - 1] = j * P;
    if (mode == OR_CUT_NONE || range <= 1) return 0;
    uint64_t nb = or_num_buckets(m, w, B);
    /* per bucket: keys at offsets < w, and keys at offsets >= B - (w - 1) */
    uint64_t *lo = (uint64_t *)calloc(nb + 1, sizeof(uint64_t));
    uint64_t *hi = (uint64_t *)calloc(nb + 1, sizeof(uint64_t));
    if (!lo || !hi) { free(lo); free(hi); return OR_ENOMEM; }
    for (uint64_t i = 0; i < n; i++) {
        uint64_t s, c;
        or_hash(keys[i], sigma, m, w, &s, &c);
        uint32_t off = (uint32_t)(s % B);
        if (off < w) lo[s / B]++;
        if (off >= B - (w - 1)) hi[s / B]++;
    }
    uint64_t R = range < P / B ? range : P / B;
    for (uint64_t j = 1; j < K; j++) {
        uint64_t b0 = j * P / B, best_b = b0;
        int64_t best = 0;
        for (uint64_t b = b0; b < b0 + R && b < nb; b++) {
            int64_t bumped = (int64_t)lo[b], prev = b > 0 ? (int64_t)hi[b - 1] : 0;
            int64_t score = mode == OR_CUT_MINBUMP ? bumped : (mode == OR_CUT_MAXPREV ? -prev : bumped - prev);
            if (b == b0 || score < best) { best = score; best_b = b; }
        }
        cuts[j - 1] = best_b * B;
    }
    free(lo); free(hi);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Whole structure.                                                          */
/* ------------------------------------------------------------------------ */

void or_default_params(or_params *p)
{
    memset(p, 0, sizeof(*p));
    p->r = 8;
    p->w = 64;
    p->B = 128;
    p->levels[0] = 0; p->levels[1] = 32; p->levels[2] = 64; p->levels[3] = 128;
    p->alpha = 1.015;   /* calibrated: ~1.0% total overhead at n=2^20, r=8 */
    p->layers = 4;
    p->partition_slots = 65536;
    p->min_partition_slots = 4096;
    p->lower_partition_slots = 4096;
    p->cut_search = OR_CUT_NONE;
    p->cut_search_range = 50;
    p->seed = 0x5EED5EED5EED5EEDULL;
    p->fb_max_retries = 16;
    p->fb_slack = 0.1;
}

void or_free(or_struct *s)
{
    if (!s) return;
    for (uint32_t l = 0; l <= OR_MAX_LAYERS; l++) {
        free(s->layer[l].thresh);
        free(s->layer[l].z);
        free(s->layer[l].texact);
        free(s->layer[l].cuts);
    }
    memset(s, 0, sizeof(*s));
}

/*
 * Build the whole layered structure.  cut_P[l] overrides the partition size
 * of layer l (0 = use params); this lets tests give the oracle explicit cut
 * lists.  Returns 0, OR_UNSOLVABLE, OR_EINVAL or OR_ENOMEM.
 */
int or_build(const uint64_t *keys, const uint32_t *vals, uint64_t n,
             const or_params *p, or_struct *out, or_stats *st)
{
    return or_build_mt(keys, vals, n, p, out, st, 1);
}

/* or_build with each bumping layer's partitions spread over nthreads host
 * threads (1 = serial); the result is the same for every nthreads. */
int or_build_mt(const uint64_t *keys, const uint32_t *vals, uint64_t n,
                const or_params *p, or_struct *out, or_stats *st, unsigned nthreads)
{
    memset(out, 0, sizeof(*out));
    if (p->r < 1 || p->r > 32 || p->w != 64 || p->B % 64 != 0 || p->B < 64 ||
        p->layers > OR_MAX_LAYERS || p->levels[0] != 0 || p->levels[3] != p->B ||
        !(p->levels[0] < p->levels[1] && p->levels[1] < p->levels[2] &&
          p->levels[2] < p->levels[3]) ||
        p->partition_slots % p->B != 0 || p->partition_slots == 0 ||
        p->lower_partition_slots % p->B != 0 ||
        !(p->alpha > 0.0) || or_forced_code(p->levels, p->w) < 0 ||
        (p->threshold_mode != OR_THRESH_2BIT && p->threshold_mode != OR_THRESH_1PLUS) ||
        p->cut_search > OR_CUT_DIFF ||
        (p->threshold_mode == OR_THRESH_1PLUS && p->B > 255))
        return OR_EINVAL;
    out->params = *p;
    out->n = n;
    uint32_t mask = (p->r >= 32) ? 0xFFFFFFFFu : ((1u << p->r) - 1u);

    uint64_t *ck = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint32_t *cv = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint64_t *nk = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    uint32_t *nv = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!ck || !cv || !nk || !nv) { free(ck); free(cv); free(nk); free(nv); return OR_ENOMEM; }
    for (uint64_t i = 0; i < n; i++) { ck[i] = keys[i]; cv[i] = vals[i] & mask; }
    uint64_t cn = n;
    int status = 0;

    for (uint32_t l = 0; l < p->layers && status == 0; l++) {
        or_layer *L = &out->layer[l];
        L->n = cn;
        L->m = or_layer_slots(cn, p->alpha, p->w);
        L->seed_index = l;
        L->nbuckets = or_num_buckets(L->m, p->w, p->B);
        /* READING: one partition per thread with at least minbpt buckets each
         * (Sec. 3) leaves deep layers, which are small, with partitions of
         * just minbpt buckets; here a fixed size per layer stands for that:
         * layer 0 is cut every partition_slots, deeper layers every
         * lower_partition_slots */
        uint64_t P = p->partition_slots;
        if (l > 0 && p->lower_partition_slots) P = p->lower_partition_slots;
        if (p->cut_P[l]) P = p->cut_P[l];
        L->nparts = or_num_partitions(L->m, P, p->min_partition_slots);
        L->part_slots = P;
        uint64_t ncuts = L->nparts ? L->nparts - 1 : 0;
        uint64_t *cuts = (uint64_t *)malloc(sizeof(uint64_t) * (ncuts ? ncuts : 1));
        if (cuts && or_search_cuts(ck, cn, L->m, or_layer_seed(p->seed, l), p->B, p->w, P, L->nparts,
                                   p->cut_search, p->cut_search_range, cuts) != 0) {
            free(cuts);
            cuts = NULL;
        }
        L->cuts = (uint64_t *)malloc(sizeof(uint64_t) * (ncuts ? ncuts : 1));
        if (L->cuts && cuts) memcpy(L->cuts, cuts, sizeof(uint64_t) * ncuts);
        const int onep = p->threshold_mode == OR_THRESH_1PLUS;
        if (onep) L->texact = (uint8_t *)calloc(L->nbuckets + 1, 1);
        else L->thresh = (uint64_t *)calloc((L->nbuckets + 31) / 32 + 1, sizeof(uint64_t));
        L->z = (uint64_t *)calloc((L->m / 64) * p->r + 1, sizeof(uint64_t));
        uint64_t nb = 0;
        if (!cuts || !L->cuts || !(onep ? (void *)L->texact : (void *)L->thresh) || !L->z) status = OR_ENOMEM;
        else
            status = or_build_layer_mt(ck, cv, cn, p->r, L->m,
                                       or_layer_seed(p->seed, l), p->levels, p->B, p->w,
                                       cuts, ncuts, 0, p->threshold_mode, L->thresh, L->texact,
                                       L->z, nk, nv, &nb, st, nthreads);
        free(cuts);
        L->nbumped = nb;
        if (st) st->bumped[l] = nb;
        uint64_t *tk = ck; ck = nk; nk = tk;
        uint32_t *tv = cv; cv = nv; nv = tv;
        cn = nb;
    }

    /* base case: no bumping, grow until it solves */
    if (status == 0) {
        or_layer *F = &out->layer[OR_MAX_LAYERS];
        F->n = cn;
        status = OR_UNSOLVABLE;
        for (uint32_t a = 0; a <= p->fb_max_retries; a++) {
            free(F->z);
            F->m = or_fallback_slots(cn, p->fb_slack, p->w, a);
            F->seed_index = p->layers + a;
            F->nbuckets = or_num_buckets(F->m, p->w, p->B);
            F->nparts = F->m ? 1 : 0;
            F->z = (uint64_t *)calloc((F->m / 64) * p->r + 1, sizeof(uint64_t));
            if (!F->z) { status = OR_ENOMEM; break; }
            uint64_t nb = 0;
            int rc = or_build_layer(ck, cv, cn, p->r, F->m,
                                    or_layer_seed(p->seed, F->seed_index), p->levels,
                                    p->B, p->w, NULL, 0, 1, NULL, F->z, nk, nv, &nb, st);
            if (rc == 0) { status = 0; out->fb_attempt = a; break; }
            if (rc != OR_FAIL) { status = rc; break; }
        }
    }
    free(ck); free(cv); free(nk); free(nv);
    if (status) or_free(out);
    return status;
}

/* Query: walk the layers; a key whose offset lies below its bucket's
 * threshold was bumped and continues in the next layer. */
uint32_t or_query_one(const or_struct *s, uint64_t key)
{
    const or_params *p = &s->params;
    for (uint32_t l = 0; l < p->layers; l++) {
        const or_layer *L = &s->layer[l];
        if (L->m == 0) return 0;
        uint64_t st, c;
        or_hash(key, or_layer_seed(p->seed, L->seed_index), L->m, p->w, &st, &c);
        uint64_t b = st / p->B;
        uint32_t off = (uint32_t)(st % p->B);
        uint32_t t;
        if (p->threshold_mode == OR_THRESH_1PLUS) {
            t = L->texact[b];
        } else {
            uint32_t code = (uint32_t)((L->thresh[b / 32] >> (2 * (b % 32))) & 3ULL);
            t = p->levels[code];
        }
        if (off < t) continue;
        return or_layer_eval(L->z, p->r, st, c);
    }
    const or_layer *F = &s->layer[OR_MAX_LAYERS];
    if (F->m == 0) return 0;
    uint64_t st, c;
    or_hash(key, or_layer_seed(p->seed, F->seed_index), F->m, p->w, &st, &c);
    return or_layer_eval(F->z, p->r, st, c);
}

void or_query(const or_struct *s, const uint64_t *keys, uint32_t *out, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++) out[i] = or_query_one(s, keys[i]);
}

/* ------------------------------------------------------------------------ */
/* Canonical export: little-endian u32/u64 fields, then the arrays.          */
/* ------------------------------------------------------------------------ */

static uint8_t *put32(uint8_t *q, uint32_t v) { memcpy(q, &v, 4); return q + 4; }
static uint8_t *put64(uint8_t *q, uint64_t v) { memcpy(q, &v, 8); return q + 8; }

/* Number of buckets of a 1+-bit layer that bump anything (flag bit set). */
static uint64_t or_flagged(const or_layer *L)
{
    uint64_t c = 0;
    for (uint64_t b = 0; b < L->nbuckets; b++) c += L->texact[b] != 0;
    return c;
}

/* Bytes of one bumping layer's threshold section in the export. */
static uint64_t or_thresh_bytes(const or_params *p, const or_layer *L)
{
    if (p->threshold_mode == OR_THRESH_1PLUS)
        return 8 * ((L->nbuckets + 63) / 64) + 8 + 8 * ((or_flagged(L) + 7) / 8);
    return 8 * ((L->nbuckets + 31) / 32);
}

/*
 * Version 1 (2-bit thresholds): per bumping layer the 2-bit code words.
 * Version 2 (1+-bit thresholds): per bumping layer the flag words (bit b%64
 * of word b/64 set iff bucket b bumps anything), a u64 count of flagged
 * buckets, then their exact thresholds as bytes in bucket order, zero-padded
 * to a multiple of 8 bytes.
 */
uint64_t or_export(const or_struct *s, uint8_t *buf, uint64_t cap)
{
    const or_params *p = &s->params;
    const int onep = p->threshold_mode == OR_THRESH_1PLUS;
    uint64_t need = 4 * 10 + 8 * 4 + (uint64_t)p->layers * 8 * 5 + 8 * 4;
    for (uint32_t l = 0; l < p->layers; l++)
        need += or_thresh_bytes(p, &s->layer[l]) + 8 * (s->layer[l].m / 64) * p->r;
    need += 8 * (s->layer[OR_MAX_LAYERS].m / 64) * p->r;
    if (!buf || cap < need) return need;
    uint8_t *q = buf;
    q = put32(q, 0x52525542u); /* "BURR" */
    q = put32(q, onep ? 2 : 1);
    q = put32(q, p->r); q = put32(q, p->w); q = put32(q, p->B); q = put32(q, p->layers);
    for (int i = 0; i < 4; i++) q = put32(q, p->levels[i]);
    uint64_t abits; memcpy(&abits, &p->alpha, 8);
    q = put64(q, p->seed); q = put64(q, abits); q = put64(q, s->n);
    q = put64(q, p->partition_slots);
    for (uint32_t l = 0; l < p->layers; l++) {
        const or_layer *L = &s->layer[l];
        q = put64(q, L->n); q = put64(q, L->m); q = put64(q, L->nparts);
        q = put64(q, L->nbuckets); q = put64(q, L->nbumped);
    }
    const or_layer *F = &s->layer[OR_MAX_LAYERS];
    q = put64(q, F->n); q = put64(q, F->m); q = put64(q, F->seed_index);
    q = put64(q, s->fb_attempt);
    for (uint32_t l = 0; l < p->layers; l++) {
        const or_layer *L = &s->layer[l];
        if (onep) {
            uint64_t nw = (L->nbuckets + 63) / 64, cnt = or_flagged(L);
            memset(q, 0, 8 * nw);
            for (uint64_t b = 0; b < L->nbuckets; b++)
                if (L->texact[b]) q[b / 8] |= (uint8_t)(1u << (b % 8));   /* little-endian words */
            q += 8 * nw;
            q = put64(q, cnt);
            uint64_t padded = 8 * ((cnt + 7) / 8), k = 0;
            memset(q, 0, padded);
            for (uint64_t b = 0; b < L->nbuckets; b++)
                if (L->texact[b]) q[k++] = L->texact[b];
            q += padded;
        } else {
            uint64_t nw = (L->nbuckets + 31) / 32;
            memcpy(q, L->thresh, 8 * nw); q += 8 * nw;
        }
        uint64_t nz = (L->m / 64) * p->r;
        memcpy(q, L->z, 8 * nz); q += 8 * nz;
    }
    uint64_t nz = (F->m / 64) * p->r;
    memcpy(q, F->z, 8 * nz); q += 8 * nz;
    return (uint64_t)(q - buf);
}

/* Space accounting: bits of all tables and thresholds, over r*n. */
double or_overhead(const or_struct *s)
{
    const or_params *p = &s->params;
    if (s->n == 0) return 0.0;
    double bits = 0;
    /* thresholds: 2 bits per bucket, or 1 bit per bucket plus 8 bits per
     * bucket that bumps (the exact threshold, 1..B) */
    for (uint32_t l = 0; l < p->layers; l++) {
        const or_layer *L = &s->layer[l];
        bits += (double)L->m * p->r;
        if (p->threshold_mode == OR_THRESH_1PLUS)
            bits += (double)L->nbuckets + 8.0 * (double)or_flagged(L);
        else
            bits += 2.0 * (double)L->nbuckets;
    }
    bits += (double)s->layer[OR_MAX_LAYERS].m * p->r;
    return bits / ((double)p->r * (double)s->n) - 1.0;
}

/* Accessors for the ctypes wrapper. */
const or_layer *or_get_layer(const or_struct *s, uint32_t l) { return &s->layer[l]; }
uint64_t or_struct_size(void) { return sizeof(or_struct); }
uint64_t or_stats_size(void) { return sizeof(or_stats); }
uint64_t or_params_size(void) { return sizeof(or_params); }
uint64_t or_layer_size(void) { return sizeof(or_layer); }
