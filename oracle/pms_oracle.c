/*
 * pms_oracle.c -- plain CPU oracle for exact planted (l,d)-motif search
 * (the PMS problem: qPMS with quorum q = n).
 *
 * TEST INFRASTRUCTURE ONLY. The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark load this file; the GPU library neither links
 * nor includes it, and nothing here includes GPU code. It shares no header,
 * helper or table with the GPU path.
 *
 * It is deliberately slow and literal: l-mers are compared character by
 * character, the search space is walked with nested loops/recursion, motifs
 * are gathered in a growable array that is sorted and de-duplicated at the
 * end. Every entry point names the definition or observation of the paper it
 * restates (section "Formal Definitions of qPMS", chapter "Our Approach").
 *
 * Conventions (the paper's readings used throughout):
 *   - alphabet order A < C < G < T, coded 0,1,2,3 as in the paper's
 *     compression example (AGGCTA -> 022130);
 *   - an l-mer of s is s[j..j+l-1] for every j in 0..m-l (Definition 2 read
 *     with its index range fixed to 1 <= i <= m-l+1);
 *   - "within d" means Hamming distance <= d (Definition 5: no more than d);
 *   - a motif set is reported as sorted, unique 64-bit keys holding 2 bits per
 *     base with position 0 in the most significant used bits, so ascending
 *     keys are lexicographic order;
 *   - the oracle_sigma_* functions at the end restate the same definitions
 *     over a general alphabet of 2..32 letters (the "Sigma" of qPMS-Sigma),
 *     reporting motifs as letters in the alphabet's own order.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)

static int code_of(uint8_t ch)
{
    switch (ch) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
    }
}

static const uint8_t LETTER[4] = {'A', 'C', 'G', 'T'};

/* Definition 3: number of positions at which two equal-length strings differ. */
int oracle_hamming(const uint8_t *a, const uint8_t *b, int l)
{
    int h = 0;
    for (int k = 0; k < l; ++k)
        if (a[k] != b[k])
            h += 1;
    return h;
}

/* Definition 4: distance from an l-mer x to a string s = minimum over the
 * l-mers of s (all m-l+1 windows). Returns l+1 if s is shorter than x. */
int oracle_distance_to_string(const uint8_t *x, int l, const uint8_t *s, int m)
{
    int best = l + 1;
    for (int j = 0; j + l <= m; ++j) {
        int h = oracle_hamming(x, s + j, l);
        if (h < best)
            best = h;
    }
    return best;
}

/* "d_H(x, s) <= d": true iff some window of s is within d of x. Same predicate
 * as oracle_distance_to_string(...) <= d, stopping at the first window found. */
static int string_has_occurrence(const uint8_t *x, int l, int d, const uint8_t *s, int m)
{
    for (int j = 0; j + l <= m; ++j)
        if (oracle_hamming(x, s + j, l) <= d)
            return 1;
    return 0;
}

/* Definition 5 with q = n: M is an (l,d)-motif of s_1..s_n iff every string
 * is within d of M. seqs is row-major n x m. */
int oracle_is_motif(const uint8_t *M, int l, int d, const uint8_t *seqs, int n, int m)
{
    for (int i = 0; i < n; ++i)
        if (!string_has_occurrence(M, l, d, seqs + (size_t)i * m, m))
            return 0;
    return 1;
}

/* Definition 5 for general q: M is an (l,d,q)-motif iff at least q of the n
 * strings are within d of M. */
int oracle_is_qmotif(const uint8_t *M, int l, int d, int q, const uint8_t *seqs, int n, int m)
{
    int hits = 0, misses = 0;
    for (int i = 0; i < n; ++i) {
        if (string_has_occurrence(M, l, d, seqs + (size_t)i * m, m))
            hits += 1;
        else
            misses += 1;
        if (hits >= q)
            return 1;          /* q strings found: it is a motif */
        if (misses > n - q)
            return 0;          /* fewer than q strings can remain */
    }
    return 0;
}

/* ---- bit-plane compression (chapter "Our Approach", "String Compression") ----
 * An l-mer is stored as ceil(log2 |Sigma|) = 2 groups of ceil(l/32) 32-bit
 * words; bit g of the code of character k goes to bit (k mod 32) of word
 * (k div 32) of group g. The distance of two compressed l-mers: XOR the two
 * copies of each group, OR the XOR results across groups, count the set bits.
 * out must hold 2*ceil(l/32) words: group 0 first, then group 1. */
int oracle_compress(const uint8_t *s, int l, uint32_t *out)
{
    int words = (l + 31) / 32;
    for (int w = 0; w < 2 * words; ++w)
        out[w] = 0;
    for (int k = 0; k < l; ++k) {
        int c = code_of(s[k]);
        if (c < 0)
            return ORACLE_EINVAL;
        for (int g = 0; g < 2; ++g)
            if ((c >> g) & 1)
                out[g * words + k / 32] |= (uint32_t)1 << (k % 32);
    }
    return ORACLE_OK;
}

static int count_set_bits(uint32_t v)
{
    int c = 0;
    while (v) {
        c += (int)(v & 1u);
        v >>= 1;
    }
    return c;
}

int oracle_compressed_distance(const uint32_t *a, const uint32_t *b, int l)
{
    int words = (l + 31) / 32;
    int h = 0;
    for (int w = 0; w < words; ++w) {
        uint32_t acc = 0;
        for (int g = 0; g < 2; ++g)
            acc |= a[g * words + w] ^ b[g * words + w];
        h += count_set_bits(acc);
    }
    return h;
}

/* ---- result sets ---- */

typedef struct {
    uint64_t *v;
    long n, cap;
    int oom;
} keyvec;

static void kv_push(keyvec *kv, uint64_t key)
{
    if (kv->oom)
        return;
    if (kv->n == kv->cap) {
        long nc = kv->cap ? 2 * kv->cap : 256;
        uint64_t *nv = (uint64_t *)realloc(kv->v, (size_t)nc * sizeof(uint64_t));
        if (!nv) {
            kv->oom = 1;
            return;
        }
        kv->v = nv;
        kv->cap = nc;
    }
    kv->v[kv->n++] = key;
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Sorts, removes duplicates, copies up to cap keys to out. Returns the number
 * of unique keys (which may exceed cap: then only cap were written). */
static long kv_finish(keyvec *kv, uint64_t *out, long cap)
{
    if (kv->oom) {
        free(kv->v);
        return ORACLE_ENOMEM;
    }
    qsort(kv->v, (size_t)kv->n, sizeof(uint64_t), cmp_u64);
    long u = 0;
    for (long i = 0; i < kv->n; ++i)
        if (u == 0 || kv->v[i] != kv->v[u - 1])
            kv->v[u++] = kv->v[i];
    for (long i = 0; i < u && i < cap; ++i)
        out[i] = kv->v[i];
    free(kv->v);
    return u;
}

/* Key of an l-mer: 2 bits per base, position 0 most significant. */
uint64_t oracle_key(const uint8_t *x, int l)
{
    uint64_t key = 0;
    for (int k = 0; k < l; ++k)
        key = (key << 2) | (uint64_t)code_of(x[k]);
    return key;
}

void oracle_decode(uint64_t key, int l, uint8_t *out)
{
    for (int k = l - 1; k >= 0; --k) {
        out[k] = LETTER[key & 3u];
        key >>= 2;
    }
}

static int valid_input(const uint8_t *seqs, int n, int m, int l, int d)
{
    if (n < 1 || l < 1 || l > 32 || m < l || d < 0 || d >= l)
        return 0;
    for (long k = 0; k < (long)n * m; ++k)
        if (code_of(seqs[k]) < 0)
            return 0;
    return 1;
}

/* ---- the d-neighbourhood B(x, d) as the tree T_d(x) of qPMSPrune ----
 * ("Previous Works", qPMSPrune: the root is x, a child differs from its parent
 * at one position to the right of the parent's last change, so a node at depth
 * h is at distance h from x; depth is at most d). Every string of B(x, d) is
 * visited exactly once. */

typedef struct {
    const uint8_t *x;   /* root l-mer */
    int q;              /* quorum used by the motif test (0: all n strings) */
    uint8_t *cur;       /* the node being visited (x with some changes) */
    int l, d;
    /* what to do with each node */
    const uint8_t *seqs;
    int n, m;
    const uint8_t *other;   /* if non-NULL: keep only nodes within d of it */
    int mode;               /* 0: motif test, 1: collect every node */
    keyvec *out;
    long visited;
    const struct packed_seqs *pk;   /* if non-NULL: the motif test on compressed l-mers */
} walk_t;

/* Every window of every sequence in compressed form (Sec. "String
 * Compression"): for l <= 32 one word per group, group 0 (bit 0 of the codes)
 * in lo[], group 1 (bit 1) in hi[], window j of string i at i * W + j. */
typedef struct packed_seqs {
    uint32_t *lo, *hi;
    int n, W, l, d;
} packed_seqs;

static int packed_build(packed_seqs *pk, const uint8_t *seqs, int n, int m, int l, int d)
{
    pk->n = n;
    pk->W = m - l + 1;
    pk->l = l;
    pk->d = d;
    pk->lo = (uint32_t *)malloc((size_t)n * pk->W * sizeof(uint32_t));
    pk->hi = (uint32_t *)malloc((size_t)n * pk->W * sizeof(uint32_t));
    if (!pk->lo || !pk->hi)
        return ORACLE_ENOMEM;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < pk->W; ++j) {
            uint32_t g[2];
            oracle_compress(seqs + (long)i * m + j, l, g);
            pk->lo[(long)i * pk->W + j] = g[0];
            pk->hi[(long)i * pk->W + j] = g[1];
        }
    return ORACLE_OK;
}

static void packed_free(packed_seqs *pk)
{
    free(pk->lo);
    free(pk->hi);
}

/* Definition 5 (q = n) on compressed l-mers: every string holds a window
 * whose compressed distance to the candidate (set bits of the OR of the two
 * groups' XORs) is at most d. The strings are taken in the order s_2, ...,
 * s_n, s_1; the order of a conjunction does not change its value. */
static int packed_is_motif(const packed_seqs *pk, const uint32_t cand[2])
{
    for (int t = 1; t <= pk->n; ++t) {
        const int i = t % pk->n;
        const uint32_t *lo = pk->lo + (long)i * pk->W, *hi = pk->hi + (long)i * pk->W;
        int found = 0;
        for (int j = 0; j < pk->W && !found; ++j)
            found = __builtin_popcount((cand[0] ^ lo[j]) | (cand[1] ^ hi[j])) <= pk->d;
        if (!found)
            return 0;
    }
    return 1;
}

static void visit_node(walk_t *w)
{
    w->visited += 1;
    if (w->other && oracle_hamming(w->cur, w->other, w->l) > w->d)
        return;
    if (w->pk) {
        uint32_t g[2];
        oracle_compress(w->cur, w->l, g);
        if (packed_is_motif(w->pk, g))
            kv_push(w->out, oracle_key(w->cur, w->l));
        return;
    }
    if (w->mode == 1 ||
        (w->q > 0 ? oracle_is_qmotif(w->cur, w->l, w->d, w->q, w->seqs, w->n, w->m)
                  : oracle_is_motif(w->cur, w->l, w->d, w->seqs, w->n, w->m)))
        kv_push(w->out, oracle_key(w->cur, w->l));
}

static void walk_tree(walk_t *w, int first_pos, int depth)
{
    visit_node(w);
    if (depth == w->d)
        return;
    for (int p = first_pos; p < w->l; ++p) {
        uint8_t orig = w->cur[p];
        for (int b = 0; b < 4; ++b) {
            if (LETTER[b] == w->x[p])
                continue;
            w->cur[p] = LETTER[b];
            walk_tree(w, p + 1, depth + 1);
        }
        w->cur[p] = orig;
    }
}

/* B(x, d) itself, as sorted keys (notation table: the sphere B(a, R)). */
long oracle_neighbourhood(const uint8_t *x, int l, int d, uint64_t *out, long cap)
{
    if (l < 1 || l > 32 || d < 0)
        return ORACLE_EINVAL;
    uint8_t cur[32];
    memcpy(cur, x, (size_t)l);
    keyvec kv = {0};
    walk_t w = {x, 0, cur, l, d, NULL, 0, 0, NULL, 1, &kv, 0};
    walk_tree(&w, 0, 0);
    return kv_finish(&kv, out, cap);
}

/* Number of nodes the tree walk of B(x, d) visits (each string once, so this
 * equals |B(x, d)|). */
long oracle_neighbourhood_visits(const uint8_t *x, int l, int d)
{
    if (l < 1 || l > 32 || d < 0)
        return ORACLE_EINVAL;
    uint8_t cur[32];
    memcpy(cur, x, (size_t)l);
    keyvec kv = {0};
    walk_t w = {x, 0, cur, l, d, NULL, 0, 0, NULL, 1, &kv, 0};
    walk_tree(&w, 0, 0);
    free(kv.v);
    return w.visited;
}

/* |B(x, d) intersect B(r, d)|, by walking B(x, d) and testing each node. */
long oracle_pair_intersection_size(const uint8_t *x, const uint8_t *r, int l, int d)
{
    uint8_t cur[32];
    memcpy(cur, x, (size_t)l);
    keyvec kv = {0};
    walk_t w = {x, 0, cur, l, d, NULL, 0, 0, r, 1, &kv, 0};
    walk_tree(&w, 0, 0);
    long n = kv.n;
    free(kv.v);
    return n;
}

/* ---- PMS solvers ---- */

typedef struct {
    const uint8_t *seqs;
    int n, m, l, d;
    int q;              /* quorum (0: n, the PMS problem) */
    int variant;        /* 0: seeds x in S_1; 1: pairs (x in S_1, r in S_2);
                           2: seeds x in S_1, motif test on compressed l-mers */
    int tid, nthreads;
    long seed_lo, seed_hi;   /* range of windows of s_1 used as seeds */
    keyvec out;
    const packed_seqs *pk;   /* variant 2 */
} job_t;

static void *solve_worker(void *arg)
{
    job_t *j = (job_t *)arg;
    const uint8_t *s1 = j->seqs;
    const uint8_t *s2 = j->n > 1 ? j->seqs + j->m : NULL;
    uint8_t cur[32];
    const long W = (long)j->m - j->l + 1;
    for (long x0 = j->seed_lo + j->tid; x0 < j->seed_hi; x0 += j->nthreads) {
        /* seed x0 numbers the l-mers of s_1, s_2, ... in order (W per string) */
        const uint8_t *x = s1 + (x0 / W) * (long)j->m + (x0 % W);
        if (j->variant != 1 || s2 == NULL) {
            /* Observation 3.1 with q = n: every motif is within d of some
             * l-mer x of s_1, so the candidates are the union of B(x, d). */
            memcpy(cur, x, (size_t)j->l);
            walk_t w = {x, j->q, cur, j->l, j->d, j->seqs, j->n, j->m, NULL, 0, &j->out, 0,
                        j->variant == 2 ? j->pk : NULL};
            walk_tree(&w, 0, 0);
        } else {
            /* Observation 3.3 with q = n: a motif is within d of an l-mer x
             * of s_1 and of an l-mer r of s_2, so it lies in
             * B(x, d) intersect B(r, d), and then d_H(x, r) <= 2d. */
            for (int r0 = 0; r0 + j->l <= j->m; ++r0) {
                const uint8_t *r = s2 + r0;
                if (oracle_hamming(x, r, j->l) > 2 * j->d)
                    continue;
                memcpy(cur, x, (size_t)j->l);
                walk_t w = {x, 0, cur, j->l, j->d, j->seqs, j->n, j->m, r, 0, &j->out, 0};
                walk_tree(&w, 0, 0);
            }
        }
    }
    return NULL;
}

static long run_solver(const uint8_t *seqs, int n, int m, int l, int d, int q, int variant,
                       long seed_lo, long seed_hi, int threads, uint64_t *out, long cap)
{
    if (!valid_input(seqs, n, m, l, d) || q < 0 || q > n)
        return ORACLE_EINVAL;
    long W = (long)m - l + 1;
    /* Observation 3.1: seeds from the l-mers of s_1..s_{n-q+1} (only s_1 for q = n) */
    const long nseeds = (q > 0 ? (long)(n - q + 1) : 1L) * W;
    if (seed_lo < 0)
        seed_lo = 0;
    if (seed_hi > nseeds)
        seed_hi = nseeds;
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    packed_seqs pk = {0};
    if (variant == 2 && packed_build(&pk, seqs, n, m, l, d) != ORACLE_OK) {
        packed_free(&pk);
        return ORACLE_ENOMEM;
    }
    job_t *jobs = (job_t *)calloc((size_t)threads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        packed_free(&pk);
        return ORACLE_ENOMEM;
    }
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (job_t){seqs, n, m, l, d, q, variant, t, threads, seed_lo, seed_hi, {0}, &pk};
        if (threads == 1 || pthread_create(&th[t], NULL, solve_worker, &jobs[t]) != 0) {
            solve_worker(&jobs[t]);
            th[t] = 0;
        }
    }
    keyvec all = {0};
    for (int t = 0; t < threads; ++t) {
        if (th[t])
            pthread_join(th[t], NULL);
        if (jobs[t].out.oom)
            all.oom = 1;
        for (long i = 0; i < jobs[t].out.n; ++i)
            kv_push(&all, jobs[t].out.v[i]);
        free(jobs[t].out.v);
    }
    free(jobs);
    free(th);
    packed_free(&pk);
    return kv_finish(&all, out, cap);
}

/* All (l,d)-motifs of seqs (n x m, row-major ASCII), seeds x over all of S_1.
 * Returns the number of motifs (sorted unique keys in out, at most cap written)
 * or a negative error. */
long oracle_solve(const uint8_t *seqs, int n, int m, int l, int d, int threads,
                  uint64_t *out, long cap)
{
    return run_solver(seqs, n, m, l, d, 0, 0, 0, (long)m - l + 1, threads, out, cap);
}

/* The motifs lying in B(x, d) for the seeds x = s_1[j..j+l-1], j in
 * [seed_lo, seed_hi): a bounded slice of oracle_solve's work. */
long oracle_solve_seeds(const uint8_t *seqs, int n, int m, int l, int d, long seed_lo,
                        long seed_hi, int threads, uint64_t *out, long cap)
{
    return run_solver(seqs, n, m, l, d, 0, 0, seed_lo, seed_hi, threads, out, cap);
}

/* The same motif set through pairs (x in S_1, r in S_2, d_H(x,r) <= 2d). */
long oracle_solve_pairs(const uint8_t *seqs, int n, int m, int l, int d, int threads,
                        uint64_t *out, long cap)
{
    return run_solver(seqs, n, m, l, d, 0, 1, 0, (long)m - l + 1, threads, out, cap);
}

/* oracle_solve_pairs restricted to the seeds x = s_1[j..j+l-1], j in
 * [seed_lo, seed_hi): a bounded slice of its work. */
long oracle_solve_pairs_seeds(const uint8_t *seqs, int n, int m, int l, int d, long seed_lo, long seed_hi,
                              int threads, uint64_t *out, long cap)
{
    return run_solver(seqs, n, m, l, d, 0, 1, seed_lo, seed_hi, threads, out, cap);
}

/* The motifs lying in B(x, d) for the seeds x = s_1[j..j+l-1], j in
 * [seed_lo, seed_hi), as oracle_solve_seeds, with the motif test of
 * Definition 5 run on compressed l-mers (Sec. "String Compression": every
 * window is compressed once, a candidate's distance to it is the set bits of
 * the OR of the XORed groups, equal to Definition 3). Same result, a few
 * times faster; used to write expected motif sets of large instances. */
long oracle_solve_packed(const uint8_t *seqs, int n, int m, int l, int d, long seed_lo, long seed_hi, int threads,
                         uint64_t *out, long cap)
{
    return run_solver(seqs, n, m, l, d, 0, 2, seed_lo, seed_hi, threads, out, cap);
}

/* qPMS (the qPMS definition, quorum q <= n): all (l,d,q)-motifs. Seeds are
 * the l-mers of s_1..s_{n-q+1} (Observation 3.1: a string within d of at
 * least q strings is within d of one of any n - q + 1 of them). */
long oracle_solve_quorum(const uint8_t *seqs, int n, int m, int l, int d, int q, int threads, uint64_t *out,
                         long cap)
{
    if (q < 1)
        return ORACLE_EINVAL;
    return run_solver(seqs, n, m, l, d, q, 0, 0, (long)(n - q + 1) * (m - l + 1), threads, out, cap);
}

/* The (l,d,q)-motifs lying in B(x, d) for seeds x numbered
 * [seed_lo, seed_hi) over the l-mers of s_1, s_2, ... (W per string). */
long oracle_solve_quorum_seeds(const uint8_t *seqs, int n, int m, int l, int d, int q, long seed_lo, long seed_hi,
                               int threads, uint64_t *out, long cap)
{
    if (q < 1)
        return ORACLE_EINVAL;
    return run_solver(seqs, n, m, l, d, q, 0, seed_lo, seed_hi, threads, out, cap);
}

/* Pattern-driven exhaustive search with a quorum: all 4^l strings tested
 * with oracle_is_qmotif. Only for tiny l. */
long oracle_bruteforce_quorum(const uint8_t *seqs, int n, int m, int l, int d, int q, uint64_t *out, long cap)
{
    if (!valid_input(seqs, n, m, l, d) || l > 12 || q < 1 || q > n)
        return ORACLE_EINVAL;
    keyvec kv = {0};
    uint8_t cand[32];
    uint64_t total = (uint64_t)1 << (2 * l);
    for (uint64_t key = 0; key < total; ++key) {
        oracle_decode(key, l, cand);
        if (oracle_is_qmotif(cand, l, d, q, seqs, n, m))
            kv_push(&kv, key);
    }
    return kv_finish(&kv, out, cap);
}

/* Pattern-driven exhaustive search ("Exact PMS Algorithms", pattern driven
 * approach): test all 4^l strings. Only for tiny l. */
long oracle_bruteforce(const uint8_t *seqs, int n, int m, int l, int d, uint64_t *out, long cap)
{
    if (!valid_input(seqs, n, m, l, d) || l > 12)
        return ORACLE_EINVAL;
    keyvec kv = {0};
    uint8_t cand[32];
    uint64_t total = (uint64_t)1 << (2 * l);
    for (uint64_t key = 0; key < total; ++key) {
        oracle_decode(key, l, cand);
        if (oracle_is_motif(cand, l, d, seqs, n, m))
            kv_push(&kv, key);
    }
    return kv_finish(&kv, out, cap);
}

/* ==== general alphabets (chapter "Our Approach": qPMS-Sigma) ====
 * The same definitions over an alphabet Sigma given as sigma distinct bytes,
 * 2 <= sigma <= 32; letter b of the alphabet has index b, and motif sets are
 * ordered lexicographically by index (for the alphabet "ACGT" this is the
 * order above). Motifs come back as l bytes each, in that order, unique. */

static int sigma_index(const uint8_t *alphabet, int sigma, uint8_t ch)
{
    for (int b = 0; b < sigma; ++b)
        if (alphabet[b] == ch)
            return b;
    return -1;
}

static int valid_alphabet(const uint8_t *alphabet, int sigma)
{
    if (!alphabet || sigma < 2 || sigma > 32)
        return 0;
    for (int a = 0; a < sigma; ++a)
        for (int b = a + 1; b < sigma; ++b)
            if (alphabet[a] == alphabet[b])
                return 0;
    return 1;
}

/* ceil(log2 sigma): the number of bit-plane groups of the compression. */
int oracle_sigma_groups(int sigma)
{
    int g = 0;
    while ((1 << g) < sigma)
        g += 1;
    return g;
}

/* String Compression for a general alphabet: ceil(log2 sigma) groups of
 * ceil(l/32) words; bit g of the index of character k goes to bit (k mod 32)
 * of word (k div 32) of group g. out holds groups * ceil(l/32) words. */
int oracle_sigma_compress(const uint8_t *alphabet, int sigma, const uint8_t *s, int l, uint32_t *out)
{
    if (!valid_alphabet(alphabet, sigma))
        return ORACLE_EINVAL;
    int words = (l + 31) / 32, groups = oracle_sigma_groups(sigma);
    for (int w = 0; w < groups * words; ++w)
        out[w] = 0;
    for (int k = 0; k < l; ++k) {
        int c = sigma_index(alphabet, sigma, s[k]);
        if (c < 0)
            return ORACLE_EINVAL;
        for (int g = 0; g < groups; ++g)
            if ((c >> g) & 1)
                out[g * words + k / 32] |= (uint32_t)1 << (k % 32);
    }
    return ORACLE_OK;
}

/* Distance of two compressed l-mers: XOR group by group, OR across groups,
 * count the set bits. */
int oracle_sigma_compressed_distance(const uint32_t *a, const uint32_t *b, int l, int groups)
{
    int words = (l + 31) / 32;
    int h = 0;
    for (int w = 0; w < words; ++w) {
        uint32_t acc = 0;
        for (int g = 0; g < groups; ++g)
            acc |= a[g * words + w] ^ b[g * words + w];
        h += count_set_bits(acc);
    }
    return h;
}

/* Growable array of motifs as 32-byte records of letter indices (zero padded,
 * so byte-wise comparison is the lexicographic order by index). */
typedef struct {
    uint8_t *v;
    long n, cap;
    int oom;
} recvec;

static void rv_push(recvec *rv, const uint8_t *rec)
{
    if (rv->oom)
        return;
    if (rv->n == rv->cap) {
        long nc = rv->cap ? 2 * rv->cap : 256;
        uint8_t *nv = (uint8_t *)realloc(rv->v, (size_t)nc * 32);
        if (!nv) {
            rv->oom = 1;
            return;
        }
        rv->v = nv;
        rv->cap = nc;
    }
    memcpy(rv->v + (size_t)rv->n * 32, rec, 32);
    rv->n += 1;
}

static int cmp_rec(const void *a, const void *b)
{
    return memcmp(a, b, 32);
}

/* Sorts and de-duplicates the records and writes up to cap motifs (l letters
 * each) to out. Returns the number of unique motifs (may exceed cap). */
static long rv_finish(recvec *rv, const uint8_t *alphabet, int l, uint8_t *out, long cap)
{
    if (rv->oom) {
        free(rv->v);
        return ORACLE_ENOMEM;
    }
    qsort(rv->v, (size_t)rv->n, 32, cmp_rec);
    long u = 0;
    for (long i = 0; i < rv->n; ++i)
        if (u == 0 || memcmp(rv->v + (size_t)i * 32, rv->v + (size_t)(u - 1) * 32, 32) != 0)
            memmove(rv->v + (size_t)u++ * 32, rv->v + (size_t)i * 32, 32);
    for (long i = 0; i < u && i < cap; ++i)
        for (int k = 0; k < l; ++k)
            out[(size_t)i * l + k] = alphabet[rv->v[(size_t)i * 32 + k]];
    free(rv->v);
    return u;
}

static int valid_sigma_input(const uint8_t *alphabet, int sigma, const uint8_t *seqs, int n, int m, int l, int d,
                             int q)
{
    if (!valid_alphabet(alphabet, sigma) || n < 1 || l < 1 || l > 32 || m < l || d < 0 || d >= l || q < 0 || q > n)
        return 0;
    for (long k = 0; k < (long)n * m; ++k)
        if (sigma_index(alphabet, sigma, seqs[k]) < 0)
            return 0;
    return 1;
}

/* B(x, d) over Sigma as the tree T_d(x) of qPMSPrune: a child changes one
 * position to the right of its parent's last change to one of the sigma - 1
 * other letters. */
typedef struct {
    const uint8_t *alphabet;
    int sigma;
    const uint8_t *x;
    uint8_t *cur;
    int l, d, q;           /* q = 0: all n strings */
    const uint8_t *seqs;
    int n, m;
    int mode;              /* 0: motif test, 1: collect every node */
    recvec *out;
    long visited;
} swalk_t;

static void sigma_visit(swalk_t *w)
{
    w->visited += 1;
    if (w->mode == 1 ||
        (w->q > 0 ? oracle_is_qmotif(w->cur, w->l, w->d, w->q, w->seqs, w->n, w->m)
                  : oracle_is_motif(w->cur, w->l, w->d, w->seqs, w->n, w->m))) {
        uint8_t rec[32] = {0};
        for (int k = 0; k < w->l; ++k)
            rec[k] = (uint8_t)sigma_index(w->alphabet, w->sigma, w->cur[k]);
        rv_push(w->out, rec);
    }
}

static void sigma_walk(swalk_t *w, int first_pos, int depth)
{
    sigma_visit(w);
    if (depth < w->d) {
        for (int p = first_pos; p < w->l; ++p) {
            uint8_t orig = w->cur[p];
            for (int b = 0; b < w->sigma; ++b) {
                if (w->alphabet[b] == w->x[p])
                    continue;
                w->cur[p] = w->alphabet[b];
                sigma_walk(w, p + 1, depth + 1);
            }
            w->cur[p] = orig;
        }
    }
}

/* Number of nodes the walk of B(x, d) over Sigma visits (= |B(x, d)|). */
long oracle_sigma_neighbourhood_visits(const uint8_t *alphabet, int sigma, const uint8_t *x, int l, int d)
{
    if (!valid_alphabet(alphabet, sigma) || l < 1 || l > 32 || d < 0)
        return ORACLE_EINVAL;
    uint8_t cur[32];
    memcpy(cur, x, (size_t)l);
    recvec rv = {0};
    swalk_t w = {alphabet, sigma, x, cur, l, d, 0, NULL, 0, 0, 1, &rv, 0};
    sigma_walk(&w, 0, 0);
    free(rv.v);
    return w.visited;
}

typedef struct {
    const uint8_t *alphabet;
    int sigma;
    const uint8_t *seqs;
    int n, m, l, d, q;
    int tid, nthreads;
    long seed_lo, seed_hi;
    recvec out;
} sjob_t;

static void *sigma_worker(void *arg)
{
    sjob_t *j = (sjob_t *)arg;
    uint8_t cur[32];
    const long W = (long)j->m - j->l + 1;
    for (long x0 = j->seed_lo + j->tid; x0 < j->seed_hi; x0 += j->nthreads) {
        /* Observation 3.1: every (l,d,q)-motif is within d of an l-mer of one
         * of s_1..s_{n-q+1}; seeds are numbered over those strings, W each */
        const uint8_t *x = j->seqs + (x0 / W) * (long)j->m + (x0 % W);
        memcpy(cur, x, (size_t)j->l);
        swalk_t w = {j->alphabet, j->sigma, x, cur, j->l, j->d, j->q, j->seqs, j->n, j->m, 0, &j->out, 0};
        sigma_walk(&w, 0, 0);
    }
    return NULL;
}

/* All (l,d,q)-motifs over Sigma (q = 0 or q = n: the PMS problem) lying in
 * B(x, d) for the seeds x numbered [seed_lo, seed_hi) over the l-mers of
 * s_1..s_{n-q+1}; seed_hi < 0 means all seeds. out receives up to cap motifs
 * of l bytes; returns their number or a negative error. */
long oracle_sigma_solve_seeds(const uint8_t *alphabet, int sigma, const uint8_t *seqs, int n, int m, int l, int d,
                              int q, long seed_lo, long seed_hi, int threads, uint8_t *out, long cap)
{
    if (!valid_sigma_input(alphabet, sigma, seqs, n, m, l, d, q))
        return ORACLE_EINVAL;
    if (q == n)
        q = 0;
    const long W = (long)m - l + 1;
    const long nseeds = (long)(q > 0 ? n - q + 1 : 1) * W;
    if (seed_lo < 0)
        seed_lo = 0;
    if (seed_hi < 0 || seed_hi > nseeds)
        seed_hi = nseeds;
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    sjob_t *jobs = (sjob_t *)calloc((size_t)threads, sizeof(sjob_t));
    pthread_t *th = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!jobs || !th) {
        free(jobs);
        free(th);
        return ORACLE_ENOMEM;
    }
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (sjob_t){alphabet, sigma, seqs, n, m, l, d, q, t, threads, seed_lo, seed_hi, {0}};
        if (threads == 1 || pthread_create(&th[t], NULL, sigma_worker, &jobs[t]) != 0) {
            sigma_worker(&jobs[t]);
            th[t] = 0;
        }
    }
    recvec all = {0};
    for (int t = 0; t < threads; ++t) {
        if (th[t])
            pthread_join(th[t], NULL);
        if (jobs[t].out.oom)
            all.oom = 1;
        for (long i = 0; i < jobs[t].out.n; ++i)
            rv_push(&all, jobs[t].out.v + (size_t)i * 32);
        free(jobs[t].out.v);
    }
    free(jobs);
    free(th);
    return rv_finish(&all, alphabet, l, out, cap);
}

long oracle_sigma_solve(const uint8_t *alphabet, int sigma, const uint8_t *seqs, int n, int m, int l, int d, int q,
                        int threads, uint8_t *out, long cap)
{
    return oracle_sigma_solve_seeds(alphabet, sigma, seqs, n, m, l, d, q, 0, -1, threads, out, cap);
}

/* Pattern-driven exhaustive search over Sigma: all sigma^l strings, each
 * tested against Definition 5. Only for sigma^l <= 2^24. */
long oracle_sigma_bruteforce(const uint8_t *alphabet, int sigma, const uint8_t *seqs, int n, int m, int l, int d,
                             int q, uint8_t *out, long cap)
{
    if (!valid_sigma_input(alphabet, sigma, seqs, n, m, l, d, q))
        return ORACLE_EINVAL;
    double total = 1.0;
    for (int k = 0; k < l; ++k)
        total *= sigma;
    if (total > (double)(1 << 24))
        return ORACLE_EINVAL;
    if (q == n)
        q = 0;
    recvec rv = {0};
    uint8_t idx[32] = {0}, cand[32];
    for (;;) {
        for (int k = 0; k < l; ++k)
            cand[k] = alphabet[idx[k]];
        if (q > 0 ? oracle_is_qmotif(cand, l, d, q, seqs, n, m) : oracle_is_motif(cand, l, d, seqs, n, m))
            rv_push(&rv, idx);
        /* next string: base-sigma counter, last position fastest */
        int k = l - 1;
        while (k >= 0 && idx[k] == sigma - 1)
            idx[k--] = 0;
        if (k < 0)
            break;
        idx[k] += 1;
    }
    return rv_finish(&rv, alphabet, l, out, cap);
}
