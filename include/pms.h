/*
 * pms.h -- C ABI of the GB300 library for exact planted (l,d)-motif search.
 *
 * The problem (paper: "Formal Definitions of qPMS", Definitions 1-5 and the
 * qPMS definition with quorum q = n, i.e. the PMS problem): given n DNA
 * sequences s_1..s_n of length m and integers l, d, report every l-mer M over
 * {A,C,G,T} such that each s_i has an l-mer (a window s_i[j..j+l-1]) within
 * Hamming distance d of M.
 *
 * All entry points return 0 (PMS_OK) or a negative PMS_E* code; none throws
 * or aborts. A context is used by one call at a time (calls on one context
 * are serialised by an internal mutex); distinct contexts are independent.
 *
 * Sequences are passed as row-major n x m arrays of the ASCII bytes 'A', 'C',
 * 'G', 'T' (any other byte is PMS_EINVAL). Motifs are returned as 64-bit
 * codes, 2 bits per base (A=0, C=1, G=2, T=3, the order of the paper's
 * compression example), position 0 in the most significant used bits, so
 * ascending codes are lexicographic order; pms_decode turns one back into
 * text. Every motif set is returned sorted ascending and without duplicates.
 *
 * Limits of this build: 1 <= l <= 32 (one 32-bit word per bit-plane),
 * 0 <= d < l, 1 <= n <= 64, l <= m <= 65536.
 */
#ifndef PMS_H
#define PMS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PMS_OK 0
#define PMS_EINVAL (-1)    /* bad argument or a byte that is not A/C/G/T */
#define PMS_ENOMEM (-2)    /* device memory budget or allocation exhausted */
#define PMS_ECUDA (-3)     /* a CUDA call failed; pms_last_error has the text */
#define PMS_ETIMEDOUT (-4) /* pms_wait: the ticket did not complete in time */
#define PMS_ETOOMANY (-5)  /* more motifs (with duplicates) than the result
                              capacity; count still holds the raw count */
#define PMS_EBUSY (-6)     /* the served queue is full */
#define PMS_ENOTFOUND (-7) /* unknown or already released ticket */
#define PMS_ESCRATCH (-8)  /* instance too large for the fixed scratch of
                              pms_solve_device_noalloc */
#define PMS_ECANCELED (-9) /* pms_wait: the ticket was withdrawn by pms_cancel */

#define PMS_LMAX 32
#define PMS_NMAX 64

typedef struct pms_ctx pms_ctx;

/* One problem instance. seqs: host memory, row-major n x m ASCII. */
typedef struct {
    const uint8_t *seqs;
    int n, m, l, d;
} pms_instance;

/* The answer for one instance. motifs points into memory owned by the
 * context (pms_solve, pms_solve_batch: valid until the next solve call on
 * the context or pms_destroy) or by the ticket (pms_wait: valid until
 * pms_release of that ticket or pms_destroy). */
typedef struct {
    int status;             /* PMS_OK or a negative code for this instance */
    const uint64_t *motifs; /* sorted unique motif codes */
    size_t count;           /* number of motifs (raw count on PMS_ETOOMANY) */
} pms_result;

/* Tunables. Zero in any field selects the default (or the tuned value). */
typedef struct {
    int ctas_per_sm;       /* resident CTAs of the verification kernel per SM */
    int chunk_work;        /* target work of one queue item, in candidate units */
    int grab;              /* tree-node filter: 0 = the tuned value, else 1;
                              1 = lane-asynchronous walk: every lane takes one
                              node through the rows, leaves a row at the
                              node's own first feasible occurrence and takes
                              the next node at once (default); g > 1 =
                              breadth-first batches of up to 128 nodes that
                              shrink to g nodes as a queue item runs out
                              (g >= 128: fixed batches of 128) */
    size_t max_motifs;     /* raw motif capacity per instance (rounded to 2^k) */
    int count_work;        /* 1: also count comparisons (slower; for profiling) */
    int serve_wave_items;  /* served form: size of a verification wave in units of
                              65536 candidate units (0: about 6.4e9 units) */
    int serve_max_inflight;/* served form: requests resident on the device */
    int smem_rows;         /* at most this many feasible occurrences of a seed are
                              kept in shared memory (0: as many as fit); a seed
                              with up to three times as many keeps only their
                              mismatch masks there and reads their planes from
                              global memory; larger row sets are read from
                              global memory */
    int autotune;          /* 1: tune each new instance class before solving it */
    int seed_mode;         /* 0: every seed x of s_1 searches B(x, d) as a tree
                              (Observation 3.1); 1: pair seeds (x in s_1, r in s_2,
                              d_H(x, r) <= 2d) search B(x, d) & B(r, d)
                              (Observation 3.3), except seeds with a pair
                              closer than d + 1, which keep the tree form.
                              Plain and batched solves; the served and
                              allocation-free forms use 0. */
    int quorum;            /* q of the qPMS problem (Definition 5): report the
                              l-mers within d of at least q of the n sequences.
                              0 or q >= n: q = n, the PMS problem. With q < n the
                              seeds are the l-mers of s_1..s_{n-q+1}
                              (Observation 3.1) and every candidate may miss up
                              to n - q sequences. Plain and batched solves; the
                              served and allocation-free forms solve q = n. */
    int partial_rows;      /* one more level of the tree T_d(x) between a node P
                              (its set of changed positions) and its leaves: the
                              letters on the changed positions above the three
                              lowest are fixed first, and such a partial
                              candidate is kept only if each of the first
                              partial_rows rows (smallest first) holds an
                              occurrence that a leaf below it could still reach
                              within d; only the kept partials' leaves are
                              tested (the row shrinking of the paper's
                              depth-first search, one level deep).
                              0: tuned value, else the default (8 rows when
                              d >= 5 and fewer than 0.15 windows of a random
                              sequence are expected within d of a candidate;
                              none otherwise); -1: no partial
                              level; k > 0: k rows. Tree form, q = n. */
    int graph;             /* solves (pms_solve, pms_solve_device,
                              pms_solve_batch) replay a CUDA graph captured
                              on the second call of each plan (the same
                              instance shapes and options), with the call's
                              input and output pointers patched in:
                              0 = on (default), replays carry no timing
                              events: pms_stats.ms_kernel and ms_verify read
                              -1 after a replay (an event node between two
                              kernels costs their launch overlap, about
                              17 us per plain (15,4) solve on GB300);
                              1 = on, with the device-time events recorded
                              inside the graph; -1 = launch kernel by kernel
                              (device times always recorded) */
    int triple_rows;       /* three-string feasibility below a tree node (the
                              TraverStringRef feasibility theorem for three
                              strings, applied to the seed x and pairs of
                              occurrences): an occurrence u of the smallest
                              row is kept for a node only if, for each of the
                              next triple_rows rows, some occurrence w leaves
                              a string of the node within d of both u and w;
                              the node is dropped when no u is left, and its
                              leaves meet only the kept u. Tree form, q = n.
                              0: the default (d >= 4 and fewer than 0.25
                              windows of a random sequence expected within d
                              of a candidate: 4 rows, 8 when d >= 5; off
                              otherwise); -1: off; k > 0: k rows. */
} pms_options;

/* A tuned schedule for one instance class (l, d, n rounded up to a power of
 * two, m rounded up to a power of two). */
typedef struct {
    int chunk_work;   /* candidate units per queue item */
    int prune_rows;   /* rows the tree-node filter applies before leaves are expanded */
    int ctas_per_sm;  /* resident CTAs of the verification kernel */
    int grab;         /* node batch policy (as pms_options.grab) */
    int partial_rows; /* rows tested at the partial-candidate level (-1: none) */
    double ms;        /* device time of the pipeline on the tuning instance */
} pms_tuning;

/* Work counters of the last solve (pms_solve / pms_solve_device /
 * pms_solve_batch / pms_solve_sigma). For the DNA solves the comparison
 * counters are filled only when pms_options.count_work was set for that
 * solve; pms_solve_sigma always fills them (subsets = tree nodes visited,
 * candidates_tested = checks of full candidates, cmp_rows / cmp_reduce /
 * cmp_verify = window, node-bound and candidate-versus-row comparisons). */
typedef struct {
    uint64_t candidates;        /* size of the searched space: sum over seeds of |B(x,d)| */
    uint64_t subsets;           /* position subsets visited (tree nodes at which substitutions start) */
    uint64_t subsets_pruned;    /* subsets dismissed by the feasible-occurrence bound */
    uint64_t candidates_tested; /* candidates compared explicitly against occurrences */
    uint64_t cmp_rows;          /* l-mer comparisons building feasible-occurrence rows */
    uint64_t cmp_reduce;        /* comparisons applying the subset bound to rows */
    uint64_t cmp_verify;        /* candidate-versus-occurrence comparisons */
    uint64_t seeds_infeasible;  /* seeds with an empty row (no motif possible) */
    double ms_total;            /* wall time of the call, host clock */
    double ms_kernel;           /* device time from the first to the last kernel;
                                   -1 after a graph replay with pms_options.graph = 0 */
    double ms_verify;           /* device time of the verification kernel alone (-1 as ms_kernel) */
    uint64_t serve_waves;       /* served form, cumulative: verification waves launched */
    uint64_t serve_overlapped_waves;     /* waves holding chunks of more than one request */
    uint64_t serve_max_requests_per_wave;
    uint64_t graph_replays;     /* cumulative: solves enqueued by replaying a captured graph */
} pms_stats;

/* Creates a context on CUDA device `device`. mem_budget_bytes caps the device
 * memory the context may hold (0 = no cap beyond the device's). The context
 * owns a CUDA stream until pms_set_stream replaces it. */
int pms_create(pms_ctx **out, int device, size_t mem_budget_bytes);

/* Issue all further work on `cuda_stream` (a cudaStream_t, e.g. a PyTorch
 * stream's handle); NULL returns to the context's own stream. */
int pms_set_stream(pms_ctx *h, void *cuda_stream);

/* Route the context's device allocations through alloc/free (e.g. a caching
 * allocator). alloc(bytes, user) returns a device pointer or NULL;
 * free_(ptr, user) releases it. Must be called before the first solve. */
int pms_set_allocator(pms_ctx *h, void *(*alloc)(size_t bytes, void *user),
                      void (*free_)(void *ptr, void *user), void *user);

int pms_set_options(pms_ctx *h, const pms_options *opt);
int pms_get_options(const pms_ctx *h, pms_options *opt);

/* Solves one instance from host memory (Definitions 1-5 with q = n; the
 * candidate set is the union of B(x, d) over the l-mers x of s_1,
 * Observation 3.1). seqs: host, read only during the call. On success
 * *motifs points to *count sorted unique codes owned by h (valid until the
 * next solve on h or pms_destroy). Blocks until the result is on the host.
 * Bytes other than A/C/G/T are detected by the packing kernel: the call
 * then returns PMS_EINVAL, with *count = 0, and pms_last_error names the
 * first such byte. The bytes are copied into a pinned host buffer of the
 * context. For small instances (n*m*max(l, (m-l+1)/16) up to 1 MiB) the
 * packing kernel reads them there, and result blocks of up to 1 MiB are
 * written by the sort kernel into another pinned buffer, so such a call
 * issues no copy of its own; larger ones are copied each way. */
int pms_solve(pms_ctx *h, const uint8_t *seqs, int n, int m, int l, int d,
              const uint64_t **motifs, size_t *count);

/* Device-resident form of pms_solve: d_seqs is a device pointer to n*m
 * ASCII bytes; the sorted unique codes are written to d_motifs (device,
 * room for `capacity` codes) and d_status (device, 4 x uint32) receives
 * {raw count, unique count, flags, 0}; flags bit 0 = invalid byte in the
 * input, bit 1 = raw motifs exceeded the context's max_motifs. Enqueued on
 * the context's stream; returns without waiting. Inputs are read and outputs
 * written only by kernels on that stream. */
int pms_solve_device(pms_ctx *h, const uint8_t *d_seqs, int n, int m, int l, int d,
                     uint64_t *d_motifs, size_t capacity, uint32_t *d_status);

/* General alphabets (the "Sigma" of qPMS-Sigma, chapter "Our Approach"):
 * the (l,d,q)-motifs of n strings over an alphabet of sigma letters
 * (Definitions 1-5), e.g. the twenty amino acids of protein sequences.
 *   alphabet: host, sigma distinct bytes (no terminator needed), 2 <= sigma
 *             <= 32; letter a of the alphabet has index a, and every
 *             l-mer is compressed into ceil(log2 sigma) bit-planes
 *             (section "String Compression").
 *   seqs:     host, row-major n x m bytes, each one of the alphabet's letters;
 *             read only during the call.
 *   q:        quorum (0 or n: every string must hold an occurrence, the PMS
 *             problem; 1 <= q < n: at least q strings, seeds then taken from
 *             s_1..s_{n-q+1} by Observation 3.1).
 * Limits: those of pms_solve (1 <= n <= PMS_NMAX, 1 <= l <= PMS_LMAX,
 * l <= m <= 65536, 0 <= d < l) and d <= 16.
 * On success *motifs points to *count motifs of l bytes each (letters of the
 * alphabet, motif after motif, no separators), sorted lexicographically by
 * letter index (the alphabet's own order) and unique; the memory is owned by
 * h and valid until the next pms_solve_sigma on h or pms_destroy. The raw
 * candidate buffer holds max_motifs keys (default 65536) and grows once, up
 * to 2^22, when the first pass needs more; past that (or past an explicit
 * max_motifs) the call returns PMS_ETOOMANY with *count = the raw count.
 * Errors: PMS_EINVAL (null pointer, bad sigma, repeated letter, a byte not in
 * the alphabet, parameters out of range), PMS_ENOMEM, PMS_ECUDA,
 * PMS_ETOOMANY. Blocks until the result is on the host; pms_get_stats then
 * reports this solve's counters (always counted) and device times. */
int pms_solve_sigma(pms_ctx *h, const uint8_t *alphabet, int sigma, const uint8_t *seqs, int n, int m, int l,
                    int d, int q, const uint8_t **motifs, size_t *count);

/* Solves k independent instances in one pass: one upload, one packing
 * launch, one persistent verification launch whose CTAs take (instance,
 * seed, chunk) items from a device work queue, one segmented sort/unique
 * launch, one download. out[i] receives instance i's result (memory owned
 * by h as for pms_solve). Returns PMS_OK if the batch ran; per-instance
 * errors are in out[i].status. */
int pms_solve_batch(pms_ctx *h, const pms_instance *inst, int k, pms_result *out);

/* Served form (continuous batching). pms_submit validates and copies the
 * instance and returns a ticket at once; the first submit on a context
 * starts its scheduler thread, its own CUDA stream and a request pool (a
 * device block of up to 1 GiB, at most half of what the budget leaves).
 * The scheduler admits requests in arrival order while a slot
 * (serve_max_inflight, default 64) and pool room are free, and launches
 * verification waves whose work queue holds chunks of every admitted request
 * (oldest first, about serve_wave_items x 65536 candidate units per wave):
 * a request that arrives while others run joins the next wave, so their work
 * overlaps on the device. pms_wait blocks up to timeout_ms (negative: no
 * limit) for the ticket's result; PMS_ETIMEDOUT leaves the ticket valid.
 * pms_release frees a completed ticket (PMS_EBUSY while it is running). */
int pms_submit(pms_ctx *h, const pms_instance *inst, uint64_t *ticket);
int pms_wait(pms_ctx *h, uint64_t ticket, int timeout_ms, pms_result *out);
int pms_release(pms_ctx *h, uint64_t ticket);

/* Served form: withdraws a ticket that is still queued (not yet admitted to
 * the device). Its pms_wait then reports status PMS_ECANCELED, and
 * pms_release frees it as usual. Returns PMS_OK (also for a ticket that has
 * already finished: its result stands), PMS_EBUSY (admitted: it runs to
 * completion), PMS_ENOTFOUND. No counterpart in the paper. */
int pms_cancel(pms_ctx *h, uint64_t ticket);

/* Fault injection for tests of the error paths (no counterpart in the
 * paper). Host-side only: the failing call is never made, so no GPU fault
 * is involved. After `after` further operations of `kind` succeed, the next
 * `count` fail (count 0 clears the injection):
 *   PMS_FAULT_ALLOC   device allocations of the context fail, so the call
 *                     that needs the memory returns PMS_ENOMEM;
 *   PMS_FAULT_UPLOAD  uploads of input sequences fail: a pms_solve or
 *                     pms_solve_batch call returns PMS_ECUDA, a served
 *                     request ends with status PMS_ECUDA (other requests
 *                     are not affected).
 * Returns PMS_OK or PMS_EINVAL. */
#define PMS_FAULT_ALLOC 1
#define PMS_FAULT_UPLOAD 2
int pms_inject_fault(pms_ctx *h, int kind, int after, int count);

/* Autotuner (no counterpart in the paper; it picks the schedule of the
 * verification kernel). pms_autotune times the device pipeline on a
 * synthetic instance of the class (n, m, l, d) (uniform random bases) for a
 * few settings, coordinate by coordinate: rows applied by the tree-node
 * filter, work per queue item, CTAs per SM, node batch policy; the best is
 * kept in the context
 * for the class (l, d, n and m rounded up to powers of two) and used by every
 * later solve of that class, and copied to *out when out is non-null.
 * pms_save_tuning / pms_load_tuning write / read the context's table as text
 * (one class per line). Options chunk_work / ctas_per_sm, when set,
 * override the tuned values. */
int pms_autotune(pms_ctx *h, int n, int m, int l, int d, pms_tuning *out);
int pms_save_tuning(const pms_ctx *h, const char *path);
int pms_load_tuning(pms_ctx *h, const char *path);

/* Work counters and timing of the last solve. Waits for that solve's kernels
 * if they are still running and it recorded device-time events; a graph
 * replayed with pms_options.graph = 0 records none, and its ms_kernel /
 * ms_verify read -1 without waiting. */
int pms_get_stats(const pms_ctx *h, pms_stats *out);

/* Writes the l letters of `code` and a terminating NUL to out (l + 1 bytes). */
int pms_decode(uint64_t code, int l, char *out);

/* Text of the last error on h (empty string if none); valid until the next
 * call on h. */
const char *pms_last_error(const pms_ctx *h);

/* Measures the issue rate of one integer instruction class on the context's
 * device with a dedicated probe kernel: kind 0 = POPC, 1 = LOP3, 2 = IADD3,
 * 3 = IMNMX (min). *per_clk_per_sm receives results per SM per SM clock
 * (thread-level operations), from `clock64` deltas inside the kernel. */
int pms_probe_int_rate(pms_ctx *h, int kind, double *per_clk_per_sm);

/* The architecture the library's device code was built for, as the CUDA
 * runtime reports it for the packing kernel on `device`
 * (cudaFuncGetAttributes binaryVersion: major * 10 + minor, 103 for
 * sm_103a). No counterpart in the paper; a build check. Returns PMS_OK,
 * PMS_EINVAL (null pointer) or PMS_ECUDA (no such device, or no device code
 * for it). */
int pms_kernel_binary_version(int device, int *version);

/* Releases the context, its device memory, stream and scheduler thread. */
void pms_destroy(pms_ctx *h);

/* Allocation-free form of pms_solve_device, for callers that may not
 * allocate device memory once they are running: applications whose device
 * memory is planned up front and handed out only by their own allocator,
 * and hosts in which cudaMalloc/cudaFree are off limits because they can
 * block, synchronize the device or fail under memory pressure at a time the
 * caller cannot control. The paper has no counterpart; this is plumbing.
 *
 * It needs no context. Every intermediate buffer (window planes,
 * compatibility masks, raw motif codes and their sort buffer, counters,
 * descriptors, per-CTA row scratch) is carved from one fixed array of
 * 16 MiB that the library's device code reserves on each GPU it is loaded
 * on and holds until the process exits; nothing is allocated per call.
 * The caller passes, as for pms_solve_device, device pointers to the n*m
 * ASCII input bytes, to room for `capacity` motif codes (d_motifs), and to
 * 4 x uint32 of status {raw count, unique count, flags, 0}; the work is
 * enqueued on `cuda_stream` (NULL: the legacy default stream) of the
 * current device and the call returns without waiting. The call's small
 * descriptor block travels inside the launches' parameters, so no host
 * memory of the call is read after it returns.
 *
 * Limits: besides the pms_solve_device limits, the instance's buffers plus
 * the row scratch of at least one CTA must fit in the 16 MiB (n = 20,
 * m = 600 needs about 2 MiB plus 0.13 MiB per CTA, and gets about 100
 * CTAs); larger instances return PMS_ESCRATCH before any work is queued.
 * At most 65536 raw motif codes (duplicates included) are kept: more set
 * status flag bit 1, as with max_motifs.
 *
 * Set-up: the first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and loads the kernels' constant tables
 * with that device current; make that first call before any stream capture
 * is begun. All calls share the one array and it keeps whatever the last
 * call left there (the counters a call relies on are cleared at its start),
 * so calls whose work overlaps on the GPU -- on different streams, or from
 * different threads without ordering -- race and corrupt each other's
 * results; order them on one stream. Returns PMS_OK, PMS_EINVAL,
 * PMS_ESCRATCH or PMS_ECUDA. */
int pms_solve_device_noalloc(const uint8_t *d_seqs, int n, int m, int l, int d, uint64_t *d_motifs,
                             size_t capacity, uint32_t *d_status, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PMS_H */
