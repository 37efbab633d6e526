// pms_internal.h -- device data layout shared by the kernels (pms_kernels.cu)
// and the host runtime (pms_runtime.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pms {

constexpr int kLMax = 32;      // one 32-bit word per bit-plane
constexpr int kNMax = 64;      // sequences per instance
constexpr int kWarps = 8;      // warps per CTA of the packing, mask and pair kernels
constexpr int kThreads = kWarps * 32;
// Warps per CTA of the verification kernel.
#ifndef PMS_MAIN_WARPS
#define PMS_MAIN_WARPS 8
#endif
constexpr int kMainWarps = PMS_MAIN_WARPS;
constexpr int kMainThreads = kMainWarps * 32;
constexpr int kRbCap = 128;    // entries of a subset-reduced occurrence row kept in shared memory
constexpr int kListCap = 192;  // surviving candidates a warp buffers before checking further rows
constexpr int kSubBatch = 128; // tree nodes (position subsets) a warp filters together
constexpr int kRowSmemCap = 2560;  // feasible occurrences of one seed held in shared memory (padded)
constexpr int kRowSmemCapSmall = 1280;  // the same in the 4-CTAs-per-SM form of the verification kernel

// Flags reported per instance.
constexpr uint32_t kFlagInvalidByte = 1u;
constexpr uint32_t kFlagOverflow = 2u;

// One instance as the kernels see it. Offsets index the arenas below.
struct InstDev {
    int n, m, l, d;
    int W;                 // windows per sequence: m - l + 1
    int NW;                // 32-bit words of one compatibility mask row: ceil(W / 32)
    int cps;               // queue chunks per seed
    int grab;              // 0: fixed node batches; 1: lane-asynchronous walk; > 1: guided batches shrinking to this size
    int ctab;              // offset (ints) of this instance's table in the chunk arena:
                           //   levoff[0..d+1] then cps pairs (g0, g1)
    int prune_rows;        // rows checked for a feasible occurrence before leaves are tested
    long long seq_off;     // byte offset of the n x m input bytes in the sequence arena
    long long plane_off;   // offset (uint2) of the n x W window planes
    long long raw_off;     // offset (uint64) of the raw motif buffer (and of its sort twin)
    long long compat_off;  // offset (uint32) of the W x (n-1) x NW compatibility masks
    long long rlen_off;    // offset (int) of the W x (n-1) row sizes (set bits of each mask row)
    long long seed_off;    // offset of this instance's seeds in the per-seed mode array
    int cps_b;             // pair mode: queue items per seed (blocks of 64 windows of s_2)
    int q;                 // quorum: a motif needs q of the n sequences (q = n: PMS)
    int nseed;             // sequences whose l-mers are seeds: n - q + 1
    int partial_rows;      // rows a partial candidate (letters fixed above the 3 lowest changed positions)
                           //   is tested against before its leaves; 0: no partial level
    uint32_t raw_cap;      // capacity of the raw motif buffer (power of two)
    int triple_rows;       // rows after the first whose occurrences are tested in pairs with the first
                           //   row's (three-string feasibility below a node); 0: no such test
};

// A contiguous range of queue items: chunks [chunk_lo, chunk_hi) of instance
// `inst`; work_lo is the global item index of chunk_lo. cps == 0: the
// instance's chunking (chunk c is chunk c % cps of seed c / cps); cps > 0: this
// segment's own, chunk c being chunk c % cps of seed seed_lo + c / cps, with
// the chunk table at ctab.
struct Segment {
    long long work_lo;
    int inst;
    int chunk_lo, chunk_hi;
    int cps;
    int seed_lo;
    int ctab;
};

// Per-instance status written by the sort/unique kernel.
struct StatusDev {
    uint32_t raw_count;    // motifs emitted, duplicates included
    uint32_t unique_count; // motifs after sort/unique (written to the dense output)
    uint32_t flags;
    uint32_t dense_off;    // first code of this instance in the dense output
};

// Work counters (count mode), indices into a uint64 array.
enum Counter {
    kCntSubsets = 0,
    kCntPruned,
    kCntTested,
    kCntCmpRows,
    kCntCmpReduce,
    kCntCmpVerify,
    kCntSeedsInfeasible,
    kCntNum
};

struct MainParams {
    const InstDev *inst;
    const Segment *seg;
    int nseg;
    long long total;              // queue items in this launch
    unsigned long long *head;     // queue head (zeroed before the launch)
    const uint2 *planes;
    const uint32_t *compat;       // seed x row compatibility masks (d_H <= 2d)
    const int *rowlen;            // seed x row sizes of those masks
    const int *ctab;
    uint64_t *raw;                // raw motif codes
    uint32_t *raw_count;          // per instance
    uint32_t *flags;              // per instance
    uint32_t *scratch;            // per CTA: 3 * rows_cap words (masks, then planes), used when a
                                  // seed's rows exceed shared memory
    int rows_cap;                 // max (n - 1) * (W + 3) over the instances, rounded up to a multiple of 4
    int smem_rows_cap;            // row entries a seed may keep in shared memory (<= kRowSmemCap)
    unsigned long long *counters; // kCntNum entries (count mode)
    const uint8_t *mode;          // per seed: 0 = tree over B(x, d), 1 = pairs (x, r); null: all 0
    // Node-level work sharing of the lane walk (null: each item's nodes are
    // claimed by its own CTA only). Per queue item g (zeroed before the
    // launch): item_claim[2g] = nodes claimed so far, item_claim[2g + 1] = the
    // nodes its claimers last saw unclaimed (a hint for CTAs looking for work).
    // steal_state[0]: cursor of the candidates examined by CTAs whose queue ran
    // out; steal_state[1]: items whose nodes are all claimed.
    int *item_claim;
    unsigned int *steal_state;
};

// Seed modes of the pair form.
constexpr uint8_t kModeTree = 0;
constexpr uint8_t kModePair = 1;

// Launch wrappers (pms_kernels.cu).
cudaError_t launch_pack(const InstDev *inst, int ninst, const long long *win_prefix, long long total_windows,
                        const uint8_t *seqs, uint2 *planes, uint32_t *flags, int blocks, cudaStream_t st);
cudaError_t launch_compat(const InstDev *inst, int ninst, const long long *row_prefix, long long total_rows,
                          const uint2 *planes, uint32_t *compat, int *rowlen, int blocks, cudaStream_t st);
// One-instance form of launch_pack + launch_compat: a CTA per (sequence, 16
// seeds) packs the sequence's windows in shared memory (W <= the staging
// capacity), writes the planes and builds the masks; bytes other than A/C/G/T
// set flags[0].
bool compat_rows_fits(int W);
cudaError_t launch_compat_rows(const InstDev *inst, int n, long long seeds, const uint8_t *seqs, uint2 *planes,
                               uint32_t *compat, int *rowlen, uint32_t *flags, cudaStream_t st);
const void *compat_rows_kernel_fn();
// small_rows: the form with kRowSmemCapSmall row entries in shared memory and
// 4 resident CTAs per SM (for instances whose seeds have few feasible
// occurrences); otherwise kRowSmemCap entries and 3 CTAs per SM.
cudaError_t launch_main(const MainParams &p, int blocks, bool count_mode, cudaStream_t st, bool small_rows = false);
cudaError_t launch_pairs(const MainParams &p, int blocks, bool count_mode, cudaStream_t st);
cudaError_t pairs_occupancy(int *blocks_per_sm, bool count_mode);
cudaError_t launch_classify(const InstDev *inst, int ninst, const long long *seed_prefix, long long total_seeds,
                            const uint2 *planes, const uint32_t *compat, uint8_t *mode, int blocks, cudaStream_t st);
cudaError_t main_occupancy(int *blocks_per_sm, bool count_mode, bool small_rows = false);
size_t main_smem_bytes(bool small_rows = false);
cudaError_t launch_sort_unique(const InstDev *inst, const int *inst_list, int nlist, uint64_t *raw, uint64_t *tmp,
                               const uint32_t *raw_count, const uint32_t *flags, StatusDev *status,
                               uint64_t *dense, uint32_t dense_cap, uint32_t *dense_total,
                               cudaStream_t st);
cudaError_t init_tables();
// Host handles of the pack and sort/unique kernels (to find their nodes in a captured graph).
const void *pack_kernel_fn();
const void *sort_unique_kernel_fn();
cudaError_t launch_probe(int kind, int iters, int blocks, unsigned long long *cycles, unsigned long long *sink,
                         cudaStream_t st);

// ---------------------------------------------------------------- general alphabets (pms_sigma.cu)
//
// The qPMS-Sigma form over an alphabet of 2..32 letters: ceil(log2 sigma)
// bit-planes per window, one seed per queue item, the tree of changed-position
// sets walked by the threads of a CTA, letters enumerated depth-first per node.

constexpr int kSigMaxD = 16;        // changed positions per candidate
constexpr int kSigMaxPlanes = 5;    // ceil(log2 32)
constexpr int kSigThreads = 256;    // threads of the search kernel's CTA
constexpr int kSigSortThreads = 1024;
constexpr int kSigSmemSmall = 64 * 1024;    // rows of one seed in shared memory: 3 CTAs per SM
constexpr int kSigSmemLarge = 100 * 1024;   // the same for seeds with many rows: 2 CTAs per SM (with the
                                            // kernel's 10 KB of static per-warp state, 2 x 110 KB <= 228 KB)
#ifndef PMS_SIG_LIST_CAP
#define PMS_SIG_LIST_CAP 16384
#endif
constexpr int kSigListCap = PMS_SIG_LIST_CAP;   // words of row lists per warp of the search kernel

// Work counters of the search kernel (always on), indices into a uint64 array.
enum SigCounter {
    kSgSeeds = 0,        // seeds taken from the queue
    kSgSeedsInfeasible,  // seeds with too many sequences lacking a feasible occurrence
    kSgNodes,            // position subsets (tree nodes) visited
    kSgNodesPruned,      // subsets dismissed by the node bound
    kSgChecks,           // depth-first checks of partial and full candidates
    kSgLeaves,           // checks of full candidates (every changed position fixed)
    kSgCmpRows,          // window comparisons building the rows
    kSgCmpReduce,        // node-bound comparisons popc(D ^ P)
    kSgCmpVerify,        // candidate-versus-row comparisons
    kSgCntNum
};

// byte -> letter index (0xFF: not a letter of the alphabet), or index -> letter
struct SigmaMap {
    uint8_t v[256];
};

struct SigmaParams {
    const uint32_t *planes;        // plane g of window (i, j) at g * n * W + i * W + j
    int n, m, l, d, b, sigma, W;
    int miss_max;                  // sequences a motif may miss: n - q
    int nseeds;                    // seeds: the windows of s_1..s_{n-q+1}
    long long nodes;               // position subsets per seed: sum over k <= d of C(l, k)
    unsigned int *head;            // seed queue head (zeroed before the launch)
    unsigned long long *raw;       // motif keys, 3 words each (most significant first)
    unsigned long long *raw_count; // keys emitted (may exceed raw_cap)
    unsigned long long raw_cap;    // keys the raw buffer holds (a power of two)
    unsigned long long *counters;  // kSgCntNum
    uint32_t *scratch;             // per CTA (1 + b) * scratch_rows words (scratch_rows even), for seeds whose rows exceed smem_rows
    int scratch_rows;
    int smem_rows;                 // rows a seed keeps in shared memory
    uint32_t *lists;               // per warp list_cap words: row lists of the depth-first search (may be null)
    int list_cap;
};

int sigma_planes(int sigma);
size_t sigma_row_bytes(int b, int l);   // shared or scratch bytes of one seed row
int sigma_smem_rows(int b, int l, bool large);
cudaError_t sigma_init_tables();
cudaError_t sigma_main_occupancy(int b, int l, bool large, int *blocks_per_sm);
cudaError_t launch_sigma_pack(const uint8_t *seqs, int n, int m, int l, int b, const SigmaMap &map, uint32_t *planes,
                              uint32_t *flags, cudaStream_t st);
cudaError_t launch_sigma_main(const SigmaParams &p, int blocks, cudaStream_t st);
// Device state of the sort/unique kernel's CTAs (one grid, all CTAs resident):
// hist holds sigma_sort_hist_words(ctas) words (per-CTA digit counts, digit
// totals, per-CTA unique counts); bar two words, zeroed before the launch.
// bar[1] != 0 after the launch: a CTA gave up waiting at a grid barrier and
// the output is not valid.
struct SigSortGrid {
    unsigned int *hist;
    unsigned int *bar;
    int ctas;
};
size_t sigma_sort_hist_words(int ctas);
// CTAs of the sort/unique grid on the current device (all resident at once).
cudaError_t sigma_sort_ctas(int *ctas);
// raw: cap keys of three words; tmp: room for as many (the radix sort's second buffer)
cudaError_t launch_sigma_sort_unique(unsigned long long *raw, unsigned long long *tmp,
                                     const unsigned long long *raw_count, unsigned long long cap, int l, int b,
                                     const SigmaMap &letters, uint8_t *out, unsigned long long *unique_count,
                                     const SigSortGrid &grid, cudaStream_t st);

}  // namespace pms
