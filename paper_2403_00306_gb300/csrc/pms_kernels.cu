// pms_kernels.cu -- sm_103a kernels of the exact planted (l,d)-motif search.
//
// Method (the paper's chapter "Our Approach" and the algorithms it builds on):
//   * every l-mer is held as two 32-bit bit-planes (bit 1 and bit 0 of the
//     A0 C1 G2 T3 codes, position k in bit k); the Hamming distance of two
//     l-mers is popc((a.hi ^ b.hi) | (a.lo ^ b.lo)) (Sec. "String Compression");
//   * candidates are the strings of B(x, d) for the l-mers x of s_1
//     (Observation 3.1 with q = n), explored as the tree T_d(x) of qPMSPrune:
//     a node is the set P of changed positions, its leaves the 3^|P| choices
//     of new letters;
//   * for each seed x and sequence s_i (i >= 2) the feasible occurrences are
//     the windows w with d_H(x, w) <= 2d (PMS8's pair-distance preprocessing;
//     any motif within d of x can only be within d of such a window); rows are
//     checked smallest first (PMS8: "sort rows by size");
//   * a node P keeps only the occurrences with popc(D_w ^ P) <= d, where D_w
//     is the mismatch mask of x and w: on P the candidate differs from x, so
//     it mismatches w wherever w agrees with x, and off P it mismatches w
//     wherever x does. A node with an empty reduced row has no motif among
//     its 3^|P| leaves (the branch-and-bound of qPMSPrune, applied per node);
//     each lane walks one node through the rows with this bound;
//   * below a surviving node, partial candidates (letters fixed above the
//     three lowest changed positions) are tested with the exact bound over
//     their leaves, or the 81 leaves of a 4-position node are handled as a
//     bit set;
//   * each surviving leaf is verified against the reduced rows with packed
//     XOR/OR/popc, warp ballots compact the survivors between rows, and the
//     motifs are appended with one atomic per warp, then sorted and
//     de-duplicated per instance.
#include "pms_internal.h"

#include <algorithm>

namespace pms {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

// Row-entry quads a lane of the node walk tests per step (4: 16 entries).
#ifndef PMS_WALK_QUADS
#define PMS_WALK_QUADS 4
#endif
constexpr int kWalkQuads = PMS_WALK_QUADS;
static_assert(kWalkQuads >= 2 && kWalkQuads % 2 == 0, "the walk step loads quads in pairs");

__constant__ uint32_t c_binom[kLMax + 1][kLMax + 1];  // C(a, b), 0 when b > a
__constant__ unsigned long long c_pow3[kLMax + 1];
// Leaf sets of a node with at most 4 changed positions p_0 < p_1 < ...: leaf
// v = sum v_i 3^i takes letter x[p_i] XOR (v_i + 1) (2-bit codes) at p_i.
// c_digit[i][v][w]: word w of the set of leaves (v < 81) with v_i = v.
__constant__ uint32_t c_digit[4][3][3];

struct __align__(16) WarpSmem {
    uint2 rb0[kRbCap + 4];      // row 0 reduced by the current subset
    uint2 rb1[kRbCap + 4];      // scratch reduced row for rows 1..
    uint2 list[kListCap];       // candidates that survived row 0
    uint32_t subs[kSubBatch];   // position subsets being filtered
    union {
        struct {
            uint8_t lmiss[kListCap];    // quorum form: rows each listed candidate has missed
            uint8_t smiss[kSubBatch];   // quorum form: rows each subset has missed
        } q;
        uint32_t stash[68];             // node walk: its state parked while leaves are expanded
    } u;
};

struct __align__(16) CtaSmem {
    uint32_t binom[kLMax + 1][kLMax + 1];
    int row_len[kNMax];      // indexed by sequence
    int row_off[kNMax];      // indexed by sequence: first entry of its row (multiple of 4)
    int row_order[kNMax];    // sequences 1..n-1, smallest row first
    int rank_off4[kNMax];    // by rank in that order: first entry quad of the row
    int rank_len4[kNMax];    // by rank in that order: entry quads of the row (padded size / 4)
    unsigned long long g;
    int inst, seed, chunk;
    int cached_inst, cached_seed;
    int feasible;
    int rows_in_smem;        // 1: D and planes in shared memory; 2: D only (planes in global scratch); 0: neither
    int total_rows;
    int next;                // next subset index of the chunk to claim
    int ctab;                // chunk table of the current item
    int stolen;              // the current item was joined after the queue ran out
    int pad;
};

// Colex unranking of the rank-th k-subset of {0..l-1} (combinatorial number
// system): bit c of the result is set for each chosen position c. `binom` is
// the C(a, b) table (a copy in shared memory, as lanes index it differently).
__device__ __forceinline__ uint32_t unrank_subset(uint32_t rank, int k, int l, const uint32_t (*binom)[kLMax + 1])
{
    uint32_t P = 0;
    int c = l - 1;
    for (int j = k; j >= 1; --j) {
        while (binom[c][j] > rank)
            --c;
        P |= 1u << c;
        rank -= binom[c][j];
        --c;
    }
    return P;
}

__device__ __forceinline__ uint64_t to_key(uint32_t h, uint32_t lo, int l)
{
    uint64_t key = 0;
    for (int k = 0; k < l; ++k)
        key = (key << 2) | (uint64_t)((((h >> k) & 1u) << 1) | ((lo >> k) & 1u));
    return key;
}

// Position of the r-th (0-based) set bit of v, for 0 <= r < popc(v): a binary
// search over the bit counts of the halves, quarters, ... of the word.
__device__ __forceinline__ int nth_set_bit(uint32_t v, int r)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int cnt = __popc(v & ((1u << w) - 1u));
        if (r >= cnt) {
            r -= cnt;
            v >>= w;
            pos += w;
        }
    }
    return pos;
}

// A seed's feasible occurrences: per entry the mismatch mask D of the seed
// and the window, and the window's planes; rows are padded to a multiple of 4
// entries with copies of their last entry.
struct Rows {
    const uint32_t *D;
    const uint2 *HL;
};

// Keeps the occurrences w of one row with popc(D_w ^ P) <= d; writes up to
// kRbCap of their planes to rb, pads rb to a multiple of 4 entries, and
// returns how many qualify.
__device__ __forceinline__ int reduce_row(const uint32_t *D, const uint2 *HL, int len, uint32_t P, int d, uint2 *rb,
                                          int lane, uint32_t lt)
{
    int k = 0;
    for (int e0 = 0; e0 < len; e0 += 32) {
        const int e = e0 + lane;
        bool keep = false;
        if (e < len)
            keep = __popc(D[e] ^ P) <= d;
        const uint32_t bal = __ballot_sync(kFull, keep);
        if (keep) {
            const int pos = k + __popc(bal & lt);
            if (pos < kRbCap)
                rb[pos] = HL[e];
        }
        k += __popc(bal);
    }
    __syncwarp();
    if (k > 0 && k <= kRbCap && lane < 4)
        rb[k + lane] = rb[k - 1];
    __syncwarp();
    return k;
}

// Is some entry of a reduced row (shared memory, padded to 4) within d of (ch, cl)?
__device__ __forceinline__ bool check_smem(const uint2 *rb, int k, uint32_t ch, uint32_t cl, int d)
{
    int m0 = 64, m1 = 64;
    for (int e = 0; e < k; e += 4) {
        const uint4 a = *reinterpret_cast<const uint4 *>(rb + e);
        const uint4 b = *reinterpret_cast<const uint4 *>(rb + e + 2);
        m0 = min(m0, __popc((ch ^ a.x) | (cl ^ a.y)));
        m1 = min(m1, __popc((ch ^ a.z) | (cl ^ a.w)));
        m0 = min(m0, __popc((ch ^ b.x) | (cl ^ b.y)));
        m1 = min(m1, __popc((ch ^ b.z) | (cl ^ b.w)));
    }
    return min(m0, m1) <= d;
}

// Same test against a full (unreduced) row; used when the reduced row does
// not fit in the warp's buffer.
__device__ __forceinline__ bool check_row(const uint2 *HL, int len, uint32_t ch, uint32_t cl, int d)
{
    int mn = 64;
    for (int e = 0; e < len; ++e) {
        const uint2 w = HL[e];
        mn = min(mn, __popc((ch ^ w.x) | (cl ^ w.y)));
    }
    return mn <= d;
}

struct WarpCtx {
    const MainParams *p;
    InstDev in;
    int I;
    int lane;
    uint32_t lt;
    uint32_t xh, xl;           // the seed l-mer
    Rows rows;                 // feasible occurrences of the seed (shared or global memory)
    const CtaSmem *cs;
    WarpSmem *ws;
    unsigned long long *cnt;   // per-thread counters (count mode)
};

template <bool kCount>
__device__ __forceinline__ void emit(const WarpCtx &c, const uint2 *list, int N)
{
    const MainParams &p = *c.p;
    for (int b = 0; b < N; b += 32) {
        const int idx = b + c.lane;
        const bool has = idx < N;
        uint64_t key = 0;
        if (has) {
            const uint2 v = list[idx];
            key = to_key(v.x, v.y, c.in.l);
        }
        const uint32_t bal = __ballot_sync(kFull, has);
        uint32_t base = 0;
        if (c.lane == 0)
            base = atomicAdd(&p.raw_count[c.I], (uint32_t)__popc(bal));
        base = __shfl_sync(kFull, base, 0);
        const uint32_t pos = base + __popc(bal & c.lt);
        if (has) {
            if (pos < c.in.raw_cap)
                p.raw[c.in.raw_off + pos] = key;
            else
                atomicOr(&p.flags[c.I], kFlagOverflow);
        }
    }
    __syncwarp();
}

// Checks the buffered candidates against rows 1.. (row 0 already passed),
// compacting survivors in place; emits those that pass every row.
template <bool kCount>
__device__ __forceinline__ void finish_list(const WarpCtx &c, uint32_t P, int N)
{
    const InstDev &in = c.in;
    const int nrows = in.n - 1;
    uint2 *list = c.ws->list;
    __syncwarp();
    for (int r = 1; r < nrows && N > 0; ++r) {
        const int ri = c.cs->row_order[r];
        const int len = c.cs->row_len[ri];
        const int off = c.cs->row_off[ri];
        const int k = reduce_row(c.rows.D + off, c.rows.HL + off, len, P, in.d, c.ws->rb1, c.lane, c.lt);
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpReduce] += len;
        if (k == 0) {
            N = 0;
            break;
        }
        const bool sm = k <= kRbCap;
        int newN = 0;
        for (int b = 0; b < N; b += 32) {
            const int idx = b + c.lane;
            const bool alive = idx < N;
            uint2 v = make_uint2(0u, 0u);
            if (alive)
                v = list[idx];
            bool hit = false;
            if (alive) {
                hit = sm ? check_smem(c.ws->rb1, k, v.x, v.y, in.d) : check_row(c.rows.HL + off, len, v.x, v.y, in.d);
                if (kCount)
                    c.cnt[kCntCmpVerify] += sm ? k : len;
            }
            __syncwarp();
            const uint32_t bal = __ballot_sync(kFull, hit);
            if (hit)
                list[newN + __popc(bal & c.lt)] = v;
            newN += __popc(bal);
        }
        __syncwarp();
        N = newN;
    }
    if (N > 0)
        emit<kCount>(c, list, N);
}

// The leaf walk of one node: every active lane tests the leaves of its
// letter choices on the lowest positions of P, two per step (the odometer
// state after one increment is computed alongside, so the two tests are
// independent), against row 0 reduced by P; hits are appended to the warp's
// list (which is checked against the other rows when it fills up). kReg > 0:
// the reduced row (at most kReg entries, padded copies included) is held in
// registers; kReg == 0: read from shared memory, or from the full row when the
// reduction overflowed; kReg < 0: no rows (n = 1), every leaf is kept.
template <bool kCount, int kReg>
__device__ __forceinline__ int leaf_loop(const WarpCtx &c, uint32_t P, uint32_t Phi, uint32_t ch0, uint32_t cl0,
                                         bool active, unsigned long long iters, int k0, int len0, int off0)
{
    const int d = c.in.d;
    const bool sm0 = k0 <= kRbCap;
    uint2 e[kReg > 0 ? kReg : 1];
    if constexpr (kReg > 0) {
#pragma unroll
        for (int i = 0; i < kReg; ++i)
            e[i] = c.ws->rb0[i < k0 ? i : k0 - 1];
    }
    uint2 *list = c.ws->list;
    uint32_t Dh = 0u, Dl = Phi;
    int listN = 0;
    for (unsigned long long it = 0; it < iters; it += 2) {
        const bool two = it + 1 < iters;
        const uint32_t both = Dh & Dl;
        const uint32_t open = Phi & ~both;
        const uint32_t q = open & (0u - open);
        const uint32_t below = Phi & (q - 1u);
        const uint32_t Dh2 = (Dh & ~below) | q;
        const uint32_t Dl2 = (Dl | below) ^ q;
        const uint32_t ch_a = ch0 ^ Dh, cl_a = cl0 ^ Dl;
        const uint32_t ch_b = ch0 ^ Dh2, cl_b = cl0 ^ Dl2;
        bool hit_a = false, hit_b = false;
        if (active) {
            if constexpr (kReg < 0) {
                hit_a = true;
                hit_b = two;
            } else if constexpr (kReg == 1) {
                hit_a = __popc((ch_a ^ e[0].x) | (cl_a ^ e[0].y)) <= d;
                hit_b = two && __popc((ch_b ^ e[0].x) | (cl_b ^ e[0].y)) <= d;
            } else if constexpr (kReg > 0) {
                int a0 = 64, a1 = 64, b0m = 64, b1m = 64;
#pragma unroll
                for (int i = 0; i < kReg; i += 2) {
                    a0 = min(a0, __popc((ch_a ^ e[i].x) | (cl_a ^ e[i].y)));
                    b0m = min(b0m, __popc((ch_b ^ e[i].x) | (cl_b ^ e[i].y)));
                    a1 = min(a1, __popc((ch_a ^ e[i + 1].x) | (cl_a ^ e[i + 1].y)));
                    b1m = min(b1m, __popc((ch_b ^ e[i + 1].x) | (cl_b ^ e[i + 1].y)));
                }
                hit_a = min(a0, a1) <= d;
                hit_b = two && min(b0m, b1m) <= d;
            } else if (sm0) {
                int a0 = 64, a1 = 64, b0m = 64, b1m = 64;
                for (int i = 0; i < k0; i += 4) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(c.ws->rb0 + i);
                    const uint4 v = *reinterpret_cast<const uint4 *>(c.ws->rb0 + i + 2);
                    a0 = min(a0, __popc((ch_a ^ u.x) | (cl_a ^ u.y)));
                    b0m = min(b0m, __popc((ch_b ^ u.x) | (cl_b ^ u.y)));
                    a1 = min(a1, __popc((ch_a ^ u.z) | (cl_a ^ u.w)));
                    b1m = min(b1m, __popc((ch_b ^ u.z) | (cl_b ^ u.w)));
                    a0 = min(a0, __popc((ch_a ^ v.x) | (cl_a ^ v.y)));
                    b0m = min(b0m, __popc((ch_b ^ v.x) | (cl_b ^ v.y)));
                    a1 = min(a1, __popc((ch_a ^ v.z) | (cl_a ^ v.w)));
                    b1m = min(b1m, __popc((ch_b ^ v.z) | (cl_b ^ v.w)));
                }
                hit_a = min(a0, a1) <= d;
                hit_b = two && min(b0m, b1m) <= d;
            } else {
                hit_a = check_row(c.rows.HL + off0, len0, ch_a, cl_a, d);
                hit_b = two && check_row(c.rows.HL + off0, len0, ch_b, cl_b, d);
            }
            if (kCount) {
                c.cnt[kCntTested] += two ? 2 : 1;
                c.cnt[kCntCmpVerify] += (unsigned long long)(two ? 2 : 1) * (kReg < 0 ? 0 : (sm0 ? k0 : len0));
            }
        }
        const uint32_t bal_a = __ballot_sync(kFull, hit_a);
        const uint32_t bal_b = __ballot_sync(kFull, hit_b);
        if (bal_a | bal_b) {
            if (hit_a)
                list[listN + __popc(bal_a & c.lt)] = make_uint2(ch_a, cl_a);
            listN += __popc(bal_a);
            if (hit_b)
                list[listN + __popc(bal_b & c.lt)] = make_uint2(ch_b, cl_b);
            listN += __popc(bal_b);
            if (listN > kListCap - 64) {
                finish_list<kCount>(c, P, listN);
                listN = 0;
            }
        }
        // advance the odometer by two
        const uint32_t both2 = Dh2 & Dl2;
        const uint32_t open2 = Phi & ~both2;
        const uint32_t q2 = open2 & (0u - open2);
        const uint32_t below2 = Phi & (q2 - 1u);
        Dh = (Dh2 & ~below2) | q2;
        Dl = (Dl2 | below2) ^ q2;
    }
    return listN;
}

// Lower bound on the distance from a window w to every leaf that agrees with
// the partial candidate (ph, pl) outside the free positions Plow and differs
// from the seed x on each of them: mismatches outside Plow, plus the free
// positions where w agrees with x (the leaf must differ from x there).
__device__ __forceinline__ int partial_bound(uint32_t ph, uint32_t pl, uint2 w, uint32_t xh, uint32_t xl,
                                             uint32_t Plow)
{
    return __popc(((ph ^ w.x) | (pl ^ w.y)) & ~Plow) + __popc(Plow & ~((xh ^ w.x) | (xl ^ w.y)));
}

// One more tree level between a node P and its leaves. A partial candidate
// fixes the letters on the positions Phi of P above its three lowest (Plow);
// it survives a row only if some occurrence w of the row has
// partial_bound <= d, since every leaf below it is at least that far from w.
// Lanes own partials (32 per group, numbered like the odometer's states),
// test them against row 0 reduced by P and then rows 1..partial_rows-1,
// reduced in turn, stopping once no partial of the group is left; the warp
// then tests the leaves of the surviving partials only (27 lanes own the
// letters on Plow, two partials per step) against row 0, and the hits go on
// to the other rows through the warp's list.
template <bool kCount, int kReg>
__device__ __forceinline__ int partial_walk(const WarpCtx &c, uint32_t P, uint32_t Phi, uint32_t Plow,
                                            uint32_t DhLo, uint32_t DlLo, bool active, int h, int k0, int len0,
                                            int off0)
{
    const int d = c.in.d;
    const int R = min(c.in.partial_rows, c.in.n - 1);
    const bool sm0 = k0 <= kRbCap;
    uint2 e[kReg > 0 ? kReg : 1];
    if constexpr (kReg > 0) {
#pragma unroll
        for (int i = 0; i < kReg; ++i)
            e[i] = c.ws->rb0[i < k0 ? i : k0 - 1];
    }
    uint2 *list = c.ws->list;
    const uint32_t npart = (uint32_t)c_pow3[h];   // h <= 20, so 3^h < 2^32
    int listN = 0;
    for (uint32_t g0 = 0; g0 < npart; g0 += 32) {
        const uint32_t pidx = g0 + (uint32_t)c.lane;
        bool live = pidx < npart;
        // odometer state number pidx: base-3 digits over Phi, lowest position first
        uint32_t Dh = 0u, Dl = 0u;
        {
            uint32_t r = pidx;
            uint32_t t = Phi;
            while (t) {
                const uint32_t b = t & (0u - t);
                t ^= b;
                const uint32_t r3 = r / 3u;
                const uint32_t dg = r - 3u * r3;
                r = r3;
                Dh |= dg >= 1u ? b : 0u;
                Dl |= dg != 1u ? b : 0u;
            }
        }
        const uint32_t ph = c.xh ^ Dh, pl = c.xl ^ Dl;
        if (live) {
            int mn = 64;
            if constexpr (kReg > 0) {
#pragma unroll
                for (int i = 0; i < kReg; ++i)
                    mn = min(mn, partial_bound(ph, pl, e[i], c.xh, c.xl, Plow));
            } else if (sm0) {
                for (int i = 0; i < k0; ++i)
                    mn = min(mn, partial_bound(ph, pl, c.ws->rb0[i], c.xh, c.xl, Plow));
            } else {
                for (int i = 0; i < len0; ++i)
                    mn = min(mn, partial_bound(ph, pl, c.rows.HL[off0 + i], c.xh, c.xl, Plow));
            }
            live = mn <= d;
            if (kCount)
                c.cnt[kCntCmpReduce] += sm0 ? k0 : len0;
        }
        for (int r = 1; r < R; ++r) {
            if (!__any_sync(kFull, live))
                break;
            const int ri = c.cs->row_order[r];
            const int len = c.cs->row_len[ri];
            const int off = c.cs->row_off[ri];
            const int k = reduce_row(c.rows.D + off, c.rows.HL + off, len, P, d, c.ws->rb1, c.lane, c.lt);
            if (kCount && c.lane == 0)
                c.cnt[kCntCmpReduce] += len;
            if (live) {
                int mn = 64;
                if (k <= kRbCap) {
                    for (int i = 0; i < k; ++i)
                        mn = min(mn, partial_bound(ph, pl, c.ws->rb1[i], c.xh, c.xl, Plow));
                } else {
                    for (int i = 0; i < len; ++i)
                        mn = min(mn, partial_bound(ph, pl, c.rows.HL[off + i], c.xh, c.xl, Plow));
                }
                live = mn <= d;
                if (kCount)
                    c.cnt[kCntCmpReduce] += k <= kRbCap ? k : len;
            }
        }
        uint32_t mask = __ballot_sync(kFull, live);
        while (mask) {
            const int pa = __ffs(mask) - 1;
            mask &= mask - 1u;
            const bool two = mask != 0u;
            const int pb = two ? __ffs(mask) - 1 : pa;
            if (two)
                mask &= mask - 1u;
            const uint32_t ch_a = __shfl_sync(kFull, ph, pa) ^ DhLo, cl_a = __shfl_sync(kFull, pl, pa) ^ DlLo;
            const uint32_t ch_b = __shfl_sync(kFull, ph, pb) ^ DhLo, cl_b = __shfl_sync(kFull, pl, pb) ^ DlLo;
            bool hit_a = false, hit_b = false;
            if (active) {
                if constexpr (kReg == 1) {
                    hit_a = __popc((ch_a ^ e[0].x) | (cl_a ^ e[0].y)) <= d;
                    hit_b = two && __popc((ch_b ^ e[0].x) | (cl_b ^ e[0].y)) <= d;
                } else if constexpr (kReg > 0) {
                    int a0 = 64, a1 = 64, b0m = 64, b1m = 64;
#pragma unroll
                    for (int i = 0; i < kReg; i += 2) {
                        a0 = min(a0, __popc((ch_a ^ e[i].x) | (cl_a ^ e[i].y)));
                        b0m = min(b0m, __popc((ch_b ^ e[i].x) | (cl_b ^ e[i].y)));
                        a1 = min(a1, __popc((ch_a ^ e[i + 1].x) | (cl_a ^ e[i + 1].y)));
                        b1m = min(b1m, __popc((ch_b ^ e[i + 1].x) | (cl_b ^ e[i + 1].y)));
                    }
                    hit_a = min(a0, a1) <= d;
                    hit_b = two && min(b0m, b1m) <= d;
                } else if (sm0) {
                    hit_a = check_smem(c.ws->rb0, k0, ch_a, cl_a, d);
                    hit_b = two && check_smem(c.ws->rb0, k0, ch_b, cl_b, d);
                } else {
                    hit_a = check_row(c.rows.HL + off0, len0, ch_a, cl_a, d);
                    hit_b = two && check_row(c.rows.HL + off0, len0, ch_b, cl_b, d);
                }
                if (kCount) {
                    c.cnt[kCntTested] += two ? 2 : 1;
                    c.cnt[kCntCmpVerify] += (unsigned long long)(two ? 2 : 1) * (sm0 ? k0 : len0);
                }
            }
            const uint32_t bal_a = __ballot_sync(kFull, hit_a);
            const uint32_t bal_b = __ballot_sync(kFull, hit_b);
            if (bal_a | bal_b) {
                if (hit_a)
                    list[listN + __popc(bal_a & c.lt)] = make_uint2(ch_a, cl_a);
                listN += __popc(bal_a);
                if (hit_b)
                    list[listN + __popc(bal_b & c.lt)] = make_uint2(ch_b, cl_b);
                listN += __popc(bal_b);
                if (listN > kListCap - 64) {
                    finish_list<kCount>(c, P, listN);
                    listN = 0;
                }
            }
        }
    }
    return listN;
}

// The three-string feasibility test of TraverStringRef, for a node P of seed
// x and a pair of occurrences: u of row 0 (rb0, reduced by P) and w of a later
// row. A string c of node P equals x outside P and differs from x on P. Let
// t_u = popc(D_u ^ P): the mismatches of c and u it cannot avoid (outside P
// where u differs from x, and on P where u agrees with x); likewise t_w. On the
// positions of P where u and w both differ from x, c can match both when
// u = w there, but only one of them when u, w and x are three different
// letters; with F the number of those positions, some c of node P is within d
// of both u and w exactly when t_u + t_w + F <= 2d (t_u, t_w <= d hold for
// reduced rows). Every motif of node P is within d of an occurrence u of row 0
// that passes this test with some occurrence w of each other row, so row 0
// keeps only such u (lane i tests entry i, rows 1..triple_rows in size order)
// and the node is dropped when none is left. Returns the new size of rb0
// (padded to a multiple of 4 like reduce_row); k0 <= 32.
template <bool kCount>
__device__ __forceinline__ int triple_filter(const WarpCtx &c, uint32_t P, int k0)
{
    const InstDev &in = c.in;
    const int d = in.d;
    const int R = min(in.triple_rows + 1, in.n - 1);
    uint2 u = make_uint2(0u, 0u);
    uint32_t Du = 0u;
    int tu = 0;
    bool alive = c.lane < k0;
    if (alive) {
        u = c.ws->rb0[c.lane];
        Du = (u.x ^ c.xh) | (u.y ^ c.xl);
        tu = __popc(Du ^ P);
    }
    for (int r = 1; r < R; ++r) {
        if (!__any_sync(kFull, alive))
            break;
        const int ri = c.cs->row_order[r];
        const int len = c.cs->row_len[ri];
        const int off = c.cs->row_off[ri];
        const int k = reduce_row(c.rows.D + off, c.rows.HL + off, len, P, d, c.ws->rb1, c.lane, c.lt);
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpReduce] += len;
        if (k > kRbCap)
            continue;   // the reduced row did not fit its buffer: this row is not used
        bool ok = false;
        if (alive) {
            for (int i = 0; i < k; ++i) {
                const uint2 w = c.ws->rb1[i];
                const uint32_t Dw = (w.x ^ c.xh) | (w.y ^ c.xl);
                const uint32_t Euw = (u.x ^ w.x) | (u.y ^ w.y);
                ok |= tu + __popc(Dw ^ P) + __popc(Du & Dw & Euw & P) <= 2 * d;
            }
            if (kCount)
                c.cnt[kCntCmpVerify] += k;
        }
        alive = alive && ok;
    }
    const uint32_t bal = __ballot_sync(kFull, alive);
    const int nk = __popc(bal);
    __syncwarp();
    if (alive)
        c.ws->rb0[__popc(bal & c.lt)] = u;
    __syncwarp();
    if (nk > 0 && c.lane < 4)
        c.ws->rb0[nk + c.lane] = c.ws->rb0[nk - 1];
    __syncwarp();
    return nk;
}

// The leaves of a node P with lev <= 4 changed positions as a set of up to 81
// bits, verified row by row. For an occurrence w of a row reduced by P, a leaf
// c is within d of w iff the matches of c and w on P reach t = lev + m_out - d,
// where m_out = popc(D_w & ~P) (outside P every leaf equals x) and a match at
// p_i needs w != x there and v_i = (x XOR w at p_i) - 1. The leaves of w are
// therefore "at least t of the digit sets c_digit[i][a_i]" over the positions
// where w differs from x, built with running at-least-1..4 unions; one lane per
// occurrence, the row's set is the OR over its occurrences and the node's
// leaves the AND over rows, stopping once it is empty.
template <bool kCount>
__device__ __forceinline__ void expand_bits(const WarpCtx &c, uint32_t P, int lev, int k0)
{
    const InstDev &in = c.in;
    const int d = in.d;
    const int nrows = in.n - 1;
    uint32_t b[4];
    {
        uint32_t t = P;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            b[i] = t & (0u - t);
            t ^= b[i];
        }
    }
    const int nleaf = (int)c_pow3[lev];
    if (kCount && c.lane == 0)
        c.cnt[kCntTested] += nleaf;
    uint32_t alive[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int lo = 32 * q;
        alive[q] = nleaf <= lo ? 0u : (nleaf >= lo + 32 ? ~0u : (1u << (nleaf - lo)) - 1u);
    }
    for (int r = 0; r < nrows; ++r) {
        const int ri = c.cs->row_order[r];
        const int len = c.cs->row_len[ri];
        const int off = c.cs->row_off[ri];
        // row 0 is already reduced (and possibly cut by the three-string test) in rb0
        int k = k0;
        if (r > 0) {
            k = reduce_row(c.rows.D + off, c.rows.HL + off, len, P, d, c.ws->rb1, c.lane, c.lt);
            if (kCount && c.lane == 0)
                c.cnt[kCntCmpReduce] += len;
        }
        const uint2 *rb = r > 0 ? c.ws->rb1 : c.ws->rb0;
        const bool sm = k <= kRbCap;
        const int cnt = sm ? k : len;   // occurrences scanned: the reduced row, or the full row
        uint32_t rowm[3] = {0u, 0u, 0u};
        for (int e0 = 0; e0 < cnt; e0 += 32) {
            const int e = e0 + c.lane;
            uint32_t m0 = 0u, m1 = 0u, m2 = 0u;
            if (e < cnt) {
                const uint2 w = sm ? rb[e] : c.rows.HL[off + e];
                const uint32_t eh = w.x ^ c.xh, el = w.y ^ c.xl;
                const uint32_t Dw = eh | el;
                const int t = lev + __popc(Dw & ~P) - d;
                if (__popc(Dw ^ P) <= d) {   // the node bound (always true for a reduced row)
                    if (t <= 0) {
                        m0 = m1 = m2 = ~0u;
                    } else {
                        uint32_t a1[3] = {0u, 0u, 0u}, a2[3] = {0u, 0u, 0u}, a3[3] = {0u, 0u, 0u},
                                 a4[3] = {0u, 0u, 0u};
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int code = ((eh & b[i]) ? 2 : 0) | ((el & b[i]) ? 1 : 0);
                            if (i < lev && code != 0) {
#pragma unroll
                                for (int q = 0; q < 3; ++q) {
                                    const uint32_t M = c_digit[i][code - 1][q];
                                    a4[q] |= a3[q] & M;
                                    a3[q] |= a2[q] & M;
                                    a2[q] |= a1[q] & M;
                                    a1[q] |= M;
                                }
                            }
                        }
                        m0 = t == 1 ? a1[0] : (t == 2 ? a2[0] : (t == 3 ? a3[0] : (t == 4 ? a4[0] : 0u)));
                        m1 = t == 1 ? a1[1] : (t == 2 ? a2[1] : (t == 3 ? a3[1] : (t == 4 ? a4[1] : 0u)));
                        m2 = t == 1 ? a1[2] : (t == 2 ? a2[2] : (t == 3 ? a3[2] : (t == 4 ? a4[2] : 0u)));
                    }
                }
            }
            rowm[0] |= __reduce_or_sync(kFull, m0);
            rowm[1] |= __reduce_or_sync(kFull, m1);
            rowm[2] |= __reduce_or_sync(kFull, m2);
        }
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpVerify] +=
                (unsigned long long)cnt * (__popc(alive[0]) + __popc(alive[1]) + __popc(alive[2]));
        alive[0] &= rowm[0];
        alive[1] &= rowm[1];
        alive[2] &= rowm[2];
        if ((alive[0] | alive[1] | alive[2]) == 0u)
            return;
    }
    // the surviving leaves: lane q of each 32-leaf word builds leaf 32 * word + q
    uint2 *list = c.ws->list;
    int N = 0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const bool has = (alive[q] >> c.lane) & 1u;
        if (has) {
            int v = 32 * q + c.lane;
            uint32_t Dh = 0u, Dl = 0u;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int dg = v % 3;
                v /= 3;
                if (i < lev) {
                    Dh |= dg >= 1 ? b[i] : 0u;
                    Dl |= dg != 1 ? b[i] : 0u;
                }
            }
            list[N + __popc(alive[q] & c.lt)] = make_uint2(c.xh ^ Dh, c.xl ^ Dl);
        }
        N += __popc(alive[q]);
    }
    __syncwarp();
    emit<kCount>(c, list, N);
}

// The leaves of one tree node P (|P| = lev) that survived the row filter.
// Lanes own the letter choices on the lowest min(lev, 3) positions of P (27
// lanes at most); every lane walks the choices on the remaining positions
// with a base-3 odometer kept as two masks (Dh, Dl) over those positions:
// state (0,1) -> (1,0) -> (1,1) -> carry, i.e. XOR deltas 1, 2, 3 of the
// 2-bit codes. Each leaf is tested against row 0 reduced by P; the hits go
// to the warp's list and on to the other rows.
template <bool kCount>
__device__ __forceinline__ void expand_subset(const WarpCtx &c, uint32_t P)
{
    const InstDev &in = c.in;
    const int d = in.d;
    const int nrows = in.n - 1;
    const int lev = __popc(P);

    int k0 = 0, len0 = 0, off0 = 0;
    if (nrows > 0) {
        const int r0 = c.cs->row_order[0];
        len0 = c.cs->row_len[r0];
        off0 = c.cs->row_off[r0];
        k0 = reduce_row(c.rows.D + off0, c.rows.HL + off0, len0, P, d, c.ws->rb0, c.lane, c.lt);
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpReduce] += len0;
        if (k0 == 0)
            return;
        if (in.triple_rows > 0 && nrows > 1 && k0 <= 32) {
            k0 = triple_filter<kCount>(c, P, k0);
            if (k0 == 0)
                return;
        }
    }

    // 81 leaves as a bit set (measured faster than the leaf list at 4 changed
    // positions, (15,4) 0.132 -> 0.128 ms, (13,4) 1.81 -> 1.77 ms; slower with
    // fewer leaves, (11,3) 0.316 -> 0.339 ms)
    if (nrows > 0 && lev == 4 && in.partial_rows == 0) {
        expand_bits<kCount>(c, P, lev, k0);
        return;
    }

    uint32_t t = P;
    const uint32_t b0 = t & (0u - t);
    t ^= b0;
    const uint32_t b1 = t & (0u - t);
    t ^= b1;
    const uint32_t b2 = t & (0u - t);
    t ^= b2;
    const uint32_t Phi = t;
    const int nlo = lev < 3 ? lev : 3;
    const int nlanes = nlo == 0 ? 1 : (nlo == 1 ? 3 : (nlo == 2 ? 9 : 27));
    const bool active = c.lane < nlanes;
    const int dg0 = c.lane % 3, dg1 = (c.lane / 3) % 3, dg2 = (c.lane / 9) % 3;
    const uint32_t DhLo = (dg0 >= 1 ? b0 : 0u) | (dg1 >= 1 ? b1 : 0u) | (dg2 >= 1 ? b2 : 0u);
    const uint32_t DlLo = (dg0 != 1 ? b0 : 0u) | (dg1 != 1 ? b1 : 0u) | (dg2 != 1 ? b2 : 0u);
    const uint32_t ch0 = c.xh ^ DhLo, cl0 = c.xl ^ DlLo;
    const unsigned long long iters = c_pow3[lev - nlo];

    int listN = 0;
    if (nrows > 0 && in.partial_rows > 0 && lev > nlo && lev - nlo <= 20) {
        const uint32_t Plow = b0 | b1 | b2;
        const int h = lev - nlo;
        // few variants: every one is inlined with its list flush, and at
        // (19,6) more of them cost more in instruction-cache misses than the
        // register-held rows save (measured 28.3 -> 18.7 ms with these two)
        if (k0 <= 1)
            listN = partial_walk<kCount, 1>(c, P, Phi, Plow, DhLo, DlLo, active, h, k0, len0, off0);
        else
            listN = partial_walk<kCount, 0>(c, P, Phi, Plow, DhLo, DlLo, active, h, k0, len0, off0);
    } else if (nrows == 0)
        listN = leaf_loop<kCount, -1>(c, P, Phi, ch0, cl0, active, iters, k0, len0, off0);
    else if (k0 <= 1)
        listN = leaf_loop<kCount, 1>(c, P, Phi, ch0, cl0, active, iters, k0, len0, off0);
    else if (k0 <= 2)
        listN = leaf_loop<kCount, 2>(c, P, Phi, ch0, cl0, active, iters, k0, len0, off0);
    else if (k0 <= 4)
        listN = leaf_loop<kCount, 4>(c, P, Phi, ch0, cl0, active, iters, k0, len0, off0);
    else
        listN = leaf_loop<kCount, 0>(c, P, Phi, ch0, cl0, active, iters, k0, len0, off0);
    if (listN > 0)
        finish_list<kCount>(c, P, listN);
}

// Breadth-first filter of the subsets in ws->subs[0..N): for the first
// prune_rows rows in size order, a subset P stays only if the row holds an
// occurrence with popc(D_w ^ P) <= d (the bound every leaf of P must meet).
// Lanes own subsets, row entries are read by all lanes at once; survivors are
// compacted after each row. Returns the number of survivors.
template <bool kCount>
__device__ __forceinline__ int filter_subsets(const WarpCtx &c, int N)
{
    const InstDev &in = c.in;
    const int d = in.d;
    const int nrows = min(in.prune_rows, in.n - 1);
    uint32_t *subs = c.ws->subs;
    for (int r = 0; r < nrows && N > 0; ++r) {
        const int ri = c.cs->row_order[r];
        const int len = c.cs->row_len[ri];
        const uint4 *D4 = reinterpret_cast<const uint4 *>(c.rows.D + c.cs->row_off[ri]);
        const int len4 = (len + 3) >> 2;
        int newN = 0;
        // two subsets per lane share every 16-byte load of row entries
        for (int b = 0; b < N; b += 64) {
            const int i0 = b + c.lane, i1 = b + 32 + c.lane;
            const bool al0 = i0 < N, al1 = i1 < N;
            const uint32_t P0 = al0 ? subs[i0] : 0u, P1 = al1 ? subs[i1] : 0u;
            int m00 = 64, m01 = 64, m10 = 64, m11 = 64;
            int e4 = 0;
            for (; e4 < len4; ++e4) {
                const uint4 v = D4[e4];
                m00 = min(m00, __popc(v.x ^ P0));
                m10 = min(m10, __popc(v.x ^ P1));
                m01 = min(m01, __popc(v.y ^ P0));
                m11 = min(m11, __popc(v.y ^ P1));
                m00 = min(m00, __popc(v.z ^ P0));
                m10 = min(m10, __popc(v.z ^ P1));
                m01 = min(m01, __popc(v.w ^ P0));
                m11 = min(m11, __popc(v.w ^ P1));
                if ((e4 & 3) == 3 &&
                    __all_sync(kFull, (!al0 || min(m00, m01) <= d) && (!al1 || min(m10, m11) <= d))) {
                    ++e4;
                    break;
                }
            }
            if (kCount)
                c.cnt[kCntCmpReduce] += 4ull * e4 * ((al0 ? 1 : 0) + (al1 ? 1 : 0));
            const bool pass0 = al0 && min(m00, m01) <= d;
            const bool pass1 = al1 && min(m10, m11) <= d;
            __syncwarp();
            const uint32_t bal0 = __ballot_sync(kFull, pass0);
            const uint32_t bal1 = __ballot_sync(kFull, pass1);
            if (pass0)
                subs[newN + __popc(bal0 & c.lt)] = P0;
            if (pass1)
                subs[newN + __popc(bal0) + __popc(bal1 & c.lt)] = P1;
            newN += __popc(bal0) + __popc(bal1);
        }
        __syncwarp();
        N = newN;
    }
    return N;
}

// Lane-asynchronous node filter of a chunk: every lane holds one tree node P
// and its position in the rows (row rank r, entry quad e4); each step a lane
// tests the next 4 * kWalkQuads entries of its own row with the bound popc(D_w ^ P) <= d.
// A hit moves the lane's node to the next row, a row scanned to its end
// dismisses the node, a node that passes the last filtered row goes to the
// expansion queue, and a free lane takes the next node of the warp's pool at
// once. So every node stops scanning a row at its own first hit (the
// sequential early-exit rule) instead of waiting for the slowest node of a
// batch. The pool holds nodes claimed a sixteenth of the chunk (4 to 64) at a
// time, each lane unranking one and stepping to the next by Gosper's step.
// subs[0..64) is the pool, subs[64..128) the queue.
//
// walk_run runs the walk until 32 or more nodes are queued or the chunk is
// done, and returns the queue length; the caller expands the queued nodes
// and calls it again. Between calls the walk's state is parked in the warp's
// shared memory (stash[0..32): each lane's node; stash[32..64): its row rank,
// quad and whether it holds a node; stash[64..67): pool position, pool size,
// chunk exhausted), so that no register is held across the leaf expansion.
__device__ __forceinline__ void walk_init(const WarpCtx &c)
{
    uint32_t *st = c.ws->u.stash;
    st[c.lane] = 0u;
    st[32 + c.lane] = 0u;
    if (c.lane < 4)
        st[64 + c.lane] = 0u;
    __syncwarp();
}

template <bool kCount>
__device__ __forceinline__ int walk_run(const WarpCtx &c, const int *tab, int g0, int g1, CtaSmem &cs, int *claim_ctr,
                                        int claim_base, unsigned int *items_out, bool &finished)
{
    const InstDev &in = c.in;
    const int d = in.d;
    const int nrows = min(in.prune_rows, in.n - 1);
    uint32_t *pool = c.ws->subs;
    uint32_t *queue = c.ws->subs + 64;
    uint32_t *st = c.ws->u.stash;
    const uint4 *D4 = reinterpret_cast<const uint4 *>(c.rows.D);
    const int nw = (int)(blockDim.x >> 5);
    const int claim = (g1 - g0 + 2 * nw - 1) / (2 * nw);
    const volatile uint32_t *vst = st;
    uint32_t P = vst[c.lane];
    const uint32_t w0 = vst[32 + c.lane];
    int r = (int)(w0 & 0xffu);
    int e4 = (int)((w0 >> 8) & 0x7fffffu);
    bool has = (w0 >> 31) != 0u;
    int pool_pos = (int)vst[64], pool_n = (int)vst[65];
    bool exhausted = vst[66] != 0u;
    int left_seen = (int)vst[67] - 1;   // unclaimed nodes after this warp's last claim (-1: none yet)
    int off4 = 0, len4 = 0;
    if (nrows > 0) {
        const int rr = min(r, nrows - 1);
        off4 = cs.rank_off4[rr];
        len4 = cs.rank_len4[rr];
    }
    int qn = 0;
    finished = false;
    __syncwarp();
    for (;;) {
        uint32_t freem = __ballot_sync(kFull, !has);
        if (freem) {
            int avail = pool_n - pool_pos;
            if (avail < __popc(freem) && !exhausted) {
                // move the unstarted rest to the front and claim more; claims
                // are sized so that every warp of the CTA gets a share of small chunks
                uint32_t keep = 0u;
                if (c.lane < avail)
                    keep = pool[pool_pos + c.lane];
                __syncwarp();
                if (c.lane < avail)
                    pool[c.lane] = keep;
                // guided: claim about half a warp's share of what was left unclaimed
                // at this warp's last claim, so the item's last nodes stay in the
                // shared counter instead of in one warp's pool
                const int share = left_seen < 0 ? claim : (left_seen + 2 * nw - 1) / (2 * nw);
                const int want = min(64 - avail, max(4, min(claim, share)));
                int start = 0;
                if (c.lane == 0) {
                    start = claim_base + atomicAdd(claim_ctr, want);
                    if (items_out) {
                        // shared counter: publish what is left, count the item once when it runs out
                        claim_ctr[1] = max(0, g1 - (start + want));
                        if (start < g1 && start + want >= g1)
                            atomicAdd(items_out, 1u);
                    }
                }
                start = __shfl_sync(kFull, start, 0);
                left_seen = max(0, g1 - (start + want));
                const int got = start < g1 ? min(want, g1 - start) : 0;
                if (start + want >= g1)
                    exhausted = true;
                // each lane unranks node start + 2j and steps to node start + 2j + 1:
                // the next k-subset in colex order is the next larger integer with k
                // bits set (Gosper's step), or the first (k+1)-subset at a level end
                for (int j = 2 * c.lane; j < got; j += 64) {
                    const int g = start + j;
                    int lev = 0;
                    while (tab[lev + 1] <= g)
                        ++lev;
                    const uint32_t P0 = unrank_subset((uint32_t)(g - tab[lev]), lev, in.l, cs.binom);
                    pool[avail + j] = P0;
                    if (j + 1 < got) {
                        uint32_t P1;
                        if (g + 1 < tab[lev + 1]) {
                            const uint32_t low = P0 & (0u - P0);
                            const uint32_t up = P0 + low;
                            P1 = up | (((P0 ^ up) >> 2) >> (__ffs(P0) - 1));
                        } else {
                            P1 = (1u << (lev + 1)) - 1u;
                        }
                        pool[avail + j + 1] = P1;
                    }
                }
                __syncwarp();
                if (kCount && c.lane == 0)
                    c.cnt[kCntSubsets] += got;
                pool_pos = 0;
                pool_n = avail + got;
                avail = pool_n;
            }
            const int take = min(__popc(freem), avail);
            const int rank = __popc(freem & c.lt);
            if (!has && rank < take) {
                P = pool[pool_pos + rank];
                r = 0;
                e4 = 0;
                has = true;
                if (nrows > 0) {
                    off4 = cs.rank_off4[0];
                    len4 = cs.rank_len4[0];
                }
            }
            pool_pos += take;
        }
        if (!__any_sync(kFull, has)) {
            finished = true;
            break;
        }
        // one step of every lane: the next 4 * kWalkQuads entries of its row, as selects
        // rather than branches (a lane without a node reads the first quad of
        // the rows and ignores the result)
        bool done = false;
        if (nrows == 0) {
            done = has;
        } else {
            const int a4 = has ? off4 + e4 : 0;
            const int lim = has ? len4 - e4 : 1;   // quads left in the row (>= 1)
            // quads past the row's end re-read quad e4 (no effect on the minimum)
            int mA = 64, mB = 64;
#pragma unroll
            for (int q = 0; q < kWalkQuads; q += 2) {
                const uint4 u = D4[lim > q ? a4 + q : a4];
                const uint4 v = D4[lim > q + 1 ? a4 + q + 1 : a4];
                mA = min(mA, min(min(__popc(u.x ^ P), __popc(u.y ^ P)), min(__popc(u.z ^ P), __popc(u.w ^ P))));
                mB = min(mB, min(min(__popc(v.x ^ P), __popc(v.y ^ P)), min(__popc(v.z ^ P), __popc(v.w ^ P))));
            }
            const int mn = min(mA, mB);
            if (kCount && has)
                c.cnt[kCntCmpReduce] += 4 * min(lim, kWalkQuads);
            const bool hit = has && mn <= d;
            e4 = hit ? 0 : e4 + kWalkQuads;
            r += hit ? 1 : 0;
            done = hit && r == nrows;
            if (hit && r < nrows) {
                off4 = cs.rank_off4[r];
                len4 = cs.rank_len4[r];
            }
            const bool dismiss = has && !hit && e4 >= len4;
            if (kCount && dismiss)
                c.cnt[kCntPruned] += 1;
            has = has && !dismiss;
        }
        // nodes that passed every filtered row go to the expansion queue
        const uint32_t bal = __ballot_sync(kFull, done);
        if (done) {
            queue[qn + __popc(bal & c.lt)] = P;
            has = false;
        }
        qn += __popc(bal);
        if (qn >= 32)
            break;
    }
    st[c.lane] = P;
    st[32 + c.lane] = (uint32_t)r | ((uint32_t)e4 << 8) | (has ? 0x80000000u : 0u);
    if (c.lane == 0) {
        st[64] = (uint32_t)pool_pos;
        st[65] = (uint32_t)pool_n;
        st[66] = exhausted ? 1u : 0u;
        st[67] = (uint32_t)(left_seen + 1);
    }
    __syncwarp();
    return qn;
}

// ---------------------------------------------------------------------------
// Quorum form (qPMS, q < n): a motif needs q of the n sequences, i.e. the
// seed's own sequence and q - 1 of the n - 1 rows; a candidate may miss up
// to n - q rows. Nodes and leaves carry a count of missed rows instead of
// being dropped at the first miss.

// Appends the codes of the lanes with `has` set to the instance's raw motifs.
__device__ __forceinline__ void emit_lanes(const WarpCtx &c, bool has, uint2 v)
{
    const MainParams &p = *c.p;
    const uint32_t bal = __ballot_sync(kFull, has);
    if (!bal)
        return;
    uint32_t base = 0;
    if (c.lane == 0)
        base = atomicAdd(&p.raw_count[c.I], (uint32_t)__popc(bal));
    base = __shfl_sync(kFull, base, 0);
    if (has) {
        const uint32_t pos = base + __popc(bal & c.lt);
        if (pos < c.in.raw_cap)
            p.raw[c.in.raw_off + pos] = to_key(v.x, v.y, c.in.l);
        else
            atomicOr(&p.flags[c.I], kFlagOverflow);
    }
}

// The listed leaves of node P against every row in order: a leaf is emitted
// as soon as it hits q - 1 rows, dropped once it misses more than n - q.
template <bool kCount>
__device__ __forceinline__ void finish_list_q(const WarpCtx &c, uint32_t P, int N)
{
    const InstDev &in = c.in;
    const int nrows = in.n - 1;
    const int budget = in.n - in.q, need = in.q - 1;
    uint2 *list = c.ws->list;
    uint8_t *lm = c.ws->u.q.lmiss;
    __syncwarp();
    for (int r = 0; r < nrows && N > 0; ++r) {
        const int ri = c.cs->row_order[r];
        const int len = c.cs->row_len[ri];
        const int off = c.cs->row_off[ri];
        const int k = len > 0 ? reduce_row(c.rows.D + off, c.rows.HL + off, len, P, in.d, c.ws->rb1, c.lane, c.lt) : 0;
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpReduce] += len;
        const bool sm = k <= kRbCap;
        int newN = 0;
        for (int b = 0; b < N; b += 32) {
            const int idx = b + c.lane;
            const bool alive = idx < N;
            uint2 v = make_uint2(0u, 0u);
            int ms = 0;
            if (alive) {
                v = list[idx];
                ms = lm[idx];
            }
            bool hit = false;
            if (alive && k > 0) {
                hit = sm ? check_smem(c.ws->rb1, k, v.x, v.y, in.d) : check_row(c.rows.HL + off, len, v.x, v.y, in.d);
                if (kCount)
                    c.cnt[kCntCmpVerify] += sm ? k : len;
            }
            if (alive && !hit)
                ++ms;
            const bool accept = alive && (r + 1 - ms) >= need;
            const bool keep = alive && !accept && ms <= budget;
            __syncwarp();
            emit_lanes(c, accept, v);
            const uint32_t bal = __ballot_sync(kFull, keep);
            if (keep) {
                const int pos = newN + __popc(bal & c.lt);
                list[pos] = v;
                lm[pos] = (uint8_t)ms;
            }
            newN += __popc(bal);
        }
        __syncwarp();
        N = newN;
    }
    __syncwarp();
}

// Every leaf of a node that survived the quorum filter goes through the rows.
template <bool kCount>
__device__ __forceinline__ void expand_subset_q(const WarpCtx &c, uint32_t P)
{
    const int lev = __popc(P);
    uint32_t t = P;
    const uint32_t b0 = t & (0u - t);
    t ^= b0;
    const uint32_t b1 = t & (0u - t);
    t ^= b1;
    const uint32_t b2 = t & (0u - t);
    t ^= b2;
    const uint32_t Phi = t;
    const int nlo = lev < 3 ? lev : 3;
    const int nlanes = nlo == 0 ? 1 : (nlo == 1 ? 3 : (nlo == 2 ? 9 : 27));
    const bool active = c.lane < nlanes;
    const int dg0 = c.lane % 3, dg1 = (c.lane / 3) % 3, dg2 = (c.lane / 9) % 3;
    const uint32_t DhLo = (dg0 >= 1 ? b0 : 0u) | (dg1 >= 1 ? b1 : 0u) | (dg2 >= 1 ? b2 : 0u);
    const uint32_t DlLo = (dg0 != 1 ? b0 : 0u) | (dg1 != 1 ? b1 : 0u) | (dg2 != 1 ? b2 : 0u);
    const uint32_t ch0 = c.xh ^ DhLo, cl0 = c.xl ^ DlLo;
    const unsigned long long iters = c_pow3[lev - nlo];
    uint2 *list = c.ws->list;
    int listN = 0;
    uint32_t Dh = 0u, Dl = Phi;
    for (unsigned long long it = 0; it < iters; ++it) {
        const uint32_t bal = __ballot_sync(kFull, active);
        if (active) {
            const int pos = listN + __popc(bal & c.lt);
            list[pos] = make_uint2(ch0 ^ Dh, cl0 ^ Dl);
            c.ws->u.q.lmiss[pos] = 0;
            if (kCount)
                c.cnt[kCntTested] += 1;
        }
        listN += __popc(bal);
        if (listN > kListCap - 32) {
            finish_list_q<kCount>(c, P, listN);
            listN = 0;
        }
        const uint32_t both = Dh & Dl;
        const uint32_t open = Phi & ~both;
        const uint32_t q = open & (0u - open);
        const uint32_t below = Phi & (q - 1u);
        Dh = (Dh & ~below) | q;
        Dl = (Dl | below) ^ q;
    }
    if (listN > 0)
        finish_list_q<kCount>(c, P, listN);
}

// Node filter with a miss budget: a node is dismissed once more than n - q of
// the filtered rows hold no occurrence meeting its bound.
template <bool kCount>
__device__ __forceinline__ int filter_subsets_q(const WarpCtx &c, int N)
{
    const InstDev &in = c.in;
    const int d = in.d;
    const int budget = in.n - in.q;
    const int nrows = min(in.prune_rows, in.n - 1);
    uint32_t *subs = c.ws->subs;
    uint8_t *sm = c.ws->u.q.smiss;
    for (int r = 0; r < nrows && N > 0; ++r) {
        const int ri = c.cs->row_order[r];
        const int len = c.cs->row_len[ri];
        const uint4 *D4 = reinterpret_cast<const uint4 *>(c.rows.D + c.cs->row_off[ri]);
        const int len4 = (len + 3) >> 2;
        int newN = 0;
        for (int b = 0; b < N; b += 32) {
            const int idx = b + c.lane;
            const bool alive = idx < N;
            const uint32_t P = alive ? subs[idx] : 0u;
            int ms = alive ? sm[idx] : 0;
            int m0 = 64, m1 = 64;
            for (int e4 = 0; e4 < len4; ++e4) {
                const uint4 v = D4[e4];
                m0 = min(m0, __popc(v.x ^ P));
                m1 = min(m1, __popc(v.y ^ P));
                m0 = min(m0, __popc(v.z ^ P));
                m1 = min(m1, __popc(v.w ^ P));
            }
            if (kCount && alive)
                c.cnt[kCntCmpReduce] += 4ull * len4;
            if (alive && min(m0, m1) > d)
                ++ms;
            const bool keep = alive && ms <= budget;
            __syncwarp();
            const uint32_t bal = __ballot_sync(kFull, keep);
            if (keep) {
                const int pos = newN + __popc(bal & c.lt);
                subs[pos] = P;
                sm[pos] = (uint8_t)ms;
            }
            newN += __popc(bal);
        }
        __syncwarp();
        N = newN;
    }
    return N;
}

// Queue item g of a launch: its instance, seed, chunk and chunk table.
struct ItemRef {
    int inst, seed, chunk, ctab;
};

__device__ __forceinline__ ItemRef decode_item(const MainParams &p, long long g)
{
    int lo = 0, hi = p.nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.seg[mid].work_lo <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    const Segment s = p.seg[lo];
    const int cidx = s.chunk_lo + (int)(g - s.work_lo);
    const int cps = s.cps > 0 ? s.cps : p.inst[s.inst].cps;
    return ItemRef{s.inst, s.seed_lo + cidx / cps, cidx % cps, s.cps > 0 ? s.ctab : p.inst[s.inst].ctab};
}

// Fewest unclaimed nodes an item must have for a CTA whose queue ran out to
// join it, and the rounds such a CTA looks for one before it stops.
constexpr int kStealMinNodes = 64;
constexpr int kStealTries = 16;

// Warp-cooperative choice of an item to join once the queue has run out: in
// each round the lanes read the unclaimed-node hints of 32 consecutive
// steal-cursor positions (the cursor cycles over the last items handed out,
// newest first) and the warp takes the item with the most if that is at least
// kStealMinNodes. A fruitless round sleeps a microsecond (items handed out
// last may not have published a hint yet). Returns the item, or -1 once every
// item's nodes are claimed or after kStealTries rounds.
__device__ __forceinline__ long long find_victim(const MainParams &p, int lane)
{
    const long long span = min(p.total, 2LL * (long long)gridDim.x);
    for (int t = 0; t < kStealTries; ++t) {
        unsigned int c0 = 0, ex = 0;
        if (lane == 0) {
            ex = *reinterpret_cast<volatile unsigned int *>(p.steal_state + 1);
            c0 = atomicAdd(p.steal_state, 32u);
        }
        ex = __shfl_sync(kFull, ex, 0);
        c0 = __shfl_sync(kFull, c0, 0);
        if ((long long)ex >= p.total)
            return -1;
        const long long g = p.total - 1 - (long long)((c0 + (unsigned int)lane) % (unsigned long long)span);
        const int left = *reinterpret_cast<volatile const int *>(p.item_claim + 2 * g + 1);
        int best = left;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            best = max(best, __shfl_xor_sync(kFull, best, o));
        if (best >= kStealMinNodes) {
            const int src = __ffs(__ballot_sync(kFull, left == best)) - 1;
            return __shfl_sync(kFull, g, src);
        }
        __nanosleep(1000);
    }
    return -1;
}

// Marks all nodes of item g claimed (an item that is done, or whose seed has
// no motif); the first to do so counts it in steal_state[1].
__device__ __forceinline__ void exhaust_item(const MainParams &p, long long g, int nodes)
{
    const int old = atomicMax(p.item_claim + 2 * g, nodes);
    if (old < nodes)
        atomicAdd(p.steal_state + 1, 1u);
}

// Gathers the feasible occurrences of seed `seed` (windows within 2d, from
// the compatibility masks) into shared memory when they fit, else into this
// CTA's global scratch, rows ordered smallest first and padded to multiples of
// 4 entries with copies of their last entry. Warp 0 derives the row order and
// offsets from the precomputed row sizes (two rows per lane, n <= 64) while
// every thread loads mask words; then each row's words are prefix-counted (a
// warp per row) and every thread fills destination slots directly: the slot's
// row by a binary search over the row offsets, its mask word by a binary
// search over the word counts, the window as the word's r-th set bit. So the
// only dependent global loads are one mask word and one window per slot, all
// issued by all threads at once. `scratch` (the warps' per-warp areas, unused
// between items) holds the mask words and counts; rows whose masks exceed it
// (more than 32 words, i.e. W > 1024, or too many rows) are gathered by the
// per-warp form below it. Works for any number of warps per CTA.

__device__ __forceinline__ void build_rows(const MainParams &p, const InstDev &in, int seed, CtaSmem &cs,
                                           uint32_t *smem_D, uint2 *smem_HL, uint32_t *glob_D, uint2 *glob_HL,
                                           int warp, int lane, unsigned long long *cnt, uint32_t *scratch)
{
    const int n = in.n, NW = in.NW, W = in.W, R = n - 1;
    const int *rl = p.rowlen + in.rlen_off + (size_t)seed * R;
    const uint32_t *mask = p.compat + in.compat_off + (size_t)seed * R * NW;
    const int nthreads = (int)blockDim.x, nwarps = nthreads >> 5;
    const int scratch_words = nwarps * (int)(sizeof(WarpSmem) / sizeof(uint32_t));
    const bool fast = NW <= 32 && 2 * R * NW <= scratch_words;
    uint32_t *sbits = scratch, *spre = scratch + R * NW;
    if (fast) {
        // every (row, word) of the seed's masks: the bits and their count
        for (int t = threadIdx.x; t < R * NW; t += nthreads) {
            const uint32_t b = __ldg(mask + t);
            sbits[t] = b;
            spre[t] = (uint32_t)__popc(b);
        }
    }
    if (warp == 0) {
        const int big = 0x7fffffff;
        const int la = lane < R ? rl[lane] : big;            // size of row (sequence) lane + 1
        const int lb = lane + 32 < R ? rl[lane + 32] : big;  // size of row lane + 33
        int ra = 0, rb = 0;                                  // ranks in smallest-first order
        for (int j = 0; j < R; ++j) {
            const int lj = __shfl_sync(kFull, j < 32 ? la : lb, j & 31);
            ra += (lj < la) || (lj == la && j < lane);
            rb += (lj < lb) || (lj == lb && j < lane + 32);
        }
        const int pa = lane < R ? (la + 3) & ~3 : 0, pb = lane + 32 < R ? (lb + 3) & ~3 : 0;
        int oa = 0, ob = 0, total = 0;                       // offsets: padded sizes of the rows ranked before
        for (int j = 0; j < R; ++j) {
            const int rj = __shfl_sync(kFull, j < 32 ? ra : rb, j & 31);
            const int pj = __shfl_sync(kFull, j < 32 ? pa : pb, j & 31);
            oa += rj < ra ? pj : 0;
            ob += rj < rb ? pj : 0;
            total += pj;
        }
        // a seed is hopeless when more rows are empty than the quorum may miss
        const int nempty = __popc(__ballot_sync(kFull, lane < R && la == 0)) +
                           __popc(__ballot_sync(kFull, lane + 32 < R && lb == 0));
        if (lane < R) {
            cs.row_len[lane + 1] = la;
            cs.row_off[lane + 1] = oa;
            cs.row_order[ra] = lane + 1;
            cs.rank_off4[ra] = oa >> 2;
            cs.rank_len4[ra] = pa >> 2;
        }
        if (lane + 32 < R) {
            cs.row_len[lane + 33] = lb;
            cs.row_off[lane + 33] = ob;
            cs.row_order[rb] = lane + 33;
            cs.rank_off4[rb] = ob >> 2;
            cs.rank_len4[rb] = pb >> 2;
        }
        if (lane == 0) {
            cs.total_rows = total;
            cs.feasible = nempty <= in.n - in.q;
            // the mismatch masks D, which every node scans, stay in shared memory up
            // to three times as many entries (the planes' room holds them too); only
            // the planes of occurrences that pass a node's bound are then read from
            // the global scratch
            cs.rows_in_smem = total <= p.smem_rows_cap ? 1 : (total <= 3 * p.smem_rows_cap ? 2 : 0);
            if (cnt)
                cnt[kCntCmpRows] += (unsigned long long)R * W;
        }
    }
    __syncthreads();
    if (!cs.feasible)
        return;
    uint32_t *Dd = cs.rows_in_smem != 0 ? smem_D : glob_D;
    uint2 *Hd = cs.rows_in_smem == 1 ? smem_HL : glob_HL;
    const uint2 *pl = p.planes + in.plane_off;
    const uint2 x = pl[seed];
    const int si = seed / W;   // the seed's own sequence has no row
    if (fast) {
        // exclusive prefix counts of each row's words (a warp per row)
        for (int k = warp; k < R; k += nwarps) {
            const int c = lane < NW ? (int)spre[k * NW + lane] : 0;
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o)
                    incl += y;
            }
            if (lane < NW)
                spre[k * NW + lane] = (uint32_t)(incl - c);
        }
        __syncthreads();
        const int total = cs.total_rows;
        for (int slot = threadIdx.x; slot < total; slot += nthreads) {
            // the rank whose padded row holds this slot: the last rank with offset <= slot
            int lo = 0, hi = R - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cs.rank_off4[mid] * 4 <= slot)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            // (an empty row shares its offset with the next rank and the rows are ordered by
            // size, so the last rank at or below the slot is a row with entries)
            const int i = cs.row_order[lo];
            const int len = cs.row_len[i];
            const int e = min(slot - cs.rank_off4[lo] * 4, len - 1);   // padding repeats the last entry
            const uint32_t *pre = spre + (i - 1) * NW;
            int t = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1)
                if (t + step < NW && (int)pre[t + step] <= e)
                    t += step;
            const int bt = nth_set_bit(sbits[(i - 1) * NW + t], e - (int)pre[t]);
            const uint2 *s = pl + (size_t)(i - 1 < si ? i - 1 : i) * W;
            const uint2 w = __ldg(s + 32 * t + bt);
            Hd[slot] = w;
            Dd[slot] = (x.x ^ w.x) | (x.y ^ w.y);
        }
        __syncthreads();
        return;
    }
    for (int i = 1 + warp; i < n; i += nwarps) {
        const uint32_t *mr = mask + (size_t)(i - 1) * NW;
        const uint2 *s = pl + (size_t)(i - 1 < si ? i - 1 : i) * W;
        const int off = cs.row_off[i];
        const int len = cs.row_len[i];
        int base = 0;
        for (int k0 = 0; k0 < NW; k0 += 32) {
            const int k = k0 + lane;
            const uint32_t bits = k < NW ? mr[k] : 0u;
            const int c = __popc(bits);
            int incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o)
                    incl += y;
            }
            const int chunk = __shfl_sync(kFull, incl, 31);
            // entry e of these 32 words goes to lane e % 32: its word t is the
            // number of words whose inclusive count is <= e, its bit the
            // (e - exclusive count of t)-th set bit of word t; all lanes load
            // their window at once
            for (int e0 = 0; e0 < chunk; e0 += 32) {
                const int e = e0 + lane;
                int t = 0;
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int v = __shfl_sync(kFull, incl, t + step - 1);
                    if (v <= e)
                        t += step;
                }
                const uint32_t wb = __shfl_sync(kFull, bits, t);
                const int before = __shfl_sync(kFull, incl, t) - __shfl_sync(kFull, c, t);
                if (e < chunk) {
                    const int bt = nth_set_bit(wb, e - before);
                    const uint2 w = s[32 * (k0 + t) + bt];
                    Hd[off + base + e] = w;
                    Dd[off + base + e] = (x.x ^ w.x) | (x.y ^ w.y);
                }
            }
            base += chunk;
        }
        __syncwarp();
        const int padded = (len + 3) & ~3;
        if (len > 0 && lane < padded - len) {
            Hd[off + len + lane] = Hd[off + len - 1];
            Dd[off + len + lane] = Dd[off + len - 1];
        }
    }
    __syncthreads();
}

// kRowsCap: row entries held in shared memory; kMinBlocks: resident CTAs per
// SM the register allocation is bounded for (3 with 2560 entries, 4 with 1280).
template <bool kCount, int kRowsCap, int kMinBlocks>
__global__ void __launch_bounds__(kMainThreads, kMinBlocks) main_kernel(MainParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem *wsm = reinterpret_cast<WarpSmem *>(smem_raw);
    uint32_t *smem_D = reinterpret_cast<uint32_t *>(smem_raw + kMainWarps * sizeof(WarpSmem));
    uint2 *smem_HL = reinterpret_cast<uint2 *>(smem_raw + kMainWarps * sizeof(WarpSmem) + kRowsCap * sizeof(uint32_t));
    CtaSmem &cs = *reinterpret_cast<CtaSmem *>(smem_raw + kMainWarps * sizeof(WarpSmem) +
                                               kRowsCap * (sizeof(uint32_t) + sizeof(uint2)));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    // rows_cap is a multiple of 4 words, so each CTA's slice and its plane
    // part start on 16-byte boundaries (the row loops use 16-byte loads)
    uint32_t *glob_D = p.scratch + (size_t)blockIdx.x * 3 * (size_t)p.rows_cap;
    uint2 *glob_HL = reinterpret_cast<uint2 *>(glob_D + p.rows_cap);
    unsigned long long cnt[kCount ? kCntNum : 1];
#pragma unroll
    for (int i = 0; i < (kCount ? kCntNum : 1); ++i)
        cnt[i] = 0;

    if (threadIdx.x == 0) {
        cs.cached_inst = -1;
        cs.cached_seed = -1;
        cs.feasible = 0;
    }
    for (int i = threadIdx.x; i < (kLMax + 1) * (kLMax + 1); i += blockDim.x)
        (&cs.binom[0][0])[i] = (&c_binom[0][0])[i];
    // launched as a programmatic dependent of the previous kernel: nothing
    // above reads its output; wait here until it has completed and its
    // writes are visible (without the launch attribute this returns at once)
    asm volatile("griddepcontrol.wait;" ::: "memory");
    bool draining = false;   // warp 0: the queue has run out, items are joined through the steal cursor
    for (;;) {
        if (warp == 0) {
            long long g = -1;
            if (!draining) {
                unsigned long long h = 0;
                if (lane == 0)
                    h = atomicAdd(p.head, 1ull);
                h = __shfl_sync(kFull, h, 0);
                if (h < (unsigned long long)p.total)
                    g = (long long)h;
                else
                    draining = p.item_claim != nullptr;
            }
            bool stolen = false;
            if (g < 0 && draining) {
                g = find_victim(p, lane);
                stolen = g >= 0;
            }
            if (lane == 0) {
                cs.g = g < 0 ? ~0ull : (unsigned long long)g;
                cs.stolen = stolen;
                if (g >= 0) {
                    const ItemRef it = decode_item(p, g);
                    cs.inst = it.inst;
                    cs.seed = it.seed;
                    cs.chunk = it.chunk;
                    cs.ctab = it.ctab;
                }
            }
        }
        __syncthreads();
        if (cs.g == ~0ull) {
            // no item left for this CTA: the sort kernel may launch (it waits
            // for this grid to complete before it reads anything)
            asm volatile("griddepcontrol.launch_dependents;");
            break;
        }
        const int I = cs.inst, seed = cs.seed, chunk = cs.chunk;
        const InstDev in = p.inst[I];
        const int *tab = p.ctab + cs.ctab;
        const int g0 = tab[in.d + 2 + 2 * chunk];
        const int g1 = tab[in.d + 2 + 2 * chunk + 1];
        if (p.mode && p.mode[in.seed_off + seed] != kModeTree) {
            if (threadIdx.x == 0 && p.item_claim)
                exhaust_item(p, (long long)cs.g, g1 - g0);
            __syncthreads();   // this seed is searched by the pair kernel
            continue;
        }
        const bool rebuild = (I != cs.cached_inst) || (seed != cs.cached_seed);
        if (rebuild) {
            build_rows(p, in, seed, cs, smem_D, smem_HL, glob_D, glob_HL, warp, lane, kCount ? cnt : nullptr,
                       reinterpret_cast<uint32_t *>(smem_raw));
            if (threadIdx.x == 0) {
                cs.cached_inst = I;
                cs.cached_seed = seed;
            }
        }
        if (threadIdx.x == 0) {
            cs.next = g0;
            // no node of an infeasible seed is searched: nothing for other CTAs to join
            if (p.item_claim && !cs.feasible)
                exhaust_item(p, (long long)cs.g, g1 - g0);
        }
        __syncthreads();
        if constexpr (kCount) {
            if (threadIdx.x == 0 && chunk == 0 && !cs.feasible && !cs.stolen)
                cnt[kCntSeedsInfeasible] += 1;
        }
        if (cs.feasible) {
            const uint2 x = p.planes[in.plane_off + seed];
            Rows rows{cs.rows_in_smem != 0 ? smem_D : glob_D, cs.rows_in_smem == 1 ? smem_HL : glob_HL};
            WarpCtx c{&p, in, I, lane, lt, x.x, x.y, rows, &cs, &wsm[warp], kCount ? cnt : nullptr};
            if (in.q < in.n) {
                // quorum form: batches of nodes with miss budgets, claimed from the
                // item's shared counter when other CTAs may join it; batches shrink
                // (guided) as the item runs out so that its warps finish together
                uint32_t *subs = wsm[warp].subs;
                int *ctr = p.item_claim ? p.item_claim + 2 * cs.g : &cs.next;
                const int base = p.item_claim ? g0 : 0;
                for (;;) {
                    int start = 0, batch = kSubBatch;
                    if (lane == 0) {
                        const int left = g1 - (base + *reinterpret_cast<volatile int *>(ctr));
                        batch = min(kSubBatch, max(32, ((left + 2 * kMainWarps - 1) / (2 * kMainWarps) + 31) & ~31));
                        start = base + atomicAdd(ctr, batch);
                        if (p.item_claim) {
                            ctr[1] = max(0, g1 - (start + batch));
                            if (start < g1 && start + batch >= g1)
                                atomicAdd(p.steal_state + 1, 1u);
                        }
                    }
                    start = __shfl_sync(kFull, start, 0);
                    batch = __shfl_sync(kFull, batch, 0);
                    if (start >= g1)
                        break;
                    const int N = min(batch, g1 - start);
                    for (int j = lane; j < N; j += 32) {
                        const int g = start + j;
                        int lev = 0;
                        while (tab[lev + 1] <= g)
                            ++lev;
                        subs[j] = unrank_subset((uint32_t)(g - tab[lev]), lev, in.l, cs.binom);
                        wsm[warp].u.q.smiss[j] = 0;
                    }
                    __syncwarp();
                    if constexpr (kCount) {
                        if (lane == 0)
                            cnt[kCntSubsets] += N;
                    }
                    const int S = filter_subsets_q<kCount>(c, N);
                    if constexpr (kCount) {
                        if (lane == 0)
                            cnt[kCntPruned] += N - S;
                    }
                    for (int sidx = 0; sidx < S; ++sidx)
                        expand_subset_q<kCount>(c, subs[sidx]);
                    __syncwarp();
                }
            } else if (in.grab == 1) {
                // nodes are claimed from the item's shared counter when other
                // CTAs may join it, else from the CTA's own
                int *ctr = p.item_claim ? p.item_claim + 2 * cs.g : &cs.next;
                const int base = p.item_claim ? g0 : 0;
                unsigned int *exh = p.item_claim ? p.steal_state + 1 : nullptr;
                walk_init(c);
                for (;;) {
                    bool fin;
                    const int qn = walk_run<kCount>(c, tab, g0, g1, cs, ctr, base, exh, fin);
                    const uint32_t *queue = wsm[warp].subs + 64;
                    for (int i = 0; i < qn; ++i)
                        expand_subset<kCount>(c, queue[i]);
                    __syncwarp();
                    if (fin)
                        break;
                }
            } else {
                uint32_t *subs = wsm[warp].subs;
                // batch filter: batches of up to kSubBatch subsets (large batches
                // keep the breadth-first filter's lanes full), small chunks split
                // so that every warp gets work; with in.grab > 1 batches shrink
                // toward in.grab as the chunk runs out (guided self-scheduling);
                // in.grab == 1 selects the lane walk above instead
                const int per_warp = (g1 - g0 + 2 * kMainWarps - 1) / (2 * kMainWarps);
                const int fixed = min(kSubBatch, max(32, (per_warp + 31) & ~31));
                for (;;) {
                    int start = 0, batch = fixed;
                    if (lane == 0) {
                        if (in.grab > 1) {
                            const int left = g1 - *reinterpret_cast<volatile int *>(&cs.next);
                            batch = min(fixed, max(in.grab, ((left + 2 * kMainWarps - 1) / (2 * kMainWarps) + 31) & ~31));
                        }
                        start = atomicAdd(&cs.next, batch);
                    }
                    start = __shfl_sync(kFull, start, 0);
                    batch = __shfl_sync(kFull, batch, 0);
                    if (start >= g1)
                        break;
                    const int N = min(batch, g1 - start);
                    for (int j = lane; j < N; j += 32) {
                        const int g = start + j;
                        int lev = 0;
                        while (tab[lev + 1] <= g)
                            ++lev;
                        subs[j] = unrank_subset((uint32_t)(g - tab[lev]), lev, in.l, cs.binom);
                    }
                    __syncwarp();
                    if constexpr (kCount) {
                        if (lane == 0)
                            cnt[kCntSubsets] += N;
                    }
                    const int S = filter_subsets<kCount>(c, N);
                    if constexpr (kCount) {
                        if (lane == 0)
                            cnt[kCntPruned] += N - S;
                    }
                    for (int sidx = 0; sidx < S; ++sidx)
                        expand_subset<kCount>(c, subs[sidx]);
                    __syncwarp();
                }
            }
        }
        // warp 0 is past its last claim, so every node of the item is claimed
        if (threadIdx.x == 0 && p.item_claim)
            exhaust_item(p, (long long)cs.g, g1 - g0);
        __syncthreads();
    }
    if constexpr (kCount) {
#pragma unroll
        for (int i = 0; i < kCntNum; ++i) {
            unsigned long long v = cnt[i];
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0 && v)
                atomicAdd(&p.counters[i], v);
        }
    }
}

// ---------------------------------------------------------------------------
// Pair form (Observation 3.3 with q = n): a motif is within d of an l-mer x
// of s_1 and of an l-mer r of s_2, so it lies in B(x, d) & B(r, d), and
// d_H(x, r) <= 2d (the s_2 row of x's compatibility masks). Let D = d_H(x, r),
// Delta the positions where x and r differ. A string c of the intersection
// changes a of the l - D agreeing positions (3 letters each), gives t of the
// differing positions a third letter (2 each), keeps x's letter on e_x of the
// others and takes r's on the rest, with a + t + (D - t - e_x) <= d and
// a + t + e_x <= d. Such c can only be within d of a window w if
// popc(mism(x, w) & mism(r, w)) <= min(2d, 3d - D): c agrees with x or r
// everywhere except on at most min(d, 2d - D) positions.

// Pair bound for one row entry w (D_w = mism(x, w) is stored with the entry).
__device__ __forceinline__ bool pair_ok(uint32_t Dw, uint2 w, uint2 r, int bound)
{
    return __popc(Dw & ((r.x ^ w.x) | (r.y ^ w.y))) <= bound;
}

__device__ __forceinline__ bool row_has_pair(const uint32_t *D, const uint2 *HL, int len, uint2 r, int bound, int lane)
{
    for (int e0 = 0; e0 < len; e0 += 32) {
        const int e = e0 + lane;
        const bool q = e < len && pair_ok(D[e], HL[e], r, bound);
        if (__any_sync(kFull, q))
            return true;
    }
    return false;
}

// Row entries meeting the pair bound, into rb (padded to 4); returns how many.
__device__ __forceinline__ int reduce_row_pair(const uint32_t *D, const uint2 *HL, int len, uint2 r, int bound,
                                               uint2 *rb, int lane, uint32_t lt)
{
    int k = 0;
    for (int e0 = 0; e0 < len; e0 += 32) {
        const int e = e0 + lane;
        uint2 w = make_uint2(0u, 0u);
        bool keep = false;
        if (e < len) {
            w = HL[e];
            keep = pair_ok(D[e], w, r, bound);
        }
        const uint32_t bal = __ballot_sync(kFull, keep);
        if (keep) {
            const int pos = k + __popc(bal & lt);
            if (pos < kRbCap)
                rb[pos] = w;
        }
        k += __popc(bal);
    }
    __syncwarp();
    if (k > 0 && k <= kRbCap && lane < 4)
        rb[k + lane] = rb[k - 1];
    __syncwarp();
    return k;
}

struct PairCtx {
    uint2 r;          // planes of the s_2 window
    int bound;        // pair bound
    int row0;         // sequence of the first verified row (smallest of s_3..s_n)
};

// Candidates of one pair that passed row 0: checked against the other rows
// (s_3..s_n without row 0, each reduced by the pair bound), then emitted.
template <bool kCount>
__device__ __forceinline__ void finish_list_pair(const WarpCtx &c, const PairCtx &pc, int N)
{
    const InstDev &in = c.in;
    const int nrows = in.n - 1;
    uint2 *list = c.ws->list;
    __syncwarp();
    for (int rr = 0; rr < nrows && N > 0; ++rr) {
        const int ri = c.cs->row_order[rr];
        if (ri == 1 || ri == pc.row0)
            continue;
        const int len = c.cs->row_len[ri];
        const int off = c.cs->row_off[ri];
        const int k = reduce_row_pair(c.rows.D + off, c.rows.HL + off, len, pc.r, pc.bound, c.ws->rb1, c.lane, c.lt);
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpReduce] += len;
        if (k == 0) {
            N = 0;
            break;
        }
        const bool sm = k <= kRbCap;
        int newN = 0;
        for (int b = 0; b < N; b += 32) {
            const int idx = b + c.lane;
            const bool alive = idx < N;
            uint2 v = make_uint2(0u, 0u);
            if (alive)
                v = list[idx];
            bool hit = false;
            if (alive) {
                hit = sm ? check_smem(c.ws->rb1, k, v.x, v.y, in.d) : check_row(c.rows.HL + off, len, v.x, v.y, in.d);
                if (kCount)
                    c.cnt[kCntCmpVerify] += sm ? k : len;
            }
            __syncwarp();
            const uint32_t bal = __ballot_sync(kFull, hit);
            if (hit)
                list[newN + __popc(bal & c.lt)] = v;
            newN += __popc(bal);
        }
        __syncwarp();
        N = newN;
    }
    if (N > 0)
        emit<kCount>(c, list, N);
}

// Deposit table of the differing positions: lut[16 k + v] = the positions of
// Delta numbered 4k..4k+3 selected by the 4 bits of v.
__device__ __forceinline__ void build_deposit_lut(uint32_t Delta, uint32_t *lut, int lane)
{
    for (int e = lane; e < 128; e += 32) {
        const int k = e >> 4, v = e & 15;
        uint32_t m = Delta;
        for (int s = 0; s < 4 * k; ++s)
            m &= m - 1u;
        uint32_t dep = 0;
        for (int j = 0; j < 4; ++j) {
            const uint32_t low = m & (0u - m);
            if ((v >> j) & 1)
                dep |= low;
            m ^= low;
        }
        lut[e] = dep;
    }
    __syncwarp();
}

// Maps a mask over the numbered differing positions to the positions themselves.
__device__ __forceinline__ uint32_t deposit_delta(uint32_t c, const uint32_t *lut, int nibbles)
{
    uint32_t r = 0;
    for (int k = 0; k < nibbles; ++k)
        r |= lut[k * 16 + ((c >> (4 * k)) & 15u)];
    return r;
}

// Inserts a 0 bit at every set position of Tc (ascending), i.e. maps a mask
// over the differing positions outside T onto the numbering of all of them.
__device__ __forceinline__ uint32_t skip_positions(uint32_t c, uint32_t Tc)
{
    while (Tc) {
        const uint32_t low = Tc & (0u - Tc);
        const uint32_t below = low - 1u;
        c = ((c & ~below) << 1) | (c & below);
        Tc ^= low;
    }
    return c;
}

// Next k-subset in colex order (next larger integer with the same popcount).
__device__ __forceinline__ uint32_t next_combination(uint32_t v)
{
    const uint32_t u = v & (0u - v);
    const uint32_t w = v + u;
    return w | (((w ^ v) >> 2) >> (__ffs(v) - 1));
}

// All leaves of one pair: classes (a, t, e_x) in a warp-uniform loop; inside a
// class the choices on agreeing positions, the third-letter set T and its
// letters are warp-uniform too, and lanes own contiguous ranges of the e_x
// subsets (unranked once, then stepped in colex order).
template <bool kCount, int kReg>
__device__ __forceinline__ void pair_leaves(const WarpCtx &c, const PairCtx &pc, uint32_t Delta, uint32_t Agree, int D,
                                            int k0, int len0, int off0, const uint32_t (*binom)[kLMax + 1])
{
    const InstDev &in = c.in;
    const int d = in.d, l = in.l;
    const bool no_rows = in.n <= 2;
    const uint32_t GH = c.xh ^ pc.r.x, GL = c.xl ^ pc.r.y;   // per position XOR code of x and r
    uint32_t *lut = c.ws->subs;
    build_deposit_lut(Delta, lut, c.lane);
    const int nib = (D + 3) >> 2;
    uint2 e[kReg > 0 ? kReg : 1];
    if constexpr (kReg > 0) {
#pragma unroll
        for (int i = 0; i < kReg; ++i)
            e[i] = c.ws->rb0[i < k0 ? i : k0 - 1];
    }
    const bool sm0 = k0 <= kRbCap;
    uint2 *list = c.ws->list;
    int listN = 0;
    const int nAg = l - D;
    for (int a = 0; a <= min(d, nAg); ++a) {
        for (int t = 0; t <= min(D, d - a); ++t) {
            for (int ex = 0; ex <= D - t; ++ex) {
                const int er = D - t - ex;
                if (a + t + er > d || a + t + ex > d)
                    continue;
                const uint32_t nA = binom[nAg][a], nT = binom[D][t], nE = binom[D - t][ex];
                const uint32_t per = (nE + 31) / 32;              // e_x subsets per lane
                const uint32_t lo = min(nE, c.lane * per), hi = min(nE, lo + per);
                // first e_x subset of this lane (numbered over the D - t positions outside T)
                const uint32_t e_first = lo < hi ? unrank_subset(lo, ex, D - t, binom) : 0u;
                uint32_t Pa = a ? ((1u << a) - 1u) : 0u;           // compact a-subset of the agreeing positions
                for (uint32_t iA = 0; iA < nA; ++iA) {
                    // deposit Pa onto the agreeing positions
                    uint32_t PaM = 0, m = Agree, q = Pa;
                    while (q) {
                        const uint32_t low = m & (0u - m);
                        if (q & 1u)
                            PaM |= low;
                        m ^= low;
                        q >>= 1;
                    }
                    // odometer over the letters of the a changed agreeing positions
                    uint32_t DhA = 0u, DlA = PaM;
                    const unsigned long long nsub = c_pow3[a];
                    for (unsigned long long sub = 0; sub < nsub; ++sub) {
                        uint32_t Tc = t ? ((1u << t) - 1u) : 0u;   // compact t-subset of the differing positions
                        for (uint32_t iT = 0; iT < nT; ++iT) {
                            const uint32_t TM = deposit_delta(Tc, lut, nib);
                            const uint32_t R = Delta & ~TM;
                            for (uint32_t wbits = 0; wbits < (1u << t); ++wbits) {
                                // third letters on T: choice bits spread over T's positions
                                uint32_t Wm = 0, mt = TM, wb = wbits;
                                while (wb) {
                                    const uint32_t low = mt & (0u - mt);
                                    if (wb & 1u)
                                        Wm |= low;
                                    mt ^= low;
                                    wb >>= 1;
                                }
                                const uint32_t dHT = (Wm | (GL & ~GH)) & TM;
                                const uint32_t dLT = ((GH & ~GL) | (Wm ^ (GH & GL))) & TM;
                                const uint32_t bh = c.xh ^ DhA ^ dHT ^ (GH & R);
                                const uint32_t bl = c.xl ^ DlA ^ dLT ^ (GL & R);
                                uint32_t ec = e_first;
                                for (uint32_t i0 = 0; i0 < per; ++i0) {
                                    const bool act = lo + i0 < hi;
                                    const uint32_t Ex = act ? deposit_delta(skip_positions(ec, Tc), lut, nib) : 0u;
                                    const uint32_t ch = bh ^ (GH & Ex), cl = bl ^ (GL & Ex);
                                    bool hit = false;
                                    if (act) {
                                        if (no_rows) {
                                            hit = true;
                                        } else if constexpr (kReg > 0) {
                                            int m0 = 64, m1 = 64;
#pragma unroll
                                            for (int i = 0; i < kReg; i += 2) {
                                                m0 = min(m0, __popc((ch ^ e[i].x) | (cl ^ e[i].y)));
                                                m1 = min(m1, __popc((ch ^ e[i + 1].x) | (cl ^ e[i + 1].y)));
                                            }
                                            hit = min(m0, m1) <= d;
                                        } else {
                                            hit = sm0 ? check_smem(c.ws->rb0, k0, ch, cl, d)
                                                      : check_row(c.rows.HL + off0, len0, ch, cl, d);
                                        }
                                        if (kCount) {
                                            c.cnt[kCntTested] += 1;
                                            c.cnt[kCntCmpVerify] += no_rows ? 0 : (sm0 ? k0 : len0);
                                        }
                                        if (ex > 0 && lo + i0 + 1 < hi)
                                            ec = next_combination(ec);
                                    }
                                    const uint32_t bal = __ballot_sync(kFull, hit);
                                    if (bal) {
                                        if (hit)
                                            list[listN + __popc(bal & c.lt)] = make_uint2(ch, cl);
                                        listN += __popc(bal);
                                        if (listN > kListCap - 32) {
                                            finish_list_pair<kCount>(c, pc, listN);
                                            listN = 0;
                                        }
                                    }
                                }
                            }
                            if (t > 0 && iT + 1 < nT)
                                Tc = next_combination(Tc);
                        }
                        // odometer step over PaM (as in the tree form)
                        const uint32_t both = DhA & DlA;
                        const uint32_t open = PaM & ~both;
                        const uint32_t qq = open & (0u - open);
                        const uint32_t below = PaM & (qq - 1u);
                        DhA = (DhA & ~below) | qq;
                        DlA = (DlA | below) ^ qq;
                    }
                    if (a > 0 && iA + 1 < nA)
                        Pa = next_combination(Pa);
                }
            }
        }
    }
    if (listN > 0)
        finish_list_pair<kCount>(c, pc, listN);
}

template <bool kCount>
__device__ __forceinline__ void process_pair(const WarpCtx &c, uint2 r, const uint32_t (*binom)[kLMax + 1])
{
    const InstDev &in = c.in;
    const int d = in.d, l = in.l;
    const uint32_t lmask = l == 32 ? 0xffffffffu : ((1u << l) - 1u);
    const uint32_t Delta = ((c.xh ^ r.x) | (c.xl ^ r.y)) & lmask;
    const int D = __popc(Delta);
    const uint32_t Agree = lmask & ~Delta;
    PairCtx pc{r, min(2 * d, 3 * d - D), 0};
    if (kCount && c.lane == 0)
        c.cnt[kCntSubsets] += 1;
    // every row s_3..s_n must hold an occurrence meeting the pair bound
    const int nrows = in.n - 1;
    int r0 = 0;
    for (int rr = 0; rr < nrows; ++rr) {
        const int ri = c.cs->row_order[rr];
        if (ri == 1)
            continue;
        if (r0 == 0)
            r0 = ri;
        const int off = c.cs->row_off[ri];
        const bool ok = row_has_pair(c.rows.D + off, c.rows.HL + off, c.cs->row_len[ri], r, pc.bound, c.lane);
        if (kCount && c.lane == 0)
            c.cnt[kCntCmpReduce] += c.cs->row_len[ri];
        if (!ok) {
            if (kCount && c.lane == 0)
                c.cnt[kCntPruned] += 1;
            return;
        }
    }
    pc.row0 = r0;
    int k0 = 0, len0 = 0, off0 = 0;
    if (r0) {
        len0 = c.cs->row_len[r0];
        off0 = c.cs->row_off[r0];
        k0 = reduce_row_pair(c.rows.D + off0, c.rows.HL + off0, len0, r, pc.bound, c.ws->rb0, c.lane, c.lt);
        if (k0 == 0)
            return;
    }
    if (!r0 || k0 > 8)
        pair_leaves<kCount, 0>(c, pc, Delta, Agree, D, k0, len0, off0, binom);
    else if (k0 <= 4)
        pair_leaves<kCount, 4>(c, pc, Delta, Agree, D, k0, len0, off0, binom);
    else
        pair_leaves<kCount, 8>(c, pc, Delta, Agree, D, k0, len0, off0, binom);
}

// Pair-form kernel: queue items are (instance, seed x, block of 64 windows of
// s_2); the CTA gathers x's feasible occurrences, its warps take the pairs
// (x, r) of the block (r within 2d of x) one at a time. Seeds whose mode is
// not kModePair are left to the tree kernel.
template <bool kCount>
__global__ void __launch_bounds__(kThreads, 2) pair_kernel(MainParams p)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    WarpSmem *wsm = reinterpret_cast<WarpSmem *>(smem_raw);
    uint32_t *smem_D = reinterpret_cast<uint32_t *>(smem_raw + kWarps * sizeof(WarpSmem));
    uint2 *smem_HL = reinterpret_cast<uint2 *>(smem_raw + kWarps * sizeof(WarpSmem) + kRowSmemCap * sizeof(uint32_t));
    CtaSmem &cs = *reinterpret_cast<CtaSmem *>(smem_raw + kWarps * sizeof(WarpSmem) +
                                               kRowSmemCap * (sizeof(uint32_t) + sizeof(uint2)));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t *glob_D = p.scratch + (size_t)blockIdx.x * 3 * (size_t)p.rows_cap;
    uint2 *glob_HL = reinterpret_cast<uint2 *>(glob_D + p.rows_cap);
    unsigned long long cnt[kCount ? kCntNum : 1];
#pragma unroll
    for (int i = 0; i < (kCount ? kCntNum : 1); ++i)
        cnt[i] = 0;
    if (threadIdx.x == 0) {
        cs.cached_inst = -1;
        cs.cached_seed = -1;
        cs.feasible = 0;
    }
    for (int i = threadIdx.x; i < (kLMax + 1) * (kLMax + 1); i += blockDim.x)
        (&cs.binom[0][0])[i] = (&c_binom[0][0])[i];
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned long long g = atomicAdd(p.head, 1ull);
            cs.g = g;
            if (g < (unsigned long long)p.total) {
                int lo = 0, hi = p.nseg - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (p.seg[mid].work_lo <= (long long)g)
                        lo = mid;
                    else
                        hi = mid - 1;
                }
                const Segment s = p.seg[lo];
                const int cidx = s.chunk_lo + (int)((long long)g - s.work_lo);
                const int cps = p.inst[s.inst].cps_b;
                cs.inst = s.inst;
                cs.seed = cidx / cps;
                cs.chunk = cidx % cps;
            }
        }
        __syncthreads();
        if (cs.g >= (unsigned long long)p.total)
            break;
        const int I = cs.inst, seed = cs.seed, chunk = cs.chunk;
        const InstDev in = p.inst[I];
        if (!p.mode || p.mode[in.seed_off + seed] != kModePair) {
            __syncthreads();
            continue;
        }
        const bool rebuild = (I != cs.cached_inst) || (seed != cs.cached_seed);
        if (rebuild) {
            build_rows(p, in, seed, cs, smem_D, smem_HL, glob_D, glob_HL, warp, lane, kCount ? cnt : nullptr,
                       reinterpret_cast<uint32_t *>(smem_raw));
            if (threadIdx.x == 0) {
                cs.cached_inst = I;
                cs.cached_seed = seed;
            }
        }
        if (threadIdx.x == 0)
            cs.next = 0;
        __syncthreads();
        if (cs.feasible) {
            const uint2 *pl = p.planes + in.plane_off;
            const uint2 x = pl[seed];
            Rows rows{cs.rows_in_smem != 0 ? smem_D : glob_D, cs.rows_in_smem == 1 ? smem_HL : glob_HL};
            WarpCtx c{&p, in, I, lane, lt, x.x, x.y, rows, &cs, &wsm[warp], kCount ? cnt : nullptr};
            // the pairs of this block: set bits of x's s_2 mask words 2 chunk, 2 chunk + 1
            const uint32_t *mrow = p.compat + in.compat_off + (size_t)seed * (in.n - 1) * in.NW;
            const int w0 = 2 * chunk;
            const uint32_t m0 = w0 < in.NW ? mrow[w0] : 0u;
            const uint32_t m1 = w0 + 1 < in.NW ? mrow[w0 + 1] : 0u;
            const int npairs = __popc(m0) + __popc(m1);
            for (;;) {
                int q = 0;
                if (lane == 0)
                    q = atomicAdd(&cs.next, 1);
                q = __shfl_sync(kFull, q, 0);
                if (q >= npairs)
                    break;
                // q-th set bit of (m0, m1)
                int bit;
                if (q < __popc(m0)) {
                    bit = __fns(m0, 0, q + 1);
                } else {
                    bit = 32 + __fns(m1, 0, q - __popc(m0) + 1);
                }
                const int rw = 64 * chunk + bit;
                process_pair<kCount>(c, pl[(size_t)in.W + rw], cs.binom);
            }
        }
        __syncthreads();
    }
    if constexpr (kCount) {
#pragma unroll
        for (int i = 0; i < kCntNum; ++i) {
            unsigned long long v = cnt[i];
            for (int o = 16; o > 0; o >>= 1)
                v += __shfl_xor_sync(kFull, v, o);
            if (lane == 0 && v)
                atomicAdd(&p.counters[i], v);
        }
    }
}

// Seed modes: a seed uses the pair form unless one of its pairs is closer
// than d + 1 (then the intersection B(x, d) & B(r, d) is large and dominated
// by changes on agreeing positions, which the tree form covers better).
__global__ void classify_kernel(const InstDev *__restrict__ inst, int ninst, const long long *__restrict__ seed_prefix,
                                long long total_seeds, const uint2 *__restrict__ planes,
                                const uint32_t *__restrict__ compat, uint8_t *__restrict__ mode)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < total_seeds; q += warps) {
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (seed_prefix[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        const InstDev in = inst[lo];
        const int j = (int)(q - seed_prefix[lo]);
        bool close = in.n < 2;
        if (!close) {
            const uint2 *pl = planes + in.plane_off;
            const uint2 x = pl[j];
            const uint32_t *mrow = compat + in.compat_off + (size_t)j * (in.n - 1) * in.NW;
            for (int w0 = 0; w0 < in.W && !close; w0 += 32) {
                const int w = w0 + lane;
                bool c = false;
                if (w < in.W && ((mrow[w >> 5] >> (w & 31)) & 1u)) {
                    const uint2 r = pl[(size_t)in.W + w];
                    c = __popc((x.x ^ r.x) | (x.y ^ r.y)) <= in.d;
                }
                close = __any_sync(kFull, c);
            }
        }
        if (lane == 0)
            mode[in.seed_off + j] = close ? kModeTree : kModePair;
    }
}

// Compatibility masks (the pair-distance table of PMS8): for every seed
// x = s_1[j..j+l-1] and every sequence i >= 2, bit w of row (j, i) is set iff
// d_H(x, s_i[w..w+l-1]) <= 2d. One warp per (instance, seed, row).
__global__ void compat_kernel(const InstDev *__restrict__ inst, int ninst, const long long *__restrict__ row_prefix,
                              long long total_rows, const uint2 *__restrict__ planes, uint32_t *__restrict__ compat,
                              int *__restrict__ rowlen)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long q = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < total_rows; q += warps) {
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (row_prefix[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        const InstDev in = inst[lo];
        const long long local = q - row_prefix[lo];
        // seed j numbers the l-mers of the seed sequences (W each); row k of a
        // seed of sequence si is sequence k (k < si) or k + 1 (k >= si)
        const int j = (int)(local / (in.n - 1)), k = (int)(local % (in.n - 1));
        const int si = j / in.W;
        const int i = k < si ? k : k + 1;
        const uint2 *pl = planes + in.plane_off;
        const uint2 x = pl[j];
        const uint2 *s = pl + (size_t)i * in.W;
        uint32_t *out = compat + in.compat_off + (size_t)local * in.NW;
        const int lim = 2 * in.d;
        int total = 0;
        // four 32-window groups per step, their loads issued together
        for (int w0 = 0; w0 < in.W; w0 += 128) {
            uint2 e[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int w = w0 + 32 * u + lane;
                e[u] = w < in.W ? s[w] : make_uint2(~x.x, ~x.y);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int w = w0 + 32 * u + lane;
                const bool keep = w < in.W && __popc((x.x ^ e[u].x) | (x.y ^ e[u].y)) <= lim;
                const uint32_t bal = __ballot_sync(kFull, keep);
                total += __popc(bal);
                if (lane == 0 && w0 + 32 * u < in.W)
                    out[(w0 >> 5) + u] = bal;
            }
        }
        if (lane == 0)
            rowlen[in.rlen_off + local] = total;
    }
}

// The same masks for a one-instance plan, by row, with the packing folded in:
// a CTA reads the bytes of one sequence i once, as two bit-planes of the whole
// sequence (a ballot per 32 positions), cuts every window's planes out of them
// with funnel shifts (the CTA of the first seed block also writes them out for
// the later kernels and flags bytes other than A/C/G/T), packs the planes of
// its 16 seeds (2 per warp, one byte per lane and two ballots), and builds row
// i of those seeds' masks from the staged planes. The planes are thus read
// from L2 not at all, and the separate pack launch is not needed.
constexpr int kCompatSeedsPerCta = 16;
constexpr int kCompatStageMax = 4096;   // windows of one sequence staged in shared memory

__device__ __forceinline__ uint32_t base_code(uint32_t ch)
{
    return ((ch >> 1) ^ (ch >> 2)) & 3u;   // A0 C1 G2 T3
}

__global__ void __launch_bounds__(256) compat_rows_kernel(const InstDev *__restrict__ inst,
                                                          const uint8_t *__restrict__ seqs, uint2 *__restrict__ planes,
                                                          uint32_t *__restrict__ compat, int *__restrict__ rowlen,
                                                          uint32_t *__restrict__ flags)
{
    __shared__ uint2 srow[kCompatStageMax];
    __shared__ uint32_t shi[(kCompatStageMax + kLMax) / 32 + 2], slo[(kCompatStageMax + kLMax) / 32 + 2];
    __shared__ int sbad;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n = inst->n, m = inst->m, l = inst->l, W = inst->W, NW = inst->NW, lim = 2 * inst->d;
    const int seeds = inst->nseed * W;
    const int i = (int)(blockIdx.x % (unsigned)n);             // the sequence of this CTA's rows
    const int jb = (int)(blockIdx.x / (unsigned)n) * kCompatSeedsPerCta;
    const uint8_t *sq = seqs + inst->seq_off;
    const uint32_t lmask = l == 32 ? ~0u : (1u << l) - 1u;
    // the verification kernel may launch now: its CTAs set up their shared
    // memory and then wait for this grid to complete (griddepcontrol.wait)
    asm volatile("griddepcontrol.launch_dependents;");
    if (threadIdx.x == 0)
        sbad = 0;
    __syncthreads();
    // sequence i as two bit-planes of m bits (32 positions per word, a ballot each)
    const int nwords = (m + 31) / 32;
    bool bad = false;
    for (int wi = warp; wi < nwords; wi += kWarps) {
        const int k = 32 * wi + lane;
        const uint32_t ch = k < m ? sq[(size_t)i * m + k] : (uint32_t)'A';
        bad |= !(ch == 'A' || ch == 'C' || ch == 'G' || ch == 'T');
        const uint32_t code = base_code(ch);
        const uint32_t hb = __ballot_sync(kFull, (code >> 1) & 1u), lb = __ballot_sync(kFull, code & 1u);
        if (lane == 0) {
            shi[wi] = hb;
            slo[wi] = lb;
        }
    }
    if (threadIdx.x < 2) {   // the word past the end, read by the last windows' funnel shifts
        shi[nwords + threadIdx.x] = 0u;
        slo[nwords + threadIdx.x] = 0u;
    }
    if (bad)
        sbad = 1;
    // this warp's seeds: windows of the seed sequences, packed from the bytes
    constexpr int kPer = kCompatSeedsPerCta / kWarps;
    uint2 xs[kPer];
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int j = jb + warp * kPer + t;
        xs[t] = make_uint2(0u, 0u);
        if (j < seeds) {   // uniform across the warp
            const int si = j / W, w = j - si * W;
            const uint32_t code = lane < l ? base_code(sq[(size_t)si * m + w + lane]) : 0u;
            xs[t] = make_uint2(__ballot_sync(kFull, (code >> 1) & 1u) & lmask, __ballot_sync(kFull, code & 1u) & lmask);
        }
    }
    __syncthreads();
    // window w: bits w .. w + l - 1 of the sequence's planes
    uint2 *pl_i = planes + inst->plane_off + (size_t)i * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const int q = w >> 5, r = w & 31;
        const uint2 e = make_uint2(__funnelshift_r(shi[q], shi[q + 1], r) & lmask,
                                   __funnelshift_r(slo[q], slo[q + 1], r) & lmask);
        srow[w] = e;
        if (jb == 0)
            pl_i[w] = e;
    }
    if (jb == 0 && threadIdx.x == 0 && sbad)
        atomicOr(&flags[0], kFlagInvalidByte);
    __syncthreads();
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
        const int j = jb + warp * kPer + t;
        const int si = j / W;   // the seed's own sequence has no row
        if (j >= seeds || si == i)
            continue;
        const int k = i < si ? i : i - 1;
        const long long local = (long long)j * (n - 1) + k;
        uint32_t *out = compat + inst->compat_off + local * NW;
        const uint2 x = xs[t];
        int total = 0;
#pragma unroll 4
        for (int w0 = 0; w0 < W; w0 += 32) {
            const int w = w0 + lane;
            bool keep = false;
            if (w < W) {
                const uint2 e = srow[w];
                keep = __popc((x.x ^ e.x) | (x.y ^ e.y)) <= lim;
            }
            const uint32_t bal = __ballot_sync(kFull, keep);
            total += __popc(bal);
            if (lane == 0)
                out[w0 >> 5] = bal;
        }
        if (lane == 0)
            rowlen[inst->rlen_off + local] = total;
    }
}

// Window planes for every (instance, sequence, window); flags bytes that are not A/C/G/T.
__global__ void pack_kernel(const InstDev *__restrict__ inst, int ninst, const long long *__restrict__ win_prefix,
                            long long total, const uint8_t *__restrict__ seqs, uint2 *__restrict__ planes,
                            uint32_t *__restrict__ flags)
{
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = ninst - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (win_prefix[mid] <= q)
                lo = mid;
            else
                hi = mid - 1;
        }
        const InstDev in = inst[lo];
        const long long local = q - win_prefix[lo];
        const int i = (int)(local / in.W), w = (int)(local % in.W);
        const uint8_t *s = seqs + in.seq_off + (size_t)i * in.m + w;
        uint32_t h = 0, lo_bits = 0;
        bool bad = false;
        for (int k = 0; k < in.l; ++k) {
            const uint32_t ch = s[k];
            bad |= !(ch == 'A' || ch == 'C' || ch == 'G' || ch == 'T');
            const uint32_t code = ((ch >> 1) ^ (ch >> 2)) & 3u;  // A0 C1 G2 T3
            h |= (code >> 1) << k;
            lo_bits |= (code & 1u) << k;
        }
        planes[in.plane_off + local] = make_uint2(h, lo_bits);
        if (bad)
            atomicOr(&flags[lo], kFlagInvalidByte);
    }
}

constexpr int kSortThreads = 1024;
constexpr uint32_t kSortSmemKeys = 8192;   // bitonic sort in shared memory up to this many codes

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *warp_tot, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t t = lane < nw ? warp_tot[lane] : 0u;
        uint32_t ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, ti, o);
            if (lane >= o)
                ti += y;
        }
        if (lane < nw)
            warp_tot[lane] = ti - t;
        if (lane == 31)
            *total = ti;
    }
    __syncthreads();
    const uint32_t r = warp_tot[warp] + incl - v;
    __syncthreads();
    return r;
}

// Stable LSD radix sort (8-bit digits) of n codes of `bits` significant bits
// by one CTA; ping-pongs between a and t and returns the buffer holding the
// sorted codes. smem: 2 x 32 x 256 counters plus 256 bin bases.
__device__ uint64_t *block_radix_sort(uint64_t *a, uint64_t *t, uint32_t n, int bits, uint32_t *smem)
{
    uint32_t *cnt = smem;                 // [32][256] per-warp digit counts of a tile
    uint32_t *off = smem + 32 * 256;      // [32][256] per-warp digit offsets of a tile
    uint32_t *bin = smem + 2 * 32 * 256;  // [256] running bin starts
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t *src = a, *dst = t;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int i = threadIdx.x; i < 2 * 32 * 256 + 256; i += blockDim.x)
            smem[i] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
            atomicAdd(&bin[(uint32_t)(src[i] >> shift) & 255u], 1u);
        __syncthreads();
        if (warp == 0) {
            uint32_t run = 0;
            for (int b0 = 0; b0 < 256; b0 += 32) {
                const uint32_t v = bin[b0 + lane];
                uint32_t incl = v;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                bin[b0 + lane] = run + incl - v;
                run += __shfl_sync(kFull, incl, 31);
            }
        }
        __syncthreads();
        for (uint32_t t0 = 0; t0 < n; t0 += blockDim.x) {
            const uint32_t i = t0 + threadIdx.x;
            const bool valid = i < n;
            const uint64_t key = valid ? src[i] : 0ull;
            const uint32_t dig = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
            const uint32_t peers = __match_any_sync(kFull, dig);
            const uint32_t rank = __popc(peers & lt);
            if (valid && rank == 0)
                cnt[warp * 256 + dig] = __popc(peers);
            __syncthreads();
            if (threadIdx.x < 256) {
                uint32_t run = bin[threadIdx.x];
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                    off[w * 256 + threadIdx.x] = run;
                    run += cnt[w * 256 + threadIdx.x];
                    cnt[w * 256 + threadIdx.x] = 0;
                }
                bin[threadIdx.x] = run;
            }
            __syncthreads();
            if (valid)
                dst[off[warp * 256 + dig] + rank] = key;
            __syncthreads();
        }
        uint64_t *x = src;
        src = dst;
        dst = x;
    }
    return src;
}

// One CTA per instance: the raw codes sorted (bitonic in shared memory when
// they fit, else radix sort through the instance's twin buffer), duplicates
// removed, unique codes appended to the dense output.
__global__ void __launch_bounds__(kSortThreads)
    sort_unique_kernel(const InstDev *__restrict__ inst, const int *__restrict__ inst_list, uint64_t *raw,
                       uint64_t *tmp, const uint32_t *__restrict__ raw_count, const uint32_t *__restrict__ flags,
                       StatusDev *__restrict__ status, uint64_t *__restrict__ dense, uint32_t dense_cap,
                       uint32_t *dense_total)
{
    extern __shared__ __align__(16) uint64_t sk[];
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t s_total, s_base, s_run;
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the producing kernel has completed
    const int I = inst_list ? inst_list[blockIdx.x] : (int)blockIdx.x;
    const InstDev in = inst[I];
    const uint32_t rc = raw_count[I];
    const uint32_t n = rc < in.raw_cap ? rc : in.raw_cap;
    uint64_t *a = raw + in.raw_off;
    uint32_t P2 = 1;
    while (P2 < n)
        P2 <<= 1;
    const uint64_t *buf;
    if (P2 <= kSortSmemKeys) {
        for (uint32_t i = threadIdx.x; i < P2; i += blockDim.x)
            sk[i] = i < n ? a[i] : ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= P2; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < P2; i += blockDim.x) {
                    const uint32_t ixj = i ^ j;
                    if (ixj > i) {
                        const uint64_t x = sk[i], y = sk[ixj];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) {
                            sk[i] = y;
                            sk[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        buf = sk;
    } else {
        buf = block_radix_sort(a, tmp + in.raw_off, n, 2 * in.l, reinterpret_cast<uint32_t *>(sk));
        __syncthreads();
    }
    uint32_t local = 0;
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
        local += (i == 0 || buf[i] != buf[i - 1]) ? 1u : 0u;
    (void)block_exclusive_scan(local, warp_tot, &s_total);
    if (threadIdx.x == 0) {
        const uint32_t base = atomicAdd(dense_total, s_total);
        s_base = base;
        s_run = 0;
        uint32_t f = flags[I];
        if (rc > in.raw_cap || base + s_total > dense_cap)
            f |= kFlagOverflow;
        status[I] = StatusDev{rc, s_total, f, base};
    }
    __syncthreads();
    for (uint32_t t0 = 0; t0 < n; t0 += blockDim.x) {
        const uint32_t i = t0 + threadIdx.x;
        const bool keep = i < n && (i == 0 || buf[i] != buf[i - 1]);
        const uint32_t ex = block_exclusive_scan(keep ? 1u : 0u, warp_tot, &s_total);
        const uint32_t pos = s_base + s_run + ex;
        if (keep && pos < dense_cap)
            dense[pos] = buf[i];
        __syncthreads();
        if (threadIdx.x == 0)
            s_run += s_total;
        __syncthreads();
    }
}

// Integer pipe probe: each thread runs 8 independent chains of one
// instruction class; thread 0 of each CTA records the SM clock cycles the
// loop took between two CTA barriers.
template <int kKind>
__global__ void __launch_bounds__(1024) probe_kernel(int iters, unsigned long long *cycles, unsigned long long *sink)
{
    uint32_t a[8];
#pragma unroll
    for (int u = 0; u < 8; ++u)
        a[u] = threadIdx.x * 2654435761u + u * 40503u + blockIdx.x;
    const uint32_t b = blockIdx.x | 0x01010101u, c2 = threadIdx.x | 0x10000001u;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (kKind == 0) {
                    a[u] = __popc(a[u]) + a[u];           // POPC + IADD chain
                } else if (kKind == 1) {
                    a[u] = (a[u] ^ b) | (a[u] & c2);      // LOP3 chain
                } else if (kKind == 2) {
                    a[u] = a[u] + b + c2;                 // IADD3 chain
                } else {
                    // one l-mer comparison as in the verification loop
                    a[u] = min(a[u], (uint32_t)__popc((b ^ a[(u + 1) & 7]) | (c2 ^ a[(u + 3) & 7])) + (uint32_t)i);
                }
            }
        }
    }
    __syncthreads();
    const long long t1 = clock64();
    uint32_t s = 0;
#pragma unroll
    for (int u = 0; u < 8; ++u)
        s ^= a[u];
    if (s == 0x12345678u)
        atomicAdd(sink, 1ull);
    if (threadIdx.x == 0)
        cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
}

}  // namespace

cudaError_t init_tables()
{
    uint32_t binom[kLMax + 1][kLMax + 1] = {};
    for (int a = 0; a <= kLMax; ++a) {
        binom[a][0] = 1;
        for (int b = 1; b <= a; ++b)
            binom[a][b] = binom[a - 1][b - 1] + (b <= a - 1 ? binom[a - 1][b] : 0u);
    }
    unsigned long long pow3[kLMax + 1];
    pow3[0] = 1;
    for (int i = 1; i <= kLMax; ++i)
        pow3[i] = pow3[i - 1] * 3ull;
    uint32_t digit[4][3][3] = {};
    for (int v = 0; v < 81; ++v) {
        int r = v;
        for (int i = 0; i < 4; ++i, r /= 3)
            digit[i][r % 3][v >> 5] |= 1u << (v & 31);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_binom, binom, sizeof(binom));
    if (e == cudaSuccess)
        e = cudaMemcpyToSymbol(c_digit, digit, sizeof(digit));
    if (e != cudaSuccess)
        return e;
    return cudaMemcpyToSymbol(c_pow3, pow3, sizeof(pow3));
}

// Resident CTAs per SM each form's registers are bounded for: with 8-warp
// CTAs 4 (the small-rows form, 64 registers) and 3 (the other, 80); with
// wider CTAs as many as keep 32 warps per SM (64 registers).
constexpr int kMinBlocksSmall = kMainWarps >= 32 ? 1 : 32 / kMainWarps;
constexpr int kMinBlocksLarge = kMainWarps == 8 ? 3 : kMinBlocksSmall;

size_t main_smem_bytes(bool small_rows)
{
    const int rows = small_rows ? kRowSmemCapSmall : kRowSmemCap;
    return kMainWarps * sizeof(WarpSmem) + rows * (sizeof(uint32_t) + sizeof(uint2)) + sizeof(CtaSmem);
}

namespace {

template <bool kCount, int kRowsCap, int kMinBlocks>
cudaError_t occupancy_of(int *blocks_per_sm, size_t smem)
{
    cudaError_t e = cudaFuncSetAttribute(main_kernel<kCount, kRowsCap, kMinBlocks>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_kernel<kCount, kRowsCap, kMinBlocks>,
                                                         kMainThreads, smem);
}

}  // namespace

cudaError_t main_occupancy(int *blocks_per_sm, bool count_mode, bool small_rows)
{
    const size_t smem = main_smem_bytes(small_rows);
    if (small_rows)
        return count_mode ? occupancy_of<true, kRowSmemCapSmall, kMinBlocksSmall>(blocks_per_sm, smem)
                          : occupancy_of<false, kRowSmemCapSmall, kMinBlocksSmall>(blocks_per_sm, smem);
    return count_mode ? occupancy_of<true, kRowSmemCap, kMinBlocksLarge>(blocks_per_sm, smem)
                      : occupancy_of<false, kRowSmemCap, kMinBlocksLarge>(blocks_per_sm, smem);
}

// Launch configuration of a programmatic dependent launch: the kernel may be
// scheduled before the previous kernel in the stream has completed, and
// waits for it with griddepcontrol.wait before touching its output. After a
// copy, a memset or an event the stream orders it as usual.
static cudaLaunchConfig_t dependent_launch(cudaLaunchAttribute *attr, int blocks, int threads, size_t smem,
                                           cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t launch_main(const MainParams &p, int blocks, bool count_mode, cudaStream_t st, bool small_rows)
{
    const size_t smem = main_smem_bytes(small_rows);
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = dependent_launch(attr, blocks, kMainThreads, smem, st);
    if (small_rows) {
        if (count_mode)
            return cudaLaunchKernelEx(&cfg, main_kernel<true, kRowSmemCapSmall, kMinBlocksSmall>, p);
        return cudaLaunchKernelEx(&cfg, main_kernel<false, kRowSmemCapSmall, kMinBlocksSmall>, p);
    }
    if (count_mode)
        return cudaLaunchKernelEx(&cfg, main_kernel<true, kRowSmemCap, kMinBlocksLarge>, p);
    return cudaLaunchKernelEx(&cfg, main_kernel<false, kRowSmemCap, kMinBlocksLarge>, p);
}

cudaError_t launch_compat(const InstDev *inst, int ninst, const long long *row_prefix, long long total_rows,
                          const uint2 *planes, uint32_t *compat, int *rowlen, int blocks, cudaStream_t st)
{
    compat_kernel<<<blocks, 256, 0, st>>>(inst, ninst, row_prefix, total_rows, planes, compat, rowlen);
    return cudaGetLastError();
}

bool compat_rows_fits(int W)
{
    return W <= kCompatStageMax;
}

cudaError_t launch_compat_rows(const InstDev *inst, int n, long long seeds, const uint8_t *seqs, uint2 *planes,
                               uint32_t *compat, int *rowlen, uint32_t *flags, cudaStream_t st)
{
    const long long blocks = (long long)n * ((seeds + kCompatSeedsPerCta - 1) / kCompatSeedsPerCta);
    compat_rows_kernel<<<(unsigned)blocks, kThreads, 0, st>>>(inst, seqs, planes, compat, rowlen, flags);
    return cudaGetLastError();
}

const void *compat_rows_kernel_fn()
{
    return reinterpret_cast<const void *>(compat_rows_kernel);
}

cudaError_t pairs_occupancy(int *blocks_per_sm, bool count_mode)
{
    const size_t smem = main_smem_bytes();
    cudaError_t e;
    if (count_mode) {
        e = cudaFuncSetAttribute(pair_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pair_kernel<true>, kThreads, smem);
    }
    e = cudaFuncSetAttribute(pair_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pair_kernel<false>, kThreads, smem);
}

cudaError_t launch_pairs(const MainParams &p, int blocks, bool count_mode, cudaStream_t st)
{
    const size_t smem = main_smem_bytes();
    if (count_mode)
        pair_kernel<true><<<blocks, kThreads, smem, st>>>(p);
    else
        pair_kernel<false><<<blocks, kThreads, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_classify(const InstDev *inst, int ninst, const long long *seed_prefix, long long total_seeds,
                            const uint2 *planes, const uint32_t *compat, uint8_t *mode, int blocks, cudaStream_t st)
{
    classify_kernel<<<blocks, 256, 0, st>>>(inst, ninst, seed_prefix, total_seeds, planes, compat, mode);
    return cudaGetLastError();
}

const void *pack_kernel_fn()
{
    return reinterpret_cast<const void *>(pack_kernel);
}

const void *sort_unique_kernel_fn()
{
    return reinterpret_cast<const void *>(sort_unique_kernel);
}

cudaError_t launch_pack(const InstDev *inst, int ninst, const long long *win_prefix, long long total_windows,
                        const uint8_t *seqs, uint2 *planes, uint32_t *flags, int blocks, cudaStream_t st)
{
    pack_kernel<<<blocks, 256, 0, st>>>(inst, ninst, win_prefix, total_windows, seqs, planes, flags);
    return cudaGetLastError();
}

cudaError_t launch_sort_unique(const InstDev *inst, const int *inst_list, int nlist, uint64_t *raw, uint64_t *tmp,
                               const uint32_t *raw_count, const uint32_t *flags, StatusDev *status,
                               uint64_t *dense, uint32_t dense_cap, uint32_t *dense_total, cudaStream_t st)
{
    const size_t smem = std::max<size_t>(kSortSmemKeys * sizeof(uint64_t), (2 * 32 * 256 + 256) * sizeof(uint32_t));
    static thread_local int attr_set_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_set_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(sort_unique_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
        attr_set_dev = dev;
    }
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = dependent_launch(attr, nlist, kSortThreads, smem, st);
    return cudaLaunchKernelEx(&cfg, sort_unique_kernel, inst, inst_list, raw, tmp, raw_count, flags, status, dense,
                              dense_cap, dense_total);
}

cudaError_t launch_probe(int kind, int iters, int blocks, unsigned long long *cycles, unsigned long long *sink,
                         cudaStream_t st)
{
    switch (kind) {
    case 0: probe_kernel<0><<<blocks, 1024, 0, st>>>(iters, cycles, sink); break;
    case 1: probe_kernel<1><<<blocks, 1024, 0, st>>>(iters, cycles, sink); break;
    case 2: probe_kernel<2><<<blocks, 1024, 0, st>>>(iters, cycles, sink); break;
    default: probe_kernel<3><<<blocks, 1024, 0, st>>>(iters, cycles, sink); break;
    }
    return cudaGetLastError();
}

}  // namespace pms
