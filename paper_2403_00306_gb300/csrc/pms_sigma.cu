// pms_sigma.cu -- exact (l,d,q)-motif search over a general alphabet (the
// qPMS-Sigma form of the paper's chapter "Our Approach": an alphabet Sigma of
// sigma letters, every l-mer compressed into ceil(log2 sigma) groups of 32-bit
// words, the distance of two compressed l-mers = popc of the OR over groups of
// the group-wise XOR; section "String Compression").
//
// What is searched (Definitions 1-5, Observation 3.1). Every motif M lies in
// B(x, d) for a window x of one of s_1..s_{n-q+1}; these windows are the seeds.
// For a seed x the candidates are the strings c with d_H(c, x) <= d, organised
// as the tree T_d(x) of qPMSPrune ("Previous Works"): a node is the set P of
// changed positions (|P| <= d), its leaves the choices of a letter other than
// x[p] at every p in P.
//
// Data per seed (one CTA). Rows: the feasible occurrences of x, i.e. the
// windows w of the other sequences with d_H(x, w) <= 2d (no candidate of B(x, d)
// can be within d of any other window), stored as D_w = mismatch mask of x and
// w plus w's bit-planes, grouped by sequence, in shared memory (global memory
// scratch when a seed has more rows than fit).
//
// Work per node P (one thread):
//  1. node bound: any candidate c of node P has d_H(c, w) >= popc(D_w ^ P)
//     (positions of D_w outside P keep x's letter and mismatch w; positions of
//     P outside D_w carry a letter other than x[p] = w[p]), so P survives only
//     if all but n - q of the other sequences hold a row with
//     popc(D_w ^ P) <= d;
//  2. letter classes: at a changed position p the letters that matter are the
//     ones the surviving rows hold there (L_p); every other letter differs
//     from all of them and from x[p], so all such letters are interchangeable
//     and one representative stands for them (expanded at output);
//  3. depth-first over the positions of P in ascending order: with the letters
//     of the first t positions fixed, a row's distance is at least the
//     mismatches outside the positions not fixed yet, and a prefix is
//     abandoned as soon as more than n - q sequences have no row within d
//     under that bound; at full depth the bound is the exact distance.
// Output keys hold ceil(log2 sigma) bits per letter index, first letter most
// significant (192 bits, three words), so ascending keys are the lexicographic
// order of the alphabet as given; the sort/unique kernel sorts,
// de-duplicates and decodes them into letters (one CTA for small outputs,
// the whole grid otherwise).
#include <cstdint>
#include <cuda_runtime.h>

#include "pms_internal.h"

namespace pms {

// 1: a node whose row lists fit takes the list form even where the pivot form
// applies (protein (9,4), n = 20, m = 600: 231 -> 121 ms with 16384-word
// lists; (11,4) 0.79 -> 0.89 ms, (9,3) unchanged)
#ifndef PMS_SIG_LISTS_BEFORE_PIVOT
#define PMS_SIG_LISTS_BEFORE_PIVOT 1
#endif
constexpr bool kSigListsBeforePivot = PMS_SIG_LISTS_BEFORE_PIVOT != 0;

__constant__ uint32_t c_sg_binom[33][33];
static uint32_t h_sg_binom[33][33];   // host copy (filled by sigma_init_tables)

__host__ __device__ inline uint32_t sg_binom(int a, int k)
{
#ifdef __CUDA_ARCH__
    return c_sg_binom[a][k];
#else
    return h_sg_binom[a][k];
#endif
}

__host__ __device__ inline int sg_popc(uint32_t v)
{
#ifdef __CUDA_ARCH__
    return __popc(v);
#else
    return __builtin_popcount(v);
#endif
}

__host__ __device__ inline int sg_popc64(unsigned long long v)
{
#ifdef __CUDA_ARCH__
    return __popcll(v);
#else
    return __builtin_popcountll(v);
#endif
}

// index of the lowest set bit (v != 0)
__host__ __device__ inline int sg_ctz(uint32_t v)
{
#ifdef __CUDA_ARCH__
    return __ffs(v) - 1;
#else
    return __builtin_ctz(v);
#endif
}

// bit j of v's set bits, counted from the lowest (j < popc(v))
__host__ __device__ inline int sg_nth_bit(uint32_t v, int j)
{
    for (; j > 0; --j)
        v &= v - 1;
    return sg_ctz(v);
}

// letter index at position p of an l-mer held as b planes (plane g at pl[g * stride])
__host__ __device__ inline int sg_letter_at(const uint32_t *pl, int stride, int b, int p)
{
    int a = 0;
    for (int g = 0; g < b; ++g)
        a |= (int)((pl[g * stride] >> p) & 1u) << g;
    return a;
}

// appends b bits to a 192-bit key (k0 most significant)
__host__ __device__ inline void sg_key_push(unsigned long long &k0, unsigned long long &k1, unsigned long long &k2,
                                            int b, int a)
{
    k0 = (k0 << b) | (k1 >> (64 - b));
    k1 = (k1 << b) | (k2 >> (64 - b));
    k2 = (k2 << b) | (unsigned long long)a;
}

// The r-th position subset in the order |P| = 0, 1, ..., d, and within a size
// colexicographically (combinatorial number system: the subset
// {c_k > ... > c_1} has rank sum_i C(c_i, i)). r < sum_{k <= d} C(l, k).
__host__ __device__ inline uint32_t sg_unrank(long long r, int l)
{
    int k = 0;
    while (r >= (long long)sg_binom(l, k)) {
        r -= sg_binom(l, k);
        ++k;
    }
    uint32_t P = 0;
    for (int i = k; i >= 1; --i) {
        int c = i - 1;
        while (c + 1 < l && (long long)sg_binom(c + 1, i) <= r)
            ++c;
        P |= 1u << c;
        r -= sg_binom(c, i);
    }
    return P;
}

// Rows hold their b planes in one 64-bit word (plane g at bits g l .. g l + l - 1)
// when that fits and saves room: 12 bytes a row instead of 4 (1 + b).
__host__ __device__ inline bool sg_packed_rows(int b, int l)
{
    return b >= 2 && b * l <= 64;
}

// One seed's rows as the node search reads them.
struct SgSeed {
    const uint32_t *D;    // row e: mismatch mask against x
    const uint32_t *Pl;   // unpacked rows: row e's plane g at Pl[g * stride + e]
    const unsigned long long *Pk;   // packed rows: row e's planes in Pk[e]
    bool packed;
    int stride;
    const int *off;       // rows of sequence i: [off[i], off[i + 1]); the seed's own sequence has none
    int n, l, d, b, miss_max, sx;
    uint32_t full;        // the sigma letter bits
    uint32_t x[kSigMaxPlanes];
};

// plane g of row e
__host__ __device__ inline uint32_t sg_plane(const SgSeed &S, int g, int e)
{
    if (S.packed)
        return (uint32_t)(S.Pk[e] >> (g * S.l)) & (S.l == 32 ? 0xFFFFFFFFu : (1u << S.l) - 1u);
    return S.Pl[g * S.stride + e];
}

// letter index of row e at position p
__host__ __device__ inline int sg_row_letter(const SgSeed &S, int e, int p)
{
    if (S.packed) {
        const unsigned long long w = S.Pk[e] >> p;
        int a = 0;
        for (int g = 0; g < S.b; ++g)
            a |= (int)((w >> (g * S.l)) & 1ull) << g;
        return a;
    }
    return sg_letter_at(S.Pl + e, S.stride, S.b, p);
}

// Work of one node by one thread (32-bit; summed over the warp into 64-bit counters after each node).
struct SgCount {
    unsigned int nodes, pruned, checks, leaves, reduce, verify;
};

// The threads that search one node together: a warp on the GPU (rows split
// over the lanes, decisions by vote), a single thread in host builds.
struct SgWarp {
    int lane;
    static constexpr int width = 32;
    __device__ bool any(bool p) const { return __any_sync(0xFFFFFFFFu, p); }
    __device__ uint32_t or_all(uint32_t v) const
    {
        for (int s = 16; s > 0; s >>= 1)
            v |= __shfl_xor_sync(0xFFFFFFFFu, v, s);
        return v;
    }
    __device__ unsigned long long bcast(unsigned long long v) const { return __shfl_sync(0xFFFFFFFFu, v, 0); }
    __device__ int from(int v, int src) const { return __shfl_sync(0xFFFFFFFFu, v, src); }
    __device__ uint32_t ballot(bool p) const { return __ballot_sync(0xFFFFFFFFu, p); }
    __device__ void sync() const { __syncwarp(); }
    __device__ void or_into(uint32_t *a, uint32_t v) const { atomicOr(a, v); }
    // lanes below this one with a vote in bal
    __device__ int rank(uint32_t bal) const { return __popc(bal & ((1u << lane) - 1u)); }
    __device__ unsigned long long or_all64(unsigned long long v) const
    {
        return ((unsigned long long)or_all((uint32_t)(v >> 32)) << 32) | or_all((uint32_t)v);
    }
    __device__ unsigned long long sum(unsigned long long v) const
    {
        for (int s = 16; s > 0; s >>= 1)
            v += __shfl_xor_sync(0xFFFFFFFFu, v, s);
        return v;
    }
};

struct SgSingle {
    int lane = 0;
    static constexpr int width = 1;
    __host__ __device__ bool any(bool p) const { return p; }
    __host__ __device__ uint32_t or_all(uint32_t v) const { return v; }
    __host__ __device__ unsigned long long bcast(unsigned long long v) const { return v; }
    __host__ __device__ int from(int v, int) const { return v; }
    __host__ __device__ uint32_t ballot(bool p) const { return p ? 1u : 0u; }
    __host__ __device__ void sync() const {}
    __host__ __device__ void or_into(uint32_t *a, uint32_t v) const { *a |= v; }
    __host__ __device__ int rank(uint32_t) const { return 0; }
    __host__ __device__ unsigned long long or_all64(unsigned long long v) const { return v; }
    __host__ __device__ unsigned long long sum(unsigned long long v) const { return v; }
};

// The first row of sequence i (in the lanes' scan order) within d of c,
// positions in U (changed positions whose letter is not fixed yet) ignored, or
// -1. Rows failing the node bound popc(D ^ P) <= d cannot be within d of any
// candidate of node P and are passed over. The lanes take every width-th row;
// the trip count and the result are uniform.
template <class G>
__host__ __device__ inline int sg_seq_find(const SgSeed &S, const G &grp, int i, uint32_t P, const uint32_t *c,
                                           uint32_t keep, SgCount &ct)
{
    for (int e0 = S.off[i]; e0 < S.off[i + 1]; e0 += G::width) {
        const int e = e0 + grp.lane;
        bool hit = false;
        if (e < S.off[i + 1]) {
            ct.reduce++;
            if (sg_popc(S.D[e] ^ P) <= S.d) {
                ct.verify++;
                uint32_t mm = 0;
                for (int g = 0; g < S.b; ++g)
                    mm |= c[g] ^ sg_plane(S, g, e);
                hit = sg_popc(mm & keep) <= S.d;
            }
        }
        const uint32_t bal = grp.ballot(hit);
        if (bal)
            return e0 + sg_ctz(bal);
    }
    return -1;
}

// Step 3's test: all but miss_max of the other sequences hold a row within d
// of c (positions in U ignored). Two orderings make it cheap without changing
// its answer: the row that held sequence i's occurrence at an earlier check
// (wit[i]) is tried before the scan -- any row of the sequence gives a valid
// lower bound -- and the sequence that failed the previous check (fail) is
// tested first, since the siblings of a rejected prefix tend to fail on it too.
// Every lane writes the same witness, so each lane reads back its own write.
template <class G>
__host__ __device__ inline bool sg_check(const SgSeed &S, const G &grp, uint32_t P, const uint32_t *c, uint32_t U,
                                         SgCount &ct, int *wit, int &fail)
{
    const uint32_t keep = ~U;
    int misses = 0;
    for (int step = -1; step < S.n; ++step) {
        const int i = step < 0 ? fail : step;
        if (i < 0 || i == S.sx || (step >= 0 && i == fail))
            continue;
        const int w = wit[i];
        bool hit = false;
        if (w >= 0) {
            ct.verify++;
            uint32_t mm = 0;
            for (int g = 0; g < S.b; ++g)
                mm |= c[g] ^ sg_plane(S, g, w);
            hit = sg_popc(mm & keep) <= S.d;
        }
        if (!hit) {
            const int e = sg_seq_find(S, grp, i, P, c, keep, ct);
            if (e >= 0) {
                hit = true;
                wit[i] = e;
            }
        }
        if (!hit && ++misses > S.miss_max) {
            fail = i;
            return false;
        }
    }
    return true;
}

// Step 1, the node bound: all but miss_max of the other sequences hold a row
// with popc(D ^ P) <= d.
template <class G>
__host__ __device__ inline bool sg_bound(const SgSeed &S, const G &grp, uint32_t P, SgCount &ct)
{
    int misses = 0;
    for (int i = 0; i < S.n; ++i) {
        if (i == S.sx)
            continue;
        bool found = false;
        for (int e0 = S.off[i]; e0 < S.off[i + 1]; e0 += G::width) {
            const int e = e0 + grp.lane;
            bool hit = false;
            if (e < S.off[i + 1]) {
                ct.reduce++;
                hit = sg_popc(S.D[e] ^ P) <= S.d;
            }
            if (grp.any(hit)) {
                found = true;
                break;
            }
        }
        if (!found && ++misses > S.miss_max)
            return false;
    }
    return true;
}

// The state of one node's search. Every value in it is the same for all the
// threads of the group, so a warp keeps one copy in shared memory: each lane
// writes the same value and a warp barrier follows every write, so no lane
// reads a value a lagging lane is about to overwrite. The letter masks L are
// built with atomic ORs between two barriers.
struct SgState {
    int pos[kSigMaxD];     // the changed positions, ascending
    int ch[kSigMaxD];      // the letter chosen at each
    int used[kSigMaxD];    // mismatches against the pivot row up to each depth
    int wl[kSigMaxD];      // the pivot row's letter where it differs from x (-1 elsewhere)
    uint32_t L[kSigMaxD];  // letters the rows passing the bound hold there
    uint32_t T[kSigMaxD];  // the choices: L and one representative of the rest
    uint32_t Wl[kSigMaxD]; // the interchangeable letters the representative stands for
    int lo[kSigMaxD];      // list form: the rows alive before depth t are list[lo[t] .. hi[t])
    int hi[kSigMaxD];
    uint32_t Tc[kSigMaxD]; // list form: the choices left for the current prefix at each depth
    uint32_t smask[kNMax]; // list form: per sequence, the letters its rows allow at the next position
};

// A group's buffer for the row lists of the list form of the depth-first
// search (null: that form is not used). An entry packs the row index (bits
// 0..20), its sequence (bits 21..26) and its distance bound (bits 27..31).
struct SgLists {
    uint32_t *buf;
    int cap;
};
constexpr int kSgListRowBits = 21;
constexpr uint32_t kSgListRowMask = (1u << kSgListRowBits) - 1u;

// Writes the motifs a full candidate stands for: at a position whose letter is
// the representative of the interchangeable letters Wl[t], every letter of
// Wl[t]. k = 0: the seed itself. One lane reserves the slots, the lanes split
// the writes.
template <class G, class Sink>
__host__ __device__ void sg_emit(const SgSeed &S, const G &grp, const int *pos, const int *ch, const uint32_t *Wl,
                                 int k, Sink &sink)
{
    unsigned long long count = 1;
    for (int t = 0; t < k; ++t)
        if (Wl[t] && ch[t] == sg_ctz(Wl[t])) {
            count *= (unsigned long long)sg_popc(Wl[t]);
            if (count > (1ull << 40))
                count = 1ull << 40;   // far beyond any capacity: reported as overflow
        }
    unsigned long long base = 0;
    if (grp.lane == 0)
        base = sink.reserve(count);
    base = grp.bcast(base);
    const unsigned long long todo = sink.room(base, count);
    for (unsigned long long e = grp.lane; e < todo; e += G::width) {
        int letter[kSigMaxD];
        unsigned long long r = e;
        for (int t = 0; t < k; ++t) {
            if (Wl[t] && ch[t] == sg_ctz(Wl[t])) {
                const unsigned long long nt = (unsigned long long)sg_popc(Wl[t]);
                letter[t] = sg_nth_bit(Wl[t], (int)(r % nt));
                r /= nt;
            } else {
                letter[t] = ch[t];
            }
        }
        unsigned long long k0 = 0, k1 = 0, k2 = 0;
        int t = 0;
        for (int p = 0; p < S.l; ++p) {
            int a;
            if (t < k && pos[t] == p)
                a = letter[t++];
            else
                a = sg_letter_at(S.x, 1, S.b, p);
            sg_key_push(k0, k1, k2, S.b, a);
        }
        sink.put(base + e, k0, k1, k2);
    }
}

// Step 3: depth-first over the letter choices T[t] of the changed positions
// pos[0..k-1]. With a pivot row (pivot: its letters in wl) a choice is taken
// only while at most `slack` of the changed positions where the row differs
// from x carry a letter other than the row's, which keeps the row within d of
// the candidate.
template <class G, class Sink>
__host__ __device__ void sg_dfs(const SgSeed &S, const G &grp, uint32_t P, int k, SgState &st, bool pivot, int slack,
                                SgCount &ct, Sink &sink, int *wit, int &fail)
{
    const bool lead = grp.lane == 0;
    uint32_t c[kSigMaxPlanes];
    for (int g = 0; g < kSigMaxPlanes; ++g)
        c[g] = S.x[g];
    int t = 0;
    st.ch[0] = sg_ctz(st.T[0]);
    grp.sync();
    for (;;) {
        bool ok = false;
        const int ct_t = st.ch[t];
        const int u = (t > 0 ? st.used[t - 1] : 0) + ((pivot && st.wl[t] >= 0 && ct_t != st.wl[t]) ? 1 : 0);
        if (!pivot || u <= slack) {
            st.used[t] = u;
            grp.sync();
            const uint32_t bit = 1u << st.pos[t];
            for (int g = 0; g < S.b; ++g)
                c[g] = ((ct_t >> g) & 1) ? (c[g] | bit) : (c[g] & ~bit);
            const uint32_t U = P & ~(uint32_t)((2ull << st.pos[t]) - 1ull);   // changed positions above pos[t]
            if (lead) {
                ct.checks++;
                if (t == k - 1)
                    ct.leaves++;
            }
            ok = sg_check(S, grp, P, c, U, ct, wit, fail);
        }
        if (ok) {
            if (t == k - 1) {
                sg_emit(S, grp, st.pos, st.ch, st.Wl, k, sink);
            } else {
                ++t;
                st.ch[t] = sg_ctz(st.T[t]);
                grp.sync();
                continue;
            }
        }
        // the next choice at this depth, else back up
        for (;;) {
            const uint32_t rest = st.T[t] & ~(uint32_t)((2ull << st.ch[t]) - 1ull);
            if (rest) {
                const int nx = sg_ctz(rest);
                grp.sync();
                st.ch[t] = nx;
                grp.sync();
                break;
            }
            if (--t < 0)
                return;
        }
    }
}

// Step 3 with the row set shrunk depth by depth (the row filtering of the
// paper's depth-first search, TraverStringRef_Tree / qPMSPrune): the rows that
// pass the node bound are listed once with their bound popc(D ^ P), the
// mismatches no letter choice can avoid. Fixing letter a at the next changed
// position p raises the bound of a row by one exactly when the row differs
// from x at p (bit p of D) and holds a letter other than a there (where it
// agrees with x, a != x[p] already counts); a row whose bound exceeds d is
// within d of no string below the prefix and leaves the list. The prefix is
// abandoned when more than miss_max sequences have no row left. So each depth
// tests only the rows the previous depth kept, each with one letter
// comparison, instead of looking for an occurrence in every sequence again.
// For q = n the kept rows also say which letters can come next: at the next
// changed position a sequence allows every letter if one of its rows has
// slack there (a bound below d, or agreement with x at that position), else
// only the letters its rows hold there; a letter that some sequence does not
// allow would leave it without a row, so only letters every sequence allows
// are tried (the same prefixes fail, without a scan of the list).
// The lists of the depths on the current path are kept one after another in
// the group's buffer (the caller checks they fit: at most n0 (k + 1)).

// Adds the letters `allow` of a kept entry to the mask of its sequence
// (st.smask, atomic ORs; sg_allowed synchronises the group before reading).
template <class G>
__host__ __device__ inline void sg_allow_into(SgState &st, const G &grp, bool keep, int seq, uint32_t allow)
{
    if (keep)
        grp.or_into(&st.smask[seq], allow);
}

// The letters every sequence (but the seed's own) allows: the AND of st.smask.
template <class G>
__host__ __device__ inline uint32_t sg_allowed(const SgSeed &S, SgState &st, const G &grp)
{
    grp.sync();
    uint32_t miss = 0;
    for (int i = grp.lane; i < S.n; i += G::width)
        if (i != S.sx)
            miss |= ~st.smask[i];
    return ~grp.or_all(miss);
}

template <class G>
__host__ __device__ inline void sg_allow_clear(const SgSeed &S, SgState &st, const G &grp)
{
    grp.sync();
    for (int i = grp.lane; i < S.n; i += G::width)
        st.smask[i] = 0u;
    grp.sync();
}

template <class G, class Sink>
__host__ __device__ void sg_dfs_rows(const SgSeed &S, const G &grp, int k, SgState &st, SgCount &ct, Sink &sink,
                                     uint32_t *buf, int n0)
{
    const bool lead = grp.lane == 0;
    const bool narrow = S.miss_max == 0;   // q = n: choices narrowed by the rows' letters
    uint32_t tc0 = st.T[0];
    if (narrow) {   // the letters the node's rows allow at the first position
        sg_allow_clear(S, st, grp);
        const int p0 = st.pos[0];
        for (int j0 = 0; j0 < n0; j0 += G::width) {
            const int j = j0 + grp.lane;
            uint32_t allow = 0;
            int seq = 0;
            if (j < n0) {
                const uint32_t v = buf[j];
                const int e = (int)(v & kSgListRowMask);
                seq = (int)((v >> kSgListRowBits) & 63u);
                allow = ((int)(v >> 27) < S.d || !((S.D[e] >> p0) & 1u))
                            ? ~0u
                            : 1u << sg_row_letter(S, e, p0);
            }
            sg_allow_into(st, grp, j < n0, seq, allow);
        }
        tc0 &= sg_allowed(S, st, grp);
    }
    if (!tc0)
        return;
    int t = 0;
    if (lead) {
        st.lo[0] = 0;
        st.hi[0] = n0;
    }
    grp.sync();
    st.Tc[0] = tc0;
    st.ch[0] = sg_ctz(tc0);
    grp.sync();
    for (;;) {
        const int plo = st.lo[t], phi = st.hi[t];
        const int p = st.pos[t], a = st.ch[t];
        const bool track = narrow && t + 1 < k;   // the next position's letters
        const int pn = track ? st.pos[t + 1] : 0;
        if (track)
            sg_allow_clear(S, st, grp);
        int w = phi;
        unsigned long long present = 0;
        for (int j0 = plo; j0 < phi; j0 += G::width) {
            const int j = j0 + grp.lane;
            bool keep = false;
            uint32_t v = 0, allow = 0;
            if (j < phi) {
                v = buf[j];
                const int e = (int)(v & kSgListRowMask);
                int dist = (int)(v >> 27);
                if ((S.D[e] >> p) & 1u) {
                    ct.verify++;
                    dist += sg_row_letter(S, e, p) != a ? 1 : 0;
                }
                keep = dist <= S.d;
                v = (v & ((1u << 27) - 1u)) | ((uint32_t)dist << 27);
                if (keep) {
                    present |= 1ull << ((v >> kSgListRowBits) & 63u);
                    if (track)
                        allow = (dist < S.d || !((S.D[e] >> pn) & 1u))
                                    ? ~0u
                                    : 1u << sg_row_letter(S, e, pn);
                }
            }
            const uint32_t bal = grp.ballot(keep);
            if (keep)
                buf[w + grp.rank(bal)] = v;
            w += sg_popc(bal);
            if (track)
                sg_allow_into(st, grp, keep, (int)((v >> kSgListRowBits) & 63u), allow);
        }
        present = grp.or_all64(present);
        if (lead) {
            ct.checks++;
            if (t == k - 1)
                ct.leaves++;
        }
        bool ok = (S.n - 1) - sg_popc64(present) <= S.miss_max;   // the seed's own sequence has no rows
        uint32_t tcn = 0;
        if (ok && t + 1 < k) {
            tcn = st.T[t + 1];
            if (track)
                tcn &= sg_allowed(S, st, grp);
            ok = tcn != 0;
        }
        if (ok) {
            if (t == k - 1) {
                sg_emit(S, grp, st.pos, st.ch, st.Wl, k, sink);
            } else {
                grp.sync();
                if (lead) {
                    st.lo[t + 1] = phi;
                    st.hi[t + 1] = w;
                }
                ++t;
                grp.sync();
                st.Tc[t] = tcn;
                st.ch[t] = sg_ctz(tcn);
                grp.sync();
                continue;
            }
        }
        // the next choice at this depth, else back up
        for (;;) {
            const uint32_t rest = st.Tc[t] & ~(uint32_t)((2ull << st.ch[t]) - 1ull);
            if (rest) {
                const int nx = sg_ctz(rest);
                grp.sync();
                st.ch[t] = nx;
                grp.sync();
                break;
            }
            if (--t < 0)
                return;
        }
    }
}

// The search below one tree node P (steps 1-3 of the file comment), by one
// group of threads in lockstep: every branch below depends only on values the
// whole group shares.
template <class G, class Sink>
__host__ __device__ void sg_node(const SgSeed &S, const G &grp, uint32_t P, SgCount &ct, Sink &sink, int *wit,
                                 SgState &st, SgLists lists)
{
    const bool lead = grp.lane == 0;
    if (lead)
        ct.nodes++;
    if (!sg_bound(S, grp, P, ct)) {
        if (lead)
            ct.pruned++;
        return;
    }
    const int k = sg_popc(P);
    if (k == 0) {   // the seed itself; the bound was its exact distance to every row
        if (lead) {
            ct.checks++;
            ct.leaves++;
        }
        sg_emit(S, grp, nullptr, nullptr, nullptr, 0, sink);
        return;
    }
    {
        uint32_t M = P;
        for (int t = 0; t < k; ++t) {
            st.pos[t] = sg_ctz(M);
            M &= M - 1;
            st.L[t] = 0;
        }
    }
    grp.sync();
    // step 2: the letters the rows passing the bound hold at the changed
    // positions, and the sequence with the fewest such rows (the pivot); the
    // passing rows are also listed for the list form of step 3 while the list
    // fits the group's buffer
    int piv = -1, piv_rows = 0;
    const bool listing = lists.buf != nullptr && S.off[S.n] <= (int)kSgListRowMask + 1;
    int n0 = 0;
    for (int i = 0; i < S.n; ++i) {
        if (i == S.sx)
            continue;
        int cnt = 0;
        for (int e0 = S.off[i]; e0 < S.off[i + 1]; e0 += G::width) {
            const int e = e0 + grp.lane;
            bool pass = false;
            int bound = 0;
            if (e < S.off[i + 1]) {
                ct.reduce++;
                const uint32_t De = S.D[e];
                bound = sg_popc(De ^ P);
                pass = bound <= S.d;
                if (pass) {
                    uint32_t M = De & P;
                    while (M) {
                        const int p = sg_ctz(M);
                        M &= M - 1;
                        grp.or_into(&st.L[sg_popc(P & ((1u << p) - 1u))],
                                    1u << sg_row_letter(S, e, p));
                    }
                }
            }
            const uint32_t bal = grp.ballot(pass);
            if (listing && pass && n0 + grp.rank(bal) < lists.cap)
                lists.buf[n0 + grp.rank(bal)] = (uint32_t)e | ((uint32_t)i << kSgListRowBits) | ((uint32_t)bound << 27);
            cnt += sg_popc(bal);
            n0 += sg_popc(bal);
        }
        if (piv < 0 || cnt < piv_rows) {
            piv = i;
            piv_rows = cnt;
        }
    }
    grp.sync();
    for (int t = 0; t < k; ++t) {
        const uint32_t Lt = st.L[t];
        const uint32_t Wt = S.full & ~Lt & ~(1u << sg_letter_at(S.x, 1, S.b, st.pos[t]));
        st.Wl[t] = Wt;
        st.T[t] = Lt | (Wt & (0u - Wt));   // the rows' letters and one representative of the rest
    }
    for (int j = grp.lane; j < S.n; j += G::width)
        wit[j] = -1;
    grp.sync();
    int fail = -1;
    // Pivot form (q = n; Observation 3.3 applied to the node): every motif of
    // node P lies within d of one of the pivot's rows that pass the bound, so
    // walking, row by row, only the letters that keep that row within d covers
    // them all (a motif near several such rows is found once per row; the
    // sort/unique step removes the copies). Chosen when the pivot has few rows
    // against large choice sets.
    const int est_plain = sg_popc(st.T[0]) * (k >= 2 ? sg_popc(st.T[1]) : 1);
    const bool lists_fit = listing && (long long)n0 * (k + 1) <= (long long)lists.cap;
    if (S.miss_max == 0 && piv >= 0 && piv_rows * k < est_plain && !(kSigListsBeforePivot && lists_fit)) {
        for (int e = S.off[piv]; e < S.off[piv + 1]; ++e) {
            const uint32_t De = S.D[e];
            if (lead)
                ct.reduce++;
            const int slack = S.d - sg_popc(De ^ P);
            if (slack < 0)
                continue;
            grp.sync();
            for (int t = 0; t < k; ++t)
                st.wl[t] = ((De >> st.pos[t]) & 1u) ? sg_row_letter(S, e, st.pos[t]) : -1;
            wit[piv] = e;
            grp.sync();
            sg_dfs(S, grp, P, k, st, true, slack, ct, sink, wit, fail);
        }
    } else if (lists_fit) {
        sg_dfs_rows(S, grp, k, st, ct, sink, lists.buf, n0);
    } else {
        sg_dfs(S, grp, P, k, st, false, 0, ct, sink, wit, fail);
    }
}

// --------------------------------------------------------------------- kernels

// Output of the search kernel: room for raw_cap keys, the count may run past it.
struct SgDeviceSink {
    unsigned long long *raw;
    unsigned long long *count;
    unsigned long long cap;
    __host__ __device__ unsigned long long reserve(unsigned long long c)
    {
#ifdef __CUDA_ARCH__
        return atomicAdd(count, c);
#else
        const unsigned long long b = *count;
        *count += c;
        return b;
#endif
    }
    __host__ __device__ unsigned long long room(unsigned long long base, unsigned long long c) const
    {
        return base >= cap ? 0ull : (c < cap - base ? c : cap - base);
    }
    __host__ __device__ void put(unsigned long long slot, unsigned long long k0, unsigned long long k1,
                                 unsigned long long k2)
    {
        raw[3 * slot] = k0;
        raw[3 * slot + 1] = k1;
        raw[3 * slot + 2] = k2;
    }
};

// One thread per window: letter indices into b bit-planes; a byte outside the
// alphabet sets flags[0] bit 0.
__global__ void sigma_pack_kernel(const uint8_t *__restrict__ seqs, int n, int m, int l, int b, SigmaMap map,
                                  uint32_t *__restrict__ planes, uint32_t *__restrict__ flags)
{
    const int W = m - l + 1;
    const long long NW = (long long)n * W;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < NW;
         w += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(w / W);
        const int j = (int)(w - (long long)i * W);
        const uint8_t *s = seqs + (size_t)i * m + j;
        uint32_t pl[kSigMaxPlanes] = {0u, 0u, 0u, 0u, 0u};
        bool bad = false;
        for (int k = 0; k < l; ++k) {
            const unsigned a = map.v[s[k]];
            if (a == 0xFFu) {
                bad = true;
                continue;
            }
            for (int g = 0; g < kSigMaxPlanes; ++g)
                pl[g] |= ((a >> g) & 1u) << k;
        }
        if (bad)
            atomicOr(flags, 1u);
        for (int g = 0; g < b; ++g)
            planes[(size_t)g * NW + w] = pl[g];
    }
}

// Persistent CTAs take one seed at a time from the queue: rows of the seed
// (two passes over every window: count per sequence, then place), then the
// tree nodes of the seed, claimed one at a time by the CTA's warps.
__global__ void __launch_bounds__(kSigThreads, 3) sigma_main_kernel(SigmaParams p)
{
    extern __shared__ __align__(16) uint32_t sg_rows_smem[];
    __shared__ int s_cnt[kNMax], s_cur[kNMax], s_off[kNMax + 1];
    __shared__ int s_seed, s_skip;
    __shared__ unsigned long long s_next;
    __shared__ int s_wit[kSigThreads / 32][kNMax];   // per warp: witness row of each sequence
    __shared__ SgState s_state[kSigThreads / 32];     // per warp: the node search's state
    __shared__ unsigned long long s_ct[kSgCntNum];
    const int tid = threadIdx.x;
    for (int c = tid; c < kSgCntNum; c += blockDim.x)
        s_ct[c] = 0;
    unsigned long long cmp_rows = 0, seeds = 0, infeasible = 0;
    SgDeviceSink sink{p.raw, p.raw_count, p.raw_cap};
    const int NW = p.n * p.W;
    for (;;) {
        if (tid == 0)
            s_seed = (int)atomicAdd(p.head, 1u);
        if (tid < p.n)
            s_cnt[tid] = 0;
        __syncthreads();
        const int seed = s_seed;
        if (seed >= p.nseeds)
            break;
        const int sx = seed / p.W;
        const int xw = sx * p.W + (seed - sx * p.W);
        SgSeed S;
        for (int g = 0; g < kSigMaxPlanes; ++g)
            S.x[g] = g < p.b ? p.planes[(size_t)g * NW + xw] : 0u;
        for (int w = tid; w < NW; w += blockDim.x) {
            const int i = w / p.W;
            if (i == sx)
                continue;
            uint32_t mm = 0;
            for (int g = 0; g < p.b; ++g)
                mm |= S.x[g] ^ p.planes[(size_t)g * NW + w];
            cmp_rows++;
            if (__popc(mm) <= 2 * p.d)
                atomicAdd(&s_cnt[i], 1);
        }
        __syncthreads();
        if (tid == 0) {
            int o = 0, misses = 0;
            for (int i = 0; i < p.n; ++i) {
                s_off[i] = o;
                s_cur[i] = o;
                o += s_cnt[i];
                if (i != sx && s_cnt[i] == 0)
                    ++misses;
            }
            s_off[p.n] = o;
            s_skip = misses > p.miss_max;
            s_next = 0;
            seeds++;
            if (s_skip)
                infeasible++;
        }
        __syncthreads();
        if (!s_skip) {
            const int total = s_off[p.n];
            const bool packed = sg_packed_rows(p.b, p.l);
            uint32_t *rows;
            int stride;
            if (total <= p.smem_rows) {
                rows = sg_rows_smem;
                stride = p.smem_rows;
            } else {
                rows = p.scratch + (size_t)blockIdx.x * (1 + p.b) * p.scratch_rows;
                stride = p.scratch_rows;
            }
            for (int w = tid; w < NW; w += blockDim.x) {
                const int i = w / p.W;
                if (i == sx)
                    continue;
                uint32_t pl[kSigMaxPlanes];
                uint32_t mm = 0;
                for (int g = 0; g < p.b; ++g) {
                    pl[g] = p.planes[(size_t)g * NW + w];
                    mm |= S.x[g] ^ pl[g];
                }
                if (__popc(mm) <= 2 * p.d) {
                    const int e = atomicAdd(&s_cur[i], 1);
                    rows[e] = mm;
                    if (packed) {
                        unsigned long long pk = 0;
                        for (int g = 0; g < p.b; ++g)
                            pk |= (unsigned long long)pl[g] << (g * p.l);
                        reinterpret_cast<unsigned long long *>(rows + stride)[e] = pk;
                    } else {
                        for (int g = 0; g < p.b; ++g)
                            rows[(size_t)(1 + g) * stride + e] = pl[g];
                    }
                }
            }
            __syncthreads();
            S.D = rows;
            S.Pl = rows + stride;
            S.Pk = reinterpret_cast<const unsigned long long *>(rows + stride);   // stride is even
            S.packed = packed;
            S.stride = stride;
            S.off = s_off;
            S.n = p.n;
            S.l = p.l;
            S.d = p.d;
            S.b = p.b;
            S.miss_max = p.miss_max;
            S.sx = sx;
            S.full = p.sigma == 32 ? 0xFFFFFFFFu : (1u << p.sigma) - 1u;
            // each warp claims the seed's nodes one at a time
            const SgWarp grp{tid & 31};
            for (;;) {
                unsigned long long r = 0;
                if (grp.lane == 0)
                    r = atomicAdd(&s_next, 1ull);
                r = grp.bcast(r);
                if (r >= (unsigned long long)p.nodes)
                    break;
                SgCount ct{};
                const SgLists lists{p.lists ? p.lists + ((size_t)blockIdx.x * (kSigThreads / 32) + (tid >> 5)) *
                                                              (size_t)p.list_cap
                                            : nullptr,
                                    p.list_cap};
                sg_node(S, grp, sg_unrank((long long)r, p.l), ct, sink, s_wit[tid >> 5], s_state[tid >> 5], lists);
                const unsigned long long red = grp.sum(ct.reduce), ver = grp.sum(ct.verify);
                if (grp.lane == 0) {   // node, check and leaf counts are the lead lane's
                    atomicAdd(&s_ct[kSgNodes], (unsigned long long)ct.nodes);
                    atomicAdd(&s_ct[kSgNodesPruned], (unsigned long long)ct.pruned);
                    atomicAdd(&s_ct[kSgChecks], (unsigned long long)ct.checks);
                    atomicAdd(&s_ct[kSgLeaves], (unsigned long long)ct.leaves);
                    atomicAdd(&s_ct[kSgCmpReduce], red);
                    atomicAdd(&s_ct[kSgCmpVerify], ver);
                }
            }
        }
        __syncthreads();   // rows, offsets and s_seed are rewritten for the next seed
    }
    atomicAdd(&s_ct[kSgCmpRows], cmp_rows);
    if (tid == 0) {
        s_ct[kSgSeeds] += seeds;
        s_ct[kSgSeedsInfeasible] += infeasible;
    }
    __syncthreads();
    if (tid < kSgCntNum)
        atomicAdd(&p.counters[tid], s_ct[tid]);
}

__host__ __device__ inline bool sg_less(const unsigned long long *a, const unsigned long long *b)
{
    if (a[0] != b[0])
        return a[0] < b[0];
    if (a[1] != b[1])
        return a[1] < b[1];
    return a[2] < b[2];
}

// Largest output sorted by the bitonic network of one CTA; more keys take the
// radix sort of the whole grid.
constexpr unsigned long long kSigBitonicMax = 4096;
// Shared memory of the sort: per-warp digit counts and offsets of a tile, and the 256 bin starts.
constexpr size_t kSigSortSmem = (2 * (kSigSortThreads / 32) * 256 + 256) * sizeof(unsigned int);
// Polls of a grid barrier (about a tenth of a microsecond apart) before a CTA gives up.
constexpr unsigned int kSigBarrierPolls = 1u << 23;

__device__ __forceinline__ unsigned int sg_ld_acquire(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier of all CTAs of the sort (they are all resident: cooperative
// launch). bar[0] counts arrivals and is never reset within a launch, so the
// k-th barrier is passed once it reaches k * gridDim.x. A CTA that polls
// kSigBarrierPolls times in vain, or finds bar[1] set, sets bar[1] and gets
// false; so does every CTA after it.
__device__ bool sg_grid_barrier(unsigned int *bar, unsigned int &k, int *s_ok)
{
    __syncthreads();
    ++k;
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned int target = k * gridDim.x;
        for (unsigned int poll = 0; sg_ld_acquire(bar) < target; ++poll) {
            if (poll >= kSigBarrierPolls || sg_ld_acquire(bar + 1) != 0u) {
                atomicOr(bar + 1, 1u);
                ok = 0;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Exclusive prefix sum of v over the CTA's threads in thread order; *total
// gets the sum. Every thread calls it. scratch: 33 words of shared memory.
__device__ unsigned int sg_block_scan(unsigned int v, unsigned int *scratch, unsigned int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        scratch[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned int s = lane < nw ? scratch[lane] : 0u;
        unsigned int si = s;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned int y = __shfl_up_sync(0xFFFFFFFFu, si, o);
            if (lane >= o)
                si += y;
        }
        if (lane < nw)
            scratch[lane] = si - s;
        if (lane == 31)
            scratch[32] = si;
    }
    __syncthreads();
    const unsigned int r = scratch[warp] + incl - v;
    *total = scratch[32];
    __syncthreads();   // scratch is free for the next call
    return r;
}

// Key i of the sorted keys is the first of its value: i == 0 or key i - 1 differs.
__device__ __forceinline__ bool sg_first_of_value(const unsigned long long *key, unsigned long long i)
{
    return i == 0 || __ldcg(key + 3 * i) != __ldcg(key + 3 * i - 3) ||
           __ldcg(key + 3 * i + 1) != __ldcg(key + 3 * i - 2) || __ldcg(key + 3 * i + 2) != __ldcg(key + 3 * i - 1);
}

// First occurrences among the sorted keys lo..hi-1.
__device__ unsigned long long sg_count_unique(const unsigned long long *key, unsigned long long lo,
                                              unsigned long long hi, unsigned int *scratch)
{
    unsigned int c = 0;
    for (unsigned long long i = lo + threadIdx.x; i < hi; i += blockDim.x)
        c += sg_first_of_value(key, i) ? 1u : 0u;
    unsigned int total;
    sg_block_scan(c, scratch, &total);
    return total;
}

// Decodes the first occurrences among the sorted keys lo..hi-1 into l letters
// each, in key order, as motifs base, base + 1, ... of out. Returns how many.
__device__ unsigned long long sg_unique_decode(const unsigned long long *key, unsigned long long lo,
                                               unsigned long long hi, unsigned long long base, int l, int b,
                                               const SigmaMap &letters, uint8_t *out, unsigned int *scratch)
{
    const unsigned long long base0 = base;
    for (unsigned long long start = lo; start < hi; start += blockDim.x) {
        const unsigned long long i = start + threadIdx.x;
        const bool f = i < hi && sg_first_of_value(key, i);
        unsigned int total;
        const unsigned int at = sg_block_scan(f ? 1u : 0u, scratch, &total);
        if (f) {
            const unsigned long long k3[3] = {__ldcg(key + 3 * i), __ldcg(key + 3 * i + 1), __ldcg(key + 3 * i + 2)};
            const unsigned long long idx = base + at;
            for (int p = 0; p < l; ++p) {
                const int s = b * (l - 1 - p);
                int a = 0;
                for (int j = 0; j < b; ++j) {
                    const int bit = s + j;
                    a |= (int)((k3[2 - (bit >> 6)] >> (bit & 63)) & 1ull) << j;
                }
                out[idx * l + p] = letters.v[a];
            }
        }
        base += total;
    }
    return base - base0;
}

// Sorts, de-duplicates and decodes the raw keys. Up to kSigBitonicMax keys:
// CTA 0 alone, by a bitonic network padded with all-ones keys to a power of
// two (within the buffer's power-of-two capacity). More: every CTA, by a
// stable LSD radix sort with 8-bit digits over the key's low l * b bits (bit
// i in word 2 - i / 64; a digit never straddles two words), ping-ponging
// between raw and tmp. Each CTA owns a contiguous tile of the keys; a pass
// counts its tile's digits, turns the counts into exclusive offsets (digit
// major, CTA minor: the digits are shared out over the CTAs), and scatters
// the tile blockDim keys at a time (ranks within a warp by __match_any_sync,
// warps in order), so equal digits keep their order. Grid barriers separate
// the phases; keys and counts written by other CTAs are read through L2.
__global__ void __launch_bounds__(kSigSortThreads) sigma_sort_unique_kernel(
    unsigned long long *raw, unsigned long long *tmp, const unsigned long long *__restrict__ raw_count,
    unsigned long long cap, int l, int b, SigmaMap letters, uint8_t *__restrict__ out,
    unsigned long long *__restrict__ unique_count, SigSortGrid grid)
{
    extern __shared__ unsigned int sg_sort_smem[];
    __shared__ unsigned int s_scan[33];
    __shared__ int s_ok;
    const int tid = threadIdx.x, nt = blockDim.x;
    const unsigned long long N = *raw_count < cap ? *raw_count : cap;
    if (N <= kSigBitonicMax) {
        if (blockIdx.x != 0)
            return;
        unsigned long long P2 = 1;
        while (P2 < N)
            P2 <<= 1;
        for (unsigned long long i = tid; i < P2; i += nt)
            if (i >= N)
                raw[3 * i] = raw[3 * i + 1] = raw[3 * i + 2] = ~0ull;
        __syncthreads();
        for (unsigned long long k = 2; k <= P2; k <<= 1) {
            for (unsigned long long j = k >> 1; j > 0; j >>= 1) {
                for (unsigned long long i = tid; i < P2; i += nt) {
                    const unsigned long long ixj = i ^ j;
                    if (ixj > i) {
                        unsigned long long *a = raw + 3 * i, *c = raw + 3 * ixj;
                        const bool up = (i & k) == 0;
                        if (up ? sg_less(c, a) : sg_less(a, c)) {
                            for (int w = 0; w < 3; ++w) {
                                const unsigned long long v = a[w];
                                a[w] = c[w];
                                c[w] = v;
                            }
                        }
                    }
                }
                __syncthreads();
            }
        }
        const unsigned long long u = sg_unique_decode(raw, 0, N, 0, l, b, letters, out, s_scan);
        if (tid == 0)
            *unique_count = u;
        return;
    }

    const unsigned int G = gridDim.x, cta = blockIdx.x;
    unsigned int *hist = grid.hist;        // [256][G]: digit counts, then their exclusive offsets
    unsigned int *tot = hist + 256 * G;    // [256]: keys per digit
    unsigned int *ucount = tot + 256;      // [G]: first occurrences per tile
    const int nw = nt >> 5, lane = tid & 31, warp = tid >> 5;
    const unsigned int lt = (1u << lane) - 1u;
    unsigned int *cnt = sg_sort_smem;              // [nw][256] per-warp digit counts of a group of keys
    unsigned int *off = sg_sort_smem + nw * 256;   // [nw][256] per-warp digit offsets of a group
    unsigned int *bin = sg_sort_smem + 2 * nw * 256;
    const unsigned long long tile = (N + G - 1) / G;
    const unsigned long long lo = min(N, (unsigned long long)cta * tile), hi = min(N, lo + tile);
    unsigned int k = 0;   // grid barriers passed
    unsigned long long *src = raw, *dst = tmp;
    const int bits = l * b;
    for (int shift = 0; shift < bits; shift += 8) {
        const int word = 2 - (shift >> 6), sh = shift & 63;
        for (int i = tid; i < 2 * nw * 256 + 256; i += nt)
            sg_sort_smem[i] = 0u;
        __syncthreads();
        for (unsigned long long i = lo + tid; i < hi; i += nt)
            atomicAdd(&bin[(unsigned int)(__ldcg(src + 3 * i + word) >> sh) & 255u], 1u);
        __syncthreads();
        if (tid < 256)
            hist[tid * G + cta] = bin[tid];
        if (!sg_grid_barrier(grid.bar, k, &s_ok))
            return;
        for (unsigned int t = cta; t < 256u; t += G) {
            unsigned int run = 0;
            for (unsigned int c0 = 0; c0 < G; c0 += nt) {
                const unsigned int c = c0 + tid;
                const unsigned int v = c < G ? __ldcg(hist + t * G + c) : 0u;
                unsigned int sum;
                const unsigned int ex = sg_block_scan(v, s_scan, &sum);
                if (c < G)
                    hist[t * G + c] = run + ex;
                run += sum;
            }
            if (tid == 0)
                tot[t] = run;
        }
        if (!sg_grid_barrier(grid.bar, k, &s_ok))
            return;
        {
            // this tile's first slot of digit t: the keys of smaller digits,
            // then the keys of digit t in earlier tiles
            const unsigned int v = tid < 256 ? __ldcg(tot + tid) : 0u;
            unsigned int sum;
            const unsigned int ex = sg_block_scan(v, s_scan, &sum);
            if (tid < 256)
                bin[tid] = ex + __ldcg(hist + tid * G + cta);
        }
        __syncthreads();
        for (unsigned long long t0 = lo; t0 < hi; t0 += nt) {
            const unsigned long long i = t0 + tid;
            const bool valid = i < hi;
            unsigned long long k0 = 0, k1 = 0, k2 = 0;
            unsigned int dig = 256u;
            if (valid) {
                k0 = __ldcg(src + 3 * i);
                k1 = __ldcg(src + 3 * i + 1);
                k2 = __ldcg(src + 3 * i + 2);
                const unsigned long long w = word == 0 ? k0 : (word == 1 ? k1 : k2);
                dig = (unsigned int)(w >> sh) & 255u;
            }
            const unsigned int peers = __match_any_sync(0xFFFFFFFFu, dig);
            const unsigned int rank = __popc(peers & lt);
            if (valid && rank == 0)
                cnt[warp * 256 + dig] = __popc(peers);
            __syncthreads();
            if (tid < 256) {
                unsigned int run = bin[tid];
                for (int w = 0; w < nw; ++w) {
                    off[w * 256 + tid] = run;
                    run += cnt[w * 256 + tid];
                    cnt[w * 256 + tid] = 0u;
                }
                bin[tid] = run;
            }
            __syncthreads();
            if (valid) {
                const unsigned int at = off[warp * 256 + dig] + rank;
                dst[3 * (unsigned long long)at] = k0;
                dst[3 * (unsigned long long)at + 1] = k1;
                dst[3 * (unsigned long long)at + 2] = k2;
            }
            __syncthreads();
        }
        if (!sg_grid_barrier(grid.bar, k, &s_ok))
            return;
        unsigned long long *x = src;
        src = dst;
        dst = x;
    }
    // unique + decode: each tile's first occurrences, placed after those of the earlier tiles
    const unsigned long long mine = sg_count_unique(src, lo, hi, s_scan);
    if (tid == 0)
        ucount[cta] = (unsigned int)mine;
    if (!sg_grid_barrier(grid.bar, k, &s_ok))
        return;
    unsigned long long base = 0;
    for (unsigned int c0 = 0; c0 < cta; c0 += nt) {
        const unsigned int c = c0 + tid;
        unsigned int sum;
        sg_block_scan(c < cta ? __ldcg(ucount + c) : 0u, s_scan, &sum);
        base += sum;
    }
    sg_unique_decode(src, lo, hi, base, l, b, letters, out, s_scan);
    if (cta == G - 1 && tid == 0)
        *unique_count = base + mine;
}

// --------------------------------------------------------------------- host side

int sigma_planes(int sigma)
{
    int g = 0;
    while ((1 << g) < sigma)
        ++g;
    return g;
}

size_t sigma_row_bytes(int b, int l)
{
    return sg_packed_rows(b, l) ? 12 : (size_t)4 * (1 + b);
}

int sigma_smem_rows(int b, int l, bool large)
{
    return (int)((large ? kSigSmemLarge : kSigSmemSmall) / sigma_row_bytes(b, l)) & ~1;   // even: 8-byte packed words
}

cudaError_t sigma_init_tables()
{
    for (int a = 0; a <= 32; ++a)
        for (int k = 0; k <= 32; ++k)
            h_sg_binom[a][k] = k > a ? 0u : (k == 0 || k == a ? 1u : h_sg_binom[a - 1][k - 1] + h_sg_binom[a - 1][k]);
    cudaError_t e = cudaMemcpyToSymbol(c_sg_binom, h_sg_binom, sizeof h_sg_binom);
    if (e != cudaSuccess)
        return e;
    e = cudaFuncSetAttribute(sigma_sort_unique_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSigSortSmem);
    if (e != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(sigma_main_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSigSmemLarge);
}

cudaError_t sigma_main_occupancy(int b, int l, bool large, int *blocks_per_sm)
{
    const size_t smem = sigma_row_bytes(b, l) * sigma_smem_rows(b, l, large);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, sigma_main_kernel, kSigThreads, smem);
}

cudaError_t launch_sigma_pack(const uint8_t *seqs, int n, int m, int l, int b, const SigmaMap &map, uint32_t *planes,
                              uint32_t *flags, cudaStream_t st)
{
    const long long NW = (long long)n * (m - l + 1);
    const int threads = 256;
    const int blocks = (int)((NW + threads - 1) / threads);
    sigma_pack_kernel<<<blocks, threads, 0, st>>>(seqs, n, m, l, b, map, planes, flags);
    return cudaGetLastError();
}

cudaError_t launch_sigma_main(const SigmaParams &p, int blocks, cudaStream_t st)
{
    const size_t smem = sigma_row_bytes(p.b, p.l) * p.smem_rows;
    sigma_main_kernel<<<blocks, kSigThreads, smem, st>>>(p);
    return cudaGetLastError();
}

size_t sigma_sort_hist_words(int ctas)
{
    return (size_t)257 * ctas + 256;
}

cudaError_t sigma_sort_ctas(int *ctas)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sigma_sort_unique_kernel, kSigSortThreads,
                                                          kSigSortSmem);
    if (e != cudaSuccess)
        return e;
    *ctas = per_sm > 0 ? sms : 1;   // one CTA per SM, all resident
    return cudaSuccess;
}

cudaError_t launch_sigma_sort_unique(unsigned long long *raw, unsigned long long *tmp,
                                     const unsigned long long *raw_count, unsigned long long cap, int l, int b,
                                     const SigmaMap &letters, uint8_t *out, unsigned long long *unique_count,
                                     const SigSortGrid &grid, cudaStream_t st)
{
    // a cooperative launch: it fails rather than start CTAs that could not all be resident
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned int)grid.ctas);
    cfg.blockDim = dim3(kSigSortThreads);
    cfg.dynamicSmemBytes = kSigSortSmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sigma_sort_unique_kernel, raw, tmp, raw_count, cap, l, b, letters, out,
                              unique_count, grid);
}

}  // namespace pms
