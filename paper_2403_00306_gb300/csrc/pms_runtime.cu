// pms_runtime.cu -- host runtime behind the C ABI of include/pms.h:
// contexts, device-memory budget and arenas, plan building (queue chunks),
// the plain / device-resident / batched solves and the served scheduler.
#include "pms_internal.h"
#include "../../include/pms.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <set>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

using namespace pms;

namespace {

constexpr size_t kAlign = 256;
constexpr int kDefaultChunkWork = 1 << 20;
constexpr int kDefaultGrab = 1;         // node filter: the lane-asynchronous walk
constexpr uint32_t kInlineKeys = 512;   // codes downloaded together with the status block

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Rows tested at the partial-candidate level when no tuned value exists
// (-1: no partial level). The level pays when a random window is rarely within
// d of a candidate (E = expected such windows per sequence of a uniform
// i.i.d. instance, small for (17,5) and (19,6), about 0.5 for (13,4) and
// (15,5), where it was measured slower) and the tree has nodes with more than
// three changed positions (d >= 5).
// Expected windows of a uniform i.i.d. sequence of length m within d of a
// fixed l-mer: (m - l + 1) P(Binomial(l, 3/4) <= d).
double expected_near(int m, int l, int d)
{
    double p = 0, c = 1;
    for (int i = 0; i <= d; ++i) {
        p += c * std::pow(0.75, i) * std::pow(0.25, l - i);
        c = c * (l - i) / (i + 1);
    }
    return (m - l + 1) * p;
}

int default_partial_rows(int n, int m, int l, int d)
{
    (void)n;
    if (d < 5)
        return -1;
    return expected_near(m, l, d) < 0.15 ? 8 : -1;
}

// Rows the three-string test below a tree node pairs with the first when no
// option selects them (-1: none). It pays where a random window is rarely
// within d of a candidate (E = expected_near below 0.25: (15,4) E = 0.07,
// 0.115 -> 0.104 ms with 4 rows; (17,5) 1.69 -> 1.07 ms and (19,6) 18.9 ->
// 12.7 ms with 8; n = 20, m = 600) and costs where nodes keep many
// occurrences ((13,4), E = 0.58: 1.79 -> 2.35 ms with 2 rows; (11,3) and
// (9,2), d < 4, likewise slower).
int default_triple_rows(int n, int m, int l, int d)
{
    (void)n;
    if (d < 4 || expected_near(m, l, d) >= 0.25)
        return -1;
    return d >= 5 ? 8 : 4;
}

uint32_t pow2_at_least(size_t v)
{
    uint32_t p = 1;
    while (p < v && p < (1u << 31))
        p <<= 1;
    return p;
}

double now_ms()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint64_t binom(int a, int b)
{
    if (b < 0 || b > a)
        return 0;
    uint64_t r = 1;
    for (int i = 1; i <= b; ++i)
        r = r * (uint64_t)(a - b + i) / (uint64_t)i;
    return r;
}

uint64_t ball_size(int l, int d)
{
    uint64_t s = 0, p3 = 1;
    for (int i = 0; i <= d; ++i, p3 *= 3)
        s += binom(l, i) * p3;
    return s;
}

// The queue chunks of one seed for (l, d): levoff[0..d+1] (first subset index
// of each level in the seed's subset sequence), then (g0, g1) ranges. A node
// at level i costs 3^i leaf units plus kNodeUnits for its row filter; the
// seed's nodes are cut into round(total / work) ranges of equal cost (at
// least one), so that no chunk is a small remainder.
constexpr double kNodeUnits = 24.0;

struct ChunkTable {
    std::vector<int> tab;
    int cps = 0;
};

ChunkTable make_chunks(int l, int d, int work)
{
    ChunkTable ct;
    std::vector<int> lev(d + 2, 0);
    for (int i = 0; i <= d; ++i)
        lev[i + 1] = lev[i] + (int)binom(l, i);
    double total = 0;
    for (int i = 0; i <= d; ++i)
        total += (double)binom(l, i) * (std::pow(3.0, i) + kNodeUnits);
    const int k = std::max(1, (int)std::lround(total / std::max(1, work)));
    std::vector<int> cuts;
    double acc = 0;
    int start = 0, g = 0, made = 0;
    for (int i = 0; i <= d; ++i) {
        const double w = std::pow(3.0, i) + kNodeUnits;
        long long remaining = (long long)binom(l, i);
        while (remaining > 0) {
            // nodes of this level until the next cut (at (made + 1) / k of the total)
            const double next_cut = total * (made + 1) / k;
            const long long room = made + 1 < k ? std::max(1LL, (long long)std::ceil((next_cut - acc) / w)) : remaining;
            const long long take = std::min(room, remaining);
            acc += take * w;
            remaining -= take;
            g += (int)take;
            if (made + 1 < k && acc >= next_cut - 1e-9) {
                cuts.push_back(start);
                cuts.push_back(g);
                start = g;
                ++made;
            }
        }
    }
    if (start < g) {
        cuts.push_back(start);
        cuts.push_back(g);
    }
    ct.tab = lev;
    ct.tab.insert(ct.tab.end(), cuts.begin(), cuts.end());
    ct.cps = (int)cuts.size() / 2;
    return ct;
}


// The chunks of one seed cut into k ranges of equal cost (as make_chunks).
ChunkTable make_chunks_k(int l, int d, int k)
{
    double total = 0;
    for (int i = 0; i <= d; ++i)
        total += (double)binom(l, i) * (std::pow(3.0, i) + kNodeUnits);
    return make_chunks(l, d, (int)std::max(1.0, std::floor(total / k)));
}

}  // namespace

// ---------------------------------------------------------------------------------- context

struct Served;

struct pms_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    void *(*ualloc)(size_t, void *) = nullptr;
    void (*ufree)(void *, void *) = nullptr;
    void *uuser = nullptr;
    size_t budget = 0;     // 0: unlimited
    size_t used = 0;
    std::recursive_mutex mu;
    std::string err;
    pms_options opt{};
    int num_sms = 0;
    int occ[2] = {0, 0};   // CTAs per SM of the verification kernel (plain, count mode)
    int occ_small[2] = {0, 0};  // same for its small-rows form
    int occ_pair[2] = {0, 0};  // same for the pair-form kernel
    pms_stats stats{};
    std::map<std::tuple<int, int, int>, ChunkTable> ctab_cache;

    struct DBuf {
        void *p = nullptr;
        size_t cap = 0;
    };
    DBuf d_seqs, d_planes, d_raw, d_tmp, d_compat, d_rowlen, d_mode, d_meta, d_ctr, d_scratch, d_result;
    // general-alphabet solves (pms_solve_sigma)
    DBuf d_sg_seqs, d_sg_planes, d_sg_ctr, d_sg_raw, d_sg_out, d_sg_scratch, d_sg_lists, d_sg_hist;
    bool sigma_ready = false;   // binomial table and kernel attributes loaded on the device
    int sg_sort_ctas = 1;       // CTAs of the sort/unique grid
    void *h_sg = nullptr;       // pinned, mapped: counters block, then the input letters
    size_t h_sg_cap = 0;
    void *h_sg_out = nullptr;   // pinned, mapped: decoded motifs of small outputs
    size_t h_sg_out_cap = 0;
    std::vector<uint8_t> owned_sigma;   // letters returned by the last pms_solve_sigma
    void *h_result = nullptr;   // pinned, mapped: results of host-memory solves
    size_t h_result_cap = 0;
    void *h_in = nullptr;       // pinned, mapped: inputs of host-memory solves
    size_t h_in_cap = 0;
    void *h_meta = nullptr;     // pinned staging for descriptors and inputs
    size_t h_meta_cap = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evm0 = nullptr, evm1 = nullptr;
    bool stats_pending = false;   // device times / counters of the last solve not read yet
    bool stats_timed = false;     // the last solve recorded its device-time events
    bool stats_count = false;
    size_t stats_k = 0;

    std::vector<std::vector<uint64_t>> owned;   // result codes returned by the last solve call
    Served *served = nullptr;

    // Captured pipelines of one-instance plans (CUDA graphs), keyed by the
    // options and the plan's descriptors; replayed with the input and output
    // pointers of each call patched into the packing node (the pack kernel, or
    // the pack + masks kernel of one-instance plans) and the sort/unique node.
    struct Graph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t x = nullptr;
        cudaGraphNode_t pack = nullptr, sort = nullptr;
        cudaKernelNodeParams pack_p{}, sort_p{};
        // the pointers the executable graph holds now (its nodes are updated only when a call's differ)
        const void *applied_seqs = nullptr;
        const void *applied_status = nullptr, *applied_dense = nullptr;
        uint32_t applied_cap = 0;
        struct {
            const void *inst;
            int ninst;
            const void *win_prefix;
            long long total;
            const void *seqs;
            void *planes;
            void *flags;
        } pv{};
        struct {
            const void *inst;
            const void *list;
            void *raw;
            void *tmp;
            const void *raw_count;
            const void *flags;
            void *status;
            void *dense;
            uint32_t dense_cap;
            void *dense_total;
        } sv{};
        struct {
            const void *inst;
            const void *seqs;
            void *planes;
            void *compat;
            void *rowlen;
            void *flags;
        } rv{};                // the one-instance pack + masks kernel, when the plan uses it
        bool input_rows = false;   // the node `pack` is that kernel (input pointer: argument 1)
        void *pack_args[7] = {};
        void *rows_args[6] = {};
        void *sort_args[10] = {};
        DBuf meta;             // this plan's descriptors (the kernels of the graph read them)
        uint64_t gen = 0;      // buffer generation the graph was captured with
        uint64_t candidates = 0;
        uint64_t last_use = 0;
    };
    std::map<std::string, Graph> graphs;
    std::set<std::string> seen_plans;   // plans run once kernel by kernel (captured on the next call)
    cudaStream_t cap_stream = nullptr;
    uint64_t buf_gen = 0;      // bumped whenever a device buffer is freed or moved
    uint64_t use_tick = 0;
    uint64_t graph_replays = 0;   // solves enqueued by replaying a captured graph

    // Injected host-side failures (pms_inject_fault), per kind: operations
    // that still succeed first, then operations that fail. Read and changed
    // with mu held.
    struct Fault {
        int after = 0, count = 0;
    } faults[3];
    bool inject(int kind)
    {
        Fault &f = faults[kind];
        if (f.count <= 0)
            return false;
        if (f.after > 0) {
            --f.after;
            return false;
        }
        --f.count;
        return true;
    }

    int fail(int code, const char *fmt, ...)
    {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        err = buf;
        return code;
    }
    int cuda_fail(cudaError_t e, const char *what)
    {
        return fail(e == cudaErrorMemoryAllocation ? PMS_ENOMEM : PMS_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    }

    void *dev_alloc(size_t bytes)
    {
        if (budget && used + bytes > budget)
            return nullptr;
        if (inject(PMS_FAULT_ALLOC))
            return nullptr;
        void *p = nullptr;
        if (ualloc) {
            p = ualloc(bytes, uuser);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p)
            used += bytes;
        return p;
    }
    void dev_free(void *p, size_t bytes)
    {
        if (!p)
            return;
        if (ufree)
            ufree(p, uuser);
        else
            cudaFree(p);
        used -= bytes;
    }
    // Grow-only device buffer. Returns PMS_OK or PMS_ENOMEM.
    int ensure(DBuf &b, size_t bytes)
    {
        bytes = round_up(std::max<size_t>(bytes, 1), kAlign);
        if (b.cap >= bytes)
            return PMS_OK;
        if (b.p) {
            cudaStreamSynchronize(stream);
            dev_free(b.p, b.cap);
            b.p = nullptr;
            b.cap = 0;
            ++buf_gen;   // captured graphs that use the old buffer are stale
        }
        const size_t want = std::max(bytes, (size_t)(bytes * 5 / 4));
        void *p = dev_alloc(want);
        if (!p) {
            p = dev_alloc(bytes);
            if (!p)
                return fail(PMS_ENOMEM, "device allocation of %zu bytes refused (budget %zu, in use %zu)", bytes,
                            budget, used);
            b.cap = bytes;
        } else {
            b.cap = want;
        }
        b.p = p;
        return PMS_OK;
    }
    int ensure_host(void *&p, size_t &cap, size_t bytes, unsigned int flags = cudaHostAllocDefault)
    {
        if (cap >= bytes)
            return PMS_OK;
        if (p) {
            cudaStreamSynchronize(stream);
            cudaFreeHost(p);
            p = nullptr;
            cap = 0;
        }
        bytes = round_up(std::max(bytes, cap * 2), 4096);
        cudaError_t e = cudaHostAlloc(&p, bytes, flags);
        if (e != cudaSuccess) {
            p = nullptr;
            return cuda_fail(e, "cudaHostAlloc");
        }
        cap = bytes;
        return PMS_OK;
    }

    // Autotuned schedules per instance class (l, d, n bucket, m bucket).
    struct Tuning {
        int chunk_work = 0;
        int prune_rows = 0;   // 0: all rows
        int ctas_per_sm = 0;
        int grab = 0;         // node filter (InstDev.grab; 0: the default)
        int partial_rows = 0; // rows of the partial-candidate level: -1 none, 0 default, k > 0
        double ms = 0;
    };
    std::map<std::tuple<int, int, int, int>, Tuning> tuned;
    static int bucket(int v)
    {
        int b = 1;
        while (b < v)
            b <<= 1;
        return b;
    }
    const Tuning *tuning(int n, int m, int l, int d) const
    {
        auto it = tuned.find(std::make_tuple(l, d, bucket(n), bucket(m)));
        return it == tuned.end() ? nullptr : &it->second;
    }
    // 0: no fixed value (the plan sizes chunks from its total work)
    int chunk_work_for(int n, int m, int l, int d) const
    {
        if (opt.chunk_work > 0)
            return opt.chunk_work;
        const Tuning *t = tuning(n, m, l, d);
        return t && t->chunk_work > 0 ? t->chunk_work : 0;
    }
    // node filter of the verification kernel (InstDev.grab): 1 = lane walk
    // (default), g > 1 = breadth-first batches shrinking to g nodes
    int grab_for(int n, int m, int l, int d) const
    {
        if (opt.grab > 0)
            return opt.grab;
        const Tuning *t = tuning(n, m, l, d);
        return t && t->grab > 0 ? t->grab : kDefaultGrab;
    }
    // rows the partial-candidate level tests (0: no partial level)
    int partial_rows_for(int n, int m, int l, int d) const
    {
        int v = opt.partial_rows;
        if (v == 0) {
            const Tuning *t = tuning(n, m, l, d);
            v = t ? t->partial_rows : 0;
        }
        if (v == 0)
            v = default_partial_rows(n, m, l, d);
        return v < 0 ? 0 : std::min(v, n - 1);
    }
    // rows the three-string test pairs with the first (0: no test)
    int triple_rows_for(int n, int m, int l, int d) const
    {
        int v = opt.triple_rows;
        if (v == 0)
            v = default_triple_rows(n, m, l, d);
        return v < 0 ? 0 : std::min(v, n - 2);
    }
    int prune_rows_for(int n, int m, int l, int d) const
    {
        const Tuning *t = tuning(n, m, l, d);
        return t && t->prune_rows > 0 ? std::min(t->prune_rows, n - 1) : n - 1;
    }

    const ChunkTable &chunks(int l, int d, int work = 0)
    {
        if (work <= 0)
            work = opt.chunk_work > 0 ? opt.chunk_work : kDefaultChunkWork;
        auto key = std::make_tuple(l, d, work);
        auto it = ctab_cache.find(key);
        if (it == ctab_cache.end())
            it = ctab_cache.emplace(key, make_chunks(l, d, work)).first;
        return it->second;
    }
};

// Checks one instance's parameters. Returns PMS_OK or PMS_EINVAL (with text).
static int check_params(pms_ctx *h, int n, int m, int l, int d)
{
    if (n < 1 || n > PMS_NMAX)
        return h->fail(PMS_EINVAL, "n = %d outside [1, %d]", n, PMS_NMAX);
    if (l < 1 || l > PMS_LMAX)
        return h->fail(PMS_EINVAL, "l = %d outside [1, %d]", l, PMS_LMAX);
    if (m < l || m > 65536)
        return h->fail(PMS_EINVAL, "m = %d outside [l, 65536]", m);
    if (d < 0 || d >= l)
        return h->fail(PMS_EINVAL, "d = %d outside [0, l)", d);
    uint64_t subsets = 0;
    for (int i = 0; i <= d; ++i)
        subsets += binom(l, i);
    if (subsets > (uint64_t)INT32_MAX)
        return h->fail(PMS_EINVAL, "(l, d) = (%d, %d): subset space too large", l, d);
    return PMS_OK;
}

static int check_bytes(pms_ctx *h, const uint8_t *s, size_t len)
{
    // a table lookup per byte, OR-accumulated over blocks (no branch per byte)
    static const struct Table {
        uint8_t bad[256];
        Table()
        {
            for (int c = 0; c < 256; ++c)
                bad[c] = (c == 'A' || c == 'C' || c == 'G' || c == 'T') ? 0 : 1;
        }
    } t;
    size_t i = 0;
    for (; i + 64 <= len; i += 64) {
        unsigned acc = 0;
        for (size_t j = 0; j < 64; ++j)
            acc |= t.bad[s[i + j]];
        if (acc)
            break;
    }
    for (; i < len; ++i)
        if (t.bad[s[i]])
            return h->fail(PMS_EINVAL, "byte %zu (0x%02x) is not one of A, C, G, T", i, s[i]);
    return PMS_OK;
}

// ------------------------------------------------------------------------- plan of one launch

namespace {

struct InstSpec {
    int n, m, l, d;
    const uint8_t *host_seqs;   // may be null (device-resident input)
    uint32_t raw_cap = 0;       // 0: from max_motifs or the estimate
};

// Host image of everything the kernels need for a set of instances.
struct Plan {
    std::vector<InstDev> inst;
    std::vector<Segment> seg;
    std::vector<long long> win_prefix;
    std::vector<long long> row_prefix;   // compatibility rows: sum of W * (n - 1)
    bool small_rows = false;             // verification kernel in its small-rows form (4 CTAs per SM)
    std::vector<long long> seed_prefix;  // seeds: sum of W
    std::vector<Segment> seg_pair;       // pair-form queue (blocks of 64 windows of s_2 per seed)
    long long total_pair_items = 0;
    long long total_seeds = 0;
    bool pair_mode = false;
    std::vector<int> ctab;
    long long total_items = 0;
    long long total_windows = 0;
    long long total_rows = 0;
    size_t seq_bytes = 0, planes = 0, raw = 0, compat = 0, rowlen = 0;
    int rows_cap = 1;
    uint64_t candidates = 0;
};

// Byte layout of the descriptor block (device d_meta, pinned h_meta).
struct MetaLayout {
    size_t inst, seg, win, rowp, seedp, segp, ctab, total;
    MetaLayout(const Plan &p)
    {
        size_t o = 0;
        inst = o;
        o = round_up(o + p.inst.size() * sizeof(InstDev), 16);
        seg = o;
        o = round_up(o + p.seg.size() * sizeof(Segment), 16);
        win = o;
        o = round_up(o + p.win_prefix.size() * sizeof(long long), 16);
        rowp = o;
        o = round_up(o + p.row_prefix.size() * sizeof(long long), 16);
        seedp = o;
        o = round_up(o + p.seed_prefix.size() * sizeof(long long), 16);
        segp = o;
        o = round_up(o + p.seg_pair.size() * sizeof(Segment), 16);
        ctab = o;
        o = round_up(o + p.ctab.size() * sizeof(int), 16);
        total = o;
    }
};

// Counters block (d_ctr): head, work counters, dense_total, then per instance
// raw_count and flags, then (items > 0) the steal cursor and the nodes claimed
// of every queue item, for the verification kernel's work sharing.
struct CtrLayout {
    size_t head, head_pair, work, dense_total, raw_count, flags, steal, claim, total;
    CtrLayout(size_t k, size_t items = 0)
    {
        head = 0;
        head_pair = 8;
        work = 16;
        dense_total = work + kCntNum * 8;
        raw_count = round_up(dense_total + 4, 16);
        flags = round_up(raw_count + 4 * k, 16);
        steal = round_up(flags + 4 * k, 16);
        claim = steal + 16;
        total = round_up(claim + 8 * items, 256);
    }
};

// Result block (d_result): StatusDev per instance, then the dense codes.
struct ResLayout {
    size_t status, dense, total;
    uint32_t dense_cap;
    ResLayout(size_t k, size_t dense_keys)
    {
        status = 0;
        dense = round_up(k * sizeof(StatusDev), 16);
        dense_cap = (uint32_t)dense_keys;
        total = dense + dense_keys * 8;
    }
};

}  // namespace

// Expected raw motif count (duplicates included) of an FM-like instance under
// independence: W |B(x,d)| q^(n-1), q = P(a random sequence has a window
// within d of a fixed l-mer). Sizes the raw buffer; overflow triggers a retry.
static double expected_raw(int n, int m, int l, int d, int quorum = 0)
{
    const int W = m - l + 1;
    const double nb = (double)ball_size(l, d);
    const double p = std::min(1.0, nb / std::pow(4.0, l));
    const double q = 1.0 - std::pow(1.0 - p, W);
    if (quorum <= 0 || quorum >= n)
        return W * nb * std::pow(q, n - 1);
    // quorum form: seeds from n - quorum + 1 sequences, a candidate needs
    // quorum - 1 of the other n - 1 sequences: binomial tail
    double tail = 0;
    for (int i = quorum - 1; i <= n - 1; ++i)
        tail += (double)binom(n - 1, i) * std::pow(q, i) * std::pow(1.0 - q, n - 1 - i);
    return (double)(n - quorum + 1) * W * nb * tail;
}

static uint32_t default_cap(const pms_ctx *h, const InstSpec &s, bool single)
{
    if (s.raw_cap)
        return s.raw_cap;
    if (h->opt.max_motifs)
        return pow2_at_least(h->opt.max_motifs);
    const double est = 4.0 * expected_raw(s.n, s.m, s.l, s.d, h->opt.quorum) + 256.0;
    const size_t lo = single ? (size_t)1 << 16 : (size_t)1 << 12;
    return pow2_at_least(std::min<double>(std::max<double>(est, lo), (double)(1u << 24)));
}

static int default_prune_rows(int n, int d)
{
    (void)d;
    return n - 1;
}

// Resident CTAs per SM of the verification kernel for an instance class: the
// occupancy, capped by the option or by the class's tuned value.
static int plan_occ(const pms_ctx *h, int n, int m, int l, int d, bool count_mode, bool small_rows)
{
    int occ = small_rows ? h->occ_small[count_mode ? 1 : 0] : h->occ[count_mode ? 1 : 0];
    if (h->opt.ctas_per_sm > 0) {
        occ = std::min(occ, h->opt.ctas_per_sm);
    } else {
        const pms_ctx::Tuning *t = h->tuning(n, m, l, d);
        if (t && t->ctas_per_sm > 0)
            occ = std::min(occ, t->ctas_per_sm);
    }
    return std::max(occ, 1);
}

// Expected feasible occurrences of one seed of a uniform i.i.d. instance:
// (n - 1) rows of W windows, each within 2d of the seed with probability
// P(Binomial(l, 3/4) <= 2d), plus the rows' padding.
// Expected feasible occurrences per seed up to which a plan takes the
// verification kernel's 4-CTA form (1280 entries in shared memory; seeds with
// up to three times as many keep their mismatch masks there and read the
// planes of passing occurrences from global memory). Measured: (19,6), about
// 1900 per seed, 12.1 -> 11.3 ms in this form; (13,4) at m = 600, about 2400
// per seed, 1.70 -> 1.75 ms, so it keeps the 3-CTA form with 2560 entries.
constexpr double kSmallFormRows = 1.6 * kRowSmemCapSmall;

static double expected_seed_rows(int n, int m, int l, int d)
{
    double p = 0, c = 1;
    for (int i = 0; i <= std::min(2 * d, l); ++i) {
        p += c * std::pow(0.75, i) * std::pow(0.25, l - i);
        c = c * (l - i) / (i + 1);
    }
    return (n - 1) * ((m - l + 1) * p + 3.0);
}

static Plan make_plan(pms_ctx *h, const std::vector<InstSpec> &specs)
{
    Plan P;
    // the small-rows form when every instance's seeds are expected to keep
    // their rows in its shared memory (seeds with more, such as those near the
    // planted copies, read their rows from the CTA's global scratch)
    P.small_rows = h->occ_small[0] > h->occ[0];
    for (const InstSpec &s : specs)
        if (expected_seed_rows(s.n, s.m, s.l, s.d) > kSmallFormRows)
            P.small_rows = false;
    long long work = 0;
    const int adaptive = kDefaultChunkWork;   // untuned classes: about 2^20 candidate units per queue item
    bool quorum_used = false;
    for (size_t k = 0; k < specs.size(); ++k) {
        const InstSpec &s = specs[k];
        InstDev in{};
        in.n = s.n;
        in.m = s.m;
        in.l = s.l;
        in.d = s.d;
        in.W = s.m - s.l + 1;
        in.NW = (in.W + 31) / 32;
        in.q = (h->opt.quorum > 0 && h->opt.quorum < s.n) ? h->opt.quorum : s.n;
        in.nseed = s.n - in.q + 1;
        const long long seeds = (long long)in.nseed * in.W;
        const int cw = h->chunk_work_for(s.n, s.m, s.l, s.d);
        const ChunkTable &ct = h->chunks(s.l, s.d, cw > 0 ? cw : adaptive);
        in.cps = ct.cps;
        in.grab = h->grab_for(s.n, s.m, s.l, s.d);
        in.prune_rows = h->prune_rows_for(s.n, s.m, s.l, s.d);
        in.partial_rows = h->partial_rows_for(s.n, s.m, s.l, s.d);
        in.triple_rows = h->triple_rows_for(s.n, s.m, s.l, s.d);
        in.ctab = (int)P.ctab.size();
        P.ctab.insert(P.ctab.end(), ct.tab.begin(), ct.tab.end());
        in.seq_off = (long long)P.seq_bytes;
        P.seq_bytes += round_up((size_t)s.n * s.m, 16);
        in.plane_off = (long long)P.planes;
        P.planes += (size_t)s.n * in.W;
        in.raw_off = (long long)P.raw;
        in.raw_cap = default_cap(h, s, specs.size() == 1);
        P.raw += in.raw_cap;
        in.compat_off = (long long)P.compat;
        P.compat += (size_t)seeds * (s.n - 1) * in.NW;
        in.rlen_off = (long long)P.rowlen;
        P.rowlen += (size_t)seeds * (s.n - 1);
        P.win_prefix.push_back(P.total_windows);
        P.total_windows += (long long)s.n * in.W;
        P.row_prefix.push_back(P.total_rows);
        P.total_rows += seeds * (s.n - 1);
        in.seed_off = P.total_seeds;
        P.seed_prefix.push_back(P.total_seeds);
        P.total_seeds += in.W;
        in.cps_b = (in.W + 63) / 64;
        P.seg_pair.push_back(Segment{P.total_pair_items, (int)k, 0, in.W * in.cps_b, 0});
        P.total_pair_items += (long long)in.W * in.cps_b;
        P.rows_cap = std::max(P.rows_cap, (int)round_up((size_t)(s.n - 1) * (in.W + 3), 4));
        const int chunks = (int)(seeds * in.cps);
        // one instance of whole-seed items whose last round would occupy only r
        // of the B CTAs: the r seeds of that round are cut into floor(B / r)
        // equal-cost chunks each, so that the round ends with all CTAs busy
        const long long B =
            (long long)h->num_sms * plan_occ(h, s.n, s.m, s.l, s.d, h->opt.count_work != 0, P.small_rows);
        const long long r = seeds % B;
        const int kk = r > 0 ? (int)std::min<long long>(B / r, 16) : 0;
        if (specs.size() == 1 && in.cps == 1 && seeds > B && kk >= 2) {
            const ChunkTable ct2 = make_chunks_k(s.l, s.d, kk);
            const int whole = (int)(seeds - r);
            P.seg.push_back(Segment{work, (int)k, 0, whole, 0, 0, 0});
            work += whole;
            const int ctab2 = (int)P.ctab.size();
            P.ctab.insert(P.ctab.end(), ct2.tab.begin(), ct2.tab.end());
            P.seg.push_back(Segment{work, (int)k, 0, (int)(r * ct2.cps), ct2.cps, whole, ctab2});
            work += r * ct2.cps;
        } else {
            P.seg.push_back(Segment{work, (int)k, 0, chunks, 0, 0, 0});
            work += chunks;
        }
        P.candidates += (uint64_t)seeds * ball_size(s.l, s.d);
        if (in.q < in.n)
            quorum_used = true;
        P.inst.push_back(in);
    }
    P.total_items = work;
    P.pair_mode = h->opt.seed_mode == 1 && !quorum_used;   // pair seeds are for q = n
    return P;
}

// Records a timing event. Inside a stream capture (a graph's launches) the
// event is a node of its own, recorded by every replay; an event node between
// two kernels costs the launch overlap of the pair (about 17 us per plain
// (15,4) solve on GB300), so graphs carry them only when pms_options.graph
// asks for timed replays.
static void record_event(const pms_ctx *h, cudaEvent_t ev, cudaStream_t st, bool capturing)
{
    if (!capturing)
        cudaEventRecord(ev, st);
    else if (h->opt.graph >= 1)
        cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
}

// CTAs of the verification kernel for a plan: resident CTAs per SM (capped by
// the option or the tuned value of the first instance's class) x SMs, at most
// two per queue item (CTAs without an item of their own join the items that
// have the most unclaimed tree nodes).
static int plan_blocks(const pms_ctx *h, const Plan &P, bool count_mode)
{
    const int occ = P.inst.empty()
                        ? std::max(1, h->occ[count_mode ? 1 : 0])
                        : plan_occ(h, P.inst[0].n, P.inst[0].m, P.inst[0].l, P.inst[0].d, count_mode, P.small_rows);
    return (int)std::min<long long>((long long)h->num_sms * occ, std::max<long long>(2 * P.total_items, 1));
}

// Host image of a plan's descriptors (layout ml) at dst.
static void fill_meta(const Plan &P, const MetaLayout &ml, char *hm)
{
    std::memcpy(hm + ml.inst, P.inst.data(), P.inst.size() * sizeof(InstDev));
    std::memcpy(hm + ml.seg, P.seg.data(), P.seg.size() * sizeof(Segment));
    std::memcpy(hm + ml.win, P.win_prefix.data(), P.win_prefix.size() * sizeof(long long));
    std::memcpy(hm + ml.rowp, P.row_prefix.data(), P.row_prefix.size() * sizeof(long long));
    std::memcpy(hm + ml.seedp, P.seed_prefix.data(), P.seed_prefix.size() * sizeof(long long));
    std::memcpy(hm + ml.segp, P.seg_pair.data(), P.seg_pair.size() * sizeof(Segment));
    std::memcpy(hm + ml.ctab, P.ctab.data(), P.ctab.size() * sizeof(int));
}

// Enqueues the whole pipeline of a plan on h->stream. d_seq_src: device
// address of the input bytes (internal arena or user memory). Descriptors are
// staged in h->h_meta and uploaded. Output: status/dense in the result block.
// meta_dev: when given, the plan's descriptors are already on the device
// there (a captured graph's own copy) and are neither staged nor uploaded.
static int enqueue_plan(pms_ctx *h, const Plan &P, const uint8_t *d_seq_src, StatusDev *status_out,
                        uint64_t *dense_out, uint32_t dense_cap, bool count_mode, char *meta_dev = nullptr)
{
    const size_t k = P.inst.size();
    MetaLayout ml(P);
    CtrLayout cl(k, (size_t)P.total_items);
    int rc;
    if ((rc = h->ensure(h->d_meta, ml.total)) || (rc = h->ensure(h->d_ctr, cl.total)) ||
        (rc = h->ensure(h->d_planes, P.planes * sizeof(uint2))) || (rc = h->ensure(h->d_raw, P.raw * 8)) ||
        (rc = h->ensure(h->d_tmp, P.raw * 8)) || (rc = h->ensure(h->d_compat, P.compat * 4)) ||
        (rc = h->ensure(h->d_rowlen, P.rowlen * 4)) || (rc = h->ensure(h->d_mode, (size_t)P.total_seeds)))
        return rc;
    const int blocks = plan_blocks(h, P, count_mode);
    if ((rc = h->ensure(h->d_scratch, (size_t)blocks * 3 * (size_t)P.rows_cap * sizeof(uint32_t))))
        return rc;
    cudaStream_t st = h->stream;
    if (!meta_dev)
        h->stats_timed = true;
    char *dm = meta_dev ? meta_dev : (char *)h->d_meta.p;
    char *dc = (char *)h->d_ctr.p;
    cudaError_t e;
    if (!meta_dev) {
        if ((rc = h->ensure_host(h->h_meta, h->h_meta_cap, ml.total)))
            return rc;
        char *hm = (char *)h->h_meta;
        fill_meta(P, ml, hm);
        if ((e = cudaMemcpyAsync(dm, hm, ml.total, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return h->cuda_fail(e, "upload descriptors");
    }
    if ((e = cudaMemsetAsync(dc, 0, cl.total, st)) != cudaSuccess)
        return h->cuda_fail(e, "clear counters");
    const InstDev *d_inst = (const InstDev *)(dm + ml.inst);
    uint32_t *d_flags = (uint32_t *)(dc + cl.flags);
    uint32_t *d_rawcnt = (uint32_t *)(dc + cl.raw_count);
    record_event(h, h->ev0, st, meta_dev != nullptr);
    const bool by_rows = P.total_rows > 0 && k == 1 && compat_rows_fits(P.inst[0].W);
    if (by_rows) {
        // one instance: packing and masks in one kernel, a CTA per (sequence, 16 seeds)
        const InstDev &i0 = P.inst[0];
        if ((e = launch_compat_rows(d_inst, i0.n, (long long)i0.nseed * i0.W, d_seq_src, (uint2 *)h->d_planes.p,
                                    (uint32_t *)h->d_compat.p, (int *)h->d_rowlen.p, d_flags, st)) != cudaSuccess)
            return h->cuda_fail(e, "compatibility kernel");
    } else {
        const int pack_blocks = (int)std::min<long long>((P.total_windows + 255) / 256, (long long)h->num_sms * 8);
        if ((e = launch_pack(d_inst, (int)k, (const long long *)(dm + ml.win), P.total_windows, d_seq_src,
                             (uint2 *)h->d_planes.p, d_flags, std::max(pack_blocks, 1), st)) != cudaSuccess)
            return h->cuda_fail(e, "pack kernel");
    }
    if (P.total_rows > 0 && !by_rows) {
        const int cw_blocks = (int)std::min<long long>((P.total_rows + 7) / 8, (long long)h->num_sms * 16);
        if ((e = launch_compat(d_inst, (int)k, (const long long *)(dm + ml.rowp), P.total_rows,
                               (const uint2 *)h->d_planes.p, (uint32_t *)h->d_compat.p, (int *)h->d_rowlen.p,
                               std::max(cw_blocks, 1), st)) !=
            cudaSuccess)
            return h->cuda_fail(e, "compatibility kernel");
    }
    if (P.pair_mode && P.total_seeds > 0) {
        const int cb = (int)std::min<long long>((P.total_seeds + 7) / 8, (long long)h->num_sms * 16);
        if ((e = launch_classify(d_inst, (int)k, (const long long *)(dm + ml.seedp), P.total_seeds,
                                 (const uint2 *)h->d_planes.p, (const uint32_t *)h->d_compat.p, (uint8_t *)h->d_mode.p,
                                 std::max(cb, 1), st)) != cudaSuccess)
            return h->cuda_fail(e, "classify kernel");
    }
    MainParams mp{};
    mp.mode = P.pair_mode ? (const uint8_t *)h->d_mode.p : nullptr;
    mp.inst = d_inst;
    mp.seg = (const Segment *)(dm + ml.seg);
    mp.nseg = (int)P.seg.size();
    mp.total = P.total_items;
    mp.head = (unsigned long long *)(dc + cl.head);
    mp.planes = (const uint2 *)h->d_planes.p;
    mp.compat = (const uint32_t *)h->d_compat.p;
    mp.rowlen = (const int *)h->d_rowlen.p;
    mp.ctab = (const int *)(dm + ml.ctab);
    mp.raw = (uint64_t *)h->d_raw.p;
    mp.raw_count = d_rawcnt;
    mp.flags = d_flags;
    mp.scratch = (uint32_t *)h->d_scratch.p;
    mp.rows_cap = P.rows_cap;
    const int rows_cap_smem = P.small_rows ? kRowSmemCapSmall : kRowSmemCap;
    mp.smem_rows_cap = h->opt.smem_rows > 0 ? std::min(h->opt.smem_rows, rows_cap_smem) : rows_cap_smem;
    mp.counters = (unsigned long long *)(dc + cl.work);
    mp.item_claim = (int *)(dc + cl.claim);
    mp.steal_state = (unsigned int *)(dc + cl.steal);
    record_event(h, h->evm0, st, meta_dev != nullptr);
    if (P.total_items > 0 && (e = launch_main(mp, blocks, count_mode, st, P.small_rows)) != cudaSuccess)
        return h->cuda_fail(e, "verification kernel");
    if (P.pair_mode && P.total_pair_items > 0) {
        MainParams pp = mp;
        pp.item_claim = nullptr;   // the pair kernel claims pairs within its own CTA
        pp.steal_state = nullptr;
        pp.seg = (const Segment *)(dm + ml.segp);
        pp.nseg = (int)P.seg_pair.size();
        pp.total = P.total_pair_items;
        pp.head = (unsigned long long *)(dc + cl.head_pair);
        int occp = std::max(1, h->occ_pair[count_mode ? 1 : 0]);
        const int pblocks = (int)std::min<long long>((long long)h->num_sms * occp, P.total_pair_items);
        if (pblocks > blocks && (rc = h->ensure(h->d_scratch, (size_t)pblocks * 3 * (size_t)P.rows_cap * 4)))
            return rc;
        pp.scratch = (uint32_t *)h->d_scratch.p;
        if ((e = launch_pairs(pp, pblocks, count_mode, st)) != cudaSuccess)
            return h->cuda_fail(e, "pair kernel");
    }
    record_event(h, h->evm1, st, meta_dev != nullptr);
    if ((e = launch_sort_unique(d_inst, nullptr, (int)k, (uint64_t *)h->d_raw.p, (uint64_t *)h->d_tmp.p, d_rawcnt,
                                d_flags, status_out,
                                dense_out, dense_cap, (uint32_t *)(dc + cl.dense_total), st)) != cudaSuccess)
        return h->cuda_fail(e, "sort/unique kernel");
    record_event(h, h->ev1, st, meta_dev != nullptr);
    return PMS_OK;
}

// ------------------------------------------------------------------ captured graphs

constexpr size_t kMaxGraphs = 32;

static void destroy_graph(pms_ctx *h, pms_ctx::Graph &G)
{
    if (G.x)
        cudaGraphExecDestroy(G.x);
    if (G.g)
        cudaGraphDestroy(G.g);
    h->dev_free(G.meta.p, G.meta.cap);
    G = pms_ctx::Graph{};
}

static void clear_graphs(pms_ctx *h)
{
    if (h->graphs.empty())
        return;
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    for (auto &kv : h->graphs)
        destroy_graph(h, kv.second);
    h->graphs.clear();
}

// Captures the launches of plan P (descriptor image `key`, which this call
// has just run kernel by kernel) into a graph with its own descriptor copy.
// Failure leaves no graph; the plan then keeps running kernel by kernel.
static void capture_graph(pms_ctx *h, const std::string &key, const Plan &P, const MetaLayout &ml,
                          const uint8_t *d_seq_src, StatusDev *status_out, uint64_t *dense_out, uint32_t dense_cap)
{
    if (h->graphs.size() >= kMaxGraphs) {
        auto lru = h->graphs.begin();
        for (auto it = h->graphs.begin(); it != h->graphs.end(); ++it)
            if (it->second.last_use < lru->second.last_use)
                lru = it;
        cudaStreamSynchronize(h->stream);
        destroy_graph(h, lru->second);
        h->graphs.erase(lru);
    }
    pms_ctx::Graph G;
    if (h->ensure(G.meta, ml.total))
        return;
    // the descriptors this call uploaded, copied in stream order
    cudaError_t e = cudaMemcpyAsync(G.meta.p, h->d_meta.p, ml.total, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess && !h->cap_stream)
        e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    const uint64_t gen = h->buf_gen;
    int rc = PMS_ECUDA;
    if (e == cudaSuccess && (e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed)) == cudaSuccess) {
        cudaStream_t saved = h->stream;
        h->stream = h->cap_stream;
        rc = enqueue_plan(h, P, d_seq_src, status_out, dense_out, dense_cap, false, (char *)G.meta.p);
        h->stream = saved;
        e = cudaStreamEndCapture(h->cap_stream, &G.g);
    }
    if (rc == PMS_OK && e == cudaSuccess && G.g && h->buf_gen == gen)
        e = cudaGraphInstantiate(&G.x, G.g, 0);
    else if (e == cudaSuccess)
        e = cudaErrorUnknown;
    // the two nodes whose arguments change from call to call
    if (e == cudaSuccess) {
        size_t nn = 0;
        cudaGraphGetNodes(G.g, nullptr, &nn);
        std::vector<cudaGraphNode_t> nodes(nn);
        if (nn)
            cudaGraphGetNodes(G.g, nodes.data(), &nn);
        for (cudaGraphNode_t nd : nodes) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel)
                continue;
            cudaKernelNodeParams kp{};
            if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess || !kp.kernelParams)
                continue;
            if (kp.func == compat_rows_kernel_fn()) {
                G.pack = nd;
                G.pack_p = kp;
                G.input_rows = true;
                void **a = kp.kernelParams;
                std::memcpy(&G.rv.inst, a[0], sizeof G.rv.inst);
                std::memcpy(&G.rv.seqs, a[1], sizeof G.rv.seqs);
                std::memcpy(&G.rv.planes, a[2], sizeof G.rv.planes);
                std::memcpy(&G.rv.compat, a[3], sizeof G.rv.compat);
                std::memcpy(&G.rv.rowlen, a[4], sizeof G.rv.rowlen);
                std::memcpy(&G.rv.flags, a[5], sizeof G.rv.flags);
            } else if (kp.func == pack_kernel_fn()) {
                G.pack = nd;
                G.pack_p = kp;
                void **a = kp.kernelParams;
                std::memcpy(&G.pv.inst, a[0], sizeof G.pv.inst);
                std::memcpy(&G.pv.ninst, a[1], sizeof G.pv.ninst);
                std::memcpy(&G.pv.win_prefix, a[2], sizeof G.pv.win_prefix);
                std::memcpy(&G.pv.total, a[3], sizeof G.pv.total);
                std::memcpy(&G.pv.seqs, a[4], sizeof G.pv.seqs);
                std::memcpy(&G.pv.planes, a[5], sizeof G.pv.planes);
                std::memcpy(&G.pv.flags, a[6], sizeof G.pv.flags);
            } else if (kp.func == sort_unique_kernel_fn()) {
                G.sort = nd;
                G.sort_p = kp;
                void **a = kp.kernelParams;
                std::memcpy(&G.sv.inst, a[0], sizeof G.sv.inst);
                std::memcpy(&G.sv.list, a[1], sizeof G.sv.list);
                std::memcpy(&G.sv.raw, a[2], sizeof G.sv.raw);
                std::memcpy(&G.sv.tmp, a[3], sizeof G.sv.tmp);
                std::memcpy(&G.sv.raw_count, a[4], sizeof G.sv.raw_count);
                std::memcpy(&G.sv.flags, a[5], sizeof G.sv.flags);
                std::memcpy(&G.sv.status, a[6], sizeof G.sv.status);
                std::memcpy(&G.sv.dense, a[7], sizeof G.sv.dense);
                std::memcpy(&G.sv.dense_cap, a[8], sizeof G.sv.dense_cap);
                std::memcpy(&G.sv.dense_total, a[9], sizeof G.sv.dense_total);
            }
        }
        if (!G.pack || !G.sort)
            e = cudaErrorUnknown;
        G.applied_seqs = G.input_rows ? G.rv.seqs : G.pv.seqs;
        G.applied_status = G.sv.status;
        G.applied_dense = G.sv.dense;
        G.applied_cap = G.sv.dense_cap;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_graph(h, G);
        return;
    }
    G.gen = gen;
    G.candidates = P.candidates;
    G.last_use = ++h->use_tick;
    pms_ctx::Graph &S = h->graphs[key];
    S = G;
    // argument pointers into the stored copy
    S.pack_args[0] = &S.pv.inst;
    S.pack_args[1] = &S.pv.ninst;
    S.pack_args[2] = &S.pv.win_prefix;
    S.pack_args[3] = &S.pv.total;
    S.pack_args[4] = &S.pv.seqs;
    S.pack_args[5] = &S.pv.planes;
    S.pack_args[6] = &S.pv.flags;
    S.rows_args[0] = &S.rv.inst;
    S.rows_args[1] = &S.rv.seqs;
    S.rows_args[2] = &S.rv.planes;
    S.rows_args[3] = &S.rv.compat;
    S.rows_args[4] = &S.rv.rowlen;
    S.rows_args[5] = &S.rv.flags;
    S.sort_args[0] = &S.sv.inst;
    S.sort_args[1] = &S.sv.list;
    S.sort_args[2] = &S.sv.raw;
    S.sort_args[3] = &S.sv.tmp;
    S.sort_args[4] = &S.sv.raw_count;
    S.sort_args[5] = &S.sv.flags;
    S.sort_args[6] = &S.sv.status;
    S.sort_args[7] = &S.sv.dense;
    S.sort_args[8] = &S.sv.dense_cap;
    S.sort_args[9] = &S.sv.dense_total;
}

// Enqueues a plan: a plan seen before (one instance or a batch: the same
// options, grid and descriptors) replays the graph captured on its second
// call, with this call's input and output pointers; count-mode solves and
// plans seen once go kernel by kernel.
static int enqueue_plan_graph(pms_ctx *h, const Plan &P, const uint8_t *d_seq_src, StatusDev *status_out,
                              uint64_t *dense_out, uint32_t dense_cap, bool count_mode)
{
    if (h->opt.graph < 0 || count_mode)
        return enqueue_plan(h, P, d_seq_src, status_out, dense_out, dense_cap, count_mode);
    MetaLayout ml(P);
    // key: options, the verification kernel's grid, the descriptors
    std::string key((const char *)&h->opt, sizeof h->opt);
    const int blocks = plan_blocks(h, P, count_mode);
    key.append((const char *)&blocks, sizeof blocks);
    const size_t ko = key.size();
    key.resize(ko + ml.total, '\0');
    fill_meta(P, ml, &key[ko]);
    auto it = h->graphs.find(key);
    if (it != h->graphs.end() && it->second.gen == h->buf_gen) {
        pms_ctx::Graph &G = it->second;
        const bool new_in = d_seq_src != G.applied_seqs;
        const bool new_out = status_out != G.applied_status || dense_out != G.applied_dense ||
                             dense_cap != G.applied_cap;
        G.pv.seqs = d_seq_src;
        G.rv.seqs = d_seq_src;
        G.sv.status = status_out;
        G.sv.dense = dense_out;
        G.sv.dense_cap = dense_cap;
        cudaKernelNodeParams pp = G.pack_p, sp = G.sort_p;
        pp.kernelParams = G.input_rows ? G.rows_args : G.pack_args;
        pp.extra = nullptr;
        sp.kernelParams = G.sort_args;
        sp.extra = nullptr;
        cudaError_t e;
        if ((new_in && (e = cudaGraphExecKernelNodeSetParams(G.x, G.pack, &pp)) != cudaSuccess) ||
            (new_out && (e = cudaGraphExecKernelNodeSetParams(G.x, G.sort, &sp)) != cudaSuccess) ||
            (e = cudaGraphLaunch(G.x, h->stream)) != cudaSuccess)
            return h->cuda_fail(e, "graph launch");
        G.applied_seqs = d_seq_src;
        G.applied_status = status_out;
        G.applied_dense = dense_out;
        G.applied_cap = dense_cap;
        G.last_use = ++h->use_tick;
        ++h->graph_replays;
        h->stats_timed = h->opt.graph >= 1;
        return PMS_OK;
    }
    if (it != h->graphs.end()) {
        cudaStreamSynchronize(h->stream);
        destroy_graph(h, it->second);
        h->graphs.erase(it);
    }
    int rc = enqueue_plan(h, P, d_seq_src, status_out, dense_out, dense_cap, count_mode);
    if (rc)
        return rc;
    // capture on a plan's second call, so that one-off shapes pay no capture
    if (h->seen_plans.size() > 4 * kMaxGraphs)
        h->seen_plans.clear();
    if (!h->seen_plans.insert(key).second) {
        h->seen_plans.erase(key);
        capture_graph(h, key, P, ml, d_seq_src, status_out, dense_out, dense_cap);
    }
    return PMS_OK;
}

// Records what the host knows of the last solve; device times and counters
// are read by collect_stats once its events have completed.
static void begin_stats(pms_ctx *h, const Plan &P, bool count_mode, double t0)
{
    pms_stats s{};
    s.candidates = P.candidates;
    s.ms_total = now_ms() - t0;
    h->stats = s;
    h->stats_pending = true;
    h->stats_count = count_mode;
    h->stats_k = P.inst.size();
}

static void collect_stats(pms_ctx *h)
{
    if (!h->stats_pending)
        return;
    h->stats_pending = false;
    pms_stats &s = h->stats;
    if (!h->stats_timed) {   // a graph replayed without its timing events
        s.ms_kernel = -1.0;
        s.ms_verify = -1.0;
        return;
    }
    if (cudaEventSynchronize(h->ev1) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (h->stats_count) {
        unsigned long long c[kCntNum] = {};
        CtrLayout cl(h->stats_k);
        cudaMemcpy(c, (char *)h->d_ctr.p + cl.work, sizeof c, cudaMemcpyDeviceToHost);
        s.subsets = c[kCntSubsets];
        s.subsets_pruned = c[kCntPruned];
        s.candidates_tested = c[kCntTested];
        s.cmp_rows = c[kCntCmpRows];
        s.cmp_reduce = c[kCntCmpReduce];
        s.cmp_verify = c[kCntCmpVerify];
        s.seeds_infeasible = c[kCntSeedsInfeasible];
    }
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess)
        s.ms_kernel = ms;
    if (cudaEventElapsedTime(&ms, h->evm0, h->evm1) == cudaSuccess)
        s.ms_verify = ms;
    cudaGetLastError();
}

static int status_code(const StatusDev &s)
{
    if (s.flags & kFlagInvalidByte)
        return PMS_EINVAL;
    if (s.flags & kFlagOverflow)
        return PMS_ETOOMANY;
    return PMS_OK;
}

// Runs a plan whose inputs come from host memory and downloads all results
// into h->h_result. On return (PMS_OK) statuses and codes are on the host.
// Most bytes that the kernels of a host-memory solve read from, or write
// to, mapped pinned memory instead of a copy. The packing kernels read each
// input byte several times (once per CTA of a sequence's seed blocks, or once
// per window that covers it), so inputs count with that factor.
constexpr size_t kZeroCopyBytes = (size_t)1 << 20;

static int run_host_plan(pms_ctx *h, const Plan &P, const std::vector<InstSpec> &specs, double t0)
{
    const size_t k = P.inst.size();
    const bool count_mode = h->opt.count_work != 0;
    int rc;
    if ((rc = h->ensure(h->d_seqs, P.seq_bytes)))
        return rc;
    size_t dense_keys = 0;
    for (const InstDev &in : P.inst)
        dense_keys += in.raw_cap;
    ResLayout rl(k, dense_keys);
    if ((rc = h->ensure(h->d_result, rl.total)))
        return rc;
    // Inputs are staged in mapped pinned memory. Small ones are read there by
    // the packing kernel itself and small result blocks are written straight
    // into mapped pinned memory, so such a solve makes no copy calls.
    size_t host_reads = 0;
    for (const InstSpec &s : specs)
        host_reads += (size_t)s.n * s.m * (size_t)std::max(s.l, (s.m - s.l + 1 + 15) / 16);
    const bool zc_in = host_reads <= kZeroCopyBytes, zc_out = rl.total <= kZeroCopyBytes;
    const size_t inline_bytes = rl.dense + (size_t)kInlineKeys * 8;
    if ((rc = h->ensure_host(h->h_in, h->h_in_cap, P.seq_bytes, cudaHostAllocMapped)) ||
        (rc = h->ensure_host(h->h_result, h->h_result_cap, zc_out ? rl.total : inline_bytes, cudaHostAllocMapped)))
        return rc;
    char *stage = (char *)h->h_in;
    for (size_t i = 0; i < k; ++i)
        std::memcpy(stage + P.inst[i].seq_off, specs[i].host_seqs, (size_t)specs[i].n * specs[i].m);
    cudaStream_t st = h->stream;
    if (h->inject(PMS_FAULT_UPLOAD))
        return h->fail(PMS_ECUDA, "upload sequences: failure injected by pms_inject_fault");
    cudaError_t e;
    void *in_dev = nullptr, *res_dev = nullptr;
    if ((e = cudaHostGetDevicePointer(&in_dev, h->h_in, 0)) != cudaSuccess ||
        (e = cudaHostGetDevicePointer(&res_dev, h->h_result, 0)) != cudaSuccess)
        return h->cuda_fail(e, "mapped host buffers");
    if (!zc_in) {
        if ((e = cudaMemcpyAsync(h->d_seqs.p, stage, P.seq_bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return h->cuda_fail(e, "upload sequences");
        in_dev = h->d_seqs.p;
    }
    char *dr = zc_out ? (char *)res_dev : (char *)h->d_result.p;
    if ((rc = enqueue_plan_graph(h, P, (const uint8_t *)in_dev, (StatusDev *)(dr + rl.status),
                                 (uint64_t *)(dr + rl.dense), rl.dense_cap, count_mode)))
        return rc;
    // otherwise statuses and the first codes in one download
    if (!zc_out &&
        (e = cudaMemcpyAsync(h->h_result, dr, std::min(inline_bytes, rl.total), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess)
        return h->cuda_fail(e, "download results");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
        return h->cuda_fail(e, "solve");
    const StatusDev *sd = (const StatusDev *)h->h_result;
    uint64_t total = 0;
    for (size_t i = 0; i < k; ++i)
        total = std::max<uint64_t>(total, (uint64_t)sd[i].dense_off + sd[i].unique_count);
    if (!zc_out && total > kInlineKeys) {
        const size_t need = rl.dense + total * 8;
        if (need > h->h_result_cap) {
            std::vector<char> keep((const char *)h->h_result, (const char *)h->h_result + rl.dense);
            void *np = nullptr;
            if ((e = cudaHostAlloc(&np, round_up(need, 4096), cudaHostAllocMapped)) != cudaSuccess)
                return h->cuda_fail(e, "cudaHostAlloc");
            cudaFreeHost(h->h_result);
            h->h_result = np;
            h->h_result_cap = round_up(need, 4096);
            std::memcpy(h->h_result, keep.data(), keep.size());
        }
        if ((e = cudaMemcpyAsync((char *)h->h_result + rl.dense, dr + rl.dense, total * 8, cudaMemcpyDeviceToHost,
                                 st)) != cudaSuccess)
            return h->cuda_fail(e, "download codes");
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
            return h->cuda_fail(e, "download codes");
    }
    begin_stats(h, P, count_mode, t0);
    collect_stats(h);
    return PMS_OK;
}

struct InstOut {
    int status = PMS_OK;
    uint32_t raw_count = 0;
    std::vector<uint64_t> codes;
};

// Solves instances from host memory; instances whose raw motif buffer
// overflowed are solved again with a larger buffer (unless the caller fixed
// max_motifs), so the returned sets are complete.
static int autotune_missing(pms_ctx *h, const std::vector<InstSpec> &specs);

static int solve_specs(pms_ctx *h, std::vector<InstSpec> specs, std::vector<InstOut> &out, double t0)
{
    if (int rc = autotune_missing(h, specs))
        return rc;
    out.assign(specs.size(), InstOut{});
    std::vector<int> todo(specs.size());
    for (size_t i = 0; i < specs.size(); ++i)
        todo[i] = (int)i;
    uint64_t candidates = 0;
    while (!todo.empty()) {
        std::vector<InstSpec> sub;
        for (int i : todo)
            sub.push_back(specs[i]);
        Plan P = make_plan(h, sub);
        candidates += P.candidates;
        int rc = run_host_plan(h, P, sub, t0);
        if (rc)
            return rc;
        const StatusDev *sd = (const StatusDev *)h->h_result;
        ResLayout rl(sub.size(), 0);
        const uint64_t *dense = (const uint64_t *)((const char *)h->h_result + rl.dense);
        std::vector<int> again;
        for (size_t j = 0; j < sub.size(); ++j) {
            const int idx = todo[j];
            const uint32_t cap = P.inst[j].raw_cap;
            const bool overflow = sd[j].raw_count > cap;
            if (overflow && !(sd[j].flags & kFlagInvalidByte) && !h->opt.max_motifs && cap < (1u << 26)) {
                specs[idx].raw_cap = pow2_at_least(std::max<size_t>((size_t)cap * 8, (size_t)sd[j].raw_count * 2));
                again.push_back(idx);
                continue;
            }
            InstOut &o = out[idx];
            o.status = status_code(sd[j]);
            o.raw_count = sd[j].raw_count;
            o.codes.assign(dense + sd[j].dense_off, dense + sd[j].dense_off + sd[j].unique_count);
        }
        todo.swap(again);
    }
    h->stats.candidates = candidates;
    return PMS_OK;
}

// ----------------------------------------------------------------------------- autotuner

// Tunes the schedule of one instance class by coordinate descent on a
// synthetic instance of that class (uniform random bases), timing the
// device pipeline with CUDA events: first how many rows the node filter
// applies before leaves are expanded, then the work per queue item, then
// the resident CTAs per SM. The best setting is stored for the class.
static int autotune_class(pms_ctx *h, int n, int m, int l, int d, pms_ctx::Tuning &best)
{
    std::vector<uint8_t> seqs((size_t)n * m);
    uint64_t x = 0x9E3779B97F4A7C15ull ^ ((uint64_t)n << 40) ^ ((uint64_t)m << 20) ^ ((uint64_t)l << 8) ^ (uint64_t)d;
    static const uint8_t letters[4] = {'A', 'C', 'G', 'T'};
    for (auto &c : seqs) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        c = letters[(x >> 33) & 3u];
    }
    const auto key = std::make_tuple(l, d, pms_ctx::bucket(n), pms_ctx::bucket(m));
    const pms_options saved = h->opt;
    h->opt.chunk_work = 0;
    h->opt.ctas_per_sm = 0;
    h->opt.count_work = 0;
    h->opt.grab = 0;
    h->opt.partial_rows = 0;
    h->opt.graph = -1;   // every trial timed by its own events, never a graph replay
    std::vector<InstSpec> specs{InstSpec{n, m, l, d, seqs.data()}};
    auto run = [&](const pms_ctx::Tuning &t, double &ms) -> int {
        h->tuned[key] = t;
        double bestms = 1e30;
        for (int rep = 0; rep < 2; ++rep) {
            Plan P = make_plan(h, specs);
            const int rc = run_host_plan(h, P, specs, now_ms());
            if (rc)
                return rc;
            bestms = std::min(bestms, h->stats.ms_kernel);
        }
        ms = bestms;
        return PMS_OK;
    };
    pms_ctx::Tuning cur;
    cur.chunk_work = kDefaultChunkWork;
    cur.prune_rows = n - 1;
    // resident CTAs of the kernel form this class's plans use
    const bool small = h->occ_small[0] > h->occ[0] && expected_seed_rows(n, m, l, d) <= kSmallFormRows;
    const int occ0 = std::max(1, small ? h->occ_small[0] : h->occ[0]);
    cur.ctas_per_sm = occ0;
    cur.partial_rows = default_partial_rows(n, m, l, d);
    cur.grab = kDefaultGrab;
    int rc = run(cur, cur.ms);
    std::vector<int> prune_c = {n - 1, 8, 4, 2, 1};
    std::vector<int> work_c = {1 << 16, 1 << 18, 1 << 20, 1 << 22};
    std::vector<int> cta_c;
    for (int c = occ0; c >= 1 && (int)cta_c.size() < 2; --c)
        cta_c.push_back(c);
    std::vector<int> grab_c = {1, 128, 32};
    std::vector<int> partial_c = {-1, 1, 2, 4};
    for (int dim = 0; dim < 5 && rc == PMS_OK; ++dim) {
        const std::vector<int> &vals =
            dim == 0 ? prune_c : (dim == 1 ? work_c : (dim == 2 ? cta_c : (dim == 3 ? grab_c : partial_c)));
        for (int v : vals) {
            pms_ctx::Tuning t = cur;
            if (dim == 0) {
                if (v > n - 1 || v == cur.prune_rows)
                    continue;
                t.prune_rows = v;
            } else if (dim == 1) {
                if (v == cur.chunk_work)
                    continue;
                t.chunk_work = v;
            } else if (dim == 2) {
                if (v == cur.ctas_per_sm)
                    continue;
                t.ctas_per_sm = v;
            } else if (dim == 3) {
                if (v == cur.grab)
                    continue;
                t.grab = v;
            } else {
                if (v == cur.partial_rows || v > n - 1)
                    continue;
                t.partial_rows = v;
            }
            if ((rc = run(t, t.ms)))
                break;
            if (t.ms < cur.ms)
                cur = t;
        }
    }
    h->opt = saved;
    if (rc) {
        h->tuned.erase(key);
        return rc;
    }
    h->tuned[key] = cur;
    clear_graphs(h);   // tuned launch shapes are not part of a graph's key
    best = cur;
    return PMS_OK;
}

// Tunes every class of `specs` not tuned yet (pms_options.autotune).
static int autotune_missing(pms_ctx *h, const std::vector<InstSpec> &specs)
{
    if (!h->opt.autotune)
        return PMS_OK;
    for (const InstSpec &s : specs) {
        if (h->tuning(s.n, s.m, s.l, s.d))
            continue;
        pms_ctx::Tuning t;
        const int rc = autotune_class(h, s.n, s.m, s.l, s.d, t);
        if (rc)
            return rc;
    }
    return PMS_OK;
}

// ----------------------------------------------------------------------------- served form

// Served form: continuous batching. A scheduler thread admits submitted
// requests while the request pool (a budgeted device block sub-allocated
// first-fit) has room, uploads and packs each on admission, and launches
// verification "waves": one persistent launch of the verification kernel
// whose queue is the union of chunk ranges of every admitted request, oldest
// first, up to a work budget. A request that arrives while waves run joins
// the next wave, so its work overlaps the remaining work of the others. When
// a wave holds a request's last chunks, that request's sort/unique and
// download are enqueued right after the wave; an event per request reports
// completion. No kernel waits on another: all ordering is stream order.

struct Request {
    uint64_t ticket = 0;
    std::vector<uint8_t> seqs;
    int n = 0, m = 0, l = 0, d = 0, W = 0;
    int state = 0;                 // 0 pending, 1 admitted, 2 finishing, 3 done
    int slot = -1;
    size_t arena_off = 0, arena_bytes = 0;
    uint32_t raw_cap = 0;
    size_t dense_rel = 0, status_rel = 0;   // offsets in the arena
    long long chunks_total = 0, chunks_next = 0;
    double units_per_chunk = 1.0;
    cudaEvent_t done_ev = nullptr;
    int status = PMS_OK;
    std::vector<uint64_t> codes;
    size_t count = 0;
};

struct PoolAlloc {
    std::map<size_t, size_t> free_;   // offset -> length
    void reset(size_t s)
    {
        free_.clear();
        if (s)
            free_[0] = s;
    }
    bool alloc(size_t bytes, size_t &off)
    {
        bytes = round_up(bytes, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_.erase(it);
                if (rest)
                    free_[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes, kAlign);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

// A request's arena in the pool (offsets relative to the arena start).
struct ReqLayout {
    size_t seqs, planes, compat, rowlen, raw, tmp, dense, status, ctab, total;
    ReqLayout(int n, int m, int W, uint32_t raw_cap, size_t ctab_ints)
    {
        size_t o = 0;
        auto take = [&](size_t b) {
            const size_t r = o;
            o = round_up(o + b, kAlign);
            return r;
        };
        seqs = take((size_t)n * m);
        planes = take((size_t)n * W * sizeof(uint2));
        compat = take((size_t)W * (n - 1) * ((W + 31) / 32) * sizeof(uint32_t));
        rowlen = take((size_t)W * (n - 1) * sizeof(int));
        raw = take((size_t)raw_cap * 8);
        tmp = take((size_t)raw_cap * 8);   // directly after raw: the sort's twin buffer
        dense = take((size_t)raw_cap * 8);
        status = take(sizeof(StatusDev) + kInlineKeys * 8);
        ctab = take(ctab_ints * sizeof(int));
        total = o;
    }
};

struct Served {
    pms_ctx *h = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::deque<Request *> pending;
    std::vector<Request *> active;                 // admitted, not done (admission order)
    std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
    cudaStream_t st = nullptr;
    int slots = 0;
    std::vector<int> free_slots;
    char *pool = nullptr;
    size_t pool_bytes = 0;
    PoolAlloc palloc;
    InstDev *d_inst = nullptr;       // [slots]
    uint32_t *d_cnt = nullptr;       // raw_count[slots], flags[slots], dense_total[slots], zero[4], ids[slots]
    InstDev *h_inst = nullptr;       // pinned [slots]
    char *h_stage = nullptr;         // pinned [slots]: status block + inline codes of a finishing request
    static constexpr size_t kStage = sizeof(StatusDev) + kInlineKeys * 8;
    int *h_ctab = nullptr;           // pinned [slots][kCtabMax]
    static constexpr int kCtabMax = 8192;
    static constexpr int kRing = 4;
    char *d_ring = nullptr;          // per wave: head + segments
    char *h_ring = nullptr;          // pinned
    size_t ring_stride = 0;
    cudaEvent_t ring_ev[kRing] = {};
    int ring_pos = 0;
    uint32_t *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    long long rows_cap = 0;
    int blocks = 0;
    std::vector<cudaEvent_t> wave_ev;   // in-flight waves
    std::string fatal;
    long long waves = 0, max_reqs_per_wave = 0, overlapped_waves = 0;
};

// d_cnt words: raw_count[slots], flags[slots], dense_total[slots], then an
// 8-word zero block (8-byte aligned; the prefix array of one-instance
// launches), then the slot ids 0..slots-1 (instance lists of the sorts).
static size_t srv_zero_word(int slots) { return round_up(3 * (size_t)slots, 2); }
static size_t srv_cnt_words(int slots) { return srv_zero_word(slots) + 8 + (size_t)slots; }
static uint32_t *srv_rawcnt(Served *S) { return S->d_cnt; }
static uint32_t *srv_flags(Served *S) { return S->d_cnt + S->slots; }
static uint32_t *srv_dense_total(Served *S) { return S->d_cnt + 2 * S->slots; }
static long long *srv_zero(Served *S) { return (long long *)(S->d_cnt + srv_zero_word(S->slots)); }
static int *srv_ids(Served *S) { return (int *)(S->d_cnt + srv_zero_word(S->slots) + 8); }

static void served_loop(Served *S);

static int served_start(pms_ctx *h)
{
    if (h->served)
        return PMS_OK;
    auto S = std::make_unique<Served>();
    S->h = h;
    S->slots = h->opt.serve_max_inflight > 0 ? h->opt.serve_max_inflight : 64;
    size_t pool = (size_t)1 << 30;
    if (h->budget) {
        const size_t left = h->budget > h->used ? h->budget - h->used : 0;
        pool = std::min(pool, left / 2);
    }
    if (pool < ((size_t)1 << 20))
        return h->fail(PMS_ENOMEM, "served form: the memory budget leaves no room for a request pool");
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking)) != cudaSuccess)
        return h->cuda_fail(e, "served stream");
    const size_t cnt_words = srv_cnt_words(S->slots);
    S->pool = (char *)h->dev_alloc(pool);
    S->d_inst = (InstDev *)h->dev_alloc(S->slots * sizeof(InstDev));
    S->d_cnt = (uint32_t *)h->dev_alloc(cnt_words * 4);
    S->ring_stride = round_up(8 + (size_t)S->slots * sizeof(Segment), 256);
    S->d_ring = (char *)h->dev_alloc(S->ring_stride * Served::kRing);
    bool ok = S->pool && S->d_inst && S->d_cnt && S->d_ring;
    if (ok)
        ok = cudaHostAlloc((void **)&S->h_inst, S->slots * sizeof(InstDev), cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&S->h_ctab, (size_t)S->slots * Served::kCtabMax * sizeof(int),
                           cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&S->h_ring, S->ring_stride * Served::kRing, cudaHostAllocDefault) == cudaSuccess &&
             cudaHostAlloc((void **)&S->h_stage, S->slots * Served::kStage, cudaHostAllocDefault) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        h->dev_free(S->pool, pool);
        h->dev_free(S->d_inst, S->slots * sizeof(InstDev));
        h->dev_free(S->d_cnt, cnt_words * 4);
        h->dev_free(S->d_ring, S->ring_stride * Served::kRing);
        if (S->h_inst)
            cudaFreeHost(S->h_inst);
        if (S->h_ctab)
            cudaFreeHost(S->h_ctab);
        if (S->h_ring)
            cudaFreeHost(S->h_ring);
        if (S->h_stage)
            cudaFreeHost(S->h_stage);
        cudaStreamDestroy(S->st);
        return h->fail(PMS_ENOMEM, "served form: device or pinned memory for the request pool is not available");
    }
    S->pool_bytes = pool;
    S->palloc.reset(pool);
    std::vector<uint32_t> init(cnt_words, 0);
    int *ids = (int *)(init.data() + srv_zero_word(S->slots) + 8);
    for (int i = 0; i < S->slots; ++i)
        ids[i] = i;
    cudaMemcpy(S->d_cnt, init.data(), cnt_words * 4, cudaMemcpyHostToDevice);
    for (auto &ev : S->ring_ev)
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    for (int i = S->slots - 1; i >= 0; --i)
        S->free_slots.push_back(i);
    int occ = std::max(1, h->occ[0]);
    if (h->opt.ctas_per_sm > 0)
        occ = std::min(occ, h->opt.ctas_per_sm);
    S->blocks = h->num_sms * occ;
    h->served = S.release();
    h->served->th = std::thread(served_loop, h->served);
    return PMS_OK;
}

static void served_stop(pms_ctx *h)
{
    Served *S = h->served;
    if (!S)
        return;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    S->th.join();
    cudaStreamSynchronize(S->st);
    for (auto &kv : S->all)
        if (kv.second->done_ev)
            cudaEventDestroy(kv.second->done_ev);
    for (auto &ev : S->ring_ev)
        cudaEventDestroy(ev);
    for (auto ev : S->wave_ev)
        cudaEventDestroy(ev);
    const size_t cnt_words = srv_cnt_words(S->slots);
    h->dev_free(S->pool, S->pool_bytes);
    h->dev_free(S->d_inst, S->slots * sizeof(InstDev));
    h->dev_free(S->d_cnt, cnt_words * 4);
    h->dev_free(S->d_ring, S->ring_stride * Served::kRing);
    if (S->d_scratch)
        h->dev_free(S->d_scratch, S->scratch_bytes);
    cudaFreeHost(S->h_inst);
    cudaFreeHost(S->h_ctab);
    cudaFreeHost(S->h_ring);
    cudaFreeHost(S->h_stage);
    cudaStreamDestroy(S->st);
    delete S;
    h->served = nullptr;
}

// Admission: a slot and an arena must be free. Uploads the request, packs
// its windows and builds its compatibility masks (stream order).
static bool served_admit(Served *S, Request *r)
{
    pms_ctx *h = S->h;
    if (S->free_slots.empty())
        return false;
    std::lock_guard<std::recursive_mutex> hg(h->mu);
    const int cw = h->chunk_work_for(r->n, r->m, r->l, r->d);
    const ChunkTable &ct = h->chunks(r->l, r->d, cw > 0 ? cw : kDefaultChunkWork);
    if ((int)ct.tab.size() > Served::kCtabMax) {
        r->status = PMS_EINVAL;
        return true;
    }
    if (h->inject(PMS_FAULT_UPLOAD)) {   // this request's upload fails: it ends with the error
        r->status = PMS_ECUDA;
        return true;
    }
    InstSpec spec{r->n, r->m, r->l, r->d, nullptr};
    r->raw_cap = default_cap(h, spec, true);
    ReqLayout L(r->n, r->m, r->W, r->raw_cap, ct.tab.size());
    if (L.total > S->pool_bytes) {
        r->status = PMS_ENOMEM;   // can never fit
        return true;
    }
    size_t off;
    if (!S->palloc.alloc(L.total, off))
        return false;
    r->slot = S->free_slots.back();
    S->free_slots.pop_back();
    r->arena_off = off;
    r->arena_bytes = L.total;
    r->dense_rel = L.dense;
    r->status_rel = L.status;
    r->chunks_total = (long long)r->W * ct.cps;
    r->chunks_next = 0;
    double units = 0;
    for (int i = 0; i <= r->d; ++i)
        units += (double)binom(r->l, i) * (std::pow(3.0, i) + kNodeUnits);
    r->units_per_chunk = std::max(1.0, units / ct.cps);
    InstDev &in = S->h_inst[r->slot];
    in = InstDev{};
    in.n = r->n;
    in.m = r->m;
    in.l = r->l;
    in.d = r->d;
    in.W = r->W;
    in.NW = (r->W + 31) / 32;
    in.cps = ct.cps;
    in.grab = h->grab_for(r->n, r->m, r->l, r->d);
    in.prune_rows = h->prune_rows_for(r->n, r->m, r->l, r->d);
    in.partial_rows = h->partial_rows_for(r->n, r->m, r->l, r->d);
    in.triple_rows = h->triple_rows_for(r->n, r->m, r->l, r->d);
    in.q = r->n;
    in.nseed = 1;
    in.seq_off = (long long)(off + L.seqs);
    in.plane_off = (long long)((off + L.planes) / sizeof(uint2));
    in.raw_off = (long long)((off + L.raw) / 8);
    in.compat_off = (long long)((off + L.compat) / 4);
    in.rlen_off = (long long)((off + L.rowlen) / 4);
    in.ctab = (int)((off + L.ctab) / sizeof(int));
    in.raw_cap = r->raw_cap;
    int *hc = S->h_ctab + (size_t)r->slot * Served::kCtabMax;
    std::memcpy(hc, ct.tab.data(), ct.tab.size() * sizeof(int));
    cudaStream_t st = S->st;
    cudaMemcpyAsync(S->pool + off + L.seqs, r->seqs.data(), r->seqs.size(), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(S->pool + off + L.ctab, hc, ct.tab.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(S->d_inst + r->slot, &in, sizeof(InstDev), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(srv_rawcnt(S) + r->slot, 0, 4, st);
    cudaMemsetAsync(srv_flags(S) + r->slot, 0, 4, st);
    cudaMemsetAsync(srv_dense_total(S) + r->slot, 0, 4, st);
    const long long windows = (long long)r->n * r->W;
    launch_pack(S->d_inst + r->slot, 1, srv_zero(S), windows, (const uint8_t *)S->pool, (uint2 *)S->pool,
                srv_flags(S) + r->slot, (int)std::max<long long>(1, std::min<long long>((windows + 255) / 256, h->num_sms * 8)),
                st);
    const long long rows = (long long)r->W * (r->n - 1);
    if (rows > 0)
        launch_compat(S->d_inst + r->slot, 1, srv_zero(S), rows, (const uint2 *)S->pool, (uint32_t *)S->pool,
                      (int *)S->pool,
                      (int)std::max<long long>(1, std::min<long long>((rows + 7) / 8, (long long)h->num_sms * 16)), st);
    r->state = 1;
    return true;
}

static void served_fail_all(Served *S, const std::string &why)
{
    S->fatal = why;
    for (Request *r : S->active) {
        r->status = PMS_ECUDA;
        r->state = 3;
    }
    for (Request *r : S->pending) {
        r->status = PMS_ECUDA;
        r->state = 3;
    }
    S->active.clear();
    S->pending.clear();
    S->cv_done.notify_all();
}

static void served_finish(Served *S, Request *r)
{
    const char *stage = S->h_stage + (size_t)r->slot * Served::kStage;
    const StatusDev sd = *(const StatusDev *)stage;
    const uint64_t *inl = (const uint64_t *)(stage + sizeof(StatusDev));
    r->status = status_code(sd);
    const uint32_t u = std::min<uint32_t>(sd.unique_count, r->raw_cap);
    if (u <= kInlineKeys) {
        r->codes.assign(inl, inl + u);
    } else {
        r->codes.resize(u);
        cudaMemcpy(r->codes.data(), S->pool + r->arena_off + r->dense_rel, (size_t)u * 8, cudaMemcpyDeviceToHost);
    }
    r->count = r->status == PMS_ETOOMANY ? sd.raw_count : r->codes.size();
    S->palloc.release(r->arena_off, r->arena_bytes);
    S->free_slots.push_back(r->slot);
    r->slot = -1;
    r->state = 3;
}

static void served_loop(Served *S)
{
    pms_ctx *h = S->h;
    cudaSetDevice(h->device);
    std::unique_lock<std::mutex> lk(S->mu);
    // about 6.4e9 candidate units per wave by default: at (13,4), m ~ 1200 one
    // seed item runs for several milliseconds, so shorter waves spend much of
    // their time in the tail (the mixed Poisson workload at 200 requests/s:
    // p50 88 -> 34 ms, p99 275 -> 142 ms against 8e8)
    const double wave_units = h->opt.serve_wave_items > 0 ? (double)h->opt.serve_wave_items * 65536.0 : 6.4e9;
    while (!S->stop) {
        bool progressed = false;
        // 1. admit in arrival order while a slot and pool room are free
        while (!S->pending.empty()) {
            Request *r = S->pending.front();
            if (!served_admit(S, r))
                break;
            S->pending.pop_front();
            if (r->state == 0) {   // rejected at admission
                r->state = 3;
                S->cv_done.notify_all();
            } else {
                S->active.push_back(r);
            }
            progressed = true;
        }
        // 2. a wave over all admitted requests with chunks left (at most 2 in flight)
        while (!S->wave_ev.empty() && cudaEventQuery(S->wave_ev.front()) == cudaSuccess) {
            cudaEventDestroy(S->wave_ev.front());
            S->wave_ev.erase(S->wave_ev.begin());
        }
        std::vector<Segment> segs;
        std::vector<Request *> finishing;
        if (S->wave_ev.size() < 2) {
            long long items = 0;
            double units = 0;
            long long need_rows = 0;
            for (Request *r : S->active) {
                if (r->state != 1 || r->chunks_next >= r->chunks_total)
                    continue;
                if (units >= wave_units || (int)segs.size() >= S->slots)
                    break;
                long long take = (long long)std::ceil((wave_units - units) / r->units_per_chunk);
                take = std::max<long long>(1, std::min(take, r->chunks_total - r->chunks_next));
                segs.push_back(Segment{items, r->slot, (int)r->chunks_next, (int)(r->chunks_next + take), 0});
                r->chunks_next += take;
                items += take;
                units += take * r->units_per_chunk;
                need_rows = std::max<long long>(need_rows, (long long)round_up((size_t)(r->n - 1) * (r->W + 3), 4));
                if (r->chunks_next >= r->chunks_total)
                    finishing.push_back(r);
            }
            if (!segs.empty()) {
                cudaError_t e = cudaSuccess;
                if (need_rows > S->rows_cap) {
                    std::lock_guard<std::recursive_mutex> hg(h->mu);
                    cudaStreamSynchronize(S->st);
                    if (S->d_scratch)
                        h->dev_free(S->d_scratch, S->scratch_bytes);
                    S->d_scratch = nullptr;
                    S->rows_cap = need_rows;
                    // row scratch for every CTA of a wave; under a tight budget the
                    // waves get fewer CTAs rather than failing
                    while (S->blocks > 0) {
                        S->scratch_bytes = (size_t)S->blocks * 3 * (size_t)S->rows_cap * 4;
                        S->d_scratch = (uint32_t *)h->dev_alloc(S->scratch_bytes);
                        if (S->d_scratch)
                            break;
                        S->blocks /= 2;
                    }
                    if (!S->d_scratch) {
                        served_fail_all(S, "served form: no memory for the row scratch");
                        break;
                    }
                }
                const int rp = S->ring_pos;
                S->ring_pos = (S->ring_pos + 1) % Served::kRing;
                cudaEventSynchronize(S->ring_ev[rp]);
                char *hr = S->h_ring + rp * S->ring_stride;
                char *dr = S->d_ring + rp * S->ring_stride;
                const unsigned long long zero = 0;
                std::memcpy(hr, &zero, 8);
                std::memcpy(hr + 8, segs.data(), segs.size() * sizeof(Segment));
                e = cudaMemcpyAsync(dr, hr, 8 + segs.size() * sizeof(Segment), cudaMemcpyHostToDevice, S->st);
                MainParams mp{};
                mp.inst = S->d_inst;
                mp.seg = (const Segment *)(dr + 8);
                mp.nseg = (int)segs.size();
                mp.total = items;
                mp.head = (unsigned long long *)dr;
                mp.planes = (const uint2 *)S->pool;
                mp.compat = (const uint32_t *)S->pool;
                mp.rowlen = (const int *)S->pool;
                mp.ctab = (const int *)S->pool;
                mp.raw = (uint64_t *)S->pool;
                mp.raw_count = srv_rawcnt(S);
                mp.flags = srv_flags(S);
                mp.scratch = S->d_scratch;
                mp.rows_cap = (int)S->rows_cap;
                mp.smem_rows_cap = h->opt.smem_rows > 0 ? std::min(h->opt.smem_rows, kRowSmemCap) : kRowSmemCap;
                mp.counters = nullptr;
                if (e == cudaSuccess)
                    e = launch_main(mp, (int)std::min<long long>(S->blocks, items), false, S->st);
                cudaEventRecord(S->ring_ev[rp], S->st);
                for (Request *r : finishing) {
                    char *base = S->pool + r->arena_off;
                    char *stage = S->h_stage + (size_t)r->slot * Served::kStage;
                    if (e == cudaSuccess)
                        e = launch_sort_unique(S->d_inst, srv_ids(S) + r->slot, 1, (uint64_t *)S->pool,
                                               (uint64_t *)S->pool + r->raw_cap, srv_rawcnt(S), srv_flags(S),
                                               (StatusDev *)(base + r->status_rel) - r->slot,
                                               (uint64_t *)(base + r->dense_rel), r->raw_cap,
                                               srv_dense_total(S) + r->slot, S->st);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(stage, base + r->status_rel, sizeof(StatusDev), cudaMemcpyDeviceToHost,
                                            S->st);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(stage + sizeof(StatusDev), base + r->dense_rel, kInlineKeys * 8,
                                            cudaMemcpyDeviceToHost, S->st);
                    cudaEventCreateWithFlags(&r->done_ev, cudaEventDisableTiming);
                    cudaEventRecord(r->done_ev, S->st);
                    r->state = 2;
                }
                cudaEvent_t wev;
                cudaEventCreateWithFlags(&wev, cudaEventDisableTiming);
                cudaEventRecord(wev, S->st);
                S->wave_ev.push_back(wev);
                S->waves += 1;
                S->max_reqs_per_wave = std::max<long long>(S->max_reqs_per_wave, (long long)segs.size());
                if (segs.size() > 1)
                    S->overlapped_waves += 1;
                if (e != cudaSuccess) {
                    cudaGetLastError();
                    served_fail_all(S, std::string("served wave: ") + cudaGetErrorString(e));
                    break;
                }
                progressed = true;
            }
        }
        // 3. completions
        bool device_error = false;
        for (size_t i = 0; i < S->active.size();) {
            Request *r = S->active[i];
            cudaError_t q = r->state == 2 ? cudaEventQuery(r->done_ev) : cudaErrorNotReady;
            if (q != cudaSuccess && q != cudaErrorNotReady) {
                device_error = true;
                S->fatal = std::string("served request: ") + cudaGetErrorString(q);
                break;
            }
            if (r->state == 2 && q == cudaSuccess) {
                cudaEventDestroy(r->done_ev);
                r->done_ev = nullptr;
                served_finish(S, r);
                S->active.erase(S->active.begin() + i);
                S->cv_done.notify_all();
                progressed = true;
            } else {
                ++i;
            }
        }
        if (device_error) {
            cudaGetLastError();
            served_fail_all(S, S->fatal);
            continue;
        }
        if (!progressed) {
            if (S->active.empty() && S->pending.empty())
                S->cv_work.wait(lk);
            else
                S->cv_work.wait_for(lk, std::chrono::microseconds(200));
        }
    }
}


// -------------------------------------------------------------------------------- C ABI

extern "C" {

int pms_create(pms_ctx **out, int device, size_t mem_budget_bytes)
{
    if (!out)
        return PMS_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return PMS_ECUDA;
    }
    auto *h = new pms_ctx();
    h->device = device;
    h->budget = mem_budget_bytes;
    cudaError_t e;
    if ((e = cudaSetDevice(device)) != cudaSuccess || (e = init_tables()) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
        (e = main_occupancy(&h->occ[0], false)) != cudaSuccess || (e = main_occupancy(&h->occ[1], true)) != cudaSuccess ||
        (e = main_occupancy(&h->occ_small[0], false, true)) != cudaSuccess ||
        (e = main_occupancy(&h->occ_small[1], true, true)) != cudaSuccess ||
        (e = pairs_occupancy(&h->occ_pair[0], false)) != cudaSuccess ||
        (e = pairs_occupancy(&h->occ_pair[1], true)) != cudaSuccess ||
        (e = cudaEventCreate(&h->ev0)) != cudaSuccess || (e = cudaEventCreate(&h->ev1)) != cudaSuccess ||
        (e = cudaEventCreate(&h->evm0)) != cudaSuccess || (e = cudaEventCreate(&h->evm1)) != cudaSuccess) {
        cudaGetLastError();
        pms_destroy(h);
        return PMS_ECUDA;
    }
    h->stream = h->own_stream;
    *out = h;
    return PMS_OK;
}

int pms_set_stream(pms_ctx *h, void *cuda_stream)
{
    if (!h)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    h->stream = cuda_stream ? (cudaStream_t)cuda_stream : h->own_stream;
    return PMS_OK;
}

int pms_set_allocator(pms_ctx *h, void *(*alloc)(size_t, void *), void (*free_)(void *, void *), void *user)
{
    if (!h || (!alloc) != (!free_))
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    if (h->used)
        return h->fail(PMS_EBUSY, "allocator must be set before the first solve");
    h->ualloc = alloc;
    h->ufree = free_;
    h->uuser = user;
    return PMS_OK;
}

int pms_set_options(pms_ctx *h, const pms_options *opt)
{
    if (!h || !opt)
        return PMS_EINVAL;
    if (opt->ctas_per_sm < 0 || opt->chunk_work < 0 || opt->grab < 0 || opt->serve_wave_items < 0 || opt->smem_rows < 0 ||
        opt->seed_mode < 0 || opt->seed_mode > 1 || opt->quorum < 0 || opt->partial_rows < -1 || opt->graph < -1 || opt->triple_rows < -1 ||
        opt->serve_max_inflight < 0 || opt->serve_max_inflight > 1024)
        return h->fail(PMS_EINVAL, "negative option");
    std::lock_guard<std::recursive_mutex> g(h->mu);
    h->opt = *opt;
    return PMS_OK;
}

int pms_get_options(const pms_ctx *h, pms_options *opt)
{
    if (!h || !opt)
        return PMS_EINVAL;
    *opt = h->opt;
    return PMS_OK;
}

int pms_solve(pms_ctx *h, const uint8_t *seqs, int n, int m, int l, int d, const uint64_t **motifs, size_t *count)
{
    if (!h)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    const double t0 = now_ms();
    h->err.clear();
    if (!seqs || !motifs || !count)
        return h->fail(PMS_EINVAL, "null argument");
    *motifs = nullptr;
    *count = 0;
    int rc;
    if ((rc = check_params(h, n, m, l, d)))
        return rc;
    // The packing kernels flag bytes other than A/C/G/T in the instance's
    // status; only then are the bytes scanned here, to name the first one.
    cudaSetDevice(h->device);
    std::vector<InstSpec> specs{InstSpec{n, m, l, d, seqs}};
    std::vector<InstOut> res;
    if ((rc = solve_specs(h, specs, res, t0)))
        return rc;
    h->owned.resize(1);
    h->owned[0].swap(res[0].codes);
    *motifs = h->owned[0].data();
    *count = h->owned[0].size();
    rc = res[0].status;
    if (rc == PMS_ETOOMANY) {
        *count = res[0].raw_count;
        return h->fail(rc, "%u motifs (with duplicates) exceed the capacity; raise max_motifs", res[0].raw_count);
    }
    if (rc) {
        h->owned[0].clear();
        *motifs = nullptr;
        *count = 0;
        if (rc == PMS_EINVAL && check_bytes(h, seqs, (size_t)n * m))
            return PMS_EINVAL;
        return h->fail(rc, "invalid input byte");
    }
    return PMS_OK;
}

int pms_solve_device(pms_ctx *h, const uint8_t *d_seqs, int n, int m, int l, int d, uint64_t *d_motifs,
                     size_t capacity, uint32_t *d_status)
{
    if (!h)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    const double t0 = now_ms();
    h->err.clear();
    if (!d_seqs || !d_motifs || !d_status || capacity == 0)
        return h->fail(PMS_EINVAL, "null argument or zero capacity");
    int rc;
    if ((rc = check_params(h, n, m, l, d)))
        return rc;
    cudaSetDevice(h->device);
    std::vector<InstSpec> specs{InstSpec{n, m, l, d, nullptr}};
    if ((rc = autotune_missing(h, specs)))
        return rc;
    Plan P = make_plan(h, specs);
    const uint32_t cap = (uint32_t)std::min<size_t>(capacity, 0xffffffffu);
    if ((rc = enqueue_plan_graph(h, P, d_seqs, (StatusDev *)d_status, d_motifs, cap, h->opt.count_work != 0)))
        return rc;
    begin_stats(h, P, h->opt.count_work != 0, t0);
    return PMS_OK;
}

int pms_solve_batch(pms_ctx *h, const pms_instance *inst, int k, pms_result *out)
{
    if (!h)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    const double t0 = now_ms();
    h->err.clear();
    if (!inst || !out || k < 1)
        return h->fail(PMS_EINVAL, "null argument or k < 1");
    std::vector<InstSpec> specs;
    std::vector<int> which;   // index into inst of each valid instance
    for (int i = 0; i < k; ++i) {
        out[i] = pms_result{PMS_OK, nullptr, 0};
        const pms_instance &q = inst[i];
        int rc = q.seqs ? check_params(h, q.n, q.m, q.l, q.d) : h->fail(PMS_EINVAL, "null sequences");
        if (!rc)
            rc = check_bytes(h, q.seqs, (size_t)q.n * q.m);
        if (rc) {
            out[i].status = rc;
            continue;
        }
        specs.push_back(InstSpec{q.n, q.m, q.l, q.d, q.seqs});
        which.push_back(i);
    }
    h->err.clear();
    if (specs.empty())
        return PMS_OK;
    cudaSetDevice(h->device);
    std::vector<InstOut> res;
    int rc;
    if ((rc = solve_specs(h, specs, res, t0)))
        return rc;
    h->owned.assign(specs.size(), {});
    for (size_t j = 0; j < specs.size(); ++j) {
        pms_result &r = out[which[j]];
        h->owned[j].swap(res[j].codes);
        r.status = res[j].status;
        r.motifs = h->owned[j].data();
        r.count = r.status == PMS_ETOOMANY ? res[j].raw_count : h->owned[j].size();
    }
    return PMS_OK;
}

int pms_submit(pms_ctx *h, const pms_instance *inst, uint64_t *ticket)
{
    if (!h)
        return PMS_EINVAL;
    if (!inst || !ticket || !inst->seqs)
        return h->fail(PMS_EINVAL, "null argument");
    {
        std::lock_guard<std::recursive_mutex> g(h->mu);
        int rc = check_params(h, inst->n, inst->m, inst->l, inst->d);
        if (!rc)
            rc = check_bytes(h, inst->seqs, (size_t)inst->n * inst->m);
        if (!rc) {
            cudaSetDevice(h->device);
            rc = served_start(h);
        }
        if (rc)
            return rc;
    }
    Served *S = h->served;
    auto r = std::make_unique<Request>();
    r->seqs.assign(inst->seqs, inst->seqs + (size_t)inst->n * inst->m);
    r->n = inst->n;
    r->m = inst->m;
    r->l = inst->l;
    r->d = inst->d;
    r->W = inst->m - inst->l + 1;
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (!S->fatal.empty())
            return h->fail(PMS_ECUDA, "%s", S->fatal.c_str());
        if (S->pending.size() >= 65536)
            return h->fail(PMS_EBUSY, "served queue full");
        r->ticket = S->next_ticket++;
        *ticket = r->ticket;
        S->pending.push_back(r.get());
        S->all.emplace(r->ticket, std::move(r));
    }
    S->cv_work.notify_all();
    return PMS_OK;
}

int pms_wait(pms_ctx *h, uint64_t ticket, int timeout_ms, pms_result *out)
{
    if (!h || !out)
        return PMS_EINVAL;
    Served *S = h->served;
    if (!S)
        return PMS_ENOTFOUND;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end())
        return PMS_ENOTFOUND;
    Request *r = it->second.get();
    auto done = [&] { return r->state == 3; };
    if (timeout_ms < 0)
        S->cv_done.wait(lk, done);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return PMS_ETIMEDOUT;
    *out = pms_result{r->status, r->codes.data(), r->status == PMS_ETOOMANY ? r->count : r->codes.size()};
    return PMS_OK;
}

int pms_release(pms_ctx *h, uint64_t ticket)
{
    if (!h)
        return PMS_EINVAL;
    Served *S = h->served;
    if (!S)
        return PMS_ENOTFOUND;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end())
        return PMS_ENOTFOUND;
    if (it->second->state != 3)
        return PMS_EBUSY;
    S->all.erase(it);
    return PMS_OK;
}

int pms_cancel(pms_ctx *h, uint64_t ticket)
{
    if (!h)
        return PMS_EINVAL;
    Served *S = h->served;
    if (!S)
        return PMS_ENOTFOUND;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->all.find(ticket);
        if (it == S->all.end())
            return PMS_ENOTFOUND;
        Request *r = it->second.get();
        if (r->state == 3)
            return PMS_OK;   // already finished: its result stands
        auto q = std::find(S->pending.begin(), S->pending.end(), r);
        if (r->state != 0 || q == S->pending.end())
            return PMS_EBUSY;   // on the device
        S->pending.erase(q);
        r->status = PMS_ECANCELED;
        r->state = 3;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
    return PMS_OK;
}

int pms_inject_fault(pms_ctx *h, int kind, int after, int count)
{
    if (!h || kind < PMS_FAULT_ALLOC || kind > PMS_FAULT_UPLOAD || after < 0 || count < 0)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    h->faults[kind] = pms_ctx::Fault{after, count};
    return PMS_OK;
}

int pms_autotune(pms_ctx *h, int n, int m, int l, int d, pms_tuning *out)
{
    if (!h)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    h->err.clear();
    int rc = check_params(h, n, m, l, d);
    if (rc)
        return rc;
    cudaSetDevice(h->device);
    pms_ctx::Tuning t;
    if ((rc = autotune_class(h, n, m, l, d, t)))
        return rc;
    if (out)
        *out = pms_tuning{t.chunk_work, t.prune_rows, t.ctas_per_sm, t.grab, t.partial_rows, t.ms};
    return PMS_OK;
}

int pms_save_tuning(const pms_ctx *h, const char *path)
{
    if (!h || !path)
        return PMS_EINVAL;
    pms_ctx *hm = const_cast<pms_ctx *>(h);
    std::lock_guard<std::recursive_mutex> g(hm->mu);
    FILE *f = std::fopen(path, "w");
    if (!f)
        return hm->fail(PMS_EINVAL, "cannot write %s", path);
    std::fprintf(f, "# l d n_bucket m_bucket chunk_work prune_rows ctas_per_sm grab partial_rows ms\n");
    for (const auto &kv : h->tuned)
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d %.6f\n", std::get<0>(kv.first), std::get<1>(kv.first),
                     std::get<2>(kv.first), std::get<3>(kv.first), kv.second.chunk_work, kv.second.prune_rows,
                     kv.second.ctas_per_sm, kv.second.grab, kv.second.partial_rows, kv.second.ms);
    std::fclose(f);
    return PMS_OK;
}

int pms_load_tuning(pms_ctx *h, const char *path)
{
    if (!h || !path)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    FILE *f = std::fopen(path, "r");
    if (!f)
        return h->fail(PMS_EINVAL, "cannot read %s", path);
    char line[256];
    int loaded = 0;
    while (std::fgets(line, sizeof line, f)) {
        if (line[0] == '#')
            continue;
        int l, d, nb, mb, cw, pr, cta, gr, pp;
        double ms;
        if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %lf", &l, &d, &nb, &mb, &cw, &pr, &cta, &gr, &pp, &ms) != 10)
            continue;
        if (l < 1 || l > PMS_LMAX || d < 0 || d >= l || cw < 0 || pr < 0 || cta < 0 || gr < 0 || pp < -1)
            continue;
        pms_ctx::Tuning t;
        t.chunk_work = cw;
        t.prune_rows = pr;
        t.ctas_per_sm = cta;
        t.grab = gr;
        t.partial_rows = pp;
        t.ms = ms;
        h->tuned[std::make_tuple(l, d, nb, mb)] = t;
        clear_graphs(h);
        ++loaded;
    }
    std::fclose(f);
    return loaded > 0 ? PMS_OK : h->fail(PMS_EINVAL, "no tuning entries in %s", path);
}

int pms_get_stats(const pms_ctx *h, pms_stats *out)
{
    if (!h || !out)
        return PMS_EINVAL;
    pms_ctx *hm = const_cast<pms_ctx *>(h);
    {
        std::lock_guard<std::recursive_mutex> g(hm->mu);
        cudaSetDevice(hm->device);
        collect_stats(hm);
        *out = h->stats;
        out->graph_replays = h->graph_replays;
    }
    // lock order: the scheduler takes its own lock before the context's, so
    // the context lock is never held while taking the scheduler's
    if (Served *S = hm->served) {
        std::lock_guard<std::mutex> sg(S->mu);
        out->serve_waves = (uint64_t)S->waves;
        out->serve_overlapped_waves = (uint64_t)S->overlapped_waves;
        out->serve_max_requests_per_wave = (uint64_t)S->max_reqs_per_wave;
    }
    return PMS_OK;
}

int pms_decode(uint64_t code, int l, char *out)
{
    if (!out || l < 1 || l > PMS_LMAX)
        return PMS_EINVAL;
    static const char letters[4] = {'A', 'C', 'G', 'T'};
    for (int k = l - 1; k >= 0; --k) {
        out[k] = letters[code & 3u];
        code >>= 2;
    }
    out[l] = '\0';
    return PMS_OK;
}

const char *pms_last_error(const pms_ctx *h)
{
    return h ? h->err.c_str() : "null context";
}

int pms_probe_int_rate(pms_ctx *h, int kind, double *per_clk_per_sm)
{
    if (!h || !per_clk_per_sm || kind < 0 || kind > 3)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    cudaSetDevice(h->device);
    const int blocks = h->num_sms;
    const int iters = 4096;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, (blocks + 1) * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return h->fail(PMS_ENOMEM, "probe buffer");
    }
    cudaMemsetAsync(d, 0, (blocks + 1) * sizeof(unsigned long long), h->stream);
    cudaError_t e = launch_probe(kind, iters, blocks, d + 1, d, h->stream);
    std::vector<unsigned long long> cyc(blocks);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cyc.data(), d + 1, blocks * sizeof(unsigned long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(h->stream);
    cudaFree(d);
    if (e != cudaSuccess)
        return h->cuda_fail(e, "probe");
    std::sort(cyc.begin(), cyc.end());
    const double c = (double)cyc[cyc.size() / 2];
    const double ops = 1024.0 * iters * 4 * 8;   // threads x iterations x unroll x chains
    *per_clk_per_sm = ops / std::max(c, 1.0);
    return PMS_OK;
}

int pms_kernel_binary_version(int device, int *version)
{
    if (!version)
        return PMS_EINVAL;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PMS_ECUDA;
    }
    cudaFuncAttributes a{};
    const cudaError_t e = cudaFuncGetAttributes(&a, pack_kernel_fn());
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PMS_ECUDA;
    }
    *version = a.binaryVersion;
    return PMS_OK;
}

// General alphabets (qPMS-Sigma). Host input, one seed per queue item of the
// search kernel; the raw key buffer grows once if the first pass overflows it.
int pms_solve_sigma(pms_ctx *h, const uint8_t *alphabet, int sigma, const uint8_t *seqs, int n, int m, int l, int d,
                    int q, const uint8_t **motifs, size_t *count)
{
    if (!h)
        return PMS_EINVAL;
    std::lock_guard<std::recursive_mutex> g(h->mu);
    const double t0 = now_ms();
    h->err.clear();
    if (!alphabet || !seqs || !motifs || !count)
        return h->fail(PMS_EINVAL, "null argument");
    *motifs = nullptr;
    *count = 0;
    if (sigma < 2 || sigma > 32)
        return h->fail(PMS_EINVAL, "sigma = %d outside [2, 32]", sigma);
    SigmaMap map, letters;
    memset(map.v, 0xFF, sizeof map.v);
    memset(letters.v, 0, sizeof letters.v);
    for (int a = 0; a < sigma; ++a) {
        if (map.v[alphabet[a]] != 0xFF)
            return h->fail(PMS_EINVAL, "letter 0x%02x repeated in the alphabet", alphabet[a]);
        map.v[alphabet[a]] = (uint8_t)a;
        letters.v[a] = alphabet[a];
    }
    int rc;
    if ((rc = check_params(h, n, m, l, d)))
        return rc;
    if (d > kSigMaxD)
        return h->fail(PMS_EINVAL, "d = %d above %d", d, kSigMaxD);
    if (q < 0 || q > n)
        return h->fail(PMS_EINVAL, "q = %d outside [0, n]", q);
    const size_t nm = (size_t)n * m;
    for (size_t i = 0; i < nm; ++i)
        if (map.v[seqs[i]] == 0xFF)
            return h->fail(PMS_EINVAL, "byte %zu (0x%02x) is not a letter of the alphabet", i, seqs[i]);
    cudaSetDevice(h->device);
    cudaError_t e;
    if (!h->sigma_ready) {
        if ((e = sigma_init_tables()) != cudaSuccess || (e = sigma_sort_ctas(&h->sg_sort_ctas)) != cudaSuccess)
            return h->cuda_fail(e, "general-alphabet tables");
        h->sigma_ready = true;
    }
    const int qe = q == 0 ? n : q;
    const int b = sigma_planes(sigma), W = m - l + 1;
    long long nodes = 0;
    for (int k = 0; k <= d; ++k)
        nodes += (long long)binom(l, k);
    const int nseeds = (n - qe + 1) * W;
    // rows a seed is expected to have: the windows of the other sequences
    // within 2d of it, each position differing with probability (sigma-1)/sigma;
    // the larger shared-memory form when the smaller would send seeds to global memory
    const int max_rows = (n - 1) * W;
    double p_row = 0;
    {
        const double pm = (double)(sigma - 1) / sigma;
        for (int j = 0; j <= std::min(2 * d, l); ++j)
            p_row += (double)binom(l, j) * std::pow(pm, j) * std::pow(1.0 - pm, l - j);
    }
    const bool large = p_row * max_rows > 0.8 * sigma_smem_rows(b, l, false);
    int occ = 0;
    if ((e = sigma_main_occupancy(b, l, large, &occ)) != cudaSuccess)
        return h->cuda_fail(e, "occupancy");
    occ = std::max(occ, 1);
    const int per_sm = h->opt.ctas_per_sm > 0 ? std::min(h->opt.ctas_per_sm, occ) : occ;
    int blocks = (int)std::max(1LL, std::min<long long>((long long)h->num_sms * per_sm, nseeds));
    const int smem_rows = sigma_smem_rows(b, l, large);
    const int scratch_rows = (max_rows + 1) & ~1;   // even: packed rows are 8-byte words
    if (max_rows > smem_rows) {
        // every CTA may need global scratch for a seed's rows: keep it within 2 GiB
        // (the persistent CTAs take seeds from a queue, so fewer CTAs only take longer);
        // PMS_SIGMA_SCRATCH_CAP (bytes) lowers that cap, so that tests reach the capped grid
        size_t cap_bytes = (size_t)2 << 30;
        if (const char *env = std::getenv("PMS_SIGMA_SCRATCH_CAP")) {
            const unsigned long long v = std::strtoull(env, nullptr, 10);
            if (v > 0 && v < cap_bytes)
                cap_bytes = (size_t)v;
        }
        const size_t per_cta = (size_t)4 * (1 + b) * scratch_rows;
        blocks = (int)std::max<size_t>(1, std::min<size_t>(blocks, cap_bytes / per_cta));
    }
    const size_t NW = (size_t)n * W;
    // head, raw count, unique count, flags, work counters, the sort's grid barrier (2 words)
    const size_t bar_off = 32 + 8 * (size_t)kSgCntNum, ctr_bytes = bar_off + 8;
    const bool capped = h->opt.max_motifs > 0;
    unsigned long long cap = pow2_at_least(capped ? h->opt.max_motifs : ((size_t)1 << 16));
    constexpr unsigned long long kRetryMax = 1ull << 22;
    if ((rc = h->ensure(h->d_sg_seqs, nm)) || (rc = h->ensure(h->d_sg_planes, (size_t)4 * b * NW)) ||
        (rc = h->ensure(h->d_sg_ctr, ctr_bytes)) ||
        (rc = h->ensure(h->d_sg_hist, 4 * sigma_sort_hist_words(h->sg_sort_ctas))))
        return rc;
    if (max_rows > smem_rows && (rc = h->ensure(h->d_sg_scratch, (size_t)4 * blocks * (1 + b) * scratch_rows)))
        return rc;
    // per warp: the row lists of the search's depths (nodes whose lists would not fit keep the
    // search without them; without room for the buffer within the budget, every node does)
    int list_cap = kSigListCap;
    if (h->ensure(h->d_sg_lists, (size_t)4 * blocks * (kSigThreads / 32) * list_cap) != PMS_OK) {
        list_cap = 0;
        h->err.clear();
    }
    if ((rc = h->ensure_host(h->h_sg, h->h_sg_cap, 256 + nm, cudaHostAllocMapped)))
        return rc;
    char *h_ctr = (char *)h->h_sg;
    memcpy(h_ctr + 256, seqs, nm);
    // inputs of up to 1 MiB are read by the packing kernel in the mapped
    // staging buffer, and outputs of up to 1 MiB written by the sort kernel
    // into a mapped buffer: no copy each way
    void *sg_dev = nullptr, *out_dev = nullptr;
    if ((e = cudaHostGetDevicePointer(&sg_dev, h->h_sg, 0)) != cudaSuccess)
        return h->cuda_fail(e, "mapped host buffers");
    const bool zc_in = nm * (size_t)l <= kZeroCopyBytes;   // every window's l letters
    const uint8_t *seq_src = zc_in ? (const uint8_t *)sg_dev + 256 : (const uint8_t *)h->d_sg_seqs.p;
    bool zc_out = false;
    unsigned long long raw = 0, uniq = 0, ctr[kSgCntNum] = {};
    uint32_t flags = 0, bar[2] = {};
    cudaStream_t st = h->stream;
    for (int attempt = 0;; ++attempt) {
        // raw keys (three words each) and, after them, the sort's second buffer
        if ((rc = h->ensure(h->d_sg_raw, (size_t)48 * cap)) || (rc = h->ensure(h->d_sg_out, (size_t)l * cap)))
            return rc;
        zc_out = (size_t)l * cap <= kZeroCopyBytes;
        if (zc_out) {
            if ((rc = h->ensure_host(h->h_sg_out, h->h_sg_out_cap, (size_t)l * cap, cudaHostAllocMapped)))
                return rc;
            if ((e = cudaHostGetDevicePointer(&out_dev, h->h_sg_out, 0)) != cudaSuccess)
                return h->cuda_fail(e, "mapped host buffers");
        }
        uint8_t *out_ptr = zc_out ? (uint8_t *)out_dev : (uint8_t *)h->d_sg_out.p;
        char *c = (char *)h->d_sg_ctr.p;
        SigmaParams p{};
        p.planes = (const uint32_t *)h->d_sg_planes.p;
        p.n = n;
        p.m = m;
        p.l = l;
        p.d = d;
        p.b = b;
        p.sigma = sigma;
        p.W = W;
        p.miss_max = n - qe;
        p.nseeds = nseeds;
        p.nodes = nodes;
        p.head = (unsigned int *)c;
        p.raw = (unsigned long long *)h->d_sg_raw.p;
        p.raw_count = (unsigned long long *)(c + 8);
        p.raw_cap = cap;
        p.counters = (unsigned long long *)(c + 32);
        p.scratch = max_rows > smem_rows ? (uint32_t *)h->d_sg_scratch.p : nullptr;
        p.scratch_rows = scratch_rows;
        p.smem_rows = smem_rows;
        p.lists = list_cap > 0 ? (uint32_t *)h->d_sg_lists.p : nullptr;
        p.list_cap = list_cap;
        if ((!zc_in &&
             (e = cudaMemcpyAsync(h->d_sg_seqs.p, h_ctr + 256, nm, cudaMemcpyHostToDevice, st)) != cudaSuccess) ||
            (e = cudaMemsetAsync(c, 0, ctr_bytes, st)) != cudaSuccess || (e = cudaEventRecord(h->ev0, st)) != cudaSuccess ||
            (e = launch_sigma_pack(seq_src, n, m, l, b, map, (uint32_t *)h->d_sg_planes.p,
                                   (uint32_t *)(c + 24), st)) != cudaSuccess ||
            (e = cudaEventRecord(h->evm0, st)) != cudaSuccess || (e = launch_sigma_main(p, blocks, st)) != cudaSuccess ||
            (e = cudaEventRecord(h->evm1, st)) != cudaSuccess ||
            (e = launch_sigma_sort_unique(p.raw, p.raw + 3 * cap, p.raw_count, cap, l, b, letters,
                                          out_ptr, (unsigned long long *)(c + 16),
                                          SigSortGrid{(unsigned int *)h->d_sg_hist.p, (unsigned int *)(c + bar_off),
                                                      h->sg_sort_ctas},
                                          st)) != cudaSuccess ||
            (e = cudaEventRecord(h->ev1, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(h_ctr, c, ctr_bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return h->cuda_fail(e, "general-alphabet solve");
        memcpy(&raw, h_ctr + 8, 8);
        memcpy(&uniq, h_ctr + 16, 8);
        memcpy(&flags, h_ctr + 24, 4);
        memcpy(ctr, h_ctr + 32, sizeof ctr);
        memcpy(bar, h_ctr + bar_off, sizeof bar);
        if (bar[1] != 0)
            return h->fail(PMS_ECUDA, "general-alphabet sort: a CTA timed out at a grid barrier");
        if (raw > cap && !capped && attempt == 0 && raw <= kRetryMax) {
            cap = pow2_at_least((size_t)raw);
            continue;
        }
        break;
    }
    if (flags & 1u)
        return h->fail(PMS_EINVAL, "byte outside the alphabet");
    const size_t keep = (size_t)std::min(uniq, cap);
    h->owned_sigma.resize(std::max<size_t>(keep * l, 1));
    if (keep && zc_out)
        memcpy(h->owned_sigma.data(), h->h_sg_out, keep * l);
    else if (keep && ((e = cudaMemcpyAsync(h->owned_sigma.data(), h->d_sg_out.p, keep * l, cudaMemcpyDeviceToHost,
                                           st)) != cudaSuccess ||
                      (e = cudaStreamSynchronize(st)) != cudaSuccess))
        return h->cuda_fail(e, "result copy");
    pms_stats s{};
    double nb = 0;
    for (int k = 0; k <= d; ++k)
        nb += (double)binom(l, k) * std::pow((double)(sigma - 1), k);
    s.candidates = (uint64_t)std::min(nb * nseeds, 1.8e19);
    s.subsets = ctr[kSgNodes];
    s.subsets_pruned = ctr[kSgNodesPruned];
    s.candidates_tested = ctr[kSgLeaves];
    s.cmp_rows = ctr[kSgCmpRows];
    s.cmp_reduce = ctr[kSgCmpReduce];
    s.cmp_verify = ctr[kSgCmpVerify];
    s.seeds_infeasible = ctr[kSgSeedsInfeasible];
    float ms = 0;
    if (cudaEventElapsedTime(&ms, h->ev0, h->ev1) == cudaSuccess)
        s.ms_kernel = ms;
    if (cudaEventElapsedTime(&ms, h->evm0, h->evm1) == cudaSuccess)
        s.ms_verify = ms;
    cudaGetLastError();
    s.ms_total = now_ms() - t0;
    h->stats = s;
    h->stats_pending = false;
    *motifs = h->owned_sigma.data();
    *count = keep;
    if (raw > cap) {
        *count = (size_t)raw;
        return h->fail(PMS_ETOOMANY, "%llu motifs (with duplicates) exceed the capacity; raise max_motifs", raw);
    }
    return PMS_OK;
}

void pms_destroy(pms_ctx *h)
{
    if (!h)
        return;
    cudaSetDevice(h->device);
    served_stop(h);
    if (h->stream)
        cudaStreamSynchronize(h->stream);
    clear_graphs(h);
    if (h->cap_stream)
        cudaStreamDestroy(h->cap_stream);
    pms_ctx::DBuf *bufs[] = {&h->d_seqs, &h->d_planes, &h->d_raw, &h->d_tmp, &h->d_compat, &h->d_rowlen, &h->d_mode, &h->d_meta, &h->d_ctr, &h->d_scratch, &h->d_result,
                             &h->d_sg_seqs, &h->d_sg_planes, &h->d_sg_ctr, &h->d_sg_raw, &h->d_sg_out, &h->d_sg_scratch,
                             &h->d_sg_lists, &h->d_sg_hist};
    for (auto *b : bufs)
        h->dev_free(b->p, b->cap);
    if (h->h_result)
        cudaFreeHost(h->h_result);
    if (h->h_in)
        cudaFreeHost(h->h_in);
    if (h->h_meta)
        cudaFreeHost(h->h_meta);
    if (h->h_sg)
        cudaFreeHost(h->h_sg);
    if (h->h_sg_out)
        cudaFreeHost(h->h_sg_out);
    if (h->ev0)
        cudaEventDestroy(h->ev0);
    if (h->ev1)
        cudaEventDestroy(h->ev1);
    if (h->evm0)
        cudaEventDestroy(h->evm0);
    if (h->evm1)
        cudaEventDestroy(h->evm1);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    delete h;
}

}  // extern "C"

// ------------------------------------------------------------ allocation-free entry point
//
// pms_solve_device_noalloc runs the same pipeline as pms_solve_device for
// callers that are not allowed to allocate device memory: every buffer it
// needs comes from one fixed array in this file, reserved on each GPU when the
// library's device code is loaded there and kept until the process exits.

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)16 << 20;   // the fixed array: 16 MiB per GPU
constexpr uint32_t kNoAllocRawCap = 1u << 16;               // raw motif codes (duplicates included)
constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocMetaInts = 16384;                      // descriptor block: 64 KiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch on this GPU
    int num_sms = 0;
    int occ = 1;
};

std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

// The descriptor block reaches the fixed array as kernel parameters, a piece
// of up to kParamPieceBytes per launch: the bytes are copied into the launch
// when it is enqueued, so no host buffer has to outlive the call (a copy
// from a stack buffer would leave the stream reading freed host memory).
constexpr int kParamPieceBytes = 4000;   // within the classic 4 KiB parameter space

struct ParamPiece {
    unsigned char b[kParamPieceBytes];
};

__global__ void store_piece_kernel(ParamPiece piece, unsigned char *dst, int nbytes)
{
    for (int i = threadIdx.x; i < nbytes; i += blockDim.x)
        dst[i] = piece.b[i];
}

cudaError_t store_bytes(unsigned char *dst, const void *src, size_t nbytes, cudaStream_t st)
{
    const unsigned char *s = static_cast<const unsigned char *>(src);
    for (size_t o = 0; o < nbytes; o += kParamPieceBytes) {
        ParamPiece piece;
        const int k = (int)std::min<size_t>(kParamPieceBytes, nbytes - o);
        std::memcpy(piece.b, s + o, (size_t)k);
        store_piece_kernel<<<1, 256, 0, st>>>(piece, dst + o, k);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// Once per device, with that device current: the array's device address,
// the kernels' constant tables and launch attributes.
int noalloc_setup(int dev, NoAllocDevice **out)
{
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return PMS_EINVAL;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    NoAllocDevice &nd = g_noalloc_dev[dev];
    if (!nd.ready) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return PMS_ECUDA;
        }
        if ((e = init_tables()) != cudaSuccess || (e = main_occupancy(&nd.occ, false)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&nd.num_sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) {
            cudaGetLastError();
            return PMS_ECUDA;
        }
        nd.base = (unsigned char *)ptr;
        nd.occ = std::max(nd.occ, 1);
        nd.ready = true;
    }
    *out = &nd;
    return PMS_OK;
}

// The chunk table of one seed for (l, d), written into a caller array
// (no heap): levoff[0..d+1] then (g0, g1) pairs. Returns the number of ints
// written, or -1 if `cap` is too small. Same cuts as make_chunks.
int chunk_table_into(int l, int d, int work, int *out, int cap, int *cps)
{
    if (d + 2 > cap)
        return -1;
    out[0] = 0;
    for (int i = 0; i <= d; ++i)
        out[i + 1] = out[i] + (int)binom(l, i);
    int n = d + 2, pairs = 0;
    double acc = 0;
    int start = 0, g = 0;
    for (int i = 0; i <= d; ++i) {
        const double w = std::pow(3.0, i) + 24.0;
        long long remaining = (long long)binom(l, i);
        while (remaining > 0) {
            const long long room = (long long)std::ceil(std::max(1.0, (work - acc) / w));
            const long long take = std::min(room, remaining);
            acc += take * w;
            remaining -= take;
            g += (int)take;
            if (acc >= work) {
                if (n + 2 > cap)
                    return -1;
                out[n++] = start;
                out[n++] = g;
                ++pairs;
                start = g;
                acc = 0;
            }
        }
    }
    if (start < g) {
        if (n + 2 > cap)
            return -1;
        out[n++] = start;
        out[n++] = g;
        ++pairs;
    }
    *cps = pairs;
    return n;
}

}  // namespace

extern "C" int pms_solve_device_noalloc(const uint8_t *d_seqs, int n, int m, int l, int d, uint64_t *d_motifs,
                                        size_t capacity, uint32_t *d_status, void *cuda_stream)
{
    if (!d_seqs || !d_motifs || !d_status || capacity == 0)
        return PMS_EINVAL;
    if (n < 1 || n > PMS_NMAX || l < 1 || l > PMS_LMAX || m < l || m > 65536 || d < 0 || d >= l)
        return PMS_EINVAL;
    uint64_t subsets = 0;
    for (int i = 0; i <= d; ++i)
        subsets += binom(l, i);
    if (subsets > (uint64_t)INT32_MAX)
        return PMS_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PMS_ECUDA;
    }
    NoAllocDevice *nd = nullptr;
    int rc = noalloc_setup(dev, &nd);
    if (rc)
        return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // descriptors, built on the stack and enqueued by value (store_bytes)
    struct Meta {
        InstDev inst;
        Segment seg;
        long long win_prefix;
        long long row_prefix;
        int ctab[kNoAllocMetaInts];
    };
    static_assert(sizeof(Meta) <= 80 * 1024, "descriptor block");
    Meta meta;
    std::memset(&meta, 0, offsetof(Meta, ctab));
    int cps = 0;
    const int nct = chunk_table_into(l, d, kDefaultChunkWork, meta.ctab, kNoAllocMetaInts, &cps);
    if (nct < 0)
        return PMS_ESCRATCH;
    InstDev &in = meta.inst;
    in.n = n;
    in.m = m;
    in.l = l;
    in.d = d;
    in.W = m - l + 1;
    in.NW = (in.W + 31) / 32;
    in.cps = cps;
    in.grab = kDefaultGrab;   // the lane-asynchronous node walk, as in the other paths
    in.prune_rows = default_prune_rows(n, d);
    {
        const int pr = default_partial_rows(n, m, l, d);
        in.partial_rows = pr < 0 ? 0 : std::min(pr, n - 1);
    }
    in.q = n;        // the PMS problem
    in.nseed = 1;
    in.ctab = 0;
    in.seq_off = 0;
    in.plane_off = 0;
    in.raw_off = 0;
    in.compat_off = 0;
    in.raw_cap = kNoAllocRawCap;
    const long long items = (long long)in.W * cps;
    meta.seg = Segment{0, 0, 0, (int)items, 0};
    meta.win_prefix = 0;
    meta.row_prefix = 0;
    const size_t meta_bytes = offsetof(Meta, ctab) + (size_t)nct * sizeof(int);

    // carve the fixed array
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = round_up(off + bytes, kAlign);
        return o;
    };
    const size_t o_meta = take(meta_bytes);
    CtrLayout cl(1);
    const size_t o_ctr = take(cl.total);
    const size_t o_planes = take((size_t)n * in.W * sizeof(uint2));
    const size_t o_compat = take((size_t)in.W * (n - 1) * in.NW * sizeof(uint32_t));
    const size_t o_rowlen = take((size_t)in.W * (n - 1) * sizeof(int));
    const size_t o_raw = take((size_t)kNoAllocRawCap * 8);
    const size_t o_tmp = take((size_t)kNoAllocRawCap * 8);
    // a multiple of 4 words keeps every CTA's slice 16-byte aligned (vector loads)
    const long long rows_cap = std::max<long long>(4, (long long)round_up((size_t)(n - 1) * (in.W + 3), 4));
    const size_t per_cta = (size_t)3 * rows_cap * sizeof(uint32_t);
    if (off > kNoAllocScratchBytes || kNoAllocScratchBytes - off < per_cta)
        return PMS_ESCRATCH;
    const long long fit = (long long)((kNoAllocScratchBytes - off) / per_cta);
    const int blocks = (int)std::max<long long>(
        1, std::min<long long>(std::min<long long>((long long)nd->num_sms * nd->occ, items), fit));
    const size_t o_rows = take((size_t)blocks * per_cta);
    unsigned char *base = nd->base;

    cudaError_t e;
    if ((e = store_bytes(base + o_meta, &meta, meta_bytes, st)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + o_ctr, 0, cl.total, st)) != cudaSuccess) {
        cudaGetLastError();
        return PMS_ECUDA;
    }
    const InstDev *d_inst = (const InstDev *)(base + o_meta + offsetof(Meta, inst));
    unsigned char *dc = base + o_ctr;
    uint32_t *d_flags = (uint32_t *)(dc + cl.flags);
    uint32_t *d_rawcnt = (uint32_t *)(dc + cl.raw_count);
    const long long windows = (long long)n * in.W;
    const int pack_blocks = (int)std::max<long long>(1, std::min<long long>((windows + 255) / 256, (long long)nd->num_sms * 8));
    if ((e = launch_pack(d_inst, 1, (const long long *)(base + o_meta + offsetof(Meta, win_prefix)), windows, d_seqs,
                         (uint2 *)(base + o_planes), d_flags, pack_blocks, st)) != cudaSuccess)
        return PMS_ECUDA;
    const long long rows = (long long)in.W * (n - 1);
    if (rows > 0) {
        const int cw_blocks = (int)std::max<long long>(1, std::min<long long>((rows + 7) / 8, (long long)nd->num_sms * 16));
        if ((e = launch_compat(d_inst, 1, (const long long *)(base + o_meta + offsetof(Meta, row_prefix)), rows,
                               (const uint2 *)(base + o_planes), (uint32_t *)(base + o_compat),
                               (int *)(base + o_rowlen), cw_blocks, st)) !=
            cudaSuccess)
            return PMS_ECUDA;
    }
    MainParams mp{};
    mp.inst = d_inst;
    mp.seg = (const Segment *)(base + o_meta + offsetof(Meta, seg));
    mp.nseg = 1;
    mp.total = items;
    mp.head = (unsigned long long *)(dc + cl.head);
    mp.planes = (const uint2 *)(base + o_planes);
    mp.compat = (const uint32_t *)(base + o_compat);
    mp.rowlen = (const int *)(base + o_rowlen);
    mp.ctab = (const int *)(base + o_meta + offsetof(Meta, ctab));
    mp.raw = (uint64_t *)(base + o_raw);
    mp.raw_count = d_rawcnt;
    mp.flags = d_flags;
    mp.scratch = (uint32_t *)(base + o_rows);
    mp.rows_cap = (int)rows_cap;
    mp.smem_rows_cap = kRowSmemCap;
    mp.counters = (unsigned long long *)(dc + cl.work);
    if ((e = launch_main(mp, blocks, false, st)) != cudaSuccess)
        return PMS_ECUDA;
    const uint32_t cap = (uint32_t)std::min<size_t>(capacity, 0xffffffffu);
    if ((e = launch_sort_unique(d_inst, nullptr, 1, (uint64_t *)(base + o_raw), (uint64_t *)(base + o_tmp), d_rawcnt,
                                d_flags, (StatusDev *)d_status, d_motifs, cap, (uint32_t *)(dc + cl.dense_total),
                                st)) != cudaSuccess)
        return PMS_ECUDA;
    return PMS_OK;
}
