// Host build of the general-alphabet node search with the warp's lane-parallel
// form: 32 host threads run sg_node together on every node, exchanging votes,
// broadcasts and sums through barriers (the collectives the GPU warp performs
// with __ballot_sync / __shfl_sync), sharing the per-warp state and witness
// rows as the kernel's shared memory does, and splitting every row scan over
// the 32 lanes. Prints the sorted unique motifs, one per line.
// argv[2], if 1: packed rows where b l <= 64 (the kernel's layout then).
// Input on stdin: "alphabet n m l d q" then the n sequences; argv[1], if
// given: the capacity of the warp's shared row-list buffer (0, the default:
// the depth-first search without row lists).
#include "../../paper_2403_00306_gb300/csrc/pms_sigma.cu"

#include <algorithm>
#include <cstdlib>
#include <array>
#include <barrier>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

using namespace pms;

namespace {

struct Exchange {
    std::barrier<> bar{32};
    uint32_t vote[32];
    unsigned long long val[32];
    std::mutex mu;
};

// The interface of pms::SgWarp, on host threads.
struct LockstepWarp {
    Exchange *x;
    int lane;
    static constexpr int width = 32;
    __host__ __device__ uint32_t ballot(bool p) const
    {
        uint32_t b = 0;
#ifndef __CUDA_ARCH__
        x->vote[lane] = p ? 1u : 0u;
        x->bar.arrive_and_wait();
        for (int i = 0; i < 32; ++i)
            b |= x->vote[i] << i;
        x->bar.arrive_and_wait();
#endif
        return b;
    }
    __host__ __device__ bool any(bool p) const { return ballot(p) != 0; }
    __host__ __device__ unsigned long long sum(unsigned long long v) const
    {
        unsigned long long s = 0;
#ifndef __CUDA_ARCH__
        x->val[lane] = v;
        x->bar.arrive_and_wait();
        for (int i = 0; i < 32; ++i)
            s += x->val[i];
        x->bar.arrive_and_wait();
#endif
        return s;
    }
    __host__ __device__ uint32_t or_all(uint32_t v) const
    {
        uint32_t s = 0;
#ifndef __CUDA_ARCH__
        x->val[lane] = v;
        x->bar.arrive_and_wait();
        for (int i = 0; i < 32; ++i)
            s |= (uint32_t)x->val[i];
        x->bar.arrive_and_wait();
#endif
        return s;
    }
    __host__ __device__ unsigned long long bcast(unsigned long long v) const
    {
        unsigned long long r = v;
#ifndef __CUDA_ARCH__
        if (lane == 0)
            x->val[0] = v;
        x->bar.arrive_and_wait();
        r = x->val[0];
        x->bar.arrive_and_wait();
#endif
        return r;
    }
    __host__ __device__ void sync() const
    {
#ifndef __CUDA_ARCH__
        x->bar.arrive_and_wait();
#endif
    }
    __host__ __device__ void or_into(uint32_t *a, uint32_t v) const
    {
#ifndef __CUDA_ARCH__
        std::lock_guard<std::mutex> g(x->mu);
        *a |= v;
#endif
    }
    __host__ __device__ int rank(uint32_t bal) const { return __builtin_popcount(bal & ((1u << lane) - 1u)); }
    __host__ __device__ int from(int v, int src) const
    {
        int r = v;
#ifndef __CUDA_ARCH__
        x->val[lane] = (unsigned long long)(unsigned)v;
        x->bar.arrive_and_wait();
        r = (int)(unsigned)x->val[src];
        x->bar.arrive_and_wait();
#endif
        return r;
    }
    __host__ __device__ unsigned long long or_all64(unsigned long long v) const
    {
        unsigned long long s = 0;
#ifndef __CUDA_ARCH__
        x->val[lane] = v;
        x->bar.arrive_and_wait();
        for (int i = 0; i < 32; ++i)
            s |= x->val[i];
        x->bar.arrive_and_wait();
#endif
        return s;
    }
};

// One lane reserves (between two barriers of the group), every lane writes its own slots.
struct HostSink {
    std::vector<std::array<unsigned long long, 3>> *v;
    unsigned long long *count;
    std::mutex *mu;
    __host__ __device__ unsigned long long reserve(unsigned long long c)
    {
        unsigned long long b = 0;
#ifndef __CUDA_ARCH__
        std::lock_guard<std::mutex> g(*mu);
        b = *count;
        *count += c;
        v->resize(*count);
#endif
        return b;
    }
    __host__ __device__ unsigned long long room(unsigned long long, unsigned long long c) const { return c; }
    __host__ __device__ void put(unsigned long long s, unsigned long long a, unsigned long long b, unsigned long long c)
    {
#ifndef __CUDA_ARCH__
        std::lock_guard<std::mutex> g(*mu);
        (*v)[s] = {a, b, c};
#endif
    }
};

}  // namespace

int main(int argc, char **argv)
{
    const int list_cap = argc > 1 ? atoi(argv[1]) : 0;
    const bool want_packed = argc > 2 && atoi(argv[2]) != 0;   // packed rows where b and l allow them
    std::vector<uint32_t> list_buf((size_t)std::max(list_cap, 1));   // the warp's, shared by its lanes
    char alpha[64];
    int n, m, l, d, q;
    if (scanf("%63s %d %d %d %d %d", alpha, &n, &m, &l, &d, &q) != 6)
        return 2;
    std::vector<std::string> seqs(n);
    static char buf[70000];
    for (int i = 0; i < n; ++i) {
        if (scanf("%69999s", buf) != 1)
            return 2;
        seqs[i] = buf;
    }
    sigma_init_tables();   // fills the host binomial table; the device copy may fail without a GPU
    cudaGetLastError();
    const int sigma = (int)strlen(alpha), b = sigma_planes(sigma), W = m - l + 1;
    int idx[256];
    for (int c = 0; c < 256; ++c)
        idx[c] = -1;
    for (int a = 0; a < sigma; ++a)
        idx[(unsigned char)alpha[a]] = a;
    const int qe = q == 0 ? n : q;
    std::vector<uint32_t> planes((size_t)b * n * W, 0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < W; ++j)
            for (int k = 0; k < l; ++k) {
                const int a = idx[(unsigned char)seqs[i][j + k]];
                for (int g = 0; g < b; ++g)
                    planes[(size_t)g * n * W + i * W + j] |= ((a >> g) & 1u) << k;
            }
    long long nodes = 0;
    for (int k = 0; k <= d; ++k)
        nodes += sg_binom(l, k);
    std::vector<std::array<unsigned long long, 3>> keys;
    unsigned long long cnt = 0;
    std::mutex sink_mu;
    Exchange ex;
    SgState st;          // the warp's shared state
    int wit[kNMax];      // the warp's witness rows
    for (int seed = 0; seed < (n - qe + 1) * W; ++seed) {
        const int sx = seed / W;
        SgSeed S;
        for (int g = 0; g < kSigMaxPlanes; ++g)
            S.x[g] = g < b ? planes[(size_t)g * n * W + seed] : 0u;
        std::vector<int> off(n + 1);
        std::vector<uint32_t> D;
        std::vector<std::vector<uint32_t>> Pl(b);
        int misses = 0;
        for (int i = 0; i < n; ++i) {
            off[i] = (int)D.size();
            if (i == sx)
                continue;
            const size_t before = D.size();
            for (int j = 0; j < W; ++j) {
                uint32_t mm = 0;
                for (int g = 0; g < b; ++g)
                    mm |= S.x[g] ^ planes[(size_t)g * n * W + i * W + j];
                if (__builtin_popcount(mm) <= 2 * d) {
                    D.push_back(mm);
                    for (int g = 0; g < b; ++g)
                        Pl[g].push_back(planes[(size_t)g * n * W + i * W + j]);
                }
            }
            if (D.size() == before)
                ++misses;
        }
        off[n] = (int)D.size();
        if (misses > n - qe)
            continue;
        const int stride = (std::max<int>(1, (int)D.size()) + 1) & ~1;
        std::vector<uint32_t> rows((size_t)(1 + b) * stride);
        const bool packed = want_packed && sg_packed_rows(b, l);
        for (size_t e = 0; e < D.size(); ++e) {
            rows[e] = D[e];
            if (packed) {
                unsigned long long pk = 0;
                for (int g = 0; g < b; ++g)
                    pk |= (unsigned long long)Pl[g][e] << (g * l);
                std::memcpy(&rows[stride + 2 * e], &pk, sizeof pk);
            } else {
                for (int g = 0; g < b; ++g)
                    rows[(size_t)(1 + g) * stride + e] = Pl[g][e];
            }
        }
        S.D = rows.data();
        S.Pl = rows.data() + stride;
        S.Pk = reinterpret_cast<const unsigned long long *>(rows.data() + stride);
        S.packed = packed;
        S.stride = stride;
        S.off = off.data();
        S.n = n;
        S.l = l;
        S.d = d;
        S.b = b;
        S.miss_max = n - qe;
        S.sx = sx;
        S.full = sigma == 32 ? 0xFFFFFFFFu : (1u << sigma) - 1u;
        std::vector<std::thread> lanes;
        for (int lane = 0; lane < 32; ++lane)
            lanes.emplace_back([&, lane] {
                LockstepWarp grp{&ex, lane};
                HostSink sink{&keys, &cnt, &sink_mu};
                for (long long r = 0; r < nodes; ++r) {
                    SgCount ct{};
                    sg_node(S, grp, sg_unrank(r, l), ct, sink, wit, st,
                            SgLists{list_cap > 0 ? list_buf.data() : nullptr, list_cap});
                    grp.sync();   // the kernel's next node claim is a warp-wide shuffle
                }
            });
        for (auto &t : lanes)
            t.join();
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    for (const auto &k : keys) {
        std::string s(l, '?');
        for (int p = 0; p < l; ++p) {
            const int sh = b * (l - 1 - p);
            int a = 0;
            for (int j = 0; j < b; ++j) {
                const int bit = sh + j;
                a |= (int)((k[2 - (bit >> 6)] >> (bit & 63)) & 1ull) << j;
            }
            s[p] = alpha[a];
        }
        printf("%s\n", s.c_str());
    }
    return 0;
}
