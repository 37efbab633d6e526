// Host build of the general-alphabet node search (the same sg_node / sg_unrank
// code the search kernel runs, with a one-thread group) for the CPU tests:
// rows are built on the host in the kernel's layout, every node of every seed
// is searched, and the sorted unique motifs are printed, one per line.
// Input on stdin: "alphabet n m l d q" then the n sequences; or "unrank l d",
// which prints the position subset (as a bit mask) of every node rank instead.
// argv[1], if given: the capacity of the group's row-list buffer (0, the
// default: the depth-first search without row lists); argv[2], if 1: rows
// with their planes packed in one 64-bit word where b l <= 64 (the kernel's
// layout then), else one word per plane.
#include "../../paper_2403_00306_gb300/csrc/pms_sigma.cu"

#include <algorithm>
#include <cstdlib>
#include <array>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace pms;

namespace {

struct HostSink {
    std::vector<std::array<unsigned long long, 3>> *v;
    unsigned long long *count;
    __host__ __device__ unsigned long long reserve(unsigned long long c)
    {
        const unsigned long long b = *count;
        *count += c;
#ifndef __CUDA_ARCH__
        v->resize(*count);
#endif
        return b;
    }
    __host__ __device__ unsigned long long room(unsigned long long, unsigned long long c) const { return c; }
    __host__ __device__ void put(unsigned long long s, unsigned long long a, unsigned long long b, unsigned long long c)
    {
#ifndef __CUDA_ARCH__
        (*v)[s] = {a, b, c};
#endif
    }
};

}  // namespace

int main(int argc, char **argv)
{
    const int list_cap = argc > 1 ? atoi(argv[1]) : 0;
    const bool want_packed = argc > 2 && atoi(argv[2]) != 0;   // packed rows where b and l allow them
    std::vector<uint32_t> list_buf((size_t)std::max(list_cap, 1));
    char alpha[64];
    int n, m, l, d, q;
    if (scanf("%63s", alpha) != 1)
        return 2;
    if (strcmp(alpha, "unrank") == 0) {
        if (scanf("%d %d", &l, &d) != 2)
            return 2;
        sigma_init_tables();
        cudaGetLastError();
        long long nodes = 0;
        for (int k = 0; k <= d; ++k)
            nodes += sg_binom(l, k);
        for (long long r = 0; r < nodes; ++r)
            printf("%u\n", sg_unrank(r, l));
        return 0;
    }
    if (scanf("%d %d %d %d %d", &n, &m, &l, &d, &q) != 5)
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
    HostSink sink{&keys, &cnt};
    SgSingle one;
    int wit[kNMax];
    SgState st;
    unsigned long long tot_nodes = 0, tot_pruned = 0;
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
            for (int j = W - 1; j >= 0; --j) {   // another row order than the kernel's
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
        for (long long r = 0; r < nodes; ++r) {
            SgCount ct{};
            sg_node(S, one, sg_unrank(r, l), ct, sink, wit, st,
                    SgLists{list_cap > 0 ? list_buf.data() : nullptr, list_cap});
            tot_nodes += ct.nodes;
            tot_pruned += ct.pruned;
        }
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    fprintf(stderr, "nodes %llu pruned %llu raw %llu\n", tot_nodes, tot_pruned, cnt);
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
