// Seeded multi-edge-type (MET) LDPC ensemble on the host: the synthetic code
// family the decoder is benchmarked on (the paper's PEG-built MET codes,
// Results "GPU-based error correction speed" and Table 1, are not available;
// this family has their shape).
//
//  * n_c = round(core_frac n) core VNs.  The first round(0.4 n_c) have 2
//    type-1 edges, the rest 3, to m1 = n_c - round(R n) type-1 checks; each
//    has d2 type-2 edges to the m2 = n - n_c type-2 checks.
//  * m2 degree-1 VNs; degree-1 VN n_c + j attaches to type-2 check j (the
//    "ignored" VNs of Table 1).
//  * Each edge type's check sockets are dealt as evenly as possible (floor or
//    ceil of the mean per check), shuffled, and paired with the VN sockets in
//    order; a repeated (VN, check) pair is re-paired by swapping its check
//    socket with a uniformly drawn socket of the same type until none is left.
//  * VN and check labels are finally shuffled, and the edges sorted by
//    (check, VN).
//
// Random numbers: xoshiro256** (Blackman and Vigna) seeded through splitmix64
// from (seed, n, d2); bounded integers by Lemire's multiply-and-reject
// method; shuffles by Fisher-Yates.  The same arguments give the same graph on
// every machine.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

namespace {

uint64_t splitmix64(uint64_t &x) {
    x += 0x9E3779B97F4A7C15ull;
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

struct Rng {
    uint64_t s[4];
    Rng(uint64_t seed, uint64_t a, uint64_t b) {
        uint64_t x = seed;
        x ^= splitmix64(a);
        x ^= rotl(splitmix64(b), 17);
        for (uint64_t &w : s) w = splitmix64(x);
    }
    uint64_t next() {
        const uint64_t r = rotl(s[1] * 5, 7) * 9;
        const uint64_t t = s[1] << 17;
        s[2] ^= s[0];
        s[3] ^= s[1];
        s[1] ^= s[2];
        s[0] ^= s[3];
        s[2] ^= t;
        s[3] = rotl(s[3], 45);
        return r;
    }
    // uniform in [0, bound), bound >= 1, without modulo bias
    uint64_t below(uint64_t bound) {
        unsigned __int128 m = static_cast<unsigned __int128>(next()) * bound;
        uint64_t lo = static_cast<uint64_t>(m);
        if (lo < bound) {
            const uint64_t thr = (0 - bound) % bound;
            while (lo < thr) {
                m = static_cast<unsigned __int128>(next()) * bound;
                lo = static_cast<uint64_t>(m);
            }
        }
        return static_cast<uint64_t>(m >> 64);
    }
    template <typename T>
    void shuffle(std::vector<T> &v) {
        for (size_t i = v.size(); i > 1; --i) std::swap(v[i - 1], v[static_cast<size_t>(below(i))]);
    }
};

struct Shape {
    int64_t n_c, m1, m2, n_two, e1, e2, e3;
};

int shape_of(double rate, int32_t n, int32_t d2, double core_frac, Shape *sh) {
    if (!(rate > 0.0 && rate < 1.0) || !(core_frac > 0.0 && core_frac < 1.0) || n < 2 || d2 < 1)
        return mld::fail(MLD_EINVAL, "ensemble: need 0 < rate < 1, 0 < core_frac < 1, n >= 2, d2 >= 1");
    sh->n_c = std::llround(core_frac * n);
    sh->m2 = n - sh->n_c;
    sh->m1 = sh->n_c - std::llround(rate * n);
    if (sh->n_c < 1 || sh->m1 < 1 || sh->m2 < 1)
        return mld::fail(MLD_EINVAL, "ensemble: degenerate sizes (core VNs, type-1 or type-2 checks < 1)");
    sh->n_two = std::llround(0.4 * static_cast<double>(sh->n_c));
    sh->e1 = 2 * sh->n_two + 3 * (sh->n_c - sh->n_two);
    sh->e2 = sh->n_c * static_cast<int64_t>(d2);
    sh->e3 = sh->m2;
    if (sh->e1 + sh->e2 + sh->e3 > (int64_t{1} << 30)) return mld::fail(MLD_EINVAL, "ensemble: more than 2^30 edges");
    return MLD_OK;
}

// check label per socket: each of m checks gets floor or ceil of e/m sockets
std::vector<int32_t> deal(int64_t e, int64_t m) {
    std::vector<int32_t> c(static_cast<size_t>(e));
    const int64_t base = e / m, extra = e % m;
    size_t k = 0;
    for (int64_t j = 0; j < m; ++j) {
        const int64_t cnt = base + (j < extra ? 1 : 0);
        for (int64_t t = 0; t < cnt; ++t) c[k++] = static_cast<int32_t>(j);
    }
    return c;
}

// swap check sockets until no (v, c) pair repeats; false if it does not settle
bool repair(const std::vector<int32_t> &v, std::vector<int32_t> &c, int64_t m, Rng &rng) {
    const size_t e = v.size();
    std::vector<int64_t> key(e);
    std::vector<size_t> order(e);
    for (int round = 0; round < 10000; ++round) {
        for (size_t i = 0; i < e; ++i) key[i] = static_cast<int64_t>(v[i]) * m + c[i];
        std::iota(order.begin(), order.end(), size_t{0});
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return key[a] < key[b]; });
        std::vector<size_t> dup;
        for (size_t i = 1; i < e; ++i)
            if (key[order[i]] == key[order[i - 1]]) dup.push_back(order[i]);
        if (dup.empty()) return true;
        std::sort(dup.begin(), dup.end());
        for (size_t i : dup) std::swap(c[i], c[static_cast<size_t>(rng.below(e))]);
    }
    return false;
}

}  // namespace

extern "C" int mld_ensemble_size(double rate, int32_t n, int32_t d2, double core_frac, int64_t *n_edges,
                                 int32_t *n_cn) {
    mld::clear_error();
    Shape sh;
    const int s = shape_of(rate, n, d2, core_frac, &sh);
    if (s != MLD_OK) return s;
    if (n_edges) *n_edges = sh.e1 + sh.e2 + sh.e3;
    if (n_cn) *n_cn = static_cast<int32_t>(sh.m1 + sh.m2);
    return MLD_OK;
}

extern "C" int mld_ensemble_edges(double rate, int32_t n, int32_t d2, double core_frac, uint64_t seed,
                                  int32_t *edge_vn, int32_t *edge_cn, uint8_t *edge_type, int64_t capacity) {
    mld::clear_error();
    Shape sh;
    int s = shape_of(rate, n, d2, core_frac, &sh);
    if (s != MLD_OK) return s;
    const int64_t e_total = sh.e1 + sh.e2 + sh.e3;
    if (!edge_vn || !edge_cn) return mld::fail(MLD_EINVAL, "ensemble_edges: null output");
    if (capacity < e_total) return mld::fail(MLD_EINVAL, "ensemble_edges: capacity below mld_ensemble_size");
    Rng rng(seed, static_cast<uint64_t>(n), static_cast<uint64_t>(d2));

    // type-1 edges: 2 sockets for the first n_two core VNs, 3 for the rest
    std::vector<int32_t> v1;
    v1.reserve(static_cast<size_t>(sh.e1));
    for (int64_t v = 0; v < sh.n_c; ++v)
        for (int t = 0; t < (v < sh.n_two ? 2 : 3); ++t) v1.push_back(static_cast<int32_t>(v));
    std::vector<int32_t> c1 = deal(sh.e1, sh.m1);
    rng.shuffle(c1);
    if (!repair(v1, c1, sh.m1, rng)) return mld::fail(MLD_EGRAPH, "ensemble: type-1 re-pairing did not settle");
    // type-2 edges of core VNs
    std::vector<int32_t> v2;
    v2.reserve(static_cast<size_t>(sh.e2));
    for (int64_t v = 0; v < sh.n_c; ++v)
        for (int32_t t = 0; t < d2; ++t) v2.push_back(static_cast<int32_t>(v));
    std::vector<int32_t> c2 = deal(sh.e2, sh.m2);
    rng.shuffle(c2);
    if (!repair(v2, c2, sh.m2, rng)) return mld::fail(MLD_EGRAPH, "ensemble: type-2 re-pairing did not settle");

    // relabelling of VNs and checks
    const int64_t m = sh.m1 + sh.m2;
    std::vector<int32_t> vlab(static_cast<size_t>(n)), clab(static_cast<size_t>(m));
    std::iota(vlab.begin(), vlab.end(), 0);
    std::iota(clab.begin(), clab.end(), 0);
    rng.shuffle(vlab);
    rng.shuffle(clab);

    struct E { int32_t c, v; uint8_t t; };
    std::vector<E> edges;
    edges.reserve(static_cast<size_t>(e_total));
    for (size_t i = 0; i < v1.size(); ++i) edges.push_back({clab[c1[i]], vlab[v1[i]], 0});
    for (size_t i = 0; i < v2.size(); ++i) edges.push_back({clab[sh.m1 + c2[i]], vlab[v2[i]], 1});
    for (int64_t j = 0; j < sh.m2; ++j)
        edges.push_back({clab[sh.m1 + j], vlab[sh.n_c + j], 2});
    std::sort(edges.begin(), edges.end(), [](const E &a, const E &b) { return a.c != b.c ? a.c < b.c : a.v < b.v; });
    for (size_t i = 0; i < edges.size(); ++i) {
        edge_vn[i] = edges[i].v;
        edge_cn[i] = edges[i].c;
        if (edge_type) edge_type[i] = edges[i].t;
    }
    return MLD_OK;
}

extern "C" int mld_graph_generate(double rate, int32_t n, int32_t d2, uint64_t seed, mld_graph **out) {
    mld::clear_error();
    if (!out) return mld::fail(MLD_EINVAL, "graph_generate: null output");
    double core_frac;
    if (rate == 0.1) core_frac = 0.20;
    else if (rate == 0.05) core_frac = 0.12;
    else if (rate == 0.02) core_frac = 0.06;
    else return mld::fail(MLD_EINVAL, "graph_generate: rate must be 0.1, 0.05 or 0.02 (mld_ensemble_edges takes any)");
    int64_t e = 0;
    int32_t m = 0;
    int s = mld_ensemble_size(rate, n, d2, core_frac, &e, &m);
    if (s != MLD_OK) return s;
    std::vector<int32_t> ev(static_cast<size_t>(e)), ec(static_cast<size_t>(e));
    std::vector<uint8_t> et(static_cast<size_t>(e));
    s = mld_ensemble_edges(rate, n, d2, core_frac, seed, ev.data(), ec.data(), et.data(), e);
    if (s != MLD_OK) return s;
    return mld_graph_create(ev.data(), ec.data(), et.data(), e, n, m, out);
}
