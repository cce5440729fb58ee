// Host-side construction of the decoder's graph store from an edge list.
//
// The paper keeps H as "one file of VNs in order plus one file of the
// VN-to-check mapping, roles swappable" (Results, "High speed error
// correction with MET-LDPC codes").  Here the same information is a
// check-major edge list (the message order) plus a VN-major permutation of
// it, with degree-1 VNs split off because their outgoing message never
// changes (Table 1, "Ignored VNs"; Discussion).
#include <algorithm>
#include <cstring>
#include <numeric>

#include "internal.h"

namespace mld {

static thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

void clear_error() { g_last_error.clear(); }

const char *last_error_text() { return g_last_error.c_str(); }

int build_host_graph(const int32_t *edge_vn, const int32_t *edge_cn,
                     const uint8_t *edge_type, int64_t n_edges, int32_t n_vn,
                     int32_t n_cn, HostGraph *out) {
    if (n_vn < 0 || n_cn < 0 || n_edges < 0)
        return fail(MLD_EINVAL, "graph: negative size");
    if (n_edges > 0 && (!edge_vn || !edge_cn))
        return fail(MLD_EINVAL, "graph: null edge array");
    // 2^30: 32-bit check and edge indices (and strided check loops) never overflow
    if (n_edges > (int64_t{1} << 30))
        return fail(MLD_EGRAPH, "graph: more than 2^30 edges");
    HostGraph &g = *out;
    g = HostGraph();
    g.n_vn = n_vn;
    g.n_cn = n_cn;
    g.n_edges = n_edges;

    std::vector<int32_t> vdeg(n_vn, 0), cdeg(n_cn, 0);
    for (int64_t k = 0; k < n_edges; ++k) {
        const int32_t v = edge_vn[k], c = edge_cn[k];
        if (v < 0 || v >= n_vn || c < 0 || c >= n_cn)
            return fail(MLD_EGRAPH, "graph: edge " + std::to_string(k) + " has an index out of range");
        if (edge_type && edge_type[k] >= MLD_MAX_EDGE_TYPES)
            return fail(MLD_EGRAPH, "graph: edge type out of range at edge " + std::to_string(k));
        vdeg[v]++;
        cdeg[c]++;
    }
    // check-major order of all edges, ties broken by VN -> detects repeats
    std::vector<int32_t> order(n_edges);
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        if (edge_cn[a] != edge_cn[b]) return edge_cn[a] < edge_cn[b];
        return edge_vn[a] < edge_vn[b];
    });
    for (int64_t i = 1; i < n_edges; ++i)
        if (edge_cn[order[i]] == edge_cn[order[i - 1]] && edge_vn[order[i]] == edge_vn[order[i - 1]])
            return fail(MLD_EGRAPH, "graph: repeated (VN, check) pair at edge " + std::to_string(order[i]));

    // internal VN numbering
    std::vector<int32_t> core_id(n_vn, -1);
    for (int32_t v = 0; v < n_vn; ++v)
        if (vdeg[v] != 1) core_id[v] = g.n_core++;
    g.n_deg1 = n_vn - g.n_core;
    g.e_core = static_cast<int32_t>(n_edges - g.n_deg1);
    g.unit.assign(n_vn, -1);
    for (int32_t v = 0; v < n_vn; ++v)
        if (core_id[v] >= 0) g.unit[v] = core_id[v];

    // edges of each caller check in `order`, and its (dc, dd) class key
    std::vector<int64_t> ustart(static_cast<size_t>(n_cn) + 1, 0);
    for (int32_t c = 0; c < n_cn; ++c) ustart[c + 1] = ustart[c] + cdeg[c];
    std::vector<int32_t> dcs(n_cn, 0), dds(n_cn, 0);
    for (int64_t k = 0; k < n_edges; ++k) {
        if (core_id[edge_vn[k]] >= 0) dcs[edge_cn[k]]++;
        else dds[edge_cn[k]]++;
    }
    auto key = [&](int32_t c) -> int64_t {
        return (dcs[c] + dds[c] <= kMaxRegDeg) ? static_cast<int64_t>(dcs[c]) * 64 + dds[c] : (1LL << 40);
    };
    g.cuser.resize(n_cn);
    std::iota(g.cuser.begin(), g.cuser.end(), 0);
    std::stable_sort(g.cuser.begin(), g.cuser.end(), [&](int32_t a, int32_t b) { return key(a) < key(b); });

    g.cptr.assign(static_cast<size_t>(n_cn) + 1, 0);
    g.dptr.assign(static_cast<size_t>(n_cn) + 1, 0);
    g.col.resize(g.e_core);
    g.etype_core.resize(g.e_core);
    g.etype_deg1.resize(g.n_deg1);
    int32_t ce = 0, slot = 0;
    for (int32_t ci = 0; ci < n_cn; ++ci) {
        const int32_t c = g.cuser[ci];
        g.cptr[ci] = ce;
        g.dptr[ci] = slot;
        for (int64_t i = ustart[c]; i < ustart[c + 1]; ++i) {
            const int32_t k = order[i];
            const int32_t v = edge_vn[k];
            const uint8_t t = edge_type ? edge_type[k] : 0;
            if (core_id[v] >= 0) {
                g.col[ce] = core_id[v];
                g.etype_core[ce] = t;
                ++ce;
            } else {
                g.unit[v] = g.n_core + slot;
                g.etype_deg1[slot] = t;
                ++slot;
            }
        }
        g.max_check_deg = std::max(g.max_check_deg, cdeg[c]);
        // open a new class when the key changes
        const bool regular = dcs[c] + dds[c] <= kMaxRegDeg;
        if (g.classes.empty() || key(c) != key(g.cuser[g.classes.back().c0])) {
            CheckClass cl;
            cl.c0 = ci;
            cl.count = 0;
            cl.dc = regular ? dcs[c] : -1;
            cl.dd = regular ? dds[c] : -1;
            cl.e0 = g.cptr[ci];
            cl.s0 = g.dptr[ci];
            g.classes.push_back(cl);
        }
        g.classes.back().count++;
    }
    g.cptr[n_cn] = ce;
    g.dptr[n_cn] = slot;
    // (core edges of a check are ascending in core id: `order` is ascending in
    // VN and core ids preserve the natural order)

    // VN-major view of the core edges
    g.vptr.assign(static_cast<size_t>(g.n_core) + 1, 0);
    for (int32_t e = 0; e < g.e_core; ++e) g.vptr[g.col[e] + 1]++;
    for (int32_t v = 0; v < g.n_core; ++v) g.vptr[v + 1] += g.vptr[v];
    g.vedge.resize(g.e_core);
    std::vector<int32_t> fill(g.vptr.begin(), g.vptr.end() - 1);
    for (int32_t e = 0; e < g.e_core; ++e) g.vedge[fill[g.col[e]]++] = e;
    for (int32_t v = 0; v < n_vn; ++v) g.max_vn_deg = std::max(g.max_vn_deg, vdeg[v]);
    return MLD_OK;
}

int build_layers(const HostGraph &h, const int32_t *layer_of_check, int32_t n_layers, LayerTables *out) {
    const int32_t m = h.n_cn;
    // class of every internal check
    std::vector<int32_t> cls_of(m, 0);
    for (size_t k = 0; k < h.classes.size(); ++k)
        for (int32_t i = 0; i < h.classes[k].count; ++i) cls_of[h.classes[k].c0 + i] = static_cast<int32_t>(k);
    std::vector<int32_t> lay(m, 0);  // layer of internal check
    int32_t nl = 0;
    if (layer_of_check) {
        if (n_layers < 1 && m > 0) return fail(MLD_EINVAL, "layers: n_layers < 1");
        for (int32_t ci = 0; ci < m; ++ci) {
            const int32_t L = layer_of_check[h.cuser[ci]];
            if (L < 0 || L >= n_layers)
                return fail(MLD_EINVAL, "layers: layer of check " + std::to_string(h.cuser[ci]) + " out of range");
            lay[ci] = L;
        }
        nl = n_layers;
    } else {
        // first fit per class, in the class's check order; layers numbered
        // class after class
        // first fit needs at most (checks sharing a VN with the check) + 1 layers
        const int32_t maxc = std::max<int32_t>(1, h.max_vn_deg) * std::max<int32_t>(1, h.max_check_deg) + 1;
        const int32_t words = (maxc + 63) / 64;
        std::vector<uint64_t> used;
        for (const CheckClass &cl : h.classes) {
            if (cl.dc == 0 && cl.dd == 0) {
                for (int32_t i = 0; i < cl.count; ++i) lay[cl.c0 + i] = nl;
                continue;
            }
            used.assign(static_cast<size_t>(h.n_core) * words, 0ull);
            int32_t top = 0;
            for (int32_t i = 0; i < cl.count; ++i) {
                const int32_t ci = cl.c0 + i;
                int32_t L = 0;
                for (;; ++L) {
                    bool free = true;
                    for (int32_t e = h.cptr[ci]; e < h.cptr[ci + 1] && free; ++e)
                        if ((used[static_cast<size_t>(h.col[e]) * words + L / 64] >> (L % 64)) & 1ull) free = false;
                    if (free) break;
                }
                for (int32_t e = h.cptr[ci]; e < h.cptr[ci + 1]; ++e)
                    used[static_cast<size_t>(h.col[e]) * words + L / 64] |= 1ull << (L % 64);
                lay[ci] = nl + L;
                top = std::max(top, L + 1);
            }
            nl += top;
        }
    }
    // internal checks ordered by (layer, class, position)
    std::vector<int32_t> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
        if (lay[a] != lay[b]) return lay[a] < lay[b];
        return cls_of[a] < cls_of[b];
    });
    // no core VN twice in a layer
    std::vector<int32_t> stamp(h.n_core, -1);
    for (int32_t ci : ord)
        for (int32_t e = h.cptr[ci]; e < h.cptr[ci + 1]; ++e) {
            if (stamp[h.col[e]] == lay[ci])
                return fail(MLD_EGRAPH, "layers: two checks of layer " + std::to_string(lay[ci]) +
                                            " share a VN of degree >= 2 (check " + std::to_string(h.cuser[ci]) + ")");
            stamp[h.col[e]] = lay[ci];
        }
    LayerTables t;
    t.lchk.reserve(m);
    t.leptr.reserve(static_cast<size_t>(m) + 1);
    t.lcol.reserve(h.e_core);
    for (int32_t i = 0; i < m; ++i) {
        const int32_t ci = ord[i];
        const CheckClass &cl = h.classes[cls_of[ci]];
        if (cl.dc == 0 && cl.dd == 0) continue;  // nothing to send
        const int32_t p = static_cast<int32_t>(t.lchk.size());
        const int32_t e = static_cast<int32_t>(t.lcol.size());
        if (t.launches.empty() || t.launches.back().layer != lay[ci] || t.launches.back().cls != cls_of[ci])
            t.launches.push_back(LayerLaunch{lay[ci], cls_of[ci], p, 0, e});
        t.launches.back().count++;
        t.lchk.push_back(ci);
        t.leptr.push_back(e);
        for (int32_t k = h.cptr[ci]; k < h.cptr[ci + 1]; ++k) t.lcol.push_back(h.col[k]);
    }
    t.leptr.push_back(static_cast<int32_t>(t.lcol.size()));
    t.layer_user.assign(m, 0);
    for (int32_t ci = 0; ci < m; ++ci) t.layer_user[h.cuser[ci]] = lay[ci];
    t.n_layers = nl;
    *out = std::move(t);
    return MLD_OK;
}

}  // namespace mld
