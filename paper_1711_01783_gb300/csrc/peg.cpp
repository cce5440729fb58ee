// Progressive edge growth (PEG) for multi-edge-type Tanner graphs, on the
// host.  The paper's codes are built this way from multi-edge-type degree
// distributions (Results, "GPU-based error correction speed"; Table 1); the
// library offers it so that codes of any distribution can be decoded.
//
// VNs are connected in order of increasing total degree (ties by index),
// each VN's edges type by type.  An edge of type t from VN v goes to a check
// that accepts t and is not yet a neighbour of v, among the farthest from v
// in the graph built so far: unreachable ones if any, else those at the
// largest breadth-first level (v's neighbours are level 1).  Among those the
// lowest current degree wins, then the lowest priority.  The search from v
// stops as soon as every check accepting t has been reached, since deeper
// levels cannot change the choice.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

namespace {

struct Key {
    int32_t deg, prio, c;
    bool operator<(const Key &o) const { return std::tie(deg, prio, c) < std::tie(o.deg, o.prio, o.c); }
};

}  // namespace

extern "C" int mld_peg_edges(int32_t n_vn, int32_t n_types, const int32_t *deg, int32_t n_cn,
                             const uint32_t *mask, const int32_t *prio, int64_t capacity, int32_t *edge_vn,
                             int32_t *edge_cn, uint8_t *edge_type, int64_t *n_edges) {
    mld::clear_error();
    if (n_vn < 0 || n_cn < 0 || n_types < 1 || n_types > MLD_MAX_EDGE_TYPES || !n_edges ||
        (n_vn > 0 && !deg) || (n_cn > 0 && !mask))
        return mld::fail(MLD_EINVAL, "peg: bad arguments");
    int64_t total = 0;
    std::vector<int64_t> vdeg(n_vn, 0);
    for (int32_t t = 0; t < n_types; ++t)
        for (int32_t v = 0; v < n_vn; ++v) {
            const int32_t d = deg[static_cast<int64_t>(t) * n_vn + v];
            if (d < 0) return mld::fail(MLD_EINVAL, "peg: negative degree");
            vdeg[v] += d;
            total += d;
        }
    if (total > (int64_t{1} << 30)) return mld::fail(MLD_EINVAL, "peg: more than 2^30 edges");
    if (capacity < total || (total > 0 && (!edge_vn || !edge_cn || !edge_type)))
        return mld::fail(MLD_EINVAL, "peg: output capacity " + std::to_string(capacity) + " < " +
                                         std::to_string(total) + " edges");
    auto pri = [&](int32_t c) { return prio ? prio[c] : c; };

    std::vector<int32_t> order(n_vn);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return vdeg[a] < vdeg[b]; });
    // VN adjacency in place (final degrees are known), checks grow
    std::vector<int64_t> vstart(static_cast<size_t>(n_vn) + 1, 0);
    for (int32_t v = 0; v < n_vn; ++v) vstart[v + 1] = vstart[v] + vdeg[v];
    std::vector<int32_t> vadj(static_cast<size_t>(total));
    std::vector<int32_t> vcnt(n_vn, 0);
    std::vector<std::vector<int32_t>> cadj(n_cn);
    std::vector<int32_t> cdeg(n_cn, 0);
    // per type: checks taking it, ordered by (degree, priority)
    std::vector<std::set<Key>> byt(n_types);
    std::vector<int64_t> n_of_type(n_types, 0);
    for (int32_t c = 0; c < n_cn; ++c)
        for (int32_t t = 0; t < n_types; ++t)
            if ((mask[c] >> t) & 1u) {
                byt[t].insert(Key{0, pri(c), c});
                n_of_type[t]++;
            }
    // breadth-first search state: stamps avoid clearing per search
    std::vector<int32_t> cstamp(n_cn, -1), clevel(n_cn, 0), vstamp(n_vn, -1);
    std::vector<int32_t> frontier, next_v, new_c;
    std::vector<std::vector<int32_t>> at_level;  // type-t checks first reached at each level
    int32_t stamp = 0;
    int64_t k = 0;
    for (int32_t v : order) {
        for (int32_t t = 0; t < n_types; ++t) {
            const int32_t dt = deg[static_cast<int64_t>(t) * n_vn + v];
            for (int32_t rep = 0; rep < dt; ++rep, ++stamp) {
                // levels from v; stop once every check taking t is reached
                int64_t reached_t = 0;
                int32_t lv = 0;
                at_level.clear();
                frontier.assign(1, v);
                vstamp[v] = stamp;
                while (!frontier.empty() && reached_t < n_of_type[t]) {
                    ++lv;
                    new_c.clear();
                    at_level.emplace_back();
                    for (int32_t u : frontier)
                        for (int64_t i = vstart[u]; i < vstart[u] + vcnt[u]; ++i) {
                            const int32_t c = vadj[i];
                            if (cstamp[c] == stamp) continue;
                            cstamp[c] = stamp;
                            clevel[c] = lv;
                            new_c.push_back(c);
                            if ((mask[c] >> t) & 1u) {
                                ++reached_t;
                                at_level.back().push_back(c);
                            }
                        }
                    next_v.clear();
                    for (int32_t c : new_c)
                        for (int32_t w : cadj[c])
                            if (vstamp[w] != stamp) {
                                vstamp[w] = stamp;
                                next_v.push_back(w);
                            }
                    frontier.swap(next_v);
                }
                int32_t pick = -1;
                if (reached_t < n_of_type[t]) {
                    // some check taking t is out of reach: the lightest of those
                    for (const Key &key : byt[t])
                        if (cstamp[key.c] != stamp) {
                            pick = key.c;
                            break;
                        }
                } else {
                    // the deepest level (>= 2: level 1 are v's neighbours) holding such checks
                    for (int32_t l = static_cast<int32_t>(at_level.size()); l >= 2 && pick < 0; --l) {
                        const Key *best = nullptr;
                        Key cur{};
                        for (int32_t c : at_level[l - 1]) {
                            const Key kc{cdeg[c], pri(c), c};
                            if (!best || kc < cur) {
                                cur = kc;
                                best = &cur;
                            }
                        }
                        if (best) pick = cur.c;
                    }
                }
                if (pick < 0)
                    return mld::fail(MLD_EGRAPH, "peg: no check left for an edge of type " + std::to_string(t) +
                                                     " of VN " + std::to_string(v));
                for (int32_t t2 = 0; t2 < n_types; ++t2)
                    if ((mask[pick] >> t2) & 1u) {
                        byt[t2].erase(Key{cdeg[pick], pri(pick), pick});
                        byt[t2].insert(Key{cdeg[pick] + 1, pri(pick), pick});
                    }
                cdeg[pick]++;
                vadj[vstart[v] + vcnt[v]++] = pick;
                cadj[pick].push_back(v);
                edge_vn[k] = v;
                edge_cn[k] = pick;
                edge_type[k] = static_cast<uint8_t>(t);
                ++k;
            }
        }
    }
    *n_edges = k;
    return MLD_OK;
}
