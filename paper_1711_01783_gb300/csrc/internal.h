// Internal declarations shared by the host graph store (graph.cpp) and the
// CUDA decoder (decoder.cu).  Not part of the public ABI (include/metldpc.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "metldpc.h"

namespace mld {

// Record an error for mld_last_error() and return `code`.
int fail(int code, const std::string &msg);
// Clear the thread's error text.
void clear_error();

// Graph store in the decoder's internal numbering (built on the host, then
// copied to the device).
//
//  * Core VNs (degree != 1) are numbered 0..n_core-1 in natural order.
//  * Degree-1 VNs get "slots" 0..n_deg1-1 in the order of their check, so that
//    the slots of check c are the contiguous range dptr[c]..dptr[c+1].
//  * Core edges are numbered check-major: the core edges of check c are
//    cptr[c]..cptr[c+1] (sorted by core VN), col[e] is the core VN of edge e.
//    This is also the order of the stored check-to-variable messages.
//  * vptr/vedge is the VN-major view (CSC): the core edges of core VN v are
//    vedge[vptr[v]..vptr[v+1]], ascending.
//  * unit[j] maps natural VN j to its internal index: core VN index, or
//    n_core + slot for a degree-1 VN.
//  * Checks are renumbered so that checks with the same number of core edges
//    (dc) and degree-1 VNs (dd) are contiguous ("classes").  Inside a class
//    with dc + dd <= kMaxRegDeg the edge range of a check is computed from its
//    position (e0 + j*dc, s0 + j*dd) instead of loaded.  Checks of higher
//    degree form one irregular class (dc = -1) that uses cptr/dptr.
//    cuser[c] is the caller's index of internal check c (cint is its inverse,
//    kept on the device to scatter syndrome bits into internal order).
constexpr int kMaxRegDeg = 8;

struct CheckClass {
    int32_t c0, count;  // internal checks c0 .. c0+count-1
    int32_t dc, dd;     // core edges and degree-1 VNs per check (dc = -1: irregular)
    int32_t e0, s0;     // first core edge and first degree-1 slot of the class
};

struct HostGraph {
    int32_t n_vn = 0, n_cn = 0;
    int64_t n_edges = 0;
    int32_t n_core = 0, n_deg1 = 0;
    int32_t e_core = 0;
    int32_t max_check_deg = 0, max_vn_deg = 0;
    std::vector<int32_t> cptr, col, dptr, vptr, vedge, unit, cuser;
    std::vector<CheckClass> classes;
    std::vector<uint8_t> etype_core, etype_deg1;
};

// One launch of the check update: a check class with its grid size for one
// slab width.  `deg` = dc + dd for a class held in registers (1..kMaxRegDeg),
// or -1 for checks read through cptr/dptr.
struct ClassLaunch {
    int32_t c0, count, dc, deg, e0, s0, blocks;
};

int build_host_graph(const int32_t *edge_vn, const int32_t *edge_cn,
                     const uint8_t *edge_type, int64_t n_edges, int32_t n_vn,
                     int32_t n_cn, HostGraph *out);

// Layered schedule: the checks of one layer share no core VN.  A layer's
// checks of one class form one launch.  Layered decoders number their
// messages in launch order, so that the messages of a launch are one
// contiguous run: position p (0 .. checks with edges - 1) is a check in
// (layer, class, class position) order, lchk[p] its internal id, its core
// edges the layered edges leptr[p] .. leptr[p+1], lcol[e] the core VN of
// layered edge e.  A launch covers positions p0 .. p0+count-1 and layered
// edges e0 .. (one class: e0 + k dc for its k-th check).
struct LayerLaunch {
    int32_t layer, cls, p0, count, e0;
};
struct LayerTables {
    std::vector<LayerLaunch> launches;
    std::vector<int32_t> lchk, leptr, lcol, layer_user;
    int32_t n_layers = 0;
};

// Validate a layering (layer of every check in the caller's numbering; NULL
// computes a first fit per class) and build the layered tables.
int build_layers(const HostGraph &h, const int32_t *layer_of_check, int32_t n_layers, LayerTables *out);

}  // namespace mld

struct mld_graph {
    mld::HostGraph h;
    int device = 0;
    // device copies of the index arrays
    int32_t *cptr = nullptr, *col = nullptr, *dptr = nullptr;
    int32_t *vptr = nullptr, *vedge = nullptr, *unit = nullptr, *cint = nullptr;
    uint8_t *etype_core = nullptr, *etype_deg1 = nullptr;
    // check-update launches per slab width (8, 16, 32, 64)
    std::vector<mld::ClassLaunch> launches[4];
    // every check is in a register class (enables the fused syndrome check)
    bool fusable = false;
    // every check with edges is in a register class (posterior accumulation,
    // layered schedule)
    bool acc_ok = false;
    // layered schedule: launches in order, the layer of every check in the
    // caller's numbering, and the device copies of the layered tables
    std::vector<mld::LayerLaunch> layer_launches;
    std::vector<int32_t> layer_user;
    int32_t n_layers = 0;
    int32_t *lchk = nullptr, *leptr = nullptr, *lcol = nullptr;
    uint64_t layers_gen = 0;  // counts layerings set (device loops record it)
};
