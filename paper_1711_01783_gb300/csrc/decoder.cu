// Batched syndrome-based flooding sum-product BP decoder for sm_103a.
//
// Method: arXiv:1711.01783, Methods, Steps 1-5 (Eqs. 1-5) in the LLR domain
// (closing paragraph of the Methods), with the GPU organisation of Results,
// "High speed error correction with MET-LDPC codes" re-designed for GB300:
//
//  * Codewords are interleaved in slabs of W (the paper's "raw key
//    permutation"): the message of edge e for slab s is W consecutive values,
//    so each graph gather or scatter moves whole 128-byte lines.
//  * The only per-edge state is the check-to-variable message r of the core
//    edges (stored float or half).  Core-VN posteriors L_v are kept in float;
//    the check update forms the extrinsic q = L_v - r_old itself, so no
//    variable-to-check array exists.
//  * Degree-1 VNs are skipped during the iterations (Table 1 "Ignored VNs",
//    Discussion): their variable-to-check message is always the channel LLR,
//    read by the check update; their posterior comes from the last check
//    update.  This is exact.
//  * One thread owns 4 codewords of one check (or one VN); check-degree
//    reductions stay in registers, and the leave-one-out sums of phi are
//    prefix + suffix sums, so no total-minus-own cancellation occurs.
//  * Hard decisions are bit-sliced (one bit per codeword, W/8 bytes per node),
//    so the syndrome check of Step 5 is a bit-exact XOR over edges.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.cuh"


// Check-update launches for each slab width: one per check class that has
// edges, with its grid size.
void build_class_tables(mld_graph *g) {
    const int widths[4] = {8, 16, 32, 64};
    for (int wi = 0; wi < 4; ++wi) {
        const int tpc = widths[wi] / kK;
        std::vector<ClassLaunch> &out = g->launches[wi];
        out.clear();
        for (const mld::CheckClass &cl : g->h.classes) {
            if (cl.dc == 0 && cl.dd == 0) continue;  // checks without edges: nothing to send
            ClassLaunch l;
            l.c0 = cl.c0;
            l.count = cl.count;
            l.dc = cl.dc;
            l.deg = cl.dc < 0 ? -1 : cl.dc + cl.dd;
            l.e0 = cl.e0;
            l.s0 = cl.s0;
            l.blocks = grid_x(static_cast<int64_t>(cl.count) * tpc);
            out.push_back(l);
        }
    }
    // the fused syndrome check needs every check in a register class (the
    // checks without edges and the irregular class are not covered)
    g->fusable = true;
    for (const mld::CheckClass &cl : g->h.classes)
        if (cl.dc < 0 || cl.dd > 1 || cl.dc + cl.dd > mld::kMaxRegDeg || (cl.dc == 0 && cl.dd == 0))
            g->fusable = false;
    // posterior accumulation: every check with edges in a register class
    g->acc_ok = true;
    for (const mld::CheckClass &cl : g->h.classes)
        if (!(cl.dc == 0 && cl.dd == 0) && (cl.dc < 0 || cl.dd > 1 || cl.dc + cl.dd > mld::kMaxRegDeg))
            g->acc_ok = false;
}

namespace {

void decoder_free(mld_decoder *d) {
    if (!d) return;
    mld::tape_release(d);
    if (d->r) cudaFree(d->r);
    d->r = nullptr;
    dfree(d->Lv); dfree(d->lch); dfree(d->lch1); dfree(d->post1); dfree(d->phi1);
    dfree(d->Lv2); dfree(d->Lv3);
    dfree(d->hb_core); dfree(d->hb1); dfree(d->sbits);
    dfree(d->done); dfree(d->fail); dfree(d->iters); dfree(d->conv); dfree(d->status);
    if (d->status_host) cudaFreeHost(d->status_host);
    d->status_host = nullptr;
    dfree(d->in_stage); dfree(d->sigma_stage); dfree(d->post_stage);
    dfree(d->syn_stage); dfree(d->bits_stage);
    for (auto &t : d->timed) { d->event_pool.push_back(t.a); d->event_pool.push_back(t.b); }
    d->timed.clear();
    for (cudaEvent_t e : d->event_pool) cudaEventDestroy(e);
    d->event_pool.clear();
    if (d->ev_fork) cudaEventDestroy(d->ev_fork);
    if (d->ev_join) cudaEventDestroy(d->ev_join);
    if (d->side) cudaStreamDestroy(d->side);
    d->ev_fork = d->ev_join = nullptr;
    d->side = nullptr;
    for (auto &lg : d->loops) cudaGraphExecDestroy(lg.exec);
    d->loops.clear();
    if (d->cap) cudaStreamDestroy(d->cap);
    d->cap = nullptr;
    dfree(d->lctr);
}

// The device address of a page-locked, mapped host buffer; null for any
// other pointer (pageable memory is staged instead).
const void *mapped_host(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // an unregistered pointer is not an error here
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

const char *array_name(int id) {
    static const char *names[] = {"?", "cptr", "col", "dptr", "vptr", "vedge", "unit", "cint", "lchk", "leptr",
                                  "lcol"};
    return (id >= 1 && id <= 10) ? names[id] : names[0];
}

std::string graph_fault_text(const int32_t st[4]) {
    return std::string("graph store corrupted on the device: ") + array_name(st[1]) + "[" + std::to_string(st[2]) +
           "] holds " + std::to_string(st[3]) + ", out of its range";
}

// Checked decoders: validate the graph store on the device, wait for the
// result, and refuse to decode a corrupted store (no decode kernel runs).
int validate_store(mld_decoder *d, cudaStream_t st) {
    const mld_graph *g = d->g;
    const mld::HostGraph &h = g->h;
    MLD_CUDA(cudaMemsetAsync(d->status, 0, 4 * sizeof(int32_t), st));
    const bool lay = d->schedule == MLD_SCHED_LAYERED && g->lchk;
    ValidateArgs va{g->cptr, g->col, g->dptr, g->vptr, g->vedge, g->unit, g->cint,
                    lay ? g->lchk : nullptr, lay ? g->leptr : nullptr, lay ? g->lcol : nullptr,
                    h.n_vn, h.n_cn, h.n_core, h.n_deg1, h.e_core,
                    0, d->status};
    if (lay) {
        int32_t np = 0;
        for (const mld::LayerLaunch &ll : g->layer_launches) np += ll.count;
        va.n_lpos = np;
    }
    int64_t top = std::max<int64_t>({static_cast<int64_t>(h.e_core), static_cast<int64_t>(h.n_vn) + 1,
                                     static_cast<int64_t>(h.n_cn) + 1, static_cast<int64_t>(va.n_lpos) + 1});
    k_validate_graph<<<static_cast<int>(std::min<int64_t>((top + kBlock - 1) / kBlock, 152 * 16)), kBlock, 0, st>>>(va);
    MLD_LAUNCHED("k_validate_graph");
    MLD_CUDA(cudaMemcpyAsync(d->status_host, d->status, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MLD_CUDA(cudaStreamSynchronize(st));
    if (d->status_host[0] != 0) return mld::fail(d->status_host[0], graph_fault_text(d->status_host));
    return MLD_OK;
}

int decode_common(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syndrome,
                  int32_t batch, int32_t max_iters, uint32_t flags, uint8_t *bits_out,
                  float *post_out, uint8_t *converged, int32_t *iters_used, void *stream,
                  bool y_mode) {
    mld::clear_error();
    if (!d) return mld::fail(MLD_EINVAL, "decode: null decoder");
    if (flags & ~(MLD_EARLY_TERM | MLD_DEVICE_PTRS)) return mld::fail(MLD_EINVAL, "decode: unknown flag");
    if (batch < 0 || batch > d->max_batch)
        return mld::fail(MLD_EINVAL, "decode: batch " + std::to_string(batch) + " outside [0, " +
                                         std::to_string(d->max_batch) + "]");
    if (max_iters < 0) return mld::fail(MLD_EINVAL, "decode: negative max_iters");
    if (batch == 0) return MLD_OK;
    const mld::HostGraph &h = d->g->h;
    if ((h.n_vn > 0 && (!in || !bits_out)) || (h.n_cn > 0 && !syndrome) || !converged || !iters_used ||
        (y_mode && !sigma))
        return mld::fail(MLD_EINVAL, "decode: null data pointer");
    int s = check_device(d->device);
    if (s != MLD_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (d->checked && d->status_host) {
        s = validate_store(d, st);
        if (s != MLD_OK) return s;
    }
    const bool dev = (flags & MLD_DEVICE_PTRS) != 0;
    const bool et = (flags & MLD_EARLY_TERM) != 0;
    const size_t nb = static_cast<size_t>(batch) * h.n_vn;
    const size_t mb = static_cast<size_t>(batch) * h.n_cn;
    const float *din = in;
    const float *dsig = y_mode ? sigma : nullptr;
    const uint8_t *dsyn = syndrome;
    uint8_t *dbits = bits_out;
    float *dpost = post_out;
    // Host buffers that are page-locked and mapped into the device's address
    // space (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory) are
    // read and written by the layout kernels directly over the host link;
    // other host buffers are staged through device copies.
    const float *min = nullptr, *msig = nullptr;
    const uint8_t *msyn = nullptr;
    uint8_t *mbits = nullptr;
    float *mpost = nullptr;
    if (!dev) {
        min = static_cast<const float *>(mapped_host(in));
        msyn = static_cast<const uint8_t *>(mapped_host(syndrome));
        msig = y_mode ? static_cast<const float *>(mapped_host(sigma)) : nullptr;
        mbits = static_cast<uint8_t *>(const_cast<void *>(mapped_host(bits_out)));
        mpost = post_out ? static_cast<float *>(const_cast<void *>(mapped_host(post_out))) : nullptr;
        if (min) din = min;
        else {
            if (nb) MLD_CUDA(cudaMemcpyAsync(d->in_stage, in, nb * sizeof(float), cudaMemcpyHostToDevice, st));
            din = d->in_stage;
        }
        if (msyn) dsyn = msyn;
        else {
            if (mb) MLD_CUDA(cudaMemcpyAsync(d->syn_stage, syndrome, mb, cudaMemcpyHostToDevice, st));
            dsyn = d->syn_stage;
        }
        if (y_mode) {
            if (msig) dsig = msig;
            else {
                MLD_CUDA(cudaMemcpyAsync(d->sigma_stage, sigma, sizeof(float) * batch, cudaMemcpyHostToDevice, st));
                dsig = d->sigma_stage;
            }
        }
        dbits = mbits ? mbits : d->bits_stage;
        dpost = post_out ? (mpost ? mpost : d->post_stage) : nullptr;
    }
    s = (d->msg == MLD_MSG_F16)
            ? mld::run_decode_f16(d, din, dsig, dsyn, batch, max_iters, et, dbits, dpost, converged, iters_used, st, dev)
            : mld::run_decode_f32(d, din, dsig, dsyn, batch, max_iters, et, dbits, dpost, converged, iters_used, st, dev);
    if (s != MLD_OK) return s;
    if (!dev) {
        if (nb && !mbits) MLD_CUDA(cudaMemcpyAsync(bits_out, d->bits_stage, nb, cudaMemcpyDeviceToHost, st));
        if (post_out && nb && !mpost)
            MLD_CUDA(cudaMemcpyAsync(post_out, d->post_stage, nb * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    return MLD_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *mld_last_error(void) { return mld::last_error_text(); }

const char *mld_version(void) { return "metldpc 0.1.0 sm_103a"; }

int mld_graph_create(const int32_t *edge_vn, const int32_t *edge_cn, const uint8_t *edge_type,
                     int64_t n_edges, int32_t n_vn, int32_t n_cn, mld_graph **out) {
    mld::clear_error();
    if (!out) return mld::fail(MLD_EINVAL, "graph_create: null out");
    mld_graph *g = new (std::nothrow) mld_graph();
    if (!g) return mld::fail(MLD_ENOMEM, "graph_create: host allocation");
    int s = mld::build_host_graph(edge_vn, edge_cn, edge_type, n_edges, n_vn, n_cn, &g->h);
    if (s == MLD_OK) {
        cudaError_t e = cudaGetDevice(&g->device);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaGetDevice");
    }
    if (s == MLD_OK) s = upload(&g->cptr, g->h.cptr);
    if (s == MLD_OK) s = upload(&g->col, g->h.col);
    if (s == MLD_OK) s = upload(&g->dptr, g->h.dptr);
    if (s == MLD_OK) s = upload(&g->vptr, g->h.vptr);
    if (s == MLD_OK) s = upload(&g->vedge, g->h.vedge);
    if (s == MLD_OK) s = upload(&g->unit, g->h.unit);
    if (s == MLD_OK) {
        std::vector<int32_t> cint(g->h.n_cn);
        for (int32_t i = 0; i < g->h.n_cn; ++i) cint[g->h.cuser[i]] = i;
        s = upload(&g->cint, cint);
    }
    if (s == MLD_OK) s = upload(&g->etype_core, g->h.etype_core);
    if (s == MLD_OK) s = upload(&g->etype_deg1, g->h.etype_deg1);
    if (s != MLD_OK) {
        mld_graph_destroy(g);
        return s;
    }
    build_class_tables(g);
    *out = g;
    return MLD_OK;
}

int mld_graph_destroy(mld_graph *g) {
    if (!g) return MLD_OK;
    dfree(g->cptr); dfree(g->col); dfree(g->dptr); dfree(g->vptr); dfree(g->vedge);
    dfree(g->unit); dfree(g->cint); dfree(g->etype_core); dfree(g->etype_deg1);
    dfree(g->lchk); dfree(g->leptr); dfree(g->lcol);
    delete g;
    return MLD_OK;
}

int mld_graph_stats_get(const mld_graph *g, mld_graph_stats *out) {
    mld::clear_error();
    if (!g || !out) return mld::fail(MLD_EINVAL, "graph_stats_get: null pointer");
    const mld::HostGraph &h = g->h;
    out->n_vn = h.n_vn;
    out->n_cn = h.n_cn;
    out->n_edges = h.n_edges;
    out->n_core = h.n_core;
    out->n_deg1 = h.n_deg1;
    out->e_core = h.e_core;
    out->max_check_deg = h.max_check_deg;
    out->max_vn_deg = h.max_vn_deg;
    return MLD_OK;
}

int mld_graph_index_arrays(const mld_graph *g, mld_index_arrays *out) {
    mld::clear_error();
    if (!g || !out) return mld::fail(MLD_EINVAL, "graph_index_arrays: null pointer");
    const mld::HostGraph &h = g->h;
    out->cptr = g->cptr;   out->n_cptr = h.n_cn + 1;
    out->col = g->col;     out->n_col = h.e_core;
    out->dptr = g->dptr;   out->n_dptr = h.n_cn + 1;
    out->vptr = g->vptr;   out->n_vptr = h.n_core + 1;
    out->vedge = g->vedge; out->n_vedge = h.e_core;
    out->unit = g->unit;   out->n_unit = h.n_vn;
    out->cint = g->cint;   out->n_cint = h.n_cn;
    return MLD_OK;
}

int mld_graph_set_layers(mld_graph *g, const int32_t *layer_of_check, int32_t n_layers) {
    mld::clear_error();
    if (!g) return mld::fail(MLD_EINVAL, "graph_set_layers: null graph");
    mld::LayerTables t;
    int s = mld::build_layers(g->h, layer_of_check, n_layers, &t);
    if (s != MLD_OK) return s;
    s = check_device(g->device);
    if (s != MLD_OK) return s;
    int32_t *lchk = nullptr, *leptr = nullptr, *lcol = nullptr;
    s = upload(&lchk, t.lchk);
    if (s == MLD_OK) s = upload(&leptr, t.leptr);
    if (s == MLD_OK) s = upload(&lcol, t.lcol);
    if (s != MLD_OK) {
        dfree(lchk); dfree(leptr); dfree(lcol);
        return s;
    }
    dfree(g->lchk); dfree(g->leptr); dfree(g->lcol);
    g->lchk = lchk;
    g->leptr = leptr;
    g->lcol = lcol;
    g->layer_launches = std::move(t.launches);
    g->layer_user = std::move(t.layer_user);
    g->n_layers = t.n_layers;
    g->layers_gen++;
    return MLD_OK;
}

int mld_graph_layers_get(const mld_graph *g, int32_t *layer_of_check, int32_t *n_layers) {
    mld::clear_error();
    if (!g || !n_layers) return mld::fail(MLD_EINVAL, "graph_layers_get: null pointer");
    if (!g->lchk) return mld::fail(MLD_EINVAL, "graph_layers_get: the graph has no layering");
    *n_layers = g->n_layers;
    if (layer_of_check) std::copy(g->layer_user.begin(), g->layer_user.end(), layer_of_check);
    return MLD_OK;
}

int mld_decoder_create(const mld_graph *g, const mld_opts *opts, mld_decoder **out) {
    mld::clear_error();
    if (!g || !opts || !out) return mld::fail(MLD_EINVAL, "decoder_create: null pointer");
    for (int i = 0; i < 6; ++i)
        if (opts->reserved[i] != 0) return mld::fail(MLD_EINVAL, "decoder_create: reserved field not zero");
    if (opts->checked != 0 && opts->checked != 1) return mld::fail(MLD_EINVAL, "decoder_create: checked must be 0 or 1");
    if (opts->staging != MLD_STAGE_DIRECT && opts->staging != MLD_STAGE_BULK && opts->staging != MLD_STAGE_BULK_LSU)
        return mld::fail(MLD_EINVAL, "decoder_create: unknown staging");
    if (opts->check_rule != MLD_CHECK_SUM_PRODUCT && opts->check_rule != MLD_CHECK_MIN_SUM)
        return mld::fail(MLD_EINVAL, "decoder_create: unknown check_rule");
    if (opts->check_rule == MLD_CHECK_MIN_SUM &&
        (!(opts->ms_offset >= 0.f) || !std::isfinite(opts->ms_offset)))
        return mld::fail(MLD_EINVAL, "decoder_create: ms_offset must be finite and >= 0");
    if (opts->vn_update != MLD_VN_GATHER && opts->vn_update != MLD_VN_ACCUMULATE)
        return mld::fail(MLD_EINVAL, "decoder_create: unknown vn_update");
    if (opts->schedule != MLD_SCHED_FLOODING && opts->schedule != MLD_SCHED_LAYERED)
        return mld::fail(MLD_EINVAL, "decoder_create: unknown schedule");
    if (opts->msg_dtype != MLD_MSG_F32 && opts->msg_dtype != MLD_MSG_F16)
        return mld::fail(MLD_EINVAL, "decoder_create: unknown msg_dtype");
    if (opts->max_batch < 1) return mld::fail(MLD_EINVAL, "decoder_create: max_batch < 1");
    if (!(opts->lmax >= 0.f) || !std::isfinite(opts->lmax) || opts->lmax > 60.f)
        return mld::fail(MLD_EINVAL, "decoder_create: lmax must be in (0, 60]");
    int W = opts->slab_width;
    if (W == 0) W = (opts->msg_dtype == MLD_MSG_F16) ? 64 : 32;
    if (W != 8 && W != 16 && W != 32 && W != 64) return mld::fail(MLD_EINVAL, "decoder_create: slab_width");
    if (opts->vn_update == MLD_VN_ACCUMULATE) {
        if (W != ((opts->msg_dtype == MLD_MSG_F16) ? 64 : 32))
            return mld::fail(MLD_EINVAL, "decoder_create: posterior accumulation needs the default slab width");
        if (!g->acc_ok)
            return mld::fail(MLD_EINVAL, "decoder_create: posterior accumulation needs every check to have at "
                                         "most 8 edges and at most one degree-1 VN");
    }
    if (opts->check_rule == MLD_CHECK_MIN_SUM &&
        (W != ((opts->msg_dtype == MLD_MSG_F16) ? 64 : 32) || opts->schedule != MLD_SCHED_FLOODING ||
         opts->vn_update != MLD_VN_GATHER))
        return mld::fail(MLD_EINVAL, "decoder_create: min-sum needs the default slab width, the flooding "
                                     "schedule and MLD_VN_GATHER");
    if (opts->schedule == MLD_SCHED_LAYERED) {
        if (W != ((opts->msg_dtype == MLD_MSG_F16) ? 64 : 32))
            return mld::fail(MLD_EINVAL, "decoder_create: the layered schedule needs the default slab width");
        if (opts->vn_update != MLD_VN_GATHER)
            return mld::fail(MLD_EINVAL, "decoder_create: the layered schedule updates posteriors in place "
                                         "(vn_update must be MLD_VN_GATHER)");
    }
    int s = check_device(g->device);
    if (s != MLD_OK) return s;
    if (opts->staging != MLD_STAGE_DIRECT) {
        const cudaError_t ce = mld::prepare_staged_f16();
        if (ce != cudaSuccess) return cuda_fail(ce, "decoder_create: staged kernels");
    }
    if (opts->schedule == MLD_SCHED_LAYERED && !g->lchk) {
        // no layering given: the default first fit per check class
        s = mld_graph_set_layers(const_cast<mld_graph *>(g), nullptr, 0);
        if (s != MLD_OK) return s;
    }
    mld_decoder *d = new (std::nothrow) mld_decoder();
    if (!d) return mld::fail(MLD_ENOMEM, "decoder_create: host allocation");
    d->g = g;
    d->device = g->device;
    d->msg = opts->msg_dtype;
    d->W = W;
    d->vn_update = opts->vn_update;
    d->schedule = opts->schedule;
    d->check_rule = opts->check_rule;
    d->checked = opts->checked != 0;
    d->staging = opts->staging;
    d->ms_off_i = opts->check_rule == MLD_CHECK_MIN_SUM ? opts->ms_offset * 1.4426950408889634f : 0.f;
    d->max_batch = opts->max_batch;
    d->max_slabs = (opts->max_batch + W - 1) / W;
    set_units(d, opts->lmax > 0.f ? opts->lmax : 25.f);
    const mld::HostGraph &h = g->h;
    const size_t S = d->max_slabs;
    const size_t msz = d->msg == MLD_MSG_F16 ? 2 : 4;
    const size_t DW = (W + 31) / 32;
    const size_t NB = W / 8;
    const size_t nb = static_cast<size_t>(d->max_batch) * h.n_vn;
    cudaError_t e = cudaMalloc(&d->r, std::max<size_t>(1, S * h.e_core * W * msz));
    if (e != cudaSuccess) {
        d->r = nullptr;
        s = mld::fail(e == cudaErrorMemoryAllocation ? MLD_ENOMEM : MLD_ECUDA, "cudaMalloc messages");
    }
    if (s == MLD_OK) s = dalloc(&d->Lv, S * h.n_core * W);
    if (s == MLD_OK) s = dalloc(&d->lch, S * h.n_core * W);
    if (s == MLD_OK && d->vn_update == MLD_VN_ACCUMULATE) s = dalloc(&d->Lv2, S * h.n_core * W);
    if (s == MLD_OK && d->vn_update == MLD_VN_ACCUMULATE) s = dalloc(&d->Lv3, S * h.n_core * W);
    if (s == MLD_OK) s = dalloc(&d->lch1, S * h.n_deg1 * W);
    if (s == MLD_OK) s = dalloc(&d->post1, S * h.n_deg1 * W);
    if (s == MLD_OK) s = dalloc(&d->phi1, S * h.n_deg1 * W);
    if (s == MLD_OK) s = dalloc(&d->hb_core, S * h.n_core * NB);
    if (s == MLD_OK) s = dalloc(&d->hb1, 2 * S * h.n_deg1 * NB);  // two buffers (iteration parity)
    if (s == MLD_OK) s = dalloc(&d->sbits, S * h.n_cn * NB);
    if (s == MLD_OK) s = dalloc(&d->done, S * DW);
    if (s == MLD_OK) s = dalloc(&d->fail, 2 * S * DW);  // two buffers (iteration parity) for plans
    if (s == MLD_OK) s = dalloc(&d->iters, S * W);
    if (s == MLD_OK) s = dalloc(&d->conv, S * W);
    if (s == MLD_OK) s = dalloc(&d->status, 4);
    if (s == MLD_OK && d->checked) {
        cudaError_t ce = cudaHostAlloc(reinterpret_cast<void **>(&d->status_host), 4 * sizeof(int32_t),
                                       cudaHostAllocDefault);
        if (ce != cudaSuccess) {
            d->status_host = nullptr;
            s = cuda_fail(ce, "decoder_create: status word");
        }
    }
    if (s == MLD_OK) s = dalloc(&d->in_stage, nb);
    if (s == MLD_OK) s = dalloc(&d->sigma_stage, static_cast<size_t>(d->max_batch));
    if (s == MLD_OK) s = dalloc(&d->post_stage, nb);
    if (s == MLD_OK) s = dalloc(&d->syn_stage, static_cast<size_t>(d->max_batch) * h.n_cn);
    if (s == MLD_OK) s = dalloc(&d->bits_stage, nb);
    if (s == MLD_OK) s = dalloc(&d->lctr, 2);
    if (s == MLD_OK) {
        cudaError_t ce = cudaStreamCreateWithFlags(&d->cap, cudaStreamNonBlocking);
        if (ce != cudaSuccess) s = cuda_fail(ce, "decoder_create: capture stream");
    }
    if (s == MLD_OK) {
        cudaError_t ce = cudaStreamCreateWithFlags(&d->side, cudaStreamNonBlocking);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&d->ev_fork, cudaEventDisableTiming);
        if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&d->ev_join, cudaEventDisableTiming);
        if (ce != cudaSuccess) s = cuda_fail(ce, "decoder_create: side stream");
    }
    if (s == MLD_OK) {
        cudaError_t e2 = cudaMemset(d->status, 0, 4 * sizeof(int32_t));
        if (e2 != cudaSuccess) s = cuda_fail(e2, "cudaMemset");
    }
    if (s != MLD_OK) {
        decoder_free(d);
        delete d;
        return s;
    }
    *out = d;
    return MLD_OK;
}

int mld_decoder_destroy(mld_decoder *d) {
    if (!d) return MLD_OK;
    decoder_free(d);
    delete d;
    return MLD_OK;
}

int mld_decode(mld_decoder *d, const float *llr, const uint8_t *syndrome, int32_t batch,
               int32_t max_iters, uint32_t flags, uint8_t *bits_out, float *post_out,
               uint8_t *converged, int32_t *iters_used, void *stream) {
    return decode_common(d, llr, nullptr, syndrome, batch, max_iters, flags, bits_out, post_out,
                         converged, iters_used, stream, false);
}

int mld_decode_y(mld_decoder *d, const float *y, const float *sigma, const uint8_t *syndrome,
                 int32_t batch, int32_t max_iters, uint32_t flags, uint8_t *bits_out,
                 float *post_out, uint8_t *converged, int32_t *iters_used, void *stream) {
    return decode_common(d, y, sigma, syndrome, batch, max_iters, flags, bits_out, post_out,
                         converged, iters_used, stream, true);
}

int mld_decode_status(mld_decoder *d) {
    mld::clear_error();
    if (!d) return mld::fail(MLD_EINVAL, "decode_status: null decoder");
    int32_t v[4] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpy(v, d->status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "decode_status");
    if (v[0] == MLD_ETIMEOUT)
        return mld::fail(MLD_ETIMEOUT, "decode_status: a staged check update gave up waiting for a bulk copy");
    return v[0] == 0 ? MLD_OK : mld::fail(v[0], graph_fault_text(v));
}

int mld_decoder_test_stall(mld_decoder *d, int32_t bytes) {
    mld::clear_error();
    if (!d) return mld::fail(MLD_EINVAL, "decoder_test_stall: null decoder");
    if (bytes < 0 || bytes > 65536) return mld::fail(MLD_EINVAL, "decoder_test_stall: bytes outside [0, 65536]");
    if (bytes != d->stall_test && !d->loops.empty()) {
        // the early-termination loop graphs hold the launch arguments they
        // were captured with: drop them (after the device is idle)
        MLD_CUDA(cudaDeviceSynchronize());
        for (auto &lg : d->loops) cudaGraphExecDestroy(lg.exec);
        d->loops.clear();
    }
    d->stall_test = bytes;
    return MLD_OK;
}

int mld_decoder_timing_enable(mld_decoder *d, int enable) {
    mld::clear_error();
    if (!d) return mld::fail(MLD_EINVAL, "timing_enable: null decoder");
    if (enable < 0) return mld::fail(MLD_EINVAL, "timing_enable: negative period");
    d->timing = enable != 0;
    d->timing_every = enable > 0 ? enable : 1;
    return MLD_OK;
}

int mld_decoder_timing_read(mld_decoder *d, mld_timing *out) {
    mld::clear_error();
    if (!d || !out) return mld::fail(MLD_EINVAL, "timing_read: null pointer");
    std::memset(out, 0, sizeof(*out));
    int status = MLD_OK;
    for (auto &t : d->timed) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(t.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e != cudaSuccess && status == MLD_OK) status = cuda_fail(e, "timing_read");
        switch (t.cls) {
            case kClsCheck: out->check_ms += ms; out->check_timed++; break;
            case kClsVar: out->var_ms += ms; out->var_timed++; break;
            case kClsSyn: out->syndrome_ms += ms; out->syndrome_timed++; break;
            default: out->layout_ms += ms; out->layout_timed++; break;
        }
        d->event_pool.push_back(t.a);
        d->event_pool.push_back(t.b);
    }
    d->timed.clear();
    out->check_launches = d->launches[kClsCheck];
    out->var_launches = d->launches[kClsVar];
    out->syndrome_launches = d->launches[kClsSyn];
    out->layout_launches = d->launches[kClsLayout];
    for (int64_t &n : d->launches) n = 0;
    return status;
}

int mld_phi_eval(int32_t msg_dtype, const float *x, float *out, int64_t n, void *stream) {
    mld::clear_error();
    if (msg_dtype != MLD_MSG_F32 && msg_dtype != MLD_MSG_F16) return mld::fail(MLD_EINVAL, "phi_eval: msg_dtype");
    if (n < 0 || (n > 0 && (!x || !out))) return mld::fail(MLD_EINVAL, "phi_eval: bad arguments");
    if (n == 0) return MLD_OK;
    const float lmax = 25.f;
    const float amin = static_cast<float>(phi_host(25.0));
    const float kLog2e = 1.442695040888963407f, kLn2 = 0.693147180559945309f;
    const float lmax_i = static_cast<float>(25.0 * 1.4426950408889634074);
    const float amin_i = static_cast<float>(phi_host(25.0) * 1.4426950408889634074);
    if (msg_dtype == MLD_MSG_F16)
        k_phi_eval<kFitB2H><<<grid_x(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n, kLog2e, lmax_i,
                                                                                     amin_i, kLn2);
    else
        k_phi_eval<kFitB2><<<grid_x(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n, kLog2e, lmax_i,
                                                                                    amin_i, kLn2);
    (void)lmax;
    (void)amin;
    MLD_LAUNCHED("k_phi_eval");
    return MLD_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free decode: working memory in a file-scope device array
// ===========================================================================
namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[MLD_NOALLOC_SCRATCH_BYTES];

constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_base[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device `dev`.  In host
// code the array's name is only a host-side stand-in, so the address is looked
// up once per device and cached.
int noalloc_base(int dev, void **out) {
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return mld::fail(MLD_EINVAL, "decode_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_fail(e, "decode_noalloc: the static scratch array could not be reserved on this device "
                                "(its module loads with the first call under lazy loading; make a warm-up "
                                "call before the device's memory is taken): cudaGetSymbolAddress");
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return MLD_OK;
}

// Offsets of the working buffers inside the scratch array (256-byte aligned).
struct NoallocLayout {
    size_t r, Lv, lch, lch1, post1, phi1, hb_core, hb1, sbits, done, fail, iters, conv, total;
};

NoallocLayout noalloc_layout(const mld::HostGraph &h, int W, size_t msz, int slabs) {
    NoallocLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (std::max<size_t>(bytes, 1) + 255) & ~static_cast<size_t>(255);
        return o;
    };
    const size_t S = static_cast<size_t>(slabs);
    const size_t NB = W / 8, DW = (W + 31) / 32;
    L.r = take(S * h.e_core * W * msz);
    L.Lv = take(S * h.n_core * W * sizeof(float));
    L.lch = take(S * h.n_core * W * sizeof(float));
    L.lch1 = take(S * h.n_deg1 * W * sizeof(float));
    L.post1 = take(S * h.n_deg1 * W * sizeof(float));
    L.phi1 = take(S * h.n_deg1 * W * sizeof(float));
    L.hb_core = take(S * h.n_core * NB);
    L.hb1 = take(2 * S * h.n_deg1 * NB);
    L.sbits = take(S * h.n_cn * NB);
    L.done = take(S * DW * sizeof(uint32_t));
    L.fail = take(2 * S * DW * sizeof(uint32_t));
    L.iters = take(S * W * sizeof(int32_t));
    L.conv = take(S * W);
    L.total = off;
    return L;
}

}  // namespace

extern "C" int mld_decode_noalloc(const mld_graph *g, int32_t msg_dtype, const float *llr,
                                  const uint8_t *syndrome, int32_t batch, int32_t max_iters,
                                  uint32_t flags, uint8_t *bits_out, float *post_out,
                                  uint8_t *converged, int32_t *iters_used, void *stream) {
    mld::clear_error();
    if (!g) return mld::fail(MLD_EINVAL, "decode_noalloc: null graph");
    if (msg_dtype != MLD_MSG_F32 && msg_dtype != MLD_MSG_F16)
        return mld::fail(MLD_EINVAL, "decode_noalloc: unknown msg_dtype");
    if (flags & ~(MLD_EARLY_TERM | MLD_DEVICE_PTRS)) return mld::fail(MLD_EINVAL, "decode_noalloc: unknown flag");
    if (batch < 0 || max_iters < 0) return mld::fail(MLD_EINVAL, "decode_noalloc: negative batch or max_iters");
    if (batch == 0) return MLD_OK;
    const mld::HostGraph &h = g->h;
    if ((h.n_vn > 0 && (!llr || !bits_out)) || (h.n_cn > 0 && !syndrome) || !converged || !iters_used)
        return mld::fail(MLD_EINVAL, "decode_noalloc: null data pointer");
    int s = check_device(g->device);
    if (s != MLD_OK) return s;
    const int W = msg_dtype == MLD_MSG_F16 ? 64 : 32;
    const size_t msz = msg_dtype == MLD_MSG_F16 ? 2 : 4;
    const int slabs = (batch + W - 1) / W;
    const NoallocLayout L = noalloc_layout(h, W, msz, slabs);
    if (L.total > static_cast<size_t>(MLD_NOALLOC_SCRATCH_BYTES))
        return mld::fail(MLD_EINVAL, "decode_noalloc: this graph and batch need " + std::to_string(L.total) +
                                         " bytes of scratch; the static array holds " +
                                         std::to_string(static_cast<size_t>(MLD_NOALLOC_SCRATCH_BYTES)));
    void *base_v = nullptr;
    s = noalloc_base(g->device, &base_v);
    if (s != MLD_OK) return s;
    unsigned char *base = static_cast<unsigned char *>(base_v);
    // a decoder view onto the scratch array: nothing here is freed
    mld_decoder d;
    d.g = g;
    d.device = g->device;
    d.msg = msg_dtype;
    d.W = W;
    d.max_batch = batch;
    d.max_slabs = slabs;
    set_units(&d, 25.f);
    d.r = base + L.r;
    d.Lv = reinterpret_cast<float *>(base + L.Lv);
    d.lch = reinterpret_cast<float *>(base + L.lch);
    d.lch1 = reinterpret_cast<float *>(base + L.lch1);
    d.post1 = reinterpret_cast<float *>(base + L.post1);
    d.phi1 = reinterpret_cast<float *>(base + L.phi1);
    d.hb_core = base + L.hb_core;
    d.hb1 = base + L.hb1;
    d.sbits = base + L.sbits;
    d.done = reinterpret_cast<uint32_t *>(base + L.done);
    d.fail = reinterpret_cast<uint32_t *>(base + L.fail);
    d.iters = reinterpret_cast<int32_t *>(base + L.iters);
    d.conv = base + L.conv;
    const bool et = (flags & MLD_EARLY_TERM) != 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return msg_dtype == MLD_MSG_F16
               ? mld::run_decode_f16(&d, llr, nullptr, syndrome, batch, max_iters, et, bits_out, post_out,
                                    converged, iters_used, st, true)
               : mld::run_decode_f32(&d, llr, nullptr, syndrome, batch, max_iters, et, bits_out, post_out,
                                   converged, iters_used, st, true);
}
