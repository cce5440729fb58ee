// Uneven batches: many codewords over several Tanner graphs (different
// rates and lengths), each group with its own iteration cap, decoded by one
// schedule of launches that is captured once into a CUDA graph and replayed
// with a single launch.
//
// The paper decodes a batch of codewords of one code with a fixed number of
// iterations (Results, "High speed error correction with MET-LDPC codes";
// Discussion).  Here every launch of the schedule covers the work of all
// jobs that share its kernel shape: a device table of segments (job, block
// range) tells each block which job, slab and check class it serves.  With
// early termination (Methods, Step 5) each codeword stops at its first
// syndrome match; its slab is skipped once all its codewords have stopped.
#include <map>
#include <tuple>

#include "kernels.cuh"

namespace {

// Everything a block needs to know about one job, resident in device memory.
struct JobDev {
    CnArgs cn;
    VnArgs vn;
    SynArgs sy;
    InArgs in;
    OutArgs out;
    const uint8_t *syn;
    const int32_t *cint;
    uint8_t *sbits;
    uint32_t *done, *fail;   // fail: two buffers of slabs*DW words (iteration parity)
    int32_t *iters;
    uint8_t *conv;
    int32_t n_vn, n_cn, batch, slabs, W;
};

// One job's share of a launch: blocks block0 .. block0 + bps*slabs - 1.
struct Seg {
    int32_t job, block0, bps, slabs, flags;
    ClassLaunch cl;
};

__device__ __forceinline__ int find_seg(const Seg *segs, int nseg) {
    int k = 0;
    while (k + 1 < nseg && static_cast<int32_t>(blockIdx.x) >= segs[k + 1].block0) ++k;
    return k;
}

// Check arguments of job j at iteration l: the degree-1 decision buffer of
// l's parity, and for the fused syndrome check (seg flag 2, l >= 2) the
// buffers of iteration l-1.
template <int W>
__device__ __forceinline__ CnArgs job_cn(const JobDev &j, const Seg &sg, int32_t l) {
    constexpr int DW = (W + 31) / 32;
    CnArgs a = j.cn;
    a.final_pass = sg.flags & 1;
    const size_t h1 = static_cast<size_t>(j.slabs) * a.n_deg1 * (W / 8);
    a.hb1 = j.cn.hb1 + static_cast<size_t>(l & 1) * h1;
    a.hb1_prev = j.cn.hb1 + static_cast<size_t>((l - 1) & 1) * h1;
    a.fail_prev = j.fail + static_cast<size_t>((l - 1) & 1) * j.slabs * DW;
    a.fuse = ((sg.flags & 2) && l >= 2) ? 1 : 0;
    return a;
}

// The decisions-only form (with the fused syndrome) runs 7 blocks per SM:
// at 8 its posterior-sign bookkeeping spills.
template <typename MsgT, int W, int DC, int DD, bool HARD1>
__global__ void __launch_bounds__(kBlock, (DC + DD <= 6 ? (HARD1 ? 7 : 8) : 6))
    km_check(const JobDev *jobs, const Seg *segs, int nseg, int32_t l) {
    const Seg sg = segs[find_seg(segs, nseg)];
    const CnArgs a = job_cn<W>(jobs[sg.job], sg, l);
    const int local = blockIdx.x - sg.block0;
    const int slab = local / sg.bps;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    // the segment's grid is capped for looped classes (build_plan)
    check_class_body<MsgT, W, DC, DD, HARD1>(a, sg.cl, static_cast<int64_t>(local % sg.bps) * blockDim.x + threadIdx.x,
                                             sg.bps, slab);
}

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) km_check_irregular(const JobDev *jobs, const Seg *segs, int nseg,
                                                             int32_t l) {
    const Seg sg = segs[find_seg(segs, nseg)];
    const CnArgs a = job_cn<W>(jobs[sg.job], sg, l);
    const int local = blockIdx.x - sg.block0;
    const int slab = local / sg.bps;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    check_irregular<MsgT, W>(a, sg.cl, static_cast<int64_t>(local % sg.bps) * blockDim.x + threadIdx.x, slab);
}

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) km_var(const JobDev *jobs, const Seg *segs, int nseg) {
    const Seg sg = segs[find_seg(segs, nseg)];
    VnArgs a = jobs[sg.job].vn;
    a.want_bits = sg.flags & 1;
    const int local = blockIdx.x - sg.block0;
    const int slab = local / sg.bps;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    var_body<MsgT, W>(a, static_cast<int64_t>(local % sg.bps) * blockDim.x + threadIdx.x, slab);
}

// parity: which of the two fail buffers this iteration uses
template <int W>
__global__ void __launch_bounds__(kBlock) km_syndrome(const JobDev *jobs, const Seg *segs, int nseg, int parity) {
    constexpr int DW = (W + 31) / 32;
    const Seg sg = segs[find_seg(segs, nseg)];
    const JobDev &j = jobs[sg.job];
    SynArgs a = j.sy;
    a.fail = j.fail + parity * j.slabs * DW;
    a.hb1 = j.sy.hb1 + static_cast<size_t>(parity) * j.slabs * a.n_deg1 * (W / 8);
    const int local = blockIdx.x - sg.block0;
    const int slab = local / sg.bps;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    syndrome_body<W>(a, static_cast<int64_t>(local % sg.bps) * blockDim.x + threadIdx.x,
                     static_cast<int64_t>(sg.bps) * blockDim.x, slab);
}

// Reads this iteration's fail words and clears the other buffer for the next.
template <int W>
__global__ void __launch_bounds__(kBlock) km_lane(const JobDev *jobs, const Seg *segs, int nseg, int32_t l,
                                                  int parity) {
    constexpr int DW = (W + 31) / 32;
    const Seg sg = segs[find_seg(segs, nseg)];
    const JobDev &j = jobs[sg.job];
    const int t = (blockIdx.x - sg.block0) * blockDim.x + threadIdx.x;
    lane_body<W>(j.done, j.fail + parity * j.slabs * DW, j.iters, j.conv, j.batch, l, j.cn.et, t);
    if (t < j.slabs * DW) j.fail[(1 - parity) * j.slabs * DW + t] = 0u;
}

template <int W, int F>
__global__ void __launch_bounds__(kBlock) km_interleave(const JobDev *jobs, const Seg *segs, int nseg) {
    const Seg sg = segs[find_seg(segs, nseg)];
    const int local = blockIdx.x - sg.block0;
    interleave_body<W, F>(jobs[sg.job].in, local % sg.bps, local / sg.bps);
}

template <int W>
__global__ void __launch_bounds__(kBlock) km_syndrome_in(const JobDev *jobs, const Seg *segs, int nseg) {
    const Seg sg = segs[find_seg(segs, nseg)];
    const JobDev &j = jobs[sg.job];
    const int local = blockIdx.x - sg.block0;
    syndrome_in_body<W>(j.syn, j.cint, j.n_cn, j.batch, j.sbits, local % sg.bps, local / sg.bps);
}

template <int W>
__global__ void __launch_bounds__(kBlock) km_deinterleave(const JobDev *jobs, const Seg *segs, int nseg) {
    const Seg sg = segs[find_seg(segs, nseg)];
    const int local = blockIdx.x - sg.block0;
    deinterleave_body<W>(jobs[sg.job].out, local % sg.bps, local / sg.bps);
}

// ---------------------------------------------------------------------------
// schedule
// ---------------------------------------------------------------------------
enum OpKind { kOpMemset, kOpInterleave, kOpSynIn, kOpHard, kOpCheck, kOpVar, kOpSyn, kOpLane, kOpOut };

struct Op {
    int kind = 0, half = 0, W = 0, dc = 0, dd = 0, parity = 0;
    int hard1 = 0;  // check ops: degree-1 decisions only
    int32_t l = 0;
    int seg0 = 0, nseg = 0, blocks = 0;
    // memset / hard-decision ops
    void *ptr = nullptr;
    size_t bytes = 0;
    const float *post = nullptr;
    int32_t count = 0;
    uint8_t *hb = nullptr;
    int slabs = 0;
};

}  // namespace

struct mld_plan {
    int device = 0;
    JobDev *d_jobs = nullptr;
    Seg *d_segs = nullptr;
    std::vector<Op> ops;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

int width_index(int W) { return W == 8 ? 0 : (W == 16 ? 1 : (W == 32 ? 2 : 3)); }

template <typename MsgT, int W>
void launch_check_op(const mld_plan *p, const Op &op, cudaStream_t st) {
    const JobDev *J = p->d_jobs;
    const Seg *S = p->d_segs + op.seg0;
#define MLD_CASE(DCV, DDV)                                                                          \
    if (op.dc == (DCV) && op.dd == (DDV)) {                                                         \
        if (op.hard1) km_check<MsgT, W, DCV, DDV, true><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg, op.l); \
        else km_check<MsgT, W, DCV, DDV, false><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg, op.l);      \
        return;                                                                                     \
    }
    MLD_CASE(1, 0) MLD_CASE(2, 0) MLD_CASE(3, 0) MLD_CASE(4, 0)
    MLD_CASE(5, 0) MLD_CASE(6, 0) MLD_CASE(7, 0) MLD_CASE(8, 0)
    MLD_CASE(0, 1) MLD_CASE(1, 1) MLD_CASE(2, 1) MLD_CASE(3, 1)
    MLD_CASE(4, 1) MLD_CASE(5, 1) MLD_CASE(6, 1) MLD_CASE(7, 1)
#undef MLD_CASE
    km_check_irregular<MsgT, W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg, op.l);
}

template <int W>
void launch_op_w(const mld_plan *p, const Op &op, cudaStream_t st) {
    const JobDev *J = p->d_jobs;
    const Seg *S = p->d_segs + op.seg0;
    switch (op.kind) {
        case kOpInterleave:
            if (op.half) km_interleave<W, kFitB2H><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg);
            else km_interleave<W, kFitB2><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg);
            break;
        case kOpSynIn: km_syndrome_in<W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg); break;
        case kOpHard:
            k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(op.count) * (W / 8)), op.slabs), kBlock, 0, st>>>(
                op.post, op.count, op.hb);
            break;
        case kOpCheck:
            if (op.half) launch_check_op<__half, W>(p, op, st);
            else launch_check_op<float, W>(p, op, st);
            break;
        case kOpVar:
            if (op.half) km_var<__half, W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg);
            else km_var<float, W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg);
            break;
        case kOpSyn: km_syndrome<W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg, op.parity); break;
        case kOpLane: km_lane<W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg, op.l, op.parity); break;
        case kOpOut: km_deinterleave<W><<<op.blocks, kBlock, 0, st>>>(J, S, op.nseg); break;
        default: break;
    }
}

int enqueue(const mld_plan *p, cudaStream_t st) {
    for (const Op &op : p->ops) {
        if (op.kind == kOpMemset) {
            MLD_CUDA(cudaMemsetAsync(op.ptr, 0, op.bytes, st));
            continue;
        }
        switch (op.W) {
            case 8: launch_op_w<8>(p, op, st); break;
            case 16: launch_op_w<16>(p, op, st); break;
            case 32: launch_op_w<32>(p, op, st); break;
            default: launch_op_w<64>(p, op, st); break;
        }
        MLD_LAUNCHED("multi-job kernel");
    }
    return MLD_OK;
}

void plan_free(mld_plan *p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    dfree(p->d_jobs);
    dfree(p->d_segs);
    delete p;
}

// Builds the jobs' device descriptors and the launch schedule.
int build_plan(const mld_job *jobs, int32_t n_jobs, uint32_t flags, mld_plan *p,
               std::vector<JobDev> &jd, std::vector<Seg> &segs) {
    const bool et = (flags & MLD_EARLY_TERM) != 0;
    int sm_count = 152;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, p->device);
    int32_t lmax_iters = 0;
    for (int32_t j = 0; j < n_jobs; ++j) {
        const mld_job &jb = jobs[j];
        mld_decoder *d = jb.decoder;
        const mld::HostGraph &h = d->g->h;
        const int W = d->W;
        const int slabs = (jb.batch + W - 1) / W;
        JobDev x{};
        const bool y_mode = jb.sigma != nullptr;
        x.cn = CnArgs{d->g->cptr, d->g->col, d->g->dptr, h.n_cn, h.n_core, h.n_deg1, h.e_core, d->r, d->Lv,
                      d->lch1, d->phi1, d->post1, d->hb1, d->sbits, d->done, d->lmax_i, d->amin_i, 0, et ? 1 : 0,
                      0, jb.batch, d->hb1, d->fail};
        x.vn = VnArgs{d->g->vptr, d->g->vedge, h.n_core, h.e_core, d->r, d->lch, d->Lv, d->hb_core, d->done, 0,
                      et ? 1 : 0};
        x.sy = SynArgs{d->g->cptr, d->g->col, d->g->dptr, h.n_cn, h.n_core, h.n_deg1, d->sbits, d->hb_core,
                       d->hb1, d->fail, d->done, et ? 1 : 0, jb.batch};
        x.in = InArgs{jb.in, y_mode ? jb.sigma : nullptr, d->g->unit, h.n_vn, h.n_core, h.n_deg1, jb.batch,
                      d->lmax, d->scale_in, d->lmax_i, d->amin_i, d->lch, d->Lv, d->lch1, d->post1, d->phi1};
        x.out = OutArgs{d->g->unit, h.n_vn, h.n_core, h.n_deg1, jb.batch, d->Lv, d->post1, d->hb1, jb.iters_used,
                        static_cast<size_t>(slabs) * h.n_deg1 * (W / 8), jb.bits_out,
                        jb.post_out, d->scale_out};
        x.syn = jb.syndrome;
        x.cint = d->g->cint;
        x.sbits = d->sbits;
        x.done = d->done;
        x.fail = d->fail;
        x.iters = jb.iters_used;
        x.conv = jb.converged;
        x.n_vn = h.n_vn;
        x.n_cn = h.n_cn;
        x.batch = jb.batch;
        x.slabs = slabs;
        x.W = W;
        jd.push_back(x);
        lmax_iters = std::max(lmax_iters, jb.max_iters);
    }

    // one op per group key; segments of the group are the jobs' shares
    using Key = std::tuple<int, int, int, int, int, int>;  // kind, half, W, dc, dd, hard1
    auto flush = [&](std::map<Key, std::vector<Seg>> &groups, int32_t l, int parity) {
        for (auto &kv : groups) {
            Op op;
            op.kind = std::get<0>(kv.first);
            op.half = std::get<1>(kv.first);
            op.W = std::get<2>(kv.first);
            op.dc = std::get<3>(kv.first);
            op.dd = std::get<4>(kv.first);
            op.hard1 = std::get<5>(kv.first);
            op.l = l;
            op.parity = parity;
            op.seg0 = static_cast<int>(segs.size());
            op.nseg = static_cast<int>(kv.second.size());
            int32_t b0 = 0;
            for (Seg s : kv.second) {
                s.block0 = b0;
                b0 += s.bps * s.slabs;
                segs.push_back(s);
            }
            op.blocks = b0;
            if (op.blocks > 0) p->ops.push_back(op);
            else segs.resize(op.seg0);
        }
        groups.clear();
    };
    auto seg = [](int32_t job, int32_t bps, int32_t slabs, int32_t fl) {
        Seg s{};
        s.job = job;
        s.bps = bps;
        s.slabs = slabs;
        s.flags = fl;
        return s;
    };
    std::map<Key, std::vector<Seg>> groups;

    // prologue: clear messages and per-codeword state, interleave inputs
    for (int32_t j = 0; j < n_jobs; ++j) {
        const mld_decoder *d = jobs[j].decoder;
        const mld::HostGraph &h = d->g->h;
        const size_t msz = d->msg == MLD_MSG_F16 ? 2 : 4;
        const size_t DW = (d->W + 31) / 32;
        Op m;
        m.kind = kOpMemset;
        m.ptr = d->r;
        m.bytes = static_cast<size_t>(jd[j].slabs) * h.e_core * d->W * msz;
        if (m.bytes) p->ops.push_back(m);
        m.ptr = d->done;
        m.bytes = sizeof(uint32_t) * jd[j].slabs * DW;
        p->ops.push_back(m);
        m.ptr = d->fail;
        m.bytes = 2 * sizeof(uint32_t) * jd[j].slabs * DW;
        p->ops.push_back(m);
    }
    for (int32_t j = 0; j < n_jobs; ++j) {
        const mld_decoder *d = jobs[j].decoder;
        const int half = d->msg == MLD_MSG_F16;
        if (jd[j].n_vn > 0)
            groups[Key{kOpInterleave, half, d->W, 0, 0, 0}].push_back(seg(j, (jd[j].n_vn + 31) / 32, jd[j].slabs, 0));
        if (jd[j].n_cn > 0)
            groups[Key{kOpSynIn, 0, d->W, 0, 0, 0}].push_back(seg(j, (jd[j].n_cn + 31) / 32, jd[j].slabs, 0));
    }
    flush(groups, 0, 0);

    auto syndrome_round = [&](const std::vector<int32_t> &js, int32_t l) {
        const int parity = l & 1;
        for (int32_t j : js) {
            const mld_decoder *d = jobs[j].decoder;
            const int bps = syndrome_blocks(jd[j].n_cn, sm_count);
            if (jd[j].n_cn > 0) groups[Key{kOpSyn, 0, d->W, 0, 0, 0}].push_back(seg(j, bps, jd[j].slabs, 0));
        }
        flush(groups, l, parity);
        for (int32_t j : js) {
            const mld_decoder *d = jobs[j].decoder;
            const int lanes = std::max(jd[j].batch, jd[j].slabs * ((d->W + 31) / 32));
            groups[Key{kOpLane, 0, d->W, 0, 0, 0}].push_back(seg(j, (lanes + kBlock - 1) / kBlock, 1, 0));
        }
        flush(groups, l, parity);
    };

    // jobs with no iteration: decisions from the channel values
    {
        std::vector<int32_t> zero;
        for (int32_t j = 0; j < n_jobs; ++j) {
            if (jobs[j].max_iters != 0) continue;
            mld_decoder *d = jobs[j].decoder;
            const mld::HostGraph &h = d->g->h;
            Op op;
            op.kind = kOpHard;
            op.W = d->W;
            op.slabs = jd[j].slabs;
            if (h.n_core > 0) {
                op.post = d->Lv;
                op.count = h.n_core;
                op.hb = d->hb_core;
                p->ops.push_back(op);
            }
            if (h.n_deg1 > 0) {
                op.post = d->post1;
                op.count = h.n_deg1;
                op.hb = d->hb1;
                p->ops.push_back(op);
            }
            zero.push_back(j);
        }
        if (!zero.empty()) syndrome_round(zero, 0);
    }

    // early termination without soft output: degree-1 decisions only, and for
    // graphs whose checks are all in register classes the syndrome of
    // iteration l-1 is formed inside check pass l (then only the last
    // iteration gets a separate syndrome check)
    auto hard1_job = [&](int32_t j) { return et && !jobs[j].post_out; };
    auto fused_job = [&](int32_t j) { return hard1_job(j) && jobs[j].decoder->g->fusable; };
    for (int32_t l = 1; l <= lmax_iters; ++l) {
        std::vector<int32_t> active, checked, lanes;
        for (int32_t j = 0; j < n_jobs; ++j)
            if (jobs[j].max_iters >= l) active.push_back(j);
        for (int32_t j : active) {
            const mld_decoder *d = jobs[j].decoder;
            const int half = d->msg == MLD_MSG_F16;
            const int fl = ((et || l == jobs[j].max_iters) ? 1 : 0) | (fused_job(j) ? 2 : 0);
            for (const ClassLaunch &cl : d->g->launches[width_index(d->W)]) {
                const int dd = cl.deg - cl.dc;
                const bool regular = cl.dc >= 0 && (dd == 0 || dd == 1);
                // looped register classes (at most 6 terms) run on a capped
                // grid of two waves (7 blocks per SM for the decisions-only form)
                const bool looped = regular && cl.deg <= 6;
                const int hard1 = (hard1_job(j) && regular) ? 1 : 0;
                const int cap = sm_count * (hard1 ? 14 : 16);
                Seg s = seg(j, looped ? std::max(1, std::min(cl.blocks, cap)) : cl.blocks, jd[j].slabs, fl);
                s.cl = cl;
                groups[Key{kOpCheck, half, d->W, regular ? cl.dc : -1, regular ? dd : -1, hard1}].push_back(s);
            }
            if (fused_job(j) && l >= 2) lanes.push_back(j);
        }
        flush(groups, l, 0);
        // the codewords of fused jobs whose iteration l-1 satisfied every check
        // stop there (the lane op also clears the other fail buffer)
        if (!lanes.empty()) {
            for (int32_t j : lanes) {
                const mld_decoder *d = jobs[j].decoder;
                const int nl = std::max(jd[j].batch, jd[j].slabs * ((d->W + 31) / 32));
                groups[Key{kOpLane, 0, d->W, 0, 0, 0}].push_back(seg(j, (nl + kBlock - 1) / kBlock, 1, 0));
            }
            flush(groups, l - 1, (l - 1) & 1);
        }
        for (int32_t j : active) {
            const mld_decoder *d = jobs[j].decoder;
            const int half = d->msg == MLD_MSG_F16;
            const int fl = (et || l == jobs[j].max_iters) ? 1 : 0;
            const int tpc = d->W / kK;
            const int bps = grid_x(static_cast<int64_t>(d->g->h.n_core) * tpc);
            if (d->g->h.n_core > 0) groups[Key{kOpVar, half, d->W, 0, 0, 0}].push_back(seg(j, bps, jd[j].slabs, fl));
            if (fl && (!fused_job(j) || l == jobs[j].max_iters)) checked.push_back(j);
        }
        flush(groups, l, 0);
        if (!checked.empty()) syndrome_round(checked, l);
    }

    for (int32_t j = 0; j < n_jobs; ++j)
        if (jd[j].n_vn > 0)
            groups[Key{kOpOut, 0, jobs[j].decoder->W, 0, 0, 0}].push_back(seg(j, (jd[j].n_vn + 31) / 32, jd[j].slabs, 0));
    flush(groups, 0, 0);
    return MLD_OK;
}

int validate_jobs(const mld_job *jobs, int32_t n_jobs, uint32_t flags, int *device) {
    if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return mld::fail(MLD_EINVAL, "plan: bad job list");
    if (flags & ~(MLD_EARLY_TERM | MLD_DEVICE_PTRS)) return mld::fail(MLD_EINVAL, "plan: unknown flag");
    int dev = -1;
    MLD_CUDA(cudaGetDevice(&dev));
    *device = dev;
    for (int32_t j = 0; j < n_jobs; ++j) {
        const mld_job &jb = jobs[j];
        const std::string at = "plan: job " + std::to_string(j) + ": ";
        if (!jb.decoder) return mld::fail(MLD_EINVAL, at + "null decoder");
        if (jb.decoder->device != dev) return mld::fail(MLD_EINVAL, at + "decoder belongs to another device");
        if (jb.batch < 1 || jb.batch > jb.decoder->max_batch) return mld::fail(MLD_EINVAL, at + "batch out of range");
        if (jb.max_iters < 0) return mld::fail(MLD_EINVAL, at + "negative max_iters");
        if (jb.decoder->schedule != MLD_SCHED_FLOODING || jb.decoder->check_rule != MLD_CHECK_SUM_PRODUCT)
            return mld::fail(MLD_EINVAL, at + "plans run flooding sum-product (layered or min-sum decoder given)");
        const mld::HostGraph &h = jb.decoder->g->h;
        if ((h.n_vn > 0 && (!jb.in || !jb.bits_out)) || (h.n_cn > 0 && !jb.syndrome) || !jb.converged ||
            !jb.iters_used)
            return mld::fail(MLD_EINVAL, at + "null data pointer");
        for (int32_t k = 0; k < j; ++k)
            if (jobs[k].decoder == jb.decoder) return mld::fail(MLD_EINVAL, at + "decoder shared with job " + std::to_string(k));
    }
    return MLD_OK;
}

}  // namespace

extern "C" {

int mld_plan_create(const mld_job *jobs, int32_t n_jobs, uint32_t flags, mld_plan **out) {
    mld::clear_error();
    if (!out) return mld::fail(MLD_EINVAL, "plan_create: null out");
    int dev = 0;
    int s = validate_jobs(jobs, n_jobs, flags, &dev);
    if (s != MLD_OK) return s;
    mld_plan *p = new (std::nothrow) mld_plan();
    if (!p) return mld::fail(MLD_ENOMEM, "plan_create: host allocation");
    p->device = dev;
    std::vector<JobDev> jd;
    std::vector<Seg> segs;
    s = build_plan(jobs, n_jobs, flags, p, jd, segs);
    if (s == MLD_OK) s = upload(&p->d_jobs, jd);
    if (s == MLD_OK) s = upload(&p->d_segs, segs);
    cudaStream_t cs = nullptr;
    if (s == MLD_OK) {
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamCreate");
    }
    if (s == MLD_OK) {
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamBeginCapture");
        if (s == MLD_OK) {
            const int es = enqueue(p, cs);
            e = cudaStreamEndCapture(cs, &p->graph);
            if (es != MLD_OK) s = es;
            else if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamEndCapture");
        }
    }
    if (s == MLD_OK) {
        cudaError_t e = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (e != cudaSuccess) s = cuda_fail(e, "cudaGraphInstantiate");
    }
    if (cs) cudaStreamDestroy(cs);
    if (s != MLD_OK) {
        plan_free(p);
        return s;
    }
    *out = p;
    return MLD_OK;
}

int mld_plan_launch(mld_plan *p, void *stream) {
    mld::clear_error();
    if (!p) return mld::fail(MLD_EINVAL, "plan_launch: null plan");
    int s = check_device(p->device);
    if (s != MLD_OK) return s;
    MLD_CUDA(cudaGraphLaunch(p->exec, static_cast<cudaStream_t>(stream)));
    return MLD_OK;
}

int mld_plan_stats(const mld_plan *p, int64_t *launches) {
    mld::clear_error();
    if (!p || !launches) return mld::fail(MLD_EINVAL, "plan_stats: null pointer");
    int64_t n = 0;
    for (const Op &op : p->ops) n += (op.kind == kOpMemset) ? 0 : 1;
    *launches = n;
    return MLD_OK;
}

int mld_plan_destroy(mld_plan *p) {
    if (!p) return MLD_OK;
    plan_free(p);
    return MLD_OK;
}

int mld_decode_multi(const mld_job *jobs, int32_t n_jobs, uint32_t flags, void *stream) {
    mld::clear_error();
    mld_plan *p = nullptr;
    int s = mld_plan_create(jobs, n_jobs, flags, &p);
    if (s != MLD_OK) return s;
    s = mld_plan_launch(p, stream);
    if (s == MLD_OK) {
        cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) s = cuda_fail(e, "cudaStreamSynchronize");
    }
    plan_free(p);
    return s;
}

}  // extern "C"
