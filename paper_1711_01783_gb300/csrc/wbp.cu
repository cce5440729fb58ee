// Differentiable weighted BP: forward over T unrolled iterations with a
// learnable scale per (iteration, edge type) on every variable-to-check
// message, and its adjoint (reverse mode), checkpointed every k iterations.
//
// Forward (LLR domain, Methods Eqs. 2-5, with weights):
//   x_e^t = L_v^{t-1} - r_e^{t-1}     (degree-1 VN: x = L_ch)
//   q_e^t = clamp(w[t][type(e)] * x_e^t)
//   r_e^t = check update of the q^t (syndrome sign, phi, clamps)
//   L_v^t = L_ch(v) + sum_e r_e^t;   output L^T.
// All weights 1 is plain BP.  The adjoint differentiates every step exactly
// (clamps: 1 strictly inside, 0 outside; sign factors: 0; phi' = -1/sinh),
// recomputing each segment of k iterations from its stored messages.
#include "kernels.cuh"

namespace {

constexpr int kMaxTerms = 16;  // check degree supported by weighted BP
constexpr int kMaxTypes = MLD_MAX_EDGE_TYPES;

struct WArgs {
    const int32_t *cptr, *col, *dptr, *vptr, *vedge;
    const uint8_t *et_core, *et_deg1;
    int32_t n_cn, n_core, n_deg1, e_core, n_types;
    const uint8_t *sbits;
    const float *lch, *lch1;   // interleaved channel LLRs (clamped)
    const float *w;            // [T][n_types] weights, device
    float lmax, amin;
};

__device__ __forceinline__ float inv_sinh(float x) { return 1.0f / sinhf(x); }

// Recomputes the forward quantities of one check (at most DMAX terms) for 4
// codewords at iteration t from r^{t-1} (rp) and L_v^{t-1} (lvp).  Loops run
// to DMAX with the check's degree as a guard, so the arrays stay in
// registers for small DMAX.
template <int W, int DMAX>
struct CheckState {
    int nce, deg;
    int32_t e0, s0;
    float x[DMAX][kK], q[DMAX][kK], f[DMAX][kK], pre[DMAX][kK];
    float wt[DMAX];
    int ty[DMAX];
    float sg[kK];  // product of signs and syndrome sign over all terms

    __device__ __forceinline__ void load(const WArgs &a, int c, int slab, int lane0, int t, const float *rp,
                                         const float *lvp) {
        constexpr int NB = W / 8;
        e0 = a.cptr[c];
        nce = a.cptr[c + 1] - e0;
        s0 = a.dptr[c];
        deg = nce + (a.dptr[c + 1] - s0);
        const uint32_t sb =
            (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >> (lane0 & 7));
        const float *wt_row = a.w + static_cast<size_t>(t - 1) * a.n_types;
#pragma unroll
        for (int k = 0; k < kK; ++k) sg[k] = ((sb >> k) & 1u) ? -1.f : 1.f;
        float acc[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            if (i >= deg) continue;
            float4 xv;
            if (i < nce) {
                const int32_t e = e0 + i;
                const float4 lv = ldf4(lvp + (static_cast<size_t>(slab) * a.n_core + a.col[e]) * W + lane0);
                const float4 ro = ldf4(rp + (static_cast<size_t>(slab) * a.e_core + e) * W + lane0);
                xv = make_float4(lv.x - ro.x, lv.y - ro.y, lv.z - ro.z, lv.w - ro.w);
                ty[i] = a.et_core[e];
            } else {
                const int32_t sl = s0 + i - nce;
                xv = ldf4(a.lch1 + (static_cast<size_t>(slab) * a.n_deg1 + sl) * W + lane0);
                ty[i] = a.et_deg1[sl];
            }
            wt[i] = wt_row[ty[i]];
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                x[i][k] = f4get(xv, k);
                q[i][k] = clampf(wt[i] * x[i][k], -a.lmax, a.lmax);
                f[i][k] = phi_f<kFitNat>(clampf(fabsf(q[i][k]), a.amin, a.lmax));
                if (q[i][k] < 0.f) sg[k] = -sg[k];
                pre[i][k] = acc[k];
                acc[k] += f[i][k];
            }
        }
    }
};

// Forward check update of iteration t for checks c0 .. c0+count-1 of at most
// DMAX terms (messages updated in place; degree-1 posteriors written when
// `last`).  The loops run to the compile-time DMAX with the check's degree
// as a guard, so the per-term arrays stay in registers for small DMAX.
template <int W, int DMAX>
__global__ void __launch_bounds__(kBlock) kw_check_fwd(WArgs a, float *r, const float *lv, float *post1, int t,
                                                       int last, int32_t c0, int32_t count) {
    constexpr int TPC = W / kK;
    constexpr int NB = W / 8;
    const int slab = blockIdx.y;
    const int64_t lt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (lt / TPC >= count) return;
    const int32_t c = c0 + static_cast<int32_t>(lt / TPC);
    const int lane0 = static_cast<int>(lt % TPC) * kK;
    const int32_t e0 = a.cptr[c], nce = a.cptr[c + 1] - e0;
    const int32_t s0 = a.dptr[c], deg = nce + (a.dptr[c + 1] - s0);
    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >> (lane0 & 7));
    const float *wt_row = a.w + static_cast<size_t>(t - 1) * a.n_types;
    float sg[kK], q[DMAX][kK], f[DMAX][kK], pre[DMAX][kK];
#pragma unroll
    for (int k = 0; k < kK; ++k) sg[k] = ((sb >> k) & 1u) ? -1.f : 1.f;
    float acc[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < DMAX; ++i) {
        if (i < deg) {
            float4 xv;
            float wt;
            if (i < nce) {
                const int32_t e = e0 + i;
                const float4 l = ldf4(lv + (static_cast<size_t>(slab) * a.n_core + a.col[e]) * W + lane0);
                const float4 ro = ldf4(r + (static_cast<size_t>(slab) * a.e_core + e) * W + lane0);
                xv = make_float4(l.x - ro.x, l.y - ro.y, l.z - ro.z, l.w - ro.w);
                wt = wt_row[a.et_core[e]];
            } else {
                const int32_t sl = s0 + i - nce;
                xv = ldf4(a.lch1 + (static_cast<size_t>(slab) * a.n_deg1 + sl) * W + lane0);
                wt = wt_row[a.et_deg1[sl]];
            }
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                q[i][k] = clampf(wt * f4get(xv, k), -a.lmax, a.lmax);
                f[i][k] = phi_f<kFitNat>(clampf(fabsf(q[i][k]), a.amin, a.lmax));
                if (q[i][k] < 0.f) sg[k] = -sg[k];
                pre[i][k] = acc[k];
                acc[k] += f[i][k];
            }
        }
    }
    float suf[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = DMAX - 1; i >= 0; --i) {
        if (i >= deg) continue;
        const bool core = i < nce;
        if (core || last) {
            float4 rv;
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                const float o = clampf(pre[i][k] + suf[k], a.amin, a.lmax);
                const float m = fminf(phi_f<kFitNat>(o), a.lmax);
                const float sgn = (q[i][k] < 0.f) ? -sg[k] : sg[k];  // sign of the other terms
                f4set(rv, k, sgn * m);
            }
            if (core) {
                *reinterpret_cast<float4 *>(r + (static_cast<size_t>(slab) * a.e_core + e0 + i) * W + lane0) = rv;
            } else {
                const size_t o = (static_cast<size_t>(slab) * a.n_deg1 + s0 + i - nce) * W + lane0;
                const float4 l = ldf4(a.lch1 + o);
                *reinterpret_cast<float4 *>(post1 + o) = make_float4(l.x + rv.x, l.y + rv.y, l.z + rv.z, l.w + rv.w);
            }
        }
#pragma unroll
        for (int k = 0; k < kK; ++k) suf[k] += f[i][k];
    }
}

// Forward check update of one class: DMAX = the class's degree (at most
// kMaxRegDeg), or kMaxTerms for the irregular class.
template <int W>
void launch_check_fwd(const WArgs &wa, const mld::ClassLaunch &cl, float *r, const float *lv, float *post1, int t,
                      int last, int slabs, cudaStream_t st) {
    const dim3 grid(cl.blocks, slabs);
    switch (cl.deg) {
#define MLD_FWD(DV) \
        case DV: kw_check_fwd<W, DV><<<grid, kBlock, 0, st>>>(wa, r, lv, post1, t, last, cl.c0, cl.count); return;
        MLD_FWD(1) MLD_FWD(2) MLD_FWD(3) MLD_FWD(4) MLD_FWD(5) MLD_FWD(6) MLD_FWD(7) MLD_FWD(8)
#undef MLD_FWD
        default: kw_check_fwd<W, kMaxTerms><<<grid, kBlock, 0, st>>>(wa, r, lv, post1, t, last, cl.c0, cl.count);
    }
}

// Adjoint of the check update of iteration t.
//   gr   : dloss/dr^t for core edges (read)
//   gd1  : dloss/dr^t of degree-1 edges (only at t = T; else null)
//   gx   : dloss/dx^t for core edges (written)
//   glch1: dloss/dL_ch of degree-1 VNs (accumulated)
//   gwp  : per-block partial dloss/dw[t][type] (written, [gridDim.x*gridDim.y][n_types])
template <int W, int DMAX>
__global__ void __launch_bounds__(kBlock) kw_check_bwd(WArgs a, const float *rp, const float *lvp, const float *gr,
                                                       const float *gd1, float *gx, float *glch1, float *gwp, int t,
                                                       int32_t c0, int32_t count, int32_t part0) {
    constexpr int TPC = W / kK;
    __shared__ float red[kBlock / 32][kMaxTypes];
    const int slab = blockIdx.y;
    const int64_t lt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    float gw[kMaxTypes];
#pragma unroll
    for (int k = 0; k < kMaxTypes; ++k) gw[k] = 0.f;
    if (lt / TPC < count) {
        const int32_t c = c0 + static_cast<int32_t>(lt / TPC);
        const int lane0 = static_cast<int>(lt % TPC) * kK;
        CheckState<W, DMAX> s;
        s.load(a, c, slab, lane0, t, rp, lvp);
        // g_o_i = sign_i * g_r_i * phi'(o_i) where o_i is strictly inside the clamp
        float go[DMAX][kK];
        float suf[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = DMAX - 1; i >= 0; --i) {
            if (i >= s.deg) continue;
            const bool core = i < s.nce;
            float4 g = make_float4(0.f, 0.f, 0.f, 0.f);
            if (core)
                g = ldf4(gr + (static_cast<size_t>(slab) * a.e_core + s.e0 + i) * W + lane0);
            else if (gd1)
                g = ldf4(gd1 + (static_cast<size_t>(slab) * a.n_deg1 + s.s0 + i - s.nce) * W + lane0);
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                const float o = s.pre[i][k] + suf[k];
                const float sgn = (s.q[i][k] < 0.f) ? -s.sg[k] : s.sg[k];
                go[i][k] = (o > a.amin && o < a.lmax) ? -sgn * f4get(g, k) * inv_sinh(o) : 0.f;
                suf[k] += s.f[i][k];
            }
        }
        // g_f_j = sum_{i != j} g_o_i (prefix + suffix), then back through phi, |.|, clamp, weight
        float gpre[DMAX][kK];
        float acc[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < DMAX; ++i) {
            if (i >= s.deg) continue;
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                gpre[i][k] = acc[k];
                acc[k] += go[i][k];
            }
        }
        float gsuf[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = DMAX - 1; i >= 0; --i) {
            if (i >= s.deg) continue;
            float gxd[kK];
            float gwi = 0.f;  // this term's weight gradient over the 4 codewords
#pragma unroll
            for (int k = 0; k < kK; ++k) {
                const float gf = gpre[i][k] + gsuf[k];
                gsuf[k] += go[i][k];
                const float aq = fabsf(s.q[i][k]);
                const float ga = (aq > a.amin && aq < a.lmax) ? -gf * inv_sinh(aq) : 0.f;
                const float gq = s.q[i][k] > 0.f ? ga : (s.q[i][k] < 0.f ? -ga : 0.f);
                const float p = s.wt[i] * s.x[i][k];
                const float gp = (p > -a.lmax && p < a.lmax) ? gq : 0.f;
                gwi += gp * s.x[i][k];
                gxd[k] = gp * s.wt[i];
            }
#pragma unroll
            for (int k = 0; k < kMaxTypes; ++k) gw[k] += (k == s.ty[i]) ? gwi : 0.f;
            const float4 gxv = make_float4(gxd[0], gxd[1], gxd[2], gxd[3]);
            if (i < s.nce) {
                *reinterpret_cast<float4 *>(gx + (static_cast<size_t>(slab) * a.e_core + s.e0 + i) * W + lane0) = gxv;
            } else {
                float *pp = glch1 + (static_cast<size_t>(slab) * a.n_deg1 + s.s0 + i - s.nce) * W + lane0;
                float4 o = *reinterpret_cast<float4 *>(pp);
                o.x += gxv.x; o.y += gxv.y; o.z += gxv.z; o.w += gxv.w;
                *reinterpret_cast<float4 *>(pp) = o;
            }
        }
    }
    // block partial sums of the weight gradient (deterministic order)
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int k = 0; k < a.n_types; ++k) {
        float v = gw[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < a.n_types) {
        float v = 0.f;
        for (int i = 0; i < kBlock / 32; ++i) v += red[i][threadIdx.x];
        gwp[(static_cast<size_t>(part0) + static_cast<size_t>(blockIdx.y) * gridDim.x + blockIdx.x) * a.n_types +
            threadIdx.x] = v;
    }
}

// Adjoint check update of one class; its block partials start at part0.
template <int W>
void launch_check_bwd(const WArgs &wa, const mld::ClassLaunch &cl, const float *rp, const float *lvp,
                      const float *gr, const float *gd1, float *gx, float *glch1, float *gwp, int t, int slabs,
                      int32_t part0, cudaStream_t st) {
    const dim3 grid(cl.blocks, slabs);
    switch (cl.deg) {
#define MLD_BWD(DV)                                                                                         \
        case DV:                                                                                            \
            kw_check_bwd<W, DV><<<grid, kBlock, 0, st>>>(wa, rp, lvp, gr, gd1, gx, glch1, gwp, t, cl.c0,    \
                                                         cl.count, part0);                                  \
            return;
        MLD_BWD(1) MLD_BWD(2) MLD_BWD(3) MLD_BWD(4) MLD_BWD(5) MLD_BWD(6) MLD_BWD(7) MLD_BWD(8)
#undef MLD_BWD
        default:
            kw_check_bwd<W, kMaxTerms><<<grid, kBlock, 0, st>>>(wa, rp, lvp, gr, gd1, gx, glch1, gwp, t, cl.c0,
                                                                cl.count, part0);
    }
}

// Adjoint of x_e^t = L_ch(v) + sum_{e' != e} r_{e'}^{t-1} at core VN v:
// G = sum_e gx_e; dL_ch += G; dr_{e'}^{t-1} = G - gx_{e'} (when t > 1).
template <int W>
__global__ void __launch_bounds__(kBlock) kw_var_bwd(WArgs a, const float *gx, float *glch, float *gr_prev) {
    constexpr int TPC = W / kK;
    const int slab = blockIdx.y;
    const int64_t lt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int32_t v = static_cast<int32_t>(lt / TPC);
    if (v >= a.n_core) return;
    const int lane0 = static_cast<int>(lt % TPC) * kK;
    const size_t ebase = static_cast<size_t>(slab) * a.e_core;
    float4 G = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int32_t j = a.vptr[v]; j < a.vptr[v + 1]; ++j) {
        const float4 g = ldf4(gx + (ebase + a.vedge[j]) * W + lane0);
        G.x += g.x; G.y += g.y; G.z += g.z; G.w += g.w;
    }
    float *gl = glch + (static_cast<size_t>(slab) * a.n_core + v) * W + lane0;
    float4 o = *reinterpret_cast<float4 *>(gl);
    o.x += G.x; o.y += G.y; o.z += G.z; o.w += G.w;
    *reinterpret_cast<float4 *>(gl) = o;
    if (gr_prev) {
        for (int32_t j = a.vptr[v]; j < a.vptr[v + 1]; ++j) {
            const size_t idx = (ebase + a.vedge[j]) * W + lane0;
            const float4 g = ldf4(gx + idx);
            *reinterpret_cast<float4 *>(gr_prev + idx) = make_float4(G.x - g.x, G.y - g.y, G.z - g.z, G.w - g.w);
        }
    }
}

// dloss/dr^T of core edge e = dloss/dL_v(e) (the posterior is L_ch + sum r^T).
template <int W>
__global__ void __launch_bounds__(kBlock) kw_grad_edges(WArgs a, const float *gl_core, float *gr) {
    constexpr int TPC = W / kK;
    const int slab = blockIdx.y;
    const int64_t lt = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int32_t v = static_cast<int32_t>(lt / TPC);
    if (v >= a.n_core) return;
    const int lane0 = static_cast<int>(lt % TPC) * kK;
    const float4 g = ldf4(gl_core + (static_cast<size_t>(slab) * a.n_core + v) * W + lane0);
    for (int32_t j = a.vptr[v]; j < a.vptr[v + 1]; ++j)
        *reinterpret_cast<float4 *>(gr + ((static_cast<size_t>(slab) * a.e_core + a.vedge[j]) * W + lane0)) = g;
}

// Natural [B][n] -> interleaved core / degree-1 arrays (32 VNs x W codewords per block).
template <int W>
__global__ void __launch_bounds__(kBlock) kw_interleave(const float *in, const int32_t *unit, int32_t n_vn,
                                                        int32_t n_core, int32_t n_deg1, int32_t batch, float *core,
                                                        float *deg1, float *deg1_copy) {
    __shared__ float tile[W][33];
    const int slab = blockIdx.y;
    const int32_t j0 = blockIdx.x * 32;
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int w = idx / 32, jj = idx % 32;
        const int b = slab * W + w;
        const int32_t j = j0 + jj;
        tile[w][jj] = (b < batch && j < n_vn) ? in[static_cast<size_t>(b) * n_vn + j] : 0.f;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int jj = idx / W, w = idx % W;
        const int32_t j = j0 + jj;
        if (j >= n_vn) continue;
        const int32_t u = unit[j];
        const float v = tile[w][jj];
        if (u < n_core) {
            core[(static_cast<size_t>(slab) * n_core + u) * W + w] = v;
        } else {
            const size_t o = (static_cast<size_t>(slab) * n_deg1 + (u - n_core)) * W + w;
            deg1[o] = v;
            deg1_copy[o] = v;
        }
    }
}

// Interleaved gradients -> natural [B][n], zero where the input LLR was clamped.
template <int W>
__global__ void __launch_bounds__(kBlock) kw_deinterleave(const float *core, const float *deg1, const float *lch,
                                                          const float *lch1, const int32_t *unit, int32_t n_vn,
                                                          int32_t n_core, int32_t n_deg1, int32_t batch, float lmax,
                                                          float *out) {
    __shared__ float tile[32][W + 1];
    const int slab = blockIdx.y;
    const int32_t j0 = blockIdx.x * 32;
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int jj = idx / W, w = idx % W;
        const int32_t j = j0 + jj;
        float v = 0.f;
        if (j < n_vn) {
            const int32_t u = unit[j];
            size_t o;
            float l;
            if (u < n_core) {
                o = (static_cast<size_t>(slab) * n_core + u) * W + w;
                v = core[o];
                l = lch[o];
            } else {
                o = (static_cast<size_t>(slab) * n_deg1 + (u - n_core)) * W + w;
                v = deg1[o];
                l = lch1[o];
            }
            if (!(fabsf(l) < lmax)) v = 0.f;  // L_ch = clamp(llr): no gradient when clamped
        }
        tile[jj][w] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int w = idx / 32, jj = idx % 32;
        const int b = slab * W + w;
        const int32_t j = j0 + jj;
        if (b < batch && j < n_vn) out[static_cast<size_t>(b) * n_vn + j] = tile[jj][w];
    }
}

// Sum over the per-block partials of each weight type in a fixed order
// (strided over the threads, then a shared-memory tree), so the result does
// not depend on scheduling.
constexpr int kReduceThreads = 256;
__global__ void __launch_bounds__(kReduceThreads) kw_reduce_dw(const float *gwp, int blocks, int n_types,
                                                               float *dw_row) {
    __shared__ float part[kReduceThreads];
    for (int k = 0; k < n_types; ++k) {
        float v = 0.f;
        for (int b = threadIdx.x; b < blocks; b += kReduceThreads) v += gwp[static_cast<size_t>(b) * n_types + k];
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = kReduceThreads / 2; o > 0; o >>= 1) {
            if (static_cast<int>(threadIdx.x) < o) part[threadIdx.x] += part[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) dw_row[k] = part[0];
        __syncthreads();
    }
}

}  // namespace

struct mld_tape {
    mld_decoder *d = nullptr;
    int32_t batch = 0, T = 0, k = 1, n_types = 0, slabs = 0;
    float *w = nullptr;                 // [T][n_types]
    std::vector<float *> ckpt;          // r^{k}, r^{2k}, ... (r^0 = 0)
    float *seg_r = nullptr, *seg_lv = nullptr;  // k message / posterior arrays
    float *gr = nullptr, *gx = nullptr;          // edge gradients
    float *glch = nullptr, *glch1 = nullptr, *gd1 = nullptr;
    float *gwp = nullptr;
    int gwp_blocks = 0;
    // The iterations of the forward and the segments of the adjoint, as
    // CUDA graphs over this tape's (and its decoder's) fixed buffers:
    // captured at first use, replayed by later calls with this tape.
    cudaGraphExec_t fwd_exec = nullptr, bwd_exec = nullptr;
    float *dw = nullptr;  // [T][n_types], copied to the caller's dw
};

namespace {

void tape_free(mld_tape *t) {
    if (!t) return;
    if (t->fwd_exec) cudaGraphExecDestroy(t->fwd_exec);
    if (t->bwd_exec) cudaGraphExecDestroy(t->bwd_exec);
    dfree(t->dw);
    dfree(t->w);
    for (float *&p : t->ckpt) dfree(p);
    dfree(t->seg_r); dfree(t->seg_lv); dfree(t->gr); dfree(t->gx);
    dfree(t->glch); dfree(t->glch1); dfree(t->gd1); dfree(t->gwp);
    delete t;
}

// Enqueues `enqueue(stream)` on st through the CUDA graph *exec: captured
// on the decoder's capture stream the first time (so that a few hundred
// small launches become one), replayed after.  Where capture is not
// possible (no capture stream, or another capture owns this thread) the
// work is launched directly.
template <typename F>
int run_graph(mld_decoder *d, cudaGraphExec_t *exec, cudaStream_t st, F &&enqueue) {
    if (!*exec) {
        if (!d->cap) return enqueue(st);
        cudaError_t e = cudaStreamBeginCapture(d->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return enqueue(st);
        }
        const int s = enqueue(d->cap);
        cudaGraph_t gr = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(d->cap, &gr);
        if (s != MLD_OK || ec != cudaSuccess) {
            if (gr) cudaGraphDestroy(gr);
            return s != MLD_OK ? s : cuda_fail(ec, "weighted BP: graph capture");
        }
        e = cudaGraphInstantiate(exec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            *exec = nullptr;
            return cuda_fail(e, "weighted BP: graph instantiation");
        }
    }
    MLD_CUDA(cudaGraphLaunch(*exec, st));
    return MLD_OK;
}

WArgs wargs(const mld_decoder *d, const float *w, int n_types) {
    const mld::HostGraph &h = d->g->h;
    return WArgs{d->g->cptr, d->g->col, d->g->dptr, d->g->vptr, d->g->vedge, d->g->etype_core, d->g->etype_deg1,
                 h.n_cn, h.n_core, h.n_deg1, h.e_core, n_types, d->sbits, d->lch, d->lch1, w, d->lmax, d->amin};
}

// Forward iterations t = t_begin+1 .. t_end on messages r / posteriors lv.
template <int W>
int forward_iters(mld_decoder *d, const WArgs &wa, float *r, float *lv, int t_begin, int t_end, int T, int slabs,
                  cudaStream_t st, mld_tape *tape, float *seg_r, float *seg_lv) {
    const mld::HostGraph &h = d->g->h;
    constexpr int TPC = W / kK;
    const size_t rsz = static_cast<size_t>(slabs) * h.e_core * W;
    const size_t lsz = static_cast<size_t>(slabs) * h.n_core * W;
    VnArgs va{d->g->vptr, d->g->vedge, h.n_core, h.e_core, r, d->lch, lv, d->hb_core, d->done, 0, 0};
    for (int t = t_begin + 1; t <= t_end; ++t) {
        if (seg_r) {  // keep r^{t-1}, L^{t-1} for the adjoint of iteration t
            MLD_CUDA(cudaMemcpyAsync(seg_r + (t - 1 - t_begin) * rsz, r, rsz * sizeof(float), cudaMemcpyDeviceToDevice, st));
            MLD_CUDA(cudaMemcpyAsync(seg_lv + (t - 1 - t_begin) * lsz, lv, lsz * sizeof(float),
                                     cudaMemcpyDeviceToDevice, st));
        }
        for (const mld::ClassLaunch &cl : d->g->launches[W == 8 ? 0 : (W == 16 ? 1 : (W == 32 ? 2 : 3))]) {
            launch_check_fwd<W>(wa, cl, r, lv, d->post1, t, t == T ? 1 : 0, slabs, st);
            MLD_LAUNCHED("kw_check_fwd");
        }
        if (h.n_core > 0) {
            k_var_update<float, W><<<dim3(grid_x(static_cast<int64_t>(h.n_core) * TPC), slabs), kBlock, 0, st>>>(va);
            MLD_LAUNCHED("k_var_update");
        }
        if (tape && !seg_r && t % tape->k == 0 && t < T)
            MLD_CUDA(cudaMemcpyAsync(tape->ckpt[t / tape->k - 1], r, rsz * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    return MLD_OK;
}

template <int W>
int wbp_forward_w(mld_decoder *d, const float *llr, const uint8_t *syn, int32_t batch, int32_t T, mld_tape *tape,
                  const float *w, int n_types, float *soft, cudaStream_t st) {
    const mld::HostGraph &h = d->g->h;
    const int slabs = (batch + W - 1) / W;
    const size_t rsz = static_cast<size_t>(slabs) * h.e_core * W;
    if (rsz) MLD_CUDA(cudaMemsetAsync(d->r, 0, rsz * sizeof(float), st));
    // weighted BP works in nats: no scaling on entry or exit
    InArgs ia{llr, nullptr, d->g->unit, h.n_vn, h.n_core, h.n_deg1, batch, d->lmax, 1.f, d->lmax, d->amin,
              d->lch, d->Lv, d->lch1, d->post1, d->phi1};
    if (h.n_vn > 0) {
        k_interleave_in<W, kFitNat><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(ia);
        MLD_LAUNCHED("k_interleave_in");
    }
    if (h.n_cn > 0) {
        k_syndrome_in<W><<<dim3((h.n_cn + 31) / 32, slabs), kBlock, 0, st>>>(syn, d->g->cint, h.n_cn, batch, d->sbits);
        MLD_LAUNCHED("k_syndrome_in");
    }
    const WArgs wa = wargs(d, w, n_types);
    auto iters = [&](cudaStream_t s2) {
        return forward_iters<W>(d, wa, static_cast<float *>(d->r), d->Lv, 0, T, T, slabs, s2, tape, nullptr,
                                nullptr);
    };
    // with a tape every buffer the iterations touch is fixed for the tape's
    // life (the weights were copied into it), so they run as a graph
    int s = tape ? run_graph(d, &tape->fwd_exec, st, iters) : iters(st);
    if (s != MLD_OK) return s;
    OutArgs oa{d->g->unit, h.n_vn, h.n_core, h.n_deg1, batch, d->Lv, d->post1, d->hb1, nullptr, 0, d->bits_stage,
               soft, 1.f};
    if (h.n_vn > 0) {
        k_deinterleave_out<W><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(oa);
        MLD_LAUNCHED("k_deinterleave_out");
    }
    return MLD_OK;
}

template <int W>
int wbp_backward_w(mld_tape *tp, const float *dsoft, float *dw, float *dllr, cudaStream_t st) {
    mld_decoder *d = tp->d;
    const mld::HostGraph &h = d->g->h;
    constexpr int TPC = W / kK;
    const int slabs = tp->slabs, T = tp->T, K = tp->k;
    const size_t rsz = static_cast<size_t>(slabs) * h.e_core * W;
    const size_t lsz = static_cast<size_t>(slabs) * h.n_core * W;
    const size_t dsz = static_cast<size_t>(slabs) * h.n_deg1 * W;
    const WArgs wa = wargs(d, tp->w, tp->n_types);
    const dim3 vgrid(grid_x(static_cast<int64_t>(h.n_core) * TPC), slabs);
    const std::vector<mld::ClassLaunch> &classes = d->g->launches[W == 8 ? 0 : (W == 16 ? 1 : (W == 32 ? 2 : 3))];
    int32_t parts = 0;  // block partials of one adjoint check pass
    for (const mld::ClassLaunch &cl : classes) parts += cl.blocks * slabs;

    // dloss/dL^T: into dL_ch (the posterior is L_ch + sum r^T) and onto r^T
    if (lsz) MLD_CUDA(cudaMemsetAsync(tp->glch, 0, lsz * sizeof(float), st));
    if (dsz) MLD_CUDA(cudaMemsetAsync(tp->glch1, 0, dsz * sizeof(float), st));
    if (h.n_vn > 0) {
        kw_interleave<W><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(
            dsoft, d->g->unit, h.n_vn, h.n_core, h.n_deg1, tp->batch, tp->glch, tp->glch1, tp->gd1);
        MLD_LAUNCHED("kw_interleave");
    }
    // from dL^T on, every buffer is the tape's or the decoder's: the
    // segments run as a graph (dw into the tape, then copied out)
    auto segments = [&](cudaStream_t s2) -> int {
        if (h.n_core > 0) {
            kw_grad_edges<W><<<vgrid, kBlock, 0, s2>>>(wa, tp->glch, tp->gr);
            MLD_LAUNCHED("kw_grad_edges");
        }
        float *r = static_cast<float *>(d->r);
        for (int t0 = ((T - 1) / K) * K; t0 >= 0; t0 -= K) {
            const int t1 = std::min(t0 + K, T);
            // recompute r^{t0} .. r^{t1-1} and L^{t0} .. L^{t1-1}
            if (t0 == 0) {
                if (rsz) MLD_CUDA(cudaMemsetAsync(r, 0, rsz * sizeof(float), s2));
            } else {
                MLD_CUDA(cudaMemcpyAsync(r, tp->ckpt[t0 / K - 1], rsz * sizeof(float), cudaMemcpyDeviceToDevice, s2));
            }
            if (h.n_core > 0) {
                VnArgs va{d->g->vptr, d->g->vedge, h.n_core, h.e_core, r, d->lch, d->Lv, d->hb_core, d->done, 0, 0};
                k_var_update<float, W><<<vgrid, kBlock, 0, s2>>>(va);
                MLD_LAUNCHED("k_var_update");
            }
            int s = forward_iters<W>(d, wa, r, d->Lv, t0, t1 - 1, T, slabs, s2, tp, tp->seg_r, tp->seg_lv);
            if (s != MLD_OK) return s;
            // r^{t1-1}, L^{t1-1} are now in r / d->Lv; store them as the last segment entry
            MLD_CUDA(cudaMemcpyAsync(tp->seg_r + (t1 - 1 - t0) * rsz, r, rsz * sizeof(float), cudaMemcpyDeviceToDevice, s2));
            MLD_CUDA(cudaMemcpyAsync(tp->seg_lv + (t1 - 1 - t0) * lsz, d->Lv, lsz * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s2));
            for (int t = t1; t > t0; --t) {
                const float *rp = tp->seg_r + (t - 1 - t0) * rsz;
                const float *lvp = tp->seg_lv + (t - 1 - t0) * lsz;
                if (parts > 0) {
                    int32_t part0 = 0;
                    for (const mld::ClassLaunch &cl : classes) {
                        launch_check_bwd<W>(wa, cl, rp, lvp, tp->gr, t == T ? tp->gd1 : nullptr, tp->gx, tp->glch1,
                                            tp->gwp, t, slabs, part0, s2);
                        MLD_LAUNCHED("kw_check_bwd");
                        part0 += cl.blocks * slabs;
                    }
                    kw_reduce_dw<<<1, kReduceThreads, 0, s2>>>(tp->gwp, parts, tp->n_types,
                                                               tp->dw + static_cast<size_t>(t - 1) * tp->n_types);
                    MLD_LAUNCHED("kw_reduce_dw");
                } else {
                    MLD_CUDA(cudaMemsetAsync(tp->dw + static_cast<size_t>(t - 1) * tp->n_types, 0,
                                             sizeof(float) * tp->n_types, s2));
                }
                if (h.n_core > 0) {
                    kw_var_bwd<W><<<vgrid, kBlock, 0, s2>>>(wa, tp->gx, tp->glch, t > 1 ? tp->gr : nullptr);
                    MLD_LAUNCHED("kw_var_bwd");
                }
            }
        }
        return MLD_OK;
    };
    int sg = run_graph(d, &tp->bwd_exec, st, segments);
    if (sg != MLD_OK) return sg;
    MLD_CUDA(cudaMemcpyAsync(dw, tp->dw, sizeof(float) * T * tp->n_types, cudaMemcpyDeviceToDevice, st));
    if (h.n_vn > 0) {
        kw_deinterleave<W><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(
            tp->glch, tp->glch1, d->lch, d->lch1, d->g->unit, h.n_vn, h.n_core, h.n_deg1, tp->batch, d->lmax, dllr);
        MLD_LAUNCHED("kw_deinterleave");
    }
    return MLD_OK;
}

template <typename T>
int talloc(T **p, size_t n) { return dalloc(p, n); }

// A decoder keeps the buffers of its last destroyed tape and hands them to
// the next forward of the same shape, so a training loop allocates (and
// frees, which waits for the device) once instead of every step.
mld_tape *take_spare(mld_decoder *d, int32_t slabs, int32_t T, int32_t k, int32_t n_types) {
    mld_tape *tp = d->tape_spare;
    if (!tp) return nullptr;
    d->tape_spare = nullptr;
    if (tp->slabs == slabs && tp->T == T && tp->k == k && tp->n_types == n_types) return tp;
    tape_free(tp);
    return nullptr;
}

}  // namespace

namespace mld {
// Decoder teardown: frees the spare tape and detaches a tape still alive (it
// frees its own buffers when destroyed).
void tape_release(mld_decoder *d) {
    if (d->tape_spare) tape_free(d->tape_spare);
    d->tape_spare = nullptr;
    if (d->tape_live) d->tape_live->d = nullptr;
    d->tape_live = nullptr;
}
}  // namespace mld

extern "C" {

int mld_wbp_forward(mld_decoder *d, const float *llr, const uint8_t *syndrome, int32_t batch, const float *w,
                    int32_t n_types, int32_t T, int32_t ckpt_k, float *soft_out, mld_tape **tape, void *stream) {
    mld::clear_error();
    if (!d) return mld::fail(MLD_EINVAL, "wbp_forward: null decoder");
    if (d->msg != MLD_MSG_F32) return mld::fail(MLD_EINVAL, "wbp_forward: the decoder must store float messages");
    if (batch < 1 || batch > d->max_batch) return mld::fail(MLD_EINVAL, "wbp_forward: batch out of range");
    if (T < 1 || ckpt_k < 1) return mld::fail(MLD_EINVAL, "wbp_forward: T and ckpt_k must be >= 1");
    if (n_types < 1 || n_types > MLD_MAX_EDGE_TYPES) return mld::fail(MLD_EINVAL, "wbp_forward: n_types");
    const mld::HostGraph &h = d->g->h;
    if (h.max_check_deg > kMaxTerms)
        return mld::fail(MLD_EINVAL, "wbp_forward: check degree above " + std::to_string(kMaxTerms));
    for (uint8_t ty : h.etype_core)
        if (ty >= n_types) return mld::fail(MLD_EINVAL, "wbp_forward: an edge type is >= n_types");
    for (uint8_t ty : h.etype_deg1)
        if (ty >= n_types) return mld::fail(MLD_EINVAL, "wbp_forward: an edge type is >= n_types");
    if ((h.n_vn > 0 && (!llr || !soft_out)) || (h.n_cn > 0 && !syndrome) || !w)
        return mld::fail(MLD_EINVAL, "wbp_forward: null data pointer");
    int s = check_device(d->device);
    if (s != MLD_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int W = d->W;
    const int slabs = (batch + W - 1) / W;
    mld_tape *tp = nullptr;
    const float *wdev = w;
    if (tape) {
        tp = take_spare(d, slabs, T, std::min(ckpt_k, T), n_types);
        if (tp) {
            tp->batch = batch;
            cudaError_t e = cudaMemcpyAsync(tp->w, w, sizeof(float) * T * n_types, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) {
                tape_free(tp);
                return cuda_fail(e, "wbp_forward: copy weights");
            }
        }
    }
    if (tape && !tp) {
        tp = new (std::nothrow) mld_tape();
        if (!tp) return mld::fail(MLD_ENOMEM, "wbp_forward: host allocation");
        tp->d = d;
        tp->batch = batch;
        tp->T = T;
        tp->k = std::min(ckpt_k, T);
        tp->n_types = n_types;
        tp->slabs = slabs;
        const size_t rsz = static_cast<size_t>(slabs) * h.e_core * W;
        const size_t lsz = static_cast<size_t>(slabs) * h.n_core * W;
        const size_t dsz = static_cast<size_t>(slabs) * h.n_deg1 * W;
        s = talloc(&tp->w, static_cast<size_t>(T) * n_types);
        if (s == MLD_OK) s = talloc(&tp->dw, static_cast<size_t>(T) * n_types);
        for (int c = tp->k; s == MLD_OK && c < T; c += tp->k) {
            float *p = nullptr;
            s = talloc(&p, rsz);
            tp->ckpt.push_back(p);
        }
        if (s == MLD_OK) s = talloc(&tp->seg_r, rsz * tp->k);
        if (s == MLD_OK) s = talloc(&tp->seg_lv, lsz * tp->k);
        if (s == MLD_OK) s = talloc(&tp->gr, rsz);
        if (s == MLD_OK) s = talloc(&tp->gx, rsz);
        if (s == MLD_OK) s = talloc(&tp->glch, lsz);
        if (s == MLD_OK) s = talloc(&tp->glch1, dsz);
        if (s == MLD_OK) s = talloc(&tp->gd1, dsz);
        tp->gwp_blocks = 0;
        for (const mld::ClassLaunch &cl : d->g->launches[W == 8 ? 0 : (W == 16 ? 1 : (W == 32 ? 2 : 3))])
            tp->gwp_blocks += cl.blocks * slabs;
        if (s == MLD_OK) s = talloc(&tp->gwp, static_cast<size_t>(std::max(1, tp->gwp_blocks)) * n_types);
        if (s == MLD_OK) {
            cudaError_t e = cudaMemcpyAsync(tp->w, w, sizeof(float) * T * n_types, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) s = cuda_fail(e, "wbp_forward: copy weights");
        }
        if (s != MLD_OK) {
            tape_free(tp);
            return s;
        }
    }
    if (tp) wdev = tp->w;
    switch (W) {
        case 8: s = wbp_forward_w<8>(d, llr, syndrome, batch, T, tp, wdev, n_types, soft_out, st); break;
        case 16: s = wbp_forward_w<16>(d, llr, syndrome, batch, T, tp, wdev, n_types, soft_out, st); break;
        case 32: s = wbp_forward_w<32>(d, llr, syndrome, batch, T, tp, wdev, n_types, soft_out, st); break;
        default: s = wbp_forward_w<64>(d, llr, syndrome, batch, T, tp, wdev, n_types, soft_out, st); break;
    }
    if (s != MLD_OK) {
        tape_free(tp);
        return s;
    }
    if (tape) {
        *tape = tp;
        d->tape_live = tp;
    }
    return MLD_OK;
}

int mld_wbp_backward(mld_tape *tp, const float *dsoft, float *dw, float *dllr, void *stream) {
    mld::clear_error();
    if (!tp || !dsoft || !dw || !dllr) return mld::fail(MLD_EINVAL, "wbp_backward: null pointer");
    int s = check_device(tp->d->device);
    if (s != MLD_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (tp->d->W) {
        case 8: return wbp_backward_w<8>(tp, dsoft, dw, dllr, st);
        case 16: return wbp_backward_w<16>(tp, dsoft, dw, dllr, st);
        case 32: return wbp_backward_w<32>(tp, dsoft, dw, dllr, st);
        default: return wbp_backward_w<64>(tp, dsoft, dw, dllr, st);
    }
}

int mld_tape_destroy(mld_tape *tp) {
    if (!tp) return MLD_OK;
    mld_decoder *d = tp->d;
    if (d && d->tape_live == tp) d->tape_live = nullptr;
    if (d && !d->tape_spare) {
        d->tape_spare = tp;  // buffers kept for the next forward of this shape
        return MLD_OK;
    }
    tape_free(tp);
    return MLD_OK;
}

}  // extern "C"
