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

#include "internal.h"
#include "phi_poly.h"

namespace mld {
const char *last_error_text();
}

namespace {

constexpr int kK = 4;          // codewords per thread
constexpr int kBlock = 256;

// ---------------------------------------------------------------------------
// phi(x) = -ln tanh(x/2) in float, for x in [phi(lmax), lmax].
// Two pieces (see gen_phi_poly.py): below MLD_PHI_X0, ln2 - ln x - t Ps(t)
// with t = x^2; above, e Pl(e^2) with e = exp(-x).  ln and exp come from
// the MUFU base-2 approximations.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mufu_lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Piece below MLD_PHI_X0.  HALF selects the shorter fit used with half
// message storage (error ~3e-6, far below half's 2^-11 rounding).
template <bool HALF>
__device__ __forceinline__ float phi_small(float x) {
    const float kLn2 = 0.693147180559945309f;
    const float t = x * x;
    float ps;
    if constexpr (HALF) {
        ps = fmaf(MLD_PHIH_S2, t, MLD_PHIH_S1);
        ps = fmaf(ps, t, MLD_PHIH_S0);
    } else {
        ps = fmaf(MLD_PHI_S4, t, MLD_PHI_S3);
        ps = fmaf(ps, t, MLD_PHI_S2);
        ps = fmaf(ps, t, MLD_PHI_S1);
        ps = fmaf(ps, t, MLD_PHI_S0);
    }
    return fmaf(-t, ps, fmaf(-kLn2, mufu_lg2(x), kLn2));
}

// Piece at and above MLD_PHI_X0.
template <bool HALF>
__device__ __forceinline__ float phi_large(float x) {
    const float kLog2e = 1.442695040888963407f;
    const float e = mufu_ex2(-kLog2e * x);
    const float z = e * e;
    float pl;
    if constexpr (HALF) {
        pl = fmaf(MLD_PHIH_L2, z, MLD_PHIH_L1);
        pl = fmaf(pl, z, MLD_PHIH_L0);
    } else {
        pl = fmaf(MLD_PHI_L3, z, MLD_PHI_L2);
        pl = fmaf(pl, z, MLD_PHI_L1);
        pl = fmaf(pl, z, MLD_PHI_L0);
    }
    return e * pl;
}

// Branch-free choice x < th ? a : b (both operands are already computed).
__device__ __forceinline__ float sel_lt(float x, float th, float a, float b) {
    float r;
    asm("{\n\t.reg .pred p;\n\tsetp.lt.f32 p, %1, %2;\n\tselp.f32 %0, %3, %4, p;\n\t}"
        : "=f"(r) : "f"(x), "f"(th), "f"(a), "f"(b));
    return r;
}

// phi of one value: both pieces are evaluated and the right one selected
// without branches, so the compiler can interleave independent chains.
template <bool HALF>
__device__ __forceinline__ float phi_f(float x) {
    return sel_lt(x, MLD_PHI_X0, phi_small<HALF>(x), phi_large<HALF>(x));
}

template <bool HALF>
__device__ __forceinline__ float4 phi4(float4 x) {
    return make_float4(phi_f<HALF>(x.x), phi_f<HALF>(x.y), phi_f<HALF>(x.z), phi_f<HALF>(x.w));
}

template <typename T> struct IsHalf { static constexpr bool value = false; };
template <> struct IsHalf<__half> { static constexpr bool value = true; };

__device__ __forceinline__ float clampf(float x, float lo, float hi) {
    return fminf(fmaxf(x, lo), hi);
}

// ---------------------------------------------------------------------------
// 4-codeword vector access for each message storage type
// ---------------------------------------------------------------------------
template <typename T> struct Msg;
template <> struct Msg<float> {
    static __device__ __forceinline__ float4 load(const float *p) {
        return *reinterpret_cast<const float4 *>(p);
    }
    static __device__ __forceinline__ void store(float *p, float4 v) {
        *reinterpret_cast<float4 *>(p) = v;
    }
};
template <> struct Msg<__half> {
    static __device__ __forceinline__ float4 load(const __half *p) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    static __device__ __forceinline__ void store(__half *p, float4 v) {
        const __half2 a = __floats2half2_rn(v.x, v.y);
        const __half2 b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t *>(&a);
        u.y = *reinterpret_cast<const uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};

__device__ __forceinline__ float4 ldf4(const float *p) {
    return __ldg(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ float f4get(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4 &v, int k, float x) {
    if (k == 0) v.x = x; else if (k == 1) v.y = x; else if (k == 2) v.z = x; else v.w = x;
}

__device__ __forceinline__ unsigned pair_mask() {
    return 0x3u << ((threadIdx.x & 31u) & ~1u);
}

// done-bit nibble of the 4 codewords starting at lane0 of a slab
template <int W>
__device__ __forceinline__ uint32_t done_nibble(const uint32_t *done, int slab, int lane0) {
    constexpr int DW = (W + 31) / 32;
    return (done[slab * DW + lane0 / 32] >> (lane0 & 31)) & 0xFu;
}

template <int W>
__device__ __forceinline__ bool slab_all_done(const uint32_t *done, int slab) {
    constexpr int DW = (W + 31) / 32;
    constexpr uint32_t full = W >= 32 ? 0xFFFFFFFFu : ((1u << W) - 1u);
    for (int i = 0; i < DW; ++i)
        if (done[slab * DW + i] != full) return false;
    return true;
}

// ---------------------------------------------------------------------------
// Check update (Eqs. 2-3 with the syndrome sign), one iteration.
// ---------------------------------------------------------------------------
struct CnArgs {
    const int32_t *cptr, *col, *dptr;
    int32_t n_cn, n_core, n_deg1, e_core;
    void *r;               // [slab][e_core][W] messages
    const float *Lv;       // [slab][n_core][W] core posteriors of the previous iteration
    const float *lch1;     // [slab][n_deg1][W] degree-1 channel LLRs
    const float *phi1;     // [slab][n_deg1][W] phi(|L_ch|) with the sign of L_ch (constant)
    float *post1;          // [slab][n_deg1][W] degree-1 posteriors (final / ET pass)
    uint8_t *hb1;          // [slab][n_deg1][W/8] degree-1 hard decisions
    const uint8_t *sbits;  // [slab][n_cn][W/8] syndrome bits
    const uint32_t *done;  // [slab][ceil(W/32)] converged lanes (ET)
    float lmax, amin;
    int final_pass, et;
};

template <typename MsgT, int W>
__device__ __forceinline__ void emit_deg1(const CnArgs &a, int slab, int slot, int lane0,
                                          float4 rv, uint32_t donenib, bool valid) {
    constexpr int NB = W / 8;
    const size_t base = (static_cast<size_t>(slab) * a.n_deg1 + slot) * W + lane0;
    const float4 l = ldf4(a.lch1 + base);  // in range: the slot of a real check
    float4 post = make_float4(l.x + rv.x, l.y + rv.y, l.z + rv.z, l.w + rv.w);
    uint32_t nib = (post.x < 0.f) | ((post.y < 0.f) << 1) | ((post.z < 0.f) << 2) | ((post.w < 0.f) << 3);
    uint8_t *hb = a.hb1 + (static_cast<size_t>(slab) * a.n_deg1 + slot) * NB + lane0 / 8;
    if (donenib && valid) {  // converged lanes keep the decision of their last iteration
        const float4 old = *reinterpret_cast<const float4 *>(a.post1 + base);
        if (donenib & 1) post.x = old.x;
        if (donenib & 2) post.y = old.y;
        if (donenib & 4) post.z = old.z;
        if (donenib & 8) post.w = old.w;
        const uint32_t oldnib = (static_cast<uint32_t>(*hb) >> (lane0 & 7)) & 0xFu;
        nib = (nib & ~donenib) | (oldnib & donenib);
    }
    if (valid) *reinterpret_cast<float4 *>(a.post1 + base) = post;
    const uint32_t other = __shfl_xor_sync(pair_mask(), nib, 1);
    if (valid && (lane0 & 7) == 0) *hb = static_cast<uint8_t>(nib | (other << 4));
}

template <typename MsgT, int W>
__device__ __forceinline__ void store_r(const CnArgs &a, MsgT *rp, float4 rv, uint32_t donenib) {
    if (donenib) {  // converged lanes keep their messages frozen
        const float4 old = Msg<MsgT>::load(rp);
        if (donenib & 1) rv.x = old.x;
        if (donenib & 2) rv.y = old.y;
        if (donenib & 4) rv.z = old.z;
        if (donenib & 8) rv.w = old.w;
    }
    Msg<MsgT>::store(rp, rv);
}

using mld::ClassLaunch;

__device__ __forceinline__ uint32_t fbits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ float bitsf(uint32_t x) { return __uint_as_float(x); }
constexpr uint32_t kSign = 0x80000000u;

// Checks of one class: DC core edges and DD degree-1 VNs per check, all
// terms in registers.  Threads past the class end work on its last check and
// store nothing (so a whole shuffle pair stays active).
template <typename MsgT, int W, int DC, int DD>
__device__ __forceinline__ void check_regular(const CnArgs &a, const ClassLaunch &cl, int64_t lt, int slab) {
    constexpr int TPC = W / kK;
    constexpr int NB = W / 8;
    constexpr int D = DC + DD;
    constexpr int dc = DC;
    constexpr bool H = IsHalf<MsgT>::value;
    const int32_t count = cl.count;
    int32_t j = static_cast<int32_t>(lt / TPC);
    const bool valid = j < count;
    if (!valid) j = count - 1;
    const int lane0 = static_cast<int>(lt % TPC) * kK;
    const int32_t c = cl.c0 + j;
    const int32_t e0 = cl.e0 + j * dc;
    const int32_t s0 = cl.s0 + j * (D - dc);
    const float lmax = a.lmax, amin = a.amin;

    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >>
         (lane0 & 7));
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    MsgT *rb = static_cast<MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    const float *lvb = a.Lv + static_cast<size_t>(slab) * a.n_core * W + lane0;
    const float *p1b = a.phi1 + static_cast<size_t>(slab) * a.n_deg1 * W + lane0;

    int32_t vidx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) vidx[i] = (i < dc) ? __ldg(a.col + e0 + i) : 0;

    // pass 1: f = phi(|q|) carrying the sign of q in its sign bit; the top
    // bit of par accumulates the sign parity (syndrome bit included).  For a
    // degree-1 VN q is its channel LLR, whose f was formed once on entry.
    float f[D][kK];
    uint32_t par[kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) par[kk] = ((sb >> kk) & 1u) << 31;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i < dc) {
            const float4 lv = ldf4(lvb + static_cast<size_t>(vidx[i]) * W);
            const float4 ro = Msg<MsgT>::load(rb + static_cast<size_t>(e0 + i) * W);
            const float4 q = make_float4(lv.x - ro.x, lv.y - ro.y, lv.z - ro.z, lv.w - ro.w);
            const float4 m = make_float4(clampf(fabsf(q.x), amin, lmax), clampf(fabsf(q.y), amin, lmax),
                                         clampf(fabsf(q.z), amin, lmax), clampf(fabsf(q.w), amin, lmax));
            const float4 ph = phi4<H>(m);
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                const uint32_t qb = fbits(f4get(q, kk));
                f[i][kk] = bitsf(fbits(f4get(ph, kk)) | (qb & kSign));
                par[kk] ^= qb;
            }
        } else {
            const float4 p = ldf4(p1b + static_cast<size_t>(s0 + i - dc) * W);
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                f[i][kk] = f4get(p, kk);
                par[kk] ^= fbits(f[i][kk]);
            }
        }
    }
    // exclusive prefix sums of |f|
    float pre[D][kK];
    {
        float acc[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < D; ++i) {
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                pre[i][kk] = acc[kk];
                acc[kk] += fabsf(f[i][kk]);
            }
        }
    }
    // pass 2 (backwards): leave-one-out sum = prefix + suffix
    float suf[kK] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        if (i < dc || a.final_pass) {
            // every other term contributes phi(|q|) >= phi(lmax) ~ amin, so for
            // D >= 2 the sum is already >= amin (up to rounding) and for D >= 3
            // phi of it stays below lmax; only the needed clamps are applied
            float4 o = make_float4(fminf(pre[i][0] + suf[0], lmax), fminf(pre[i][1] + suf[1], lmax),
                                   fminf(pre[i][2] + suf[2], lmax), fminf(pre[i][3] + suf[3], lmax));
            if (D == 1) o = make_float4(amin, amin, amin, amin);
            float4 m = phi4<H>(o);
            if (D <= 2) m = make_float4(fminf(m.x, lmax), fminf(m.y, lmax), fminf(m.z, lmax), fminf(m.w, lmax));
            float4 rv;
#pragma unroll
            for (int kk = 0; kk < kK; ++kk)
                f4set(rv, kk, bitsf(fbits(f4get(m, kk)) | ((par[kk] ^ fbits(f[i][kk])) & kSign)));
            if (i < dc) {
                if (valid) store_r<MsgT, W>(a, rb + static_cast<size_t>(e0 + i) * W, rv, donenib);
            } else {
                emit_deg1<MsgT, W>(a, slab, s0 + i - dc, lane0, rv, donenib, valid);
            }
        }
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) suf[kk] += fabsf(f[i][kk]);
    }
}

// Checks of any degree, edges read through cptr/dptr; leave-one-out sums as
// total minus own term.  Threads of a check pair stay together; nothing here
// needs the whole warp.
template <typename MsgT, int W>
__device__ __forceinline__ void check_irregular(const CnArgs &a, const ClassLaunch &cl, int64_t lt, int slab) {
    constexpr int TPC = W / kK;
    constexpr int NB = W / 8;
    constexpr bool H = IsHalf<MsgT>::value;
    const int32_t j = static_cast<int32_t>(lt / TPC);
    if (j >= cl.count) return;
    const int lane0 = static_cast<int>(lt % TPC) * kK;
    const int32_t c = cl.c0 + j;
    const int32_t e0 = a.cptr[c], e1 = a.cptr[c + 1];
    const int32_t s0 = a.dptr[c], s1 = a.dptr[c + 1];
    const int nce = e1 - e0;
    const int deg = nce + (s1 - s0);
    const float lmax = a.lmax, amin = a.amin;
    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >>
         (lane0 & 7));
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    MsgT *rb = static_cast<MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    const float *lvb = a.Lv + static_cast<size_t>(slab) * a.n_core * W + lane0;
    const float *l1b = a.lch1 + static_cast<size_t>(slab) * a.n_deg1 * W + lane0;
    auto input = [&](int i) -> float4 {
        if (i < nce) {
            const float4 lv = ldf4(lvb + static_cast<size_t>(__ldg(a.col + e0 + i)) * W);
            const float4 ro = Msg<MsgT>::load(rb + static_cast<size_t>(e0 + i) * W);
            return make_float4(lv.x - ro.x, lv.y - ro.y, lv.z - ro.z, lv.w - ro.w);
        }
        return ldf4(l1b + static_cast<size_t>(s0 + i - nce) * W);  // q = L_ch
    };
    float S[kK] = {0.f, 0.f, 0.f, 0.f};
    uint32_t par[kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) par[kk] = ((sb >> kk) & 1u) << 31;
    for (int i = 0; i < deg; ++i) {
        const float4 q = input(i);
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) {
            const float qk = f4get(q, kk);
            par[kk] ^= fbits(qk);
            S[kk] += phi_f<H>(clampf(fabsf(qk), amin, lmax));
        }
    }
    for (int i = 0; i < deg; ++i) {
        const bool out_core = i < nce;
        if (!out_core && !a.final_pass) continue;
        const float4 q = input(i);
        float4 rv;
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) {
            const float qk = f4get(q, kk);
            const float fk = phi_f<H>(clampf(fabsf(qk), amin, lmax));
            const float mk = fminf(phi_f<H>(clampf(S[kk] - fk, amin, lmax)), lmax);
            f4set(rv, kk, bitsf(fbits(mk) | ((par[kk] ^ fbits(qk)) & kSign)));
        }
        if (out_core)
            store_r<MsgT, W>(a, rb + static_cast<size_t>(e0 + i) * W, rv, donenib);
        else
            emit_deg1<MsgT, W>(a, slab, s0 + i - nce, lane0, rv, donenib, true);
    }
}

// One check class per launch, its shape (DC, DD) a compile-time constant: the
// register arrays are sized exactly and only this class's code is hot.
template <typename MsgT, int W, int DC, int DD>
__global__ void __launch_bounds__(kBlock, (DC + DD <= 6 ? 4 : 3)) k_check_update(CnArgs a, ClassLaunch cl) {
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;  // block-uniform
    check_regular<MsgT, W, DC, DD>(a, cl, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, slab);
}

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) k_check_update_irregular(CnArgs a, ClassLaunch cl) {
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    check_irregular<MsgT, W>(a, cl, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, slab);
}

// Classes with at most one degree-1 VN per check and at most kMaxRegDeg terms
// run the register kernel for their shape; any other class (possible in
// caller graphs, not in the MET ensembles) runs the streaming kernel.
template <typename MsgT, int W>
void launch_check_class(const CnArgs &ca, const ClassLaunch &cl, int slabs, cudaStream_t st) {
    const dim3 grid(cl.blocks, slabs);
    const int dd = cl.deg - cl.dc;
#define MLD_CASE(DCV, DDV) \
    case (DCV) * 2 + (DDV): k_check_update<MsgT, W, DCV, DDV><<<grid, kBlock, 0, st>>>(ca, cl); return;
    if (cl.dc >= 0 && (dd == 0 || dd == 1)) {
        switch (cl.dc * 2 + dd) {
            MLD_CASE(1, 0) MLD_CASE(2, 0) MLD_CASE(3, 0) MLD_CASE(4, 0)
            MLD_CASE(5, 0) MLD_CASE(6, 0) MLD_CASE(7, 0) MLD_CASE(8, 0)
            MLD_CASE(0, 1) MLD_CASE(1, 1) MLD_CASE(2, 1) MLD_CASE(3, 1)
            MLD_CASE(4, 1) MLD_CASE(5, 1) MLD_CASE(6, 1) MLD_CASE(7, 1)
            default: break;
        }
    }
#undef MLD_CASE
    k_check_update_irregular<MsgT, W><<<grid, kBlock, 0, st>>>(ca, cl);
}

// ---------------------------------------------------------------------------
// Variable update (Eqs. 4-5) for core VNs: L_v = L_ch + sum of incoming r.
// ---------------------------------------------------------------------------
struct VnArgs {
    const int32_t *vptr, *vedge;
    int32_t n_core, e_core;
    const void *r;
    const float *lch;   // [slab][n_core][W]
    float *Lv;          // [slab][n_core][W]
    uint8_t *hb;        // [slab][n_core][W/8]
    const uint32_t *done;
    int want_bits, et;
};

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) k_var_update(VnArgs a) {
    constexpr int TPC = W / kK;
    constexpr int NB = W / 8;
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int32_t v = static_cast<int32_t>(t / TPC);
    if (v >= a.n_core) return;
    const int lane0 = static_cast<int>(t % TPC) * kK;
    const size_t vrow = (static_cast<size_t>(slab) * a.n_core + v) * W + lane0;
    const MsgT *rb = static_cast<const MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    float4 acc = ldf4(a.lch + vrow);
    int32_t j = a.vptr[v];
    const int32_t j1 = a.vptr[v + 1];
    for (; j + 4 <= j1; j += 4) {
        const int32_t ea = __ldg(a.vedge + j), eb = __ldg(a.vedge + j + 1);
        const int32_t ec = __ldg(a.vedge + j + 2), ed = __ldg(a.vedge + j + 3);
        const float4 ra = Msg<MsgT>::load(rb + static_cast<size_t>(ea) * W);
        const float4 rbv = Msg<MsgT>::load(rb + static_cast<size_t>(eb) * W);
        const float4 rc = Msg<MsgT>::load(rb + static_cast<size_t>(ec) * W);
        const float4 rd = Msg<MsgT>::load(rb + static_cast<size_t>(ed) * W);
        acc.x += ra.x; acc.y += ra.y; acc.z += ra.z; acc.w += ra.w;
        acc.x += rbv.x; acc.y += rbv.y; acc.z += rbv.z; acc.w += rbv.w;
        acc.x += rc.x; acc.y += rc.y; acc.z += rc.z; acc.w += rc.w;
        acc.x += rd.x; acc.y += rd.y; acc.z += rd.z; acc.w += rd.w;
    }
    for (; j < j1; ++j) {
        const float4 ra = Msg<MsgT>::load(rb + static_cast<size_t>(__ldg(a.vedge + j)) * W);
        acc.x += ra.x; acc.y += ra.y; acc.z += ra.z; acc.w += ra.w;
    }
    *reinterpret_cast<float4 *>(a.Lv + vrow) = acc;
    if (a.want_bits) {
        const uint32_t nib = (acc.x < 0.f) | ((acc.y < 0.f) << 1) | ((acc.z < 0.f) << 2) | ((acc.w < 0.f) << 3);
        const uint32_t other = __shfl_xor_sync(pair_mask(), nib, 1);
        if ((lane0 & 7) == 0)
            a.hb[(static_cast<size_t>(slab) * a.n_core + v) * NB + lane0 / 8] = static_cast<uint8_t>(nib | (other << 4));
    }
}

// ---------------------------------------------------------------------------
// Syndrome check (Step 5): bit-exact XOR of hard decisions over each check.
// fail[slab] collects, per codeword, whether any check is violated.
// ---------------------------------------------------------------------------
struct SynArgs {
    const int32_t *cptr, *col, *dptr;
    int32_t n_cn, n_core, n_deg1;
    const uint8_t *sbits, *hb_core, *hb1;
    uint32_t *fail;
    const uint32_t *done;
    int et;
};

template <int W>
__global__ void __launch_bounds__(kBlock) k_syndrome_check(SynArgs a) {
    constexpr int NB = W / 8;
    constexpr int DW = (W + 31) / 32;
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;  // block-uniform
    const int g = threadIdx.x % NB;
    const size_t cbase = static_cast<size_t>(slab) * a.n_cn;
    const uint8_t *hc = a.hb_core + static_cast<size_t>(slab) * a.n_core * NB + g;
    const uint8_t *h1 = a.hb1 + static_cast<size_t>(slab) * a.n_deg1 * NB + g;
    uint32_t acc = 0;
    const int64_t total = static_cast<int64_t>(a.n_cn) * NB;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
         t += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        const int32_t c = static_cast<int32_t>(t / NB);
        uint32_t x = a.sbits[(cbase + c) * NB + g];
        for (int32_t e = a.cptr[c]; e < a.cptr[c + 1]; ++e) x ^= hc[static_cast<size_t>(__ldg(a.col + e)) * NB];
        for (int32_t s = a.dptr[c]; s < a.dptr[c + 1]; ++s) x ^= h1[static_cast<size_t>(s) * NB];
        acc |= x;
    }
#pragma unroll
    for (int o = 16; o >= NB; o >>= 1) acc |= __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) < NB && acc)
        atomicOr(a.fail + slab * DW + (g * 8) / 32, acc << ((g * 8) & 31));
}

// per-codeword bookkeeping after a syndrome check at iteration l
template <int W>
__global__ void k_lane_update(uint32_t *done, const uint32_t *fail, int32_t *iters,
                              uint8_t *conv, int32_t batch, int32_t l, int et) {
    constexpr int DW = (W + 31) / 32;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const int slab = b / W, w = b % W;
    const int word = slab * DW + w / 32;
    const uint32_t bit = 1u << (w & 31);
    const bool ok = (fail[word] & bit) == 0u;
    if (et) {
        if (done[word] & bit) return;  // frozen at an earlier iteration
        iters[b] = l;
        conv[b] = ok ? 1 : 0;
        if (ok) atomicOr(done + word, bit);
    } else {
        iters[b] = l;
        conv[b] = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// Layout conversion: natural [B][n] rows <-> interleaved slabs.
// ---------------------------------------------------------------------------
struct InArgs {
    const float *in;      // [B][n_vn]
    const float *sigma;   // [B] or null (input is already an LLR)
    const int32_t *unit;
    int32_t n_vn, n_core, n_deg1, batch;
    float lmax, amin;
    float *lch, *Lv, *lch1, *post1, *phi1;
};

template <int W, bool HALF>
__global__ void __launch_bounds__(kBlock) k_interleave_in(InArgs a) {
    __shared__ float tile[W][33];
    const int slab = blockIdx.y;
    const int32_t j0 = blockIdx.x * 32;
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int w = idx / 32, jj = idx % 32;
        const int b = slab * W + w;
        const int32_t j = j0 + jj;
        float v = 0.f;
        if (b < a.batch && j < a.n_vn) {
            v = a.in[static_cast<size_t>(b) * a.n_vn + j];
            if (a.sigma) {
                const float s = a.sigma[b];
                v = (s > 0.f) ? v * (2.0f / (s * s)) : 0.f;
            }
            v = clampf(v, -a.lmax, a.lmax) + 0.0f;  // -0 -> +0: a zero LLR has no sign
        }
        tile[w][jj] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int jj = idx / W, w = idx % W;
        const int32_t j = j0 + jj;
        if (j >= a.n_vn) continue;
        const int32_t u = a.unit[j];
        const float v = tile[w][jj];
        if (u < a.n_core) {
            const size_t o = (static_cast<size_t>(slab) * a.n_core + u) * W + w;
            a.lch[o] = v;
            a.Lv[o] = v;
        } else {
            const size_t o = (static_cast<size_t>(slab) * a.n_deg1 + (u - a.n_core)) * W + w;
            a.lch1[o] = v;
            a.post1[o] = v;
            // the degree-1 VN's message never changes: its phi term, with the
            // sign of the LLR, is formed once here for every check update
            const float f = phi_f<HALF>(clampf(fabsf(v), a.amin, a.lmax));
            a.phi1[o] = bitsf(fbits(f) | (fbits(v) & kSign));
        }
    }
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_syndrome_in(const uint8_t *syn, const int32_t *cint, int32_t n_cn,
                                                        int32_t batch, uint8_t *sbits) {
    constexpr int NB = W / 8;
    __shared__ uint8_t tile[W][33];
    const int slab = blockIdx.y;
    const int32_t c0 = blockIdx.x * 32;  // caller's check order (coalesced reads)
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int w = idx / 32, cc = idx % 32;
        const int b = slab * W + w;
        const int32_t c = c0 + cc;
        tile[w][cc] = (b < batch && c < n_cn) ? (syn[static_cast<size_t>(b) * n_cn + c] & 1u) : 0u;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * NB; idx += blockDim.x) {
        const int cc = idx / NB, g = idx % NB;
        const int32_t c = c0 + cc;
        if (c >= n_cn) continue;
        uint32_t byte = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) byte |= static_cast<uint32_t>(tile[g * 8 + k][cc]) << k;
        sbits[(static_cast<size_t>(slab) * n_cn + cint[c]) * NB + g] = static_cast<uint8_t>(byte);
    }
}

// bit-sliced hard decisions of a float array [slab][count][W] -> [slab][count][W/8]
template <int W>
__global__ void __launch_bounds__(kBlock) k_hard_bits(const float *post, int32_t count, uint8_t *hb) {
    constexpr int NB = W / 8;
    const int slab = blockIdx.y;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (t >= static_cast<int64_t>(count) * NB) return;
    const size_t u = static_cast<size_t>(t / NB);
    const int g = static_cast<int>(t % NB);
    const float *p = post + (static_cast<size_t>(slab) * count + u) * W + g * 8;
    uint32_t byte = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) byte |= static_cast<uint32_t>(p[k] < 0.f) << k;
    hb[(static_cast<size_t>(slab) * count + u) * NB + g] = static_cast<uint8_t>(byte);
}

struct OutArgs {
    const int32_t *unit;
    int32_t n_vn, n_core, n_deg1, batch;
    const float *Lv, *post1;
    uint8_t *bits;   // [B][n_vn]
    float *post;     // [B][n_vn] or null
};

template <int W>
__global__ void __launch_bounds__(kBlock) k_deinterleave_out(OutArgs a) {
    __shared__ float tile[32][W + 1];
    const int slab = blockIdx.y;
    const int32_t j0 = blockIdx.x * 32;
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int jj = idx / W, w = idx % W;
        const int32_t j = j0 + jj;
        float v = 0.f;
        if (j < a.n_vn) {
            const int32_t u = a.unit[j];
            v = (u < a.n_core) ? a.Lv[(static_cast<size_t>(slab) * a.n_core + u) * W + w]
                               : a.post1[(static_cast<size_t>(slab) * a.n_deg1 + (u - a.n_core)) * W + w];
        }
        tile[jj][w] = v;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int w = idx / 32, jj = idx % 32;
        const int b = slab * W + w;
        const int32_t j = j0 + jj;
        if (b >= a.batch || j >= a.n_vn) continue;
        const float v = tile[jj][w];
        a.bits[static_cast<size_t>(b) * a.n_vn + j] = v < 0.f ? 1 : 0;
        if (a.post) a.post[static_cast<size_t>(b) * a.n_vn + j] = v;
    }
}

template <bool HALF>
__global__ void k_phi_eval(const float *x, float *out, int64_t n, float lmax, float amin) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fminf(phi_f<HALF>(clampf(x[i], amin, lmax)), lmax);
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
double phi_host(double x) { return std::log1p(2.0 / std::expm1(x)); }

int cuda_fail(cudaError_t e, const char *what) {
    return mld::fail(MLD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define MLD_CUDA(call)                                        \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

#define MLD_LAUNCHED(what)                                    \
    do {                                                      \
        cudaError_t e_ = cudaGetLastError();                  \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);    \
    } while (0)

template <typename T>
int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return mld::fail(e == cudaErrorMemoryAllocation ? MLD_ENOMEM : MLD_ECUDA,
                         std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    return MLD_OK;
}

template <typename T>
void dfree(T *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

template <typename T>
int upload(T **dst, const std::vector<T> &src) {
    int st = dalloc(dst, src.size());
    if (st != MLD_OK) return st;
    if (!src.empty()) MLD_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    return MLD_OK;
}

int grid_x(int64_t threads) {
    return static_cast<int>((threads + kBlock - 1) / kBlock);
}

}  // namespace

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
}

// ===========================================================================
// decoder object
// ===========================================================================
struct mld_decoder {
    const mld_graph *g = nullptr;
    int device = 0;
    int msg = MLD_MSG_F32;
    int W = 32;
    int max_batch = 0;
    int max_slabs = 0;
    float lmax = 25.f, amin = 0.f;
    void *r = nullptr;
    float *Lv = nullptr, *lch = nullptr, *lch1 = nullptr, *post1 = nullptr, *phi1 = nullptr;
    uint8_t *hb_core = nullptr, *hb1 = nullptr, *sbits = nullptr;
    uint32_t *done = nullptr, *fail = nullptr;
    int32_t *iters = nullptr;
    uint8_t *conv = nullptr;
    int32_t *status = nullptr;
    // staging buffers for host pointers
    float *in_stage = nullptr, *sigma_stage = nullptr, *post_stage = nullptr;
    uint8_t *syn_stage = nullptr, *bits_stage = nullptr;
    // kernel timing hook
    struct Timed { int cls; cudaEvent_t a, b; };
    bool timing = false;
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
};

namespace {

void decoder_free(mld_decoder *d) {
    if (!d) return;
    if (d->r) cudaFree(d->r);
    d->r = nullptr;
    dfree(d->Lv); dfree(d->lch); dfree(d->lch1); dfree(d->post1); dfree(d->phi1);
    dfree(d->hb_core); dfree(d->hb1); dfree(d->sbits);
    dfree(d->done); dfree(d->fail); dfree(d->iters); dfree(d->conv); dfree(d->status);
    dfree(d->in_stage); dfree(d->sigma_stage); dfree(d->post_stage);
    dfree(d->syn_stage); dfree(d->bits_stage);
    for (auto &t : d->timed) { d->event_pool.push_back(t.a); d->event_pool.push_back(t.b); }
    d->timed.clear();
    for (cudaEvent_t e : d->event_pool) cudaEventDestroy(e);
    d->event_pool.clear();
}

enum { kClsCheck = 0, kClsVar = 1, kClsSyn = 2, kClsLayout = 3 };

cudaEvent_t pool_event(mld_decoder *d) {
    if (!d->event_pool.empty()) {
        cudaEvent_t e = d->event_pool.back();
        d->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch one kernel through `fn`, bracketed by timing events when enabled.
template <typename F>
int timed_launch(mld_decoder *d, int cls, cudaStream_t st, const char *what, F &&fn) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (d->timing) {
        a = pool_event(d);
        b = pool_event(d);
        if (!a || !b) return mld::fail(MLD_ECUDA, "cudaEventCreate");
        MLD_CUDA(cudaEventRecord(a, st));
    }
    fn();
    MLD_LAUNCHED(what);
    if (d->timing) {
        MLD_CUDA(cudaEventRecord(b, st));
        d->timed.push_back({cls, a, b});
    }
    return MLD_OK;
}

int check_device(int want) {
    int dev = -1;
    MLD_CUDA(cudaGetDevice(&dev));
    if (dev != want)
        return mld::fail(MLD_EINVAL, "handle belongs to device " + std::to_string(want) +
                                         " but device " + std::to_string(dev) + " is current");
    return MLD_OK;
}

// Launch the full decode sequence on device buffers.
template <typename MsgT, int W>
int run_decode(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn,
               int32_t batch, int32_t iters, bool et, uint8_t *bits, float *post,
               uint8_t *conv_out, int32_t *iters_out, cudaStream_t st, bool out_dev) {
    const mld::HostGraph &h = d->g->h;
    const mld_graph *g = d->g;
    const int slabs = (batch + W - 1) / W;
    constexpr int TPC = W / kK;
    constexpr int DW = (W + 31) / 32;
    const size_t rbytes = static_cast<size_t>(slabs) * h.e_core * W * sizeof(MsgT);
    if (rbytes) MLD_CUDA(cudaMemsetAsync(d->r, 0, rbytes, st));
    MLD_CUDA(cudaMemsetAsync(d->done, 0, sizeof(uint32_t) * slabs * DW, st));

    InArgs ia{in, sigma, g->unit, h.n_vn, h.n_core, h.n_deg1, batch, d->lmax, d->amin,
              d->lch, d->Lv, d->lch1, d->post1, d->phi1};
    if (h.n_vn > 0) {
        int s = timed_launch(d, kClsLayout, st, "k_interleave_in", [&] {
            k_interleave_in<W, IsHalf<MsgT>::value><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(ia);
        });
        if (s != MLD_OK) return s;
    }
    if (h.n_cn > 0) {
        int s = timed_launch(d, kClsLayout, st, "k_syndrome_in", [&] {
            k_syndrome_in<W><<<dim3((h.n_cn + 31) / 32, slabs), kBlock, 0, st>>>(syn, g->cint, h.n_cn, batch,
                                                                                d->sbits);
        });
        if (s != MLD_OK) return s;
    }

    CnArgs ca{g->cptr, g->col, g->dptr, h.n_cn, h.n_core, h.n_deg1, h.e_core,
              d->r, d->Lv, d->lch1, d->phi1, d->post1, d->hb1, d->sbits, d->done,
              d->lmax, d->amin, 0, et ? 1 : 0};
    VnArgs va{g->vptr, g->vedge, h.n_core, h.e_core, d->r, d->lch, d->Lv, d->hb_core, d->done, 0, et ? 1 : 0};
    SynArgs sa{g->cptr, g->col, g->dptr, h.n_cn, h.n_core, h.n_deg1, d->sbits, d->hb_core, d->hb1,
               d->fail, d->done, et ? 1 : 0};
    // check-update launches, one per check class (built with the graph)
    const int wi = W == 8 ? 0 : (W == 16 ? 1 : (W == 32 ? 2 : 3));
    const std::vector<ClassLaunch> &launches = g->launches[wi];
    const dim3 vn_grid(grid_x(static_cast<int64_t>(h.n_core) * TPC), slabs);
    int sm_count = 152;
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, d->device);
    const int64_t syn_threads = static_cast<int64_t>(h.n_cn) * (W / 8);
    const int syn_blocks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(grid_x(syn_threads), 4LL * sm_count)));
    const dim3 syn_grid(syn_blocks, slabs);
    const int lane_blocks = (batch + 127) / 128;

    auto syndrome_round = [&](int32_t l, bool et_mode) -> int {
        MLD_CUDA(cudaMemsetAsync(d->fail, 0, sizeof(uint32_t) * slabs * DW, st));
        if (h.n_cn > 0) {
            sa.et = et_mode ? 1 : 0;
            int s = timed_launch(d, kClsSyn, st, "k_syndrome_check", [&] {
                k_syndrome_check<W><<<syn_grid, kBlock, 0, st>>>(sa);
            });
            if (s != MLD_OK) return s;
        }
        return timed_launch(d, kClsSyn, st, "k_lane_update", [&] {
            k_lane_update<W><<<lane_blocks, 128, 0, st>>>(d->done, d->fail, d->iters, d->conv, batch, l,
                                                           et_mode ? 1 : 0);
        });
    };

    if (iters == 0) {
        if (h.n_core > 0) {
            int s = timed_launch(d, kClsLayout, st, "k_hard_bits", [&] {
                k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_core) * (W / 8)), slabs), kBlock, 0, st>>>(
                    d->Lv, h.n_core, d->hb_core);
            });
            if (s != MLD_OK) return s;
        }
        if (h.n_deg1 > 0) {
            int s = timed_launch(d, kClsLayout, st, "k_hard_bits", [&] {
                k_hard_bits<W><<<dim3(grid_x(static_cast<int64_t>(h.n_deg1) * (W / 8)), slabs), kBlock, 0, st>>>(
                    d->post1, h.n_deg1, d->hb1);
            });
            if (s != MLD_OK) return s;
        }
        int s = syndrome_round(0, false);
        if (s != MLD_OK) return s;
    }
    for (int32_t l = 1; l <= iters; ++l) {
        const bool last = (l == iters);
        ca.final_pass = (last || et) ? 1 : 0;
        for (const ClassLaunch &cl : launches) {
            int s = timed_launch(d, kClsCheck, st, "k_check_update",
                                 [&] { launch_check_class<MsgT, W>(ca, cl, slabs, st); });
            if (s != MLD_OK) return s;
        }
        va.want_bits = (last || et) ? 1 : 0;
        if (h.n_core > 0) {
            int s = timed_launch(d, kClsVar, st, "k_var_update", [&] {
                k_var_update<MsgT, W><<<vn_grid, kBlock, 0, st>>>(va);
            });
            if (s != MLD_OK) return s;
        }
        if (et || last) {
            int s = syndrome_round(l, et);
            if (s != MLD_OK) return s;
        }
    }

    OutArgs oa{g->unit, h.n_vn, h.n_core, h.n_deg1, batch, d->Lv, d->post1, bits, post};
    if (h.n_vn > 0) {
        int s = timed_launch(d, kClsLayout, st, "k_deinterleave_out", [&] {
            k_deinterleave_out<W><<<dim3((h.n_vn + 31) / 32, slabs), kBlock, 0, st>>>(oa);
        });
        if (s != MLD_OK) return s;
    }
    const cudaMemcpyKind kind = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    MLD_CUDA(cudaMemcpyAsync(conv_out, d->conv, batch, kind, st));
    MLD_CUDA(cudaMemcpyAsync(iters_out, d->iters, sizeof(int32_t) * batch, kind, st));
    return MLD_OK;
}

template <typename MsgT>
int dispatch_w(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn, int32_t batch,
               int32_t iters, bool et, uint8_t *bits, float *post, uint8_t *conv, int32_t *it,
               cudaStream_t st, bool out_dev) {
    switch (d->W) {
        case 8: return run_decode<MsgT, 8>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        case 16: return run_decode<MsgT, 16>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        case 32: return run_decode<MsgT, 32>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        case 64: return run_decode<MsgT, 64>(d, in, sigma, syn, batch, iters, et, bits, post, conv, it, st, out_dev);
        default: return mld::fail(MLD_EINVAL, "unsupported slab width");
    }
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
    const bool dev = (flags & MLD_DEVICE_PTRS) != 0;
    const bool et = (flags & MLD_EARLY_TERM) != 0;
    const size_t nb = static_cast<size_t>(batch) * h.n_vn;
    const size_t mb = static_cast<size_t>(batch) * h.n_cn;
    const float *din = in;
    const float *dsig = y_mode ? sigma : nullptr;
    const uint8_t *dsyn = syndrome;
    uint8_t *dbits = bits_out;
    float *dpost = post_out;
    if (!dev) {
        if (nb) MLD_CUDA(cudaMemcpyAsync(d->in_stage, in, nb * sizeof(float), cudaMemcpyHostToDevice, st));
        if (mb) MLD_CUDA(cudaMemcpyAsync(d->syn_stage, syndrome, mb, cudaMemcpyHostToDevice, st));
        if (y_mode)
            MLD_CUDA(cudaMemcpyAsync(d->sigma_stage, sigma, sizeof(float) * batch, cudaMemcpyHostToDevice, st));
        din = d->in_stage;
        dsyn = d->syn_stage;
        dsig = y_mode ? d->sigma_stage : nullptr;
        dbits = d->bits_stage;
        dpost = post_out ? d->post_stage : nullptr;
    }
    s = (d->msg == MLD_MSG_F16)
            ? dispatch_w<__half>(d, din, dsig, dsyn, batch, max_iters, et, dbits, dpost, converged, iters_used, st, dev)
            : dispatch_w<float>(d, din, dsig, dsyn, batch, max_iters, et, dbits, dpost, converged, iters_used, st, dev);
    if (s != MLD_OK) return s;
    if (!dev) {
        if (nb) MLD_CUDA(cudaMemcpyAsync(bits_out, d->bits_stage, nb, cudaMemcpyDeviceToHost, st));
        if (post_out && nb)
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

int mld_decoder_create(const mld_graph *g, const mld_opts *opts, mld_decoder **out) {
    mld::clear_error();
    if (!g || !opts || !out) return mld::fail(MLD_EINVAL, "decoder_create: null pointer");
    for (int i = 0; i < 12; ++i)
        if (opts->reserved[i] != 0) return mld::fail(MLD_EINVAL, "decoder_create: reserved field not zero");
    if (opts->msg_dtype != MLD_MSG_F32 && opts->msg_dtype != MLD_MSG_F16)
        return mld::fail(MLD_EINVAL, "decoder_create: unknown msg_dtype");
    if (opts->max_batch < 1) return mld::fail(MLD_EINVAL, "decoder_create: max_batch < 1");
    if (!(opts->lmax >= 0.f) || !std::isfinite(opts->lmax) || opts->lmax > 60.f)
        return mld::fail(MLD_EINVAL, "decoder_create: lmax must be in (0, 60]");
    int W = opts->slab_width;
    if (W == 0) W = (opts->msg_dtype == MLD_MSG_F16) ? 64 : 32;
    if (W != 8 && W != 16 && W != 32 && W != 64) return mld::fail(MLD_EINVAL, "decoder_create: slab_width");
    int s = check_device(g->device);
    if (s != MLD_OK) return s;
    mld_decoder *d = new (std::nothrow) mld_decoder();
    if (!d) return mld::fail(MLD_ENOMEM, "decoder_create: host allocation");
    d->g = g;
    d->device = g->device;
    d->msg = opts->msg_dtype;
    d->W = W;
    d->max_batch = opts->max_batch;
    d->max_slabs = (opts->max_batch + W - 1) / W;
    d->lmax = opts->lmax > 0.f ? opts->lmax : 25.f;
    d->amin = static_cast<float>(phi_host(static_cast<double>(d->lmax)));
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
    if (s == MLD_OK) s = dalloc(&d->lch1, S * h.n_deg1 * W);
    if (s == MLD_OK) s = dalloc(&d->post1, S * h.n_deg1 * W);
    if (s == MLD_OK) s = dalloc(&d->phi1, S * h.n_deg1 * W);
    if (s == MLD_OK) s = dalloc(&d->hb_core, S * h.n_core * NB);
    if (s == MLD_OK) s = dalloc(&d->hb1, S * h.n_deg1 * NB);
    if (s == MLD_OK) s = dalloc(&d->sbits, S * h.n_cn * NB);
    if (s == MLD_OK) s = dalloc(&d->done, S * DW);
    if (s == MLD_OK) s = dalloc(&d->fail, S * DW);
    if (s == MLD_OK) s = dalloc(&d->iters, S * W);
    if (s == MLD_OK) s = dalloc(&d->conv, S * W);
    if (s == MLD_OK) s = dalloc(&d->status, 1);
    if (s == MLD_OK) s = dalloc(&d->in_stage, nb);
    if (s == MLD_OK) s = dalloc(&d->sigma_stage, static_cast<size_t>(d->max_batch));
    if (s == MLD_OK) s = dalloc(&d->post_stage, nb);
    if (s == MLD_OK) s = dalloc(&d->syn_stage, static_cast<size_t>(d->max_batch) * h.n_cn);
    if (s == MLD_OK) s = dalloc(&d->bits_stage, nb);
    if (s == MLD_OK) {
        cudaError_t e2 = cudaMemset(d->status, 0, sizeof(int32_t));
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
    int32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, d->status, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "decode_status");
    return v == 0 ? MLD_OK : mld::fail(v, "device-detected error");
}

int mld_decoder_timing_enable(mld_decoder *d, int enable) {
    mld::clear_error();
    if (!d) return mld::fail(MLD_EINVAL, "timing_enable: null decoder");
    d->timing = enable != 0;
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
            case kClsCheck: out->check_ms += ms; out->check_launches++; break;
            case kClsVar: out->var_ms += ms; out->var_launches++; break;
            case kClsSyn: out->syndrome_ms += ms; out->syndrome_launches++; break;
            default: out->layout_ms += ms; out->layout_launches++; break;
        }
        d->event_pool.push_back(t.a);
        d->event_pool.push_back(t.b);
    }
    d->timed.clear();
    return status;
}

int mld_phi_eval(int32_t msg_dtype, const float *x, float *out, int64_t n, void *stream) {
    mld::clear_error();
    if (msg_dtype != MLD_MSG_F32 && msg_dtype != MLD_MSG_F16) return mld::fail(MLD_EINVAL, "phi_eval: msg_dtype");
    if (n < 0 || (n > 0 && (!x || !out))) return mld::fail(MLD_EINVAL, "phi_eval: bad arguments");
    if (n == 0) return MLD_OK;
    const float lmax = 25.f;
    const float amin = static_cast<float>(phi_host(25.0));
    if (msg_dtype == MLD_MSG_F16)
        k_phi_eval<true><<<grid_x(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n, lmax, amin);
    else
        k_phi_eval<false><<<grid_x(n), kBlock, 0, static_cast<cudaStream_t>(stream)>>>(x, out, n, lmax, amin);
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
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
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
    L.hb1 = take(S * h.n_deg1 * NB);
    L.sbits = take(S * h.n_cn * NB);
    L.done = take(S * DW * sizeof(uint32_t));
    L.fail = take(S * DW * sizeof(uint32_t));
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
    d.lmax = 25.f;
    d.amin = static_cast<float>(phi_host(25.0));
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
               ? dispatch_w<__half>(&d, llr, nullptr, syndrome, batch, max_iters, et, bits_out, post_out,
                                    converged, iters_used, st, true)
               : dispatch_w<float>(&d, llr, nullptr, syndrome, batch, max_iters, et, bits_out, post_out,
                                   converged, iters_used, st, true);
}
