// Device code and host helpers shared by the translation units of
// libmetldpc.so (decoder.cu: single-graph decoding and the C ABI; multi.cu:
// batches over several graphs).  Everything here has internal linkage.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "phi_poly.h"

namespace mld {
const char *last_error_text();
}

namespace {

constexpr int kK = 4;          // codewords per thread
constexpr int kBlock = 128;

// ---------------------------------------------------------------------------
// phi(x) = -ln tanh(x/2) in float, for x in [phi(lmax), lmax].
// Three fits (see gen_phi_poly.py):
//   kFitNat : LLRs in nats (weighted BP): below MLD_PHI_X0, ln2 - ln x - t Ps(t)
//             with t = x^2; above, e Pl(e^2) with e = exp(-x).
//   kFitB2  : LLRs in bits, y = x log2 e (decoding, float storage): the same
//             map psi(y) = log2(e) phi(y ln 2) as the larger of
//             C0 - lg2 y - u Qs(u) (u = y^2; accurate below MLD_PHI2_Y0) and
//             e Ql(e^2) (e = 2^-y; accurate above); error 1.5e-7 relative.
//   kFitB2H : as kFitB2 with two coefficients per piece (half storage; error
//             2.0e-4 relative, below half's 2^-11 rounding).
// ln and exp come from the MUFU base-2 approximations.
// ---------------------------------------------------------------------------
enum Fit { kFitNat = 0, kFitB2 = 1, kFitB2H = 2 };

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

template <int F>
__device__ __forceinline__ float phi_small(float x) {
    const float t = x * x;
    float ps;
    if constexpr (F == kFitNat) {
        const float kLn2 = 0.693147180559945309f;
        ps = fmaf(MLD_PHI_S4, t, MLD_PHI_S3);
        ps = fmaf(ps, t, MLD_PHI_S2);
        ps = fmaf(ps, t, MLD_PHI_S1);
        ps = fmaf(ps, t, MLD_PHI_S0);
        return fmaf(-t, ps, fmaf(-kLn2, mufu_lg2(x), kLn2));
    } else {
        if constexpr (F == kFitB2H) {
            ps = fmaf(MLD_PHI2H_S1, t, MLD_PHI2H_S0);
        } else {
            ps = fmaf(MLD_PHI2_S3, t, MLD_PHI2_S2);
            ps = fmaf(ps, t, MLD_PHI2_S1);
            ps = fmaf(ps, t, MLD_PHI2_S0);
        }
        return fmaf(-t, ps, MLD_PHI2_C0) - mufu_lg2(x);
    }
}

template <int F>
__device__ __forceinline__ float phi_large(float x) {
    float e;
    if constexpr (F == kFitNat) e = mufu_ex2(-1.442695040888963407f * x);
    else e = mufu_ex2(-x);
    const float z = e * e;
    float pl;
    if constexpr (F == kFitNat) {
        pl = fmaf(MLD_PHI_L3, z, MLD_PHI_L2);
        pl = fmaf(pl, z, MLD_PHI_L1);
        pl = fmaf(pl, z, MLD_PHI_L0);
    } else if constexpr (F == kFitB2H) {
        pl = fmaf(MLD_PHI2H_L1, z, MLD_PHI2H_L0);
    } else {
        pl = fmaf(MLD_PHI2_L3, z, MLD_PHI2_L2);
        pl = fmaf(pl, z, MLD_PHI2_L1);
        pl = fmaf(pl, z, MLD_PHI2_L0);
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

// phi of one value: both pieces are evaluated without branches, so the
// compiler can interleave independent chains.  In the base-2 fits the top
// coefficient of Qs is positive, so past the split the small piece falls
// below the large one (to -inf), and below the split the large piece stays
// under the small one: their maximum is the right piece (near the split,
// where both are accurate, whichever is larger).  One max replaces the
// compare and select; gen_phi_poly.py checks the ordering on the whole range.
template <int F>
__device__ __forceinline__ float phi_f(float x) {
    if constexpr (F == kFitNat)
        return sel_lt(x, MLD_PHI_X0, phi_small<F>(x), phi_large<F>(x));
    else
        return fmaxf(phi_small<F>(x), phi_large<F>(x));
}

// Three-input max (sm_100 and later).
__device__ __forceinline__ float max3f(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// phi of four values with the result floored at `lo`, base-2 fits: the max
// of the two pieces and the floor in one instruction per value.  With
// lo = phi(lmax) this equals phi of the argument clamped above at lmax (phi
// decreases), and an argument of +inf gives lo (the small piece is -inf,
// the large one 0), so the clamp needs no instruction of its own.
template <int F>
__device__ __forceinline__ float4 phi4_floor(float4 x, float lo) {
    static_assert(F == kFitB2 || F == kFitB2H, "phi4_floor: base-2 fits only");
    return make_float4(max3f(phi_small<F>(x.x), phi_large<F>(x.x), lo),
                       max3f(phi_small<F>(x.y), phi_large<F>(x.y), lo),
                       max3f(phi_small<F>(x.z), phi_large<F>(x.z), lo),
                       max3f(phi_small<F>(x.w), phi_large<F>(x.w), lo));
}

template <typename T> struct IsHalf { static constexpr bool value = false; };
template <> struct IsHalf<__half> { static constexpr bool value = true; };
// the fit the decoding kernels use for a message storage type
template <typename T> struct DecodeFit { static constexpr int value = IsHalf<T>::value ? kFitB2H : kFitB2; };

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
    // store v and return the values as stored
    static __device__ __forceinline__ float4 store_get(float *p, float4 v) {
        *reinterpret_cast<float4 *>(p) = v;
        return v;
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
    static __device__ __forceinline__ float4 store_get(__half *p, float4 v) {
        const __half2 a = __floats2half2_rn(v.x, v.y);
        const __half2 b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<const uint32_t *>(&a);
        u.y = *reinterpret_cast<const uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
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
    uint8_t *hb1;          // [slab][n_deg1][W/8] degree-1 hard decisions written by this pass
    const uint8_t *sbits;  // [slab][n_cn][W/8] syndrome bits
    const uint32_t *done;  // [slab][ceil(W/32)] converged lanes (ET)
    float lmax, amin;
    int final_pass, et;
    // Fused syndrome check (early termination without soft output): this
    // pass also forms the syndrome of the previous iteration from the signs
    // of the posteriors it reads and the previous degree-1 decisions, and ORs
    // the failing codewords into fail_prev.
    int fuse;
    int32_t batch;              // codewords (later lanes are padding)
    const uint8_t *hb1_prev;    // degree-1 decisions of the previous iteration
    uint32_t *fail_prev;        // [slab][ceil(W/32)] fail words of the previous iteration
    // Posterior accumulation (fixed iterations only): each new message, as
    // stored, is added to this [slab][n_core][W] array, which holds L_ch on
    // entry and L_v of this iteration (Eq. 4) once the pass is complete.
    // Null: the variable update gathers the messages instead.
    float *acc;
    // Check rule: 0 sum-product (Eqs. 2-3), 1 offset min-sum with offset
    // ms_off (internal units).
    int rule;
    float ms_off;
    // Decoder status word (int32[4]); a staged check update whose bulk copy
    // never completes records MLD_ETIMEOUT here.  May be null elsewhere.
    int32_t *status;
    // Test of the timeout path: bytes added to the byte count that block
    // (0, 0) of a staged check update expects for its first stage, so that
    // its wait runs out (0: none).
    int32_t stall_test;
};

enum { kRuleSumProduct = 0, kRuleMinSum = 1 };

template <typename MsgT, int W>
__device__ __forceinline__ void emit_deg1(const CnArgs &a, int slab, int slot, int lane0,
                                          float4 rv, uint32_t donenib, bool valid) {
    constexpr int NB = W / 8;
    const size_t base = (static_cast<size_t>(slab) * a.n_deg1 + slot) * W + lane0;
    const float4 l = ldf4(a.lch1 + base);  // in range: the slot of a real check
    float4 post = make_float4(l.x + rv.x, l.y + rv.y, l.z + rv.z, l.w + rv.w);
    uint32_t nib = (post.x < 0.f) | ((post.y < 0.f) << 1) | ((post.z < 0.f) << 2) | ((post.w < 0.f) << 3);
    uint8_t *hb = a.hb1 + (static_cast<size_t>(slab) * a.n_deg1 + slot) * NB + lane0 / 8;
    // converged lanes keep their posterior and what this decision buffer
    // holds for them (their output is read from the buffer of their last
    // iteration's parity, which later passes leave unchanged)
    if (donenib && valid) {
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

// Decisions of a degree-1 VN for 4 codewords (bit k: codeword lane0 + k) into
// its bit-sliced byte of this pass's buffer; converged lanes keep what the
// byte holds (see emit_deg1).  Both threads of a shuffle pair must call it.
template <int W>
__device__ __forceinline__ void emit_deg1_bits(const CnArgs &a, int slab, int slot, int lane0, uint32_t nib,
                                               uint32_t donenib, bool valid) {
    constexpr int NB = W / 8;
    uint8_t *hb = a.hb1 + (static_cast<size_t>(slab) * a.n_deg1 + slot) * NB + lane0 / 8;
    if (donenib && valid) {
        const uint32_t oldnib = (static_cast<uint32_t>(*hb) >> (lane0 & 7)) & 0xFu;
        nib = (nib & ~donenib) | (oldnib & donenib);
    }
    const uint32_t other = __shfl_xor_sync(pair_mask(), nib, 1);
    if (valid && (lane0 & 7) == 0) *hb = static_cast<uint8_t>(nib | (other << 4));
}

// Message store under early termination: converged lanes keep their
// messages frozen.  The freeze is not needed for exact outputs (a converged
// codeword's posterior and decisions are frozen by the variable update and
// emit_deg1*, and no output reads its later messages), so the
// decisions-only kernels skip it (FREEZE false), which saves a reload and
// four selects per term once lanes have converged.
template <typename MsgT, int W, bool FREEZE = true>
__device__ __forceinline__ void store_r(const CnArgs &a, MsgT *rp, float4 rv, uint32_t donenib) {
    if (FREEZE && donenib) {
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

// Check j of one class (DC core edges and DD degree-1 VNs per check, all
// terms in registers), codewords lane0 .. lane0+3 of the slab.  A thread past
// the class end works on its last check and stores nothing (so a whole
// shuffle pair stays active).  HARD1: a degree-1 VN gets its decision only,
// not its posterior (early termination without soft output); FUSE (with
// HARD1): with a.fuse the call also returns the previous iteration's
// syndrome failures of the check for the thread's 4 codewords (bit k:
// codeword lane0 + k), else 0.
// Where a check's terms are read from.  TermsGlobal: straight from the
// posterior, message and degree-1 arrays, the core VNs' column indices
// loaded first; lv(i) / ro(i): posterior and stored message of core term i,
// p1(i): phi term of degree-1 term i, each for the thread's 4 codewords.
template <typename MsgT, int W, int DC>
struct TermsGlobal {
    const float *lvb;
    const MsgT *rb;
    const float *p1b;
    int32_t e0, s0;
    int32_t vidx[DC > 0 ? DC : 1];
    __device__ __forceinline__ float4 lv(int i) const { return ldf4(lvb + static_cast<size_t>(vidx[i]) * W); }
    __device__ __forceinline__ float4 ro(int i) const {
        return Msg<MsgT>::load(rb + static_cast<size_t>(e0 + i) * W);
    }
    __device__ __forceinline__ float4 p1(int i) const { return ldf4(p1b + static_cast<size_t>(s0 + i) * W); }
};

template <typename MsgT, int W, int DC, int DD, bool HARD1, bool ACC, bool FUSE, typename Terms>
__device__ __forceinline__ uint32_t check_terms(const CnArgs &a, int lane0, int slab, bool valid, int32_t e0,
                                                int32_t s0, uint32_t sb, uint32_t donenib, const Terms &t);

template <typename MsgT, int W, int DC, int DD, bool HARD1 = false, bool ACC = false, bool FUSE = HARD1>
__device__ __forceinline__ uint32_t check_regular(const CnArgs &a, const ClassLaunch &cl, int32_t j, int lane0,
                                                  int slab) {
    constexpr int NB = W / 8;
    const int32_t count = cl.count;
    const bool valid = j < count;
    if (!valid) j = count - 1;
    const int32_t c = cl.c0 + j;
    const int32_t e0 = cl.e0 + j * DC;
    const int32_t s0 = cl.s0 + j * DD;

    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >>
         (lane0 & 7));
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    TermsGlobal<MsgT, W, DC> t;
    t.rb = static_cast<const MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    t.lvb = a.Lv + static_cast<size_t>(slab) * a.n_core * W + lane0;
    t.p1b = a.phi1 + static_cast<size_t>(slab) * a.n_deg1 * W + lane0;
    t.e0 = e0;
    t.s0 = s0;
#pragma unroll
    for (int i = 0; i < DC; ++i) t.vidx[i] = __ldg(a.col + e0 + i);
    return check_terms<MsgT, W, DC, DD, HARD1, ACC, FUSE>(a, lane0, slab, valid, e0, s0, sb, donenib, t);
}

// The update of one check from its terms (read through t), codewords lane0
// .. lane0+3 of the slab; valid false: compute but store nothing.  sb: the
// check's syndrome bits for the 4 codewords (bit k: lane0 + k); donenib:
// their converged flags under early termination.
template <typename MsgT, int W, int DC, int DD, bool HARD1, bool ACC, bool FUSE, typename Terms>
__device__ __forceinline__ uint32_t check_terms(const CnArgs &a, int lane0, int slab, bool valid, int32_t e0,
                                                int32_t s0, uint32_t sb, uint32_t donenib, const Terms &t) {
    constexpr int NB = W / 8;
    constexpr int D = DC + DD;
    constexpr int dc = DC;
    constexpr int F = DecodeFit<MsgT>::value;
    const float lmax = a.lmax, amin = a.amin;
    MsgT *rb = static_cast<MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;

    // pass 1: f = phi(|q|) carrying the sign of q in its sign bit; the top
    // bit of par accumulates the sign parity (syndrome bit included).  For a
    // degree-1 VN q is its channel LLR, whose f was formed once on entry.
    float f[D][kK];
    uint32_t par[kK];
    uint32_t lvs[kK] = {0u, 0u, 0u, 0u};  // sign parity of the posteriors read (fused syndrome)
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) par[kk] = ((sb >> kk) & 1u) << 31;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i < dc) {
            const float4 lv = t.lv(i);
            if constexpr (HARD1 && FUSE) {
#pragma unroll
                for (int kk = 0; kk < kK; ++kk) lvs[kk] ^= fbits(f4get(lv, kk));
            }
            const float4 ro = t.ro(i);
            const float4 q = make_float4(lv.x - ro.x, lv.y - ro.y, lv.z - ro.z, lv.w - ro.w);
            // phi(|q|) floored at amin = phi(lmax) is phi of |q| clamped above at
            // lmax.  |q| is not clamped below: an argument under phi(lmax)
            // gives a term above lmax (up to +inf at 0), which floors every
            // other term's output at amin exactly as the clamped term would;
            // terms are only added, so no inf - inf arises
            const float4 m = make_float4(fabsf(q.x), fabsf(q.y), fabsf(q.z), fabsf(q.w));
            const float4 ph = phi4_floor<F>(m, amin);
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                const uint32_t qb = fbits(f4get(q, kk));
                f[i][kk] = bitsf(fbits(f4get(ph, kk)) | (qb & kSign));
                par[kk] ^= qb;
            }
        } else {
            const float4 p = t.p1(i - dc);
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                f[i][kk] = f4get(p, kk);
                par[kk] ^= fbits(f[i][kk]);
            }
        }
    }
    // exclusive prefix sums of |f| (pre[0], which would be 0, is not formed:
    // no addition below has a zero operand)
    float pre[D][kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
        if (D >= 2) pre[1][kk] = fabsf(f[0][kk]);
#pragma unroll
        for (int i = 2; i < D; ++i) pre[i][kk] = pre[i - 1][kk] + fabsf(f[i - 1][kk]);
    }
    // pass 2 (backwards): leave-one-out sum = prefix + suffix
    float suf[kK];
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        if (i < dc || a.final_pass) {
            // the output floored at amin is phi of the sum clamped above at
            // lmax.  Every other term is >= amin, so for D >= 3 the sum is at
            // least 2 amin and phi of it stays below lmax; for D <= 2 the
            // output is also clamped above
            float4 o;
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                float v;
                if (D == 1) v = amin;                      // no other term
                else if (i == D - 1) v = pre[i][kk];       // no suffix
                else if (i == 0) v = suf[kk];              // no prefix
                else v = pre[i][kk] + suf[kk];
                f4set(o, kk, v);
            }
            if (HARD1 && i >= dc) {
                // degree-1 VN, decisions only: the posterior L_ch + r is
                // negative when both are, or when the negative one is the
                // larger in magnitude; phi is a decreasing involution, so
                // |r| = phi(o) > |L_ch| exactly when o < phi(|L_ch|) = |f|
                uint32_t nib = 0;
#pragma unroll
                for (int kk = 0; kk < kK; ++kk) {
                    const uint32_t fb = fbits(f[i][kk]);
                    const bool l_neg = (fb & kSign) != 0;
                    const bool r_neg = ((par[kk] ^ fb) & kSign) != 0;
                    const float fl = fabsf(f[i][kk]), ov = f4get(o, kk);
                    const bool neg = (l_neg == r_neg) ? l_neg : (l_neg ? fl < ov : fl > ov);
                    nib |= static_cast<uint32_t>(neg) << kk;
                }
                emit_deg1_bits<W>(a, slab, s0 + i - dc, lane0, nib, donenib, valid);
            } else {
                float4 m = phi4_floor<F>(o, amin);
                if (D <= 2) m = make_float4(fminf(m.x, lmax), fminf(m.y, lmax), fminf(m.z, lmax), fminf(m.w, lmax));
                float4 rv;
#pragma unroll
                for (int kk = 0; kk < kK; ++kk)
                    f4set(rv, kk, bitsf(fbits(f4get(m, kk)) | ((par[kk] ^ fbits(f[i][kk])) & kSign)));
                if (i < dc) {
                    if (valid) {
                        MsgT *rp = rb + static_cast<size_t>(e0 + i) * W;
                        if constexpr (ACC) {
                            // the message as stored joins its VN's posterior
                            const float4 st = Msg<MsgT>::store_get(rp, rv);
                            // (the column index is loaded again, an L1 hit, rather than kept
                            // live through both passes)
                            const int32_t v = __ldg(a.col + e0 + i);
                            float *ap = a.acc + (static_cast<size_t>(slab) * a.n_core + v) * W + lane0;
                            atomicAdd(reinterpret_cast<float4 *>(ap), st);
                        } else if (a.et) {
                            store_r<MsgT, W, !HARD1>(a, rp, rv, donenib);
                        } else {
                            Msg<MsgT>::store(rp, rv);
                        }
                    }
                } else {
                    emit_deg1<MsgT, W>(a, slab, s0 + i - dc, lane0, rv, donenib, valid);
                }
            }
        }
        if (i > 0) {
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) suf[kk] = (i == D - 1) ? fabsf(f[i][kk]) : suf[kk] + fabsf(f[i][kk]);
        }
    }
    uint32_t fail = 0;
    if constexpr (HARD1 && FUSE) {
        if (a.fuse && valid) {
            // previous iteration: s_c XOR the decisions of the check's VNs
            // (core: posterior < 0, the sign read above; degree-1: stored bit)
            uint32_t x = sb & 0xFu;
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) x ^= (lvs[kk] >> 31) << kk;
            if (DD == 1)
                x ^= (static_cast<uint32_t>(a.hb1_prev[(static_cast<size_t>(slab) * a.n_deg1 + s0) * NB + lane0 / 8]) >>
                      (lane0 & 7)) & 0xFu;
            const int lanes = a.batch - slab * W - lane0;  // real codewords among the 4
            const uint32_t real = lanes >= kK ? 0xFu : (lanes > 0 ? (1u << lanes) - 1u : 0u);
            fail = x & real & ~donenib;
        }
    }
    return fail;
}

// ORs the fused syndrome failures of a block's threads (4 codewords each,
// at lane0) into the fail words of the slab: warp reduction, then one atomic
// per word and warp.  Every thread of the block must call it.
template <int W>
__device__ __forceinline__ void flush_fail(uint32_t *fail_slab, uint32_t nib, int lane0) {
    constexpr int DW = (W + 31) / 32;
    uint32_t lo = lane0 < 32 ? nib << lane0 : 0u;
    uint32_t hi = lane0 >= 32 ? nib << (lane0 - 32) : 0u;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo |= __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        if (DW > 1) hi |= __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (lo) atomicOr(fail_slab, lo);
        if (DW > 1 && hi) atomicOr(fail_slab + 1, hi);
    }
}

// Checks of any degree, edges read through cptr/dptr; leave-one-out sums as
// total minus own term.  Threads of a check pair stay together; nothing here
// needs the whole warp.
template <typename MsgT, int W>
__device__ __forceinline__ void check_irregular(const CnArgs &a, const ClassLaunch &cl, int64_t lt, int slab) {
    constexpr int TPC = W / kK;
    constexpr int NB = W / 8;
    constexpr int F = DecodeFit<MsgT>::value;
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
            S[kk] += phi_f<F>(clampf(fabsf(qk), amin, lmax));
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
            const float fk = phi_f<F>(clampf(fabsf(qk), amin, lmax));
            const float mk = fminf(phi_f<F>(clampf(S[kk] - fk, amin, lmax)), lmax);
            f4set(rv, kk, bitsf(fbits(mk) | ((par[kk] ^ fbits(qk)) & kSign)));
        }
        if (out_core)
            store_r<MsgT, W>(a, rb + static_cast<size_t>(e0 + i) * W, rv, donenib);
        else
            emit_deg1<MsgT, W>(a, slab, s0 + i - nce, lane0, rv, donenib, true);
    }
}

// Classes of at most 6 terms loop over their checks on a capped grid: a
// thread's set-up (indices, slab bases) is then shared by several checks.
// The 7- and 8-term classes (80 registers) take one check per thread.
template <int D> constexpr bool kLoopedClass = D <= 6;

// The threads of a class launch (t0: thread index in the slab's grid of
// `blocks` blocks): looped classes step through their checks, the others take
// one; with HARD1 the fused syndrome failures are ORed into a.fail_prev.
template <typename MsgT, int W, int DC, int DD, bool HARD1, bool ACC = false, bool FUSE = HARD1>
__device__ __forceinline__ void check_class_body(const CnArgs &a, const ClassLaunch &cl, int64_t t0,
                                                 int32_t blocks, int slab) {
    constexpr int TPC = W / kK;
    const int lane0 = static_cast<int>(t0 % TPC) * kK;
    uint32_t fail = 0;
    if constexpr (kLoopedClass<DC + DD>) {
        // a capped grid; each thread takes every stride-th check with the
        // same lanes, so its set-up is shared by several checks.  Both
        // threads of a shuffle pair belong to one check and leave together.
        const int32_t jstride = blocks * (kBlock / TPC);
        for (int32_t j = static_cast<int32_t>(t0 / TPC); j < cl.count; j += jstride)
            fail |= check_regular<MsgT, W, DC, DD, HARD1, ACC, FUSE>(a, cl, j, lane0, slab);
    } else {
        fail = check_regular<MsgT, W, DC, DD, HARD1, ACC, FUSE>(a, cl, static_cast<int32_t>(t0 / TPC), lane0, slab);
    }
    if constexpr (HARD1 && FUSE) {
        if (a.fuse) flush_fail<W>(a.fail_prev + slab * ((W + 31) / 32), fail, lane0);
    }
}

// One check class per launch, its shape (DC, DD) a compile-time constant: the
// register arrays are sized exactly and only this class's code is hot.
// HARD1 without FUSE (decisions only, the syndrome checked by its own
// kernel): 7 blocks per SM, 72 registers without spills.
template <typename MsgT, int W, int DC, int DD, bool HARD1, bool ACC = false, bool FUSE = HARD1>
__global__ void __launch_bounds__(kBlock, (DC + DD <= 6 ? ((ACC || (HARD1 && !FUSE)) ? 7 : 8) : 6))
    k_check_update(CnArgs a, ClassLaunch cl) {
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;  // block-uniform
    check_class_body<MsgT, W, DC, DD, HARD1, ACC, FUSE>(a, cl,
                                                  static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x,
                                                  static_cast<int32_t>(gridDim.x), slab);
}

// ---------------------------------------------------------------------------
// Staged check update.  The classes of at most six terms can also run with
// their operands brought into shared memory by the bulk-copy (TMA) engine
// one stage ahead of the arithmetic: a stage is G consecutive checks of the
// class (one per group of W/4 threads); its message rows and degree-1 terms
// are two contiguous copies, its posterior rows one 16-byte-aligned copy per
// core edge (issued by the thread that loaded that edge's column index a
// stage earlier).  Completion is tracked by one mbarrier per buffer (two
// buffers); the arithmetic is check_terms, reading shared memory.  Every
// wait is bounded in time: a copy that has not landed after kWaitLimitNs
// records MLD_ETIMEOUT in the status word and the block leaves, storing
// nothing for that stage.
// ---------------------------------------------------------------------------
constexpr int kStagedBlocksPerSm = 6;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for the phase of the given parity to complete; false after
// limit_ns without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}
// After a wait has run out: how long to give the copies still in flight.
constexpr unsigned long long kDrainNs = 100000000ull;
// Orders this thread's earlier generic-proxy accesses of shared memory
// before its later bulk copies into it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bulk copy global -> shared (both addresses 16-byte aligned, bytes a
// multiple of 16), completing as transaction bytes on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// 16-byte asynchronous copy global -> shared through the load/store unit
// (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// Arrive on the mbarrier once this thread's earlier cp.async copies have
// landed; counts as one of the phase's expected arrivals.
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

template <typename MsgT, int W, int DC, int DD>
struct StageShape {
    static constexpr int TPC = W / kK;                               // threads per check
    static constexpr int G = kBlock / TPC;                           // checks per stage
    static constexpr int kMsgRow = W * static_cast<int>(sizeof(MsgT));
    static constexpr int kF32Row = W * 4;
    static constexpr int kMsg = G * DC * kMsgRow;                    // message rows
    static constexpr int kP1 = G * DD * kF32Row;                     // degree-1 terms
    static constexpr int kPost = G * DC * kF32Row;                   // posterior rows
    static constexpr int kStage = kMsg + kP1 + kPost;
    static constexpr int kBytes = 2 * kStage + 2 * 8;                // two buffers, two mbarriers
    static constexpr int kPerCheck = DC * kMsgRow + DD * kF32Row + DC * kF32Row;
};

// Terms of one check in a stage buffer (pointers already at the thread's
// lane0).
template <typename MsgT, int W>
struct TermsShared {
    const float *post;
    const MsgT *msg;
    const float *phi;
    __device__ __forceinline__ float4 lv(int i) const { return *reinterpret_cast<const float4 *>(post + i * W); }
    __device__ __forceinline__ float4 ro(int i) const { return Msg<MsgT>::load(msg + i * W); }
    __device__ __forceinline__ float4 p1(int i) const { return *reinterpret_cast<const float4 *>(phi + i * W); }
};

// A capped grid; block b takes stages b, b + gridDim.x, ...  Sum-product,
// no fused syndrome (HARD1 false), no accumulation.  LSU false: each
// posterior row is one bulk copy, issued by the thread that loaded its
// column index; LSU true: every thread copies its own 16 bytes of each of
// its check's posterior rows with cp.async (the load/store unit, not the
// bulk-copy engine) and signals the stage's mbarrier when they land.
template <typename MsgT, int W, int DC, int DD, bool LSU>
__global__ void __launch_bounds__(kBlock, kStagedBlocksPerSm) k_check_staged(CnArgs a, ClassLaunch cl) {
    using S = StageShape<MsgT, W, DC, DD>;
    static_assert(DC + DD > 0 && DD <= 1, "staged classes");
    constexpr int NC = DC > 0 ? DC : 1;
    extern __shared__ __align__(128) unsigned char smem[];
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;  // block-uniform
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + 2 * S::kStage);
    const int tid = threadIdx.x;
    const int g = tid / S::TPC;
    const int lane0 = (tid % S::TPC) * kK;
    const int32_t count = cl.count;
    const int32_t stages = (count + S::G - 1) / S::G;
    const int32_t step = static_cast<int32_t>(gridDim.x);
    if (tid == 0) {
        // LSU: one arrival from thread 0 (with the byte count of the bulk
        // copies) and one from each thread's cp.async group per phase
        mbar_init(&full[0], LSU ? 1 + kBlock : 1);
        mbar_init(&full[1], LSU ? 1 + kBlock : 1);
        mbar_init_fence();
    }
    __syncthreads();
    const MsgT *rsrc = static_cast<const MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W;
    const float *lvsrc = a.Lv + static_cast<size_t>(slab) * a.n_core * W;
    const float *p1src = a.phi1 + static_cast<size_t>(slab) * a.n_deg1 * W;
    constexpr int NB = W / 8;
    constexpr uint32_t kBulkPerCheck = LSU ? DC * S::kMsgRow + DD * S::kF32Row : S::kPerCheck;

    // column indices for the posterior copies of stage st (-1: none).  Bulk:
    // thread tid < G*DC takes row tid of the stage (check tid / DC, term
    // tid % DC) in v[0].  LSU: a thread takes the DC rows of its own check.
    auto cols_of = [&](int32_t st, int32_t (&v)[NC]) {
#pragma unroll
        for (int i = 0; i < NC; ++i) v[i] = -1;
        if constexpr (DC > 0) {
            if (st >= stages) return;
            if constexpr (LSU) {
                const int32_t j = st * S::G + g;
                if (j < count) {
#pragma unroll
                    for (int i = 0; i < DC; ++i) v[i] = __ldg(a.col + cl.e0 + j * DC + i);
                }
            } else {
                if (tid >= S::G * DC) return;
                const int32_t j = st * S::G + tid / DC;
                if (j < count) v[0] = __ldg(a.col + cl.e0 + j * DC + tid % DC);
            }
        }
    };
    auto sb_of = [&](int32_t st) -> uint32_t {
        const int32_t j = min(st * S::G + g, count - 1);
        return static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + cl.c0 + j) * NB + lane0 / 8]) >>
               (lane0 & 7);
    };
    auto issue = [&](int32_t st, int buf, const int32_t (&v)[NC]) {
        unsigned char *base = smem + buf * S::kStage;
        const int32_t j0 = st * S::G;
        const int32_t nv = min(S::G, count - j0);
        if (tid == 0) {
            fence_proxy_async_smem();
            const uint32_t extra =
                (a.stall_test > 0 && blockIdx.x == 0 && blockIdx.y == 0 && st == 0) ? a.stall_test : 0;
            mbar_arrive_expect_tx(&full[buf], static_cast<uint32_t>(nv) * kBulkPerCheck + extra);
            if (DC > 0)
                bulk_g2s(base, rsrc + static_cast<size_t>(cl.e0 + j0 * DC) * W,
                         static_cast<uint32_t>(nv * DC * S::kMsgRow), &full[buf]);
            if (DD > 0)
                bulk_g2s(base + S::kMsg, p1src + static_cast<size_t>(cl.s0 + j0 * DD) * W,
                         static_cast<uint32_t>(nv * DD * S::kF32Row), &full[buf]);
        }
        if constexpr (LSU) {
            float *post = reinterpret_cast<float *>(base + S::kMsg + S::kP1) + g * DC * W + lane0;
#pragma unroll
            for (int i = 0; i < DC; ++i)
                if (v[i] >= 0) cp_async16(post + i * W, lvsrc + static_cast<size_t>(v[i]) * W + lane0);
            cp_async_arrive_noinc(&full[buf]);
        } else {
            if (v[0] >= 0) {
                if (tid != 0) fence_proxy_async_smem();
                bulk_g2s(base + S::kMsg + S::kP1 + tid * S::kF32Row, lvsrc + static_cast<size_t>(v[0]) * W,
                         static_cast<uint32_t>(S::kF32Row), &full[buf]);
            }
        }
    };

    int32_t s = static_cast<int32_t>(blockIdx.x);
    int32_t vn[NC];
    cols_of(s, vn);
    if (s < stages) issue(s, 0, vn);
    cols_of(s + step, vn);
    uint32_t sbn = s < stages ? sb_of(s) : 0u;
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    for (int k = 0; s < stages; s += step, ++k) {
        const int buf = k & 1;
        const int32_t sn = s + step;
        // the other buffer was released by the barrier that ended the
        // previous stage
        if (sn < stages) issue(sn, buf ^ 1, vn);
        cols_of(sn + step, vn);
        const uint32_t sb = sbn;
        if (sn < stages) sbn = sb_of(sn);
        const bool ok = mbar_wait(&full[buf], static_cast<uint32_t>(k >> 1) & 1u);
        int32_t j = s * S::G + g;
        const bool valid = ok && j < count;
        if (j >= count) j = count - 1;
        const unsigned char *base = smem + buf * S::kStage;
        TermsShared<MsgT, W> t;
        t.msg = reinterpret_cast<const MsgT *>(base) + g * DC * W + lane0;
        t.phi = reinterpret_cast<const float *>(base + S::kMsg) + g * DD * W + lane0;
        t.post = reinterpret_cast<const float *>(base + S::kMsg + S::kP1) + g * DC * W + lane0;
        check_terms<MsgT, W, DC, DD, false, false, false>(a, lane0, slab, valid, cl.e0 + j * DC, cl.s0 + j * DD, sb,
                                                   donenib, t);
        if (__syncthreads_or(!ok)) {
            // a copy never completed: record it, give the copies in flight
            // (this stage's and the next one's) a bounded time to land, leave
            if (tid == 0) {
                if (a.status) atomicCAS(a.status, 0, MLD_ETIMEOUT);
                mbar_wait(&full[buf], static_cast<uint32_t>(k >> 1) & 1u, kDrainNs);
                if (sn < stages) mbar_wait(&full[buf ^ 1], static_cast<uint32_t>((k + 1) >> 1) & 1u, kDrainNs);
            }
            __syncthreads();
            return;
        }
    }
}

template <typename MsgT, int W>
constexpr bool kStagedWidth = IsHalf<MsgT>::value && W == 64;

// Posterior accumulation is built for the default slab width of each
// message type (64 half, 32 float).
template <typename MsgT, int W>
constexpr bool kAccWidth = IsHalf<MsgT>::value ? W == 64 : W == 32;

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) k_check_update_irregular(CnArgs a, ClassLaunch cl) {
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    check_irregular<MsgT, W>(a, cl, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, slab);
}

// Classes with at most one degree-1 VN per check and at most kMaxRegDeg terms
// run the register kernel for their shape; any other class (possible in
// caller graphs, not in the MET ensembles) runs the streaming kernel.
// cap_blocks: grid width for the looped classes (a few waves of the GPU);
// hard1: early termination without soft output (degree-1 decisions only, and
// the fused syndrome check when ca.fuse; see check_regular).  With ca.acc set
// (fixed iterations, default slab width, register classes only) the kernels
// also add every new message to the next posteriors.
template <typename MsgT, int W>
void launch_minsum_class(const CnArgs &ca, const ClassLaunch &cl, int slabs, cudaStream_t st, int cap_blocks);

// Six staged blocks per SM need the largest shared-memory carveout; set once
// per kernel (a function attribute, not stream work) when a decoder that
// stages is created.
template <typename MsgT, int W, int DC, int DD>
cudaError_t prefer_smem_staged() {
    cudaError_t e = cudaFuncSetAttribute(k_check_staged<MsgT, W, DC, DD, false>,
                                         cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_check_staged<MsgT, W, DC, DD, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                cudaSharedmemCarveoutMaxShared);
}

inline cudaError_t prepare_staged_kernels() {
    const cudaError_t e[] = {
        prefer_smem_staged<__half, 64, 1, 0>(), prefer_smem_staged<__half, 64, 2, 0>(),
        prefer_smem_staged<__half, 64, 3, 0>(), prefer_smem_staged<__half, 64, 4, 0>(),
        prefer_smem_staged<__half, 64, 5, 0>(), prefer_smem_staged<__half, 64, 6, 0>(),
        prefer_smem_staged<__half, 64, 0, 1>(), prefer_smem_staged<__half, 64, 1, 1>(),
        prefer_smem_staged<__half, 64, 2, 1>(), prefer_smem_staged<__half, 64, 3, 1>(),
        prefer_smem_staged<__half, 64, 4, 1>(), prefer_smem_staged<__half, 64, 5, 1>()};
    for (cudaError_t x : e)
        if (x != cudaSuccess) return x;
    return cudaSuccess;
}

template <typename MsgT, int W, int DC, int DD>
void launch_staged(const CnArgs &ca, const ClassLaunch &cl, int slabs, cudaStream_t st, int staged_cap,
                   int mode) {
    using S = StageShape<MsgT, W, DC, DD>;
    static_assert(S::kBytes <= 48 * 1024, "staged buffers within the default dynamic shared memory");
    const int32_t stages = (cl.count + S::G - 1) / S::G;
    const dim3 grid(std::max(1, std::min<int32_t>(stages, staged_cap)), slabs);
    if (mode == MLD_STAGE_BULK_LSU) k_check_staged<MsgT, W, DC, DD, true><<<grid, kBlock, S::kBytes, st>>>(ca, cl);
    else k_check_staged<MsgT, W, DC, DD, false><<<grid, kBlock, S::kBytes, st>>>(ca, cl);
}

// The staged kernel, where it applies (half messages at slab width 64,
// sum-product, no fused syndrome, no accumulation, a register class of at
// most six terms with at most one degree-1 VN per check); false otherwise.
template <typename MsgT, int W>
bool try_launch_staged(const CnArgs &ca, const ClassLaunch &cl, int slabs, cudaStream_t st, int staged_cap,
                       bool hard1, int mode) {
    if constexpr (kStagedWidth<MsgT, W>) {
        const int dd = cl.deg - cl.dc;
        if (staged_cap <= 0 || hard1 || ca.acc || ca.rule != kRuleSumProduct || cl.dc < 0 || cl.deg > 6 ||
            cl.count <= 0 || (dd != 0 && dd != 1))
            return false;
        switch (cl.dc * 2 + dd) {
#define MLD_STAGED(DCV, DDV) \
    case (DCV) * 2 + (DDV): launch_staged<MsgT, W, DCV, DDV>(ca, cl, slabs, st, staged_cap, mode); return true;
            MLD_STAGED(1, 0) MLD_STAGED(2, 0) MLD_STAGED(3, 0) MLD_STAGED(4, 0) MLD_STAGED(5, 0) MLD_STAGED(6, 0)
            MLD_STAGED(0, 1) MLD_STAGED(1, 1) MLD_STAGED(2, 1) MLD_STAGED(3, 1) MLD_STAGED(4, 1) MLD_STAGED(5, 1)
#undef MLD_STAGED
            default: return false;
        }
    } else {
        (void)ca; (void)cl; (void)slabs; (void)st; (void)staged_cap; (void)hard1; (void)mode;
        return false;
    }
}

template <typename MsgT, int W>
void launch_check_class(const CnArgs &ca, const ClassLaunch &cl, int slabs, cudaStream_t st, int cap_blocks,
                        bool hard1, int staged_cap = 0, int staged_mode = MLD_STAGE_DIRECT) {
    if (ca.rule == kRuleMinSum) {
        launch_minsum_class<MsgT, W>(ca, cl, slabs, st, cap_blocks);
        return;
    }
    if (try_launch_staged<MsgT, W>(ca, cl, slabs, st, staged_cap, hard1, staged_mode)) return;
    const dim3 grid(cl.blocks, slabs);
    const dim3 capped(std::max(1, std::min(cl.blocks, cap_blocks)), slabs);
    const dim3 g = (cl.dc >= 0 && cl.deg <= 6) ? capped : grid;
    // the decisions-only kernels without the fused syndrome run 7 blocks per
    // SM: their looped grid is two waves of 7
    const dim3 capped7(std::max(1, std::min(cl.blocks, cap_blocks / 8 * 7)), slabs);
    const dim3 g7 = (cl.dc >= 0 && cl.deg <= 6) ? capped7 : grid;
    const int dd = cl.deg - cl.dc;
#define MLD_CASE(DCV, DDV)                                                                          \
    case (DCV) * 2 + (DDV):                                                                         \
        static_assert(kLoopedClass<(DCV) + (DDV)> == ((DCV) + (DDV) <= 6), "grid choice");         \
        if constexpr (kAccWidth<MsgT, W>) {                                                         \
            if (ca.acc) {                                                                           \
                k_check_update<MsgT, W, DCV, DDV, false, true><<<g, kBlock, 0, st>>>(ca, cl);      \
                return;                                                                             \
            }                                                                                       \
        }                                                                                           \
        if (hard1 && ca.fuse) k_check_update<MsgT, W, DCV, DDV, true><<<g, kBlock, 0, st>>>(ca, cl); \
        else if (hard1) k_check_update<MsgT, W, DCV, DDV, true, false, false><<<g7, kBlock, 0, st>>>(ca, cl); \
        else k_check_update<MsgT, W, DCV, DDV, false><<<g, kBlock, 0, st>>>(ca, cl);              \
        return;
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
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may be scheduled before its predecessor on
// the stream has finished; it waits here until that predecessor has
// completed and its memory is visible, then lets its own successor be
// scheduled.  Without the attribute both instructions return at once.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---------------------------------------------------------------------------
// Layered schedule: the checks are updated one layer at a time, every check
// from the latest messages.  The checks of a layer share no core VN, so a
// check owns the posteriors of its core VNs while its layer runs: it forms
// q = L_v - r_old (Eq. 4 with the current messages), the new r (Eqs. 2-3,
// as in check_regular) and L_v <- (L_v - r_old) + r_new in place.
// ---------------------------------------------------------------------------
// Layered launches number their messages contiguously: the launch's k-th
// check (internal id c) owns layered edges cl.e0 + k DC ..; a.col is the
// layered column table.  Its degree-1 slots follow the class order.  HARD1:
// a degree-1 VN gets its decision only (early termination without soft
// output), as in check_terms.
template <typename MsgT, int W, int DC, int DD, bool HARD1 = false>
__device__ __forceinline__ void check_layered(const CnArgs &a, const ClassLaunch &cl, int32_t c, int32_t k,
                                              int lane0, int slab, bool valid) {
    constexpr int D = DC + DD;
    constexpr int F = DecodeFit<MsgT>::value;
    constexpr int NB = W / 8;
    const int32_t e0 = cl.e0 + k * DC;
    const int32_t s0 = cl.s0 + (c - cl.c0) * DD;
    const float lmax = a.lmax, amin = a.amin;
    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >>
         (lane0 & 7));
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    MsgT *rb = static_cast<MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    // the posteriors are written by this kernel: plain (coherent) loads
    float *lvb = const_cast<float *>(a.Lv) + static_cast<size_t>(slab) * a.n_core * W + lane0;
    const float *p1b = a.phi1 + static_cast<size_t>(slab) * a.n_deg1 * W + lane0;

    float f[D][kK];
    uint32_t par[kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) par[kk] = ((sb >> kk) & 1u) << 31;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i < DC) {
            const int32_t v = __ldg(a.col + e0 + i);
            const float4 lv = *reinterpret_cast<const float4 *>(lvb + static_cast<size_t>(v) * W);
            const float4 ro = Msg<MsgT>::load(rb + static_cast<size_t>(e0 + i) * W);
            const float4 q = make_float4(lv.x - ro.x, lv.y - ro.y, lv.z - ro.z, lv.w - ro.w);
            const float4 m = make_float4(fabsf(q.x), fabsf(q.y), fabsf(q.z), fabsf(q.w));
            const float4 ph = phi4_floor<F>(m, amin);
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                const uint32_t qb = fbits(f4get(q, kk));
                f[i][kk] = bitsf(fbits(f4get(ph, kk)) | (qb & kSign));
                par[kk] ^= qb;
            }
        } else {
            const float4 p = ldf4(p1b + static_cast<size_t>(s0 + i - DC) * W);
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                f[i][kk] = f4get(p, kk);
                par[kk] ^= fbits(f[i][kk]);
            }
        }
    }
    float pre[D][kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
        if (D >= 2) pre[1][kk] = fabsf(f[0][kk]);
#pragma unroll
        for (int i = 2; i < D; ++i) pre[i][kk] = pre[i - 1][kk] + fabsf(f[i - 1][kk]);
    }
    float suf[kK];
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        if (i < DC || a.final_pass) {
            float4 o;
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                float v;
                if (D == 1) v = amin;
                else if (i == D - 1) v = pre[i][kk];
                else if (i == 0) v = suf[kk];
                else v = pre[i][kk] + suf[kk];
                f4set(o, kk, v);
            }
            if (HARD1 && i >= DC) {
                // decision of L_ch + r without r: see check_terms
                uint32_t nib = 0;
#pragma unroll
                for (int kk = 0; kk < kK; ++kk) {
                    const uint32_t fb = fbits(f[i][kk]);
                    const bool l_neg = (fb & kSign) != 0;
                    const bool r_neg = ((par[kk] ^ fb) & kSign) != 0;
                    const float fl = fabsf(f[i][kk]), ov = f4get(o, kk);
                    const bool neg = (l_neg == r_neg) ? l_neg : (l_neg ? fl < ov : fl > ov);
                    nib |= static_cast<uint32_t>(neg) << kk;
                }
                emit_deg1_bits<W>(a, slab, s0 + i - DC, lane0, nib, donenib, valid);
            } else {
            float4 mm = phi4_floor<F>(o, amin);
            if (D <= 2) mm = make_float4(fminf(mm.x, lmax), fminf(mm.y, lmax), fminf(mm.z, lmax), fminf(mm.w, lmax));
            float4 rv;
#pragma unroll
            for (int kk = 0; kk < kK; ++kk)
                f4set(rv, kk, bitsf(fbits(f4get(mm, kk)) | ((par[kk] ^ fbits(f[i][kk])) & kSign)));
            if (i < DC) {
                if (valid) {
                    MsgT *rp = rb + static_cast<size_t>(e0 + i) * W;
                    const float4 ro = Msg<MsgT>::load(rp);
                    if (donenib) {  // converged lanes keep their messages
                        if (donenib & 1) rv.x = ro.x;
                        if (donenib & 2) rv.y = ro.y;
                        if (donenib & 4) rv.z = ro.z;
                        if (donenib & 8) rv.w = ro.w;
                    }
                    const float4 st = Msg<MsgT>::store_get(rp, rv);
                    float *lp = lvb + static_cast<size_t>(__ldg(a.col + e0 + i)) * W;
                    const float4 lv = *reinterpret_cast<const float4 *>(lp);
                    float4 ln = make_float4((lv.x - ro.x) + st.x, (lv.y - ro.y) + st.y, (lv.z - ro.z) + st.z,
                                            (lv.w - ro.w) + st.w);
                    if (donenib) {  // and their posteriors
                        if (donenib & 1) ln.x = lv.x;
                        if (donenib & 2) ln.y = lv.y;
                        if (donenib & 4) ln.z = lv.z;
                        if (donenib & 8) ln.w = lv.w;
                    }
                    *reinterpret_cast<float4 *>(lp) = ln;
                }
            } else {
                emit_deg1<MsgT, W>(a, slab, s0 + i - DC, lane0, rv, donenib, valid);
            }
            }
        }
        if (i > 0) {
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) suf[kk] = (i == D - 1) ? fabsf(f[i][kk]) : suf[kk] + fabsf(f[i][kk]);
        }
    }
}

// One layer's checks of one class (pos[k]: internal id of the k-th), on a
// capped grid: a thread keeps its lanes and steps through every stride-th
// check, so consecutive checks of a wave read consecutive message rows.
// Both threads of a shuffle pair belong to one check and leave together.
// Blocks per SM of the layered kernels (72 registers per thread).
constexpr int kLayeredBlocksPerSm = 7;

template <typename MsgT, int W, int DC, int DD, bool HARD1>
__global__ void __launch_bounds__(kBlock, (DC + DD <= 6 ? kLayeredBlocksPerSm : 6))
    k_check_layered(CnArgs a, ClassLaunch cl, const int32_t *pos) {
    constexpr int TPC = W / kK;
    pdl_enter();  // the previous layer's messages and posteriors
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;  // block-uniform
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int lane0 = static_cast<int>(t % TPC) * kK;
    const int32_t kstride = static_cast<int32_t>(gridDim.x) * (kBlock / TPC);
    for (int32_t k = static_cast<int32_t>(t / TPC); k < cl.count; k += kstride)
        check_layered<MsgT, W, DC, DD, HARD1>(a, cl, __ldg(pos + k), k, lane0, slab, true);
}

// Layered update of a check of any degree (edges read through cptr/dptr);
// leave-one-out sums as total minus own term, as in check_irregular.  Both
// threads of a shuffle pair belong to one check.
// a.cptr: the launch's layered edge starts (check k: a.cptr[k] .. a.cptr[k+1]).
template <typename MsgT, int W>
__device__ __forceinline__ void check_layered_irregular(const CnArgs &a, int32_t c, int32_t k, int lane0,
                                                        int slab) {
    constexpr int F = DecodeFit<MsgT>::value;
    constexpr int NB = W / 8;
    const int32_t e0 = a.cptr[k], e1 = a.cptr[k + 1];
    const int32_t s0 = a.dptr[c], s1 = a.dptr[c + 1];
    const int nce = e1 - e0;
    const int deg = nce + (s1 - s0);
    const float lmax = a.lmax, amin = a.amin;
    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >>
         (lane0 & 7));
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    MsgT *rb = static_cast<MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    float *lvb = const_cast<float *>(a.Lv) + static_cast<size_t>(slab) * a.n_core * W + lane0;
    const float *l1b = a.lch1 + static_cast<size_t>(slab) * a.n_deg1 * W + lane0;
    auto input = [&](int i) -> float4 {
        if (i < nce) {
            const float4 lv = *reinterpret_cast<const float4 *>(lvb + static_cast<size_t>(__ldg(a.col + e0 + i)) * W);
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
            S[kk] += phi_f<F>(clampf(fabsf(qk), amin, lmax));
        }
    }
    // each edge's message and VN are touched only at its own i, so input(i)
    // still reads the values of pass 1
    for (int i = 0; i < deg; ++i) {
        const bool out_core = i < nce;
        if (!out_core && !a.final_pass) continue;
        const float4 q = input(i);
        float4 rv;
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) {
            const float qk = f4get(q, kk);
            const float fk = phi_f<F>(clampf(fabsf(qk), amin, lmax));
            const float mk = fminf(phi_f<F>(clampf(S[kk] - fk, amin, lmax)), lmax);
            f4set(rv, kk, bitsf(fbits(mk) | ((par[kk] ^ fbits(qk)) & kSign)));
        }
        if (out_core) {
            MsgT *rp = rb + static_cast<size_t>(e0 + i) * W;
            const float4 ro = Msg<MsgT>::load(rp);
            if (donenib) {
                if (donenib & 1) rv.x = ro.x;
                if (donenib & 2) rv.y = ro.y;
                if (donenib & 4) rv.z = ro.z;
                if (donenib & 8) rv.w = ro.w;
            }
            const float4 st = Msg<MsgT>::store_get(rp, rv);
            float *lp = lvb + static_cast<size_t>(__ldg(a.col + e0 + i)) * W;
            const float4 lv = *reinterpret_cast<const float4 *>(lp);
            float4 ln = make_float4((lv.x - ro.x) + st.x, (lv.y - ro.y) + st.y, (lv.z - ro.z) + st.z,
                                    (lv.w - ro.w) + st.w);
            if (donenib) {
                if (donenib & 1) ln.x = lv.x;
                if (donenib & 2) ln.y = lv.y;
                if (donenib & 4) ln.z = lv.z;
                if (donenib & 8) ln.w = lv.w;
            }
            *reinterpret_cast<float4 *>(lp) = ln;
        } else {
            emit_deg1<MsgT, W>(a, slab, s0 + i - nce, lane0, rv, donenib, true);
        }
    }
}

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) k_check_layered_irregular(CnArgs a, ClassLaunch cl, const int32_t *pos) {
    constexpr int TPC = W / kK;
    pdl_enter();
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int lane0 = static_cast<int>(t % TPC) * kK;
    const int32_t kstride = static_cast<int32_t>(gridDim.x) * (kBlock / TPC);
    for (int32_t k = static_cast<int32_t>(t / TPC); k < cl.count; k += kstride)  // whole checks leave together
        check_layered_irregular<MsgT, W>(a, __ldg(pos + k), k, lane0, slab);
}

// The layered schedule is built for the default slab width of each message
// type.  Classes of at most 8 terms with at most one degree-1 VN run the
// register kernel of their shape, any other class the runtime-degree kernel.
template <typename MsgT, int W>
void launch_layered(const CnArgs &ca, const ClassLaunch &cl, const int32_t *pos, int slabs, cudaStream_t st,
                    bool hard1) {
    if constexpr (kAccWidth<MsgT, W>) {
        const dim3 grid(cl.blocks, slabs);
        const int dd = cl.deg - cl.dc;
#define MLD_LCASE(DCV, DDV)                                                                          \
    case (DCV) * 2 + (DDV):                                                                          \
        if (hard1) launch_pdl(k_check_layered<MsgT, W, DCV, DDV, true>, grid, dim3(kBlock), st, ca, cl, pos); \
        else launch_pdl(k_check_layered<MsgT, W, DCV, DDV, false>, grid, dim3(kBlock), st, ca, cl, pos);     \
        return;
        if (cl.dc >= 0 && (dd == 0 || dd == 1)) {
            switch (cl.dc * 2 + dd) {
                MLD_LCASE(1, 0) MLD_LCASE(2, 0) MLD_LCASE(3, 0) MLD_LCASE(4, 0)
                MLD_LCASE(5, 0) MLD_LCASE(6, 0) MLD_LCASE(7, 0) MLD_LCASE(8, 0)
                MLD_LCASE(0, 1) MLD_LCASE(1, 1) MLD_LCASE(2, 1) MLD_LCASE(3, 1)
                MLD_LCASE(4, 1) MLD_LCASE(5, 1) MLD_LCASE(6, 1) MLD_LCASE(7, 1)
                default: break;
            }
        }
#undef MLD_LCASE
        launch_pdl(k_check_layered_irregular<MsgT, W>, grid, dim3(kBlock), st, ca, cl, pos);
    }
}

// ---------------------------------------------------------------------------
// Offset min-sum check update: the sign rule of Eqs. 2-3 (syndrome sign
// included) with magnitude max(min of the other |q| - offset, 0), |q| clamped
// at lmax.  The two smallest magnitudes and the position of the smallest give
// every leave-one-out minimum.
// ---------------------------------------------------------------------------
template <typename MsgT, int W, int DC, int DD>
__device__ __forceinline__ void check_minsum(const CnArgs &a, const ClassLaunch &cl, int32_t j, int lane0,
                                             int slab) {
    constexpr int D = DC + DD;
    constexpr int NB = W / 8;
    const int32_t c = cl.c0 + j;
    const int32_t e0 = cl.e0 + j * DC;
    const int32_t s0 = cl.s0 + j * DD;
    const float lmax = a.lmax, off = a.ms_off;
    const uint32_t sb =
        (static_cast<uint32_t>(a.sbits[(static_cast<size_t>(slab) * a.n_cn + c) * NB + lane0 / 8]) >>
         (lane0 & 7));
    const uint32_t donenib = a.et ? done_nibble<W>(a.done, slab, lane0) : 0u;
    MsgT *rb = static_cast<MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    const float *lvb = a.Lv + static_cast<size_t>(slab) * a.n_core * W + lane0;
    const float *l1b = a.lch1 + static_cast<size_t>(slab) * a.n_deg1 * W + lane0;
    float m1[kK], m2[kK];
    uint32_t par[kK], neg[kK], at[kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
        par[kk] = (sb >> kk) & 1u;
        neg[kk] = 0u;
        at[kk] = 0u;
        m1[kk] = lmax;
        m2[kk] = lmax;
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        float4 q;
        if (i < DC) {
            const float4 lv = ldf4(lvb + static_cast<size_t>(__ldg(a.col + e0 + i)) * W);
            const float4 ro = Msg<MsgT>::load(rb + static_cast<size_t>(e0 + i) * W);
            q = make_float4(lv.x - ro.x, lv.y - ro.y, lv.z - ro.z, lv.w - ro.w);
        } else {
            q = ldf4(l1b + static_cast<size_t>(s0 + i - DC) * W);  // degree-1 VN: q = L_ch
        }
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) {
            const float qk = f4get(q, kk);
            const uint32_t ng = qk < 0.f ? 1u : 0u;
            par[kk] ^= ng;
            neg[kk] |= ng << i;
            const float mg = fminf(fabsf(qk), lmax);
            const bool lt1 = mg < m1[kk];
            m2[kk] = lt1 ? m1[kk] : fminf(m2[kk], mg);
            at[kk] = lt1 ? static_cast<uint32_t>(i) : at[kk];
            m1[kk] = lt1 ? mg : m1[kk];
        }
    }
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i < DC || a.final_pass) {
            float4 rv;
#pragma unroll
            for (int kk = 0; kk < kK; ++kk) {
                const float mg = fmaxf((at[kk] == static_cast<uint32_t>(i) ? m2[kk] : m1[kk]) - off, 0.f);
                const uint32_t sg = (par[kk] ^ (neg[kk] >> i)) & 1u;
                f4set(rv, kk, sg ? -mg : mg);
            }
            if (i < DC) {
                MsgT *rp = rb + static_cast<size_t>(e0 + i) * W;
                if (a.et) store_r<MsgT, W>(a, rp, rv, donenib);
                else Msg<MsgT>::store(rp, rv);
            } else {
                emit_deg1<MsgT, W>(a, slab, s0 + i - DC, lane0, rv, donenib, true);
            }
        }
    }
}

// Any degree (edges through cptr/dptr): the same rule over two passes.
template <typename MsgT, int W>
__device__ __forceinline__ void check_minsum_irregular(const CnArgs &a, int32_t c, int lane0, int slab) {
    constexpr int NB = W / 8;
    const int32_t e0 = a.cptr[c], e1 = a.cptr[c + 1];
    const int32_t s0 = a.dptr[c], s1 = a.dptr[c + 1];
    const int nce = e1 - e0;
    const int deg = nce + (s1 - s0);
    const float lmax = a.lmax, off = a.ms_off;
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
        return ldf4(l1b + static_cast<size_t>(s0 + i - nce) * W);
    };
    float m1[kK], m2[kK];
    uint32_t par[kK];
    int at[kK];
#pragma unroll
    for (int kk = 0; kk < kK; ++kk) {
        par[kk] = (sb >> kk) & 1u;
        at[kk] = -1;
        m1[kk] = lmax;
        m2[kk] = lmax;
    }
    for (int i = 0; i < deg; ++i) {
        const float4 q = input(i);
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) {
            const float qk = f4get(q, kk);
            par[kk] ^= qk < 0.f ? 1u : 0u;
            const float mg = fminf(fabsf(qk), lmax);
            if (mg < m1[kk]) {
                m2[kk] = m1[kk];
                m1[kk] = mg;
                at[kk] = i;
            } else {
                m2[kk] = fminf(m2[kk], mg);
            }
        }
    }
    for (int i = 0; i < deg; ++i) {
        const bool out_core = i < nce;
        if (!out_core && !a.final_pass) continue;
        const float4 q = input(i);
        float4 rv;
#pragma unroll
        for (int kk = 0; kk < kK; ++kk) {
            const float mg = fmaxf((at[kk] == i ? m2[kk] : m1[kk]) - off, 0.f);
            const uint32_t sg = par[kk] ^ (f4get(q, kk) < 0.f ? 1u : 0u);
            f4set(rv, kk, sg ? -mg : mg);
        }
        if (out_core)
            store_r<MsgT, W>(a, rb + static_cast<size_t>(e0 + i) * W, rv, donenib);
        else
            emit_deg1<MsgT, W>(a, slab, s0 + i - nce, lane0, rv, donenib, true);
    }
}

// Min-sum launches loop over their checks on a capped grid (the state per
// thread is small, so every shape loops).  Both threads of a shuffle pair
// belong to one check and leave together.  80 registers: the loads of a
// check's terms are all in flight at once (64 registers spill: 0.37 -> 0.51 ms
// per pass at rate 0.1, n = 10^6, 64 codewords).
constexpr int kMinSumBlocksPerSm = 6;
template <typename MsgT, int W, int DC, int DD>
__global__ void __launch_bounds__(kBlock, kMinSumBlocksPerSm) k_check_minsum(CnArgs a, ClassLaunch cl) {
    constexpr int TPC = W / kK;
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int lane0 = static_cast<int>(t % TPC) * kK;
    const int32_t jstride = static_cast<int32_t>(gridDim.x) * (kBlock / TPC);
    for (int32_t j = static_cast<int32_t>(t / TPC); j < cl.count; j += jstride)
        check_minsum<MsgT, W, DC, DD>(a, cl, j, lane0, slab);
}

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) k_check_minsum_irregular(CnArgs a, ClassLaunch cl) {
    constexpr int TPC = W / kK;
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    const int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int lane0 = static_cast<int>(t % TPC) * kK;
    const int32_t jstride = static_cast<int32_t>(gridDim.x) * (kBlock / TPC);
    for (int32_t j = static_cast<int32_t>(t / TPC); j < cl.count; j += jstride)
        check_minsum_irregular<MsgT, W>(a, cl.c0 + j, lane0, slab);
}

// Offset min-sum is built for the default slab width of each message type.
template <typename MsgT, int W>
void launch_minsum_class(const CnArgs &ca, const ClassLaunch &cl, int slabs, cudaStream_t st, int cap_blocks) {
    if constexpr (kAccWidth<MsgT, W>) {
        const dim3 g(std::max(1, std::min(cl.blocks, cap_blocks)), slabs);
        const int dd = cl.deg - cl.dc;
#define MLD_MCASE(DCV, DDV)                                                   \
    case (DCV) * 2 + (DDV):                                                   \
        k_check_minsum<MsgT, W, DCV, DDV><<<g, kBlock, 0, st>>>(ca, cl);      \
        return;
        if (cl.dc >= 0 && (dd == 0 || dd == 1)) {
            switch (cl.dc * 2 + dd) {
                MLD_MCASE(1, 0) MLD_MCASE(2, 0) MLD_MCASE(3, 0) MLD_MCASE(4, 0)
                MLD_MCASE(5, 0) MLD_MCASE(6, 0) MLD_MCASE(7, 0) MLD_MCASE(8, 0)
                MLD_MCASE(0, 1) MLD_MCASE(1, 1) MLD_MCASE(2, 1) MLD_MCASE(3, 1)
                MLD_MCASE(4, 1) MLD_MCASE(5, 1) MLD_MCASE(6, 1) MLD_MCASE(7, 1)
                default: break;
            }
        }
#undef MLD_MCASE
        k_check_minsum_irregular<MsgT, W><<<g, kBlock, 0, st>>>(ca, cl);
    }
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
__device__ __forceinline__ void var_body(const VnArgs &a, int64_t t, int slab) {
    constexpr int TPC = W / kK;
    constexpr int NB = W / 8;
    const int32_t v = static_cast<int32_t>(t / TPC);
    if (v >= a.n_core) return;
    const int lane0 = static_cast<int>(t % TPC) * kK;
    const size_t vrow = (static_cast<size_t>(slab) * a.n_core + v) * W + lane0;
    const MsgT *rb = static_cast<const MsgT *>(a.r) + static_cast<size_t>(slab) * a.e_core * W + lane0;
    float4 acc = ldf4(a.lch + vrow);
    int32_t j = a.vptr[v];
    const int32_t j1 = a.vptr[v + 1];
    // four edges per round, every load of a round in flight together; the
    // last round's missing edges re-read the round's first row (an L1 hit)
    // and add nothing, so the sums are formed in CSC order as before
    for (; j < j1; j += 4) {
        const int32_t rem = j1 - j;
        const int32_t ea = __ldg(a.vedge + j);
        const int32_t eb = rem > 1 ? __ldg(a.vedge + j + 1) : ea;
        const int32_t ec = rem > 2 ? __ldg(a.vedge + j + 2) : ea;
        const int32_t ed = rem > 3 ? __ldg(a.vedge + j + 3) : ea;
        const float4 ra = Msg<MsgT>::load(rb + static_cast<size_t>(ea) * W);
        const float4 rbv = Msg<MsgT>::load(rb + static_cast<size_t>(eb) * W);
        const float4 rc = Msg<MsgT>::load(rb + static_cast<size_t>(ec) * W);
        const float4 rd = Msg<MsgT>::load(rb + static_cast<size_t>(ed) * W);
        acc.x += ra.x; acc.y += ra.y; acc.z += ra.z; acc.w += ra.w;
        if (rem > 1) { acc.x += rbv.x; acc.y += rbv.y; acc.z += rbv.z; acc.w += rbv.w; }
        if (rem > 2) { acc.x += rc.x; acc.y += rc.y; acc.z += rc.z; acc.w += rc.w; }
        if (rem > 3) { acc.x += rd.x; acc.y += rd.y; acc.z += rd.z; acc.w += rd.w; }
    }
    if (a.et) {
        // converged lanes keep the posterior of their last iteration (with a
        // fused syndrome check a lane is marked after its messages moved on)
        const uint32_t dn = done_nibble<W>(a.done, slab, lane0);
        if (dn) {
            const float4 old = *reinterpret_cast<const float4 *>(a.Lv + vrow);
            if (dn & 1) acc.x = old.x;
            if (dn & 2) acc.y = old.y;
            if (dn & 4) acc.z = old.z;
            if (dn & 8) acc.w = old.w;
        }
    }
    *reinterpret_cast<float4 *>(a.Lv + vrow) = acc;
    if (a.want_bits) {
        const uint32_t nib = (acc.x < 0.f) | ((acc.y < 0.f) << 1) | ((acc.z < 0.f) << 2) | ((acc.w < 0.f) << 3);
        const uint32_t other = __shfl_xor_sync(pair_mask(), nib, 1);
        if ((lane0 & 7) == 0)
            a.hb[(static_cast<size_t>(slab) * a.n_core + v) * NB + lane0 / 8] = static_cast<uint8_t>(nib | (other << 4));
    }
}

template <typename MsgT, int W>
__global__ void __launch_bounds__(kBlock) k_var_update(VnArgs a) {
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;
    var_body<MsgT, W>(a, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x, slab);
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
    int32_t batch;         // codewords in the batch (later lanes are padding)
};

// One slab's W decision bits of a node as one unsigned word.
template <int W> struct SlabWord;
template <> struct SlabWord<8> { using T = uint8_t; };
template <> struct SlabWord<16> { using T = uint16_t; };
template <> struct SlabWord<32> { using T = uint32_t; };
template <> struct SlabWord<64> { using T = unsigned long long; };

// Checks first, first + stride, ... of one slab, all W codewords of a check
// in one word: x = syndrome row XOR the decision rows of the check's VNs
// (gathered four at a time).  Every thread of the warp must call it (warp
// reduction at the end).
template <int W>
__device__ __forceinline__ void syndrome_body(const SynArgs &a, int64_t first, int64_t stride, int slab) {
    using T = typename SlabWord<W>::T;
    constexpr int DW = (W + 31) / 32;
    constexpr unsigned long long kFull = W == 64 ? ~0ull : ((1ull << W) - 1ull);
    const T *hc = reinterpret_cast<const T *>(a.hb_core) + static_cast<size_t>(slab) * a.n_core;
    const T *h1 = reinterpret_cast<const T *>(a.hb1) + static_cast<size_t>(slab) * a.n_deg1;
    const T *sr = reinterpret_cast<const T *>(a.sbits) + static_cast<size_t>(slab) * a.n_cn;
    // codewords whose outcome is already known: frozen (early termination)
    // or padding lanes past the end of the batch
    unsigned long long known = 0;
    if (a.et) {
        known = a.done[slab * DW];
        if (DW > 1) known |= static_cast<unsigned long long>(a.done[slab * DW + 1]) << 32;
    }
    const int valid = a.batch - slab * W;
    if (valid < W) known |= ~0ull << valid;
    known &= kFull;
    unsigned long long acc = 0;
    for (int64_t t = first; t < a.n_cn; t += stride) {
        // once every codeword has failed a check (or is known), further
        // checks cannot change the result
        if ((acc | known) == kFull) break;
        const int32_t c = static_cast<int32_t>(t);
        T x = sr[c];
        int32_t e = __ldg(a.cptr + c);
        const int32_t e1 = __ldg(a.cptr + c + 1);
        for (; e + 4 <= e1; e += 4) {
            const int32_t v0 = __ldg(a.col + e), v1 = __ldg(a.col + e + 1);
            const int32_t v2 = __ldg(a.col + e + 2), v3 = __ldg(a.col + e + 3);
            x ^= static_cast<T>(hc[v0] ^ hc[v1] ^ hc[v2] ^ hc[v3]);
        }
        for (; e < e1; ++e) x ^= hc[__ldg(a.col + e)];
        const int32_t s1 = __ldg(a.dptr + c + 1);
        for (int32_t s = __ldg(a.dptr + c); s < s1; ++s) x ^= h1[s];
        acc |= x;
    }
    acc &= ~known;
    uint32_t lo = static_cast<uint32_t>(acc), hi = static_cast<uint32_t>(acc >> 32);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        lo |= __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        if (DW > 1) hi |= __shfl_xor_sync(0xFFFFFFFFu, hi, o);
    }
    // set only bits not already set: most warps of a failing slab then read
    // the word instead of contending on it
    if ((threadIdx.x & 31) == 0) {
        uint32_t *fw = a.fail + slab * DW;
        if (lo && (*reinterpret_cast<volatile uint32_t *>(fw) & lo) != lo) atomicOr(fw, lo);
        if (DW > 1 && hi && (*reinterpret_cast<volatile uint32_t *>(fw + 1) & hi) != hi) atomicOr(fw + 1, hi);
    }
}

// grid width (blocks per slab) of a syndrome check over n_cn checks: one
// thread per check up to 8 blocks per SM, beyond that threads take several
// checks (and can stop early once every codeword has failed)
inline int syndrome_blocks(int64_t n_cn, int sm_count) {
    const int64_t want = (n_cn + kBlock - 1) / kBlock;
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(want, static_cast<int64_t>(sm_count) * 8)));
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_syndrome_check(SynArgs a) {
    const int slab = blockIdx.y;
    if (a.et && slab_all_done<W>(a.done, slab)) return;  // block-uniform
    syndrome_body<W>(a, static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x,
                     static_cast<int64_t>(gridDim.x) * blockDim.x, slab);
}

// per-codeword bookkeeping after a syndrome check at iteration l
template <int W>
__device__ __forceinline__ void lane_body(uint32_t *done, const uint32_t *fail, int32_t *iters,
                                          uint8_t *conv, int32_t batch, int32_t l, int et, int b) {
    constexpr int DW = (W + 31) / 32;
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

template <int W>
__global__ void k_lane_update(uint32_t *done, const uint32_t *fail, int32_t *iters,
                              uint8_t *conv, int32_t batch, int32_t l, int et) {
    lane_body<W>(done, fail, iters, conv, batch, l, et, blockIdx.x * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Early termination driven by the device: the iterations run inside a CUDA
// graph loop (a conditional WHILE node) whose body holds two iterations; the
// iteration number lives in device memory (lctr[0]: iterations before the
// body, lctr[1]: the cap), and the loop stops once every codeword has
// stopped, so no launch runs after the last codeword converges.
// ---------------------------------------------------------------------------
// Counter and cap; padding lanes of the last slab count as stopped (so a slab
// whose real codewords have all stopped is skipped).  done must be zero.
template <int W>
__global__ void k_loop_init(uint32_t *done, int32_t slabs, int32_t batch, int32_t *lctr, int32_t max_iters) {
    constexpr int DW = (W + 31) / 32;
    constexpr int WB = W >= 32 ? 32 : W;  // lanes per done word
    constexpr uint32_t full = W >= 32 ? 0xFFFFFFFFu : ((1u << W) - 1u);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        lctr[0] = 0;
        lctr[1] = max_iters;
    }
    if (i < slabs * DW) {
        const int real = batch - (i / DW) * W - (i % DW) * 32;  // real lanes in this word
        done[i] = real <= 0 ? full : (real >= WB ? 0u : (full & ~((1u << real) - 1u)));
    }
}

// Bookkeeping of iteration l = lctr[0] + off after its syndrome check (fail):
// as lane_body with early termination, and at the cap every lane stops with
// the outputs of that iteration.  Also clears the fail words the next
// iteration uses (fail_next, nwords words).
template <int W>
__global__ void k_lane_update_dev(uint32_t *done, const uint32_t *fail, uint32_t *fail_next, int32_t nwords,
                                  int32_t *iters, uint8_t *conv, int32_t batch, const int32_t *lctr, int32_t off) {
    constexpr int DW = (W + 31) / 32;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nwords) fail_next[b] = 0u;
    if (b >= batch) return;
    const int32_t l = lctr[0] + off;
    const int slab = b / W, w = b % W;
    const int word = slab * DW + w / 32;
    const uint32_t bit = 1u << (w & 31);
    if (done[word] & bit) return;  // stopped at an earlier iteration
    const bool ok = (fail[word] & bit) == 0u;
    iters[b] = l;
    conv[b] = ok ? 1 : 0;
    if (ok || l >= lctr[1]) atomicOr(done + word, bit);
}

// One warp: continue while some lane still iterates, counting the body's two
// iterations.
template <int W>
__global__ void k_loop_cond(const uint32_t *done, int32_t nwords, int32_t *lctr, cudaGraphConditionalHandle h) {
    constexpr uint32_t full = W >= 32 ? 0xFFFFFFFFu : ((1u << W) - 1u);
    bool all = true;
    for (int i = threadIdx.x; i < nwords; i += 32) all = all && (done[i] == full);
    all = __all_sync(0xFFFFFFFFu, all);
    if (threadIdx.x == 0) {
        if (!all) lctr[0] += 2;
        cudaGraphSetConditional(h, all ? 0u : 1u);
    }
}

// ---------------------------------------------------------------------------
// Graph store validation (decoders created with `checked`): every index of
// the device arrays is compared with its range, reading each array only
// within its own length.  The first violation found is recorded in st[0..3]:
// status code, array id, index, value (st[0] is claimed with a compare-and-
// swap, so concurrent finders leave one record).
// ---------------------------------------------------------------------------
struct ValidateArgs {
    const int32_t *cptr, *col, *dptr, *vptr, *vedge, *unit, *cint;
    const int32_t *lchk, *leptr, *lcol;  // layered tables or null
    int32_t n_vn, n_cn, n_core, n_deg1, e_core, n_lpos;
    int32_t *st;
};

enum { kArrCptr = 1, kArrCol, kArrDptr, kArrVptr, kArrVedge, kArrUnit, kArrCint, kArrLchk, kArrLeptr, kArrLcol };

__device__ __forceinline__ void flag_bad(int32_t *st, int arr, int64_t i, int32_t v) {
    if (atomicCAS(st, 0, MLD_EGRAPH) == 0) {
        st[1] = arr;
        st[2] = static_cast<int32_t>(i);
        st[3] = v;
    }
}

// ptr[0 .. n] must rise from 0 to `last`
__device__ __forceinline__ void check_ptr(const int32_t *ptr, int64_t n, int32_t last, int64_t i, int arr,
                                          int32_t *st) {
    if (i > n) return;
    const int32_t v = ptr[i];
    const bool bad = (i == 0 && v != 0) || (i == n && v != last) || (i < n && v > ptr[i + 1]) || v < 0 || v > last;
    if (bad) flag_bad(st, arr, i, v);
}

__device__ __forceinline__ void check_range(const int32_t *a, int64_t n, int32_t hi, int64_t i, int arr,
                                            int32_t *st) {
    if (i >= n) return;
    const int32_t v = a[i];
    if (v < 0 || v >= hi) flag_bad(st, arr, i, v);
}

__global__ void __launch_bounds__(kBlock) k_validate_graph(ValidateArgs a) {
    // every array's last index: e_core - 1, n_vn - 1, n_cn, n_core (<= n_vn), n_lpos
    int64_t top = a.e_core;
    top = top > static_cast<int64_t>(a.n_vn) + 1 ? top : static_cast<int64_t>(a.n_vn) + 1;
    top = top > static_cast<int64_t>(a.n_cn) + 1 ? top : static_cast<int64_t>(a.n_cn) + 1;
    top = top > static_cast<int64_t>(a.n_lpos) + 1 ? top : static_cast<int64_t>(a.n_lpos) + 1;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < top; i += stride) {
        check_ptr(a.cptr, a.n_cn, a.e_core, i, kArrCptr, a.st);
        check_range(a.col, a.e_core, a.n_core, i, kArrCol, a.st);
        check_ptr(a.dptr, a.n_cn, a.n_deg1, i, kArrDptr, a.st);
        check_ptr(a.vptr, a.n_core, a.e_core, i, kArrVptr, a.st);
        check_range(a.vedge, a.e_core, a.e_core, i, kArrVedge, a.st);
        check_range(a.unit, a.n_vn, a.n_vn, i, kArrUnit, a.st);
        check_range(a.cint, a.n_cn, a.n_cn, i, kArrCint, a.st);
        if (a.lchk) {
            check_range(a.lchk, a.n_lpos, a.n_cn, i, kArrLchk, a.st);
            check_ptr(a.leptr, a.n_lpos, a.e_core, i, kArrLeptr, a.st);
            check_range(a.lcol, a.e_core, a.n_core, i, kArrLcol, a.st);
        }
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
    float lmax;           // clamp of the channel LLR, nats
    float scale;          // nats -> internal units (log2 e for decoding, 1 for weighted BP)
    float lmax_i, amin_i; // phi argument clamps in internal units
    float *lch, *Lv, *lch1, *post1, *phi1;
};

// One tile of 32 natural VNs x W codewords of slab `slab`.
template <int W, int F>
__device__ __forceinline__ void interleave_body(const InArgs &a, int tile_x, int slab) {
    __shared__ float tile[W][33];
    const int32_t j0 = tile_x * 32;
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
            v = clampf(v, -a.lmax, a.lmax) * a.scale + 0.0f;  // -0 -> +0: a zero LLR has no sign
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
            const float f = phi_f<F>(clampf(fabsf(v), a.amin_i, a.lmax_i));
            a.phi1[o] = bitsf(fbits(f) | (fbits(v) & kSign));
        }
    }
}

template <int W, int F>
__global__ void __launch_bounds__(kBlock) k_interleave_in(InArgs a) {
    interleave_body<W, F>(a, blockIdx.x, blockIdx.y);
}

template <int W>
__device__ __forceinline__ void syndrome_in_body(const uint8_t *syn, const int32_t *cint, int32_t n_cn,
                                                 int32_t batch, uint8_t *sbits, int tile_x, int slab) {
    constexpr int NB = W / 8;
    __shared__ uint8_t tile[W][33];
    const int32_t c0 = tile_x * 32;  // caller's check order (coalesced reads)
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

template <int W>
__global__ void __launch_bounds__(kBlock) k_syndrome_in(const uint8_t *syn, const int32_t *cint, int32_t n_cn,
                                                        int32_t batch, uint8_t *sbits) {
    syndrome_in_body<W>(syn, cint, n_cn, batch, sbits, blockIdx.x, blockIdx.y);
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

// dst = src over n4 float4 (the posterior accumulator starts at L_ch)
__global__ void __launch_bounds__(kBlock) k_copy4(float4 *dst, const float4 *src, int64_t n4) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n4; i += stride)
        dst[i] = __ldg(src + i);
}

struct OutArgs {
    const int32_t *unit;
    int32_t n_vn, n_core, n_deg1, batch;
    const float *Lv, *post1;
    const uint8_t *hb1;  // degree-1 decisions (post1 is formed only for soft output)
    const int32_t *iters;  // iterations used per codeword: hb1 buffer (iters & 1), or null (buffer 0)
    size_t hb1_stride;     // bytes between the two hb1 buffers
    uint8_t *bits;   // [B][n_vn]
    float *post;     // [B][n_vn] or null
    float scale;     // internal units -> nats
};

template <int W>
__device__ __forceinline__ void deinterleave_body(const OutArgs &a, int tile_x, int slab) {
    constexpr int NB = W / 8;
    __shared__ float tile[32][W + 1];
    __shared__ uint8_t tbit[32][W + 1];
    const int32_t j0 = tile_x * 32;
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int jj = idx / W, w = idx % W;
        const int32_t j = j0 + jj;
        float v = 0.f;
        uint8_t bit = 0;
        if (j < a.n_vn) {
            const int32_t u = a.unit[j];
            if (u < a.n_core) {
                v = a.Lv[(static_cast<size_t>(slab) * a.n_core + u) * W + w];
                bit = v < 0.f ? 1 : 0;
            } else {
                const size_t s = static_cast<size_t>(slab) * a.n_deg1 + (u - a.n_core);
                if (a.post) v = a.post1[s * W + w];
                const int b = slab * W + w;
                const size_t buf = (a.iters && b < a.batch) ? static_cast<size_t>(a.iters[b] & 1) * a.hb1_stride : 0;
                bit = (a.hb1[buf + s * NB + w / 8] >> (w & 7)) & 1u;
            }
        }
        tile[jj][w] = v;
        tbit[jj][w] = bit;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < W * 32; idx += blockDim.x) {
        const int w = idx / 32, jj = idx % 32;
        const int b = slab * W + w;
        const int32_t j = j0 + jj;
        if (b >= a.batch || j >= a.n_vn) continue;
        a.bits[static_cast<size_t>(b) * a.n_vn + j] = tbit[jj][w];
        if (a.post) a.post[static_cast<size_t>(b) * a.n_vn + j] = tile[jj][w] * a.scale;
    }
}

template <int W>
__global__ void __launch_bounds__(kBlock) k_deinterleave_out(OutArgs a) {
    deinterleave_body<W>(a, blockIdx.x, blockIdx.y);
}

// phi of nats inputs through fit F: scale_in converts to the fit's units,
// scale_out converts the result back to nats.
template <int F>
__global__ void k_phi_eval(const float *x, float *out, int64_t n, float scale_in, float lmax, float amin,
                           float scale_out) {
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fminf(phi_f<F>(clampf(x[i] * scale_in, amin, lmax)), lmax) * scale_out;
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
    float lmax = 25.f, amin = 0.f;   // LLR clamp and phi(lmax), nats
    // internal units of the decoding kernels (bits: an LLR times log2 e)
    float lmax_i = 0.f, amin_i = 0.f, scale_in = 1.f, scale_out = 1.f;
    void *r = nullptr;
    float *Lv = nullptr, *lch = nullptr, *lch1 = nullptr, *post1 = nullptr, *phi1 = nullptr;
    uint8_t *hb_core = nullptr, *hb1 = nullptr, *sbits = nullptr;
    uint32_t *done = nullptr, *fail = nullptr;
    int32_t *iters = nullptr;
    uint8_t *conv = nullptr;
    int32_t *status = nullptr;
    // posterior accumulation (MLD_VN_ACCUMULATE): two more posterior buffers
    int vn_update = MLD_VN_GATHER;
    int schedule = MLD_SCHED_FLOODING;
    int check_rule = MLD_CHECK_SUM_PRODUCT;
    float ms_off_i = 0.f;  // min-sum offset, internal units
    int checked = 0;       // validate the graph store before every decode
    int staging = MLD_STAGE_DIRECT;  // check-update operands: direct or bulk-staged
    // weighted BP: the tape in use, and the buffers of the last destroyed one
    mld_tape *tape_live = nullptr, *tape_spare = nullptr;
    int32_t stall_test = 0;          // mld_decoder_test_stall
    int32_t *status_host = nullptr;  // page-locked copy of the status word
    // early termination run by the device: capture stream, iteration counter
    // and cap (device), and the loop graphs built so far (per batch size,
    // variant and layering of the graph)
    cudaStream_t cap = nullptr;
    int32_t *lctr = nullptr;
    struct LoopGraph { int32_t batch, variant; uint64_t layers_gen; cudaGraphExec_t exec; };
    std::vector<LoopGraph> loops;
    float *Lv2 = nullptr, *Lv3 = nullptr;
    // staging buffers for host pointers
    float *in_stage = nullptr, *sigma_stage = nullptr, *post_stage = nullptr;
    uint8_t *syn_stage = nullptr, *bits_stage = nullptr;
    // side stream for check classes run beside the largest one (null: all
    // classes on the caller's stream), with its fork and join events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // kernel timing hook
    struct Timed { int cls; cudaEvent_t a, b; };
    bool timing = false;
    int timing_every = 1;        // time every N-th iteration's launches
    bool sample_now = true;      // the launches being enqueued are timed
    int64_t launches[4] = {0, 0, 0, 0};  // kernels launched while timing is on, per class
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> event_pool;
};

namespace mld {
// decode_f16.cu / decode_f32.cu: one decode call's launch sequence for each
// message storage type (separate translation units, compiled in parallel).
int run_decode_f16(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn, int32_t batch,
                   int32_t iters, bool et, uint8_t *bits, float *post, uint8_t *conv, int32_t *it,
                   cudaStream_t st, bool out_dev);
int run_decode_f32(mld_decoder *d, const float *in, const float *sigma, const uint8_t *syn, int32_t batch,
                   int32_t iters, bool et, uint8_t *bits, float *post, uint8_t *conv, int32_t *it,
                   cudaStream_t st, bool out_dev);
// Sets the shared-memory carveout of the staged kernels that decode_f16.cu
// launches (a function attribute belongs to one translation unit's kernel).
cudaError_t prepare_staged_f16();
// wbp.cu: frees a decoder's spare weighted-BP tape, detaches a live one.
void tape_release(mld_decoder *d);
}  // namespace mld

namespace {

// Sets the clamps and the nats <-> bits scales of a decoder from its lmax.
inline void set_units(mld_decoder *d, float lmax) {
    const double kLog2e = 1.4426950408889634074;
    d->lmax = lmax;
    d->amin = static_cast<float>(std::log1p(2.0 / std::expm1(static_cast<double>(lmax))));
    d->lmax_i = static_cast<float>(lmax * kLog2e);
    d->amin_i = static_cast<float>(std::log1p(2.0 / std::expm1(static_cast<double>(lmax))) * kLog2e);
    d->scale_in = static_cast<float>(kLog2e);
    d->scale_out = static_cast<float>(1.0 / kLog2e);
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

// Launch `nk` kernels through `fn`, bracketed by one pair of timing events
// when timing is on and this launch is sampled.
template <typename F>
int timed_launch(mld_decoder *d, int cls, cudaStream_t st, const char *what, F &&fn, int nk = 1) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (d->timing) d->launches[cls] += nk;
    const bool sample = d->timing && d->sample_now;
    if (sample) {
        a = pool_event(d);
        b = pool_event(d);
        if (!a || !b) return mld::fail(MLD_ECUDA, "cudaEventCreate");
        MLD_CUDA(cudaEventRecord(a, st));
    }
    fn();
    MLD_LAUNCHED(what);
    if (sample) {
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

}  // namespace
