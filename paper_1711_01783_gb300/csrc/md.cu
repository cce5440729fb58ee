// Multidimensional reconciliation front end (d = 8) for sm_103a.
//
// The step before decoding in the paper's reconciliation (Results,
// "Information reconciliation for CV-QKD system"; Fig. 1): Bob and Alice turn
// correlated Gaussian samples Y = X + Z into Bob's bits and Alice's soft
// observation of them by rotating blocks of 8 samples onto a virtual
// binary-input AWGN channel.  Per block of 8:
//   Bob:   y' = y / |y|, u = (1 - 2 b) / sqrt 8 (b: his 8 bits),
//          alpha_i = <A_i y', u>   (i = 0..7), sends alpha and |y|;
//   Alice: (M x)_k = sum_i alpha_i (A_i x)_k with M = sum_i alpha_i A_i, and
//          LLR_k = 2 |y| (M x)_k / (sqrt 8 sigma_z^2).
// A_i is left multiplication by the basis octonion e_i.  M is orthogonal and
// M y' = u because the A_i y' form an orthonormal basis (octonion norms
// multiply).  Each A_i is a signed permutation, so both products are 64 sign
// flips and adds per block; one thread owns a block (32 contiguous bytes of
// every array), so the kernels stream: 8 B in, 4.5 B out per sample (Bob),
// 8.5 B in and 4 B out (Alice).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "internal.h"

namespace {

// ---------------------------------------------------------------------------
// Octonion basis products by the Cayley-Dickson doubling, evaluated at
// compile time.  Elements of the 2n-dimensional algebra are pairs (a, b) of
// n-dimensional ones with (a, b)(c, d) = (ac - conj(d) b, d a + b conj(c));
// for basis elements (e_i of the first half, e_{n+i} = (0, e_i)) this gives
//   e_i e_j         = e_i e_j                      (i, j < n)
//   e_i e_{n+j}     = (0, e_j e_i)
//   e_{n+i} e_j     = (0, e_i conj(e_j))
//   e_{n+i} e_{n+j} = (-conj(e_j) e_i, 0)
// with conj(e_0) = e_0 and conj(e_k) = -e_k otherwise; starting from the reals
// this builds the complex numbers, the quaternions (1, i, j, k) and the
// octonions.  prod(i, j) = s e_k is returned as (k, s).
// ---------------------------------------------------------------------------
struct BasisProduct {
    int index;
    int sign;
};

__host__ __device__ constexpr BasisProduct cd_basis(int n, int i, int j) {
    if (n == 1) return {0, 1};
    const int h = n / 2;
    const int si = (j % h == 0) ? 1 : -1;  // conj(e_j) = si e_j (within its half)
    if (i < h && j < h) return cd_basis(h, i, j);
    if (i < h) {  // (e_i, 0)(0, e_j') = (0, e_j' e_i)
        const BasisProduct p = cd_basis(h, j - h, i);
        return {h + p.index, p.sign};
    }
    if (j < h) {  // (0, e_i')(e_j, 0) = (0, e_i' conj(e_j))
        const BasisProduct p = cd_basis(h, i - h, j);
        return {h + p.index, p.sign * si};
    }
    // (0, e_i')(0, e_j') = (-conj(e_j') e_i', 0)
    const BasisProduct p = cd_basis(h, j - h, i - h);
    return {p.index, -p.sign * si};
}

// (A_i x)_k = sign * x[src] for the j with e_i e_j = +-e_k.
struct OctRows {
    int src[8][8];
    float sign[8][8];
};

__host__ __device__ constexpr OctRows oct_rows() {
    OctRows t{};
    for (int i = 0; i < 8; ++i)
        for (int j = 0; j < 8; ++j) {
            const BasisProduct p = cd_basis(8, i, j);
            t.src[i][p.index] = j;
            t.sign[i][p.index] = static_cast<float>(p.sign);
        }
    return t;
}

constexpr float kInvSqrt8 = 0.35355339059327376f;

__device__ __forceinline__ void load8(const float *p, float v[8]) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    const float4 b = *reinterpret_cast<const float4 *>(p + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

__device__ __forceinline__ void store8(float *p, const float v[8]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(v[4], v[5], v[6], v[7]);
}

__global__ void __launch_bounds__(128) k_md_bob(const float *y, const uint8_t *bits, int64_t nblk, float *alpha,
                                                float *ynorm) {
    constexpr OctRows kOct = oct_rows();  // evaluated by the compiler
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t blk = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; blk < nblk; blk += stride) {
        float v[8];
        load8(y + blk * 8, v);
        const uint2 bb = *reinterpret_cast<const uint2 *>(bits + blk * 8);
        float n2 = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) n2 = fmaf(v[k], v[k], n2);
        const float nrm = sqrtf(n2);
        // a block of zeros has no direction: take e_0 (any unit vector works)
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        float u[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const uint32_t byte = ((k < 4 ? bb.x : bb.y) >> (8 * (k & 3))) & 0xFFu;
            u[k] = (byte & 1u) ? -kInvSqrt8 : kInvSqrt8;
            v[k] = nrm > 0.f ? v[k] * inv : (k == 0 ? 1.f : 0.f);
        }
        float a[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) s = fmaf(kOct.sign[i][k] * v[kOct.src[i][k]], u[k], s);
            a[i] = s;
        }
        store8(alpha + blk * 8, a);
        ynorm[blk] = nrm;
    }
}

__global__ void __launch_bounds__(128) k_md_alice(const float *x, const float *alpha, const float *ynorm,
                                                  const float *noise_var, int64_t nblk, int64_t blk_per_row,
                                                  float *llr) {
    constexpr OctRows kOct = oct_rows();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t blk = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; blk < nblk; blk += stride) {
        float v[8], a[8], out[8];
        load8(x + blk * 8, v);
        load8(alpha + blk * 8, a);
        const float scale = 2.f * ynorm[blk] * kInvSqrt8 / noise_var[blk / blk_per_row];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float s = 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) s = fmaf(a[i], kOct.sign[i][k] * v[kOct.src[i][k]], s);
            out[k] = s * scale;
        }
        store8(llr + blk * 8, out);
    }
}

int md_fail(cudaError_t e, const char *what) {
    return mld::fail(MLD_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int grid_for(int64_t nblk) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((nblk + 127) / 128, static_cast<int64_t>(sms) * 16)));
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" int mld_md_bob(const float *y, const uint8_t *bits, int64_t count, float *alpha_out, float *ynorm_out,
                          void *stream) {
    mld::clear_error();
    if (count < 0 || count % 8 != 0) return mld::fail(MLD_EINVAL, "md_bob: count must be a multiple of 8");
    if (count == 0) return MLD_OK;
    if (!y || !bits || !alpha_out || !ynorm_out) return mld::fail(MLD_EINVAL, "md_bob: null pointer");
    if (!aligned16(y) || !aligned16(alpha_out) || (reinterpret_cast<uintptr_t>(bits) & 7u))
        return mld::fail(MLD_EINVAL, "md_bob: y and alpha_out must be 16-byte aligned, bits 8-byte aligned");
    const int64_t nblk = count / 8;
    k_md_bob<<<grid_for(nblk), 128, 0, static_cast<cudaStream_t>(stream)>>>(y, bits, nblk, alpha_out, ynorm_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLD_OK : md_fail(e, "k_md_bob");
}

extern "C" int mld_md_alice(const float *x, const float *alpha, const float *ynorm, const float *noise_var,
                            int32_t rows, int64_t row_len, float *llr_out, void *stream) {
    mld::clear_error();
    if (rows < 0 || row_len < 0 || row_len % 8 != 0)
        return mld::fail(MLD_EINVAL, "md_alice: rows >= 0 and row_len a multiple of 8 required");
    if (rows == 0 || row_len == 0) return MLD_OK;
    if (!x || !alpha || !ynorm || !noise_var || !llr_out) return mld::fail(MLD_EINVAL, "md_alice: null pointer");
    if (!aligned16(x) || !aligned16(alpha) || !aligned16(llr_out))
        return mld::fail(MLD_EINVAL, "md_alice: x, alpha and llr_out must be 16-byte aligned");
    const int64_t bpr = row_len / 8;
    const int64_t nblk = static_cast<int64_t>(rows) * bpr;
    k_md_alice<<<grid_for(nblk), 128, 0, static_cast<cudaStream_t>(stream)>>>(x, alpha, ynorm, noise_var, nblk, bpr,
                                                                              llr_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLD_OK : md_fail(e, "k_md_alice");
}
