// Double-single (float hi + float lo) arithmetic for the mixed-precision
// predictor: the error-free transformations two-sum (Knuth) and two-product
// (Dekker, with a fused multiply-add) give ~48-bit sums and products on the
// FP32 pipe. The error-free transformations contain no multiply feeding an add
// (the products are explicit fmaf), and the one plain FP32 expression uses
// round-to-nearest intrinsics, so the results do not depend on whether the
// including file lets the compiler contract multiply-adds.
#pragma once

#include <cuda_runtime.h>

namespace nb {

struct DS {
    float hi, lo;
};

__device__ __forceinline__ DS ds_split(double x)
{
    const float h = (float)x;
    return DS{h, (float)(x - (double)h)};
}

__device__ __forceinline__ float2 ds_pack(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// hi + lo renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ DS ds_norm(float s, float e)
{
    const float h = s + e;
    return DS{h, e - (h - s)};
}

__device__ __forceinline__ DS ds_add(DS x, DS y)
{
    const float s = x.hi + y.hi;
    const float bp = s - x.hi;
    float e = (x.hi - (s - bp)) + (y.hi - bp);
    e += x.lo + y.lo;
    return ds_norm(s, e);
}

__device__ __forceinline__ DS ds_mul(DS x, DS y)
{
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, e);
    e = fmaf(x.lo, y.hi, e);
    return ds_norm(p, e);
}

__device__ __forceinline__ DS ds_scale2(DS x, float pow2) { return DS{x.hi * pow2, x.lo * pow2}; }

// Hermite predictor of one particle in double-single for the mixed j-record:
// xp = x + d (v + d (a/2 + d k/6)) per component (the same polynomial as
// x + v d + a d^2/2 + k d^3/6, in Horner form), vp = v + d (a + d k/2) in FP32.
// X, V, A, K: the particle's double-single x, v, a, k per component; d: the
// time since the particle's own time, as a double-single.
__device__ __forceinline__ void ds_predict_ds(const float2 *X, const float2 *V, const float2 *A, const float2 *K, DS d,
                                              float4 &hi, float4 &lo, float4 &vel, float m)
{
    const DS sixth = {0.166666671633720398f, -4.967053879e-09f};   // 1/6 = hi + lo to ~2^-53
    const DS d6 = ds_mul(d, sixth);
    float ph[3], pl[3], pv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        DS t = ds_mul(DS{K[c].x, K[c].y}, d6);
        t = ds_add(ds_scale2(DS{A[c].x, A[c].y}, 0.5f), t);
        t = ds_mul(t, d);
        t = ds_add(DS{V[c].x, V[c].y}, t);
        t = ds_mul(t, d);
        const DS xp = ds_add(DS{X[c].x, X[c].y}, t);
        ph[c] = xp.hi;
        pl[c] = xp.lo;
        pv[c] = __fadd_rn(__fadd_rn(V[c].x, __fmul_rn(d.hi, __fadd_rn(A[c].x, __fmul_rn(d.hi, __fmul_rn(0.5f, K[c].x))))),
                          V[c].y);
    }
    hi = make_float4(ph[0], ph[1], ph[2], m);
    lo = make_float4(pl[0], pl[1], pl[2], 0.f);
    vel = make_float4(pv[0], pv[1], pv[2], 0.f);
}

__device__ __forceinline__ void ds_predict_vals(const float2 *X, const float2 *V, const float2 *A, const float2 *K,
                                                double d64, float4 &hi, float4 &lo, float4 &vel, float m)
{
    ds_predict_ds(X, V, A, K, ds_split(d64), hi, lo, vel, m);
}

// (hi, lo) - (hi2, lo2) renormalised: the difference of two double-single times on
// the FP32 pipe (a two-sum of the high parts, the low parts added to its error)
__device__ __forceinline__ DS ds_sub(DS x, DS y) { return ds_add(x, DS{-y.hi, -y.lo}); }

// The same from the state arrays x2, v2, a2, k2 ([3][np] float2 (hi, lo)) of particle i.
__device__ __forceinline__ void ds_predict(const float2 *x2, const float2 *v2, const float2 *a2, const float2 *k2,
                                           int64_t np, int64_t i, double d64, float4 &hi, float4 &lo, float4 &vel,
                                           float m)
{
    float2 X[3], V[3], A[3], K[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        X[c] = x2[c * np + i];
        V[c] = v2[c * np + i];
        A[c] = a2[c * np + i];
        K[c] = k2[c * np + i];
    }
    ds_predict_vals(X, V, A, K, d64, hi, lo, vel, m);
}

// Double-single helpers of the softened potential sums (the energy kernels of
// the single-system path and of the ensemble). The two-sum steps rely on the
// including file being compiled without multiply-add contraction.
__device__ __forceinline__ void en_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void en_fast_two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    e = b - (s - a);
}
// (ah + al) - (bh + bl) as a normalised double-single
__device__ __forceinline__ void en_diff(float ah, float al, float bh, float bl, float &h, float &l)
{
    float s, e;
    en_two_sum(ah, -bh, s, e);
    e += al - bl;
    en_fast_two_sum(s, e, h, l);
}
// h + l += bh + bl
__device__ __forceinline__ void en_acc(float &h, float &l, float bh, float bl)
{
    float s, e;
    en_two_sum(h, bh, s, e);
    e += l + bl;
    en_fast_two_sum(s, e, h, l);
}

// m_j / |r_ij| (softened) as a double-single, from double-single positions and
// mass: r = x_j - x_i and r^2 + eps^2 to ~2^-46 relative (two-sums and exact
// squares by FMA), q = (r^2 + eps^2)^(-1/2) from the MUFU estimate, one FP32 and
// one double-single Newton step (the residual 1 - r^2 y^2 is exact to 2^-46),
// error ~2^-44 relative.
__device__ __forceinline__ void en_pair(float4 j0, float4 j1, float2 xi, float2 yi, float2 zi, float2 e2, float &th,
                                        float &tl)
{
    float dh, dl, r2h, r2l, p, e;
    en_diff(j0.x, j0.y, xi.x, xi.y, dh, dl);
    r2h = dh * dh;
    r2l = fmaf(dh, dh, -r2h);
    r2l = fmaf(2.f * dh, dl, r2l);
    en_diff(j0.z, j0.w, yi.x, yi.y, dh, dl);
    p = dh * dh;
    e = fmaf(dh, dh, -p);
    e = fmaf(2.f * dh, dl, e);
    en_acc(r2h, r2l, p, e);
    en_diff(j1.x, j1.y, zi.x, zi.y, dh, dl);
    p = dh * dh;
    e = fmaf(dh, dh, -p);
    e = fmaf(2.f * dh, dl, e);
    en_acc(r2h, r2l, p, e);
    en_acc(r2h, r2l, e2.x, e2.y);
    float y = rsqrtf(r2h);
    y = y * fmaf(-0.5f * r2h * y, y, 1.5f);
    const float a2 = y * y;
    const float a2e = fmaf(y, y, -a2);
    const float c = r2h * a2;
    const float ce = fmaf(r2h, a2, -c);
    const float res = (1.f - c) - (ce + fmaf(r2h, a2e, r2l * a2));
    float qh, ql;
    en_fast_two_sum(y, 0.5f * y * res, qh, ql);
    th = j1.z * qh;
    tl = fmaf(j1.z, qh, -th);
    tl = fmaf(j1.z, ql, tl);
    tl = fmaf(j1.w, qh, tl);
}

}  // namespace nb
