// Mixed-precision pair arithmetic of Eq. (Force) and its time derivative, and
// the compensated (two-sum) accumulation helpers, shared by the force kernels
// and the ensemble kernel.
#pragma once

#include "nb_internal.cuh"

namespace nb {

constexpr int kFoldPairs = 64;     // FP32 terms per partial before a two-sum fold


struct IPart {
    float xh, yh, zh, xl, yl, zl, vx, vy, vz;
};

struct Acc7 {
    float ax, ay, az, kx, ky, kz, ph;
};

__device__ __forceinline__ void zero(Acc7 &q)
{
    q.ax = q.ay = q.az = q.kx = q.ky = q.kz = q.ph = 0.f;
}

// Particle i's fields in its pair record (lane i & 1 of every float4).
__device__ __forceinline__ void jrec_store(JPair *P, int64_t i, float xh, float yh, float zh, float m, float xl,
                                           float yl, float zl, float vx, float vy, float vz)
{
    float *r = reinterpret_cast<float *>(&P[i >> 1]);
    const int o = (int)(i & 1);
    r[0 + o] = xh;
    r[2 + o] = yh;
    r[4 + o] = zh;
    r[6 + o] = m;
    r[8 + o] = xl;
    r[10 + o] = yl;
    r[12 + o] = zl;
    r[14 + o] = vx;
    r[16 + o] = vy;
    r[18 + o] = vz;
}

__device__ __forceinline__ IPart jrec_load(const JPair *P, int64_t i)
{
    const float *r = reinterpret_cast<const float *>(&P[i >> 1]);
    const int o = (int)(i & 1);
    return IPart{r[0 + o], r[2 + o], r[4 + o], r[8 + o], r[10 + o], r[12 + o], r[14 + o], r[16 + o], r[18 + o]};
}

__device__ __forceinline__ float jrec_mass(const JPair *P, int64_t i)
{
    return reinterpret_cast<const float *>(&P[i >> 1])[6 + (int)(i & 1)];
}

// One i-j interaction. r = x_j - x_i in double-single, w = v_j - v_i,
// r2 = |r|^2 + eps^2, q = r2^{-1/2} (MUFU estimate + one Newton step),
// mu = m_j q^3, al = 3 (r.w) / r2:
//   a += mu r,  k += mu (w - al r),  phi -= m_j q.
// MASK zeroes the term when j == i (self-exclusion by index).
template <bool MASK>
__device__ __forceinline__ void pair_mixed(const float4 &h, const float4 &l, const float4 &w, const IPart &I,
                                           float eps2, Acc7 &A, bool self)
{
    float dx = (h.x - I.xh) + (l.x - I.xl);
    float dy = (h.y - I.yh) + (l.y - I.yl);
    float dz = (h.z - I.zh) + (l.z - I.zl);
    float wx = w.x - I.vx, wy = w.y - I.vy, wz = w.z - I.vz;
    float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float rw = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    float q = rsqrtf(r2);
    // one Newton-Raphson step for r2^{-1/2}: q <- q + q (1 - r2 q^2) / 2, which takes
    // the hardware estimate to about one ulp (the accuracy of a and k rests on it)
    const float e = fmaf(-r2 * q, q, 1.0f);
    q = fmaf(0.5f * q, e, q);
    if (MASK) q = self ? 0.f : q;
    float q2 = q * q;
    float mq = h.w * q;
    float mu = mq * q2;
    float al = 3.f * rw * q2;
    A.ph -= mq;
    A.ax = fmaf(mu, dx, A.ax);
    A.ay = fmaf(mu, dy, A.ay);
    A.az = fmaf(mu, dz, A.az);
    A.kx = fmaf(mu, fmaf(-al, dx, wx), A.kx);
    A.ky = fmaf(mu, fmaf(-al, dy, wy), A.ky);
    A.kz = fmaf(mu, fmaf(-al, dz, wz), A.kz);
}

// (hi, lo) += p exactly up to the rounding of lo (Knuth's two-sum), p = 0 after.
__device__ __forceinline__ void two_sum_fold(float &hi, float &lo, float &p)
{
    float s = hi + p;
    float bp = s - hi;
    float e = (hi - (s - bp)) + (p - bp);
    hi = s;
    lo += e;
    p = 0.f;
}

__device__ __forceinline__ void fold(Acc7 &hi, Acc7 &lo, Acc7 &p)
{
    two_sum_fold(hi.ax, lo.ax, p.ax);
    two_sum_fold(hi.ay, lo.ay, p.ay);
    two_sum_fold(hi.az, lo.az, p.az);
    two_sum_fold(hi.kx, lo.kx, p.kx);
    two_sum_fold(hi.ky, lo.ky, p.ky);
    two_sum_fold(hi.kz, lo.kz, p.kz);
    two_sum_fold(hi.ph, lo.ph, p.ph);
}

// (hi, lo) + (hi2, lo2) with a two-sum on the high parts.
__device__ __forceinline__ void ds_add(float &hi, float &lo, float hi2, float lo2)
{
    float s = hi + hi2;
    float bp = s - hi;
    float e = (hi - (s - bp)) + (hi2 - bp);
    e += lo + lo2;
    hi = s + e;                 // renormalise (fast two-sum)
    lo = e - (hi - s);
}

// xor-butterfly over the lanes of one group of G consecutive lanes (G | 32)
template <int G>
__device__ __forceinline__ void ds_group_reduce(float &hi, float &lo)
{
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, off);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, off);
        ds_add(hi, lo, h2, l2);
    }
}

// All seven components through the same butterfly, level by level: the shuffles
// of a level are independent and issue together (each component sees exactly the
// operations of ds_group_reduce<G>, so the results are the same bits).
template <int G>
__device__ __forceinline__ void ds_group_reduce7(Acc7 &hi, Acc7 &lo)
{
#pragma unroll
    for (int off = G / 2; off >= 1; off >>= 1) {
        float h[7], l[7];
        h[0] = __shfl_xor_sync(0xffffffffu, hi.ax, off); l[0] = __shfl_xor_sync(0xffffffffu, lo.ax, off);
        h[1] = __shfl_xor_sync(0xffffffffu, hi.ay, off); l[1] = __shfl_xor_sync(0xffffffffu, lo.ay, off);
        h[2] = __shfl_xor_sync(0xffffffffu, hi.az, off); l[2] = __shfl_xor_sync(0xffffffffu, lo.az, off);
        h[3] = __shfl_xor_sync(0xffffffffu, hi.kx, off); l[3] = __shfl_xor_sync(0xffffffffu, lo.kx, off);
        h[4] = __shfl_xor_sync(0xffffffffu, hi.ky, off); l[4] = __shfl_xor_sync(0xffffffffu, lo.ky, off);
        h[5] = __shfl_xor_sync(0xffffffffu, hi.kz, off); l[5] = __shfl_xor_sync(0xffffffffu, lo.kz, off);
        h[6] = __shfl_xor_sync(0xffffffffu, hi.ph, off); l[6] = __shfl_xor_sync(0xffffffffu, lo.ph, off);
        ds_add(hi.ax, lo.ax, h[0], l[0]);
        ds_add(hi.ay, lo.ay, h[1], l[1]);
        ds_add(hi.az, lo.az, h[2], l[2]);
        ds_add(hi.kx, lo.kx, h[3], l[3]);
        ds_add(hi.ky, lo.ky, h[4], l[4]);
        ds_add(hi.kz, lo.kz, h[5], l[5]);
        ds_add(hi.ph, lo.ph, h[6], l[6]);
    }
}

__device__ __forceinline__ float acc_get(const Acc7 &q, int c)
{
    switch (c) {
    case 0: return q.ax;
    case 1: return q.ay;
    case 2: return q.az;
    case 3: return q.kx;
    case 4: return q.ky;
    case 5: return q.kz;
    default: return q.ph;
    }
}

// ------------------------------------------------------- packed (f32x2) form
// The same interaction for two j-particles at once (the two lanes of a pair
// record) against one i-particle, with the packed FP32 instructions of sm_100+
// (__ffma2_rn, __fadd2_rn, __fmul2_rn): every operation below acts on both
// lanes, so a pair record costs about half the issue slots of two scalar
// evaluations. The i-particle is held broadcast and negated in both lanes.
struct IPk {
    float2 nxh, nyh, nzh, nxl, nyl, nzl, nvx, nvy, nvz;
};

struct AccPk {
    float2 ax, ay, az, kx, ky, kz, ph;
};

__device__ __forceinline__ IPk ipk_of(const IPart &I)
{
    return IPk{make_float2(-I.xh, -I.xh), make_float2(-I.yh, -I.yh), make_float2(-I.zh, -I.zh),
               make_float2(-I.xl, -I.xl), make_float2(-I.yl, -I.yl), make_float2(-I.zl, -I.zl),
               make_float2(-I.vx, -I.vx), make_float2(-I.vy, -I.vy), make_float2(-I.vz, -I.vz)};
}

__device__ __forceinline__ void zero(AccPk &q)
{
    const float2 z = make_float2(0.f, 0.f);
    q.ax = q.ay = q.az = q.kx = q.ky = q.kz = q.ph = z;
}

// MASK zeroes lane a (j = 2p) or b (j = 2p+1) when it is the i-particle itself.
template <bool MASK>
__device__ __forceinline__ void pair_packed(const float4 &q0, const float4 &q1, const float4 &q2, const float4 &q3,
                                            const float4 &q4, const IPk &I, float2 eps2, AccPk &A, bool self_a,
                                            bool self_b)
{
    const float2 dx = __fadd2_rn(__fadd2_rn(make_float2(q0.x, q0.y), I.nxh), __fadd2_rn(make_float2(q2.x, q2.y), I.nxl));
    const float2 dy = __fadd2_rn(__fadd2_rn(make_float2(q0.z, q0.w), I.nyh), __fadd2_rn(make_float2(q2.z, q2.w), I.nyl));
    const float2 dz = __fadd2_rn(__fadd2_rn(make_float2(q1.x, q1.y), I.nzh), __fadd2_rn(make_float2(q3.x, q3.y), I.nzl));
    const float2 wx = __fadd2_rn(make_float2(q3.z, q3.w), I.nvx);
    const float2 wy = __fadd2_rn(make_float2(q4.x, q4.y), I.nvy);
    const float2 wz = __fadd2_rn(make_float2(q4.z, q4.w), I.nvz);
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
    const float2 rw = __ffma2_rn(dx, wx, __ffma2_rn(dy, wy, __fmul2_rn(dz, wz)));
    float2 q = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
    // Newton step: t = r2 q^2 - 1, q <- q - (q/2) t (bitwise the scalar form's step)
    const float2 t = __ffma2_rn(__fmul2_rn(r2, q), q, make_float2(-1.f, -1.f));
    q = __ffma2_rn(__fmul2_rn(q, make_float2(-0.5f, -0.5f)), t, q);
    if (MASK) {
        q.x = self_a ? 0.f : q.x;
        q.y = self_b ? 0.f : q.y;
    }
    const float2 qq = __fmul2_rn(q, q);
    const float2 mq = __fmul2_rn(make_float2(q1.z, q1.w), q);
    const float2 mu = __fmul2_rn(mq, qq);
    const float2 nal = __fmul2_rn(__fmul2_rn(rw, make_float2(-3.f, -3.f)), qq);
    A.ph = __ffma2_rn(mq, make_float2(-1.f, -1.f), A.ph);
    A.ax = __ffma2_rn(mu, dx, A.ax);
    A.ay = __ffma2_rn(mu, dy, A.ay);
    A.az = __ffma2_rn(mu, dz, A.az);
    A.kx = __ffma2_rn(mu, __ffma2_rn(nal, dx, wx), A.kx);
    A.ky = __ffma2_rn(mu, __ffma2_rn(nal, dy, wy), A.ky);
    A.kz = __ffma2_rn(mu, __ffma2_rn(nal, dz, wz), A.kz);
}

// both lanes of the packed partial into the (hi, lo) two-sum accumulator; p = 0 after
__device__ __forceinline__ void fold_pk_one(float &hi, float &lo, float2 &p)
{
    float v = p.x + p.y;
    two_sum_fold(hi, lo, v);
    p = make_float2(0.f, 0.f);
}

__device__ __forceinline__ void fold(Acc7 &hi, Acc7 &lo, AccPk &p)
{
    fold_pk_one(hi.ax, lo.ax, p.ax);
    fold_pk_one(hi.ay, lo.ay, p.ay);
    fold_pk_one(hi.az, lo.az, p.az);
    fold_pk_one(hi.kx, lo.kx, p.kx);
    fold_pk_one(hi.ky, lo.ky, p.ky);
    fold_pk_one(hi.kz, lo.kz, p.kz);
    fold_pk_one(hi.ph, lo.ph, p.ph);
}

}  // namespace nb
