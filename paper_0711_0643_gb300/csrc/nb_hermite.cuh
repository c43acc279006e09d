// FP64 Hermite step arithmetic shared by the single-system step kernels and
// the ensemble kernel (Sect. 2.1 of the paper): predictor, corrector, the
// Aarseth step (Eq. timestep), power-of-two quantisation and the first step.
// Every translation unit that includes this file is compiled with
// -fmad=false, so each expression rounds operation by operation in the order
// written -- the same order as the FP64 CPU oracle, giving the same bits.
// Divisions by the constants 6, 24, 120, products with 3, 6, 12 and with powers
// of two are replaced by the exact equivalents of nb_exact.cuh (same bits, on
// the integer pipe or with less FP64 work).
#pragma once

#include <math_constants.h>

#include "nb_ds.cuh"
#include "nb_exact.cuh"
#include "nb_internal.cuh"

namespace nb {

__device__ __forceinline__ double dot3(double ux, double uy, double uz, double wx, double wy, double wz)
{
    return ux * wx + uy * wy + uz * wz;
}

// largest power of two <= x for finite x > 0
__device__ __forceinline__ double pow2_floor(double x)
{
    int e;
    (void)frexp(x, &e);
    return ldexp(1.0, e - 1);
}

// Squared norm inside [2^-120, 2^120]: its FP32 copy, square root and the
// products below stay normal.
__host__ __device__ __forceinline__ bool norm2_in_range(double S)
{
    const int e = dexpo(S);
    return e >= 1023 - 120 && e <= 1023 + 120;
}

// The quantiser needs the Aarseth step only through the largest power of two
// below it. FP32 estimate from rA = sqrt(A), rK, rP, rQ and fK = K, fP = P (all
// FP32, from FP64 squared norms in range): relative error under 2^-19 (about a
// dozen correctly rounded FP32 operations). When the estimate's significand is
// at least 2^-14 away from 1 and from 2, it has the exact step's exponent: qb is
// that power of two and the function returns true; otherwise false, and the
// caller evaluates the FP64 expression sqrt(eta (|a||a2p| + |k|^2) / (|k||a3| +
// |a2p|^2)) as the oracle does.
__host__ __device__ __forceinline__ bool aarseth_estimate(float rA, float rK, float rP, float rQ, float fK,
                                                          float fP, float eta_f, long long &qb)
{
    // separate roundings, whatever the including file's contraction setting
#ifdef __CUDA_ARCH__
    const float num = __fadd_rn(__fmul_rn(rA, rP), fK);
    const float den = __fadd_rn(__fmul_rn(rK, rQ), fP);
    const float ratio = __fdiv_rn(__fmul_rn(eta_f, num), den);
#else
    const float num = rA * rP + fK;
    const float den = rK * rQ + fP;
    const float ratio = (eta_f * num) / den;
#endif
    const int re = (fbits(ratio) >> 23) & 0xff;
    const float c32 = sqrtf(ratio);
    const int cb = fbits(c32);
    const int cm = cb & 0x7fffff;
    qb = (long long)(((cb >> 23) & 0xff) - 127 + 1023) << 52;
    return re >= 127 - 120 && re <= 127 + 120 && cm >= (1 << 9) && cm <= 0x7fffff - (1 << 10);
}

__device__ __forceinline__ double initial_step(const double *a, const double *k, double eta, double dt_max,
                                               double dt_min)
{
    const double amag = sqrt(dot3(a[0], a[1], a[2], a[0], a[1], a[2]));
    const double kmag = sqrt(dot3(k[0], k[1], k[2], k[0], k[1], k[2]));
    const double cand = (kmag > 0.0) ? eta * amag / kmag : CUDART_INF;
    if (!(cand > 0.0)) return 0.0;
    double dt = isinf(cand) ? dt_max : pow2_floor(cand);
    if (dt > dt_max) dt = dt_max;
    if (dt < dt_min) return 0.0;
    return dt;
}

// Hermite predictor of particle i (state vectors [3][np]) to time tn.
__device__ __forceinline__ void hermite_predict(const double *x, const double *v, const double *a, const double *k,
                                                const double *t, int64_t np, int64_t i, double tn, double *xp,
                                                double *vp)
{
    const double d = tn - t[i];
    const double d2 = d * d;
    const double d3 = d2 * d;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int64_t q = c * np + i;
        xp[c] = ((x[q] + v[q] * d) + (a[q] * d2) * 0.5) + div6(k[q] * d3);
        vp[c] = (v[q] + a[q] * d) + (k[q] * d2) * 0.5;
    }
}

__device__ __forceinline__ double pick4(double v0, double v1, double v2, double v3, int w)
{
    return w == 0 ? v0 : (w == 1 ? v1 : (w == 2 ? v2 : v3));
}

// hermite_correct for one particle per group of four lanes. An FP64 warp
// instruction costs the same whatever its active lanes, so lanes 0-2 carry the
// x, y, z components through the predictor and the corrector (a third of the
// instructions of one thread doing all three) and lane 3 joins for the step.
// Same results, bit for bit. Every FP64 operation is an explicit
// round-to-nearest intrinsic, so the result does not depend on whether the
// including file lets the compiler contract multiply-adds. All 32 lanes of the
// warp call it together (full-mask shuffles); lane q = lane & 3 passes
// component min(q, 2) of the new a and k. i must be a valid particle even when
// live is false: the group then computes without storing. Returns status bits;
// lane 3 of a live group also writes the new key t + dt to *key_out if given.
// g is load_group(H, i), read by the caller (the overload below reads it).
// y / 6, y / 24, y / 120 and 3 y 2^s, correctly rounded, on the integer pipe
// (nb_exact.cuh); the FP64 unit only out of line, outside the exponent window.
static __device__ __noinline__ double ddiv_slow(double y, double d) { return __ddiv_rn(y, d); }
__device__ __forceinline__ double rn_div6(double y)
{
    double q;
    return div3_int(y, 1, q) ? q : ddiv_slow(y, 6.0);
}
__device__ __forceinline__ double rn_div24(double y)
{
    double q;
    return div3_int(y, 3, q) ? q : ddiv_slow(y, 24.0);
}
__device__ __forceinline__ double rn_div120(double y)
{
    double q;
    return div15_int(y, 3, q) ? q : ddiv_slow(y, 120.0);
}
__device__ __forceinline__ double rn_mul3(double y, int s, double p)   // p = 3 * 2^s
{
    double q;
    return mul3_int(y, s, q) ? q : dmul_slow(y, p);
}
__device__ __forceinline__ double dneg(double x) { return dfrom(dbits(x) ^ (long long)0x8000000000000000ull); }
static __device__ __noinline__ float2 ds_pack_slow(double x)
{
    const float h = __double2float_rn(x);
    return make_float2(h, __double2float_rn(__dsub_rn(x, (double)h)));
}
// (RN32(x), RN32(x - RN32(x))): on the integer pipe when both parts are normal floats
__device__ __forceinline__ float2 rn_ds_pack(double x)
{
    unsigned h, l;
    if (ds_split_int(x, h, l)) return make_float2(ffrom(h), ffrom(l));
    return ds_pack_slow(x);
}
__device__ __forceinline__ double pow2_of(int e) { return dfrom((long long)(1023 + e) << 52); }

// A second copy of the double-single state, the times and the keys that
// correct_group also writes when given one (the small-block engine keeps its
// particles' copy in shared memory): element (c, i) at c * np + (i - base).
struct DsMirror {
    float2 *x2, *v2, *a2, *k2;
    float2 *t;            // times as double-single (hi, lo)
    long long *key;
    int64_t np, base;
};

// The state correct_group reads for particle i (lane q: component min(q, 2)).
struct GroupState {
    double ti, dt, x, v, ao, ko;
};
__device__ __forceinline__ GroupState load_group(const HState &H, int64_t i)
{
    const int q = threadIdx.x & 3;
    const int64_t o = (q < 3 ? q : 2) * H.np + i;
    return GroupState{H.t[i], H.dt[i], H.x[o], H.v[o], H.a[o], H.k[o]};
}

__device__ __forceinline__ int correct_group(const HState &H, int64_t i, const GroupState &g, bool live, double tn,
                                             double an, double kn, double eta, double dt_max, double dt_min,
                                             long long *key_out = nullptr, const DsMirror *mir = nullptr)
{
    const int lane = threadIdx.x & 31;
    const int q = lane & 3;
    const int c = q < 3 ? q : 2;
    const int g0 = lane & ~3;
    const unsigned full = 0xffffffffu;
    const int64_t np = H.np;
    const int64_t o = c * np + i;
    const double ti = g.ti, dt = g.dt, x = g.x, v = g.v, ao = g.ao, ko = g.ko;

    // predictor: ((x + v d) + (a d^2) / 2) + (k d^3) / 6 and (v + a d) + (k d^2) / 2;
    // corrector: a2 = -6 da / dt^2 - (4 k_old + 2 k_new) / dt,
    // a3 = 12 da / dt^3 + 6 (k_old + k_new) / dt^2, x1 = xp + a2 dt^4 / 24 + a3 dt^5 / 120,
    // v1 = vp + a2 dt^3 / 6 + a3 dt^4 / 24, a2p = a2 + a3 dt (dt is a power of two
    // in [2^-300, 2^300], so 1/dt^k are exact)
    const double d = __dsub_rn(tn, ti);
    const double da = __dsub_rn(ao, an);
    const long long dtb = dbits(dt);
    const int e = (int)((dtb >> 52) & 0x7ff) - 1023;
    double x1, v1, a2, a3;
    if (__all_sync(full, dbits(d) == dtb && e >= -204 && e <= 204)) {
        // d = dt = 2^e and every dt^k, 1/dt^k is a normal power of two: each product
        // with one of them (and with 2, 4, 1/2) is an exponent shift (scale2), the
        // same bits as the FP64 multiply below
        const double d2 = pow2_of(2 * e), d3 = pow2_of(3 * e), d4 = pow2_of(4 * e), d5 = pow2_of(5 * e);
        const double i1 = pow2_of(-e), i2 = pow2_of(-2 * e), i3 = pow2_of(-3 * e);
        const double xp = __dadd_rn(__dadd_rn(__dadd_rn(x, scale2(v, e, dt)), scale2(scale2(ao, 2 * e, d2), -1, 0.5)),
                                    rn_div6(scale2(ko, 3 * e, d3)));
        const double vp = __dadd_rn(__dadd_rn(v, scale2(ao, e, dt)), scale2(scale2(ko, 2 * e, d2), -1, 0.5));
        // -6 da, 12 da and 6 (k_old + k_new) as exact integer products (same bits)
        a2 = __dsub_rn(scale2(dneg(rn_mul3(da, 1, 6.0)), -2 * e, i2),
                       scale2(__dadd_rn(scale2(ko, 2, 4.0), scale2(kn, 1, 2.0)), -e, i1));
        a3 = __dadd_rn(scale2(rn_mul3(da, 2, 12.0), -3 * e, i3), scale2(rn_mul3(__dadd_rn(ko, kn), 1, 6.0), -2 * e, i2));
        x1 = __dadd_rn(__dadd_rn(xp, rn_div24(scale2(a2, 4 * e, d4))), rn_div120(scale2(a3, 5 * e, d5)));
        v1 = __dadd_rn(__dadd_rn(vp, rn_div6(scale2(a2, 3 * e, d3))), rn_div24(scale2(a3, 4 * e, d4)));
    } else {
        const double d2 = __dmul_rn(d, d);
        const double d3 = __dmul_rn(d2, d);
        const double xp = __dadd_rn(__dadd_rn(__dadd_rn(x, __dmul_rn(v, d)), __dmul_rn(__dmul_rn(ao, d2), 0.5)),
                                    rn_div6(__dmul_rn(ko, d3)));
        const double vp = __dadd_rn(__dadd_rn(v, __dmul_rn(ao, d)), __dmul_rn(__dmul_rn(ko, d2), 0.5));
        const double dt2 = __dmul_rn(dt, dt);
        const double dt3 = __dmul_rn(dt2, dt);
        const double dt4 = __dmul_rn(dt3, dt);
        const double dt5 = __dmul_rn(dt4, dt);
        const double idt = recip_pow2(dt);
        const double idt2 = __dmul_rn(idt, idt);
        const double idt3 = __dmul_rn(idt2, idt);
        a2 = __dsub_rn(__dmul_rn(__dmul_rn(-6.0, da), idt2),
                       __dmul_rn(__dadd_rn(__dmul_rn(4.0, ko), __dmul_rn(2.0, kn)), idt));
        a3 = __dadd_rn(__dmul_rn(__dmul_rn(12.0, da), idt3), __dmul_rn(__dmul_rn(6.0, __dadd_rn(ko, kn)), idt2));
        x1 = __dadd_rn(__dadd_rn(xp, rn_div24(__dmul_rn(a2, dt4))), rn_div120(__dmul_rn(a3, dt5)));
        v1 = __dadd_rn(__dadd_rn(vp, rn_div6(__dmul_rn(a2, dt3))), rn_div24(__dmul_rn(a3, dt4)));
    }
    const double a2p = __dadd_rn(a2, scale2(a3, e, dt));

    // The step's power of two from the FP32 estimate. Lane q gathers the three
    // component squares of vector q (a, k, a2p, a3) by rotating shuffles and sums
    // them in component order, as dot3 does, in FP32 from RN32 copies of the FP64
    // components made on the integer pipe (the estimate's error stays far inside
    // its 2^-14 decision window). The FP64 norms are formed only where the
    // estimate does not decide.
    float c0f, c1f, c2f, c3f;
    const bool ok32 = rn32_int(an, c0f) & rn32_int(kn, c1f) & rn32_int(a2p, c2f) & rn32_int(a3, c3f);
    const float t0 = sq_ftz(c0f), t1 = sq_ftz(c1f), t2 = sq_ftz(c2f), t3 = sq_ftz(c3f);
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int w = (q - r) & 3;   // lane src supplies vector (src - r) & 3
        const float mine = w == 0 ? t0 : (w == 1 ? t1 : (w == 2 ? t2 : t3));
        const int src = (q + r) & 3;
        const float got = __shfl_sync(full, mine, g0 + src);
        if (src == 0) f0 = got;
        if (src == 1) f1 = got;
        if (src == 2) f2 = got;
    }
    const float fS = (f0 + f1) + f2;
    const float rS = __fsqrt_rn(fS);
    const float rA = __shfl_sync(full, rS, g0), rK = __shfl_sync(full, rS, g0 + 1);
    const float rP = __shfl_sync(full, rS, g0 + 2), rQ = __shfl_sync(full, rS, g0 + 3);
    const float fK = __shfl_sync(full, fS, g0 + 1), fP = __shfl_sync(full, fS, g0 + 2);
    const unsigned okb = __ballot_sync(full, ok32 && norm2_f32_in_range(fS));
    long long qb = 0;
    bool pos = true;
    bool decided = aarseth_estimate(rA, rK, rP, rQ, fK, fP, __double2float_rn(eta), qb);
    decided = decided && ((okb >> g0) & 0xFu) == 0xFu;
    if (__any_sync(full, live && !decided)) {
        const double s0 = __dmul_rn(an, an), s1 = __dmul_rn(kn, kn), s2 = __dmul_rn(a2p, a2p),
                     s3 = __dmul_rn(a3, a3);
        double p0 = 0.0, p1 = 0.0, p2 = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const double mine = pick4(s0, s1, s2, s3, (q - r) & 3);
            const int src = (q + r) & 3;
            const double got = __shfl_sync(full, mine, g0 + src);
            if (src == 0) p0 = got;
            if (src == 1) p1 = got;
            if (src == 2) p2 = got;
        }
        const double S = __dadd_rn(__dadd_rn(p0, p1), p2);
        const double mag = __dsqrt_rn(S);   // the four magnitudes, one per lane
        const double mA = __shfl_sync(full, mag, g0), mK = __shfl_sync(full, mag, g0 + 1);
        const double mP = __shfl_sync(full, mag, g0 + 2), mQ = __shfl_sync(full, mag, g0 + 3);
        const double K = __shfl_sync(full, S, g0 + 1), P = __shfl_sync(full, S, g0 + 2);
        if (!decided) {
            const double num = __dadd_rn(__dmul_rn(mA, mP), K);
            const double den = __dadd_rn(__dmul_rn(mK, mQ), P);
            const double cand = den == 0.0 ? CUDART_INF : __dsqrt_rn(__ddiv_rn(__dmul_rn(eta, num), den));
            qb = pow2_floor_bits(cand);
            pos = dpositive(cand);
        }
    }
    int flags = 0;
    if (live) {
        if (q < 3) {
            if (!(dfinite(x1) && dfinite(v1) && dfinite(an) && dfinite(kn))) flags |= kStNonfinite;
            H.x[o] = x1;
            H.v[o] = v1;
            H.a[o] = an;
            H.k[o] = kn;
            if (H.x2) {
                const float2 px = rn_ds_pack(x1), pv = rn_ds_pack(v1), pa = rn_ds_pack(an), pk = rn_ds_pack(kn);
                H.x2[o] = px;
                H.v2[o] = pv;
                H.a2[o] = pa;
                H.k2[o] = pk;
                if (mir) {
                    const int64_t om = c * mir->np + (i - mir->base);
                    mir->x2[om] = px;
                    mir->v2[om] = pv;
                    mir->a2[om] = pa;
                    mir->k2[om] = pk;
                }
            }
        } else {
            const double dt_new = quantise_bits(qb, pos, dt, tn, dt_max, dt_min);
            if (dt_new == 0.0) flags |= kStUnderflow;
            const double key = __dadd_rn(tn, dt_new);
            H.t[i] = tn;
            H.dt[i] = dt_new;
            H.tn[i] = key;
            if (key_out) *key_out = dbits(key);
            if (mir) {
                mir->t[i - mir->base] = rn_ds_pack(tn);
                mir->key[i - mir->base] = dbits(key);
            }
        }
    }
    return flags;
}
__device__ __forceinline__ int correct_group(const HState &H, int64_t i, bool live, double tn, double an, double kn,
                                             double eta, double dt_max, double dt_min, long long *key_out = nullptr)
{
    return correct_group(H, i, load_group(H, i), live, tn, an, kn, eta, dt_max, dt_min, key_out);
}

}  // namespace nb
