// FP64 Hermite step arithmetic shared by the single-system step kernels and
// the ensemble kernel (Sect. 2.1 of the paper): predictor, corrector, the
// Aarseth step (Eq. timestep), power-of-two quantisation and the first step.
// Every translation unit that includes this file is compiled with
// -fmad=false, so each expression rounds operation by operation in the order
// written -- the same order as the FP64 CPU oracle, giving the same bits.
#pragma once

#include <math_constants.h>

#include "nb_ds.cuh"
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

// Power-of-two step rule: drop to the largest power of two below the candidate;
// double (once) only at times commensurate with twice the old step and within
// dt_max; otherwise keep. 0 means "below dt_min or no valid candidate".
__device__ __forceinline__ double quantise(double cand, double dt_old, double t_new, double dt_max, double dt_min)
{
    if (!(cand > 0.0)) return 0.0;
    const double q = isinf(cand) ? CUDART_INF : pow2_floor(cand);
    double dt;
    const double dt2 = 2.0 * dt_old;
    if (q < dt_old) {
        dt = q;
    } else if (q >= dt2 && dt2 <= dt_max) {
        const double u = t_new / dt2;
        dt = (u == floor(u)) ? dt2 : dt_old;
    } else {
        dt = dt_old;
    }
    if (dt > dt_max) dt = dt_max;
    if (dt < dt_min) return 0.0;
    return dt;
}

// Eq. (timestep): sqrt(eta (|a||a2p| + |k|^2) / (|k||a3| + |a2p|^2)); den = 0 sets no limit.
__device__ __forceinline__ double aarseth(const double *an, const double *kn, const double *a2p, const double *a3,
                                          double eta)
{
    const double amag = sqrt(dot3(an[0], an[1], an[2], an[0], an[1], an[2]));
    const double kmag = sqrt(dot3(kn[0], kn[1], kn[2], kn[0], kn[1], kn[2]));
    const double a2mag = sqrt(dot3(a2p[0], a2p[1], a2p[2], a2p[0], a2p[1], a2p[2]));
    const double a3mag = sqrt(dot3(a3[0], a3[1], a3[2], a3[0], a3[1], a3[2]));
    const double num = amag * a2mag + dot3(kn[0], kn[1], kn[2], kn[0], kn[1], kn[2]);
    const double den = kmag * a3mag + dot3(a2p[0], a2p[1], a2p[2], a2p[0], a2p[1], a2p[2]);
    if (den == 0.0) return CUDART_INF;
    return sqrt(eta * num / den);
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
        xp[c] = x[q] + v[q] * d + a[q] * d2 / 2.0 + k[q] * d3 / 6.0;
        vp[c] = v[q] + a[q] * d + k[q] * d2 / 2.0;
    }
}

// Hermite corrector and the new quantised step of particle i for the block time
// tn, given the new force an, kn; updates x, v, a, k, t, dt, tn in place and the
// double-single copies xd, vd, ad, kd when given (NULL: no copies).
// Returns status bits (non-finite, underflow). dt is a power of two, so dividing
// by dt, dt^2, dt^3 is the same exact scaling as multiplying by their reciprocals.
__device__ __forceinline__ int hermite_correct(double *x, double *v, double *a, double *k, double *t, double *dtv,
                                               double *tnv, float2 *xd, float2 *vd, float2 *ad, float2 *kd,
                                               int64_t np, int64_t i, double tn, const double *an,
                                               const double *kn, double eta, double dt_max, double dt_min)
{
    const double dt = dtv[i];
    double xp[3], vp[3];
    hermite_predict(x, v, a, k, t, np, i, tn, xp, vp);
    const double dt2 = dt * dt;
    const double dt3 = dt2 * dt;
    const double dt4 = dt3 * dt;
    const double dt5 = dt4 * dt;
    const double idt = 1.0 / dt;
    const double idt2 = idt * idt;
    const double idt3 = idt2 * idt;
    double x1[3], v1[3], a2[3], a3[3], a2p[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double ao = a[c * np + i], ko = k[c * np + i];
        const double da = ao - an[c];
        a2[c] = -6.0 * da * idt2 - (4.0 * ko + 2.0 * kn[c]) * idt;
        a3[c] = 12.0 * da * idt3 + 6.0 * (ko + kn[c]) * idt2;
        x1[c] = xp[c] + a2[c] * dt4 / 24.0 + a3[c] * dt5 / 120.0;
        v1[c] = vp[c] + a2[c] * dt3 / 6.0 + a3[c] * dt4 / 24.0;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) a2p[c] = a2[c] + a3[c] * dt;
    const double cand = aarseth(an, kn, a2p, a3, eta);
    const double dt_new = quantise(cand, dt, tn, dt_max, dt_min);
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c)
        finite = finite && isfinite(x1[c]) && isfinite(v1[c]) && isfinite(an[c]) && isfinite(kn[c]);
    int flags = 0;
    if (!finite) flags |= kStNonfinite;
    if (dt_new == 0.0) flags |= kStUnderflow;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        x[c * np + i] = x1[c];
        v[c * np + i] = v1[c];
        a[c * np + i] = an[c];
        k[c * np + i] = kn[c];
    }
    if (xd) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xd[c * np + i] = ds_pack(x1[c]);
            vd[c * np + i] = ds_pack(v1[c]);
            ad[c * np + i] = ds_pack(an[c]);
            kd[c * np + i] = ds_pack(kn[c]);
        }
    }
    t[i] = tn;
    dtv[i] = dt_new;
    tnv[i] = tn + dt_new;
    return flags;
}

}  // namespace nb
