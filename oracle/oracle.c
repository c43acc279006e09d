/*
 * FP64 CPU oracle for the Hermite block-timestep direct N-body path.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the CUDA library. Plain sequential
 * loops in the order of the paper's formulas (Portegies Zwart et al.,
 * "A parallel gravitational N-body kernel", Sect. 2.1). Build with
 *   gcc -O2 -ffp-contract=off [-fopenmp] -shared -fPIC
 * so that no multiply-add is fused and every result is reproducible.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ERR_NONFINITE (-3)
#define ORC_ERR_DT_UNDERFLOW (-4)
#define ORC_ERR_ARG (-1)

/* ------------------------------------------------------------------ force */

/* Eq. (Force): a_i = G sum_{j != i} m_j (r_j - r_i)/|r_j - r_i|^3, read with
 * the attractive sign and Plummer softening; the jerk is d a_i / dt along the
 * predicted motion (Sect. 2.1: "a and k ... recalculated ... using direct
 * summation"); phi_i is the matching softened potential. */
static void force_one(int64_t n, const double *m, const double *x, const double *v, double eps2,
                      int64_t i, double *ai, double *ki, double *phii)
{
    double ax = 0.0, ay = 0.0, az = 0.0;
    double kx = 0.0, ky = 0.0, kz = 0.0;
    double p = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double rx = x[3 * j + 0] - x[3 * i + 0];
        double ry = x[3 * j + 1] - x[3 * i + 1];
        double rz = x[3 * j + 2] - x[3 * i + 2];
        double wx = v[3 * j + 0] - v[3 * i + 0];
        double wy = v[3 * j + 1] - v[3 * i + 1];
        double wz = v[3 * j + 2] - v[3 * i + 2];
        double d2 = rx * rx + ry * ry + rz * rz + eps2;
        double d = sqrt(d2);
        double d3 = d2 * d;
        double d5 = d3 * d2;
        double rw = rx * wx + ry * wy + rz * wz;
        ax += m[j] * rx / d3;
        ay += m[j] * ry / d3;
        az += m[j] * rz / d3;
        kx += m[j] * (wx / d3 - 3.0 * rw * rx / d5);
        ky += m[j] * (wy / d3 - 3.0 * rw * ry / d5);
        kz += m[j] * (wz / d3 - 3.0 * rw * rz / d5);
        p -= m[j] / d;
    }
    ai[0] = ax; ai[1] = ay; ai[2] = az;
    ki[0] = kx; ki[1] = ky; ki[2] = kz;
    *phii = p;
}

void orc_force(int64_t n, const double *m, const double *x, const double *v, double eps2,
               int64_t s, const int32_t *idx, double *a, double *k, double *phi, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 1) {
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16)
        for (int64_t ii = 0; ii < s; ++ii)
            force_one(n, m, x, v, eps2, idx[ii], a + 3 * ii, k + 3 * ii, phi + ii);
        return;
    }
#else
    (void)nthreads;
#endif
    for (int64_t ii = 0; ii < s; ++ii)
        force_one(n, m, x, v, eps2, idx[ii], a + 3 * ii, k + 3 * ii, phi + ii);
}

/* -------------------------------------------------------------- predictor */

void orc_predict(int64_t n, const double *x, const double *v, const double *a, const double *k,
                 const double *t, double t_new, double *xp, double *vp)
{
    for (int64_t j = 0; j < n; ++j) {
        double d = t_new - t[j];
        double d2 = d * d;
        double d3 = d2 * d;
        for (int c = 0; c < 3; ++c) {
            int64_t q = 3 * j + c;
            xp[q] = x[q] + v[q] * d + a[q] * d2 / 2.0 + k[q] * d3 / 6.0;
            vp[q] = v[q] + a[q] * d + k[q] * d2 / 2.0;
        }
    }
}

/* -------------------------------------------------------------- corrector */

void orc_correct_one(const double *xp, const double *vp, const double *a_old, const double *k_old,
                     const double *a_new, const double *k_new, double dt,
                     double *x1, double *v1, double *a2, double *a3)
{
    double dt2 = dt * dt;
    double dt3 = dt2 * dt;
    double dt4 = dt3 * dt;
    double dt5 = dt4 * dt;
    for (int c = 0; c < 3; ++c) {
        double da = a_old[c] - a_new[c];
        a2[c] = -6.0 * da / dt2 - (4.0 * k_old[c] + 2.0 * k_new[c]) / dt;
        a3[c] = 12.0 * da / dt3 + 6.0 * (k_old[c] + k_new[c]) / dt2;
        x1[c] = xp[c] + a2[c] * dt4 / 24.0 + a3[c] * dt5 / 120.0;
        v1[c] = vp[c] + a2[c] * dt3 / 6.0 + a3[c] * dt4 / 24.0;
    }
}

static double dot3(const double *u, const double *w)
{
    return u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
}

double orc_aarseth_dt(const double *a_new, const double *k_new, const double *a2p,
                      const double *a3, double eta)
{
    double amag = sqrt(dot3(a_new, a_new));
    double kmag = sqrt(dot3(k_new, k_new));
    double a2mag = sqrt(dot3(a2p, a2p));
    double a3mag = sqrt(dot3(a3, a3));
    double num = amag * a2mag + dot3(k_new, k_new);
    double den = kmag * a3mag + dot3(a2p, a2p);
    if (den == 0.0) return INFINITY;      /* no higher derivatives: no limit */
    return sqrt(eta * num / den);
}

void orc_correct_particle(const double *xp, const double *vp, const double *a_old, const double *k_old,
                          const double *a_new, const double *k_new, double dt, double eta,
                          double *x1, double *v1, double *dt_cand)
{
    double a2[3], a3[3], a2p[3];
    orc_correct_one(xp, vp, a_old, k_old, a_new, k_new, dt, x1, v1, a2, a3);
    for (int c = 0; c < 3; ++c) a2p[c] = a2[c] + a3[c] * dt;
    *dt_cand = orc_aarseth_dt(a_new, k_new, a2p, a3, eta);
}

/* largest power of two <= x, for finite x > 0 */
static double pow2_floor(double x)
{
    int e;
    (void)frexp(x, &e);          /* x = f 2^e, f in [1/2, 1) */
    return ldexp(1.0, e - 1);
}

double orc_quantise(double dt_cand, double dt_old, double t_new, double dt_max, double dt_min)
{
    if (!(dt_cand > 0.0)) return 0.0;               /* NaN, zero or negative */
    double q = isinf(dt_cand) ? INFINITY : pow2_floor(dt_cand);
    double dt;
    double dt2 = 2.0 * dt_old;
    if (q < dt_old) {
        dt = q;
    } else if (q >= dt2 && dt2 <= dt_max) {
        double u = t_new / dt2;
        dt = (u == floor(u)) ? dt2 : dt_old;
    } else {
        dt = dt_old;
    }
    if (dt > dt_max) dt = dt_max;
    if (dt < dt_min) return 0.0;
    return dt;
}

double orc_initial_dt(const double *a, const double *k, double eta, double dt_max, double dt_min)
{
    double amag = sqrt(dot3(a, a));
    double kmag = sqrt(dot3(k, k));
    double cand = (kmag > 0.0) ? eta * amag / kmag : INFINITY;
    if (!(cand > 0.0)) return 0.0;
    double dt = isinf(cand) ? dt_max : pow2_floor(cand);
    if (dt > dt_max) dt = dt_max;
    if (dt < dt_min) return 0.0;
    return dt;
}

/* --------------------------------------------------------- block selection */

int64_t orc_next_block(int64_t n, const double *t, const double *dt, double *t_next, int32_t *idx)
{
    if (n <= 0) { *t_next = INFINITY; return 0; }
    double tmin = t[0] + dt[0];
    for (int64_t i = 1; i < n; ++i) {
        double ti = t[i] + dt[i];
        if (ti < tmin) tmin = ti;
    }
    int64_t s = 0;
    for (int64_t i = 0; i < n; ++i)
        if (t[i] + dt[i] == tmin) {
            if (idx) idx[s] = (int32_t)i;
            ++s;
        }
    *t_next = tmin;
    return s;
}

/* ----------------------------------------------------------------- energy */

void orc_energy(int64_t n, const double *m, const double *x, const double *v, double eps2,
                double *K, double *W, int nthreads)
{
    double *a = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *k = malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *phi = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int32_t *idx = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) idx[i] = (int32_t)i;
    orc_force(n, m, x, v, eps2, n, idx, a, k, phi, nthreads);
    double kin = 0.0, pot = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2];
        kin += 0.5 * m[i] * v2;
        pot += 0.5 * m[i] * phi[i];
    }
    *K = kin;
    *W = pot;
    free(a); free(k); free(phi); free(idx);
}

/* ------------------------------------------------------------- perturbers */

/* Sect. 3.1: the perturber list of a binary holds the stars with the strongest
 * effect on its internal motion, in the order the serial scan finds them, at most
 * nmax of them (the paper's N_pert = 256). The paper states the threshold as a
 * force of about 10^-7 relative to a mean force; read here as the tidal
 * perturbation of the binary: star j at distance r_j from the binary's centre of
 * mass accelerates the two members differently by about 2 m_j d / r_j^3 (d their
 * separation), against the binary's internal acceleration m_b / d^2, and it is a
 * perturber when the ratio 2 m_j d^3 / (m_b r_j^3) reaches gamma. The test is
 * taken without roots, on the sixth powers of the distances:
 *     (2 m_j)^2 d^6 >= (gamma m_b)^2 r_j^6. */
static double dist2(const double *u, const double *w)
{
    double dx = u[0] - w[0], dy = u[1] - w[1], dz = u[2] - w[2];
    return dx * dx + dy * dy + dz * dz;
}

void orc_perturbers(int64_t n, const double *m, const double *x, int32_t nbin, const int32_t *pairs,
                    double gamma, int32_t nmax, int64_t j_lo, int64_t j_hi, int32_t *lists, int32_t *counts)
{
    if (j_lo < 0) j_lo = 0;
    if (j_hi > n) j_hi = n;
    for (int32_t b = 0; b < nbin; ++b) {
        int32_t i = pairs[2 * b], k = pairs[2 * b + 1];
        double mb = m[i] + m[k];
        double cm[3];
        for (int c = 0; c < 3; ++c) cm[c] = (m[i] * x[3 * i + c] + m[k] * x[3 * k + c]) / mb;
        double d2 = dist2(x + 3 * i, x + 3 * k);
        double d6 = d2 * d2 * d2;
        double gm = gamma * mb;
        double rhs_scale = gm * gm;
        int32_t found = 0;
        for (int32_t q = 0; q < nmax; ++q) lists[(int64_t)b * nmax + q] = -1;
        for (int64_t j = j_lo; j < j_hi; ++j) {
            if (j == i || j == k) continue;
            double r2 = dist2(x + 3 * j, cm);
            double r6 = r2 * r2 * r2;
            double tm = 2.0 * m[j];
            if (tm * tm * d6 >= rhs_scale * r6) {
                if (found < nmax) lists[(int64_t)b * nmax + found] = (int32_t)j;
                ++found;
            }
        }
        counts[b] = found;
    }
}

/* ------------------------------------------------------------- integrator */

static int all_finite(const double *u, int64_t count)
{
    for (int64_t q = 0; q < count; ++q)
        if (!isfinite(u[q])) return 0;
    return 1;
}

int orc_init(orc_system *sys)
{
    int64_t n = sys->n;
    if (n < 0) return ORC_ERR_ARG;
    if (n == 0) return 0;
    int32_t *idx = malloc(sizeof(int32_t) * (size_t)n);
    double *phi = malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) { idx[i] = (int32_t)i; sys->t[i] = 0.0; }
    orc_force(n, sys->m, sys->x, sys->v, sys->eps2, n, idx, sys->a, sys->k, phi, sys->nthreads);
    int err = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (!all_finite(sys->a + 3 * i, 3) || !all_finite(sys->k + 3 * i, 3)) { err = ORC_ERR_NONFINITE; break; }
        double dt = sys->dt_fixed > 0.0 ? sys->dt_fixed
                  : orc_initial_dt(sys->a + 3 * i, sys->k + 3 * i, sys->eta, sys->dt_max, sys->dt_min);
        if (dt == 0.0 && !err) err = ORC_ERR_DT_UNDERFLOW;
        sys->dt[i] = dt;
    }
    free(idx); free(phi);
    sys->block_steps = 0;
    sys->particle_steps = 0;
    sys->interactions = 0.0;
    return err;
}

int orc_step(orc_system *sys, double *t_next_out, int64_t *s_out, int32_t *idx_out)
{
    int64_t n = sys->n;
    if (n <= 0) { *t_next_out = INFINITY; *s_out = 0; return 0; }
    int32_t *idx = malloc(sizeof(int32_t) * (size_t)n);
    double *xp = malloc(sizeof(double) * 3 * (size_t)n);
    double *vp = malloc(sizeof(double) * 3 * (size_t)n);
    double t_next;
    int64_t s = orc_next_block(n, sys->t, sys->dt, &t_next, idx);
    orc_predict(n, sys->x, sys->v, sys->a, sys->k, sys->t, t_next, xp, vp);
    double *an = malloc(sizeof(double) * 3 * (size_t)s);
    double *kn = malloc(sizeof(double) * 3 * (size_t)s);
    double *phi = malloc(sizeof(double) * (size_t)s);
    orc_force(n, sys->m, xp, vp, sys->eps2, s, idx, an, kn, phi, sys->nthreads);
    int bad_finite = 0, bad_dt = 0;
    for (int64_t ii = 0; ii < s; ++ii) {
        int64_t i = idx[ii];
        double dt = sys->dt[i];
        double x1[3], v1[3], cand;
        orc_correct_particle(xp + 3 * i, vp + 3 * i, sys->a + 3 * i, sys->k + 3 * i,
                             an + 3 * ii, kn + 3 * ii, dt, sys->eta, x1, v1, &cand);
        double dt_new = sys->dt_fixed > 0.0 ? sys->dt_fixed
                      : orc_quantise(cand, dt, t_next, sys->dt_max, sys->dt_min);
        if (!all_finite(x1, 3) || !all_finite(v1, 3) || !all_finite(an + 3 * ii, 3) ||
            !all_finite(kn + 3 * ii, 3))
            bad_finite = 1;
        if (dt_new == 0.0) bad_dt = 1;
        memcpy(sys->x + 3 * i, x1, sizeof x1);
        memcpy(sys->v + 3 * i, v1, sizeof v1);
        memcpy(sys->a + 3 * i, an + 3 * ii, 3 * sizeof(double));
        memcpy(sys->k + 3 * i, kn + 3 * ii, 3 * sizeof(double));
        sys->t[i] = t_next;
        sys->dt[i] = dt_new;
    }
    if (idx_out) memcpy(idx_out, idx, sizeof(int32_t) * (size_t)s);
    *t_next_out = t_next;
    *s_out = s;
    sys->block_steps += 1;
    sys->particle_steps += s;
    sys->interactions += (double)s * (double)n;
    free(idx); free(xp); free(vp); free(an); free(kn); free(phi);
    if (bad_finite) return ORC_ERR_NONFINITE;
    if (bad_dt) return ORC_ERR_DT_UNDERFLOW;
    return 0;
}

int orc_run(orc_system *sys, double t_end, int64_t max_steps)
{
    int64_t n = sys->n;
    int64_t done = 0;
    while (n > 0) {
        double tmin = sys->t[0] + sys->dt[0];
        for (int64_t i = 1; i < n; ++i) {
            double ti = sys->t[i] + sys->dt[i];
            if (ti < tmin) tmin = ti;
        }
        if (tmin > t_end) break;
        if (max_steps > 0 && done >= max_steps) break;
        double t_next;
        int64_t s;
        int err = orc_step(sys, &t_next, &s, NULL);
        ++done;
        if (err) return err;
    }
    return 0;
}
