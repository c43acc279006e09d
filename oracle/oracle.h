/*
 * FP64 CPU oracle for the Hermite block-timestep direct N-body path.
 *
 * TEST INFRASTRUCTURE ONLY. This oracle is a plain, slow, sequential
 * restatement of the method of Portegies Zwart et al., "A parallel
 * gravitational N-body kernel" (Sect. 2.1), used by the test-suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark. The CUDA library
 * never links, loads or calls it, and it shares no code with the library.
 *
 * Conventions (G = 1):
 *   positions, velocities, accelerations, jerks: double[n][3], row-major;
 *   masses, times, time steps, potentials: double[n];
 *   active lists: int32 indices, ascending.
 *
 * Readings of the paper that the oracle takes (the paper is silent or garbled
 * on these points):
 *   - Eq. (Force) is read as the attractive sum over (r_j - r_i) with Plummer
 *     softening eps^2 added to |r_j - r_i|^2; the jerk is the exact time
 *     derivative of that softened acceleration; phi_i = -sum m_j/(r^2+eps^2)^{1/2}.
 *   - j = i is excluded by index, never subtracted afterwards.
 *   - In the timestep criterion (Eq. timestep) a_p and k are the new
 *     acceleration and jerk at the end of the step, ddot a_p = a2 + a3 dt and
 *     ddot k = a3, with nu = eta = 0.01.
 *   - The first step uses dt = eta |a|/|k|; all steps are quantised to powers
 *     of two (see orc_quantise).
 */
#ifndef NB_ORACLE_H
#define NB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Eq. (Force), Sect. 2.1, plus its time derivative and the potential:
 * for each active i = idx[ii], ii < s, summed over j = 0..n-1 ascending, j != i:
 *   r = x_j - x_i, w = v_j - v_i, d2 = |r|^2 + eps2, d = sqrt(d2)
 *   a_i   += m_j r / d^3
 *   k_i   += m_j (w / d^3 - 3 (r.w) r / d^5)
 *   phi_i -= m_j / d
 * Outputs a, k: [s][3]; phi: [s]. nthreads > 1 splits the i loop over OpenMP
 * threads; every i-sum stays sequential over j, so results are identical. */
void orc_force(int64_t n, const double *m, const double *x, const double *v, double eps2,
               int64_t s, const int32_t *idx, double *a, double *k, double *phi, int nthreads);

/* Hermite predictor, Sect. 2.1: for every particle, with d = t_new - t[j],
 *   xp = x + v d + a d^2/2 + k d^3/6,   vp = v + a d + k d^2/2. */
void orc_predict(int64_t n, const double *x, const double *v, const double *a, const double *k,
                 const double *t, double t_new, double *xp, double *vp);

/* Hermite corrector for one particle, Sect. 2.1, with da = a_old - a_new:
 *   a2 = -6 da/dt^2 - (4 k_old + 2 k_new)/dt
 *   a3 = 12 da/dt^3 + 6 (k_old + k_new)/dt^2
 *   x  = xp + a2 dt^4/24 + a3 dt^5/120,  v = vp + a2 dt^3/6 + a3 dt^4/24.
 * All vectors are double[3]; outputs x1, v1, a2, a3. */
void orc_correct_one(const double *xp, const double *vp, const double *a_old, const double *k_old,
                     const double *a_new, const double *k_new, double dt,
                     double *x1, double *v1, double *a2, double *a3);

/* Eq. (timestep), Sect. 2.1 (Aarseth 1985):
 *   dt = sqrt(eta (|a||a2p| + |k|^2) / (|k||a3| + |a2p|^2)),  a2p = a2 + a3 dt_used. */
double orc_aarseth_dt(const double *a_new, const double *k_new, const double *a2p,
                      const double *a3, double eta);

/* Corrector plus the new step candidate for one active particle (Sect. 2.1):
 * orc_correct_one, then a2p = a2 + a3 dt (the second derivative carried to the
 * end of the step) and Eq. (timestep) with the new a and k. Writes x1, v1
 * and the unquantised candidate *dt_cand. */
void orc_correct_particle(const double *xp, const double *vp, const double *a_old, const double *k_old,
                          const double *a_new, const double *k_new, double dt, double eta,
                          double *x1, double *v1, double *dt_cand);

/* Power-of-two quantisation of a candidate step (Sect. 2.1 requires powers of
 * two; the rule itself is this library's reading): q = largest power of two
 * <= dt_cand (by frexp). If q < dt_old the step drops to q; if q >= 2 dt_old,
 * t_new is a multiple of 2 dt_old and 2 dt_old <= dt_max the step doubles
 * once; otherwise it stays dt_old. Returns 0 if the result is below dt_min,
 * or if dt_cand is not a positive finite number. */
double orc_quantise(double dt_cand, double dt_old, double t_new, double dt_max, double dt_min);

/* First step: quantised eta |a|/|k| capped at dt_max (|k| = 0 gives dt_max). */
double orc_initial_dt(const double *a, const double *k, double eta, double dt_max, double dt_min);

/* Block selection, Sect. 2.1: t_next = min_i (t_i + dt_i); idx = all i with
 * t_i + dt_i == t_next, ascending. Returns s (0 if n == 0). */
int64_t orc_next_block(int64_t n, const double *t, const double *dt, double *t_next, int32_t *idx);

/* Kinetic K = sum m v^2/2 and potential W = sum m_i phi_i / 2 (softened,
 * consistent with orc_force), from a full sum over all particles. */
void orc_energy(int64_t n, const double *m, const double *x, const double *v, double eps2,
                double *K, double *W, int nthreads);

/* Perturber lists of binaries (Sect. 3.1). Binary b = (pairs[2b], pairs[2b+1]).
 * Star j (not a member) perturbs it when its tidal acceleration across the
 * binary, relative to the binary's internal acceleration, reaches gamma:
 *     2 m_j d^3 / (m_b r_j^3) >= gamma,
 * d the members' separation, m_b their mass, r_j the distance from the binary's
 * centre of mass. Stars j in [j_lo, j_hi) are scanned in ascending index; the
 * first nmax perturbers go to lists[b][0..), in that order (unused entries -1);
 * counts[b] is the number found (it may exceed nmax). */
void orc_perturbers(int64_t n, const double *m, const double *x, int32_t nbin, const int32_t *pairs,
                    double gamma, int32_t nmax, int64_t j_lo, int64_t j_hi, int32_t *lists, int32_t *counts);

/* Integrator state. All arrays are caller-owned, length n ([n][3] for vectors). */
typedef struct {
    int64_t n;
    double *m, *x, *v, *a, *k, *t, *dt;
    double eps2, eta, dt_max, dt_min;
    double dt_fixed;   /* > 0: every particle takes this constant step (order tests) */
    int nthreads;
    /* counters */
    int64_t block_steps, particle_steps;
    double interactions;   /* sum of s*n over block steps */
} orc_system;

/* Computes a, k at t = 0 (all t = 0) and the first steps. Returns 0 or an
 * error code (-3 non-finite, -4 step underflow). */
int orc_init(orc_system *sys);

/* One block step: select, predict all, force on the block, correct, new steps.
 * Writes t_next, s and (if idx_out != NULL) the active list. Returns 0 or an
 * error code as above. */
int orc_step(orc_system *sys, double *t_next_out, int64_t *s_out, int32_t *idx_out);

/* Block steps until the next block time exceeds t_end. Returns 0 or an error.
 * With max_steps > 0 it stops after that many block steps. */
int orc_run(orc_system *sys, double t_end, int64_t max_steps);

#ifdef __cplusplus
}
#endif
#endif
