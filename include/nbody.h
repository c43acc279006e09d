/*
 * nbody.h -- C ABI of the GB300 (sm_103a) Hermite block-timestep direct N-body
 * library (libnbody.so).
 *
 * The library implements the hot path of the integrator described in
 * Portegies Zwart et al., "A parallel gravitational N-body kernel" (Sect. 2.1):
 * block selection by the smallest t_i + dt_i, the Hermite predictor for all
 * particles, the softened acceleration / jerk / potential of the active block
 * against all N predicted particles (Eq. Force), the Hermite corrector and
 * the Aarseth time step (Eq. timestep) quantised to powers of two. The
 * paper's j-parallelisation over processors (Sect. 3) becomes an on-chip
 * decomposition: j-tiles staged in shared memory, register-blocked i, and a
 * fixed-order reduction over j-splits.
 *
 * Conventions
 *   - G = 1. Vectors are double[n][3], row-major (x0 y0 z0 x1 ...).
 *   - Host pointers are caller-owned and are only read/written during the call.
 *     "_dev" entry points take device pointers of the context's device and
 *     work on the context's stream; they return before the GPU work ends.
 *   - The library allocates and owns all its device memory (freed by
 *     nb_destroy). A context is not thread-safe; use one per host thread.
 *   - Every call returns an nb_status. NB_ERR_CUDA reports a CUDA runtime
 *     error; device-side conditions (non-finite values, a time step below
 *     dt_min, a device wait that ran past its spin limit) are accumulated in
 *     a device status word and reported by the next call that synchronises
 *     (nb_next_block, nb_force_jerk, nb_step, nb_run, nb_energy, nb_get_state,
 *     nb_sync). nb_last_error() gives a one-line description.
 *   - Precision: NB_PREC_MIXED does the pair arithmetic in FP32 with
 *     double-single (hi + lo) positions and compensated partial sums; the
 *     state, predictor, corrector and energy stay FP64. NB_PREC_FP64 does all
 *     of it in FP64.
 */
#ifndef NBODY_H
#define NBODY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nb_ctx nb_ctx;

typedef enum {
    NB_OK = 0,
    NB_ERR_ARG = -1,           /* bad argument (size, NULL, order) */
    NB_ERR_CUDA = -2,          /* CUDA runtime error, or no usable device */
    NB_ERR_NONFINITE = -3,     /* a force, position or velocity became NaN/inf */
    NB_ERR_DT_UNDERFLOW = -4,  /* a quantised step fell below dt_min */
    NB_ERR_TIMEOUT = -5,       /* a device-side wait exceeded its spin limit */
    NB_ERR_STATE = -6          /* call out of order (e.g. nb_correct before nb_force_jerk) */
} nb_status;

typedef enum { NB_PREC_MIXED = 0, NB_PREC_FP64 = 1 } nb_precision;

typedef struct {
    double eta;           /* accuracy parameter nu of Eq. (timestep); default 0.01 */
    double dt_max;        /* largest step, a power of two <= 2^300; default 1/16 */
    double dt_min;        /* smallest step, >= 2^-300; default 2^-40 (below: NB_ERR_DT_UNDERFLOW) */
    int32_t precision;    /* nb_precision; default NB_PREC_MIXED */
    int32_t autotune;     /* 1: time the kernel variants per active-set size on first use */
    int64_t spin_limit;   /* iteration cap of every device-side wait; default 1<<24 */
    int32_t device;       /* CUDA device ordinal; -1 = the current device */
    int32_t inject;       /* test hook: 1 = the next force launch waits on a barrier that
                             nothing completes, so its spin limit must expire */
} nb_config;

/* Buckets of the block-size histogram: bucket b counts block steps with
 * 2^(b-1) < s <= 2^b (b = 0: s = 1). */
#define NB_SIZE_BUCKETS 32

/* Counters since nb_init (block steps, particle steps sum s, interactions sum s*N). */
typedef struct {
    int64_t block_steps;
    int64_t particle_steps;
    double interactions;
    double t_now;                         /* largest t_i */
    int64_t size_hist[NB_SIZE_BUCKETS];   /* block steps per block-size bucket */
    int64_t loop_slots;                   /* step slots the nb_run loop has run (each slot: the
                                             engine if on, the selection, predictor, force and
                                             corrector kernels; slots past t_end run as no-ops) */
} nb_counters;

/* Full particle state; arrays of length n ([n][3] for vectors), caller-owned. */
typedef struct {
    int64_t n;
    double *m, *x, *v, *a, *k, *t, *dt;
} nb_state_view;

/* Fills *cfg with the defaults listed above. */
void nb_config_default(nb_config *cfg);

/* Creates a context on cfg->device. stream: a cudaStream_t to run on, or NULL
 * for a stream the library creates (non-blocking). cfg NULL = defaults.
 * Errors: NB_ERR_ARG (ctx NULL, bad config), NB_ERR_CUDA (no device). */
nb_status nb_create(nb_ctx **ctx, const nb_config *cfg, void *stream);

/* Frees the context and its device memory. NULL is ignored. */
void nb_destroy(nb_ctx *ctx);

/* One-line description of the last error on this context ("" if none). */
const char *nb_last_error(const nb_ctx *ctx);

/* Loads n particles (m[n], x[n][3], v[n][3], host) with softening eps2 = eps^2
 * (Plummer softening; the paper's Eq. Force has none), sets t_i = 0, computes
 * a and k by a full force pass (s = n) and the first steps
 * dt_i = 2^floor(log2(eta |a|/|k|)) capped at dt_max (Sect. 2.1 is silent on
 * the start; this is the usual Aarseth start with eta_s = eta).
 * Errors: NB_ERR_ARG (n < 1 or n > 2^31-1, eps2 < 0), NB_ERR_NONFINITE,
 * NB_ERR_DT_UNDERFLOW, NB_ERR_CUDA. */
nb_status nb_init(nb_ctx *ctx, int64_t n, const double *m, const double *x, const double *v,
                  double eps2);

/* As nb_init with device pointers (same layouts). */
nb_status nb_init_dev(nb_ctx *ctx, int64_t n, const double *m_dev, const double *x_dev,
                      const double *v_dev, double eps2);

/* Block selection (Sect. 2.1, first bullet): t_next = min_i (t_i + dt_i) and the
 * active list {i : t_i + dt_i == t_next} in ascending i, kept on the device
 * for nb_force_jerk/nb_correct. Writes *t_next and *s (host). */
nb_status nb_next_block(nb_ctx *ctx, double *t_next, int64_t *s);

/* Copies the active list of the last nb_next_block (int32[s], ascending) to host. */
nb_status nb_get_active(nb_ctx *ctx, int32_t *idx);

/* Hermite predictor (Sect. 2.1): every particle j to time t:
 * x_p = x + v d + a d^2/2 + k d^3/6, v_p = v + a d + k d^2/2, d = t - t_j.
 * Writes the predicted j-records used by nb_force_jerk; the state is unchanged. */
nb_status nb_predict(nb_ctx *ctx, double t);

/* Copies the predicted positions and velocities of the last nb_predict (or of the
 * predictor step inside nb_step / nb_run) to host arrays xp[n][3], vp[n][3]
 * (either may be NULL). In mixed precision these are the j-records as the
 * force kernel sees them: hi + lo for positions, the FP32 velocity. */
nb_status nb_get_predicted(nb_ctx *ctx, double *xp, double *vp);

/* Eq. (Force) and its time derivative on the active list idx[s] (host, int32,
 * strictly ascending, each < n) against all n particles as last predicted:
 *   a_i = sum_{j != i} m_j r / (r^2+eps^2)^{3/2},
 *   k_i = sum_{j != i} m_j [ w / (r^2+eps^2)^{3/2} - 3 (r.w) r / (r^2+eps^2)^{5/2} ],
 *   phi_i = - sum_{j != i} m_j / (r^2+eps^2)^{1/2},   r = x_j - x_i, w = v_j - v_i.
 * idx NULL = the active list of the last nb_next_block (s must match it).
 * a, k: double[s][3]; phi: double[s] (host); any of them may be NULL (then that
 * output stays on the device for nb_correct). s = 0 is a no-op.
 * Errors: NB_ERR_ARG (s < 0, s > n, idx not ascending or out of range),
 * NB_ERR_NONFINITE (a result is NaN/inf), NB_ERR_TIMEOUT, NB_ERR_CUDA. */
nb_status nb_force_jerk(nb_ctx *ctx, const int32_t *idx, int64_t s, double *a, double *k,
                        double *phi);

/* As nb_force_jerk with device pointers: idx_dev int32[s] (strictly ascending,
 * each < n, not checked), a_dev/k_dev double[s][3], phi_dev double[s]; any
 * output may be NULL. Asynchronous on the context's stream. */
nb_status nb_force_jerk_dev(nb_ctx *ctx, const int32_t *idx_dev, int64_t s, double *a_dev,
                            double *k_dev, double *phi_dev);

/* The j-parallel block step of Sect. 3 (Flowchart): every rank holds the whole
 * system, sums the forces on the active block over its own share of j, the
 * partial forces are added over the ranks (the paper's MPI_Allreduce; the
 * binding's jparallel module gathers them and adds them in rank order), and
 * every rank corrects identically.
 *
 * nb_j_range: the share [*j_begin, *j_end) of rank `rank` of `world` (whole
 * 256-particle tiles, balanced; the last share ends at n).
 * nb_force_jerk_range / _dev: as nb_force_jerk / nb_force_jerk_dev, with the
 * sums over j in [j_begin, j_end) only (j_begin and j_end multiples of 256,
 * j_end may be n; an empty range gives zeros). idx NULL = the active list of
 * the last nb_next_block. The results are partial sums: nb_correct does not take
 * them (NB_ERR_STATE); add them over the ranks and pass the totals to
 * nb_correct_forces.
 * nb_correct_forces / _dev: nb_correct with the new a[s][3], k[s][3] given by
 * the caller (host / device arrays, in the order of the active list of the last
 * nb_next_block or force call). Same errors as nb_correct. */
nb_status nb_j_range(nb_ctx *ctx, int32_t rank, int32_t world, int64_t *j_begin, int64_t *j_end);
nb_status nb_force_jerk_range(nb_ctx *ctx, const int32_t *idx, int64_t s, int64_t j_begin, int64_t j_end,
                              double *a, double *k, double *phi);
nb_status nb_force_jerk_range_dev(nb_ctx *ctx, const int32_t *idx_dev, int64_t s, int64_t j_begin,
                                  int64_t j_end, double *a_dev, double *k_dev, double *phi_dev);
nb_status nb_correct_forces(nb_ctx *ctx, double t_block, const double *a, const double *k);
nb_status nb_correct_forces_dev(nb_ctx *ctx, double t_block, const double *a_dev, const double *k_dev);

/* Hermite corrector and new steps (Sect. 2.1, Eq. timestep) for the active list
 * of the last nb_force_jerk, whose members must all have t_i + dt_i == t_block
 * (the paper's "dt" argument is read as the block time; each particle's own
 * step is dt_i = t_block - t_i). Uses the forces of that call.
 * Errors: NB_ERR_STATE (no forces pending, or a member not due at t_block),
 * NB_ERR_NONFINITE, NB_ERR_DT_UNDERFLOW, NB_ERR_CUDA. */
nb_status nb_correct(nb_ctx *ctx, double t_block);

/* One block step on the device: select, predict all, force on the block,
 * correct (no host round trip); a small block runs inside the small-block
 * engine (nb_set_engine), as it does in nb_run. */
nb_status nb_step(nb_ctx *ctx);

/* Block steps until the next block time exceeds t_end (t_end must be a multiple
 * of dt_max for every particle to land on it). One CUDA-graph launch: a full
 * selection, then a while node whose body runs block steps on the device with
 * no host round trip. In mixed precision, block steps whose block is small
 * (see nb_set_engine) run inside the small-block engine: one thread-block
 * cluster doing selection, predictor, force and corrector in one kernel, step
 * after step, until a block it does not take; every other block step runs as
 * [selection at the known block time || predictor] -> force -> corrector (the
 * corrector forms the next block time; steps past t_end are no-ops). Same
 * trajectory, bit for bit, as repeated nb_step.
 * One call runs at most 2^22 block steps (then NB_ERR_STATE, "block-step cap"). */
nb_status nb_run(nb_ctx *ctx, double t_end);

/* Timings of nb_run_timed. */
typedef struct {
    double force_ms;              /* summed force-kernel time (blocks the engine does not take) */
    double phase_ms[5];           /* select, predict, force, correct, engine (phases != 0; else only
                                     [2] and [4]) */
    int64_t force_launches;       /* block steps done by the four-kernel step */
    int64_t engine_steps;         /* block steps done by the small-block engine */
    double force_interactions;    /* sum of s N over the force launches */
    double engine_interactions;   /* sum of s N over the engine's steps */
} nb_timing;

/* Same trajectory as nb_run, driven from the host one block step at a time, with
 * CUDA events around every force launch and every engine step (a short,
 * time-bounded wait kernel precedes each start event so that it is processed
 * only once the launch is queued); phases != 0 brackets the select, predict and
 * correct kernels the same way (the select that ends the loop is not counted).
 * out may be NULL. For measurement; slower than nb_run. */
nb_status nb_run_timed(nb_ctx *ctx, double t_end, int32_t phases, nb_timing *out);

/* Small-block engine (mixed precision): the largest block s_max (<= 256) that
 * nb_step / nb_run / nb_run_timed run inside the one-cluster engine kernel
 * instead of the four-kernel step (a block is also left to the four-kernel
 * step when more than 64 of its members fall into one CTA's share of the
 * particles). The paper has the step of Sect. 2.1 only; the engine is the same
 * step with the j-split of Sect. 3 across the cluster's CTAs and the partial
 * forces summed in a fixed order. s_max = 0 switches it off, -1 restores the
 * default: for n <= 4096 the largest s with s n <= 2^19 (at least 16, at most
 * 256); above 4096 particles off (there its steps cost about as much as the
 * four-kernel steps on this GPU). Without a co-schedulable 16- or 8-CTA cluster,
 * or above 1024 particles per CTA (n > 16384 on 16-CTA clusters), there is no
 * engine.
 * Errors: NB_ERR_ARG (s_max out of range, or s_max > 0 in FP64 precision).
 * nb_get_engine: the largest block the engine takes for the loaded system
 * (0 = no engine) and its cluster size; either pointer may be NULL. */
nb_status nb_set_engine(nb_ctx *ctx, int32_t s_max);
nb_status nb_get_engine(nb_ctx *ctx, int32_t *s_max, int32_t *cluster);

/* Kinetic, potential (softened, W = sum m_i phi_i / 2) and total energy of the
 * current state, on the device: K in FP64; the pair terms of W in double-single
 * arithmetic on the FP32 pipe (agrees with FP64 sums to ~1e-15 relative) with
 * FP64 per-particle and fixed-order final sums. Exact only when all t_i are
 * equal (e.g. after nb_run). Any pointer may be NULL. */
nb_status nb_energy(nb_ctx *ctx, double *E, double *K, double *W);

/* Copies the full FP64 state to / from host arrays (view->n must equal the
 * context's n; set_state also needs a consistent t, dt). */
nb_status nb_get_state(nb_ctx *ctx, nb_state_view *view);
nb_status nb_set_state(nb_ctx *ctx, const nb_state_view *view);

/* Counters since nb_init. */
nb_status nb_stats(nb_ctx *ctx, nb_counters *out);

/* Waits for the context's stream and reports pending device-side errors. */
nb_status nb_sync(nb_ctx *ctx);

/* Kernel tuning. nb_autotune times every force-kernel variant and split factor
 * for active-set sizes 1, 2, 4, ..., n on the current predicted state and keeps
 * the fastest per size bucket. nb_set_tuning forces (variant, split) for a
 * bucket (bucket b holds s in (2^(b-1), 2^b]); variant -1 restores the default.
 * split is the j-split factor at the bucket's largest size min(2^b, n); a
 * smaller block of the bucket keeps the same number of work items (i-blocks x
 * splits), so its split grows in proportion.
 * nb_get_tuning reads the table (variant[32], split[32]). */
nb_status nb_autotune(nb_ctx *ctx);
nb_status nb_set_tuning(nb_ctx *ctx, int32_t bucket, int32_t variant, int32_t split);
nb_status nb_get_tuning(nb_ctx *ctx, int32_t *variant, int32_t *split);
/* Number of force-kernel variants of the context's precision and a short name. */
int32_t nb_num_variants(const nb_ctx *ctx);
const char *nb_variant_name(const nb_ctx *ctx, int32_t variant);

/* Largest particle count accepted by nb_force_jerk_static. */
#define NB_STATIC_MAX_N 65536

/* The mixed-precision force evaluation of nb_force_jerk (same arithmetic and
 * kernel) for callers that must not allocate device memory: code inside a host
 * framework that owns the GPU's memory budget through its own pool, plugins
 * running in another application's CUDA context, and latency-critical loops
 * that cannot afford the implicit device synchronisation of cudaMalloc/cudaFree.
 * The paper has no counterpart; this is a deployment variant of Eq. (Force).
 *
 * No context and no allocation: the caller passes device pointers on the
 * current device -- m_dev[n], the predicted state x_dev[n][3], v_dev[n][3]
 * (FP64), the active list idx_dev[s] (int32, strictly ascending, each < n, not
 * checked) and the outputs a_dev[s][3], k_dev[s][3], phi_dev[s] (any output may
 * be NULL) -- and a stream (NULL = the legacy default stream). All scratch lives
 * in one fixed __device__ array of the library (about 11 MiB, held by every GPU
 * that loads the library until exit), so n is limited to NB_STATIC_MAX_N
 * (a larger n returns NB_ERR_ARG); the j-split factor is lowered as needed so
 * that the split partials (s x split entries) fit in 2^16 slots.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make this
 * first call before any stream capture. A cudaDeviceReset between calls is not
 * supported (the kept address would be stale).
 * Every call reuses the same array and leaves its contents behind, so calls
 * that overlap on the GPU (other streams, other host threads) race: serialise
 * them. The call returns after the outputs are written (it synchronises the
 * stream) and reports NB_ERR_NONFINITE, NB_ERR_TIMEOUT or NB_ERR_CUDA. */
nb_status nb_force_jerk_static(int64_t n, const double *m_dev, const double *x_dev, const double *v_dev,
                               double eps2, const int32_t *idx_dev, int64_t s, double *a_dev, double *k_dev,
                               double *phi_dev, void *stream);

/* Perturber lists of binaries (Sect. 3.1). Binary b is the particle pair
 * (pairs[2b], pairs[2b+1]). Star j (not a member) perturbs it when its tidal
 * acceleration across the binary, relative to the binary's internal
 * acceleration, reaches gamma:
 *     2 m_j d^3 / (m_b r_j^3) >= gamma
 * (d the members' separation, m_b their mass, r_j the distance from the
 * binary's centre of mass; the paper's 10^-7 is gamma = 1e-7), evaluated on the
 * context's current positions as (2 m_j)^2 d^6 >= (gamma m_b)^2 r_j^6 in FP64
 * with every operation rounded separately, in a fixed order (the CPU oracle's
 * order: the same decisions bit for bit). Stars j in [j_lo, j_hi) (j_hi < 0:
 * n) are scanned in ascending index and the first nmax perturbers go to
 * lists[b][0..) in that order — the serial code's order, which the paper's
 * parallel code restores by sorting — the rest of the row -1; counts[b] is the
 * number found (it may exceed nmax). Lists of consecutive j-ranges (one per
 * rank of the j-parallel step), concatenated in range order and cut at nmax,
 * are the list of the whole range and their counts add up. nmax in [1,
 * NB_PERT_MAX] (the paper's N_pert = 256). Host arrays: pairs[nbin][2],
 * lists[nbin][nmax], counts[nbin]; synchronous; NB_ERR_ARG for an invalid pair.
 * The _dev form takes device arrays, is asynchronous on the context's stream
 * and marks an invalid pair with counts[b] = -1 and an empty row. */
#define NB_PERT_MAX 4096
nb_status nb_perturbers(nb_ctx *ctx, int32_t nbin, const int32_t *pairs, double gamma, int32_t nmax,
                        int64_t j_lo, int64_t j_hi, int32_t *lists, int32_t *counts);
nb_status nb_perturbers_dev(nb_ctx *ctx, int32_t nbin, const int32_t *pairs_dev, double gamma, int32_t nmax,
                            int64_t j_lo, int64_t j_hi, int32_t *lists_dev, int32_t *counts_dev);

/* Batched ensemble of nc independent systems (Sect. 2.1 applied to each):
 * offsets[nc+1] delimit each system's particles in the concatenated arrays
 * m[N], x[N][3], v[N][3] (host, N = offsets[nc]); eps2[nc] per system, each
 * system at most 2^19 particles (one thread-block cluster works on a system at
 * a time). Each system keeps its own block schedule. Computes the
 * initial forces, first steps and energies (t = 0) on the device. Replaces any
 * previous ensemble of the context (the single-system state is independent). */
nb_status nb_ensemble_init(nb_ctx *ctx, int32_t nc, const int64_t *offsets, const double *m,
                           const double *x, const double *v, const double *eps2);

/* Advances every system of the ensemble to t_end in one persistent launch of
 * thread-block clusters: each cluster takes whole systems from a queue (largest
 * first) and runs their block steps with cluster barriers and distributed
 * shared memory. At most 2^20 block steps per system and call. */
nb_status nb_ensemble_run(nb_ctx *ctx, double t_end);

/* Per-system total energies E[nc] (host), computed at the end of the last
 * nb_ensemble_init (t = 0) or nb_ensemble_run. */
nb_status nb_ensemble_energy(nb_ctx *ctx, double *E);

/* Per-system counters since nb_ensemble_init (host arrays of length nc, any may
 * be NULL): block steps, particle steps (sum of s), interactions (sum of s*N). */
nb_status nb_ensemble_stats(nb_ctx *ctx, int64_t *block_steps, int64_t *particle_steps, double *interactions);

/* Full concatenated state of all systems (view->n = offsets[nc]). */
nb_status nb_ensemble_get_state(nb_ctx *ctx, nb_state_view *view);

/* Launch shape for the loaded ensemble. cluster: CTAs per thread-block cluster,
 * 2, 4, 8 or 16 (0: the default, the largest of 16, 8 and 4 whose co-resident
 * clusters keep at least 90 % of the device's CTA slots busy). split_cap: the
 * largest block (active count s) taken by the j-split, where every CTA of the
 * cluster computes all active particles against its own share of j and the
 * shares' partial forces are summed in rank order; larger blocks are dealt out
 * by i, each CTA taking a share of them against all j (0: the default,
 * min(largest system, 8192); capped at 8192). The partial-force buffer
 * (clusters x cluster x split_cap slots of 64 bytes) grows as needed. Results
 * depend on the shape through the order of the partial sums; one shape gives
 * the same bits on every run. NB_ERR_ARG for a cluster size this device cannot
 * keep resident. */
nb_status nb_ensemble_set_shape(nb_ctx *ctx, int32_t cluster, int32_t split_cap);

/* The current shape: cluster size, co-resident clusters, split cap (any may be NULL). */
nb_status nb_ensemble_get_shape(nb_ctx *ctx, int32_t *cluster, int32_t *nclusters, int32_t *split_cap);

/* Autotuner of the ensemble launch: advances the loaded ensemble by
 * t_probe (<= 0: the configuration's dt_max) under every cluster size of {16,
 * 8, 4} that the device keeps resident and every split cap of {min(largest
 * system, 8192), 4096, 2048, 1024} not above the first, timing each probe with
 * CUDA events and restoring the state after it; keeps the fastest shape (a
 * probe that ends with a status error does not count). best_ms (may be NULL)
 * receives the fastest probe's time. The ensemble's state afterwards is
 * bitwise the state before the call; it allocates a device copy of that state
 * (about 13 doubles and 13 float pairs per particle) for the duration. */
nb_status nb_ensemble_autotune(nb_ctx *ctx, double t_probe, float *best_ms);

#ifdef __cplusplus
}
#endif
#endif
