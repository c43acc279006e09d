// Internal declarations shared by the translation units of libnbody.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nbody.h"

namespace nb {

// ---------------------------------------------------------------- constants

constexpr int kThreads = 256;        // threads per CTA of the force kernels
constexpr int kJT = 256;             // j-records per shared-memory tile
constexpr int kStages = 3;           // tiles in flight per CTA
constexpr int kBuckets = 32;         // active-set size buckets (bucket b: s in (2^(b-1), 2^b])
constexpr int kPartStride = 8;       // doubles per (i, split) partial: ax ay az kx ky kz phi pad
constexpr double kPadPos = 1e18;     // position of the far-away, massless records padding j to whole tiles

// device status bits (accumulated with atomicOr, read at sync points)
constexpr int kStNonfinite = 1;
constexpr int kStUnderflow = 2;
constexpr int kStTimeout = 4;
constexpr int kStState = 8;
constexpr int kStSteps = 16;         // block-step cap reached inside nb_run

// ------------------------------------------------------------- force kernels

// Mixed-precision j-records, two particles per 80-byte record (j = 2p, 2p+1),
// interleaved so that every float4 holds two (j = 2p, j = 2p+1) pairs of one
// quantity -- the operand layout of the packed f32x2 instructions:
//   q[0] = (x_hi, x_hi', y_hi, y_hi')   q[1] = (z_hi, z_hi', m, m')
//   q[2] = (x_lo, x_lo', y_lo, y_lo')   q[3] = (z_lo, z_lo', vx, vx')
//   q[4] = (vy, vy', vz, vz')
// with x_hi = fl32(x), x_lo = fl32(x - x_hi) (double-single position), FP32
// velocity and mass. Arrays hold n_pad / 2 records.
struct JPair {
    float4 q[5];
};

struct JRecs {
    JPair *p;
};

struct Tuning {
    int32_t variant[kBuckets];
    int32_t split[kBuckets];
};

// Parameters of one force evaluation (both precisions).
// State arrays ([3][np] vectors, [np] scalars) for correct_group.
struct HState {
    double *x, *v, *a, *k, *t, *dt, *tn;
    float2 *x2, *v2, *a2, *k2;   // double-single copies (x2 == nullptr: none kept)
    int64_t np;
};

struct ForceArgs {
    int64_t n;            // particles
    int64_t n_tiles;      // ceil(n / kJT); j arrays are padded to n_tiles * kJT
    int64_t tile_lo;      // the sums run over j in tiles [tile_lo, tile_hi) only (all: 0, n_tiles);
    int64_t tile_hi;      // a sub-range gives one rank's partial forces of the j-parallel step
    JRecs j;              // mixed records
    const double *xp;     // FP64 predicted positions [3][n_pad]
    const double *vp;     // FP64 predicted velocities [3][n_pad]
    const double *m;      // masses [n_pad]
    float eps2f;
    double eps2;
    const int32_t *idx;   // active list (ascending), length *s
    int64_t idx_cap;      // readable entries of idx (>= *s): the kernel reads ahead before *s arrives
    const int64_t *s;     // active count (device)
    int64_t s_host;       // >= 0: the active count, given at launch (s is then not read)
    int32_t *idx_copy;    // non-null: the kernel copies idx[0 .. s) here and s to *s_copy
    int64_t *s_copy;      //   (a caller's device list becomes the context's without a separate launch)
    double *out_a;        // non-null: the final sums also in the caller's layouts a[s][3],
    double *out_k;        //   k[s][3], phi[s] (any may be null), with non-finite results
    double *out_phi;      //   flagged, so no separate reduction launch is needed
    double *part;         // split partials [s][split][8] (mixed: float2 (hi, lo) pairs)
    int64_t part_cap;     // capacity of part in 8-byte words
    double *fin;          // final sums [s][8]: ax ay az kx ky kz phi pad
    int32_t *tickets;     // per i-block arrival counters (zero between launches)
    int32_t *split_used;  // written by the kernel: split factor of this launch
    const Tuning *tune;   // device tuning table
    int32_t force_variant;  // >= 0: ignore the table (autotuner, tests)
    int32_t force_split;
    int32_t *status;
    int64_t spin_limit;
    int32_t inject;       // test hook (see nb_config.inject)
};

// Perturber lists of binaries (nb_perturb.cu; Sect. 3.1).
struct PertArgs {
    int64_t n, np;          // particles, stride of the [3][np] position array
    const double *m, *x;    // masses, positions [3][np]
    int32_t nbin;
    const int32_t *pairs;   // [nbin][2] member indices
    double gamma;
    int32_t nmax;
    int64_t j_lo, j_hi;     // stars scanned: [j_lo, j_hi)
    int32_t *lists;         // [nbin][nmax], -1 past the count
    int32_t *counts;        // [nbin] perturbers found (may exceed nmax); -1 for an invalid pair
};
cudaError_t launch_perturbers(const PertArgs &p, cudaStream_t st);

// Variant catalogue. Mixed: 0..kMixedVariants-1; FP64: 0..kF64Variants-1.
constexpr int kMixedVariants = 7;
constexpr int kMixedFallbackId = 4;   // tiled, one particle per thread: takes any size
constexpr int kShareVariantId = 6;    // resident j-share in 8-CTA clusters
constexpr int kF64Variants = 2;
int mixed_variant_I(int v);           // i-particles per work item
const char *mixed_variant_name(int v);
int f64_variant_I(int v);
const char *f64_variant_name(int v);

// Persistent launches: grid = fixed CTA count, work items derived from *s.
cudaError_t launch_force_mixed(const ForceArgs &a, int grid, cudaStream_t st);
cudaError_t launch_force_f64(const ForceArgs &a, int grid, cudaStream_t st);
int force_mixed_ctas_per_sm();
// Persistent grid of the mixed force kernel for n_tiles tiles of j-records (the
// resident cluster grid where the resident-share variant can run): pass it to
// launch_force_mixed, which launches clusters in that case.
int force_mixed_grid(int num_sms, int64_t n_tiles);
// Whether the resident-share variant (6) can take a j range of n_tiles tiles.
bool mixed_share_fits(int64_t n_tiles);
int force_f64_ctas_per_sm();
size_t force_mixed_smem_bytes();

// One-wave (or four-wave, for long items) split factor for nib i-blocks.
int64_t wave_split(int64_t nib, int64_t n_tiles, int64_t resident);
// Default tuning (variant, split) for an active count s.
void default_tuning(int precision, int64_t n, int64_t s, int num_sms, int ctas_per_sm, int *variant,
                    int *split);

// ------------------------------------------------------------ step kernels

struct StepArgs {
    int64_t n, n_pad;
    double *m, *x, *v, *a, *k, *t, *dt;   // state, vectors [3][n_pad]
    double *tn;                           // t + dt per particle (the block-selection key)
    float2 *x2, *v2, *a2, *k2;            // double-single copies of x, v, a, k [3][n_pad]
    JRecs j;                              // mixed records (written by predict)
    double *xp, *vp;                      // FP64 predicted records [3][n_pad]
    int precision;
    double eps2;
    double eta, dt_max, dt_min;
    int32_t *idx;                         // active list
    int64_t *s;                           // active count
    double *t_next;                       // block time
    double *t_end;                        // nb_run target
    // nb_run loop: the next block time is formed while a block is processed.
    // The selection reads this block's time from *t_known and writes the
    // smallest key above it to *t_form; the corrector lowers *t_form by every
    // new key (atomic minimum on the bit patterns). Keys of inactive particles
    // do not change, so *t_form ends as the smallest key of all: the next
    // block's *t_known. Consecutive steps swap the two slots.
    double *t_known;
    double *t_form;
    const double *fin;                    // final force sums [s][8]
    int32_t *status;
    int64_t *counters;                    // [0] block steps, [1] particle steps, [2] max block steps,
                                          // [3 + b] block-size histogram, [3 + NB_SIZE_BUCKETS] loop slots run
    double *interactions;                 // sum s*n
};

// predictor to *t_dev (non-null; with skip_past also *t_dev <= *t_end, else no-op) or t_host;
// skip_empty: no-op when the active count *a.s is 0 (the engine did the step)
cudaError_t launch_predict(const StepArgs &a, const double *t_dev, double t_host, bool skip_past, cudaStream_t st,
                           bool skip_empty = false);
// Selection. SEL_FULL: the smallest key is the block time. SEL_KNOWN (nb_run
// loop body): the block time is *t_known; also writes *t_form and, when the
// block is not to be done (past *t_end, an error, the step cap), s = 0.
// set_cond: SEL_FULL sets the while-node condition to "the first block is due"
// and writes the block time to *t_known; SEL_KNOWN sets it to "this block is done".
enum SelMode { SEL_FULL = 0, SEL_KNOWN = 1 };
cudaError_t launch_select(const StepArgs &a, SelMode mode, unsigned long long cond, bool set_cond, cudaStream_t st);
// corrector; lower_form: atomic minimum of the new keys into *t_form;
// after_force: launched with a programmatic dependency on the force kernel
// launched just before it on the stream (its first loads overlap that kernel)
cudaError_t launch_correct(const StepArgs &a, bool check_due, bool lower_form, bool after_force, cudaStream_t st);
cudaError_t launch_init_steps(const StepArgs &a, cudaStream_t st);
cudaError_t launch_reduce_out(const double *fin, const int64_t *s, int64_t s_host, double *a, double *k,
                              double *phi, int32_t *status, cudaStream_t st);
cudaError_t launch_tnext(const StepArgs &a, cudaStream_t st);
cudaError_t launch_state_to_ds(const StepArgs &a, cudaStream_t st);
cudaError_t launch_aos_to_soa(const double *src, double *dst, int64_t n, int64_t n_pad, cudaStream_t st);
cudaError_t launch_soa_to_aos(const double *src, double *dst, int64_t n, int64_t n_pad, cudaStream_t st);
cudaError_t launch_records_to_aos(const StepArgs &a, double *xp_aos, double *vp_aos, cudaStream_t st);
cudaError_t launch_fill_iota(int32_t *idx, int64_t n, cudaStream_t st);
// copies the device list src[s] to dst and writes s to *s_dev (one launch)
cudaError_t launch_set_active(const int32_t *src, int32_t *dst, int64_t s, int64_t *s_dev, cudaStream_t st);
cudaError_t launch_pad_records(const StepArgs &a, cudaStream_t st);
// caller's forces a[s][3], k[s][3] into the final-sum layout fin[s][8]
cudaError_t launch_forces_in(const double *a, const double *k, int64_t s, double *fin, cudaStream_t st);
// energy: writes K, W to out[0], out[1] (fixed-order sums)
cudaError_t launch_energy(const StepArgs &a, double *scratch, int scratch_ctas, double *out,
                          cudaStream_t st);
cudaError_t launch_check_active(const int32_t *idx, int64_t s, int64_t n, int32_t *status,
                                cudaStream_t st);
cudaError_t launch_check_due(const StepArgs &a, double t_block, cudaStream_t st);
cudaError_t launch_delay(uint64_t ns, cudaStream_t st);

// ------------------------------------------------------- small-block engine
// One thread-block cluster runs consecutive block steps whose blocks are small
// (select, predict, force, correct inside one kernel; nb_engine.cu).
constexpr int kEngMaxS = 256;             // largest block the engine takes
constexpr int kEngCap = 16;               // most members of one CTA's chunk in a block it takes
constexpr int64_t kEngMaxChunk = 1024;    // particles per CTA (their state and pair records sit in shared memory)

struct EngineArgs {
    StepArgs S;
    const double *t_in;    // block time of the first step
    double *t_out;         // at exit: the block time of the first block not done
    int64_t *s_clear;      // non-null: set to 0 when at least one step was done
    float eps2f;
    int64_t chunk;         // particles per CTA, a multiple of 16
    int32_t s_max;         // largest block taken (<= kEngMaxS)
    int32_t check_end;     // stop before a block past *S.t_end
    int64_t max_steps;     // steps of this launch (the call's cap in S.counters applies too)
};
int engine_cluster();                          // CTAs per cluster on this device, 0 = no engine
int64_t engine_chunk(int64_t n_pad, int C);    // particles per CTA
size_t engine_smem_bytes(int64_t chunk);
cudaError_t launch_engine(const EngineArgs &e, int C, cudaStream_t st);

}  // namespace nb
