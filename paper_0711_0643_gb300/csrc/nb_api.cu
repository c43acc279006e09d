// C ABI of libnbody.so: context, device memory, the block-step engine and the
// kernel tuner. See include/nbody.h for the contract of every entry point.
//
// Engine: nb_run builds (once per context) a CUDA graph
//     select -> WHILE( U x ( [engine] -> [select at the known time || predict] -> force -> correct ) )
// where each selection sets the while-node condition on the device (this block
// is due by t_end, no error) and the corrector forms the next block time while
// it corrects (see build_run_graph). The small-block engine (nb_engine.cu, mixed
// precision) runs every block step whose block is small inside one cluster
// launch and stops at the first block it does not take, which the four kernels
// after it then do. One graph launch integrates to t_end with no host round trip
// per block step; the force kernel sizes its work from the active count it reads
// on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "nb_internal.cuh"

using namespace nb;

struct nb_ensemble;
namespace nb {
void ensemble_free(nb_ensemble *e);
}

struct nb_ctx {
    nb_config cfg{};
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    int64_t n = 0, n_pad = 0, n_tiles = 0;
    double eps2 = 0.0;

    // state [3][n_pad] for vectors
    double *m = nullptr, *x = nullptr, *v = nullptr, *a = nullptr, *k = nullptr, *t = nullptr, *dt = nullptr;
    JRecs j{};
    double *xp = nullptr, *vp = nullptr;
    double *stage = nullptr;      // [3 n] staging for layout changes
    int32_t *idx = nullptr;
    int64_t *s = nullptr;
    double *t_next = nullptr, *t_end = nullptr;
    double *t_slot = nullptr;     // [2] block times of the nb_run loop (StepArgs::t_known, t_form)
    double *part = nullptr;
    int64_t part_cap = 0;
    double *fin = nullptr;          // final force sums [n_pad][8]
    int32_t *tickets = nullptr;     // per i-block arrival counters
    double *tn = nullptr;           // t + dt
    float2 *x2 = nullptr, *v2 = nullptr, *a2 = nullptr, *k2 = nullptr;   // double-single state copies
    int32_t *split_used = nullptr;
    Tuning *tune_dev = nullptr;
    Tuning tune{};
    int32_t *status = nullptr;
    int64_t *counters = nullptr;  // [0] block steps [1] particle steps [2] cap
    double *interactions = nullptr;
    double *en_scratch = nullptr;
    int en_ctas = 0;
    double *en_out = nullptr;
    double *out_a = nullptr, *out_k = nullptr, *out_phi = nullptr;

    bool have_state = false;
    bool forces_pending = false;
    int64_t block_s = -1;          // s of the last selection / force call
    bool tuned = false;

    cudaGraphExec_t run_exec = nullptr;
    std::vector<cudaEvent_t> ev;   // timing events for nb_run_timed

    std::string err;
    int inject_pending = 0;
    nb_ensemble *ens = nullptr;   // batched ensemble state (nb_ensemble.cu)

    // small-block engine (mixed precision): cluster size, particles per CTA, the
    // largest block it takes (0 = off; -1 = the default for n); t_eng is the
    // block time it leaves behind in host-driven steps
    int eng_C = 0;
    int64_t eng_chunk = 0;
    int32_t eng_smax = -1;
    double *t_eng = nullptr;
};

// Accessors used by the ensemble translation unit.
nb_ensemble *nb_ctx_ensemble(nb_ctx *ctx) { return ctx->ens; }
void nb_ctx_set_ensemble(nb_ctx *ctx, nb_ensemble *e)
{
    if (ctx->ens && ctx->ens != e) {
        cudaStreamSynchronize(ctx->stream);
        nb::ensemble_free(ctx->ens);
    }
    ctx->ens = e;
}
cudaStream_t nb_ctx_stream(nb_ctx *ctx) { return ctx->stream; }
const nb_config *nb_ctx_config(nb_ctx *ctx) { return &ctx->cfg; }
nb_status nb_ctx_fail(nb_ctx *ctx, nb_status st, const char *msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

namespace {

constexpr int64_t kMaxRunSteps = int64_t(1) << 22;   // block steps per nb_run call
constexpr int kRunUnroll = 16;                         // block steps per pass of the nb_run while node
constexpr int kRunUnrollEngine = 4;                    // the same with the engine (each runs many steps)
constexpr int64_t kEngDefaultMaxN = 4096;              // the engine is on by default up to this many particles
static_assert(kRunUnroll % 2 == 0 && kRunUnrollEngine % 2 == 0,
              "the loop's steps alternate two block-time slots");

nb_status fail(nb_ctx *c, nb_status st, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

#define CK(call)                                                                                       \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

void dfree(void *p)
{
    if (p) cudaFree(p);
}

StepArgs step_args(nb_ctx *c)
{
    StepArgs A{};
    A.n = c->n;
    A.n_pad = c->n_pad;
    A.m = c->m; A.x = c->x; A.v = c->v; A.a = c->a; A.k = c->k; A.t = c->t; A.dt = c->dt;
    A.tn = c->tn;
    A.x2 = c->x2; A.v2 = c->v2; A.a2 = c->a2; A.k2 = c->k2;
    A.j = c->j;
    A.xp = c->xp; A.vp = c->vp;
    A.precision = c->cfg.precision;
    A.eps2 = c->eps2;
    A.eta = c->cfg.eta; A.dt_max = c->cfg.dt_max; A.dt_min = c->cfg.dt_min;
    A.idx = c->idx; A.s = c->s; A.t_next = c->t_next; A.t_end = c->t_end;
    A.t_known = c->t_slot; A.t_form = c->t_slot + 1;
    A.fin = c->fin;
    A.status = c->status; A.counters = c->counters; A.interactions = c->interactions;
    return A;
}

ForceArgs force_args(nb_ctx *c, int variant = -1, int split = 0)
{
    ForceArgs F{};
    F.n = c->n;
    F.n_tiles = c->n_tiles;
    F.tile_lo = 0;
    F.tile_hi = c->n_tiles;
    F.j = c->j;
    F.xp = c->xp; F.vp = c->vp; F.m = c->m;
    F.eps2f = (float)c->eps2;
    F.eps2 = c->eps2;
    F.idx = c->idx;
    F.idx_cap = c->n_pad;
    F.s = c->s;
    F.s_host = -1;
    F.part = c->part;
    F.part_cap = c->part_cap;
    F.fin = c->fin;
    F.tickets = c->tickets;
    F.split_used = c->split_used;
    F.tune = c->tune_dev;
    F.force_variant = variant;
    F.force_split = split;
    F.status = c->status;
    F.spin_limit = c->cfg.spin_limit;
    F.inject = 0;
    return F;
}

int force_grid(nb_ctx *c)
{
    return c->cfg.precision == NB_PREC_FP64 ? c->num_sms * force_f64_ctas_per_sm() : force_mixed_grid(c->num_sms, c->n_tiles);
}

cudaError_t launch_force(nb_ctx *c, const ForceArgs &F)
{
    return c->cfg.precision == NB_PREC_FP64 ? launch_force_f64(F, force_grid(c), c->stream)
                                            : launch_force_mixed(F, force_grid(c), c->stream);
}

// force launch honouring the one-shot injection hook
cudaError_t launch_force_ctx(nb_ctx *c)
{
    ForceArgs F = force_args(c);
    if (c->inject_pending) {
        F.inject = 1;
        c->inject_pending = 0;
    }
    return launch_force(c, F);
}

// The engine's default largest block: its force phase runs on the cluster's
// SMs only, so it takes blocks whose s N is small (2^19 pair evaluations: the
// force phase then takes a few microseconds, below the full path's per-step
// overhead). Above 4096 particles it is off by default: measured on this GPU, its
// steps (~16 us at N = 16384, mostly the FP64 corrector chain and the barrier-
// separated phases on 16 SMs) plus a launch each time a large block interrupts
// it cost as much as the four-kernel steps (Plummer N = 16384 to t = 1: 686 vs
// 674 ms), while at N = 1024 it saves a fifth (58 vs 75 ms).
int32_t default_engine_smax(int64_t n)
{
    if (n > kEngDefaultMaxN) return 0;
    int64_t s = (int64_t(1) << 19) / std::max<int64_t>(n, 1);
    s = std::max<int64_t>(16, std::min<int64_t>(s, kEngMaxS));
    return (int32_t)s;
}

// Engine shape for the loaded system: mixed precision, a co-schedulable
// cluster, and each CTA's chunk of pair records within its shared memory.
void engine_setup(nb_ctx *c)
{
    c->eng_C = 0;
    c->eng_chunk = 0;
    if (c->cfg.precision != NB_PREC_MIXED || c->n < 1) return;
    const int C = engine_cluster();
    if (C < 1) return;
    const int64_t chunk = engine_chunk(c->n_pad, C);
    if (chunk < 16 || chunk > kEngMaxChunk) return;
    c->eng_C = C;
    c->eng_chunk = chunk;
}

bool engine_on(const nb_ctx *c)
{
    const int32_t smax = c->eng_smax < 0 ? default_engine_smax(c->n) : c->eng_smax;
    return c->eng_C > 0 && smax > 0;
}

EngineArgs engine_args(nb_ctx *c, const StepArgs &A, const double *t_in, double *t_out, int64_t *s_clear,
                       bool check_end, int64_t max_steps)
{
    EngineArgs e{};
    e.S = A;
    e.t_in = t_in;
    e.t_out = t_out;
    e.s_clear = s_clear;
    e.eps2f = (float)c->eps2;
    e.chunk = c->eng_chunk;
    e.s_max = c->eng_smax < 0 ? default_engine_smax(c->n) : c->eng_smax;
    e.check_end = check_end ? 1 : 0;
    e.max_steps = max_steps;
    return e;
}

void free_system(nb_ctx *c)
{
    if (c->run_exec) {
        cudaGraphExecDestroy(c->run_exec);
        c->run_exec = nullptr;
    }
    void *ptrs[] = {c->m, c->x, c->v, c->a, c->k, c->t, c->dt, c->j.p, c->xp, c->vp,
                    c->stage, c->idx, c->part, c->fin, c->tickets, c->tn, c->x2, c->v2, c->a2, c->k2, c->en_scratch,
                    c->out_a, c->out_k, c->out_phi};
    for (void *p : ptrs) dfree(p);
    c->m = c->x = c->v = c->a = c->k = c->t = c->dt = nullptr;
    c->j = JRecs{};
    c->xp = c->vp = c->stage = nullptr;
    c->idx = nullptr;
    c->part = nullptr;
    c->fin = nullptr;
    c->tickets = nullptr;
    c->tn = nullptr;
    c->x2 = c->v2 = c->a2 = c->k2 = nullptr;
    c->en_scratch = nullptr;
    c->out_a = c->out_k = c->out_phi = nullptr;
    c->n = c->n_pad = c->n_tiles = 0;
    c->have_state = false;
    c->forces_pending = false;
    c->tuned = false;
}

nb_status alloc_system(nb_ctx *ctx, int64_t n)
{
    free_system(ctx);
    ctx->n = n;
    ctx->n_tiles = (n + kJT - 1) / kJT;
    ctx->n_pad = ctx->n_tiles * kJT;
    const int64_t np = ctx->n_pad;
    CK(dalloc(&ctx->m, np));
    CK(dalloc(&ctx->x, 3 * np));
    CK(dalloc(&ctx->v, 3 * np));
    CK(dalloc(&ctx->a, 3 * np));
    CK(dalloc(&ctx->k, 3 * np));
    CK(dalloc(&ctx->t, np));
    CK(dalloc(&ctx->dt, np));
    CK(dalloc(&ctx->j.p, np / 2));
    CK(dalloc(&ctx->xp, 3 * np));
    CK(dalloc(&ctx->vp, 3 * np));
    CK(dalloc(&ctx->stage, 3 * np));
    CK(dalloc(&ctx->idx, np));
    // partials: room for s * split * 8 doubles; at least 4 splits of a full block
    ctx->part_cap = std::max<int64_t>(4 * np * kPartStride, int64_t(1) << 23);
    CK(dalloc(&ctx->part, ctx->part_cap));
    CK(dalloc(&ctx->fin, kPartStride * np));
    CK(dalloc(&ctx->tickets, np + 1));
    CK(dalloc(&ctx->tn, np));
    CK(dalloc(&ctx->x2, 3 * np));
    CK(dalloc(&ctx->v2, 3 * np));
    CK(dalloc(&ctx->a2, 3 * np));
    CK(dalloc(&ctx->k2, 3 * np));
    CK(cudaMemsetAsync(ctx->tickets, 0, (np + 1) * sizeof(int32_t), ctx->stream));
    ctx->en_ctas = (int)((n + 127) / 128) * 8;   // i-tiles of 128 x up to 8 j-splits
    CK(dalloc(&ctx->en_scratch, 2 * (size_t)ctx->en_ctas));
    CK(dalloc(&ctx->out_a, 3 * np));
    CK(dalloc(&ctx->out_k, 3 * np));
    CK(dalloc(&ctx->out_phi, np));
    CK(cudaMemsetAsync(ctx->a, 0, 3 * np * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(ctx->k, 0, 3 * np * sizeof(double), ctx->stream));
    CK(cudaMemsetAsync(ctx->t, 0, np * sizeof(double), ctx->stream));
    return NB_OK;
}

void fill_default_tuning(nb_ctx *c)
{
    for (int b = 0; b < kBuckets; ++b) {
        int64_t s = int64_t(1) << b;
        if (s > c->n) s = c->n;
        int v, S;
        default_tuning(c->cfg.precision, c->n, s, force_grid(c), 1, &v, &S);
        c->tune.variant[b] = v;
        c->tune.split[b] = S;
    }
}

nb_status upload_tuning(nb_ctx *ctx)
{
    CK(cudaMemcpyAsync(ctx->tune_dev, &ctx->tune, sizeof(Tuning), cudaMemcpyHostToDevice, ctx->stream));
    return NB_OK;
}

// Reads and clears the device status word; maps it to an nb_status.
nb_status sync_status(nb_ctx *ctx)
{
    CK(cudaStreamSynchronize(ctx->stream));
    int32_t st = 0;
    CK(cudaMemcpy(&st, ctx->status, sizeof st, cudaMemcpyDeviceToHost));
    if (st == 0) return NB_OK;
    CK(cudaMemset(ctx->status, 0, sizeof(int32_t)));
    if ((st & kStTimeout) && ctx->tickets)   // an aborted force launch may leave tickets armed
        CK(cudaMemset(ctx->tickets, 0, (ctx->n_pad + 1) * sizeof(int32_t)));
    if (st & kStTimeout) return fail(ctx, NB_ERR_TIMEOUT, "a device-side wait exceeded the spin limit");
    if (st & kStNonfinite) return fail(ctx, NB_ERR_NONFINITE, "non-finite force, position or velocity");
    if (st & kStUnderflow) return fail(ctx, NB_ERR_DT_UNDERFLOW, "time step below dt_min");
    if (st & kStState) return fail(ctx, NB_ERR_STATE, "active particle not due at the block time");
    if (st & kStSteps) return fail(ctx, NB_ERR_STATE, "block-step cap reached");
    return fail(ctx, NB_ERR_CUDA, "unknown device status %d", st);
}

// Allocation for n particles; an unchanged n keeps the buffers, the tuning
// table and (for an unchanged eps2) the captured run graph.
nb_status prepare_system(nb_ctx *ctx, int64_t n, double eps2)
{
    if (n != ctx->n || !ctx->m) {
        nb_status st = alloc_system(ctx, n);
        if (st != NB_OK) return st;
    } else {
        CK(cudaMemsetAsync(ctx->a, 0, 3 * ctx->n_pad * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(ctx->k, 0, 3 * ctx->n_pad * sizeof(double), ctx->stream));
        CK(cudaMemsetAsync(ctx->t, 0, ctx->n_pad * sizeof(double), ctx->stream));
        if (ctx->run_exec && eps2 != ctx->eps2) {   // eps2 is baked into the captured launches
            cudaGraphExecDestroy(ctx->run_exec);
            ctx->run_exec = nullptr;
        }
    }
    ctx->eps2 = eps2;
    return NB_OK;
}

// Common tail of nb_init / nb_init_dev: state x, v, m loaded (SoA), a = k = 0.
nb_status init_forces(nb_ctx *ctx)
{
    engine_setup(ctx);
    StepArgs A = step_args(ctx);
    CK(launch_pad_records(A, ctx->stream));
    CK(launch_state_to_ds(A, ctx->stream));
    CK(launch_predict(A, nullptr, 0.0, false, ctx->stream));    // t = 0, a = k = 0: records = positions
    CK(launch_fill_iota(ctx->idx, ctx->n, ctx->stream));
    CK(cudaMemcpyAsync(ctx->s, &ctx->n, sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    if (!ctx->tuned) fill_default_tuning(ctx);
    nb_status rs = upload_tuning(ctx);
    if (rs != NB_OK) return rs;
    CK(launch_force_ctx(ctx));
    CK(launch_init_steps(A, ctx->stream));
    CK(cudaMemsetAsync(ctx->counters, 0, 2 * sizeof(int64_t), ctx->stream));
    CK(cudaMemsetAsync(ctx->counters + 3, 0, (NB_SIZE_BUCKETS + 1) * sizeof(int64_t), ctx->stream));
    CK(cudaMemsetAsync(ctx->interactions, 0, sizeof(double), ctx->stream));
    ctx->have_state = true;
    ctx->forces_pending = false;
    ctx->block_s = -1;
    nb_status st = sync_status(ctx);
    if (st == NB_OK && ctx->cfg.autotune && !ctx->tuned) st = nb_autotune(ctx);
    return st;
}

nb_status check_ctx(nb_ctx *ctx, bool need_state)
{
    if (!ctx) return NB_ERR_ARG;
    ctx->err.clear();
    if (need_state && !ctx->have_state) return fail(ctx, NB_ERR_STATE, "no particles loaded (call nb_init)");
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return NB_OK;
}

// The nb_run graph: a full selection (block time = smallest key; sets the
// condition and the candidate slot), then a while node whose body is kRunUnroll
// block steps of
//     [selection of the known block time || predictor to it] -> force -> corrector.
// The next block time is formed during the block (StepArgs::t_form), so the
// selection and the predictor of a block depend only on the previous corrector
// and run side by side. Each selection sets the condition to "this block is
// done"; a step that finds no block due runs as no-ops (s = 0), and so do the
// steps after it in the body. Going round the while node costs ~5 us on this
// GPU against ~1 us between two kernels of the body, hence the unrolling.
// The corrector stays a kernel of its own: its FP64 work must spread over many
// SMs (an FP64 warp instruction holds an SM sub-partition's FP64 unit for ~70
// clocks), which the CTAs that finish the force sums of an i-block cannot do.
nb_status build_run_graph(nb_ctx *ctx)
{
    if (ctx->run_exec) return NB_OK;
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    StepArgs A = step_args(ctx);
    // 1) first selection (sets the condition)
    CK(cudaStreamBeginCaptureToGraph(ctx->stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    cudaError_t e1 = launch_select(A, SEL_FULL, (unsigned long long)h, true, ctx->stream);
    cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ctx, NB_ERR_CUDA, "graph capture (select): %s / %s", cudaGetErrorString(e1),
                    cudaGetErrorString(e2));
    }
    size_t nn = 0;
    CK(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CK(cudaGraphGetNodes(g, nodes.data(), &nn));
    // 2) while node
    cudaGraphNodeParams cp{};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t wn;
    CK(cudaGraphAddNode(&wn, g, nodes.data(), nullptr, nn, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // 3) body: the predictor forks onto a side stream and joins before the force kernel
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    cudaError_t eb = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
    if (eb == cudaSuccess) eb = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (eb == cudaSuccess) eb = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    cudaError_t ee = cudaSuccess;
    if (eb == cudaSuccess) {
        eb = cudaStreamBeginCaptureToGraph(ctx->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
        if (eb == cudaSuccess) {
            const bool eng = engine_on(ctx);
            const int unroll = eng ? kRunUnrollEngine : kRunUnroll;
            for (int u = 0; u < unroll && eb == cudaSuccess; ++u) {
                StepArgs Au = A;   // step u reads slot u % 2 and forms slot (u + 1) % 2
                Au.t_known = ctx->t_slot + (u & 1);
                Au.t_form = ctx->t_slot + ((u + 1) & 1);
                if (eng) {
                    // the small blocks from this block time on; the engine leaves the time of
                    // the first block it does not take in the same slot
                    eb = launch_engine(engine_args(ctx, Au, Au.t_known, Au.t_known, nullptr, true, kMaxRunSteps),
                                       ctx->eng_C, ctx->stream);
                }
                if (eb == cudaSuccess) eb = cudaEventRecord(fork, ctx->stream);
                if (eb == cudaSuccess) eb = cudaStreamWaitEvent(side, fork, 0);
                if (eb == cudaSuccess) eb = launch_predict(Au, Au.t_known, 0.0, true, side);
                if (eb == cudaSuccess) eb = cudaEventRecord(join, side);
                if (eb == cudaSuccess) eb = launch_select(Au, SEL_KNOWN, (unsigned long long)h, true, ctx->stream);
                if (eb == cudaSuccess) eb = cudaStreamWaitEvent(ctx->stream, join, 0);
                if (eb == cudaSuccess) eb = launch_force(ctx, force_args(ctx));
                if (eb == cudaSuccess) eb = launch_correct(Au, false, true, true, ctx->stream);
            }
            cudaGraph_t body_out = body;
            ee = cudaStreamEndCapture(ctx->stream, &body_out);
        }
    }
    if (join) cudaEventDestroy(join);
    if (fork) cudaEventDestroy(fork);
    if (side) cudaStreamDestroy(side);
    if (eb != cudaSuccess || ee != cudaSuccess) {
        cudaGraphDestroy(g);
        return fail(ctx, NB_ERR_CUDA, "graph capture (body): %s / %s", cudaGetErrorString(eb),
                    cudaGetErrorString(ee));
    }
    cudaError_t ei = cudaGraphInstantiate(&ctx->run_exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        ctx->run_exec = nullptr;
        return fail(ctx, NB_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ei));
    }
    return NB_OK;
}

nb_status set_t_end(nb_ctx *ctx, double t_end)
{
    CK(cudaMemcpyAsync(ctx->t_end, &t_end, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    return NB_OK;
}

}  // namespace

// ============================================================== C ABI

extern "C" {

void nb_config_default(nb_config *cfg)
{
    if (!cfg) return;
    cfg->eta = 0.01;
    cfg->dt_max = 1.0 / 16.0;
    cfg->dt_min = std::ldexp(1.0, -40);
    cfg->precision = NB_PREC_MIXED;
    cfg->autotune = 0;
    cfg->spin_limit = int64_t(1) << 24;
    cfg->device = -1;
    cfg->inject = 0;
}

nb_status nb_create(nb_ctx **out, const nb_config *cfg, void *stream)
{
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    nb_ctx *ctx = new nb_ctx();
    if (cfg)
        ctx->cfg = *cfg;
    else
        nb_config_default(&ctx->cfg);
    const nb_config &c = ctx->cfg;
    auto bad = [&](const char *why) {
        delete ctx;
        (void)why;
        return NB_ERR_ARG;
    };
    if (!(c.eta > 0) || !(c.dt_max > 0) || !(c.dt_min > 0) || c.dt_min > c.dt_max) return bad("steps");
    int e2;
    if (std::frexp(c.dt_max, &e2) != 0.5) return bad("dt_max must be a power of two");
    // steps stay within [2^-300, 2^300], so dt^5 and 1/dt^3 are exact powers of two
    if (c.dt_min < std::ldexp(1.0, -300) || c.dt_max > std::ldexp(1.0, 300)) return bad("step range");
    if (c.precision != NB_PREC_MIXED && c.precision != NB_PREC_FP64) return bad("precision");
    if (c.spin_limit < 1) return bad("spin_limit");
    int dev = c.device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) {
        delete ctx;
        return NB_ERR_CUDA;
    }
    if (cudaSetDevice(dev) != cudaSuccess) {
        delete ctx;
        return NB_ERR_CUDA;
    }
    ctx->device = dev;
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        delete ctx;
        return NB_ERR_CUDA;
    }
    if (stream) {
        ctx->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return NB_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    ctx->inject_pending = c.inject;
    (void)force_mixed_ctas_per_sm();   // sets kernel attributes before any graph capture
    (void)force_f64_ctas_per_sm();
    if (c.precision == NB_PREC_MIXED) (void)engine_cluster();
    bool ok = dalloc(&ctx->s, 1) == cudaSuccess && dalloc(&ctx->t_next, 1) == cudaSuccess &&
              dalloc(&ctx->t_slot, 2) == cudaSuccess &&
              dalloc(&ctx->t_end, 1) == cudaSuccess && dalloc(&ctx->split_used, 1) == cudaSuccess &&
              dalloc(&ctx->tune_dev, 1) == cudaSuccess && dalloc(&ctx->status, 1) == cudaSuccess &&
              dalloc(&ctx->counters, 4 + NB_SIZE_BUCKETS) == cudaSuccess && dalloc(&ctx->interactions, 1) == cudaSuccess &&
              dalloc(&ctx->en_out, 2) == cudaSuccess && dalloc(&ctx->t_eng, 1) == cudaSuccess;
    if (!ok) {
        nb_destroy(ctx);
        return NB_ERR_CUDA;
    }
    int64_t init_counters[4 + NB_SIZE_BUCKETS] = {0, 0, int64_t(1) << 40};
    int32_t one = 1;
    bool ok2 = cudaMemset(ctx->status, 0, sizeof(int32_t)) == cudaSuccess &&
               cudaMemcpy(ctx->counters, init_counters, sizeof init_counters, cudaMemcpyHostToDevice) ==
                   cudaSuccess &&
               cudaMemcpy(ctx->split_used, &one, sizeof one, cudaMemcpyHostToDevice) == cudaSuccess &&
               cudaMemset(ctx->interactions, 0, sizeof(double)) == cudaSuccess;
    if (!ok2) {
        nb_destroy(ctx);
        return NB_ERR_CUDA;
    }
    *out = ctx;
    return NB_OK;
}

void nb_destroy(nb_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    free_system(ctx);
    nb_ctx_set_ensemble(ctx, nullptr);
    void *ptrs[] = {ctx->s, ctx->t_next, ctx->t_slot, ctx->t_end, ctx->split_used, ctx->tune_dev, ctx->status,
                    ctx->counters, ctx->interactions, ctx->en_out, ctx->t_eng};
    for (void *p : ptrs) dfree(p);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *nb_last_error(const nb_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

nb_status nb_init(nb_ctx *ctx, int64_t n, const double *m, const double *x, const double *v, double eps2)
{
    nb_status st = check_ctx(ctx, false);
    if (st != NB_OK) return st;
    if (n < 1 || n > INT32_MAX) return fail(ctx, NB_ERR_ARG, "n = %lld out of range", (long long)n);
    if (!m || !x || !v) return fail(ctx, NB_ERR_ARG, "null input array");
    if (!(eps2 >= 0.0) || !std::isfinite(eps2)) return fail(ctx, NB_ERR_ARG, "eps2 must be finite and >= 0");
    st = prepare_system(ctx, n, eps2);
    if (st != NB_OK) return st;
    const int64_t np = ctx->n_pad;
    CK(cudaMemcpyAsync(ctx->m, m, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->stage, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_aos_to_soa(ctx->stage, ctx->x, n, np, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpyAsync(ctx->stage, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(launch_aos_to_soa(ctx->stage, ctx->v, n, np, ctx->stream));
    return init_forces(ctx);
}

nb_status nb_init_dev(nb_ctx *ctx, int64_t n, const double *m, const double *x, const double *v, double eps2)
{
    nb_status st = check_ctx(ctx, false);
    if (st != NB_OK) return st;
    if (n < 1 || n > INT32_MAX) return fail(ctx, NB_ERR_ARG, "n = %lld out of range", (long long)n);
    if (!m || !x || !v) return fail(ctx, NB_ERR_ARG, "null input array");
    if (!(eps2 >= 0.0) || !std::isfinite(eps2)) return fail(ctx, NB_ERR_ARG, "eps2 must be finite and >= 0");
    st = prepare_system(ctx, n, eps2);
    if (st != NB_OK) return st;
    const int64_t np = ctx->n_pad;
    CK(cudaMemcpyAsync(ctx->m, m, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(launch_aos_to_soa(x, ctx->x, n, np, ctx->stream));
    CK(launch_aos_to_soa(v, ctx->v, n, np, ctx->stream));
    return init_forces(ctx);
}

nb_status nb_next_block(nb_ctx *ctx, double *t_next, int64_t *s)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    StepArgs A = step_args(ctx);
    CK(launch_select(A, SEL_FULL, 0, false, ctx->stream));
    double tn;
    int64_t ss;
    CK(cudaMemcpyAsync(&tn, ctx->t_next, sizeof tn, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&ss, ctx->s, sizeof ss, cudaMemcpyDeviceToHost, ctx->stream));
    st = sync_status(ctx);
    if (st != NB_OK) return st;
    ctx->block_s = ss;
    ctx->forces_pending = false;
    if (t_next) *t_next = tn;
    if (s) *s = ss;
    return NB_OK;
}

nb_status nb_get_active(nb_ctx *ctx, int32_t *idx)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (ctx->block_s < 0) return fail(ctx, NB_ERR_STATE, "no active list (call nb_next_block)");
    if (!idx) return fail(ctx, NB_ERR_ARG, "null idx");
    if (ctx->block_s > 0)
        CK(cudaMemcpyAsync(idx, ctx->idx, ctx->block_s * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    return sync_status(ctx);
}

nb_status nb_predict(nb_ctx *ctx, double t)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!std::isfinite(t)) return fail(ctx, NB_ERR_ARG, "t must be finite");
    CK(launch_predict(step_args(ctx), nullptr, t, false, ctx->stream));
    return NB_OK;
}

nb_status nb_get_predicted(nb_ctx *ctx, double *xp, double *vp)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    const int64_t n = ctx->n;
    // stage holds 3n doubles: positions first, then velocities through out_a
    StepArgs A = step_args(ctx);
    CK(launch_records_to_aos(A, xp ? ctx->stage : nullptr, vp ? ctx->out_a : nullptr, ctx->stream));
    if (xp) CK(cudaMemcpyAsync(xp, ctx->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (vp) CK(cudaMemcpyAsync(vp, ctx->out_a, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return sync_status(ctx);
}

static nb_status force_common(nb_ctx *ctx, int64_t s, double *a_dev, double *k_dev, double *phi_dev)
{
    CK(launch_force_ctx(ctx));
    CK(launch_reduce_out(ctx->fin, nullptr, s, a_dev, k_dev, phi_dev, ctx->status, ctx->stream));
    ctx->forces_pending = true;
    ctx->block_s = s;
    return NB_OK;
}

nb_status nb_force_jerk(nb_ctx *ctx, const int32_t *idx, int64_t s, double *a, double *k, double *phi)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (s < 0 || s > ctx->n) return fail(ctx, NB_ERR_ARG, "s = %lld out of range", (long long)s);
    if (s == 0) return NB_OK;
    if (idx) {
        for (int64_t q = 0; q < s; ++q) {
            if (idx[q] < 0 || idx[q] >= ctx->n) return fail(ctx, NB_ERR_ARG, "idx[%lld] out of range", (long long)q);
            if (q > 0 && idx[q] <= idx[q - 1]) return fail(ctx, NB_ERR_ARG, "idx not strictly ascending");
        }
        CK(cudaMemcpyAsync(ctx->idx, idx, s * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->s, &s, sizeof s, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));   // idx, s are host stack/caller memory
    } else if (s != ctx->block_s) {
        return fail(ctx, NB_ERR_ARG, "s does not match the last nb_next_block");
    }
    st = force_common(ctx, s, ctx->out_a, ctx->out_k, ctx->out_phi);
    if (st != NB_OK) return st;
    if (a) CK(cudaMemcpyAsync(a, ctx->out_a, 3 * s * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (k) CK(cudaMemcpyAsync(k, ctx->out_k, 3 * s * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (phi) CK(cudaMemcpyAsync(phi, ctx->out_phi, s * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return sync_status(ctx);
}

nb_status nb_force_jerk_dev(nb_ctx *ctx, const int32_t *idx_dev, int64_t s, double *a, double *k, double *phi)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (s < 0 || s > ctx->n) return fail(ctx, NB_ERR_ARG, "s = %lld out of range", (long long)s);
    if (s == 0) return NB_OK;
    if (!idx_dev) return fail(ctx, NB_ERR_ARG, "null idx_dev");
    // one launch: the kernel reads the caller's list, copies it into the context (for
    // nb_correct) and writes the sums in the caller's layouts
    ForceArgs F = force_args(ctx);
    F.idx = idx_dev;
    F.idx_cap = s;
    F.s_host = s;
    F.idx_copy = ctx->idx;
    F.s_copy = ctx->s;
    F.out_a = a;
    F.out_k = k;
    F.out_phi = phi;
    if (ctx->inject_pending) {
        F.inject = 1;
        ctx->inject_pending = 0;
    }
    CK(launch_force(ctx, F));
    ctx->forces_pending = true;
    ctx->block_s = s;
    return NB_OK;
}

// ----- the j-parallel step (Sect. 3): partial forces over a share of j, and the
// corrector with forces summed elsewhere (over ranks)

static nb_status range_tiles(nb_ctx *ctx, int64_t j_begin, int64_t j_end, int64_t *t_lo, int64_t *t_hi)
{
    if (j_begin < 0 || j_end > ctx->n || j_begin > j_end)
        return fail(ctx, NB_ERR_ARG, "j range [%lld, %lld) outside [0, %lld)", (long long)j_begin, (long long)j_end,
                    (long long)ctx->n);
    if (j_begin % kJT != 0 || (j_end % kJT != 0 && j_end != ctx->n))
        return fail(ctx, NB_ERR_ARG, "j_begin and j_end must be multiples of %d (j_end may be n)", kJT);
    *t_lo = j_begin / kJT;
    *t_hi = (j_end + kJT - 1) / kJT;
    return NB_OK;
}

static nb_status force_range_common(nb_ctx *ctx, int64_t s, int64_t t_lo, int64_t t_hi, double *a_dev,
                                    double *k_dev, double *phi_dev)
{
    if (t_hi == t_lo) {   // an empty share: zero partial sums
        if (a_dev) CK(cudaMemsetAsync(a_dev, 0, 3 * s * sizeof(double), ctx->stream));
        if (k_dev) CK(cudaMemsetAsync(k_dev, 0, 3 * s * sizeof(double), ctx->stream));
        if (phi_dev) CK(cudaMemsetAsync(phi_dev, 0, s * sizeof(double), ctx->stream));
    } else {
        ForceArgs F = force_args(ctx);
        F.tile_lo = t_lo;
        F.tile_hi = t_hi;
        if (ctx->inject_pending) {
            F.inject = 1;
            ctx->inject_pending = 0;
        }
        CK(launch_force(ctx, F));
        CK(launch_reduce_out(ctx->fin, nullptr, s, a_dev, k_dev, phi_dev, ctx->status, ctx->stream));
    }
    ctx->forces_pending = false;   // partial sums: nb_correct does not take them
    ctx->block_s = s;
    return NB_OK;
}

nb_status nb_j_range(nb_ctx *ctx, int32_t rank, int32_t world, int64_t *j_begin, int64_t *j_end)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (world < 1 || rank < 0 || rank >= world) return fail(ctx, NB_ERR_ARG, "rank %d of %d", rank, world);
    const int64_t lo = ctx->n_tiles * rank / world, hi = ctx->n_tiles * (rank + 1) / world;
    if (j_begin) *j_begin = std::min<int64_t>(lo * kJT, ctx->n);
    if (j_end) *j_end = std::min<int64_t>(hi * kJT, ctx->n);
    return NB_OK;
}

nb_status nb_force_jerk_range(nb_ctx *ctx, const int32_t *idx, int64_t s, int64_t j_begin, int64_t j_end, double *a,
                              double *k, double *phi)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (s < 0 || s > ctx->n) return fail(ctx, NB_ERR_ARG, "s = %lld out of range", (long long)s);
    int64_t t_lo = 0, t_hi = 0;
    if ((st = range_tiles(ctx, j_begin, j_end, &t_lo, &t_hi)) != NB_OK) return st;
    if (s == 0) return NB_OK;
    if (idx) {
        for (int64_t q = 0; q < s; ++q) {
            if (idx[q] < 0 || idx[q] >= ctx->n) return fail(ctx, NB_ERR_ARG, "idx[%lld] out of range", (long long)q);
            if (q > 0 && idx[q] <= idx[q - 1]) return fail(ctx, NB_ERR_ARG, "idx not strictly ascending");
        }
        CK(cudaMemcpyAsync(ctx->idx, idx, s * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ctx->s, &s, sizeof s, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    } else if (s != ctx->block_s) {
        return fail(ctx, NB_ERR_ARG, "s does not match the last nb_next_block");
    }
    st = force_range_common(ctx, s, t_lo, t_hi, ctx->out_a, ctx->out_k, ctx->out_phi);
    if (st != NB_OK) return st;
    if (a) CK(cudaMemcpyAsync(a, ctx->out_a, 3 * s * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (k) CK(cudaMemcpyAsync(k, ctx->out_k, 3 * s * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (phi) CK(cudaMemcpyAsync(phi, ctx->out_phi, s * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return sync_status(ctx);
}

nb_status nb_force_jerk_range_dev(nb_ctx *ctx, const int32_t *idx_dev, int64_t s, int64_t j_begin, int64_t j_end,
                                  double *a_dev, double *k_dev, double *phi_dev)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (s < 0 || s > ctx->n) return fail(ctx, NB_ERR_ARG, "s = %lld out of range", (long long)s);
    int64_t t_lo = 0, t_hi = 0;
    if ((st = range_tiles(ctx, j_begin, j_end, &t_lo, &t_hi)) != NB_OK) return st;
    if (s == 0) return NB_OK;
    if (idx_dev) {
        CK(launch_set_active(idx_dev, ctx->idx, s, ctx->s, ctx->stream));
    } else if (s != ctx->block_s) {
        return fail(ctx, NB_ERR_ARG, "s does not match the last nb_next_block");
    }
    return force_range_common(ctx, s, t_lo, t_hi, a_dev, k_dev, phi_dev);
}

static nb_status correct_with(nb_ctx *ctx, double t_block)
{
    CK(cudaMemcpyAsync(ctx->t_next, &t_block, sizeof t_block, cudaMemcpyHostToDevice, ctx->stream));
    StepArgs A = step_args(ctx);
    CK(launch_check_due(A, t_block, ctx->stream));
    nb_status st = sync_status(ctx);
    if (st != NB_OK) return st;
    CK(launch_correct(A, true, false, false, ctx->stream));
    ctx->forces_pending = false;
    ctx->block_s = -1;
    return sync_status(ctx);
}

nb_status nb_correct_forces(nb_ctx *ctx, double t_block, const double *a, const double *k)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (ctx->block_s < 0) return fail(ctx, NB_ERR_STATE, "no active list (call nb_next_block)");
    if (!a || !k) return fail(ctx, NB_ERR_ARG, "null forces");
    const int64_t s = ctx->block_s;
    if (s == 0) return NB_OK;
    std::vector<double> fin((size_t)s * kPartStride, 0.0);
    for (int64_t q = 0; q < s; ++q)
        for (int c = 0; c < 3; ++c) {
            fin[q * kPartStride + c] = a[3 * q + c];
            fin[q * kPartStride + 3 + c] = k[3 * q + c];
        }
    CK(cudaMemcpyAsync(ctx->fin, fin.data(), fin.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));   // fin is host stack memory
    return correct_with(ctx, t_block);
}

nb_status nb_correct_forces_dev(nb_ctx *ctx, double t_block, const double *a_dev, const double *k_dev)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (ctx->block_s < 0) return fail(ctx, NB_ERR_STATE, "no active list (call nb_next_block)");
    if (!a_dev || !k_dev) return fail(ctx, NB_ERR_ARG, "null forces");
    const int64_t s = ctx->block_s;
    if (s == 0) return NB_OK;
    CK(launch_forces_in(a_dev, k_dev, s, ctx->fin, ctx->stream));
    return correct_with(ctx, t_block);
}

// Perturber lists (nb_perturb.cu): argument checks shared by both entry points.
static nb_status perturbers_args(nb_ctx *ctx, int32_t nbin, const void *pairs, int32_t nmax, int64_t *j_lo,
                                 int64_t *j_hi, const void *lists, const void *counts)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (nbin < 0) return fail(ctx, NB_ERR_ARG, "nbin must be >= 0");
    if (nbin > 0 && (!pairs || !lists || !counts)) return fail(ctx, NB_ERR_ARG, "null pairs, lists or counts");
    if (nmax < 1 || nmax > NB_PERT_MAX) return fail(ctx, NB_ERR_ARG, "nmax must be in [1, NB_PERT_MAX]");
    if (*j_lo < 0) *j_lo = 0;
    if (*j_hi < 0 || *j_hi > ctx->n) *j_hi = ctx->n;
    if (*j_hi < *j_lo) *j_hi = *j_lo;
    return NB_OK;
}

static PertArgs pert_args(nb_ctx *ctx, int32_t nbin, const int32_t *pairs, double gamma, int32_t nmax,
                          int64_t j_lo, int64_t j_hi, int32_t *lists, int32_t *counts)
{
    PertArgs P{};
    P.n = ctx->n;
    P.np = ctx->n_pad;
    P.m = ctx->m;
    P.x = ctx->x;
    P.nbin = nbin;
    P.pairs = pairs;
    P.gamma = gamma;
    P.nmax = nmax;
    P.j_lo = j_lo;
    P.j_hi = j_hi;
    P.lists = lists;
    P.counts = counts;
    return P;
}

nb_status nb_perturbers_dev(nb_ctx *ctx, int32_t nbin, const int32_t *pairs_dev, double gamma, int32_t nmax,
                            int64_t j_lo, int64_t j_hi, int32_t *lists_dev, int32_t *counts_dev)
{
    nb_status st = perturbers_args(ctx, nbin, pairs_dev, nmax, &j_lo, &j_hi, lists_dev, counts_dev);
    if (st != NB_OK) return st;
    if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(ctx, NB_ERR_ARG, "gamma must be finite and > 0");
    if (nbin == 0) return NB_OK;
    CK(launch_perturbers(pert_args(ctx, nbin, pairs_dev, gamma, nmax, j_lo, j_hi, lists_dev, counts_dev),
                         ctx->stream));
    return NB_OK;
}

nb_status nb_perturbers(nb_ctx *ctx, int32_t nbin, const int32_t *pairs, double gamma, int32_t nmax,
                        int64_t j_lo, int64_t j_hi, int32_t *lists, int32_t *counts)
{
    nb_status st = perturbers_args(ctx, nbin, pairs, nmax, &j_lo, &j_hi, lists, counts);
    if (st != NB_OK) return st;
    if (!(gamma > 0.0) || !std::isfinite(gamma)) return fail(ctx, NB_ERR_ARG, "gamma must be finite and > 0");
    if (nbin == 0) return NB_OK;
    for (int32_t b = 0; b < nbin; ++b) {
        const int32_t i = pairs[2 * b], k = pairs[2 * b + 1];
        if (i < 0 || k < 0 || i >= ctx->n || k >= ctx->n || i == k)
            return fail(ctx, NB_ERR_ARG, "pair %d: members must be two distinct particles", (int)b);
    }
    int32_t *dp = nullptr, *dl = nullptr, *dc = nullptr;
    cudaError_t e = cudaMalloc(&dp, sizeof(int32_t) * 2 * (size_t)nbin);
    if (e == cudaSuccess) e = cudaMalloc(&dl, sizeof(int32_t) * (size_t)nbin * nmax);
    if (e == cudaSuccess) e = cudaMalloc(&dc, sizeof(int32_t) * (size_t)nbin);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp, pairs, sizeof(int32_t) * 2 * (size_t)nbin, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = launch_perturbers(pert_args(ctx, nbin, dp, gamma, nmax, j_lo, j_hi, dl, dc), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(lists, dl, sizeof(int32_t) * (size_t)nbin * nmax, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(counts, dc, sizeof(int32_t) * (size_t)nbin, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cudaFree(dp);
    cudaFree(dl);
    cudaFree(dc);
    if (e != cudaSuccess) return fail(ctx, NB_ERR_CUDA, "perturbers: %s", cudaGetErrorString(e));
    return NB_OK;
}

nb_status nb_correct(nb_ctx *ctx, double t_block)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!ctx->forces_pending) return fail(ctx, NB_ERR_STATE, "no forces pending (call nb_force_jerk)");
    CK(cudaMemcpyAsync(ctx->t_next, &t_block, sizeof t_block, cudaMemcpyHostToDevice, ctx->stream));
    StepArgs A = step_args(ctx);
    CK(launch_check_due(A, t_block, ctx->stream));
    st = sync_status(ctx);
    if (st != NB_OK) return st;
    CK(launch_correct(A, true, false, false, ctx->stream));
    ctx->forces_pending = false;
    return sync_status(ctx);
}

nb_status nb_step(nb_ctx *ctx)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    StepArgs A = step_args(ctx);
    CK(launch_select(A, SEL_FULL, 0, false, ctx->stream));
    const bool eng = engine_on(ctx);
    if (eng) {
        // the engine takes the block if it is small (then s = 0 and the kernels below
        // do nothing), as inside nb_run
        CK(launch_engine(engine_args(ctx, A, ctx->t_next, ctx->t_eng, ctx->s, false, 1), ctx->eng_C, ctx->stream));
    }
    CK(launch_predict(A, A.t_next, 0.0, false, ctx->stream, eng));
    CK(launch_force_ctx(ctx));
    CK(launch_correct(A, false, false, false, ctx->stream));
    ctx->forces_pending = false;
    ctx->block_s = -1;
    return sync_status(ctx);
}

nb_status nb_run(nb_ctx *ctx, double t_end)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!std::isfinite(t_end)) return fail(ctx, NB_ERR_ARG, "t_end must be finite");
    st = build_run_graph(ctx);
    if (st != NB_OK) return st;
    st = set_t_end(ctx, t_end);
    if (st != NB_OK) return st;
    {
        // bound this call's device-side loop: at most kMaxRunSteps block steps
        int64_t done = 0;
        CK(cudaMemcpyAsync(&done, ctx->counters, sizeof done, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        const int64_t cap = done + kMaxRunSteps;
        CK(cudaMemcpyAsync(ctx->counters + 2, &cap, sizeof cap, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (ctx->inject_pending) {   // the hook applies to plain launches; run one step that way
        st = nb_step(ctx);
        if (st != NB_OK) return st;
    }
    CK(cudaGraphLaunch(ctx->run_exec, ctx->stream));
    ctx->forces_pending = false;
    ctx->block_s = -1;
    return sync_status(ctx);
}

nb_status nb_run_timed(nb_ctx *ctx, double t_end, int32_t phases_on, nb_timing *out)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!std::isfinite(t_end)) return fail(ctx, NB_ERR_ARG, "t_end must be finite");
    StepArgs A = step_args(ctx);
    const bool phases = phases_on != 0;
    double inter_f = 0.0, inter_e = 0.0;
    const bool eng = engine_on(ctx);
    const int32_t smax = eng ? engine_args(ctx, A, nullptr, nullptr, nullptr, false, 1).s_max : 0;
    int64_t nl = 0, ne = 0;
    double total[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // select, predict, force, correct, engine
    if (ctx->ev.size() < 10) {
        for (cudaEvent_t e : ctx->ev)
            if (e) cudaEventDestroy(e);
        ctx->ev.assign(10, nullptr);
        for (int q = 0; q < 10; ++q) CK(cudaEventCreate(&ctx->ev[q]));
    }
    // A phase is bracketed by events only after a short, time-bounded wait
    // kernel holds the stream, so that the launch and its end event are queued
    // before the start event is processed: the events then bracket the kernel
    // and not the host's launch latency.
    auto open = [&](int ph) -> cudaError_t {
        cudaError_t e = launch_delay(20000, ctx->stream);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev[2 * ph], ctx->stream);
        return e;
    };
    auto close = [&](int ph) { return cudaEventRecord(ctx->ev[2 * ph + 1], ctx->stream); };
    auto elapsed = [&](int ph) -> cudaError_t {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, ctx->ev[2 * ph], ctx->ev[2 * ph + 1]);
        total[ph] += ms;
        return e;
    };
    for (;;) {
        if (phases) CK(open(0));
        CK(launch_select(A, SEL_FULL, 0, false, ctx->stream));
        if (phases) CK(close(0));
        double tn;
        int64_t ss;
        CK(cudaMemcpyAsync(&tn, ctx->t_next, sizeof tn, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaMemcpyAsync(&ss, ctx->s, sizeof ss, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (!(tn <= t_end) || ss <= 0) break;
        if (phases) CK(elapsed(0));
        if (eng && ss <= smax) {
            // the engine decides (block size and members per chunk) as it does in nb_run
            CK(open(4));
            CK(launch_engine(engine_args(ctx, A, ctx->t_next, ctx->t_eng, ctx->s, false, 1), ctx->eng_C,
                             ctx->stream));
            CK(close(4));
            int64_t left = 0;
            int32_t stw = 0;
            CK(cudaMemcpyAsync(&left, ctx->s, sizeof left, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(&stw, ctx->status, sizeof stw, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
            CK(elapsed(4));
            if (left == 0) {
                ++ne;
                inter_e += (double)ss * (double)ctx->n;
                if (stw) break;
                continue;
            }
        }
        if (phases) CK(open(1));
        CK(launch_predict(A, A.t_next, 0.0, false, ctx->stream));
        if (phases) CK(close(1));
        CK(open(2));
        CK(launch_force_ctx(ctx));
        CK(close(2));
        if (phases) CK(open(3));
        CK(launch_correct(A, false, false, false, ctx->stream));
        if (phases) CK(close(3));
        int32_t stw = 0;
        CK(cudaMemcpyAsync(&stw, ctx->status, sizeof stw, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        CK(elapsed(2));
        if (phases) {
            CK(elapsed(1));
            CK(elapsed(3));
        }
        ++nl;
        inter_f += (double)ss * (double)ctx->n;
        if (stw) break;
    }
    if (out) {
        out->force_ms = total[2];
        for (int q = 0; q < 5; ++q) out->phase_ms[q] = total[q];
        out->force_launches = nl;
        out->engine_steps = ne;
        out->force_interactions = inter_f;
        out->engine_interactions = inter_e;
    }
    ctx->forces_pending = false;
    ctx->block_s = -1;
    return sync_status(ctx);
}

nb_status nb_energy(nb_ctx *ctx, double *E, double *K, double *W)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    CK(launch_energy(step_args(ctx), ctx->en_scratch, ctx->en_ctas, ctx->en_out, ctx->stream));
    double kw[2];
    CK(cudaMemcpyAsync(kw, ctx->en_out, sizeof kw, cudaMemcpyDeviceToHost, ctx->stream));
    st = sync_status(ctx);
    if (st != NB_OK) return st;
    if (K) *K = kw[0];
    if (W) *W = kw[1];
    if (E) *E = kw[0] + kw[1];
    return NB_OK;
}

nb_status nb_get_state(nb_ctx *ctx, nb_state_view *view)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!view || view->n != ctx->n) return fail(ctx, NB_ERR_ARG, "state view size mismatch");
    const int64_t n = ctx->n, np = ctx->n_pad;
    auto vec = [&](double *src, double *dst) -> nb_status {
        if (!dst) return NB_OK;
        CK(launch_soa_to_aos(src, ctx->stage, n, np, ctx->stream));
        CK(cudaMemcpyAsync(dst, ctx->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return NB_OK;
    };
    if (view->m) CK(cudaMemcpyAsync(view->m, ctx->m, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (view->t) CK(cudaMemcpyAsync(view->t, ctx->t, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (view->dt) CK(cudaMemcpyAsync(view->dt, ctx->dt, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if ((st = vec(ctx->x, view->x)) != NB_OK) return st;
    if ((st = vec(ctx->v, view->v)) != NB_OK) return st;
    if ((st = vec(ctx->a, view->a)) != NB_OK) return st;
    if ((st = vec(ctx->k, view->k)) != NB_OK) return st;
    return sync_status(ctx);
}

nb_status nb_set_state(nb_ctx *ctx, const nb_state_view *view)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!view || view->n != ctx->n) return fail(ctx, NB_ERR_ARG, "state view size mismatch");
    if (!view->m || !view->x || !view->v || !view->a || !view->k || !view->t || !view->dt)
        return fail(ctx, NB_ERR_ARG, "set_state needs every array");
    for (int64_t i = 0; i < ctx->n; ++i) {
        // steps must be powers of two within [dt_min, dt_max] and times multiples of them
        int e;
        const double dti = view->dt[i], ti = view->t[i];
        if (!(dti >= ctx->cfg.dt_min && dti <= ctx->cfg.dt_max) || std::frexp(dti, &e) != 0.5 ||
            !(ti >= 0.0) || !std::isfinite(ti) || std::floor(ti / dti) * dti != ti)
            return fail(ctx, NB_ERR_ARG, "state %lld: t = %g, dt = %g is not a valid block-step state",
                        (long long)i, ti, dti);
    }
    const int64_t n = ctx->n, np = ctx->n_pad;
    CK(cudaStreamSynchronize(ctx->stream));
    auto vec = [&](const double *src, double *dst) -> nb_status {
        CK(cudaMemcpyAsync(ctx->stage, src, 3 * n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        CK(launch_aos_to_soa(ctx->stage, dst, n, np, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        return NB_OK;
    };
    CK(cudaMemcpyAsync(ctx->m, view->m, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->t, view->t, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->dt, view->dt, n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    if ((st = vec(view->x, ctx->x)) != NB_OK) return st;
    if ((st = vec(view->v, ctx->v)) != NB_OK) return st;
    if ((st = vec(view->a, ctx->a)) != NB_OK) return st;
    if ((st = vec(view->k, ctx->k)) != NB_OK) return st;
    CK(launch_tnext(step_args(ctx), ctx->stream));
    CK(launch_state_to_ds(step_args(ctx), ctx->stream));
    ctx->forces_pending = false;
    ctx->block_s = -1;
    return sync_status(ctx);
}

nb_status nb_stats(nb_ctx *ctx, nb_counters *out)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (!out) return fail(ctx, NB_ERR_ARG, "null counters");
    int64_t c[4 + NB_SIZE_BUCKETS];
    double inter;
    CK(cudaMemcpyAsync(c, ctx->counters, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&inter, ctx->interactions, sizeof inter, cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<double> t(ctx->n);
    CK(cudaMemcpyAsync(t.data(), ctx->t, ctx->n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out->block_steps = c[0];
    out->particle_steps = c[1];
    out->interactions = inter;
    out->t_now = *std::max_element(t.begin(), t.end());
    for (int b = 0; b < NB_SIZE_BUCKETS; ++b) out->size_hist[b] = c[3 + b];
    out->loop_slots = c[3 + NB_SIZE_BUCKETS];
    return NB_OK;
}

nb_status nb_sync(nb_ctx *ctx)
{
    nb_status st = check_ctx(ctx, false);
    if (st != NB_OK) return st;
    return sync_status(ctx);
}

int32_t nb_num_variants(const nb_ctx *ctx)
{
    if (!ctx) return 0;
    return ctx->cfg.precision == NB_PREC_FP64 ? kF64Variants : kMixedVariants;
}

const char *nb_variant_name(const nb_ctx *ctx, int32_t v)
{
    if (!ctx || v < 0 || v >= nb_num_variants(ctx)) return "";
    return ctx->cfg.precision == NB_PREC_FP64 ? f64_variant_name(v) : mixed_variant_name(v);
}

nb_status nb_set_tuning(nb_ctx *ctx, int32_t bucket, int32_t variant, int32_t split)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (bucket < 0 || bucket >= kBuckets) return fail(ctx, NB_ERR_ARG, "bucket out of range");
    if (variant >= nb_num_variants(ctx)) return fail(ctx, NB_ERR_ARG, "variant out of range");
    if (variant < 0) {
        int64_t s = std::min<int64_t>(int64_t(1) << bucket, ctx->n);
        int vv, SS;
        default_tuning(ctx->cfg.precision, ctx->n, s, force_grid(ctx), 1, &vv, &SS);
        variant = vv;
        split = SS;
    }
    if (split < 1) return fail(ctx, NB_ERR_ARG, "split must be >= 1");
    ctx->tune.variant[bucket] = variant;
    ctx->tune.split[bucket] = split;
    return upload_tuning(ctx);
}

nb_status nb_get_tuning(nb_ctx *ctx, int32_t *variant, int32_t *split)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    if (variant) std::memcpy(variant, ctx->tune.variant, sizeof ctx->tune.variant);
    if (split) std::memcpy(split, ctx->tune.split, sizeof ctx->tune.split);
    return NB_OK;
}

nb_status nb_set_engine(nb_ctx *ctx, int32_t s_max)
{
    nb_status st = check_ctx(ctx, false);
    if (st != NB_OK) return st;
    if (s_max > kEngMaxS || s_max < -1) return fail(ctx, NB_ERR_ARG, "s_max must be in [-1, %d]", kEngMaxS);
    if (s_max > 0 && ctx->cfg.precision != NB_PREC_MIXED)
        return fail(ctx, NB_ERR_ARG, "the small-block engine exists for mixed precision only");
    if (s_max != ctx->eng_smax && ctx->run_exec) {   // the run graph holds the engine's launch
        CK(cudaStreamSynchronize(ctx->stream));
        cudaGraphExecDestroy(ctx->run_exec);
        ctx->run_exec = nullptr;
    }
    ctx->eng_smax = s_max;
    return NB_OK;
}

nb_status nb_get_engine(nb_ctx *ctx, int32_t *s_max, int32_t *cluster)
{
    nb_status st = check_ctx(ctx, false);
    if (st != NB_OK) return st;
    const bool on = ctx->have_state ? engine_on(ctx) : false;
    if (s_max) *s_max = on ? (ctx->eng_smax < 0 ? default_engine_smax(ctx->n) : ctx->eng_smax) : 0;
    if (cluster) *cluster = on ? ctx->eng_C : 0;
    return NB_OK;
}

// Autotuner: for each bucket (s = 1, 2, 4, ..., n) time every variant at a few
// split factors around its default on the current predicted records, with the
// active list 0..s-1, and keep the fastest (median of 3 launches).
nb_status nb_autotune(nb_ctx *ctx)
{
    nb_status st = check_ctx(ctx, true);
    if (st != NB_OK) return st;
    const int nv = nb_num_variants(ctx);
    const bool mixed = ctx->cfg.precision != NB_PREC_FP64;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(launch_fill_iota(ctx->idx, ctx->n, ctx->stream));
    int last_b = 0;
    while ((int64_t(1) << last_b) < ctx->n && last_b < kBuckets - 1) ++last_b;
    for (int b = 0; b <= last_b; ++b) {
        const int64_t s = std::min<int64_t>(int64_t(1) << b, ctx->n);
        CK(cudaMemcpyAsync(ctx->s, &s, sizeof s, cudaMemcpyHostToDevice, ctx->stream));
        float best = 1e30f;
        int bv = ctx->tune.variant[b], bs = ctx->tune.split[b];
        for (int v = 0; v < nv; ++v) {
            const bool share = mixed && v == kShareVariantId;
            if (share && !mixed_share_fits(ctx->n_tiles)) continue;
            const int64_t I = ctx->cfg.precision == NB_PREC_FP64 ? f64_variant_I(v) : mixed_variant_I(v);
            if (I > 4 * s && v > 0) continue;        // i-blocks mostly empty
            if (!share && (s + I - 1) / I > 4096 && v != kMixedFallbackId) continue;   // far too many small work items
            const int64_t nib = (s + I - 1) / I;
            const int64_t R = force_grid(ctx);
            // wave-aligned splits (W = nib * S just below k full waves), the default's
            // choice, a few coarse ones and 1..4; more than 16 waves of items only
            // for splits up to 4
            std::vector<int64_t> cands;
            for (int64_t S : {R / nib, 2 * R / nib, 3 * R / nib, 4 * R / nib, R / (2 * nib),
                              wave_split(nib, ctx->n_tiles, R), ctx->n_tiles / 4, ctx->n_tiles / 16, (int64_t)1,
                              (int64_t)2, (int64_t)3, (int64_t)4}) {
                S = std::min<int64_t>(std::max<int64_t>(S, 1), ctx->n_tiles);
                if (nib * S > 16 * R && S > 4) continue;
                if (std::find(cands.begin(), cands.end(), S) == cands.end()) cands.push_back(S);
            }
            if (share) cands.assign(1, 1);   // the resident-share variant has no split factor
            for (int64_t S : cands) {
                if (S * s * kPartStride > ctx->part_cap) continue;
                ForceArgs F = force_args(ctx, v, (int)S);
                float t3[3] = {0.f, 0.f, 0.f};
                CK(cudaEventRecord(e0, ctx->stream));
                CK(launch_force(ctx, F));   // warm (and a first timing)
                CK(cudaEventRecord(e1, ctx->stream));
                CK(cudaEventSynchronize(e1));
                CK(cudaEventElapsedTime(&t3[0], e0, e1));
                const int reps = t3[0] > 50.f ? 1 : 3;   // long launches: one timing is enough
                // short launches in batches of k back to back (the event timer reads in
                // steps of about a microsecond, the size of the differences being ranked)
                const int k = t3[0] < 0.2f ? std::min(32, std::max(1, (int)(0.2f / std::max(t3[0], 0.005f)))) : 1;
                for (int r = 0; r < reps; ++r) {
                    CK(cudaEventRecord(e0, ctx->stream));
                    for (int q = 0; q < k; ++q) CK(launch_force(ctx, F));
                    CK(cudaEventRecord(e1, ctx->stream));
                    CK(cudaEventSynchronize(e1));
                    CK(cudaEventElapsedTime(&t3[r], e0, e1));
                    t3[r] /= (float)k;
                }
                const float tm = reps == 3 ? std::max(std::min(t3[0], t3[1]), std::min(std::max(t3[0], t3[1]), t3[2]))
                                           : t3[0];
                if (tm < best) {
                    best = tm;
                    bv = v;
                    bs = (int)S;
                }
            }
        }
        ctx->tune.variant[b] = bv;
        ctx->tune.split[b] = bs;
    }
    for (int b = last_b + 1; b < kBuckets; ++b) {
        ctx->tune.variant[b] = ctx->tune.variant[last_b];
        ctx->tune.split[b] = ctx->tune.split[last_b];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->tuned = true;
    st = upload_tuning(ctx);
    if (st != NB_OK) return st;
    ctx->block_s = -1;
    ctx->forces_pending = false;
    return sync_status(ctx);
}

// Ensemble entry points: see nb_ensemble.cu.

}  // extern "C"
