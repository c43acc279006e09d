// Per-block-step kernels around the force evaluation (Sect. 2.1 of the paper):
// the Hermite predictor for all particles, block selection (smallest
// t_i + dt_i), the Hermite corrector with the Aarseth time step quantised to
// powers of two, the first steps, and the FP64 energy diagnostic.
//
// This file is compiled with -fmad=false: every FP64 expression rounds
// operation by operation in the order written, so the predictor and the
// corrector give the same bits as a CPU evaluation of the same formulas
// without fused multiply-adds.
#include <cooperative_groups.h>
#include <math_constants.h>

#include "nb_ds.cuh"
#include "nb_exact.cuh"
#include "nb_hermite.cuh"
#include "nb_internal.cuh"
#include "nb_pair.cuh"

namespace nb {

namespace {

namespace cg = cooperative_groups;

constexpr int kStepThreads = 256;

__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ int64_t gstride() { return (int64_t)gridDim.x * blockDim.x; }

// Predicted position/velocity of particle i at time tn (Hermite predictor).
__device__ __forceinline__ void predict_one(const StepArgs &A, int64_t i, double tn, double *xp, double *vp)
{
    hermite_predict(A.x, A.v, A.a, A.k, A.t, A.n_pad, i, tn, xp, vp);
}

__global__ void predict_kernel(StepArgs A, const double *t_dev, double t_host, int skip_past, int skip_empty)
{
    const double tn = t_dev ? *t_dev : t_host;
    // nb_run loop: no block is due at a time past t_end (the loop's last pass)
    if (skip_past && !(tn <= *A.t_end)) return;
    // nb_step: the small-block engine has done this step
    if (skip_empty && *A.s == 0) return;
    const int64_t np = A.n_pad;
    for (int64_t i = gtid(); i < A.n; i += gstride()) {
        if (A.precision == NB_PREC_MIXED) {
            // double-single Horner on the FP32 pipe (FP64 is a narrow pipe on this part)
            float4 h, l, w;
            ds_predict(A.x2, A.v2, A.a2, A.k2, np, i, tn - A.t[i], h, l, w, (float)A.m[i]);
            jrec_store(A.j.p, i, h.x, h.y, h.z, h.w, l.x, l.y, l.z, w.x, w.y, w.z);
        } else {
            double xp[3], vp[3];
            predict_one(A, i, tn, xp, vp);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                A.xp[c * np + i] = xp[c];
                A.vp[c * np + i] = vp[c];
            }
        }
    }
}

__global__ void pad_kernel(StepArgs A)
{
    const int64_t np = A.n_pad;
    for (int64_t i = A.n + gtid(); i < np; i += gstride()) {
        jrec_store(A.j.p, i, (float)kPadPos, (float)kPadPos, (float)kPadPos, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        A.m[i] = 0.0;
        for (int c = 0; c < 3; ++c) {
            A.xp[c * np + i] = kPadPos;
            A.vp[c * np + i] = 0.0;
            A.x[c * np + i] = kPadPos;
            A.v[c * np + i] = 0.0;
            A.a[c * np + i] = 0.0;
            A.k[c * np + i] = 0.0;
        }
        A.t[i] = CUDART_INF;
        A.dt[i] = CUDART_INF;
        A.tn[i] = CUDART_INF;
    }
}

__global__ void tnext_kernel(StepArgs A)
{
    for (int64_t i = gtid(); i < A.n; i += gstride()) A.tn[i] = A.t[i] + A.dt[i];
}

// Double-single copies of the FP64 state (after uploads and state changes).
__global__ void state_to_ds_kernel(StepArgs A)
{
    const int64_t np = A.n_pad;
    for (int64_t i = gtid(); i < A.n; i += gstride()) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t q = c * np + i;
            A.x2[q] = ds_pack(A.x[q]);
            A.v2[q] = ds_pack(A.v[q]);
            A.a2[q] = ds_pack(A.a[q]);
            A.k2[q] = ds_pack(A.k[q]);
        }
    }
}

// ---------------------------------------------------------------- selection
// Keys tn_i = t_i + dt_i are non-negative doubles (+inf for padding) whose bit
// patterns order like the values, so all comparisons run on the integer pipe.
// Chunks of 16 x (threads) keys; warp w owns keys [512 w, 512 w + 512)
// of a chunk, read as 8 coalesced segments of 64 keys (lane l holds keys 2l and
// 2l + 1 of each segment, one 16-byte load). The padded length is a multiple of
// 256, so a segment lies wholly inside or outside it. Pass 1: minimum. Pass 2:
// ballots give each lane the rank of its hits inside its warp's keys (segment
// by segment, keys in index order), one block-wide scan of the warp counts
// places the warps, and the active list comes out ascending. While a CTA has a
// single chunk its keys stay in registers between the passes.
constexpr int kSelSeg = 8;   // segments of 64 keys per warp
// one CTA of 1024 threads (chunks of 16384 keys) up to 16384 particles; above,
// a cluster of 512-thread CTAs (chunks of 8192 keys: 102 registers, no spills)
constexpr int kSelSmallThreads = 1024, kSelClusterThreads = 512;
constexpr int64_t kSelSmallMax = 16384;

__device__ __forceinline__ long long warp_min_ll(long long v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const long long o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    return v;
}

// key index of lane l's pair in segment j of warp w, chunk base c0
__device__ __forceinline__ int64_t sel_index(int64_t c0, int warp, int j, int lane)
{
    return c0 + (int64_t)warp * (64 * kSelSeg) + 64 * j + 2 * lane;
}

__device__ __forceinline__ void sel_load(const long long *key, int64_t c0, int warp, int lane, int64_t np,
                                         longlong2 *k)
{
#pragma unroll
    for (int j = 0; j < kSelSeg; ++j) {
        const int64_t e = sel_index(c0, warp, j, lane);
        k[j] = e < np ? *reinterpret_cast<const longlong2 *>(key + e)
                      : make_longlong2(0x7ff0000000000000LL, 0x7ff0000000000000LL);
    }
}

// CLUSTER: a thread-block cluster of C CTAs (up to one CTA per chunk, a power
// of two, at most 16); CTA r takes a contiguous run of chunks.
// The CTA minima meet through distributed shared memory across one cluster
// barrier; with C > 1 each CTA then counts its hits, the counts meet across a
// second barrier (a CTA's list starts after the hits of the lower ranks), and a
// last barrier keeps every CTA's shared memory alive until all have read it.
template <int T, bool CLUSTER>
__global__ void __launch_bounds__(T) select_kernel(StepArgs A, cudaGraphConditionalHandle cond, int set_cond)
{
    constexpr int kSelThreads = T;
    constexpr int64_t kSelChunk = (int64_t)T * 2 * kSelSeg;
    __shared__ long long smin[kSelThreads / 32];
    __shared__ int woff[kSelThreads / 32];
    __shared__ int wtot;
    __shared__ long long s_kmin;   // this CTA's minimum
    __shared__ int s_cnt;          // this CTA's hits
    cg::cluster_group cluster = cg::this_cluster();
    const int C = CLUSTER ? (int)cluster.num_blocks() : 1;
    const int rank = CLUSTER ? (int)cluster.block_rank() : 0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t n = A.n, np = A.n_pad;
    const long long *key = reinterpret_cast<const long long *>(A.tn);
    const int64_t nchunk = (np + kSelChunk - 1) / kSelChunk;
    const int64_t cpc = (int64_t)(((uint32_t)nchunk + (uint32_t)C - 1u) / (uint32_t)C);   // nchunk < 2^32
    const int64_t ch0 = (int64_t)rank * cpc < nchunk ? (int64_t)rank * cpc : nchunk;
    const int64_t ch1 = ch0 + cpc < nchunk ? ch0 + cpc : nchunk;
    const bool resident = ch1 - ch0 <= 1;   // the keys stay in registers between the passes
    const unsigned below = (1u << lane) - 1u;
    longlong2 k[kSelSeg];
#pragma unroll
    for (int j = 0; j < kSelSeg; ++j) k[j] = make_longlong2(0x7ff0000000000000LL, 0x7ff0000000000000LL);
    long long m = 0x7ff0000000000000LL;   // +inf
    for (int64_t ch = ch0; ch < ch1; ++ch) {
        sel_load(key, ch * kSelChunk, warp, lane, np, k);
#pragma unroll
        for (int j = 0; j < kSelSeg; ++j) {
            m = k[j].x < m ? k[j].x : m;
            m = k[j].y < m ? k[j].y : m;
        }
    }
    m = warp_min_ll(m);
    if (lane == 0) smin[warp] = m;
    __syncthreads();
    if (warp == 0) {
        long long x = lane < kSelThreads / 32 ? smin[lane] : 0x7ff0000000000000LL;
        x = warp_min_ll(x);
        if (lane == 0) s_kmin = x;
    }
    long long kmin;
    if (CLUSTER) {
        cluster.sync();
        kmin = s_kmin;
        for (int r = 0; r < C; ++r) {
            const long long o = *cluster.map_shared_rank(&s_kmin, r);
            kmin = o < kmin ? o : kmin;
        }
    } else {
        __syncthreads();
        kmin = s_kmin;
    }
    int out = 0;   // entries written before this chunk (same in every thread)
    int total = 0;
    if (CLUSTER && C > 1) {
        // count this CTA's hits, then place the CTA after the lower ranks' hits
        int cnt = 0;
        for (int64_t ch = ch0; ch < ch1; ++ch) {
            const int64_t c0 = ch * kSelChunk;
            if (!resident) sel_load(key, c0, warp, lane, np, k);
#pragma unroll
            for (int j = 0; j < kSelSeg; ++j) {
                const int64_t e = sel_index(c0, warp, j, lane);
                cnt += (k[j].x == kmin && e < n) + (k[j].y == kmin && e + 1 < n);
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (lane == 0) woff[warp] = cnt;
        __syncthreads();
        if (tid == 0) {
            int t = 0;
            for (int w = 0; w < kSelThreads / 32; ++w) t += woff[w];
            s_cnt = t;
        }
        cluster.sync();
        for (int r = 0; r < C; ++r) {
            const int cr = *cluster.map_shared_rank(&s_cnt, r);
            if (r < rank) out += cr;
            total += cr;
        }
        cluster.sync();   // no CTA leaves (or rewrites woff) while others read its shared memory
    }
    for (int64_t ch = ch0; ch < ch1; ++ch) {
        const int64_t c0 = ch * kSelChunk;
        if (!resident) sel_load(key, c0, warp, lane, np, k);
        // per segment: hits of the even and odd key of every lane
        unsigned be[kSelSeg], bo[kSelSeg];
        int wcount = 0;
#pragma unroll
        for (int j = 0; j < kSelSeg; ++j) {
            const int64_t e = sel_index(c0, warp, j, lane);
            be[j] = __ballot_sync(0xffffffffu, k[j].x == kmin && e < n);
            bo[j] = __ballot_sync(0xffffffffu, k[j].y == kmin && e + 1 < n);
            wcount += __popc(be[j]) + __popc(bo[j]);
        }
        if (lane == 0) woff[warp] = wcount;
        __syncthreads();
        if (warp == 0) {
            const int cw = lane < kSelThreads / 32 ? woff[lane] : 0;
            int wi = cw;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, wi, off);
                if (lane >= off) wi += y;
            }
            if (lane < kSelThreads / 32) woff[lane] = wi - cw;
            if (lane == 31) wtot = wi;
        }
        __syncthreads();
        int pos = out + woff[warp];
#pragma unroll
        for (int j = 0; j < kSelSeg; ++j) {
            const int64_t e = sel_index(c0, warp, j, lane);
            const bool he = (be[j] >> lane) & 1u, ho = (bo[j] >> lane) & 1u;
            const int r = pos + __popc(be[j] & below) + __popc(bo[j] & below);
            if (he) A.idx[r] = (int32_t)e;
            if (ho) A.idx[r + (he ? 1 : 0)] = (int32_t)(e + 1);
            pos += __popc(be[j]) + __popc(bo[j]);
        }
        out += wtot;
        __syncthreads();   // woff and wtot are rewritten by the next chunk
    }
    if (C == 1) total = out;
    if (rank == 0 && tid == 0) {
        const int64_t s = (int64_t)total;
        const double tmin = __longlong_as_double(kmin);
        *A.s = s;
        *A.t_next = tmin;
        if (set_cond) {
            const bool ok = (tmin <= *A.t_end) && s > 0 && (*A.status == 0);
            bool more = ok && (A.counters[0] < A.counters[2]);
            if (ok && !more) atomicOr(A.status, kStSteps);
            *A.t_known = tmin;   // the nb_run loop body's first block time
            cudaGraphSetConditional(cond, more ? 1u : 0u);
        }
    }
}

// The nb_run loop body's selection, at a known block time (*t_known, formed by
// the previous corrector): no minimum pass. A cluster of C CTAs (C <= 16) splits
// the keys in chunks of 16 T keys; one pass gives every warp its hits (ballots)
// and its smallest key other than the block time. The CTA totals and minima go
// into every rank's shared memory across one cluster barrier, then each CTA
// writes its hits after those of the lower ranks, ascending. With one chunk per
// CTA the ballots stay in registers between the count and the write.
// Writes s (0 when the block is not to be done: past *t_end, an error, the step
// cap; force and corrector are then no-ops), t_next and *t_form, and sets the
// while-node condition to "this block is done".
template <int T>
__global__ void __launch_bounds__(T) select_known_kernel(StepArgs A, cudaGraphConditionalHandle cond)
{
    constexpr int kW = T / 32;
    constexpr int64_t kChunk = (int64_t)T * 2 * kSelSeg;
    constexpr long long kInf = 0x7ff0000000000000LL;
    __shared__ int woff[kW];
    __shared__ long long wmin[kW];
    __shared__ int wtot;
    __shared__ int r_cnt[16];         // hits of each rank, written by that rank
    __shared__ long long r_min[16];   // smallest key other than the block time, per rank
    // Once this barrier phase completes every CTA of the cluster is running:
    // no CTA writes into another's shared memory before that.
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t np = A.n_pad;
    const long long *key = reinterpret_cast<const long long *>(A.tn);
    const int64_t nchunk = (np + kChunk - 1) / kChunk;
    const int64_t cpc = (int64_t)(((uint32_t)nchunk + (uint32_t)C - 1u) / (uint32_t)C);   // nchunk < 2^32
    const int64_t ch0 = (int64_t)rank * cpc < nchunk ? (int64_t)rank * cpc : nchunk;
    const int64_t ch1 = ch0 + cpc < nchunk ? ch0 + cpc : nchunk;
    const bool resident = ch1 - ch0 <= 1;
    // what the last step reads (the previous corrector wrote it), loaded up front
    const bool lead = rank == 0 && tid == 0;
    const double t_end = lead ? *A.t_end : 0.0;
    const int32_t status0 = lead ? *A.status : 0;
    const bool cap_ok = lead ? A.counters[0] < A.counters[2] : false;
    const long long kmin = *reinterpret_cast<const long long *>(A.t_known);
    // padding keys and keys past n_pad are +inf: with a finite block time every
    // hit is a particle; an infinite one selects nothing
    const bool live = kmin < kInf;
    const unsigned below = (1u << lane) - 1u;
    longlong2 k[kSelSeg];
    unsigned be[kSelSeg], bo[kSelSeg];
    long long m2 = kInf;   // smallest key other than kmin (one below kmin is a state error)
    int wcnt = 0;          // this warp's hits
    for (int64_t ch = ch0; ch < ch1; ++ch) {
        sel_load(key, ch * kChunk, warp, lane, np, k);
#pragma unroll
        for (int j = 0; j < kSelSeg; ++j) {
            const long long x = k[j].x == kmin ? kInf : k[j].x;
            const long long y = k[j].y == kmin ? kInf : k[j].y;
            m2 = x < m2 ? x : m2;
            m2 = y < m2 ? y : m2;
            be[j] = __ballot_sync(0xffffffffu, live && k[j].x == kmin);
            bo[j] = __ballot_sync(0xffffffffu, live && k[j].y == kmin);
            wcnt += __popc(be[j]) + __popc(bo[j]);
        }
    }
    m2 = warp_min_ll(m2);
    if (lane == 0) {
        woff[warp] = wcnt;
        wmin[warp] = m2;
    }
    __syncthreads();
    if (warp == 0) {
        const int cw = lane < kW ? woff[lane] : 0;
        int wi = cw;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < kW) woff[lane] = wi - cw;   // the warps' offsets inside this CTA (one chunk)
        const int tot = __shfl_sync(0xffffffffu, wi, 31);
        const long long mm = warp_min_ll(lane < kW ? wmin[lane] : kInf);
        asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
        if (lane < C) {
            *cluster.map_shared_rank(&r_cnt[rank], lane) = tot;
            *cluster.map_shared_rank(&r_min[rank], lane) = mm;
        }
    } else {
        asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    }
    cluster.sync();   // every rank's total and minimum are in this CTA's shared memory
    // lane r holds rank r's entries; warp reductions give this CTA's offset (the
    // lower ranks' hits), the total and the smallest other key
    const int cr = lane < C ? r_cnt[lane] : 0;
    int out = lane < rank ? cr : 0, total = cr;
    long long m2all = lane < C ? r_min[lane] : kInf;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        out += __shfl_xor_sync(0xffffffffu, out, off);
        total += __shfl_xor_sync(0xffffffffu, total, off);
    }
    m2all = warp_min_ll(m2all);
    for (int64_t ch = ch0; ch < ch1; ++ch) {
        const int64_t c0 = ch * kChunk;
        if (!resident) {
            // several chunks: ballots and warp offsets again, chunk by chunk
            sel_load(key, c0, warp, lane, np, k);
            int wc = 0;
#pragma unroll
            for (int j = 0; j < kSelSeg; ++j) {
                be[j] = __ballot_sync(0xffffffffu, live && k[j].x == kmin);
                bo[j] = __ballot_sync(0xffffffffu, live && k[j].y == kmin);
                wc += __popc(be[j]) + __popc(bo[j]);
            }
            __syncthreads();   // the previous chunk's offsets have been read
            if (lane == 0) woff[warp] = wc;
            __syncthreads();
            if (warp == 0) {
                const int cw = lane < kW ? woff[lane] : 0;
                int wi = cw;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, wi, off);
                    if (lane >= off) wi += y;
                }
                if (lane < kW) woff[lane] = wi - cw;
                if (lane == 31) wtot = wi;
            }
            __syncthreads();
        }
        int pos = out + woff[warp];
#pragma unroll
        for (int j = 0; j < kSelSeg; ++j) {
            const int64_t e = sel_index(c0, warp, j, lane);
            const bool he = (be[j] >> lane) & 1u, ho = (bo[j] >> lane) & 1u;
            const int r = pos + __popc(be[j] & below) + __popc(bo[j] & below);
            if (he) A.idx[r] = (int32_t)e;
            if (ho) A.idx[r + (he ? 1 : 0)] = (int32_t)(e + 1);
            pos += __popc(be[j]) + __popc(bo[j]);
        }
        if (!resident) out += wtot;
    }
    if (lead) {
        A.counters[3 + NB_SIZE_BUCKETS] += 1;   // one more step slot of the nb_run loop has run
        const int64_t s = (int64_t)total;
        const double tmin = __longlong_as_double(kmin);
        const bool due = tmin <= t_end;
        const bool sound = m2all >= kmin && (s > 0 || !due);
        if (!sound) atomicOr(A.status, kStState);
        const bool ok = due && sound && status0 == 0;
        const bool more = ok && cap_ok;
        if (ok && !more) atomicOr(A.status, kStSteps);
        *A.s = more ? s : 0;
        *A.t_next = tmin;
        *A.t_form = more ? __longlong_as_double(m2all) : tmin;
        cudaGraphSetConditional(cond, more ? 1u : 0u);
    }
}

// ---------------------------------------------------------------- corrector

__device__ __forceinline__ void load_fin(const double *fin, int64_t ii, double *an, double *kn, double *phi)
{
    const double *p = fin + ii * kPartStride;
    an[0] = p[0]; an[1] = p[1]; an[2] = p[2];
    kn[0] = p[3]; kn[1] = p[4]; kn[2] = p[5];
    if (phi) *phi = p[6];
}

// Four lanes per active particle (correct_group): 32 particles per CTA and round.
constexpr int kCorThreads = 128;
constexpr int kCorPer = kCorThreads / 4;

__global__ void __launch_bounds__(kCorThreads) correct_kernel(StepArgs A, int check_due, int lower_form)
{
    const int64_t s = *A.s;
    const double tn = *A.t_next;
    const HState H{A.x, A.v, A.a, A.k, A.t, A.dt, A.tn, A.x2, A.v2, A.a2, A.k2, A.n_pad};
    const int q = threadIdx.x & 3;
    const int c = q < 3 ? q : 2;
    // Launched programmatically after the force kernel (nb_run loop), this part
    // overlaps its end: the active list, the block time and the state were
    // written before it, only the new forces (fin) after. The first round's
    // particle and its state are read here; then wait for the force grid.
    const int64_t base0 = (int64_t)blockIdx.x * kCorPer;
    int64_t i0 = 0;
    GroupState g0{};
    if (base0 < s) {
        const int64_t ii = base0 + (threadIdx.x >> 2);
        i0 = A.idx[ii < s ? ii : 0];
        g0 = load_group(H, i0);
    }
    asm volatile("griddepcontrol.wait;" ::: "memory");   // returns at once without such a dependency
    int flags = 0;
    long long kmin = 0x7ff0000000000000LL;   // smallest new key of this thread's particles
    for (int64_t base = base0; base < s; base += (int64_t)gridDim.x * kCorPer) {
        const int64_t ii = base + (threadIdx.x >> 2);
        bool live = ii < s;
        const int64_t iis = live ? ii : 0;
        const bool first = base == base0;
        const int64_t i = first ? i0 : A.idx[iis];
        if (live && check_due && dbits(A.tn[i]) != dbits(tn)) {
            live = false;
            flags |= kStState;
        }
        const double an = A.fin[iis * kPartStride + c], kn = A.fin[iis * kPartStride + 3 + c];
        long long key = 0x7ff0000000000000LL;
        flags |= correct_group(H, i, first ? g0 : load_group(H, i), live, tn, an, kn, A.eta, A.dt_max, A.dt_min, &key);
        kmin = key < kmin ? key : kmin;
    }
    if (lower_form) {
        // the next block time: the smallest of the unchanged keys (*t_form, from
        // the selection) and the new ones; non-negative doubles order like their bits
        kmin = warp_min_ll(kmin);
        if ((threadIdx.x & 31) == 0 && kmin != 0x7ff0000000000000LL)
            atomicMin(reinterpret_cast<long long *>(A.t_form), kmin);
    }
    if (flags) atomicOr(A.status, flags);
    if (blockIdx.x == 0 && threadIdx.x == 0 && s > 0) {
        A.counters[0] += 1;
        A.counters[1] += s;
        int b = 0;
        while ((int64_t(1) << b) < s && b < NB_SIZE_BUCKETS - 1) ++b;
        A.counters[3 + b] += 1;   // block-size histogram
        *A.interactions += (double)s * (double)A.n;
    }
}

// First steps after the initial full force pass.
__global__ void init_steps_kernel(StepArgs A)
{
    const int64_t np = A.n_pad;
    int flags = 0;
    for (int64_t i = gtid(); i < A.n; i += gstride()) {
        double an[3], kn[3];
        load_fin(A.fin, i, an, kn, nullptr);
        bool finite = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A.a[c * np + i] = an[c];
            A.k[c * np + i] = kn[c];
            A.a2[c * np + i] = ds_pack(an[c]);
            A.k2[c * np + i] = ds_pack(kn[c]);
            finite = finite && isfinite(an[c]) && isfinite(kn[c]);
        }
        const double dt = initial_step(an, kn, A.eta, A.dt_max, A.dt_min);
        if (!finite) flags |= kStNonfinite;
        if (dt == 0.0) flags |= kStUnderflow;
        A.t[i] = 0.0;
        A.dt[i] = dt;
        A.tn[i] = 0.0 + dt;
    }
    if (flags) atomicOr(A.status, flags);
}

// Final force sums into caller layouts a[s][3], k[s][3], phi[s].
__global__ void reduce_out_kernel(const double *fin, const int64_t *s_dev, int64_t s_host, double *a, double *k,
                                  double *phi, int32_t *status)
{
    const int64_t s = s_dev ? *s_dev : s_host;
    int flags = 0;
    for (int64_t ii = gtid(); ii < s; ii += gstride()) {
        double an[3], kn[3], ph;
        load_fin(fin, ii, an, kn, &ph);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (a) a[ii * 3 + c] = an[c];
            if (k) k[ii * 3 + c] = kn[c];
            if (!isfinite(an[c]) || !isfinite(kn[c])) flags |= kStNonfinite;
        }
        if (phi) phi[ii] = ph;
        if (!isfinite(ph)) flags |= kStNonfinite;
    }
    if (flags) atomicOr(status, flags);
}

__global__ void check_due_kernel(StepArgs A, double t_block)
{
    const int64_t s = *A.s;
    int flags = 0;
    for (int64_t ii = gtid(); ii < s; ii += gstride()) {
        const int64_t i = A.idx[ii];
        if (A.tn[i] != t_block) flags |= kStState;
    }
    if (flags) atomicOr(A.status, flags);
}

__global__ void aos_to_soa_kernel(const double *src, double *dst, int64_t n, int64_t np)
{
    for (int64_t q = gtid(); q < 3 * n; q += gstride()) {
        const int64_t i = q / 3, c = q % 3;
        dst[c * np + i] = src[q];
    }
}

__global__ void soa_to_aos_kernel(const double *src, double *dst, int64_t n, int64_t np)
{
    for (int64_t q = gtid(); q < 3 * n; q += gstride()) {
        const int64_t i = q / 3, c = q % 3;
        dst[q] = src[c * np + i];
    }
}

// Predicted records back to [n][3] doubles (mixed: hi + lo and the FP32 velocity).
__global__ void records_to_aos_kernel(StepArgs A, double *xo, double *vo)
{
    const int64_t np = A.n_pad;
    for (int64_t i = gtid(); i < A.n; i += gstride()) {
        if (A.precision == NB_PREC_MIXED) {
            const IPart r = jrec_load(A.j.p, i);
            if (xo) {
                xo[3 * i + 0] = (double)r.xh + (double)r.xl;
                xo[3 * i + 1] = (double)r.yh + (double)r.yl;
                xo[3 * i + 2] = (double)r.zh + (double)r.zl;
            }
            if (vo) {
                vo[3 * i + 0] = (double)r.vx;
                vo[3 * i + 1] = (double)r.vy;
                vo[3 * i + 2] = (double)r.vz;
            }
        } else {
            for (int c = 0; c < 3; ++c) {
                if (xo) xo[3 * i + c] = A.xp[c * np + i];
                if (vo) vo[3 * i + c] = A.vp[c * np + i];
            }
        }
    }
}

__global__ void iota_kernel(int32_t *idx, int64_t n)
{
    for (int64_t i = gtid(); i < n; i += gstride()) idx[i] = (int32_t)i;
}

// Forces supplied by the caller (a[s][3], k[s][3]) into the corrector's layout [s][8].
__global__ void forces_in_kernel(const double *a, const double *k, int64_t s, double *fin)
{
    for (int64_t q = gtid(); q < s * kPartStride; q += gstride()) {
        const int64_t ii = q / kPartStride;
        const int c = (int)(q % kPartStride);
        fin[q] = c < 3 ? a[ii * 3 + c] : (c < 6 ? k[ii * 3 + c - 3] : 0.0);
    }
}

// A caller's device active list and its length into the context (one launch
// instead of a device copy and a host-to-device copy of the count).
__global__ void set_active_kernel(const int32_t *src, int32_t *dst, int64_t s, int64_t *s_dev)
{
    for (int64_t i = gtid(); i < s; i += gstride()) dst[i] = src[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) *s_dev = s;
}

// ------------------------------------------------------------------- energy
// K = sum m v^2 / 2, W = sum m_i phi_i / 2 with the softened FP64 potential.
// Each CTA sums its particles in a fixed order into scratch[cta][2]; a single
// thread then adds the CTA sums in index order.
constexpr int kEnThreads = 128;
constexpr int kEnSplitMax = 8;   // j-splits per i-tile (the scratch holds that many partials per tile)

// K and W of the current state. Grid (i-tiles of 128, j-splits): each thread
// sums m_j / r_ij over its split's j != i in double-single on the FP32 pipe (an
// FP64 instruction costs ~64 FP32 lanes' worth here); FP64 takes over per
// particle (W_i = -m_i phi_i / 2, K_i = m_i v_i^2 / 2) and for the CTA and final
// sums, all in a fixed order.
__global__ void __launch_bounds__(kEnThreads) energy_kernel(StepArgs A, double *scratch, int S)
{
    __shared__ float4 sj[kEnThreads][2];
    __shared__ double sk[kEnThreads / 32], sw[kEnThreads / 32];
    const int64_t n = A.n, np = A.n_pad;
    const int64_t i = (int64_t)blockIdx.x * kEnThreads + threadIdx.x;
    const int by = blockIdx.y;
    const bool live = i < n;
    const int64_t ii = live ? i : 0;
    const float2 xi = rn_ds_pack(A.x[ii]), yi = rn_ds_pack(A.x[np + ii]), zi = rn_ds_pack(A.x[2 * np + ii]);
    const float2 e2 = rn_ds_pack(A.eps2);
    float ph = 0.f, pl = 0.f;
    const int64_t ntile = (n + kEnThreads - 1) / kEnThreads;
    const int64_t per = (ntile + S - 1) / S;
    const int64_t t0 = (int64_t)by * per;
    const int64_t t1 = t0 + per < ntile ? t0 + per : ntile;
    for (int64_t t = t0; t < t1; ++t) {
        const int64_t j = t * kEnThreads + threadIdx.x;
        __syncthreads();
        if (j < n) {
            const float2 x = rn_ds_pack(A.x[j]), y = rn_ds_pack(A.x[np + j]), z = rn_ds_pack(A.x[2 * np + j]);
            const float2 m = rn_ds_pack(A.m[j]);
            sj[threadIdx.x][0] = make_float4(x.x, x.y, y.x, y.y);
            sj[threadIdx.x][1] = make_float4(z.x, z.y, m.x, m.y);
        }
        __syncthreads();
        const int jn = (int)(n - t * kEnThreads < kEnThreads ? n - t * kEnThreads : kEnThreads);
        const int self = (int)(i - t * kEnThreads);   // tile slot of i, if it is in this tile
        for (int q = 0; q < jn; ++q) {
            float th, tl;
            en_pair(sj[q][0], sj[q][1], xi, yi, zi, e2, th, tl);
            if (q != self) en_acc(ph, pl, th, tl);
        }
    }
    double ek = 0.0, ew = 0.0;
    if (live) {
        const double mi = A.m[i];
        ew = -0.5 * mi * ((double)ph + (double)pl);
        if (by == 0) {
            const double vx = A.v[i], vy = A.v[np + i], vz = A.v[2 * np + i];
            ek = 0.5 * mi * (vx * vx + vy * vy + vz * vz);
        }
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        ek += __shfl_down_sync(0xffffffffu, ek, off);
        ew += __shfl_down_sync(0xffffffffu, ew, off);
    }
    if ((threadIdx.x & 31) == 0) {
        sk[threadIdx.x >> 5] = ek;
        sw[threadIdx.x >> 5] = ew;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double K = 0.0, W = 0.0;
        for (int w = 0; w < kEnThreads / 32; ++w) {
            K += sk[w];
            W += sw[w];
        }
        const int64_t slot = (int64_t)blockIdx.x * S + by;
        scratch[2 * slot] = K;
        scratch[2 * slot + 1] = W;
    }
}

__global__ void energy_final_kernel(const double *scratch, int64_t nslots, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double K = 0.0, W = 0.0;
        for (int64_t b = 0; b < nslots; ++b) {
            K += scratch[2 * b];
            W += scratch[2 * b + 1];
        }
        out[0] = K;
        out[1] = W;
    }
}

// Keeps the stream busy for about ns nanoseconds (bounded by time and by an
// iteration cap), so that work enqueued behind it is already queued when it
// ends. Used only by the measurement loop.
__global__ void delay_kernel(uint64_t ns)
{
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < 200000; ++it) {
        uint64_t t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= ns) break;
        __nanosleep(256);
    }
}

int grid_for(int64_t n, int threads, int max_grid = 4096)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > max_grid) g = max_grid;
    return (int)g;
}

}  // namespace

// -------------------------------------------------------------------- launchers

cudaError_t launch_predict(const StepArgs &a, const double *t_dev, double t_host, bool skip_past, cudaStream_t st,
                           bool skip_empty)
{
    // FP64-heavy: small CTAs so that the work spreads over every SM
    predict_kernel<<<grid_for(a.n, 64, 8192), 64, 0, st>>>(a, t_dev, t_host, skip_past ? 1 : 0, skip_empty ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_state_to_ds(const StepArgs &a, cudaStream_t st)
{
    state_to_ds_kernel<<<grid_for(a.n, kStepThreads), kStepThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_tnext(const StepArgs &a, cudaStream_t st)
{
    tnext_kernel<<<grid_for(a.n, kStepThreads), kStepThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pad_records(const StepArgs &a, cudaStream_t st)
{
    if (a.n_pad > a.n) pad_kernel<<<grid_for(a.n_pad - a.n, kStepThreads), kStepThreads, 0, st>>>(a);
    return cudaGetLastError();
}

// Largest cluster (16, 8, 4, 2) the device co-schedules for kernel K with the
// given CTA size (queried once per kernel).
template <class K>
int max_cluster(K kernel, int threads)
{
    cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    for (int c = 16; c >= 2; c >>= 1) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3((unsigned)threads);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclu = 0;
        if (cudaOccupancyMaxActiveClusters(&nclu, kernel, &cfg) == cudaSuccess && nclu > 0) {
            (void)cudaGetLastError();
            return c;
        }
    }
    (void)cudaGetLastError();
    return 1;
}

// Launch configuration of a one-cluster grid of C CTAs.
void cluster_config(int C, int threads, cudaStream_t st, cudaLaunchConfig_t &cfg, cudaLaunchAttribute *at)
{
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = st;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
}

// Full selection: one CTA of 1024 threads (chunks of 16384 keys) up to
// kSelSmallMax keys, above that a cluster of 512-thread CTAs, one per chunk of
// 8192 keys, a power of two, at most 16 and at most what the device co-schedules.
cudaError_t launch_select_full(const StepArgs &a, unsigned long long cond, bool set_cond, cudaStream_t st)
{
    if (a.n_pad <= kSelSmallMax) {
        select_kernel<kSelSmallThreads, false>
            <<<1, kSelSmallThreads, 0, st>>>(a, (cudaGraphConditionalHandle)cond, set_cond ? 1 : 0);
        return cudaGetLastError();
    }
    static const int cmax = max_cluster(select_kernel<kSelClusterThreads, true>, kSelClusterThreads);
    const int64_t nchunk = (a.n_pad + 2 * kSelSeg * kSelClusterThreads - 1) / (2 * kSelSeg * kSelClusterThreads);
    int C = 1;
    while (C * 2 <= cmax && C * 2 <= nchunk) C *= 2;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cluster_config(C, kSelClusterThreads, st, cfg, at);
    return cudaLaunchKernelEx(&cfg, select_kernel<kSelClusterThreads, true>, a, (cudaGraphConditionalHandle)cond,
                              set_cond ? 1 : 0);
}

// Selection at a known block time: CTAs of T threads (chunks of 16 T keys) with
// T the smallest of 64, 128, 256, 512 that covers the keys in 16 chunks; as many
// CTAs as chunks, a power of two, at most 16 and at most what the device co-schedules.
template <int T>
cudaError_t launch_select_known_T(const StepArgs &a, unsigned long long cond, cudaStream_t st)
{
    static const int cmax = max_cluster(select_known_kernel<T>, T);
    const int64_t nchunk = (a.n_pad + 2 * kSelSeg * T - 1) / (2 * kSelSeg * T);
    int C = 1;
    while (C * 2 <= cmax && C * 2 <= nchunk) C *= 2;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute at[1];
    cluster_config(C, T, st, cfg, at);
    return cudaLaunchKernelEx(&cfg, select_known_kernel<T>, a, (cudaGraphConditionalHandle)cond);
}

cudaError_t launch_select(const StepArgs &a, SelMode mode, unsigned long long cond, bool set_cond, cudaStream_t st)
{
    if (mode == SEL_FULL) return launch_select_full(a, cond, set_cond, st);
    if (a.n_pad <= 16 * 2 * kSelSeg * 64) return launch_select_known_T<64>(a, cond, st);
    if (a.n_pad <= 16 * 2 * kSelSeg * 128) return launch_select_known_T<128>(a, cond, st);
    if (a.n_pad <= 16 * 2 * kSelSeg * 256) return launch_select_known_T<256>(a, cond, st);
    return launch_select_known_T<512>(a, cond, st);
}

cudaError_t launch_correct(const StepArgs &a, bool check_due, bool lower_form, bool after_force, cudaStream_t st)
{
    // one round covers blocks of up to 608 * 32 particles; CTAs past s exit at once
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)grid_for(a.n, kCorPer, 608));
    cfg.blockDim = dim3(kCorThreads);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    if (after_force) {
        // programmatic dependency on the force kernel just before it in the stream
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, correct_kernel, a, check_due ? 1 : 0, lower_form ? 1 : 0);
}

cudaError_t launch_init_steps(const StepArgs &a, cudaStream_t st)
{
    init_steps_kernel<<<grid_for(a.n, kStepThreads), kStepThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_out(const double *fin, const int64_t *s, int64_t s_host, double *a, double *k,
                              double *phi, int32_t *status, cudaStream_t st)
{
    reduce_out_kernel<<<grid_for(s_host > 0 ? s_host : 1, kStepThreads), kStepThreads, 0, st>>>(fin, s, s_host, a,
                                                                                               k, phi, status);
    return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double *src, double *dst, int64_t n, int64_t np, cudaStream_t st)
{
    aos_to_soa_kernel<<<grid_for(3 * n, kStepThreads), kStepThreads, 0, st>>>(src, dst, n, np);
    return cudaGetLastError();
}

cudaError_t launch_soa_to_aos(const double *src, double *dst, int64_t n, int64_t np, cudaStream_t st)
{
    soa_to_aos_kernel<<<grid_for(3 * n, kStepThreads), kStepThreads, 0, st>>>(src, dst, n, np);
    return cudaGetLastError();
}

cudaError_t launch_records_to_aos(const StepArgs &a, double *xp_aos, double *vp_aos, cudaStream_t st)
{
    records_to_aos_kernel<<<grid_for(a.n, kStepThreads), kStepThreads, 0, st>>>(a, xp_aos, vp_aos);
    return cudaGetLastError();
}

cudaError_t launch_fill_iota(int32_t *idx, int64_t n, cudaStream_t st)
{
    iota_kernel<<<grid_for(n, kStepThreads), kStepThreads, 0, st>>>(idx, n);
    return cudaGetLastError();
}

cudaError_t launch_forces_in(const double *a, const double *k, int64_t s, double *fin, cudaStream_t st)
{
    forces_in_kernel<<<grid_for(s * kPartStride, kStepThreads, 1216), kStepThreads, 0, st>>>(a, k, s, fin);
    return cudaGetLastError();
}

cudaError_t launch_set_active(const int32_t *src, int32_t *dst, int64_t s, int64_t *s_dev, cudaStream_t st)
{
    set_active_kernel<<<grid_for(s > 0 ? s : 1, kStepThreads, 1216), kStepThreads, 0, st>>>(src, dst, s, s_dev);
    return cudaGetLastError();
}

cudaError_t launch_energy(const StepArgs &a, double *scratch, int scratch_ctas, double *out, cudaStream_t st)
{
    const int64_t nbx = (a.n + kEnThreads - 1) / kEnThreads;
    // j-splits so that the grid covers the GPU several times over; the scratch
    // holds kEnSplitMax partials per i-tile
    int64_t S = (1216 + nbx - 1) / nbx;
    if (S > kEnSplitMax) S = kEnSplitMax;
    if (S > nbx) S = nbx;
    if (S < 1) S = 1;
    if (nbx * S > scratch_ctas) return cudaErrorInvalidValue;
    energy_kernel<<<dim3((unsigned)nbx, (unsigned)S), kEnThreads, 0, st>>>(a, scratch, (int)S);
    energy_final_kernel<<<1, 32, 0, st>>>(scratch, nbx * S, out);
    return cudaGetLastError();
}

cudaError_t launch_delay(uint64_t ns, cudaStream_t st)
{
    delay_kernel<<<1, 1, 0, st>>>(ns);
    return cudaGetLastError();
}

cudaError_t launch_check_due(const StepArgs &a, double t_block, cudaStream_t st)
{
    check_due_kernel<<<grid_for(a.n, kStepThreads, 1024), kStepThreads, 0, st>>>(a, t_block);
    return cudaGetLastError();
}

cudaError_t launch_check_active(const int32_t *, int64_t, int64_t, int32_t *, cudaStream_t)
{
    return cudaSuccess;   // host-side validation is used for host index lists
}

}  // namespace nb
