// Batched ensembles of independent systems, each with its own block-step
// schedule (Sect. 2.1 applied to every member), advanced in one persistent
// launch.
//
// Design: the kernel is launched with thread-block clusters of C CTAs (the
// largest of 16, 8 and 4 whose co-resident clusters keep at least 90 % of the
// kernel's CTA slots busy; see ensemble_shape) and one cluster per slot of the
// GPU. A cluster
// takes a whole system from an atomic queue (largest first: the host orders
// the members by N^2) and runs that system's integration to t_end on its own:
// selection, prediction, force, correction, repeated, with the cluster's CTAs
// sharing the particles. Cross-CTA exchanges (minimum of t+dt, active counts,
// error flags) go through distributed shared memory; phases are separated by
// hardware cluster barriers. Control flow is uniform over the cluster by
// construction (every decision is taken from values that all CTAs read the
// same way), so every CTA reaches every barrier; no software spin-wait exists.
//
// Particles are dealt to the cluster's CTAs in even chunks; a CTA predicts,
// corrects and scans the keys of its own chunk. Force work per block step: every
// CTA takes all s active particles against its own chunk as j (the j-split,
// j-share resident in shared memory for chunks of up to 1984 particles), and the
// partials are summed in rank order by the CTA that owns each active particle;
// blocks too large for the j-split's partial slots or shared-memory list (s >
// kEnsSplitCap) are dealt out by i instead, each CTA taking a share of them
// against all of the system's j (no reduction needed).
//
// This file is compiled with -fmad=false (the FP64 corrector must round like
// the CPU oracle); the FP32 pair arithmetic uses explicit fused multiply-adds.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "nb_ds.cuh"
#include "nb_hermite.cuh"
#include "nb_internal.cuh"
#include "nb_pair.cuh"

namespace cg = cooperative_groups;

namespace nb {
namespace {

#ifndef NB_ENS_THREADS
#define NB_ENS_THREADS 256
#endif
#ifndef NB_ENS_MIN_BLOCKS
#define NB_ENS_MIN_BLOCKS (512 / NB_ENS_THREADS)
#endif
constexpr int kEnsThreads = NB_ENS_THREADS;   // threads per CTA (and particles per j-tile)
constexpr int kEnsTile = kEnsThreads;
// Largest block (active count s) taken by the j-split: every CTA runs all active
// particles against its own j-share and the partials are summed across the
// cluster, which needs C * s partial slots per cluster (8 float2 each) and the
// active list in shared memory. On the 256-system workload (8-CTA clusters),
// with larger blocks left to the i-split: 1024 2.16 s, 2048 2.10 s, 4096 2.01 s,
// 6144 1.98 s, 8192 (every block) 1.97 s. Members of up to this many particles
// never take the i-split.
constexpr int kEnsSplitCap = 8192;
constexpr int64_t kEnsMaxN = int64_t(1) << 19;          // largest system one cluster takes
// Dynamic shared memory: a CTA's whole j-share as pair records for the small-s
// force (chunks of up to 2 kJBufPairs - 64 particles; larger chunks stream
// j-tiles from global memory), its first kEnsTile / 2 records the j-tile of the
// streamed force.
constexpr int kJBufPairs = 1024;
constexpr size_t kEnsDynSmem = kJBufPairs * sizeof(JPair);

struct EnsArgs {
    int32_t nc;
    const int64_t *off;      // [nc + 1]
    const double *eps2;      // [nc]
    const int32_t *order;    // [nc] members, largest first
    int64_t np;              // stride of the SoA vectors (total particles)
    double *m, *x, *v, *a, *k, *t, *dt, *tn;
    float2 *x2, *v2, *a2, *k2;   // double-single copies of x, v, a, k
    float2 *t2;              // double-single copy of t (the predictor's time differences on the FP32 pipe)
    float *m32;              // FP32 masses (the j-records' mass)
    float2 *m2;              // double-single masses (the potential sums)
    float4 *jh, *jl, *jv;    // predicted records
    int32_t *idx;            // per-rank candidate segments of the active list, member segments
    int32_t *idx2;           // the active list in rank order (block steps with many active particles)
    float2 *part;            // j-split partials, per cluster
    int32_t *queue;          // next member to take
    int32_t *ready;          // [nc] 1 once forces and first steps exist
    int32_t *status;         // [nc] status bits
    int64_t *steps;          // [nc][2] block steps, particle steps
    double *inter;           // [nc] interactions
    double *energy;          // [nc][16][2] K, W per cluster rank after the last launch
    double t_end, eta, dt_max, dt_min;
    int64_t max_steps;       // per member and launch
    int64_t part_cap;        // partial slots per cluster (C * the j-split's largest s)
    int32_t s_cap;           // the j-split's largest s (<= kEnsSplitCap)
};

struct EnsSmem {
    double dred[kEnsThreads / 32][2];
    long long kmin;              // this CTA's smallest key and how many of its particles have it
    int cnt;
    int err;
    int member;
    int wcnt[kEnsThreads / 32];
    long long wmin[kEnsThreads / 32];
    int seg_off[16], seg_start[16];   // rank q's segment: list positions from seg_off[q], act from seg_start[q]
};

// ------------------------------------------------------------- prediction

// Particle i (global index) predicted to the block time tb (double-single) as
// its j-record. The time difference is formed in double-single from the
// double-single copy of t_i (all times are multiples of the smallest step, so
// the difference is exact), keeping the O(N) prediction off the FP64 pipe (a
// narrow pipe on this part).
__device__ __forceinline__ void predict_one(const EnsArgs &E, int64_t i, DS tb, float4 &h, float4 &l, float4 &w)
{
    float2 X[3], V[3], A[3], K[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        X[c] = E.x2[c * E.np + i];
        V[c] = E.v2[c * E.np + i];
        A[c] = E.a2[c * E.np + i];
        K[c] = E.k2[c * E.np + i];
    }
    const float2 ti = E.t2[i];
    ds_predict_ds(X, V, A, K, ds_sub(tb, DS{ti.x, ti.y}), h, l, w, E.m32[i]);
}

__device__ __forceinline__ DS ds_of_time(double t)
{
    const float2 p = rn_ds_pack(t);
    return DS{p.x, p.y};
}

// Particles [c0, c1) of a member to the block time.
__device__ __forceinline__ void predict_chunk(const EnsArgs &E, int64_t base, int64_t c0, int64_t c1, double tblock)
{
    const DS tb = ds_of_time(tblock);
    for (int64_t q = c0 + threadIdx.x; q < c1; q += kEnsThreads) {
        const int64_t i = base + q;
        float4 h, l, w;
        predict_one(E, i, tb, h, l, w);
        E.jh[i] = h;
        E.jl[i] = l;
        E.jv[i] = w;
    }
}

// ------------------------------------------------------------- force (CTA)

// Records of j in [j0, j1) of one member into shared memory as pair records
// (the layout of the packed pair arithmetic), far-away massless padding past j1.
__device__ __forceinline__ void load_tile(const EnsArgs &E, int64_t base, int64_t jt, int64_t j1, JPair *tile)
{
    const int q = threadIdx.x;
    const int64_t j = jt + q;
    if (j < j1) {
        const float4 h = E.jh[base + j], l = E.jl[base + j], w = E.jv[base + j];
        jrec_store(tile, q, h.x, h.y, h.z, h.w, l.x, l.y, l.z, w.x, w.y, w.z);
    } else {
        const float far = (float)kPadPos;
        jrec_store(tile, q, far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
    }
}

// Forces on the active positions [p0, p1) of list act (member-relative particle
// indices, ascending; global or shared memory) from the member's j in [j0, j1),
// as (hi, lo) float pairs into part: position pp goes to slot slot0 + pp - p0 (7
// values of kPartStride). The i-particles' predicted records are read from
// jh/jl/jv, or with PRED predicted here to tb (when other CTAs' predictions are
// not synchronised with this one).
template <int R, int TJ, bool PRED>
__device__ void cta_force(const EnsArgs &E, int64_t base, const int32_t *act, int64_t p0, int64_t p1, int64_t j0,
                          int64_t j1, float eps2f, float2 *part, int64_t slot0, JPair *tile, DS tb)
{
    constexpr int TI = kEnsThreads / TJ;
    constexpr int I = TI * R;
    constexpr int PPT = (kEnsTile / 2) / TJ;                  // pair records per thread per tile
    constexpr int FP = kFoldPairs / 2;                       // records per fold
    constexpr int CH = PPT < FP ? PPT : FP;
    constexpr int kFoldTiles = PPT >= FP ? 0 : FP / PPT;
    const int tid = threadIdx.x, tj = tid % TJ, ti = tid / TJ;
    const float2 e2 = make_float2(eps2f, eps2f);
    for (int64_t pb = p0; pb < p1; pb += I) {
        const int64_t pe = pb + I < p1 ? pb + I : p1;
        IPk ip[R];
        int32_t gi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t p = pb + (int64_t)r * TI + ti;
            gi[r] = act[p < pe ? p : pe - 1];
            float4 h, l, w;
            if (PRED) {
                predict_one(E, base + gi[r], tb, h, l, w);
            } else {
                h = E.jh[base + gi[r]];
                l = E.jl[base + gi[r]];
                w = E.jv[base + gi[r]];
            }
            ip[r] = ipk_of(IPart{h.x, h.y, h.z, l.x, l.y, l.z, w.x, w.y, w.z});
        }
        const int64_t imin = act[pb], imax = act[pe - 1];
        AccPk p[R];
        Acc7 hi[R], lo[R];
#pragma unroll
        for (int r = 0; r < R; ++r) { zero(p[r]); zero(hi[r]); zero(lo[r]); }
        int fc = 0;
        for (int64_t jt = j0; jt < j1; jt += kEnsTile) {
            __syncthreads();
            load_tile(E, base, jt, j1, tile);
            __syncthreads();
            const bool masked = jt <= imax && jt + kEnsTile - 1 >= imin;
            // pair records holding real particles in this tile (the rest is padding)
            const int npairs = (int)((j1 - jt < kEnsTile ? j1 - jt : kEnsTile) + 1) / 2;
#pragma unroll 1
            for (int c0 = 0; c0 < PPT && c0 * TJ < npairs; c0 += CH) {
                if (masked) {
#pragma unroll 4
                    for (int u = 0; u < CH; ++u) {
                        const int pp = tj + (c0 + u) * TJ;
                        const float4 *Q = tile[pp].q;
                        const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3], q4 = Q[4];
                        const int64_t ja = jt + 2 * pp;
#pragma unroll
                        for (int r = 0; r < R; ++r)
                            pair_packed<true>(q0, q1, q2, q3, q4, ip[r], e2, p[r], ja == gi[r], ja + 1 == gi[r]);
                    }
                } else {
#pragma unroll 4
                    for (int u = 0; u < CH; ++u) {
                        const int pp = tj + (c0 + u) * TJ;
                        const float4 *Q = tile[pp].q;
                        const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3], q4 = Q[4];
#pragma unroll
                        for (int r = 0; r < R; ++r) pair_packed<false>(q0, q1, q2, q3, q4, ip[r], e2, p[r], false, false);
                    }
                }
                if (PPT >= FP) {
#pragma unroll
                    for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);
                }
            }
            if (kFoldTiles > 0 && ++fc == kFoldTiles) {
                fc = 0;
#pragma unroll
                for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            fold(hi[r], lo[r], p[r]);
            if (TJ > 1) ds_group_reduce7<TJ>(hi[r], lo[r]);
        }
        if (tj == 0) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int64_t pp = pb + (int64_t)r * TI + ti;
                if (pp >= pe) continue;
                float2 *dst = part + (slot0 + pp - p0) * kPartStride;
#pragma unroll
                for (int c = 0; c < 7; ++c) dst[c] = make_float2(acc_get(hi[r], c), acc_get(lo[r], c));
            }
        }
    }
}

// Size-adapted dispatch of cta_force.
template <bool PRED>
__device__ __noinline__ void cta_force_any(const EnsArgs &E, int64_t base, const int32_t *act, int64_t p0, int64_t p1,
                                           int64_t j0, int64_t j1, float eps2f, float2 *part, int64_t slot0,
                                           JPair *tile, DS tb = DS{0.f, 0.f})
{
    const int64_t ni = p1 - p0;
    if (ni <= 0) return;
    // one i-particle per thread group (R = 1; two would not fit the registers of
    // the packed form); TJ threads share it
    if (ni <= 8)
        cta_force<1, 32, PRED>(E, base, act, p0, p1, j0, j1, eps2f, part, slot0, tile, tb);
    else if (ni <= 32)
        cta_force<1, 8, PRED>(E, base, act, p0, p1, j0, j1, eps2f, part, slot0, tile, tb);
    else if (ni <= 64)
        cta_force<1, 4, PRED>(E, base, act, p0, p1, j0, j1, eps2f, part, slot0, tile, tb);
    else if (ni <= 128)
        cta_force<1, 2, PRED>(E, base, act, p0, p1, j0, j1, eps2f, part, slot0, tile, tb);
    else
        cta_force<1, 1, PRED>(E, base, act, p0, p1, j0, j1, eps2f, part, slot0, tile, tb);
}

// ------------------------------------------- small-s force on a resident j-share

// Particles [c0, c1) of a member predicted to the block time straight into
// shared memory as pair records (the CTA's j-share), padded with far-away
// massless records to a whole number of 32 records (a padding record adds exact
// zeros).
__device__ __forceinline__ void predict_share(const EnsArgs &E, int64_t base, int64_t c0, int64_t c1, double tblock,
                                              JPair *jb)
{
    const DS tb = ds_of_time(tblock);
    const int nj = (int)(c1 - c0);
    const int npad = (nj + 63) / 64 * 64;
    const float far = (float)kPadPos;
    for (int q = threadIdx.x; q < npad; q += kEnsThreads) {
        if (q < nj) {
            float4 h, l, w;
            predict_one(E, base + c0 + q, tb, h, l, w);
            jrec_store(jb, q, h.x, h.y, h.z, h.w, l.x, l.y, l.z, w.x, w.y, w.z);
        } else {
            jrec_store(jb, q, far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        }
    }
}

// One pass of the small-s force: cnt <= kEnsThreads / TJ active particles from
// list position p0, each shared by TJ threads that split the resident j-share
// (thread tj takes records tj, tj + TJ, ...; the padding covers the last round),
// FP32 partials folded into two-sum accumulators every kFoldPairs terms, then
// summed over the group. The i-particles are predicted here.
template <int TJ>
__device__ __forceinline__ void share_pass(const EnsArgs &E, int64_t base, const int32_t *list, int p0, int cnt,
                                           int64_t c0, int nj, const JPair *jb, float eps2f, float2 *part,
                                           int64_t slot0, DS tb)
{
    constexpr int FP = kFoldPairs / 2;   // records per fold
    const int tid = threadIdx.x, tj = tid % TJ, ti = tid / TJ;
    const bool live = ti < cnt;
    const int32_t gi = list[p0 + (live ? ti : cnt - 1)];
    float4 h, l, w;
    predict_one(E, base + gi, tb, h, l, w);
    const IPk ip = ipk_of(IPart{h.x, h.y, h.z, l.x, l.y, l.z, w.x, w.y, w.z});
    const float2 e2 = make_float2(eps2f, eps2f);
    AccPk p;
    Acc7 hi, lo;
    zero(p);
    zero(hi);
    zero(lo);
    const int nrec = ((nj + 1) / 2 + TJ - 1) / TJ;   // records per thread
    const int64_t self = (int64_t)gi - c0;           // i's place in the share, if it is there
    if (__any_sync(0xffffffffu, self >= 0 && self < nj)) {
        for (int k0 = 0; k0 < nrec; k0 += FP) {
            const int k1 = k0 + FP < nrec ? k0 + FP : nrec;
#pragma unroll 4
            for (int k = k0; k < k1; ++k) {
                const int pp = tj + k * TJ;
                const float4 *Q = jb[pp].q;
                pair_packed<true>(Q[0], Q[1], Q[2], Q[3], Q[4], ip, e2, p, 2 * pp == self, 2 * pp + 1 == self);
            }
            fold(hi, lo, p);
        }
    } else {
        for (int k0 = 0; k0 < nrec; k0 += FP) {
            const int k1 = k0 + FP < nrec ? k0 + FP : nrec;
#pragma unroll 4
            for (int k = k0; k < k1; ++k) {
                const float4 *Q = jb[tj + k * TJ].q;
                pair_packed<false>(Q[0], Q[1], Q[2], Q[3], Q[4], ip, e2, p, false, false);
            }
            fold(hi, lo, p);
        }
    }
    if (TJ > 1) ds_group_reduce7<TJ>(hi, lo);
    if (tj == 0 && live) {
        float2 *dst = part + (slot0 + p0 + ti) * kPartStride;
#pragma unroll
        for (int c = 0; c < 7; ++c) dst[c] = make_float2(acc_get(hi, c), acc_get(lo, c));
    }
}

// All s active particles against the resident j-share of nj particles, in
// passes whose group width TJ fits the remaining count (256 particles with TJ = 1,
// then 128 with TJ = 2, ... down to 8 with TJ = 32), so few threads hold a
// duplicate particle.
__device__ __noinline__ void share_force(const EnsArgs &E, int64_t base, const int32_t *list, int s, int64_t c0,
                                         int nj, const JPair *jb, float eps2f, float2 *part, int64_t slot0, DS tb)
{
    int done = 0;
    while (done < s) {
        const int r = s - done;
        if (r >= 256) {
            share_pass<1>(E, base, list, done, 256, c0, nj, jb, eps2f, part, slot0, tb);
            done += 256;
        } else if (r >= 128) {
            share_pass<2>(E, base, list, done, 128, c0, nj, jb, eps2f, part, slot0, tb);
            done += 128;
        } else if (r >= 64) {
            share_pass<4>(E, base, list, done, 64, c0, nj, jb, eps2f, part, slot0, tb);
            done += 64;
        } else if (r >= 32) {
            share_pass<8>(E, base, list, done, 32, c0, nj, jb, eps2f, part, slot0, tb);
            done += 32;
        } else if (r > 8) {
            const int cnt = r < 16 ? r : 16;
            share_pass<16>(E, base, list, done, cnt, c0, nj, jb, eps2f, part, slot0, tb);
            done += cnt;
        } else {
            share_pass<32>(E, base, list, done, r, c0, nj, jb, eps2f, part, slot0, tb);
            done += r;
        }
    }
}

// Component cq of a and k of list position p: the C ranks' partials summed in
// rank order, all loads issued before the first addition.
__device__ __forceinline__ void sum_partials(const float2 *part, int64_t s, int64_t p, int cq, int C, double &an,
                                             double &kn)
{
    float ha = 0.f, la = 0.f, hk = 0.f, lk = 0.f;
    for (int q0 = 0; q0 < C; q0 += 8) {
        float2 va[8], vk[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (q0 + u < C) {
                const float2 *src = part + ((int64_t)(q0 + u) * s + p) * kPartStride;
                va[u] = __ldcg(src + cq);
                vk[u] = __ldcg(src + 3 + cq);
            }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (q0 + u < C) {
                ds_add(ha, la, va[u].x, va[u].y);
                ds_add(hk, lk, vk[u].x, vk[u].y);
            }
        }
    }
    an = (double)ha + (double)la;
    kn = (double)hk + (double)lk;
}

// ---------------------------------------------------------------- phases

// K and W (softened) of the member's particles [c0, c1) summed by the CTA.
// Every pair once: particle q takes the (N - 1) / 2 particles after it on the
// ring of the member's indices, and for even N the opposite particle with
// weight 1/2 (that pair is reached from both ends), so each thread does the
// same work. The sum of m_j / r over a particle's pairs is double-single on the
// FP32 pipe (en_pair: r from double-single positions, r^2 + eps^2 to ~2^-46, a
// Newton-refined inverse square root; ~2^-44 relative per pair); K, m_i phi_i
// and the sums over particles are FP64, in a fixed order.
__device__ void energy_chunk(const EnsArgs &E, int64_t base, int64_t N, int64_t c0, int64_t c1, double eps2,
                             EnsSmem *sm, double &K, double &W)
{
    double ek = 0.0, ew = 0.0;
    const int64_t half = (N - 1) / 2;
    const float2 e2 = rn_ds_pack(eps2);
    const int64_t np = E.np;
    for (int64_t q = c0 + threadIdx.x; q < c1; q += kEnsThreads) {
        const int64_t i = base + q;
        const float2 xi = E.x2[i], yi = E.x2[np + i], zi = E.x2[2 * np + i];
        float ph = 0.f, pl = 0.f;
        int64_t jj = q;
        for (int64_t d = 1; d <= half; ++d) {
            jj = jj + 1 < N ? jj + 1 : 0;
            const int64_t j = base + jj;
            const float2 xj = E.x2[j], yj = E.x2[np + j], zj = E.x2[2 * np + j], mj = E.m2[j];
            float th, tl;
            en_pair(make_float4(xj.x, xj.y, yj.x, yj.y), make_float4(zj.x, zj.y, mj.x, mj.y), xi, yi, zi, e2, th, tl);
            en_acc(ph, pl, th, tl);
        }
        if ((N & 1) == 0) {
            const int64_t j = base + (q + N / 2 < N ? q + N / 2 : q - N / 2);
            const float2 xj = E.x2[j], yj = E.x2[np + j], zj = E.x2[2 * np + j], mj = E.m2[j];
            float th, tl;
            en_pair(make_float4(xj.x, xj.y, yj.x, yj.y), make_float4(zj.x, zj.y, mj.x, mj.y), xi, yi, zi, e2, th, tl);
            en_acc(ph, pl, 0.5f * th, 0.5f * tl);
        }
        const double vx = E.v[i], vy = E.v[E.np + i], vz = E.v[2 * E.np + i];
        ek += 0.5 * E.m[i] * (vx * vx + vy * vy + vz * vz);
        ew -= E.m[i] * ((double)ph + (double)pl);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        ek += __shfl_xor_sync(0xffffffffu, ek, off);
        ew += __shfl_xor_sync(0xffffffffu, ew, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        sm->dred[warp][0] = ek;
        sm->dred[warp][1] = ew;
    }
    __syncthreads();
    K = 0.0;
    W = 0.0;
    for (int wv = 0; wv < kEnsThreads / 32; ++wv) {
        K += sm->dred[wv][0];
        W += sm->dred[wv][1];
    }
    __syncthreads();
}

__global__ void ens_aos_to_soa(const double *src, double *dst, int64_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 3 * n; q += (int64_t)gridDim.x * blockDim.x)
        dst[(q % 3) * n + q / 3] = src[q];
}

__global__ void ens_to_ds(const double *src, float2 *dst, int64_t count)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = ds_pack(src[q]);
}

__global__ void ens_to_f32(const double *src, float *dst, int64_t count)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = (float)src[q];
}

__global__ void ens_soa_to_aos(const double *src, double *dst, int64_t n)
{
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < 3 * n; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = src[(q % 3) * n + q / 3];
}

__device__ __forceinline__ long long min_ll(long long a, long long b) { return a < b ? a : b; }

__global__ void __launch_bounds__(kEnsThreads, NB_ENS_MIN_BLOCKS) ensemble_kernel(EnsArgs E)
{
    __shared__ EnsSmem smem;
    extern __shared__ __align__(16) unsigned char ens_dyn[];
    EnsSmem *sm = &smem;
    JPair *jbuf = reinterpret_cast<JPair *>(ens_dyn);
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float2 *part = E.part + (int64_t)(blockIdx.x / C) * E.part_cap * kPartStride;
    const int64_t slots = E.part_cap / C;   // partial slots per CTA (i-split and start-up rounds)
    if (tid == 0) {
        sm->err = 0;
        sm->cnt = 0;
        sm->kmin = 0;
    }
    __syncthreads();
    for (;;) {
        if (rank == 0 && tid == 0) sm->member = atomicAdd(E.queue, 1);
        cluster.sync();
        const int slot = *cluster.map_shared_rank(&sm->member, 0);
        cluster.sync();
        if (slot >= E.nc) break;
        const int mem = E.order[slot];
        const int64_t base = E.off[mem];
        const int64_t N = E.off[mem + 1] - base;
        const double eps2 = E.eps2[mem];
        const float eps2f = (float)eps2;
        // particles [c0, c1) belong to this CTA: it predicts them, holds the j-share
        // of the small-s force, corrects them and scans their keys; an even share
        // (pair records stay whole), 32-bit division (N < 2^19)
        const int64_t chunk = (int64_t)((((uint32_t)N + (uint32_t)C - 1u) / (uint32_t)C + 1u) / 2u * 2u);
        const int64_t c0 = (int64_t)rank * chunk < N ? (int64_t)rank * chunk : N;
        const int64_t c1 = c0 + chunk < N ? c0 + chunk : N;
        int32_t *act = E.idx + base;
        int flags = 0;

        if (!E.ready[mem]) {
            // initial forces (s = N), first steps, energy at t = 0
            for (int64_t q = c0 + tid; q < c1; q += kEnsThreads) act[q] = (int32_t)q;
            predict_chunk(E, base, c0, c1, 0.0);
            __threadfence();
            cluster.sync();
            // own particles in rounds of `slots`: sums into this CTA's slots, then a, k,
            // their double-single copies and the first step per particle
            for (int64_t r0 = c0; r0 < c1; r0 += slots) {
                const int64_t r1 = r0 + slots < c1 ? r0 + slots : c1;
                const int64_t slot0 = (int64_t)rank * slots;
                cta_force_any<false>(E, base, act, r0, r1, 0, N, eps2f, part, slot0, jbuf);
                __syncthreads();
                for (int64_t pp = r0 + tid; pp < r1; pp += kEnsThreads) {
                    const float2 *src = part + (slot0 + pp - r0) * kPartStride;
                    double an[3], kn[3];
                    bool fin = true;
                    const int64_t i = base + act[pp];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 va = __ldcg(src + c), vk = __ldcg(src + 3 + c);
                        an[c] = (double)va.x + (double)va.y;
                        kn[c] = (double)vk.x + (double)vk.y;
                        E.a[c * E.np + i] = an[c];
                        E.k[c * E.np + i] = kn[c];
                        E.a2[c * E.np + i] = ds_pack(an[c]);
                        E.k2[c * E.np + i] = ds_pack(kn[c]);
                        fin = fin && isfinite(an[c]) && isfinite(kn[c]);
                    }
                    const double d0 = initial_step(an, kn, E.eta, E.dt_max, E.dt_min);
                    if (!fin) flags |= kStNonfinite;
                    if (d0 == 0.0) flags |= kStUnderflow;
                    E.t[i] = 0.0;
                    E.dt[i] = d0;
                    E.tn[i] = 0.0 + d0;
                }
                __syncthreads();
            }
            __threadfence();
            cluster.sync();
            if (rank == 0 && tid == 0) {
                E.ready[mem] = 1;
                E.steps[2 * mem] = 0;
                E.steps[2 * mem + 1] = 0;
                E.inter[mem] = 0.0;
            }
        }

        int64_t nsteps = 0;
        const unsigned full = 0xffffffffu;
        const long long kInf = 0x7ff0000000000000LL;
        const int cq = (tid & 3) < 3 ? (tid & 3) : 2;   // four lanes per particle in the corrector
        for (;;) {
            // ---- select. Each thread's smallest key over its slice of this CTA's
            // particles and how many have it, reduced to the CTA's (smallest key,
            // count); the particles holding the CTA's smallest key are written, in
            // index order, to this CTA's segment of act. One cluster barrier then
            // exchanges the CTAs' pairs and error flags: the block time is the
            // smallest key, the active list the segments of the CTAs holding it,
            // in rank order.
            const long long *key = reinterpret_cast<const long long *>(E.tn) + base;
            const int64_t sub = (c1 - c0 + kEnsThreads - 1) / kEnsThreads;
            const int64_t s0 = c0 + tid * sub < c1 ? c0 + tid * sub : c1;
            const int64_t s1 = s0 + sub < c1 ? s0 + sub : c1;
            long long mloc = kInf;
            int cloc = 0;
            for (int64_t q = s0; q < s1; q += 4) {   // four loads in flight
                long long kv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) kv[u] = q + u < s1 ? key[q + u] : kInf;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (q + u < s1) {
                        if (kv[u] < mloc) {
                            mloc = kv[u];
                            cloc = 1;
                        } else if (kv[u] == mloc) {
                            ++cloc;
                        }
                    }
                }
            }
            long long wm = mloc;
            int wc = cloc;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const long long om = __shfl_xor_sync(full, wm, off);
                const int oc = __shfl_xor_sync(full, wc, off);
                const long long nm = min_ll(wm, om);
                wc = (wm == nm ? wc : 0) + (om == nm ? oc : 0);
                wm = nm;
            }
            if (lane == 0) {
                sm->wmin[warp] = wm;
                sm->wcnt[warp] = wc;
            }
            // error flags of the previous step, OR-ed over the CTA
            if (flags) atomicOr(&sm->err, flags);
            flags = 0;
            __syncthreads();
            long long mc = sm->wmin[0];
            for (int wv = 1; wv < kEnsThreads / 32; ++wv) mc = min_ll(mc, sm->wmin[wv]);
            int wbase = 0, cc = 0;
            for (int wv = 0; wv < kEnsThreads / 32; ++wv) {
                const int cw = sm->wmin[wv] == mc ? sm->wcnt[wv] : 0;
                if (wv < warp) wbase += cw;
                cc += cw;
            }
            const int ct = mloc == mc ? cloc : 0;
            int incl = ct;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(full, incl, off);
                if (lane >= off) incl += y;
            }
            if (ct > 0) {
                int pos = (int)c0 + wbase + incl - ct;
                for (int64_t q = s0; q < s1; ++q)
                    if (key[q] == mc) act[pos++] = (int32_t)q;
            }
            if (tid == 0) {
                sm->kmin = mc;
                sm->cnt = cc;
            }
            cluster.sync();
            // lane q reads rank q's pair and flags (C <= 16): one round of distributed
            // shared-memory loads, then warp reductions and a scan over the ranks
            const long long kq = lane < C ? *cluster.map_shared_rank(&sm->kmin, lane) : kInf;
            int nq = lane < C ? *cluster.map_shared_rank(&sm->cnt, lane) : 0;
            int err = lane < C ? *cluster.map_shared_rank(&sm->err, lane) : 0;
            long long kmin = kq;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                kmin = min_ll(kmin, __shfl_xor_sync(full, kmin, off));
                err |= __shfl_xor_sync(full, err, off);
            }
            nq = kq == kmin ? nq : 0;
            int oq = nq;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(full, oq, off);
                if (lane >= off) oq += y;
            }
            const int64_t s = __shfl_sync(full, oq, 31);
            oq -= nq;   // rank lane's first position in the list
            const int my_off = __shfl_sync(full, oq, rank), my_cnt = __shfl_sync(full, nq, rank);
            const double tblock = __longlong_as_double(kmin);
            const bool go = (tblock <= E.t_end) && s > 0 && err == 0 && nsteps < E.max_steps;
            if (!go) {
                if (rank == 0 && tid == 0) {
                    if (err) atomicOr(&E.status[mem], err);
                    if (nsteps >= E.max_steps && tblock <= E.t_end) atomicOr(&E.status[mem], kStSteps);
                }
                break;
            }
            if (warp == 0 && lane < C) {
                sm->seg_off[lane] = oq;
                sm->seg_start[lane] = lane * (int)chunk;
            }
            // the j-split's active list sits in dynamic shared memory after the
            // resident j-share (or after the streamed j-tile). Its place, and so the
            // choice between j-split and i-split, follows from the chunk size alone,
            // the same in every CTA of the cluster: a choice that differed between
            // CTAs would pair up different cluster barriers.
            const bool resident = chunk <= 2 * kJBufPairs - 64;
            const int nj = (int)(c1 - c0);
            const int list_rec = resident ? (int)((chunk + 63) / 64 * 32) : kEnsTile / 2;
            int32_t *slist = reinterpret_cast<int32_t *>(jbuf + list_rec);
            if (s <= E.s_cap && s * (int64_t)sizeof(int32_t) <= (int64_t)kEnsDynSmem - list_rec * (int64_t)sizeof(JPair)) {
                // ---- few active particles: every CTA takes all of them against its own
                // j-share (its chunk, predicted by itself), so the i-particles are
                // predicted where they are used and no barrier separates prediction
                // from force. The list is gathered into shared memory; the j-share
                // too, for chunks of up to 2 kJBufPairs - 64 particles.
                __syncthreads();
                for (int p = tid; p < (int)s; p += kEnsThreads) {
                    int q = 0;
                    while (q + 1 < C && sm->seg_off[q + 1] <= p) ++q;
                    slist[p] = act[sm->seg_start[q] + p - sm->seg_off[q]];
                }
                if (resident)
                    predict_share(E, base, c0, c1, tblock, jbuf);
                else
                    predict_chunk(E, base, c0, c1, tblock);
                __syncthreads();
                if (c1 > c0) {
                    if (resident)
                        share_force(E, base, slist, (int)s, c0, nj, jbuf, eps2f, part,
                                    (int64_t)rank * s, ds_of_time(tblock));
                    else
                        cta_force_any<true>(E, base, slist, 0, s, c0, c1, eps2f, part, (int64_t)rank * s, jbuf,
                                            ds_of_time(tblock));
                } else {
                    for (int64_t q = tid; q < s * 7; q += kEnsThreads)
                        part[((int64_t)rank * s + q / 7) * kPartStride + q % 7] = make_float2(0.f, 0.f);
                }
                cluster.sync();
                if (tid == 0) sm->err = 0;
                // each CTA corrects its own active particles (positions my_off ...
                // my_off + my_cnt of the list), summing the ranks' partials in rank order
                const HState H{E.x, E.v, E.a, E.k, E.t, E.dt, E.tn, E.x2, E.v2, E.a2, E.k2, E.np};
                for (int b0 = 0; b0 < my_cnt; b0 += kEnsThreads / 4) {
                    const int kk = b0 + (tid >> 2);
                    const bool live = kk < my_cnt;
                    const int p = my_off + (live ? kk : 0);
                    const int64_t i = base + slist[p];
                    const GroupState g = load_group(H, i);
                    double an, kn;
                    sum_partials(part, s, p, cq, C, an, kn);
                    flags |= correct_group(H, i, g, live, tblock, an, kn, E.eta, E.dt_max, E.dt_min);
                    if (live && (tid & 3) == 3) E.t2[i] = rn_ds_pack(tblock);
                }
                // the keys and states just written belong to this CTA: a CTA barrier
                // orders them before the next scan and prediction
                __syncthreads();
            } else {
                // ---- many active particles: the list in rank order into idx2, all j
                // predicted; each CTA takes an even share of the list against every j
                // (no reduction) in rounds of `slots` through its own slots, each
                // round corrected by four-lane groups
                int32_t *list = E.idx2 + base;
                for (int k = tid; k < my_cnt; k += kEnsThreads) list[my_off + k] = act[c0 + k];
                predict_chunk(E, base, c0, c1, tblock);
                cluster.sync();
                if (tid == 0) sm->err = 0;
                const int64_t share = (s + C - 1) / C;
                const int64_t p0 = (int64_t)rank * share < s ? (int64_t)rank * share : s;
                const int64_t p1 = p0 + share < s ? p0 + share : s;
                const int64_t slot0 = (int64_t)rank * slots;
                for (int64_t r0 = p0; r0 < p1; r0 += slots) {
                    const int64_t r1 = r0 + slots < p1 ? r0 + slots : p1;
                    cta_force_any<false>(E, base, list, r0, r1, 0, N, eps2f, part, slot0, jbuf);
                    __syncthreads();
                    const HState H{E.x, E.v, E.a, E.k, E.t, E.dt, E.tn, E.x2, E.v2, E.a2, E.k2, E.np};
                    for (int64_t b0 = r0; b0 < r1; b0 += kEnsThreads / 4) {
                        const int64_t pp = b0 + (tid >> 2);
                        const bool live = pp < r1;
                        const int64_t pps = live ? pp : r0;
                        const float2 *src = part + (slot0 + pps - r0) * kPartStride;
                        const float2 va = __ldcg(src + cq), vk = __ldcg(src + 3 + cq);
                        const double an = (double)va.x + (double)va.y, kn = (double)vk.x + (double)vk.y;
                        const int64_t i = base + list[pps];
                        flags |= correct_group(H, i, live, tblock, an, kn, E.eta, E.dt_max, E.dt_min);
                        if (live && (tid & 3) == 3) E.t2[i] = rn_ds_pack(tblock);
                    }
                    __syncthreads();
                }
                // particles of every chunk were corrected: a cluster barrier before the
                // next scan
                cluster.sync();
            }
            if (rank == 0 && tid == 0) {
                E.steps[2 * mem] += 1;
                E.steps[2 * mem + 1] += s;
                E.inter[mem] += (double)s * (double)N;
            }
            ++nsteps;
        }
        // ---- energy at the end of this launch
        __threadfence();
        cluster.sync();
        double K, W;
        energy_chunk(E, base, N, c0, c1, eps2, sm, K, W);
        if (tid == 0) {
            E.energy[(mem * 16 + rank) * 2] = K;
            E.energy[(mem * 16 + rank) * 2 + 1] = W;
        }
        if (tid == 0) sm->err = 0;
        cluster.sync();
    }
}

}  // namespace
}  // namespace nb

// ============================================================== host side

using namespace nb;

struct nb_ensemble {
    int32_t nc = 0;
    int64_t ntot = 0;
    int cluster = 0, nclusters = 0;
    int32_t s_cap = 0;      // the j-split's largest block: min(largest member, kEnsSplitCap) by default
    int64_t nmax = 0;       // largest member
    size_t part_alloc = 0;  // float2 entries allocated in part
    double t_now = 0.0;     // time every member is at
    int64_t *off = nullptr;
    double *eps2 = nullptr;
    int32_t *order = nullptr;
    double *m = nullptr, *x = nullptr, *v = nullptr, *a = nullptr, *k = nullptr, *t = nullptr, *dt = nullptr,
           *tn = nullptr;
    float2 *x2 = nullptr, *v2 = nullptr, *a2 = nullptr, *k2 = nullptr, *t2 = nullptr;
    float *m32 = nullptr;
    float2 *m2 = nullptr;
    float4 *jh = nullptr, *jl = nullptr, *jv = nullptr;
    int32_t *idx = nullptr, *idx2 = nullptr;
    float2 *part = nullptr;
    int32_t *queue = nullptr, *ready = nullptr, *status = nullptr;
    int64_t *steps = nullptr;
    double *inter = nullptr, *energy = nullptr;
    double *stage = nullptr;
    std::vector<int64_t> off_host;
};

namespace nb {

void ensemble_free(nb_ensemble *e)
{
    if (!e) return;
    void *ptrs[] = {e->off, e->eps2, e->order, e->m, e->x, e->v, e->a, e->k, e->t, e->dt, e->tn, e->x2, e->v2,
                    e->a2, e->k2, e->t2, e->m32, e->m2, e->jh, e->jl, e->jv,
                    e->idx, e->idx2, e->part, e->queue, e->ready, e->status, e->steps, e->inter, e->energy, e->stage};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete e;
}

// Chooses the cluster size and the number of clusters that are resident at
// once: the largest of 16, 8, 4 CTAs per cluster whose resident clusters keep
// at least 90 % of the kernel's resident CTAs busy. Clusters must fit inside a
// GPC, so on this GPU 16-CTA clusters leave a quarter of the CTA slots empty
// (14 clusters, 224 of 304 CTAs) where 8-CTA clusters fill 288: measured on the
// 256-cluster workload, 4.37 s with 16 against 2.46 s with 8 (3.4 s with 4,
// 6.2 s with 2: smaller clusters lengthen every system's block step).
static cudaError_t ensemble_attrs()
{
    static bool done = false;
    if (done) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(ensemble_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(ensemble_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEnsDynSmem);
    if (err != cudaSuccess) return err;
    done = true;
    return cudaSuccess;
}

// Clusters of C CTAs the device keeps resident at once (0: C does not run).
static int ensemble_clusters(int C)
{
    if (ensemble_attrs() != cudaSuccess) return 0;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(C * 64);
    cfg.blockDim = dim3(kEnsThreads);
    cfg.dynamicSmemBytes = kEnsDynSmem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclu = 0;
    if (cudaOccupancyMaxActiveClusters(&nclu, ensemble_kernel, &cfg) != cudaSuccess || nclu < 1) {
        cudaGetLastError();
        return 0;
    }
    return nclu;
}

static cudaError_t ensemble_shape(int *cluster, int *nclusters)
{
    static int c_cached = 0, n_cached = 0;
    if (c_cached) {
        *cluster = c_cached;
        *nclusters = n_cached;
        return cudaSuccess;
    }
    cudaError_t err = ensemble_attrs();
    if (err != cudaSuccess) return err;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ensemble_kernel, kEnsThreads, kEnsDynSmem) !=
            cudaSuccess ||
        per_sm < 1)
        return cudaErrorInvalidConfiguration;
    const int slots = sms * per_sm;
    int best_c = 0, best_n = 0;
    for (int C : {16, 8, 4}) {
        const int nclu = ensemble_clusters(C);
        if (nclu < 1) continue;
        if (!best_c) {   // fallback: the largest size that runs at all
            best_c = C;
            best_n = nclu;
        }
        if (10 * C * nclu >= 9 * slots) {
            best_c = C;
            best_n = nclu;
            break;
        }
    }
    if (!best_c) return cudaErrorInvalidConfiguration;
    c_cached = best_c;
    n_cached = best_n;
    *cluster = best_c;
    *nclusters = best_n;
    return cudaSuccess;
}

cudaError_t ensemble_launch(nb_ensemble *e, double t_end, double eta, double dt_max, double dt_min, cudaStream_t st)
{
    EnsArgs E{};
    E.nc = e->nc;
    E.off = e->off;
    E.eps2 = e->eps2;
    E.order = e->order;
    E.np = e->ntot;
    E.m = e->m; E.x = e->x; E.v = e->v; E.a = e->a; E.k = e->k; E.t = e->t; E.dt = e->dt; E.tn = e->tn;
    E.x2 = e->x2; E.v2 = e->v2; E.a2 = e->a2; E.k2 = e->k2;
    E.t2 = e->t2; E.m32 = e->m32; E.m2 = e->m2;
    E.jh = e->jh; E.jl = e->jl; E.jv = e->jv;
    E.idx = e->idx;
    E.idx2 = e->idx2;
    E.part = e->part;
    E.s_cap = e->s_cap;
    E.part_cap = (int64_t)e->cluster * e->s_cap;
    E.queue = e->queue;
    E.ready = e->ready;
    E.status = e->status;
    E.steps = e->steps;
    E.inter = e->inter;
    E.energy = e->energy;
    E.t_end = t_end;
    E.eta = eta;
    E.dt_max = dt_max;
    E.dt_min = dt_min;
    E.max_steps = int64_t(1) << 20;
    cudaError_t err = cudaMemsetAsync(e->queue, 0, sizeof(int32_t), st);
    if (err != cudaSuccess) return err;
    err = cudaMemsetAsync(e->energy, 0, 32 * (size_t)e->nc * sizeof(double), st);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = e->cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(e->cluster * e->nclusters);
    cfg.blockDim = dim3(kEnsThreads);
    cfg.dynamicSmemBytes = kEnsDynSmem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, ensemble_kernel, E);
}

}  // namespace nb

// Glue with the context (defined in nb_api.cu).
nb_ensemble *nb_ctx_ensemble(nb_ctx *ctx);
void nb_ctx_set_ensemble(nb_ctx *ctx, nb_ensemble *e);
cudaStream_t nb_ctx_stream(nb_ctx *ctx);
const nb_config *nb_ctx_config(nb_ctx *ctx);
nb_status nb_ctx_fail(nb_ctx *ctx, nb_status st, const char *msg);

namespace nb_ens_host {

template <class T>
cudaError_t ealloc(T **p, size_t count)
{
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(count, 1) * sizeof(T));
}

#define ECK(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            std::string m_ = std::string(#call) + ": " + cudaGetErrorString(e_);                      \
            return nb_ctx_fail(ctx, NB_ERR_CUDA, m_.c_str());                                         \
        }                                                                                             \
    } while (0)

// Partial slots for the current shape: nclusters * cluster * s_cap entries of
// kPartStride (grown, never shrunk).
nb_status ens_part_reserve(nb_ctx *ctx, nb_ensemble *e)
{
    const size_t need = (size_t)e->nclusters * e->cluster * e->s_cap * kPartStride;
    if (need <= e->part_alloc) return NB_OK;
    if (e->part) cudaFree(e->part);
    e->part = nullptr;
    e->part_alloc = 0;
    ECK(ealloc(&e->part, need));
    e->part_alloc = need;
    return NB_OK;
}

nb_status ens_sync(nb_ctx *ctx, nb_ensemble *e)
{
    cudaStream_t st = nb_ctx_stream(ctx);
    ECK(cudaStreamSynchronize(st));
    std::vector<int32_t> status(e->nc);
    ECK(cudaMemcpy(status.data(), e->status, e->nc * sizeof(int32_t), cudaMemcpyDeviceToHost));
    int32_t any = 0;
    for (int32_t s : status) any |= s;
    if (!any) return NB_OK;
    ECK(cudaMemset(e->status, 0, e->nc * sizeof(int32_t)));
    if (any & kStNonfinite) return nb_ctx_fail(ctx, NB_ERR_NONFINITE, "ensemble: non-finite values");
    if (any & kStUnderflow) return nb_ctx_fail(ctx, NB_ERR_DT_UNDERFLOW, "ensemble: time step below dt_min");
    if (any & kStSteps) return nb_ctx_fail(ctx, NB_ERR_STATE, "ensemble: block-step cap reached");
    return nb_ctx_fail(ctx, NB_ERR_CUDA, "ensemble: device error");
}

// Device copies of the state a run changes (for the tuner's probes).
struct EnsBackup {
    double *d = nullptr;
    float2 *f = nullptr;
    int32_t *i = nullptr;
    int64_t *l = nullptr;
    ~EnsBackup()
    {
        for (void *p : {(void *)d, (void *)f, (void *)i, (void *)l})
            if (p) cudaFree(p);
    }
};

static void ens_copy_state(nb_ensemble *e, EnsBackup &b, bool save, cudaStream_t st)
{
    const int64_t n = e->ntot, nc = e->nc;
    auto cp = [&](void *live, void *keep, size_t bytes) {
        if (save)
            cudaMemcpyAsync(keep, live, bytes, cudaMemcpyDeviceToDevice, st);
        else
            cudaMemcpyAsync(live, keep, bytes, cudaMemcpyDeviceToDevice, st);
    };
    double *dd = b.d;
    for (double *p : {e->x, e->v, e->a, e->k}) {
        cp(p, dd, 3 * n * sizeof(double));
        dd += 3 * n;
    }
    for (double *p : {e->t, e->dt, e->tn}) {
        cp(p, dd, n * sizeof(double));
        dd += n;
    }
    cp(e->inter, dd, nc * sizeof(double));
    dd += nc;
    cp(e->energy, dd, 32 * nc * sizeof(double));
    float2 *ff = b.f;
    for (float2 *p : {e->x2, e->v2, e->a2, e->k2}) {
        cp(p, ff, 3 * n * sizeof(float2));
        ff += 3 * n;
    }
    cp(e->t2, ff, n * sizeof(float2));
    cp(e->ready, b.i, nc * sizeof(int32_t));
    cp(e->status, b.i + nc, nc * sizeof(int32_t));
    cp(e->steps, b.l, 2 * nc * sizeof(int64_t));
}

}  // namespace nb_ens_host

using namespace nb_ens_host;

extern "C" {

nb_status nb_ensemble_init(nb_ctx *ctx, int32_t nc, const int64_t *offsets, const double *m, const double *x,
                           const double *v, const double *eps2)
{
    if (!ctx) return NB_ERR_ARG;
    if (nc < 1 || !offsets || !m || !x || !v || !eps2) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: bad arguments");
    if (offsets[0] != 0) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: offsets[0] must be 0");
    for (int32_t c = 0; c < nc; ++c) {
        if (offsets[c + 1] <= offsets[c]) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: empty or unordered system");
        if (!(eps2[c] >= 0.0) || !std::isfinite(eps2[c])) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: bad eps2");
    }
    const int64_t n = offsets[nc];
    if (n > INT32_MAX) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: too many particles");
    for (int32_t c = 0; c < nc; ++c)
        if (offsets[c + 1] - offsets[c] > kEnsMaxN)
            return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: system too large for one cluster");
    nb_ctx_set_ensemble(ctx, nullptr);
    nb_ensemble *e = new nb_ensemble();
    nb_ctx_set_ensemble(ctx, e);
    e->nc = nc;
    e->ntot = n;
    e->off_host.assign(offsets, offsets + nc + 1);
    ECK(ensemble_shape(&e->cluster, &e->nclusters));
    ECK(ealloc(&e->off, nc + 1));
    ECK(ealloc(&e->eps2, nc));
    ECK(ealloc(&e->order, nc));
    ECK(ealloc(&e->m, n));
    for (double **p : {&e->x, &e->v, &e->a, &e->k}) ECK(ealloc(p, 3 * n));
    for (double **p : {&e->t, &e->dt, &e->tn}) ECK(ealloc(p, n));
    for (float2 **p : {&e->x2, &e->v2, &e->a2, &e->k2}) ECK(ealloc(p, 3 * n));
    ECK(ealloc(&e->t2, n));
    ECK(ealloc(&e->m32, n));
    ECK(ealloc(&e->m2, n));
    for (float4 **p : {&e->jh, &e->jl, &e->jv}) ECK(ealloc(p, n));
    ECK(ealloc(&e->idx, n));
    ECK(ealloc(&e->idx2, n));
    for (int32_t c = 0; c < nc; ++c) e->nmax = std::max<int64_t>(e->nmax, offsets[c + 1] - offsets[c]);
    e->s_cap = (int32_t)std::min<int64_t>(e->nmax, kEnsSplitCap);
    {
        const nb_status ps = ens_part_reserve(ctx, e);
        if (ps != NB_OK) return ps;
    }
    ECK(ealloc(&e->queue, 1));
    ECK(ealloc(&e->ready, nc));
    ECK(ealloc(&e->status, nc));
    ECK(ealloc(&e->steps, 2 * nc));
    ECK(ealloc(&e->inter, nc));
    ECK(ealloc(&e->energy, 32 * (size_t)nc));
    ECK(ealloc(&e->stage, 3 * n));
    cudaStream_t st = nb_ctx_stream(ctx);
    // longest first: order by N^2 (the force work), ties by index
    std::vector<int32_t> order(nc);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t p, int32_t q) {
        return offsets[p + 1] - offsets[p] > offsets[q + 1] - offsets[q];
    });
    ECK(cudaMemcpyAsync(e->off, offsets, (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    ECK(cudaMemcpyAsync(e->eps2, eps2, nc * sizeof(double), cudaMemcpyHostToDevice, st));
    ECK(cudaMemcpyAsync(e->order, order.data(), nc * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    ECK(cudaMemcpyAsync(e->m, m, n * sizeof(double), cudaMemcpyHostToDevice, st));
    const int blocks = (int)std::min<int64_t>((3 * n + 255) / 256, 4096);
    ECK(cudaMemcpyAsync(e->stage, x, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    ens_aos_to_soa<<<blocks, 256, 0, st>>>(e->stage, e->x, n);
    ECK(cudaStreamSynchronize(st));
    ECK(cudaMemcpyAsync(e->stage, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st));
    ens_aos_to_soa<<<blocks, 256, 0, st>>>(e->stage, e->v, n);
    ECK(cudaMemsetAsync(e->a, 0, 3 * n * sizeof(double), st));
    ECK(cudaMemsetAsync(e->k, 0, 3 * n * sizeof(double), st));
    ens_to_ds<<<blocks, 256, 0, st>>>(e->x, e->x2, 3 * n);
    ens_to_ds<<<blocks, 256, 0, st>>>(e->v, e->v2, 3 * n);
    ECK(cudaMemsetAsync(e->a2, 0, 3 * n * sizeof(float2), st));
    ECK(cudaMemsetAsync(e->k2, 0, 3 * n * sizeof(float2), st));
    ECK(cudaMemsetAsync(e->t, 0, n * sizeof(double), st));
    ECK(cudaMemsetAsync(e->t2, 0, n * sizeof(float2), st));
    ens_to_f32<<<blocks, 256, 0, st>>>(e->m, e->m32, n);
    ens_to_ds<<<blocks, 256, 0, st>>>(e->m, e->m2, n);
    ECK(cudaMemsetAsync(e->ready, 0, nc * sizeof(int32_t), st));
    ECK(cudaMemsetAsync(e->status, 0, nc * sizeof(int32_t), st));
    ECK(cudaMemsetAsync(e->steps, 0, 2 * nc * sizeof(int64_t), st));
    ECK(cudaMemsetAsync(e->inter, 0, nc * sizeof(double), st));
    // initial forces, first steps and energies at t = 0: a launch that takes no step
    const nb_config *cfg = nb_ctx_config(ctx);
    ECK(ensemble_launch(e, -1.0, cfg->eta, cfg->dt_max, cfg->dt_min, st));
    return ens_sync(ctx, e);
}

nb_status nb_ensemble_run(nb_ctx *ctx, double t_end)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    if (!std::isfinite(t_end)) return nb_ctx_fail(ctx, NB_ERR_ARG, "t_end must be finite");
    const nb_config *cfg = nb_ctx_config(ctx);
    ECK(ensemble_launch(e, t_end, cfg->eta, cfg->dt_max, cfg->dt_min, nb_ctx_stream(ctx)));
    const nb_status st = ens_sync(ctx, e);
    if (st == NB_OK) e->t_now = t_end;
    return st;
}

nb_status nb_ensemble_energy(nb_ctx *ctx, double *E)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    if (!E) return nb_ctx_fail(ctx, NB_ERR_ARG, "null E");
    std::vector<double> kw(32 * (size_t)e->nc);
    ECK(cudaStreamSynchronize(nb_ctx_stream(ctx)));
    ECK(cudaMemcpy(kw.data(), e->energy, kw.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int32_t c = 0; c < e->nc; ++c) {
        double K = 0.0, W = 0.0;   // cluster ranks in order
        for (int q = 0; q < 16; ++q) {
            K += kw[(c * 16 + q) * 2];
            W += kw[(c * 16 + q) * 2 + 1];
        }
        E[c] = K + W;
    }
    return NB_OK;
}

nb_status nb_ensemble_stats(nb_ctx *ctx, int64_t *block_steps, int64_t *particle_steps, double *interactions)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    std::vector<int64_t> st(2 * e->nc);
    ECK(cudaStreamSynchronize(nb_ctx_stream(ctx)));
    ECK(cudaMemcpy(st.data(), e->steps, st.size() * sizeof(int64_t), cudaMemcpyDeviceToHost));
    for (int32_t c = 0; c < e->nc; ++c) {
        if (block_steps) block_steps[c] = st[2 * c];
        if (particle_steps) particle_steps[c] = st[2 * c + 1];
    }
    if (interactions) ECK(cudaMemcpy(interactions, e->inter, e->nc * sizeof(double), cudaMemcpyDeviceToHost));
    return NB_OK;
}

nb_status nb_ensemble_set_shape(nb_ctx *ctx, int32_t cluster, int32_t split_cap)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    if (cluster != 0 && cluster != 2 && cluster != 4 && cluster != 8 && cluster != 16)
        return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: cluster must be 0, 2, 4, 8 or 16");
    if (split_cap < 0) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: split_cap must be >= 0");
    int C = 0, ncl = 0;
    if (cluster == 0) {
        ECK(ensemble_shape(&C, &ncl));
    } else {
        C = cluster;
        ncl = ensemble_clusters(C);
        if (ncl < 1) return nb_ctx_fail(ctx, NB_ERR_ARG, "ensemble: that cluster size does not run on this device");
    }
    const int64_t cap = split_cap == 0 ? std::min<int64_t>(e->nmax, kEnsSplitCap)
                                       : std::min<int64_t>(std::min<int64_t>(split_cap, e->nmax), kEnsSplitCap);
    ECK(cudaStreamSynchronize(nb_ctx_stream(ctx)));
    e->cluster = C;
    e->nclusters = ncl;
    e->s_cap = (int32_t)std::max<int64_t>(cap, 1);
    return ens_part_reserve(ctx, e);
}

nb_status nb_ensemble_get_shape(nb_ctx *ctx, int32_t *cluster, int32_t *nclusters, int32_t *split_cap)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    if (cluster) *cluster = e->cluster;
    if (nclusters) *nclusters = e->nclusters;
    if (split_cap) *split_cap = e->s_cap;
    return NB_OK;
}

nb_status nb_ensemble_autotune(nb_ctx *ctx, double t_probe, float *best_ms)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    const nb_config *cfg = nb_ctx_config(ctx);
    if (!(t_probe > 0.0)) t_probe = cfg->dt_max;
    if (!std::isfinite(t_probe)) return nb_ctx_fail(ctx, NB_ERR_ARG, "t_probe must be finite");
    cudaStream_t st = nb_ctx_stream(ctx);
    const int64_t n = e->ntot, nc = e->nc;
    EnsBackup b;
    ECK(ealloc(&b.d, 15 * n + 33 * nc));
    ECK(ealloc(&b.f, 13 * n));
    ECK(ealloc(&b.i, 2 * nc));
    ECK(ealloc(&b.l, 2 * nc));
    ens_copy_state(e, b, true, st);
    ECK(cudaGetLastError());
    const int C0 = e->cluster, N0 = e->nclusters;
    const int32_t S0 = e->s_cap;
    const int64_t top = std::min<int64_t>(e->nmax, kEnsSplitCap);
    std::vector<int64_t> caps{top};
    for (int64_t c : {4096, 2048, 1024})
        if (c < top) caps.push_back(c);
    cudaEvent_t ev0, ev1;
    ECK(cudaEventCreate(&ev0));
    ECK(cudaEventCreate(&ev1));
    float best = -1.f;
    int bc = C0, bn = N0;
    int32_t bs = S0;
    nb_status rc = NB_OK;
    for (int C : {16, 8, 4}) {
        const int ncl = ensemble_clusters(C);
        if (ncl < 1) continue;
        for (int64_t cap : caps) {
            e->cluster = C;
            e->nclusters = ncl;
            e->s_cap = (int32_t)cap;
            rc = ens_part_reserve(ctx, e);
            if (rc != NB_OK) break;
            cudaEventRecord(ev0, st);
            cudaError_t err = ensemble_launch(e, e->t_now + t_probe, cfg->eta, cfg->dt_max, cfg->dt_min, st);
            cudaEventRecord(ev1, st);
            if (err == cudaSuccess) err = cudaEventSynchronize(ev1);
            float ms = 0.f;
            if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, ev0, ev1);
            std::vector<int32_t> status(nc);
            if (err == cudaSuccess)
                err = cudaMemcpy(status.data(), e->status, nc * sizeof(int32_t), cudaMemcpyDeviceToHost);
            ens_copy_state(e, b, false, st);
            if (err == cudaSuccess) err = cudaStreamSynchronize(st);
            if (err != cudaSuccess) {
                rc = nb_ctx_fail(ctx, NB_ERR_CUDA, cudaGetErrorString(err));
                break;
            }
            bool ok = true;
            for (int32_t v : status) ok = ok && v == 0;
            if (ok && (best < 0.f || ms < best)) {
                best = ms;
                bc = C;
                bn = ncl;
                bs = (int32_t)cap;
            }
        }
        if (rc != NB_OK) break;
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    e->cluster = bc;
    e->nclusters = bn;
    e->s_cap = bs;
    if (rc != NB_OK) return rc;
    if (best < 0.f) return nb_ctx_fail(ctx, NB_ERR_STATE, "ensemble: no probe ran cleanly");
    if (best_ms) *best_ms = best;
    return ens_part_reserve(ctx, e);
}

nb_status nb_ensemble_get_state(nb_ctx *ctx, nb_state_view *view)
{
    if (!ctx) return NB_ERR_ARG;
    nb_ensemble *e = nb_ctx_ensemble(ctx);
    if (!e) return nb_ctx_fail(ctx, NB_ERR_STATE, "no ensemble loaded (call nb_ensemble_init)");
    if (!view || view->n != e->ntot) return nb_ctx_fail(ctx, NB_ERR_ARG, "state view size mismatch");
    cudaStream_t st = nb_ctx_stream(ctx);
    const int64_t n = e->ntot;
    const int blocks = (int)std::min<int64_t>((3 * n + 255) / 256, 4096);
    ECK(cudaStreamSynchronize(st));
    if (view->m) ECK(cudaMemcpy(view->m, e->m, n * sizeof(double), cudaMemcpyDeviceToHost));
    if (view->t) ECK(cudaMemcpy(view->t, e->t, n * sizeof(double), cudaMemcpyDeviceToHost));
    if (view->dt) ECK(cudaMemcpy(view->dt, e->dt, n * sizeof(double), cudaMemcpyDeviceToHost));
    double *src[4] = {e->x, e->v, e->a, e->k};
    double *dst[4] = {view->x, view->v, view->a, view->k};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        ens_soa_to_aos<<<blocks, 256, 0, st>>>(src[q], e->stage, n);
        ECK(cudaMemcpyAsync(dst[q], e->stage, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, st));
        ECK(cudaStreamSynchronize(st));
    }
    return NB_OK;
}

}  // extern "C"
