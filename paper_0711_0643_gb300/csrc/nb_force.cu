// Force + jerk + potential of the active block against all N predicted
// particles: Eq. (Force) of Sect. 2.1 with Plummer softening, its exact time
// derivative, and the softened potential.
//
// The paper splits the j-sum over processors and adds the partial forces with
// MPI_Allreduce (Sect. 3). Here the split is on one chip:
//   * a work item = (i-block, j-split); every CTA of a persistent grid loops
//     over work items derived on the device from the active count s, so the
//     launch needs no host round trip and can live inside a CUDA graph;
//   * j-records stream through shared memory in tiles of kJT records, copied
//     by the TMA bulk engine (cp.async.bulk + mbarrier, kStages in flight);
//   * each thread holds R i-particles in registers and sweeps the tile with
//     TJ threads sharing each i (TJ > 1 splits j inside the CTA when s is small);
//   * partials are reduced in a fixed order (lane shuffles, then the split
//     index): the last CTA to finish an i-block (an arrival ticket, no waiting)
//     sums that block's split partials in ascending split order, so results
//     are bitwise reproducible run to run.
//
// Mixed precision: positions arrive as double-single (hi, lo) pairs so that
// r = x_j - x_i keeps ~46 bits even for close pairs (velocities are FP32: the
// jerk error is set by the FP32 pair arithmetic, not by w); the pair
// arithmetic is FP32 on packed f32x2 instructions over the two particles of a
// pair record, with one MUFU reciprocal square root per particle refined by a
// Newton step; per-thread FP32 partial sums over at most kFoldPairs
// pairs are folded into (hi, lo) two-sum accumulators, and the cross-thread
// reductions combine (hi, lo) pairs with two-sums too (FP64 is a narrow pipe on
// this part; only the final per-split partial is converted to double).
#include <cooperative_groups.h>

#include <cstddef>

#include "nb_internal.cuh"
#include "nb_pair.cuh"

namespace cg = cooperative_groups;

namespace nb {

namespace {

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion counted on the mbarrier (TMA).
// Both addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: false if the spin limit expired.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int64_t limit)
{
    for (int it = 0; it < 64; ++it)
        if (mbar_test(bar, parity)) return true;
    for (int64_t it = 64; it < limit; ++it) {
        if (mbar_test(bar, parity)) return true;
        __nanosleep(64);
    }
    return false;
}

// ------------------------------------------------------------ shared memory

constexpr int kMaxRC = 2 * 7;   // R * components, largest R over variants

constexpr int kPT = kJT / 2;    // pair records per tile
constexpr int kRing = 6;        // tiles in flight in the TMA streaming variant

// Resident-share variant: clusters of kShareC CTAs, CTA r holding up to
// kShareRec pair records of the j range in shared memory, the active list dealt
// out to the clusters in chunks of up to kShareSlots particles.
constexpr int kShareC = 8;
constexpr int kShareRec = 1024;
constexpr int kShareSlots = 256;

// The staging buffers come last, so that the resident-share variant's larger
// buffer can take their place and run past the end of the struct: the kernel
// instantiation without that variant is launched with sizeof(Smem) bytes, the
// one with it with kSmemShare bytes.
struct __align__(128) Smem {
    float2 red[kThreads / 32][kMaxRC];
    uint64_t bar[kRing];
    uint64_t inject_bar;
    int64_t s;                 // active count of this launch
    Tuning tune;               // the device tuning table, read once per CTA
    int32_t idx_pre[kThreads]; // the first kThreads entries of the active list, read with s
    int abort;
    int last;
    alignas(128) union {
        JPair tile[kStages][kPT];   // tile variants
        JPair ring[kRing][kPT];     // TMA streaming variant
    };
};

struct ShareBuf {
    JPair rec[kShareRec];            // this CTA's share of the j-records
    float2 slot[kShareSlots][7];     // (hi, lo) partials of the chunk's particles
};

constexpr size_t kSmemShare = (offsetof(Smem, tile) + sizeof(ShareBuf) + 127) / 128 * 128;

__device__ __forceinline__ ShareBuf *shb(Smem *sm) { return reinterpret_cast<ShareBuf *>(&sm->tile[0][0]); }

__device__ __forceinline__ int bucket_of(int64_t s)
{
    // bucket b holds s in (2^(b-1), 2^b]; s = 1 -> 0
    int b = 0;
    while ((int64_t(1) << b) < s && b < kBuckets - 1) ++b;
    return b;
}

// a / b for a >= 0, b > 0. A 64-bit division is a long dependent instruction
// chain on this GPU (several of them sat on the critical path of every launch);
// the 32-bit one is short, and the sizes of a launch fit in 32 bits.
__device__ __forceinline__ int64_t qdiv(int64_t a, int64_t b)
{
    if ((((uint64_t)a | (uint64_t)b) >> 32) == 0) return (int64_t)((uint32_t)a / (uint32_t)b);
    return a / b;
}

// The table's split is the one for its bucket's largest size s_ref = min(2^b, n);
// a smaller block of the bucket keeps the same number of work items (i-blocks x
// splits), so a wave-aligned choice stays wave-aligned.
__device__ __forceinline__ int table_split(int S_ref, int b, int64_t s, int64_t n, int64_t I)
{
    const int64_t s_ref = (int64_t(1) << b) < n ? (int64_t(1) << b) : n;
    const int64_t nib_ref = qdiv(s_ref + I - 1, I), nib = qdiv(s + I - 1, I);
    const int64_t S = qdiv((int64_t)S_ref * nib_ref, nib);
    return S < 1 ? 1 : (S > (1 << 30) ? (1 << 30) : (int)S);
}

// Entry jj < s of the active list (the first kThreads from shared memory).
__device__ __forceinline__ int32_t idx_at(const ForceArgs &A, const Smem *sm, int64_t jj)
{
    return jj < kThreads ? sm->idx_pre[jj] : A.idx[jj];
}

// Split factor clamp shared by both precisions.
__device__ __forceinline__ int clamp_split(int S, int64_t n_tiles, int64_t s, int64_t cap)
{
    if (S < 1) S = 1;
    if (S > n_tiles) S = (int)n_tiles;
    int64_t lim = qdiv(cap, s * kPartStride);
    if (lim < 1) lim = 1;
    if (S > lim) S = (int)lim;
    return S;
}

// Split partial of active particle ii from split by, as (hi, lo) float pairs.
__device__ __forceinline__ float2 *part2(const ForceArgs &A, int64_t ii, int by, int S)
{
    return reinterpret_cast<float2 *>(A.part) + (ii * S + by) * kPartStride;
}

__device__ __forceinline__ void write_part(const ForceArgs &A, int64_t ii, int by, int S, const Acc7 &hi,
                                           const Acc7 &lo)
{
    float2 *dst = part2(A, ii, by, S);
#pragma unroll
    for (int c = 0; c < 7; ++c) dst[c] = make_float2(acc_get(hi, c), acc_get(lo, c));
}

// Final sum of component c (ax ay az kx ky kz phi) of active particle ii: into
// fin and, when the launch has them, the caller's layouts.
__device__ __forceinline__ void put_final(const ForceArgs &A, int64_t ii, int c, double v)
{
    A.fin[ii * kPartStride + c] = v;
    double *dst = c < 3 ? A.out_a : (c < 6 ? A.out_k : A.out_phi);
    if (dst) {
        dst[c < 6 ? ii * 3 + (c % 3) : ii] = v;
        if (!isfinite(v)) atomicOr(A.status, kStNonfinite);
    }
}

// Active count of a launch and the optional copy of the caller's list into the
// context (grid-stride; every CTA takes part).
__device__ __forceinline__ int64_t launch_s(const ForceArgs &A) { return A.s_host >= 0 ? A.s_host : *A.s; }

__device__ __forceinline__ void copy_list(const ForceArgs &A, int64_t s)
{
    if (!A.idx_copy) return;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < s; q += (int64_t)gridDim.x * blockDim.x)
        A.idx_copy[q] = A.idx[q];
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.s_copy = s;
}

// Called by every thread after a work item has written its partials. The CTA
// that completes the i-block (ticket S - 1) adds the block's S partials in split
// order with two-sums and writes the FP64 results; it then re-arms the ticket.
__device__ void finish_item(const ForceArgs &A, int64_t s, int64_t bx, int S, int64_t I, Smem *sm)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(&A.tickets[bx], 1);
        sm->last = (t == S - 1);
    }
    __syncthreads();
    if (sm->last) {
        __threadfence();
        const int64_t ib0 = bx * I;
        const int64_t ib1 = ib0 + I < s ? ib0 + I : s;
        const int cnt = (int)(ib1 - ib0) * 7;
        if (S <= 4) {
            // few splits: one thread per (particle, component)
            for (int q = threadIdx.x; q < cnt; q += kThreads) {
                const int64_t ii = ib0 + q / 7;
                const int c = q % 7;
                const float2 *src = reinterpret_cast<const float2 *>(A.part) + ii * S * kPartStride + c;
                float h = 0.f, l = 0.f;
                for (int sp = 0; sp < S; ++sp) {
                    const float2 v = __ldcg(src + sp * kPartStride);
                    ds_add(h, l, v.x, v.y);
                }
                put_final(A, ii, c, (double)h + (double)l);
            }
        } else {
            // many splits. The order of every addition is the split order per lane, then a
            // fixed tree over lanes, so the batching of the loads does not change the result.
            constexpr int kFinUnroll = 4;
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            const float2 *base = reinterpret_cast<const float2 *>(A.part);
            if (cnt <= kThreads / 32) {
                // one particle: a warp per component; lane l adds splits l, l + 32, ...
                // (kFinUnroll loads per round), then a butterfly of two-sums over the lanes
                if (warp < cnt) {
                    const float2 *src = base + (ib0 + warp / 7) * S * kPartStride + warp % 7;
                    float h = 0.f, l = 0.f;
                    for (int sp0 = lane; sp0 < S; sp0 += 32 * kFinUnroll) {
                        float2 v[kFinUnroll];
#pragma unroll
                        for (int u = 0; u < kFinUnroll; ++u)
                            v[u] = sp0 + 32 * u < S ? __ldcg(src + (sp0 + 32 * u) * kPartStride) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int u = 0; u < kFinUnroll; ++u)
                            if (sp0 + 32 * u < S) ds_add(h, l, v[u].x, v[u].y);
                    }
                    ds_group_reduce<32>(h, l);
                    if (lane == 0) put_final(A, ib0 + warp / 7, warp % 7, (double)h + (double)l);
                }
            } else {
                // a warp per particle: the particle's S partials are S x 64 contiguous
                // bytes, read with 16-byte loads (kFinLoads issued together). Lane l takes
                // components 2 (l % 4) and 2 (l % 4) + 1 of splits l / 4, l / 4 + 8, ... and
                // adds them in ascending split order; a fixed tree over the eight lanes of
                // each component pair (lane distance 4, 8, 16) finishes the sum.
                constexpr int kFinLoads = 16;
                const int qc = lane & 3, sub = lane >> 2;
                const int np = (int)(ib1 - ib0);
                for (int pi = warp; pi < np; pi += kThreads / 32) {
                    const int64_t ii = ib0 + pi;
                    const float4 *src = reinterpret_cast<const float4 *>(A.part) + ii * S * (kPartStride / 2) + qc;
                    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
                    for (int sp0 = sub; sp0 < S; sp0 += 8 * kFinLoads) {
                        float4 v[kFinLoads];
#pragma unroll
                        for (int u = 0; u < kFinLoads; ++u) {
                            const int sp = sp0 + 8 * u;
                            v[u] = sp < S ? __ldcg(src + (int64_t)sp * (kPartStride / 2)) : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int u = 0; u < kFinLoads; ++u)
                            if (sp0 + 8 * u < S) {
                                ds_add(h0, l0, v[u].x, v[u].y);
                                if (qc < 3) ds_add(h1, l1, v[u].z, v[u].w);   // component 7 is padding
                            }
                    }
#pragma unroll
                    for (int off = 4; off <= 16; off <<= 1) {
                        const float a0 = __shfl_xor_sync(0xffffffffu, h0, off), b0 = __shfl_xor_sync(0xffffffffu, l0, off);
                        const float a1 = __shfl_xor_sync(0xffffffffu, h1, off), b1 = __shfl_xor_sync(0xffffffffu, l1, off);
                        ds_add(h0, l0, a0, b0);
                        ds_add(h1, l1, a1, b1);
                    }
                    if (sub == 0) {
                        put_final(A, ii, 2 * qc, (double)h0 + (double)l0);
                        if (qc < 3) put_final(A, ii, 2 * qc + 1, (double)h1 + (double)l1);
                    }
                }
            }
        }
        if (threadIdx.x == 0) A.tickets[bx] = 0;
    }
    __syncthreads();
}

// ------------------------------------------------------- streamed variant
// TI = 1: all threads share the same R i-particles; each thread walks its own
// pair records straight from global memory (coalesced float4 loads), so no
// shared staging is needed. For small active blocks.
template <int R>
__device__ void work_stream(const ForceArgs &A, int64_t s, int64_t bx, int by, int S, Smem *sm)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tper = qdiv(A.tile_hi - A.tile_lo + S - 1, S);
    const int64_t t0 = A.tile_lo + (int64_t)by * tper;
    const int64_t t1 = t0 + tper < A.tile_hi ? t0 + tper : A.tile_hi;
    const int64_t p0 = t0 * kPT, p1 = t1 * kPT;
    // this thread's first pair record moves into L1 while the i-particle loads
    // are in flight (a prefetch holds no registers)
    if (p0 + tid < p1) {
        const char *a = reinterpret_cast<const char *>(A.j.p + p0 + tid);
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(a + 64));
    }
    IPk ip[R];
    int32_t gi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int64_t ii = bx * R + r;
        gi[r] = idx_at(A, sm, ii < s ? ii : s - 1);
        ip[r] = ipk_of(jrec_load(A.j.p, gi[r]));
    }
    const float2 e2 = make_float2(A.eps2f, A.eps2f);
    AccPk p[R];
    Acc7 hi[R], lo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { zero(p[r]); zero(hi[r]); zero(lo[r]); }
    // two pair records per thread in flight (their loads are issued together),
    // a fold after every kFoldPairs / 2 records
    int cnt = 0;
    for (int64_t pp = p0 + tid; pp < p1; pp += 2 * kThreads) {
        const int64_t pq = pp + kThreads < p1 ? pp + kThreads : pp;
        float4 a0, a1, a2, a3, a4, b0, b1, b2, b3, b4;
        {
            const float4 *q = A.j.p[pp].q;
            const float4 *w = A.j.p[pq].q;
            a0 = __ldg(q); a1 = __ldg(q + 1); a2 = __ldg(q + 2); a3 = __ldg(q + 3); a4 = __ldg(q + 4);
            b0 = __ldg(w); b1 = __ldg(w + 1); b2 = __ldg(w + 2); b3 = __ldg(w + 3); b4 = __ldg(w + 4);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
            pair_packed<true>(a0, a1, a2, a3, a4, ip[r], e2, p[r], 2 * pp == gi[r], 2 * pp + 1 == gi[r]);
        if (pq != pp) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                pair_packed<true>(b0, b1, b2, b3, b4, ip[r], e2, p[r], 2 * pq == gi[r], 2 * pq + 1 == gi[r]);
        }
        cnt += 2;
        if (cnt >= kFoldPairs / 2) {
            cnt = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);
    // fixed-order reduction: lanes (xor tree of two-sums), then warps in ascending order
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ds_group_reduce7<32>(hi[r], lo[r]);
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 7; ++c) sm->red[warp][r * 7 + c] = make_float2(acc_get(hi[r], c), acc_get(lo[r], c));
        }
    }
    __syncthreads();
    if (tid < R * 7) {
        float h = sm->red[0][tid].x, l = sm->red[0][tid].y;
#pragma unroll
        for (int wv = 1; wv < kThreads / 32; ++wv) ds_add(h, l, sm->red[wv][tid].x, sm->red[wv][tid].y);
        int r = tid / 7, c = tid % 7;
        int64_t ii = bx * R + r;
        if (ii < s) part2(A, ii, by, S)[c] = make_float2(h, l);
    }
    __syncthreads();
}

// --------------------------------------------------- TMA streaming variant
// TI = 1: all threads share one i-particle; the item's j-tiles stream through a
// ring of kRing shared-memory stages filled by the TMA bulk engine, so that
// kRing x 10 KB per CTA are in flight without holding registers (for blocks of
// one or two particles the evaluation is bound by reading the j-records). The
// two halves of the CTA take consecutive tiles, a thread one pair record of its
// half's tile.
__device__ __forceinline__ void issue_ring(const ForceArgs &A, Smem *sm, int64_t tile, int st)
{
    constexpr uint32_t bytes = kPT * sizeof(JPair);
    mbar_arrive_expect_tx(&sm->bar[st], bytes);
    bulk_g2s(sm->ring[st], A.j.p + tile * kPT, bytes, &sm->bar[st]);
}

__device__ void work_stream_tma(const ForceArgs &A, int64_t s, int64_t bx, int by, int S, Smem *sm, uint32_t &git)
{
    static_assert(kThreads == 2 * kPT, "each half of the CTA takes one tile");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t tper = qdiv(A.tile_hi - A.tile_lo + S - 1, S);
    const int64_t t0 = A.tile_lo + (int64_t)by * tper;
    const int64_t t1 = t0 + tper < A.tile_hi ? t0 + tper : A.tile_hi;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    if (tid == 0) {
        const int64_t pro = nt < kRing ? nt : kRing;
        for (int64_t q = 0; q < pro; ++q) issue_ring(A, sm, t0 + q, (int)((git + q) % kRing));
    }
    const int32_t gi = idx_at(A, sm, bx < s ? bx : s - 1);
    const IPk ip = ipk_of(jrec_load(A.j.p, gi));
    const float2 e2 = make_float2(A.eps2f, A.eps2f);
    const int half = tid / kPT, r = tid % kPT;
    AccPk p;
    Acc7 hi, lo;
    zero(p);
    zero(hi);
    zero(lo);
    int cnt = 0;
    for (int64_t q = 0; q < nt; q += 2) {
        const int64_t qh = q + half;
        if (qh < nt) {
            const uint32_t g = git + (uint32_t)qh;
            const int st = (int)(g % kRing);
            if (!mbar_wait(&sm->bar[st], (g / kRing) & 1u, A.spin_limit)) {
                sm->abort = 1;
            } else {
                const float4 *Q = sm->ring[st][r].q;
                const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3], q4 = Q[4];
                const int64_t ja = (t0 + qh) * kJT + 2 * r;
                pair_packed<true>(q0, q1, q2, q3, q4, ip, e2, p, ja == gi, ja + 1 == gi);
                if (++cnt == kFoldPairs / 2) {
                    cnt = 0;
                    fold(hi, lo, p);
                }
            }
        }
        __syncthreads();   // both tiles read: their stages may be refilled
        if (sm->abort) {
            // a wait ran out: drain what this CTA still has in flight (bounded), then stop
            // (tiles q .. q + kRing - 1 were issued; each wait is bounded)
            if (tid == 0) {
                for (int64_t qq = q; qq < nt && qq < q + kRing; ++qq) {
                    const uint32_t gg = git + (uint32_t)qq;
                    (void)mbar_wait(&sm->bar[gg % kRing], (gg / kRing) & 1u, A.spin_limit);
                }
            }
            git += (uint32_t)nt;
            return;
        }
        if (tid == 0) {
            for (int64_t qq = q + kRing; qq < q + kRing + 2 && qq < nt; ++qq)
                issue_ring(A, sm, t0 + qq, (int)((git + qq) % kRing));
        }
    }
    git += (uint32_t)nt;
    fold(hi, lo, p);
    // fixed-order reduction: lanes (xor tree of two-sums), then warps in ascending order
    ds_group_reduce7<32>(hi, lo);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 7; ++c) sm->red[warp][c] = make_float2(acc_get(hi, c), acc_get(lo, c));
    }
    __syncthreads();
    if (tid < 7) {
        float h = sm->red[0][tid].x, l = sm->red[0][tid].y;
#pragma unroll
        for (int wv = 1; wv < kThreads / 32; ++wv) ds_add(h, l, sm->red[wv][tid].x, sm->red[wv][tid].y);
        if (bx < s) part2(A, bx, by, S)[tid] = make_float2(h, l);
    }
    __syncthreads();
}

// ----------------------------------------------------------- tiled variant
// TI = kThreads / TJ thread groups, each holding R i-particles; the TJ threads
// of a group take interleaved pair records of each shared-memory tile.
template <int R, int TJ, bool MASK>
__device__ __forceinline__ void sweep_tile(const Smem *sm, int st, int tj, int64_t j0, const IPk *ip,
                                           const int32_t *gi, float2 e2, AccPk *p, Acc7 *hi, Acc7 *lo)
{
    constexpr int PPT = kPT / TJ;                           // pair records per thread per tile
    constexpr int FP = kFoldPairs / 2;                      // records per fold
    constexpr int CH = PPT < FP ? PPT : FP;
    const JPair *T = sm->tile[st];
#pragma unroll 1
    for (int c0 = 0; c0 < PPT; c0 += CH) {
#pragma unroll 4
        for (int u = 0; u < CH; ++u) {
            const int pp = tj + (c0 + u) * TJ;
            const float4 q0 = T[pp].q[0], q1 = T[pp].q[1], q2 = T[pp].q[2], q3 = T[pp].q[3], q4 = T[pp].q[4];
            const int64_t ja = j0 + 2 * pp;
#pragma unroll
            for (int r = 0; r < R; ++r)
                pair_packed<MASK>(q0, q1, q2, q3, q4, ip[r], e2, p[r], MASK && ja == gi[r], MASK && ja + 1 == gi[r]);
        }
        if (PPT >= FP) {
#pragma unroll
            for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);
        }
    }
}

__device__ __forceinline__ void issue_tile(const ForceArgs &A, Smem *sm, int64_t tile, int st)
{
    constexpr uint32_t bytes = kPT * sizeof(JPair);
    mbar_arrive_expect_tx(&sm->bar[st], bytes);
    bulk_g2s(sm->tile[st], A.j.p + tile * kPT, bytes, &sm->bar[st]);
}

template <int R, int TJ>
__device__ void work_tile(const ForceArgs &A, int64_t s, int64_t bx, int by, int S, Smem *sm, uint32_t &git)
{
    constexpr int TI = kThreads / TJ;
    constexpr int I = TI * R;
    constexpr int PPT = kPT / TJ;
    constexpr int kFoldTiles = PPT >= kFoldPairs / 2 ? 0 : (kFoldPairs / 2) / PPT;   // 0: folded inside the sweep
    static_assert(TJ <= 32 && (32 % TJ) == 0, "TJ must divide a warp");
    const int tid = threadIdx.x, tj = tid % TJ, ti = tid / TJ;
    const int64_t tper = qdiv(A.tile_hi - A.tile_lo + S - 1, S);
    const int64_t t0 = A.tile_lo + (int64_t)by * tper;
    const int64_t t1 = t0 + tper < A.tile_hi ? t0 + tper : A.tile_hi;
    const int64_t nt = t1 > t0 ? t1 - t0 : 0;
    // the first tiles are in flight before the i-particle loads
    if (tid == 0) {
        const int64_t pro = nt < kStages - 1 ? nt : kStages - 1;
        for (int64_t q = 0; q < pro; ++q) issue_tile(A, sm, t0 + q, (int)((git + q) % kStages));
    }

    IPk ip[R];
    int32_t gi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int64_t ii = bx * I + (int64_t)r * TI + ti;
        gi[r] = idx_at(A, sm, ii < s ? ii : s - 1);
        ip[r] = ipk_of(jrec_load(A.j.p, gi[r]));
    }
    const float2 e2 = make_float2(A.eps2f, A.eps2f);
    // index range of this i-block (the active list ascends), for self-exclusion
    const int64_t ib0 = bx * I;
    const int64_t ib1 = (ib0 + I < s ? ib0 + I : s) - 1;
    const int64_t imin = idx_at(A, sm, ib0), imax = idx_at(A, sm, ib1);

    AccPk p[R];
    Acc7 hi[R], lo[R];
#pragma unroll
    for (int r = 0; r < R; ++r) { zero(p[r]); zero(hi[r]); zero(lo[r]); }
    int fc = 0;
    for (int64_t q = 0; q < nt; ++q) {
        const uint32_t g = git + (uint32_t)q;
        const int st = (int)(g % kStages);
        if (tid == 0 && q + kStages - 1 < nt)
            issue_tile(A, sm, t0 + q + kStages - 1, (int)((g + kStages - 1) % kStages));
        if (!mbar_wait(&sm->bar[st], (g / kStages) & 1u, A.spin_limit)) sm->abort = 1;
        const int64_t j0 = (t0 + q) * kJT;
        if (j0 <= imax && j0 + kJT - 1 >= imin)
            sweep_tile<R, TJ, true>(sm, st, tj, j0, ip, gi, e2, p, hi, lo);
        else
            sweep_tile<R, TJ, false>(sm, st, tj, j0, ip, gi, e2, p, hi, lo);
        if (kFoldTiles > 0 && ++fc == kFoldTiles) {
            fc = 0;
#pragma unroll
            for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);
        }
        __syncthreads();
        if (sm->abort) {
            // a wait ran out: drain what this CTA still has in flight (bounded), then stop
            if (tid == 0) {
                for (int64_t qq = q + 1; qq < nt && qq < q + kStages; ++qq) {
                    const uint32_t gg = git + (uint32_t)qq;
                    (void)mbar_wait(&sm->bar[gg % kStages], (gg / kStages) & 1u, A.spin_limit);
                }
            }
            git += (uint32_t)nt;
            return;
        }
    }
    git += (uint32_t)nt;
#pragma unroll
    for (int r = 0; r < R; ++r) fold(hi[r], lo[r], p[r]);

#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (TJ > 1) ds_group_reduce7<TJ>(hi[r], lo[r]);
        const int64_t ii = bx * I + (int64_t)r * TI + ti;
        if (tj == 0 && ii < s) write_part(A, ii, by, S, hi[r], lo[r]);
    }
}

// -------------------------------------------------------------- variants

// 0: stream R=1 (I=1)      1: stream R=2 (I=2)      2: tile R=1 TJ=32 (I=8)
// 3: tile R=1 TJ=8 (I=32)  4: tile R=1 TJ=1 (I=256) 5: TMA stream R=1 (I=1)
// 6: resident share (cluster launch; the split factor is unused)
constexpr int kMixedFallback = kMixedFallbackId;   // the variant of an out-of-range table entry
constexpr int kShareVariant = kShareVariantId;
__host__ __device__ __forceinline__ int mixed_I(int v)
{
    switch (v) {
    case 0: return 1;
    case 1: return 2;
    case 2: return 8;
    case 3: return 32;
    case 5: return 1;
    case 6: return 1;
    default: return 256;
    }
}

// ------------------------------------------------- resident-share variant
// For j ranges of up to kShareC * kShareRec pair records. The launch runs as
// clusters of kShareC CTAs; CTA r of a cluster copies records [r * rper, (r + 1)
// * rper) of the range into shared memory once (bulk copies on one mbarrier),
// padded with far-away massless records to whole rounds of 32. The clusters deal
// out the active list in chunks (chunk k to cluster k mod clusters); every CTA of
// the cluster runs the whole chunk against its share in passes whose group
// width TJ fits the remaining count, leaving (hi, lo) partials in its shared
// memory. After a cluster barrier, CTA r sums positions r, r + kShareC, ... of
// the chunk over the kShareC CTAs in rank order through distributed shared
// memory and writes the FP64 results; a second barrier frees the slots. No
// global partial slots, tickets or fences; the same bits on every run.

// rper: records per CTA, a multiple of 32 (0 when the range does not fit)
__device__ __forceinline__ int64_t share_rper(const ForceArgs &A)
{
    const int64_t nrec = (A.tile_hi - A.tile_lo) * kPT;
    const int64_t rper = ((nrec + kShareC - 1) / kShareC + 31) / 32 * 32;
    return rper <= kShareRec ? rper : 0;
}

// One pass: cnt particles from list position p0 into slots slot0 ..., TJ threads
// per particle taking records tj, tj + TJ, ... of the share (nr rounds).
template <int TJ>
__device__ __forceinline__ void share_pass(const ForceArgs &A, Smem *sm, int64_t p0, int cnt, int slot0,
                                           int64_t rec0, int nrec, int nr)
{
    constexpr int FP = kFoldPairs / 2;   // records per fold
    const int tid = threadIdx.x, tj = tid % TJ, ti = tid / TJ;
    const bool live = ti < cnt;
    const int32_t gi = idx_at(A, sm, p0 + (live ? ti : cnt - 1));
    const IPk ip = ipk_of(jrec_load(A.j.p, gi));
    const float2 e2 = make_float2(A.eps2f, A.eps2f);
    AccPk p;
    Acc7 hi, lo;
    zero(p);
    zero(hi);
    zero(lo);
    // i's place in the share, if it is there (else a value no record matches);
    // one loop with the self test in it keeps the code small: each launch runs
    // its passes once, from a cold instruction cache
    const int64_t self = (int64_t)gi - 2 * rec0;
    const int selfi = self >= 0 && self < 2 * (int64_t)nrec ? (int)self : -2;
    const JPair *R = shb(sm)->rec;
    for (int k0 = 0; k0 < nr; k0 += FP) {
        const int k1 = k0 + FP < nr ? k0 + FP : nr;
#pragma unroll 2
        for (int k = k0; k < k1; ++k) {
            const int pp = tj + k * TJ;
            const float4 *Q = R[pp].q;
            pair_packed<true>(Q[0], Q[1], Q[2], Q[3], Q[4], ip, e2, p, 2 * pp == selfi, 2 * pp + 1 == selfi);
        }
        fold(hi, lo, p);
    }
    if (TJ > 1) ds_group_reduce7<TJ>(hi, lo);
    if (tj == 0 && live) {
#pragma unroll
        for (int c = 0; c < 7; ++c) shb(sm)->slot[slot0 + ti][c] = make_float2(acc_get(hi, c), acc_get(lo, c));
    }
}

// A pass for cnt <= 4 particles with 256 / cnt threads each (whole warps): lanes
// then warps of a particle summed in ascending order.
__device__ __forceinline__ void share_pass_wide(const ForceArgs &A, Smem *sm, int64_t p0, int cnt, int slot0,
                                                int64_t rec0, int nrec, int nrec32)
{
    constexpr int FP = kFoldPairs / 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int W = cnt == 1 ? 8 : (cnt == 2 ? 4 : 2);   // warps per particle
    const int TW = 32 * W;                            // threads per particle
    const int ti = tid / TW, tj = tid % TW;
    const bool live = ti < cnt;
    const int32_t gi = idx_at(A, sm, p0 + (live ? ti : cnt - 1));
    const IPk ip = ipk_of(jrec_load(A.j.p, gi));
    const float2 e2 = make_float2(A.eps2f, A.eps2f);
    AccPk p;
    Acc7 hi, lo;
    zero(p);
    zero(hi);
    zero(lo);
    const int64_t self = (int64_t)gi - 2 * rec0;
    const int selfi = self >= 0 && self < 2 * (int64_t)nrec ? (int)self : -2;
    const JPair *R = shb(sm)->rec;
    const int nr = (nrec32 + TW - 1) / TW;
    int f = 0;
    for (int k = 0; k < nr; ++k) {
        const int pp = tj + k * TW;
        if (pp < nrec32) {
            const float4 *Q = R[pp].q;
            pair_packed<true>(Q[0], Q[1], Q[2], Q[3], Q[4], ip, e2, p, 2 * pp == selfi, 2 * pp + 1 == selfi);
        }
        if (++f == FP) {
            f = 0;
            fold(hi, lo, p);
        }
    }
    fold(hi, lo, p);
    ds_group_reduce7<32>(hi, lo);
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < 7; ++c) sm->red[warp][c] = make_float2(acc_get(hi, c), acc_get(lo, c));
    }
    __syncthreads();
    if (tid < cnt * 7) {
        const int t = tid / 7, c = tid % 7;
        float h = sm->red[t * W][c].x, l = sm->red[t * W][c].y;
        for (int wv = 1; wv < W; ++wv) ds_add(h, l, sm->red[t * W + wv][c].x, sm->red[t * W + wv][c].y);
        shb(sm)->slot[slot0 + t][c] = make_float2(h, l);
    }
    __syncthreads();
}

// The whole launch of the resident-share variant for this CTA.
__device__ __noinline__ void share_force(const ForceArgs &A, int64_t s, Smem *sm, int64_t rper)
{
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int q = blockIdx.x / kShareC, ncl = gridDim.x / kShareC;
    const int tid = threadIdx.x;
    const int64_t rtot = (A.tile_hi - A.tile_lo) * kPT;
    const int64_t rec0 = A.tile_lo * kPT + (int64_t)rank * rper;
    const int64_t rlim = A.tile_lo * kPT + rtot;
    const int nrec = (int)(rec0 < rlim ? (rlim - rec0 < rper ? rlim - rec0 : rper) : 0);
    const int nrec32 = (nrec + 31) / 32 * 32;
    // chunks: ceil(s / clusters) particles each (at most kShareSlots)
    int64_t csz = (s + ncl - 1) / ncl;
    if (csz > kShareSlots) csz = kShareSlots;
    const int64_t nchunk = (s + csz - 1) / csz;
    if (q >= nchunk) return;   // the whole cluster has nothing to do (uniform over it)
    // the share: bulk copies of at most 16 KB on one mbarrier, padding by the threads
    bool ok = true;
    if (nrec > 0) {
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)nrec * (uint32_t)sizeof(JPair);
            mbar_arrive_expect_tx(&sm->bar[0], bytes);
            constexpr int kPiece = 200;   // records per copy (16000 bytes)
            for (int r0 = 0; r0 < nrec; r0 += kPiece) {
                const int nr = nrec - r0 < kPiece ? nrec - r0 : kPiece;
                bulk_g2s(shb(sm)->rec + r0, A.j.p + rec0 + r0, (uint32_t)nr * (uint32_t)sizeof(JPair), &sm->bar[0]);
            }
        }
    }
    {
        const float far = (float)kPadPos;
        for (int qq = 2 * nrec + tid; qq < 2 * nrec32; qq += kThreads)
            jrec_store(shb(sm)->rec, qq, far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
    }
    if (nrec > 0 && !mbar_wait(&sm->bar[0], 0, A.spin_limit)) {
        ok = false;
        if (tid == 0) atomicOr(A.status, kStTimeout);
    }
    __syncthreads();
    for (int64_t k = q; k < nchunk; k += ncl) {
        const int64_t c0 = k * csz;
        const int cnt = (int)(c0 + csz < s ? csz : s - c0);
        if (ok) {
            int done = 0;
            while (done < cnt) {
                const int r = cnt - done;
                if (r >= 256) {
                    share_pass<1>(A, sm, c0 + done, 256, done, rec0, nrec, nrec32);
                    done += 256;
                } else if (r >= 128) {
                    share_pass<2>(A, sm, c0 + done, 128, done, rec0, nrec, nrec32 / 2);
                    done += 128;
                } else if (r >= 64) {
                    share_pass<4>(A, sm, c0 + done, 64, done, rec0, nrec, nrec32 / 4);
                    done += 64;
                } else if (r >= 32) {
                    share_pass<8>(A, sm, c0 + done, 32, done, rec0, nrec, nrec32 / 8);
                    done += 32;
                } else if (r > 8) {
                    const int n16 = r < 16 ? r : 16;
                    share_pass<16>(A, sm, c0 + done, n16, done, rec0, nrec, nrec32 / 16);
                    done += n16;
                } else if (r > 4) {
                    share_pass<32>(A, sm, c0 + done, r, done, rec0, nrec, nrec32 / 32);
                    done += r;
                } else {
                    share_pass_wide(A, sm, c0 + done, r, done, rec0, nrec, nrec32);
                    done += r;
                }
            }
        } else {
            for (int qq = tid; qq < cnt * 7; qq += kThreads)
                shb(sm)->slot[qq / 7][qq % 7] = make_float2(0.f, 0.f);
        }
        cl.sync();
        // rank r sums positions r, r + kShareC, ...: one (position, component) per thread
        for (int t = tid; t < ((cnt + kShareC - 1) / kShareC) * 7; t += kThreads) {
            const int pl = rank + kShareC * (t / 7), c = t % 7;
            if (pl < cnt) {
                float2 v[kShareC];
#pragma unroll
                for (int u = 0; u < kShareC; ++u) v[u] = *cl.map_shared_rank(&shb(sm)->slot[pl][c], u);
                float h = 0.f, l = 0.f;
#pragma unroll
                for (int u = 0; u < kShareC; ++u) ds_add(h, l, v[u].x, v[u].y);
                put_final(A, c0 + pl, c, (double)h + (double)l);
            }
        }
        cl.sync();
    }
    if (!ok && nrec > 0 && tid == 0) (void)mbar_wait(&sm->bar[0], 0, A.spin_limit);   // drain before exit
}

// SHARE: the instantiation with the resident-share variant (launched as clusters
// with kSmemShare bytes); without it the kernel has no cluster code and the
// plain shared-memory size.
template <bool SHARE>
__global__ void __launch_bounds__(kThreads, 2) force_mixed_kernel(ForceArgs A)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem *sm = reinterpret_cast<Smem *>(smem_raw);
    const int tid = threadIdx.x;
    // a launch that depends on this one programmatically (the nb_run loop's
    // corrector) may start now: it reads only what was written before this kernel
    // until it waits for this grid's completion
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    // read ahead of s: entries past s are stale and never used (idx_cap >= s)
    const int32_t ipre = tid < A.idx_cap ? A.idx[tid] : 0;
    if (tid == 0) {
        for (int st = 0; st < kRing; ++st) mbar_init(&sm->bar[st], 1);
        mbar_init(&sm->inject_bar, 1);
        fence_mbar_init();
        sm->abort = 0;
        sm->s = launch_s(A);
    }
    // the active count and the whole tuning table in one round trip
    if (A.force_variant < 0 && tid < 2 * kBuckets) {
        if (tid < kBuckets)
            sm->tune.variant[tid] = A.tune->variant[tid];
        else
            sm->tune.split[tid - kBuckets] = A.tune->split[tid - kBuckets];
    }
    sm->idx_pre[tid] = ipre;
    __syncthreads();
    const int64_t s = sm->s;
    if (s <= 0) return;
    copy_list(A, s);
    if (A.inject) {
        // Test hook: wait on a barrier that no one arrives on; the spin limit must
        // expire and the kernel must report it. No copy is in flight here.
        if (!mbar_wait(&sm->inject_bar, 0, A.spin_limit) && tid == 0) atomicOr(A.status, kStTimeout);
        return;
    }
    int variant, S;
    if (A.force_variant >= 0) {
        variant = A.force_variant;
        S = A.force_split;
    } else {
        const int b = bucket_of(s);
        variant = sm->tune.variant[b];
        if (variant < 0 || variant >= kMixedVariants) variant = kMixedFallback;
        S = table_split(sm->tune.split[b], b, s, A.n, mixed_I(variant));
    }
    if (variant < 0 || variant >= kMixedVariants) variant = kMixedFallback;
    if (variant == kShareVariant) {
        // needs the cluster launch and a j range that fits the shares (the same
        // answer in every CTA of a cluster)
        if constexpr (SHARE) {
            const int64_t rper = share_rper(A);
            if (cg::this_cluster().num_blocks() == kShareC && rper > 0) {
                if (blockIdx.x == 0 && tid == 0) *A.split_used = kShareC;
                share_force(A, s, sm, rper);
                return;
            }
        }
        variant = kMixedFallback;   // (a launch without clusters: one split)
        S = 1;
    }
    S = clamp_split(S, A.tile_hi - A.tile_lo, s, A.part_cap);
    if (blockIdx.x == 0 && tid == 0) *A.split_used = S;
    const int64_t I = mixed_I(variant);
    const int64_t nib = qdiv(s + I - 1, I);
    const int64_t W = nib * S;
    uint32_t git = 0;
    for (int64_t w = blockIdx.x; w < W; w += gridDim.x) {
        const int64_t bx = qdiv(w, S);
        const int by = (int)(w - bx * S);
        switch (variant) {
        case 0: work_stream<1>(A, s, bx, by, S, sm); break;
        case 1: work_stream<2>(A, s, bx, by, S, sm); break;
        case 2: work_tile<1, 32>(A, s, bx, by, S, sm, git); break;
        case 3: work_tile<1, 8>(A, s, bx, by, S, sm, git); break;
        case 5: work_stream_tma(A, s, bx, by, S, sm, git); break;
        default: work_tile<1, 1>(A, s, bx, by, S, sm, git); break;
        }
        if (sm->abort) {
            if (tid == 0) atomicOr(A.status, kStTimeout);
            return;
        }
        finish_item(A, s, bx, S, I, sm);
    }
}

// ------------------------------------------------------------ FP64 kernels
// The plain FP64 path: same decomposition, double arithmetic throughout and
// j-data read through the read-only cache (all lanes of a warp read the same
// j in the i-loop variant, one broadcast transaction).

__device__ __forceinline__ void pair_f64(double xj, double yj, double zj, double mj, double vxj, double vyj,
                                         double vzj, const double *xi, double eps2, double *acc, bool self)
{
    double dx = xj - xi[0], dy = yj - xi[1], dz = zj - xi[2];
    double wx = vxj - xi[3], wy = vyj - xi[4], wz = vzj - xi[5];
    double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    double rw = fma(dx, wx, fma(dy, wy, dz * wz));
    double q = self ? 0.0 : rsqrt(r2);
    double q2 = q * q;
    double mq = mj * q;
    double mu = mq * q2;
    double al = 3.0 * rw * q2;
    acc[6] -= mq;
    acc[0] = fma(mu, dx, acc[0]);
    acc[1] = fma(mu, dy, acc[1]);
    acc[2] = fma(mu, dz, acc[2]);
    acc[3] = fma(mu, fma(-al, dx, wx), acc[3]);
    acc[4] = fma(mu, fma(-al, dy, wy), acc[4]);
    acc[5] = fma(mu, fma(-al, dz, wz), acc[5]);
}

__device__ __forceinline__ void load_i64(const ForceArgs &A, int32_t i, double *xi)
{
    const int64_t np = A.n_tiles * kJT;
    xi[0] = A.xp[i]; xi[1] = A.xp[np + i]; xi[2] = A.xp[2 * np + i];
    xi[3] = A.vp[i]; xi[4] = A.vp[np + i]; xi[5] = A.vp[2 * np + i];
}

__device__ void work_f64_stream(const ForceArgs &A, int64_t s, int64_t bx, int by, int S, double (*red)[7])
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t gi = A.idx[bx < s ? bx : s - 1];
    double xi[6];
    load_i64(A, gi, xi);
    const int64_t np = A.n_tiles * kJT;
    const int64_t tper = qdiv(A.tile_hi - A.tile_lo + S - 1, S);
    const int64_t t0 = A.tile_lo + (int64_t)by * tper;
    const int64_t t1 = t0 + tper < A.tile_hi ? t0 + tper : A.tile_hi;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t j = t0 * kJT + tid; j < t1 * kJT; j += kThreads)
        pair_f64(__ldg(A.xp + j), __ldg(A.xp + np + j), __ldg(A.xp + 2 * np + j), __ldg(A.m + j),
                 __ldg(A.vp + j), __ldg(A.vp + np + j), __ldg(A.vp + 2 * np + j), xi, A.eps2, acc, j == gi);
#pragma unroll
    for (int c = 0; c < 7; ++c) {
        double x = acc[c];
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
        if (lane == 0) red[warp][c] = x;
    }
    __syncthreads();
    if (tid < 7) {
        double x = 0.0;
        for (int wv = 0; wv < kThreads / 32; ++wv) x += red[wv][tid];
        if (bx < s) A.part[(bx * S + by) * kPartStride + tid] = x;
    }
    __syncthreads();
}

__device__ void work_f64_iloop(const ForceArgs &A, int64_t s, int64_t bx, int by, int S)
{
    const int tid = threadIdx.x;
    const int64_t ii = bx * kThreads + tid;
    const int32_t gi = A.idx[ii < s ? ii : s - 1];
    double xi[6];
    load_i64(A, gi, xi);
    const int64_t np = A.n_tiles * kJT;
    const int64_t tper = qdiv(A.tile_hi - A.tile_lo + S - 1, S);
    const int64_t t0 = A.tile_lo + (int64_t)by * tper;
    const int64_t t1 = t0 + tper < A.tile_hi ? t0 + tper : A.tile_hi;
    double acc[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int64_t j = t0 * kJT; j < t1 * kJT; ++j)
        pair_f64(__ldg(A.xp + j), __ldg(A.xp + np + j), __ldg(A.xp + 2 * np + j), __ldg(A.m + j),
                 __ldg(A.vp + j), __ldg(A.vp + np + j), __ldg(A.vp + 2 * np + j), xi, A.eps2, acc, j == gi);
    if (ii < s) {
        double *dst = A.part + (ii * S + by) * kPartStride;
        for (int c = 0; c < 7; ++c) dst[c] = acc[c];
    }
}

// FP64 counterpart of finish_item: FP64 sums in split order.
__device__ void finish_item_f64(const ForceArgs &A, int64_t s, int64_t bx, int S, int64_t I, int *last)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(&A.tickets[bx], 1);
        *last = (t == S - 1);
    }
    __syncthreads();
    if (*last) {
        __threadfence();
        const int64_t ib0 = bx * I;
        const int64_t ib1 = ib0 + I < s ? ib0 + I : s;
        const int64_t cnt = (ib1 - ib0) * 7;
        for (int64_t q = threadIdx.x; q < cnt; q += kThreads) {
            const int64_t ii = ib0 + q / 7;
            const int c = (int)(q % 7);
            const double *src = A.part + ii * S * kPartStride + c;
            double x = 0.0;
            // eight loads in flight, added in split order
            for (int sp0 = 0; sp0 < S; sp0 += 8) {
                double v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) v[u] = sp0 + u < S ? __ldcg(src + (sp0 + u) * kPartStride) : 0.0;
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (sp0 + u < S) x += v[u];
            }
            put_final(A, ii, c, x);
        }
        if (threadIdx.x == 0) A.tickets[bx] = 0;
    }
    __syncthreads();
}

__host__ __device__ __forceinline__ int f64_I(int v) { return v == 0 ? 1 : kThreads; }

__global__ void __launch_bounds__(kThreads) force_f64_kernel(ForceArgs A)
{
    __shared__ double red[kThreads / 32][7];
    __shared__ uint64_t inject_bar;
    __shared__ int last;
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int64_t s = launch_s(A);
    if (s <= 0) return;
    copy_list(A, s);
    if (A.inject) {
        if (threadIdx.x == 0) {
            mbar_init(&inject_bar, 1);
            fence_mbar_init();
        }
        __syncthreads();
        if (!mbar_wait(&inject_bar, 0, A.spin_limit) && threadIdx.x == 0) atomicOr(A.status, kStTimeout);
        return;
    }
    int variant, S;
    if (A.force_variant >= 0) {
        variant = A.force_variant;
        S = A.force_split;
    } else {
        const int b = bucket_of(s);
        variant = A.tune->variant[b];
        if (variant < 0 || variant >= kF64Variants) variant = kF64Variants - 1;
        S = table_split(A.tune->split[b], b, s, A.n, f64_I(variant));
    }
    if (variant < 0 || variant >= kF64Variants) variant = kF64Variants - 1;
    S = clamp_split(S, A.tile_hi - A.tile_lo, s, A.part_cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *A.split_used = S;
    const int64_t I = f64_I(variant);
    const int64_t W = qdiv(s + I - 1, I) * S;
    for (int64_t w = blockIdx.x; w < W; w += gridDim.x) {
        const int64_t bx = qdiv(w, S);
        const int by = (int)(w - bx * S);
        if (variant == 0)
            work_f64_stream(A, s, bx, by, S, red);
        else
            work_f64_iloop(A, s, bx, by, S);
        finish_item_f64(A, s, bx, S, I, &last);
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

int mixed_variant_I(int v) { return mixed_I(v); }

const char *mixed_variant_name(int v)
{
    switch (v) {
    case 0: return "stream R=1";
    case 1: return "stream R=2";
    case 2: return "tile R=1 TJ=32";
    case 3: return "tile R=1 TJ=8";
    case 4: return "tile R=1 TJ=1";
    case 5: return "TMA stream R=1";
    case 6: return "resident share (8-CTA clusters)";
    default: return "?";
    }
}

int f64_variant_I(int v) { return f64_I(v); }

const char *f64_variant_name(int v) { return v == 0 ? "f64 stream" : "f64 i-loop"; }

size_t force_mixed_smem_bytes() { return sizeof(Smem); }

static int g_mixed_occ = -1, g_f64_occ = -1, g_mixed_grid = -1;

int force_mixed_ctas_per_sm()
{
    if (g_mixed_occ < 0) {
        cudaFuncSetAttribute(force_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(Smem));
        cudaFuncSetAttribute(force_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSmemShare);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, force_mixed_kernel<false>, kThreads, sizeof(Smem)) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
        g_mixed_occ = occ;
    }
    return g_mixed_occ;
}

// For particle counts whose j-records fit the resident shares of one cluster,
// the mixed kernel runs as clusters of kShareC CTAs (the resident-share variant
// needs them; the others ignore them). Its persistent grid is then the number of
// clusters the device keeps resident at once times kShareC, so that no CTA of
// the grid waits for another to finish (a CTA of a late cluster would hold its
// work items until then); 0 when cluster launches are not available. Larger
// particle counts (and that case) launch SMs x resident CTAs without clusters.
static int mixed_cluster_grid()
{
    if (g_mixed_grid < 0) {
        (void)force_mixed_ctas_per_sm();
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kShareC;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(kShareC * 64);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmemShare;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, force_mixed_kernel<true>, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            ncl = 0;
        }
        g_mixed_grid = ncl * kShareC;
    }
    return g_mixed_grid;
}

bool mixed_share_fits(int64_t n_tiles)
{
    const int64_t rper = ((n_tiles * kPT + kShareC - 1) / kShareC + 31) / 32 * 32;
    return rper <= kShareRec && mixed_cluster_grid() > 0;
}

int force_mixed_grid(int num_sms, int64_t n_tiles)
{
    return mixed_share_fits(n_tiles) ? mixed_cluster_grid() : num_sms * force_mixed_ctas_per_sm();
}

int force_f64_ctas_per_sm()
{
    if (g_f64_occ < 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, force_f64_kernel, kThreads, 0) != cudaSuccess ||
            occ < 1)
            occ = 1;
        g_f64_occ = occ;
    }
    return g_f64_occ;
}

cudaError_t launch_force_mixed(const ForceArgs &a, int grid, cudaStream_t st)
{
    (void)force_mixed_ctas_per_sm();   // sets the dynamic shared-memory attribute once
    if (mixed_share_fits(a.n_tiles) && grid % kShareC == 0) {
        cudaLaunchConfig_t cfg{};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kShareC;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kThreads);
        cfg.dynamicSmemBytes = kSmemShare;
        cfg.stream = st;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, force_mixed_kernel<true>, a);
    }
    force_mixed_kernel<false><<<grid, kThreads, sizeof(Smem), st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_force_f64(const ForceArgs &a, int grid, cudaStream_t st)
{
    force_f64_kernel<<<grid, kThreads, 0, st>>>(a);
    return cudaGetLastError();
}

// Work items are i-blocks x j-splits over a grid of R = SMs x resident CTAs;
// a launch takes ceil(W / R) waves of items, so W just above a multiple of R
// wastes most of a wave. One full wave (S = R / nib) unless items would then be
// long (64 tiles or more): then the split in [S, 4 S] whose items fill their
// waves best. At least 4 tiles per item.
int64_t wave_split(int64_t nib, int64_t n_tiles, int64_t resident)
{
    int64_t S = std::max<int64_t>(1, resident / nib);
    if (n_tiles / S >= 64) {
        int64_t best = S;
        double best_eff = 0.0;
        for (int64_t c = S; c <= 4 * S; ++c) {
            const int64_t W = nib * c;
            const double eff = (double)W / (double)(((W + resident - 1) / resident) * resident);
            if (eff > best_eff + 1e-9) {
                best_eff = eff;
                best = c;
            }
        }
        S = best;
    }
    S = std::min<int64_t>(S, std::max<int64_t>(1, n_tiles / 4));
    return std::max<int64_t>(1, std::min<int64_t>(S, n_tiles));
}

void default_tuning(int precision, int64_t n, int64_t s, int num_sms, int ctas_per_sm, int *variant, int *split)
{
    const int64_t n_tiles = (n + kJT - 1) / kJT;
    const int64_t resident = (int64_t)num_sms * ctas_per_sm;
    int v;
    if (precision == NB_PREC_FP64) {
        v = s <= 64 ? 0 : 1;
    } else if (mixed_share_fits(n_tiles) && s > 16 && s <= 8192) {
        // the j-records fit the resident shares of a cluster: no split partials in L2
        v = kShareVariant;
    } else if (n <= 65536) {
        // j-records stay in L2 and are cheap to re-read: stream variants (every
        // thread of a CTA on the same 1 or 2 i-particles) win while blocks are small
        v = s <= (n <= 32768 ? 64 : 16) ? 0 : s <= 1024 ? 1 : s <= 1536 ? 2 : s <= 12288 ? 3 : 4;
    } else {
        // large N: re-reading all j per i-particle costs more than it hides
        v = s <= 1 ? 0 : s <= 4 ? 1 : s <= 32 ? 2 : s <= 512 ? 3 : 4;
    }
    const int64_t I = precision == NB_PREC_FP64 ? f64_I(v) : mixed_I(v);
    *variant = v;
    *split = (int)wave_split((s + I - 1) / I, n_tiles, resident);
}

}  // namespace nb
