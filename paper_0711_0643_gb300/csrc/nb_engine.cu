// Small-block engine: consecutive block steps with small active blocks, each a
// full step of Sect. 2.1 (selection by the smallest t_i + dt_i, Hermite
// predictor for all particles, Eq. (Force) with its jerk and potential on the
// block, corrector and Eq. (timestep) quantised to powers of two), run inside
// one kernel by one thread-block cluster.
//
// Why: with a few active particles a block step is a chain of dependent phases
// whose arithmetic is small; as four kernels per step (selection, predictor,
// force, corrector) the launch gaps and the kernels' own start-up dominate. The
// cluster keeps the whole chain on chip and replaces each kernel boundary by a
// hardware cluster barrier.
//
// Decomposition (the paper's j-parallelisation, Sect. 3, on the cluster's CTAs):
// CTA r owns the particles [r c, (r + 1) c) (c = chunk). Per step it
//   1. finds its chunk's members of the block (keys t + dt equal to the block
//      time; ascending) and the smallest other key; pushes its member count into
//      every CTA's shared memory;
//   2. predicts its members to the block time (the double-single predictor of
//      the full path, same bits) and pushes their records to every CTA;
//   -- cluster barrier: every CTA knows every chunk's count, hence the block
//      size s and each chunk's offset; if the block is too large for the engine
//      (s > s_max, or more than kEngCap members in one chunk), past t_end, or
//      the step budget is used up, every CTA stops here, leaving the block time
//      for the full path;
//   3. predicts its whole chunk into pair records in shared memory, orders the
//      s members it received, and sums their forces over its own chunk only
//      (packed f32x2 pair arithmetic, two-sum folds and reductions: the force
//      kernel's arithmetic), pushing the (hi, lo) partial sums to each member's
//      owner;
//   -- cluster barrier;
//   4. corrects its own members: four lanes per particle add the C partial sums
//      in rank order (the paper's global sum of partial forces, in a fixed order)
//      and run the FP64 corrector, Aarseth step and quantisation of the full path
//      (same bits given the same forces); the smallest key of its chunk after the
//      step is pushed into every CTA;
//   -- cluster barrier: the smallest of those is the next block time.
// Each CTA keeps its chunk's double-single state, times and keys in shared memory
// for the whole launch (loaded once; the corrector updates its members' copies as
// it writes the FP64 state), so the per-step selection and prediction read only
// shared memory and run on the FP32 pipe (the time differences t_block - t_j in
// double-single: FP64 is a narrow pipe on this part).
// No software spin-wait exists: every branch is taken identically by all CTAs
// (each decision uses values every CTA holds), so every CTA reaches every
// barrier. Results are bitwise reproducible and do not depend on how many steps
// one launch takes (nb_step runs the engine for one step, nb_run until a block
// it does not take).
//
// This file is compiled with -fmad=false (the FP64 corrector rounds like the
// CPU oracle); the FP32 pair arithmetic uses explicit fused multiply-adds.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "nb_ds.cuh"
#include "nb_hermite.cuh"
#include "nb_internal.cuh"
#include "nb_pair.cuh"

namespace cg = cooperative_groups;

namespace nb {
namespace {

constexpr int kEngThreads = 512;
constexpr int kEngWarps = kEngThreads / 32;
constexpr int kEngMaxC = 16;
constexpr long long kInfBits = 0x7ff0000000000000LL;
static_assert(kEngCap <= 8 * (kEngWarps - 1), "the last warp must hold no member (four lanes per member)");
static_assert(kEngMaxC * kEngCap <= kEngThreads, "one thread per (rank, member) when pushing records");

// predicted record of an active particle: (x_hi, y_hi, z_hi, index bits), (x_lo, y_lo, z_lo, 0), (vx, vy, vz, 0)
struct __align__(16) IRec {
    float4 h, l, w;
};

// Shared memory of one CTA. Everything another CTA needs is pushed into the
// reader's shared memory (distributed shared-memory stores) before a cluster
// barrier, so every read after a barrier is local.
struct __align__(16) EngSmem {
    IRec inbox[kEngMaxC][kEngCap];          // [q][k]: member k of rank q's chunk, pushed by rank q
    IRec ilist[kEngMaxS];                   // all members in block order (copied from the inbox)
    float2 part_in[kEngCap][kEngMaxC][8];   // [k][q]: rank q's partial sums (hi, lo) for this chunk's member k
    int2 qmap[kEngMaxS];                    // block position -> (owner rank, member index there)
    IRec own_rec[kEngCap];                  // this chunk's members' predicted records
    int own_idx[kEngCap];                   // this chunk's members (particle indices, ascending)
    int rank_base[kEngMaxC];                // block position of each rank's first member
    float2 red[kEngWarps][7];               // per-warp sums (blocks of up to 16)
    long long slot_min[kEngMaxC];           // written by rank q: the smallest key of its chunk after the step
    int slot_err[kEngMaxC];                 // written by rank q: its status bits of the step
    int slot_cnt[kEngMaxC];                 // written by rank q: its chunk's members of the block
    int wcnt[kEngWarps];
    long long wmin[kEngWarps];
    int wflags[kEngWarps];
};

__device__ __forceinline__ long long min_ll(long long a, long long b) { return a < b ? a : b; }

__device__ __forceinline__ long long warp_min(long long v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = min_ll(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

__device__ __forceinline__ IPk ipk_of_rec(const IRec &R)
{
    return ipk_of(IPart{R.h.x, R.h.y, R.h.z, R.l.x, R.l.y, R.l.z, R.w.x, R.w.y, R.w.z});
}

// Sends the (hi, lo) partial sums of block position q to the member's owner.
__device__ __forceinline__ void push_part(cg::cluster_group &cluster, EngSmem *sm, int q, int rank, const Acc7 &hi,
                                          const Acc7 &lo)
{
    const int2 o = sm->qmap[q];
    float2 *dst = cluster.map_shared_rank(&sm->part_in[o.y][rank][0], o.x);
#pragma unroll
    for (int c = 0; c < 7; ++c) dst[c] = make_float2(acc_get(hi, c), acc_get(lo, c));
}

// Partial sums of one member (predicted record ip, index gi) over pair records
// [rb, re) of the chunk, lanes interleaved with stride TJ starting at lane tj.
// MASK: the member's own pair is left out by index (the engine always masks: one
// instantiation per width keeps the kernel's code, and its instruction-cache
// footprint, small).
template <bool MASK, int TJ>
__device__ __forceinline__ void sweep(const JPair *recs, int64_t j0, int rb, int re, int tj, const IPk &ip, int gi,
                                      float2 e2, Acc7 &hi, Acc7 &lo)
{
    AccPk p;
    zero(p);
    int cnt = 0;
#pragma unroll 4
    for (int r = rb + tj; r < re; r += TJ) {
        const float4 *Q = recs[r].q;
        const float4 q0 = Q[0], q1 = Q[1], q2 = Q[2], q3 = Q[3], q4 = Q[4];
        const int64_t ja = j0 + 2 * (int64_t)r;
        pair_packed<MASK>(q0, q1, q2, q3, q4, ip, e2, p, MASK && ja == gi, MASK && ja + 1 == gi);
        if (++cnt == kFoldPairs / 2) {
            cnt = 0;
            fold(hi, lo, p);
        }
    }
    fold(hi, lo, p);
}

// Blocks of more than 16: TJ lanes per member (TJ = 8), each CTA thread group
// takes members in rounds; the group's lanes reduce with two-sums in a fixed order.
template <int TJ>
__device__ void force_groups(cg::cluster_group &cluster, EngSmem *sm, const JPair *recs, int64_t j0, int64_t j1,
                             int nrec, int s, float2 e2, int rank)
{
    constexpr int kGroups = kEngThreads / TJ;
    const int tid = threadIdx.x, tj = tid % TJ, g = tid / TJ;
    for (int base = 0; base < s; base += kGroups) {
        const int q = base + g;
        const int qq = q < s ? q : s - 1;
        const IRec R = sm->ilist[qq];
        const int gi = __float_as_int(R.h.w);
        const IPk ip = ipk_of_rec(R);
        Acc7 hi, lo;
        zero(hi);
        zero(lo);
        sweep<true, TJ>(recs, j0, 0, nrec, tj, ip, gi, e2, hi, lo);
        ds_group_reduce7<TJ>(hi, lo);
        if (tj == 0 && q < s) push_part(cluster, sm, q, rank, hi, lo);
    }
}

__global__ void __launch_bounds__(kEngThreads, 1) engine_kernel(EngineArgs E)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    EngSmem *sm = reinterpret_cast<EngSmem *>(smem_raw);
    JPair *recs = reinterpret_cast<JPair *>(smem_raw + sizeof(EngSmem));
    const int64_t ch = E.chunk;
    // this chunk's double-single state [3][ch] and times, keys and masses
    float2 *cx = reinterpret_cast<float2 *>(recs + ch / 2);
    float2 *cv = cx + 3 * ch, *ca = cv + 3 * ch, *ck = ca + 3 * ch;
    float2 *ct = ck + 3 * ch;
    long long *ckey = reinterpret_cast<long long *>(ct + ch);
    float *cm = reinterpret_cast<float *>(ckey + ch);
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned full = 0xffffffffu;
    const StepArgs &A = E.S;
    const int64_t n = A.n, np = A.n_pad;
    const int64_t j0 = (int64_t)rank * E.chunk < np ? (int64_t)rank * E.chunk : np;
    const int64_t j1 = j0 + E.chunk < np ? j0 + E.chunk : np;
    const int nrec = (int)((j1 - j0) / 2);
    const long long *key = reinterpret_cast<const long long *>(A.tn);
    const HState H{A.x, A.v, A.a, A.k, A.t, A.dt, A.tn, A.x2, A.v2, A.a2, A.k2, A.n_pad};
    const DsMirror mir{cx, cv, ca, ck, ct, ckey, ch, j0};
    for (int64_t i = j0 + tid; i < j0 + ch; i += kEngThreads) {
        const int64_t li = i - j0;
        const bool real = i < n;   // padding (and a short last chunk): +inf keys, never selected
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            cx[c * ch + li] = real ? A.x2[c * np + i] : make_float2(0.f, 0.f);
            cv[c * ch + li] = real ? A.v2[c * np + i] : make_float2(0.f, 0.f);
            ca[c * ch + li] = real ? A.a2[c * np + i] : make_float2(0.f, 0.f);
            ck[c * ch + li] = real ? A.k2[c * np + i] : make_float2(0.f, 0.f);
        }
        ct[li] = real ? rn_ds_pack(A.t[i]) : make_float2(0.f, 0.f);
        ckey[li] = real ? key[i] : kInfBits;
        cm[li] = real ? (float)A.m[i] : 0.f;
    }
    __syncthreads();
    const float2 e2 = make_float2(E.eps2f, E.eps2f);
    // step budget of this launch (this call's cap on block steps included), the
    // block time and a pending error: the same values in every thread of the cluster
    int64_t budget = E.max_steps;
    {
        const int64_t left = A.counters[2] - A.counters[0];
        if (left < budget) budget = left;
    }
    const bool clean = *A.status == 0;
    const double t_end = E.check_end ? *A.t_end : 0.0;
    long long tb = *reinterpret_cast<const long long *>(E.t_in);
    int64_t steps = 0;
    // no CTA writes into another's shared memory before every CTA of the cluster
    // runs: arrive here, wait before the first such write
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    bool waited = false;
    for (;;) {
        const double tbd = __longlong_as_double(tb);
        const float2 tb2 = rn_ds_pack(tbd);   // the block time as a double-single
        const DS tbs{tb2.x, tb2.y};
        if (!clean || steps >= budget || !(tb < kInfBits) || (E.check_end && !(tbd <= t_end))) break;

        // ---- 1. this chunk's members (keys == block time), ascending, and the smallest other key
        long long m2 = kInfBits;
        int hits = 0;
        for (int64_t c0 = j0; c0 < j1; c0 += 2 * kEngThreads) {
            const int64_t e = c0 + 2 * (int64_t)tid;
            const longlong2 kv = e < j1 ? *reinterpret_cast<const longlong2 *>(ckey + (e - j0))
                                        : make_longlong2(kInfBits, kInfBits);
            const bool h0 = kv.x == tb, h1 = kv.y == tb;
            m2 = min_ll(m2, h0 ? kInfBits : kv.x);
            m2 = min_ll(m2, h1 ? kInfBits : kv.y);
            const unsigned b0 = __ballot_sync(full, h0), b1 = __ballot_sync(full, h1);
            if (lane == 0) sm->wcnt[warp] = __popc(b0) + __popc(b1);
            __syncthreads();
            int woff = 0, tot = 0;
#pragma unroll
            for (int w = 0; w < kEngWarps; ++w) {
                const int cw = sm->wcnt[w];
                woff += w < warp ? cw : 0;
                tot += cw;
            }
            const unsigned below = (1u << lane) - 1u;
            const int pos = hits + woff + __popc(b0 & below) + __popc(b1 & below);
            if (h0 && pos < kEngCap) sm->own_idx[pos] = (int)e;
            if (h1 && pos + (h0 ? 1 : 0) < kEngCap) sm->own_idx[pos + (h0 ? 1 : 0)] = (int)(e + 1);
            hits += tot;
            __syncthreads();   // wcnt is rewritten by the next segment
        }
        const int hk = hits < kEngCap ? hits : kEngCap;

        // ---- 2. predict this chunk's members (the chunk itself only once the block is
        // known to be taken) and push their records to every CTA
        for (int q = tid; q < hk; q += kEngThreads) {
            const int i = sm->own_idx[q];
            const int64_t li = i - j0;
            float2 X[3], V[3], Ac[3], K[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                X[c] = cx[c * ch + li];
                V[c] = cv[c * ch + li];
                Ac[c] = ca[c * ch + li];
                K[c] = ck[c * ch + li];
            }
            float4 h, l, w;
            ds_predict_ds(X, V, Ac, K, ds_sub(tbs, DS{ct[li].x, ct[li].y}), h, l, w, cm[li]);
            sm->own_rec[q] = IRec{make_float4(h.x, h.y, h.z, __int_as_float(i)), make_float4(l.x, l.y, l.z, 0.f),
                                  make_float4(w.x, w.y, w.z, 0.f)};
        }
        // the corrector's FP64 state of this thread's member (four lanes per member),
        // in flight during the force phase; a quad past the members works on member 0
        // without storing (correct_group needs a valid particle, and one with the
        // members' step keeps its fast path)
        const int hq = tid >> 2;
        const bool qlive = hq < hk;
        const int icor = hk > 0 ? sm->own_idx[qlive ? hq : 0] : (int)j0;
        GroupState gs{};
        if (hk > 0 && warp * 8 < hk) gs = load_group(H, icor);
        __syncthreads();
        if (!waited) {
            asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
            waited = true;
        }
        if (tid < C) *cluster.map_shared_rank(&sm->slot_cnt[rank], tid) = hits;
        if (tid < hk * C) {
            const int k = tid / C, dst = tid % C;
            *cluster.map_shared_rank(&sm->inbox[rank][k], dst) = sm->own_rec[k];
        }
        cluster.sync();

        // ---- the block: its size, this chunk's offset; does the engine take it?
        int s = 0, mx = 0;
        {
            const int cq = lane < C ? sm->slot_cnt[lane] : 0;
            int total = cq, big = cq;
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                total += __shfl_xor_sync(full, total, o);
                big = max(big, __shfl_xor_sync(full, big, o));
            }
            s = total;
            mx = big;
        }
        if (s < 1 || s > E.s_max || mx > kEngCap) break;

        // ---- 3. the chunk's pair records; the members in block order (rank by rank);
        // then the partial sums over this chunk, pushed to each member's owner
        if (warp == 0) {
            const int cq = lane < C ? sm->slot_cnt[lane] : 0;
            int incl = cq;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(full, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane < C) sm->rank_base[lane] = incl - cq;
        }
        for (int64_t i = j0 + tid; i < j1; i += kEngThreads) {
            const int64_t li = i - j0;
            if (i < n) {
                float2 X[3], V[3], Ac[3], K[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    X[c] = cx[c * ch + li];
                    V[c] = cv[c * ch + li];
                    Ac[c] = ca[c * ch + li];
                    K[c] = ck[c * ch + li];
                }
                float4 h, l, w;
                ds_predict_ds(X, V, Ac, K, ds_sub(tbs, DS{ct[li].x, ct[li].y}), h, l, w, cm[li]);
                jrec_store(recs, li, h.x, h.y, h.z, h.w, l.x, l.y, l.z, w.x, w.y, w.z);
            } else {
                const float far = (float)kPadPos;
                jrec_store(recs, li, far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (tid < C * kEngCap) {
            const int r = tid / kEngCap, k = tid % kEngCap;
            if (r < C && k < sm->slot_cnt[r]) {
                const int q = sm->rank_base[r] + k;
                sm->ilist[q] = sm->inbox[r][k];
                sm->qmap[q] = make_int2(r, k);
            }
        }
        __syncthreads();
        if (s <= 16) {
            // G warps per member (G = 16 / s rounded to a power of two), lanes over
            // pair records; the G warps' sums are added in warp order
            const int sp = s <= 1 ? 1 : s <= 2 ? 2 : s <= 4 ? 4 : s <= 8 ? 8 : 16;
            const int G = kEngWarps / sp;
            const int q = warp / G, part = warp % G;
            if (q < s) {
                const IRec R = sm->ilist[q];
                const int gi = __float_as_int(R.h.w);
                const IPk ip = ipk_of_rec(R);
                const int rb = (int)((int64_t)nrec * part / G), re = (int)((int64_t)nrec * (part + 1) / G);
                Acc7 hi, lo;
                zero(hi);
                zero(lo);
                sweep<true, 32>(recs, j0, rb, re, lane, ip, gi, e2, hi, lo);
                ds_group_reduce7<32>(hi, lo);
                if (lane == 0) {
#pragma unroll
                    for (int c = 0; c < 7; ++c) sm->red[warp][c] = make_float2(acc_get(hi, c), acc_get(lo, c));
                }
            }
            __syncthreads();
            // warp c adds component c of each member's G warp sums by a butterfly over
            // groups of G lanes (lane l holds warp l's sum; lanes past the members add zeros)
            if (warp < 7) {
                const int c = warp;
                const bool has = lane < kEngWarps && lane / G < s;
                float h = has ? sm->red[lane][c].x : 0.f, l = has ? sm->red[lane][c].y : 0.f;
                for (int off = G / 2; off >= 1; off >>= 1) {
                    const float h2 = __shfl_xor_sync(full, h, off), l2 = __shfl_xor_sync(full, l, off);
                    ds_add(h, l, h2, l2);
                }
                if (has && lane % G == 0) {
                    const int2 o = sm->qmap[lane / G];
                    *cluster.map_shared_rank(&sm->part_in[o.y][rank][c], o.x) = make_float2(h, l);
                }
            }
        } else {
            force_groups<8>(cluster, sm, recs, j0, j1, nrec, s, e2, rank);
        }
        cluster.sync();

        // ---- 4. correct this chunk's members: the ranks' partial sums in rank order,
        // then the FP64 corrector
        int flags = 0;
        long long tmin = m2;
        if (warp * 8 < hk) {   // warps holding at least one member (quads 8w .. 8w + 7)
            const int c = (tid & 3) < 3 ? (tid & 3) : 2;
            const int k = qlive ? hq : 0;
            float2 va[kEngMaxC], vk[kEngMaxC];
#pragma unroll
            for (int r = 0; r < kEngMaxC; ++r) {
                va[r] = r < C ? sm->part_in[k][r][c] : make_float2(0.f, 0.f);
                vk[r] = r < C ? sm->part_in[k][r][3 + c] : make_float2(0.f, 0.f);
            }
            float ha = 0.f, la = 0.f, hk_ = 0.f, lk = 0.f;
#pragma unroll
            for (int r = 0; r < kEngMaxC; ++r) {
                if (r < C) {
                    ds_add(ha, la, va[r].x, va[r].y);
                    ds_add(hk_, lk, vk[r].x, vk[r].y);
                }
            }
            const double an = (double)ha + (double)la, kn = (double)hk_ + (double)lk;
            long long newkey = kInfBits;
            flags |= correct_group(H, icor, gs, qlive, tbd, an, kn, A.eta, A.dt_max, A.dt_min, &newkey, &mir);
            tmin = min_ll(tmin, newkey);
        }
        tmin = warp_min(tmin);
        flags = (int)__reduce_or_sync(full, (unsigned)flags);
        if (lane == 0) {
            sm->wmin[warp] = tmin;
            sm->wflags[warp] = flags;
        }
        __syncthreads();
        if (rank == 0 && tid == 0) {
            A.counters[0] += 1;
            A.counters[1] += s;
            int b = 0;
            while ((int64_t(1) << b) < s && b < NB_SIZE_BUCKETS - 1) ++b;
            A.counters[3 + b] += 1;
            *A.interactions += (double)s * (double)n;
        }
        ++steps;
        // The last warp (which holds no member: kEngCap members take warps 0 and 1)
        // publishes this chunk's smallest key and status bits to every CTA and
        // arrives with release semantics; the other warps arrive relaxed, so the
        // barrier does not wait for the corrector's global stores (nothing in this
        // cluster reads them before the next kernel; this CTA's own next reads of
        // them follow a CTA barrier).
        if (warp == kEngWarps - 1) {
            long long mm = lane < kEngWarps ? sm->wmin[lane] : kInfBits;
            int ff = lane < kEngWarps ? sm->wflags[lane] : 0;
            mm = warp_min(mm);
            ff = (int)__reduce_or_sync(full, (unsigned)ff);
            if (lane < C) {
                *cluster.map_shared_rank(&sm->slot_min[rank], lane) = mm;
                *cluster.map_shared_rank(&sm->slot_err[rank], lane) = ff;
            }
            asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
        } else {
            asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
        }
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");

        // ---- the next block time: the smallest key of all chunks
        long long nxt = lane < C ? sm->slot_min[lane] : kInfBits;
        int err = lane < C ? sm->slot_err[lane] : 0;
        nxt = warp_min(nxt);
        err = (int)__reduce_or_sync(full, (unsigned)err);
        tb = nxt;
        if (err) {
            if (rank == 0 && tid == 0) atomicOr(A.status, err);
            break;
        }
    }
    if (!waited) asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    if (rank == 0 && tid == 0) {
        *E.t_out = __longlong_as_double(tb);
        if (steps > 0 && E.s_clear) *E.s_clear = 0;
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

// shared memory: the exchange areas, the chunk's pair records, and its state copy
// (x, v, a, k double-single [3][chunk] float2 each, times, keys, masses)
size_t engine_smem_bytes(int64_t chunk)
{
    return sizeof(EngSmem) + (size_t)(chunk / 2) * sizeof(JPair) +
           (size_t)chunk * (12 * sizeof(float2) + sizeof(float2) + sizeof(long long) + sizeof(float));
}

// Cluster size of the engine for this device (16 if co-schedulable with the
// largest shared-memory footprint, else 8, else 0 = no engine); queried once.
int engine_cluster()
{
    static int cached = -1;
    if (cached >= 0) return cached;
    cached = 0;
    const size_t smem = engine_smem_bytes(kEngMaxChunk);
    if (cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(engine_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        (void)cudaGetLastError();
        return cached;
    }
    for (int c : {16, 8}) {
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3((unsigned)c);
        cfg.blockDim = dim3(kEngThreads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)c;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclu = 0;
        if (cudaOccupancyMaxActiveClusters(&nclu, engine_kernel, &cfg) == cudaSuccess && nclu > 0) {
            cached = c;
            break;
        }
        (void)cudaGetLastError();
    }
    return cached;
}

int64_t engine_chunk(int64_t n_pad, int C)
{
    if (C < 1) return 0;
    const int64_t c = (n_pad + C - 1) / C;
    return (c + 15) / 16 * 16;
}

cudaError_t launch_engine(const EngineArgs &e, int C, cudaStream_t st)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(kEngThreads);
    cfg.dynamicSmemBytes = engine_smem_bytes(e.chunk);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, engine_kernel, e);
}

}  // namespace nb
