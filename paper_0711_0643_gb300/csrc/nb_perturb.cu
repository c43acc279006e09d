// Perturber lists of binaries (Sect. 3.1 of the paper): for each binary, the
// stars that perturb its internal motion, in the order a serial scan over the
// star index finds them, at most nmax of them, with the count of all.
//
// The paper gives the threshold as a force of about 10^-7 relative to a mean
// force. It is read here as the tidal perturbation of the binary: star j at
// distance r_j from the binary's centre of mass accelerates the two members
// differently by about 2 m_j d / r_j^3 (d their separation), against the
// binary's internal acceleration m_b / d^2, and it is a perturber when the ratio
// 2 m_j d^3 / (m_b r_j^3) reaches gamma. The test is taken without roots, on
// sixth powers, as (2 m_j)^2 d^6 >= (gamma m_b)^2 r_j^6, every FP64 operation an
// explicit round-to-nearest one in a fixed order (the decision is an integer
// result and must not depend on operation fusing).
//
// One CTA per binary walks the stars in chunks of 256 in ascending index: each
// thread tests one star, warp ballots and a CTA prefix place the perturbers of
// the chunk after those already found, so the list comes out in the serial
// order by construction (the paper restores that order after its parallel
// search by broadcasting and sorting the lists). A j-range restricts the scan to
// one rank's share of the stars; lists of consecutive ranges concatenated in
// range order and cut at nmax give the list of the whole range.
#include "nb_internal.cuh"

namespace nb {
namespace {

constexpr int kPertThreads = 256;

__device__ __forceinline__ double d2_of(double ux, double uy, double uz, double wx, double wy, double wz)
{
    const double dx = __dsub_rn(ux, wx), dy = __dsub_rn(uy, wy), dz = __dsub_rn(uz, wz);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

__global__ void __launch_bounds__(kPertThreads) perturbers_kernel(PertArgs P)
{
    __shared__ int wcnt[kPertThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int64_t np = P.np;
    for (int32_t b = blockIdx.x; b < P.nbin; b += gridDim.x) {
        const int32_t i = P.pairs[2 * b], k = P.pairs[2 * b + 1];
        int32_t *list = P.lists + (int64_t)b * P.nmax;
        if (i < 0 || k < 0 || i >= P.n || k >= P.n || i == k) {
            // an invalid pair: an empty list and a negative count
            for (int q = tid; q < P.nmax; q += kPertThreads) list[q] = -1;
            if (tid == 0) P.counts[b] = -1;
            continue;
        }
        const double mi = P.m[i], mk = P.m[k];
        const double mb = __dadd_rn(mi, mk);
        double cm[3], xi[3], xk[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            xi[c] = P.x[c * np + i];
            xk[c] = P.x[c * np + k];
            cm[c] = __ddiv_rn(__dadd_rn(__dmul_rn(mi, xi[c]), __dmul_rn(mk, xk[c])), mb);
        }
        const double d2 = d2_of(xi[0], xi[1], xi[2], xk[0], xk[1], xk[2]);
        const double d6 = __dmul_rn(__dmul_rn(d2, d2), d2);
        const double gm = __dmul_rn(P.gamma, mb);
        const double rhs = __dmul_rn(gm, gm);
        int found = 0;   // the same in every thread
        for (int64_t j0 = P.j_lo; j0 < P.j_hi; j0 += kPertThreads) {
            const int64_t j = j0 + tid;
            bool pert = false;
            if (j < P.j_hi && j != i && j != k) {
                const double r2 = d2_of(P.x[j], P.x[np + j], P.x[2 * np + j], cm[0], cm[1], cm[2]);
                const double r6 = __dmul_rn(__dmul_rn(r2, r2), r2);
                const double tm = __dmul_rn(2.0, P.m[j]);
                pert = __dmul_rn(__dmul_rn(tm, tm), d6) >= __dmul_rn(rhs, r6);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, pert);
            if (lane == 0) wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
#pragma unroll
            for (int w = 0; w < kPertThreads / 32; ++w) {
                const int cw = wcnt[w];
                before += w < warp ? cw : 0;
                total += cw;
            }
            const int pos = found + before + __popc(bal & below);
            if (pert && pos < P.nmax) list[pos] = (int32_t)j;
            found += total;
            __syncthreads();   // wcnt is rewritten by the next chunk
        }
        for (int q = found + tid; q < P.nmax; q += kPertThreads) list[q] = -1;
        if (tid == 0) P.counts[b] = found;
    }
}

}  // namespace

cudaError_t launch_perturbers(const PertArgs &p, cudaStream_t st)
{
    if (p.nbin <= 0) return cudaSuccess;
    const int grid = (int)(p.nbin < 65535 ? p.nbin : 65535);
    perturbers_kernel<<<grid, kPertThreads, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace nb
