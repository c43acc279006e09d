// nb_force_jerk_static: the mixed-precision force evaluation without any
// device allocation, for callers that may not allocate GPU memory themselves.
//
// Typical such callers: code running inside a host framework that owns the
// device's memory budget through its own pool and forbids raw cudaMalloc;
// plugins loaded into another application's process and CUDA context; and
// latency-critical loops that must not pay the implicit device synchronisation
// of cudaMalloc/cudaFree. They pass inputs and outputs; every intermediate
// buffer (the double-single j-records, the split partials, the final sums,
// the arrival tickets, the active count and the status word) lives in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "nb_ds.cuh"
#include "nb_internal.cuh"
#include "nb_pair.cuh"

namespace nb {
namespace {

constexpr int64_t kStaticMaxN = NB_STATIC_MAX_N;
constexpr int64_t kStaticTiles = (kStaticMaxN + kJT - 1) / kJT;
constexpr int64_t kStaticPad = kStaticTiles * kJT;
constexpr int64_t kStaticPartWords = int64_t(1) << 19;   // split partials: 4 MiB

// byte offsets inside the array (all multiples of 256)
constexpr size_t kOffRec = 0;
constexpr size_t kOffPart = kOffRec + (kStaticPad / 2) * sizeof(JPair);
constexpr size_t kOffFin = kOffPart + kStaticPartWords * 8;
constexpr size_t kOffTickets = kOffFin + kStaticPad * kPartStride * sizeof(double);
constexpr size_t kOffS = kOffTickets + ((kStaticPad + 1) * sizeof(int32_t) + 255) / 256 * 256;
constexpr size_t kOffSplit = kOffS + 256;
constexpr size_t kOffStatus = kOffSplit + 256;
constexpr size_t kStaticBytes = kOffStatus + 256;

static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

// Per-device address of g_scratch (set up on the first call on each device).
std::mutex g_mu;
unsigned char *g_addr[256] = {};

// Double-single records of the caller's FP64 predicted state, far-away massless
// padding up to a whole tile, cleared tickets, the active count, a clear status.
__global__ void static_setup_kernel(const double *m, const double *x, const double *v, int64_t n, int64_t s,
                                    unsigned char *base)
{
    JPair *rec = reinterpret_cast<JPair *>(base + kOffRec);
    int32_t *tickets = reinterpret_cast<int32_t *>(base + kOffTickets);
    const int64_t npad = (n + kJT - 1) / kJT * kJT;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < npad; i += stride) {
        if (i < n) {
            const DS px = ds_split(x[3 * i]), py = ds_split(x[3 * i + 1]), pz = ds_split(x[3 * i + 2]);
            jrec_store(rec, i, px.hi, py.hi, pz.hi, (float)m[i], px.lo, py.lo, pz.lo, (float)v[3 * i],
                       (float)v[3 * i + 1], (float)v[3 * i + 2]);
        } else {
            const float far = (float)kPadPos;
            jrec_store(rec, i, far, far, far, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f);
        }
        tickets[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        tickets[npad] = 0;
        *reinterpret_cast<int64_t *>(base + kOffS) = s;
        *reinterpret_cast<int32_t *>(base + kOffStatus) = 0;
    }
}

}  // namespace
}  // namespace nb

using namespace nb;

extern "C" nb_status nb_force_jerk_static(int64_t n, const double *m_dev, const double *x_dev, const double *v_dev,
                                          double eps2, const int32_t *idx_dev, int64_t s, double *a_dev,
                                          double *k_dev, double *phi_dev, void *stream)
{
    if (n < 1 || n > kStaticMaxN || s < 0 || s > n) return NB_ERR_ARG;
    if (!m_dev || !x_dev || !v_dev || (s > 0 && !idx_dev)) return NB_ERR_ARG;
    if (!(eps2 >= 0.0) || !std::isfinite(eps2)) return NB_ERR_ARG;
    if (s == 0) return NB_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return NB_ERR_CUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return NB_ERR_CUDA;
            g_addr[dev] = static_cast<unsigned char *>(p);
        }
        base = g_addr[dev];
    }
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NB_ERR_CUDA;
    const int64_t n_tiles = (n + kJT - 1) / kJT;
    const int grid = force_mixed_grid(num_sms, n_tiles);
    int variant = 0, split = 1;
    default_tuning(NB_PREC_MIXED, n, s, grid, 1, &variant, &split);
    // the split partials must fit: s * split * 8 words
    const int64_t max_split = kStaticPartWords / (s * kPartStride);
    if (max_split < 1) return NB_ERR_ARG;
    if (split > max_split) split = (int)max_split;
    if (split > n_tiles) split = (int)n_tiles;
    if (split < 1) split = 1;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t npad = n_tiles * kJT;
    int blocks = (int)std::min<int64_t>((npad + 255) / 256, 4096);
    static_setup_kernel<<<blocks, 256, 0, st>>>(m_dev, x_dev, v_dev, n, s, base);
    if (cudaGetLastError() != cudaSuccess) return NB_ERR_CUDA;

    ForceArgs F{};
    F.n = n;
    F.n_tiles = n_tiles;
    F.tile_lo = 0;
    F.tile_hi = n_tiles;
    F.j.p = reinterpret_cast<JPair *>(base + kOffRec);
    F.eps2f = (float)eps2;
    F.eps2 = eps2;
    F.idx = idx_dev;
    F.idx_cap = s;
    F.s = reinterpret_cast<const int64_t *>(base + kOffS);
    F.s_host = -1;
    F.part = reinterpret_cast<double *>(base + kOffPart);
    F.part_cap = kStaticPartWords;
    F.fin = reinterpret_cast<double *>(base + kOffFin);
    F.tickets = reinterpret_cast<int32_t *>(base + kOffTickets);
    F.split_used = reinterpret_cast<int32_t *>(base + kOffSplit);
    F.tune = nullptr;
    F.force_variant = variant;
    F.force_split = split;
    F.status = reinterpret_cast<int32_t *>(base + kOffStatus);
    F.spin_limit = int64_t(1) << 24;
    F.inject = 0;
    if (launch_force_mixed(F, grid, st) != cudaSuccess) return NB_ERR_CUDA;
    if (launch_reduce_out(F.fin, F.s, s, a_dev, k_dev, phi_dev, F.status, st) != cudaSuccess) return NB_ERR_CUDA;
    // the status word is read in stream order (no wait on other streams' work)
    int32_t status = 0;
    if (cudaMemcpyAsync(&status, F.status, sizeof status, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return NB_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return NB_ERR_CUDA;
    if (status & kStTimeout) return NB_ERR_TIMEOUT;
    if (status & kStNonfinite) return NB_ERR_NONFINITE;
    return status ? NB_ERR_CUDA : NB_OK;
}
