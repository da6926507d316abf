// Allocation-free variant of the CFL time-step reduction (gks_cfl_dt_noalloc).
//
// Some callers cannot allocate device memory at the moment they need the time
// step: time loops of solvers that reserve all memory at start-up and forbid
// allocation afterwards, and hosts whose device memory belongs to another
// allocator (a framework's caching pool).  For them this entry point computes
// the same step as gks_cfl_dt without calling cudaMalloc, cudaFree or any
// allocating routine: the block minima of the two-stage reduction live in the
// file-scope array below, which every GPU that loads the library holds until
// the process exits.
#include <cfloat>
#include <mutex>

#include "gks_internal.h"

namespace gks {
namespace {

constexpr int kNoallocMaxBlocks = 16384;   // 128 KiB of scratch: up to 16384 * 256 = 4,194,304 cells
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_dt_scratch[kNoallocMaxBlocks];

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

// Per-cell CFL bound of the caller-ordered state (w[v * T + perm[i]] belongs to
// internal cell i), block minimum into scratch[blockIdx.x].
__global__ void k_cfl_partial_static(const int32_t *__restrict__ perm, const double *__restrict__ inrad,
                                     const double *__restrict__ w, int64_t T, double gamma, double mu,
                                     double *__restrict__ scratch)
{
    __shared__ double sh[kBlock];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double dti = DBL_MAX;
    if (i < T) {
        const int64_t c = perm[i];
        const double rho = w[c], u = w[T + c] / rho, v = w[2 * T + c] / rho;
        const double p = (gamma - 1.0) * (w[3 * T + c] - 0.5 * rho * (u * u + v * v));
        const double r = inrad[i];
        dti = r / (sqrt(u * u + v * v) + sqrt(gamma * p / rho) + 2.0 * mu / (rho * r));
        if (!(dti > 0.0)) dti = 0.0;
    }
    sh[threadIdx.x] = dti;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[blockIdx.x] = sh[0];
}

__global__ void k_cfl_final_static(const double *__restrict__ scratch, int nblk, double cfl, double *dt_out)
{
    __shared__ double sh[kBlock];
    double m = DBL_MAX;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) m = fmin(m, scratch[b]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *dt_out = cfl * sh[0];
}

// Device address of the scratch array on the current device, looked up once
// per device and kept for the life of the process (a device reset that moves
// the array is documented as the end of this entry point's use).
gks_status scratch_address(int dev, double **out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("gks_cfl_dt_noalloc: device ordinal %d beyond %d", dev, kMaxDevices);
        return GKS_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_dt_scratch);
        if (e != cudaSuccess || !p) {
            set_error("gks_cfl_dt_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return GKS_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return GKS_OK;
}

}  // namespace
}  // namespace gks

using namespace gks;

extern "C" gks_status gks_cfl_dt_noalloc(const gks_mesh *m, const double *w, double *dt_dev, void *stream)
{
    if (!m || !w || !dt_dev) {
        set_error("gks_cfl_dt_noalloc: NULL argument");
        return GKS_EINVAL;
    }
    if (m->n_case != 1) {
        set_error("gks_cfl_dt_noalloc: the handle holds %d cases; it takes a single mesh", m->n_case);
        return GKS_EINVAL;
    }
    const int64_t T = m->d.T;
    const int64_t nblk = (T + kBlock - 1) / kBlock;
    if (nblk > kNoallocMaxBlocks) {
        set_error("gks_cfl_dt_noalloc: %lld cells exceed the maximum of %lld of the static scratch",
                  (long long)T, (long long)kNoallocMaxBlocks * kBlock);
        return GKS_EINVAL;
    }
    int prev = -1;
    GKS_CUDA(cudaGetDevice(&prev));
    if (prev != m->device) GKS_CUDA(cudaSetDevice(m->device));
    double *scratch = nullptr;
    gks_status st = scratch_address(m->device, &scratch);
    if (st == GKS_OK) {
        cudaStream_t s = (cudaStream_t)stream;
        k_cfl_partial_static<<<(unsigned)nblk, kBlock, 0, s>>>(m->d.perm, m->d.inrad, w, T, m->cfg.gamma, m->cfg.mu,
                                                                scratch);
        note_launch();
        k_cfl_final_static<<<1, kBlock, 0, s>>>(scratch, (int)nblk, m->cfg.cfl, dt_dev);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            set_error("gks_cfl_dt_noalloc: launch failed: %s", cudaGetErrorString(e));
            st = GKS_ECUDA;
        }
    }
    if (prev != m->device) cudaSetDevice(prev);
    return st;
}
