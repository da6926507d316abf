// Measurement probes (not part of the scheme): the throughput of the FP64 and
// FP32 fused multiply-add pipes and of streaming HBM reads and copies on the
// GPU the library runs on.  The benchmark times them with CUDA events and uses
// the results as the measured roofs of the kernels the FMA pipes or HBM bound.
// Also the pair arithmetic and the bounded wait of the solver on their own,
// for the tests.
#include "gks_df.cuh"
#include "gks_internal.h"
#include "gks_wait.cuh"

namespace gks {
namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;               // independent dependency chains per thread

// kChains chains of a = a * b + c per thread, iters times each: 2 kChains iters
// flops per thread.  b < 1 keeps the chains bounded; the sum is written so that
// nothing is dead code.
template <typename R>
__global__ void __launch_bounds__(kProbeThreads) k_fma_chain(int iters, R b, R c, R *sink)
{
    R a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = R(threadIdx.x + k) * R(1e-3);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;
    }
    R s = R(0);
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    if (s == R(-12345.0)) sink[blockIdx.x] = s;     // never true; keeps the chains live
}

// Sum of the 16-byte words of a buffer (grid-stride, 4 words in flight per thread).
__global__ void __launch_bounds__(kProbeThreads) k_read(const float4 *__restrict__ p, int64_t n, double *sink)
{
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const float4 a = __ldcs(p + i), b = __ldcs(p + i + stride), c = __ldcs(p + i + 2 * stride),
                     d = __ldcs(p + i + 3 * stride);
        acc += (a.x + a.y + a.z + a.w) + (b.x + b.y + b.z + b.w) + (c.x + c.y + c.z + c.w) + (d.x + d.y + d.z + d.w);
    }
    for (; i < n; i += stride) {
        const float4 a = __ldcs(p + i);
        acc += a.x + a.y + a.z + a.w;
    }
    if (acc == -12345.0f) sink[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kProbeThreads) k_copy(const float4 *__restrict__ s, float4 *__restrict__ d, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) __stcs(d + i, __ldcs(s + i));
}

// One double-FP32 function per element: the argument is split into an FP32
// pair by integer operations, the result widened to FP64.
__global__ void k_df_eval(int op, int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                          double *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dfm::df a = dfm::split_double(x[i]);
    dfm::df r = {0.0f, 0.0f};
    switch (op) {
    case GKS_DF_SPLIT: r = a; break;
    case GKS_DF_EXP: r = dfm::exp(a); break;
    case GKS_DF_EXPM1: r = dfm::expm1(a); break;
    case GKS_DF_ERFCX: r = dfm::erfcx(a); break;
    case GKS_DF_SQRT: r = dfm::sqrt(a); break;
    case GKS_DF_DIV: r = dfm::div(a, dfm::split_double(y[i])); break;
    case GKS_DF_MUL: r = dfm::mul(a, dfm::split_double(y[i])); break;
    case GKS_DF_ADD: r = dfm::add(a, dfm::split_double(y[i])); break;
    case GKS_DF_RECIP: r = dfm::recip(a); break;
    default: break;
    }
    if (op == GKS_DF_SPLIT) {
        out[2 * i] = (double)r.hi;             // the pair itself
        out[2 * i + 1] = (double)r.lo;
    } else {
        out[2 * i] = dfm::to_double(r);
        out[2 * i + 1] = 0.0;
    }
}

gks_status grid_of(int per_sm, unsigned *g)
{
    int dev = 0, nsm = 0;
    GKS_CUDA(cudaGetDevice(&dev));
    GKS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    *g = (unsigned)(nsm * per_sm);
    return GKS_OK;
}

// One thread waits for *flag == 1 (set first when set != 0); out[0] = 1 if
// the wait gave up, out[1] = nanoseconds it took.
__global__ void k_wait_probe(int32_t *flag, int32_t *err, int set, uint64_t limit_ns, int64_t *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (set) publish(flag, 1);
    const uint64_t t0 = global_ns();
    const bool ok = bounded_wait(flag, 1, err, limit_ns);
    out[0] = ok ? 0 : 1;
    out[1] = (int64_t)(global_ns() - t0);
}

}  // namespace
}  // namespace gks

using namespace gks;

extern "C" gks_status gks_probe_wait(int64_t limit_ns, int32_t set_flag, int32_t *timed_out, int64_t *waited_ns,
                                     void *stream)
{
    if (!timed_out || limit_ns < 1 || limit_ns > 10000000000LL) {
        set_error("gks_probe_wait: NULL timed_out or limit outside [1, 1e10] ns");
        return GKS_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t *buf = nullptr;                 // [0] flag, [1] error word, [2..3] results
    GKS_CUDA(cudaMalloc(&buf, 4 * sizeof(int64_t)));
    int64_t h[2] = {0, 0};
    cudaError_t e = cudaMemsetAsync(buf, 0, 4 * sizeof(int64_t), s);
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32, 0, s>>>(reinterpret_cast<int32_t *>(buf), reinterpret_cast<int32_t *>(buf + 1),
                                      set_flag ? 1 : 0, (uint64_t)limit_ns, buf + 2);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, buf + 2, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) {
        set_error("gks_probe_wait: %s", cudaGetErrorString(e));
        return GKS_ECUDA;
    }
    *timed_out = (int32_t)h[0];
    if (waited_ns) *waited_ns = h[1];
    return GKS_OK;
}

extern "C" gks_status gks_probe_fma(int32_t fp64, int32_t blocks_per_sm, int32_t iters, double *sink, void *stream,
                                    double *flops)
{
    if (!sink || blocks_per_sm <= 0 || iters <= 0) {
        set_error("gks_probe_fma: NULL sink or non-positive size");
        return GKS_EINVAL;
    }
    unsigned g = 0;
    gks_status st = grid_of(blocks_per_sm, &g);
    if (st != GKS_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (fp64)
        k_fma_chain<double><<<g, kProbeThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink);
    else
        k_fma_chain<float><<<g, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, reinterpret_cast<float *>(sink));
    note_launch();
    GKS_CUDA(cudaGetLastError());
    if (flops) *flops = 2.0 * kChains * 8.0 * iters * (double)g * kProbeThreads;
    return GKS_OK;
}

extern "C" gks_status gks_probe_read(const void *buf, int64_t bytes, double *sink, void *stream)
{
    if (!buf || !sink || bytes < 16 || (bytes & 15) || ((uintptr_t)buf & 15)) {
        set_error("gks_probe_read: buffer must be 16-byte aligned and a positive multiple of 16 bytes");
        return GKS_EINVAL;
    }
    unsigned g = 0;
    gks_status st = grid_of(4, &g);
    if (st != GKS_OK) return st;
    k_read<<<g, kProbeThreads, 0, (cudaStream_t)stream>>>(static_cast<const float4 *>(buf), bytes / 16, sink);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

extern "C" gks_status gks_probe_copy(const void *src, void *dst, int64_t bytes, void *stream)
{
    if (!src || !dst || bytes < 16 || (bytes & 15) || ((uintptr_t)src & 15) || ((uintptr_t)dst & 15)) {
        set_error("gks_probe_copy: buffers must be 16-byte aligned and a positive multiple of 16 bytes");
        return GKS_EINVAL;
    }
    unsigned g = 0;
    gks_status st = grid_of(4, &g);
    if (st != GKS_OK) return st;
    k_copy<<<g, kProbeThreads, 0, (cudaStream_t)stream>>>(static_cast<const float4 *>(src), static_cast<float4 *>(dst),
                                                        bytes / 16);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

extern "C" gks_status gks_probe_df(int32_t op, int64_t n, const double *x, const double *y, double *out, void *stream)
{
    if (op < GKS_DF_SPLIT || op > GKS_DF_RECIP || n < 0 || (n > 0 && (!x || !out)) ||
        ((op == GKS_DF_DIV || op == GKS_DF_MUL || op == GKS_DF_ADD) && n > 0 && !y)) {
        set_error("gks_probe_df: bad operation or NULL array");
        return GKS_EINVAL;
    }
    if (n == 0) return GKS_OK;
    k_df_eval<<<(unsigned)((n + kProbeThreads - 1) / kProbeThreads), kProbeThreads, 0, (cudaStream_t)stream>>>(op, n, x,
                                                                                                             y, out);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}
