// CLS reconstruction on the device (Sec. III): right-hand side, operator
// application, block ILU(0) preconditioner and restarted GMRES.
//
// Four independent systems (rho, rho u, rho v, E) share one operator; every
// kernel handles one cell and all four variables, so each block of the
// operator is read once per application.  Vectors are SoA [var][dof][cell] in
// RCM order.  GMRES (Saad & Schultz 1986) is right-preconditioned, uses
// classical Gram-Schmidt (twice, CGS2, in FP64 mode), and keeps per-variable
// state on the device (running/converged masks); reductions go through
// per-block partial sums and a fixed-order second pass, so results are
// deterministic.  The Krylov basis is stored unnormalised, V_k = vn_k v_k,
// with the norms vn_k on the device: the normalisation is folded into the
// Gram-Schmidt coefficients, the Hessenberg entries and the final combination,
// which saves one read and one write of the new vector per iteration.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "gks_internal.h"
#include "gks_wait.cuh"

namespace gks {
namespace {

constexpr int NV = 4, ND = 5, NX = 20;
constexpr int kDotThreads = 256;       // threads per block of the dot-product kernel
constexpr int kDotMaxTiles = 65535;    // grid.y limit of the dot-product kernel

// Per-variable control words ctl[16]: [0..3] active (needs more work), [4..7]
// running (iterating in the current cycle), [8..11] Krylov vectors in the
// cycle, [12..15] iterations so far.

// acc += sa [e1 + dx e3 + dy e4 | e2 + dx e4 + dy e5] (g1, g2): the off-diagonal
// block O_ij = alpha [...] applied to the gradient entries (g1, g2) of
// neighbour j, scaled by sa = +-alpha, with sax = sa dx, say = sa dy; all FMAs
template <typename R>
__device__ __forceinline__ void oacc(R sa, R sax, R say, R g1, R g2, R *acc)
{
    acc[0] = fma(sa, g1, acc[0]);
    acc[1] = fma(sa, g2, acc[1]);
    acc[2] = fma(sax, g1, acc[2]);
    acc[3] = fma(say, g1, fma(sax, g2, acc[3]));
    acc[4] = fma(say, g2, acc[4]);
}

// acc[0..1] += sr [x0 + dx x2 + dy x3 | x1 + dx x3 + dy x4] (srx = sr dx, sry =
// sr dy): the transpose form that the global normal equations (Eq. (33)) add
// to an off-diagonal block from the neighbour's own equations, applied to all
// five unknowns x of the neighbour
template <typename R>
__device__ __forceinline__ void racc(R sr, R srx, R sry, const R *x, R *acc)
{
    acc[0] = fma(sr, x[0], fma(srx, x[2], fma(sry, x[3], acc[0])));
    acc[1] = fma(sr, x[1], fma(srx, x[3], fma(sry, x[4], acc[1])));
}

// 2^e exactly (|e| <= 1022)
__device__ __forceinline__ double pow2(int e)
{
    e = e < -1022 ? -1022 : (e > 1023 ? 1023 : e);
    return __longlong_as_double((long long)(e + 1023) << 52);
}

// Block reduction of NV values; thread 0 of the block gets the totals.
__device__ __forceinline__ void block_sum4(double *v, double *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) sh[warp * NV + q] = v[q];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        for (int q = 0; q < NV; ++q) {
            double s = 0.0;
            for (int k = 0; k < nw; ++k) s += sh[k * NV + q];
            v[q] = s;
        }
    }
    __syncthreads();
}

// r_i = sum_j a0_ij (ubar_j - ubar_i), Eq. (25) with b_ij = (ubar_j - ubar_i, 0, 0)
// with partial sums of |b|^2 per block and variable in part[blk][v][1]
__global__ void k_rhs(DeviceMesh d, const double *__restrict__ w, double *__restrict__ b, double *__restrict__ part,
                      int pstride)
{
    __shared__ double sh[32 * NV];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double nb[NV] = {0, 0, 0, 0};
    if (i < T) {
        double acc[NX];
#pragma unroll
        for (int q = 0; q < NX; ++q) acc[q] = 0.0;
        double wi[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) wi[v] = w[v * T + i];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int j = d.nb[s * T + i];
            if (j < 0) continue;
            double a[ND];
#pragma unroll
            for (int l = 0; l < ND; ++l) a[l] = d.a0[(s * ND + l) * T + i];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double du = w[v * T + j] - wi[v];
#pragma unroll
                for (int l = 0; l < ND; ++l) acc[v * ND + l] += a[l] * du;
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v)
#pragma unroll
            for (int l = 0; l < ND; ++l) {
                const double bv = acc[v * ND + l];
                b[(v * ND + l) * T + i] = bv;
                nb[v] += bv * bv;
            }
    }
    block_sum4(nb, sh);
    if (threadIdx.x == 0)
        for (int v = 0; v < NV; ++v) part[(blockIdx.x * NV + v) * pstride + 1] = nb[v];
}

// acc = (K x)_i, the operator row of cell i applied to x (TM arithmetic).
// Every load (neighbour indices, blocks, the neighbours' gradient entries, own
// data) is issued before the arithmetic; a missing neighbour reads the cell's
// own entries with a zero block.
// G: extended stencil (global normal equations and / or second-derivative
// equations): the transpose form with the reverse-slot coefficients arg, exrg,
// eyrg (racc) and the diagonal coupling bdg of the unknowns 3..5; unused
// otherwise.
template <typename TX, typename TM, bool G = false>
__device__ __forceinline__ void cell_apply(const DeviceMesh &d, const TM *__restrict__ Dg, const TM *__restrict__ alg,
                                           const TM *__restrict__ exg, const TM *__restrict__ eyg,
                                           const TX *__restrict__ x, int64_t i, TM *acc,
                                           const TM *__restrict__ arg = nullptr, const TM *__restrict__ exrg = nullptr,
                                           const TM *__restrict__ eyrg = nullptr, const TM *__restrict__ bdgg = nullptr)
{
    const int64_t T = d.T;
    int64_t jn[3];
    TM sa[3], sax[3], say[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int j = d.nb[s * T + i];
        jn[s] = j >= 0 ? j : i;
        sa[s] = j >= 0 ? -alg[s * T + i] : TM(0);
        sax[s] = sa[s] * exg[s * T + i];
        say[s] = sa[s] * eyg[s * T + i];
    }
    TM g[3][2 * NV];
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            g[s][2 * v] = TM(x[(v * ND + 0) * T + jn[s]]);
            g[s][2 * v + 1] = TM(x[(v * ND + 1) * T + jn[s]]);
        }
    TM Dm[15];
#pragma unroll
    for (int q = 0; q < 15; ++q) Dm[q] = Dg[q * T + i];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        TM xv[ND];
#pragma unroll
        for (int l = 0; l < ND; ++l) xv[l] = TM(x[(v * ND + l) * T + i]);
        // symmetric 5x5 times vector
        acc[v * ND + 0] = Dm[0] * xv[0] + Dm[1] * xv[1] + Dm[2] * xv[2] + Dm[3] * xv[3] + Dm[4] * xv[4];
        acc[v * ND + 1] = Dm[1] * xv[0] + Dm[5] * xv[1] + Dm[6] * xv[2] + Dm[7] * xv[3] + Dm[8] * xv[4];
        acc[v * ND + 2] = Dm[2] * xv[0] + Dm[6] * xv[1] + Dm[9] * xv[2] + Dm[10] * xv[3] + Dm[11] * xv[4];
        acc[v * ND + 3] = Dm[3] * xv[0] + Dm[7] * xv[1] + Dm[10] * xv[2] + Dm[12] * xv[3] + Dm[13] * xv[4];
        acc[v * ND + 4] = Dm[4] * xv[0] + Dm[8] * xv[1] + Dm[11] * xv[2] + Dm[13] * xv[3] + Dm[14] * xv[4];
    }
#pragma unroll
    for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int v = 0; v < NV; ++v) oacc(sa[s], sax[s], say[s], g[s][2 * v], g[s][2 * v + 1], acc + v * ND);
    if (G) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const bool has = jn[s] != i;
            const TM sr = has ? -arg[s * T + i] : TM(0);
            const TM srx = sr * exrg[s * T + i], sry = sr * eyrg[s * T + i];
            const TM sb = has ? -bdgg[s * T + i] : TM(0);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                TM xj[ND];
#pragma unroll
                for (int l = 0; l < ND; ++l) xj[l] = TM(x[(v * ND + l) * T + jn[s]]);
                racc(sr, srx, sry, xj, acc + v * ND);
#pragma unroll
                for (int l = 2; l < ND; ++l) acc[v * ND + l] = fma(sb, xj[l], acc[v * ND + l]);
            }
        }
    }
}

// y = K x (mode 0), or y = 2^-e (b - K x) with partial sums of |y|^2 of the
// stored y (mode 1), e = sexp[system] (0 when sexp is NULL): an FP32 Krylov
// basis keeps its first vector near unit size whatever the size of b.
// K_ii = D_i (symmetric, 15 stored values), K_ij = -O_ij.  TX: type of x, TM:
// type of the operator data and of the arithmetic (mode 1 is FP64 only), TY:
// type of y.
template <typename TX, typename TM, typename TY, bool G = false>
__global__ void k_spmv(DeviceMesh d, const TM *__restrict__ Dg, const TM *__restrict__ alg,
                       const TM *__restrict__ exg, const TM *__restrict__ eyg, const TX *__restrict__ x,
                       TY *__restrict__ y, int mode, const double *__restrict__ b, double *__restrict__ part,
                       int pstride, const int32_t *__restrict__ sexp = nullptr, const TM *__restrict__ arg = nullptr,
                       const TM *__restrict__ exrg = nullptr, const TM *__restrict__ eyrg = nullptr,
                       const TM *__restrict__ bdgg = nullptr)
{
    __shared__ double sh[32 * NV];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double nr[NV] = {0, 0, 0, 0};
    if (i < T) {
        TM acc[NX];
        cell_apply<TX, TM, G>(d, Dg, alg, exg, eyg, x, i, acc, arg, exrg, eyrg, bdgg);
        if (mode == 0) {
#pragma unroll
            for (int q = 0; q < NX; ++q) y[q * T + i] = TY(acc[q]);
        } else {
            const int c = d.blk_case[blockIdx.x];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double sig = sexp ? pow2(-sexp[4 * c + v]) : 1.0;
#pragma unroll
                for (int l = 0; l < ND; ++l) {
                    const double rv = b[(v * ND + l) * T + i] - double(acc[v * ND + l]);
                    const TY st = TY(rv * sig);
                    y[(v * ND + l) * T + i] = st;
                    nr[v] += double(st) * double(st);
                }
            }
        }
    }
    if (mode >= 1) {
        block_sum4(nr, sh);
        if (threadIdx.x == 0)
            for (int v = 0; v < NV; ++v) part[(blockIdx.x * NV + v) * pstride + 0] = nr[v];
    }
}

// y = K z with the first Gram-Schmidt pass fused in (the FP32-basis inner
// cycles): each thread keeps its cell's y_i in registers and forms the
// products with V_0..V_j at the same cell, so the new basis vector is not read
// back from HBM by a separate dot-product kernel.  part[blk][v][k] =
// sum over the block's cells of <V_k, y>_v: FP32 products and warp sums (as
// k_dots), each warp's sums widened to FP64 and added across the block's warps
// in order.  Deterministic; a different summation order than k_dots, so the
// iterates agree with the unfused path to rounding.  J > 0: the Arnoldi index
// j = J - 1 is a compile-time constant, the products with all J basis vectors
// are formed before one block-wide pass sums them (one barrier instead of two
// per vector); the same operations in the same order as the loop over k.
template <int J = 0>
__global__ void __launch_bounds__(kBlock, 3)
    k_spmv_dots(DeviceMesh d, const float *__restrict__ Dg, const float *__restrict__ alg,
                const float *__restrict__ exg, const float *__restrict__ eyg, const float *__restrict__ x,
                float *__restrict__ y, const float *__restrict__ V, int j, double *__restrict__ part, int pstride)
{
    __shared__ float sh[kBlock / 32][J > 0 ? J : 1][NV];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[NX];
#pragma unroll
    for (int q = 0; q < NX; ++q) acc[q] = 0.0f;
    if (i < T) {
        cell_apply<float, float, false>(d, Dg, alg, exg, eyg, x, i, acc);
#pragma unroll
        for (int q = 0; q < NX; ++q) y[q * T + i] = acc[q];
    }
    const int64_t vs = (int64_t)NX * T;
    if constexpr (J > 0) {
        float sv[J][NV];
#pragma unroll
        for (int k = 0; k < J; ++k)
#pragma unroll
            for (int v = 0; v < NV; ++v) sv[k][v] = 0.0f;
        if (i < T) {
#pragma unroll
            for (int k = 0; k < J; ++k) {
                const float *vk = V + k * vs;
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int l = 0; l < ND; ++l) sv[k][v] = fmaf(vk[(v * ND + l) * T + i], acc[v * ND + l], sv[k][v]);
            }
        }
#pragma unroll
        for (int k = 0; k < J; ++k)
#pragma unroll
            for (int v = 0; v < NV; ++v)
                for (int o = 16; o > 0; o >>= 1) sv[k][v] += __shfl_down_sync(0xffffffffu, sv[k][v], o);
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < J; ++k)
#pragma unroll
                for (int v = 0; v < NV; ++v) sh[warp][k][v] = sv[k][v];
        __syncthreads();
        if (threadIdx.x < J * NV) {
            const int k = threadIdx.x / NV, v = threadIdx.x % NV;
            double t = 0.0;
            for (int w = 0; w < kBlock / 32; ++w) t += double(sh[w][k][v]);
            part[(blockIdx.x * NV + v) * pstride + k] = t;
        }
    } else {
        for (int k = 0; k <= j; ++k) {
            float sv[NV] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (i < T) {
                const float *vk = V + k * vs;
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int l = 0; l < ND; ++l) sv[v] = fmaf(vk[(v * ND + l) * T + i], acc[v * ND + l], sv[v]);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v)
                for (int o = 16; o > 0; o >>= 1) sv[v] += __shfl_down_sync(0xffffffffu, sv[v], o);
            if (lane == 0)
#pragma unroll
                for (int v = 0; v < NV; ++v) sh[warp][0][v] = sv[v];
            __syncthreads();
            if (threadIdx.x < NV) {
                double t = 0.0;
                for (int w = 0; w < kBlock / 32; ++w) t += double(sh[w][0][threadIdx.x]);
                part[(blockIdx.x * NV + threadIdx.x) * pstride + k] = t;
            }
            __syncthreads();
        }
    }
}

// ---- double-FP32 arithmetic for the refinement residual of the mixed mode.
// A value is the unevaluated sum h + l of two FP32 numbers (about 48
// significant bits; Dekker 1971).  The product of two high parts is exact as
// p + e with e = fma(a, b, -p); sums use Knuth's TwoSum (TAOCP vol. 2, 4.2.2),
// whose rounding error is exact; the small cross terms a_h b_l + a_l b_h are
// plain FP32.  The _rn intrinsics keep the compiler from contracting or
// reordering these steps.  GB300 runs FP32 at 64 times its FP64 rate, so the
// 13 FP32 operations of a product-sum cost far less than one DFMA.

// 2^-e v = h + l on the integer pipe (no FP64 instruction; e is applied to the
// exponent field): h holds the upper 24 significant bits (truncated), l the
// next 29 rounded to 24, so |2^-e v - h - l| <= 2^-47 |2^-e v|.  The residual
// scales each system by 2^-e ~ 1/|b|, against which smaller parts do not
// count: below 2^-74 only h is kept, below 2^-126 nothing (with operator
// entries <= 2^30 either drop is under 2^-68 |2^-e b| per term).  Returns
// false for 2^-e v >= 2^128 or a value that is not finite; that cell then
// takes the FP64 operator.
__device__ __forceinline__ bool df_split(double v, int e, float &h, float &l)
{
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const unsigned hw = (unsigned)(u >> 32), lw = (unsigned)u;
    const int E = (int)((hw >> 20) & 0x7FFu);           // biased FP64 exponent
    const int Es = E - e;                                // that of 2^-e v
    h = l = 0.0f;
    if (E == 2047 || (E != 0 && Es > 1150)) return false;
    if (E == 0 || Es < 897) return true;                 // zero, FP64 subnormal, or negligible
    const unsigned sgn = hw & 0x80000000u;
    h = __uint_as_float(sgn | ((unsigned)(Es - 896) << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    if (Es >= 949) {
        // the remaining 29 bits times 2^(Es - 1075), a normal FP32 power of two here
        const float r = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), __uint_as_float((unsigned)(Es - 948) << 23));
        l = sgn ? -r : r;
    }
    return true;
}

// (sh, sl) += (ah, al) (bh, bl)
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float &sh, float &sl)
{
    const float p = __fmul_rn(ah, bh);
    const float e = __fmaf_rn(ah, bh, -p);
    const float t = __fadd_rn(sh, p);
    const float z = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, __fadd_rn(e, __fmaf_rn(ah, bl, __fmul_rn(al, bh)))));
}

// (bh, bl) - (sh, sl), rounded to FP32
__device__ __forceinline__ float df_sub_round(float bh, float bl, float sh, float sl)
{
    const float t = __fsub_rn(bh, sh);
    const float z = __fsub_rn(t, bh);
    const float err = __fadd_rn(__fsub_rn(bh, __fsub_rn(t, z)), __fsub_rn(-sh, z));
    return __fadd_rn(t, __fadd_rn(err, __fsub_rn(bl, sl)));
}

// FP64 fallback of k_resid_df for variable v of cell i: out = 2^-e (b - K x)
template <bool G>
__device__ __noinline__ void resid64_cell(const DeviceMesh &d, const double *__restrict__ x,
                                          const double *__restrict__ b, int64_t i, int v, int e, float *out)
{
    double acc[NX];
    cell_apply<double, double, G>(d, d.D, d.alpha, d.ex, d.ey, x, i, acc, d.alr, d.exr, d.eyr, d.bdg);
    for (int l = 0; l < ND; ++l) out[l] = float((b[(v * ND + l) * d.T + i] - acc[v * ND + l]) * pow2(-e));
}

// V_0 = 2^-e (b - K x) in FP32 and partial |V_0|^2 (as k_spmv mode 1 with an
// FP32 basis), in double-FP32 arithmetic: the operator as FP32 pairs D2 ([30][T]:
// the 15 diagonal-block values, then their low parts) and S2 ([18][T]: sa,
// sa dx, sa dy of each neighbour, then their low parts), 2^-e x and 2^-e b
// split on the fly, so the sums come out scaled.  One thread per cell and
// variable (the double-FP32 chains are latency-bound: many small threads hide
// it better than one thread per cell); block q of the 1-D grid takes variable
// q % 4 of cell block q / 4, so the four blocks of a cell block run together
// and share the operator through L2.  A value outside the split range sends
// the thread to the FP64 operator.  Each thread's five squares are summed in
// FP32 (the scaled vector is near unit size).  G: global normal equations, the
// transpose form from the reverse-slot pairs SR2 ([18][T], as S2) on all five
// unknowns of each neighbour.
template <bool G>
__global__ void __launch_bounds__(kBlock, 4) k_resid_df(DeviceMesh d, const float *__restrict__ D2,
                                                       const float *__restrict__ S2, const double *__restrict__ x,
                                                       float *__restrict__ y, const double *__restrict__ b,
                                                       double *__restrict__ part, int pstride,
                                                       const int32_t *__restrict__ sexp,
                                                       const float *__restrict__ SR2 = nullptr,
                                                       const float *__restrict__ SB2 = nullptr)
{
    __shared__ double sh[kBlock / 32];
    const int64_t T = d.T;
    const int v = blockIdx.x & 3;
    const int64_t blk = blockIdx.x >> 2;
    const int64_t i = blk * kBlock + threadIdx.x;
    double nr = 0.0;
    if (i < T) {
        const int e = sexp[4 * d.blk_case[blk] + v];
        int64_t jn[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int j = d.nb[s * T + i];
            jn[s] = j >= 0 ? j : i;
        }
        // the cell's own block first, then the neighbours: the two phases keep
        // fewer values live (no spills at the register cap), and the sums run
        // in the same order
        constexpr int NG = G ? ND : 2;                    // neighbour unknowns used
        double xv[ND], gv[3][NG], bv[ND];
        float dp[30], op[18], rp[G ? 18 : 1], bp[G ? 6 : 1];
#pragma unroll
        for (int l = 0; l < ND; ++l) xv[l] = x[(v * ND + l) * T + i];
#pragma unroll
        for (int q = 0; q < 30; ++q) dp[q] = D2[q * T + i];
        bool ok = true;
        float xh[ND], xl[ND], gh[3][NG], gl[3][NG], ah[ND], al[ND], out[ND];
#pragma unroll
        for (int l = 0; l < ND; ++l) {
            ok &= df_split(xv[l], e, xh[l], xl[l]);
            ah[l] = al[l] = 0.0f;
        }
        // symmetric 5x5 block: entry (a, k) in the upper-triangle order
        constexpr int kIdx[5][5] = {{0, 1, 2, 3, 4}, {1, 5, 6, 7, 8}, {2, 6, 9, 10, 11}, {3, 7, 10, 12, 13},
                                    {4, 8, 11, 13, 14}};
#pragma unroll
        for (int a = 0; a < ND; ++a)
#pragma unroll
            for (int k = 0; k < ND; ++k) df_mac(dp[kIdx[a][k]], dp[15 + kIdx[a][k]], xh[k], xl[k], ah[a], al[a]);
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int l = 0; l < NG; ++l) gv[s][l] = x[(v * ND + l) * T + jn[s]];
#pragma unroll
        for (int q = 0; q < 18; ++q) op[q] = S2[q * T + i];
        if (G) {
#pragma unroll
            for (int q = 0; q < 18; ++q) rp[q] = SR2[q * T + i];
#pragma unroll
            for (int q = 0; q < 6; ++q) bp[q] = SB2[q * T + i];
        }
#pragma unroll
        for (int l = 0; l < ND; ++l) bv[l] = b[(v * ND + l) * T + i];
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int l = 0; l < NG; ++l) ok &= df_split(gv[s][l], e, gh[s][l], gl[s][l]);
        // off-diagonal block of neighbour s (see oacc): sa, sax = sa dx, say = sa dy
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int q = 3 * s;
            df_mac(op[q], op[9 + q], gh[s][0], gl[s][0], ah[0], al[0]);
            df_mac(op[q], op[9 + q], gh[s][1], gl[s][1], ah[1], al[1]);
            df_mac(op[q + 1], op[10 + q], gh[s][0], gl[s][0], ah[2], al[2]);
            df_mac(op[q + 1], op[10 + q], gh[s][1], gl[s][1], ah[3], al[3]);
            df_mac(op[q + 2], op[11 + q], gh[s][0], gl[s][0], ah[3], al[3]);
            df_mac(op[q + 2], op[11 + q], gh[s][1], gl[s][1], ah[4], al[4]);
            if (G) {
                // transpose form (see racc): rows 0 and 1 from all five unknowns
                df_mac(rp[q], rp[9 + q], gh[s][0], gl[s][0], ah[0], al[0]);
                df_mac(rp[q + 1], rp[10 + q], gh[s][NG > 2 ? 2 : 0], gl[s][NG > 2 ? 2 : 0], ah[0], al[0]);
                df_mac(rp[q + 2], rp[11 + q], gh[s][NG > 3 ? 3 : 0], gl[s][NG > 3 ? 3 : 0], ah[0], al[0]);
                df_mac(rp[q], rp[9 + q], gh[s][1], gl[s][1], ah[1], al[1]);
                df_mac(rp[q + 1], rp[10 + q], gh[s][NG > 3 ? 3 : 0], gl[s][NG > 3 ? 3 : 0], ah[1], al[1]);
                df_mac(rp[q + 2], rp[11 + q], gh[s][NG > 4 ? 4 : 0], gl[s][NG > 4 ? 4 : 0], ah[1], al[1]);
                // diagonal coupling of the unknowns 3..5 (second-derivative equations)
#pragma unroll
                for (int l = 2; l < ND; ++l)
                    df_mac(bp[s], bp[3 + s], gh[s][NG > l ? l : 0], gl[s][NG > l ? l : 0], ah[l], al[l]);
            }
        }
#pragma unroll
        for (int l = 0; l < ND; ++l) {
            float bh, bl;
            ok &= df_split(bv[l], e, bh, bl);
            out[l] = df_sub_round(bh, bl, ah[l], al[l]);
        }
        if (!ok) resid64_cell<G>(d, x, b, i, v, e, out);   // a value outside the split range
        float sq = 0.0f;
#pragma unroll
        for (int l = 0; l < ND; ++l) {
            y[(v * ND + l) * T + i] = out[l];
            sq = __fmaf_rn(out[l], out[l], sq);
        }
        nr = double(sq);
    }
    for (int o = 16; o > 0; o >>= 1) nr += __shfl_down_sync(0xffffffffu, nr, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nr;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) t += sh[w];
        part[(blk * NV + v) * pstride + 0] = t;
    }
}

// 2^e f as an FP64 value, formed on the integer pipe (exact; an FP32 subnormal
// f, below 2^-126 of the scale, counts as zero)
__device__ __forceinline__ double f2d_pow2(float f, int e)
{
    const unsigned u = __float_as_uint(f);
    const int ef = (int)((u >> 23) & 0xFFu);
    if (ef == 0) return 0.0;
    const long long E = (long long)ef - 127 + 1023 + e;
    if (E <= 0 || E >= 2047) return double(f) * pow2(e);
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)E << 52) |
                                    ((unsigned long long)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}

// The right-hand side of k_rhs in double-FP32 arithmetic (the FP32-basis
// solve).  GB300's FP64 pipe made the FP64 kernel (92 FP64 operations per
// cell) its bottleneck; here a cell and variable take the power of two 2^e of
// their largest difference w_j - w_i (formed in FP64), split the scaled
// differences on the integer pipe, multiply them exactly by the weights as FP32
// pairs a0p ([30][T]: the 15 high parts, then the low parts) and sum with
// compensation (df_mac); the normalised pair (high + low, 48 bits) is widened
// on the integer pipe and added in FP64: 32 FP64 operations per cell, b to
// about 2^-48 relative at any magnitude.  A difference that does not split
// (not finite) sends the cell to FP64.  part[blk][v][1] gets the block's |b|^2:
// the scaled high parts squared in FP32, rescaled to the warp's largest 2^e,
// summed in FP32 within the warp and in FP64 across warps.
__global__ void __launch_bounds__(kBlock, 3) k_rhs_df(DeviceMesh d, const float *__restrict__ a0p,
                                                      const double *__restrict__ w, double *__restrict__ b,
                                                      double *__restrict__ part, int pstride)
{
    __shared__ double sh[(kBlock / 32) * NV];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float ss[NV] = {0.0f, 0.0f, 0.0f, 0.0f};      // scaled |b|^2 of this cell
    int ev[NV] = {-1022, -1022, -1022, -1022};    // the scales 2^e
    if (i < T) {
        double wi[NV], du[3][NV];
        int js[3];
        // the cell's weights first: their loads overlap the neighbour gathers
        float ah[3][ND], al[3][ND];
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int l = 0; l < ND; ++l) {
                ah[s][l] = a0p[(s * ND + l) * T + i];
                al[s][l] = a0p[(15 + s * ND + l) * T + i];
            }
#pragma unroll
        for (int v = 0; v < NV; ++v) wi[v] = w[v * T + i];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            js[s] = d.nb[s * T + i];
#pragma unroll
            for (int v = 0; v < NV; ++v) du[s][v] = js[s] >= 0 ? w[v * T + js[s]] - wi[v] : 0.0;
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            int em = 1;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const int E = (int)(((unsigned)__double2hiint(du[s][v]) >> 20) & 0x7FFu);
                em = E > em ? E : em;
            }
            ev[v] = (em == 2047 ? 1023 : em) - 1023;
        }
        // with 2^e the largest difference of its variable, a difference fails to
        // split only when it is not finite: that sends the cell to FP64
        bool ok = true;
#pragma unroll
        for (int s = 0; s < 3; ++s)
#pragma unroll
            for (int v = 0; v < NV; ++v) ok &= isfinite(du[s][v]);
        if (ok) {
            // one variable at a time (ten accumulators live, not forty); each sum
            // runs over the neighbours in order, as the FP64 kernel's does
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                float sh_[ND], sl_[ND];
#pragma unroll
                for (int l = 0; l < ND; ++l) sh_[l] = sl_[l] = 0.0f;
#pragma unroll
                for (int s = 0; s < 3; ++s) {
                    if (js[s] < 0) continue;
                    float dh, dl;
                    df_split(du[s][v], ev[v], dh, dl);
#pragma unroll
                    for (int l = 0; l < ND; ++l) df_mac(ah[s][l], al[s][l], dh, dl, sh_[l], sl_[l]);
                }
#pragma unroll
                for (int l = 0; l < ND; ++l) {
                    // normalise (TwoSum): h + lo = sh + sl exactly
                    const float h = __fadd_rn(sh_[l], sl_[l]);
                    const float z = __fsub_rn(h, sh_[l]);
                    const float lo = __fadd_rn(__fsub_rn(sh_[l], __fsub_rn(h, z)), __fsub_rn(sl_[l], z));
                    b[(v * ND + l) * T + i] = f2d_pow2(h, ev[v]) + f2d_pow2(lo, ev[v]);
                    ss[v] = __fmaf_rn(h, h, ss[v]);
                }
            }
        } else {
            // FP64 as in k_rhs; the norm from the values scaled by 2^-e
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                double acc[ND] = {0.0, 0.0, 0.0, 0.0, 0.0};
                for (int s = 0; s < 3; ++s) {
                    if (js[s] < 0) continue;
                    for (int l = 0; l < ND; ++l) acc[l] += d.a0[(s * ND + l) * T + i] * du[s][v];
                }
                for (int l = 0; l < ND; ++l) {
                    b[(v * ND + l) * T + i] = acc[l];
                    const float h = float(acc[l] * pow2(-ev[v]));
                    ss[v] = __fmaf_rn(h, h, ss[v]);
                }
            }
        }
    }
    // |b|^2 = sum 2^(2e) ss: rescaled to the warp's largest e in FP32 (smaller
    // terms that underflow are below 2^-126 of the largest), summed in FP32
    // within the warp, widened once per warp and summed in FP64 across warps
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        int em = ev[v];
        for (int o = 16; o > 0; o >>= 1) em = max(em, __shfl_xor_sync(0xffffffffu, em, o));
        const int k = 2 * (ev[v] - em);           // <= 0
        float c = k >= -126 ? ss[v] * __uint_as_float((unsigned)(127 + k) << 23) : 0.0f;
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if (lane == 0) sh[warp * NV + v] = double(c) * pow2(em) * pow2(em);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int v = 0; v < NV; ++v) {
            double t = 0.0;
            for (int k = 0; k < kBlock / 32; ++k) t += sh[k * NV + v];
            part[(blockIdx.x * NV + v) * pstride + 1] = t;
        }
}

// Forward block-ILU relation for the listed rows (or all rows when rows == nullptr):
//   z_i = P_i (r_i + sum_{k<i} O_ik zin_k)      (use_nb = 0: z_i = P_i r_i)
// use_nb = 2: the first sweep with the block-diagonal pass folded in, zin_k =
// P_k r_k formed here from the lower neighbours' factors and right-hand sides
// (rounded to TZ as the separate pass stores them), which saves the write and
// the re-read of that pass; the neighbours' data mostly comes from L2.
// TR: type of r, TZ: type of z, TM: type of the factors and of the arithmetic.
// rcopy (may be NULL): also store TZ(r_i), so that later sweeps read r in the
// working precision (same values as converting r again).  Own data (r, P) is
// loaded before the neighbour gathers so that the two overlap.
// TP: storage type of the factors (TM, or FP16 for the mixed mode's FP32
// preconditioner), widened to TM on load.
// G: global normal equations, the transpose form with the reverse-slot
// coefficients arg, exrg, eyrg on all five unknowns of the neighbour.
// a neighbour's value: through L2 in the sync-free solves (written by another
// block of the same launch), a plain load otherwise
template <bool SF, typename T>
__device__ __forceinline__ T ldx(const T *p)
{
    if constexpr (SF) return __ldcg(p);
    else return *p;
}

// A bounded wait of the sync-free solves gives up after 1 s (a correct solve
// waits a few microseconds per level).
constexpr uint64_t kWaitLimitNs = 1000000000ull;

// The forward relation of row i (see k_ilu_fwd).  SF: the sync-free exact
// solve, which waits for each lower neighbour's ready tag before reading its
// value (through L2) and publishes its own row's tag after the store.
template <typename TR, typename TZ, typename TM, typename TP, bool G, bool SF>
__device__ __forceinline__ void ilu_fwd_row(const DeviceMesh &d, const TP *__restrict__ Pg,
                                            const TP *__restrict__ alg, const TP *__restrict__ exg,
                                            const TP *__restrict__ eyg, int64_t i, const TR *r, const TZ *zin,
                                            TZ *zout, int use_nb, TZ *__restrict__ rcopy, const TP *__restrict__ arg,
                                            const TP *__restrict__ exrg, const TP *__restrict__ eyrg,
                                            const TP *__restrict__ bdgg, int32_t *sf_flag, int32_t sf_tag,
                                            int32_t *sf_err)
{
    const int64_t T = d.T;
    TM y[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) y[k] = TM(r[k * T + i]);
    TM Pm[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) Pm[k] = TM(Pg[k * T + i]);
    if (rcopy)
#pragma unroll
        for (int k = 0; k < NX; ++k) rcopy[k * T + i] = TZ(y[k]);
    if (SF) {
        // every lower neighbour's tag first (one round trip for all of them)
        const int32_t *wf[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int j = d.nb[s * T + i];
            wf[s] = (j >= 0 && j < i) ? sf_flag + j : nullptr;
        }
        bounded_wait_all(wf[0], wf[1], wf[2], sf_tag, sf_err, kWaitLimitNs);
    }
    if (use_nb) {
        // unknowns of a neighbour that its off-diagonal block reaches
        constexpr int NA = G ? ND : 2;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            // every slot's loads are issued (a slot that is not a lower
            // neighbour reads the cell's own data, which is discarded), only the
            // accumulation is conditional: the gathers of the slots overlap
            const int jn = d.nb[s * T + i];
            const bool lower = jn >= 0 && jn < i;
            const int64_t j = lower ? jn : i;
            const TM sa = TM(alg[s * T + i]), sax = sa * TM(exg[s * T + i]), say = sa * TM(eyg[s * T + i]);
            TM zn[NV][NA];
            if (use_nb == 2) {
                TM rj[NX];
#pragma unroll
                for (int k = 0; k < NX; ++k) rj[k] = TM(r[k * T + j]);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    TM pa[ND];
#pragma unroll
                    for (int c = 0; c < ND; ++c) pa[c] = TM(Pg[(a * ND + c) * T + j]);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        TM t = TM(0);
#pragma unroll
                        for (int c = 0; c < ND; ++c) t = fma(pa[c], rj[v * ND + c], t);
                        zn[v][a] = TM(TZ(t));
                    }
                }
            } else if (SF) {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int a = 0; a < NA; ++a) zn[v][a] = TM(__ldcg(zin + (v * ND + a) * T + j));
            } else {
#pragma unroll
                for (int v = 0; v < NV; ++v)
#pragma unroll
                    for (int a = 0; a < NA; ++a) zn[v][a] = TM(zin[(v * ND + a) * T + j]);
            }
            if (!lower) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v) oacc(sa, sax, say, zn[v][0], zn[v][1], y + v * ND);
            if constexpr (G) {
                const TM sr = TM(arg[s * T + i]), srx = sr * TM(exrg[s * T + i]), sry = sr * TM(eyrg[s * T + i]);
                const TM sb = TM(bdgg[s * T + i]);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    racc(sr, srx, sry, zn[v], y + v * ND);
#pragma unroll
                    for (int l = 2; l < ND; ++l) y[v * ND + l] = fma(sb, zn[v][l], y[v * ND + l]);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < ND; ++a) {
            TM s = TM(0);
#pragma unroll
            for (int c = 0; c < ND; ++c) s = fma(Pm[a * ND + c], y[v * ND + c], s);
            zout[(v * ND + a) * T + i] = TZ(s);
        }
    if (SF) publish(sf_flag + i, sf_tag);
}

template <typename TR, typename TZ, typename TM, typename TP = TM, bool G = false>
__global__ void k_ilu_fwd(DeviceMesh d, const TP *__restrict__ Pg, const TP *__restrict__ alg,
                          const TP *__restrict__ exg, const TP *__restrict__ eyg, const int32_t *__restrict__ rows,
                          int64_t nrows, const TR *r, const TZ *zin, TZ *zout, int use_nb, TZ *__restrict__ rcopy,
                          const TP *__restrict__ arg = nullptr, const TP *__restrict__ exrg = nullptr,
                          const TP *__restrict__ eyrg = nullptr, const TP *__restrict__ bdgg = nullptr)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nrows) return;
    const int64_t i = rows ? rows[q] : q;
    ilu_fwd_row<TR, TZ, TM, TP, G, false>(d, Pg, alg, exg, eyg, i, r, zin, zout, use_nb, rcopy, arg, exrg, eyrg,
                                          bdgg, nullptr, 0, nullptr);
}

// Backward block-ILU relation: x_i = z_i + P_i sum_{j>i} O_ij xin_j (own data
// loaded before the neighbour gathers; with no upper neighbour the sum is 0
// and x_i = z_i exactly).
template <typename TZ, typename TM, typename TP, bool G, bool SF>
__device__ __forceinline__ void ilu_bwd_row(const DeviceMesh &d, const TP *__restrict__ Pg,
                                            const TP *__restrict__ alg, const TP *__restrict__ exg,
                                            const TP *__restrict__ eyg, int64_t i, const TZ *z, const TZ *xin,
                                            TZ *xout, const TP *__restrict__ arg, const TP *__restrict__ exrg,
                                            const TP *__restrict__ eyrg, const TP *__restrict__ bdgg,
                                            int32_t *sf_flag, int32_t sf_tag, int32_t *sf_err)
{
    const int64_t T = d.T;
    TM zi[NX], y[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) {
        zi[k] = TM(z[k * T + i]);
        y[k] = TM(0);
    }
    TM Pm[25];
#pragma unroll
    for (int k = 0; k < 25; ++k) Pm[k] = TM(Pg[k * T + i]);
    if (SF) {
        // every upper neighbour's tag first (one round trip for all of them)
        const int32_t *wf[3];
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const int j = d.nb[s * T + i];
            wf[s] = j > i ? sf_flag + j : nullptr;
        }
        bounded_wait_all(wf[0], wf[1], wf[2], sf_tag, sf_err, kWaitLimitNs);
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int j = d.nb[s * T + i];
        if (j <= i) continue;
        const TM sa = TM(alg[s * T + i]), sax = sa * TM(exg[s * T + i]), say = sa * TM(eyg[s * T + i]);
#pragma unroll
        for (int v = 0; v < NV; ++v)
            oacc(sa, sax, say, TM(ldx<SF>(xin + (v * ND + 0) * T + j)), TM(ldx<SF>(xin + (v * ND + 1) * T + j)),
                 y + v * ND);
        if (G) {
            const TM sr = TM(arg[s * T + i]), srx = sr * TM(exrg[s * T + i]), sry = sr * TM(eyrg[s * T + i]);
            const TM sb = TM(bdgg[s * T + i]);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                TM xj[ND];
#pragma unroll
                for (int l = 0; l < ND; ++l) xj[l] = TM(ldx<SF>(xin + (v * ND + l) * T + j));
                racc(sr, srx, sry, xj, y + v * ND);
#pragma unroll
                for (int l = 2; l < ND; ++l) y[v * ND + l] = fma(sb, xj[l], y[v * ND + l]);
            }
        }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < ND; ++a) {
            TM s = zi[v * ND + a];
#pragma unroll
            for (int c = 0; c < ND; ++c) s = fma(Pm[a * ND + c], y[v * ND + c], s);
            xout[(v * ND + a) * T + i] = TZ(s);
        }
    if (SF) publish(sf_flag + i, sf_tag);
}

template <typename TZ, typename TM, typename TP = TM, bool G = false>
__global__ void __launch_bounds__(kBlock, sizeof(TM) == 4 ? 3 : 1)
    k_ilu_bwd(DeviceMesh d, const TP *__restrict__ Pg, const TP *__restrict__ alg, const TP *__restrict__ exg,
              const TP *__restrict__ eyg, const int32_t *__restrict__ rows, int64_t nrows, const TZ *z, const TZ *xin,
              TZ *xout, const TP *__restrict__ arg = nullptr, const TP *__restrict__ exrg = nullptr,
              const TP *__restrict__ eyrg = nullptr, const TP *__restrict__ bdgg = nullptr)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nrows) return;
    const int64_t i = rows ? rows[q] : q;
    ilu_bwd_row<TZ, TM, TP, G, false>(d, Pg, alg, exg, eyg, i, z, xin, xout, arg, exrg, eyrg, bdgg, nullptr, 0,
                                      nullptr);
}

// ---- sync-free exact triangular solves (GKS_PC_ILU_EXACT).  One launch per
// relation instead of one per level: persistent blocks take tickets for
// kBlock-row ranges in RCM order (forward: increasing rows, backward:
// decreasing), so a block only ever waits on rows of tickets taken before its
// own, by blocks that are already running; within a range a row waits on
// lower (upper) rows of the same range, which earlier threads finish (threads
// of a warp make independent progress).  Every row waits for its lower
// (upper) neighbours' tags (bounded_wait, at most kWaitLimitNs each), reads
// their values through L2 and publishes its own tag.  The tags of the two
// relations of application e are 2e + 1 and 2e + 2, so no flag is reset
// between applications.  ctl: [0] epoch e, [1] forward and [2] backward
// tickets, [3] sticky wait error.  The arithmetic of a row is that of the
// level-scheduled launches, so the results are the same bit for bit.

constexpr int kSfBlocksPerSm = 2;       // persistent blocks per SM of the sync-free solves

// Next application: new epoch, tickets back to 0 (clear = 1: only the error word).
__global__ void k_sf_begin(int32_t *ctl, int clear)
{
    if (threadIdx.x != 0) return;
    if (clear) {
        ctl[3] = 0;
        return;
    }
    ctl[0] += 1;
    ctl[1] = 0;
    ctl[2] = 0;
}

template <typename TR, typename TZ, typename TM, typename TP, bool G>
__global__ void __launch_bounds__(kBlock) k_ilu_fwd_sf(DeviceMesh d, const TP *__restrict__ Pg,
                                                       const TP *__restrict__ alg, const TP *__restrict__ exg,
                                                       const TP *__restrict__ eyg, const TR *r, TZ *z,
                                                       int32_t *flag, int32_t *ctl,
                                                       const TP *__restrict__ arg = nullptr,
                                                       const TP *__restrict__ exrg = nullptr,
                                                       const TP *__restrict__ eyrg = nullptr,
                                                       const TP *__restrict__ bdgg = nullptr)
{
    __shared__ int32_t ticket;
    const int64_t T = d.T;
    const int64_t nt = (T + kBlock - 1) / kBlock;
    const int32_t tag = 2 * ctl[0] + 1;
    for (;;) {
        if (threadIdx.x == 0) ticket = atomicAdd(ctl + 1, 1);
        __syncthreads();
        const int64_t tk = ticket;
        __syncthreads();
        if (tk >= nt) return;
        const int64_t i = tk * kBlock + threadIdx.x;
        if (i < T)
            ilu_fwd_row<TR, TZ, TM, TP, G, true>(d, Pg, alg, exg, eyg, i, r, z, z, 1, nullptr, arg, exrg, eyrg, bdgg,
                                                 flag, tag, ctl + 3);
    }
}

template <typename TZ, typename TM, typename TP, bool G>
__global__ void __launch_bounds__(kBlock) k_ilu_bwd_sf(DeviceMesh d, const TP *__restrict__ Pg,
                                                       const TP *__restrict__ alg, const TP *__restrict__ exg,
                                                       const TP *__restrict__ eyg, TZ *x, int32_t *flag,
                                                       int32_t *ctl, const TP *__restrict__ arg = nullptr,
                                                       const TP *__restrict__ exrg = nullptr,
                                                       const TP *__restrict__ eyrg = nullptr,
                                                       const TP *__restrict__ bdgg = nullptr)
{
    __shared__ int32_t ticket;
    const int64_t T = d.T;
    const int64_t nt = (T + kBlock - 1) / kBlock;
    const int32_t tag = 2 * ctl[0] + 2;
    for (;;) {
        if (threadIdx.x == 0) ticket = atomicAdd(ctl + 2, 1);
        __syncthreads();
        const int64_t tk = ticket;
        __syncthreads();
        if (tk >= nt) return;
        const int64_t i = T - 1 - (tk * kBlock + threadIdx.x);
        if (i >= 0)
            ilu_bwd_row<TZ, TM, TP, G, true>(d, Pg, alg, exg, eyg, i, x, x, x, arg, exrg, eyrg, bdgg, flag, tag,
                                             ctl + 3);
    }
}

// ---- two backward preconditioner sweeps per launch: the second sweep of a
// cell needs its upper neighbours' first-sweep values, which each thread forms
// itself from the neighbours' own data (factors, z, and their upper
// neighbours' values), with exactly the arithmetic and roundings of a separate
// first sweep, so the results are the same bit for bit.  One launch instead of
// two reads each cell's factors and z once and writes x once; the neighbours'
// data mostly comes from L2 (a neighbour is a few hundred to a thousand cells
// away in RCM order).  Measured at 1M cells (ncu, one launch): 101 us against
// 55 + 59 us for the two sweeps.  The same fusion of the forward pair (which
// also has to form the neighbours' neighbours' z^0 = P r) took 195 us against
// 69 + 56 us, its three levels of dependent gathers exposed, and is not used.
// Per-cell equations only (the global normal equations' reverse slots keep one
// sweep per launch).

// x^{q+2} = B(B(x^q)) with B(x)_i = z_i + P_i sum_{j>i} O_ij x_j: two backward
// sweeps in one launch (x^q = xin; x^0 = z).
template <typename TZ, typename TM, typename TP>
__global__ void __launch_bounds__(kBlock, sizeof(TM) == 4 ? 3 : 2) k_ilu_bwd2(DeviceMesh d, const TP *__restrict__ Pg,
                                                      const TP *__restrict__ alg, const TP *__restrict__ exg,
                                                      const TP *__restrict__ eyg, const TZ *z, const TZ *xin,
                                                      TZ *xout)
{
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    TM y[NX];
#pragma unroll
    for (int k = 0; k < NX; ++k) y[k] = TM(0);
#pragma unroll 1
    for (int s = 0; s < 3; ++s) {
        const int j = d.nb[s * T + i];
        if (j <= i) continue;
        const TM sa = TM(alg[s * T + i]), sax = sa * TM(exg[s * T + i]), say = sa * TM(eyg[s * T + i]);
        // the first sweep at j, rows 0 and 1: x^{q+1}_j = z_j + P_j sum_{k>j} O_jk x^q_k
        TM yj[NX];
#pragma unroll
        for (int q = 0; q < NX; ++q) yj[q] = TM(0);
        // the three slots' loads issued together (a slot that is not an upper
        // neighbour of j reads j's own values, discarded); only the sums are
        // conditional, in slot order
#pragma unroll
        for (int s2 = 0; s2 < 3; ++s2) {
            const int kn = d.nb[s2 * T + j];
            const bool upper = kn > j;
            const int64_t k = upper ? kn : j;
            const TM sb = TM(alg[s2 * T + j]), sbx = sb * TM(exg[s2 * T + j]), sby = sb * TM(eyg[s2 * T + j]);
            TM xk[NV][2];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                xk[v][0] = TM(xin[(v * ND + 0) * T + k]);
                xk[v][1] = TM(xin[(v * ND + 1) * T + k]);
            }
            if (!upper) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v) oacc(sb, sbx, sby, xk[v][0], xk[v][1], yj + v * ND);
        }
        TM x1[NV][2];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            TM pa[ND];
#pragma unroll
            for (int c = 0; c < ND; ++c) pa[c] = TM(Pg[(a * ND + c) * T + j]);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                TM t = TM(z[(v * ND + a) * T + j]);
#pragma unroll
                for (int c = 0; c < ND; ++c) t = fma(pa[c], yj[v * ND + c], t);
                x1[v][a] = TM(TZ(t));
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) oacc(sa, sax, say, x1[v][0], x1[v][1], y + v * ND);
    }
    // the cell's own factor and z last, after the gathers (fewer values live
    // while the neighbours' first sweep is formed)
    TM Pm[25], zi[NX];
#pragma unroll
    for (int k = 0; k < 25; ++k) Pm[k] = TM(Pg[k * T + i]);
#pragma unroll
    for (int k = 0; k < NX; ++k) zi[k] = TM(z[k * T + i]);
#pragma unroll
    for (int v = 0; v < NV; ++v)
#pragma unroll
        for (int a = 0; a < ND; ++a) {
            TM t = zi[v * ND + a];
#pragma unroll
            for (int c = 0; c < ND; ++c) t = fma(Pm[a * ND + c], y[v * ND + c], t);
            xout[(v * ND + a) * T + i] = TZ(t);
        }
}

// Partial dot products <V_k, w> of the four variables over one block of
// kBlock cells: grid (k, block), blockIdx.x = k so that the j + 1 blocks of a
// cell block run together and read w once from HBM.  64 threads per variable,
// four cells each (64 apart), all 40 loads issued before the sums (read-only
// kernels need many bytes in flight); the warp sums then the two warps of a
// variable give part[blk][v][k].  Fixed order: the sums are deterministic.
// TB: type of the stored basis.  An FP64 basis is multiplied and summed in
// FP64; an FP32 basis (the inner cycles of the mixed mode) in FP32 within a
// warp (640 products), each warp's sum then widened once and summed across
// warps and blocks in FP64, so that the FP64 pipe sees almost nothing.
template <typename TB>
__global__ void __launch_bounds__(kDotThreads, 3) k_dots(int64_t T, int64_t nblk, const TB *__restrict__ V,
                                                         const TB *__restrict__ w, double *__restrict__ part,
                                                         int pstride)
{
    constexpr int kPerVar = kDotThreads / NV;          // 64 threads (two warps) per variable
    constexpr int kCells = kBlock / kPerVar;           // 4 cells per thread
    __shared__ double sh[kDotThreads / 32];
    const int k = blockIdx.x;
    const int v = threadIdx.x / kPerVar, t = threadIdx.x % kPerVar;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const TB *vk = V + (int64_t)k * NX * T + (int64_t)v * ND * T;
    const TB *wv = w + (int64_t)v * ND * T;
    for (int64_t b = blockIdx.y; b < nblk; b += gridDim.y) {
        const int64_t c0 = b * kBlock + t;
        TB st = TB(0);
#pragma unroll
        for (int q = 0; q < kCells; ++q) {
            const int64_t i = c0 + q * kPerVar;
#pragma unroll
            for (int l = 0; l < ND; ++l) st = i < T ? fma(vk[l * T + i], wv[l * T + i], st) : st;
        }
        // warp sum in the basis precision, widened once per warp
        for (int o = 16; o > 0; o >>= 1) st += __shfl_down_sync(0xffffffffu, st, o);
        if (lane == 0) sh[warp] = double(st);
        __syncthreads();
        if (threadIdx.x < NV) part[(b * NV + threadIdx.x) * pstride + k] = sh[2 * threadIdx.x] + sh[2 * threadIdx.x + 1];
        __syncthreads();
    }
}

// w -= sum_{k<=j} c[s][k] V_k for running systems s = case * 4 + v (c: the
// Gram-Schmidt coefficients of the unnormalised basis), w = 0 for the others;
// optional partial |w|^2 per block.  The arithmetic is in the basis precision
// TB (FP32 for the inner cycles of the mixed mode); the block's coefficients
// are rounded to TB once, in shared memory.  J > 0: the Arnoldi index j = J - 1
// is a compile-time constant and every load of the four systems is issued
// before the arithmetic (systems that are not running read their vectors too
// and store zeros), for more bytes in flight per thread; the same operations
// in the same order as the loop over k.
template <typename TB, int J = 0>
__global__ void k_orth_update(DeviceMesh d, const TB *__restrict__ V, TB *__restrict__ w, int j,
                              const double *__restrict__ hc, int hstride, const int32_t *__restrict__ ctl, int ns,
                              double *__restrict__ part, int pstride, int want_norm)
{
    if (J > 0) j = J - 1;
    __shared__ double sh[32 * NV];
    __shared__ TB shc[NV][kMaxRestart];
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t vs = (int64_t)NX * T;
    const int c = d.blk_case[blockIdx.x];
    for (int q = threadIdx.x; q < NV * (j + 1); q += blockDim.x)
        shc[q / (j + 1)][q % (j + 1)] = TB(hc[(4 * c + q / (j + 1)) * hstride + q % (j + 1)]);
    __syncthreads();
    TB nrm[NV] = {0, 0, 0, 0};
    if (J > 0 && i < T) {
        bool run[NV];
        TB wv[NV][ND], vk[NV][J > 0 ? J : 1][ND];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            run[v] = ctl[kCtlRunning * ns + 4 * c + v] != 0;
#pragma unroll
            for (int l = 0; l < ND; ++l) wv[v][l] = w[(v * ND + l) * T + i];
#pragma unroll
            for (int k = 0; k < J; ++k)
#pragma unroll
                for (int l = 0; l < ND; ++l) vk[v][k][l] = V[k * vs + (v * ND + l) * T + i];
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
#pragma unroll
            for (int k = 0; k < J; ++k)
#pragma unroll
                for (int l = 0; l < ND; ++l) wv[v][l] = fma(-shc[v][k], vk[v][k][l], wv[v][l]);
#pragma unroll
            for (int l = 0; l < ND; ++l) {
                const TB o = run[v] ? wv[v][l] : TB(0);
                w[(v * ND + l) * T + i] = o;
                nrm[v] = fma(o, o, nrm[v]);
            }
        }
    } else if (i < T) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const int sy = 4 * c + v;
            if (!ctl[kCtlRunning * ns + sy]) {
#pragma unroll
                for (int l = 0; l < ND; ++l) w[(v * ND + l) * T + i] = TB(0);
                continue;
            }
            TB wv[ND];
#pragma unroll
            for (int l = 0; l < ND; ++l) wv[l] = w[(v * ND + l) * T + i];
            for (int k = 0; k <= j; ++k) {
                const TB hk = shc[v][k];
                const TB *vk = V + k * vs;
#pragma unroll
                for (int l = 0; l < ND; ++l) wv[l] = fma(-hk, vk[(v * ND + l) * T + i], wv[l]);
            }
#pragma unroll
            for (int l = 0; l < ND; ++l) {
                w[(v * ND + l) * T + i] = wv[l];
                nrm[v] = fma(wv[l], wv[l], nrm[v]);
            }
        }
    }
    if (want_norm) {
        double nd[NV];
        if (std::is_same<TB, float>::value) {
            // warp sums in FP32, widened once per warp
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                for (int o = 16; o > 0; o >>= 1) nrm[v] += __shfl_down_sync(0xffffffffu, nrm[v], o);
                if (lane == 0) sh[warp * NV + v] = double(nrm[v]);
            }
            __syncthreads();
            if (threadIdx.x == 0)
                for (int v = 0; v < NV; ++v) {
                    double t = 0.0;
                    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w * NV + v];
                    nd[v] = t;
                }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) nd[v] = double(nrm[v]);
            block_sum4(nd, sh);
        }
        if (threadIdx.x == 0)
            for (int v = 0; v < NV; ++v) part[(blockIdx.x * NV + v) * pstride + 0] = nd[v];
    }
}

// Segmented sums over the partial-sum rows of each case (cell blocks,
// seg[c]..seg[c+1]), fixed order:
// out[s][q] (op) sum_{b in case(s)} part[b][v(s)][q], q < nq; op 0 store, 1 add,
// 2 store sqrt.  With vn given, also co[s][q] = sum / vn[s][q]^2 (the
// Gram-Schmidt coefficient of the unnormalised basis vector q).  One block of
// kReduceThreads per (q, s): grid (nq, ns).
constexpr int kReduceThreads = 256;

// sum of at(b) over b = b0 + t, b0 + t + kReduceThreads, ... < b1 (t the
// thread), added in that order as the plain loop does, so the sum is the same
// bit for bit; the loads are issued eight at a time, so a thread waits for a
// few L2 round trips instead of one per term (a case's 4,000 cell blocks at 1M
// are 16 terms per thread)
template <typename F>
__device__ __forceinline__ double strided_sum(int b0, int b1, F &&at)
{
    constexpr int U = 8;
    double acc = 0.0;
    for (int b = b0 + (int)threadIdx.x; b < b1; b += U * kReduceThreads) {
        double t[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int bb = b + u * kReduceThreads;
            t[u] = bb < b1 ? at(bb) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (b + u * kReduceThreads < b1) acc += t[u];
    }
    return acc;
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce(const double *__restrict__ part,
                                                           const int32_t *__restrict__ seg, int pstride, double *out,
                                                           int ostride, int op, const double *__restrict__ vn = nullptr,
                                                           int vstride = 0, double *co = nullptr, int cstride = 0)
{
    __shared__ double sh[kReduceThreads / 32];
    const int q = blockIdx.x, sy = blockIdx.y, c = sy >> 2, v = sy & 3;
    const int b0 = seg[c], b1 = seg[c + 1];
    double acc = strided_sum(b0, b1, [&](int b) { return part[((int64_t)b * NV + v) * pstride + q]; });
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        acc = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) acc += sh[w];
        if (op == 0) out[sy * ostride + q] = acc;
        else if (op == 1) out[sy * ostride + q] += acc;
        else out[sy * ostride + q] = sqrt(acc);
        if (co) {
            const double n = vn[sy * vstride + q];
            co[sy * cstride + q] = n > 0.0 ? acc / (n * n) : 0.0;
        }
    }
}

// h[s][q] += h2[s][q], q <= j (second Gram-Schmidt pass)
__global__ void k_hadd(double *hc, int hstride, const double *__restrict__ h2, int h2stride, int j, int ns)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ns * (j + 1); t += gridDim.x * blockDim.x) {
        const int sy = t / (j + 1), q = t % (j + 1);
        hc[sy * hstride + q] += h2[sy * h2stride + q];
    }
}

// Arnoldi index j of system sy (running systems only): the new Hessenberg
// column from the raw sums hc, the earlier rotations applied, a new rotation,
// the rotated residual g and the stopping test.
__device__ __forceinline__ void givens_step(int sy, int j, int m, const double *__restrict__ hc, int hstride,
                                            double *vn, double *H, double *cs, double *sn, double *g, int32_t *ctl,
                                            int ns, const double *__restrict__ bnorm,
                                            const double *__restrict__ beta, double rtol, double eta, int maxit)
{
    if (!ctl[kCtlRunning * ns + sy]) return;
    // Hessenberg column of the normalised basis: h_kj = <V_k, u_j> / (vn_k vn_j),
    // h_{j+1,j} = |V_{j+1}| / vn_j; the new vector's norm becomes vn_{j+1}
    double h[kMaxRestart + 1];
    const double nj = vn[sy * (m + 1) + j];
    for (int k = 0; k <= j; ++k) h[k] = hc[sy * hstride + k] / (vn[sy * (m + 1) + k] * nj);
    const double hnext = hc[sy * hstride + j + 1];
    h[j + 1] = hnext / nj;
    vn[sy * (m + 1) + j + 1] = hnext;
    for (int k = 0; k < j; ++k) {
        const double c = cs[sy * m + k], s = sn[sy * m + k];
        const double t0 = h[k], t1 = h[k + 1];
        h[k] = c * t0 + s * t1;
        h[k + 1] = -s * t0 + c * t1;
    }
    const double dd = hypot(h[j], h[j + 1]);
    const double c = dd > 0.0 ? h[j] / dd : 1.0, s = dd > 0.0 ? h[j + 1] / dd : 0.0;
    cs[sy * m + j] = c;
    sn[sy * m + j] = s;
    h[j] = dd;
    for (int k = 0; k <= j; ++k) H[((int64_t)sy * (m + 1) + k) * m + j] = h[k];
    const double gj = g[sy * (m + 1) + j];
    g[sy * (m + 1) + j + 1] = -s * gj;
    g[sy * (m + 1) + j] = c * gj;
    ctl[kCtlJv * ns + sy] = j + 1;
    ctl[kCtlIters * ns + sy] += 1;
    // stop the cycle at the target, or (mixed precision, eta > 0) once the inner
    // residual has dropped by eta: the FP64 refinement residual then restarts it
    const double gn = fabs(g[sy * (m + 1) + j + 1]);
    if (gn <= rtol * bnorm[sy] || gn <= eta * beta[sy] || !(hnext > 0.0) || ctl[kCtlIters * ns + sy] >= maxit ||
        j + 1 == m)
        ctl[kCtlRunning * ns + sy] = 0;
}

// The last reduction of an Arnoldi index (|V_{j+1}| of system blockIdx.y into
// hc[.][j + 1], as k_reduce with op 2) followed by that system's Givens step
// in thread 0, which saves a launch per index.
__global__ void __launch_bounds__(kReduceThreads) k_norm_givens(const double *__restrict__ part,
                                                                const int32_t *__restrict__ seg, int pstride, int j,
                                                                int m, double *hc, int hstride, double *vn, double *H,
                                                                double *cs, double *sn, double *g, int32_t *ctl,
                                                                int ns, const double *__restrict__ bnorm,
                                                                const double *__restrict__ beta, double rtol,
                                                                double eta, int maxit)
{
    __shared__ double sh[kReduceThreads / 32];
    const int sy = blockIdx.y, c = sy >> 2, v = sy & 3;
    const int b0 = seg[c], b1 = seg[c + 1];
    double acc = strided_sum(b0, b1, [&](int b) { return part[((int64_t)b * NV + v) * pstride]; });
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        acc = 0.0;
        for (int w = 0; w < kReduceThreads / 32; ++w) acc += sh[w];
        hc[sy * hstride + j + 1] = sqrt(acc);
        givens_step(sy, j, m, hc, hstride, vn, H, cs, sn, g, ctl, ns, bnorm, beta, rtol, eta, maxit);
    }
}

// y = H^{-1} g on the first jv columns (upper triangular after the rotations).
__global__ void k_backsolve(int m, const double *__restrict__ H, const double *__restrict__ g, double *y,
                            const int32_t *__restrict__ ctl, int ns)
{
    const int sy = blockIdx.x * blockDim.x + threadIdx.x;
    if (sy >= ns) return;
    const int jv = ctl[kCtlJv * ns + sy];
    for (int k = jv - 1; k >= 0; --k) {
        double s = g[sy * (m + 1) + k];
        for (int q = k + 1; q < jv; ++q) s -= H[((int64_t)sy * (m + 1) + k) * m + q] * y[sy * m + q];
        y[sy * m + k] = s / H[((int64_t)sy * (m + 1) + k) * m + k];
    }
}

// y_k /= vn_k: coefficients of the unnormalised preconditioned vectors
// With sexp given (FP32 basis, rows [current][next] exponents e of the scale
// 2^-e of the first basis vector): y is also scaled by 2^-e of the current
// cycle (the combination adds 2^e sum y_k Z_k, so its FP32 sums stay near unit
// size), and the next residual's exponent comes from the cycle's estimate
// |g_jv| of its norm (at least 1e-3 rtol |b|).
// y32 (optional): an FP32 copy of the result for the FP32 combination.
__global__ void k_scale_y(int m, double *y, const double *__restrict__ vn, const int32_t *__restrict__ ctl, int ns,
                          const double *__restrict__ g = nullptr, const double *__restrict__ bnorm = nullptr,
                          double rtol = 0.0, int32_t *sexp = nullptr, float *y32 = nullptr)
{
    const int sy = blockIdx.x * blockDim.x + threadIdx.x;
    if (sy >= ns) return;
    const int jv = ctl[kCtlJv * ns + sy];
    const double f = sexp ? pow2(-sexp[sy]) : 1.0;
    for (int k = 0; k < jv; ++k) {
        y[sy * m + k] = sexp ? y[sy * m + k] / vn[sy * (m + 1) + k] * f : y[sy * m + k] / vn[sy * (m + 1) + k];
        if (y32) y32[sy * m + k] = float(y[sy * m + k]);
    }
    if (sexp && jv > 0) {
        const double est = fmax(fabs(g[sy * (m + 1) + jv]), 1e-3 * rtol * bnorm[sy]);
        if (est > 0.0 && est < 1e300) sexp[ns + sy] = max(-1000, ilogb(est));
    }
}

// x += sum_{k<jv} y_k Z_k with Z_k = M^{-1} V_k kept from the iterations
// x += sum_k y[s][k] Z_k.  FP64 path: FP64 sums.  Mixed path (FP32 Z): the
// correction of one inner cycle is formed in FP32 (it only has to be accurate to
// the inner tolerance; the next FP64 residual measures what is left) and added
// to x in FP64, so the FP64 pipe sees one add per value instead of one
// conversion and one FMA per value and Krylov vector.  With sexp given (FP32
// basis): y carries 2^-e of the cycle (see k_scale_y) and the sum is scaled
// back by 2^e in FP64 (exact).
// y32 (FP32 Z only, optional): the FP32 copy of y, read instead of converting
// y per thread; the scaled value 2^e acc is formed exactly on the integer pipe
// (f2d_pow2), so the FP64 pipe sees one add per value.
template <typename TZ>
__global__ void k_combine_z(DeviceMesh d, const TZ *__restrict__ Z, const double *__restrict__ y, int m,
                            const int32_t *__restrict__ ctl, int ns, double *__restrict__ x,
                            const int32_t *__restrict__ sexp = nullptr, const float *__restrict__ y32 = nullptr)
{
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    const int v = blockIdx.y;                          // one variable per grid row
    const int sy = 4 * d.blk_case[blockIdx.x] + v;
    const int jv = ctl[kCtlJv * ns + sy];
    if (jv <= 0) return;
    const int64_t vs = (int64_t)NX * T;
    TZ acc[ND] = {0, 0, 0, 0, 0};
    for (int k = 0; k < jv; ++k) {
        const TZ yk = y32 ? TZ(y32[sy * m + k]) : TZ(y[sy * m + k]);
#pragma unroll
        for (int l = 0; l < ND; ++l) acc[l] += yk * Z[k * vs + (v * ND + l) * T + i];
    }
    if (sexp) {
        const int e = sexp[sy];
        if (std::is_same<TZ, float>::value) {
            // 2^e acc as an FP64 value formed on the integer pipe (exact; no
            // conversion instruction on the FP64 pipe), one FP64 add per value
#pragma unroll
            for (int l = 0; l < ND; ++l) x[(v * ND + l) * T + i] += f2d_pow2(float(acc[l]), e);
        } else {
            const double f = pow2(e);
#pragma unroll
            for (int l = 0; l < ND; ++l) x[(v * ND + l) * T + i] += double(acc[l]) * f;
        }
    } else {
#pragma unroll
        for (int l = 0; l < ND; ++l) x[(v * ND + l) * T + i] += double(acc[l]);
    }
}

// Warm start of solve n (cases not done) from the last solutions
// x = s_{n-1}, xp = s_{n-2}, xpp = s_{n-3}: order 0 keeps x, order 1 takes
// 2 x - xp, order 2 takes 3 x - 3 xp + xpp (polynomial extrapolation in the
// step index).  The history shifts by an exchange of the two buffers' roles,
// which follow the parity of the device's solve count n (k_mark_noconv raises
// it after the solve): the old x goes into xpp's buffer (the next xp), and
// xp's buffer (the next xpp) already holds s_{n-2}, so one vector is written
// instead of two.  Cells of finished cases keep their history: their two
// buffers exchange contents, which the exchange of roles undoes.
__global__ void k_warm(DeviceMesh d, double *__restrict__ x, double *__restrict__ h0, double *__restrict__ h1,
                       const int32_t *__restrict__ done, const int64_t *__restrict__ nsolve, int max_order)
{
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    // n solves so far: the two history buffers swap roles after every solve, and
    // the extrapolation uses as many past solutions as exist
    const int64_t n = *nsolve;
    double *__restrict__ xp = (n & 1) ? h1 : h0;
    double *__restrict__ xpp = (n & 1) ? h0 : h1;
    const int order = (max_order >= 2 && n >= 3) ? 2 : (n >= 2 ? 1 : 0);
    if (done[d.blk_case[blockIdx.x]]) {
#pragma unroll 4
        for (int q = 0; q < NX; ++q) {
            const double b = xp[q * T + i], c = xpp[q * T + i];
            xp[q * T + i] = c;
            xpp[q * T + i] = b;
        }
        return;
    }
#pragma unroll 4
    for (int q = 0; q < NX; ++q) {
        const double a = x[q * T + i];
        if (order == 2) x[q * T + i] = 3.0 * (a - xp[q * T + i]) + xpp[q * T + i];
        else if (order == 1) x[q * T + i] = 2.0 * a - xp[q * T + i];
        xpp[q * T + i] = a;
    }
}

// Start (first = 1) or restart of every system: sums[s][0] = |r|^2,
// sums[s][1] = |b|^2.  Systems of finished cases stay inactive.
// Scale of the first residual of a solve: next exponent sexp[ns + s] = e with 2^-e B in [1, 2),
// B = max(|b|, |b_prev|) (sums[s][1] = |b|^2, bnorm = |b| of the previous
// solve, 0 at first): the warm start solved the previous system, so its
// residual is of the order of B at most; e = 0 when B = 0.
__global__ void k_sigma(const double *__restrict__ sums, int sstride, const double *__restrict__ bnorm,
                        int32_t *sexp, int ns)
{
    const int sy = blockIdx.x * blockDim.x + threadIdx.x;
    if (sy >= ns) return;
    const double bn = fmax(sqrt(sums[sy * sstride + 1]), bnorm[sy]);
    sexp[ns + sy] = bn > 0.0 && bn < 1e300 ? max(-1000, ilogb(bn)) : 0;
}

// sums[s][0] = |V_0|^2 of the stored first basis vector V_0 = 2^-e r (e: the
// next exponent sexp[ns + s], which becomes the current one sexp[s]; e = 0
// when sexp is NULL), sums[s][1] = |b|^2 (first solve of a step).
__global__ void k_start(const double *__restrict__ sums, int sstride, double *bnorm, double *beta, double *vn, int m,
                        int32_t *ctl, int ns, const int32_t *__restrict__ done, double rtol, int maxit, int first,
                        int32_t *sexp = nullptr)
{
    const int sy = blockIdx.x * blockDim.x + threadIdx.x;
    if (sy >= ns) return;
    // |b| comes with the first residual; restarts reuse it
    const double vn0 = sqrt(sums[sy * sstride + 0]);
    double be = vn0;
    if (sexp) {
        be = vn0 * pow2(sexp[ns + sy]);
        sexp[sy] = sexp[ns + sy];
    }
    const double bn = first ? sqrt(sums[sy * sstride + 1]) : bnorm[sy];
    if (first) {
        bnorm[sy] = bn;
        ctl[kCtlIters * ns + sy] = 0;
        ctl[kCtlActive * ns + sy] = !done[sy >> 2];
    }
    beta[sy] = be;
    vn[sy * (m + 1)] = vn0;                            // V_0 = 2^-e r, v_0 = r / beta
    const int act = ctl[kCtlActive * ns + sy] && bn > 0.0 && be > rtol * bn && ctl[kCtlIters * ns + sy] < maxit;
    ctl[kCtlActive * ns + sy] = act;
    ctl[kCtlRunning * ns + sy] = act;
    ctl[kCtlJv * ns + sy] = 0;
}

// flags[0] = any active system, flags[1] = any running system (one block).
__global__ void k_any(const int32_t *__restrict__ ctl, int ns, int32_t *flags)
{
    __shared__ int sh[2];
    if (threadIdx.x < 2) sh[threadIdx.x] = 0;
    __syncthreads();
    int a = 0, r = 0;
    for (int sy = threadIdx.x; sy < ns; sy += blockDim.x) {
        a |= ctl[kCtlActive * ns + sy];
        r |= ctl[kCtlRunning * ns + sy];
    }
    if (a) atomicOr(&sh[0], 1);
    if (r) atomicOr(&sh[1], 1);
    __syncthreads();
    if (threadIdx.x < 2) flags[threadIdx.x] = sh[threadIdx.x];
}

// Condition of the device-controlled solve (one block): any system active
// (which = 0, the cycle loop) or running (which = 1, the next Arnoldi index).
// Thread 0 counts the run in ctr[slot] (slot >= 0) and sets the handle (set).
// guard 1 starts the solve's cycle count; guard 2 counts a cycle and ends the
// loop once more than limit cycles ran (each cycle takes at least one
// iteration of every active system, which stops at maxit, so the limit
// maxit + 1 is a backstop that a correct solve never reaches).
__global__ void k_cond(const int32_t *__restrict__ ctl, int ns, int which, cudaGraphConditionalHandle h, int set,
                       int64_t *ctr, int slot, int guard, int64_t limit)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int a = 0;
    for (int sy = threadIdx.x; sy < ns; sy += blockDim.x) a |= ctl[(which ? kCtlRunning : kCtlActive) * ns + sy];
    if (a) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x != 0) return;
    unsigned v = any ? 1u : 0u;
    if (slot >= 0) ctr[slot] += 1;
    if (guard == 1) ctr[kCtrGuard] = 0;
    if (guard == 2 && ++ctr[kCtrGuard] > limit) v = 0u;
    if (set) cudaGraphSetConditional(h, v);
}

// Condition of the device-controlled step loop (one block): any case not done,
// and the loops of this launch (run_ctl[0]) below its limit (run_ctl[1]).
// entry = 1 before the loop (no loops yet); otherwise at the end of a loop,
// which it counts in run_ctl[0] and in ctr[kCtrRun].
__global__ void k_run_cond(const int32_t *__restrict__ done, int n, int64_t *run_ctl, int64_t *ctr,
                           cudaGraphConditionalHandle h, int entry)
{
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    int a = 0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) a |= done[c] == 0;
    if (a) atomicOr(&any, 1);
    __syncthreads();
    if (threadIdx.x != 0) return;
    int64_t loops = 0;
    if (!entry) {
        loops = run_ctl[0] + 1;
        ctr[kCtrRun] += 1;
    }
    run_ctl[0] = loops;
    cudaGraphSetConditional(h, (any && loops < run_ctl[1]) ? 1u : 0u);
}

// g = beta e_1 for active systems.
__global__ void k_init_g(double *g, int m, const double *__restrict__ beta, const int32_t *__restrict__ ctl, int ns)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ns * (m + 1); t += gridDim.x * blockDim.x) {
        const int sy = t / (m + 1);
        g[t] = (t % (m + 1) == 0 && ctl[kCtlActive * ns + sy]) ? beta[sy] : 0.0;
    }
}

__global__ void k_zero_trivial(DeviceMesh d, double *__restrict__ x, const double *__restrict__ bnorm)
{
    const int64_t T = d.T;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= T) return;
    const int c = d.blk_case[blockIdx.x];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        if (bnorm[4 * c + v] > 0.0) continue;
#pragma unroll
        for (int l = 0; l < ND; ++l) x[(v * ND + l) * T + i] = 0.0;
    }
}

// status[c] |= noconv for cases with a system that stopped above the tolerance,
// and |= timeout for every active case if a wait of the sync-free ILU solves
// gave up during the solve (sf_err, may be NULL); the solve count of the warm
// start (k_warm) goes up by one
__global__ void k_mark_noconv(const double *__restrict__ bnorm, const double *__restrict__ beta,
                              const int32_t *__restrict__ done, int ns, double rtol, int32_t *status,
                              int64_t *nsolve, const int32_t *sf_err)
{
    const int sy = blockIdx.x * blockDim.x + threadIdx.x;
    if (sy == 0) ++*nsolve;
    if (sy >= ns || done[sy >> 2]) return;
    if (bnorm[sy] > 0.0 && beta[sy] > rtol * bnorm[sy]) atomicOr(&status[sy >> 2], kStatusNoConv);
    if (sf_err && *sf_err) atomicOr(&status[sy >> 2], kStatusTimeout);
}

inline unsigned nblocks(int64_t n) { return (unsigned)((n + kBlock - 1) / kBlock); }

// k_orth_update with the Arnoldi index unrolled for the first four indices
// (the inner cycles of the mixed mode rarely go further)
template <typename TB>
void launch_orth_update(const DeviceMesh &d, unsigned nb, cudaStream_t q, const TB *V, TB *w, int j,
                        const double *hc, int hstride, const int32_t *ctl, int ns, double *part, int pstride,
                        int want_norm)
{
    switch (j) {
    case 0: k_orth_update<TB, 1><<<nb, kBlock, 0, q>>>(d, V, w, j, hc, hstride, ctl, ns, part, pstride, want_norm); break;
    case 1: k_orth_update<TB, 2><<<nb, kBlock, 0, q>>>(d, V, w, j, hc, hstride, ctl, ns, part, pstride, want_norm); break;
    case 2: k_orth_update<TB, 3><<<nb, kBlock, 0, q>>>(d, V, w, j, hc, hstride, ctl, ns, part, pstride, want_norm); break;
    case 3: k_orth_update<TB, 4><<<nb, kBlock, 0, q>>>(d, V, w, j, hc, hstride, ctl, ns, part, pstride, want_norm); break;
    default: k_orth_update<TB><<<nb, kBlock, 0, q>>>(d, V, w, j, hc, hstride, ctl, ns, part, pstride, want_norm);
    }
}

// The reverse-slot coefficients of the global normal equations for the ILU
// kernels (all NULL for the per-cell equations).
template <typename TP>
struct RevSlots {
    const TP *a = nullptr, *x = nullptr, *y = nullptr, *b = nullptr;
};

// dst = M^{-1} src (block ILU(0) on the RCM order).  TZ, TM: storage and
// arithmetic precision of the application; TP: storage of the factors; tA, tB:
// work buffers of type TZ; rev: reverse slots of the global normal equations.
template <typename TR, typename TZ, typename TM, typename TP = TM>
gks_status precond_t(gks_mesh *m, const TP *Pg, const TP *alg, const TP *exg, const TP *eyg, const TR *src,
                     TZ *dst, TZ *tA, TZ *tB, TZ *rz, cudaStream_t s, RevSlots<TP> rev = {})
{
    DeviceMesh &d = m->d;
    const int64_t T = d.T;
    // forward / backward relation, the global variant when reverse slots are given
    auto fwd = [&](int64_t n, const int32_t *rows, auto r, const TZ *zin, TZ *zout, int use_nb, TZ *rc) {
        using TRx = std::remove_cv_t<std::remove_pointer_t<decltype(r)>>;
        if (rev.a)
            k_ilu_fwd<TRx, TZ, TM, TP, true><<<nblocks(n), kBlock, 0, s>>>(d, Pg, alg, exg, eyg, rows, n, r, zin, zout,
                                                                          use_nb, rc, rev.a, rev.x, rev.y, rev.b);
        else
            k_ilu_fwd<TRx, TZ, TM, TP, false><<<nblocks(n), kBlock, 0, s>>>(d, Pg, alg, exg, eyg, rows, n, r, zin,
                                                                           zout, use_nb, rc);
        note_launch();
    };
    auto bwd = [&](int64_t n, const int32_t *rows, const TZ *z, const TZ *xin, TZ *xout) {
        if (rev.a)
            k_ilu_bwd<TZ, TM, TP, true><<<nblocks(n), kBlock, 0, s>>>(d, Pg, alg, exg, eyg, rows, n, z, xin, xout,
                                                                     rev.a, rev.x, rev.y, rev.b);
        else
            k_ilu_bwd<TZ, TM, TP, false><<<nblocks(n), kBlock, 0, s>>>(d, Pg, alg, exg, eyg, rows, n, z, xin, xout);
        note_launch();
    };
    if (m->cfg.precond == GKS_PC_ILU_EXACT) {
        // sync-free: a new epoch, then one launch per relation
        Work &k = m->wk;
        k_sf_begin<<<1, 32, 0, s>>>(k.sf_ctl, 0);
        note_launch();
        const unsigned g = (unsigned)std::min<int64_t>(nblocks(T), (int64_t)k.sm_count * kSfBlocksPerSm);
        if (rev.a)
            k_ilu_fwd_sf<TR, TZ, TM, TP, true><<<g, kBlock, 0, s>>>(d, Pg, alg, exg, eyg, src, dst, k.sf_flag,
                                                                    k.sf_ctl, rev.a, rev.x, rev.y, rev.b);
        else
            k_ilu_fwd_sf<TR, TZ, TM, TP, false><<<g, kBlock, 0, s>>>(d, Pg, alg, exg, eyg, src, dst, k.sf_flag,
                                                                     k.sf_ctl);
        note_launch();
        if (rev.a)
            k_ilu_bwd_sf<TZ, TM, TP, true><<<g, kBlock, 0, s>>>(d, Pg, alg, exg, eyg, dst, k.sf_flag, k.sf_ctl,
                                                                rev.a, rev.x, rev.y, rev.b);
        else
            k_ilu_bwd_sf<TZ, TM, TP, false><<<g, kBlock, 0, s>>>(d, Pg, alg, exg, eyg, dst, k.sf_flag, k.sf_ctl);
        note_launch();
    } else if (m->cfg.precond == GKS_PC_ILU_LEVELS) {
        const auto &lp = m->lvl_lo_ptr;
        for (size_t l = 0; l + 1 < lp.size(); ++l)
            fwd(lp[l + 1] - lp[l], d.lvl_lo + lp[l], src, dst, dst, 1, (TZ *)nullptr);
        const auto &up = m->lvl_up_ptr;
        for (size_t l = 0; l + 1 < up.size(); ++l) bwd(up[l + 1] - up[l], d.lvl_up + up[l], dst, dst, dst);
    } else if (m->cfg.precond == GKS_PC_BJACOBI) {
        fwd(T, nullptr, src, nullptr, dst, 0, (TZ *)nullptr);     // z = P r, the block-diagonal inverse
    } else {
        // sweeps: forward z^0 = P r, z^{q+1} = F(z^q); backward x^0 = z, x^{q+1} = B(x^q)
        const int ns = m->cfg.ilu_sweeps;
        const int nsb = m->cfg.ilu_sweeps_bwd < 0 ? ns : m->cfg.ilu_sweeps_bwd;
        // z^0 folded into the first sweep (ilu_fuse_first) or a pass of its own
        const bool fuse = ns > 0 && m->cfg.ilu_fuse_first;
        // two backward sweeps per launch where a pair follows (the per-cell
        // equations; same results as one sweep per launch)
        const bool pairs = !rev.a && m->cfg.ilu_sweep_pairs;   // backward relation only
        const int nf = fuse ? ns : ns + 1;   // forward launches
        TZ *za = (nf % 2 == 1) ? tA : dst;   // buffers chosen so that z ends in tA
        TZ *zb = (nf % 2 == 1) ? dst : tA;
        // a wider source is rounded to TZ once, in the first pass, for the sweeps
        TZ *rc = (sizeof(TR) > sizeof(TZ) && ns > 0) ? rz : nullptr;
        fwd(T, nullptr, src, nullptr, za, fuse ? 2 : 0, rc);
        for (int q = fuse ? 1 : 0; q < ns; ++q) {
            if (rc)
                fwd(T, nullptr, (const TZ *)rc, za, zb, 1, (TZ *)nullptr);
            else
                fwd(T, nullptr, src, za, zb, 1, (TZ *)nullptr);
            std::swap(za, zb);
        }
        if (nsb == 0) {
            GKS_CUDA(cudaMemcpyAsync(dst, za, sizeof(TZ) * NX * T, cudaMemcpyDeviceToDevice, s));
        } else {
            // launches: pairs of sweeps, then a single one if nsb is odd
            const int npair = pairs ? nsb / 2 : 0, nb = npair + (nsb - 2 * npair);
            TZ *xa = za;                                    // x^0 = z (in za)
            TZ *xb = (nb % 2 == 1) ? dst : (za == tB ? tA : tB);
            for (int q = 0; q < nb; ++q) {
                if (q < npair) {
                    k_ilu_bwd2<TZ, TM, TP><<<nblocks(T), kBlock, 0, s>>>(d, Pg, alg, exg, eyg, za, xa, xb);
                    note_launch();
                } else {
                    bwd(T, nullptr, za, xa, xb);
                }
                xa = xb;
                xb = (xb == dst) ? tB : dst;
            }
        }
    }
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

template <typename TR>
gks_status precond(gks_mesh *m, const TR *src, double *dst, cudaStream_t s)
{
    DeviceMesh &d = m->d;
    return precond_t<TR, double, double>(m, d.P, d.alpha, d.ex, d.ey, src, dst, m->wk.t2, m->wk.t3, nullptr, s,
                                         {d.alr, d.exr, d.eyr, d.bdg});
}

template <typename TR>
gks_status precond32(gks_mesh *m, const TR *src, float *dst, cudaStream_t s)
{
    DeviceMesh &d = m->d;
    if (d.P16)   // FP16 factors (ilu_fp16), FP32 arithmetic
        return precond_t<TR, float, float, __half>(m, d.P16, d.alpha16, d.ex16, d.ey16, src, dst, m->wk.t2_32,
                                                   m->wk.t3_32, m->wk.r32, s, {d.alr16, d.exr16, d.eyr16, d.bdg16});
    return precond_t<TR, float, float>(m, d.P32, d.alpha32, d.ex32, d.ey32, src, dst, m->wk.t2_32, m->wk.t3_32,
                                       m->wk.r32, s, {d.alr32, d.exr32, d.eyr32, d.bdg32});
}

// Any active / any running system into the pinned host flags (no synchronisation).
gks_status enqueue_flags(gks_mesh *m, cudaStream_t s)
{
    const int slot = prof_start(m, kProfCtl, s);
    k_any<<<1, kBlock, 0, s>>>(m->wk.ctl, m->wk.ns, m->wk.flags);
    note_launch();
    GKS_CUDA(cudaMemcpyAsync(m->wk.h_flags, m->wk.flags, sizeof(int32_t) * 2, cudaMemcpyDeviceToHost, s));
    prof_stop(m, slot, s);
    return GKS_OK;
}

// Add what the device-controlled solves ran since the last call (counters
// already copied to h_ctr, stream synchronised) to the launch and work totals.
void take_counters(gks_mesh *m)
{
    SolveGraphs &g = *m->graphs;
    for (int q = 0; q < kCtrLen; ++q) {
        const int64_t d = g.h_ctr[q] - g.ctr_seen[q];
        g.ctr_seen[q] = g.h_ctr[q];
        if (q < kCtrCycles && d > 0) {
            if (q < (int)g.whole_iter_launches.size()) g_launches.fetch_add(d * g.whole_iter_launches[q]);
            m->prof.arnoldi += d;
            m->prof.precond += d;
            m->prof.arnoldi_jsum += d * (q + 1);
        } else if (q == kCtrCycles && d > 0) {
            g_launches.fetch_add(d * g.whole_cycle_launches);
            m->prof.residuals += d;
        } else if (q == kCtrRun && d > 0) {
            // loops of the step-loop graph: their kernels outside the solve's
            // cycles, and the first residual of each loop's solve
            g_launches.fetch_add(d * g.run_loop_launches);
            m->prof.residuals += d;
        }
    }
}

// Graphs are used unless disabled or the profiler (events between kernels) is on;
// a change of a knob baked into the captured kernel arguments drops them.
bool prepare_graphs(gks_mesh *m)
{
    if (m->cfg.no_graphs == 1 || m->prof.mask) return false;
    if (!m->graphs) m->graphs = new SolveGraphs;
    SolveGraphs &g = *m->graphs;
    if (g.disabled) return false;
    const gks_config &c = m->cfg;
    if (g.sweeps != c.ilu_sweeps || g.sweeps_bwd != c.ilu_sweeps_bwd || g.fuse != c.ilu_fuse_first ||
        g.pairs != c.ilu_sweep_pairs || g.spmv_dots != c.spmv_dots ||
        g.precond != c.precond ||
        g.maxit != c.gmres_maxit || g.eta != c.inner_rtol ||
        g.rtol != c.gmres_rtol || (int)g.iter.size() != m->wk.m) {
        if (g.whole || g.run) flush_solve_counters(m);
        destroy_graph_execs(&g);
        g.sweeps = c.ilu_sweeps;
        g.sweeps_bwd = c.ilu_sweeps_bwd;
        g.fuse = c.ilu_fuse_first;
        g.pairs = c.ilu_sweep_pairs;
        g.spmv_dots = c.spmv_dots;
        g.precond = c.precond;
        g.maxit = c.gmres_maxit;
        g.eta = c.inner_rtol;
        g.rtol = c.gmres_rtol;
        g.iter.assign(m->wk.m, nullptr);
        g.iter_launches.assign(m->wk.m, 0);
    }
    return true;
}

// Capture enq(stream) into *exec on the private stream; *nl = kernels captured.
template <typename F>
gks_status capture_part(gks_mesh *m, cudaGraphExec_t *exec, int64_t *nl, F &&enq)
{
    SolveGraphs &g = *m->graphs;
    if (!g.cap) GKS_CUDA(cudaStreamCreateWithFlags(&g.cap, cudaStreamNonBlocking));
    const int64_t l0 = g_launches.load();
    GKS_CUDA(cudaStreamBeginCapture(g.cap, cudaStreamCaptureModeThreadLocal));
    const gks_status st = enq(g.cap);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g.cap, &graph);
    const int64_t n = g_launches.load() - l0;
    g_launches.fetch_sub(n, std::memory_order_relaxed);   // captured, not run
    if (st != GKS_OK || e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st != GKS_OK ? st : GKS_ECUDA;
    }
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        cudaGetLastError();
        return GKS_ECUDA;
    }
    *nl = n;
    return GKS_OK;
}

// Run one part of the solve on s and wait for its host flags: a replay of its
// graph (captured on first use), or the launches themselves.
template <typename F>
gks_status run_part(gks_mesh *m, bool use_graph, cudaGraphExec_t *exec, int64_t *nl, cudaStream_t s, F &&enq)
{
    use_graph = use_graph && !m->graphs->disabled;
    if (use_graph && !*exec && capture_part(m, exec, nl, enq) != GKS_OK) {
        m->graphs->disabled = true;                   // fall back to direct launches for good
        use_graph = false;
    }
    if (use_graph) {
        GKS_CUDA(cudaGraphLaunch(*exec, s));
        g_launches.fetch_add(*nl, std::memory_order_relaxed);
    } else {
        const gks_status st = enq(s);
        if (st != GKS_OK) return st;
    }
    GKS_CUDA(cudaStreamSynchronize(s));
    return GKS_OK;
}

// Append enq(stream) to graph g after the nodes deps[0..nd) by capture on the
// private stream; *sink = the last captured node, *nl = kernels captured.
template <typename F>
gks_status capture_into(gks_mesh *m, cudaGraph_t g, const cudaGraphNode_t *deps, size_t nd, cudaGraphNode_t *sink,
                        int64_t *nl, F &&enq)
{
    SolveGraphs &G = *m->graphs;
    if (!G.cap) GKS_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking));
    const int64_t l0 = g_launches.load();
    GKS_CUDA(cudaStreamBeginCaptureToGraph(G.cap, g, deps, nullptr, nd, cudaStreamCaptureModeThreadLocal));
    const gks_status st = enq(G.cap);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t *tail = nullptr;
    size_t nt = 0;
    const cudaError_t e = cudaStreamGetCaptureInfo(G.cap, &cs, nullptr, nullptr, &tail, nullptr, &nt);
    const cudaGraphNode_t last = (e == cudaSuccess && nt == 1) ? tail[0] : nullptr;
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(G.cap, &out);
    const int64_t n = g_launches.load() - l0;
    g_launches.fetch_sub(n, std::memory_order_relaxed);   // captured, not run
    if (st != GKS_OK || e != cudaSuccess || e2 != cudaSuccess || !last) {
        cudaGetLastError();
        return st != GKS_OK ? st : GKS_ECUDA;
    }
    *sink = last;
    *nl = n;
    return GKS_OK;
}

// Add a conditional node (if / while, one body) on handle h after dep.
gks_status add_cond(cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                    cudaGraphConditionalNodeType type, cudaGraphNode_t *node, cudaGraph_t *body)
{
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    GKS_CUDA(cudaGraphAddNode(node, g, &dep, nullptr, 1, &p));
    *body = p.conditional.phGraph_out[0];
    return GKS_OK;
}

// The device counters of the device-controlled graphs (allocated once per handle).
gks_status ensure_counters(gks_mesh *m, cudaStream_t s)
{
    SolveGraphs &G = *m->graphs;
    if (G.ctr) return GKS_OK;
    GKS_CUDA(cudaMalloc(&G.ctr, sizeof(int64_t) * kCtrLen));
    GKS_CUDA(cudaMallocHost(&G.h_ctr, sizeof(int64_t) * kCtrLen));
    GKS_CUDA(cudaMemsetAsync(G.ctr, 0, sizeof(int64_t) * kCtrLen, s));
    G.ctr_seen.assign(kCtrLen, 0);
    return GKS_OK;
}

// A device-controlled solve built as part of a larger graph: into g after dep
// (NULL: with no dependency); sink receives its last node, launches the kernels
// that run once per solve (the start part and what follows the cycle loop).
struct SolveEmbed {
    cudaGraph_t g = nullptr;
    cudaGraphNode_t dep = nullptr;
    cudaGraphNode_t sink = nullptr;
    int64_t launches = 0;
};

// The device-controlled solve as one executable graph (or, with emb, as nodes
// of the caller's graph):
//   start; c = any active
//   while (c) { i_0 = any running
//               if (i_0) { Arnoldi 0; i_1 = any running
//                          if (i_1) { Arnoldi 1; ... if (i_{m-1}) { Arnoldi m-1 } } }
//               restart; c = any active (and within the cycle limit) }
// The condition kernels replace the host flags of the per-part graphs; the
// conditions of an index are only evaluated once the one before it has run.
template <typename SB, typename IB, typename RB>
gks_status build_whole(gks_mesh *m, cudaStream_t s, SB &&start_body, IB &&iter_body, RB &&restart_body,
                       SolveEmbed *emb = nullptr)
{
    SolveGraphs &G = *m->graphs;
    Work &k = m->wk;
    const int ns = k.ns, mm = k.m;
    const int64_t limit = (int64_t)m->cfg.gmres_maxit + 1;
    if (const gks_status r = ensure_counters(m, s); r != GKS_OK) return r;
    int64_t *ctr = G.ctr;
    const int32_t *ctl = k.ctl;
    cudaGraph_t top = emb ? emb->g : nullptr;
    if (!emb) GKS_CUDA(cudaGraphCreate(&top, 0));
    const size_t ndep = emb && emb->dep ? 1 : 0;
    gks_status st = GKS_OK;
    std::vector<int64_t> nl_iter(mm, 0);
    int64_t nl_start = 0, nl_c0 = 0, nl_restart = 0;
    do {
        cudaGraphConditionalHandle h_outer, h_next;
        if (cudaGraphConditionalHandleCreate(&h_outer, top, 0, 0) != cudaSuccess) { st = GKS_ECUDA; break; }
        cudaGraphNode_t sink, wnode, inode;
        cudaGraph_t wbody, ibody;
        st = capture_into(m, top, ndep ? &emb->dep : nullptr, ndep, &sink, &nl_start, [&](cudaStream_t q) -> gks_status {
            gks_status r = start_body(q);
            if (r != GKS_OK) return r;
            k_cond<<<1, kBlock, 0, q>>>(ctl, ns, 0, h_outer, 1, ctr, -1, 1, limit); note_launch();
            return GKS_OK;
        });
        if (st != GKS_OK || (st = add_cond(top, sink, h_outer, cudaGraphCondTypeWhile, &wnode, &wbody)) != GKS_OK)
            break;
        if (cudaGraphConditionalHandleCreate(&h_next, wbody, 0, 0) != cudaSuccess) { st = GKS_ECUDA; break; }
        st = capture_into(m, wbody, nullptr, 0, &sink, &nl_c0, [&](cudaStream_t q) -> gks_status {
            k_cond<<<1, kBlock, 0, q>>>(ctl, ns, 1, h_next, 1, ctr, -1, 0, limit); note_launch();
            return GKS_OK;
        });
        if (st != GKS_OK || (st = add_cond(wbody, sink, h_next, cudaGraphCondTypeIf, &inode, &ibody)) != GKS_OK)
            break;
        st = capture_into(m, wbody, &inode, 1, &sink, &nl_restart, [&](cudaStream_t q) -> gks_status {
            gks_status r = restart_body(q);
            if (r != GKS_OK) return r;
            k_cond<<<1, kBlock, 0, q>>>(ctl, ns, 0, h_outer, 1, ctr, kCtrCycles, 2, limit); note_launch();
            return GKS_OK;
        });
        if (st != GKS_OK) break;
        for (int j = 0; j < mm && st == GKS_OK; ++j) {
            const bool more = j + 1 < mm;
            if (more && cudaGraphConditionalHandleCreate(&h_next, ibody, 0, 0) != cudaSuccess) {
                st = GKS_ECUDA;
                break;
            }
            st = capture_into(m, ibody, nullptr, 0, &sink, &nl_iter[j], [&](cudaStream_t q) -> gks_status {
                gks_status r = iter_body(q, j);
                if (r != GKS_OK) return r;
                k_cond<<<1, kBlock, 0, q>>>(ctl, ns, 1, h_next, more ? 1 : 0, ctr, j, 0, limit); note_launch();
                return GKS_OK;
            });
            if (st == GKS_OK && more) st = add_cond(ibody, sink, h_next, cudaGraphCondTypeIf, &inode, &ibody);
        }
        if (st != GKS_OK) break;
        if (emb) {
            emb->sink = wnode;
        } else if (cudaGraphInstantiate(&G.whole, top, 0) != cudaSuccess) {
            G.whole = nullptr;
            st = GKS_ECUDA;
        }
    } while (false);
    if (!emb) cudaGraphDestroy(top);
    cudaGetLastError();
    if (st != GKS_OK) return st;
    G.whole_start_launches = nl_start;
    G.whole_cycle_launches = nl_c0 + nl_restart;
    G.whole_iter_launches = nl_iter;
    return GKS_OK;
}

// part[blk][v][k] = partial <V_k, w>, k <= j, per cell block
template <typename TB>
gks_status dots(gks_mesh *m, const TB *V, const TB *w, int j, double *part, int ps, cudaStream_t s)
{
    const int64_t nblk = m->wk.nblk;
    const dim3 g((unsigned)(j + 1), (unsigned)std::min<int64_t>(nblk, kDotMaxTiles));
    k_dots<TB><<<g, kDotThreads, 0, s>>>(m->d.T, nblk, V, w, part, ps);
    note_launch();
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

inline unsigned sblocks(int n) { return (unsigned)((n + 127) / 128); }

}  // namespace

// Solve the CLS systems of every case for the right-hand sides built from
// m->wk.w; the solutions (and warm starts) are m->wk.x.  GMRES cycles of all
// systems run in lockstep: every launch covers all cases, and per-system masks
// stop the systems that have converged.
// The whole solve with the Krylov basis stored as TB (double, or float in the
// mixed mode with basis_fp32).  With emb the device-controlled solve and its
// closing kernel are built into the caller's graph instead of run.
template <typename TB>
gks_status cls_solve_t(gks_mesh *m, TB *V, cudaStream_t s, int32_t *iters, double *relres, int32_t *converged,
                       SolveEmbed *emb = nullptr)
{
    DeviceMesh &d = m->d;
    Work &k = m->wk;
    const int64_t T = d.T;
    const int mm = k.m;
    const int ps = mm + 2;
    const int ns = k.ns;
    const unsigned nb = (unsigned)k.nblk;
    const double rtol = m->cfg.gmres_rtol;
    const int maxit = m->cfg.gmres_maxit;
    const int64_t vs = (int64_t)NX * T;
    const bool mixed = m->cfg.precision == GKS_MIXED;
    // mixed precision: an inner GMRES cycle (FP32 operator and ILU) stops once its
    // residual estimate has dropped by inner_rtol; the FP64 residual of the next
    // refinement sweep then measures the true error
    const double eta = mixed ? m->cfg.inner_rtol : 0.0;
    gks_status st;

    // FP32 basis: first basis vector scaled by a power of two; exponents per
    // system, [current cycle][next residual]
    int32_t *sx = std::is_same<TB, float>::value ? k.sexp : nullptr;
    const int32_t *sxn = sx ? sx + ns : nullptr;
    // V_0 = 2^-e (b - K x) and partial |V_0|^2: double-FP32 arithmetic into the
    // FP32 basis when the operator has FP32 pairs, FP64 arithmetic otherwise
    // operator applications y = K x (mode 0) or the FP64 residual (mode 1); the
    // global normal equations' variant when the mesh has reverse slots
    auto spmv64 = [&](cudaStream_t q, const double *xs, TB *y, int mode, const double *bb, const int32_t *se) {
        if (d.alr)
            k_spmv<double, double, TB, true><<<nb, kBlock, 0, q>>>(d, d.D, d.alpha, d.ex, d.ey, xs, y, mode, bb,
                                                                   k.part, ps, se, d.alr, d.exr, d.eyr, d.bdg);
        else
            k_spmv<double, double, TB, false><<<nb, kBlock, 0, q>>>(d, d.D, d.alpha, d.ex, d.ey, xs, y, mode, bb,
                                                                    k.part, ps, se);
    };
    auto spmv32 = [&](cudaStream_t q, const float *xs, TB *y) {
        if (d.alr32)
            k_spmv<float, float, TB, true><<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, xs, y, 0,
                                                                 nullptr, nullptr, 0, nullptr, d.alr32, d.exr32,
                                                                 d.eyr32, d.bdg32);
        else
            k_spmv<float, float, TB, false><<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, xs, y, 0,
                                                                  nullptr, nullptr, 0);
    };
    // the FP32-basis solve forms b in double-FP32 arithmetic when the weights fit
    const bool rhs_df = std::is_same<TB, float>::value && d.a0p;
    auto residual = [&](cudaStream_t q) -> gks_status {
        if (std::is_same<TB, float>::value && d.D2) {
            if (d.SR2)
                k_resid_df<true><<<4 * nb, kBlock, 0, q>>>(d, d.D2, d.S2, k.x, reinterpret_cast<float *>(V), k.b,
                                                           k.part, ps, sxn, d.SR2, d.SB2);
            else
                k_resid_df<false><<<4 * nb, kBlock, 0, q>>>(d, d.D2, d.S2, k.x, reinterpret_cast<float *>(V), k.b,
                                                            k.part, ps, sxn);
        } else {
            spmv64(q, k.x, V, 1, k.b, sxn);
        }
        note_launch();
        GKS_CUDA(cudaGetLastError());
        return GKS_OK;
    };
    // the three fixed launch sequences (the per-part graphs end each with the
    // flags for the host, the whole-solve graph with a condition kernel)
    auto start_body = [&](cudaStream_t q) -> gks_status {
        int slot = prof_start(m, kProfCtl, q);
        if (m->cfg.precond == GKS_PC_ILU_EXACT) {
            k_sf_begin<<<1, 32, 0, q>>>(k.sf_ctl, 1);      // a new solve: clear the wait error
            note_launch();
        }
        if (rhs_df)
            k_rhs_df<<<nb, kBlock, 0, q>>>(d, d.a0p, k.w, k.b, k.part, ps);
        else
            k_rhs<<<nb, kBlock, 0, q>>>(d, k.w, k.b, k.part, ps);
        note_launch();
        if (sx) {
            // the FP32 basis stores its first vector scaled by a power of two 2^-e
            k_reduce<<<dim3(1, ns), kReduceThreads, 0, q>>>(k.part + 1, d.case_blk, ps, k.hcol + 1, ps, 0);
            note_launch();
            k_sigma<<<sblocks(ns), 128, 0, q>>>(k.hcol, ps, k.bnorm, k.sexp, ns); note_launch();
        }
        prof_stop(m, slot, q);
        slot = prof_start(m, kProfResid, q);
        // residual r = b - K x, written straight into the basis slot V_0 (v_0 = V_0 / beta)
        if (const gks_status r = residual(q); r != GKS_OK) return r;
        k_reduce<<<dim3(sx ? 1 : 2, ns), kReduceThreads, 0, q>>>(k.part, d.case_blk, ps, k.hcol, ps, 0);
        note_launch();
        prof_stop(m, slot, q);
        slot = prof_start(m, kProfCtl, q);
        k_start<<<sblocks(ns), 128, 0, q>>>(k.hcol, ps, k.bnorm, k.beta, k.vn, mm, k.ctl, ns, k.done, rtol, maxit,
                                             1, sx);
        note_launch();
        k_zero_trivial<<<nb, kBlock, 0, q>>>(d, k.x, k.bnorm); note_launch();
        k_init_g<<<sblocks(ns * (mm + 1)), 128, 0, q>>>(k.g, mm, k.beta, k.ctl, ns); note_launch();
        prof_stop(m, slot, q);
        GKS_CUDA(cudaGetLastError());
        return GKS_OK;
    };
    auto iter_body = [&](cudaStream_t q, int j) -> gks_status {
        TB *vj = V + j * vs, *vj1 = V + (j + 1) * vs;
        gks_status st;
        int slot = prof_start(m, kProfIlu, q);
        // Z_j = M^{-1} V_j, kept for the update of x at the end of the cycle
        if ((st = mixed ? precond32(m, vj, k.Z32 + j * vs, q) : precond(m, vj, k.Z + j * vs, q)) != GKS_OK)
            return st;
        prof_stop(m, slot, q);
        slot = prof_start(m, kProfSpmv, q);
        // the FP32 basis with the per-cell equations: the operator kernel also
        // forms the first Gram-Schmidt products (k_spmv_dots)
        const bool fused_dots = std::is_same<TB, float>::value && !d.alr32 && m->cfg.spmv_dots;
        if (fused_dots) {
            float *yv = reinterpret_cast<float *>(vj1);
            const float *Vf = reinterpret_cast<const float *>(V);
            const float *zj = k.Z32 + j * vs;
            switch (j) {     // the first four Arnoldi indices unrolled (the inner cycles rarely go further)
            case 0: k_spmv_dots<1><<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, zj, yv, Vf, j, k.part, ps); break;
            case 1: k_spmv_dots<2><<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, zj, yv, Vf, j, k.part, ps); break;
            case 2: k_spmv_dots<3><<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, zj, yv, Vf, j, k.part, ps); break;
            case 3: k_spmv_dots<4><<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, zj, yv, Vf, j, k.part, ps); break;
            default: k_spmv_dots<<<nb, kBlock, 0, q>>>(d, d.D32, d.alpha32, d.ex32, d.ey32, zj, yv, Vf, j, k.part, ps);
            }
        } else if (mixed) {
            spmv32(q, k.Z32 + j * vs, vj1);
        } else {
            spmv64(q, k.Z + j * vs, vj1, 0, nullptr, nullptr);
        }
        note_launch();
        prof_stop(m, slot, q);
        slot = prof_start(m, kProfOrth, q);
        // classical Gram-Schmidt: twice in FP64 mode; once in the mixed mode, whose
        // cycles only reduce the residual by inner_rtol before an FP64 restart
        if (!fused_dots && (st = dots<TB>(m, V, vj1, j, k.part, ps, q)) != GKS_OK) return st;
        k_reduce<<<dim3(j + 1, ns), kReduceThreads, 0, q>>>(k.part, d.case_blk, ps, k.hcol, ps, 0, k.vn, mm + 1,
                                                             k.hco, ps);
        note_launch();
        launch_orth_update<TB>(d, nb, q, V, vj1, j, k.hco, ps, k.ctl, ns, k.part, ps, mixed ? 1 : 0);
        note_launch();
        if (!mixed) {
            if ((st = dots<TB>(m, V, vj1, j, k.part, ps, q)) != GKS_OK) return st;
            k_reduce<<<dim3(j + 1, ns), kReduceThreads, 0, q>>>(k.part, d.case_blk, ps, k.y, mm, 0, k.vn, mm + 1,
                                                                 k.hco, ps);
            note_launch();
            launch_orth_update<TB>(d, nb, q, V, vj1, j, k.hco, ps, k.ctl, ns, k.part, ps, 1); note_launch();
            k_hadd<<<sblocks(ns * (j + 1)), 128, 0, q>>>(k.hcol, ps, k.y, mm, j, ns); note_launch();
        }
        // |V_{j+1}| and the Givens step of every system
        k_norm_givens<<<dim3(1, ns), kReduceThreads, 0, q>>>(k.part, d.case_blk, ps, j, mm, k.hcol, ps, k.vn, k.H,
                                                              k.cs, k.sn, k.g, k.ctl, ns, k.bnorm, k.beta, rtol, eta,
                                                              maxit);
        note_launch();
        prof_stop(m, slot, q);
        GKS_CUDA(cudaGetLastError());
        return GKS_OK;
    };
    auto restart_body = [&](cudaStream_t q) -> gks_status {
        int slot = prof_start(m, kProfCorr, q);
        k_backsolve<<<sblocks(ns), 128, 0, q>>>(mm, k.H, k.g, k.y, k.ctl, ns); note_launch();
        k_scale_y<<<sblocks(ns), 128, 0, q>>>(mm, k.y, k.vn, k.ctl, ns, k.g, k.bnorm, rtol, sx,
                                               mixed ? k.y32 : nullptr);
        note_launch();
        if (mixed)
            k_combine_z<float><<<dim3(nb, NV), kBlock, 0, q>>>(d, k.Z32, k.y, mm, k.ctl, ns, k.x, sx, k.y32);
        else
            k_combine_z<double><<<dim3(nb, NV), kBlock, 0, q>>>(d, k.Z, k.y, mm, k.ctl, ns, k.x);
        note_launch();
        prof_stop(m, slot, q);
        slot = prof_start(m, kProfResid, q);
        if (const gks_status r = residual(q); r != GKS_OK) return r;
        k_reduce<<<dim3(1, ns), kReduceThreads, 0, q>>>(k.part, d.case_blk, ps, k.hcol, ps, 0); note_launch();
        prof_stop(m, slot, q);
        slot = prof_start(m, kProfCtl, q);
        k_start<<<sblocks(ns), 128, 0, q>>>(k.hcol, ps, k.bnorm, k.beta, k.vn, mm, k.ctl, ns, k.done, rtol, maxit,
                                             0, sx);
        note_launch();
        k_init_g<<<sblocks(ns * (mm + 1)), 128, 0, q>>>(k.g, mm, k.beta, k.ctl, ns); note_launch();
        prof_stop(m, slot, q);
        GKS_CUDA(cudaGetLastError());
        return GKS_OK;
    };
    auto with_flags = [&](cudaStream_t q, gks_status r) { return r != GKS_OK ? r : enqueue_flags(m, q); };
    auto start_part = [&](cudaStream_t q) { return with_flags(q, start_body(q)); };
    auto iter_part = [&](cudaStream_t q, int j) { return with_flags(q, iter_body(q, j)); };
    auto restart_part = [&](cudaStream_t q) { return with_flags(q, restart_body(q)); };

    const bool use_graph = prepare_graphs(m);
    SolveGraphs *G = use_graph ? m->graphs : nullptr;
    bool whole = false;
    // the whole-solve graph holds every Arnoldi index up front: with the
    // level-by-level exact ILU (two launches per level) that is too many nodes
    // on large meshes, whose per-step graphs are built only for the indices used
    const bool few_nodes = m->cfg.precond != GKS_PC_ILU_LEVELS || m->lvl_lo_ptr.size() + m->lvl_up_ptr.size() <= 256;
    if (emb) {
        if (!G || !few_nodes || G->disabled || m->cfg.no_graphs != 0) return GKS_EINVAL;
        if ((st = build_whole(m, s, start_body, iter_body, restart_body, emb)) != GKS_OK) return st;
        int64_t nl = 0;
        st = capture_into(m, emb->g, &emb->sink, 1, &emb->sink, &nl, [&](cudaStream_t q) -> gks_status {
            k_mark_noconv<<<sblocks(ns), 128, 0, q>>>(k.bnorm, k.beta, k.done, ns, rtol, k.status, k.nsolve,
                                                         m->cfg.precond == GKS_PC_ILU_EXACT ? k.sf_ctl + 3 : nullptr);
            note_launch();
            GKS_CUDA(cudaGetLastError());
            return GKS_OK;
        });
        emb->launches = G->whole_start_launches + nl;
        return st;
    }
    if (G && few_nodes && !G->disabled && !G->whole_failed && m->cfg.no_graphs != 2) {
        if (!G->whole && build_whole(m, s, start_body, iter_body, restart_body) != GKS_OK) {
            G->whole_failed = true;                     // per-part graphs with host control from now on
            cudaGetLastError();
        }
        whole = G->whole != nullptr;
    }
    cudaGraphExec_t none = nullptr;
    int64_t none_n = 0;
    if (whole) {
        GKS_CUDA(cudaGraphLaunch(G->whole, s));
        g_launches.fetch_add(G->whole_start_launches, std::memory_order_relaxed);
        m->prof.residuals += 1;
    } else {
        if ((st = run_part(m, use_graph, G ? &G->start : &none, G ? &G->start_launches : &none_n, s,
                           start_part)) != GKS_OK)
            return st;
        m->prof.residuals += 1;
    }
    while (!whole && k.h_flags[0]) {
        for (int j = 0; j < mm; ++j) {
            m->prof.precond += 1;
            m->prof.arnoldi += 1;
            m->prof.arnoldi_jsum += j + 1;
            st = run_part(m, use_graph, G ? &G->iter[j] : &none, G ? &G->iter_launches[j] : &none_n, s,
                          [&](cudaStream_t q) { return iter_part(q, j); });
            if (st != GKS_OK) return st;
            if (!k.h_flags[1]) break;
        }
        if ((st = run_part(m, use_graph, G ? &G->restart : &none, G ? &G->restart_launches : &none_n, s,
                           restart_part)) != GKS_OK)
            return st;
        m->prof.residuals += 1;
    }
    k_mark_noconv<<<sblocks(ns), 128, 0, s>>>(k.bnorm, k.beta, k.done, ns, rtol, k.status, k.nsolve,
                                              m->cfg.precond == GKS_PC_ILU_EXACT ? k.sf_ctl + 3 : nullptr);
    note_launch();
    if (iters || relres || converged) {
        std::vector<int32_t> it(ns);
        std::vector<double> be(ns), bn(ns);
        GKS_CUDA(cudaMemcpyAsync(it.data(), k.ctl + kCtlIters * ns, sizeof(int32_t) * ns, cudaMemcpyDeviceToHost, s));
        GKS_CUDA(cudaMemcpyAsync(be.data(), k.beta, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        GKS_CUDA(cudaMemcpyAsync(bn.data(), k.bnorm, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        if (whole)
            GKS_CUDA(cudaMemcpyAsync(G->h_ctr, G->ctr, sizeof(int64_t) * kCtrLen, cudaMemcpyDeviceToHost, s));
        GKS_CUDA(cudaStreamSynchronize(s));
        if (whole) take_counters(m);
        int32_t conv = 1;
        for (int q = 0; q < ns; ++q) {
            const double rr = bn[q] > 0.0 ? be[q] / bn[q] : 0.0;
            if (iters) iters[q] = it[q];
            if (relres) relres[q] = rr;
            if (rr > rtol) conv = 0;
        }
        if (converged) *converged = conv;
    }
    return GKS_OK;
}

namespace {

// the extrapolated warm start of the next solve (if configured)
gks_status launch_warm(gks_mesh *m, cudaStream_t s)
{
    Work &k = m->wk;
    if (!m->cfg.warm_extrap) return GKS_OK;
    const int slot = prof_start(m, kProfCtl, s);
    k_warm<<<(unsigned)k.nblk, kBlock, 0, s>>>(m->d, k.x, k.x_prev, k.x_prev2, k.done, k.nsolve, m->cfg.warm_extrap);
    note_launch();
    prof_stop(m, slot, s);
    GKS_CUDA(cudaGetLastError());
    return GKS_OK;
}

// The step loop as a graph (see run_graph_launch):
//   c = any case not done and a loop limit above 0
//   while (c) { CFL step, clipped to the end times; warm start;
//               the device-controlled solve; solve count and convergence marks;
//               iteration sums; limiter; flux; update; per-case clocks;
//               c = any case not done and the loops of this launch below the limit }
gks_status build_run(gks_mesh *m, cudaStream_t s)
{
    SolveGraphs &G = *m->graphs;
    Work &k = m->wk;
    const int n = m->n_case;
    if (const gks_status r = ensure_counters(m, s); r != GKS_OK) return r;
    if (!G.h_run) GKS_CUDA(cudaMallocHost(&G.h_run, sizeof(int64_t)));
    int64_t *ctr = G.ctr;
    cudaGraph_t top = nullptr;
    GKS_CUDA(cudaGraphCreate(&top, 0));
    gks_status st = GKS_OK;
    int64_t nl_entry = 0, nl_a = 0, nl_b = 0;
    SolveEmbed e;
    do {
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, top, 0, 0) != cudaSuccess) { st = GKS_ECUDA; break; }
        cudaGraphNode_t sink, wnode;
        cudaGraph_t body;
        st = capture_into(m, top, nullptr, 0, &sink, &nl_entry, [&](cudaStream_t q) -> gks_status {
            k_run_cond<<<1, kBlock, 0, q>>>(k.done, n, k.run_ctl, ctr, h, 1); note_launch();
            return GKS_OK;
        });
        if (st != GKS_OK || (st = add_cond(top, sink, h, cudaGraphCondTypeWhile, &wnode, &body)) != GKS_OK) break;
        st = capture_into(m, body, nullptr, 0, &sink, &nl_a, [&](cudaStream_t q) -> gks_status {
            gks_status r;
            if ((r = launch_cfl_dt(m, k.w, k.dt, q)) != GKS_OK) return r;
            if ((r = launch_clip_only(m, q)) != GKS_OK) return r;
            return launch_warm(m, q);
        });
        if (st != GKS_OK) break;
        e.g = body;
        e.dep = sink;
        st = k.V32 ? cls_solve_t<float>(m, k.V32, s, nullptr, nullptr, nullptr, &e)
                   : cls_solve_t<double>(m, k.V, s, nullptr, nullptr, nullptr, &e);
        if (st != GKS_OK) break;
        st = capture_into(m, body, &e.sink, 1, &sink, &nl_b, [&](cudaStream_t q) -> gks_status {
            gks_status r;
            if ((r = launch_acc_iters(m, q)) != GKS_OK) return r;
            if (m->cfg.limiter && (r = launch_limiter(m, k.w, k.x, q)) != GKS_OK) return r;
            if ((r = launch_flux(m, k.w, m->cfg.limiter ? k.xl : k.x, 0.0, k.dt, k.flux, q)) != GKS_OK) return r;
            if ((r = launch_update(m, k.w, k.flux, q)) != GKS_OK) return r;
            if ((r = launch_after_step(m, q)) != GKS_OK) return r;
            k_run_cond<<<1, kBlock, 0, q>>>(k.done, n, k.run_ctl, ctr, h, 0); note_launch();
            GKS_CUDA(cudaGetLastError());
            return GKS_OK;
        });
        if (st != GKS_OK) break;
        if (cudaGraphInstantiate(&G.run, top, 0) != cudaSuccess) {
            G.run = nullptr;
            st = GKS_ECUDA;
        }
    } while (false);
    cudaGraphDestroy(top);
    cudaGetLastError();
    if (st != GKS_OK) return st;
    G.run_loop_launches = nl_a + e.launches + nl_b;
    G.run_cfg = m->cfg;
    return GKS_OK;
}

}  // namespace

gks_status cls_solve(gks_mesh *m, cudaStream_t s, int32_t *iters, double *relres, int32_t *converged)
{
    Work &k = m->wk;
    if (const gks_status st = launch_warm(m, s); st != GKS_OK) return st;
    return k.V32 ? cls_solve_t<float>(m, k.V32, s, iters, relres, converged)
                 : cls_solve_t<double>(m, k.V, s, iters, relres, converged);
}

gks_status run_graph_launch(gks_mesh *m, int64_t max_steps, cudaStream_t s, bool *used)
{
    *used = false;
    if (m->cfg.no_graphs != 0 || !prepare_graphs(m)) return GKS_OK;
    SolveGraphs &G = *m->graphs;
    if (G.run_failed || G.disabled) return GKS_OK;
    if (G.run && std::memcmp(&G.run_cfg, &m->cfg, sizeof(gks_config)) != 0) {
        flush_solve_counters(m);                   // counted with the old graph's launch numbers
        cudaGraphExecDestroy(G.run);
        G.run = nullptr;
    }
    if (!G.run && build_run(m, s) != GKS_OK) {
        G.run_failed = true;                       // the host loop from now on
        cudaGetLastError();
        return GKS_OK;
    }
    *G.h_run = max_steps;
    GKS_CUDA(cudaMemcpyAsync(m->wk.run_ctl + 1, G.h_run, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    GKS_CUDA(cudaGraphLaunch(G.run, s));
    g_launches.fetch_add(1, std::memory_order_relaxed);   // the entry condition
    *used = true;
    return GKS_OK;
}

void flush_solve_counters(gks_mesh *m)
{
    SolveGraphs *g = m->graphs;
    if (!g || !g->ctr) return;
    if (cudaDeviceSynchronize() == cudaSuccess &&
        cudaMemcpy(g->h_ctr, g->ctr, sizeof(int64_t) * kCtrLen, cudaMemcpyDeviceToHost) == cudaSuccess)
        take_counters(m);
    cudaGetLastError();
}

void destroy_graph_execs(SolveGraphs *g)
{
    for (cudaGraphExec_t &e : g->iter)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    if (g->start) cudaGraphExecDestroy(g->start);
    if (g->restart) cudaGraphExecDestroy(g->restart);
    if (g->whole) cudaGraphExecDestroy(g->whole);
    if (g->run) cudaGraphExecDestroy(g->run);
    g->start = g->restart = g->whole = g->run = nullptr;
}

}  // namespace gks
