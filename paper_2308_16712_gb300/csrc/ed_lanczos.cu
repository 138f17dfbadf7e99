// ed_lanczos.cu -- the Krylov eigensolver that consumes the matvec (the paper's
// Background: Lanczos needs hundreds of matrix-vector products).
//
// Recurrence (fp64 on the GPU):  v_0 = x0 / |x0|,
//   w = H v_j,  alpha_j = Re <v_j, w>,  w -= alpha_j v_j + beta_j v_{j-1},
//   beta_{j+1} = |w|,  v_{j+1} = w / beta_{j+1}.
// Dot products and norms are compensated (Neumaier) sums over a fixed
// partition, so a second pass reproduces alpha/beta bit for bit.  The lowest
// eigenpair of the tridiagonal matrix comes from Sturm-count bisection and
// inverse iteration in a single-thread kernel.  With ED_LANCZOS_F32_MATVEC the
// matvec runs in fp32 (its input is the fp32 copy of v_j written by the
// normalisation kernel) and the Ritz vector is refined by a few fp64 Lanczos
// steps started from it.  The returned energy is the fp64 Rayleigh quotient of
// the final vector, with its fp64 residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "ed_kernels.cuh"

namespace edk {
namespace {

constexpr int kRedThreads = 256;
constexpr int kRefineSteps = 6;

// ---- compensated sums ------------------------------------------------------
// fp64 is the scarce resource on this GPU, so each thread sums its few dozen
// elements with plain fp64 fused multiply-adds into two accumulators, and only
// the merges across threads and blocks are compensated: Knuth's branch-free
// TwoSum carries the rounding error of every merge in a second word.
struct KSum {
    double s, c;
};

__device__ __forceinline__ KSum two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ KSum ksum_merge(KSum a, KSum b)
{
    KSum r = two_sum(a.s, b.s);
    r.c += a.c + b.c;
    return r;
}

// Block-wide merge of (s, c) pairs in a fixed tree order; result in thread 0.
__device__ KSum block_ksum(KSum k)
{
    __shared__ double sm_s[kRedThreads / 32], sm_c[kRedThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        KSum other{__shfl_down_sync(0xffffffffu, k.s, o), __shfl_down_sync(0xffffffffu, k.c, o)};
        k = ksum_merge(k, other);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sm_s[wid] = k.s;
        sm_c[wid] = k.c;
    }
    __syncthreads();
    if (wid == 0) {
        k = lane < kRedThreads / 32 ? KSum{sm_s[lane], sm_c[lane]} : KSum{0.0, 0.0};
        for (int o = 16; o > 0; o >>= 1) {
            KSum other{__shfl_down_sync(0xffffffffu, k.s, o), __shfl_down_sync(0xffffffffu, k.c, o)};
            k = ksum_merge(k, other);
        }
    }
    __syncthreads();
    return k;
}

// Sum of the per-block partials (fixed order), every block computes the same value.
__device__ double reduce_partials(const double2 *part, int nparts)
{
    KSum k{0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
        k = ksum_merge(k, KSum{part[i].x, part[i].y});
    k = block_ksum(k);
    __shared__ double total;
    if (threadIdx.x == 0)
        total = k.s + k.c;
    __syncthreads();
    return total;
}


// ---- vector element access (real or complex, fp64 or fp32) -------------------
template <bool kC> struct Vec;
template <> struct Vec<false> {
    using D = double;
    using F = float;
    __device__ static double dot(double a, double b) { return a * b; }
    __device__ static double dotf(double a, float b) { return a * (double)b; }
    __device__ static double norm2(double a) { return a * a; }
    __device__ static double up(float a) { return (double)a; }
    __device__ static float down(double a) { return (float)a; }
    __device__ static double axpby(double w, double a, double v, double b, double p) { return fma(-b, p, fma(-a, v, w)); }
    __device__ static double scale(double w, double s) { return w * s; }
    __device__ static double zero() { return 0.0; }
    __device__ static double fma_acc(double acc, double y, double v) { return acc + y * v; }
};
template <> struct Vec<true> {
    using D = double2;
    using F = float2;
    __device__ static double dot(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }
    __device__ static double dotf(double2 a, float2 b) { return a.x * (double)b.x + a.y * (double)b.y; }
    __device__ static double norm2(double2 a) { return a.x * a.x + a.y * a.y; }
    __device__ static double2 up(float2 a) { return make_double2(a.x, a.y); }
    __device__ static float2 down(double2 a) { return make_float2((float)a.x, (float)a.y); }
    __device__ static double2 axpby(double2 w, double a, double2 v, double b, double2 p)
    {
        return make_double2(fma(-b, p.x, fma(-a, v.x, w.x)), fma(-b, p.y, fma(-a, v.y, w.y)));
    }
    __device__ static double2 scale(double2 w, double s) { return make_double2(w.x * s, w.y * s); }
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 fma_acc(double2 acc, double y, double2 v)
    {
        return make_double2(acc.x + y * v.x, acc.y + y * v.y);
    }
};

// The block that finishes last: every block stores its partial (thread 0),
// fences, and takes a ticket; the one that draws gridDim.x - 1 knows every
// partial is visible.  Nothing waits, so no block can stall another.
__device__ bool is_last_block(unsigned int *ticket)
{
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    return last;
}

// The sum of the block partials in block order (the same merge order as
// reduce_partials), read through L2; valid in thread 0.
__device__ double sum_partials_l2(const double2 *part, int nparts)
{
    KSum k{0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const double2 p = __ldcg(part + i);
        k = ksum_merge(k, KSum{p.x, p.y});
    }
    k = block_ksum(k);
    return k.s + k.c;
}

// partial[b] = compensated sum over this block's slice of Re<a_i, b_i>; with a
// ticket, the last block also stores the total in out[*jp] (out[0] without a
// step index) and resets the ticket.  Four elements per iteration, loads
// first, for memory-level parallelism.
template <bool kC, bool kF32>
__global__ void __launch_bounds__(kRedThreads) k_dot_part(const typename Vec<kC>::D *a, const void *bv,
                                                           uint64_t n, double2 *part, unsigned int *ticket,
                                                           double *out, const int *jp = nullptr)
{
    using VT = Vec<kC>;
    using B = std::conditional_t<kF32, typename VT::F, typename VT::D>;
    const B *bp = reinterpret_cast<const B *>(bv);
    auto dotv = [](typename VT::D x, B y) {
        if constexpr (kF32)
            return VT::dotf(x, y);
        else
            return VT::dot(x, y);
    };
    double s0 = 0.0, s1 = 0.0;
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    const uint64_t bs = blockDim.x;
    uint64_t i = lo + threadIdx.x;
    for (; i + 3 * bs < hi; i += 4 * bs) {
        const typename VT::D a0 = a[i], a1 = a[i + bs], a2 = a[i + 2 * bs], a3 = a[i + 3 * bs];
        const B b0 = bp[i], b1 = bp[i + bs], b2 = bp[i + 2 * bs], b3 = bp[i + 3 * bs];
        s0 += dotv(a0, b0);
        s1 += dotv(a1, b1);
        s0 += dotv(a2, b2);
        s1 += dotv(a3, b3);
    }
    for (; i < hi; i += bs)
        s0 += dotv(a[i], bp[i]);
    const KSum k = block_ksum(two_sum(s0, s1));
    if (threadIdx.x == 0)
        part[blockIdx.x] = make_double2(k.s, k.c);
    if (ticket && is_last_block(ticket)) {
        const double t = sum_partials_l2(part, gridDim.x);
        if (threadIdx.x == 0) {
            out[jp ? *jp : 0] = t;
            *ticket = 0;
        }
    }
}

template <bool kC>
__global__ void __launch_bounds__(kRedThreads) k_norm_part(const typename Vec<kC>::D *a, uint64_t n, double2 *part)
{
    using VT = Vec<kC>;
    double s0 = 0.0, s1 = 0.0;
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    uint64_t i = lo + threadIdx.x;
    for (; i + blockDim.x < hi; i += 2 * blockDim.x) {
        s0 += VT::norm2(a[i]);
        s1 += VT::norm2(a[i + blockDim.x]);
    }
    if (i < hi)
        s0 += VT::norm2(a[i]);
    const KSum k = block_ksum(two_sum(s0, s1));
    if (threadIdx.x == 0)
        part[blockIdx.x] = make_double2(k.s, k.c);
}

// w = w_in - alpha_j v - beta_j vp (alpha_j and beta_j already stored); norm
// partials of w; with a ticket, the last block stores sqrt(|w|^2) in *beta_out.
// With a step index jp, alpha, beta_j and beta_out are offset by *jp.
template <bool kC, bool kF32>
__global__ void __launch_bounds__(kRedThreads) k_update(const void *w_in, typename Vec<kC>::D *w,
                                                         const typename Vec<kC>::D *v,
                                                         const typename Vec<kC>::D *vp, uint64_t n,
                                                         const double *alpha, const double *beta_j,
                                                         double2 *norm_part, unsigned int *ticket,
                                                         double *beta_out, const int *jp = nullptr)
{
    if (jp) {
        alpha += *jp;
        beta_j += *jp;
        beta_out += *jp;
    }
    using VT = Vec<kC>;
    using D = typename VT::D;
    using WI = std::conditional_t<kF32, typename VT::F, D>;
    const WI *wp = reinterpret_cast<const WI *>(w_in);
    auto upw = [](WI x) {
        if constexpr (kF32)
            return VT::up(x);
        else
            return x;
    };
    const double a = *alpha;
    const double b = vp ? *beta_j : 0.0;
    double s0 = 0.0, s1 = 0.0;
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    const uint64_t bs = blockDim.x;
    uint64_t i = lo + threadIdx.x;
    for (; i + 3 * bs < hi; i += 4 * bs) {
        D wv[4], vv[4], pv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            wv[u] = upw(wp[i + u * bs]);
            vv[u] = v[i + u * bs];
            pv[u] = vp ? vp[i + u * bs] : VT::zero();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const D r = VT::axpby(wv[u], a, vv[u], b, pv[u]);
            w[i + u * bs] = r;
            if (u & 1)
                s1 += VT::norm2(r);
            else
                s0 += VT::norm2(r);
        }
    }
    for (; i < hi; i += bs) {
        const D r = VT::axpby(upw(wp[i]), a, v[i], b, vp ? vp[i] : VT::zero());
        w[i] = r;
        s0 += VT::norm2(r);
    }
    const KSum k = block_ksum(two_sum(s0, s1));
    if (threadIdx.x == 0)
        norm_part[blockIdx.x] = make_double2(k.s, k.c);
    if (ticket && is_last_block(ticket)) {
        const double t = sum_partials_l2(norm_part, gridDim.x);
        if (threadIdx.x == 0) {
            *beta_out = sqrt(fmax(t, 0.0));
            *ticket = 0;
        }
    }
}

// beta_{j+1} = sqrt(sum of the norm partials) in one block (after the
// reorthogonalisation has replaced w and its partials)
__global__ void __launch_bounds__(kRedThreads) k_norm_final(const double2 *part, int nparts, double *beta)
{
    const double t = reduce_partials(part, nparts);
    if (threadIdx.x == 0)
        *beta = sqrt(fmax(t, 0.0));
}

// v_out = w / beta (zero on breakdown); fp32 copy; four elements per thread
// per iteration.  With a step index jp: beta is offset by *jp, and with a
// store, the vector is also written as stored vector *jp + 1.
template <bool kC>
__global__ void __launch_bounds__(kRedThreads) k_normalize(const typename Vec<kC>::D *w,
                                                            typename Vec<kC>::D *v_out,
                                                            typename Vec<kC>::F *x32, uint64_t n,
                                                            const double *beta, const int *jp = nullptr,
                                                            typename Vec<kC>::D *store = nullptr)
{
    using VT = Vec<kC>;
    if (jp) {
        beta += *jp;
        if (store)
            store += (uint64_t)(*jp + 1) * n;
    }
    const double b = *beta;
    const double s = b > 0.0 ? 1.0 / b : 0.0;
    const uint64_t G = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * G < n; i += 4 * G) {
        typename VT::D r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            r[u] = VT::scale(w[i + u * G], s);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            v_out[i + u * G] = r[u];
            if (x32)
                x32[i + u * G] = VT::down(r[u]);
            if (jp && store)
                store[i + u * G] = r[u];
        }
    }
    for (; i < n; i += G) {
        const typename VT::D r = VT::scale(w[i], s);
        v_out[i] = r;
        if (x32)
            x32[i] = VT::down(r);
        if (jp && store)
            store[i] = r;
    }
}

// acc += y[j] * v   (Ritz vector accumulation, second pass); with a step
// index jp, j = *jp and the first step (j = 0) overwrites acc
template <bool kC>
__global__ void k_axpy_coef(typename Vec<kC>::D *acc, const typename Vec<kC>::D *v, const double *y, int j,
                            uint64_t n, int first, const int *jp = nullptr)
{
    using VT = Vec<kC>;
    if (jp) {
        j = *jp;
        first = j == 0;
    }
    const double c = y[j];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        acc[i] = VT::fma_acc(first ? VT::zero() : acc[i], c, v[i]);
}

__global__ void k_step_set(int *jp, int v) { *jp = v; }
__global__ void k_step_inc(int *jp) { *jp += 1; }

// psi[i] = sum_j y[j] V[j][i] over stored Krylov vectors
template <bool kC>
__global__ void k_combine(typename Vec<kC>::D *psi, const typename Vec<kC>::D *V, const double *y,
                          const int *m_eff, uint64_t n)
{
    using VT = Vec<kC>;
    const int m = *m_eff;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        typename VT::D acc = VT::zero();
        for (int j = 0; j < m; ++j)
            acc = VT::fma_acc(acc, y[j], V[(uint64_t)j * n + i]);
        psi[i] = acc;
    }
}

// x_out = x_in / sqrt(sum of partials)
template <bool kC>
__global__ void k_scale_by_norm(const typename Vec<kC>::D *in, typename Vec<kC>::D *out,
                                typename Vec<kC>::F *x32, uint64_t n, const double2 *part, int nparts)
{
    using VT = Vec<kC>;
    const double nrm = sqrt(fmax(reduce_partials(part, nparts), 0.0));
    const double s = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const typename VT::D r = VT::scale(in[i], s);
        out[i] = r;
        if (x32)
            x32[i] = VT::down(r);
    }
}

// r = a - theta b with theta = <b,a>/<b,b> (from partials); partials of |r|^2
template <bool kC>
__global__ void __launch_bounds__(kRedThreads) k_residual(const typename Vec<kC>::D *hu,
                                                           const typename Vec<kC>::D *u, uint64_t n,
                                                           const double2 *num_part,
                                                           const double2 *den_part, int nparts,
                                                           double *theta_out, double2 *res_part)
{
    using VT = Vec<kC>;
    const double num = reduce_partials(num_part, nparts);
    const double den = reduce_partials(den_part, nparts);
    const double th = num / den;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        *theta_out = th;
    double s0 = 0.0;
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        s0 += VT::norm2(VT::axpby(hu[i], th, u[i], 0.0, VT::zero()));
    const KSum k = block_ksum(KSum{s0, 0.0});
    if (threadIdx.x == 0)
        res_part[blockIdx.x] = make_double2(k.s, k.c);
}

__global__ void k_finish_residual(const double2 *res_part, const double2 *den_part, int nparts,
                                  double *out)
{
    const double r = reduce_partials(res_part, nparts);
    const double d = reduce_partials(den_part, nparts);
    if (threadIdx.x == 0)
        *out = sqrt(fmax(r, 0.0) / d);
}

// ---- full reorthogonalisation against the kept Krylov vectors ----------------
struct Part4 {  // compensated real and imaginary parts of one block's partial
    double rs, rc, is, ic;
};
// Classical Gram-Schmidt applied twice: c_k = <V_k, w> for k < kcount, then
// w -= sum_k c_k V_k.  Complex vectors use the Hermitian product.
// part[k * gridDim.x + b] = block b's slice of c_k as (re.s, re.c, im.s, im.c).
template <bool kC>
__global__ void __launch_bounds__(kRedThreads) k_reorth_dot(const typename Vec<kC>::D *V,
                                                             const typename Vec<kC>::D *w, uint64_t n,
                                                             int kcount, Part4 *part)
{
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    for (int k = 0; k < kcount; ++k) {
        const typename Vec<kC>::D *vk = V + (uint64_t)k * n;
        double sr = 0.0, si = 0.0;
        for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            if constexpr (kC) {
                const double2 a = vk[i], b = w[i];
                sr = fma(a.x, b.x, fma(a.y, b.y, sr));
                si = fma(a.x, b.y, fma(-a.y, b.x, si));
            } else {
                sr = fma(vk[i], w[i], sr);
            }
        }
        const KSum kr = block_ksum(KSum{sr, 0.0});
        KSum ki{0.0, 0.0};
        if constexpr (kC)
            ki = block_ksum(KSum{si, 0.0});
        if (threadIdx.x == 0)
            part[(uint64_t)k * gridDim.x + blockIdx.x] = Part4{kr.s, kr.c, ki.s, ki.c};
    }
}

// c[k] = sum of the block partials of coefficient k (one block per k)
__global__ void __launch_bounds__(kRedThreads) k_reorth_coef(const Part4 *part, int nparts, double2 *c)
{
    const int k = blockIdx.x;
    KSum r{0.0, 0.0}, im{0.0, 0.0};
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
        const Part4 p = part[(uint64_t)k * nparts + b];
        r = ksum_merge(r, KSum{p.rs, p.rc});
        im = ksum_merge(im, KSum{p.is, p.ic});
    }
    r = block_ksum(r);
    im = block_ksum(im);
    if (threadIdx.x == 0)
        c[k] = make_double2(r.s + r.c, im.s + im.c);
}

// w -= sum_k c_k V_k; norm partials of the result
template <bool kC>
__global__ void __launch_bounds__(kRedThreads) k_reorth_update(const typename Vec<kC>::D *V,
                                                                typename Vec<kC>::D *w, uint64_t n,
                                                                int kcount, const double2 *c,
                                                                double2 *norm_part)
{
    using VT = Vec<kC>;
    const uint64_t per = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t lo = min(n, blockIdx.x * per), hi = min(n, lo + per);
    double s0 = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        typename VT::D acc = w[i];
        for (int k = 0; k < kcount; ++k) {
            const double2 ck = c[k];
            const typename VT::D vk = V[(uint64_t)k * n + i];
            if constexpr (kC) {
                acc.x -= ck.x * vk.x - ck.y * vk.y;
                acc.y -= ck.x * vk.y + ck.y * vk.x;
            } else {
                acc -= ck.x * vk;
            }
        }
        w[i] = acc;
        s0 += VT::norm2(acc);
    }
    const KSum k = block_ksum(KSum{s0, 0.0});
    if (threadIdx.x == 0)
        norm_part[blockIdx.x] = make_double2(k.s, k.c);
}

// ---- tridiagonal eigensolver (one thread) ------------------------------------
// Number of eigenvalues of T (diag a, offdiag b) below x (Sturm sequence).
__device__ int sturm_count(const double *a, const double *b, int m, double x)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        const double bb = i ? b[i] * b[i] : 0.0;
        d = (a[i] - x) - (i ? bb / d : 0.0);
        if (d == 0.0)
            d = -1e-300;
        if (d < 0.0)
            ++cnt;
    }
    return cnt;
}

// Lowest eigenvalue and eigenvector of the leading m_eff x m_eff block, where
// m_eff stops at the first beta that vanishes (invariant subspace).
// a[0..m), beta[0..m]: beta[j] couples v_{j-1} and v_j (beta[0] unused).
// One warp: multisection -- each lane evaluates the Sturm count at one of 32
// interior points, which shrinks the bracket of the lowest eigenvalue 33-fold
// per round -- then inverse iteration on lane 0.  Launch with 32 threads.
__global__ void k_tridiag_lowest(const double *alpha, const double *beta, int m, double *y,
                                 double *lambda_out, int *m_eff_out, double *work)
{
    const int lane = threadIdx.x & 31;
    int me = m;
    double scale = 0.0, lo = 1e300, hi = -1e300;
    if (lane == 0) {
        for (int i = 0; i < m; ++i)
            scale = fmax(scale, fabs(alpha[i]) + fabs(beta[i + 1]));
        for (int i = 1; i < m; ++i)
            if (!(beta[i] > 1e-13 * fmax(scale, 1e-300))) {
                me = i;
                break;
            }
        for (int i = 0; i < me; ++i) {  // Gershgorin interval
            const double r = (i ? fabs(beta[i]) : 0.0) + (i + 1 < me ? fabs(beta[i + 1]) : 0.0);
            lo = fmin(lo, alpha[i] - r);
            hi = fmax(hi, alpha[i] + r);
        }
    }
    me = __shfl_sync(0xffffffffu, me, 0);
    scale = __shfl_sync(0xffffffffu, scale, 0);
    lo = __shfl_sync(0xffffffffu, lo, 0);
    hi = __shfl_sync(0xffffffffu, hi, 0);
    for (int it = 0; it < 24; ++it) {
        const double width = hi - lo;
        if (!(width > 2e-16 * fmax(fabs(lo), fabs(hi))))
            break;
        const double x = lo + width * (double)(lane + 1) / 33.0;
        const unsigned below = __ballot_sync(0xffffffffu, sturm_count(alpha, beta, me, x) >= 1);
        // first lane whose point has an eigenvalue below it
        const int f = below ? __ffs(below) - 1 : 32;
        const double nlo = f == 0 ? lo : lo + width * (double)f / 33.0;
        const double nhi = f == 32 ? hi : lo + width * (double)(f + 1) / 33.0;
        lo = nlo;
        hi = nhi;
    }
    if (lane != 0)
        return;
    const double lam = 0.5 * (lo + hi);
    // inverse iteration: (T - lam I) z = y, LU without pivoting with guarded pivots
    double *dd = work;  // pivots
    const double eps = 1e-15 * fmax(scale, 1e-300);
    for (int i = 0; i < me; ++i)
        y[i] = 1.0;
    for (int iter = 0; iter < 4; ++iter) {
        double piv = alpha[0] - lam;
        if (fabs(piv) < eps)
            piv = eps;
        dd[0] = piv;
        for (int i = 1; i < me; ++i) {
            const double l = beta[i] / dd[i - 1];
            piv = (alpha[i] - lam) - l * beta[i];
            if (fabs(piv) < eps)
                piv = eps;
            dd[i] = piv;
            y[i] -= l * y[i - 1];
        }
        y[me - 1] /= dd[me - 1];
        for (int i = me - 2; i >= 0; --i)
            y[i] = (y[i] - beta[i + 1] * y[i + 1]) / dd[i];
        double nrm = 0.0;
        for (int i = 0; i < me; ++i)
            nrm += y[i] * y[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < me; ++i)
            y[i] /= nrm;
    }
    for (int i = me; i < m; ++i)
        y[i] = 0.0;
    *lambda_out = lam;
    *m_eff_out = me;
}

// Eigenvalue number blockIdx.x (0 = lowest) of the leading m_eff x m_eff block
// (m_eff as found by k_tridiag_lowest), by the same 32-point multisection with
// the criterion "at least blockIdx.x + 1 eigenvalues below x"; NaN beyond m_eff.
// Launch with 32 threads per block, one block per eigenvalue.
__global__ void k_tridiag_kth(const double *alpha, const double *beta, int m, const int *m_eff, double *out)
{
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x;
    const int me = *m_eff;
    if (e >= me) {
        if (lane == 0)
            out[e] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double lo = 1e300, hi = -1e300;
    if (lane == 0) {
        for (int i = 0; i < me; ++i) {  // Gershgorin interval
            const double r = (i ? fabs(beta[i]) : 0.0) + (i + 1 < me ? fabs(beta[i + 1]) : 0.0);
            lo = fmin(lo, alpha[i] - r);
            hi = fmax(hi, alpha[i] + r);
        }
    }
    lo = __shfl_sync(0xffffffffu, lo, 0);
    hi = __shfl_sync(0xffffffffu, hi, 0);
    for (int it = 0; it < 24; ++it) {
        const double width = hi - lo;
        if (!(width > 2e-16 * fmax(fabs(lo), fabs(hi))))
            break;
        const double x = lo + width * (double)(lane + 1) / 33.0;
        const unsigned below = __ballot_sync(0xffffffffu, sturm_count(alpha, beta, me, x) >= e + 1);
        const int f = below ? __ffs(below) - 1 : 32;
        const double nlo = f == 0 ? lo : lo + width * (double)f / 33.0;
        const double nhi = f == 32 ? hi : lo + width * (double)(f + 1) / 33.0;
        lo = nlo;
        hi = nhi;
    }
    if (lane == 0)
        out[e] = 0.5 * (lo + hi);
}


// CUDA event pairs around every matvec launch; summed after the final sync.
struct MatvecTimer {
    std::vector<cudaEvent_t> ev;
    ~MatvecTimer()
    {
        for (cudaEvent_t e : ev)
            cudaEventDestroy(e);
    }
    cudaError_t mark(cudaStream_t st)
    {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess)
            return r;
        ev.push_back(e);
        return cudaEventRecord(e, st);
    }
    double total_ms() const
    {
        double t = 0.0;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[i], ev[i + 1]) == cudaSuccess)
                t += ms;
        }
        return t;
    }
};

// Steps replayed from a CUDA graph: -1 = for sectors of at most
// kGraphMaxDim states (launch-bound; larger sectors spend microseconds per
// launch against milliseconds per kernel), 0 = never, 1 = always.
int g_lanczos_graph = -1;
constexpr uint64_t kGraphMaxDim = 1ULL << 22;

// The capture stream and the graphs of one call, released on every exit path.
struct Graphs {
    cudaStream_t cap = nullptr;
    std::vector<cudaGraph_t> graphs;
    std::vector<cudaGraphExec_t> execs;
    ~Graphs()
    {
        for (auto g : execs)
            cudaGraphExecDestroy(g);
        for (auto g : graphs)
            cudaGraphDestroy(g);
        if (cap)
            cudaStreamDestroy(cap);
    }
};

// Work arrays of one call, from the library's stream-ordered pool.
struct Scratch {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    ~Scratch()
    {
        for (void *p : ptrs)
            ws_free(p, st);
    }
    template <typename T>
    cudaError_t get(T **p, size_t count)
    {
        cudaError_t e = ws_alloc((void **)p, std::max<size_t>(count, 1) * sizeof(T), st);
        if (e == cudaSuccess)
            ptrs.push_back((void *)*p);
        return e;
    }
};

#define ED_L_TRY(expr)                                                      \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) {                                            \
            (void)cudaGetLastError();                                       \
            return _e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA; \
        }                                                                   \
    } while (0)

template <bool kC>
ed_status run_lanczos(const ed_operator *op, const ed_basis *b, const void *x0, int steps,
                      ed_lanczos_mode mode, bool recompute, bool push, bool reorth, bool values_only, int n_eig,
                      double *eigs_out, double *e0_out, void *vec_out,
                      ed_lanczos_info *info, cudaStream_t st)
{
    using D = typename Vec<kC>::D;
    using F = typename Vec<kC>::F;
    const uint64_t n = b->dim;
    const bool f32 = mode == ED_LANCZOS_F32_MATVEC;
    const ed_dtype dt64 = kC ? ED_C128 : ED_F64, dt32 = kC ? ED_C64 : ED_F32;
    const OpView ov = make_op_view(op);
    const GroupView gv = b->group_view();
    const IndexView iv = b->index_view();
    const bool track = !b->trivial_chars;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int nparts = std::max(1, std::min<int>(sms * 8, (int)((n + kRedThreads - 1) / kRedThreads)));
    const int vgrid = std::max(1, std::min<int>(sms * 8, (int)((n + kRedThreads - 1) / kRedThreads)));

    // store the Krylov basis if it fits in half of the free memory
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    free_b += ws_cached_bytes();
    const size_t vec_bytes = n * sizeof(D);
    const bool store = !values_only && !recompute && (double)(steps + 1) * vec_bytes < 0.5 * (double)free_b;
    // push products are not bit-reproducible, so a recomputed pass would not
    // retrace the first one
    if (push && (!store || !ov.exchange_only || !(iv.htab || iv.bkt)))
        return ED_ERR_UNSUPPORTED;
    // reorthogonalisation needs every earlier Lanczos vector
    if (reorth && !store)
        return ED_ERR_UNSUPPORTED;

    const bool graph = !reorth && !push && (g_lanczos_graph == 1 || (g_lanczos_graph < 0 && n <= kGraphMaxDim));
    Scratch S(st);
    Graphs GR;
    D *V = nullptr, *w = nullptr, *ring[2] = {nullptr, nullptr}, *psi = nullptr;
    F *x32 = nullptr, *w32 = nullptr;
    double *alpha = nullptr, *beta = nullptr, *y = nullptr, *work = nullptr, *scal = nullptr;
    int *m_eff = nullptr;
    double2 *part_a = nullptr, *part_b = nullptr, *part_c = nullptr;
    if (store)
        ED_L_TRY(S.get(&V, (size_t)(steps + 1) * n));
    if (!store || graph) {  // the graph's steps run on the ring and copy into the store
        ED_L_TRY(S.get(&ring[0], n));
        ED_L_TRY(S.get(&ring[1], n));
    }
    int *jdev = nullptr;  // the step index of graph-replayed steps
    if (graph)
        ED_L_TRY(S.get(&jdev, 1));
    ED_L_TRY(S.get(&w, n));
    ED_L_TRY(S.get(&psi, n));
    if (f32) {
        ED_L_TRY(S.get(&x32, n));
        ED_L_TRY(S.get(&w32, n));
    }
    const int mref = kRefineSteps;
    const int mmax = std::max(steps, mref);
    ED_L_TRY(S.get(&alpha, mmax + 1));
    ED_L_TRY(S.get(&beta, mmax + 2));
    ED_L_TRY(S.get(&y, mmax + 1));
    ED_L_TRY(S.get(&work, 2 * (mmax + 1)));
    ED_L_TRY(S.get(&scal, 8));
    ED_L_TRY(S.get(&m_eff, 1));
    ED_L_TRY(S.get(&part_a, nparts));
    ED_L_TRY(S.get(&part_b, nparts));
    ED_L_TRY(S.get(&part_c, nparts));
    unsigned int *tickets = nullptr;  // last-block tickets of k_dot_part and k_update
    ED_L_TRY(S.get(&tickets, 2));
    ED_L_TRY(cudaMemsetAsync(tickets, 0, 2 * sizeof(unsigned int), st));
    Part4 *rpart = nullptr;
    double2 *rcoef = nullptr;
    double *d_eigs = nullptr;
    if (reorth) {
        ED_L_TRY(S.get(&rpart, (size_t)(mmax + 2) * nparts));
        ED_L_TRY(S.get(&rcoef, mmax + 2));
    }
    if (n_eig > 0)
        ED_L_TRY(S.get(&d_eigs, n_eig));
    ED_L_TRY(cudaMemsetAsync(beta, 0, (mmax + 2) * sizeof(double), st));

    int matvecs = 0;
    MatvecTimer timer;
    auto timed_matvec = [&](const void *in, void *out, ed_dtype dt) -> cudaError_t {
        ++matvecs;
        cudaError_t e = timer.mark(st);
        if (e == cudaSuccess)
            e = push ? launch_matvec_push(ov, gv, iv, track, in, out, dt, st)
                     : launch_matvec_v(ov, gv, iv, track, in, out, 1, dt, tuned_variant(b, 1, dt), st);
        if (e == cudaSuccess)
            e = timer.mark(st);
        return e;
    };
    auto H64 = [&](const D *in, D *out) -> cudaError_t { return timed_matvec(in, out, dt64); };

    // One Lanczos run of m steps from `start` (unnormalised), fp64 or fp32 matvec.
    // If Vs != nullptr, v_j is stored at Vs + j n; otherwise the ring buffers
    // are used and, if acc_y != nullptr, psi += acc_y[j] v_j is accumulated.
    auto run = [&](const D *start, int m, bool use_f32, D *Vs, const double *acc_y) -> cudaError_t {
        cudaError_t e;
        D *v0 = Vs ? Vs : ring[0];
        k_norm_part<kC><<<nparts, kRedThreads, 0, st>>>(start, n, part_a); count_launch();
        k_scale_by_norm<kC><<<vgrid, kRedThreads, 0, st>>>(start, v0, use_f32 ? x32 : nullptr, n, part_a, nparts); count_launch();
        D *vp = nullptr, *v = v0;
        for (int j = 0; j < m; ++j) {
            if (acc_y) {
                k_axpy_coef<kC><<<vgrid, kRedThreads, 0, st>>>(psi, v, acc_y, j, n, j == 0); count_launch();
            }
            if (use_f32) {
                e = timed_matvec(x32, w32, dt32);
                if (e != cudaSuccess)
                    return e;
                k_dot_part<kC, true><<<nparts, kRedThreads, 0, st>>>(v, w32, n, part_a, tickets, alpha + j); count_launch();
                k_update<kC, true><<<nparts, kRedThreads, 0, st>>>(w32, w, v, vp, n, alpha + j, beta + j, part_b,
                                                                    tickets + 1, beta + j + 1); count_launch();
            } else {
                if ((e = H64(v, w)) != cudaSuccess)
                    return e;
                k_dot_part<kC, false><<<nparts, kRedThreads, 0, st>>>(v, w, n, part_a, tickets, alpha + j); count_launch();
                k_update<kC, false><<<nparts, kRedThreads, 0, st>>>(w, w, v, vp, n, alpha + j, beta + j, part_b,
                                                                     tickets + 1, beta + j + 1); count_launch();
            }
            if (reorth && Vs) {  // against v_0 .. v_j, twice
                for (int pass = 0; pass < 2; ++pass) {
                    k_reorth_dot<kC><<<nparts, kRedThreads, 0, st>>>(Vs, w, n, j + 1, rpart); count_launch();
                    k_reorth_coef<<<j + 1, kRedThreads, 0, st>>>(rpart, nparts, rcoef); count_launch();
                    k_reorth_update<kC><<<nparts, kRedThreads, 0, st>>>(Vs, w, n, j + 1, rcoef, part_b); count_launch();
                }
                k_norm_final<<<1, kRedThreads, 0, st>>>(part_b, nparts, beta + j + 1); count_launch();
            }
            D *vn = Vs ? Vs + (uint64_t)(j + 1) * n : (vp ? vp : ring[1]);
            k_normalize<kC><<<vgrid, kRedThreads, 0, st>>>(w, vn, use_f32 ? x32 : nullptr, n, beta + j + 1); count_launch();
            vp = v;
            v = vn;
        }
        return cudaGetLastError();
    };

    // The same m steps as run(), for launch-bound sectors: step 0 eagerly, then
    // a CUDA graph of two steps (v, vp alternate between the ring buffers with
    // period two; alpha, beta and the store slot are indexed by the step index
    // on the device) replayed, and an odd last step eagerly.  Same kernels in
    // the same order, so the results equal run()'s bit for bit; products
    // inside the graph are not timed one by one.
    auto run_g = [&](const D *start, int m, bool use_f32, D *Vs, const double *acc_y) -> cudaError_t {
        cudaError_t e;
        k_norm_part<kC><<<nparts, kRedThreads, 0, st>>>(start, n, part_a); count_launch();
        k_scale_by_norm<kC><<<vgrid, kRedThreads, 0, st>>>(start, ring[0], use_f32 ? x32 : nullptr, n, part_a, nparts); count_launch();
        if (Vs && (e = cudaMemcpyAsync(Vs, ring[0], vec_bytes, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        k_step_set<<<1, 1, 0, st>>>(jdev, 0); count_launch();
        auto step = [&](const D *v, const D *vp, D *vn, cudaStream_t s) -> cudaError_t {
            if (acc_y) {
                k_axpy_coef<kC><<<vgrid, kRedThreads, 0, s>>>(psi, v, acc_y, 0, n, 0, jdev); count_launch();
            }
            cudaError_t e2;
            if (use_f32) {
                if ((e2 = launch_matvec_v(ov, gv, iv, track, x32, w32, 1, dt32, tuned_variant(b, 1, dt32), s)) !=
                    cudaSuccess)
                    return e2;
                k_dot_part<kC, true><<<nparts, kRedThreads, 0, s>>>(v, w32, n, part_a, tickets, alpha, jdev); count_launch();
                k_update<kC, true><<<nparts, kRedThreads, 0, s>>>(w32, w, v, vp, n, alpha, beta, part_b,
                                                                   tickets + 1, beta + 1, jdev); count_launch();
            } else {
                if ((e2 = launch_matvec_v(ov, gv, iv, track, v, w, 1, dt64, tuned_variant(b, 1, dt64), s)) !=
                    cudaSuccess)
                    return e2;
                k_dot_part<kC, false><<<nparts, kRedThreads, 0, s>>>(v, w, n, part_a, tickets, alpha, jdev); count_launch();
                k_update<kC, false><<<nparts, kRedThreads, 0, s>>>(w, w, v, vp, n, alpha, beta, part_b,
                                                                    tickets + 1, beta + 1, jdev); count_launch();
            }
            k_normalize<kC><<<vgrid, kRedThreads, 0, s>>>(w, vn, use_f32 ? x32 : nullptr, n, beta + 1, jdev, Vs); count_launch();
            k_step_inc<<<1, 1, 0, s>>>(jdev); count_launch();
            return cudaGetLastError();
        };
        if ((e = step(ring[0], nullptr, ring[1], st)) != cudaSuccess)
            return e;
        ++matvecs;
        int done = 1;
        if (m - done >= 2) {
            if (!GR.cap && (e = cudaStreamCreateWithFlags(&GR.cap, cudaStreamNonBlocking)) != cudaSuccess)
                return e;
            const unsigned long long c0 = launches_so_far();
            if ((e = cudaStreamBeginCapture(GR.cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess)
                return e;
            e = step(ring[1], ring[0], ring[0], GR.cap);
            if (e == cudaSuccess)
                e = step(ring[0], ring[1], ring[1], GR.cap);
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(GR.cap, &g);
            if (g)
                GR.graphs.push_back(g);
            if (e != cudaSuccess || e2 != cudaSuccess)
                return e != cudaSuccess ? e : e2;
            const unsigned per_graph = (unsigned)(launches_so_far() - c0);
            uncount_launch(per_graph);  // captured, not yet run
            cudaGraphExec_t ge = nullptr;
            if ((e = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess)
                return e;
            GR.execs.push_back(ge);
            for (; m - done >= 2; done += 2) {
                if ((e = cudaGraphLaunch(ge, st)) != cudaSuccess)
                    return e;
                count_launch(per_graph);
                matvecs += 2;
            }
        }
        if (done < m) {  // odd remainder: v in ring[1]
            if ((e = step(ring[1], ring[0], ring[0], st)) != cudaSuccess)
                return e;
            ++matvecs;
        }
        return cudaGetLastError();
    };
    auto run_any = [&](const D *start, int m, bool use_f32, D *Vs, const double *acc_y) -> cudaError_t {
        return graph ? run_g(start, m, use_f32, Vs, acc_y) : run(start, m, use_f32, Vs, acc_y);
    };

    // main pass
    ED_L_TRY(run_any((const D *)x0, steps, f32, store ? V : nullptr, nullptr));
    ED_L_TRY(cudaMemsetAsync(y, 0, (mmax + 1) * sizeof(double), st));
    k_tridiag_lowest<<<1, 32, 0, st>>>(alpha, beta, steps, y, scal + 0, m_eff, work); count_launch();
    if (n_eig > 0) {
        k_tridiag_kth<<<n_eig, 32, 0, st>>>(alpha, beta, steps, m_eff, d_eigs); count_launch();
    }
    if (values_only) {
        // lowest Ritz value; residual estimate |beta_{m+1} y_m| of the recurrence
        double ritz = 0.0;
        int me = 0;
        ED_L_TRY(cudaMemcpyAsync(&ritz, scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
        ED_L_TRY(cudaMemcpyAsync(&me, m_eff, sizeof(int), cudaMemcpyDeviceToHost, st));
        ED_L_TRY(cudaStreamSynchronize(st));
        double bl = 0.0, yl = 0.0;
        if (me > 0) {
            ED_L_TRY(cudaMemcpy(&bl, beta + me, sizeof(double), cudaMemcpyDeviceToHost));
            ED_L_TRY(cudaMemcpy(&yl, y + me - 1, sizeof(double), cudaMemcpyDeviceToHost));
        }
        if (n_eig > 0 && eigs_out)
            ED_L_TRY(cudaMemcpy(eigs_out, d_eigs, n_eig * sizeof(double), cudaMemcpyDeviceToHost));
        if (e0_out)
            *e0_out = ritz;
        if (info) {
            info->steps = me;
            info->matvecs = matvecs;
            info->ritz = ritz;
            info->e0 = ritz;
            info->residual = fabs(bl * yl);
            info->matvec_ms = timer.total_ms();
        }
        return ED_OK;
    }
    if (store) {
        k_combine<kC><<<vgrid, kRedThreads, 0, st>>>(psi, V, y, m_eff, n); count_launch();
    } else {
        ED_L_TRY(run_any((const D *)x0, steps, f32, nullptr, y));  // bit-identical second pass
    }
    ED_L_TRY(cudaGetLastError());
    double ritz = 0.0;
    int me = 0;
    ED_L_TRY(cudaMemcpyAsync(&ritz, scal + 0, sizeof(double), cudaMemcpyDeviceToHost, st));
    ED_L_TRY(cudaMemcpyAsync(&me, m_eff, sizeof(int), cudaMemcpyDeviceToHost, st));

    // fp64 refinement from the fp32-matvec Ritz vector: a short fp64 Lanczos run
    D *u = psi;
    if (f32) {
        // its mref + 1 vectors go into the main pass's Krylov store (no longer
        // needed once psi is formed) or a new one if that fits in half of the
        // free memory; else the Ritz vector comes from a second pass that
        // starts from psi and accumulates into it (psi is read only before
        // the first accumulation)
        D *Vr = nullptr;
        if (store && steps >= mref) {
            Vr = V;
        } else if (!recompute) {
            cudaMemGetInfo(&free_b, &total_b);
            free_b += ws_cached_bytes();
            if ((double)(mref + 1) * vec_bytes < 0.5 * (double)free_b)
                ED_L_TRY(S.get(&Vr, (size_t)(mref + 1) * n));
        }
        const bool store_r = Vr != nullptr;
        if (!store_r && !ring[0]) {
            ED_L_TRY(S.get(&ring[0], n));
            ED_L_TRY(S.get(&ring[1], n));
        }
        ED_L_TRY(cudaMemsetAsync(beta, 0, (mmax + 2) * sizeof(double), st));
        ED_L_TRY(run_any(psi, mref, false, Vr, nullptr));
        ED_L_TRY(cudaMemsetAsync(y, 0, (mmax + 1) * sizeof(double), st));
        k_tridiag_lowest<<<1, 32, 0, st>>>(alpha, beta, mref, y, scal + 1, m_eff, work); count_launch();
        if (store_r) {
            k_combine<kC><<<vgrid, kRedThreads, 0, st>>>(psi, Vr, y, m_eff, n); count_launch();
        } else {
            ED_L_TRY(run_any(psi, mref, false, nullptr, y));
        }
        ED_L_TRY(cudaGetLastError());
    }
    // fp64 Rayleigh quotient and residual of the final vector u
    ED_L_TRY(H64(u, w));
    k_dot_part<kC, false><<<nparts, kRedThreads, 0, st>>>(u, w, n, part_a, nullptr, nullptr); count_launch();
    k_norm_part<kC><<<nparts, kRedThreads, 0, st>>>(u, n, part_b); count_launch();
    k_residual<kC><<<nparts, kRedThreads, 0, st>>>(w, u, n, part_a, part_b, nparts, scal + 2, part_c); count_launch();
    k_finish_residual<<<1, kRedThreads, 0, st>>>(part_c, part_b, nparts, scal + 3); count_launch();
    if (vec_out)
        k_scale_by_norm<kC><<<vgrid, kRedThreads, 0, st>>>(u, (D *)vec_out, nullptr, n, part_b, nparts); count_launch();
    ED_L_TRY(cudaGetLastError());
    double res[2] = {0.0, 0.0};
    ED_L_TRY(cudaMemcpyAsync(res, scal + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (n_eig > 0 && eigs_out)
        ED_L_TRY(cudaMemcpyAsync(eigs_out, d_eigs, n_eig * sizeof(double), cudaMemcpyDeviceToHost, st));
    ED_L_TRY(cudaStreamSynchronize(st));
    if (e0_out)
        *e0_out = res[0];
    if (info) {
        info->steps = me;
        info->matvecs = matvecs;
        info->ritz = ritz;
        info->e0 = res[0];
        info->residual = res[1];
        info->matvec_ms = timer.total_ms();
    }
    return ED_OK;
}

}  // namespace
}  // namespace edk

namespace {
ed_status lanczos_entry(const ed_operator *op, const ed_basis *b, const void *x0, int steps, int mode_flags,
                        int n_eig, double *eigs_out, double tol, double *e0_out, void *vec_out,
                        ed_lanczos_info *info, void *stream)
{
    if (!op || !b || steps < 1 || steps > 10000)
        return ED_ERR_INVALID_ARG;
    const int base = mode_flags & ~(ED_LANCZOS_RECOMPUTE | ED_LANCZOS_PUSH | ED_LANCZOS_REORTH |
                                    ED_LANCZOS_VALUES_ONLY);
    if (base != ED_LANCZOS_F64 && base != ED_LANCZOS_F32_MATVEC)
        return ED_ERR_INVALID_ARG;
    if (n_eig < 0 || n_eig > steps || (n_eig > 0 && !eigs_out))
        return ED_ERR_INVALID_ARG;
    const ed_lanczos_mode mode = (ed_lanczos_mode)base;
    const bool recompute = (mode_flags & ED_LANCZOS_RECOMPUTE) != 0;
    const bool push = (mode_flags & ED_LANCZOS_PUSH) != 0;
    const bool reorth = (mode_flags & ED_LANCZOS_REORTH) != 0;
    const bool values_only = (mode_flags & ED_LANCZOS_VALUES_ONLY) != 0;
    if (values_only && vec_out)
        return ED_ERR_INVALID_ARG;
    if (b->dim == 0 || !x0)
        return ED_ERR_INVALID_ARG;
    if (((uintptr_t)x0 | (uintptr_t)vec_out) & 15)
        return ED_ERR_INVALID_ARG;
    const ed_status st = edk::check_pair(op, b);
    if (st != ED_OK)
        return st;
    const bool cplx = !(b->real_chars && op->real);
    ed_lanczos_info local{};
    ed_lanczos_info *inf = info ? info : &local;
    const ed_status r = cplx ? edk::run_lanczos<true>(op, b, x0, steps, mode, recompute, push, reorth, values_only, n_eig,
                                                      eigs_out, e0_out, vec_out, inf, (cudaStream_t)stream)
                             : edk::run_lanczos<false>(op, b, x0, steps, mode, recompute, push, reorth, values_only, n_eig,
                                                       eigs_out, e0_out, vec_out, inf, (cudaStream_t)stream);
    if (r == ED_OK && tol > 0.0 && !(inf->residual <= tol))
        return ED_ERR_NOT_CONVERGED;
    return r;
}
}  // namespace

// Test hook: steps replayed from a CUDA graph (-1 automatic, 0 never, 1
// always); returns the previous policy.
extern "C" int edx_lanczos_graph(int policy)
{
    const int old = edk::g_lanczos_graph;
    edk::g_lanczos_graph = policy < 0 ? -1 : (policy ? 1 : 0);
    return old;
}

extern "C" ed_status ed_lanczos(const ed_operator *op, const ed_basis *b, const void *x0, int steps,
                                int mode_flags, double *e0_out, void *vec_out,
                                ed_lanczos_info *info, void *stream)
{
    return lanczos_entry(op, b, x0, steps, mode_flags, 0, nullptr, 0.0, e0_out, vec_out, info, stream);
}

extern "C" ed_status ed_lanczos_eigs(const ed_operator *op, const ed_basis *b, const void *x0, int steps,
                                     int mode_flags, int n_eig, double *eigs_out, double tol, void *vec_out,
                                     ed_lanczos_info *info, void *stream)
{
    return lanczos_entry(op, b, x0, steps, mode_flags, n_eig, eigs_out, tol, nullptr, vec_out, info, stream);
}
