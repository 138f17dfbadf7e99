// ed_lanczos_multi.cu -- the Lanczos recurrence of ed_lanczos run in a batch
// of symmetry sectors at once (lowest energy of each), every matvec being one
// persistent multi-sector launch, and the steps replayed from a CUDA graph.
//
// The sectors' vectors are concatenated.  Reductions are segmented: each block
// of the vector kernels lies inside one sector, and a finalize with one block
// per sector merges that sector's block partials (compensated fp64 sums, as in
// the single-sector solver).  The step index lives on the device and is
// advanced by the last kernel of a step, so the graph of two consecutive steps
// (the Lanczos vectors alternate between two buffers) serves every step of a
// run.  The Ritz vector of each sector is formed from the stored Lanczos
// vectors, or by a second, bit-identical pass when they do not fit; in the
// fp32-matvec mode it is then refined by a short fp64 run.  The energy returned
// per sector is the fp64 Rayleigh quotient of its final vector, with its fp64
// residual.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "ed_kernels.cuh"
#include "ed_matvec_multi_impl.cuh"

namespace edk {
namespace {

constexpr int kThr = 256;
constexpr int kPerThread = 16;  // vector elements per thread in the segmented kernels
constexpr int kRefine = 6;      // fp64 refinement steps (as ed_lanczos)

// ---- compensated sums ----------------------------------------------------------
struct KS {
    double s, c;
};
__device__ __forceinline__ KS two_sum_k(double a, double b)
{
    const double s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ KS merge_k(KS a, KS b)
{
    KS r = two_sum_k(a.s, b.s);
    r.c += a.c + b.c;
    return r;
}
// block-wide merge; the result is valid in thread 0
__device__ KS block_merge(KS k)
{
    __shared__ double ss[kThr / 32], cs[kThr / 32];
    for (int o = 16; o > 0; o >>= 1)
        k = merge_k(k, KS{__shfl_down_sync(0xffffffffu, k.s, o), __shfl_down_sync(0xffffffffu, k.c, o)});
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        ss[wid] = k.s;
        cs[wid] = k.c;
    }
    __syncthreads();
    if (wid == 0) {
        k = lane < kThr / 32 ? KS{ss[lane], cs[lane]} : KS{0.0, 0.0};
        for (int o = 16; o > 0; o >>= 1)
            k = merge_k(k, KS{__shfl_down_sync(0xffffffffu, k.s, o), __shfl_down_sync(0xffffffffu, k.c, o)});
    }
    return k;
}

// ---- segment layout ----------------------------------------------------------------
struct Seg {
    int stride;               // stride of the per-sector scalar arrays
    const int *blk_sec;       // sector of each block
    const uint64_t *blk_lo;   // first element of each block
    const uint64_t *blk_hi;   // end of each block
    const int *sec_blk;       // n_sec + 1: first block of each sector
};

// element types: fp64 vector D, fp32 matvec copy F
template <bool C> struct El { using D = double; using F = float; };
template <> struct El<true> { using D = double2; using F = float2; };

__device__ __forceinline__ double re_dot(double a, double b) { return a * b; }
__device__ __forceinline__ double re_dot(double2 a, double2 b) { return fma(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ double re_dot(double a, float b) { return a * (double)b; }
__device__ __forceinline__ double re_dot(double2 a, float2 b) { return fma(a.x, (double)b.x, a.y * (double)b.y); }
__device__ __forceinline__ double nrm2(double a) { return a * a; }
__device__ __forceinline__ double nrm2(double2 a) { return fma(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double up(float a) { return a; }
__device__ __forceinline__ double2 up(float2 a) { return make_double2(a.x, a.y); }
__device__ __forceinline__ double up(double a) { return a; }
__device__ __forceinline__ double2 up(double2 a) { return a; }
__device__ __forceinline__ float down(double a) { return (float)a; }
__device__ __forceinline__ float2 down(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double zero_of(double) { return 0.0; }
__device__ __forceinline__ double2 zero_of(double2) { return make_double2(0.0, 0.0); }
// w - a v - b p
__device__ __forceinline__ double axpby(double w, double a, double v, double b, double p)
{
    return fma(-b, p, fma(-a, v, w));
}
__device__ __forceinline__ double2 axpby(double2 w, double a, double2 v, double b, double2 p)
{
    return make_double2(fma(-b, p.x, fma(-a, v.x, w.x)), fma(-b, p.y, fma(-a, v.y, w.y)));
}
__device__ __forceinline__ double scale(double w, double s) { return w * s; }
__device__ __forceinline__ double2 scale(double2 w, double s) { return make_double2(w.x * s, w.y * s); }
__device__ __forceinline__ double fmac(double acc, double y, double v) { return fma(y, v, acc); }
__device__ __forceinline__ double2 fmac(double2 acc, double y, double2 v)
{
    return make_double2(fma(y, v.x, acc.x), fma(y, v.y, acc.y));
}

// part[b] = block b's partial of Re<a, bv> (of |a|^2 when bv is null)
template <bool C, typename B>
__global__ void __launch_bounds__(kThr) k_seg_dot(Seg sg, const typename El<C>::D *a, const B *bv, double2 *part)
{
    const uint64_t lo = sg.blk_lo[blockIdx.x], hi = sg.blk_hi[blockIdx.x];
    double s0 = 0.0, s1 = 0.0;
    int par = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThr) {
        const double t = bv ? re_dot(a[i], bv[i]) : nrm2(a[i]);
        if (par)
            s1 += t;
        else
            s0 += t;
        par ^= 1;
    }
    const KS k = block_merge(two_sum_k(s0, s1));
    if (threadIdx.x == 0)
        part[blockIdx.x] = make_double2(k.s, k.c);
}

// out[s * stride + (*step) + shift] = sum of sector s's partials (its square
// root if root); one block per sector; step may be null (index 0)
__global__ void __launch_bounds__(kThr) k_seg_final(Seg sg, const double2 *part, double *out, const int *step,
                                                    int shift, int root)
{
    const int s = blockIdx.x;
    KS k{0.0, 0.0};
    for (int b = sg.sec_blk[s] + threadIdx.x; b < sg.sec_blk[s + 1]; b += kThr)
        k = merge_k(k, KS{part[b].x, part[b].y});
    k = block_merge(k);
    if (threadIdx.x == 0) {
        const double t = k.s + k.c;
        out[(size_t)s * sg.stride + (step ? *step : 0) + shift] = root ? sqrt(fmax(t, 0.0)) : t;
    }
}

// w = w_in - alpha_j v - beta_j vp (vp null: first step); partials of |w|^2
template <bool C, typename WI>
__global__ void __launch_bounds__(kThr) k_seg_update(Seg sg, const WI *w_in, typename El<C>::D *w,
                                                     const typename El<C>::D *v, const typename El<C>::D *vp,
                                                     const double *alpha, const double *beta, const int *step,
                                                     double2 *part)
{
    const int s = sg.blk_sec[blockIdx.x];
    const int j = *step;
    const double a = alpha[(size_t)s * sg.stride + j];
    const double b = beta[(size_t)s * sg.stride + j];
    const uint64_t lo = sg.blk_lo[blockIdx.x], hi = sg.blk_hi[blockIdx.x];
    double s0 = 0.0, s1 = 0.0;
    int par = 0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThr) {
        const typename El<C>::D vi = v[i];
        const typename El<C>::D r = axpby(up(w_in[i]), a, vi, b, vp ? vp[i] : zero_of(vi));
        w[i] = r;
        if (par)
            s1 += nrm2(r);
        else
            s0 += nrm2(r);
        par ^= 1;
    }
    const KS k = block_merge(two_sum_k(s0, s1));
    if (threadIdx.x == 0)
        part[blockIdx.x] = make_double2(k.s, k.c);
}

// Stored Lanczos vectors: vector q at base + q * total, fp32 or fp64; only
// q < count are kept.
struct Store {
    void *base;
    int f32;
    int count;
    uint64_t total;
};

// out = in / nrm[s * stride + q] with q = (*step) + shift (step may be null:
// q = shift), zero if that norm is 0; an fp32 copy if x32; a copy into stored
// vector q if st.base
template <bool C>
__global__ void __launch_bounds__(kThr) k_seg_scale(Seg sg, const typename El<C>::D *in, typename El<C>::D *out,
                                                    typename El<C>::F *x32, const double *nrm, const int *step,
                                                    int shift, Store st)
{
    const int s = sg.blk_sec[blockIdx.x];
    const int q = (step ? *step : 0) + shift;
    const double n = nrm[(size_t)s * sg.stride + q];
    const double sc = n > 0.0 ? 1.0 / n : 0.0;
    const bool keep = st.base && q < st.count;
    typename El<C>::D *v64 = keep && !st.f32 ? (typename El<C>::D *)st.base + (uint64_t)q * st.total : nullptr;
    typename El<C>::F *v32 = keep && st.f32 ? (typename El<C>::F *)st.base + (uint64_t)q * st.total : nullptr;
    const uint64_t lo = sg.blk_lo[blockIdx.x], hi = sg.blk_hi[blockIdx.x];
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThr) {
        const typename El<C>::D r = scale(in[i], sc);
        out[i] = r;
        if (x32)
            x32[i] = down(r);
        if (v64)
            v64[i] = r;
        if (v32)
            v32[i] = down(r);
    }
}

// psi = sum_{q < m} y[s * stride + q] v_q over the stored vectors
template <bool C>
__global__ void __launch_bounds__(kThr) k_seg_combine(Seg sg, typename El<C>::D *psi, Store st, const double *y,
                                                      int m)
{
    const int s = sg.blk_sec[blockIdx.x];
    const double *ys = y + (size_t)s * sg.stride;
    const uint64_t lo = sg.blk_lo[blockIdx.x], hi = sg.blk_hi[blockIdx.x];
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThr) {
        typename El<C>::D acc = zero_of(typename El<C>::D{});
        for (int q = 0; q < m; ++q) {
            const double c = ys[q];
            if (c == 0.0)
                continue;
            const uint64_t e = (uint64_t)q * st.total + i;
            acc = fmac(acc, c, st.f32 ? up(((const typename El<C>::F *)st.base)[e])
                                      : ((const typename El<C>::D *)st.base)[e]);
        }
        psi[i] = acc;
    }
}

// psi += y_j v_j (psi = y_0 v_0 at j = 0)
template <bool C>
__global__ void __launch_bounds__(kThr) k_seg_accum(Seg sg, typename El<C>::D *psi, const typename El<C>::D *v,
                                                    const double *y, const int *step)
{
    const int s = sg.blk_sec[blockIdx.x];
    const int j = *step;
    const double c = y[(size_t)s * sg.stride + j];
    const uint64_t lo = sg.blk_lo[blockIdx.x], hi = sg.blk_hi[blockIdx.x];
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThr) {
        const typename El<C>::D vi = v[i];
        psi[i] = fmac(j == 0 ? zero_of(vi) : psi[i], c, vi);
    }
}

// partials of |Hu - theta u|^2 with theta = num_s / den_s
template <bool C>
__global__ void __launch_bounds__(kThr) k_seg_resid(Seg sg, const typename El<C>::D *hu, const typename El<C>::D *u,
                                                    const double *num, const double *den, double2 *part)
{
    const int s = sg.blk_sec[blockIdx.x];
    const double th = num[(size_t)s * sg.stride] / den[(size_t)s * sg.stride];
    const uint64_t lo = sg.blk_lo[blockIdx.x], hi = sg.blk_hi[blockIdx.x];
    double s0 = 0.0;
    for (uint64_t i = lo + threadIdx.x; i < hi; i += kThr) {
        const typename El<C>::D ui = u[i];
        s0 += nrm2(axpby(hu[i], th, ui, 0.0, ui));
    }
    const KS k = block_merge(KS{s0, 0.0});
    if (threadIdx.x == 0)
        part[blockIdx.x] = make_double2(k.s, k.c);
}

__global__ void k_step_set(int *step, int v) { *step = v; }
__global__ void k_step_inc(int *step) { *step += 1; }

// Sturm count: eigenvalues below x of the m x m tridiagonal (a, b)
__device__ int sturm_cnt(const double *a, const double *b, int m, double x)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        d = (a[i] - x) - (i ? b[i] * b[i] / d : 0.0);
        if (d == 0.0)
            d = -1e-300;
        cnt += d < 0.0;
    }
    return cnt;
}

// One warp per sector: lowest eigenvalue of the sector's tridiagonal matrix
// (32-point multisection of the Gershgorin interval with Sturm counts) and its
// eigenvector (inverse iteration), cut at the first vanishing beta.
__global__ void k_seg_tridiag(const double *alpha, const double *beta, int stride, int m, double *y,
                              double *lam_out, int *m_eff, double *work)
{
    const int s = blockIdx.x;
    const int lane = threadIdx.x & 31;
    const double *a = alpha + (size_t)s * stride;
    const double *b = beta + (size_t)s * stride;
    double *ys = y + (size_t)s * stride;
    double *dd = work + (size_t)s * stride;
    int me = m;
    double scl = 0.0, lo = 1e300, hi = -1e300;
    if (lane == 0) {
        for (int i = 0; i < m; ++i)
            scl = fmax(scl, fabs(a[i]) + fabs(b[i + 1]));
        for (int i = 1; i < m; ++i)
            if (!(b[i] > 1e-13 * fmax(scl, 1e-300))) {
                me = i;
                break;
            }
        for (int i = 0; i < me; ++i) {
            const double r = (i ? fabs(b[i]) : 0.0) + (i + 1 < me ? fabs(b[i + 1]) : 0.0);
            lo = fmin(lo, a[i] - r);
            hi = fmax(hi, a[i] + r);
        }
    }
    me = __shfl_sync(0xffffffffu, me, 0);
    scl = __shfl_sync(0xffffffffu, scl, 0);
    lo = __shfl_sync(0xffffffffu, lo, 0);
    hi = __shfl_sync(0xffffffffu, hi, 0);
    for (int it = 0; it < 24; ++it) {
        const double wd = hi - lo;
        if (!(wd > 2e-16 * fmax(fabs(lo), fabs(hi))))
            break;
        const double x = lo + wd * (double)(lane + 1) / 33.0;
        const unsigned below = __ballot_sync(0xffffffffu, sturm_cnt(a, b, me, x) >= 1);
        const int f = below ? __ffs(below) - 1 : 32;
        const double nlo = f == 0 ? lo : lo + wd * (double)f / 33.0;
        const double nhi = f == 32 ? hi : lo + wd * (double)(f + 1) / 33.0;
        lo = nlo;
        hi = nhi;
    }
    if (lane != 0)
        return;
    const double lam = 0.5 * (lo + hi);
    const double eps = 1e-15 * fmax(scl, 1e-300);
    for (int i = 0; i < me; ++i)
        ys[i] = 1.0;
    for (int iter = 0; iter < 4; ++iter) {
        double piv = a[0] - lam;
        if (fabs(piv) < eps)
            piv = eps;
        dd[0] = piv;
        for (int i = 1; i < me; ++i) {
            const double l = b[i] / dd[i - 1];
            piv = (a[i] - lam) - l * b[i];
            if (fabs(piv) < eps)
                piv = eps;
            dd[i] = piv;
            ys[i] -= l * ys[i - 1];
        }
        ys[me - 1] /= dd[me - 1];
        for (int i = me - 2; i >= 0; --i)
            ys[i] = (ys[i] - b[i + 1] * ys[i + 1]) / dd[i];
        double nrm = 0.0;
        for (int i = 0; i < me; ++i)
            nrm += ys[i] * ys[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < me; ++i)
            ys[i] /= nrm;
    }
    for (int i = me; i < m; ++i)
        ys[i] = 0.0;
    lam_out[(size_t)s * stride] = lam;
    m_eff[s] = me;
}

// device buffers, graphs and the capture stream, released on every exit path
struct Owned {
    cudaStream_t st;  // the call's stream: work arrays are allocated and freed in its order
    std::vector<void *> ptrs;
    std::vector<cudaGraphExec_t> execs;
    std::vector<cudaGraph_t> graphs;
    cudaStream_t cap = nullptr;
    explicit Owned(cudaStream_t s) : st(s) {}
    ~Owned()
    {
        for (auto g : execs)
            cudaGraphExecDestroy(g);
        for (auto g : graphs)
            cudaGraphDestroy(g);
        for (void *p : ptrs)
            ws_free(p, st);
        if (cap)
            cudaStreamDestroy(cap);
    }
    template <typename T>
    cudaError_t get(T **p, size_t n)
    {
        const cudaError_t e = ws_alloc((void **)p, std::max<size_t>(n, 1) * sizeof(T), st);
        if (e == cudaSuccess)
            ptrs.push_back((void *)*p);
        return e;
    }
};

#define LM_TRY(expr)                                                        \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) {                                            \
            (void)cudaGetLastError();                                       \
            return _e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA; \
        }                                                                   \
    } while (0)
#define LM_CHK(expr)                        \
    do {                                    \
        cudaError_t _e = (expr);            \
        if (_e != cudaSuccess)              \
            return _e;                      \
    } while (0)

MultiArgs g_margs;  // host staging of the matvec launch arguments (copied at each launch)

template <bool C>
ed_status run_multi(const ed_operator *op, const ed_sector *sectors, int ns, int steps, bool f32,
                    bool recompute, double *e0_out, ed_lanczos_info *info, cudaStream_t st)
{
    using D = typename El<C>::D;
    using F = typename El<C>::F;
    Owned O(st);
    std::vector<uint64_t> off(ns + 1, 0);
    for (int k = 0; k < ns; ++k)
        off[k + 1] = off[k] + sectors[k].basis->dim;
    const uint64_t total = off[ns];
    // segment blocks: at most kThr * kPerThread elements of one sector each
    std::vector<int> blk_sec, sec_blk(ns + 1, 0);
    std::vector<uint64_t> blk_lo, blk_hi;
    for (int k = 0; k < ns; ++k) {
        sec_blk[k] = (int)blk_sec.size();
        for (uint64_t lo = off[k]; lo < off[k + 1]; lo += (uint64_t)kThr * kPerThread) {
            blk_sec.push_back(k);
            blk_lo.push_back(lo);
            blk_hi.push_back(std::min<uint64_t>(off[k + 1], lo + (uint64_t)kThr * kPerThread));
        }
    }
    sec_blk[ns] = (int)blk_sec.size();
    const unsigned nblk = (unsigned)blk_sec.size();
    const int stride = std::max(steps, kRefine) + 2;
    const size_t sc = (size_t)ns * stride;

    Seg sg;
    sg.stride = stride;
    {
        uint64_t *p_lo, *p_hi;
        int *p_bs, *p_sb;
        LM_TRY(O.get(&p_lo, nblk));
        LM_TRY(O.get(&p_hi, nblk));
        LM_TRY(O.get(&p_bs, nblk));
        LM_TRY(O.get(&p_sb, ns + 1));
        LM_TRY(cudaMemcpyAsync(p_lo, blk_lo.data(), nblk * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        LM_TRY(cudaMemcpyAsync(p_hi, blk_hi.data(), nblk * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
        LM_TRY(cudaMemcpyAsync(p_bs, blk_sec.data(), nblk * sizeof(int), cudaMemcpyHostToDevice, st));
        LM_TRY(cudaMemcpyAsync(p_sb, sec_blk.data(), (ns + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
        sg.blk_lo = p_lo;
        sg.blk_hi = p_hi;
        sg.blk_sec = p_bs;
        sg.sec_blk = p_sb;
    }
    D *x0, *ring0, *ring1, *w, *psi;
    F *x32 = nullptr, *w32 = nullptr;
    double *alpha, *beta, *y, *work, *lam, *nrm, *num, *den, *res;
    int *m_eff, *step;
    double2 *part;
    LM_TRY(O.get(&x0, total));
    LM_TRY(O.get(&ring0, total));
    LM_TRY(O.get(&ring1, total));
    LM_TRY(O.get(&w, total));
    LM_TRY(O.get(&psi, total));
    if (f32) {
        LM_TRY(O.get(&x32, total));
        LM_TRY(O.get(&w32, total));
    }
    for (double **p : {&alpha, &beta, &y, &work, &lam, &nrm, &num, &den, &res})
        LM_TRY(O.get(p, sc));
    LM_TRY(O.get(&m_eff, ns));
    LM_TRY(O.get(&step, 1));
    LM_TRY(O.get(&part, nblk));
    LM_TRY(cudaStreamCreateWithFlags(&O.cap, cudaStreamNonBlocking));
    for (int k = 0; k < ns; ++k)
        LM_TRY(cudaMemcpyAsync(x0 + off[k], sectors[k].d_x, (off[k + 1] - off[k]) * sizeof(D),
                               cudaMemcpyDeviceToDevice, st));

    // Lanczos vectors are kept (and the Ritz vector formed from them) when
    // they fit in half of the free memory, else the Ritz vector comes from a
    // second, bit-identical pass.  The fp32-matvec mode keeps the fp32 copies
    // the matvec consumed: its Ritz vector only starts the fp64 refinement.
    size_t free_b = 0, total_b = 0;
    LM_TRY(cudaMemGetInfo(&free_b, &total_b));
    const size_t main_bytes = (size_t)steps * total * (f32 ? sizeof(F) : sizeof(D));
    const size_t ref_bytes = (size_t)kRefine * total * sizeof(D);
    Store main_st{nullptr, f32 ? 1 : 0, steps, total}, ref_st{nullptr, 0, kRefine, total};
    if (!recompute && (double)main_bytes < 0.5 * (double)free_b) {
        if (f32) {
            F *p;
            LM_TRY(O.get(&p, (size_t)steps * total));
            main_st.base = p;
        } else {
            D *p;
            LM_TRY(O.get(&p, (size_t)steps * total));
            main_st.base = p;
        }
        free_b -= main_bytes;
    }
    if (f32 && !recompute && (double)ref_bytes < 0.5 * (double)free_b) {
        D *p;
        LM_TRY(O.get(&p, (size_t)kRefine * total));
        ref_st.base = p;
    }

    // The products: one multi-sector launch fed by the device work queue (one
    // ed_matvec launch per sector only under the per-sector test policy, for
    // sectors that each fill the GPU).
    int dev = 0, sms = 0;
    LM_TRY(cudaGetDevice(&dev));
    LM_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint64_t min_dim = ~0ull;
    for (int k = 0; k < ns; ++k)
        min_dim = std::min<uint64_t>(min_dim, sectors[k].basis->dim);
    const bool per_sector = multi_policy_get() == 2 && min_dim >= (uint64_t)sms * 2048;
    const OpView ov = make_op_view(op);
    const ed_basis *b0 = sectors[0].basis;
    bool track = false;
    int max_order = 0;
    for (int k = 0; k < ns; ++k) {
        track = track || !sectors[k].basis->trivial_chars;
        max_order = std::max(max_order, sectors[k].basis->order);
    }
    auto matvec = [&](const void *xin, void *yout, bool single, cudaStream_t s) -> cudaError_t {
        const size_t esize = single ? sizeof(F) : sizeof(D);
        if (per_sector) {
            const ed_dtype dt = single ? (C ? ED_C64 : ED_F32) : (C ? ED_C128 : ED_F64);
            for (int k = 0; k < ns; ++k) {
                const ed_basis *b = sectors[k].basis;
                LM_CHK(launch_matvec(ov, b->group_view(), b->index_view(), !b->trivial_chars,
                                     (const char *)xin + off[k] * esize, (char *)yout + off[k] * esize, 1,
                                     dt, s));
            }
            return cudaSuccess;
        }
        MultiArgs &a = g_margs;
        a.op = ov;
        a.g = b0->group_view();
        a.g.flip = 0;  // spin inversion is per sector
        a.nvec = 1;
        a.max_order = max_order;
        a.n_sectors = ns;
        uint64_t tiles = 0;
        for (int k = 0; k < ns; ++k) {
            const ed_basis *b = sectors[k].basis;
            const GroupView gv = b->group_view();
            const IndexView iv = b->index_view();
            SectorDesc &d = a.sec[k];
            d.keys = iv.keys;
            d.states = iv.states;
            d.norms = iv.norms;
            sector_index_from(d, b);
            d.chi = gv.fact ? gv.fchi : gv.chi;
            d.chif = gv.fact ? gv.fchif : gv.chif;
            d.x = (const char *)xin + off[k] * esize;
            d.y = (char *)yout + off[k] * esize;
            d.dim = b->dim;
            d.tile_begin = tiles;
            d.flip = b->spin_inversion != 0;
            tiles += (b->dim + 31) / 32;
        }
        a.total_tiles = tiles;
        const cudaError_t ce = batch_ctl(s, &a.ctl);  // first used in the eager step 0, before any capture
        if (ce != cudaSuccess)
            return ce;
        return multi_launch_any(a, track, single ? (C ? ED_C64 : ED_F32) : (C ? ED_C128 : ED_F64), s);
    };

    // Lanczos step j (j on the device): w = H v - alpha_j v - beta_j vp,
    // beta_{j+1} = |w|, vn = w / beta_{j+1} (kept as vector j + 1 if stored);
    // with acc, psi += y_j v first
    auto step_body = [&](D *v, D *vp, D *vn, bool single, bool acc, Store keep,
                         cudaStream_t s) -> cudaError_t {
        if (acc) {
            k_seg_accum<C><<<nblk, kThr, 0, s>>>(sg, psi, v, y, step); count_launch();
        }
        if (single) {
            LM_CHK(matvec(x32, w32, true, s));
            k_seg_dot<C, F><<<nblk, kThr, 0, s>>>(sg, v, w32, part); count_launch();
            k_seg_final<<<ns, kThr, 0, s>>>(sg, part, alpha, step, 0, 0); count_launch();
            k_seg_update<C, F><<<nblk, kThr, 0, s>>>(sg, w32, w, v, vp, alpha, beta, step, part); count_launch();
        } else {
            LM_CHK(matvec(v, w, false, s));
            k_seg_dot<C, D><<<nblk, kThr, 0, s>>>(sg, v, w, part); count_launch();
            k_seg_final<<<ns, kThr, 0, s>>>(sg, part, alpha, step, 0, 0); count_launch();
            k_seg_update<C, D><<<nblk, kThr, 0, s>>>(sg, w, w, v, vp, alpha, beta, step, part); count_launch();
        }
        k_seg_final<<<ns, kThr, 0, s>>>(sg, part, beta, step, 1, 1); count_launch();
        k_seg_scale<C><<<nblk, kThr, 0, s>>>(sg, w, vn, single ? x32 : nullptr, beta, step, 1, keep); count_launch();
        k_step_inc<<<1, 1, 0, s>>>(step); count_launch();
        return cudaGetLastError();
    };

    // m Lanczos steps from `start` (unnormalised), keeping the vectors in
    // `keep` if it has a base.  Step 0 runs eagerly; the rest alternate
    // ring1 -> ring0 -> ring1 and replay a captured pair of steps.
    auto run = [&](const D *start, int m, bool single, bool acc, Store keep) -> cudaError_t {
        k_seg_dot<C, D><<<nblk, kThr, 0, st>>>(sg, start, (const D *)nullptr, part); count_launch();
        k_seg_final<<<ns, kThr, 0, st>>>(sg, part, nrm, nullptr, 0, 1); count_launch();
        k_seg_scale<C><<<nblk, kThr, 0, st>>>(sg, start, ring0, single ? x32 : nullptr, nrm, nullptr, 0, keep); count_launch();
        LM_CHK(cudaMemsetAsync(beta, 0, sc * sizeof(double), st));
        k_step_set<<<1, 1, 0, st>>>(step, 0); count_launch();
        LM_CHK(step_body(ring0, nullptr, ring1, single, acc, keep, st));
        int done = 1;
        if (m - done >= 2) {
            // capture steps (v = ring1, vp = ring0 -> ring0) and (ring0, ring1 -> ring1)
            const unsigned long long c0 = launches_so_far();
            LM_CHK(cudaStreamBeginCapture(O.cap, cudaStreamCaptureModeRelaxed));
            cudaError_t e = step_body(ring1, ring0, ring0, single, acc, keep, O.cap);
            if (e == cudaSuccess)
                e = step_body(ring0, ring1, ring1, single, acc, keep, O.cap);
            cudaGraph_t g = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(O.cap, &g);
            if (g)
                O.graphs.push_back(g);
            LM_CHK(e);
            LM_CHK(e2);
            const unsigned per_graph = (unsigned)(launches_so_far() - c0);
            uncount_launch(per_graph);  // captured, not yet run
            cudaGraphExec_t ge = nullptr;
            LM_CHK(cudaGraphInstantiate(&ge, g, 0));
            O.execs.push_back(ge);
            for (; m - done >= 2; done += 2) {
                LM_CHK(cudaGraphLaunch(ge, st));
                count_launch(per_graph);
            }
        }
        if (done < m)  // odd remainder; the current vector is in ring1
            LM_CHK(step_body(ring1, ring0, ring0, single, acc, keep, st));
        return cudaGetLastError();
    };
    auto tridiag = [&](int m) -> cudaError_t {
        LM_CHK(cudaMemsetAsync(y, 0, sc * sizeof(double), st));
        k_seg_tridiag<<<ns, 32, 0, st>>>(alpha, beta, stride, m, y, lam, m_eff, work); count_launch();
        return cudaGetLastError();
    };
    // m steps from start, then psi = the lowest Ritz vector of every sector
    const Store none{nullptr, 0, 0, total};
    int matvecs = 0;
    auto ritz_vectors = [&](const D *start, int m, bool single, Store keep) -> cudaError_t {
        LM_CHK(run(start, m, single, false, keep));
        LM_CHK(tridiag(m));
        matvecs += m;
        if (keep.base) {
            k_seg_combine<C><<<nblk, kThr, 0, st>>>(sg, psi, keep, y, m); count_launch();
            return cudaGetLastError();
        }
        matvecs += m;
        return run(start, m, single, true, none);  // bit-identical second pass
    };

    LM_TRY(ritz_vectors(x0, steps, f32, main_st));
    std::vector<double> h_lam(sc);
    std::vector<int> h_meff(ns);
    LM_TRY(cudaMemcpyAsync(h_lam.data(), lam, sc * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_TRY(cudaMemcpyAsync(h_meff.data(), m_eff, ns * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (f32) {  // fp64 refinement started from the fp32-matvec Ritz vectors
        LM_TRY(cudaMemcpyAsync(x0, psi, total * sizeof(D), cudaMemcpyDeviceToDevice, st));
        LM_TRY(ritz_vectors(x0, kRefine, false, ref_st));
    }
    // fp64 Rayleigh quotient and residual of psi, per sector
    LM_TRY(matvec(psi, w, false, st));
    ++matvecs;
    k_seg_dot<C, D><<<nblk, kThr, 0, st>>>(sg, psi, w, part); count_launch();
    k_seg_final<<<ns, kThr, 0, st>>>(sg, part, num, nullptr, 0, 0); count_launch();
    k_seg_dot<C, D><<<nblk, kThr, 0, st>>>(sg, psi, (const D *)nullptr, part); count_launch();
    k_seg_final<<<ns, kThr, 0, st>>>(sg, part, den, nullptr, 0, 0); count_launch();
    k_seg_resid<C><<<nblk, kThr, 0, st>>>(sg, w, psi, num, den, part); count_launch();
    k_seg_final<<<ns, kThr, 0, st>>>(sg, part, res, nullptr, 0, 0); count_launch();
    bool want_vec = false;
    for (int k = 0; k < ns; ++k)
        want_vec = want_vec || sectors[k].d_y;
    if (want_vec) {  // normalised vectors: psi / |psi| per sector, copied out
        k_seg_dot<C, D><<<nblk, kThr, 0, st>>>(sg, psi, (const D *)nullptr, part); count_launch();
        k_seg_final<<<ns, kThr, 0, st>>>(sg, part, nrm, nullptr, 0, 1); count_launch();
        k_seg_scale<C><<<nblk, kThr, 0, st>>>(sg, psi, w, nullptr, nrm, nullptr, 0, none); count_launch();
        for (int k = 0; k < ns; ++k)
            if (sectors[k].d_y)
                LM_TRY(cudaMemcpyAsync(sectors[k].d_y, w + off[k], (off[k + 1] - off[k]) * sizeof(D),
                                       cudaMemcpyDeviceToDevice, st));
    }
    LM_TRY(cudaGetLastError());
    std::vector<double> hn(sc), hd(sc), hr(sc);
    LM_TRY(cudaMemcpyAsync(hn.data(), num, sc * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_TRY(cudaMemcpyAsync(hd.data(), den, sc * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_TRY(cudaMemcpyAsync(hr.data(), res, sc * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_TRY(cudaStreamSynchronize(st));
    for (int k = 0; k < ns; ++k) {
        const size_t q = (size_t)k * stride;
        const double e0 = hn[q] / hd[q];
        if (e0_out)
            e0_out[k] = e0;
        if (info) {
            info[k].steps = h_meff[k];
            info[k].matvecs = matvecs;
            info[k].ritz = h_lam[q];
            info[k].e0 = e0;
            info[k].residual = std::sqrt(std::max(hr[q], 0.0) / hd[q]);
            info[k].matvec_ms = 0.0;
        }
    }
    return ED_OK;
}

#undef LM_CHK
#undef LM_TRY

}  // namespace
}  // namespace edk

extern "C" ed_status ed_lanczos_multi(const ed_operator *op, const ed_sector *sectors, int n_sectors, int steps,
                                      int mode, ed_dtype dtype, double *e0_out, ed_lanczos_info *info,
                                      void *stream)
{
    using namespace edk;
    if (!op || !sectors || n_sectors < 1 || n_sectors > kMaxSectors || steps < 1 || steps > 10000)
        return ED_ERR_INVALID_ARG;
    const int base = mode & ~ED_LANCZOS_RECOMPUTE;
    if (base != ED_LANCZOS_F64 && base != ED_LANCZOS_F32_MATVEC)
        return ED_ERR_INVALID_ARG;
    if (dtype != ED_F64 && dtype != ED_C128)
        return ED_ERR_INVALID_ARG;
    const ed_basis *b0 = sectors[0].basis;
    if (!b0)
        return ED_ERR_INVALID_ARG;
    for (int s = 0; s < n_sectors; ++s) {
        const ed_basis *b = sectors[s].basis;
        if (!b || b->n_sites != b0->n_sites || b->n_perm != b0->n_perm || b->perms != b0->perms)
            return ED_ERR_INVALID_ARG;
        const ed_status st = check_pair(op, b);
        if (st != ED_OK)
            return st;
        if (dtype == ED_F64 && !(b->real_chars && op->real))
            return ED_ERR_INVALID_ARG;
        const void *x = sectors[s].d_x;
        const void *y = sectors[s].d_y;
        if (b->dim == 0 || !x || (((uintptr_t)x | (uintptr_t)y) & 15))
            return ED_ERR_INVALID_ARG;
        if (!b->d_htab && !b->d_bkt)
            return ED_ERR_UNSUPPORTED;
    }
    static std::mutex mtx;  // the launch-argument staging is shared by all calls
    std::lock_guard<std::mutex> lock(mtx);
    const bool f32 = base == ED_LANCZOS_F32_MATVEC;
    const bool recompute = (mode & ED_LANCZOS_RECOMPUTE) != 0;
    cudaStream_t st = (cudaStream_t)stream;
    return dtype == ED_C128 ? run_multi<true>(op, sectors, n_sectors, steps, f32, recompute, e0_out, info, st)
                            : run_multi<false>(op, sectors, n_sectors, steps, f32, recompute, e0_out, info, st);
}
