// ed_lanczos_block.cu -- block Lanczos on p = nvec vectors at once, the
// consumer of the interleaved block product (Background: Krylov methods
// consume hundreds of products; one representative search and index lookup per
// matrix element serves all p columns of a block).
//
// Recurrence (real sectors; blocks are [dim][p], interleaved like the
// product's vectors, held as double-float pairs of fp32 arrays):  V_1 R_0 = X0 (QR),
//   W = H V_j,  C = V_j^T W,  Cp = V_{j-1}^T W,  A_j = (C + C^T) / 2,
//   W -= V_j C + V_{j-1} Cp,            (classical Gram-Schmidt against the two
//                                        last blocks: Cp replaces B_j^T)
//   W = V_{j+1} B_{j+1}                 (Cholesky QR, twice)
// so that H V_j = V_{j-1} B_j^T + V_j A_j + V_{j+1} B_{j+1} and the projected
// matrix T is block tridiagonal with bandwidth p.  Its lowest eigenpairs come
// from Sturm counts of a banded LDL^T factorisation (bisection, one warp) and
// banded inverse iteration; the Ritz vector from a second, bit-identical pass;
// the energy from a short fp64 single-vector Lanczos refinement of it
// (ed_lanczos), as in the single-vector fp32-matvec mode.
//
// Every reduction over the rows is a per-block partial in a fixed tile order,
// merged by the last block to finish in block order with compensated (TwoSum)
// merges, so both passes reproduce every coefficient bit for bit.  The
// per-element arithmetic is double-float on the fp32 pipe (see dd_acc); the
// coefficient matrices, the tile sums and all merges are fp64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "ed_kernels.cuh"

namespace edk {
namespace {

constexpr int kBlThreads = 256;
constexpr int kTileRows = 64;

struct KS {
    double s, c;
};
__device__ __forceinline__ KS ks_add(KS a, double b)
{
    const double s = a.s + b;
    const double bb = s - a.s;
    return {s, a.c + ((a.s - (s - bb)) + (b - bb))};
}
__device__ __forceinline__ KS ks_merge(KS a, KS b)
{
    KS r = ks_add(a, b.s);
    r.c += b.c;
    return r;
}

__device__ bool last_block(unsigned int *ticket)
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

// out[e] = merged block partials part[b * E + e], b in block order (the last
// block to finish runs this; every partial is visible after the ticket)
__device__ void merge_partials(const double2 *part, int E, double *out, unsigned int *ticket)
{
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        KS k{0.0, 0.0};
        for (unsigned b = 0; b < gridDim.x; ++b) {
            const double2 p = __ldcg(part + (size_t)b * E + e);
            k = ks_merge(k, KS{p.x, p.y});
        }
        out[e] = k.s + k.c;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        *ticket = 0;
}

// ---- double-float arithmetic on the fp32 pipe --------------------------------
// GB300's fp64 FMA rate is 1/74 of its fp32 rate (measured: 5.3e11 against
// 3.9e13 per second), so the per-element arithmetic of the block kernels uses
// pairs of floats (h + l, about 48 significant bits): error-free products by
// FMA and TwoSum accumulation.  Coefficient matrices, tile sums and every
// merge across threads and blocks stay fp64.
__device__ __forceinline__ void dd_acc(float xh, float xl, float yh, float yl, float &s, float &c)
{
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xh, yl, e);
    e = fmaf(xl, yh, e);
    const float t = s + p;
    const float z = t - s;
    c += ((s - (t - z)) + (p - z)) + e;
    s = t;
}

// dd_acc for a y that is exactly a float (low word zero): one FMA fewer
__device__ __forceinline__ void dd_acc1(float xh, float xl, float yh, float &s, float &c)
{
    const float p = xh * yh;
    float e = fmaf(xh, yh, -p);
    e = fmaf(xl, yh, e);
    const float t = s + p;
    const float z = t - s;
    c += ((s - (t - z)) + (p - z)) + e;
    s = t;
}

__device__ __forceinline__ void dd_split(double x, float &h, float &l)
{
    h = (float)x;
    l = (float)(x - (double)h);
}

// (h, l) += (s, c) as double-float numbers, renormalised
__device__ __forceinline__ void dd_add(float &h, float &l, float s, float c)
{
    const float t = h + s;
    const float z = t - h;
    float e = (h - (t - z)) + (s - z);
    e += l + c;
    h = t + e;
    l = e - (h - t);
}

// normalise s + c into h + l (|c| small against |s| after an accumulation)
__device__ __forceinline__ void dd_norm(float s, float c, float &h, float &l)
{
    h = s + c;
    l = c - (h - s);
}

// A tile's elements held in registers between the load of tile t + grid and
// the shared-memory store at the top of the next iteration, so that the
// global loads overlap the current tile's arithmetic.  Kind K: 0 fp32 array
// (low word 0), 1 fp64 array (split), 2 double-float block (separate high and
// low float arrays).
template <int P, int K>
struct Prefetch {
    static constexpr int kN = (kTileRows * P + kBlThreads - 1) / kBlThreads;
    float h[kN], l[kN];
    __device__ __forceinline__ void load(const void *gh, const float *gl, uint64_t r0, uint64_t n)
    {
        const uint64_t lim = n * P;
#pragma unroll
        for (int k = 0; k < kN; ++k) {
            const int e = threadIdx.x + k * kBlThreads;
            const uint64_t gi = r0 * P + (uint64_t)e;
            h[k] = 0.f;
            l[k] = 0.f;
            if (e < kTileRows * P && gi < lim) {
                if (K == 0) {
                    h[k] = reinterpret_cast<const float *>(gh)[gi];
                } else if (K == 1) {
                    dd_split(reinterpret_cast<const double *>(gh)[gi], h[k], l[k]);
                } else {
                    h[k] = reinterpret_cast<const float *>(gh)[gi];
                    l[k] = gl[gi];
                }
            }
        }
    }
    __device__ __forceinline__ void store(float *sh, float *sl) const
    {
#pragma unroll
        for (int k = 0; k < kN; ++k) {
            const int e = threadIdx.x + k * kBlThreads;
            if (e < kTileRows * P) {
                sh[e] = h[k];
                sl[e] = l[k];
            }
        }
    }
};

// Stride of the staged X tiles of the Gram kernel: one tile plus 8 floats, so
// that the two matrices' elements of one row fall in different banks.
template <int P> constexpr int kXStride = kTileRows * P + 8;

// Gram entries of a tile: entries are taken in 2 x 2 groups (a0, a0+1) x
// (b0, b0+1) of matrix m; a thread owns one group and a slice of the tile's
// rows (rows sl, sl + SL, ...), sums its four entries over them in double-
// float, adds the tile sums into renormalised double-float accumulators and
// moves those into fp64 every kFlushTiles tiles (fp64 work per row stays
// negligible; each double-float run spans at most kFlushTiles tile sums).
constexpr int kFlushTiles = 64;

struct GramAcc {
    float h[4], l[4];
    double d[4];
    int tiles;
    __device__ void init()
    {
        for (int k = 0; k < 4; ++k) {
            h[k] = l[k] = 0.f;
            d[k] = 0.0;
        }
        tiles = 0;
    }
    __device__ void flush()
    {
        for (int k = 0; k < 4; ++k) {
            d[k] += (double)h[k] + (double)l[k];
            h[k] = l[k] = 0.f;
        }
        tiles = 0;
    }
};
template <int P, int NM>
struct GramLayout {
    static constexpr int kHalf = P / 2;
    static constexpr int kGroups = NM * kHalf * kHalf;
    static constexpr int kSlices = kBlThreads / kGroups;
    static constexpr int E = NM * P * P;
};

template <int P, int NM, bool kYlow, int kXs = kTileRows * P>
__device__ __forceinline__ void gram_tile(const float *sxh, const float *sxl, const float *syh, const float *syl,
                                          GramAcc &acc)
{
    using L = GramLayout<P, NM>;
    // slices beyond the tile's rows (small P) stay idle; the others take
    // kRows rows each, unrolled with compile-time offsets
    constexpr int kActive = L::kSlices < kTileRows ? L::kSlices : kTileRows;
    constexpr int kRows = kTileRows / kActive;
    static_assert(kTileRows % kActive == 0, "slices must divide the tile");
    const int grp = threadIdx.x % L::kGroups, sl = threadIdx.x / L::kGroups;
    if (sl >= kActive)
        return;
    const int m = grp / (L::kHalf * L::kHalf), rem = grp % (L::kHalf * L::kHalf);
    const int a0 = 2 * (rem / L::kHalf), b0 = 2 * (rem % L::kHalf);
    // (a0, a0 + 1) and (b0, b0 + 1) are adjacent, 8-byte aligned pairs
    const float2 *xh = reinterpret_cast<const float2 *>(sxh + m * kXs + sl * P + a0);
    const float2 *xl = reinterpret_cast<const float2 *>(sxl + m * kXs + sl * P + a0);
    const float2 *yh = reinterpret_cast<const float2 *>(syh + sl * P + b0);
    const float2 *yl = reinterpret_cast<const float2 *>(syl + sl * P + b0);
    constexpr int kStep = kActive * P / 2;  // float2 elements between a slice's rows
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < kRows; ++i) {
        const float2 x_h = xh[i * kStep], x_l = xl[i * kStep], y_h = yh[i * kStep];
        if constexpr (kYlow) {
            const float2 y_l = yl[i * kStep];
            dd_acc(x_h.x, x_l.x, y_h.x, y_l.x, s[0], c[0]);
            dd_acc(x_h.x, x_l.x, y_h.y, y_l.y, s[1], c[1]);
            dd_acc(x_h.y, x_l.y, y_h.x, y_l.x, s[2], c[2]);
            dd_acc(x_h.y, x_l.y, y_h.y, y_l.y, s[3], c[3]);
        } else {
            dd_acc1(x_h.x, x_l.x, y_h.x, s[0], c[0]);
            dd_acc1(x_h.x, x_l.x, y_h.y, s[1], c[1]);
            dd_acc1(x_h.y, x_l.y, y_h.x, s[2], c[2]);
            dd_acc1(x_h.y, x_l.y, y_h.y, s[3], c[3]);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        dd_add(acc.h[k], acc.l[k], s[k], c[k]);
    if (++acc.tiles == kFlushTiles)
        acc.flush();
}

// Per-block partials of the Gram entries: the slices' fp64 accumulators merged
// in slice order (compensated) through shared memory; the last block to
// finish merges the blocks into out.
template <int P, int NM>
__device__ void gram_finish(GramAcc &acc, double *red, double2 *part, unsigned int *ticket, double *out)
{
    using L = GramLayout<P, NM>;
    const int grp = threadIdx.x % L::kGroups, sl = threadIdx.x / L::kGroups;
    acc.flush();
    __syncthreads();
    if (sl < L::kSlices)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            red[(sl * L::kGroups + grp) * 4 + k] = acc.d[k];
    __syncthreads();
    for (int e = threadIdx.x; e < L::E; e += blockDim.x) {
        const int m = e / (P * P), a = (e / P) % P, b = e % P;
        const int g = m * L::kHalf * L::kHalf + (a / 2) * L::kHalf + b / 2, k = (a & 1) * 2 + (b & 1);
        KS t{0.0, 0.0};
        for (int q = 0; q < L::kSlices; ++q)
            t = ks_add(t, red[(q * L::kGroups + g) * 4 + k]);
        part[(size_t)blockIdx.x * L::E + e] = make_double2(t.s, t.c);
    }
    if (last_block(ticket))
        merge_partials(part, L::E, out, ticket);
}

// Gram of NM double-float blocks X_m against Y (kind YK as in Prefetch):
// out[m][a][b] = sum_i X_m[i][a] Y[i][b].
template <int P, int NM, int YK>
__global__ void __launch_bounds__(kBlThreads) k_dd_gram(const float *X0h, const float *X0l, const float *X1h,
                                                        const float *X1l, const void *Yh, const float *Yl,
                                                        uint64_t n, double2 *part, unsigned int *ticket,
                                                        double *out, const int *stop)
{
    if (*stop)
        return;
    __shared__ __align__(16) float sxh[NM * kXStride<P>], sxl[NM * kXStride<P>];
    __shared__ __align__(16) float syh[kTileRows * P], syl[kTileRows * P];
    __shared__ double red[kBlThreads * 4];
    GramAcc acc;
    acc.init();
    const uint64_t tiles = (n + kTileRows - 1) / kTileRows;
    Prefetch<P, 2> p0, p1;
    Prefetch<P, YK> py;
    auto fetch = [&](uint64_t t) {
        p0.load(X0h, X0l, t * kTileRows, n);
        if (NM > 1)
            p1.load(X1h, X1l, t * kTileRows, n);
        py.load(Yh, Yl, t * kTileRows, n);
    };
    if (blockIdx.x < tiles)
        fetch(blockIdx.x);
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        p0.store(sxh, sxl);
        if (NM > 1)
            p1.store(sxh + kXStride<P>, sxl + kXStride<P>);
        py.store(syh, syl);
        __syncthreads();
        if (t + gridDim.x < tiles)
            fetch(t + gridDim.x);
        gram_tile<P, NM, YK != 0, kXStride<P>>(sxh, sxl, syh, syl, acc);
        __syncthreads();
    }
    gram_finish<P, NM>(acc, red, part, ticket, out);
}

// ---- row-per-thread kernels: update and Cholesky QR ---------------------------
// One thread per row: a row's P elements (high and low words) come straight
// from global memory into registers, the P x P coefficient matrix is read from
// shared memory as (high, low) pairs (broadcast, one 8-byte load per
// double-float multiply-add), and triangular coefficient matrices cost only
// their P (P + 1) / 2 nonzero entries.  A tile is kBlThreads rows; the Gram
// of the rows a tile produced is taken from a padded shared-memory copy.

// P floats of row `row` of a [n][P] block (16-byte aligned rows for P >= 4)
template <int P>
__device__ __forceinline__ void load_row(const float *g, uint64_t row, float (&v)[P])
{
    if constexpr (P % 4 == 0) {
        const float4 *q = reinterpret_cast<const float4 *>(g + row * P);
#pragma unroll
        for (int k = 0; k < P / 4; ++k) {
            const float4 t = q[k];
            v[4 * k] = t.x;
            v[4 * k + 1] = t.y;
            v[4 * k + 2] = t.z;
            v[4 * k + 3] = t.w;
        }
    } else {
        static_assert(P == 2, "block sizes 2, 4, 8, 16");
        const float2 t = reinterpret_cast<const float2 *>(g + row * P)[0];
        v[0] = t.x;
        v[1] = t.y;
    }
}

template <int P>
__device__ __forceinline__ void store_row(float *g, uint64_t row, const float (&v)[P])
{
    if constexpr (P % 4 == 0) {
        float4 *q = reinterpret_cast<float4 *>(g + row * P);
#pragma unroll
        for (int k = 0; k < P / 4; ++k)
            q[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
        reinterpret_cast<float2 *>(g + row * P)[0] = make_float2(v[0], v[1]);
    }
}

// Row of the product output Y as a double-float start value (kind YK as in
// Prefetch: 0 fp32, 1 fp64, 2 double-float)
template <int P, int YK>
__device__ __forceinline__ void load_y_row(const void *gh, const float *gl, uint64_t row, float (&s)[P],
                                           float (&c)[P])
{
    if constexpr (YK == 0) {
        load_row<P>(reinterpret_cast<const float *>(gh), row, s);
#pragma unroll
        for (int b = 0; b < P; ++b)
            c[b] = 0.f;
    } else if constexpr (YK == 1) {
        const double *q = reinterpret_cast<const double *>(gh) + row * P;
#pragma unroll
        for (int b = 0; b < P; ++b)
            dd_split(q[b], s[b], c[b]);
    } else {
        load_row<P>(reinterpret_cast<const float *>(gh), row, s);
        load_row<P>(gl, row, c);
    }
}

// Symmetric Gram of a staged tile of kBlThreads rows with row stride P + 1:
// the 2 x 2 entry groups (ga, gb) with ga <= gb (P/2 (P/2 + 1) / 2 of them),
// one per thread, with a slice of the tile's rows.
template <int P>
struct SymLayout {
    static constexpr int kHalf = P / 2;
    static constexpr int kGroups = kHalf * (kHalf + 1) / 2;
    static constexpr int kSlices = kGroups == 1 ? 256 : kGroups <= 4 ? 64 : kGroups <= 16 ? 16 : 4;
    static constexpr int kRows = kBlThreads / kSlices;  // rows per slice and tile
    static constexpr int kStride = P + 2;               // even: 8-byte aligned pairs
    static_assert(kGroups * kSlices <= kBlThreads && kBlThreads % kSlices == 0, "layout");
    __device__ static int index(int ga, int gb) { return ga * kHalf - ga * (ga - 1) / 2 + (gb - ga); }
    __device__ static void groups(int g, int &ga, int &gb)
    {
        ga = 0;
        while (g >= kHalf - ga) {
            g -= kHalf - ga;
            ++ga;
        }
        gb = ga + g;
    }
};

template <int P>
__device__ __forceinline__ void gram_tile_sym(const float *sh, const float *sl, GramAcc &acc)
{
    using L = SymLayout<P>;
    const int grp = threadIdx.x % L::kGroups, slc = threadIdx.x / L::kGroups;
    if (slc >= L::kSlices)
        return;
    int ga, gb;
    L::groups(grp, ga, gb);
    const float2 *xh = reinterpret_cast<const float2 *>(sh + slc * L::kStride + 2 * ga);
    const float2 *xl = reinterpret_cast<const float2 *>(sl + slc * L::kStride + 2 * ga);
    const float2 *yh = reinterpret_cast<const float2 *>(sh + slc * L::kStride + 2 * gb);
    const float2 *yl = reinterpret_cast<const float2 *>(sl + slc * L::kStride + 2 * gb);
    constexpr int kStep = L::kSlices * L::kStride / 2;
    float s[4] = {0.f, 0.f, 0.f, 0.f}, c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < L::kRows; ++i) {
        const float2 x_h = xh[i * kStep], x_l = xl[i * kStep], y_h = yh[i * kStep], y_l = yl[i * kStep];
        dd_acc(x_h.x, x_l.x, y_h.x, y_l.x, s[0], c[0]);
        dd_acc(x_h.x, x_l.x, y_h.y, y_l.y, s[1], c[1]);
        dd_acc(x_h.y, x_l.y, y_h.x, y_l.x, s[2], c[2]);
        dd_acc(x_h.y, x_l.y, y_h.y, y_l.y, s[3], c[3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        dd_add(acc.h[k], acc.l[k], s[k], c[k]);
    if (++acc.tiles == kFlushTiles)
        acc.flush();
}

// As gram_finish, for the symmetric layout: entry (a, b) with a/2 > b/2 is
// the transposed entry of group (b/2, a/2), so the result is exactly symmetric.
template <int P>
__device__ void gram_finish_sym(GramAcc &acc, double *red, double2 *part, unsigned int *ticket, double *out)
{
    using L = SymLayout<P>;
    const int grp = threadIdx.x % L::kGroups, slc = threadIdx.x / L::kGroups;
    acc.flush();
    __syncthreads();
    if (slc < L::kSlices)
#pragma unroll
        for (int k = 0; k < 4; ++k)
            red[(slc * L::kGroups + grp) * 4 + k] = acc.d[k];
    __syncthreads();
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int a = e / P, b = e % P;
        const bool tr = a / 2 > b / 2;
        const int g = tr ? L::index(b / 2, a / 2) : L::index(a / 2, b / 2);
        const int k = tr ? (b & 1) * 2 + (a & 1) : (a & 1) * 2 + (b & 1);
        KS t{0.0, 0.0};
        for (int q = 0; q < L::kSlices; ++q)
            t = ks_add(t, red[(q * L::kGroups + g) * 4 + k]);
        part[(size_t)blockIdx.x * P * P + e] = make_double2(t.s, t.c);
    }
    if (last_block(ticket))
        merge_partials(part, P * P, out, ticket);
}

// W = Y - X0 C0 - X1 C1 (C fp64, P x P row-major per matrix: W[i][b] -=
// sum_a X[i][a] C[a][b]), written as a double-float block; W may alias X1 or
// Y (each row is read completely by its thread before that thread writes it).
// With G: the Gram of W.
template <int P, int NM, int YK>
__global__ void __launch_bounds__(kBlThreads) k_dd_update(const float *X0h, const float *X0l, const float *X1h,
                                                          const float *X1l, const void *Yh, const float *Yl,
                                                          const double *C, float *Wh, float *Wl, uint64_t n,
                                                          double2 *part, unsigned int *ticket, double *G,
                                                          const int *stop)
{
    if (*stop)
        return;
    using L = SymLayout<P>;
    __shared__ __align__(16) float2 sc[NM * P * P];
    __shared__ __align__(16) float swh[kBlThreads * L::kStride], swl[kBlThreads * L::kStride];
    __shared__ double red[kBlThreads * 4];
    for (int e = threadIdx.x; e < NM * P * P; e += blockDim.x) {
        float h, l;
        dd_split(-C[e], h, l);
        sc[e] = make_float2(h, l);
    }
    __syncthreads();
    GramAcc acc;
    acc.init();
    const uint64_t tiles = (n + kBlThreads - 1) / kBlThreads;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t row = t * kBlThreads + threadIdx.x;
        float wh[P], wl[P];
        if (row < n) {
            float s[P], c[P];
            load_y_row<P, YK>(Yh, Yl, row, s, c);
#pragma unroll
            for (int m = 0; m < NM; ++m) {
                float xh[P], xl[P];
                load_row<P>(m ? X1h : X0h, row, xh);
                load_row<P>(m ? X1l : X0l, row, xl);
#pragma unroll
                for (int a = 0; a < P; ++a)
#pragma unroll
                    for (int b = 0; b < P; b += 2) {  // two (high, low) coefficients per load
                        const float4 q = reinterpret_cast<const float4 *>(sc + m * P * P + a * P)[b / 2];
                        dd_acc(xh[a], xl[a], q.x, q.y, s[b], c[b]);
                        dd_acc(xh[a], xl[a], q.z, q.w, s[b + 1], c[b + 1]);
                    }
            }
#pragma unroll
            for (int b = 0; b < P; ++b)
                dd_norm(s[b], c[b], wh[b], wl[b]);
            store_row<P>(Wh, row, wh);
            store_row<P>(Wl, row, wl);
        } else {
#pragma unroll
            for (int b = 0; b < P; ++b)
                wh[b] = wl[b] = 0.f;
        }
        if (G) {
#pragma unroll
            for (int b = 0; b < P; ++b) {
                swh[threadIdx.x * L::kStride + b] = wh[b];
                swl[threadIdx.x * L::kStride + b] = wl[b];
            }
            __syncthreads();
            gram_tile_sym<P>(swh, swl, acc);
            __syncthreads();
        }
    }
    if (G)
        gram_finish_sym<P>(acc, red, part, ticket, G);
}

// Cholesky QR steps on the block W (double-float, in place).  kApply = false:
// Z = W R1i (R1i fp64 upper triangular, row-major) and the Gram of Z into G2;
// kApply = true: W = W (R1i R2i), the product of the two upper triangular
// inverses formed in fp64 (CholQR2 applied at once).
template <int P, bool kApply>
__global__ void __launch_bounds__(kBlThreads) k_dd_qr(float *Wh, float *Wl, const double *R1i, const double *R2i,
                                                      uint64_t n, double2 *part, unsigned int *ticket,
                                                      double *G2, const int *stop)
{
    if (*stop)
        return;
    using L = SymLayout<P>;
    constexpr int kZ = kApply ? 1 : kBlThreads * L::kStride;
    __shared__ __align__(16) float2 sr[P * P];
    __shared__ __align__(16) float szh[kZ], szl[kZ];
    __shared__ double red[kApply ? 1 : kBlThreads * 4];
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        const int a = e / P, b = e % P;
        double v = 0.0;
        if (kApply) {
            for (int k = a; k <= b; ++k)
                v += R1i[a * P + k] * R2i[k * P + b];
        } else if (a <= b) {
            v = R1i[e];
        }
        float h, l;
        dd_split(v, h, l);
        sr[e] = make_float2(h, l);
    }
    __syncthreads();
    GramAcc acc;
    acc.init();
    const uint64_t tiles = (n + kBlThreads - 1) / kBlThreads;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t row = t * kBlThreads + threadIdx.x;
        float zh[P], zl[P];
        if (row < n) {
            float wh[P], wl[P];
            load_row<P>(Wh, row, wh);
            load_row<P>(Wl, row, wl);
#pragma unroll
            for (int b = 0; b < P; ++b) {
                float s = 0.f, c = 0.f;
#pragma unroll
                for (int a = 0; a <= b; ++a) {
                    const float2 q = sr[a * P + b];
                    dd_acc(wh[a], wl[a], q.x, q.y, s, c);
                }
                dd_norm(s, c, zh[b], zl[b]);
            }
            if (kApply) {
                store_row<P>(Wh, row, zh);
                store_row<P>(Wl, row, zl);
            }
        } else {
#pragma unroll
            for (int b = 0; b < P; ++b)
                zh[b] = zl[b] = 0.f;
        }
        if (!kApply) {
#pragma unroll
            for (int b = 0; b < P; ++b) {
                szh[threadIdx.x * L::kStride + b] = zh[b];
                szl[threadIdx.x * L::kStride + b] = zl[b];
            }
            __syncthreads();
            gram_tile_sym<P>(szh, szl, acc);
            __syncthreads();
        }
    }
    if (!kApply)
        gram_finish_sym<P>(acc, red, part, ticket, G2);
}

// psi (double-float, dim) += V_j s_j  (s_j = y[j P .. j P + P) in fp64); psi
// starts from zero when first
template <int P>
__global__ void k_dd_ritz_acc(float *ph, float *pl, const float *Vh, const float *Vl, const double *y, int j,
                              uint64_t n, int first, const int *m_eff)
{
    if (j >= *m_eff)
        return;
    float ch[P], cl[P];
#pragma unroll
    for (int a = 0; a < P; ++a)
        dd_split(y[j * P + a], ch[a], cl[a]);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        float s = first ? 0.f : ph[i], c = first ? 0.f : pl[i];
#pragma unroll
        for (int a = 0; a < P; ++a)
            dd_acc(Vh[i * P + a], Vl[i * P + a], ch[a], cl[a], s, c);
        float h, l;
        dd_norm(s, c, h, l);
        ph[i] = h;
        pl[i] = l;
    }
}

// fp64 <-> double-float conversions of whole arrays
__global__ void k_f64_to_dd(const double *x, float *h, float *l, uint64_t count)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        dd_split(x[i], h[i], l[i]);
}

__global__ void k_dd_to_f64(const float *h, const float *l, double *x, uint64_t count)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (uint64_t)gridDim.x * blockDim.x)
        x[i] = (double)h[i] + (double)l[i];
}

// Cholesky of the P x P symmetric matrix G (row-major): G = R^T R, R upper
// triangular; Ri = R^-1 (upper).  False when a pivot is not positive enough
// (rank loss: the block Krylov space stops growing).
template <int P>
__device__ bool chol_upper(const double *G, double *R, double *Ri)
{
    double scale = 0.0;
    for (int a = 0; a < P; ++a)
        scale = fmax(scale, G[a * P + a]);
    for (int e = 0; e < P * P; ++e) {
        R[e] = 0.0;
        Ri[e] = 0.0;
    }
    for (int a = 0; a < P; ++a) {
        double d = G[a * P + a];
        for (int k = 0; k < a; ++k)
            d -= R[k * P + a] * R[k * P + a];
        if (!(d > 1e-28 * scale) || !(scale > 0.0))
            return false;
        const double r = sqrt(d);
        R[a * P + a] = r;
        for (int b = a + 1; b < P; ++b) {
            double s = 0.5 * (G[a * P + b] + G[b * P + a]);
            for (int k = 0; k < a; ++k)
                s -= R[k * P + a] * R[k * P + b];
            R[a * P + b] = s / r;
        }
    }
    // inverse of the upper triangular R, column by column
    for (int b = 0; b < P; ++b) {
        Ri[b * P + b] = 1.0 / R[b * P + b];
        for (int a = b - 1; a >= 0; --a) {
            double s = 0.0;
            for (int k = a + 1; k <= b; ++k)
                s += R[a * P + k] * Ri[k * P + b];
            Ri[a * P + b] = -s / R[a * P + a];
        }
    }
    return true;
}

// Small P x P steps, one thread.  Layout of `sm` (device scratch, P*P blocks):
// [0] C   [1] Cp   [2] G   [3] R1   [4] R1i   [5] G2   [6] R2   [7] R2i
// which = 0: A_j = sym(C) -> A[j] (j = step index, 0-based);
// which = 1: R1 = chol(G);  which = 2: R2 = chol(G2), B[j + 1] = R2 R1 (the
// coupling to the next block; for j < 0 (the start block) nothing is stored).
// A failed Cholesky stops the recurrence: *stop = 1, *m_eff = j + 1 blocks.
template <int P>
__global__ void k_bl_small(double *sm, double *A, double *B, int j, int which, int *stop, int *m_eff)
{
    if (threadIdx.x != 0 || *stop)
        return;
    double *C = sm, *G = sm + 2 * P * P, *R1 = sm + 3 * P * P, *R1i = sm + 4 * P * P;
    double *G2 = sm + 5 * P * P, *R2 = sm + 6 * P * P, *R2i = sm + 7 * P * P;
    if (which == 0) {
        for (int a = 0; a < P; ++a)
            for (int b = 0; b < P; ++b)
                A[(size_t)j * P * P + a * P + b] = 0.5 * (C[a * P + b] + C[b * P + a]);
        return;
    }
    if (which == 1) {
        if (!chol_upper<P>(G, R1, R1i)) {
            *stop = 1;
            *m_eff = j + 1;
        }
        return;
    }
    if (!chol_upper<P>(G2, R2, R2i)) {
        *stop = 1;
        *m_eff = j + 1;
        return;
    }
    if (j >= 0) {
        double *Bn = B + (size_t)(j + 1) * P * P;  // B = R2 R1 (upper triangular)
        for (int a = 0; a < P; ++a)
            for (int b = 0; b < P; ++b) {
                double s = 0.0;
                for (int k = a; k <= b; ++k)
                    s += R2[a * P + k] * R1[k * P + b];
                Bn[a * P + b] = b >= a ? s : 0.0;
            }
        *m_eff = j + 1;
    }
}

// ---- eigenpairs of the block tridiagonal T (bandwidth P) ----------------------
// T(r, c): diagonal blocks A_j, T[j+1][j] = B_{j+1}, T[j][j+1] = B_{j+1}^T.
template <int P>
__device__ __forceinline__ double band_el(const double *A, const double *B, int r, int c)
{
    const int jr = r / P, a = r % P, jc = c / P, b = c % P;
    if (jr == jc)
        return A[(size_t)jr * P * P + a * P + b];
    if (jr == jc + 1)
        return B[(size_t)jr * P * P + a * P + b];
    if (jc == jr + 1)
        return B[(size_t)jc * P * P + b * P + a];
    return 0.0;
}

// Number of eigenvalues of the leading nn x nn block of T below x: negative
// pivots of the banded LDL^T of T - x I (Sylvester's law of inertia), with the
// last P rows of L kept in a ring.
template <int P>
__device__ int band_count(const double *A, const double *B, int nn, double x, double tiny)
{
    double L[P + 1][P];  // L[k % (P+1)][k - l - 1] = L(k, l), l in [k - P, k)
    double D[P + 1];
    int cnt = 0;
    for (int k = 0; k < nn; ++k) {
        const int ks = k % (P + 1);
        const int k0 = max(0, k - P);
        for (int j = k0; j < k; ++j) {
            const int js = j % (P + 1);
            double s = band_el<P>(A, B, k, j);
            for (int l = max(k0, j - P); l < j; ++l)
                s -= L[ks][k - l - 1] * D[l % (P + 1)] * L[js][j - l - 1];
            L[ks][k - j - 1] = s / D[js];
        }
        double d = band_el<P>(A, B, k, k) - x;
        for (int l = k0; l < k; ++l)
            d -= L[ks][k - l - 1] * L[ks][k - l - 1] * D[l % (P + 1)];
        if (fabs(d) < tiny)
            d = -tiny;
        D[ks] = d;
        cnt += d < 0.0;
    }
    return cnt;
}

// Eigenvalue number blockIdx.x (0 = lowest) of the leading m_eff P x m_eff P
// block by 32-point multisection; block 0 also finds the eigenvector of the
// lowest by inverse iteration (banded LDL^T with guarded pivots; scratch holds
// nn (P + 1) doubles).  Launch with 32 threads per block.
template <int P>
__global__ void k_band_eigs(const double *A, const double *B, const int *m_eff, double *eig, double *y,
                            double *scratch)
{
    const int lane = threadIdx.x & 31;
    const int nn = *m_eff * P;
    const int e = blockIdx.x;
    if (e >= nn) {
        if (lane == 0)
            eig[e] = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    double lo = 1e300, hi = -1e300, scale = 0.0;
    for (int r = 0; r < nn; ++r) {  // Gershgorin interval
        double rad = 0.0;
        for (int c = max(0, r - P); c <= min(nn - 1, r + P); ++c)
            if (c != r)
                rad += fabs(band_el<P>(A, B, r, c));
        const double d = band_el<P>(A, B, r, r);
        lo = fmin(lo, d - rad);
        hi = fmax(hi, d + rad);
        scale = fmax(scale, fabs(d) + rad);
    }
    const double tiny = 1e-300 + 1e-30 * scale;
    for (int it = 0; it < 64; ++it) {
        const double width = hi - lo;
        if (!(width > 2e-16 * fmax(fabs(lo), fabs(hi))))
            break;
        const double x = lo + width * (double)(lane + 1) / 33.0;
        const unsigned below = __ballot_sync(0xffffffffu, band_count<P>(A, B, nn, x, tiny) >= e + 1);
        const int f = below ? __ffs(below) - 1 : 32;
        const double nlo = f == 0 ? lo : lo + width * (double)f / 33.0;
        const double nhi = f == 32 ? hi : lo + width * (double)(f + 1) / 33.0;
        lo = nlo;
        hi = nhi;
    }
    if (lane != 0)
        return;
    const double lam = 0.5 * (lo + hi);
    eig[e] = lam;
    if (e != 0 || !y)
        return;
    // inverse iteration: banded LDL^T of T - lam I stored in full (row k:
    // L(k, k-1-q) at scratch[k (P+1) + q], D(k) at scratch[k (P+1) + P])
    const double eps = 1e-15 * fmax(scale, 1e-300);
    double *F = scratch;
    for (int k = 0; k < nn; ++k) {
        const int k0 = max(0, k - P);
        for (int j = k0; j < k; ++j) {
            double s = band_el<P>(A, B, k, j);
            for (int l = max(k0, j - P); l < j; ++l)
                s -= F[(size_t)k * (P + 1) + (k - l - 1)] * F[(size_t)l * (P + 1) + P] *
                     F[(size_t)j * (P + 1) + (j - l - 1)];
            F[(size_t)k * (P + 1) + (k - j - 1)] = s / F[(size_t)j * (P + 1) + P];
        }
        double d = band_el<P>(A, B, k, k) - lam;
        for (int l = k0; l < k; ++l) {
            const double Lkl = F[(size_t)k * (P + 1) + (k - l - 1)];
            d -= Lkl * Lkl * F[(size_t)l * (P + 1) + P];
        }
        if (fabs(d) < eps)
            d = d < 0.0 ? -eps : eps;
        F[(size_t)k * (P + 1) + P] = d;
    }
    for (int k = 0; k < nn; ++k)
        y[k] = 1.0;
    for (int iter = 0; iter < 4; ++iter) {
        for (int k = 0; k < nn; ++k)  // L u = y
            for (int l = max(0, k - P); l < k; ++l)
                y[k] -= F[(size_t)k * (P + 1) + (k - l - 1)] * y[l];
        for (int k = 0; k < nn; ++k)  // D
            y[k] /= F[(size_t)k * (P + 1) + P];
        for (int k = nn - 1; k >= 0; --k)  // L^T z = u
            for (int r = k + 1; r <= min(nn - 1, k + P); ++r)
                y[k] -= F[(size_t)r * (P + 1) + (r - k - 1)] * y[r];
        double nrm = 0.0;
        for (int k = 0; k < nn; ++k)
            nrm += y[k] * y[k];
        nrm = sqrt(nrm);
        for (int k = 0; k < nn; ++k)
            y[k] /= nrm;
    }
}

struct Pool {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit Pool(cudaStream_t s) : st(s) {}
    ~Pool()
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

#define ED_BL_TRY(expr)                                                     \
    do {                                                                    \
        cudaError_t _e = (expr);                                            \
        if (_e != cudaSuccess) {                                            \
            (void)cudaGetLastError();                                       \
            return _e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA; \
        }                                                                   \
    } while (0)

// Launch helpers for the product output kind (0: fp32, 1: fp64) and the
// number of earlier blocks (1 or 2) the new one is orthogonalised against.
template <int P>
void launch_gram(int nm, int yk, const float *X0h, const float *X0l, const float *X1h, const float *X1l,
                 const void *Yh, const float *Yl, uint64_t n, int grid, double2 *part, unsigned int *ticket,
                 double *out, const int *stop, cudaStream_t st)
{
#define ED_DD_GRAM(NM, YK) \
    k_dd_gram<P, NM, YK><<<grid, kBlThreads, 0, st>>>(X0h, X0l, X1h, X1l, Yh, Yl, n, part, ticket, out, stop)
    if (nm == 1) {
        if (yk == 0) ED_DD_GRAM(1, 0); else if (yk == 1) ED_DD_GRAM(1, 1); else ED_DD_GRAM(1, 2);
    } else {
        if (yk == 0) ED_DD_GRAM(2, 0); else if (yk == 1) ED_DD_GRAM(2, 1); else ED_DD_GRAM(2, 2);
    }
#undef ED_DD_GRAM
    count_launch();
}

template <int P>
void launch_update(int nm, int yk, const float *X0h, const float *X0l, const float *X1h, const float *X1l,
                   const void *Yh, const float *Yl, const double *C, float *Wh, float *Wl, uint64_t n, int grid,
                   double2 *part, unsigned int *ticket, double *G, const int *stop, cudaStream_t st)
{
#define ED_DD_UPD(NM, YK)                                                                                  \
    k_dd_update<P, NM, YK><<<grid, kBlThreads, 0, st>>>(X0h, X0l, X1h, X1l, Yh, Yl, C, Wh, Wl, n, part, ticket, \
                                                        G, stop)
    if (nm == 1) {
        if (yk == 0) ED_DD_UPD(1, 0); else if (yk == 1) ED_DD_UPD(1, 1); else ED_DD_UPD(1, 2);
    } else {
        if (yk == 0) ED_DD_UPD(2, 0); else if (yk == 1) ED_DD_UPD(2, 1); else ED_DD_UPD(2, 2);
    }
#undef ED_DD_UPD
    count_launch();
}

template <int P>
ed_status run_block(const ed_operator *op, const ed_basis *b, const double *x0, int steps, bool f32, bool reorth,
                    bool values_only, int n_eig, double *eigs_out, double *psi_out, int *steps_out,
                    int *matvecs_out, double *ritz_out, double *res_out, double *mv_ms_out, cudaStream_t st)
{
    const uint64_t n = b->dim;
    const OpView ov = make_op_view(op);
    const GroupView gv = b->group_view();
    const IndexView iv = b->index_view();
    const bool track = !b->trivial_chars;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t tiles = (n + kTileRows - 1) / kTileRows;
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * 4, tiles));
    // the row-per-thread kernels (update, QR): tiles of kBlThreads rows
    const uint64_t rtiles = (n + kBlThreads - 1) / kBlThreads;
    const int rgrid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * 4, rtiles));
    const int vgrid = (int)std::max<uint64_t>(1, std::min<uint64_t>((uint64_t)sms * 8, (n + 255) / 256));
    const size_t blk = (size_t)n * P;

    Pool S(st);
    // blocks as double-float (high and low float arrays); the high array is
    // the fp32 copy the products read
    float *Vh = nullptr, *Vl = nullptr;  // 2 blocks (ring), or steps + 1 (kept)
    const int nblocks = reorth ? steps + 1 : 2;
    float *W32 = nullptr, *ph = nullptr, *pl = nullptr;
    double *V64 = nullptr, *W64 = nullptr, *A = nullptr, *B = nullptr, *sm = nullptr;
    double *y = nullptr, *eig = nullptr, *scr = nullptr;
    double2 *part = nullptr;
    unsigned int *tickets = nullptr;
    int *flags = nullptr;  // [0] stop, [1] m_eff (running), [2] m_eff of the main pass
    ED_BL_TRY(S.get(&Vh, (size_t)nblocks * blk));
    ED_BL_TRY(S.get(&Vl, (size_t)nblocks * blk));
    if (f32) {
        ED_BL_TRY(S.get(&W32, blk));
    } else {
        ED_BL_TRY(S.get(&V64, blk));
        ED_BL_TRY(S.get(&W64, blk));
    }
    ED_BL_TRY(S.get(&ph, n));
    ED_BL_TRY(S.get(&pl, n));
    ED_BL_TRY(S.get(&A, (size_t)(steps + 1) * P * P));
    ED_BL_TRY(S.get(&B, (size_t)(steps + 2) * P * P));
    ED_BL_TRY(S.get(&sm, 8 * P * P));
    ED_BL_TRY(S.get(&y, (size_t)(steps + 1) * P));
    ED_BL_TRY(S.get(&eig, std::max(n_eig, 1)));
    ED_BL_TRY(S.get(&scr, (size_t)(steps + 1) * P * (P + 1)));
    ED_BL_TRY(S.get(&part, (size_t)grid * 2 * P * P));
    ED_BL_TRY(S.get(&tickets, 4));
    ED_BL_TRY(S.get(&flags, 3));
    ED_BL_TRY(cudaMemsetAsync(tickets, 0, 4 * sizeof(unsigned int), st));
    ED_BL_TRY(cudaMemsetAsync(A, 0, (size_t)(steps + 1) * P * P * sizeof(double), st));
    ED_BL_TRY(cudaMemsetAsync(B, 0, (size_t)(steps + 2) * P * P * sizeof(double), st));

    int matvecs = 0;
    std::vector<cudaEvent_t> ev;
    auto mark = [&]() -> cudaError_t {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess)
            return r;
        ev.push_back(e);
        return cudaEventRecord(e, st);
    };
    double *C = sm, *G = sm + 2 * P * P, *R1i = sm + 4 * P * P, *G2 = sm + 5 * P * P, *R2i = sm + 7 * P * P;
    int *stop = flags;
    const int yk = f32 ? 0 : 1;
    const MatvecVariant tuned = tuned_variant(b, P, f32 ? ED_F32 : ED_F64);
    const void *Yh = f32 ? (const void *)W32 : (const void *)W64;
    auto bh = [&](int k) { return Vh + (size_t)(reorth ? k : (k & 1)) * blk; };
    auto bl = [&](int k) { return Vl + (size_t)(reorth ? k : (k & 1)) * blk; };

    // Cholesky QR (twice) of the block (wh, wl) in place; R1 already in sm
    auto qr = [&](float *wh, float *wl, int j) {
        k_dd_qr<P, false><<<rgrid, kBlThreads, 0, st>>>(wh, wl, R1i, nullptr, n, part, tickets + 2, G2, stop);
        count_launch();
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 2, stop, flags + 1); count_launch();
        k_dd_qr<P, true><<<rgrid, kBlThreads, 0, st>>>(wh, wl, R1i, R2i, n, part, tickets + 2, nullptr, stop);
        count_launch();
    };

    // One pass of `steps` block steps from x0; with acc, psi += V_j s_j.
    auto pass = [&](bool acc) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
        if (e != cudaSuccess)
            return e;
        k_f64_to_dd<<<vgrid, 256, 0, st>>>(x0, bh(0), bl(0), blk); count_launch();
        launch_gram<P>(1, 2, bh(0), bl(0), nullptr, nullptr, bh(0), bl(0), n, grid, part, tickets, G, stop, st);
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, -1, 1, stop, flags + 1); count_launch();
        qr(bh(0), bl(0), -1);
        for (int j = 0; j < steps; ++j) {
            float *Vjh = bh(j), *Vjl = bl(j);
            const float *Vph = j ? bh(j - 1) : nullptr, *Vpl = j ? bl(j - 1) : nullptr;
            float *Wh = bh(j + 1), *Wl = bl(j + 1);  // the ring's V_{j-1} buffer, or kept block j + 1
            if (acc && !reorth) {
                k_dd_ritz_acc<P><<<vgrid, 256, 0, st>>>(ph, pl, Vjh, Vjl, y, j, n, j == 0, flags + 2);
                count_launch();
            }
            // W = H V_j (a stopped recurrence still runs the product: wasted
            // work only when the sector is smaller than the block space)
            ++matvecs;
            if ((e = mark()) != cudaSuccess)
                return e;
            if (!f32) {
                k_dd_to_f64<<<vgrid, 256, 0, st>>>(Vjh, Vjl, V64, blk); count_launch();
            }
            e = launch_matvec_v(ov, gv, iv, track, f32 ? (const void *)Vjh : (const void *)V64,
                                f32 ? (void *)W32 : (void *)W64, P, f32 ? ED_F32 : ED_F64, tuned, st);
            if (e != cudaSuccess)
                return e;
            if ((e = mark()) != cudaSuccess)
                return e;
            const int nm = j ? 2 : 1;
            launch_gram<P>(nm, yk, Vjh, Vjl, Vph, Vpl, Yh, nullptr, n, grid, part, tickets, C, stop, st);
            k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 0, stop, flags + 1); count_launch();
            launch_update<P>(nm, yk, Vjh, Vjl, Vph, Vpl, Yh, nullptr, C, Wh, Wl, n, rgrid, part, tickets + 1,
                             reorth ? nullptr : G, stop, st);
            if (reorth) {  // against every kept block, block modified Gram-Schmidt, twice
                for (int rep = 0; rep < 2; ++rep)
                    for (int i = 0; i <= j; ++i) {
                        launch_gram<P>(1, 2, bh(i), bl(i), nullptr, nullptr, Wh, Wl, n, grid, part, tickets, C,
                                       stop, st);
                        launch_update<P>(1, 2, bh(i), bl(i), nullptr, nullptr, Wh, Wl, C, Wh, Wl, n, rgrid, part,
                                         tickets + 1, nullptr, stop, st);
                    }
                launch_gram<P>(1, 2, Wh, Wl, nullptr, nullptr, Wh, Wl, n, grid, part, tickets, G, stop, st);
            }
            k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 1, stop, flags + 1); count_launch();
            qr(Wh, Wl, j);
        }
        return cudaGetLastError();
    };

    {
        cudaError_t e = pass(false);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;
        }
    }
    // m_eff = steps unless the recurrence stopped (k_bl_small wrote it)
    int me = 0;
    ED_BL_TRY(cudaMemcpyAsync(&me, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    ED_BL_TRY(cudaStreamSynchronize(st));
    if (me <= 0)
        return ED_ERR_INVALID_ARG;  // the start block has lower rank than nvec
    ED_BL_TRY(cudaMemcpyAsync(flags + 2, flags + 1, sizeof(int), cudaMemcpyDeviceToDevice, st));
    const int ne = std::max(n_eig, 1);
    k_band_eigs<P><<<ne, 32, 0, st>>>(A, B, flags + 1, eig, y, scr); count_launch();
    ED_BL_TRY(cudaGetLastError());
    std::vector<double> eh(ne);
    ED_BL_TRY(cudaMemcpyAsync(eh.data(), eig, ne * sizeof(double), cudaMemcpyDeviceToHost, st));
    *res_out = 0.0;
    if (values_only) {
        // residual estimate |B_{m+1} s_m| of the lowest Ritz pair (s_m: the
        // eigenvector's entries on the last block)
        std::vector<double> Bm((size_t)P * P), ym(P);
        ED_BL_TRY(cudaMemcpyAsync(Bm.data(), B + (size_t)me * P * P, P * P * sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
        ED_BL_TRY(cudaMemcpyAsync(ym.data(), y + (size_t)(me - 1) * P, P * sizeof(double),
                                  cudaMemcpyDeviceToHost, st));
        ED_BL_TRY(cudaStreamSynchronize(st));
        double r2 = 0.0;
        for (int a = 0; a < P; ++a) {
            double t = 0.0;
            for (int c = 0; c < P; ++c)
                t += Bm[a * P + c] * ym[c];
            r2 += t * t;
        }
        *res_out = me < steps ? 0.0 : sqrt(r2);  // a stopped recurrence spans an invariant subspace
    } else if (reorth) {
        for (int j = 0; j < me; ++j) {
            k_dd_ritz_acc<P><<<vgrid, 256, 0, st>>>(ph, pl, bh(j), bl(j), y, j, n, j == 0, flags + 2);
            count_launch();
        }
    } else {
        cudaError_t e = pass(true);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;
        }
    }
    if (!values_only) {
        k_dd_to_f64<<<vgrid, 256, 0, st>>>(ph, pl, psi_out, n); count_launch();
    }
    ED_BL_TRY(cudaStreamSynchronize(st));
    double ms = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, ev[i], ev[i + 1]) == cudaSuccess)
            ms += t;
    }
    for (cudaEvent_t e : ev)
        cudaEventDestroy(e);
    if (eigs_out)
        for (int k = 0; k < n_eig; ++k)
            eigs_out[k] = eh[k];
    *steps_out = me;
    *matvecs_out = matvecs;
    *ritz_out = eh[0];
    *mv_ms_out = ms;
    return ED_OK;
}

}  // namespace
}  // namespace edk

extern "C" ed_status ed_lanczos_block(const ed_operator *op, const ed_basis *b, const void *d_x0, int nvec,
                                      int steps, int mode, int n_eig, double *eigs_out, double *e0_out,
                                      void *d_vec_out, ed_lanczos_info *info, void *stream)
{
    using namespace edk;
    if (!op || !b || !d_x0 || steps < 1 || steps > 10000)
        return ED_ERR_INVALID_ARG;
    if (nvec != 2 && nvec != 4 && nvec != 8 && nvec != 16)
        return ED_ERR_INVALID_ARG;
    const bool reorth = (mode & ED_LANCZOS_REORTH) != 0;
    const bool values_only = (mode & ED_LANCZOS_VALUES_ONLY) != 0;
    mode &= ~(ED_LANCZOS_REORTH | ED_LANCZOS_VALUES_ONLY);
    if (values_only && d_vec_out)
        return ED_ERR_INVALID_ARG;
    if (mode != ED_LANCZOS_F64 && mode != ED_LANCZOS_F32_MATVEC)
        return ED_ERR_INVALID_ARG;
    if (n_eig < 0 || n_eig > nvec * steps || (n_eig > 0 && !eigs_out))
        return ED_ERR_INVALID_ARG;
    if (b->dim < (uint64_t)nvec || (((uintptr_t)d_x0 | (uintptr_t)d_vec_out) & 15))
        return ED_ERR_INVALID_ARG;
    const ed_status st0 = check_pair(op, b);
    if (st0 != ED_OK)
        return st0;
    if (!(b->real_chars && op->real))
        return ED_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const bool f32 = mode == ED_LANCZOS_F32_MATVEC;
    if (reorth) {  // every block is kept: it must fit in half of the free memory
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        free_b += ws_cached_bytes();
        if ((double)(steps + 1) * (double)b->dim * nvec * sizeof(double) > 0.5 * (double)free_b)
            return ED_ERR_UNSUPPORTED;
    }
    double *psi = nullptr;
    if (ws_alloc((void **)&psi, (size_t)b->dim * sizeof(double), st) != cudaSuccess) {
        (void)cudaGetLastError();
        return ED_ERR_OOM;
    }
    int steps_done = 0, matvecs = 0;
    double ritz = 0.0, mv_ms = 0.0, res_est = 0.0;
    ed_status r = ED_ERR_INVALID_ARG;
    const double *x0 = (const double *)d_x0;
    switch (nvec) {
    case 2: r = run_block<2>(op, b, x0, steps, f32, reorth, values_only, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &res_est, &mv_ms, st); break;
    case 4: r = run_block<4>(op, b, x0, steps, f32, reorth, values_only, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &res_est, &mv_ms, st); break;
    case 8: r = run_block<8>(op, b, x0, steps, f32, reorth, values_only, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &res_est, &mv_ms, st); break;
    case 16: r = run_block<16>(op, b, x0, steps, f32, reorth, values_only, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &res_est, &mv_ms, st); break;
    }
    // fp64 refinement of the Ritz vector: a short single-vector fp64 Lanczos
    // run from it, whose fp64 Rayleigh quotient and residual are returned
    ed_lanczos_info ri{};
    double e0 = 0.0;
    if (r == ED_OK && values_only) {
        e0 = ritz;
        ri.residual = res_est;
    } else if (r == ED_OK) {
        r = ed_lanczos(op, b, psi, 6, ED_LANCZOS_F64, &e0, d_vec_out, &ri, stream);
    }
    ws_free(psi, st);
    if (r != ED_OK)
        return r;
    if (e0_out)
        *e0_out = e0;
    if (info) {
        info->steps = steps_done;
        info->matvecs = matvecs + ri.matvecs;
        info->ritz = ritz;
        info->e0 = e0;
        info->residual = ri.residual;
        info->matvec_ms = mv_ms + ri.matvec_ms;
    }
    return ED_OK;
}
