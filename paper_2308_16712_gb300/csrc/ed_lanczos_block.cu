// ed_lanczos_block.cu -- block Lanczos on p = nvec vectors at once, the
// consumer of the interleaved block product (Background: Krylov methods
// consume hundreds of products; one representative search and index lookup per
// matrix element serves all p columns of a block).
//
// Recurrence (real sectors; blocks are [dim][p] fp64, interleaved like the
// product's vectors):  V_1 R_0 = X0 (QR),
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
// merges, so both passes reproduce every coefficient bit for bit.
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

template <typename T> __device__ __forceinline__ double ld_up(const T *p) { return (double)*p; }

// Stage rows [r0, r0 + kTileRows) of a [n][P] block into shared memory
// (zeros past n); coalesced: consecutive threads read consecutive elements.
template <int P, typename T>
__device__ __forceinline__ void stage(double *sm, const T *g, uint64_t r0, uint64_t n)
{
    const uint64_t base = r0 * P;
    const uint64_t lim = n * P;
    for (int e = threadIdx.x; e < kTileRows * P; e += blockDim.x) {
        const uint64_t gi = base + (uint64_t)e;
        sm[e] = gi < lim ? ld_up(g + gi) : 0.0;
    }
}

// Gram of NM fp64 blocks X_m against Y: out[m][a][b] = sum_i X_m[i][a] Y[i][b].
// A thread owns entries e = tid, tid + 256, ...; per tile it sums the tile's
// rows in a register and adds that into a compensated running sum.
template <int P, int NM, typename YT>
__global__ void __launch_bounds__(kBlThreads) k_bl_gram(const double *X0, const double *X1, const YT *Y,
                                                        uint64_t n, double2 *part, unsigned int *ticket,
                                                        double *out, const int *stop)
{
    if (*stop)
        return;
    __shared__ double sx[NM][kTileRows * P];
    __shared__ double sy[kTileRows * P];
    constexpr int E = NM * P * P;
    constexpr int EPT = (E + kBlThreads - 1) / kBlThreads;
    KS acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q)
        acc[q] = KS{0.0, 0.0};
    const uint64_t tiles = (n + kTileRows - 1) / kTileRows;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t r0 = t * kTileRows;
        stage<P>(sx[0], X0, r0, n);
        if (NM > 1)
            stage<P>(sx[NM - 1], X1, r0, n);
        stage<P>(sy, Y, r0, n);
        __syncthreads();
#pragma unroll
        for (int q = 0; q < EPT; ++q) {
            const int e = threadIdx.x + q * kBlThreads;
            if (e < E) {
                const int m = e / (P * P), a = (e / P) % P, b = e % P;
                double s = 0.0;
#pragma unroll 8
                for (int r = 0; r < kTileRows; ++r)
                    s = fma(sx[m][r * P + a], sy[r * P + b], s);
                acc[q] = ks_add(acc[q], s);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * kBlThreads;
        if (e < E)
            part[(size_t)blockIdx.x * E + e] = make_double2(acc[q].s, acc[q].c);
    }
    if (last_block(ticket))
        merge_partials(part, E, out, ticket);
}

// W = Y - X0 C0 - X1 C1 (C read from device memory, P x P row-major: W[i][b]
// -= sum_a X[i][a] C[a][b]); W may alias X1 (a tile is read completely before
// it is written).  With G: Gram partials of W^T W, merged into G by the last block.
template <int P, int NM, typename YT>
__global__ void __launch_bounds__(kBlThreads) k_bl_update(const double *X0, const double *X1, const YT *Y,
                                                          const double *C, double *W, uint64_t n,
                                                          double2 *part, unsigned int *ticket, double *G,
                                                          const int *stop)
{
    if (*stop)
        return;
    __shared__ double sx[NM][kTileRows * P];
    __shared__ double sw[kTileRows * P];
    __shared__ double sc[NM * P * P];
    for (int e = threadIdx.x; e < NM * P * P; e += blockDim.x)
        sc[e] = C[e];
    constexpr int E = P * P;
    constexpr int EPT = (E + kBlThreads - 1) / kBlThreads;
    KS acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q)
        acc[q] = KS{0.0, 0.0};
    const uint64_t tiles = (n + kTileRows - 1) / kTileRows;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t r0 = t * kTileRows;
        stage<P>(sx[0], X0, r0, n);
        if (NM > 1)
            stage<P>(sx[NM - 1], X1, r0, n);
        stage<P>(sw, Y, r0, n);
        __syncthreads();
        for (int e = threadIdx.x; e < kTileRows * P; e += blockDim.x) {
            const int r = e / P, b = e % P;
            double w = sw[e];
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
                for (int a = 0; a < P; ++a)
                    w = fma(-sx[m][r * P + a], sc[m * P * P + a * P + b], w);
            sw[e] = w;
        }
        __syncthreads();
        const uint64_t lim = n * P;
        for (int e = threadIdx.x; e < kTileRows * P; e += blockDim.x) {
            const uint64_t gi = r0 * P + (uint64_t)e;
            if (gi < lim)
                W[gi] = sw[e];
        }
        if (G) {
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int e = threadIdx.x + q * kBlThreads;
                if (e < E) {
                    const int a = e / P, b = e % P;
                    double s = 0.0;
#pragma unroll 8
                    for (int r = 0; r < kTileRows; ++r)
                        s = fma(sw[r * P + a], sw[r * P + b], s);
                    acc[q] = ks_add(acc[q], s);
                }
            }
        }
        __syncthreads();
    }
    if (!G)
        return;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * kBlThreads;
        if (e < E)
            part[(size_t)blockIdx.x * E + e] = make_double2(acc[q].s, acc[q].c);
    }
    if (last_block(ticket))
        merge_partials(part, E, G, ticket);
}

// Z = W R1i (R1i upper triangular, row-major); kApply = false: Gram partials
// of Z^T Z merged into G2; kApply = true: V = Z R2i written over W, with its
// fp32 copy V32 (may be null).  Z is formed identically in both.
template <int P, bool kApply>
__global__ void __launch_bounds__(kBlThreads) k_bl_qr(double *W, const double *R1i, const double *R2i,
                                                      float *V32, uint64_t n, double2 *part,
                                                      unsigned int *ticket, double *G2, const int *stop)
{
    if (*stop)
        return;
    __shared__ double sw[kTileRows * P];
    __shared__ double sz[kTileRows * P];
    __shared__ double s1[P * P], s2[P * P];
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        s1[e] = R1i[e];
        if (kApply)
            s2[e] = R2i[e];
    }
    constexpr int E = P * P;
    constexpr int EPT = (E + kBlThreads - 1) / kBlThreads;
    KS acc[EPT];
#pragma unroll
    for (int q = 0; q < EPT; ++q)
        acc[q] = KS{0.0, 0.0};
    const uint64_t tiles = (n + kTileRows - 1) / kTileRows;
    const uint64_t lim = n * P;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const uint64_t r0 = t * kTileRows;
        stage<P>(sw, W, r0, n);
        __syncthreads();
        for (int e = threadIdx.x; e < kTileRows * P; e += blockDim.x) {
            const int r = e / P, b = e % P;
            double z = 0.0;
            for (int a = 0; a <= b; ++a)
                z = fma(sw[r * P + a], s1[a * P + b], z);
            sz[e] = z;
        }
        __syncthreads();
        if (kApply) {
            for (int e = threadIdx.x; e < kTileRows * P; e += blockDim.x) {
                const int r = e / P, b = e % P;
                double v = 0.0;
                for (int a = 0; a <= b; ++a)
                    v = fma(sz[r * P + a], s2[a * P + b], v);
                const uint64_t gi = r0 * P + (uint64_t)e;
                if (gi < lim) {
                    W[gi] = v;
                    if (V32)
                        V32[gi] = (float)v;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < EPT; ++q) {
                const int e = threadIdx.x + q * kBlThreads;
                if (e < E) {
                    const int a = e / P, b = e % P;
                    double s = 0.0;
#pragma unroll 8
                    for (int r = 0; r < kTileRows; ++r)
                        s = fma(sz[r * P + a], sz[r * P + b], s);
                    acc[q] = ks_add(acc[q], s);
                }
            }
        }
        __syncthreads();
    }
    if (kApply)
        return;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
        const int e = threadIdx.x + q * kBlThreads;
        if (e < E)
            part[(size_t)blockIdx.x * E + e] = make_double2(acc[q].s, acc[q].c);
    }
    if (last_block(ticket))
        merge_partials(part, E, G2, ticket);
}

// psi (dim) += V_j s_j  (s_j = y[j P .. j P + P)), psi zeroed when first
template <int P>
__global__ void k_bl_ritz_acc(double *psi, const double *V, const double *y, int j, uint64_t n, int first,
                              const int *m_eff)
{
    if (j >= *m_eff)
        return;
    double c[P];
#pragma unroll
    for (int a = 0; a < P; ++a)
        c[a] = y[j * P + a];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        double acc = first ? 0.0 : psi[i];
#pragma unroll
        for (int a = 0; a < P; ++a)
            acc = fma(V[i * P + a], c[a], acc);
        psi[i] = acc;
    }
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

template <int P>
ed_status run_block(const ed_operator *op, const ed_basis *b, const double *x0, int steps, bool f32, bool reorth,
                    int n_eig, double *eigs_out, double *psi_out, int *steps_out, int *matvecs_out,
                    double *ritz_out, double *mv_ms_out, cudaStream_t st)
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
    const size_t blk = (size_t)n * P;

    Pool S(st);
    double *Vb[2] = {nullptr, nullptr}, *W64 = nullptr, *A = nullptr, *B = nullptr, *sm = nullptr;
    double *y = nullptr, *eig = nullptr, *scr = nullptr;
    float *V32 = nullptr, *W32 = nullptr;
    double2 *part = nullptr;
    unsigned int *tickets = nullptr;
    int *flags = nullptr;  // [0] stop, [1] m_eff (running), [2] m_eff of the main pass
    double *Vall = nullptr;  // every block (reorthogonalisation), steps + 1 of them
    if (reorth) {
        ED_BL_TRY(S.get(&Vall, (size_t)(steps + 1) * blk));
    } else {
        ED_BL_TRY(S.get(&Vb[0], blk));
        ED_BL_TRY(S.get(&Vb[1], blk));
    }
    if (f32) {
        ED_BL_TRY(S.get(&V32, blk));
        ED_BL_TRY(S.get(&W32, blk));
    } else {
        ED_BL_TRY(S.get(&W64, blk));
    }
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
    const ed_dtype dt = f32 ? ED_F32 : ED_F64;
    double *C = sm, *G = sm + 2 * P * P, *R1i = sm + 4 * P * P, *G2 = sm + 5 * P * P, *R2i = sm + 7 * P * P;
    int *stop = flags;

    // QR of the block in Vb[k] in place (Cholesky QR, twice); V32 refreshed
    auto qr_inplace = [&](double *Wb, int j) {
        k_bl_qr<P, false><<<grid, kBlThreads, 0, st>>>(Wb, R1i, nullptr, nullptr, n, part, tickets + 2, G2,
                                                       stop); count_launch();
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 2, stop, flags + 1); count_launch();
        k_bl_qr<P, true><<<grid, kBlThreads, 0, st>>>(Wb, R1i, R2i, V32, n, part, tickets + 2, nullptr,
                                                      stop); count_launch();
    };

    // One pass of `steps` block steps from x0.  With acc, psi += V_j s_j.
    auto pass = [&](bool acc) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
        if (e != cudaSuccess)
            return e;
        // start block: V_1 = QR(X0)
        if ((e = cudaMemcpyAsync(Vb[0], x0, blk * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        k_bl_gram<P, 1, double><<<grid, kBlThreads, 0, st>>>(Vb[0], nullptr, Vb[0], n, part, tickets, G,
                                                             stop); count_launch();
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, -1, 1, stop, flags + 1); count_launch();
        k_bl_qr<P, false><<<grid, kBlThreads, 0, st>>>(Vb[0], R1i, nullptr, nullptr, n, part, tickets + 2, G2,
                                                       stop); count_launch();
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, -1, 2, stop, flags + 1); count_launch();
        k_bl_qr<P, true><<<grid, kBlThreads, 0, st>>>(Vb[0], R1i, R2i, V32, n, part, tickets + 2, nullptr,
                                                      stop); count_launch();
        int cur = 0;
        for (int j = 0; j < steps; ++j) {
            double *V = Vb[cur], *Vp = Vb[cur ^ 1];
            if (acc) {
                k_bl_ritz_acc<P><<<grid, kBlThreads, 0, st>>>(psi_out, V, y, j, n, j == 0, flags + 2);
                count_launch();
            }
            // W = H V_j (stopped recurrences still run the product: it is
            // only skipped work for a sector smaller than the block space)
            ++matvecs;
            if ((e = mark()) != cudaSuccess)
                return e;
            e = launch_matvec(ov, gv, iv, track, f32 ? (const void *)V32 : (const void *)V,
                              f32 ? (void *)W32 : (void *)W64, P, dt, st);
            if (e != cudaSuccess)
                return e;
            if ((e = mark()) != cudaSuccess)
                return e;
            if (f32) {
                if (j == 0)
                    k_bl_gram<P, 1, float><<<grid, kBlThreads, 0, st>>>(V, nullptr, W32, n, part, tickets, C,
                                                                        stop);
                else
                    k_bl_gram<P, 2, float><<<grid, kBlThreads, 0, st>>>(V, Vp, W32, n, part, tickets, C, stop);
                count_launch();
                k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 0, stop, flags + 1); count_launch();
                if (j == 0)
                    k_bl_update<P, 1, float><<<grid, kBlThreads, 0, st>>>(V, nullptr, W32, C, Vp, n, part,
                                                                          tickets + 1, G, stop);
                else
                    k_bl_update<P, 2, float><<<grid, kBlThreads, 0, st>>>(V, Vp, W32, C, Vp, n, part,
                                                                          tickets + 1, G, stop);
                count_launch();
            } else {
                if (j == 0)
                    k_bl_gram<P, 1, double><<<grid, kBlThreads, 0, st>>>(V, nullptr, W64, n, part, tickets, C,
                                                                         stop);
                else
                    k_bl_gram<P, 2, double><<<grid, kBlThreads, 0, st>>>(V, Vp, W64, n, part, tickets, C,
                                                                         stop);
                count_launch();
                k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 0, stop, flags + 1); count_launch();
                if (j == 0)
                    k_bl_update<P, 1, double><<<grid, kBlThreads, 0, st>>>(V, nullptr, W64, C, Vp, n, part,
                                                                           tickets + 1, G, stop);
                else
                    k_bl_update<P, 2, double><<<grid, kBlThreads, 0, st>>>(V, Vp, W64, C, Vp, n, part,
                                                                           tickets + 1, G, stop);
                count_launch();
            }
            k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 1, stop, flags + 1); count_launch();
            qr_inplace(Vp, j);  // V_{j+1} in the buffer of V_{j-1}
            cur ^= 1;
        }
        return cudaGetLastError();
    };

    // With every block kept: W is orthogonalised against all earlier blocks
    // (block modified Gram-Schmidt, twice) and the Ritz vector is combined
    // from the kept blocks.
    auto pass_store = [&]() -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(flags, 0, 2 * sizeof(int), st);
        if (e != cudaSuccess)
            return e;
        if ((e = cudaMemcpyAsync(Vall, x0, blk * sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return e;
        k_bl_gram<P, 1, double><<<grid, kBlThreads, 0, st>>>(Vall, nullptr, Vall, n, part, tickets, G,
                                                             stop); count_launch();
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, -1, 1, stop, flags + 1); count_launch();
        k_bl_qr<P, false><<<grid, kBlThreads, 0, st>>>(Vall, R1i, nullptr, nullptr, n, part, tickets + 2, G2,
                                                       stop); count_launch();
        k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, -1, 2, stop, flags + 1); count_launch();
        k_bl_qr<P, true><<<grid, kBlThreads, 0, st>>>(Vall, R1i, R2i, V32, n, part, tickets + 2, nullptr,
                                                      stop); count_launch();
        for (int j = 0; j < steps; ++j) {
            double *V = Vall + (size_t)j * blk, *Vp = j ? V - blk : nullptr, *Wn = V + blk;
            ++matvecs;
            if ((e = mark()) != cudaSuccess)
                return e;
            e = launch_matvec(ov, gv, iv, track, f32 ? (const void *)V32 : (const void *)V,
                              f32 ? (void *)W32 : (void *)W64, P, dt, st);
            if (e != cudaSuccess)
                return e;
            if ((e = mark()) != cudaSuccess)
                return e;
            if (f32) {
                if (j == 0)
                    k_bl_gram<P, 1, float><<<grid, kBlThreads, 0, st>>>(V, nullptr, W32, n, part, tickets, C,
                                                                        stop);
                else
                    k_bl_gram<P, 2, float><<<grid, kBlThreads, 0, st>>>(V, Vp, W32, n, part, tickets, C, stop);
                count_launch();
                k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 0, stop, flags + 1); count_launch();
                if (j == 0)
                    k_bl_update<P, 1, float><<<grid, kBlThreads, 0, st>>>(V, nullptr, W32, C, Wn, n, part,
                                                                          tickets + 1, nullptr, stop);
                else
                    k_bl_update<P, 2, float><<<grid, kBlThreads, 0, st>>>(V, Vp, W32, C, Wn, n, part,
                                                                          tickets + 1, nullptr, stop);
            } else {
                if (j == 0)
                    k_bl_gram<P, 1, double><<<grid, kBlThreads, 0, st>>>(V, nullptr, W64, n, part, tickets, C,
                                                                         stop);
                else
                    k_bl_gram<P, 2, double><<<grid, kBlThreads, 0, st>>>(V, Vp, W64, n, part, tickets, C,
                                                                         stop);
                count_launch();
                k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 0, stop, flags + 1); count_launch();
                if (j == 0)
                    k_bl_update<P, 1, double><<<grid, kBlThreads, 0, st>>>(V, nullptr, W64, C, Wn, n, part,
                                                                           tickets + 1, nullptr, stop);
                else
                    k_bl_update<P, 2, double><<<grid, kBlThreads, 0, st>>>(V, Vp, W64, C, Wn, n, part,
                                                                           tickets + 1, nullptr, stop);
            }
            count_launch();
            for (int rep = 0; rep < 2; ++rep)
                for (int i = 0; i <= j; ++i) {
                    const double *Vi = Vall + (size_t)i * blk;
                    k_bl_gram<P, 1, double><<<grid, kBlThreads, 0, st>>>(Vi, nullptr, Wn, n, part, tickets, C,
                                                                         stop); count_launch();
                    k_bl_update<P, 1, double><<<grid, kBlThreads, 0, st>>>(Vi, nullptr, Wn, C, Wn, n, part,
                                                                           tickets + 1, nullptr, stop);
                    count_launch();
                }
            k_bl_gram<P, 1, double><<<grid, kBlThreads, 0, st>>>(Wn, nullptr, Wn, n, part, tickets, G, stop);
            count_launch();
            k_bl_small<P><<<1, 32, 0, st>>>(sm, A, B, j, 1, stop, flags + 1); count_launch();
            qr_inplace(Wn, j);
        }
        return cudaGetLastError();
    };

    // main pass, then the projected problem
    {
        cudaError_t e = reorth ? pass_store() : pass(false);
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
    int *d_me = flags + 1;
    k_band_eigs<P><<<ne, 32, 0, st>>>(A, B, d_me, eig, y, scr); count_launch();
    ED_BL_TRY(cudaGetLastError());
    std::vector<double> eh(ne);
    ED_BL_TRY(cudaMemcpyAsync(eh.data(), eig, ne * sizeof(double), cudaMemcpyDeviceToHost, st));
    // Ritz vector of the lowest: from the kept blocks, or by a second,
    // bit-identical pass
    if (reorth) {
        for (int j = 0; j < me; ++j) {
            k_bl_ritz_acc<P><<<grid, kBlThreads, 0, st>>>(psi_out, Vall + (size_t)j * blk, y, j, n, j == 0,
                                                          flags + 2);
            count_launch();
        }
    } else {
        cudaError_t e = pass(true);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;
        }
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
    mode &= ~ED_LANCZOS_REORTH;
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
        if ((double)(steps + 1) * (double)b->dim * nvec * sizeof(double) > 0.5 * (double)free_b)
            return ED_ERR_UNSUPPORTED;
    }
    double *psi = nullptr;
    if (ws_alloc((void **)&psi, (size_t)b->dim * sizeof(double), st) != cudaSuccess) {
        (void)cudaGetLastError();
        return ED_ERR_OOM;
    }
    int steps_done = 0, matvecs = 0;
    double ritz = 0.0, mv_ms = 0.0;
    ed_status r = ED_ERR_INVALID_ARG;
    const double *x0 = (const double *)d_x0;
    switch (nvec) {
    case 2: r = run_block<2>(op, b, x0, steps, f32, reorth, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &mv_ms, st); break;
    case 4: r = run_block<4>(op, b, x0, steps, f32, reorth, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &mv_ms, st); break;
    case 8: r = run_block<8>(op, b, x0, steps, f32, reorth, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &mv_ms, st); break;
    case 16: r = run_block<16>(op, b, x0, steps, f32, reorth, n_eig, eigs_out, psi, &steps_done, &matvecs, &ritz, &mv_ms, st); break;
    }
    // fp64 refinement of the Ritz vector: a short single-vector fp64 Lanczos
    // run from it, whose fp64 Rayleigh quotient and residual are returned
    ed_lanczos_info ri{};
    double e0 = 0.0;
    if (r == ED_OK)
        r = ed_lanczos(op, b, psi, 6, ED_LANCZOS_F64, &e0, d_vec_out, &ri, stream);
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
