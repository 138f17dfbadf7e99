// ed_matvec_impl.cuh -- the pull-style symmetry-adapted matvec kernel
// (Sec. "Matrix-vector product": y_i = sum_j H_ij x_j with getRow and
// stateToIndex), instantiated per precision in the ed_matvec_*.cu units.
//
// Work decomposition.  The grid is persistent; rows are dealt to warps in
// tiles of 32 (round-robin), and each warp hands its rows to its lanes on
// demand (ballot + popc), so a lane that finishes a row takes the next one
// without waiting for the others.
// A lane owns its row r: it loads r and n(r), forms the diagonal from the
// local configurations of every bond family (one word rotation and four
// popcounts per family), and then walks the off-diagonal terms of H|r> one at a
// time (bit by bit through the family masks).  All 32 lanes run the
// representative search of their current term in lockstep over the same group
// element (the mask reads are shared-memory broadcasts), then each lane looks
// the representative up in the sorted basis, gathers x at that index and
// accumulates in registers, in a fixed order: the result is deterministic and
// needs no atomics.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "ed_kernels.cuh"

namespace edk {

constexpr int kMvThreads = 256;
// The register budget is left to the compiler: capping it for more resident
// warps cost more (spills, longer dependency chains) than it gained.

struct MatvecArgs {
    OpView op;
    GroupView g;
    IndexView ix;
    const void *x;
    void *y;
    int nvec;
};

template <typename T, bool kC> struct ValT { using type = T; };
template <typename T> struct ValT<T, true> { using type = Cplx<T>; };

template <typename T> __device__ __forceinline__ Cplx<T> conjc(Cplx<T> a) { return {a.re, -a.im}; }

template <typename T> __device__ __forceinline__ Cplx<T> load_c(const double2 *p);
template <> __device__ __forceinline__ Cplx<double> load_c<double>(const double2 *p) { return {p->x, p->y}; }
template <typename T> __device__ __forceinline__ Cplx<T> load_cf(const float2 *p);
template <> __device__ __forceinline__ Cplx<float> load_cf<float>(const float2 *p) { return {p->x, p->y}; }

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// streaming stores of y (written once, not re-read by this kernel)
__device__ __forceinline__ void store_cs(float *p, float v) { __stcs(p, v); }
__device__ __forceinline__ void store_cs(double *p, double v) { __stcs(p, v); }
__device__ __forceinline__ void store_cs(Cplx<float> *p, Cplx<float> v)
{
    __stcs(reinterpret_cast<float2 *>(p), make_float2(v.re, v.im));
}
__device__ __forceinline__ void store_cs(Cplx<double> *p, Cplx<double> v)
{
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v.re, v.im));
}

// Whole rows of an interleaved [dim][nvec] block with nvec == NV: NV values
// by 16-byte loads and streaming 16-byte stores, for rows of a multiple of 16
// bytes (the block starts 16-byte aligned).  One gather instruction per 16
// bytes instead of one per value.
template <typename V, int NV>
constexpr bool kRowVec = (NV * sizeof(V)) % 16 == 0;

template <typename V, int NV>
__device__ __forceinline__ void load_row_v(const V *p, V (&out)[NV])
{
    constexpr int kW = (int)(NV * sizeof(V) / 16);
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
    uint4 w[kW];
#pragma unroll
    for (int k = 0; k < kW; ++k)
        w[k] = __ldg(q + k);
    memcpy(out, w, sizeof(w));
}

template <typename V, int NV>
__device__ __forceinline__ void store_row_v(V *p, const V (&in)[NV])
{
    constexpr int kW = (int)(NV * sizeof(V) / 16);
    uint4 w[kW];
    memcpy(w, in, sizeof(w));
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int k = 0; k < kW; ++k)
        __stcs(q + k, w[k]);
}

// Shared-memory layout: masks | chi | families | matrices | offmask | coset kinds | sqrt tables
template <typename W, typename T, bool kTrack, bool kFact>
__host__ __device__ inline void matvec_smem_layout(const GroupView &g, const OpView &op, size_t off[8])
{
    const int nm = kFact ? g.n_cos : g.n_perm;
    off[0] = 0;
    off[1] = align16(off[0] + (size_t)nm * kMaskStride * sizeof(W));
    off[2] = align16(off[1] + (kTrack ? (size_t)g.order * sizeof(Cplx<T>) : 0));
    off[3] = align16(off[2] + (size_t)op.n_fam * sizeof(OpFamily));
    off[4] = align16(off[3] + (size_t)op.n_mats * 16 * sizeof(Cplx<T>));
    off[5] = align16(off[4] + (size_t)op.n_mats * 4);
    off[6] = align16(off[5] + (kFact ? (size_t)g.n_cos : 0));
    off[7] = align16(off[6] + 2 * (size_t)(g.order + 1) * sizeof(T));
}

template <typename W, typename T, bool kTrack, bool kFact>
__host__ __device__ inline size_t matvec_smem_bytes(const GroupView &g, const OpView &op)
{
    size_t off[8];
    matvec_smem_layout<W, T, kTrack, kFact>(g, op, off);
    return off[7];
}

// bit i of the result = bit (i + delta) mod n of s  (0 < delta < n)
__device__ __forceinline__ uint32_t rot_down(uint32_t s, int delta, int n, uint32_t full)
{
    if (n == 32)
        return __funnelshift_r(s, s, delta);
    return ((s >> delta) | (s << (n - delta))) & full;
}
__device__ __forceinline__ uint64_t rot_down(uint64_t s, int delta, int n, uint64_t full)
{
    return ((s >> delta) | (s << (n - delta))) & full;
}

__device__ __forceinline__ int lowest_bit(uint32_t v) { return __ffs(v) - 1; }
__device__ __forceinline__ int lowest_bit(uint64_t v) { return __ffsll((long long)v) - 1; }
__device__ __forceinline__ int popc(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popc(uint64_t v) { return __popcll((long long)v); }

// Sites i of the family (mask M) whose bond (i, i+delta) is in local
// configuration c = 2 s_i + s_{i+delta}; t = rot_down(s, delta).
template <typename W>
__device__ __forceinline__ W config_mask(W s, W t, W M, int c)
{
    const W a = (c & 2) ? s : ~s;
    const W b = (c & 1) ? t : ~t;
    return a & b & M;
}

// min and max over the rotations of the n-bit word h (n <= 32).
// Rotation step 1 (every ring translation): the loop is unrolled over the 32
// possible amounts so that each rotation is one funnel shift by an immediate
// of the doubled word aligned to bit 32; amounts beyond n are skipped by a
// warp-uniform predicate.  Other steps use run-time shift amounts.
__device__ __forceinline__ void rot_minmax32(uint32_t h, int L, int d, int n, uint32_t full, uint32_t &mn,
                                             uint32_t &mx)
{
    uint32_t m0 = ~0u, m1 = ~0u, x0 = 0, x1 = 0;
    if (d == 1 && n == 32) {
#pragma unroll
        for (int b = 0; b < 32; b += 2) {
            const uint32_t q0 = __funnelshift_l(h, h, b);
            const uint32_t q1 = __funnelshift_l(h, h, b + 1);
            m0 = min(m0, q0);
            x0 = max(x0, q0);
            m1 = min(m1, q1);
            x1 = max(x1, q1);
        }
    } else if (d == 1) {
        // (h | h << n) << (32 - n) as a 64-bit word hi:lo; rotation by b is
        // bits [32 - b, 64 - b) masked to n bits
        const uint64_t e = ((uint64_t)h | ((uint64_t)h << n)) << (32 - n);
        const uint32_t lo = (uint32_t)e, hi = (uint32_t)(e >> 32);
#pragma unroll
        for (int b = 0; b < 32; b += 2) {
            if (b < L) {
                const uint32_t q0 = __funnelshift_rc(lo, hi, 32 - b) & full;  // clamps: b = 0 gives hi
                m0 = min(m0, q0);
                x0 = max(x0, q0);
            }
            if (b + 1 < L) {
                const uint32_t q1 = __funnelshift_r(lo, hi, 31 - b) & full;
                m1 = min(m1, q1);
                x1 = max(x1, q1);
            }
        }
    } else {
        const uint32_t lo = h | (h << n), hi = h >> (32 - n);
        for (int b = 0; b < L; ++b) {
            const uint32_t q = __funnelshift_rc(lo, hi, n - b * d) & full;
            m0 = min(m0, q);
            x0 = max(x0, q);
        }
    }
    mn = min(mn, min(m0, m1));
    mx = max(mx, max(x0, x1));
}

// Minimum over the factored group without tracking the minimiser: for every
// coset image h, the running min and max over its rotations; the spin-flipped
// candidates q ^ full have their minimum at full ^ max(q).
template <typename W>
__device__ __forceinline__ W rep_min_fact(W s, const uint8_t *kinds, const W *masks, int n_cos, int L,
                                          int d, int n, int flip, W full)
{
    W mn = ~W(0), mx = 0;
    for (int c = 0; c < n_cos; ++c) {
        const W h = coset_image(s, (int)kinds[c], masks + c * kMaskStride, n);
        if constexpr (sizeof(W) == 4) {
            rot_minmax32(h, L, d, n, full, mn, mx);
        } else {
            W q = h;
#pragma unroll 4
            for (int b = 0; b < L; ++b) {
                mn = min(mn, q);
                mx = max(mx, q);
                q = ((q << d) | (q >> (n - d))) & full;
            }
        }
    }
    return flip ? min(mn, (W)(mx ^ full)) : mn;
}

template <typename W, typename T, bool kC, bool kTrack, bool kFact, int NV>
__global__ void __launch_bounds__(kMvThreads) k_matvec(const MatvecArgs a)
{
    using V = typename ValT<T, kC>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    size_t off[8];
    matvec_smem_layout<W, T, kTrack, kFact>(a.g, a.op, off);
    W *sm_masks = reinterpret_cast<W *>(smem + off[0]);
    Cplx<T> *sm_chi = reinterpret_cast<Cplx<T> *>(smem + off[1]);
    OpFamily *sm_fam = reinterpret_cast<OpFamily *>(smem + off[2]);
    Cplx<T> *sm_mats = reinterpret_cast<Cplx<T> *>(smem + off[3]);
    uint8_t *sm_off = smem + off[4];
    uint8_t *sm_kind = smem + off[5];
    T *sm_sq = reinterpret_cast<T *>(smem + off[6]);     // sqrt(k), k = 0..order
    T *sm_isq = sm_sq + (a.g.order + 1);                  // 1/sqrt(k)

    {
        const int nm = kFact ? a.g.n_cos : a.g.n_perm;
        const W *gm;
        if (kFact)
            gm = sizeof(W) == 4 ? reinterpret_cast<const W *>(a.g.cos_masks32)
                                : reinterpret_cast<const W *>(a.g.cos_masks64);
        else
            gm = sizeof(W) == 4 ? reinterpret_cast<const W *>(a.g.masks32)
                                : reinterpret_cast<const W *>(a.g.masks64);
        for (int e = threadIdx.x; e < nm * kMaskStride; e += blockDim.x)
            sm_masks[e] = gm[e];
        if (kFact)
            for (int e = threadIdx.x; e < a.g.n_cos; e += blockDim.x)
                sm_kind[e] = a.g.cos_kind[e];
        if (kTrack) {
            const double2 *cd = kFact ? a.g.fchi : a.g.chi;
            const float2 *cf = kFact ? a.g.fchif : a.g.chif;
            for (int e = threadIdx.x; e < a.g.order; e += blockDim.x) {
                if constexpr (sizeof(T) == 8)
                    sm_chi[e] = load_c<T>(cd + e);
                else
                    sm_chi[e] = load_cf<T>(cf + e);
            }
        }
        for (int e = threadIdx.x; e < a.op.n_fam; e += blockDim.x)
            sm_fam[e] = a.op.fams[e];
        for (int e = threadIdx.x; e < a.op.n_mats * 16; e += blockDim.x) {
            if constexpr (sizeof(T) == 8)
                sm_mats[e] = load_c<T>(a.op.mats + e);
            else
                sm_mats[e] = load_cf<T>(a.op.matsf + e);
        }
        for (int e = threadIdx.x; e < a.op.n_mats * 4; e += blockDim.x)
            sm_off[e] = a.op.offmask[e];
        for (int e = threadIdx.x; e <= a.g.order; e += blockDim.x) {
            sm_sq[e] = sqrt((T)e);
            sm_isq[e] = e ? T(1) / sqrt((T)e) : T(0);
        }
    }
    __syncthreads();

    const V *__restrict__ x = reinterpret_cast<const V *>(a.x);
    V *__restrict__ y = reinterpret_cast<V *>(a.y);
    const int nvec = a.nvec;
    const int n_fam = a.op.n_fam;
    const int n = a.g.n_sites;
    const uint64_t dim = a.ix.dim;
    const W full = (W)a.g.full;
    const unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    // Rows are dealt in tiles of 32 consecutive rows, round-robin over the
    // warps of the grid: warp w takes tiles w, w + nw, w + 2 nw, ...  (the term
    // count of a row varies slowly along the sorted basis, so contiguous blocks
    // per warp would be unbalanced).  p counts the rows this warp has taken.
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    auto row_of = [&](uint64_t p) { return ((p >> 5) * nw + gw) * 32 + (p & 31); };
    uint64_t next = 0;  // warp-uniform
    const bool packed = a.ix.keys != nullptr;

    bool has = false;
    uint64_t row = 0;
    W r = 0, t = 0, fmask = 0, bits = 0, cur = 0;
    T rinv = 1;
    int f = 0, c = 0, i = 0, fdelta = 0, fmat = 0, amp = 0;
    uint32_t cpm = 0;
    V acc[NV];

    // next off-diagonal term of H|r> in (family, configuration, site, target) order
    auto advance = [&]() -> bool {
        while (true) {
            if (cpm) {
                const int cp = __ffs(cpm) - 1;
                cpm &= cpm - 1;
                const int fl = c ^ cp;
                int j = i + fdelta;
                j -= j >= n ? n : 0;
                cur = r ^ (W((fl >> 1) & 1) << i) ^ (W(fl & 1) << j);
                amp = fmat * 16 + cp * 4 + c;
                return true;
            }
            if (bits) {
                i = lowest_bit(bits);
                bits &= bits - 1;
                cpm = sm_off[fmat * 4 + c];
                continue;
            }
            if (++c == 4) {
                c = 0;
                if (++f >= n_fam)
                    return false;
                const OpFamily fm = sm_fam[f];
                fmask = (W)fm.mask;
                fmat = (int)fm.mat;
                fdelta = (int)fm.delta;
                t = rot_down(r, fdelta, n, full);
            }
            bits = sm_off[fmat * 4 + c] ? config_mask(r, t, fmask, c) : W(0);
        }
    };
    auto store_row = [&]() {
        if constexpr (kRowVec<V, NV>) {
            if (nvec == NV) {
                store_row_v<V, NV>(y + row * NV, acc);
                return;
            }
        }
#pragma unroll
        for (int v = 0; v < NV; ++v)
            if (v < nvec)
                store_cs(y + row * nvec + v, acc[v]);
    };

    bool rows_left = row_of(0) < dim;
    while (true) {
        unsigned need = __ballot_sync(kAll, !has);
        while (need != 0 && rows_left) {
            const uint64_t mine = row_of(next + __popc(need & lanes_below));
            next += __popc(need);
            if (!has && mine < dim) {
                row = mine;
                if (packed) {
                    const uint64_t k = __ldcs(a.ix.keys + row);  // streamed once: evict first
                    r = (W)(k >> 16);
                    rinv = sm_isq[k & 0xffff];
                } else {
                    r = (W)__ldg(a.ix.states + row);
                    rinv = sm_isq[__ldg(a.ix.norms + row)];
                }
                // diagonal: sum over families and configurations
                Cplx<T> d = {T(0), T(0)};
                for (int q = 0; q < n_fam; ++q) {
                    const OpFamily fm = sm_fam[q];
                    const W tq = rot_down(r, (int)fm.delta, n, full);
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const int cnt = popc(config_mask(r, tq, (W)fm.mask, cc));
                        const Cplx<T> h = sm_mats[fm.mat * 16 + cc * 5];
                        d.re += h.re * (T)cnt;
                        d.im += h.im * (T)cnt;
                    }
                }
                V xr[NV];
                if constexpr (kRowVec<V, NV>) {
                    if (nvec == NV)
                        load_row_v<V, NV>(x + row * NV, xr);
                    else
#pragma unroll
                        for (int v = 0; v < NV; ++v)
                            xr[v] = v < nvec ? x[row * nvec + v] : V{};
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        xr[v] = v < nvec ? x[row * nvec + v] : V{};
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (v < nvec) {
                        if constexpr (kC)
                            acc[v] = cmul(conjc(d), xr[v]);
                        else
                            acc[v] = d.re * xr[v];
                    }
                }
                // first family
                f = 0;
                c = -1;
                cpm = 0;
                bits = 0;
                {
                    const OpFamily fm = sm_fam[0];
                    fmask = (W)fm.mask;
                    fmat = (int)fm.mat;
                    fdelta = (int)fm.delta;
                    t = rot_down(r, fdelta, n, full);
                }
                if (advance())
                    has = true;
                else
                    store_row();
            }
            rows_left = row_of(next) < dim;
            need = __ballot_sync(kAll, !has);
        }
        if (need == kAll)
            break;  // no lane holds a row and none are left

        W best;
        int gbest = 0;
        const W s = has ? cur : W(0);
        if (kFact && a.g.prune && (sizeof(W) == 8 || kTrack)) {
            rep_search_rot1<W, kTrack>(s, sm_kind, sm_masks, a.g.n_cos, n, a.g.n_perm, a.g.flip, full, best,
                                       gbest);
        } else if (kFact) {
            if (kTrack)
                rep_search_fact<W, true>(s, sm_kind, sm_masks, a.g.n_cos, a.g.rot_L, a.g.rot_d, n,
                                         a.g.n_perm, a.g.flip, full, best, gbest);
            else
                best = rep_min_fact<W>(s, sm_kind, sm_masks, a.g.n_cos, a.g.rot_L, a.g.rot_d, n,
                                       a.g.flip, full);
        } else {
            rep_search<W, kTrack>(s, sm_masks, a.g.n_perm, a.g.flip, full, best, gbest);
        }

        if (has) {
            uint32_t jj = 0, nj = 0;
            bool found;
            if (a.ix.bkt) {
                found = find_bucketed((uint64_t)best, a.ix.bkt, a.ix.stash, a.ix.n_stash, n, a.ix.bbits,
                                      a.ix.brem, jj, nj);
            } else if (a.ix.htab) {
                found = find_hashed((uint64_t)best, a.ix, jj, nj);
            } else if (packed) {
                found = find_key((uint64_t)best, a.ix, jj, nj);
            } else {
                const int64_t j64 = find_index((uint64_t)best, a.ix);
                found = j64 >= 0;
                if (found) {
                    jj = (uint32_t)j64;
                    nj = __ldg(a.ix.norms + j64);
                }
            }
            if (found) {
                const uint64_t j = jj;
                const T ratio = sm_sq[nj] * rinv;
                const Cplx<T> h = sm_mats[amp];
                Cplx<T> coef = {h.re * ratio, -h.im * ratio};  // conj(h) sqrt(n'/n)
                if (kTrack)
                    coef = cmul(coef, sm_chi[gbest]);
                V xg[NV];
                if constexpr (kRowVec<V, NV>) {
                    if (nvec == NV)
                        load_row_v<V, NV>(x + j * NV, xg);
                    else
#pragma unroll
                        for (int v = 0; v < NV; ++v)
                            xg[v] = v < nvec ? x[j * nvec + v] : V{};
                } else {
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        xg[v] = v < nvec ? x[j * nvec + v] : V{};
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (v < nvec) {
                        const V xv = xg[v];
                        if constexpr (kC) {
                            const Cplx<T> p = cmul(coef, xv);
                            acc[v].re += p.re;
                            acc[v].im += p.im;
                        } else {
                            acc[v] += coef.re * xv;
                        }
                    }
                }
            }
            if (!advance()) {
                store_row();
                has = false;
            }
        }
    }
}

template <typename W, typename T, bool kC, bool kTrack, bool kFact, int NV>
cudaError_t matvec_launch(const MatvecArgs &a, cudaStream_t stream)
{
    auto kern = k_matvec<W, T, kC, kTrack, kFact, NV>;
    const size_t smem = matvec_smem_bytes<W, T, kTrack, kFact>(a.g, a.op);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMvThreads, smem);
    if (e != cudaSuccess)
        return e;
    const uint64_t warps_needed = (a.ix.dim + 31) / 32;
    const uint64_t blocks_needed = (warps_needed * 32 + kMvThreads - 1) / kMvThreads;
    const int grid = (int)std::min<uint64_t>(blocks_needed, (uint64_t)sms * std::max(per_sm, 1));
    kern<<<std::max(grid, 1), kMvThreads, smem, stream>>>(a); count_launch();
    return cudaGetLastError();
}

template <typename T, bool kC>
cudaError_t matvec_dispatch_prec(const MatvecArgs &a, bool track, cudaStream_t stream)
{
    const bool w32 = a.g.n_sites <= 32;
    const bool fact = a.g.fact != 0;
#define ED_MV_NV(W, TR, FA)                                                       \
    do {                                                                          \
        if (a.nvec == 1) return matvec_launch<W, T, kC, TR, FA, 1>(a, stream);    \
        if (a.nvec <= 4) return matvec_launch<W, T, kC, TR, FA, 4>(a, stream);    \
        if (a.nvec <= 8) return matvec_launch<W, T, kC, TR, FA, 8>(a, stream);    \
        return matvec_launch<W, T, kC, TR, FA, 16>(a, stream);                    \
    } while (0)
#define ED_MV_FA(W, TR)                  \
    do {                                 \
        if (fact) ED_MV_NV(W, TR, true); \
        ED_MV_NV(W, TR, false);          \
    } while (0)
    if (w32) {
        if (track) ED_MV_FA(uint32_t, true);
        ED_MV_FA(uint32_t, false);
    }
    if (track) ED_MV_FA(uint64_t, true);
    ED_MV_FA(uint64_t, false);
#undef ED_MV_FA
#undef ED_MV_NV
}

cudaError_t matvec_f64(const MatvecArgs &a, bool track, cudaStream_t s);
cudaError_t matvec_f32(const MatvecArgs &a, bool track, cudaStream_t s);
cudaError_t matvec_c128(const MatvecArgs &a, bool track, cudaStream_t s);
cudaError_t matvec_c64(const MatvecArgs &a, bool track, cudaStream_t s);

}  // namespace edk
