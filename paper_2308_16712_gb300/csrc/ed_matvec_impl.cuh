// ed_matvec_impl.cuh -- the pull-style symmetry-adapted matvec kernel
// (Sec. "Matrix-vector product": y_i = sum_j H_ij x_j with getRow and
// stateToIndex), instantiated per precision in the ed_matvec_*.cu units.
//
// Work decomposition.  The grid is persistent; the basis is cut into tiles of
// R consecutive rows (R = 32, or fewer when rows can produce many terms), dealt
// round-robin to warps.  For each tile a warp works in three phases:
//  0. each row lane loads its row r and n(r), forms the diagonal from the
//     local configurations of every bond family (one word rotation and four
//     popcounts per family), counts its off-diagonal terms, and after a warp
//     scan writes the produced states into the warp's term list in shared
//     memory;
//  A. all 32 lanes take 32 terms at a time: the representative search runs in
//     lockstep over the group (mask reads are shared-memory broadcasts), then
//     each lane looks its representative up (hash index or prefix table) and
//     writes the found index and coefficient conj(h) chi sqrt(n'/n) back;
//  B. each row lane sums its own terms, in list order, gathering x at the
//     found indices, and writes y.
// The order of every sum is fixed: the result is deterministic, with no atomics.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "ed_kernels.cuh"

namespace edk {

constexpr int kMvThreads = 128;  // 4 warps per block
constexpr int kTermCap = 512;    // term slots per warp
// The register budget is left to the compiler: capping it for more resident
// warps cost more (spills, longer dependency chains) than it gained.

struct MatvecArgs {
    OpView op;
    GroupView g;
    IndexView ix;
    const void *x;
    void *y;
    int nvec;
    int tile_rows;  // rows per tile: tile_rows * op.max_terms <= kTermCap
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

// coefficient type of a term
template <typename T, bool kC> using CoefT = typename ValT<T, kC>::type;

// Per-warp term list: slot A holds the produced state, then the found index;
// slot B holds (matrix entry | row << 16), then the coefficient.
template <typename W, typename T, bool kC>
__host__ __device__ inline size_t warp_slots_bytes()
{
    const size_t a = sizeof(W) > 4 ? sizeof(W) : 4;
    const size_t b = sizeof(CoefT<T, kC>) > 4 ? sizeof(CoefT<T, kC>) : 4;
    return align16((size_t)kTermCap * a) + align16((size_t)kTermCap * b) + align16(32 * sizeof(T));
}

// Shared-memory layout: masks | chi | families | matrices | offmask | coset kinds | sqrt tables | warp slots
template <typename W, typename T, bool kC, bool kTrack, bool kFact>
__host__ __device__ inline void matvec_smem_layout(const GroupView &g, const OpView &op, size_t off[9])
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
    off[8] = off[7] + (size_t)(kMvThreads / 32) * warp_slots_bytes<W, T, kC>();
}

template <typename W, typename T, bool kC, bool kTrack, bool kFact>
__host__ __device__ inline size_t matvec_smem_bytes(const GroupView &g, const OpView &op)
{
    size_t off[9];
    matvec_smem_layout<W, T, kC, kTrack, kFact>(g, op, off);
    return off[8];
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
    using C = CoefT<T, kC>;
    extern __shared__ __align__(16) unsigned char smem[];
    size_t off[9];
    matvec_smem_layout<W, T, kC, kTrack, kFact>(a.g, a.op, off);
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

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    unsigned char *wbase = smem + off[7] + (size_t)wib * warp_slots_bytes<W, T, kC>();
    constexpr size_t kSlotA = sizeof(W) > 4 ? sizeof(W) : 4;
    constexpr size_t kSlotB = sizeof(C) > 4 ? sizeof(C) : 4;
    unsigned char *slotA = wbase;
    unsigned char *slotB = wbase + align16((size_t)kTermCap * kSlotA);
    T *row_rinv = reinterpret_cast<T *>(slotB + align16((size_t)kTermCap * kSlotB));
    auto a_state = [&](int k) -> W & { return *reinterpret_cast<W *>(slotA + (size_t)k * kSlotA); };
    auto a_index = [&](int k) -> uint32_t & { return *reinterpret_cast<uint32_t *>(slotA + (size_t)k * kSlotA); };
    auto b_meta = [&](int k) -> uint32_t & { return *reinterpret_cast<uint32_t *>(slotB + (size_t)k * kSlotB); };
    auto b_coef = [&](int k) -> C & { return *reinterpret_cast<C *>(slotB + (size_t)k * kSlotB); };

    const V *__restrict__ x = reinterpret_cast<const V *>(a.x);
    V *__restrict__ y = reinterpret_cast<V *>(a.y);
    const int nvec = a.nvec;
    const int n_fam = a.op.n_fam;
    const int n = a.g.n_sites;
    const uint64_t dim = a.ix.dim;
    const W full = (W)a.g.full;
    const unsigned kAll = 0xffffffffu;
    const int R = a.tile_rows;
    const bool packed = a.ix.keys != nullptr;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t ntiles = (dim + R - 1) / R;

    for (uint64_t tile = gw; tile < ntiles; tile += nw) {
        // ---- phase 0: rows, diagonal, term lists ---------------------------------
        const uint64_t row = tile * (uint64_t)R + lane;
        const bool live = lane < R && row < dim;
        W r = 0;
        T rinv = 0;
        Cplx<T> diag = {T(0), T(0)};
        int cnt = 0;
        if (live) {
            uint32_t nr;
            if (packed) {
                const uint64_t k = __ldcs(a.ix.keys + row);  // streamed once: evict first
                r = (W)(k >> 16);
                nr = (uint32_t)(k & 0xffff);
            } else {
                r = (W)__ldg(a.ix.states + row);
                nr = __ldg(a.ix.norms + row);
            }
            rinv = sm_isq[nr];
            for (int q = 0; q < n_fam; ++q) {
                const OpFamily fm = sm_fam[q];
                const W tq = rot_down(r, (int)fm.delta, n, full);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int pc = popc(config_mask(r, tq, (W)fm.mask, cc));
                    const Cplx<T> h = sm_mats[fm.mat * 16 + cc * 5];
                    diag.re += h.re * (T)pc;
                    diag.im += h.im * (T)pc;
                    cnt += pc * __popc((unsigned)sm_off[fm.mat * 4 + cc]);
                }
            }
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(kAll, incl, o);
            if (lane >= o)
                incl += v;
        }
        const int first = incl - cnt;
        const int total = __shfl_sync(kAll, incl, 31);
        if (live) {
            row_rinv[lane] = rinv;
            int k = first;
            for (int q = 0; q < n_fam; ++q) {
                const OpFamily fm = sm_fam[q];
                const int delta = (int)fm.delta;
                const W tq = rot_down(r, delta, n, full);
                for (int cc = 0; cc < 4; ++cc) {
                    const uint32_t targets = sm_off[fm.mat * 4 + cc];
                    if (!targets)
                        continue;
                    W bits = config_mask(r, tq, (W)fm.mask, cc);
                    while (bits) {
                        const int i = lowest_bit(bits);
                        bits &= bits - 1;
                        int j = i + delta;
                        j -= j >= n ? n : 0;
                        uint32_t tg = targets;
                        while (tg) {
                            const int cp = __ffs(tg) - 1;
                            tg &= tg - 1;
                            const int fl = cc ^ cp;
                            a_state(k) = r ^ (W((fl >> 1) & 1) << i) ^ (W(fl & 1) << j);
                            b_meta(k) = (uint32_t)(fm.mat * 16 + cp * 4 + cc) | ((uint32_t)lane << 16);
                            ++k;
                        }
                    }
                }
            }
        }
        __syncwarp();

        // ---- phase A: search and look up 32 terms at a time ----------------------
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int k = b0 + lane;
            const bool valid = k < total;
            const W s = valid ? a_state(k) : W(0);
            W best;
            int gbest = 0;
            if (kFact) {
                if (kTrack)
                    rep_search_fact<W, true>(s, sm_kind, sm_masks, a.g.n_cos, a.g.rot_L, a.g.rot_d, n,
                                             a.g.n_perm, a.g.flip, full, best, gbest);
                else
                    best = rep_min_fact<W>(s, sm_kind, sm_masks, a.g.n_cos, a.g.rot_L, a.g.rot_d, n,
                                           a.g.flip, full);
            } else {
                rep_search<W, kTrack>(s, sm_masks, a.g.n_perm, a.g.flip, full, best, gbest);
            }
            if (valid) {
                const uint32_t meta = b_meta(k);
                uint32_t jj = 0, nj = 0;
                bool found;
                if (a.ix.htab) {
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
                C coef{};
                if (found) {
                    const T ratio = sm_sq[nj] * row_rinv[meta >> 16];
                    const Cplx<T> h = sm_mats[meta & 0xffff];
                    Cplx<T> cf = {h.re * ratio, -h.im * ratio};  // conj(h) sqrt(n'/n)
                    if (kTrack)
                        cf = cmul(cf, sm_chi[gbest]);
                    if constexpr (kC)
                        coef = cf;
                    else
                        coef = cf.re;
                }
                a_index(k) = found ? jj : 0xffffffffu;
                b_coef(k) = coef;
            }
        }
        __syncwarp();

        // ---- phase B: each row lane sums its terms in list order -----------------
        if (live) {
            V acc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                if (v < nvec) {
                    const V xv = x[row * nvec + v];
                    if constexpr (kC)
                        acc[v] = cmul(conjc(diag), xv);
                    else
                        acc[v] = diag.re * xv;
                }
            }
            for (int k = first; k < first + cnt; ++k) {
                const uint32_t j = a_index(k);
                if (j == 0xffffffffu)
                    continue;
                const C cf = b_coef(k);
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (v < nvec) {
                        const V xv = x[(uint64_t)j * nvec + v];
                        if constexpr (kC) {
                            const Cplx<T> p = cmul(cf, xv);
                            acc[v].re += p.re;
                            acc[v].im += p.im;
                        } else {
                            acc[v] += cf * xv;
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v)
                if (v < nvec)
                    store_cs(y + row * nvec + v, acc[v]);
        }
        __syncwarp();
    }
}

template <typename W, typename T, bool kC, bool kTrack, bool kFact, int NV>
cudaError_t matvec_launch(const MatvecArgs &a, cudaStream_t stream)
{
    auto kern = k_matvec<W, T, kC, kTrack, kFact, NV>;
    const size_t smem = matvec_smem_bytes<W, T, kC, kTrack, kFact>(a.g, a.op);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMvThreads, smem);
    if (e != cudaSuccess)
        return e;
    MatvecArgs args = a;
    args.tile_rows = std::max(1, std::min(32, kTermCap / std::max(1, a.op.max_terms)));
    const uint64_t tiles = (a.ix.dim + args.tile_rows - 1) / args.tile_rows;
    const uint64_t blocks_needed = (tiles + (kMvThreads / 32) - 1) / (kMvThreads / 32);
    const int grid = (int)std::min<uint64_t>(blocks_needed, (uint64_t)sms * std::max(per_sm, 1));
    kern<<<std::max(grid, 1), kMvThreads, smem, stream>>>(args); count_launch();
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
