// ed_matvec_tp.cuh -- term-parallel form of the pull matvec (Sec. "Matrix-vector
// product": y_i = sum_j H_ij x_j through getRow and stateToIndex), for
// operators whose two-site terms only exchange antiparallel spins (every
// off-diagonal entry of each 4x4 matrix couples |01> and |10>: Heisenberg, XXZ,
// J1-J2 and any U(1)-conserving two-site coupling), for one vector per
// product or a real block of 8 interleaved vectors (the row value is then the
// block's row, and every step below works on it componentwise).
//
// Work decomposition.  The grid is persistent; a warp takes a tile of 32
// consecutive rows of one sector (tiles dealt round-robin over the warps).
// Each lane loads its row, forms the diagonal and counts the row's
// off-diagonal terms (antiparallel bonds of every family); a warp scan lays
// the tile's terms out flat.  The warp then works through the flat list 32
// terms at a time: lane l takes term l of the round, finds its row and the
// bond from the row's antiparallel-bond masks (the u-th set bit), runs the
// representative search and the index lookup, gathers x and forms
// conj(h) chi sqrt(n'/n) x.  A segmented scan over the lanes (segments = rows)
// sums the round's contributions of each row, and the last lane of a segment
// adds that sum to the row's accumulator in shared memory, which holds
// diag * x_row first.  Every lane runs a search in every round (instead of
// lanes idling while others start rows or walk their term lists), and the
// summation order depends only on the tile layout: deterministic, and
// identical for a sector alone or inside a batch of sectors.
#pragma once

#include <type_traits>

#include "ed_matvec_multi_impl.cuh"

namespace edk {

constexpr int kTpThreads = 256;
constexpr int kTpWarps = kTpThreads / 32;

template <int kSec>
struct TpArgs {
    OpView op;
    GroupView g;            // lattice permutations; flip and characters per sector
    int n_sectors;
    int max_order;          // largest expanded group order among the sectors
    uint64_t total_tiles;
    BatchCtl ctl;           // work queue, status word, gate (zero: static tiles, no wait)
    SectorDesc sec[kSec];   // read from the launch parameters (constant bank)
};

// per-warp scratch: the tile's rows
template <typename W, typename T, typename V>
struct TpWarp {
    V acc[32];          // row accumulators
    W r[32];            // row states
    T rinv[32];         // 1 / sqrt(n(row))
    uint32_t off[32];   // first flat term of each row
    uint8_t p2r[32];    // row whose terms start at lane p of the current round
};

// One-family operators: each warp lists its rows' terms in shared memory once
// per tile (site i, | 0x80 for configuration |10>), n_sites bytes per row.
__host__ __device__ inline int tp_term_stride(const GroupView &g, const OpView &op)
{
    return op.n_fam == 1 ? (g.n_sites + 7) & ~7 : 0;
}

template <typename W, typename T, typename V, bool kFact>
__host__ __device__ inline void tp_smem_layout(const GroupView &g, const OpView &op, int n_sectors,
                                               int max_order, size_t off[8])
{
    const int nm = kFact ? g.n_cos : g.n_perm;
    off[0] = 0;                                                                  // masks
    off[1] = align16(off[0] + (size_t)nm * kMaskStride * sizeof(W));             // families
    off[2] = align16(off[1] + (size_t)op.n_fam * sizeof(OpFamily));              // matrices
    off[3] = align16(off[2] + (size_t)op.n_mats * 16 * sizeof(Cplx<T>));         // offmask
    off[4] = align16(off[3] + (size_t)op.n_mats * 4);                            // coset kinds
    off[5] = align16(off[4] + (kFact ? (size_t)g.n_cos : 0));                    // sqrt tables
    off[6] = align16(off[5] + 2 * (size_t)(max_order + 1) * sizeof(T));          // (sectors: parameters)
    off[7] = off[6];                                                             // warps
    (void)n_sectors;
}

template <typename W, typename T, typename V>
__host__ __device__ inline size_t tp_terms_offset(size_t warps_off)
{
    return align16(warps_off + kTpWarps * sizeof(TpWarp<W, T, V>));
}

template <typename W, typename T, typename V, bool kFact>
__host__ __device__ inline size_t tp_smem_bytes(const GroupView &g, const OpView &op, int n_sectors,
                                                int max_order)
{
    size_t off[8];
    tp_smem_layout<W, T, V, kFact>(g, op, n_sectors, max_order, off);
    return tp_terms_offset<W, T, V>(off[7]) + (size_t)kTpWarps * 32 * tp_term_stride(g, op);
}

// position of the u-th set bit of b (u < popc(b)), branch-free halving
__device__ __forceinline__ int nth_set_bit(uint32_t b, int u)
{
    int pos = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int c = __popc(b & ((1u << w) - 1u));
        const bool hi = u >= c;
        u -= hi ? c : 0;
        b = hi ? b >> w : b;
        pos += hi ? w : 0;
    }
    return pos;
}
__device__ __forceinline__ int nth_set_bit(uint64_t b, int u)
{
    const int c = __popc((uint32_t)b);
    return u >= c ? 32 + nth_set_bit((uint32_t)(b >> 32), u - c) : nth_set_bit((uint32_t)b, u);
}

template <typename T> __device__ __forceinline__ T vzero() { return T(0); }
template <> __device__ __forceinline__ Cplx<float> vzero<Cplx<float>>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ Cplx<double> vzero<Cplx<double>>() { return {0.0, 0.0}; }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
template <typename T> __device__ __forceinline__ Cplx<T> vadd(Cplx<T> a, Cplx<T> b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ float vshfl_up(float v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double vshfl_up(double v, int o) { return __shfl_up_sync(0xffffffffu, v, o); }
template <typename T> __device__ __forceinline__ Cplx<T> vshfl_up(Cplx<T> v, int o)
{
    return {__shfl_up_sync(0xffffffffu, v.re, o), __shfl_up_sync(0xffffffffu, v.im, o)};
}

// NV interleaved vectors of a real block as one value: a row of the block.
// The segmented scan and the accumulators work on it componentwise; loads and
// stores move it 16 bytes at a time.
template <typename T, int NV>
struct __align__(16) VecN {
    T v[NV];
};
template <typename T, int NV>
__device__ __forceinline__ VecN<T, NV> vadd(const VecN<T, NV> &a, const VecN<T, NV> &b)
{
    VecN<T, NV> r;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        r.v[k] = a.v[k] + b.v[k];
    return r;
}
template <typename T, int NV>
__device__ __forceinline__ VecN<T, NV> vshfl_up(const VecN<T, NV> &a, int o)
{
    VecN<T, NV> r;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        r.v[k] = __shfl_up_sync(0xffffffffu, a.v[k], o);
    return r;
}
template <typename T, int NV>
__device__ __forceinline__ VecN<T, NV> operator*(T s, const VecN<T, NV> &a)
{
    VecN<T, NV> r;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        r.v[k] = s * a.v[k];
    return r;
}
template <typename V> struct IsVecN : std::false_type {};
template <typename T, int NV> struct IsVecN<VecN<T, NV>> : std::true_type {};
template <typename V>
__device__ __forceinline__ V vzero_any()
{
    if constexpr (IsVecN<V>::value) {
        V r;
#pragma unroll
        for (int k = 0; k < (int)(sizeof(V) / sizeof(r.v[0])); ++k)
            r.v[k] = 0;
        return r;
    } else {
        return vzero<V>();
    }
}
template <typename V>
__device__ __forceinline__ V vload(const V *p)
{
    if constexpr (IsVecN<V>::value) {
        constexpr int kW = (int)(sizeof(V) / 16);
        uint4 w[kW];
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
        for (int k = 0; k < kW; ++k)
            w[k] = __ldg(q + k);
        V r;
        memcpy(&r, w, sizeof(V));
        return r;
    } else {
        return *p;
    }
}
template <typename T, int NV>
__device__ __forceinline__ void store_cs(VecN<T, NV> *p, const VecN<T, NV> &a)
{
    constexpr int kW = (int)(sizeof(VecN<T, NV>) / 16);
    uint4 w[kW];
    memcpy(w, &a, sizeof(w));
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int k = 0; k < kW; ++k)
        __stcs(q + k, w[k]);
}

// The row value of the term-parallel kernel: one scalar or complex number, or
// NV > 1 interleaved real vectors
template <typename T, bool kC, int NV>
using TpVal = std::conditional_t<(NV > 1), VecN<T, NV>, typename ValT<T, kC>::type>;

__device__ __forceinline__ void atomic_add(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void atomic_add(double *p, double v) { atomicAdd(p, v); }
template <typename T> __device__ __forceinline__ void atomic_add(Cplx<T> *p, Cplx<T> v)
{
    atomicAdd(&p->re, v.re);
    atomicAdd(&p->im, v.im);
}

// hash index entries: 8 bytes {state, index << norm_bits | norm} or 16 bytes
// {state, index | norm << 32}
template <typename W> __device__ __forceinline__ W ent_state(uint2 v) { return (W)v.x; }
template <typename W> __device__ __forceinline__ W ent_state(ulonglong2 v) { return (W)v.x; }
__device__ __forceinline__ uint32_t ent_index(uint2 v, int nb) { return v.y >> nb; }
__device__ __forceinline__ uint32_t ent_norm(uint2 v, int nb) { return v.y & ((1u << nb) - 1u); }
__device__ __forceinline__ uint32_t ent_index(ulonglong2 v, int) { return (uint32_t)v.y; }
__device__ __forceinline__ uint32_t ent_norm(ulonglong2 v, int) { return (uint32_t)(v.y >> 32); }

// Resident blocks per SM the register budget is sized for.  32-bit words with
// a hash index: 8 (32 registers; 8-32 bytes of spills, measured faster than 6
// blocks at 40 registers without them: ring N=32 fp32 1.25 against 1.38 ms).
// Otherwise 5 (48 registers, no spills; 64-bit words at 32 registers spilled
// 50-130 bytes: ring N=40 fp32 722 ms with the spills, 663 ms without).
template <typename W, int kIdx, int NV = 1>
constexpr int kTpMinBlocks = NV > 1 ? 4 : (sizeof(W) == 4 && kIdx != 2 ? 8 : 5);

// kIdx: index of the sectors -- 0 hash index with 8-byte entries, 1 with
// 16-byte entries, 2 bucketed index (find_bucketed).  NV > 1: a real block of
// NV interleaved vectors (one search and lookup per term serves them all).
template <typename W, typename T, bool kC, bool kTrack, bool kFact, int kIdx, int kSec, bool kPush = false,
          int NV = 1>
__global__ void __launch_bounds__(kTpThreads, kTpMinBlocks<W, kIdx, NV>)
    k_matvec_tp(const __grid_constant__ TpArgs<kSec> a)
{
    static_assert(NV == 1 || (!kC && !kPush), "blocks: real, pull form");
    using V = TpVal<T, kC, NV>;
    using E = std::conditional_t<kIdx == 1, ulonglong2, uint2>;
    extern __shared__ __align__(16) unsigned char smem[];
    size_t off[8];
    tp_smem_layout<W, T, V, kFact>(a.g, a.op, a.n_sectors, a.max_order, off);
    W *sm_masks = reinterpret_cast<W *>(smem + off[0]);
    OpFamily *sm_fam = reinterpret_cast<OpFamily *>(smem + off[1]);
    Cplx<T> *sm_mats = reinterpret_cast<Cplx<T> *>(smem + off[2]);
    uint8_t *sm_off = smem + off[3];
    uint8_t *sm_kind = smem + off[4];
    T *sm_sq = reinterpret_cast<T *>(smem + off[5]);
    T *sm_isq = sm_sq + (a.max_order + 1);
    const SectorDesc *sm_sec = a.sec;  // launch parameters: warp-uniform reads
    TpWarp<W, T, V> *sm_warp = reinterpret_cast<TpWarp<W, T, V> *>(smem + off[7]);
    const int tstride = tp_term_stride(a.g, a.op);
    uint8_t *sm_terms = smem + tp_terms_offset<W, T, V>(off[7]) + (size_t)(threadIdx.x >> 5) * 32 * tstride;
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
        for (int e = threadIdx.x; e <= a.max_order; e += blockDim.x) {
            sm_sq[e] = sqrt((T)e);
            sm_isq[e] = e ? T(1) / sqrt((T)e) : T(0);
        }
    }
    if (!pass_gate(a.ctl))  // includes the barrier after the table loads
        return;

    const unsigned kAll = 0xffffffffu;
    const int n_fam = a.op.n_fam;
    const int n = a.g.n_sites;
    const W full = (W)a.g.full;
    const int lane = threadIdx.x & 31;
    TpWarp<W, T, V> &ws = sm_warp[threadIdx.x >> 5];
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;

    uint64_t taken = 0;
    for (uint64_t tile = next_tile(a.ctl, taken, gw, nw); tile < a.total_tiles;
         tile = next_tile(a.ctl, taken, gw, nw)) {
        int sec = 0;
        if (kSec > 1) {  // last sector with tile_begin <= tile (warp-uniform)
            int lo = 0, hi = a.n_sectors - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sm_sec[mid].tile_begin <= tile)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            sec = lo;
        }
        const SectorDesc &sd = sm_sec[sec];
        const V *__restrict__ x = reinterpret_cast<const V *>(sd.x);
        const int flip = sd.flip;

        // ---- rows: state, norm, diagonal, number of off-diagonal terms ----
        const uint64_t row = (tile - sd.tile_begin) * 32 + lane;
        const bool valid = row < sd.dim;
        W r = 0;
        T rinv = T(0);
        uint32_t nt = 0;
        V acc = vzero_any<V>();
        if (valid) {
            if (sd.keys) {
                const uint64_t k = __ldcs(sd.keys + row);  // streamed once: evict first
                r = (W)(k >> 16);
                rinv = sm_isq[k & 0xffff];
            } else {
                r = (W)__ldg(sd.states + row);
                rinv = sm_isq[__ldg(sd.norms + row)];
            }
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
                    if ((cc == 1 || cc == 2) && sm_off[fm.mat * 4 + cc])
                        nt += (uint32_t)cnt;
                }
            }
            const V xv = vload(x + row);
            if constexpr (kPush) {
                // push form: the row's x is scattered, not gathered; the
                // diagonal goes to y like every other contribution
                acc = xv;
                V dv;
                if constexpr (kC)
                    dv = cmul(conjc(d), xv);
                else
                    dv = d.re * xv;
                atomic_add(reinterpret_cast<V *>(sd.y) + row, dv);
            } else if constexpr (kC) {
                acc = cmul(conjc(d), xv);
            } else {
                acc = d.re * xv;
            }
        }
        // flat layout of the tile's terms: exclusive scan of the counts
        uint32_t incl = nt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kAll, incl, o);
            if (lane >= o)
                incl += v;
        }
        const uint32_t total = __shfl_sync(kAll, incl, 31);
        const uint32_t offl = incl - nt;
        ws.acc[lane] = acc;
        ws.r[lane] = r;
        ws.rinv[lane] = rinv;
        ws.off[lane] = offl;
        if (n_fam == 1 && nt) {  // list the row's antiparallel bonds once per tile
            const OpFamily fm = sm_fam[0];
            const W tq = rot_down(r, (int)fm.delta, n, full);
            int k = 0;
#pragma unroll
            for (int cc = 1; cc <= 2; ++cc) {
                if (sm_off[fm.mat * 4 + cc]) {
                    W bits = config_mask(r, tq, (W)fm.mask, cc);
                    while (bits) {
                        sm_terms[lane * tstride + k++] = (uint8_t)(lowest_bit(bits) | (cc == 2 ? 0x80 : 0));
                        bits &= bits - 1;
                    }
                }
            }
        }
        __syncwarp();

        const E *__restrict__ hent = reinterpret_cast<const E *>(sd.hent);
        const uint32_t *__restrict__ htab = sd.htab;
        const int hbits = sd.hbits, norm_bits = sd.norm_bits;
        for (uint32_t base = 0; base < total; base += 32) {
            // rows whose terms start in this round, and the row carried in
            const bool starts = nt > 0 && offl >= base && offl < base + 32;
            if (starts)
                ws.p2r[offl - base] = (uint8_t)lane;
            const unsigned M = __reduce_or_sync(kAll, starts ? 1u << (offl - base) : 0u);
            const unsigned carry = __ballot_sync(kAll, nt > 0 && offl < base && offl + nt > base);
            __syncwarp();
            const uint32_t t = base + lane;
            const bool act = t < total;
            const unsigned le = M & (kAll >> (31 - lane));  // segment starts at or below this lane
            const int spos = le ? 31 - __clz((int)le) : -1;
            const int rho = le ? (int)ws.p2r[spos] : (carry ? __ffs((int)carry) - 1 : 0);

            // this lane's term: the u-th antiparallel bond of row rho, in
            // (family, configuration |01> then |10>, site) order
            W s = 0;
            int amp = 0;
            if (act && n_fam == 1) {
                const W rr = ws.r[rho];
                const uint32_t code = sm_terms[rho * tstride + (t - ws.off[rho])];
                const OpFamily fm = sm_fam[0];
                const int i = (int)(code & 63u);
                const int cc = code & 0x80u ? 2 : 1;
                amp = (int)fm.mat * 16 + (3 - cc) * 4 + cc;
                int j = i + (int)fm.delta;
                j -= j >= n ? n : 0;
                s = rr ^ (W(1) << i) ^ (W(1) << j);
            } else if (act) {
                const W rr = ws.r[rho];
                int u = (int)(t - ws.off[rho]);
                W sel = 0;
                int su = 0, sdelta = 0;
                for (int q = 0; q < n_fam; ++q) {
                    const OpFamily fm = sm_fam[q];
                    const W tq = rot_down(rr, (int)fm.delta, n, full);
#pragma unroll
                    for (int cc = 1; cc <= 2; ++cc) {
                        if (sm_off[fm.mat * 4 + cc]) {
                            const W bits = config_mask(rr, tq, (W)fm.mask, cc);
                            const int cnt = popc(bits);
                            if (u >= 0 && u < cnt) {
                                sel = bits;
                                su = u;
                                sdelta = (int)fm.delta;
                                amp = (int)fm.mat * 16 + (3 - cc) * 4 + cc;
                            }
                            u -= cnt;
                        }
                    }
                }
                const int i = nth_set_bit(sel, su);
                int j = i + sdelta;
                j -= j >= n ? n : 0;
                s = rr ^ (W(1) << i) ^ (W(1) << j);
            }

            // representative search (every lane; idle lanes search s = 0)
            W best;
            int gbest = 0;
            if (kFact && a.g.prune && (sizeof(W) == 8 || kTrack)) {
                rep_search_rot1<W, kTrack>(s, sm_kind, sm_masks, a.g.n_cos, n, a.g.n_perm, flip, full, best,
                                           gbest);
            } else if (kFact) {
                if (kTrack)
                    rep_search_fact<W, true>(s, sm_kind, sm_masks, a.g.n_cos, a.g.rot_L, a.g.rot_d, n,
                                             a.g.n_perm, flip, full, best, gbest);
                else
                    best = rep_min_fact<W>(s, sm_kind, sm_masks, a.g.n_cos, a.g.rot_L, a.g.rot_d, n, flip,
                                           full);
            } else {
                rep_search<W, kTrack>(s, sm_masks, a.g.n_perm, flip, full, best, gbest);
            }

            // stateToIndex through the bucket of the hash index, gather, scale
            V val = vzero_any<V>();
            if (act) {
                uint32_t jidx = 0, jnorm = 0;
                bool found = false;
                if constexpr (kIdx == 2) {
                    found = find_bucketed((uint64_t)best, sd.bkt, sd.stash, sd.n_stash, n, sd.bbits, sd.brem, jidx,
                                          jnorm);
                } else {
                    const uint32_t bk = hash_bucket((uint64_t)best, hbits);
                    const uint32_t e1 = __ldg(htab + bk + 1);
                    for (uint32_t e = __ldg(htab + bk); e < e1; ++e) {
                        const E v = __ldg(hent + e);
                        if (ent_state<W>(v) == best) {
                            jidx = ent_index(v, norm_bits);
                            jnorm = ent_norm(v, norm_bits);
                            found = true;
                            break;
                        }
                    }
                }
                if (found) {
                    {
                        const T ratio = sm_sq[jnorm] * ws.rinv[rho];
                        const Cplx<T> h = sm_mats[amp];
                        Cplx<T> coef = {h.re * ratio, -h.im * ratio};  // conj(h) sqrt(n'/n)
                        if (kTrack) {
                            Cplx<T> ch;
                            if constexpr (sizeof(T) == 8)
                                ch = load_c<T>(sd.chi + gbest);
                            else
                                ch = load_cf<T>(sd.chif + gbest);
                            coef = cmul(coef, ch);
                        }
                        if constexpr (kPush) {
                            // H Hermitian: H[r'][r] = conj(H[r][r']); this term adds
                            // conj(coef) x_r to y_r'
                            const V xr = ws.acc[rho];
                            V pv;
                            if constexpr (kC)
                                pv = cmul(conjc(coef), xr);
                            else
                                pv = coef.re * xr;
                            atomic_add(reinterpret_cast<V *>(sd.y) + jidx, pv);
                        } else {
                            const V xv = vload(x + jidx);
                            if constexpr (kC)
                                val = cmul(coef, xv);
                            else
                                val = coef.re * xv;
                        }
                    }
                }
            }
            if constexpr (!kPush) {
                // segmented inclusive scan: lanes spos..lane belong to the same row
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const V up = vshfl_up(val, o);
                    if (lane >= o && lane - o >= spos)
                        val = vadd(val, up);
                }
                const bool seg_end = act && (lane == 31 || t + 1 == total || ((M >> (lane + 1)) & 1u));
                if (seg_end)
                    ws.acc[rho] = vadd(ws.acc[rho], val);
            }
            __syncwarp();
        }
        if (!kPush && valid)
            store_cs(reinterpret_cast<V *>(sd.y) + row, ws.acc[lane]);
        __syncwarp();
    }
}

template <typename W, typename T, bool kC, bool kTrack, bool kFact, int kIdx, int kSec, bool kPush = false,
          int NV = 1>
cudaError_t tp_launch(const TpArgs<kSec> &a, cudaStream_t stream)
{
    using V = TpVal<T, kC, NV>;
    auto kern = k_matvec_tp<W, T, kC, kTrack, kFact, kIdx, kSec, kPush, NV>;
    const size_t smem = tp_smem_bytes<W, T, V, kFact>(a.g, a.op, a.n_sectors, a.max_order);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTpThreads, smem);
    if (e != cudaSuccess)
        return e;
    const uint64_t blocks_needed = (a.total_tiles + kTpWarps - 1) / kTpWarps;
    const int grid = (int)std::min<uint64_t>(blocks_needed, (uint64_t)sms * std::max(per_sm, 1));
    kern<<<std::max(grid, 1), kTpThreads, smem, stream>>>(a); count_launch();
    return cudaGetLastError();
}

// idx: index kind of every sector of the batch (they must agree): 0 hash
// index with 8-byte entries, 1 with 16-byte entries, 2 bucketed index; kPush:
// the transposed (push) form with atomic scatter into y, which must be zero
template <typename T, bool kC, int kSec, bool kPush = false, int NV = 1>
cudaError_t tp_dispatch(const TpArgs<kSec> &a, bool track, int idx, cudaStream_t stream)
{
    const bool w32 = a.g.n_sites <= 32;
    const bool fact = a.g.fact != 0;
#define ED_TP_FA(W, TR, IX)                                                                 \
    do {                                                                                    \
        if (fact) return tp_launch<W, T, kC, TR, true, IX, kSec, kPush, NV>(a, stream);     \
        return tp_launch<W, T, kC, TR, false, IX, kSec, kPush, NV>(a, stream);              \
    } while (0)
#define ED_TP_TR(W, IX)                  \
    do {                                 \
        if (track) ED_TP_FA(W, true, IX); \
        ED_TP_FA(W, false, IX);          \
    } while (0)
    if (idx == 2) {
        if (w32) ED_TP_TR(uint32_t, 2);
        ED_TP_TR(uint64_t, 2);
    }
    if (w32) {
        if (idx == 1) ED_TP_TR(uint32_t, 1);
        ED_TP_TR(uint32_t, 0);
    }
    ED_TP_TR(uint64_t, 1);
#undef ED_TP_TR
#undef ED_TP_FA
}

// The term-parallel kernel applies when every off-diagonal entry of every
// family's matrix couples configurations 1 and 2 (|01> <-> |10>).
bool tp_operator_ok(const ed_operator *op);

// index kind of a sector for tp_dispatch
inline int tp_index_kind(const SectorDesc &d) { return d.bkt ? 2 : (d.hwide ? 1 : 0); }

// one sector (tp_single_*) or a batch (tp_multi_*), nvec = 1; idx as tp_dispatch
cudaError_t tp_single_f64(const TpArgs<1> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_single_f32(const TpArgs<1> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_single_c128(const TpArgs<1> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_single_c64(const TpArgs<1> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_multi_f64(const TpArgs<kMaxSectors> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_multi_f32(const TpArgs<kMaxSectors> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_multi_c128(const TpArgs<kMaxSectors> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_multi_c64(const TpArgs<kMaxSectors> &a, bool track, int idx, cudaStream_t s);
// push form (ablation), one sector, y zeroed by the caller
cudaError_t tp_push(const TpArgs<1> &a, bool track, int idx, ed_dtype dtype, cudaStream_t s);
// one sector, a real block of 8 interleaved vectors
cudaError_t tp_single_f64_nv8(const TpArgs<1> &a, bool track, int idx, cudaStream_t s);
cudaError_t tp_single_f32_nv8(const TpArgs<1> &a, bool track, int idx, cudaStream_t s);

}  // namespace edk
