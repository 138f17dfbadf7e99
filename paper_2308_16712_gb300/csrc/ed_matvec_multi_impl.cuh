// ed_matvec_multi_impl.cuh -- many symmetry sectors in one persistent launch
// (the matvec of Sec. "Matrix-vector product" for a batch of sectors that share
// one lattice permutation group and differ in characters, spin inversion, U(1)
// sector, basis and vectors).
//
// The row tiles of all sectors form one list (tile_begin[s] = first tile of
// sector s); warps take tiles round-robin and hand rows to lanes on demand as
// in the single-sector kernel, so every lane may hold a row of a different
// sector.  The group loop is shared (same permutations for all sectors); the
// spin-inversion candidates, the characters and the index search are per lane.
#pragma once

#include "ed_matvec_impl.cuh"

namespace edk {

constexpr int kMaxSectors = 160;

struct SectorDesc {
    const uint64_t *keys;     // state << 16 | norm (or null: states + norms)
    const uint64_t *states;
    const uint16_t *norms;
    const uint32_t *htab;     // hash index (this or the bucketed index is required)
    const void *hent;
    const uint64_t *bkt;      // bucketed index (IndexView), or null
    const ulonglong2 *stash;
    uint32_t n_stash;
    int bbits, brem;
    const double2 *chi;       // characters in the order of the search used
    const float2 *chif;
    const void *x;
    void *y;
    uint64_t dim;
    uint64_t tile_begin;      // first tile of this sector in the batch
    int hbits, hwide, norm_bits, flip;
};

// ---------------------------------------------------------------------------
// Work queue and failure detection of the batched (many-sector) launches.
// Tiles are handed out by a device counter (warp lane 0 takes the next tile
// with an atomic add), in the order of the sector table -- largest sectors
// first -- so that the small sectors' tiles fill the tail of the launch.
// Optionally (a test hook) every block first waits for a gate word that a
// producer would set; the wait is bounded (0.5 s by the global timer, and an
// iteration cap), and when it runs out the block records kStatusTimeout in
// the status word and leaves without touching any vector: the launch ends,
// the context stays usable, and ed_stream_status reports ED_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
constexpr unsigned long long kGateTimeoutNs = 500000000ull;

struct BatchCtl {
    unsigned long long *queue;  // next tile to hand out, zeroed before the launch (null: static tiles)
    unsigned int *status;       // device status word (or null)
    const volatile int *gate;   // wait until *gate != 0 before any work (null: no wait)
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait of the block on the gate; false (status recorded) when it ran out.
__device__ __forceinline__ bool pass_gate(const BatchCtl &c)
{
    __shared__ int open_gate;
    if (threadIdx.x == 0) {
        open_gate = 1;
        if (c.gate) {
            const unsigned long long t0 = global_ns();
            for (int it = 0; *c.gate == 0; ++it) {
                if (global_ns() - t0 > kGateTimeoutNs || it > (1 << 22)) {
                    if (c.status)
                        atomicOr(c.status, kStatusTimeout);
                    open_gate = 0;
                    break;
                }
                __nanosleep(1000);
            }
        }
    }
    __syncthreads();
    return open_gate != 0;
}

// next tile of a warp: from the queue (lane 0's atomic add, broadcast), or
// the static round-robin sequence gw, gw + nw, ... (k = tiles taken so far)
__device__ __forceinline__ uint64_t next_tile(const BatchCtl &c, uint64_t &k, uint64_t gw, uint64_t nw)
{
    if (c.queue) {
        unsigned long long t = 0;
        if ((threadIdx.x & 31) == 0)
            t = atomicAdd(c.queue, 1ull);
        return __shfl_sync(0xffffffffu, t, 0);
    }
    return (k++) * nw + gw;
}

// the index of a basis as a sector descriptor sees it (the hash index, or the
// bucketed index where the basis has one)
inline void sector_index_from(SectorDesc &d, const ed_basis *b)
{
    d.htab = b->d_htab;
    d.hent = b->d_hent;
    d.hbits = b->hbits;
    d.hwide = b->hwide;
    d.norm_bits = b->norm_bits;
    d.bkt = b->d_bkt;
    d.stash = b->d_stash;
    d.n_stash = b->n_stash;
    d.bbits = b->bbits;
    d.brem = b->brem;
}

struct MultiArgs {
    OpView op;
    GroupView g;              // permutation tables shared by all sectors
    int n_sectors;
    int nvec;
    int max_order;            // largest expanded group order in the batch
    uint64_t total_tiles;
    BatchCtl ctl;
    SectorDesc sec[kMaxSectors];  // read from the launch parameters (constant bank)
};

template <typename W, typename T, bool kTrack, bool kFact>
__host__ __device__ inline void multi_smem_layout(const GroupView &g, const OpView &op, int n_sectors,
                                                  int max_order, size_t off[7])
{
    const int nm = kFact ? g.n_cos : g.n_perm;
    off[0] = 0;                                                                  // masks
    off[1] = align16(off[0] + (size_t)nm * kMaskStride * sizeof(W));             // families
    off[2] = align16(off[1] + (size_t)op.n_fam * sizeof(OpFamily));              // matrices
    off[3] = align16(off[2] + (size_t)op.n_mats * 16 * sizeof(Cplx<T>));         // offmask
    off[4] = align16(off[3] + (size_t)op.n_mats * 4);                            // coset kinds
    off[5] = align16(off[4] + (kFact ? (size_t)g.n_cos : 0));                    // sqrt tables
    off[6] = align16(off[5] + 2 * (size_t)(max_order + 1) * sizeof(T));          // sectors
}

template <typename W, typename T, bool kTrack, bool kFact>
__host__ __device__ inline size_t multi_smem_bytes(const GroupView &g, const OpView &op, int n_sectors,
                                                   int max_order)
{
    size_t off[7];
    multi_smem_layout<W, T, kTrack, kFact>(g, op, n_sectors, max_order, off);
    return align16(off[6]);
}

// group search with a per-lane spin-inversion flag (the candidate loop itself
// is uniform across the warp)
template <typename W, bool kTrack, bool kFact>
__device__ __forceinline__ void search_lane(W s, const uint8_t *kinds, const W *masks, const GroupView &g,
                                            int lane_flip, W full, W &best, int &gbest)
{
    if (kFact && g.prune && (sizeof(W) == 8 || kTrack)) {
        rep_search_rot1<W, kTrack>(s, kinds, masks, g.n_cos, g.n_sites, g.n_perm, lane_flip, full, best, gbest);
        return;
    }
    if (kFact && !kTrack) {
        best = rep_min_fact<W>(s, kinds, masks, g.n_cos, g.rot_L, g.rot_d, g.n_sites, lane_flip, full);
        gbest = 0;
        return;
    }
    W bst = ~W(0);
    int gb = 0;
    auto take = [&](W q, int gi) {
        if (kTrack) {
            if (q < bst) {
                bst = q;
                gb = gi;
            }
        } else {
            bst = min(bst, q);
        }
    };
    if (kFact) {
        for_each_image<W>(s, kinds, masks, g.n_cos, g.rot_L, g.rot_d, g.n_sites, g.n_perm, 0, full,
                          [&](W q, int gi) {
                              take(q, gi);
                              if (lane_flip)
                                  take(q ^ full, gi + g.n_perm);
                              return false;
                          });
    } else {
        for (int p = 0; p < g.n_perm; ++p) {
            const W q = benes_apply(s, masks + p * kMaskStride);
            take(q, p);
            if (lane_flip)
                take(q ^ full, p + g.n_perm);
        }
    }
    best = bst;
    gbest = gb;
}

template <typename W, typename T, bool kC, bool kTrack, bool kFact, int NV>
__global__ void __launch_bounds__(kMvThreads) k_matvec_multi(const __grid_constant__ MultiArgs a)
{
    using V = typename ValT<T, kC>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    size_t off[7];
    multi_smem_layout<W, T, kTrack, kFact>(a.g, a.op, a.n_sectors, a.max_order, off);
    W *sm_masks = reinterpret_cast<W *>(smem + off[0]);
    OpFamily *sm_fam = reinterpret_cast<OpFamily *>(smem + off[1]);
    Cplx<T> *sm_mats = reinterpret_cast<Cplx<T> *>(smem + off[2]);
    uint8_t *sm_off = smem + off[3];
    uint8_t *sm_kind = smem + off[4];
    T *sm_sq = reinterpret_cast<T *>(smem + off[5]);
    T *sm_isq = sm_sq + (a.max_order + 1);
    const SectorDesc *sm_sec = a.sec;  // launch parameters: warp-uniform reads
    if (!pass_gate(a.ctl))
        return;
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
    __syncthreads();

    const int nvec = a.nvec;
    const int n_fam = a.op.n_fam;
    const int n = a.g.n_sites;
    const W full = (W)a.g.full;
    const unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lanes_below = (1u << lane) - 1u;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    auto sector_of = [&](uint64_t tile) {
        int lo = 0, hi = a.n_sectors - 1;  // last sector with tile_begin <= tile
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm_sec[mid].tile_begin <= tile)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    };
    uint64_t next = 0;  // warp-uniform

    bool has = false;
    int sec = 0;
    uint64_t row = 0;
    W r = 0, t = 0, fmask = 0, bits = 0, cur = 0;
    T rinv = 1;
    int f = 0, c = 0, i = 0, fdelta = 0, fmat = 0, amp = 0;
    uint32_t cpm = 0;
    V acc[NV];

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
        V *y = reinterpret_cast<V *>(sm_sec[sec].y);
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

    // The warp's rows come in the order of the tiles it takes: positions
    // [base, base + 32) are the rows of tile t_cur, [base + 32, base + 64)
    // those of t_nxt (taken when a ballot round reaches into it).
    const uint64_t kNone = ~0ull;
    uint64_t taken = 0, base = 0;
    uint64_t t_cur = next_tile(a.ctl, taken, gw, nw), t_nxt = kNone;
    bool rows_left = t_cur < a.total_tiles;
    while (true) {
        unsigned need = __ballot_sync(kAll, !has);
        while (need != 0 && rows_left) {
            const uint32_t cnt = __popc(need);
            if (next + cnt > base + 32 && t_nxt == kNone)
                t_nxt = next_tile(a.ctl, taken, gw, nw);
            const uint64_t p = next + __popc(need & lanes_below);
            next += cnt;
            const uint64_t tile = p < base + 32 ? t_cur : t_nxt;
            if (!has && tile < a.total_tiles) {
                sec = sector_of(tile);
                const SectorDesc &sd = sm_sec[sec];
                const uint64_t rw = (tile - sd.tile_begin) * 32 + (p & 31);
                if (rw < sd.dim) {
                    row = rw;
                    const V *x = reinterpret_cast<const V *>(sd.x);
                    if (sd.keys) {
                        const uint64_t k = __ldcs(sd.keys + row);
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
                            const int pc = popc(config_mask(r, tq, (W)fm.mask, cc));
                            const Cplx<T> h = sm_mats[fm.mat * 16 + cc * 5];
                            d.re += h.re * (T)pc;
                            d.im += h.im * (T)pc;
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
            }
            if (next >= base + 32) {
                base += 32;
                t_cur = t_nxt;
                t_nxt = kNone;
                if (t_cur == kNone)
                    t_cur = next_tile(a.ctl, taken, gw, nw);
            }
            rows_left = t_cur < a.total_tiles;
            need = __ballot_sync(kAll, !has);
        }
        if (need == kAll)
            break;

        W best;
        int gbest = 0;
        const int lane_flip = has ? sm_sec[sec].flip : 0;
        search_lane<W, kTrack, kFact>(has ? cur : W(0), sm_kind, sm_masks, a.g, lane_flip, full, best, gbest);

        if (has) {
            const SectorDesc &sd = sm_sec[sec];
            IndexView ix;
            ix.keys = sd.keys;
            ix.states = sd.states;
            ix.norms = sd.norms;
            ix.dim = sd.dim;
            ix.htab = sd.htab;
            ix.hent = sd.hent;
            ix.hbits = sd.hbits;
            ix.hwide = sd.hwide;
            ix.norm_bits = sd.norm_bits;
            uint32_t jj = 0, nj = 0;
            const bool found = sd.bkt ? find_bucketed((uint64_t)best, sd.bkt, sd.stash, sd.n_stash, n, sd.bbits,
                                                      sd.brem, jj, nj)
                                      : find_hashed((uint64_t)best, ix, jj, nj);
            if (found) {
                const uint64_t j = jj;
                const T ratio = sm_sq[nj] * rinv;
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
                const V *x = reinterpret_cast<const V *>(sd.x);
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
                            const Cplx<T> pr = cmul(coef, xv);
                            acc[v].re += pr.re;
                            acc[v].im += pr.im;
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
cudaError_t multi_launch(const MultiArgs &a, cudaStream_t stream)
{
    auto kern = k_matvec_multi<W, T, kC, kTrack, kFact, NV>;
    const size_t smem = multi_smem_bytes<W, T, kTrack, kFact>(a.g, a.op, a.n_sectors, a.max_order);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMvThreads, smem);
    if (e != cudaSuccess)
        return e;
    const uint64_t blocks_needed = (a.total_tiles * 32 + kMvThreads - 1) / kMvThreads;
    const int grid = (int)std::min<uint64_t>(blocks_needed, (uint64_t)sms * std::max(per_sm, 1));
    kern<<<std::max(grid, 1), kMvThreads, smem, stream>>>(a); count_launch();
    return cudaGetLastError();
}

template <typename T, bool kC>
cudaError_t multi_dispatch_prec(const MultiArgs &a, bool track, cudaStream_t stream)
{
    const bool w32 = a.g.n_sites <= 32;
    const bool fact = a.g.fact != 0;
#define ED_MM_NV(W, TR, FA)                                                      \
    do {                                                                         \
        if (a.nvec == 1) return multi_launch<W, T, kC, TR, FA, 1>(a, stream);    \
        if (a.nvec <= 4) return multi_launch<W, T, kC, TR, FA, 4>(a, stream);    \
        if (a.nvec <= 8) return multi_launch<W, T, kC, TR, FA, 8>(a, stream);    \
        return multi_launch<W, T, kC, TR, FA, 16>(a, stream);                    \
    } while (0)
#define ED_MM_FA(W, TR)                  \
    do {                                 \
        if (fact) ED_MM_NV(W, TR, true); \
        ED_MM_NV(W, TR, false);          \
    } while (0)
    if (w32) {
        if (track) ED_MM_FA(uint32_t, true);
        ED_MM_FA(uint32_t, false);
    }
    if (track) ED_MM_FA(uint64_t, true);
    ED_MM_FA(uint64_t, false);
#undef ED_MM_FA
#undef ED_MM_NV
}

// control words of a batched launch on stream s (a fresh work-queue counter,
// zeroed on s; the status word; the gate when a stall is injected)
cudaError_t batch_ctl(cudaStream_t s, BatchCtl *out);
void set_inject_stall(bool on);
int multi_policy_get();

cudaError_t multi_f64(const MultiArgs &a, bool track, cudaStream_t s);
cudaError_t multi_f32(const MultiArgs &a, bool track, cudaStream_t s);
cudaError_t multi_c128(const MultiArgs &a, bool track, cudaStream_t s);
cudaError_t multi_c64(const MultiArgs &a, bool track, cudaStream_t s);
cudaError_t multi_launch_any(const MultiArgs &a, bool track, ed_dtype dtype, cudaStream_t s);

}  // namespace edk
