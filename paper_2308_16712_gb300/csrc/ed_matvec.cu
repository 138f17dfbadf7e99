// ed_matvec.cu -- kernel choice and dtype dispatch of the matvec.
#include "ed_matvec_tp.cuh"

namespace edk {

int g_kernel_policy = 0;

// The library's kernel rule for one vector of an exchange-only operator: the
// term-parallel kernel in single precision, and in double precision for
// 64-bit words (ring N=36 / 40 fp64: 42.5 / 714 ms against 45.1 / 750 ms
// row-per-lane); row-per-lane otherwise.
bool use_term_parallel(int nvec, const OpView &op, ed_dtype dtype, int n_sites)
{
    if (nvec != 1 || !op.exchange_only || g_kernel_policy == 1)
        return false;
    return g_kernel_policy == 2 || dtype == ED_F32 || dtype == ED_C64 || n_sites > 32;
}

static TpArgs<1> single_tp_args(const OpView &op, const GroupView &g, const IndexView &ix, const void *x,
                                void *y)
{
    TpArgs<1> t;
    t.op = op;
    t.g = g;
    t.ctl = BatchCtl{nullptr, nullptr, nullptr};  // one sector: static tiles, no gate
    t.n_sectors = 1;
    t.max_order = g.order;
    t.total_tiles = (ix.dim + 31) / 32;
    SectorDesc &d = t.sec[0];
    d.keys = ix.keys;
    d.states = ix.states;
    d.norms = ix.norms;
    d.htab = ix.htab;
    d.hent = ix.hent;
    d.chi = g.fact ? g.fchi : g.chi;
    d.chif = g.fact ? g.fchif : g.chif;
    d.x = x;
    d.y = y;
    d.dim = ix.dim;
    d.tile_begin = 0;
    d.hbits = ix.hbits;
    d.hwide = ix.hwide;
    d.norm_bits = ix.norm_bits;
    d.bkt = ix.bkt;
    d.stash = ix.stash;
    d.n_stash = ix.n_stash;
    d.bbits = ix.bbits;
    d.brem = ix.brem;
    d.flip = g.flip;
    return t;
}

// The push form (ablation): y = 0, then every term scattered atomically.
cudaError_t launch_matvec_push(const OpView &op, const GroupView &g, const IndexView &ix, bool track,
                               const void *x, void *y, ed_dtype dtype, cudaStream_t stream)
{
    const size_t vb = (dtype == ED_F64 || dtype == ED_C64) ? 8 : dtype == ED_F32 ? 4 : 16;
    cudaError_t e = cudaMemsetAsync(y, 0, ix.dim * vb, stream);
    if (e != cudaSuccess)
        return e;
    const TpArgs<1> t = single_tp_args(op, g, ix, x, y);
    return tp_push(t, track, tp_index_kind(t.sec[0]), dtype, stream);
}

cudaError_t launch_matvec(const OpView &op, const GroupView &g, const IndexView &ix, bool track,
                          const void *x, void *y, int nvec, ed_dtype dtype, cudaStream_t stream)
{
    return launch_matvec_v(op, g, ix, track, x, y, nvec, dtype, MatvecVariant{}, stream);
}

cudaError_t launch_matvec_v(const OpView &op, GroupView g, const IndexView &ix, bool track, const void *x,
                            void *y, int nvec, ed_dtype dtype, MatvecVariant v, cudaStream_t stream)
{
    if (v.prune >= 0 && g.fact && g.rot_d == 1)
        g.prune = v.prune;
    // the term-parallel kernel: one vector (use_term_parallel), or a real
    // block of 8 vectors: by default in fp32 (ring N=32 / 36 / 40: 1.69 /
    // 43.6 / 724 ms against 2.04 / 48.4 / 788 ms row-per-lane), in fp64 when
    // the autotuner or the test policy chooses it (its segmented scan adds on
    // the slow fp64 pipe)
    const bool block8 = nvec == 8 && (dtype == ED_F64 || dtype == ED_F32);
    const bool tp_ok = (ix.htab || ix.bkt) && (nvec == 1 || block8) && op.exchange_only;
    const bool rule = block8 ? (g_kernel_policy == 2 || (g_kernel_policy == 0 && dtype == ED_F32))
                             : use_term_parallel(nvec, op, dtype, g.n_sites);
    const bool tp = tp_ok && (v.kernel == 2 || (v.kernel == 0 && rule));
    if (tp) {
        const TpArgs<1> t = single_tp_args(op, g, ix, x, y);
        const int k = tp_index_kind(t.sec[0]);
        if (block8)
            return dtype == ED_F64 ? tp_single_f64_nv8(t, track, k, stream) : tp_single_f32_nv8(t, track, k, stream);
        switch (dtype) {
        case ED_F64: return tp_single_f64(t, track, k, stream);
        case ED_F32: return tp_single_f32(t, track, k, stream);
        case ED_C128: return tp_single_c128(t, track, k, stream);
        case ED_C64: return tp_single_c64(t, track, k, stream);
        }
        return cudaErrorInvalidValue;
    }
    const MatvecArgs a{op, g, ix, x, y, nvec};
    switch (dtype) {
    case ED_F64: return matvec_f64(a, track, stream);
    case ED_F32: return matvec_f32(a, track, stream);
    case ED_C128: return matvec_c128(a, track, stream);
    case ED_C64: return matvec_c64(a, track, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace edk

// ---------------------------------------------------------------------------
// Exact count of the stored nonzeros of H in a sector: every off-diagonal term
// whose representative is in the basis, plus one diagonal entry per row.  One
// thread per row; counts are summed with integer atomics (order-independent).
// ---------------------------------------------------------------------------
namespace edk {
namespace {

template <typename W, bool kFact>
__global__ void __launch_bounds__(256) k_count_nnz(const OpView op, const GroupView g, const IndexView ix,
                                                   unsigned long long *total)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nm = kFact ? g.n_cos : g.n_perm;
    W *sm_masks = reinterpret_cast<W *>(smem);
    uint8_t *sm_kind = reinterpret_cast<uint8_t *>(sm_masks + (size_t)nm * kMaskStride);
    const W *gm;
    if (kFact)
        gm = sizeof(W) == 4 ? reinterpret_cast<const W *>(g.cos_masks32) : reinterpret_cast<const W *>(g.cos_masks64);
    else
        gm = sizeof(W) == 4 ? reinterpret_cast<const W *>(g.masks32) : reinterpret_cast<const W *>(g.masks64);
    for (int e = threadIdx.x; e < nm * kMaskStride; e += blockDim.x)
        sm_masks[e] = gm[e];
    if (kFact)
        for (int e = threadIdx.x; e < g.n_cos; e += blockDim.x)
            sm_kind[e] = g.cos_kind[e];
    __syncthreads();
    const W full = (W)g.full;
    const int n = g.n_sites;
    unsigned long long cnt = 0;
    for (uint64_t row = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; row < ix.dim;
         row += (uint64_t)gridDim.x * blockDim.x) {
        const W r = (W)ix.states[row];
        cnt += 1;  // the diagonal entry
        for (int q = 0; q < op.n_fam; ++q) {
            const OpFamily fm = op.fams[q];
            int j = 0;
            const W tq = (W)(((uint64_t)r >> fm.delta | (uint64_t)r << (n - fm.delta)) & g.full);
            for (int cc = 0; cc < 4; ++cc) {
                const uint32_t targets = op.offmask[fm.mat * 4 + cc];
                if (!targets)
                    continue;
                const W a = (cc & 2) ? r : (W)~r, b = (cc & 1) ? tq : (W)~tq;
                W bits = a & b & (W)fm.mask;
                while (bits) {
                    const int i = sizeof(W) == 4 ? __ffs((uint32_t)bits) - 1 : __ffsll((long long)bits) - 1;
                    bits &= bits - 1;
                    j = i + (int)fm.delta;
                    j -= j >= n ? n : 0;
                    uint32_t tg = targets;
                    while (tg) {
                        const int cp = __ffs(tg) - 1;
                        tg &= tg - 1;
                        const int fl = cc ^ cp;
                        const W s = r ^ (W((fl >> 1) & 1) << i) ^ (W(fl & 1) << j);
                        W best;
                        int gb;
                        if (kFact && g.prune && sizeof(W) == 8)
                            rep_search_rot1<W, false>(s, sm_kind, sm_masks, g.n_cos, n, g.n_perm, g.flip, full,
                                                      best, gb);
                        else if (kFact)
                            rep_search_fact<W, false>(s, sm_kind, sm_masks, g.n_cos, g.rot_L, g.rot_d, n, g.n_perm,
                                                      g.flip, full, best, gb);
                        else
                            rep_search<W, false>(s, sm_masks, g.n_perm, g.flip, full, best, gb);
                        cnt += find_index((uint64_t)best, ix) >= 0 ? 1 : 0;
                    }
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0)
        atomicAdd(total, cnt);
}

template <typename W, bool kFact>
cudaError_t nnz_launch(const OpView &op, const GroupView &g, const IndexView &ix, unsigned long long *total,
                       cudaStream_t stream)
{
    const int nm = kFact ? g.n_cos : g.n_perm;
    const size_t smem = (size_t)nm * kMaskStride * sizeof(W) + (size_t)g.n_cos + 16;
    auto kern = k_count_nnz<W, kFact>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((ix.dim + 255) / 256, 152 * 16));
    kern<<<(unsigned)blocks, 256, smem, stream>>>(op, g, ix, total); count_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_count_nnz(const OpView &op, const GroupView &g, const IndexView &ix,
                             unsigned long long *total, cudaStream_t stream)
{
    if (g.n_sites <= 32)
        return g.fact ? nnz_launch<uint32_t, true>(op, g, ix, total, stream)
                      : nnz_launch<uint32_t, false>(op, g, ix, total, stream);
    return g.fact ? nnz_launch<uint64_t, true>(op, g, ix, total, stream)
                  : nnz_launch<uint64_t, false>(op, g, ix, total, stream);
}

}  // namespace edk

extern "C" void edx_kernel_policy(int policy) { edk::g_kernel_policy = policy; }
