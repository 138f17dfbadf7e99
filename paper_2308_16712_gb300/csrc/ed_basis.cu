// ed_basis.cu -- basis build (Sec. "States enumeration"): the range of
// fixed-popcount states is split into chunks of consecutive combinations; each
// thread unranks its chunk start (combinatorial number system, colex order =
// ascending integers) and walks the chunk with Gosper's next-combination step,
// keeping the states that are their orbit's minimum with nonzero norm.  A count
// pass, an exclusive scan and a write pass give an order-preserving compaction,
// so the result is ascending without a sort.  Then the prefix table used by
// "stateToIndex" is built over it.
#include <cuda_runtime.h>

#include <algorithm>

#include "ed_kernels.cuh"

namespace edk {
namespace {

constexpr int kEnumThreads = 256;

// Device-detected invariant violations of the kernels in this file (bit 0:
// a chunk's write pass disagreed with its count pass).  Read and cleared by
// ed_stream_status.
__device__ unsigned int g_basis_status;

__device__ __forceinline__ uint64_t unrank_colex(uint64_t rank, int n, int k, const uint64_t *binom)
{
    uint64_t s = 0;
    int hi = n;
    for (int i = k; i >= 1; --i) {
        int c = hi - 1;
        while (__ldg(binom + c * 65 + i) > rank)
            --c;
        s |= 1ULL << c;
        rank -= __ldg(binom + c * 65 + i);
        hi = c;
    }
    return s;
}

// Gosper's hack: the next larger integer with the same popcount.
__device__ __forceinline__ uint64_t next_combination(uint64_t s)
{
    const uint64_t u = s & (~s + 1ULL);
    const uint64_t v = s + u;
    return v | (((v ^ s) >> 2) >> (__ffsll((long long)s) - 1));
}

// Orbit norm of s if s is the minimum of its orbit, else 0.  Norm = number of
// group elements fixing s, or 0 when a fixing element has chi != 1.
template <typename W>
__device__ __forceinline__ int rep_norm(W s, const W *sm_masks, const uint32_t *sm_one, int n_perm,
                                        int flip, W full)
{
    int stab = 0;
    bool ok = true;
    for (int p = 0; p < n_perm; ++p) {
        const W q = benes_apply(s, sm_masks + p * kMaskStride);
        if (q < s)
            return 0;
        if (q == s) {
            ++stab;
            ok = ok && chi_is_one(sm_one, p);
        }
        if (flip) {
            const W f = q ^ full;
            if (f < s)
                return 0;
            if (f == s) {
                ++stab;
                ok = ok && chi_is_one(sm_one, p + n_perm);
            }
        }
    }
    return ok ? stab : 0;
}

// Same test over the factored group (rotation subgroup x coset representatives).
template <typename W>
__device__ __forceinline__ int rep_norm_fact(W s, const uint8_t *kinds, const W *masks,
                                             const uint32_t *one, const GroupView &g, W full)
{
    int stab = 0;
    bool ok = true, rep = true;
    for_each_image<W>(s, kinds, masks, g.n_cos, g.rot_L, g.rot_d, g.n_sites, g.n_perm, g.flip, full,
                      [&](W q, int gi) {
                          if (q < s) {
                              rep = false;
                              return true;
                          }
                          if (q == s) {
                              ++stab;
                              ok = ok && chi_is_one(one, gi);
                          }
                          return false;
                      });
    return (rep && ok) ? stab : 0;
}

__host__ __device__ inline size_t enum_smem_bytes(const GroupView &g, size_t wbytes, bool fact)
{
    const int nm = fact ? g.n_cos : g.n_perm;
    return (size_t)nm * kMaskStride * wbytes + ((g.order + 31) / 32) * 4 + ((nm + 15) / 16) * 16;
}

template <typename W, bool kU1, bool kWrite, bool kFact>
__global__ void __launch_bounds__(kEnumThreads) k_enumerate(EnumPlan plan, GroupView g,
                                                            uint32_t *counts,
                                                            const uint64_t *offsets,
                                                            uint64_t *states, uint16_t *norms)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nm = kFact ? g.n_cos : g.n_perm;
    W *sm_masks = reinterpret_cast<W *>(smem);
    uint32_t *sm_one = reinterpret_cast<uint32_t *>(smem + (size_t)nm * kMaskStride * sizeof(W));
    uint8_t *sm_kind = reinterpret_cast<uint8_t *>(sm_one + (g.order + 31) / 32);
    const W *gm;
    if (kFact)
        gm = sizeof(W) == 4 ? reinterpret_cast<const W *>(g.cos_masks32)
                            : reinterpret_cast<const W *>(g.cos_masks64);
    else
        gm = sizeof(W) == 4 ? reinterpret_cast<const W *>(g.masks32)
                            : reinterpret_cast<const W *>(g.masks64);
    for (int e = threadIdx.x; e < nm * kMaskStride; e += blockDim.x)
        sm_masks[e] = gm[e];
    for (int e = threadIdx.x; e < (g.order + 31) / 32; e += blockDim.x)
        sm_one[e] = kFact ? g.fchi_one[e] : g.chi_one[e];
    if (kFact)
        for (int e = threadIdx.x; e < g.n_cos; e += blockDim.x)
            sm_kind[e] = g.cos_kind[e];
    __syncthreads();
    const W full = (W)g.full;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < plan.n_chunks;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t r0 = c * plan.chunk;
        const uint64_t cnt = min(plan.chunk, plan.total - r0);
        uint64_t s = kU1 ? unrank_colex(r0, plan.n_sites, plan.n_up, plan.binom) : r0;
        uint32_t kept = 0;
        uint64_t out = kWrite ? offsets[c] : 0;
        uint32_t *cflags = plan.flags ? plan.flags + c * plan.flag_words : nullptr;
        uint32_t word = 0;
        for (uint64_t q = 0; q < cnt; ++q) {
            int nrm;
            if (kWrite && cflags) {  // only the states the count pass kept
                if ((q & 31) == 0)
                    word = cflags[q >> 5];
                nrm = (word >> (q & 31)) & 1u
                          ? (kFact ? rep_norm_fact<W>((W)s, sm_kind, sm_masks, sm_one, g, full)
                                   : rep_norm<W>((W)s, sm_masks, sm_one, g.n_perm, g.flip, full))
                          : 0;
            } else {
                nrm = kFact ? rep_norm_fact<W>((W)s, sm_kind, sm_masks, sm_one, g, full)
                            : rep_norm<W>((W)s, sm_masks, sm_one, g.n_perm, g.flip, full);
            }
            if (nrm) {
                if (kWrite) {
                    states[out] = s;
                    norms[out] = (uint16_t)nrm;
                    ++out;
                }
                ++kept;
            }
            if (!kWrite && cflags) {
                word |= (nrm ? 1u : 0u) << (q & 31);
                if ((q & 31) == 31 || q + 1 == cnt) {
                    cflags[q >> 5] = word;
                    word = 0;
                }
            }
            if (q + 1 < cnt)
                s = kU1 ? next_combination(s) : s + 1;
        }
        if (!kWrite)
            counts[c] = kept;
        else if (offsets[c] + kept != offsets[c + 1])
            atomicOr(&g_basis_status, 1u);
    }
}

template <typename W, bool kU1, bool kWrite, bool kFact>
cudaError_t enum_launch(const EnumPlan &plan, const GroupView &g, uint32_t *counts,
                        const uint64_t *offsets, uint64_t *states, uint16_t *norms,
                        cudaStream_t stream)
{
    auto kern = k_enumerate<W, kU1, kWrite, kFact>;
    const size_t smem = enum_smem_bytes(g, sizeof(W), kFact);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kEnumThreads, smem);
    if (e != cudaSuccess)
        return e;
    const uint64_t want = (plan.n_chunks + kEnumThreads - 1) / kEnumThreads;
    const int grid = (int)std::min<uint64_t>(want, (uint64_t)sms * std::max(per_sm, 1));
    kern<<<std::max(grid, 1), kEnumThreads, smem, stream>>>(plan, g, counts, offsets, states, norms); count_launch();
    return cudaGetLastError();
}

template <bool kWrite>
cudaError_t enum_dispatch(const EnumPlan &plan, const GroupView &g, uint32_t *counts,
                          const uint64_t *offsets, uint64_t *states, uint16_t *norms,
                          cudaStream_t stream)
{
    const bool u1 = plan.n_up >= 0;
#define ED_ENUM(W, U1)                                                                           \
    return g.fact ? enum_launch<W, U1, kWrite, true>(plan, g, counts, offsets, states, norms, stream) \
                  : enum_launch<W, U1, kWrite, false>(plan, g, counts, offsets, states, norms, stream)
    if (plan.n_sites <= 32) {
        if (u1)
            ED_ENUM(uint32_t, true);
        ED_ENUM(uint32_t, false);
    }
    if (u1)
        ED_ENUM(uint64_t, true);
    ED_ENUM(uint64_t, false);
#undef ED_ENUM
}

// ---------------------------------------------------------------------------
// exclusive scan, uint32 -> uint64 (reduce per block, scan block sums in one
// block with a running carry, rescan each block)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *sm_warp, uint64_t &total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += t;
    }
    if (lane == 31)
        sm_warp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint64_t w = lane < (int)(blockDim.x >> 5) ? sm_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o)
                w += t;
        }
        sm_warp[lane] = w;  // inclusive warp-total prefix
    }
    __syncthreads();
    total = sm_warp[(blockDim.x >> 5) - 1];
    const uint64_t before = wid ? sm_warp[wid - 1] : 0;
    __syncthreads();
    return before + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *in, uint64_t n, uint64_t *bsum)
{
    __shared__ uint64_t sm[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint64_t v = 0;
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n)
            v += in[base + k];
    uint64_t total;
    block_exclusive_scan(v, sm, total);
    if (threadIdx.x == 0)
        bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_bsums(uint64_t *bsum, uint64_t nb, uint64_t *grand)
{
    __shared__ uint64_t sm[32];
    uint64_t carry = 0;
    for (uint64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const uint64_t i = b0 + threadIdx.x;
        const uint64_t v = i < nb ? bsum[i] : 0;
        uint64_t total;
        const uint64_t ex = block_exclusive_scan(v, sm, total);
        if (i < nb)
            bsum[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0)
        *grand = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *in, uint64_t n,
                                                            const uint64_t *bsum, uint64_t *out)
{
    __shared__ uint64_t sm[32];
    const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
    uint32_t items[kScanItems];
    uint64_t v = 0;
    for (int k = 0; k < kScanItems; ++k) {
        items[k] = base + k < n ? in[base + k] : 0;
        v += items[k];
    }
    uint64_t total;
    uint64_t run = bsum[blockIdx.x] + block_exclusive_scan(v, sm, total);
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n)
            out[base + k] = run;
        run += items[k];
    }
}

// ---------------------------------------------------------------------------
// prefix table, sortedness check, state -> index
// ---------------------------------------------------------------------------
__global__ void k_prefix_table(IndexView ix, uint32_t *tab)
{
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ix.tab_size)
        return;
    uint64_t lo = 0, hi = ix.dim;  // first i with key(states[i]) >= t
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (prefix_key(ix.states[mid], ix.e_lo, ix.mbits) < t)
            lo = mid + 1;
        else
            hi = mid;
    }
    tab[t] = (uint32_t)lo;
}

__global__ void k_hash_count(const uint64_t *states, uint64_t dim, int hbits, uint32_t *counts)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(counts + hash_bucket(states[i], hbits), 1u);
}

__global__ void k_offsets_to_u32(const uint64_t *offsets, uint64_t n, uint32_t *out)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (uint32_t)offsets[i];
}

// The order of entries inside a bucket depends on atomic timing; lookups
// compare states, so the result of a lookup does not.
__global__ void k_hash_fill(const uint64_t *states, const uint16_t *norms, uint64_t dim, int hbits,
                            uint32_t *cursor, void *entries, int wide, int norm_bits)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = states[i];
        const uint32_t pos = atomicAdd(cursor + hash_bucket(s, hbits), 1u);
        if (wide)
            reinterpret_cast<ulonglong2 *>(entries)[pos] =
                make_ulonglong2(s, (uint64_t)i | ((uint64_t)norms[i] << 32));
        else
            reinterpret_cast<uint2 *>(entries)[pos] =
                make_uint2((uint32_t)s, ((uint32_t)i << norm_bits) | norms[i]);
    }
}

// Slot order inside a bucket depends on atomic timing; a lookup compares the
// tag, so its result does not.
__global__ void k_bucket_fill(const uint64_t *states, const uint16_t *norms, uint64_t dim, int n, int bbits,
                              int brem, uint32_t *cnt, uint64_t *bkt, ulonglong2 *stash, uint32_t *n_stash,
                              uint32_t stash_cap)
{
    const uint32_t bmask = (uint32_t)((1ULL << bbits) - 1);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t s = states[i];
        const uint64_t m = bucket_mix(s, n);
        const uint32_t rem = (uint32_t)m & ((1u << brem) - 1u);
        uint32_t b = (uint32_t)(m >> brem);
        const uint64_t hi = ((uint64_t)norms[i] << (brem + 1)) | ((uint64_t)rem << 1);
        const uint64_t e = i | (hi << 32);
        uint32_t slot = atomicAdd(cnt + b, 1u);
        if (slot < kBucketSlots) {
            bkt[((uint64_t)b << 2) + slot] = e;
            continue;
        }
        b ^= bucket_alt(rem, bmask);
        slot = atomicAdd(cnt + b, 1u);
        if (slot < kBucketSlots) {
            bkt[((uint64_t)b << 2) + slot] = e | (1ULL << 32);
            continue;
        }
        const uint32_t k = atomicAdd(n_stash, 1u);
        if (k < stash_cap)
            stash[k] = make_ulonglong2(s, i | ((uint64_t)norms[i] << 32));
    }
}

__global__ void k_max_bucket(const uint32_t *tab, uint64_t tab_size, uint32_t *out)
{
    uint32_t m = 0;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tab_size;
         t += (uint64_t)gridDim.x * blockDim.x)
        m = max(m, tab[t + 1] - tab[t]);
    for (int o = 16; o > 0; o >>= 1)
        m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, m);
}

__global__ void k_pack_keys(const uint64_t *states, const uint16_t *norms, uint64_t dim, uint64_t *keys)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x)
        keys[i] = (states[i] << 16) | norms[i];
}

__global__ void k_check_sorted(const uint64_t *states, uint64_t dim, int *flag)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i < dim;
         i += (uint64_t)gridDim.x * blockDim.x)
        if (states[i - 1] >= states[i])
            atomicOr(flag, 1);
}

__global__ void k_index(IndexView ix, const uint64_t *q, int64_t *out, uint64_t n)
{
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = find_index(q[i], ix);
}

}  // namespace

cudaError_t basis_status_take(unsigned int *status)
{
    unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(status, g_basis_status, sizeof(unsigned int));
    if (e == cudaSuccess && *status)
        e = cudaMemcpyToSymbol(g_basis_status, &zero, sizeof(unsigned int));
    return e;
}

cudaError_t launch_enum_count(const EnumPlan &plan, const GroupView &g, uint32_t *counts,
                              cudaStream_t stream)
{
    return enum_dispatch<false>(plan, g, counts, nullptr, nullptr, nullptr, stream);
}

cudaError_t launch_enum_write(const EnumPlan &plan, const GroupView &g, const uint64_t *offsets,
                              uint64_t *states, uint16_t *norms, cudaStream_t stream)
{
    return enum_dispatch<true>(plan, g, nullptr, offsets, states, norms, stream);
}

size_t scan_tmp_words(uint64_t n)
{
    return (n + kScanTile - 1) / kScanTile + 1;
}

cudaError_t launch_scan(const uint32_t *counts, uint64_t n, uint64_t *offsets, uint64_t *tmp,
                        cudaStream_t stream)
{
    const uint64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0)
        return cudaMemsetAsync(offsets, 0, sizeof(uint64_t), stream);
    k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, stream>>>(counts, n, tmp); count_launch();
    k_scan_bsums<<<1, kScanThreads, 0, stream>>>(tmp, nb, offsets + n); count_launch();
    k_scan_down<<<(unsigned)nb, kScanThreads, 0, stream>>>(counts, n, tmp, offsets); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_prefix_table(const IndexView &ix, uint32_t *tab, cudaStream_t stream)
{
    const uint64_t n = ix.tab_size + 1;
    k_prefix_table<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(ix, tab); count_launch();
    return cudaGetLastError();
}

static unsigned grid_for(uint64_t n)
{
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, 65536));
}

cudaError_t launch_hash_count(const uint64_t *states, uint64_t dim, int hbits, uint32_t *counts,
                              cudaStream_t stream)
{
    if (!dim)
        return cudaSuccess;
    k_hash_count<<<grid_for(dim), 256, 0, stream>>>(states, dim, hbits, counts); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_offsets_to_u32(const uint64_t *offsets, uint64_t n, uint32_t *out, cudaStream_t stream)
{
    k_offsets_to_u32<<<grid_for(n), 256, 0, stream>>>(offsets, n, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hash_fill(const uint64_t *states, const uint16_t *norms, uint64_t dim, int hbits,
                             uint32_t *cursor, void *entries, int wide, int norm_bits,
                             cudaStream_t stream)
{
    if (!dim)
        return cudaSuccess;
    k_hash_fill<<<grid_for(dim), 256, 0, stream>>>(states, norms, dim, hbits, cursor, entries, wide,
                                                    norm_bits); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_bucket_fill(const uint64_t *states, const uint16_t *norms, uint64_t dim, int n_sites,
                               int bbits, int brem, uint32_t *cnt, uint64_t *bkt, ulonglong2 *stash,
                               uint32_t *n_stash, uint32_t stash_cap, cudaStream_t stream)
{
    if (!dim)
        return cudaSuccess;
    k_bucket_fill<<<grid_for(dim), 256, 0, stream>>>(states, norms, dim, n_sites, bbits, brem, cnt, bkt, stash,
                                                      n_stash, stash_cap); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_max_bucket(const uint32_t *tab, uint64_t tab_size, uint32_t *out, cudaStream_t stream)
{
    const uint64_t blocks = std::max<uint64_t>(1, std::min<uint64_t>((tab_size + 255) / 256, 4096));
    k_max_bucket<<<(unsigned)blocks, 256, 0, stream>>>(tab, tab_size, out); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pack_keys(const uint64_t *states, const uint16_t *norms, uint64_t dim, uint64_t *keys,
                             cudaStream_t stream)
{
    if (dim == 0)
        return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((dim + 255) / 256, 65536);
    k_pack_keys<<<(unsigned)blocks, 256, 0, stream>>>(states, norms, dim, keys); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_check_sorted(const uint64_t *states, uint64_t dim, int *flag, cudaStream_t stream)
{
    if (dim < 2)
        return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((dim + 255) / 256, 65536);
    k_check_sorted<<<(unsigned)blocks, 256, 0, stream>>>(states, dim, flag); count_launch();
    return cudaGetLastError();
}

cudaError_t launch_index(const IndexView &ix, const uint64_t *query, int64_t *out, uint64_t n,
                         cudaStream_t stream)
{
    k_index<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(ix, query, out, n); count_launch();
    return cudaGetLastError();
}

}  // namespace edk
