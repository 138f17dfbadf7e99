// ed_internal.cuh -- device-side building blocks shared by the basis and matvec
// kernels: the word-level Benes network that applies a site permutation, the
// representative search over the symmetry group, the "stateToIndex" search in
// the sorted basis (Sec. "Matrix-vector product"), and the handle layouts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <vector>

#include "../../include/ed.h"

namespace edk {

// ---------------------------------------------------------------------------
// Benes networks on a machine word.  A permutation of the 2^L bit positions of
// a word is realised by 2L-1 "delta swap" stages with shifts
// 2^(L-1), ..., 2, 1, 2, ..., 2^(L-1); stage i exchanges bits p and p + d(i)
// wherever bit p of its mask is set.  Masks are stored padded to 12 words per
// permutation so that they can be fetched as 16-byte vectors.
// ---------------------------------------------------------------------------
constexpr int kMaskStride = 12;

template <typename W> struct WordInfo;
template <> struct WordInfo<uint32_t> { static constexpr int kLog = 5; static constexpr int kBits = 32; };
template <> struct WordInfo<uint64_t> { static constexpr int kLog = 6; static constexpr int kBits = 64; };

__host__ __device__ constexpr int benes_shift(int log2w, int stage)
{
    return stage < log2w ? (1 << (log2w - 1 - stage)) : (1 << (stage - log2w + 1));
}

template <typename W, typename M>
__device__ __forceinline__ W delta_swap(W x, M mask, int d)
{
    const W m = (W)mask;
    W t = ((x >> d) ^ x) & m;
    return x ^ t ^ (t << d);
}

// Apply one permutation, masks in shared memory (16-byte aligned, 12 words).
__device__ __forceinline__ uint32_t benes_apply(uint32_t x, const uint32_t *m)
{
    const uint4 a = *reinterpret_cast<const uint4 *>(m);
    const uint4 b = *reinterpret_cast<const uint4 *>(m + 4);
    const uint32_t c = m[8];
    x = delta_swap(x, a.x, 16);
    x = delta_swap(x, a.y, 8);
    x = delta_swap(x, a.z, 4);
    x = delta_swap(x, a.w, 2);
    x = delta_swap(x, b.x, 1);
    x = delta_swap(x, b.y, 2);
    x = delta_swap(x, b.z, 4);
    x = delta_swap(x, b.w, 8);
    x = delta_swap(x, c, 16);
    return x;
}

__device__ __forceinline__ uint64_t benes_apply(uint64_t x, const uint64_t *m)
{
    const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(m);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(m + 2);
    const ulonglong2 c = *reinterpret_cast<const ulonglong2 *>(m + 4);
    const ulonglong2 e = *reinterpret_cast<const ulonglong2 *>(m + 6);
    const ulonglong2 f = *reinterpret_cast<const ulonglong2 *>(m + 8);
    const uint64_t g = m[10];
    x = delta_swap(x, a.x, 32);
    x = delta_swap(x, a.y, 16);
    x = delta_swap(x, b.x, 8);
    x = delta_swap(x, b.y, 4);
    x = delta_swap(x, c.x, 2);
    x = delta_swap(x, c.y, 1);
    x = delta_swap(x, e.x, 2);
    x = delta_swap(x, e.y, 4);
    x = delta_swap(x, f.x, 8);
    x = delta_swap(x, f.y, 16);
    x = delta_swap(x, g, 32);
    return x;
}

// ---------------------------------------------------------------------------
// Device views of the handles (plain structs passed by value to kernels).
// ---------------------------------------------------------------------------
struct GroupView {
    int n_sites;
    int n_perm;        // lattice elements (the permutations)
    int flip;          // 1 if spin inversion doubles the group
    int order;         // n_perm * (1 + flip); expanded index: p (plain), p + n_perm (flipped)
    uint64_t full;     // low n_sites bits set
    const uint32_t *masks32;  // n_perm x kMaskStride (used when n_sites <= 32)
    const uint64_t *masks64;  // n_perm x kMaskStride
    const double2 *chi;       // order entries, expanded
    const float2 *chif;       // same, single precision
    const uint32_t *chi_one;  // bitset over the expanded order: chi == 1
    // Factored form G = { rho^b h_c F^f }: rho = rotation of the n_sites-bit word
    // by rot_d bits (order rot_L), h_c = coset representatives applied first.
    // Expanded factored index: c * rot_L + b (+ n_perm if flipped).
    int fact;                 // 1 if the factored form is available
    int rot_L, rot_d, n_cos;
    int prune;                // 1: rot_d == 1; the kernels then use the pruned search
                              // (rep_search_rot1) for 64-bit words and for tracked
                              // minimisers; 32-bit words without tracking keep the
                              // exhaustive funnel-shift loop, which measured faster
    const uint8_t *cos_kind;  // n_cos: 0 identity, 1 bit reversal, 2 Benes network
    const uint32_t *cos_masks32;  // n_cos x kMaskStride
    const uint64_t *cos_masks64;  // n_cos x kMaskStride
    const double2 *fchi;      // order entries, factored index
    const float2 *fchif;
    const uint32_t *fchi_one;
};

struct IndexView {
    const uint64_t *states;  // ascending basis
    const uint16_t *norms;   // orbit norms
    const uint64_t *keys;    // state << 16 | norm (n_sites <= 48), else null
    uint64_t dim;
    const uint32_t *tab;     // prefix offsets, tab_size + 1 entries
    uint64_t tab_size;
    int e_lo, e_hi;          // bit-length range covered by the table
    int mbits;               // mantissa bits of the table key
    int probe_iters;         // halving steps that reduce the largest bucket to one entry, + 1
    // hash index: bucket b = hash(state) holds entries hent[htab[b] .. htab[b+1])
    const uint32_t *htab;    // 2^hbits + 1 offsets (null: use the prefix table)
    const void *hent;        // entries: 8 bytes (state:32 | packed index,norm:32) or 16 bytes
    int hbits;               // log2 of the bucket count
    int hwide;               // 1: 16-byte entries {state, index | norm << 32}
    int norm_bits;           // 8-byte entries: low norm_bits of the packed word hold the norm
    // bucketed index (replaces the hash index above when present): one 32-byte
    // bucket of four 8-byte entries per lookup, see find_bucketed
    const uint64_t *bkt;     // 2^bbits buckets x 4 entries, or null
    const ulonglong2 *stash; // ascending {state, index | norm << 32} of keys whose two buckets were full
    uint32_t n_stash;
    int bbits;               // log2 of the bucket count
    int brem;                // remainder bits kept per entry: n_sites - bbits
};

// ---------------------------------------------------------------------------
// Bucketed index ("stateToIndex" with one memory access).  A product over a
// sector far larger than L2 is bound by the rate of random DRAM accesses: on
// GB300 random 32-byte reads saturate near 4e10/s and 64-byte reads near
// 2.3e10/s, whatever their footprint beyond a few GiB, so each lookup reads
// exactly one aligned 32-byte bucket (one sector) holding up to four entries,
// instead of a bucket offset and then an entry.  The state s is mapped by
// an invertible mix m of its n bits; the top bbits of m choose the bucket and
// the low brem bits (the remainder) are stored, so that (bucket, remainder)
// identifies m and hence s with a 64-bit entry:
//   bits  0..31  index in the basis (dim < 2^32 - 1, so 0xFFFFFFFF marks empty)
//   bits 32..    tag = remainder << 1 | alt, then the orbit norm above the tag
// A key goes to the first free slot of its primary bucket, else of its
// alternative bucket (primary XOR a nonzero function of the remainder; alt = 1
// in the tag), else to a small sorted stash.  Slots fill in order, so a key is
// in its alternative bucket only if its primary bucket's last slot is used,
// and in the stash only if both are full.
// ---------------------------------------------------------------------------
constexpr int kBucketSlots = 4;

__host__ __device__ __forceinline__ uint64_t bucket_mix(uint64_t s, int n)
{
    const uint64_t full = n >= 64 ? ~0ULL : ((1ULL << n) - 1);
    uint64_t m = (s * 0x9E3779B97F4A7C15ULL) & full;  // odd multiplier: a bijection mod 2^n
    m ^= m >> ((n + 1) >> 1);                         // xorshift: a bijection on n bits
    return (m * 0xD6E8FEB86659FD93ULL) & full;
}

__host__ __device__ __forceinline__ uint32_t bucket_alt(uint32_t rem, uint32_t bmask)
{
    return (uint32_t)((((uint64_t)rem * 0x9E3779B97F4A7C15ULL) >> 40) | 1u) & bmask;  // odd: nonzero
}

__device__ __forceinline__ bool find_bucketed(uint64_t s, const uint64_t *bkt, const ulonglong2 *stash,
                                              uint32_t n_stash, int n, int bbits, int brem, uint32_t &idx,
                                              uint32_t &norm)
{
    const uint64_t m = bucket_mix(s, n);
    const uint32_t rem = (uint32_t)m & ((1u << brem) - 1u);
    const uint32_t tmask = (2u << brem) - 1u;
    uint32_t b = (uint32_t)(m >> brem);
    uint32_t tag = rem << 1;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(bkt + ((uint64_t)b << 2));
        ulonglong2 v[kBucketSlots / 2];
#pragma unroll
        for (int k = 0; k < kBucketSlots / 2; ++k)
            v[k] = __ldg(p + k);
#pragma unroll
        for (int k = 0; k < kBucketSlots; ++k) {
            const uint64_t e = (k & 1) ? v[k >> 1].y : v[k >> 1].x;
            const uint32_t lo = (uint32_t)e, hi = (uint32_t)(e >> 32);
            if (((hi ^ tag) & tmask) == 0 && lo != 0xFFFFFFFFu) {
                idx = lo;
                norm = hi >> (brem + 1);
                return true;
            }
        }
        if ((uint32_t)v[kBucketSlots / 2 - 1].y == 0xFFFFFFFFu)
            return false;  // primary (or alternative) bucket not full
        b ^= bucket_alt(rem, (1u << bbits) - 1u);
        tag |= 1u;
    }
    uint32_t lo = 0, hi = n_stash;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(&stash[mid].x) < s)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo < n_stash) {
        const ulonglong2 e = __ldg(stash + lo);
        if (e.x == s) {
            idx = (uint32_t)e.y;
            norm = (uint32_t)(e.y >> 32);
            return true;
        }
    }
    return false;
}

__host__ __device__ __forceinline__ uint32_t hash_bucket(uint64_t s, int hbits)
{
    return (uint32_t)((s * 0x9E3779B97F4A7C15ULL) >> (64 - hbits));
}

// stateToIndex through the hash index: scans the state's bucket (about one
// entry on average; the entries of a bucket are contiguous).
__device__ __forceinline__ bool find_hashed(uint64_t s, const IndexView &ix, uint32_t &idx, uint32_t &norm)
{
    const uint32_t b = hash_bucket(s, ix.hbits);
    uint32_t e = __ldg(ix.htab + b);
    const uint32_t end = __ldg(ix.htab + b + 1);
    if (ix.hwide) {
        const ulonglong2 *ent = reinterpret_cast<const ulonglong2 *>(ix.hent);
        for (; e < end; ++e) {
            const ulonglong2 v = __ldg(ent + e);
            if (v.x == s) {
                idx = (uint32_t)v.y;
                norm = (uint32_t)(v.y >> 32);
                return true;
            }
        }
    } else {
        const uint2 *ent = reinterpret_cast<const uint2 *>(ix.hent);
        for (; e < end; ++e) {
            const uint2 v = __ldg(ent + e);
            if (v.x == (uint32_t)s) {
                idx = v.y >> ix.norm_bits;
                norm = v.y & ((1u << ix.norm_bits) - 1u);
                return true;
            }
        }
    }
    return false;
}

// Monotone bucket key of a state: (bit length - e_lo, next mbits bits below the
// leading one).  Ascending states give non-decreasing keys.
__host__ __device__ __forceinline__ uint64_t prefix_key(uint64_t s, int e_lo, int mbits)
{
#ifdef __CUDA_ARCH__
    const int bl = 64 - __clzll((long long)s);
#else
    const int bl = s ? 64 - __builtin_clzll(s) : 0;
#endif
    uint64_t mant = 0;
    if (mbits > 0 && bl >= 2)
        mant = (s << (65 - bl)) >> (64 - mbits);
    return ((uint64_t)(bl - e_lo) << mbits) | mant;
}

// "stateToIndex": position of s in the ascending basis or -1.
static __device__ __noinline__ int64_t find_index(uint64_t s, const IndexView &ix)
{
    const int bl = 64 - __clzll((long long)s);
    if (bl < ix.e_lo || bl > ix.e_hi)
        return -1;
    const uint64_t t = prefix_key(s, ix.e_lo, ix.mbits);
    uint64_t lo = __ldg(ix.tab + t);
    uint64_t hi = __ldg(ix.tab + t + 1);
    const uint64_t end = hi;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (__ldg(ix.states + mid) < s)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < end && __ldg(ix.states + lo) == s) ? (int64_t)lo : -1;
}

// stateToIndex over the packed keys (state << 16 | norm): the probe that finds
// the state also delivers its orbit norm.  Indices are 32-bit (dim < 2^32).
static __device__ __noinline__ bool find_key(uint64_t s, const IndexView &ix, uint32_t &idx, uint32_t &norm)
{
    const int bl = 64 - __clzll((long long)s);
    if (bl < ix.e_lo || bl > ix.e_hi)
        return false;
    const uint64_t t = prefix_key(s, ix.e_lo, ix.mbits);
    uint32_t lo = __ldg(ix.tab + t);
    uint32_t hi = __ldg(ix.tab + t + 1);
    const uint32_t end = hi;
    const uint64_t target = s << 16;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(ix.keys + mid) < target)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo >= end)
        return false;
    const uint64_t k = __ldg(ix.keys + lo);
    if ((k >> 16) != s)
        return false;
    idx = lo;
    norm = (uint32_t)(k & 0xffff);
    return true;
}

__device__ __forceinline__ bool chi_is_one(const uint32_t *bits, int g)
{
    return (bits[g >> 5] >> (g & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Representative search: best = min over the expanded group of g.s, gbest =
// the expanded index of the first minimiser in visiting order.  The loop over
// the group is uniform across the warp (every lane applies the same element at
// the same time), so mask reads from shared memory are broadcasts.
// ---------------------------------------------------------------------------
template <typename W, bool kTrack>
__device__ __forceinline__ void rep_search(W s, const W *sm_masks, int n_perm, int flip, W full,
                                           W &best, int &gbest)
{
    best = ~W(0);
    gbest = 0;
    if (flip) {
        for (int p = 0; p < n_perm; ++p) {
            const W q = benes_apply(s, sm_masks + p * kMaskStride);
            const W f = q ^ full;
            if (kTrack) {
                if (q < best) { best = q; gbest = p; }
                if (f < best) { best = f; gbest = p + n_perm; }
            } else {
                best = min(best, min(q, f));
            }
        }
    } else {
        for (int p = 0; p < n_perm; ++p) {
            const W q = benes_apply(s, sm_masks + p * kMaskStride);
            if (kTrack) {
                if (q < best) { best = q; gbest = p; }
            } else {
                best = min(best, q);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Representative search over the factored group.  For every coset
// representative h (identity, bit reversal of the n-bit word, or a Benes
// network) the image h.s is rotated through all rot_L positions; each rotated
// word q and its complement q ^ full (spin inversion) are candidates.  The
// coset loop and the rotation loop are uniform across the warp.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t reverse_bits(uint32_t s, int n) { return __brev(s) >> (32 - n); }
__device__ __forceinline__ uint64_t reverse_bits(uint64_t s, int n) { return __brevll(s) >> (64 - n); }

template <typename W>
__device__ __forceinline__ W coset_image(W s, int kind, const W *masks, int n)
{
    if (kind == 0)
        return s;
    if (kind == 1)
        return reverse_bits(s, n);
    return benes_apply(s, masks);
}

// Visits every candidate of the factored group: f(candidate, factored index).
// 32-bit words: rotation by k of the n-bit word is one funnel shift of the
// doubled word (h | h << n).
template <typename F>
__device__ __forceinline__ void for_each_image32(uint32_t s, const uint8_t *kinds, const uint32_t *masks,
                                                 int n_cos, int L, int d, int n, int n_perm, int flip,
                                                 uint32_t full, F &&f)
{
    for (int c = 0; c < n_cos; ++c) {
        const uint32_t h = coset_image(s, (int)kinds[c], masks + c * kMaskStride, n);
        const uint32_t lo = n == 32 ? h : (h | (h << n));
        const uint32_t hi = n == 32 ? h : (h >> (32 - n));
        const int base = c * L;
        if (n == 32) {
            for (int b = 0; b < L; ++b) {
                const uint32_t q = __funnelshift_l(h, h, b * d);
                if (f(q, base + b))
                    return;
                if (flip && f(~q, base + b + n_perm))
                    return;
            }
        } else {
            for (int b = 0; b < L; ++b) {
                const uint32_t q = __funnelshift_rc(lo, hi, n - b * d) & full;
                if (f(q, base + b))
                    return;
                if (flip && f(q ^ full, base + b + n_perm))
                    return;
            }
        }
    }
}

// 64-bit words: the rotation is applied incrementally, rho = rotate by d.
template <typename F>
__device__ __forceinline__ void for_each_image64(uint64_t s, const uint8_t *kinds, const uint64_t *masks,
                                                 int n_cos, int L, int d, int n, int n_perm, int flip,
                                                 uint64_t full, F &&f)
{
    for (int c = 0; c < n_cos; ++c) {
        uint64_t q = coset_image(s, (int)kinds[c], masks + c * kMaskStride, n);
        const int base = c * L;
        for (int b = 0; b < L; ++b) {
            if (f(q, base + b))
                return;
            if (flip && f(q ^ full, base + b + n_perm))
                return;
            q = ((q << d) | (q >> (n - d))) & full;
        }
    }
}

template <typename W, typename F>
__device__ __forceinline__ void for_each_image(W s, const uint8_t *kinds, const W *masks, int n_cos, int L,
                                               int d, int n, int n_perm, int flip, W full, F &&f)
{
    if constexpr (sizeof(W) == 4)
        for_each_image32(s, kinds, masks, n_cos, L, d, n, n_perm, flip, full, f);
    else
        for_each_image64(s, kinds, masks, n_cos, L, d, n, n_perm, flip, full, f);
}

template <typename W, bool kTrack>
__device__ __forceinline__ void rep_search_fact(W s, const uint8_t *kinds, const W *masks, int n_cos, int L,
                                                int d, int n, int n_perm, int flip, W full, W &best,
                                                int &gbest)
{
    W bst = ~W(0);
    int gb = 0;
    for_each_image<W>(s, kinds, masks, n_cos, L, d, n, n_perm, flip, full, [&](W q, int g) {
        if (kTrack) {
            if (q < bst) {
                bst = q;
                gb = g;
            }
        } else {
            bst = min(bst, q);
        }
        return false;
    });
    best = bst;
    gbest = gb;
}

// ---------------------------------------------------------------------------
// Pruned search for a rotation step of one site (every translation of a ring).
//
// Compared as unsigned integers, a rotation of an n-bit word h is the smaller
// the longer the run of zeros it starts with (at bit n-1).  The minimum over
// all n rotations therefore brings the top of one of the LONGEST zero runs of
// h to bit n-1, and only those rotations need to be formed and compared.  With
// spin inversion the complement of a rotation starts with the complemented
// bits, so a longest run of ones qualifies as well: the candidates are the tops
// of the longest runs of equal bits (a zero run gives the plain rotation, a
// one run the complemented one).  The tops are found bit-parallel: with
// X_k = {p : bits p, p-1, ..., p-k+1 of h are equal} (zeros only, without
// spin inversion), X_{k+1} = X_2 & rotl(X_k, 1); the last nonempty X_k holds
// exactly the tops of the longest runs.  The bit reversal maps the runs of h to
// mirrored runs of the same lengths, so the candidates of the reversal image
// are the mirrored bottoms of those runs (the tops rotated down by length - 1),
// with no second pass.  The minimum equals the brute-force minimum over the
// rotations of every coset image; the minimiser may differ only by an element
// of the stabiliser of the minimum.
// ---------------------------------------------------------------------------
// rotation of the n-bit word x up by b (0 <= b < n): bit p goes to p + b mod n
template <typename W>
__device__ __forceinline__ W rotl_n(W x, int b, int n, W full)
{
    if constexpr (sizeof(W) == 4) {
        if (n == 32)
            return __funnelshift_l(x, x, b);
        return ((x << b) | (x >> (n - b))) & full;
    } else {
        if (n == 64)
            return (x << b) | (x >> ((64 - b) & 63));
        return ((x << b) | (x >> (n - b))) & full;
    }
}

// Tops of the longest runs of equal bits of h (of zeros only when !flip), and
// the length of those runs.  A word without such a run structure (all bits
// equal, or no zero at all without spin inversion: every rotation is the same
// word) gives the single candidate top n - 1 (rotation 0) and length n.
template <typename W>
__device__ __forceinline__ W run_tops(W h, int n, int flip, W full, int &len)
{
    const W r1 = rotl_n(h, 1, n, full);  // bit p of r1 = bit p-1 of h
    const W x2 = flip ? (W)(~(h ^ r1) & full) : (W)(~(h | r1) & full);
    W cur = flip ? full : (W)(~h & full);
    if (x2 == full || cur == 0) {
        len = n;
        return W(1) << (n - 1);
    }
    // x2 != full: X_k is empty once k - 1 >= n, so the loop ends within n steps
    len = 1;
    while (true) {
        const W nxt = x2 & rotl_n(cur, 1, n, full);
        if (nxt == 0)
            break;
        cur = nxt;
        ++len;
    }
    return cur;
}

template <typename W>
__device__ __forceinline__ int lowest_set(W v)
{
    if constexpr (sizeof(W) == 4)
        return __ffs((int)v) - 1;
    else
        return __ffsll((long long)v) - 1;
}

// Candidates of one coset image h (coset c): the rotations that bring a top in
// `tops` to bit n - 1, complemented where the run there is a run of ones.
template <typename W, bool kTrack>
__device__ __forceinline__ void rot1_candidates(W h, W tops, int c, int n, int n_perm, int flip, W full,
                                                W &best, int &gbest)
{
    while (tops) {
        const int p = lowest_set(tops);
        tops &= tops - 1;
        const int b = n - 1 - p;
        W q = rotl_n(h, b, n, full);
        int gi = c * n + b;
        if (flip && ((h >> p) & 1)) {
            q ^= full;
            gi += n_perm;
        }
        if (kTrack) {
            if (q < best) {
                best = q;
                gbest = gi;
            }
        } else {
            best = min(best, q);
        }
    }
}

// Minimum over the factored group when its rotations step by one site (rot_L
// = n); gbest is a factored index of a minimiser.  `flip` may differ per lane.
template <typename W, bool kTrack>
__device__ __forceinline__ void rep_search_rot1(W s, const uint8_t *kinds, const W *masks, int n_cos, int n,
                                                int n_perm, int flip, W full, W &best, int &gbest)
{
    W bst = ~W(0);
    int gb = 0;
    int len0;
    const W t0 = run_tops(s, n, flip, full, len0);
    for (int c = 0; c < n_cos; ++c) {
        const int kind = kinds[c];
        W h, tops;
        if (kind == 0) {
            h = s;
            tops = t0;
        } else if (kind == 1) {
            h = reverse_bits(s, n);
            const int dn = len0 - 1;  // bottoms = tops rotated down by len - 1
            tops = reverse_bits(rotl_n(t0, dn ? n - dn : 0, n, full), n);
        } else {
            h = benes_apply(s, masks + c * kMaskStride);
            int l;
            tops = run_tops(h, n, flip, full, l);
        }
        rot1_candidates<W, kTrack>(h, tops, c, n, n_perm, flip, full, bst, gb);
    }
    best = bst;
    gbest = gb;
}

// ---------------------------------------------------------------------------
// small complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct Cplx { T re, im; };

// A "rotation family" of two-site terms: every site i in `mask` is coupled to
// site (i + delta) mod n_sites by the same 4x4 matrix `mat`.  Any term list is
// a union of such families (group the terms by matrix and by site offset), so
// a row's local configurations on all bonds of a family come from one word
// rotation and a few logic operations.
struct OpFamily {
    uint64_t mask;
    uint32_t mat;
    uint32_t delta;
};

template <typename T>
__device__ __forceinline__ Cplx<T> cmul(Cplx<T> a, Cplx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}

}  // namespace edk

// ---------------------------------------------------------------------------
// Handle layouts (host side).
// ---------------------------------------------------------------------------
struct ed_basis {
    int device = 0;
    int n_sites = 0, n_up = 0, spin_inversion = 0;
    int n_perm = 0, order = 0;
    bool trivial_chars = false;  // every expanded character equals 1
    bool real_chars = false;     // every expanded character is real
    std::vector<int32_t> perms;  // n_perm x n_sites
    std::vector<double> chars;   // n_perm x 2
    uint64_t dim = 0;
    // device arrays
    uint64_t *d_states = nullptr;
    uint16_t *d_norms = nullptr;
    uint64_t *d_keys = nullptr;  // state << 16 | norm, n_sites <= 48
    uint32_t *d_tab = nullptr;
    uint32_t *d_masks32 = nullptr;
    uint64_t *d_masks64 = nullptr;
    double2 *d_chi = nullptr;
    float2 *d_chif = nullptr;
    uint32_t *d_chi_one = nullptr;
    // factored form (see GroupView)
    bool fact = false;
    int rot_L = 1, rot_d = 0, n_cos = 0;
    uint8_t *d_cos_kind = nullptr;
    uint32_t *d_cos_masks32 = nullptr;
    uint64_t *d_cos_masks64 = nullptr;
    double2 *d_fchi = nullptr;
    float2 *d_fchif = nullptr;
    uint32_t *d_fchi_one = nullptr;
    uint64_t tab_size = 0;
    int e_lo = 0, e_hi = 0, mbits = 0;
    uint32_t max_bucket = 0;
    int probe_iters = 1;
    // hash index
    uint32_t *d_htab = nullptr;
    void *d_hent = nullptr;
    int hbits = 0, hwide = 0, norm_bits = 0;
    uint32_t hash_max_bucket = 0;
    // bucketed index (IndexView; built instead of the hash index for large sectors)
    uint64_t *d_bkt = nullptr;
    ulonglong2 *d_stash = nullptr;
    uint32_t n_stash = 0;
    int bbits = 0, brem = 0;

    edk::GroupView group_view() const;
    edk::IndexView index_view() const;
};

struct ed_operator {
    int n_sites = 0, n_terms = 0, n_mats = 0;
    std::vector<int32_t> sites;       // n_terms x 2
    std::vector<int32_t> mat_of_term; // n_terms
    std::vector<double> mats;         // n_mats x 16 x 2: coeff * h, deduplicated
    int max_offdiag = 0;              // max off-diagonal entries one row can produce
    bool real = true;                 // every matrix entry real
    // host copies of the device tables
    std::vector<edk::OpFamily> h_fams;
    std::vector<double2> h_mats;
    std::vector<float2> h_matsf;
    std::vector<uint8_t> h_offmask;
    // device tables
    edk::OpFamily *d_fams = nullptr;  // rotation families of the terms
    double2 *d_mats = nullptr;        // n_mats x 16
    float2 *d_matsf = nullptr;
    uint8_t *d_offmask = nullptr;     // n_mats x 4: bit c' set if h[c'][c] != 0, c' != c
    mutable std::atomic<const ed_basis *> checked{nullptr};  // last basis verified symmetric
};
