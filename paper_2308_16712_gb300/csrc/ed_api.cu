// ed_api.cu -- the C ABI: argument and group validation, Benes routing of the
// site permutations, handle management and dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <vector>

#include "ed_kernels.cuh"

using cplx = std::complex<double>;

namespace {

constexpr double kChiTol = 1e-9;

#define ED_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) {                           \
            (void)cudaGetLastError();                      \
            return _e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA; \
        }                                                  \
    } while (0)

// ---------------------------------------------------------------------------
// Benes routing.  `sigma` maps local position a -> local destination sigma[a]
// inside the sub-network [base, base + 2^lsub).  Every token (bit) is sent to
// the lower or the upper half by the input stage such that the two tokens of
// an input pair (a, a ^ d) and the two tokens bound for an output pair
// (b, b ^ d) take different halves (2-colouring of even cycles), the halves
// are routed recursively, and the output stage puts each token in place.
// ---------------------------------------------------------------------------
void benes_route(int lsub, int base, const std::vector<int> &sigma, int ltot,
                 std::vector<uint64_t> &masks)
{
    const int m = 1 << lsub;
    if (m == 2) {
        if (sigma[0] == 1)
            masks[ltot - 1] |= 1ULL << base;
        return;
    }
    const int d = m / 2;
    std::vector<int> inv(m), side(m, -1);
    for (int a = 0; a < m; ++a)
        inv[sigma[a]] = a;
    for (int a0 = 0; a0 < m; ++a0) {
        if (side[a0] >= 0)
            continue;
        int a = a0;
        while (side[a] < 0) {
            side[a] = 0;
            const int ap = a ^ d;
            side[ap] = 1;
            a = inv[sigma[ap] ^ d];
        }
    }
    const int level = lsub - 1;
    const int in_stage = ltot - 1 - level, out_stage = ltot - 1 + level;
    std::vector<int> lower(d), upper(d);
    for (int a = 0; a < m; ++a) {
        if (a < d && side[a] == 1)
            masks[in_stage] |= 1ULL << (base + a);
        (side[a] == 0 ? lower : upper)[a & (d - 1)] = sigma[a] & (d - 1);
    }
    for (int b = 0; b < d; ++b)
        if (side[inv[b]] == 1)
            masks[out_stage] |= 1ULL << (base + b);
    benes_route(lsub - 1, base, lower, ltot, masks);
    benes_route(lsub - 1, base + d, upper, ltot, masks);
}

// Masks (2*log2w - 1 stages) realising "bit i moves to perm[i]" on a w-bit word.
std::vector<uint64_t> benes_masks(int log2w, int n, const int32_t *perm)
{
    const int w = 1 << log2w;
    std::vector<int> sigma(w);
    for (int i = 0; i < w; ++i)
        sigma[i] = i < n ? perm[i] : i;
    std::vector<uint64_t> masks(2 * log2w - 1, 0);
    benes_route(log2w, 0, sigma, log2w, masks);
    return masks;
}

// ---------------------------------------------------------------------------
// group checks: each row a permutation, identity present, no repeats, closed
// under composition (a.b)[i] = a[b[i]], chi a unitary homomorphism.
// ---------------------------------------------------------------------------
ed_status validate_group(int n, int ne, const int32_t *perms, const double *chars)
{
    std::map<std::vector<int32_t>, int> index;
    bool has_identity = false;
    for (int g = 0; g < ne; ++g) {
        std::vector<int32_t> p(perms + (size_t)g * n, perms + (size_t)(g + 1) * n);
        std::vector<char> seen(n, 0);
        bool ident = true;
        for (int i = 0; i < n; ++i) {
            if (p[i] < 0 || p[i] >= n || seen[p[i]])
                return ED_ERR_NOT_A_GROUP;
            seen[p[i]] = 1;
            ident = ident && p[i] == i;
        }
        has_identity = has_identity || ident;
        if (!index.emplace(p, g).second)
            return ED_ERR_NOT_A_GROUP;
        const cplx c(chars[2 * g], chars[2 * g + 1]);
        if (!std::isfinite(c.real()) || !std::isfinite(c.imag()) ||
            std::abs(std::abs(c) - 1.0) > kChiTol)
            return ED_ERR_BAD_CHARACTER;
        if (ident && std::abs(c - 1.0) > kChiTol)
            return ED_ERR_BAD_CHARACTER;
    }
    if (!has_identity)
        return ED_ERR_NOT_A_GROUP;
    std::vector<int32_t> comp(n);
    for (int a = 0; a < ne; ++a) {
        for (int b = 0; b < ne; ++b) {
            for (int i = 0; i < n; ++i)
                comp[i] = perms[(size_t)a * n + perms[(size_t)b * n + i]];
            auto it = index.find(comp);
            if (it == index.end())
                return ED_ERR_NOT_A_GROUP;
            const int c = it->second;
            const cplx ca(chars[2 * a], chars[2 * a + 1]), cb(chars[2 * b], chars[2 * b + 1]);
            const cplx cc(chars[2 * c], chars[2 * c + 1]);
            if (std::abs(cc - ca * cb) > kChiTol)
                return ED_ERR_BAD_CHARACTER;
        }
    }
    return ED_OK;
}

uint64_t binomial(int n, int k)
{
    if (k < 0 || k > n)
        return 0;
    unsigned __int128 r = 1;
    for (int i = 1; i <= k; ++i)
        r = r * (unsigned)(n - k + i) / (unsigned)i;
    return (uint64_t)r;
}

template <typename T>
cudaError_t upload(T **dst, const T *src, size_t count)
{
    cudaError_t e = cudaMalloc((void **)dst, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess)
        return e;
    if (count)
        e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// Factored form of the lattice group: the largest cyclic subgroup acting as a
// rotation of the n-bit word (site i -> i + d mod n, smallest such d) and one
// representative per coset {rho^b h}, preferring the identity, then the bit
// reversal (site i -> n - 1 - i), else any element (applied by a Benes network).
struct Factorization {
    int L = 1, d = 0;
    std::vector<int> rep;       // user element index of each coset representative
    std::vector<uint8_t> kind;  // 0 identity, 1 reversal, 2 Benes
    std::vector<int> elem;      // (c * L + b) -> user element index of rho^b h_c
};

bool factorize(int n, int ne, const int32_t *perms, Factorization &F)
{
    std::map<std::vector<int32_t>, int> index;
    for (int g = 0; g < ne; ++g)
        index.emplace(std::vector<int32_t>(perms + (size_t)g * n, perms + (size_t)(g + 1) * n), g);
    int d = 0;
    for (int cand = 1; cand < n && !d; ++cand) {
        if (n % cand)
            continue;
        std::vector<int32_t> rot(n);
        for (int i = 0; i < n; ++i)
            rot[i] = (i + cand) % n;
        if (index.count(rot))
            d = cand;
    }
    if (!d || d >= 32)
        return false;
    const int L = n / d;
    if (ne % L)
        return false;
    F.L = L;
    F.d = d;
    std::vector<int> coset_of(ne, -1);
    std::vector<int32_t> q(n), ident(n), rev(n);
    for (int i = 0; i < n; ++i) {
        ident[i] = i;
        rev[i] = n - 1 - i;
    }
    for (int g = 0; g < ne; ++g) {
        if (coset_of[g] >= 0)
            continue;
        const int c = (int)F.rep.size();
        std::vector<int> members(L);
        for (int b = 0; b < L; ++b) {
            for (int i = 0; i < n; ++i)
                q[i] = (perms[(size_t)g * n + i] + b * d) % n;
            auto it = index.find(q);
            if (it == index.end())
                return false;
            members[b] = it->second;
            coset_of[it->second] = c;
        }
        // representative: identity, else reversal, else g itself
        int rep = g, kind = 2;
        for (int m : members) {
            std::vector<int32_t> p(perms + (size_t)m * n, perms + (size_t)(m + 1) * n);
            if (p == ident) {
                rep = m;
                kind = 0;
                break;
            }
            if (p == rev && kind == 2) {
                rep = m;
                kind = 1;
            }
        }
        F.rep.push_back(rep);
        F.kind.push_back((uint8_t)kind);
    }
    const int nc = (int)F.rep.size();
    F.elem.assign((size_t)nc * L, -1);
    for (int c = 0; c < nc; ++c) {
        for (int b = 0; b < L; ++b) {
            for (int i = 0; i < n; ++i)
                q[i] = (perms[(size_t)F.rep[c] * n + i] + b * d) % n;
            F.elem[(size_t)c * L + b] = index.at(q);
        }
    }
    return nc * L == ne;
}

bool g_force_generic = false;
bool g_force_prefix = false;
bool g_force_all_rotations = false;  // test hook: factored search over every rotation
// Index built by ed_basis_build: 0 = the bucketed index for sectors of at
// least kBucketAutoDim states (where the hash index no longer fits in L2 and
// every lookup is DRAM traffic), else the hash index; 1 = always the hash
// index; 2 = the bucketed index wherever its entry fits in 64 bits.
int g_index_policy = 0;
constexpr uint64_t kBucketAutoDim = 1ULL << 23;

// Bucketed index over the basis (see find_bucketed): 2^bbits >= dim / 1.8
// buckets of four slots (at 1.8 keys per bucket about 3 % of the keys go to
// their alternative bucket and 0.2 % to the stash).  Returns false (and leaves nothing allocated) when
// the entry does not fit in 64 bits, allocation fails or the stash would
// overflow; the caller then builds the hash index.
bool build_bucket_index(ed_basis *b, int norm_bits, cudaStream_t stream)
{
    const uint64_t dim = b->dim;
    int bb = 1;
    while (bb < 31 && (double)dim > 1.8 * (double)(1ULL << bb))
        ++bb;
    const int brem = b->n_sites - bb;
    if (brem < 0 || brem + 1 + norm_bits > 32 || dim >= 0xFFFFFFFFULL)
        return false;
    const uint64_t nbk = 1ULL << bb;
    const uint32_t cap = (uint32_t)std::min<uint64_t>(dim, std::max<uint64_t>(4096, dim >> 6));
    uint64_t *d_bkt = nullptr;
    uint32_t *d_cnt = nullptr;
    ulonglong2 *d_st = nullptr;
    cudaError_t e = edk::ws_alloc((void **)&d_bkt, nbk * edk::kBucketSlots * sizeof(uint64_t), stream);
    if (e == cudaSuccess)
        e = edk::ws_alloc((void **)&d_cnt, (nbk + 1) * sizeof(uint32_t), stream);  // + the stash counter
    if (e == cudaSuccess)
        e = edk::ws_alloc((void **)&d_st, (size_t)cap * sizeof(ulonglong2), stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_bkt, 0xFF, nbk * edk::kBucketSlots * sizeof(uint64_t), stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_cnt, 0, (nbk + 1) * sizeof(uint32_t), stream);
    if (e == cudaSuccess)
        e = edk::launch_bucket_fill(b->d_states, b->d_norms, dim, b->n_sites, bb, brem, d_cnt, d_bkt, d_st,
                                    d_cnt + nbk, cap, stream);
    uint32_t n_st = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&n_st, d_cnt + nbk, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(stream);
    std::vector<ulonglong2> st;
    if (e == cudaSuccess && n_st > 0 && n_st <= cap) {
        // the stash is searched by binary search: sort it by state on the host
        st.resize(n_st);
        e = cudaMemcpy(st.data(), d_st, n_st * sizeof(ulonglong2), cudaMemcpyDeviceToHost);
        std::sort(st.begin(), st.end(), [](const ulonglong2 &a, const ulonglong2 &c) { return a.x < c.x; });
    }
    edk::ws_free(d_cnt, stream);
    edk::ws_free(d_st, stream);
    ulonglong2 *d_stash = nullptr;
    if (e == cudaSuccess && n_st > 0 && n_st <= cap) {
        e = edk::ws_alloc((void **)&d_stash, n_st * sizeof(ulonglong2), stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_stash, st.data(), n_st * sizeof(ulonglong2), cudaMemcpyHostToDevice, stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(stream);
    }
    if (e != cudaSuccess || n_st > cap) {
        (void)cudaGetLastError();
        edk::ws_free(d_bkt, stream);
        edk::ws_free(d_stash, stream);
        return false;
    }
    b->d_bkt = d_bkt;
    b->d_stash = d_stash;
    b->n_stash = n_st;
    b->bbits = bb;
    b->brem = brem;
    return true;
}

void free_basis(ed_basis *b)
{
    if (!b)
        return;
    // every launch that may still read the arrays has finished before they
    // go back to the pool (the large ones) or to the device
    cudaDeviceSynchronize();
    cudaFree(b->d_cos_kind);
    cudaFree(b->d_cos_masks32);
    cudaFree(b->d_cos_masks64);
    cudaFree(b->d_fchi);
    cudaFree(b->d_fchif);
    cudaFree(b->d_fchi_one);
    edk::ws_free(b->d_states, 0);
    edk::ws_free(b->d_norms, 0);
    edk::ws_free(b->d_keys, 0);
    edk::ws_free(b->d_htab, 0);
    edk::ws_free(b->d_hent, 0);
    edk::ws_free(b->d_bkt, 0);
    edk::ws_free(b->d_stash, 0);
    edk::ws_free(b->d_tab, 0);
    cudaFree(b->d_masks32);
    cudaFree(b->d_masks64);
    cudaFree(b->d_chi);
    cudaFree(b->d_chif);
    cudaFree(b->d_chi_one);
    delete b;
}

// Does the operator commute with every element of the (expanded) group?
// Terms are summed per ordered site pair into 4x4 matrices; an element maps
// the term on (i, j) to (perm[i], perm[j]) and, if it flips, conjugates the
// matrix by X (x) X.
bool operator_is_symmetric(const ed_operator *op, int n_perm, const int32_t *perms,
                           int spin_inversion)
{
    using Key = std::pair<int, int>;
    auto canon = [&](const int32_t *pm, bool flip) {
        std::map<Key, std::vector<cplx>> out;
        for (int t = 0; t < op->n_terms; ++t) {
            int i = op->sites[2 * t], j = op->sites[2 * t + 1];
            if (pm) {
                i = pm[i];
                j = pm[j];
            }
            const double *mm = op->mats.data() + (size_t)op->mat_of_term[t] * 32;
            std::vector<cplx> h(16);
            for (int r = 0; r < 4; ++r)
                for (int c = 0; c < 4; ++c) {
                    int rr = flip ? 3 - r : r, cc = flip ? 3 - c : c;
                    h[rr * 4 + cc] = cplx(mm[2 * (r * 4 + c)], mm[2 * (r * 4 + c) + 1]);
                }
            if (i > j) {  // swap the tensor factors: index 2a+b -> 2b+a
                std::vector<cplx> s(16);
                auto sw = [](int x) { return ((x & 1) << 1) | (x >> 1); };
                for (int r = 0; r < 4; ++r)
                    for (int c = 0; c < 4; ++c)
                        s[sw(r) * 4 + sw(c)] = h[r * 4 + c];
                h = s;
                std::swap(i, j);
            }
            auto &acc = out[Key(i, j)];
            if (acc.empty())
                acc.assign(16, cplx(0));
            for (int e = 0; e < 16; ++e)
                acc[e] += h[e];
        }
        return out;
    };
    const auto ref = canon(nullptr, false);
    double scale = 0;
    for (auto &kv : ref)
        for (auto &v : kv.second)
            scale = std::max(scale, std::abs(v));
    const double tol = 1e-12 * std::max(1.0, scale);
    auto same = [&](const std::map<Key, std::vector<cplx>> &m) {
        auto val = [&](const std::map<Key, std::vector<cplx>> &x, const Key &k, int e) {
            auto it = x.find(k);
            return it == x.end() ? cplx(0) : it->second[e];
        };
        for (auto &kv : ref)
            for (int e = 0; e < 16; ++e)
                if (std::abs(val(m, kv.first, e) - kv.second[e]) > tol)
                    return false;
        for (auto &kv : m)
            for (int e = 0; e < 16; ++e)
                if (std::abs(val(ref, kv.first, e) - kv.second[e]) > tol)
                    return false;
        return true;
    };
    for (int g = 0; g < n_perm; ++g) {
        const int32_t *pm = perms + (size_t)g * op->n_sites;
        if (!same(canon(pm, false)))
            return false;
        if (spin_inversion && !same(canon(pm, true)))
            return false;
    }
    return true;
}


// The host part of an operator: scaled, deduplicated matrices and the packed
// term table.  Arguments must already be validated.
ed_operator *build_operator_host(int n_sites, int n_terms, const double *coeff,
                                 const int32_t *sites, const double *local)
{
    ed_operator *op = new ed_operator();
    op->n_sites = n_sites;
    op->n_terms = n_terms;
    op->sites.assign(sites, sites + 2 * (size_t)n_terms);
    // scaled matrices coeff_t * h_t, deduplicated
    std::map<std::vector<double>, int> seen;
    for (int t = 0; t < n_terms; ++t) {
        const cplx c(coeff[2 * t], coeff[2 * t + 1]);
        std::vector<double> m(32);
        for (int e = 0; e < 16; ++e) {
            const cplx v = c * cplx(local[(size_t)t * 32 + 2 * e], local[(size_t)t * 32 + 2 * e + 1]);
            m[2 * e] = v.real();
            m[2 * e + 1] = v.imag();
            if (v.imag() != 0.0)
                op->real = false;
        }
        auto it = seen.find(m);
        int id;
        if (it == seen.end()) {
            id = (int)seen.size();
            seen.emplace(m, id);
            op->mats.insert(op->mats.end(), m.begin(), m.end());
        } else {
            id = it->second;
        }
        op->mat_of_term.push_back(id);
    }
    op->n_mats = (int)seen.size();
    if (op->n_mats > 65535) {
        delete op;
        return nullptr;
    }
    std::vector<uint8_t> offmask((size_t)op->n_mats * 4, 0);
    std::vector<double2> md((size_t)op->n_mats * 16);
    std::vector<float2> mf((size_t)op->n_mats * 16);
    for (int k = 0; k < op->n_mats; ++k) {
        for (int e = 0; e < 16; ++e) {
            const double re = op->mats[(size_t)k * 32 + 2 * e], im = op->mats[(size_t)k * 32 + 2 * e + 1];
            md[(size_t)k * 16 + e] = make_double2(re, im);
            mf[(size_t)k * 16 + e] = make_float2((float)re, (float)im);
            const int r = e / 4, c = e % 4;
            if (r != c && (re != 0.0 || im != 0.0))
                offmask[(size_t)k * 4 + c] |= (uint8_t)(1u << r);
        }
    }
    // the most off-diagonal elements one row can produce
    int worst = 0;
    for (int t = 0; t < n_terms; ++t) {
        int best = 0;
        for (int c = 0; c < 4; ++c)
            best = std::max(best, __builtin_popcount(offmask[(size_t)op->mat_of_term[t] * 4 + c]));
        worst += best;
    }
    op->max_offdiag = worst;
    // rotation families: terms grouped by (matrix, (j - i) mod n); a site that
    // occurs twice in one group opens another family of the same kind
    std::map<std::pair<int, int>, std::vector<size_t>> open_fams;
    for (int t = 0; t < n_terms; ++t) {
        const int i = sites[2 * t], j = sites[2 * t + 1];
        const int delta = ((j - i) % n_sites + n_sites) % n_sites;
        auto &list = open_fams[{op->mat_of_term[t], delta}];
        bool placed = false;
        for (size_t f : list) {
            if (!((op->h_fams[f].mask >> i) & 1ULL)) {
                op->h_fams[f].mask |= 1ULL << i;
                placed = true;
                break;
            }
        }
        if (!placed) {
            list.push_back(op->h_fams.size());
            op->h_fams.push_back(edk::OpFamily{1ULL << i, (uint32_t)op->mat_of_term[t], (uint32_t)delta});
        }
    }
    op->h_mats = std::move(md);
    op->h_matsf = std::move(mf);
    op->h_offmask = std::move(offmask);
    return op;
}

edk::OpView op_view(const ed_operator *op)
{
    // exchange only: no off-diagonal entry leaves configurations 1 and 2, and
    // each of them only reaches the other
    int exch = 1;
    for (int k = 0; k < op->n_mats; ++k) {
        const uint8_t *m = op->h_offmask.data() + (size_t)k * 4;
        if (m[0] || m[3] || (m[1] & ~4u) || (m[2] & ~2u))
            exch = 0;
    }
    return edk::OpView{(int)op->h_fams.size(), op->n_mats, op->max_offdiag, op->d_fams, op->d_mats,
                       op->d_matsf, op->d_offmask, exch};
}

}  // namespace

namespace edk {

OpView make_op_view(const ed_operator *op) { return op_view(op); }

int index_policy_get() { return g_index_policy; }
void index_policy_set(int policy) { g_index_policy = policy; }

// Validated host tables for counting a sector with the generic group search
// (used by the allocation-free count entry point).
ed_status count_tables_host(int n_sites, int n_up, int spin_inversion, int n_elems,
                            const int32_t *perms, const double *chars,
                            std::vector<uint32_t> &masks32, std::vector<uint64_t> &masks64,
                            std::vector<uint32_t> &chi_one)
{
    if (!perms || !chars)
        return ED_ERR_INVALID_ARG;
    if (n_sites < 1 || n_sites > 64 || n_elems < 1 || n_elems > 1024)
        return ED_ERR_INVALID_ARG;
    if (n_up < -1 || n_up > n_sites || (n_up == -1 && n_sites > 40))
        return ED_ERR_INVALID_ARG;
    if (spin_inversion < -1 || spin_inversion > 1)
        return ED_ERR_INVALID_ARG;
    if (spin_inversion != 0 && n_up != -1 && 2 * n_up != n_sites)
        return ED_ERR_INVALID_ARG;
    const ed_status st = validate_group(n_sites, n_elems, perms, chars);
    if (st != ED_OK)
        return st;
    const int order = n_elems * (spin_inversion ? 2 : 1);
    chi_one.assign((order + 31) / 32, 0);
    for (int g = 0; g < order; ++g) {
        const int p = g % n_elems;
        cplx c(chars[2 * p], chars[2 * p + 1]);
        if (g >= n_elems)
            c *= (double)spin_inversion;
        if (std::abs(c - 1.0) < kChiTol)
            chi_one[g / 32] |= 1u << (g % 32);
    }
    masks32.assign((size_t)n_elems * kMaskStride, 0);
    masks64.assign((size_t)n_elems * kMaskStride, 0);
    for (int g = 0; g < n_elems; ++g) {
        const int32_t *pm = perms + (size_t)g * n_sites;
        if (n_sites <= 32) {
            auto m = benes_masks(5, n_sites, pm);
            for (int k = 0; k < 9; ++k)
                masks32[(size_t)g * kMaskStride + k] = (uint32_t)m[k];
        }
        auto m = benes_masks(6, n_sites, pm);
        for (int k = 0; k < 11; ++k)
            masks64[(size_t)g * kMaskStride + k] = m[k];
    }
    return ED_OK;
}

uint64_t binomial_host(int n, int k) { return binomial(n, k); }

static std::atomic<unsigned long long> g_launches{0};
void count_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
void uncount_launch(unsigned n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
unsigned long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

// Operator/basis compatibility and the symmetry check (cached per basis).
ed_status check_pair(const ed_operator *op, const ed_basis *b)
{
    if (!op || !b)
        return ED_ERR_INVALID_ARG;
    if (op->n_sites != b->n_sites)
        return ED_ERR_INVALID_ARG;
    if (op->checked.load() == b)
        return ED_OK;
    if (!operator_is_symmetric(op, b->n_perm, b->perms.data(), b->spin_inversion))
        return ED_ERR_SYMMETRY_MISMATCH;
    op->checked.store(b);
    return ED_OK;
}

}  // namespace edk

edk::GroupView ed_basis::group_view() const
{
    edk::GroupView g;
    g.n_sites = n_sites;
    g.n_perm = n_perm;
    g.flip = spin_inversion != 0;
    g.order = order;
    g.full = n_sites >= 64 ? ~0ULL : ((1ULL << n_sites) - 1);
    g.masks32 = d_masks32;
    g.masks64 = d_masks64;
    g.chi = d_chi;
    g.chif = d_chif;
    g.chi_one = d_chi_one;
    g.fact = fact && !g_force_generic;
    g.rot_L = rot_L;
    g.rot_d = rot_d;
    g.n_cos = n_cos;
    g.prune = g.fact && rot_d == 1 && !g_force_all_rotations;
    g.cos_kind = d_cos_kind;
    g.cos_masks32 = d_cos_masks32;
    g.cos_masks64 = d_cos_masks64;
    g.fchi = d_fchi;
    g.fchif = d_fchif;
    g.fchi_one = d_fchi_one;
    return g;
}

edk::IndexView ed_basis::index_view() const
{
    edk::IndexView v{d_states, d_norms, d_keys, dim, d_tab, tab_size, e_lo, e_hi, mbits, probe_iters};
    const bool use_hash = (d_htab || d_bkt) && !g_force_prefix;
    v.htab = use_hash ? d_htab : nullptr;
    v.hent = use_hash ? d_hent : nullptr;
    v.hbits = hbits;
    v.hwide = hwide;
    v.norm_bits = norm_bits;
    v.bkt = use_hash ? d_bkt : nullptr;
    v.stash = d_stash;
    v.n_stash = n_stash;
    v.bbits = bbits;
    v.brem = brem;
    return v;
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

ed_status ed_stream_status(void *stream)
{
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return ED_ERR_CUDA;
    }
    unsigned int st = 0, bst = 0;
    if (edk::basis_status_take(&st) != cudaSuccess || edk::batch_status_take(&bst) != cudaSuccess) {
        (void)cudaGetLastError();
        return ED_ERR_CUDA;
    }
    if (st)
        return ED_ERR_INTERNAL;
    return (bst & edk::kStatusTimeout) ? ED_ERR_TIMEOUT : ED_OK;
}

const char *ed_status_string(ed_status s)
{
    switch (s) {
    case ED_OK: return "ok";
    case ED_ERR_INVALID_ARG: return "invalid argument";
    case ED_ERR_NOT_A_GROUP: return "permutations do not form a group";
    case ED_ERR_BAD_CHARACTER: return "characters are not a one-dimensional unitary representation";
    case ED_ERR_SYMMETRY_MISMATCH: return "operator does not commute with the symmetry group";
    case ED_ERR_OOM: return "device out of memory";
    case ED_ERR_CUDA: return "CUDA runtime error";
    case ED_ERR_INTERNAL: return "device-side invariant check failed";
    case ED_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case ED_ERR_NOT_CONVERGED: return "not converged";
    case ED_ERR_UNSUPPORTED: return "unsupported by this build";
    }
    return "unknown status";
}

}  // extern "C"

namespace {
// The basis build; with count_only != null it stops after the count pass and
// the scan and returns the sector dimension there (no basis is kept).
ed_status basis_build_impl(int n_sites, int n_up, int spin_inversion, int n_elems,
                           const int32_t *perms, const double *chars, void *stream_, ed_basis **out,
                           uint64_t *count_only)
{
    if ((!out && !count_only) || !perms || !chars)
        return ED_ERR_INVALID_ARG;
    if (out)
        *out = nullptr;
    // argument and group validation, the chi == 1 bitset and the Benes masks:
    // the same host tables as the allocation-free count
    std::vector<uint32_t> m32, one;
    std::vector<uint64_t> m64;
    ed_status st = edk::count_tables_host(n_sites, n_up, spin_inversion, n_elems, perms, chars, m32, m64, one);
    if (st != ED_OK)
        return st;
    cudaStream_t stream = (cudaStream_t)stream_;

    ed_basis *b = new ed_basis();
    cudaGetDevice(&b->device);
    b->n_sites = n_sites;
    b->n_up = n_up;
    b->spin_inversion = spin_inversion;
    b->n_perm = n_elems;
    b->order = n_elems * (spin_inversion ? 2 : 1);
    b->perms.assign(perms, perms + (size_t)n_elems * n_sites);
    b->chars.assign(chars, chars + 2 * (size_t)n_elems);

    // expanded characters: plain elements, then flipped ones (times z)
    std::vector<double2> chi(b->order);
    std::vector<float2> chif(b->order);
    b->trivial_chars = true;
    b->real_chars = true;
    for (int g = 0; g < b->order; ++g) {
        const int p = g % n_elems;
        cplx c(chars[2 * p], chars[2 * p + 1]);
        if (g >= n_elems)
            c *= (double)spin_inversion;
        chi[g] = make_double2(c.real(), c.imag());
        chif[g] = make_float2((float)c.real(), (float)c.imag());
        b->trivial_chars = b->trivial_chars && ((one[g / 32] >> (g % 32)) & 1u);
        b->real_chars = b->real_chars && std::abs(c.imag()) < kChiTol;
    }
#define ED_B_TRY(expr)                           \
    do {                                         \
        cudaError_t _e = (expr);                 \
        if (_e != cudaSuccess) {                 \
            (void)cudaGetLastError();            \
            free_basis(b);                       \
            edk::ws_free(d_counts, stream);      \
            edk::ws_free(d_flags, stream);       \
            edk::ws_free(d_offsets, stream);     \
            edk::ws_free(d_tmp, stream);         \
            cudaFree(d_binom);                   \
            cudaFree(d_flag);                    \
            return _e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA; \
        }                                        \
    } while (0)
    uint32_t *d_counts = nullptr, *d_flags = nullptr;
    uint64_t *d_offsets = nullptr, *d_tmp = nullptr, *d_binom = nullptr;
    int *d_flag = nullptr;
    ED_B_TRY(upload(&b->d_masks32, m32.data(), m32.size()));
    ED_B_TRY(upload(&b->d_masks64, m64.data(), m64.size()));
    ED_B_TRY(upload(&b->d_chi, chi.data(), chi.size()));
    ED_B_TRY(upload(&b->d_chif, chif.data(), chif.size()));
    ED_B_TRY(upload(&b->d_chi_one, one.data(), one.size()));
    {
        Factorization F;
        if (factorize(n_sites, n_elems, perms, F)) {
            const int nc = (int)F.rep.size();
            std::vector<uint32_t> cm32((size_t)nc * edk::kMaskStride, 0);
            std::vector<uint64_t> cm64((size_t)nc * edk::kMaskStride, 0);
            for (int c = 0; c < nc; ++c) {
                const int32_t *pm = perms + (size_t)F.rep[c] * n_sites;
                if (n_sites <= 32) {
                    auto m = benes_masks(5, n_sites, pm);
                    for (int st2 = 0; st2 < 9; ++st2)
                        cm32[(size_t)c * edk::kMaskStride + st2] = (uint32_t)m[st2];
                }
                auto m = benes_masks(6, n_sites, pm);
                for (int st2 = 0; st2 < 11; ++st2)
                    cm64[(size_t)c * edk::kMaskStride + st2] = m[st2];
            }
            std::vector<double2> fchi(b->order);
            std::vector<float2> fchif(b->order);
            std::vector<uint32_t> fone((b->order + 31) / 32, 0);
            for (int g = 0; g < b->order; ++g) {
                const int fi = g % n_elems;            // factored index within one flip half
                const int src = F.elem[fi] + (g >= n_elems ? n_elems : 0);  // expanded index
                fchi[g] = chi[src];
                fchif[g] = chif[src];
                if ((one[src / 32] >> (src % 32)) & 1u)
                    fone[g / 32] |= 1u << (g % 32);
            }
            ED_B_TRY(upload(&b->d_cos_kind, F.kind.data(), F.kind.size()));
            ED_B_TRY(upload(&b->d_cos_masks32, cm32.data(), cm32.size()));
            ED_B_TRY(upload(&b->d_cos_masks64, cm64.data(), cm64.size()));
            ED_B_TRY(upload(&b->d_fchi, fchi.data(), fchi.size()));
            ED_B_TRY(upload(&b->d_fchif, fchif.data(), fchif.size()));
            ED_B_TRY(upload(&b->d_fchi_one, fone.data(), fone.size()));
            b->fact = true;
            b->rot_L = F.L;
            b->rot_d = F.d;
            b->n_cos = nc;
        }
    }

    // enumeration plan
    std::vector<uint64_t> binom(65 * 65);
    for (int n = 0; n <= 64; ++n)
        for (int k = 0; k <= 64; ++k)
            binom[n * 65 + k] = binomial(n, k);
    ED_B_TRY(upload(&d_binom, binom.data(), binom.size()));
    edk::EnumPlan plan;
    plan.n_sites = n_sites;
    plan.n_up = n_up;
    plan.total = n_up < 0 ? (1ULL << n_sites) : binomial(n_sites, n_up);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const uint64_t threads = (uint64_t)sms * 2048 * 4;
    plan.chunk = std::max<uint64_t>(16, (plan.total + threads - 1) / threads);
    plan.n_chunks = (plan.total + plan.chunk - 1) / plan.chunk;
    plan.binom = d_binom;
    const edk::GroupView gv = b->group_view();

    ED_B_TRY(edk::ws_alloc((void **)&d_counts, plan.n_chunks * sizeof(uint32_t), stream));
    ED_B_TRY(edk::ws_alloc((void **)&d_offsets, (plan.n_chunks + 1) * sizeof(uint64_t), stream));
    ED_B_TRY(edk::ws_alloc((void **)&d_tmp, edk::scan_tmp_words(plan.n_chunks) * sizeof(uint64_t), stream));
    if (!count_only) {  // kept-state bits for the write pass, when they take <= 1/8 of free memory
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const uint64_t words = (plan.chunk + 31) / 32;
        const uint64_t bytes = plan.n_chunks * words * sizeof(uint32_t);
        if (bytes <= free_b / 8 && edk::ws_alloc((void **)&d_flags, bytes, stream) == cudaSuccess) {
            plan.flags = d_flags;
            plan.flag_words = (uint32_t)words;
        }
        (void)cudaGetLastError();
    }
    ED_B_TRY(edk::launch_enum_count(plan, gv, d_counts, stream));
    ED_B_TRY(edk::launch_scan(d_counts, plan.n_chunks, d_offsets, d_tmp, stream));
    uint64_t dim = 0;
    ED_B_TRY(cudaMemcpyAsync(&dim, d_offsets + plan.n_chunks, sizeof(uint64_t),
                             cudaMemcpyDeviceToHost, stream));
    ED_B_TRY(cudaStreamSynchronize(stream));
    if (count_only) {
        *count_only = dim;
        free_basis(b);
        edk::ws_free(d_counts, stream); edk::ws_free(d_offsets, stream); edk::ws_free(d_tmp, stream);
        cudaFree(d_binom);
        return ED_OK;
    }
    if (dim >= (1ULL << 32)) {
        free_basis(b);
        edk::ws_free(d_counts, stream); edk::ws_free(d_flags, stream); edk::ws_free(d_offsets, stream);
        edk::ws_free(d_tmp, stream); cudaFree(d_binom);
        return ED_ERR_UNSUPPORTED;
    }
    b->dim = dim;
    ED_B_TRY(edk::ws_alloc((void **)&b->d_states, std::max<uint64_t>(dim, 1) * sizeof(uint64_t), stream));
    ED_B_TRY(edk::ws_alloc((void **)&b->d_norms, std::max<uint64_t>(dim, 1) * sizeof(uint16_t), stream));
    ED_B_TRY(edk::launch_enum_write(plan, gv, d_offsets, b->d_states, b->d_norms, stream));

    // prefix table over the bit-length range of the basis
    uint64_t ends[2] = {0, 0};
    if (dim) {
        ED_B_TRY(cudaMemcpyAsync(&ends[0], b->d_states, 8, cudaMemcpyDeviceToHost, stream));
        ED_B_TRY(cudaMemcpyAsync(&ends[1], b->d_states + dim - 1, 8, cudaMemcpyDeviceToHost, stream));
        ED_B_TRY(cudaStreamSynchronize(stream));
    }
    auto bitlen = [](uint64_t s) { return s ? 64 - __builtin_clzll(s) : 0; };
    b->e_lo = bitlen(ends[0]);
    b->e_hi = bitlen(ends[1]);
    const int n_exp = b->e_hi - b->e_lo + 1;
    int mb = 0;
    while (mb < 26 && ((uint64_t)n_exp << (mb + 1)) * 2 <= std::max<uint64_t>(dim, 1))
        ++mb;
    b->mbits = mb;
    b->tab_size = (uint64_t)n_exp << mb;
    ED_B_TRY(edk::ws_alloc((void **)&b->d_tab, (b->tab_size + 1) * sizeof(uint32_t), stream));
    ED_B_TRY(edk::launch_prefix_table(b->index_view(), b->d_tab, stream));
    ED_B_TRY(cudaMalloc(&d_flag, 2 * sizeof(int)));
    ED_B_TRY(cudaMemsetAsync(d_flag, 0, 2 * sizeof(int), stream));
    ED_B_TRY(edk::launch_check_sorted(b->d_states, dim, d_flag, stream));
    ED_B_TRY(edk::launch_max_bucket(b->d_tab, b->tab_size, reinterpret_cast<uint32_t *>(d_flag + 1), stream));
    int flag[2] = {0, 0};
    ED_B_TRY(cudaMemcpyAsync(flag, d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, stream));
    ED_B_TRY(cudaStreamSynchronize(stream));
    b->max_bucket = (uint32_t)flag[1];
    {
        unsigned int dev_status = 0;
        ED_B_TRY(edk::basis_status_take(&dev_status));
        flag[0] |= (int)dev_status;
    }
    bool bucketed = false;
    // index kind: the test policy, else the autotuner's choice for sectors
    // like this one, else the bucketed index from kBucketAutoDim states on
    const int tuned = g_index_policy == 0 ? edk::tuned_index_kind(n_sites, b->order, spin_inversion != 0, dim) : 0;
    const bool want_bucket = g_index_policy == 2 || (g_index_policy == 0 && (tuned ? tuned == 2 : dim >= kBucketAutoDim));
    if (dim && want_bucket) {
        int nb = 1;
        while ((1 << nb) <= b->order)
            ++nb;
        bucketed = build_bucket_index(b, nb, stream);
    }
    if (dim && !bucketed) {
        // hash index: 2^hbits >= dim / 2 buckets (one to two states per bucket)
        int hb = 1;
        while ((2ULL << hb) < dim)
            ++hb;
        b->hbits = hb;
        int nb = 1;
        while ((1 << nb) <= b->order)
            ++nb;
        int ib = 1;
        while ((1ULL << ib) < dim)
            ++ib;
        b->norm_bits = nb;
        b->hwide = !(n_sites <= 32 && ib + nb <= 32);
        const uint64_t T = 1ULL << hb;
        uint32_t *d_hcount = nullptr;
        uint64_t *d_hoff = nullptr, *d_htmp = nullptr;
        cudaError_t he = edk::ws_alloc((void **)&d_hcount, T * sizeof(uint32_t), stream);
        if (he == cudaSuccess)
            he = edk::ws_alloc((void **)&d_hoff, (T + 1) * sizeof(uint64_t), stream);
        if (he == cudaSuccess)
            he = edk::ws_alloc((void **)&d_htmp, edk::scan_tmp_words(T) * sizeof(uint64_t), stream);
        if (he == cudaSuccess)
            he = edk::ws_alloc((void **)&b->d_htab, (T + 1) * sizeof(uint32_t), stream);
        if (he == cudaSuccess)
            he = edk::ws_alloc((void **)&b->d_hent, dim * (b->hwide ? 16 : 8), stream);
        if (he == cudaSuccess)
            he = cudaMemsetAsync(d_hcount, 0, T * sizeof(uint32_t), stream);
        if (he == cudaSuccess)
            he = edk::launch_hash_count(b->d_states, dim, hb, d_hcount, stream);
        if (he == cudaSuccess)
            he = edk::launch_scan(d_hcount, T, d_hoff, d_htmp, stream);
        if (he == cudaSuccess)
            he = edk::launch_offsets_to_u32(d_hoff, T + 1, b->d_htab, stream);
        if (he == cudaSuccess)  // reuse the count array as the fill cursor
            he = cudaMemcpyAsync(d_hcount, b->d_htab, T * sizeof(uint32_t), cudaMemcpyDeviceToDevice, stream);
        if (he == cudaSuccess)
            he = edk::launch_hash_fill(b->d_states, b->d_norms, dim, hb, d_hcount, b->d_hent, b->hwide,
                                       b->norm_bits, stream);
        uint32_t hmax = 0;
        uint32_t *d_hmax = reinterpret_cast<uint32_t *>(d_flag);
        if (he == cudaSuccess)
            he = cudaMemsetAsync(d_hmax, 0, sizeof(uint32_t), stream);
        if (he == cudaSuccess)
            he = edk::launch_max_bucket(b->d_htab, T, d_hmax, stream);
        if (he == cudaSuccess)
            he = cudaMemcpyAsync(&hmax, d_hmax, sizeof(uint32_t), cudaMemcpyDeviceToHost, stream);
        if (he == cudaSuccess)
            he = cudaStreamSynchronize(stream);
        edk::ws_free(d_hcount, stream);
        edk::ws_free(d_hoff, stream);
        edk::ws_free(d_htmp, stream);
        ED_B_TRY(he);
        b->hash_max_bucket = hmax;
        // packed keys (state << 16 | norm) for the products' row loads and the
        // prefix-table search: one 8-byte load instead of two streams.  The
        // bucketed index goes without them (rows then read states and norms):
        // at 3.2e9 states they would take 25.6 GB beside the states.
        if (n_sites <= 48) {
            ED_B_TRY(edk::ws_alloc((void **)&b->d_keys, dim * sizeof(uint64_t), stream));
            ED_B_TRY(edk::launch_pack_keys(b->d_states, b->d_norms, dim, b->d_keys, stream));
        }
    }
    {
        int k = 1;  // steps that reduce the largest bucket to one entry, plus the final probe
        while ((1u << (k - 1)) < std::max<uint32_t>(b->max_bucket, 1))
            ++k;
        b->probe_iters = k;
    }
    edk::ws_free(d_counts, stream);
    edk::ws_free(d_flags, stream);
    edk::ws_free(d_offsets, stream);
    edk::ws_free(d_tmp, stream);
    cudaFree(d_binom);
    cudaFree(d_flag);
#undef ED_B_TRY
    if (flag[0]) {
        free_basis(b);
        return ED_ERR_INTERNAL;
    }
    *out = b;
    return ED_OK;
}

}  // namespace

extern "C" {

ed_status ed_basis_build(int n_sites, int n_up, int spin_inversion, int n_elems,
                         const int32_t *perms, const double *chars, void *stream, ed_basis **out)
{
    return basis_build_impl(n_sites, n_up, spin_inversion, n_elems, perms, chars, stream, out, nullptr);
}

ed_status ed_basis_count(int n_sites, int n_up, int spin_inversion, int n_elems, const int32_t *perms,
                         const double *chars, void *stream, uint64_t *dim)
{
    if (!dim)
        return ED_ERR_INVALID_ARG;
    return basis_build_impl(n_sites, n_up, spin_inversion, n_elems, perms, chars, stream, nullptr, dim);
}

ed_status ed_basis_size(const ed_basis *b, uint64_t *dim)
{
    if (!b || !dim)
        return ED_ERR_INVALID_ARG;
    *dim = b->dim;
    return ED_OK;
}

ed_status ed_basis_states(const ed_basis *b, const uint64_t **s, const uint16_t **n)
{
    if (!b || !s || !n)
        return ED_ERR_INVALID_ARG;
    *s = b->d_states;
    *n = b->d_norms;
    return ED_OK;
}

ed_status ed_basis_is_real(const ed_basis *b, int *is_real)
{
    if (!b || !is_real)
        return ED_ERR_INVALID_ARG;
    *is_real = b->real_chars ? 1 : 0;
    return ED_OK;
}

ed_status ed_basis_index(const ed_basis *b, const uint64_t *q, int64_t *idx, uint64_t n,
                         void *stream)
{
    if (!b || (n && (!q || !idx)))
        return ED_ERR_INVALID_ARG;
    if (!n)
        return ED_OK;
    ED_CUDA_TRY(edk::launch_index(b->index_view(), q, idx, n, (cudaStream_t)stream));
    return ED_OK;
}

void ed_basis_destroy(ed_basis *b)
{
    if (b)
        cudaDeviceSynchronize();
    free_basis(b);
}

ed_status ed_operator_create(int n_sites, int n_terms, const double *coeff, const int32_t *sites,
                             const double *local, ed_operator **out)
{
    if (!out || !coeff || !sites || !local)
        return ED_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_sites < 1 || n_sites > 64 || n_terms < 1 || n_terms > 4096)
        return ED_ERR_INVALID_ARG;
    for (int t = 0; t < n_terms; ++t) {
        const int i = sites[2 * t], j = sites[2 * t + 1];
        if (i < 0 || j < 0 || i >= n_sites || j >= n_sites || i == j)
            return ED_ERR_INVALID_ARG;
    }
    for (size_t e = 0; e < (size_t)n_terms * 32; ++e)
        if (!std::isfinite(local[e]))
            return ED_ERR_INVALID_ARG;
    ed_operator *op = build_operator_host(n_sites, n_terms, coeff, sites, local);
    if (!op)
        return ED_ERR_INVALID_ARG;
    cudaError_t e = upload(&op->d_fams, op->h_fams.data(), op->h_fams.size());
    if (e == cudaSuccess)
        e = upload(&op->d_mats, op->h_mats.data(), op->h_mats.size());
    if (e == cudaSuccess)
        e = upload(&op->d_matsf, op->h_matsf.data(), op->h_matsf.size());
    if (e == cudaSuccess)
        e = upload(&op->d_offmask, op->h_offmask.data(), op->h_offmask.size());
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        ed_operator_destroy(op);
        return e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA;
    }
    *out = op;
    return ED_OK;
}

void ed_operator_destroy(ed_operator *op)
{
    if (!op)
        return;
    cudaDeviceSynchronize();
    cudaFree(op->d_fams);
    cudaFree(op->d_mats);
    cudaFree(op->d_matsf);
    cudaFree(op->d_offmask);
    delete op;
}

static ed_status check_matvec_args(const ed_operator *op, const ed_basis *b, const void *x, const void *y,
                                   int nvec, ed_dtype dtype)
{
    if (!op || !b)
        return ED_ERR_INVALID_ARG;
    if (nvec < 1 || nvec > 16)
        return ED_ERR_INVALID_ARG;
    if (dtype != ED_F64 && dtype != ED_F32 && dtype != ED_C128 && dtype != ED_C64)
        return ED_ERR_INVALID_ARG;
    const bool cplx_dtype = dtype == ED_C128 || dtype == ED_C64;
    if (!cplx_dtype && !(b->real_chars && op->real))
        return ED_ERR_INVALID_ARG;
    if (b->dim && (!x || !y))
        return ED_ERR_INVALID_ARG;
    if (((uintptr_t)x | (uintptr_t)y) & 15)
        return ED_ERR_INVALID_ARG;
    if (x == y && b->dim)
        return ED_ERR_INVALID_ARG;
    return edk::check_pair(op, b);
}

ed_status ed_matvec(const ed_operator *op, const ed_basis *b, const void *x, void *y, int nvec,
                    ed_dtype dtype, void *stream)
{
    const ed_status st = check_matvec_args(op, b, x, y, nvec, dtype);
    if (st != ED_OK)
        return st;
    if (!b->dim)
        return ED_OK;
    ED_CUDA_TRY(edk::launch_matvec_v(op_view(op), b->group_view(), b->index_view(), !b->trivial_chars, x, y,
                                     nvec, dtype, edk::tuned_variant(b, nvec, dtype), (cudaStream_t)stream));
    return ED_OK;
}

// Ablation hook (not part of the public header): y = H x by the transposed
// (push) form, one vector, atomic adds into y.  Same arguments as ed_matvec
// with nvec = 1; needs the hash index and an exchange-only operator
// (ED_ERR_UNSUPPORTED otherwise).  Not deterministic in the last bits.
ed_status edx_matvec_push(const ed_operator *op, const ed_basis *b, const void *x, void *y, ed_dtype dtype,
                          void *stream)
{
    const ed_status st = check_matvec_args(op, b, x, y, 1, dtype);
    if (st != ED_OK || !b->dim)
        return st;
    const edk::OpView ov = op_view(op);
    if (!b->d_htab || !ov.exchange_only)
        return ED_ERR_UNSUPPORTED;
    ED_CUDA_TRY(edk::launch_matvec_push(ov, b->group_view(), b->index_view(), !b->trivial_chars, x, y, dtype,
                                        (cudaStream_t)stream));
    return ED_OK;
}

// Diagnostics hook: exact number of stored nonzeros of H in the sector
// (allocates an 8-byte counter; synchronises the device).  Returns 0 or -1.
int edx_count_nnz(const ed_operator *op, const ed_basis *b, unsigned long long *out)
{
    if (!op || !b || !out || edk::check_pair(op, b) != ED_OK)
        return -1;
    *out = 0;
    if (!b->dim)
        return 0;
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess)
        return -1;
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = edk::launch_count_nnz(op_view(op), b->group_view(), b->index_view(), d, 0);
    if (e == cudaSuccess)
        e = cudaMemcpy(out, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : -1;
}

// Test hook (not part of the public header): 1 = use the generic Benes search
// for every group even when the factored form is available (both paths are
// then exercised by the same parity tests).  Affects later launches.
void edx_force_generic(int on) { g_force_generic = on != 0; }

// Test hook: 1 = the factored search visits every rotation of every coset
// image (no pruning to the tops of the longest runs), so that the pruned and
// the exhaustive factored search run through the same parity tests.
void edx_force_all_rotations(int on) { g_force_all_rotations = on != 0; }

// Host-only test hook: the factored form the library finds for a permutation
// group (returns the number of cosets, 0 if there is none); kinds_out gets one
// byte per coset (0 identity, 1 reversal, 2 Benes), at most ne entries.
int edx_factorize(int n, int ne, const int32_t *perms, int *rot_L, int *rot_d, uint8_t *kinds_out)
{
    if (n < 1 || n > 64 || ne < 1 || !perms)
        return -1;
    Factorization F;
    if (!factorize(n, ne, perms, F))
        return 0;
    if (rot_L) *rot_L = F.L;
    if (rot_d) *rot_d = F.d;
    if (kinds_out)
        std::copy(F.kind.begin(), F.kind.end(), kinds_out);
    return (int)F.rep.size();
}

// Test hook: 1 = the matvec finds indices through the prefix table and binary
// search even where the hash index exists.  Affects later launches.
void edx_force_prefix_search(int on) { g_force_prefix = on != 0; }

// Test hook: the index later basis builds make (0 automatic, 1 hash index,
// 2 bucketed index wherever its entry fits).
void edx_index_policy(int policy) { g_index_policy = policy; }

// Diagnostics hook: whether a basis has the bucketed index, its log2 bucket
// count and the number of stashed keys.
int edx_basis_bucket(const ed_basis *b, int *bbits, uint32_t *n_stash)
{
    if (!b)
        return -1;
    if (bbits) *bbits = b->bbits;
    if (n_stash) *n_stash = b->n_stash;
    return b->d_bkt ? 1 : 0;
}

// Diagnostics hook: largest bucket of the hash index and its entry width.
int edx_basis_hash(const ed_basis *b, int *hbits, uint32_t *max_bucket, int *wide)
{
    if (!b)
        return -1;
    if (hbits) *hbits = b->hbits;
    if (max_bucket) *max_bucket = b->hash_max_bucket;
    if (wide) *wide = b->hwide;
    return b->d_htab ? 1 : 0;
}

// Diagnostics hook: prefix-table shape of a basis (entries, largest bucket,
// probe steps of the index search).
int edx_basis_table(const ed_basis *b, uint64_t *tab_size, uint32_t *max_bucket, int *probe_iters)
{
    if (!b)
        return -1;
    if (tab_size) *tab_size = b->tab_size;
    if (max_bucket) *max_bucket = b->max_bucket;
    if (probe_iters) *probe_iters = b->probe_iters;
    return 0;
}

// Diagnostics hook: whether a basis uses the factored search, and its shape.
int edx_basis_factored(const ed_basis *b, int *rot_L, int *rot_d, int *n_cos)
{
    if (!b)
        return -1;
    if (rot_L) *rot_L = b->rot_L;
    if (rot_d) *rot_d = b->rot_d;
    if (n_cos) *n_cos = b->n_cos;
    return b->fact ? 1 : 0;
}

// Diagnostics hook (not part of the public header): kernel launches issued by
// the library since it was loaded.
unsigned long long edx_launch_count(void) { return edk::g_launches.load(); }

// Host-only test hook (not part of the public header): the Benes masks the
// library computes for one permutation, 2*log2w - 1 words.
int edx_benes_masks(int log2w, int n, const int32_t *perm, uint64_t *masks_out)
{
    if (log2w < 1 || log2w > 6 || n < 1 || n > (1 << log2w) || !perm || !masks_out)
        return -1;
    auto m = benes_masks(log2w, n, perm);
    std::copy(m.begin(), m.end(), masks_out);
    return (int)m.size();
}

// Host-only test hook: validate a term list and a permutation group and run the
// operator symmetry check without touching the GPU.  Returns 1 if the operator
// commutes with the group (spin inversion included when nonzero), 0 if not,
// -1 on invalid terms.
int edx_terms_commute(int n_sites, int n_terms, const double *coeff, const int32_t *sites,
                      const double *local, int n_perm, const int32_t *perms, int spin_inversion)
{
    if (n_sites < 1 || n_sites > 64 || n_terms < 1 || !coeff || !sites || !local || !perms)
        return -1;
    for (int t = 0; t < n_terms; ++t) {
        const int i = sites[2 * t], j = sites[2 * t + 1];
        if (i < 0 || j < 0 || i >= n_sites || j >= n_sites || i == j)
            return -1;
    }
    ed_operator *op = build_operator_host(n_sites, n_terms, coeff, sites, local);
    if (!op)
        return -1;
    const int r = operator_is_symmetric(op, n_perm, perms, spin_inversion) ? 1 : 0;
    delete op;
    return r;
}

// Host-only test hook: number of rotation families the term list splits into
// (-1 on invalid terms).
int edx_operator_families(int n_sites, int n_terms, const double *coeff, const int32_t *sites,
                          const double *local)
{
    if (n_sites < 1 || n_sites > 64 || n_terms < 1 || !coeff || !sites || !local)
        return -1;
    for (int t = 0; t < n_terms; ++t) {
        const int i = sites[2 * t], j = sites[2 * t + 1];
        if (i < 0 || j < 0 || i >= n_sites || j >= n_sites || i == j)
            return -1;
    }
    ed_operator *op = build_operator_host(n_sites, n_terms, coeff, sites, local);
    if (!op)
        return -1;
    const int r = (int)op->h_fams.size();
    delete op;
    return r;
}

// Host-only test hook: the group validation of ed_basis_build as a status.
int edx_validate_group(int n_sites, int n_elems, const int32_t *perms, const double *chars)
{
    return (int)validate_group(n_sites, n_elems, perms, chars);
}

}  // extern "C"
