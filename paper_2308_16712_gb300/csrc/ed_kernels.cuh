// ed_kernels.cuh -- launch wrappers exported by the kernel translation units to
// the host API (ed_api.cu).  All functions enqueue on `stream` and return the
// CUDA error of the launch.
#pragma once

#include "ed_internal.cuh"

namespace edk {

// Library-owned, stream-ordered device memory (see ed_pool.cu): allocations
// and frees are ordered on stream s; freed memory stays cached for later calls.
cudaError_t ws_alloc(void **p, size_t bytes, cudaStream_t s);
cudaError_t ws_free(void *p, cudaStream_t s);
// Bytes the pool holds freed and ready for reuse (counted as free memory when
// a solver decides whether its vectors fit).
size_t ws_cached_bytes();

// Kernel launches issued by the library since it was loaded (diagnostics).
void count_launch(unsigned n = 1);
// Takes back n counted launches (kernels recorded into a graph by stream
// capture are counted again each time the graph is launched).
void uncount_launch(unsigned n);
unsigned long long launches_so_far();

// ---- basis build (Sec. "States enumeration") --------------------------------
struct EnumPlan {
    int n_sites;
    int n_up;            // -1: all 2^n_sites states
    uint64_t total;      // states to visit
    uint64_t chunk;      // states per thread
    uint64_t n_chunks;
    const uint64_t *binom;  // device (65 x 65) binomial table
    // Optional: one bit per visited state, set by the count pass for the
    // states it keeps (flag_words 32-bit words per chunk); the write pass then
    // tests only those states again (for their norms) instead of all of them.
    uint32_t *flags = nullptr;
    uint32_t flag_words = 0;
};

// Reads and clears the basis kernels' device status word (synchronous).
cudaError_t basis_status_take(unsigned int *status);
// Status word of the batched matvec launches: kStatusTimeout = a block gave up
// a bounded wait.  Reads and clears the word of the current device.
constexpr unsigned kStatusTimeout = 2u;
cudaError_t batch_status_take(unsigned int *st);
// Pass 1: per-chunk representative counts.
cudaError_t launch_enum_count(const EnumPlan &plan, const GroupView &g, uint32_t *counts,
                              cudaStream_t stream);
// Pass 2: write representatives and norms at offsets[chunk].
cudaError_t launch_enum_write(const EnumPlan &plan, const GroupView &g, const uint64_t *offsets,
                              uint64_t *states, uint16_t *norms, cudaStream_t stream);
// Exclusive scan of n uint32 counts into n + 1 uint64 offsets (offsets[n] = total).
// `tmp` must hold scan_tmp_words(n) uint64 words.
size_t scan_tmp_words(uint64_t n);
cudaError_t launch_scan(const uint32_t *counts, uint64_t n, uint64_t *offsets, uint64_t *tmp,
                        cudaStream_t stream);
// Prefix table over the ascending basis.
cudaError_t launch_prefix_table(const IndexView &ix, uint32_t *tab, cudaStream_t stream);
// Hash index build: counts[b] += 1 for every state's bucket (counts zeroed),
// then (after an exclusive scan into offsets) entries scattered into buckets.
cudaError_t launch_hash_count(const uint64_t *states, uint64_t dim, int hbits, uint32_t *counts,
                              cudaStream_t stream);
cudaError_t launch_offsets_to_u32(const uint64_t *offsets, uint64_t n, uint32_t *out, cudaStream_t stream);
cudaError_t launch_hash_fill(const uint64_t *states, const uint16_t *norms, uint64_t dim, int hbits,
                             uint32_t *cursor, void *entries, int wide, int norm_bits,
                             cudaStream_t stream);
// Bucketed index build: every basis state into the first free slot of its
// primary bucket, else of its alternative bucket, else appended to the stash
// (at most stash_cap entries; *n_stash counts every stash insertion, so a value
// above stash_cap means entries were dropped).  bkt must be all ones (empty),
// cnt (2^bbits counters) zero.
cudaError_t launch_bucket_fill(const uint64_t *states, const uint16_t *norms, uint64_t dim, int n_sites,
                               int bbits, int brem, uint32_t *cnt, uint64_t *bkt, ulonglong2 *stash,
                               uint32_t *n_stash, uint32_t stash_cap, cudaStream_t stream);
// *out = max over buckets of tab[t+1] - tab[t] (*out must start at 0)
cudaError_t launch_max_bucket(const uint32_t *tab, uint64_t tab_size, uint32_t *out, cudaStream_t stream);
// keys[i] = states[i] << 16 | norms[i]
cudaError_t launch_pack_keys(const uint64_t *states, const uint16_t *norms, uint64_t dim, uint64_t *keys,
                             cudaStream_t stream);
// Sets *flag to 1 if the basis is not strictly ascending.
cudaError_t launch_check_sorted(const uint64_t *states, uint64_t dim, int *flag, cudaStream_t stream);

// ---- state -> index -----------------------------------------------------------
cudaError_t launch_index(const IndexView &ix, const uint64_t *query, int64_t *out, uint64_t n,
                         cudaStream_t stream);

// ---- matvec (Sec. "Matrix-vector product") --------------------------------------
struct OpView {
    int n_fam;
    int n_mats;
    int max_terms;           // most off-diagonal terms one row can produce
    const OpFamily *fams;    // rotation families
    const double2 *mats;     // n_mats x 16, coeff * h
    const float2 *matsf;
    const uint8_t *offmask;  // n_mats x 4: bit c' set if h[c'][c] != 0, c' != c
    int exchange_only;       // every off-diagonal entry couples |01> and |10>
};

// Host tables (generic group search) for counting a sector; validates the group.
ed_status count_tables_host(int n_sites, int n_up, int spin_inversion, int n_elems,
                            const int32_t *perms, const double *chars,
                            std::vector<uint32_t> &masks32, std::vector<uint64_t> &masks64,
                            std::vector<uint32_t> &chi_one);
uint64_t binomial_host(int n, int k);

// The index ed_basis_build makes (test hook and autotuner): 0 automatic,
// 1 hash index, 2 bucketed index where its entry fits.
int index_policy_get();
void index_policy_set(int policy);

// Operator/basis compatibility check (n_sites, symmetry); cached per basis.
ed_status check_pair(const ed_operator *op, const ed_basis *b);
OpView make_op_view(const ed_operator *op);

// *total += stored nonzeros of H in the sector (off-diagonal terms found in
// the basis plus one diagonal entry per row)
cudaError_t launch_count_nnz(const OpView &op, const GroupView &g, const IndexView &ix,
                             unsigned long long *total, cudaStream_t stream);

cudaError_t launch_matvec(const OpView &op, const GroupView &g, const IndexView &ix, bool track,
                          const void *x, void *y, int nvec, ed_dtype dtype, cudaStream_t stream);
// A product variant: kernel 0 = the library's rule (use_term_parallel),
// 1 = row-per-lane, 2 = term-parallel (where it applies); prune -1 = the
// group's own setting, 0 = every rotation, 1 = the pruned search (rotation
// step one site only).
struct MatvecVariant {
    int kernel = 0;
    int prune = -1;
};
cudaError_t launch_matvec_v(const OpView &op, GroupView g, const IndexView &ix, bool track, const void *x,
                            void *y, int nvec, ed_dtype dtype, MatvecVariant v, cudaStream_t stream);
// The variant ed_autotune found fastest for this basis, nvec and dtype on the
// current GPU (the default variant when none was tuned).
MatvecVariant tuned_variant(const ed_basis *b, int nvec, ed_dtype dtype);
// The index kind (1 hash, 2 bucketed) ed_autotune_index found faster for
// sectors like this one on the current GPU, or 0 when none was tuned.
int tuned_index_kind(int n_sites, int order, int flip, uint64_t dim);
// The transposed (push) form, one vector, for the ablation hook: y zeroed,
// then every contribution added atomically (order-dependent rounding).
cudaError_t launch_matvec_push(const OpView &op, const GroupView &g, const IndexView &ix, bool track,
                               const void *x, void *y, ed_dtype dtype, cudaStream_t stream);

// Kernel choice for one vector and an exchange-only operator: 0 = the
// term-parallel kernel in single precision, the row-per-lane kernel in double
// precision (where the term-parallel kernel's fp64 segmented sums cost more
// than they save); 1 = always row-per-lane; 2 = always term-parallel.
extern int g_kernel_policy;
bool use_term_parallel(int nvec, const OpView &op, ed_dtype dtype, int n_sites);

}  // namespace edk
