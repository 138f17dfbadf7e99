/*
 * ed.h -- C ABI of the GB300 symmetry-adapted exact-diagonalization hot path.
 *
 * The library implements the two operations the paper builds its exact
 * diagonalization on, for spin-1/2 systems on one GPU:
 *
 *  - the basis of symmetry representatives (Sec. "States enumeration";
 *    Background, Fig. 1: U(1) restriction and lattice symmetries), stored as
 *    one ascending uint64 array with an integer orbit norm per element;
 *  - the matrix-free matrix-vector product y_i = sum_j H_ij x_j over that
 *    basis (Sec. "Matrix-vector product"), computed row by row ("pull"),
 *    without atomics, by generating H|r> term by term, mapping every produced
 *    state to its representative and finding that representative's index by
 *    search in the sorted basis ("stateToIndex");
 *
 * plus the Krylov eigensolver that consumes it (Background: Lanczos).
 *
 * Conventions (used by every call):
 *  - site i <-> bit i of a uint64 state, bit value 1 = spin up; at most 64 sites.
 *  - a group element is a site permutation perm (site i goes to site perm[i]:
 *    bit perm[i] of g.s equals bit i of s) with a character chi (complex, |chi|=1).
 *    Spin inversion F (complement all n_sites bits) is added by the library as
 *    a direct-product factor with character z = spin_inversion.
 *  - representative rep(s) = min over the group of g.s (unsigned compare);
 *    orbit norm n(s) = |Stab(s)| if chi == 1 on the stabilizer, else 0; the
 *    basis holds the states with s == rep(s) and n(s) != 0, ascending.
 *  - matrix element (pull form): for row r and each term of H|r> = sum_s h_s|s>
 *    with r' = rep(s) = g*.s:  y_r += conj(h_s) chi(g*) sqrt(n(r')/n(r)) x_idx(r').
 *  - vectors are device arrays laid out [dim][nvec] (nvec values of one basis
 *    row are contiguous), 16-byte aligned; complex values are (re, im) pairs.
 *
 * Ownership: handles are created and destroyed by the library and are not
 * modified after creation (they may be used from several streams at once).
 * Device arrays passed in (x, y, queries, results) belong to the caller.
 * Host arrays passed in are only read during the call.
 *
 * Errors: every call returns an ed_status.  Argument and shape errors are
 * detected on the host before any launch.  A `stream` argument is a
 * cudaStream_t (NULL = the legacy default stream); calls that take one enqueue
 * their work on it and return without synchronising unless stated otherwise.
 */
#ifndef ED_H
#define ED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ED_OK = 0,
    ED_ERR_INVALID_ARG = 1,      /* null pointer, size out of range, misaligned array */
    ED_ERR_NOT_A_GROUP = 2,      /* not closed, no identity, repeated element, not a permutation */
    ED_ERR_BAD_CHARACTER = 3,    /* |chi| != 1 or chi(a b) != chi(a) chi(b) (tolerance 1e-9) */
    ED_ERR_SYMMETRY_MISMATCH = 4,/* the operator does not commute with the group */
    ED_ERR_OOM = 5,              /* device allocation failed */
    ED_ERR_CUDA = 6,             /* a CUDA runtime call failed */
    ED_ERR_INTERNAL = 7,         /* a device-side invariant check failed */
    ED_ERR_NOT_CONVERGED = 8,    /* Lanczos residual above the requested tolerance */
    ED_ERR_UNSUPPORTED = 9,      /* valid request outside what this build implements */
    ED_ERR_TIMEOUT = 10          /* a bounded device-side wait ran out (reported by ed_stream_status) */
} ed_status;

typedef enum {
    ED_F64 = 0,  /* double                     */
    ED_F32 = 1,  /* float                      */
    ED_C128 = 2, /* complex double, (re, im)   */
    ED_C64 = 3   /* complex float, (re, im)    */
} ed_dtype;

typedef struct ed_basis ed_basis;
typedef struct ed_operator ed_operator;

/*
 * ed_release_cached_memory -- the library takes the arrays it allocates itself
 * (the solvers' work vectors, the basis build's temporaries, the large arrays
 * of a basis) from a stream-ordered device memory pool of its own, which keeps
 * up to min(8 GiB, 1/16 of the device memory) of freed memory cached for the
 * next call (allocating and freeing gigabytes with cudaMalloc / cudaFree costs
 * milliseconds and synchronises the device).  This call returns the cached
 * memory to the device.  Errors: ED_ERR_CUDA.
 */
ed_status ed_release_cached_memory(void);

/* Human-readable name of a status code (static string). */
const char *ed_status_string(ed_status status);

/*
 * ed_stream_status -- errors found on the device by work enqueued earlier.
 * The paper's runtime needs no such call (its errors surface synchronously);
 * here kernels run asynchronously and record violated invariants in a device
 * status word instead of trapping (e.g. the enumeration's write pass finding a
 * chunk whose count differs from its count pass; a batched launch whose
 * blocks gave up a bounded wait).  Synchronises `stream`, then reads and
 * clears the words.
 * Returns ED_OK, ED_ERR_INTERNAL (an invariant failed), ED_ERR_TIMEOUT (a
 * bounded wait ran out; the launch ended without touching its outputs) or
 * ED_ERR_CUDA (an asynchronous launch or execution error).
 */
ed_status ed_stream_status(void *stream);

/*
 * ed_basis_build -- enumerate the representatives of one symmetry sector
 * (Sec. "States enumeration": chunked filter of the bitstring range; the
 * filter condition is the representative test and nonzero orbit norm above).
 *
 *   n_sites        1..64
 *   n_up           number of up spins (U(1) sector, Background / Fig. 1), 0..n_sites;
 *                  -1 = no U(1) restriction (then n_sites <= 40)
 *   spin_inversion 0 (not used), +1 or -1 (its character z); nonzero requires
 *                  2*n_up == n_sites or n_up == -1
 *   n_elems        number of lattice group elements, 1..1024
 *   perms          host, n_elems x n_sites int32, row g = permutation of element g
 *   chars          host, n_elems x 2 double (re, im) = chi(g); must be a
 *                  one-dimensional unitary representation of the permutation group
 *   stream         cudaStream_t for the enumeration kernels
 *   out            receives the new handle
 *
 * The call synchronises `stream` (to size its arrays) and returns with the
 * basis ready; its large arrays come from the library's memory pool (see
 * ed_release_cached_memory).  Device memory per state: 10 bytes (states and
 * norms) plus about 1 byte of prefix table, plus the index: about 18-36 bytes
 * for the bucketed index (sectors of 2^23 states or more; 32-byte buckets,
 * one per 1.8 states or fewer), else 10-20 bytes for the hash index and 8 for
 * packed (state, norm) keys.  Errors:
 * ED_ERR_INVALID_ARG, ED_ERR_NOT_A_GROUP, ED_ERR_BAD_CHARACTER, ED_ERR_OOM,
 * ED_ERR_CUDA, ED_ERR_INTERNAL.
 */
ed_status ed_basis_build(int n_sites, int n_up, int spin_inversion, int n_elems,
                         const int32_t *perms, const double *chars, void *stream,
                         ed_basis **out);

/*
 * ed_basis_count -- the sector dimension only: the count pass of the
 * enumeration and its scan, without keeping the basis (Table 2 of the paper
 * lists such dimensions, up to 48 spins, which no single GPU could store).
 * Arguments as ed_basis_build; the dimension may exceed 2^32.  The per-chunk
 * counts and the scan's arrays come from the library's memory pool and go
 * back to it; the group and binomial tables are allocated with cudaMalloc and
 * freed (which synchronises the device).  Synchronises `stream`.
 */
ed_status ed_basis_count(int n_sites, int n_up, int spin_inversion, int n_elems,
                         const int32_t *perms, const double *chars, void *stream, uint64_t *dim);

/* Number of representatives (the sector dimension). */
ed_status ed_basis_size(const ed_basis *basis, uint64_t *dim);

/* Borrowed device pointers to the ascending states (dim x uint64) and the
 * orbit norms (dim x uint16).  Valid until ed_basis_destroy. */
ed_status ed_basis_states(const ed_basis *basis, const uint64_t **d_states,
                          const uint16_t **d_norms);

/* 1 if every character (spin inversion included) is real, else 0: real
 * sectors may use ED_F64 / ED_F32 vectors, complex ones need ED_C128 / ED_C64. */
ed_status ed_basis_is_real(const ed_basis *basis, int *is_real);

/*
 * ed_basis_index -- "stateToIndex" (Sec. "Matrix-vector product"): position
 * of each query state in the basis, or -1 if it is not a basis element.
 *   d_query  device, n x uint64;  d_index  device, n x int64 (written).
 */
ed_status ed_basis_index(const ed_basis *basis, const uint64_t *d_query, int64_t *d_index,
                         uint64_t n, void *stream);

/* Release the basis and its device memory (synchronises the device). */
void ed_basis_destroy(ed_basis *basis);

/*
 * ed_basis_count_noalloc -- the sector dimension (the number of
 * representatives ed_basis_build would keep), computed without allocating any
 * device memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc -- an application whose memory pool or
 * caching allocator already owns the device memory, or a latency-critical
 * path on which cudaMalloc / cudaFree (which synchronise the device) are not
 * allowed.
 *
 *   arguments   as ed_basis_build, with at most 512 lattice elements
 *               (n_elems > 512 returns ED_ERR_INVALID_ARG: the scratch has a
 *               fixed size) and at most 2^42 enumerated states (C(n_sites,
 *               n_up), or 2^n_sites without U(1); C(44, 22) fits): the
 *               enumeration has at most 2^18 chunks of at most 2^24 states,
 *               and a larger sector returns ED_ERR_UNSUPPORTED before any
 *               CUDA call (count it with ed_basis_count)
 *   dim_out     host, receives the dimension
 *
 * All scratch (group tables, per-chunk counts, scan offsets; about 3.2 MB) is
 * one fixed device array inside the library, present on every device that
 * loads it until the process exits.  The first call on a device looks up the
 * array's device address (make that first call before any stream capture).
 * Every call reuses the same array: calls that overlap on the GPU (different
 * streams or host threads at once) race and must be serialised by the caller.
 * The call enqueues on `stream` and synchronises it before returning.
 * Errors: as ed_basis_build, plus ED_ERR_INVALID_ARG for n_elems > 512 and
 * ED_ERR_UNSUPPORTED for more than 2^42 enumerated states.
 */
ed_status ed_basis_count_noalloc(int n_sites, int n_up, int spin_inversion, int n_elems,
                                 const int32_t *perms, const double *chars, void *stream,
                                 uint64_t *dim_out);

/*
 * ed_operator_create -- H = sum_t coeff_t * h_t acting on the site pair
 * (sites[2t], sites[2t+1]) (the analytic Hamiltonian the matrix elements are
 * generated from, Sec. "Matrix-vector product", getRow / getManyRows).
 *
 *   n_sites  1..64
 *   n_terms  1..4096
 *   coeff    host, n_terms x 2 double (re, im)
 *   sites    host, n_terms x 2 int32, two distinct sites in [0, n_sites)
 *   local    host, n_terms x 16 x 2 double: the 4x4 complex matrix h_t on
 *            |s_i s_j>, row-major, row/column index 2*s_i + s_j
 *
 * H must be Hermitian for the matrix elements above to be those of H.
 * Errors: ED_ERR_INVALID_ARG.
 */
ed_status ed_operator_create(int n_sites, int n_terms, const double *coeff,
                             const int32_t *sites, const double *local, ed_operator **out);

void ed_operator_destroy(ed_operator *op);

/*
 * ed_matvec -- y = H x over the basis (Sec. "Matrix-vector product",
 * y_i = sum_j H_ij x_j), overwriting y.
 *
 *   d_x, d_y  device, dim x nvec of `dtype`, 16-byte aligned, not overlapping
 *   nvec      1..16 vectors multiplied at once (one representative search per
 *             matrix element serves all of them)
 *   dtype     ED_F64 / ED_F32 (real sectors only) or ED_C128 / ED_C64;
 *             the arithmetic is done in that precision
 *
 * Two kernels: rows handed to lanes (each lane walks its row's terms), and,
 * for nvec = 1 in single precision (and in double precision above 32 sites)
 * or an fp32 block of nvec = 8, with an operator whose off-diagonal entries
 * only exchange antiparallel spins (|01> <-> |10>), a term-parallel
 * kernel (a warp lays a tile's terms out flat, one term per lane per round,
 * and sums each row with a segmented warp scan).  The two sum a row's terms in
 * different orders, so a column of an nvec > 1 product may differ from the
 * nvec = 1 product in the last bits.  ed_autotune replaces this rule (and the
 * choice of representative search) by measured choices for sectors of the
 * same shape.  On a real block of 8 vectors the term-parallel kernel sums
 * every column in the order of its single-vector form.
 *
 * No allocation and no host synchronisation.  Deterministic: the same inputs
 * give bit-identical y.  Errors: ED_ERR_INVALID_ARG (including a complex
 * sector with a real dtype, or operator/basis with different n_sites),
 * ED_ERR_SYMMETRY_MISMATCH, ED_ERR_CUDA.
 */
ed_status ed_matvec(const ed_operator *op, const ed_basis *basis, const void *d_x, void *d_y,
                    int nvec, ed_dtype dtype, void *stream);

/* One sector of a batched product: y = H x over `basis` (x, y as in ed_matvec). */
typedef struct {
    const ed_basis *basis;
    const void *d_x;
    void *d_y;
} ed_sector;

/*
 * ed_matvec_multi -- y_s = H x_s for up to 160 symmetry sectors in one
 * persistent launch (the matvec of Sec. "Matrix-vector product" applied to a
 * batch of sectors of uneven dimension, so that no launch tail is paid per
 * sector).  The launch's warps take 32-row tiles from a device work queue (an
 * atomic counter over the tiles of all sectors, largest sectors first), the
 * role the paper's producer/consumer balancing plays across nodes.  Every basis must be built from the same n_sites and the same list
 * of lattice permutations (characters, spin inversion and n_up may differ);
 * dtype must be complex if any sector is.  Sectors with dimension 0 are
 * skipped.  Results equal those of ed_matvec on each sector, bit for bit.
 *
 *   sectors   host array of n_sectors entries
 *   nvec, dtype, stream   as ed_matvec
 *
 * No allocation; no host synchronisation.  Errors: ED_ERR_INVALID_ARG (also
 * for sectors with different permutations), ED_ERR_SYMMETRY_MISMATCH,
 * ED_ERR_CUDA.
 */
ed_status ed_matvec_multi(const ed_operator *op, const ed_sector *sectors, int n_sectors, int nvec,
                          ed_dtype dtype, void *stream);

/* Lanczos precision modes. */
typedef enum {
    ED_LANCZOS_F64 = 0,        /* fp64 matvec, fp64 recurrence                     */
    ED_LANCZOS_F32_MATVEC = 1, /* fp32 matvec, fp64 recurrence and fp64 refinement */
    ED_LANCZOS_RECOMPUTE = 16, /* flag: form the Ritz vector (and that of the fp64
                                  refinement) by a second pass even when the
                                  Krylov vectors would fit in memory              */
    ED_LANCZOS_PUSH = 32,      /* flag (ed_lanczos only): products by the transposed
                                  ("push") form -- every term added to y at its
                                  representative's index with an atomic add, the
                                  paper's distributed product.  Faster on GB300 (no
                                  x gather, no per-row sums) but y, and so E0, vary
                                  in the last bits from run to run.  Needs the
                                  Krylov vectors kept in memory and an operator
                                  whose off-diagonal entries only exchange
                                  antiparallel spins; ED_ERR_UNSUPPORTED otherwise */
    ED_LANCZOS_REORTH = 64     /* flag (ed_lanczos, ed_lanczos_eigs): reorthogonalise
                                  every new Lanczos vector against all earlier ones
                                  (classical Gram-Schmidt, twice, fp64), which keeps
                                  the Ritz values free of spurious copies so that the
                                  low excited states come out too; costs about
                                  4 j vector reads at step j.  Needs the Krylov
                                  vectors kept in memory; ED_ERR_UNSUPPORTED otherwise */,
    ED_LANCZOS_VALUES_ONLY = 128 /* flag (ed_lanczos, ed_lanczos_block): the Ritz
                                  values of the main run only -- no Ritz vector,
                                  no second pass, no refinement; e0 is the lowest
                                  Ritz value and residual the recurrence's own
                                  estimate |beta_{m+1} s_m| (|B_{m+1} s_m| for
                                  blocks) of |H psi - e0 psi|; d_vec_out must be
                                  NULL */
} ed_lanczos_mode;

typedef struct {
    int steps;            /* Lanczos steps taken (stops early on an invariant subspace) */
    int matvecs;          /* matrix-vector products performed, refinement included */
    double ritz;          /* lowest Ritz value of the tridiagonal matrix */
    double e0;            /* returned energy: fp64 Rayleigh quotient of the Ritz vector */
    double residual;      /* |H psi - e0 psi| / |psi| in fp64 */
    double matvec_ms;     /* device time spent in the matvec kernels, summed over
                             the products launched one by one (CUDA events on
                             `stream` around each); ed_lanczos replays the steps
                             of sectors of at most 2^22 states from a CUDA graph
                             and does not time those products (0)               */
} ed_lanczos_info;

/*
 * ed_lanczos -- lowest eigenvalue of H in the sector by the Lanczos
 * recurrence (Background: Krylov methods consume hundreds of matvecs).
 *
 *   d_x0      device start vector, dim values: double for real sectors,
 *             (re, im) double pairs for complex ones; need not be normalised
 *   steps     1..10000 Lanczos steps (no restart)
 *   mode      ED_LANCZOS_F64 or ED_LANCZOS_F32_MATVEC, optionally OR-ed with
 *             ED_LANCZOS_RECOMPUTE or ED_LANCZOS_PUSH
 *   e0_out    host, receives the energy (may be NULL)
 *   d_vec_out device, dim values as d_x0, receives the normalised ground-state
 *             approximation (may be NULL)
 *   info      host, filled (may be NULL)
 *
 * The alpha/beta recurrence, dot products (compensated fp64 sums) and the
 * tridiagonal eigensolve run in fp64 on the GPU.  The Ritz vector is formed
 * from stored Krylov vectors when they fit in device memory, else by a second,
 * bit-identical pass of the recurrence.  It is then refined in fp64: a few
 * fp64 Lanczos steps started from it (their vectors stored, or recomputed by
 * a second pass in the same way), whose lowest Ritz value is returned
 * together with its residual.  Work memory beyond the caller's vectors: four
 * fp64 vectors, plus two fp32 vectors in the fp32-matvec mode, when the
 * Krylov vectors are not stored.  Sectors of at most 2^22 states are
 * launch-bound: there the steps after the first are replayed from a CUDA
 * graph of two steps (same kernels, same results).  Not to be called while
 * `stream` is being captured.  Takes its work vectors from the library's
 * memory pool (see ed_release_cached_memory); synchronises `stream` before
 * returning.
 * Errors: ED_ERR_INVALID_ARG, ED_ERR_SYMMETRY_MISMATCH, ED_ERR_UNSUPPORTED
 * (ED_LANCZOS_PUSH not applicable), ED_ERR_OOM, ED_ERR_CUDA.
 */
ed_status ed_lanczos(const ed_operator *op, const ed_basis *basis, const void *d_x0, int steps,
                     int mode, double *e0_out, void *d_vec_out, ed_lanczos_info *info,
                     void *stream);

/*
 * ed_lanczos_eigs -- ed_lanczos that also returns the lowest n_eig Ritz values
 * of the main run's tridiagonal matrix (Sturm-count multisection for each),
 * the estimates of the lowest n_eig eigenvalues of H in the sector.
 *
 *   n_eig     0..steps
 *   eigs_out  host, n_eig values, ascending; NaN past the dimension of the
 *             Krylov space actually built (a sector smaller than `steps`)
 *   tol       > 0: return ED_ERR_NOT_CONVERGED (with every output filled) when
 *             the fp64 residual |H psi - e0 psi| / |psi| of the returned state
 *             exceeds tol; <= 0: no check
 *   other arguments as ed_lanczos (the refined lowest energy is in info->e0)
 *
 * Without ED_LANCZOS_REORTH the plain recurrence loses orthogonality once the
 * lowest Ritz value has converged and may then repeat converged values
 * ("ghosts") among the higher ones; with it, the values are those of an
 * orthonormal Krylov basis.  In the fp32-matvec mode the values carry the fp32
 * products' error (about 1e-7 relative); only the lowest is refined.
 * Errors as ed_lanczos, ED_ERR_INVALID_ARG for n_eig out of range,
 * ED_ERR_NOT_CONVERGED as above.
 */
ed_status ed_lanczos_eigs(const ed_operator *op, const ed_basis *basis, const void *d_x0, int steps,
                          int mode, int n_eig, double *eigs_out, double tol, void *d_vec_out,
                          ed_lanczos_info *info, void *stream);

/*
 * ed_lanczos_block -- lowest eigenvalues of H in a real sector by the block
 * Lanczos recurrence on nvec vectors at once (Background: Krylov methods
 * consume hundreds of matrix-vector products; here every product is one
 * interleaved block product, in which one representative search and index
 * lookup per matrix element serves all nvec columns, Sec. "Matrix-vector
 * product").
 *
 *   d_x0      device start block, dim x nvec doubles laid out [dim][nvec]
 *             (need not be orthonormal; must have rank nvec)
 *   nvec      block size: 2, 4, 8 or 16
 *   steps     1..10000 block steps (no restart); the recurrence stops early
 *             when the block Krylov space stops growing
 *   mode      ED_LANCZOS_F64 (fp64 block products) or ED_LANCZOS_F32_MATVEC
 *             (products of the block's fp32 copy), optionally OR-ed with
 *             ED_LANCZOS_REORTH: every block is kept and each new one is
 *             orthogonalised against all earlier ones (block modified
 *             Gram-Schmidt, twice), so that the higher Ritz values carry no
 *             spurious copies of converged ones; needs the blocks to fit in
 *             half of the free memory (ED_ERR_UNSUPPORTED otherwise)
 *   n_eig     0..nvec*steps lowest Ritz values to return in eigs_out (host,
 *             ascending; NaN past the dimension of the space built)
 *   e0_out    host, the refined lowest energy (may be NULL)
 *   d_vec_out device, dim doubles, the normalised ground-state approximation
 *             (may be NULL)
 *   info      host (may be NULL); steps = block steps taken, matvecs = block
 *             products plus the refinement's single products, ritz = lowest
 *             Ritz value of the block recurrence
 *
 * The blocks and their coefficient matrices are fp64: for every step
 * C = V_j^T W and Cp = V_{j-1}^T W of the product W = H V_j (compensated
 * fp64 sums over a fixed partition), W -= V_j C + V_{j-1} Cp, and a Cholesky
 * QR applied twice gives the next block and the coupling B_{j+1}.  The lowest
 * eigenpair of the block tridiagonal matrix (bandwidth nvec) is found on the
 * GPU by bisection with Sturm counts of its banded LDL^T factorisation and by
 * inverse iteration; the Ritz vector by a second, bit-identical pass (no
 * block is stored); the energy is then refined exactly as ed_lanczos's
 * fp32-matvec mode does (a short fp64 single-vector Lanczos run from the
 * Ritz vector; fp64 Rayleigh quotient and residual).  Memory: three blocks
 * of fp64 (two in the fp32 mode, plus two fp32 blocks) from the library's
 * pool.  Synchronises `stream` before returning.
 * Errors: ED_ERR_INVALID_ARG (also nvec not in {2, 4, 8, 16}, a sector
 * smaller than nvec or a start block of lower rank), ED_ERR_SYMMETRY_MISMATCH,
 * ED_ERR_UNSUPPORTED (complex sectors or operators), ED_ERR_OOM, ED_ERR_CUDA.
 */
ed_status ed_lanczos_block(const ed_operator *op, const ed_basis *basis, const void *d_x0, int nvec, int steps,
                           int mode, int n_eig, double *eigs_out, double *e0_out, void *d_vec_out,
                           ed_lanczos_info *info, void *stream);

/*
 * ed_lanczos_multi -- lowest eigenvalue of H in each of up to 160 symmetry
 * sectors, by the recurrence of ed_lanczos run on all sectors together
 * (Sec. "Introduction": symmetries make H block diagonal, one independent
 * eigenproblem of reduced dimension per block; here many blocks at once).
 * Every product is one multi-sector launch as in ed_matvec_multi (tiles from
 * a device work queue); the vector updates and the compensated fp64 dot
 * products are segmented per sector; each run of steps is captured once as a
 * CUDA graph of two steps and replayed.
 * The sectors follow the rules of ed_matvec_multi (same n_sites and lattice
 * permutations); every sector must be non-empty.
 *
 *   sectors   host array; d_x = device start vector (dim values of `dtype`,
 *             need not be normalised), d_y = device output for the normalised
 *             ground-state approximation (may be NULL)
 *   steps     1..10000 Lanczos steps, the same for every sector; a sector that
 *             reaches an invariant subspace stops contributing early
 *   mode      ED_LANCZOS_F64 or ED_LANCZOS_F32_MATVEC, optionally OR-ed with
 *             ED_LANCZOS_RECOMPUTE (form the Ritz vectors by a second pass even
 *             when the Lanczos vectors would fit in memory)
 *   dtype     ED_F64 (every sector and H real) or ED_C128: the type of d_x, d_y
 *   e0_out    host, n_sectors energies (may be NULL)
 *   info      host, n_sectors entries (may be NULL); matvecs counts the batched
 *             products; matvec_ms is 0 (products inside a graph are not timed
 *             one by one)
 *
 * The Lanczos vectors are kept when they fit in half of the free device
 * memory (in the fp32-matvec mode as the fp32 copies the products consumed:
 * that Ritz vector only starts the fp64 refinement), else the Ritz vectors
 * come from a second, bit-identical pass.  Per sector the energy is the fp64
 * Rayleigh quotient of its final vector, as ed_lanczos returns.  Takes its
 * work vectors from the library's memory pool (five fp64 vectors of the
 * summed dimension, two fp32 ones in the fp32-matvec mode, and the kept
 * Lanczos vectors); synchronises
 * `stream` before returning.  Not to be called while `stream` is being
 * captured.  Errors: ED_ERR_INVALID_ARG, ED_ERR_SYMMETRY_MISMATCH,
 * ED_ERR_UNSUPPORTED (a basis without the hash index), ED_ERR_OOM, ED_ERR_CUDA.
 */
ed_status ed_lanczos_multi(const ed_operator *op, const ed_sector *sectors, int n_sectors, int steps,
                           int mode, ed_dtype dtype, double *e0_out, ed_lanczos_info *info,
                           void *stream);

/*
 * ed_autotune -- choose, by measurement on this GPU, how ed_matvec (and the
 * solvers) run the product for this basis, nvec and dtype: the row-per-lane or
 * the term-parallel kernel (the latter for single vectors of operators whose
 * off-diagonal entries only exchange antiparallel spins), and the pruned or
 * the exhaustive rotation search (rings: rotation step one site).  The paper
 * has no counterpart (its kernels are generated once for a CPU).  Every
 * candidate runs a warm-up and three timed products (CUDA events on
 * `stream`, best of three) on the caller's x and y (as ed_matvec: device,
 * dim x nvec, 16-byte aligned; y is overwritten); the fastest is kept in the
 * library's tuning table, keyed by (GPU name, n_sites, group order, spin
 * inversion, log2 of the dimension, nvec, dtype, index kind), and used by
 * every later product on a matching basis.  With the environment variable
 * ED_TUNE_FILE naming a file, the table is read from it on first use and
 * each choice is appended to it.  Synchronises `stream`.
 *
 *   out   host (may be NULL): kernel (0 the library's rule, 1 row-per-lane,
 *         2 term-parallel), search (-1 not applicable, 0 every rotation,
 *         1 pruned), index (1 hash, 2 bucketed), ms_default (the rule's
 *         product), ms_best (the chosen one), variants_timed
 * Errors: ED_ERR_INVALID_ARG, ED_ERR_SYMMETRY_MISMATCH, ED_ERR_CUDA.
 */
typedef struct {
    int kernel;
    int search;
    int index;
    double ms_default;
    double ms_best;
    int variants_timed;
} ed_tune_result;

ed_status ed_autotune(const ed_operator *op, const ed_basis *basis, const void *d_x, void *d_y, int nvec,
                      ed_dtype dtype, ed_tune_result *out, void *stream);

/*
 * ed_autotune_index -- choose the index (hash index, or bucketed index with
 * one 32-byte bucket per lookup) that later ed_basis_build calls make for
 * sectors like this one (same GPU, n_sites, group order, spin inversion and
 * log2 of the dimension): builds the sector with each index (arguments as
 * ed_basis_build; both bases exist at once), runs ed_autotune on each with
 * zero vectors of nvec columns of dtype from the library's memory pool, and
 * keeps the faster index (written to ED_TUNE_FILE as ed_autotune does).  out
 * receives the chosen index's result, with ms_default = the default product
 * on the hash index.  Errors: as ed_basis_build and ed_autotune, ED_ERR_OOM.
 */
ed_status ed_autotune_index(const ed_operator *op, int n_sites, int n_up, int spin_inversion, int n_elems,
                            const int32_t *perms, const double *chars, int nvec, ed_dtype dtype,
                            ed_tune_result *out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ED_H */
