/*
 * ed_oracle.c -- plain, slow, obviously correct CPU reference for the
 * symmetry-adapted spin-1/2 exact-diagonalization hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * cpu_baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path, and must never be used as a fallback for it.
 *
 * What it computes (the paper leaves the representative condition to its
 * refs; the readings below are the ones this project uses throughout):
 *
 *  - Encoding (Background, Fig. 1): site i <-> bit i of a uint64, 1 = up.
 *    A group element g = (perm, flip, chi) maps state s to g.s with
 *    bit perm[i] of g.s = bit i of s, then all n bits complemented if flip.
 *  - U(1) restriction (Background, Fig. 1): only states with popcount n_up.
 *  - Representative (States enumeration): rep(s) = min over g of g.s as an
 *    unsigned integer, found here by applying every group element bit by bit.
 *  - Orbit norm: n(s) = sum over the stabilizer of conj(chi(g)); for a
 *    one-dimensional character this is |Stab(s)| when chi == 1 on the
 *    stabilizer, else 0.  Stored as that integer.
 *  - Basis: ascending list of all s with s == rep(s) and n(s) != 0; the index
 *    of a state is its position (Background: basis elements vs indices).
 *  - Matrix-vector product (Sec. "Matrix-vector product", y_i = sum_j H_ij x_j,
 *    pull form): for row r and every term of H|r> = sum_s h_s |s>, with
 *    r' = rep(s) = g*.s:  y_r += conj(h_s) chi(g*) sqrt(n(r')/n(r)) x_idx(r').
 *    Terms whose representative has norm 0 vanish and are dropped.
 *
 * Everything is fp64 / complex128; no blocking, fusion or reordering.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_CHI_TOL 1e-9

/* ------------------------------------------------------------------------ */
/* group action                                                              */
/* ------------------------------------------------------------------------ */

static uint64_t low_mask(int n) { return n >= 64 ? ~0ULL : ((1ULL << n) - 1ULL); }

/* g.s for one group element, one bit at a time. */
uint64_t orc_apply(int n, const int32_t *perm, int flip, uint64_t s)
{
    uint64_t out = 0;
    for (int i = 0; i < n; ++i)
        if ((s >> i) & 1ULL)
            out |= 1ULL << perm[i];
    if (flip)
        out ^= low_mask(n);
    return out;
}

typedef struct {
    int n;              /* sites */
    int ng;             /* group order (spin inversion already expanded) */
    const int32_t *perm; /* ng x n */
    const uint8_t *flip; /* ng */
    const double *chi;   /* ng x 2 (re, im) */
} orc_group;

static double complex chi_of(const orc_group *G, int g)
{
    return G->chi[2 * g] + I * G->chi[2 * g + 1];
}

static int chi_is_one(const orc_group *G, int g)
{
    return cabs(chi_of(G, g) - 1.0) < ORC_CHI_TOL;
}

/* Orbit norm of s: |Stab(s)| if chi == 1 on the stabilizer, else 0.
 * Also returns the complex stabilizer sum for self-checks. */
static int norm_of(const orc_group *G, uint64_t s, double complex *stab_sum)
{
    int stab = 0, all_one = 1;
    double complex acc = 0;
    for (int g = 0; g < G->ng; ++g) {
        if (orc_apply(G->n, G->perm + (size_t)g * G->n, G->flip[g], s) == s) {
            ++stab;
            acc += conj(chi_of(G, g));
            if (!chi_is_one(G, g))
                all_one = 0;
        }
    }
    if (stab_sum)
        *stab_sum = acc;
    return all_one ? stab : 0;
}

/* rep(s), the character of the first argmin g*, and n(rep(s)).
 * Returns 0 normally, -1 if two argmins carry different characters while
 * the norm is nonzero (which the theory forbids). */
static int state_info(const orc_group *G, uint64_t s, uint64_t *rep,
                      double complex *chi_star, int *norm)
{
    uint64_t best = ~0ULL;
    int gbest = -1;
    for (int g = 0; g < G->ng; ++g) {
        uint64_t t = orc_apply(G->n, G->perm + (size_t)g * G->n, G->flip[g], s);
        if (gbest < 0 || t < best) {
            best = t;
            gbest = g;
        }
    }
    *rep = best;
    *chi_star = chi_of(G, gbest);
    *norm = norm_of(G, best, NULL);
    if (*norm != 0) {
        for (int g = 0; g < G->ng; ++g) {
            uint64_t t = orc_apply(G->n, G->perm + (size_t)g * G->n, G->flip[g], s);
            if (t == best && cabs(chi_of(G, g) - *chi_star) > 1e-9)
                return -1;
        }
    }
    return 0;
}

/* Exported single-state query: rep, chi(g*) (re,im), norm, and the complex
 * stabilizer sum of rep.  Return value as state_info. */
int orc_state_info(int n, int ng, const int32_t *perm, const uint8_t *flip,
                   const double *chi, uint64_t s, uint64_t *rep, double *chi_star,
                   int *norm, double *stab_sum)
{
    orc_group G = {n, ng, perm, flip, chi};
    double complex cs, ss;
    int rc = state_info(&G, s, rep, &cs, norm);
    norm_of(&G, *rep, &ss);
    chi_star[0] = creal(cs);
    chi_star[1] = cimag(cs);
    stab_sum[0] = creal(ss);
    stab_sum[1] = cimag(ss);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* basis enumeration (States enumeration)                                    */
/* ------------------------------------------------------------------------ */

/* Next combination in colexicographic order of the set bit positions
 * c[0] < c[1] < ... < c[k-1] (which is ascending order of the integer).
 * Returns 0 when there is none. */
static int next_combination(int *c, int k, int n)
{
    int j = 0;
    while (j < k) {
        int limit = (j + 1 < k) ? c[j + 1] : n;
        if (c[j] + 1 < limit)
            break;
        ++j;
    }
    if (j == k)
        return 0;
    c[j] += 1;
    for (int i = 0; i < j; ++i)
        c[i] = i;
    return 1;
}

static uint64_t combination_state(const int *c, int k)
{
    uint64_t s = 0;
    for (int i = 0; i < k; ++i)
        s |= 1ULL << c[i];
    return s;
}

static int keep_state(const orc_group *G, uint64_t s, uint16_t *norm)
{
    for (int g = 0; g < G->ng; ++g)
        if (orc_apply(G->n, G->perm + (size_t)g * G->n, G->flip[g], s) < s)
            return 0;
    int nm = norm_of(G, s, NULL);
    *norm = (uint16_t)nm;
    return nm != 0;
}

/* All representatives with nonzero norm, ascending.  n_up < 0: no U(1)
 * restriction (all 2^n states; n <= 30).  Writes at most cap entries and
 * returns the total count (or -1 on bad arguments). */
int64_t orc_enumerate(int n, int n_up, int ng, const int32_t *perm, const uint8_t *flip,
                      const double *chi, uint64_t *states, uint16_t *norms, int64_t cap)
{
    orc_group G = {n, ng, perm, flip, chi};
    int64_t count = 0;
    uint16_t nm;
    if (n_up < 0) {
        if (n > 30)
            return -1;
        for (uint64_t s = 0; s < (1ULL << n); ++s) {
            if (keep_state(&G, s, &nm)) {
                if (count < cap) {
                    states[count] = s;
                    norms[count] = nm;
                }
                ++count;
            }
        }
        return count;
    }
    if (n_up > n)
        return -1;
    int c[64];
    for (int i = 0; i < n_up; ++i)
        c[i] = i;
    do {
        uint64_t s = combination_state(c, n_up);
        if (keep_state(&G, s, &nm)) {
            if (count < cap) {
                states[count] = s;
                norms[count] = nm;
            }
            ++count;
        }
    } while (n_up > 0 && next_combination(c, n_up, n));
    return count;
}

/* The first `count` states of popcount n_up in ascending order, starting at
 * the given combination (used for bounded timing samples). */
int64_t orc_enumerate_slice(int n, int n_up, int ng, const int32_t *perm,
                            const uint8_t *flip, const double *chi, uint64_t first_state,
                            int64_t count, int64_t *n_kept)
{
    orc_group G = {n, ng, perm, flip, chi};
    int c[64], k = 0;
    for (int i = 0; i < n; ++i)
        if ((first_state >> i) & 1ULL)
            c[k++] = i;
    if (k != n_up)
        return -1;
    int64_t done = 0, kept = 0;
    uint16_t nm;
    do {
        uint64_t s = combination_state(c, n_up);
        kept += keep_state(&G, s, &nm);
        ++done;
    } while (done < count && next_combination(c, n_up, n));
    *n_kept = kept;
    return done;
}

/* ------------------------------------------------------------------------ */
/* the Hamiltonian: H = sum_t coeff_t * h_t(i_t, j_t)                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_terms;
    const double *coeff; /* n_terms x 2 */
    const int32_t *sites; /* n_terms x 2 */
    const double *local;  /* n_terms x 16 x 2, h[row][col], index 2*s_i + s_j */
} orc_operator;

/* Every (amplitude, state) of H|r>, diagonal entries included; returns the
 * number written (at most cap). */
static int column_of(const orc_operator *H, uint64_t r, double complex *amp, uint64_t *st,
                     int cap)
{
    int m = 0;
    for (int t = 0; t < H->n_terms; ++t) {
        int i = H->sites[2 * t], j = H->sites[2 * t + 1];
        int si = (int)((r >> i) & 1ULL), sj = (int)((r >> j) & 1ULL);
        int col = 2 * si + sj;
        double complex c = H->coeff[2 * t] + I * H->coeff[2 * t + 1];
        for (int row = 0; row < 4; ++row) {
            const double *e = H->local + ((size_t)t * 16 + row * 4 + col) * 2;
            double complex h = e[0] + I * e[1];
            if (h == 0)
                continue;
            uint64_t s = r & ~((1ULL << i) | (1ULL << j));
            s |= (uint64_t)(row >> 1) << i;
            s |= (uint64_t)(row & 1) << j;
            if (m < cap) {
                amp[m] = c * h;
                st[m] = s;
            }
            ++m;
        }
    }
    return m;
}

static int64_t find_index(const uint64_t *basis, int64_t dim, uint64_t s)
{
    int64_t lo = 0, hi = dim;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (basis[mid] < s)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < dim && basis[lo] == s) ? lo : -1;
}

/* The nonzero matrix elements of row `row` as (column index, value) pairs,
 * duplicates not merged.  Returns the count, or -1 if a representative with
 * nonzero norm is missing from the basis, -2 on a character inconsistency. */
static int row_elements(const orc_group *G, const orc_operator *H, const uint64_t *basis,
                        const uint16_t *norms, int64_t dim, int64_t row, int64_t *cols,
                        double complex *vals, int cap)
{
    enum { MAXC = 4096 };
    double complex amp[MAXC];
    uint64_t st[MAXC];
    uint64_t r = basis[row];
    double nr = (double)norms[row];
    int m = column_of(H, r, amp, st, MAXC);
    if (m > MAXC)
        return -3;
    int out = 0;
    for (int q = 0; q < m; ++q) {
        uint64_t rp;
        double complex chi;
        int nrp;
        if (state_info(G, st[q], &rp, &chi, &nrp) != 0)
            return -2;
        if (nrp == 0)
            continue;
        int64_t j = find_index(basis, dim, rp);
        if (j < 0)
            return -1;
        if (out < cap) {
            cols[out] = j;
            vals[out] = conj(amp[q]) * chi * sqrt((double)nrp / nr);
        }
        ++out;
    }
    return out;
}

/* y = H x over the whole basis; x, y complex128 interleaved [dim][nvec]. */
int orc_matvec(int n, int ng, const int32_t *perm, const uint8_t *flip, const double *chi,
               int n_terms, const double *coeff, const int32_t *sites, const double *local,
               const uint64_t *basis, const uint16_t *norms, int64_t dim, int nvec,
               const double *x, double *y)
{
    orc_group G = {n, ng, perm, flip, chi};
    orc_operator H = {n_terms, coeff, sites, local};
    enum { CAP = 4096 };
    int64_t cols[CAP];
    double complex vals[CAP];
    for (int64_t r = 0; r < dim; ++r) {
        int m = row_elements(&G, &H, basis, norms, dim, r, cols, vals, CAP);
        if (m < 0)
            return m;
        for (int v = 0; v < nvec; ++v) {
            double complex acc = 0;
            for (int q = 0; q < m; ++q) {
                const double *xe = x + 2 * (cols[q] * nvec + v);
                acc += vals[q] * (xe[0] + I * xe[1]);
            }
            y[2 * (r * nvec + v)] = creal(acc);
            y[2 * (r * nvec + v) + 1] = cimag(acc);
        }
    }
    return 0;
}

/* The sector matrix in COO form (duplicates not merged).  Returns the number
 * of entries (writes at most cap) or a negative error. */
int64_t orc_coo(int n, int ng, const int32_t *perm, const uint8_t *flip, const double *chi,
                int n_terms, const double *coeff, const int32_t *sites, const double *local,
                const uint64_t *basis, const uint16_t *norms, int64_t dim, int64_t *rows,
                int64_t *cols, double *vals, int64_t cap)
{
    orc_group G = {n, ng, perm, flip, chi};
    orc_operator H = {n_terms, coeff, sites, local};
    enum { CAP = 4096 };
    int64_t c[CAP];
    double complex v[CAP];
    int64_t total = 0;
    for (int64_t r = 0; r < dim; ++r) {
        int m = row_elements(&G, &H, basis, norms, dim, r, c, v, CAP);
        if (m < 0)
            return m;
        for (int q = 0; q < m; ++q) {
            if (total < cap) {
                rows[total] = r;
                cols[total] = c[q];
                vals[2 * total] = creal(v[q]);
                vals[2 * total + 1] = cimag(v[q]);
            }
            ++total;
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* rows evaluated from states alone (sizes where the basis cannot be built)  */
/* ------------------------------------------------------------------------ */

/* The paper's 64-bit mixer (Sec. "Hashed distribution"), used as the
 * counter-based generator of the input vector x keyed by the state. */
static uint64_t mix64(uint64_t x)
{
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

static double unif_pm1(uint64_t seed, uint64_t counter)
{
    uint64_t h = mix64(seed + counter * 0x9E3779B97F4A7C15ULL);
    return 2.0 * ((double)(h >> 11) * 0x1.0p-53) - 1.0;
}

static double complex x_of_state(uint64_t seed, uint64_t s, int nvec, int v, int cplx)
{
    uint64_t c = s * (uint64_t)nvec + (uint64_t)v;
    if (cplx)
        return unif_pm1(seed, 2 * c) + I * unif_pm1(seed, 2 * c + 1);
    return unif_pm1(seed, c);
}

/* For each given row state r (which must be a representative with nonzero
 * norm), y(r) = sum over H|r> of conj(h) chi(g*) sqrt(n(r')/n(r)) x(r'),
 * where x(r') is the state-keyed random vector.  Also returns the number of
 * stored elements of each row: off-diagonal terms whose representative has
 * nonzero norm, plus one for the diagonal.  Returns 0, or -2 / -4 (row not a
 * representative). */
int orc_rows_statex(int n, int ng, const int32_t *perm, const uint8_t *flip,
                    const double *chi, int n_terms, const double *coeff,
                    const int32_t *sites, const double *local, const uint64_t *row_states,
                    int64_t n_rows, uint64_t seed, int nvec, int cplx, double *y,
                    int32_t *nnz)
{
    orc_group G = {n, ng, perm, flip, chi};
    orc_operator H = {n_terms, coeff, sites, local};
    enum { MAXC = 4096 };
    double complex amp[MAXC];
    uint64_t st[MAXC];
    for (int64_t q = 0; q < n_rows; ++q) {
        uint64_t r = row_states[q];
        uint64_t rr;
        double complex cr;
        int nr;
        if (state_info(&G, r, &rr, &cr, &nr) != 0)
            return -2;
        if (rr != r || nr == 0)
            return -4;
        int m = column_of(&H, r, amp, st, MAXC);
        int offdiag = 0;
        for (int v = 0; v < nvec; ++v) {
            y[2 * (q * nvec + v)] = 0.0;
            y[2 * (q * nvec + v) + 1] = 0.0;
        }
        for (int e = 0; e < m; ++e) {
            uint64_t rp;
            double complex chi_s;
            int nrp;
            if (state_info(&G, st[e], &rp, &chi_s, &nrp) != 0)
                return -2;
            if (nrp == 0)
                continue;
            if (st[e] != r)
                ++offdiag;
            double complex coef = conj(amp[e]) * chi_s * sqrt((double)nrp / (double)nr);
            for (int v = 0; v < nvec; ++v) {
                double complex add = coef * x_of_state(seed, rp, nvec, v, cplx);
                y[2 * (q * nvec + v)] += creal(add);
                y[2 * (q * nvec + v) + 1] += cimag(add);
            }
        }
        nnz[q] = offdiag + 1; /* off-diagonal elements plus the one diagonal */
    }
    return 0;
}
