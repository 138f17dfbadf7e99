// ed_tune.cu -- the autotuner of the product: which kernel (row-per-lane or
// term-parallel), which group search (pruned to the longest runs, or every
// rotation) and which index (hash or bucketed) run fastest for a kind of
// sector on this GPU.  Choices are measured (CUDA events, best of three after
// a warm-up) and kept in a table keyed by (GPU name, n_sites, group order,
// spin inversion, log2 of the dimension, nvec, dtype, index kind); with the
// environment variable ED_TUNE_FILE set, the table is read from that file on
// first use and every new choice is appended to it, so later processes reuse
// it.  ed_matvec and the solvers take the tuned variant when one exists.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ed_kernels.cuh"

namespace edk {
namespace {

using ProdKey = std::tuple<std::string, int, int, int, int, int, int, int>;  // gpu n order flip log2dim nvec dtype idx
using IdxKey = std::tuple<std::string, int, int, int, int>;                 // gpu n order flip log2dim

std::mutex g_tune_mutex;
bool g_loaded = false;
std::map<ProdKey, MatvecVariant> g_prod;
std::map<IdxKey, int> g_index;

// device name of the current device, cached per device (called with the
// table's mutex held)
std::string gpu_name()
{
    static std::map<int, std::string> names;
    int dev = 0;
    cudaGetDevice(&dev);
    auto it = names.find(dev);
    if (it != names.end())
        return it->second;
    cudaDeviceProp p;
    std::string s = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? std::string(p.name) : "unknown";
    for (char &c : s)
        if (c == ' ' || c == '|')
            c = '_';
    names[dev] = s;
    return s;
}

int log2_dim(uint64_t dim)
{
    int l = 0;
    while (l < 63 && (2ULL << l) <= dim)
        ++l;
    return l;
}

// ED_TUNE_FILE lines: "P gpu n order flip log2dim nvec dtype idx kernel prune"
//                     "I gpu n order flip log2dim kind"
void load_locked()
{
    if (g_loaded)
        return;
    g_loaded = true;
    const char *path = std::getenv("ED_TUNE_FILE");
    if (!path || !*path)
        return;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return;
    char kind = 0;
    char gpu[256];
    while (std::fscanf(f, " %c %255s", &kind, gpu) == 2) {
        if (kind == 'P') {
            int n, order, flip, l2, nvec, dt, idx, kern, prune;
            if (std::fscanf(f, "%d %d %d %d %d %d %d %d %d", &n, &order, &flip, &l2, &nvec, &dt, &idx, &kern,
                            &prune) != 9)
                break;
            g_prod[ProdKey{gpu, n, order, flip, l2, nvec, dt, idx}] = MatvecVariant{kern, prune};
        } else if (kind == 'I') {
            int n, order, flip, l2, k;
            if (std::fscanf(f, "%d %d %d %d %d", &n, &order, &flip, &l2, &k) != 5)
                break;
            g_index[IdxKey{gpu, n, order, flip, l2}] = k;
        } else {
            break;
        }
    }
    std::fclose(f);
}

void append_line(const std::string &line)
{
    const char *path = std::getenv("ED_TUNE_FILE");
    if (!path || !*path)
        return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fputs(line.c_str(), f);
        std::fclose(f);
    }
}

int index_kind_of(const ed_basis *b) { return b->d_bkt ? 2 : 1; }

ProdKey prod_key(const ed_basis *b, int nvec, ed_dtype dtype)
{
    return ProdKey{gpu_name(), b->n_sites, b->order, b->spin_inversion != 0 ? 1 : 0, log2_dim(b->dim), nvec,
                   (int)dtype, index_kind_of(b)};
}

// best of three product launches after a warm-up, CUDA events on the stream
cudaError_t time_variant(const ed_operator *op, const ed_basis *b, const void *x, void *y, int nvec,
                         ed_dtype dtype, MatvecVariant v, cudaStream_t st, double *ms)
{
    const OpView ov = make_op_view(op);
    const GroupView gv = b->group_view();
    const IndexView iv = b->index_view();
    const bool track = !b->trivial_chars;
    cudaError_t e = launch_matvec_v(ov, gv, iv, track, x, y, nvec, dtype, v, st);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best = 1e300;
    for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        e = launch_matvec_v(ov, gv, iv, track, x, y, nvec, dtype, v, st);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess)
            e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess)
            best = std::min(best, (double)t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace

MatvecVariant tuned_variant(const ed_basis *b, int nvec, ed_dtype dtype)
{
    if (g_kernel_policy != 0)  // a test hook forces a kernel: no tuned choice
        return MatvecVariant{};
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_locked();
    if (g_prod.empty())
        return MatvecVariant{};
    auto it = g_prod.find(prod_key(b, nvec, dtype));
    return it == g_prod.end() ? MatvecVariant{} : it->second;
}

int tuned_index_kind(int n_sites, int order, int flip, uint64_t dim)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    load_locked();
    if (g_index.empty())
        return 0;
    auto it = g_index.find(IdxKey{gpu_name(), n_sites, order, flip ? 1 : 0, log2_dim(dim)});
    return it == g_index.end() ? 0 : it->second;
}

// candidate variants of the product for this basis (the default first)
static std::vector<MatvecVariant> product_variants(const ed_operator *op, const ed_basis *b, int nvec,
                                                   ed_dtype dtype)
{
    const OpView ov = make_op_view(op);
    const GroupView gv = b->group_view();
    const bool tp_ok = (b->d_htab || b->d_bkt) && (nvec == 1 || (nvec == 8 && (dtype == ED_F64 || dtype == ED_F32))) &&
                       ov.exchange_only;
    const bool prune_ok = gv.fact && gv.rot_d == 1;
    std::vector<MatvecVariant> v{MatvecVariant{0, -1}};
    for (int k : {1, 2}) {
        if (k == 2 && !tp_ok)
            continue;
        for (int p : {0, 1}) {
            if (!prune_ok && p == 1)
                continue;
            v.push_back(MatvecVariant{k, prune_ok ? p : -1});
        }
    }
    return v;
}

}  // namespace edk

extern "C" ed_status ed_autotune(const ed_operator *op, const ed_basis *b, const void *d_x, void *d_y, int nvec,
                                 ed_dtype dtype, ed_tune_result *out, void *stream)
{
    using namespace edk;
    if (!op || !b || !d_x || !d_y || d_x == d_y || nvec < 1 || nvec > 16 ||
        (((uintptr_t)d_x | (uintptr_t)d_y) & 15))
        return ED_ERR_INVALID_ARG;
    if (dtype != ED_F64 && dtype != ED_F32 && dtype != ED_C128 && dtype != ED_C64)
        return ED_ERR_INVALID_ARG;
    const ed_status st0 = check_pair(op, b);
    if (st0 != ED_OK)
        return st0;
    if ((dtype == ED_F64 || dtype == ED_F32) && !(b->real_chars && op->real))
        return ED_ERR_INVALID_ARG;
    if (!b->dim)
        return ED_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const std::vector<MatvecVariant> cand = product_variants(op, b, nvec, dtype);
    double ms_default = 0.0, ms_best = 1e300;
    MatvecVariant best{};
    for (size_t i = 0; i < cand.size(); ++i) {
        double ms = 0.0;
        const cudaError_t e = time_variant(op, b, d_x, d_y, nvec, dtype, cand[i], st, &ms);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return ED_ERR_CUDA;
        }
        if (i == 0)
            ms_default = ms;
        if (ms < ms_best) {
            ms_best = ms;
            best = cand[i];
        }
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        load_locked();
        const ProdKey k = prod_key(b, nvec, dtype);
        g_prod[k] = best;
        char line[512];
        std::snprintf(line, sizeof line, "P %s %d %d %d %d %d %d %d %d %d\n", std::get<0>(k).c_str(),
                      std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), std::get<5>(k),
                      std::get<6>(k), std::get<7>(k), best.kernel, best.prune);
        append_line(line);
    }
    if (out) {
        out->kernel = best.kernel;
        out->search = best.prune;
        out->index = b->d_bkt ? 2 : 1;
        out->ms_default = ms_default;
        out->ms_best = ms_best;
        out->variants_timed = (int)cand.size();
    }
    return ED_OK;
}

extern "C" ed_status ed_autotune_index(const ed_operator *op, int n_sites, int n_up, int spin_inversion,
                                       int n_elems, const int32_t *perms, const double *chars, int nvec,
                                       ed_dtype dtype, ed_tune_result *out, void *stream)
{
    using namespace edk;
    if (!op || nvec < 1 || nvec > 16)
        return ED_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ed_tune_result r[2] = {};
    ed_basis *bases[2] = {nullptr, nullptr};
    ed_status s = ED_OK;
    const int saved = index_policy_get();
    uint64_t dim = 0;
    int order = 0;
    for (int k = 0; k < 2 && s == ED_OK; ++k) {
        index_policy_set(k == 0 ? 1 : 2);  // hash, then bucketed
        s = ed_basis_build(n_sites, n_up, spin_inversion, n_elems, perms, chars, stream, &bases[k]);
        index_policy_set(saved);
        if (s != ED_OK)
            break;
        dim = bases[k]->dim;
        order = bases[k]->order;
        if (k == 1 && !bases[1]->d_bkt)
            break;  // the bucketed index does not apply (entry too narrow): hash stays
        const size_t vb = (dtype == ED_F64 || dtype == ED_C64) ? 8 : dtype == ED_F32 ? 4 : 16;
        void *x = nullptr, *y = nullptr;
        if (ws_alloc(&x, dim * nvec * vb, st) != cudaSuccess || ws_alloc(&y, dim * nvec * vb, st) != cudaSuccess) {
            ws_free(x, st);
            (void)cudaGetLastError();
            s = ED_ERR_OOM;
            break;
        }
        cudaMemsetAsync(x, 0, dim * nvec * vb, st);
        s = ed_autotune(op, bases[k], x, y, nvec, dtype, &r[k], stream);
        ws_free(x, st);
        ws_free(y, st);
    }
    const bool both = s == ED_OK && bases[1] && bases[1]->d_bkt && r[1].ms_best > 0.0;
    const int kind = both && r[1].ms_best < r[0].ms_best ? 2 : 1;
    for (ed_basis *b : bases)
        if (b)
            ed_basis_destroy(b);
    if (s != ED_OK)
        return s;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        load_locked();
        const IdxKey k{gpu_name(), n_sites, order, spin_inversion != 0 ? 1 : 0, log2_dim(dim)};
        g_index[k] = kind;
        char line[512];
        std::snprintf(line, sizeof line, "I %s %d %d %d %d %d\n", std::get<0>(k).c_str(), std::get<1>(k),
                      std::get<2>(k), std::get<3>(k), std::get<4>(k), kind);
        append_line(line);
    }
    if (out) {
        *out = kind == 2 ? r[1] : r[0];
        out->index = kind;
        out->ms_default = r[0].ms_default;
    }
    return ED_OK;
}

// Test hook: forget every tuned choice (the file, if any, is not touched).
extern "C" void edx_tune_reset(void)
{
    std::lock_guard<std::mutex> lock(edk::g_tune_mutex);
    edk::g_prod.clear();
    edk::g_index.clear();
    edk::g_loaded = true;
}
