// ed_noalloc.cu -- counting the representatives of a sector without any
// device allocation.
//
// ed_basis_build allocates its work arrays (per-chunk counts, scan offsets)
// and the basis itself.  Some callers cannot do that: an application that has
// handed the whole device memory to its own pool or caching allocator has none
// left for a library's cudaMalloc, and a latency-critical path cannot afford
// cudaMalloc / cudaFree, which synchronise the device.  For them this file
// offers the count pass of the basis build with all of its scratch -- the
// group tables, the binomial table, the per-chunk counts and the scan
// offsets -- carved out of one file-scope device array of fixed size.
//
// Host code cannot pass that array's name to a kernel (in host code the name
// is only a host-side stand-in), so the device address is looked up once per
// device with cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "ed_kernels.cuh"

namespace {

constexpr int kNoAllocMaxElems = 512;                // lattice elements (before spin inversion)
constexpr uint64_t kNoAllocMaxChunks = 1ULL << 18;   // enumeration chunks per call
// States one thread enumerates (a chunk).  The per-chunk count is a uint32,
// and the bound also caps a thread's work: at most 2^18 x 2^24 = 2^42 states
// per call (C(44, 22) = 2.1e12 fits; larger sectors need ed_basis_count).
constexpr uint64_t kNoAllocMaxChunkStates = 1ULL << 24;
constexpr int kNoAllocMaxDevices = 64;

// byte offsets of the carved regions (each 256-byte aligned)
constexpr size_t al(size_t v) { return (v + 255) & ~size_t(255); }
constexpr size_t kOffMasks32 = 0;
constexpr size_t kOffMasks64 = al(kOffMasks32 + (size_t)kNoAllocMaxElems * edk::kMaskStride * 4);
constexpr size_t kOffChiOne = al(kOffMasks64 + (size_t)kNoAllocMaxElems * edk::kMaskStride * 8);
constexpr size_t kOffBinom = al(kOffChiOne + (2 * kNoAllocMaxElems + 31) / 32 * 4);
constexpr size_t kOffCounts = al(kOffBinom + 65 * 65 * 8);
constexpr size_t kOffOffsets = al(kOffCounts + kNoAllocMaxChunks * 4);
constexpr size_t kOffTmp = al(kOffOffsets + (kNoAllocMaxChunks + 1) * 8);
// the scan's work region: scan_tmp_words(n) words, n / 4096 + 1 for the
// current scan tile, checked against this size before every launch
constexpr size_t kScratchBytes = al(kOffTmp + ((kNoAllocMaxChunks + 4095) / 4096 + 1) * 8);

// The scratch of every call, on every device that loads the library (about
// 3.2 MB, held until the process exits).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mutex;
unsigned char *g_scratch_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).
cudaError_t scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" ed_status ed_basis_count_noalloc(int n_sites, int n_up, int spin_inversion, int n_elems,
                                            const int32_t *perms, const double *chars,
                                            void *stream_, uint64_t *dim_out)
{
    if (!dim_out)
        return ED_ERR_INVALID_ARG;
    if (n_elems > kNoAllocMaxElems)
        return ED_ERR_INVALID_ARG;  // beyond the fixed scratch capacity
    std::vector<uint32_t> m32, one;
    std::vector<uint64_t> m64;
    const ed_status st = edk::count_tables_host(n_sites, n_up, spin_inversion, n_elems, perms,
                                                chars, m32, m64, one);
    if (st != ED_OK)
        return st;
    // the enumeration plan, and its size checks, before any CUDA call
    edk::EnumPlan plan;
    plan.n_sites = n_sites;
    plan.n_up = n_up;
    plan.total = n_up < 0 ? (1ULL << n_sites) : edk::binomial_host(n_sites, n_up);
    plan.chunk = std::max<uint64_t>(16, (plan.total + kNoAllocMaxChunks - 1) / kNoAllocMaxChunks);
    plan.n_chunks = (plan.total + plan.chunk - 1) / plan.chunk;
    if (plan.chunk > kNoAllocMaxChunkStates)
        return ED_ERR_UNSUPPORTED;  // more states than the fixed scratch and per-thread bound allow
    if (edk::scan_tmp_words(plan.n_chunks) * sizeof(uint64_t) > kScratchBytes - kOffTmp)
        return ED_ERR_INTERNAL;     // the scan's work region would not fit the scratch
    cudaStream_t stream = (cudaStream_t)stream_;
    unsigned char *base = nullptr;
#define ED_NA_TRY(expr)                       \
    do {                                      \
        cudaError_t _e = (expr);              \
        if (_e != cudaSuccess) {              \
            (void)cudaGetLastError();         \
            return ED_ERR_CUDA;               \
        }                                     \
    } while (0)
    ED_NA_TRY(scratch_address(&base));
    uint32_t *d_m32 = reinterpret_cast<uint32_t *>(base + kOffMasks32);
    uint64_t *d_m64 = reinterpret_cast<uint64_t *>(base + kOffMasks64);
    uint32_t *d_one = reinterpret_cast<uint32_t *>(base + kOffChiOne);
    uint64_t *d_binom = reinterpret_cast<uint64_t *>(base + kOffBinom);
    uint32_t *d_counts = reinterpret_cast<uint32_t *>(base + kOffCounts);
    uint64_t *d_offsets = reinterpret_cast<uint64_t *>(base + kOffOffsets);
    uint64_t *d_tmp = reinterpret_cast<uint64_t *>(base + kOffTmp);

    std::vector<uint64_t> binom(65 * 65);
    for (int a = 0; a <= 64; ++a)
        for (int k = 0; k <= 64; ++k)
            binom[a * 65 + k] = edk::binomial_host(a, k);
    // every region the kernels read is rewritten here, so nothing from an
    // earlier call survives into this one
    ED_NA_TRY(cudaMemcpyAsync(d_m32, m32.data(), m32.size() * 4, cudaMemcpyHostToDevice, stream));
    ED_NA_TRY(cudaMemcpyAsync(d_m64, m64.data(), m64.size() * 8, cudaMemcpyHostToDevice, stream));
    ED_NA_TRY(cudaMemcpyAsync(d_one, one.data(), one.size() * 4, cudaMemcpyHostToDevice, stream));
    ED_NA_TRY(cudaMemcpyAsync(d_binom, binom.data(), binom.size() * 8, cudaMemcpyHostToDevice, stream));

    edk::GroupView g{};
    g.n_sites = n_sites;
    g.n_perm = n_elems;
    g.flip = spin_inversion != 0;
    g.order = n_elems * (spin_inversion ? 2 : 1);
    g.full = n_sites >= 64 ? ~0ULL : ((1ULL << n_sites) - 1);
    g.masks32 = d_m32;
    g.masks64 = d_m64;
    g.chi_one = d_one;
    g.fact = 0;

    plan.binom = d_binom;

    ED_NA_TRY(edk::launch_enum_count(plan, g, d_counts, stream));
    ED_NA_TRY(edk::launch_scan(d_counts, plan.n_chunks, d_offsets, d_tmp, stream));
    uint64_t dim = 0;
    ED_NA_TRY(cudaMemcpyAsync(&dim, d_offsets + plan.n_chunks, sizeof(uint64_t),
                              cudaMemcpyDeviceToHost, stream));
    ED_NA_TRY(cudaStreamSynchronize(stream));
#undef ED_NA_TRY
    *dim_out = dim;
    return ED_OK;
}
