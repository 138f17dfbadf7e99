// ed_matvec_multi.cu -- the batched multi-sector matvec: argument checks,
// sector table and dtype dispatch.
#include <algorithm>
#include <mutex>
#include <vector>

#include "ed_matvec_tp.cuh"

namespace edk {

// Per-device control words of the batched launches: a ring of work-queue
// counters (a call takes the next one and zeroes it on its stream, so calls
// in flight on different streams use different counters unless more than
// kQueueRing overlap), the status word and the gate word of the stall test.
namespace {
constexpr int kQueueRing = 64;
constexpr int kCtlDevices = 64;
struct CtlWords {
    unsigned long long *queues = nullptr;  // kQueueRing counters
    unsigned int *status = nullptr;
    int *gate = nullptr;                   // stays 0: nothing opens it
    unsigned next = 0;
};
std::mutex g_ctl_mutex;
CtlWords g_ctl[kCtlDevices];
bool g_inject_stall = false;
// 0 and 1: one batched launch (measured faster than per-sector launches on
// all 140 XXZ N=28 sectors, also for single vectors in single precision:
// 51.7 against 54.4 ms); 2: one launch per sector where the term-parallel
// kernel applies (test hook)
int g_multi_policy = 0;
}  // namespace

cudaError_t batch_ctl(cudaStream_t s, BatchCtl *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kCtlDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_ctl_mutex);
    CtlWords &c = g_ctl[dev];
    if (!c.queues) {
        void *p = nullptr;
        const size_t bytes = kQueueRing * sizeof(unsigned long long) + 2 * sizeof(int);
        if ((e = cudaMalloc(&p, bytes)) != cudaSuccess)
            return e;
        if ((e = cudaMemset(p, 0, bytes)) != cudaSuccess)
            return e;
        c.queues = static_cast<unsigned long long *>(p);
        c.status = reinterpret_cast<unsigned int *>(c.queues + kQueueRing);
        c.gate = reinterpret_cast<int *>(c.status + 1);
    }
    unsigned long long *q = c.queues + (c.next++ % kQueueRing);
    if ((e = cudaMemsetAsync(q, 0, sizeof(*q), s)) != cudaSuccess)
        return e;
    *out = BatchCtl{q, c.status, g_inject_stall ? c.gate : nullptr};
    return cudaSuccess;
}

cudaError_t batch_status_take(unsigned int *st)
{
    *st = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kCtlDevices)
        return e;
    std::lock_guard<std::mutex> lock(g_ctl_mutex);
    CtlWords &c = g_ctl[dev];
    if (!c.status)
        return cudaSuccess;
    if ((e = cudaMemcpy(st, c.status, sizeof(unsigned int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    return *st ? cudaMemset(c.status, 0, sizeof(unsigned int)) : cudaSuccess;
}

void set_inject_stall(bool on) { g_inject_stall = on; }

cudaError_t multi_f64(const MultiArgs &a, bool track, cudaStream_t s) { return multi_dispatch_prec<double, false>(a, track, s); }
cudaError_t multi_f32(const MultiArgs &a, bool track, cudaStream_t s) { return multi_dispatch_prec<float, false>(a, track, s); }
cudaError_t multi_c128(const MultiArgs &a, bool track, cudaStream_t s) { return multi_dispatch_prec<double, true>(a, track, s); }
cudaError_t multi_c64(const MultiArgs &a, bool track, cudaStream_t s) { return multi_dispatch_prec<float, true>(a, track, s); }

// The batched product: the term-parallel kernel where use_term_parallel
// chooses it (its warps take tiles of one sector each), else the row-per-lane
// multi-sector kernel.
cudaError_t multi_launch_any(const MultiArgs &a, bool track, ed_dtype dtype, cudaStream_t s)
{
    bool same_kind = true;
    for (int k = 1; k < a.n_sectors; ++k)
        same_kind = same_kind && tp_index_kind(a.sec[k]) == tp_index_kind(a.sec[0]);
    if (same_kind && use_term_parallel(a.nvec, a.op, dtype, a.g.n_sites)) {
        const int kind = a.n_sectors > 0 ? tp_index_kind(a.sec[0]) : 0;
        static thread_local TpArgs<kMaxSectors> t;  // host staging (17 KB); copied at launch
        t.op = a.op;
        t.g = a.g;
        t.n_sectors = a.n_sectors;
        t.max_order = a.max_order;
        t.total_tiles = a.total_tiles;
        t.ctl = a.ctl;
        for (int k = 0; k < a.n_sectors; ++k)
            t.sec[k] = a.sec[k];
        switch (dtype) {
        case ED_F64: return tp_multi_f64(t, track, kind, s);
        case ED_F32: return tp_multi_f32(t, track, kind, s);
        case ED_C128: return tp_multi_c128(t, track, kind, s);
        case ED_C64: return tp_multi_c64(t, track, kind, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (dtype) {
    case ED_F64: return multi_f64(a, track, s);
    case ED_F32: return multi_f32(a, track, s);
    case ED_C128: return multi_c128(a, track, s);
    case ED_C64: return multi_c64(a, track, s);
    }
    return cudaErrorInvalidValue;
}
}  // namespace edk

// Test hook: 1 = every later batched launch first waits on a gate word that
// nothing opens (an injected stall of the producer); its bounded wait runs
// out and ed_stream_status reports ED_ERR_TIMEOUT.
extern "C" void edx_inject_stall(int on) { edk::set_inject_stall(on != 0); }

namespace edk {
void set_multi_policy(int p) { g_multi_policy = p; }
int multi_policy_get() { return g_multi_policy; }
}  // namespace edk

// Test hook: 0 = the library's rule (one batched launch), 1 = the same,
// 2 = one launch per sector where the term-parallel kernel applies and every
// sector alone fills the GPU.
extern "C" void edx_multi_policy(int policy) { edk::set_multi_policy(policy); }

extern "C" ed_status ed_matvec_multi(const ed_operator *op, const ed_sector *sectors, int n_sectors, int nvec,
                                     ed_dtype dtype, void *stream)
{
    using namespace edk;
    if (!op || !sectors || n_sectors < 1 || n_sectors > kMaxSectors || nvec < 1 || nvec > 16)
        return ED_ERR_INVALID_ARG;
    if (dtype != ED_F64 && dtype != ED_F32 && dtype != ED_C128 && dtype != ED_C64)
        return ED_ERR_INVALID_ARG;
    const bool cplx = dtype == ED_C128 || dtype == ED_C64;
    const ed_basis *b0 = sectors[0].basis;
    if (!b0)
        return ED_ERR_INVALID_ARG;
    static MultiArgs args;  // 17 KB: built on the host, passed by value to the kernel
    static std::mutex args_mutex;
    std::lock_guard<std::mutex> lock(args_mutex);
    args.op = make_op_view(op);
    args.g = b0->group_view();
    args.nvec = nvec;
    args.max_order = 0;
    bool track = false;
    int m = 0;
    uint64_t tiles = 0;
    // the tile list (and the work queue) runs through the sectors largest first
    std::vector<int> order(n_sectors);
    for (int s = 0; s < n_sectors; ++s)
        order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int u, int v) {
        const uint64_t du = sectors[u].basis ? sectors[u].basis->dim : 0;
        const uint64_t dv = sectors[v].basis ? sectors[v].basis->dim : 0;
        return du > dv;
    });
    for (int oi = 0; oi < n_sectors; ++oi) {
        const int s = order[oi];
        const ed_basis *b = sectors[s].basis;
        if (!b || b->n_sites != b0->n_sites || b->n_perm != b0->n_perm || b->perms != b0->perms)
            return ED_ERR_INVALID_ARG;  // every sector must use the same lattice permutations
        const ed_status st = check_pair(op, b);
        if (st != ED_OK)
            return st;
        if (!cplx && !(b->real_chars && op->real))
            return ED_ERR_INVALID_ARG;
        if (!b->dim)
            continue;
        const void *x = sectors[s].d_x;
        void *y = sectors[s].d_y;
        if (!x || !y || x == y || (((uintptr_t)x | (uintptr_t)y) & 15))
            return ED_ERR_INVALID_ARG;
        if (!b->d_htab && !b->d_bkt)
            return ED_ERR_UNSUPPORTED;
        const GroupView gv = b->group_view();
        const IndexView iv = b->index_view();
        SectorDesc &d = args.sec[m++];
        d.keys = iv.keys;
        d.states = iv.states;
        d.norms = iv.norms;
        sector_index_from(d, b);
        d.chi = gv.fact ? gv.fchi : gv.chi;
        d.chif = gv.fact ? gv.fchif : gv.chif;
        d.x = x;
        d.y = y;
        d.dim = b->dim;
        d.tile_begin = tiles;
        d.flip = b->spin_inversion != 0;
        tiles += (b->dim + 31) / 32;
        track = track || !b->trivial_chars;
        args.max_order = std::max(args.max_order, b->order);
    }
    args.n_sectors = m;
    args.total_tiles = tiles;
    if (!m)
        return ED_OK;
    // the shared search uses the larger flip-expanded order only for the
    // characters, which are per sector; the group view's own flip is unused
    args.g.flip = 0;
    // One vector in single precision, every sector large enough to fill the
    // GPU alone (one row per resident thread): a term-parallel launch per
    // sector, measured faster than one batched launch for such sectors (all
    // 140 XXZ N=28 sectors: 58 against 142 ms).  The same kernel and
    // arguments as ed_matvec, so the results are the same bits.
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    bool all_large = true;
    for (int s = 0; s < n_sectors; ++s)
        all_large = all_large && (!sectors[s].basis->dim || sectors[s].basis->dim >= (uint64_t)sms * 2048);
    cudaError_t e = cudaSuccess;
    const bool per_sector = g_multi_policy == 2 && all_large;
    if (per_sector && use_term_parallel(nvec, args.op, dtype, args.g.n_sites)) {
        for (int s = 0; s < n_sectors && e == cudaSuccess; ++s) {
            const ed_basis *b = sectors[s].basis;
            if (b->dim)
                e = launch_matvec(args.op, b->group_view(), b->index_view(), !b->trivial_chars, sectors[s].d_x,
                                  sectors[s].d_y, nvec, dtype, (cudaStream_t)stream);
        }
    } else {
        e = batch_ctl((cudaStream_t)stream, &args.ctl);
        if (e == cudaSuccess)
            e = multi_launch_any(args, track, dtype, (cudaStream_t)stream);
    }
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return ED_ERR_CUDA;
    }
    return ED_OK;
}
