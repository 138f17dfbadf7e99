// ed_matvec_push.cu -- the transposed ("push") form of the matvec, kept as an
// ablation of the pull form (Sec. "Matrix-vector product": the paper's
// distributed product pushes every column's contributions to the owners of
// the target rows).  Each term of H|r> adds its element to y at the index of
// its representative with an atomic add, so y needs no segmented sums, no x
// gathers and no per-row ownership, but the order of the additions (and the
// last bits of y) varies from run to run.
#include "ed_matvec_tp.cuh"

namespace edk {

cudaError_t tp_push(const TpArgs<1> &a, bool track, int idx, ed_dtype dtype, cudaStream_t s)
{
    switch (dtype) {
    case ED_F64: return tp_dispatch<double, false, 1, true>(a, track, idx, s);
    case ED_F32: return tp_dispatch<float, false, 1, true>(a, track, idx, s);
    case ED_C128: return tp_dispatch<double, true, 1, true>(a, track, idx, s);
    case ED_C64: return tp_dispatch<float, true, 1, true>(a, track, idx, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace edk
