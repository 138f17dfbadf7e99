// ed_matvec_tp_nv8.cu -- instantiation of the term-parallel matvec kernel for
// one sector and a real block of 8 interleaved vectors (fp64 and fp32).
#include "ed_matvec_tp.cuh"

namespace edk {
cudaError_t tp_single_f64_nv8(const TpArgs<1> &a, bool track, int idx, cudaStream_t s)
{
    return tp_dispatch<double, false, 1, false, 8>(a, track, idx, s);
}
cudaError_t tp_single_f32_nv8(const TpArgs<1> &a, bool track, int idx, cudaStream_t s)
{
    return tp_dispatch<float, false, 1, false, 8>(a, track, idx, s);
}
}  // namespace edk
