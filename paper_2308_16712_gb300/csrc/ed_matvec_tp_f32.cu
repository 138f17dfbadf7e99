// ed_matvec_tp_f32.cu -- instantiation of the term-parallel matvec kernels
// for float arithmetic, one sector and batches of sectors.
#include "ed_matvec_tp.cuh"

namespace edk {
cudaError_t tp_single_f32(const TpArgs<1> &a, bool track, int idx, cudaStream_t s)
{
    return tp_dispatch<float, false, 1>(a, track, idx, s);
}
cudaError_t tp_multi_f32(const TpArgs<kMaxSectors> &a, bool track, int idx, cudaStream_t s)
{
    return tp_dispatch<float, false, kMaxSectors>(a, track, idx, s);
}
}  // namespace edk
