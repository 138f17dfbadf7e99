// ed_matvec_tp_c64.cu -- instantiation of the term-parallel matvec kernels
// for complex float arithmetic, one sector and batches of sectors.
#include "ed_matvec_tp.cuh"

namespace edk {
cudaError_t tp_single_c64(const TpArgs<1> &a, bool track, int idx, cudaStream_t s)
{
    return tp_dispatch<float, true, 1>(a, track, idx, s);
}
cudaError_t tp_multi_c64(const TpArgs<kMaxSectors> &a, bool track, int idx, cudaStream_t s)
{
    return tp_dispatch<float, true, kMaxSectors>(a, track, idx, s);
}
}  // namespace edk
