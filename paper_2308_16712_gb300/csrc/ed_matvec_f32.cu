// ed_matvec_f32.cu -- instantiation of the matvec kernels for float arithmetic
// (real vectors).
#include "ed_matvec_impl.cuh"

namespace edk {
cudaError_t matvec_f32(const MatvecArgs &a, bool track, cudaStream_t s)
{
    return matvec_dispatch_prec<float, false>(a, track, s);
}
}  // namespace edk
