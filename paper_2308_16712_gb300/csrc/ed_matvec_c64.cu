// ed_matvec_c64.cu -- instantiation of the matvec kernels for float arithmetic
// (complex vectors).
#include "ed_matvec_impl.cuh"

namespace edk {
cudaError_t matvec_c64(const MatvecArgs &a, bool track, cudaStream_t s)
{
    return matvec_dispatch_prec<float, true>(a, track, s);
}
}  // namespace edk
