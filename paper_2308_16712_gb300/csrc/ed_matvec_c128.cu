// ed_matvec_c128.cu -- instantiation of the matvec kernels for double arithmetic
// (complex vectors).
#include "ed_matvec_impl.cuh"

namespace edk {
cudaError_t matvec_c128(const MatvecArgs &a, bool track, cudaStream_t s)
{
    return matvec_dispatch_prec<double, true>(a, track, s);
}
}  // namespace edk
