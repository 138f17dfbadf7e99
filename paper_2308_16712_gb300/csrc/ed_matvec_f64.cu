// ed_matvec_f64.cu -- instantiation of the matvec kernels for double arithmetic
// (real vectors).
#include "ed_matvec_impl.cuh"

namespace edk {
cudaError_t matvec_f64(const MatvecArgs &a, bool track, cudaStream_t s)
{
    return matvec_dispatch_prec<double, false>(a, track, s);
}
}  // namespace edk
