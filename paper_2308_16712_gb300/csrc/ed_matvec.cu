// ed_matvec.cu -- dtype dispatch of the matvec kernels.
#include "ed_matvec_impl.cuh"

namespace edk {

cudaError_t launch_matvec(const OpView &op, const GroupView &g, const IndexView &ix, bool track,
                          const void *x, void *y, int nvec, ed_dtype dtype, cudaStream_t stream)
{
    const MatvecArgs a{op, g, ix, x, y, nvec};
    switch (dtype) {
    case ED_F64: return matvec_f64(a, track, stream);
    case ED_F32: return matvec_f32(a, track, stream);
    case ED_C128: return matvec_c128(a, track, stream);
    case ED_C64: return matvec_c64(a, track, stream);
    }
    return cudaErrorInvalidValue;
}

}  // namespace edk
