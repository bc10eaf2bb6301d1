// Pair kernels for the M4 kernel serving the wrap list: periodic leaves whose
// pair vectors may miss the minimum image.
#include "sph_pairs.cuh"

namespace sph {

cudaError_t density_launches_m4_wrap(const BatchView &b, int precision, int use_pred, cudaStream_t st)
{
    if (!(b.dens_mask & 0x00ff)) return cudaSuccess;
    return density_classes<SPH_KERNEL_M4, true>(b, precision, use_pred, st);
}

cudaError_t force_launches_m4_wrap(const BatchView &b, int precision, cudaStream_t st)
{
    if (!(b.lpp_mask & 0x0f)) return cudaSuccess;
    return force_classes<SPH_KERNEL_M4, true>(b, precision, st);
}

}  // namespace sph
