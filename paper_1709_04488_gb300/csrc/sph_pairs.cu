// Pair kernels for the M4 cubic spline, the slow density path (any kernel)
// and the launch sequence of the density and force passes.
#include "sph_pairs.cuh"

namespace sph {

cudaError_t density_launches_m4(const BatchView &b, int precision, int use_pred, cudaStream_t st)
{
    if (!(b.dens_mask & 0x00ff)) return cudaSuccess;
    return density_classes<SPH_KERNEL_M4, false>(b, precision, use_pred, st);
}

cudaError_t force_launches_m4(const BatchView &b, int precision, cudaStream_t st)
{
    if (!(b.lpp_mask & 0x0f)) return cudaSuccess;
    return force_classes<SPH_KERNEL_M4, false>(b, precision, st);
}

// Order: the common launches of every class (which put the periodic leaves
// whose pair vectors may miss the minimum image on the wrap list), the
// wrap-list launches (periodic batches), then the slow density path.
cudaError_t launch_density(const BatchView &b, int precision, int use_pred, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    const bool tasks = b.block_on && b.block_tasks;
    if (!tasks) {  // (block-step ticks with tasks: the wrap-list launch serves them)
        e = density_launches_m4(b, precision, use_pred, st);
        if (e == cudaSuccess) e = density_launches_m6(b, precision, use_pred, st);
    }
    const bool wrap = b.any_periodic || b.any_gravity || tasks;
    if (e == cudaSuccess && wrap) e = density_launches_m4_wrap(b, precision, use_pred, st);
    if (e == cudaSuccess && wrap) e = density_launches_m6_wrap(b, precision, use_pred, st);
    if (e != cudaSuccess) return e;
    if (precision == SPH_PREC_FP64) run_density_fallback<double>(b, use_pred, st);
    else run_density_fallback<float>(b, use_pred, st);
    return cudaGetLastError();
}

cudaError_t launch_block_tasks(const BatchView &b, int precision, cudaStream_t st)
{
    const unsigned grid = (unsigned)dev_info().sm_count * 4;
    if (precision == SPH_PREC_FP64) k_block_tasks<double><<<grid, 256, 0, st>>>(b, 1);
    else k_block_tasks<float><<<grid, 256, 0, st>>>(b, 1);
    return cudaGetLastError();
}

cudaError_t launch_block_leaf_tick(const BatchView &b, int precision, cudaStream_t st)
{
    const unsigned grid = (unsigned)dev_info().sm_count * 8;
    if (precision == SPH_PREC_FP64) k_block_leaf_tick<double, dbl4><<<grid, 256, 0, st>>>(b, 1);
    else k_block_leaf_tick<float, float4><<<grid, 256, 0, st>>>(b, 1);
    return cudaGetLastError();
}

cudaError_t launch_forces(const BatchView &b, int precision, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if (!(b.block_on && b.block_tasks)) {  // (block-step ticks with tasks: the wrap-list launch serves them)
        e = force_launches_m4(b, precision, st);
        if (e == cudaSuccess) e = force_launches_m6(b, precision, st);
    }
    if (e == cudaSuccess && (b.any_periodic || b.any_general)) e = force_launches_m4_wrap(b, precision, st);
    if (e == cudaSuccess && (b.any_periodic || b.any_general)) e = force_launches_m6_wrap(b, precision, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace sph
