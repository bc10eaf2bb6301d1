// ALU ceiling of the pair kernels: the throughput of independent fused
// multiply-add chains across every SM, in FP32 (the pair arithmetic of the
// mixed path) and in FP64 (the plain FP64 path).  The pair kernels are bound
// by this pipe, not by a dense contraction, so their roofline fraction is
// taken against this measured number.  The paper has no counterpart: it
// reports no hardware ceilings.
//
// Each thread runs kChains independent chains x <- x a + b (a just below 1,
// b small, so values stay finite); 2 flop per fused multiply-add.  The grid
// fills every SM with kBlocksPerSM blocks of kThreads threads, enough warps
// to cover the pipe latency.  A store guarded by a data-dependent test that
// never holds keeps the chains live.
#include <cmath>

#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 64;
constexpr int kThreads = 256;
constexpr int kBlocksPerSM = 8;

__device__ double g_peak_sink;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_chain(T a, T b, int reps)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = T(threadIdx.x) * T(1e-3) + T(c);
    for (int r = 0; r < reps; ++r) {
#pragma unroll
        for (int k = 0; k < kUnroll; ++k) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == T(-1.2345e-7)) g_peak_sink = (double)s;
}

template <typename T>
int timed_launch(int reps, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float &ms)
{
    const long long blocks = (long long)dev_info().sm_count * kBlocksPerSM;
    cudaEventRecord(e0, st);
    k_fma_chain<T><<<(unsigned)blocks, kThreads, 0, st>>>(T(0.999999), T(1e-7), reps);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) return fail(SPH_ECUDA, "sph_alu_peak: %s", cudaGetErrorString(e));
    return SPH_OK;
}

template <typename T>
int measure(double target_ms, cudaStream_t st, double *tflops, double *ms_out)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return fail(SPH_ECUDA, "sph_alu_peak: cudaEventCreate");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(SPH_ECUDA, "sph_alu_peak: cudaEventCreate");
    }
    // calibrate the repetition count on a short launch, then time one launch
    // of about target_ms
    int reps = 16;
    float ms = 0.f;
    int rc = timed_launch<T>(reps, st, e0, e1, ms);
    for (int k = 0; rc == SPH_OK && k < 6 && ms < 0.2 * target_ms && reps < (1 << 24); ++k) {
        const double f = ms > 1e-3 ? 0.5 * target_ms / ms : 64.0;
        reps = (int)fmin((double)reps * fmax(2.0, fmin(f, 64.0)), (double)(1 << 24));
        rc = timed_launch<T>(reps, st, e0, e1, ms);
    }
    if (rc == SPH_OK) {
        const double f = ms > 1e-3 ? target_ms / ms : 1.0;
        reps = (int)fmax(1.0, fmin((double)reps * f, (double)(1 << 26)));
        rc = timed_launch<T>(reps, st, e0, e1, ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPH_OK) return rc;
    const double threads = (double)dev_info().sm_count * kBlocksPerSM * kThreads;
    const double flop = 2.0 * threads * kChains * kUnroll * (double)reps;
    *tflops = flop / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    return SPH_OK;
}

}  // namespace

}  // namespace sph

extern "C" int sph_alu_peak(int precision, double target_ms, double *tflops, double *ms, void *stream)
{
    using namespace sph;
    if (!tflops) return fail(SPH_EINVAL, "sph_alu_peak: tflops is NULL");
    if (precision != SPH_PREC_MIXED && precision != SPH_PREC_FP64)
        return fail(SPH_EINVAL, "sph_alu_peak: precision must be SPH_PREC_MIXED (FP32) or SPH_PREC_FP64");
    if (!(target_ms > 0.0) || target_ms > 10000.0)
        return fail(SPH_EINVAL, "sph_alu_peak: target_ms must be in (0, 10000]");
    cudaStream_t st = (cudaStream_t)stream;
    return precision == SPH_PREC_FP64 ? measure<double>(target_ms, st, tflops, ms)
                                      : measure<float>(target_ms, st, tflops, ms);
}
