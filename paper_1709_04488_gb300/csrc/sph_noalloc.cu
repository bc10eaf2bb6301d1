// An entry point that allocates nothing: the density solve and the force
// evaluation of one problem, with all of its scratch memory in a fixed array
// compiled into the library.
//
// Who needs it: code that may not create device allocations of its own.  A
// host that owns every byte of device memory through its own pool (so that a
// raw allocation would bypass its accounting or fail once the pool has
// reserved the free memory), a plug-in called back from such a host, or a
// real-time loop that must not enter the CUDA allocator can still call
// this with its own input and output arrays.  The price is a fixed scratch
// area that every GPU using the library keeps until the process exits, and a
// cap on the problem size.
#include <mutex>

#include "sph_internal.cuh"

namespace {

using namespace sph;

// Largest problem the fixed scratch holds, and its size.  24 MiB holds the
// workspace layout of every option for 32768 particles: the FP64 layout
// (15 MiB) plus self-gravity's buffers (partial sums of split partner
// ranges, the tree walk's copies; the FP64 tree walk's layout is the
// largest, 22 MiB), plus the diagnostics record.  noalloc_max_n() finds the
// largest n for a layout that would not fit (a guard: none does now).
constexpr long long kNoAllocMaxN = 32768;
constexpr size_t kNoAllocBytes = (size_t)24 << 20;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array per device, looked up once per device.
void *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

int scratch_for_current_device(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(SPH_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(SPH_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(SPH_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SPH_OK;
}

// Bytes of the fixed scratch one call of n particles with parameters p uses.
size_t noalloc_bytes(const sph_params *p, long long n)
{
    Carver c{nullptr};
    c.take<ProbDiag>(1);
    BatchView b;
    memset(&b, 0, sizeof b);
    carve_tables(c, b, 1);
    carve_arrays(c, b, n, 1, p->precision, p->gravity ? gravity_chunks(n, p->grav_theta) : 0,
                 p->gravity && p->grav_theta > 0);
    return c.off;
}

// Largest n (<= kNoAllocMaxN) whose layout fits the fixed scratch for p.
long long noalloc_max_n(const sph_params *p)
{
    if (noalloc_bytes(p, kNoAllocMaxN) <= kNoAllocBytes) return kNoAllocMaxN;
    long long lo = 0, hi = kNoAllocMaxN;  // fits(lo), !fits(hi)
    while (hi - lo > 1) {
        const long long mid = (lo + hi) / 2;
        if (noalloc_bytes(p, mid) <= kNoAllocBytes) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Writes the problem table and clears everything a call must find at zero.
__global__ void k_noalloc_init(BatchView b, ProbStatic ps)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        b.prob[0] = ps;
        b.prob_base[0] = 0;
        b.prob_base[1] = ps.n;
        memset(b.dyn, 0, sizeof(ProbDyn));
        memset(ps.diag, 0, sizeof(ProbDiag));
    }
    if (blockIdx.x == 0) b.counters[threadIdx.x] = 0;  // kNumCounters threads
}

}  // namespace

extern "C" int sph_density_forces_noalloc(const sph_params *p, int64_t n, const sph_state *state, void *stream)
{
    int rc = validate(p);
    if (rc) return rc;
    if (n < 0 || n > kNoAllocMaxN)
        return fail(SPH_EINVAL, "n = %lld: the allocation-free entry point takes at most %lld particles",
                    (long long)n, kNoAllocMaxN);
    if (noalloc_bytes(p, n) > kNoAllocBytes)
        return fail(SPH_ENOSPACE,
                    "n = %lld does not fit the allocation-free entry point's fixed scratch with these "
                    "parameters (self-gravity needs extra buffers): at most %lld particles",
                    (long long)n, noalloc_max_n(p));
    if (!state) return fail(SPH_EINVAL, "state is NULL");
    if (n > 0) {
        const double *req[] = {state->x, state->y, state->z, state->vx, state->vy, state->vz, state->u,
                               state->m, state->h, state->rho, state->omega, state->P, state->c,
                               state->ax, state->ay, state->az, state->du, state->vsig};
        for (const double *q : req)
            if (!q) return fail(SPH_EINVAL, "a state array is NULL");
        if (p->av_switch && (!state->alpha || !state->dalpha))
            return fail(SPH_EINVAL, "the viscosity switch needs state.alpha and state.dalpha");
    }
    void *base = nullptr;
    rc = scratch_for_current_device(&base);
    if (rc) return rc;
    // lay the workspace out inside the fixed array
    Carver c{(char *)base};
    ProbDiag *diag = c.take<ProbDiag>(1);
    BatchView b;
    memset(&b, 0, sizeof b);
    carve_tables(c, b, 1);
    carve_arrays(c, b, n, 1, p->precision, p->gravity ? gravity_chunks(n, p->grav_theta) : 0,
                 p->gravity && p->grav_theta > 0);
    if (c.off > kNoAllocBytes)  // (checked above; kept as a guard on the layout)
        return fail(SPH_ENOSPACE, "fixed scratch too small for %lld particles", (long long)n);
    const int lpp = lpp_of(p, n);
    b.ntot = n;
    b.key_bits = key_bits_for(1);
    b.key_lo = key_low_bits(n);
    b.lpp_mask = mask_of(lpp, p->kernel);
    b.dens_mask = dens_class_bit(lpp, 0, p->kernel);  // masses are not inspected here: distance-and-mass lists
    b.any_isolated = p->periodic ? 0 : 1;
    b.any_periodic = p->periodic ? 1 : 0;
    b.any_general = (p->av_switch || p->ac_signal || p->gravity) ? 1 : 0;
    b.any_gravity = p->gravity ? 1 : 0;
    b.any_cd = p->av_switch == SPH_AV_CULLEN_DEHNEN ? 1 : 0;
    b.grav_blocks = p->gravity ? gravity_blocks(n, p->grav_theta) : 0;
    b.grav_split = p->gravity && gravity_chunks(n, p->grav_theta) > 1;
    b.any_grav_tree = p->gravity && p->grav_theta > 0;
    ProbStatic ps;
    memset(&ps, 0, sizeof ps);
    ps.x = state->x;
    ps.y = state->y;
    ps.z = state->z;
    ps.vx = state->vx;
    ps.vy = state->vy;
    ps.vz = state->vz;
    ps.u = state->u;
    ps.m = state->m;
    ps.h = state->h;
    ps.rho = state->rho;
    ps.omega = state->omega;
    ps.P = state->P;
    ps.c = state->c;
    ps.ax = state->ax;
    ps.ay = state->ay;
    ps.az = state->az;
    ps.du = state->du;
    ps.vsig = state->vsig;
    ps.alpha = state->alpha;
    ps.dalpha = state->dalpha;
    ps.n = n;
    ps.base = 0;
    ps.diag = diag;
    ps.lpp = lpp;
    ps.ph = phys_of(p);
    ps.gchunks = p->gravity ? gravity_chunks(n, p->grav_theta) : 0;
    cudaStream_t st = (cudaStream_t)stream;
    const int prec = p->precision;
    cudaError_t e;
#define NA_TRY(x)                                                                                  \
    do {                                                                                           \
        e = (x);                                                                                   \
        if (e != cudaSuccess) return fail(SPH_ECUDA, "%s: %s", #x, cudaGetErrorString(e));         \
    } while (0)
    k_noalloc_init<<<1, kNumCounters, 0, st>>>(b, ps);
    NA_TRY(cudaGetLastError());
    NA_TRY(cudaMemsetAsync(b.zero_lo, 0, b.zero_bytes, st));
    NA_TRY(launch_reset_step(b, 1, st));
    NA_TRY(launch_domain_and_keys(b, st));
    NA_TRY(launch_radix_sort(b, st));
    NA_TRY(launch_gather(b, st));
    NA_TRY(launch_build_leaves(b, prec, st));
    NA_TRY(launch_density(b, prec, 0, st));
    NA_TRY(launch_refit(b, prec, st));
    NA_TRY(launch_forces(b, prec, st));
    launch_gravity(b, prec, st);
    NA_TRY(cudaGetLastError());
    NA_TRY(launch_kick_close(b, 0, 1, st));
    if (p->flags & SPH_FLAG_ASYNC) return SPH_OK;
    NA_TRY(cudaStreamSynchronize(st));
    unsigned status = 0;
    NA_TRY(cudaMemcpy(&status, &diag->status, sizeof status, cudaMemcpyDeviceToHost));
#undef NA_TRY
    return status_to_code(status);
}
