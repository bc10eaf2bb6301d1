// Hierarchical block time-steps (Sec. 2.1.4) with the Saitoh & Makino
// limiter, for one problem per context.  One block step takes every particle
// from one synchronisation point to the next, Delta t_MAX later: levels
// l = 0 .. L step by Delta t_MAX / 2^l, and time is counted in ticks of
// Delta t_MAX / 2^L.  At every tick where some particle's step ends, all
// particles drift with their half-step velocities, and the particles whose
// step ends (the active ones) get a new h and density and new forces from
// the positions and predicted v and u of all, the closing half kick and the
// opening half kick of their next step; the others keep the h, density,
// pressure and sound speed of their last solve.  The
// force pass of the wrap-list launch serves them: it records the largest
// level among each active particle's neighbours (the predictive limiter) and
// lifts inactive neighbours more than block_gap levels below (the reactive
// one).  Every rule is taken on integer levels and ticks, so both precisions
// make the same decisions from the same step lengths.
//
// The kick, drift and prediction arithmetic is written with explicit
// rounding, operation for operation as the reference formulas state it.
//
// The schedule lives on the device (Delta t_MAX, the tick length, the current
// and next event ticks), so the host can enqueue the ticks as the body of a
// graph loop whose condition the last kernel of each tick sets: no host round
// trip between ticks.
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kBlockThreads = 256;

__device__ __forceinline__ unsigned long long dbits(double v)
{
    return (unsigned long long)__double_as_longlong(v);  // positive doubles order as integers
}

// lowest level l <= L whose step Delta t_MAX / 2^l is at most dt
__device__ __forceinline__ int level_of(double dt, double dtmax, int L)
{
    int l = 0;
    while (l < L && ldexp(dtmax, -l) > dt) ++l;
    return l;
}

// the CFL step of Eq. SPH_DT from the last force evaluation and, with
// gravity, the acceleration condition of Eq. SPH_DTACCEL
__device__ __forceinline__ double particle_dt(const ProbStatic &ps, long long i)
{
    double d = __ddiv_rn(__dmul_rn(ps.ph.c_cfl, ps.h[i]), ps.vsig[i]);
    if (ps.ph.gravity) {
        const double a2 = __dadd_rn(__dadd_rn(__dmul_rn(ps.ax[i], ps.ax[i]), __dmul_rn(ps.ay[i], ps.ay[i])),
                                    __dmul_rn(ps.az[i], ps.az[i]));
        const double a = __dsqrt_rn(a2);
        if (a > 0) {
            const double gdt = __dmul_rn(ps.ph.c_grav, __dsqrt_rn(__ddiv_rn(ps.h[i], a)));
            if (gdt < d) d = gdt;
        }
    }
    return d;
}

__device__ __forceinline__ double kick(double v, double a, double d) { return __dadd_rn(v, __dmul_rn(a, d)); }

// half of `ticks` ticks of length tau
__device__ __forceinline__ double half_ticks(long long ticks, double tau)
{
    return __dmul_rn(__dmul_rn(0.5, (double)ticks), tau);
}

__device__ __forceinline__ double bits_d(long long v) { return __longlong_as_double(v); }

__global__ void k_block_init(BatchView b)
{
    b.scratch64[0] = (long long)dbits(INFINITY);  // smallest step
    b.scratch64[1] = 0;                           // largest step
    b.scratch64[2] = 0x7fffffffffffffffLL;        // next tick where a step ends
    b.scratch64[3] = 0;                           // particle force evaluations
    b.scratch64[4] = 0;                           // the block starts at tick 0
    b.scratch64[8] = 0;                           // ticks taken
    b.scratch64[9] = 0;
}

__global__ void __launch_bounds__(kBlockThreads) k_block_dt(BatchView b)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double lo = INFINITY, hi = 0.0;
    if (g < b.ntot) {
        const ProbStatic &ps = b.prob[0];
        lo = hi = particle_dt(ps, g - ps.base);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if ((threadIdx.x & 31) == 0) {
        if (lo < INFINITY) atomicMin((unsigned long long *)&b.scratch64[0], dbits(lo));
        atomicMax((unsigned long long *)&b.scratch64[1], dbits(hi));
    }
}

// Delta t_MAX: the largest step, or 2^L times the smallest if that is less;
// no finite positive step leaves Delta t_MAX = 0 and a non-finite status
__global__ void k_block_plan(BatchView b, int L)
{
    const double dmin = bits_d(b.scratch64[0]), dmax = bits_d(b.scratch64[1]);
    double dtmax = 0.0, tau = 0.0;
    if (dmin > 0 && dmin < INFINITY) {
        const double cap = ldexp(dmin, L);
        dtmax = dmax < cap ? dmax : cap;
        tau = ldexp(dtmax, -L);
    } else {
        atomicOr(&b.prob[0].diag->status, ST_NONFINITE);
    }
    b.scratch64[6] = __double_as_longlong(dtmax);
    b.scratch64[7] = __double_as_longlong(tau);
}

__device__ __forceinline__ void next_event(const BatchView &b, long long t)
{
    const long long m = warp_min(t);
    if ((threadIdx.x & 31) == 0) atomicMin((unsigned long long *)&b.scratch64[2], (unsigned long long)m);
}

// each particle's opening step: level from its CFL step, raised to within
// block_gap of its neighbours' largest level, and the opening half kick
__global__ void __launch_bounds__(kBlockThreads) k_block_open(BatchView b, int L)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const double dtmax = bits_d(b.scratch64[6]), tau = bits_d(b.scratch64[7]);
    long long t1 = 0x7fffffffffffffffLL;
    if (g < b.ntot && dtmax > 0) {
        const ProbStatic &ps = b.prob[0];
        const long long i = g - ps.base;
        int l = level_of(particle_dt(ps, i), dtmax, L);
        const int lim = b.bnml[g] - ps.ph.block_gap;
        if (l < lim) l = lim;
        b.blev[g] = l;
        b.bt0[g] = 0;
        b.bt1[g] = (int)((1LL << L) >> l);
        t1 = b.bt1[g];
        const double hd = half_ticks(t1, tau);
        const long long n = b.ntot;
        b.bvh[g] = kick(ps.vx[i], ps.ax[i], hd);
        b.bvh[n + g] = kick(ps.vy[i], ps.ay[i], hd);
        b.bvh[2 * n + g] = kick(ps.vz[i], ps.az[i], hd);
        b.bvh[3 * n + g] = ps.ph.eos == SPH_EOS_ADIABATIC ? kick(ps.u[i], ps.du[i], hd) : ps.u[i];
        b.bvh[4 * n + g] = ps.ph.av_switch ? kick(ps.alpha[i], ps.dalpha[i], hd) : 0.0;
    }
    next_event(b, t1);
}

// the loop's gate before the first tick: the first event tick must lie in
// (0, 2^L] and nothing may have failed
__global__ void k_block_gate(BatchView b, int L, int use_cond, cudaGraphConditionalHandle cond)
{
    ProbDiag *d = b.prob[0].diag;
    const long long N = 1LL << L, next = b.scratch64[2];
    bool go = d->status == 0;
    if (go && !(next > 0 && next <= N)) {
        atomicOr(&d->status, ST_SCHEDULE);
        go = false;
    }
    b.scratch64[9] = go ? 1 : 0;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// a tick starts: it advances to the next event tick; with tree reuse, the
// branch condition says whether this tick sorts and builds the leaves
__global__ void k_block_tick_begin(BatchView b, int every, int use_cond, cudaGraphConditionalHandle cond)
{
    b.scratch64[5] = b.scratch64[2];
    b.counters[kBlockTasks] = 0;
    if (use_cond) cudaGraphSetConditional(cond, b.scratch64[8] % every == 0 ? 1u : 0u);
}

// a tick ends: the next one follows unless the block is complete or a
// status is set; the next event tick must lie after this one
__global__ void k_block_tick_end(BatchView b, int L, int use_cond, cudaGraphConditionalHandle cond)
{
    ProbDiag *d = b.prob[0].diag;
    const long long N = 1LL << L, k1 = b.scratch64[5], next = b.scratch64[2];
    b.scratch64[4] = k1;
    b.scratch64[8] += 1;
    bool go = d->status == 0 && k1 < N;
    if (go && !(next > k1 && next <= N)) {
        atomicOr(&d->status, ST_SCHEDULE);
        go = false;
    }
    b.scratch64[9] = go ? 1 : 0;
    if (use_cond) cudaGraphSetConditional(cond, go ? 1u : 0u);
}

// drift every particle from tick k0 to tick k1, mark the particles whose
// step ends at k1, predict v, u and alpha at k1 for the force pass
__global__ void __launch_bounds__(kBlockThreads) k_block_drift(BatchView b)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k0 = b.scratch64[4], k1 = b.scratch64[5];
    const double tau = bits_d(b.scratch64[7]);
    bool due = false;
    if (g < b.ntot) {
        const ProbStatic &ps = b.prob[0];
        const PhysParams &ph = ps.ph;
        const long long i = g - ps.base, n = b.ntot;
        const double dk = __dmul_rn((double)(k1 - k0), tau);
        double *X[3] = {ps.x, ps.y, ps.z};
        const double *A[3] = {ps.ax, ps.ay, ps.az};
        double *VP[3] = {b.vpx, b.vpy, b.vpz};
        const int t0 = b.bt0[g], t1 = b.bt1[g];
        const double dp = __dmul_rn(__dmul_rn((double)(2 * k1 - t0 - t1), 0.5), tau);  // t - t_mid
        for (int a = 0; a < 3; ++a) {
            const double vh = b.bvh[a * n + g];
            double x = __dadd_rn(X[a][i], __dmul_rn(vh, dk));
            if (ph.periodic) {
                const double lo = ph.box_lo[a], Lb = ph.box_len[a];
                if (x >= lo + Lb) x -= Lb;
                else if (x < lo) x += Lb;
            }
            X[a][i] = x;
            VP[a][g] = kick(vh, A[a][i], dp);
        }
        b.up[g] = ph.eos == SPH_EOS_ADIABATIC ? kick(b.bvh[3 * n + g], ps.du[i], dp) : ps.u[i];
        if (ph.av_switch) b.ap[g] = kick(b.bvh[4 * n + g], ps.dalpha[i], dp);
        b.breq[g] = -1;
        due = t1 == k1;
    }
    const unsigned m = __ballot_sync(0xffffffffu, due);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long *)&b.scratch64[3], (unsigned long long)__popc(m));
}

// sorted staging of the levels for the force pass: +(level + 1) where the
// step ends at tick k, -(level + 1) elsewhere
template <typename T>
__global__ void __launch_bounds__(kBlockThreads) k_block_stage(BatchView b)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= b.ntot) return;
    const long long k = b.scratch64[5];
    const int g = b.perm[s];
    const T v = (T)(b.blev[g] + 1);
    ((T *)b.slev)[s] = b.bt1[g] == k ? v : -v;
}

// the tick's tasks for the pair kernels: each leaf with particles whose step
// ends now gives one task per 32 / block_lanes of them (in sorted order), so
// that a task's block_lanes lanes per particle and its box (of those
// particles only) keep the pair kernels' latency short when few particles
// of a leaf are due
template <typename T>
__global__ void __launch_bounds__(kBlockThreads) k_block_tasks(BatchView b)
{
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) {
        const int st = b.leaf_start[leaf], n = b.leaf_start[leaf + 1] - st;  // (n <= 32)
        const bool due = lane < n && ((const T *)b.slev)[st + (lane < n ? lane : 0)] > T(0);
        const int d = __popc(__ballot_sync(0xffffffffu, due));
        const int size = 32 / b.block_lanes, nt = (d + size - 1) / size;
        int base = 0;
        if (lane == 0 && nt > 0) base = atomicAdd(&b.counters[kBlockTasks], nt);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < nt) b.btask[base + lane] = (leaf << 5) | (lane * size);
    }
}

// after the force pass at tick k: closing half kick of the active particles
// and, before the end of the block, the level and opening half kick of their
// next step; inactive particles lifted by the reactive limiter end their
// step at the next tick of their new level's grid
__global__ void __launch_bounds__(kBlockThreads) k_block_kick(BatchView b, int L)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k = b.scratch64[5];
    const double dtmax = bits_d(b.scratch64[6]), tau = bits_d(b.scratch64[7]);
    long long tnext = 0x7fffffffffffffffLL;
    if (g < b.ntot) {
        const ProbStatic &ps = b.prob[0];
        const PhysParams &ph = ps.ph;
        const long long i = g - ps.base, n = b.ntot, N = 1LL << L;
        const bool adi = ph.eos == SPH_EOS_ADIABATIC;
        const double *A[3] = {ps.ax, ps.ay, ps.az};
        double *V[3] = {ps.vx, ps.vy, ps.vz};
        int t0 = b.bt0[g], t1 = b.bt1[g], lev = b.blev[g];
        if (t1 == k) {
            const double hd = half_ticks(t1 - t0, tau);
            for (int a = 0; a < 3; ++a) V[a][i] = kick(b.bvh[a * n + g], A[a][i], hd);
            if (adi) ps.u[i] = kick(b.bvh[3 * n + g], ps.du[i], hd);
            if (ph.av_switch) ps.alpha[i] = kick(b.bvh[4 * n + g], ps.dalpha[i], hd);
            if (k < N) {
                int l = level_of(particle_dt(ps, i), dtmax, L);
                const int lim = b.bnml[g] - ph.block_gap;
                if (l < lim) l = lim;
                if (l < lev)  // down one level, and only where synchronised
                    l = (k % (N >> (lev - 1)) == 0) ? lev - 1 : lev;
                lev = l;
                t0 = (int)k;
                t1 = (int)(k + (N >> l));
                const double hn = half_ticks(N >> l, tau);
                for (int a = 0; a < 3; ++a) b.bvh[a * n + g] = kick(V[a][i], A[a][i], hn);
                b.bvh[3 * n + g] = adi ? kick(ps.u[i], ps.du[i], hn) : ps.u[i];
                if (ph.av_switch) b.bvh[4 * n + g] = kick(ps.alpha[i], ps.dalpha[i], hn);
            }
        } else {
            const int rq = b.breq[g];
            if (rq > lev) {
                const long long stp = N >> rq;
                const long long ke = (k / stp + 1) * stp;  // next tick on the new level's grid
                if (ke < t1) {
                    const double corr = half_ticks(ke - t1, tau);
                    for (int a = 0; a < 3; ++a) b.bvh[a * n + g] = kick(b.bvh[a * n + g], A[a][i], corr);
                    if (adi) b.bvh[3 * n + g] = kick(b.bvh[3 * n + g], ps.du[i], corr);
                    if (ph.av_switch) b.bvh[4 * n + g] = kick(b.bvh[4 * n + g], ps.dalpha[i], corr);
                    t1 = (int)ke;
                    lev = rq;
                }
            }
        }
        b.bt0[g] = t0;
        b.bt1[g] = t1;
        b.blev[g] = lev;
        if (t1 > k) tnext = t1;
    }
    next_event(b, tnext);
}

__global__ void k_block_next_reset(BatchView b) { b.scratch64[2] = 0x7fffffffffffffffLL; }

__global__ void k_block_finish(BatchView b)
{
    ProbDiag *d = b.prob[0].diag;
    if (d->status) return;  // a failed block leaves the clock where it was
    d->time += bits_d(b.scratch64[6]);
    d->steps += 1;
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + kBlockThreads - 1) / kBlockThreads); }

}  // namespace

cudaError_t launch_block_dt(const BatchView &b, int L, cudaStream_t st)
{
    k_block_init<<<1, 1, 0, st>>>(b);
    k_block_dt<<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b);
    k_block_plan<<<1, 1, 0, st>>>(b, L);
    return cudaGetLastError();
}

cudaError_t launch_block_open(const BatchView &b, int L, cudaStream_t st)
{
    k_block_open<<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b, L);
    return cudaGetLastError();
}

cudaError_t launch_block_gate(const BatchView &b, int L, bool use_cond, cudaGraphConditionalHandle cond,
                              cudaStream_t st)
{
    k_block_gate<<<1, 1, 0, st>>>(b, L, use_cond ? 1 : 0, cond);
    return cudaGetLastError();
}

cudaError_t launch_block_tick_begin(const BatchView &b, int every, bool use_cond, cudaGraphConditionalHandle cond,
                                    cudaStream_t st)
{
    k_block_tick_begin<<<1, 1, 0, st>>>(b, every > 1 ? every : 1, use_cond ? 1 : 0, cond);
    return cudaGetLastError();
}

cudaError_t launch_block_drift(const BatchView &b, cudaStream_t st)
{
    k_block_drift<<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_block_stage(const BatchView &b, int precision, cudaStream_t st)
{
    if (precision == SPH_PREC_FP64) k_block_stage<double><<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b);
    else k_block_stage<float><<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_block_tasks(const BatchView &b, int precision, cudaStream_t st)
{
    const unsigned grid = (unsigned)dev_info().sm_count * 4;
    if (precision == SPH_PREC_FP64) k_block_tasks<double><<<grid, kBlockThreads, 0, st>>>(b);
    else k_block_tasks<float><<<grid, kBlockThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_block_kick(const BatchView &b, int L, cudaStream_t st)
{
    k_block_next_reset<<<1, 1, 0, st>>>(b);  // the next event is a fresh minimum over the updated steps
    k_block_kick<<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b, L);
    return cudaGetLastError();
}

cudaError_t launch_block_tick_end(const BatchView &b, int L, bool use_cond, cudaGraphConditionalHandle cond,
                                  cudaStream_t st)
{
    k_block_tick_end<<<1, 1, 0, st>>>(b, L, use_cond ? 1 : 0, cond);
    return cudaGetLastError();
}

cudaError_t launch_block_finish(const BatchView &b, cudaStream_t st)
{
    k_block_finish<<<1, 1, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace sph
