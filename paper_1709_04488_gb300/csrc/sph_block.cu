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
#include "sph_leaf.cuh"

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
    b.scratch64[10] = 0;                          // kick blocks done
    b.scratch64[11] = 0;
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
    if ((threadIdx.x & 31) == 0) {
        atomicMin((unsigned long long *)&b.scratch64[2], (unsigned long long)m);
        __threadfence();  // (before the block reports itself done)
    }
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
        b.bvh[g] = block_kick(ps.vx[i], ps.ax[i], hd);
        b.bvh[n + g] = block_kick(ps.vy[i], ps.ay[i], hd);
        b.bvh[2 * n + g] = block_kick(ps.vz[i], ps.az[i], hd);
        b.bvh[3 * n + g] = ps.ph.eos == SPH_EOS_ADIABATIC ? block_kick(ps.u[i], ps.du[i], hd) : ps.u[i];
        b.bvh[4 * n + g] = ps.ph.av_switch ? block_kick(ps.alpha[i], ps.dalpha[i], hd) : 0.0;
    }
    next_event(b, t1);
}

// A tick opens (all threads of one block): the step's counters and
// diagnostics are cleared, the tick advances to the next event tick, whose
// slot then collects a fresh minimum over the updated steps.
__device__ __forceinline__ void open_tick(const BatchView &b)
{
    const int k = threadIdx.x;
    if (k < kNumCounters) reset_counter(b, 1, k);
    if (k < b.nprob) reset_diag(b, k, 1);
    if (k == 0) {
        b.scratch64[5] = *(volatile long long *)&b.scratch64[2];  // (in L2: other blocks' minima)
        b.scratch64[2] = 0x7fffffffffffffffLL;
        b.counters[kBlockTasks] = 0;
    }
}

// after a tick (or before the first): the next tick opens if nothing failed
// and the next event tick lies after the current one and at most 2^L; the
// ticks before 2^L run as the loop, the tick at 2^L (every particle due)
// after it
__device__ __forceinline__ void schedule_next(const BatchView &b, long long k, long long N, int use_cond,
                                              cudaGraphConditionalHandle cond, cudaGraphConditionalHandle fin,
                                              int *go_s)
{
    ProbDiag *d = b.prob[0].diag;
    const long long next = *(volatile long long *)&b.scratch64[2];
    bool go = *(volatile unsigned *)&d->status == 0 && k < N && b.scratch64[8] < N;
    if (go && !(next > k && next <= N)) {
        atomicOr(&d->status, ST_SCHEDULE);
        go = false;
    }
    const bool loop = go && next < N, last = go && next == N;
    b.scratch64[9] = loop ? 1 : 0;
    b.scratch64[11] = last ? 1 : 0;
    if (use_cond) {
        cudaGraphSetConditional(cond, loop ? 1u : 0u);
        cudaGraphSetConditional(fin, last ? 1u : 0u);
    }
    *go_s = go;
}

// the loop's gate before the first tick; opens the first tick
__global__ void __launch_bounds__(128) k_block_gate(BatchView b, int L, int use_cond, cudaGraphConditionalHandle cond,
                                                    cudaGraphConditionalHandle fin)
{
    __shared__ int go_s;
    if (threadIdx.x == 0) schedule_next(b, 0, 1LL << L, use_cond, cond, fin, &go_s);
    __syncthreads();
    if (go_s) open_tick(b);
}

// graph form with tree reuse: whether this tick sorts and builds the leaves
// (the ticks k > 0 with k a multiple of tree_rebuild_every)
__global__ void k_block_tick_begin(BatchView b, int every, cudaGraphConditionalHandle cond)
{
    const long long k = b.scratch64[8];
    cudaGraphSetConditional(cond, k > 0 && k % every == 0 ? 1u : 0u);
}

__device__ __forceinline__ void count_due(const BatchView &b, bool due)
{
    const unsigned m = __ballot_sync(0xffffffffu, due);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd((unsigned long long *)&b.scratch64[3], (unsigned long long)__popc(m));
}

// drift every particle (original order), ahead of a new sort
__global__ void __launch_bounds__(kBlockThreads) k_block_drift(BatchView b)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool due = g < b.ntot && drift_one(b, g, b.scratch64[4], b.scratch64[5], bits_d(b.scratch64[7]));
    count_due(b, due);
}

// sorted particle s (after a new sort): the gather of position, mass and h
// into sorted order and the staging of its level for the force pass:
// +(level + 1) where the step ends at tick k1, -(level + 1) elsewhere
template <typename T>
__global__ void __launch_bounds__(kBlockThreads) k_block_gather(BatchView b)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long k1 = b.scratch64[5];
    if (s < b.ntot) {
        const ProbStatic &ps = b.prob[0];
        const long long g = b.perm[s], i = g - ps.base;
        b.sx[s] = ps.x[i];
        b.sy[s] = ps.y[i];
        b.sz[s] = ps.z[i];
        b.sm[s] = ps.m[i];
        b.sh[s] = ps.h[i];
        const T v = (T)(b.blev[g] + 1);
        ((T *)b.slev)[s] = b.bt1[g] == k1 ? v : -v;
    }
}

// after the force pass at tick k: closing half kick of the active particles
// and, before the end of the block, the level and opening half kick of their
// next step; inactive particles lifted by the reactive limiter end their
// step at the next tick of their new level's grid
__global__ void __launch_bounds__(kBlockThreads) k_block_kick(BatchView b, int L, int use_cond,
                                                              cudaGraphConditionalHandle cond,
                                                              cudaGraphConditionalHandle fin)
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
            // every input first (the stores below could alias them for the
            // compiler: one memory round trip each), the kicked v, u and
            // alpha kept for the next half kick
            const bool sw = ph.av_switch != 0, more = k < N;
            const double hd = half_ticks(t1 - t0, tau);
            const double vh[3] = {b.bvh[g], b.bvh[n + g], b.bvh[2 * n + g]};
            const double acc[3] = {A[0][i], A[1][i], A[2][i]};
            const double uh = b.bvh[3 * n + g], du = adi ? ps.du[i] : 0.0;
            const double ah = sw ? b.bvh[4 * n + g] : 0.0, da = sw ? ps.dalpha[i] : 0.0;
            double u = adi ? 0.0 : ps.u[i];
            const double dt = more ? particle_dt(ps, i) : 0.0;
            const int nml = more ? b.bnml[g] : 0;
            double v[3], al = 0.0;
            for (int a = 0; a < 3; ++a) {
                v[a] = block_kick(vh[a], acc[a], hd);
                V[a][i] = v[a];
            }
            if (adi) {
                u = block_kick(uh, du, hd);
                ps.u[i] = u;
            }
            if (sw) {
                al = block_kick(ah, da, hd);
                ps.alpha[i] = al;
            }
            if (more) {
                int l = level_of(dt, dtmax, L);
                const int lim = nml - ph.block_gap;
                if (l < lim) l = lim;
                if (l < lev)  // down one level, and only where synchronised
                    l = (k % (N >> (lev - 1)) == 0) ? lev - 1 : lev;
                lev = l;
                t0 = (int)k;
                t1 = (int)(k + (N >> l));
                const double hn = half_ticks(N >> l, tau);
                for (int a = 0; a < 3; ++a) b.bvh[a * n + g] = block_kick(v[a], acc[a], hn);
                b.bvh[3 * n + g] = adi ? block_kick(u, du, hn) : u;
                if (sw) b.bvh[4 * n + g] = block_kick(al, da, hn);
            }
        } else {
            const int rq = b.breq[g];
            if (rq > lev) {
                const long long stp = N >> rq;
                const long long ke = (k / stp + 1) * stp;  // next tick on the new level's grid
                if (ke < t1) {
                    const double corr = half_ticks(ke - t1, tau);
                    for (int a = 0; a < 3; ++a) b.bvh[a * n + g] = block_kick(b.bvh[a * n + g], A[a][i], corr);
                    if (adi) b.bvh[3 * n + g] = block_kick(b.bvh[3 * n + g], ps.du[i], corr);
                    if (ph.av_switch) b.bvh[4 * n + g] = block_kick(b.bvh[4 * n + g], ps.dalpha[i], corr);
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
    // the last block to finish ends the tick: the next one follows unless the
    // block is complete or a status is set; the next event tick must lie
    // after this one (read past L1: the other blocks' minima are in L2)
    __shared__ int last_s, go_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last_s = atomicAdd((unsigned long long *)&b.scratch64[10], 1ull) == (unsigned long long)gridDim.x - 1ull;
    }
    __syncthreads();
    if (!last_s) return;
    if (threadIdx.x == 0) {
        __threadfence();
        b.scratch64[10] = 0;
        b.scratch64[4] = k;
        b.scratch64[8] += 1;
        schedule_next(b, k, 1LL << L, use_cond, cond, fin, &go_s);
    }
    __syncthreads();
    if (go_s) open_tick(b);
}

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
                              cudaGraphConditionalHandle fin, cudaStream_t st)
{
    k_block_gate<<<1, 128, 0, st>>>(b, L, use_cond ? 1 : 0, cond, fin);
    return cudaGetLastError();
}

cudaError_t launch_block_tick_begin(const BatchView &b, int every, cudaGraphConditionalHandle cond,
                                    cudaStream_t st)
{
    k_block_tick_begin<<<1, 1, 0, st>>>(b, every > 1 ? every : 1, cond);
    return cudaGetLastError();
}

cudaError_t launch_block_drift(const BatchView &b, cudaStream_t st)
{
    k_block_drift<<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_block_gather(const BatchView &b, int precision, cudaStream_t st)
{
    const unsigned grid = blocks_for(b.ntot);
    if (precision == SPH_PREC_FP64) k_block_gather<double><<<grid, kBlockThreads, 0, st>>>(b);
    else k_block_gather<float><<<grid, kBlockThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_block_kick(const BatchView &b, int L, bool use_cond, cudaGraphConditionalHandle cond,
                             cudaGraphConditionalHandle fin, cudaStream_t st)
{
    k_block_kick<<<blocks_for(b.ntot), kBlockThreads, 0, st>>>(b, L, use_cond ? 1 : 0, cond, fin);
    return cudaGetLastError();
}

cudaError_t launch_block_finish(const BatchView &b, cudaStream_t st)
{
    k_block_finish<<<1, 1, 0, st>>>(b);
    return cudaGetLastError();
}

}  // namespace sph
