// Global-step leapfrog kick-drift-kick (Eqs. LFKDK1/LFKDK2), the CFL step
// (Eq. SPH_DT) and the FP64 conservation reductions, all in FP64 and in the
// caller's particle order.
//
// Reading of the paper for velocity-dependent forces: the first half kick and
// the drift use the stored a^n, du^n; the density solve and the forces are
// evaluated at the new positions with the predicted v^ = v^(n+1/2) + a^n dt/2
// and u^ = u^(n+1/2) + du^n dt/2; the closing half kick uses a^(n+1).
#include "sph_internal.cuh"

namespace sph {

namespace {

constexpr int kRedThreads = 256;

constexpr int kCloseItems = 8;  // most particles per thread in the closing kernel

__global__ void k_reset_step(BatchView b, int mode)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    reset_counters(b, mode);
    if (p < b.nprob) reset_diag(b, p, mode);
}

// step size of problem p: the caller's, else the CFL step of the last forces
__device__ __forceinline__ double step_dt(const ProbDiag *d, double dt_host)
{
    return dt_host > 0.0 ? dt_host : d->dt_next;
}

// Opening half kick and drift (Eq. LFKDK1) with the predicted v and u; block
// 0 also selects each problem's step and resets its diagnostics.
__global__ void k_kick_drift(BatchView b, double dt_host)
{
    reset_counters(b, 1);
    if (blockIdx.x == 0) {
        for (int p = threadIdx.x; p < b.nprob; p += blockDim.x) {
            ProbDiag *d = b.prob[p].diag;
            const double dt = step_dt(d, dt_host);
            reset_diag(b, p, 1);
            d->dt_cur = dt;
        }
    }
    long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= b.ntot) return;
    int p = find_problem(b.prob_base, b.nprob, g);
    const ProbStatic &ps = b.prob[p];
    const PhysParams &ph = ps.ph;
    long long i = g - ps.base;
    const double dt = step_dt(ps.diag, dt_host), hdt = 0.5 * dt;
    // every input first (the stores below could alias them for the
    // compiler: one memory round trip each)
    const bool adi = ph.eos == SPH_EOS_ADIABATIC, mm = ph.av_switch == SPH_AV_MORRIS_MONAGHAN;
    const double a[3] = {ps.ax[i], ps.ay[i], ps.az[i]};
    const double v0[3] = {ps.vx[i], ps.vy[i], ps.vz[i]};
    const double x0[3] = {ps.x[i], ps.y[i], ps.z[i]};
    const double u = ps.u[i], du = adi ? ps.du[i] : 0.0, h0 = ps.h[i];
    const float dv = b.divv ? b.divv[g] : 0.f;
    const double al0 = mm ? ps.alpha[i] : 0.0, dal = mm ? ps.dalpha[i] : 0.0;
    double *X[3] = {ps.x, ps.y, ps.z};
    double *Vv[3] = {ps.vx, ps.vy, ps.vz};
    double *VP[3] = {b.vpx, b.vpy, b.vpz};
    for (int k = 0; k < 3; ++k) {
        double vh = v0[k] + hdt * a[k];
        Vv[k][i] = vh;
        double x = x0[k] + vh * dt;
        if (ph.periodic) {
            double lo = ph.box_lo[k], L = ph.box_len[k];
            if (x >= lo + L) x -= L;
            else if (x < lo) x += L;
        }
        X[k][i] = x;
        VP[k][g] = vh + hdt * a[k];
    }
    // the h iteration starts from the continuity equation's prediction,
    // h exp(div v dt / 3) (h ~ rho^-1/3), bounded to a factor 1.25
    if (b.divv) {
        const float e = (float)(dt * (1.0 / 3.0)) * dv;
        ps.h[i] = h0 * (double)expf(fminf(fmaxf(e, -0.223f), 0.223f));  // (a starting guess: FP32 is enough)
    }
    if (adi) {
        double uh = u + hdt * du;
        ps.u[i] = uh;
        b.up[g] = uh + hdt * du;
    } else {
        b.up[g] = u;
    }
    if (mm) {  // the switch's alpha is kicked and predicted like u
        const double ah = al0 + hdt * dal;
        ps.alpha[i] = ah;
        b.ap[g] = ah + hdt * dal;
    }
}

__device__ __forceinline__ void add_diag(ProbDiag *d, const double *v)
{
    double *dst[9] = {&d->mass, &d->mom[0], &d->mom[1], &d->mom[2], &d->energy,
                      &d->fsum[0], &d->fsum[1], &d->fsum[2], &d->dEdt};
    for (int k = 0; k < 9; ++k) atomicAdd(dst[k], v[k]);
}

// Closing half kick (Eq. LFKDK2, optional) and the FP64 reductions per
// problem: each block takes items * blockDim consecutive particles and
// sums them per problem in registers, then reduces over the block when the
// whole block is in one problem (one set of atomics per block), else adds per
// thread.  Block 0 also finishes each problem's step record (CFL step of the
// forces just computed, time, step count, leaf count), which reads nothing
// this kernel writes.
__global__ void k_kick_close(BatchView b, int do_kick, int forces_ran, int items)
{
    __shared__ double red[9][kRedThreads / 32];
    __shared__ int pfirst, plast;
    if (blockIdx.x == 0) {
        for (int p = threadIdx.x; p < b.nprob; p += blockDim.x) {
            ProbDiag *d = b.prob[p].diag;
            if (forces_ran) d->dt_next = __longlong_as_double((long long)d->dt_min_bits);
            if (b.counters[kTimeoutCounter]) atomicOr(&d->status, ST_TIMEOUT);
            if (do_kick) {
                d->time += d->dt_cur;
                d->steps += 1;
            }
            d->leaves = b.dyn[p].nleaf;
            if (forces_ran) {
                // recording the force candidates in the density walk pays only
                // while they stay valid: after a step where they did not, walk
                // without recording for a while (8 steps, doubling up to 256
                // while retries keep failing), then try again
                int reused = 0;
                if (d->reuse_hold > 0) {
                    --d->reuse_hold;
                } else if (b.dyn[p].lists_stale) {
                    const int len = d->reuse_backoff > 0 ? d->reuse_backoff : kReuseHold;
                    d->reuse_hold = len;
                    d->reuse_backoff = len < 256 ? 2 * len : 256;
                } else {
                    reused = 1;
                    d->reuse_backoff = kReuseHold;
                }
                d->walk_reused = reused;
            }
        }
    }
    const long long base = (long long)blockIdx.x * blockDim.x * items;
    if (base >= b.ntot) return;
    const long long end = base + (long long)blockDim.x * items < b.ntot ? base + (long long)blockDim.x * items : b.ntot;
    if (threadIdx.x == 0) {
        pfirst = find_problem(b.prob_base, b.nprob, base);
        plast = find_problem(b.prob_base, b.nprob, end - 1);
    }
    __syncthreads();
    double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    int cur = -1;
    for (long long g = base + threadIdx.x; g < end; g += blockDim.x) {
        const int p = pfirst == plast ? pfirst : find_problem(b.prob_base, b.nprob, g);
        if (p != cur) {
            if (cur >= 0) {
                add_diag(b.prob[cur].diag, v);
                for (int k = 0; k < 9; ++k) v[k] = 0.0;
            }
            cur = p;
        }
        const ProbStatic &ps = b.prob[p];
        const PhysParams &ph = ps.ph;
        long long i = g - ps.base;
        const double hdt = 0.5 * ps.diag->dt_cur;
        double a[3] = {ps.ax[i], ps.ay[i], ps.az[i]};
        double vel[3] = {ps.vx[i], ps.vy[i], ps.vz[i]};
        double u = ps.u[i], du = ps.du[i];
        const bool adi = ph.eos == SPH_EOS_ADIABATIC;
        if (do_kick) {
            for (int k = 0; k < 3; ++k) vel[k] += hdt * a[k];
            ps.vx[i] = vel[0];
            ps.vy[i] = vel[1];
            ps.vz[i] = vel[2];
            if (adi) {
                u += hdt * du;
                ps.u[i] = u;
            }
            if (ph.av_switch == SPH_AV_MORRIS_MONAGHAN) ps.alpha[i] += hdt * ps.dalpha[i];
            if (ph.av_switch == SPH_AV_CULLEN_DEHNEN && forces_ran) {
                // Cullen & Dehnen: A = xi max(-dD/dt, 0) with dD/dt between the
                // step's two force evaluations; alpha rises to alpha_loc at once
                // and decays towards it on h / (2 av_decay v_sig)
                const double dt = 2.0 * hdt;
                const double ddot = (ps.dalpha[i] - b.cdold[g]) / dt;
                const double Aa = b.cdxi[g] * (ddot < 0.0 ? -ddot : 0.0);
                const double h = ps.h[i], h2A = h * h * Aa, vs = ps.vsig[i];
                const double aloc = h2A > 0.0 ? ph.alpha_av * h2A / (vs * vs + h2A) : 0.0;
                const double al = ps.alpha[i];
                ps.alpha[i] = al < aloc ? aloc : aloc + (al - aloc) * exp(-dt * 2.0 * ph.av_decay * vs / h);
            }
        }
        double m = ps.m[i];
        v[0] += m;
        v[1] += m * vel[0];
        v[2] += m * vel[1];
        v[3] += m * vel[2];
        v[4] += m * (0.5 * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]) + (adi ? u : 0.0));
        v[5] += m * a[0];
        v[6] += m * a[1];
        v[7] += m * a[2];
        v[8] += m * (vel[0] * a[0] + vel[1] * a[1] + vel[2] * a[2] + (adi ? du : 0.0));
    }
    if (pfirst == plast) {
        for (int k = 0; k < 9; ++k) {
            double x = warp_sum(v[k]);
            if ((threadIdx.x & 31) == 0) red[k][threadIdx.x >> 5] = x;
        }
        __syncthreads();
        if (threadIdx.x < 9) {
            double t = 0;
            for (int w = 0; w < kRedThreads / 32; ++w) t += red[threadIdx.x][w];
            ProbDiag *d = b.prob[pfirst].diag;
            double *dst[9] = {&d->mass, &d->mom[0], &d->mom[1], &d->mom[2], &d->energy,
                              &d->fsum[0], &d->fsum[1], &d->fsum[2], &d->dEdt};
            atomicAdd(dst[threadIdx.x], t);
        }
    } else if (cur >= 0) {
        add_diag(b.prob[cur].diag, v);
    }
}

}  // namespace

cudaError_t launch_reset_step(const BatchView &b, int mode, cudaStream_t st)
{
    k_reset_step<<<(b.nprob + 127) / 128, 128, 0, st>>>(b, mode);
    return cudaGetLastError();
}

cudaError_t launch_kick_drift(const BatchView &b, double dt_host, cudaStream_t st)
{
    const long long blocks = b.ntot > 0 ? (b.ntot + 255) / 256 : 1;
    k_kick_drift<<<(unsigned)blocks, 256, 0, st>>>(b, dt_host);
    return cudaGetLastError();
}

cudaError_t launch_kick_close(const BatchView &b, int do_kick, int forces_ran, cudaStream_t st)
{
    // enough blocks to fill the GPU twice, up to kCloseItems particles a thread
    const long long fill = 2LL * dev_info().sm_count * kRedThreads;
    long long items = (b.ntot + fill - 1) / fill;
    items = items < 1 ? 1 : items > kCloseItems ? kCloseItems : items;
    const long long per = (long long)kRedThreads * items;
    const long long blocks = b.ntot > 0 ? (b.ntot + per - 1) / per : 1;
    k_kick_close<<<(unsigned)blocks, kRedThreads, 0, st>>>(b, do_kick, forces_ran, (int)items);
    return cudaGetLastError();
}

}  // namespace sph
