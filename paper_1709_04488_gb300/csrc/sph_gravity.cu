// Self-gravity, long-range part of Eq. SPHSELFGRAV (Sec. 2.1.2): the
// kernel-softened attraction
//   g_i = -G sum_{j != i} m_j (phi'(r_ij,h_i) + phi'(r_ij,h_j))/2 r_hat_ij,
// phi'(r,h) = M(r/h)/r^2 (Eq. GRAVFORCEKERNEL), either by direct summation over
// every particle of the problem (grav_theta = 0, k_gravity below) or by the
// tree walk of Sec. 4.2 (k_grav_moments, k_gravity_tree further down).  The
// zeta term of the same equation runs in the force pass with the neighbours.
// During a block step only the particles whose step ends take the long range.
//
// Direct sum: two particles per thread, sorted order; the blocks of a problem cover only
// that problem's particles (each problem's first block is precomputed on the
// host), and the partner particles stream through shared memory in tiles.
// A problem too small to fill the GPU with one block per 256 particles splits
// its partners into C ranges (C depends on N alone, so a problem gives the
// same bits alone or in a batch): each block sums one range into FP64
// partials, and a second kernel adds the C partials in range order.
// Positions are taken relative to the problem's key-domain corner in FP64 and
// cast, like the leaf offsets of the pair kernels.  Each pair term is formed
// from the same staged values on both sides with explicit rounding, so
// F_ij = -F_ji bit for bit, and F_i is accumulated with TwoSum; a_i = G F_i / m_i
// in FP64 is added to the accelerations the force pass wrote.
#include "sph_pairs.cuh"

namespace sph {

namespace {

constexpr int kGravThreads = 128;  // two particles per thread: 256 per block

// M(q) of the force kernel with every operation's rounding fixed, so that
// both particles of a pair get the same bits
template <typename T>
__device__ __forceinline__ T grav_mass_rn(T q)
{
    if (q >= T(2)) return T(1);
    const T q2 = mul_rn(q, q), q3 = mul_rn(q2, q);
    if (q < T(1)) return mul_rn(mul_rn(T(4), q3), fma_rn(q2, fma_rn(T(0.125), q, T(-0.3)), T(1.0 / 3.0)));
    return mul_rn(T(4), fma_rn(q3, fma_rn(q, fma_rn(q, fma_rn(q, T(-1.0 / 24.0), T(0.3)), T(-0.75)), T(2.0 / 3.0)),
                               T(-1.0 / 60.0)));
}

// partners per range: ceil(N/C) rounded up to whole tiles
__host__ __device__ inline long long gravity_span(long long n, int c)
{
    const long long s = (n + c - 1) / c;
    return (s + 2 * kGravThreads - 1) / (2 * kGravThreads) * (2 * kGravThreads);
}

template <typename T>
struct GravVec;
template <>
struct GravVec<float> {
    using P = float4;  // position (relative to the problem's corner), mass
    using H = float2;  // h, 1/h
};
template <>
struct GravVec<double> {
    using P = dbl4;
    using H = double2;
};

// one pair term of particle (x, m, h, 1/h) with staged partner q, hq:
// -G m_i m_j phi_bar' r_hat with phi_bar' = (phi'(r,h_i) + phi'(r,h_j))/2,
// added to (ax, ay, az); the self pair (r = 0) adds nothing
template <typename T, typename P, typename H>
__device__ __forceinline__ void grav_pair(T xi, T yi, T zi, T mi, T hi, T hinv_i, const P &q, const H &hq,
                                          TwoSumAcc<T> &ax, TwoSumAcc<T> &ay, TwoSumAcc<T> &az)
{
    const T rx = sub_rn(xi, q.x), ry = sub_rn(yi, q.y), rz = sub_rn(zi, q.z);
    const T r2 = fma_rn(rz, rz, fma_rn(ry, ry, mul_rn(rx, rx)));
    const T rinv = rsqrt_t(r2);
    const T rinv2 = mul_rn(rinv, rinv);
    T fbar = rinv2;  // beyond both supports: 1/r^2
    const T r = mul_rn(r2, rinv);
    if (r < T(2) * (hi > hq.x ? hi : hq.x))
        fbar = mul_rn(mul_rn(T(0.5), add_rn(grav_mass_rn(mul_rn(r, hinv_i)), grav_mass_rn(mul_rn(r, hq.y)))), rinv2);
    const T w = r2 > T(0) ? mul_rn(mul_rn(mul_rn(mi, q.w), fbar), rinv) : T(0);  // symmetric in (i, j)
    ax.add(-mul_rn(w, rx));
    ay.add(-mul_rn(w, ry));
    az.add(-mul_rn(w, rz));
}

// Each thread serves two particles (kGravThreads apart), so that each staged
// partner is read from shared memory once per two pair terms.
template <typename T>
__global__ void __launch_bounds__(kGravThreads) k_gravity(BatchView b)
{
    using P = typename GravVec<T>::P;
    using H = typename GravVec<T>::H;
    __shared__ P tp[2 * kGravThreads];
    __shared__ H th[2 * kGravThreads];
    // problem of this block: the last one whose first block is <= blockIdx.x
    int p = 0;
    for (int lo = 0, hi = b.nprob - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (b.prob[mid].gblk0 <= (int)blockIdx.x) {
            p = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    while (p > 0 && !b.prob[p].ph.gravity) --p;  // (problems without gravity own no blocks)
    const ProbStatic &ps = b.prob[p];
    const long long base = b.prob_base[p], n = ps.n, end = base + n;
    const int C = ps.gchunks, rel = (int)blockIdx.x - ps.gblk0, ib = rel / C, ch = rel - ib * C;
    const long long span = gravity_span(n, C);
    const long long jlo = base + ch * span, jhi = jlo + span < end ? jlo + span : end;
    const long long i0 = base + (long long)ib * (2 * kGravThreads) + threadIdx.x;
    const long long i1 = i0 + kGravThreads;
    const double *ref = b.dyn[p].dom_lo;
    auto load = [&](long long i, P &x, H &h) {
        x.x = (T)(b.sx[i] - ref[0]);
        x.y = (T)(b.sy[i] - ref[1]);
        x.z = (T)(b.sz[i] - ref[2]);
        x.w = (T)b.sm[i];
        h.x = (T)b.sh[i];
        h.y = T(1) / h.x;  // the same 1/h the partner's tile holds
    };
    P x0, x1;
    H h0, h1;
    x0.x = x0.y = x0.z = x0.w = x1.x = x1.y = x1.z = x1.w = T(0);
    h0.x = h0.y = h1.x = h1.y = T(1);
    if (i0 < end) load(i0, x0, h0);
    if (i1 < end) load(i1, x1, h1);
    TwoSumAcc<T> a0x{T(0), T(0)}, a0y{T(0), T(0)}, a0z{T(0), T(0)};
    TwoSumAcc<T> a1x{T(0), T(0)}, a1y{T(0), T(0)}, a1z{T(0), T(0)};
    for (long long j0 = jlo; j0 < jhi; j0 += 2 * kGravThreads) {
        __syncthreads();  // the previous tile is consumed
        for (int t = threadIdx.x; t < 2 * kGravThreads; t += kGravThreads)
            if (j0 + t < jhi) load(j0 + t, tp[t], th[t]);
        __syncthreads();
        const int jn = (int)(jhi - j0 < 2 * kGravThreads ? jhi - j0 : 2 * kGravThreads);
#pragma unroll 4
        for (int k = 0; k < jn; ++k) {
            const P q = tp[k];
            const H hq = th[k];
            grav_pair(x0.x, x0.y, x0.z, x0.w, h0.x, h0.y, q, hq, a0x, a0y, a0z);
            grav_pair(x1.x, x1.y, x1.z, x1.w, h1.x, h1.y, q, hq, a1x, a1y, a1z);
        }
    }
    auto store = [&](long long i, const TwoSumAcc<T> &ax, const TwoSumAcc<T> &ay, const TwoSumAcc<T> &az) {
        if (b.block_on && ((const T *)b.slev)[i] < T(0)) return;  // block step: not this particle's force pass
        if (C > 1) {  // partial of range ch, layout [ch][axis][ntot]
            double *g = b.gpart + (long long)ch * 3 * b.ntot + i;
            g[0] = (double)ax.s + (double)ax.c;
            g[b.ntot] = (double)ay.s + (double)ay.c;
            g[2 * b.ntot] = (double)az.s + (double)az.c;
            return;
        }
        const long long io = (long long)b.perm[i] - ps.base;
        const double minv = ps.uniform_m ? ps.inv_m_uniform : 1.0 / ps.m[io];
        const double Gm = ps.ph.G * minv;
        ps.ax[io] += Gm * ((double)ax.s + (double)ax.c);
        ps.ay[io] += Gm * ((double)ay.s + (double)ay.c);
        ps.az[io] += Gm * ((double)az.s + (double)az.c);
    };
    if (i0 < end) store(i0, a0x, a0y, a0z);
    if (i1 < end) store(i1, a1x, a1y, a1z);
}

// Sum the partials of split problems in range order: a_i += G/m_i sum_ch F_i,ch.
template <typename T>
__global__ void __launch_bounds__(256) k_gravity_reduce(BatchView b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.ntot) return;
    if (b.block_on && ((const T *)b.slev)[i] < T(0)) return;  // block step: not this particle's force pass
    int p = 0;  // problem of particle i: the last one whose base is <= i
    for (int lo = 0, hi = b.nprob - 1; lo <= hi;) {
        const int mid = (lo + hi) >> 1;
        if (b.prob_base[mid] <= i) {
            p = mid;
            lo = mid + 1;
        } else {
            hi = mid - 1;
        }
    }
    const ProbStatic &ps = b.prob[p];
    if (!ps.ph.gravity || ps.gchunks <= 1) return;
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int ch = 0; ch < ps.gchunks; ++ch) {
        const double *g = b.gpart + (long long)ch * 3 * b.ntot + i;
        fx += g[0];
        fy += g[b.ntot];
        fz += g[2 * b.ntot];
    }
    const long long io = (long long)b.perm[i] - ps.base;
    const double Gm = ps.ph.G * (ps.uniform_m ? ps.inv_m_uniform : 1.0 / ps.m[io]);
    ps.ax[io] += Gm * fx;
    ps.ay[io] += Gm * fy;
    ps.az[io] += Gm * fz;
}

// ---------------------------------------------------------------------------
// Gravity tree walk (Sec. 4.2) over the leaves and 32-ary nodes the pair
// kernels use.  Each node carries its mass, centre of mass (relative to the
// key-domain corner), quadrupole Q_ab = sum m (3 d_a d_b - |d|^2 delta_ab)
// about the centre of mass, particle box, h_max and l^2, l the distance from
// the centre of mass to the box's farthest corner.  Moments are formed in FP64
// (leaves from the sorted particles, nodes bottom-up from their children by
// the parallel-axis shift) and stored in the staging precision; boxes are
// rounded outwards.
// ---------------------------------------------------------------------------
constexpr int kTreeThreads = 128;
constexpr int kTreeStage = 128;  // partner particles staged per warp at once

__device__ __forceinline__ float4 ldcg4(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ dbl4 ldcg4(const dbl4 *p)
{
    const double2 *q = reinterpret_cast<const double2 *>(p);
    const double2 a = __ldcg(q), c = __ldcg(q + 1);
    dbl4 r;
    r.x = a.x;
    r.y = a.y;
    r.z = c.x;
    r.w = c.y;
    return r;
}

__device__ __forceinline__ float rd_t(double v, float) { return __double2float_rd(v); }
__device__ __forceinline__ float ru_t(double v, float) { return __double2float_ru(v); }
__device__ __forceinline__ double rd_t(double v, double) { return v; }
__device__ __forceinline__ double ru_t(double v, double) { return v; }

template <typename V4>
__device__ __forceinline__ V4 mk4(double x, double y, double z, double w)
{
    V4 r;
    r.x = x;
    r.y = y;
    r.z = z;
    r.w = w;
    return r;
}

// Moments of one warp's set (one entry per lane; M = 0 where a lane holds
// nothing): centre of mass com, Q about it, box [lo, hi], h_max; written by
// lane 0 to node g.  `q` is the entry's own quadrupole about its own centre
// (zero for particles).
template <typename T>
__device__ void form_node(double M, const double (&x)[3], const double (&q)[6], const double (&lo)[3],
                          const double (&hi)[3], double hm, typename Vec4<T>::type *g)
{
    using V4 = typename Vec4<T>::type;
    const double Mt = warp_sum(M);
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = warp_sum(M * x[a]) / Mt;
    const double d[3] = {M > 0 ? x[0] - c[0] : 0.0, M > 0 ? x[1] - c[1] : 0.0, M > 0 ? x[2] - c[2] : 0.0};
    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double Q[6] = {warp_sum(q[0] + M * (3.0 * d[0] * d[0] - d2)), warp_sum(q[1] + M * (3.0 * d[0] * d[1])),
                         warp_sum(q[2] + M * (3.0 * d[0] * d[2])), warp_sum(q[3] + M * (3.0 * d[1] * d[1] - d2)),
                         warp_sum(q[4] + M * (3.0 * d[1] * d[2])), warp_sum(q[5] + M * (3.0 * d[2] * d[2] - d2))};
    double L[3], H[3];
    for (int a = 0; a < 3; ++a) {
        L[a] = warp_min(lo[a]);
        H[a] = warp_max(hi[a]);
    }
    const double hmax = warp_max(hm);
    double l2 = 0.0;  // farthest corner of the box from the centre of mass
    for (int a = 0; a < 3; ++a) {
        const double e = fmax(c[a] - L[a], H[a] - c[a]);
        l2 += e * e;
    }
    if ((threadIdx.x & 31) == 0) {
        const T t = T(0);
        g[0] = mk4<V4>(c[0], c[1], c[2], Mt);
        g[1] = mk4<V4>(Q[0], Q[1], Q[2], Q[3]);
        g[2] = mk4<V4>(Q[4], Q[5], ru_t(l2, t), ru_t(hmax, t));
        g[3] = mk4<V4>(rd_t(L[0], t), rd_t(L[1], t), rd_t(L[2], t), 0.0);
        g[4] = mk4<V4>(ru_t(H[0], t), ru_t(H[1], t), ru_t(H[2], t), 0.0);
    }
}

// The same over each group of four lanes (the level-1 node's leaves 4g ..
// 4g+3 in lanes 4g .. 4g+3): lane 4g writes group g to g_base + 5 g; empty
// groups (no mass) are written with M = 0 and are never visited.
template <typename T>
__device__ void form_groups(double M, const double (&x)[3], const double (&q)[6], const double (&lo)[3],
                            const double (&hi)[3], double hm, typename Vec4<T>::type *g_base)
{
    using V4 = typename Vec4<T>::type;
    auto gsum = [](double v) {
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        return v + __shfl_xor_sync(0xffffffffu, v, 2);
    };
    auto gmin = [](double v) {
        v = fmin(v, __shfl_xor_sync(0xffffffffu, v, 1));
        return fmin(v, __shfl_xor_sync(0xffffffffu, v, 2));
    };
    auto gmax = [](double v) {
        v = fmax(v, __shfl_xor_sync(0xffffffffu, v, 1));
        return fmax(v, __shfl_xor_sync(0xffffffffu, v, 2));
    };
    const double Mt = gsum(M);
    double c[3];
    for (int a = 0; a < 3; ++a) {
        const double s = gsum(M * x[a]);
        c[a] = Mt > 0 ? s / Mt : 0.0;
    }
    const double d[3] = {M > 0 ? x[0] - c[0] : 0.0, M > 0 ? x[1] - c[1] : 0.0, M > 0 ? x[2] - c[2] : 0.0};
    const double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double Q[6] = {gsum(q[0] + M * (3.0 * d[0] * d[0] - d2)), gsum(q[1] + M * (3.0 * d[0] * d[1])),
                         gsum(q[2] + M * (3.0 * d[0] * d[2])), gsum(q[3] + M * (3.0 * d[1] * d[1] - d2)),
                         gsum(q[4] + M * (3.0 * d[1] * d[2])), gsum(q[5] + M * (3.0 * d[2] * d[2] - d2))};
    double L[3], H[3];
    for (int a = 0; a < 3; ++a) {
        L[a] = gmin(lo[a]);
        H[a] = gmax(hi[a]);
    }
    const double hmax = gmax(hm);
    double l2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double e = Mt > 0 ? fmax(c[a] - L[a], H[a] - c[a]) : 0.0;
        l2 += e * e;
    }
    const int lane = threadIdx.x & 31;
    if ((lane & 3) == 0) {
        const T t = T(0);
        V4 *g = g_base + 5 * (lane >> 2);
        g[0] = mk4<V4>(c[0], c[1], c[2], Mt);
        g[1] = mk4<V4>(Q[0], Q[1], Q[2], Q[3]);
        g[2] = mk4<V4>(Q[4], Q[5], ru_t(l2, t), ru_t(hmax, t));
        g[3] = mk4<V4>(rd_t(Mt > 0 ? L[0] : 0.0, t), rd_t(Mt > 0 ? L[1] : 0.0, t), rd_t(Mt > 0 ? L[2] : 0.0, t), 0.0);
        g[4] = mk4<V4>(ru_t(Mt > 0 ? H[0] : 0.0, t), ru_t(Mt > 0 ? H[1] : 0.0, t), ru_t(Mt > 0 ? H[2] : 0.0, t), 0.0);
    }
}

// Leaf moments from the sorted FP64 particles, then the nodes above: the warp
// whose arrival completes a node's children forms it (the arrival counters
// are the tree build's, zero between kernels, and are cleared again here).
template <typename T>
__global__ void __launch_bounds__(256) k_grav_moments(BatchView b)
{
    using V4 = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w0; leaf < nleaf; leaf += nw) {
        const int p = b.leaf_pid[leaf];
        const ProbStatic &ps = b.prob[p];
        if (!(ps.ph.gravity && ps.ph.grav_theta > 0)) continue;
        const ProbDyn &d = b.dyn[p];
        const int st = b.leaf_start[leaf], cnt = b.leaf_start[leaf + 1] - st;
        double M = 0.0, x[3] = {0.0, 0.0, 0.0}, lo[3], hi[3], hm = 0.0;
        const double q0[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        if (lane < cnt) {
            const int i = st + lane;
            x[0] = b.sx[i] - d.dom_lo[0];
            x[1] = b.sy[i] - d.dom_lo[1];
            x[2] = b.sz[i] - d.dom_lo[2];
            M = b.sm[i];
            hm = b.sh[i];
            for (int a = 0; a < 3; ++a) lo[a] = hi[a] = x[a];
            // the walk's copy of the particle in the staging precision
            using P = typename GravVec<T>::P;
            using H = typename GravVec<T>::H;
            P e;
            H f;
            e.x = (T)x[0];
            e.y = (T)x[1];
            e.z = (T)x[2];
            e.w = (T)M;
            f.x = (T)hm;
            f.y = T(1) / f.x;
            ((P *)b.gpos)[i] = e;
            ((H *)b.gh)[i] = f;
        } else {
            for (int a = 0; a < 3; ++a) {
                lo[a] = INFINITY;
                hi[a] = -INFINITY;
            }
        }
        form_node<T>(M, x, q0, lo, hi, hm, (V4 *)b.gnode[0] + 5LL * leaf);
        // upwards
        int k = leaf - d.node_off[0];
        for (int lvl = 0; lvl < d.top_level; ++lvl) {
            const int parent = k / kBranch;
            const int nch = min(kBranch, d.node_cnt[lvl] - parent * kBranch);
            int *ctr = b.node_ctr[lvl + 1] + d.node_off[lvl + 1] + parent;
            int old = 0;
            if (lane == 0) {
                __threadfence();  // this warp's node before its arrival
                old = atomicAdd(ctr, 1);
            }
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old != nch - 1) break;
            if (lane == 0) *ctr = 0;
            __threadfence();
            double Mc = 0.0, xc[3] = {0.0, 0.0, 0.0}, qc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, lc[3], hc[3], hmc = 0.0;
            if (lane < nch) {
                const V4 *g = (const V4 *)b.gnode[lvl] + 5LL * (d.node_off[lvl] + parent * kBranch + lane);
                const V4 A = ldcg4(g), B = ldcg4(g + 1), C = ldcg4(g + 2), L = ldcg4(g + 3), H = ldcg4(g + 4);
                Mc = A.w;
                xc[0] = A.x;
                xc[1] = A.y;
                xc[2] = A.z;
                qc[0] = B.x;
                qc[1] = B.y;
                qc[2] = B.z;
                qc[3] = B.w;
                qc[4] = C.x;
                qc[5] = C.y;
                hmc = C.w;
                lc[0] = L.x;
                lc[1] = L.y;
                lc[2] = L.z;
                hc[0] = H.x;
                hc[1] = H.y;
                hc[2] = H.z;
            } else {
                for (int a = 0; a < 3; ++a) {
                    lc[a] = INFINITY;
                    hc[a] = -INFINITY;
                }
            }
            if (lvl == 0)  // a level-1 node: also its groups of four leaves
                form_groups<T>(Mc, xc, qc, lc, hc, hmc, (V4 *)b.ggrp + 40LL * (d.node_off[1] + parent));
            form_node<T>(Mc, xc, qc, lc, hc, hmc, (V4 *)b.gnode[lvl + 1] + 5LL * (d.node_off[lvl + 1] + parent));
            k = parent;
        }
    }
}

// Acceleration (per unit G) at offset r from a node's centre of mass:
// -M r/|r|^3 + Q r/|r|^5 - (5/2)(r.Q.r) r/|r|^7, added to plain sums (the
// expansion's own error, ~theta^3, is far above their rounding).
template <typename T>
__device__ __forceinline__ void multipole_acc(T rx, T ry, T rz, T M, const T (&Q)[6], T &ax, T &ay, T &az)
{
    const T r2 = rx * rx + ry * ry + rz * rz;
    const T rinv = rsqrt_t(r2), rinv2 = rinv * rinv, rinv3 = rinv2 * rinv, rinv5 = rinv3 * rinv2;
    const T qx = Q[0] * rx + Q[1] * ry + Q[2] * rz;
    const T qy = Q[1] * rx + Q[3] * ry + Q[4] * rz;
    const T qz = Q[2] * rx + Q[4] * ry + Q[5] * rz;
    const T rqr = rx * qx + ry * qy + rz * qz;
    const T k = -M * rinv3 - T(2.5) * rqr * rinv5 * rinv2;
    ax += k * rx + qx * rinv5;
    ay += k * ry + qy * rinv5;
    az += k * rz + qz * rinv5;
}

// One warp per leaf of a problem with grav_theta > 0.  The walk classifies the
// children of each visited node, one per lane: used through its multipole
// (the opening criterion holds for the whole leaf box and no pair with it is
// softened), opened, or absent.  Used nodes and the particles of opened
// leaves are staged in shared memory and summed at once; with several lanes
// per particle each lane takes every lpp-th staged entry and the lanes'
// sums are added in a fixed order at the end.
template <typename T>
__global__ void __launch_bounds__(kTreeThreads) k_gravity_tree(BatchView b)
{
    using V4 = typename Vec4<T>::type;
    using P = typename GravVec<T>::P;
    using H = typename GravVec<T>::H;
    constexpr int kW = kTreeThreads / 32;
    __shared__ P s_p[kW][kTreeStage];  // partner (x, m) or node (com, M)
    __shared__ H s_h[kW][kTreeStage];  // partner (h, 1/h)
    __shared__ T s_q[kW][32][6];       // node Q
    __shared__ int s_off[kW][32], s_st[kW][32];  // opened leaves: first staged entry, first particle
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    // the walk's query: a leaf (its box the opening criterion's), or in a
    // block-step tick a task of the particles whose step ends (up to S =
    // 32 / block_lanes of a leaf, their own box), so that the few queries
    // of a tick walk in short, parallel pieces.  (For a whole step the
    // leaves are faster: the multipole terms per particle hardly fall with
    // the smaller boxes, and the walks multiply.)
    const bool blk = b.block_on && b.block_tasks;
    const int nitem = blk ? b.counters[kBlockTasks] : b.counters[0];
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int item = w0; item < nitem; item += nw) {
        int leaf = item, k0 = 0;
        if (blk) {
            const int t = b.btask[item];
            leaf = t >> 5;
            k0 = t & 31;
        }
        const int p = b.leaf_pid[leaf];
        const ProbStatic &ps = b.prob[p];
        if (!(ps.ph.gravity && ps.ph.grav_theta > 0)) continue;
        const ProbDyn &d = b.dyn[p];
        const int lpp = blk ? b.block_lanes : ps.lpp, S = kBranch / lpp;
        const int pi = lane % S, sub = lane / S;
        const int st = b.leaf_start[leaf], cnt_leaf = b.leaf_start[leaf + 1] - st;
        // the particles of the leaf that take the long range now (block
        // step: those whose step ends), and this task's share of them
        const unsigned dm = __ballot_sync(0xffffffffu, lane < cnt_leaf &&
                                          (!b.block_on || ((const T *)b.slev)[st + (lane < cnt_leaf ? lane : 0)] > T(0)));
        const int nd = __popc(dm), cnt = min(S, max(nd - k0, 0));
        const bool due = pi < cnt;
        if (!__any_sync(0xffffffffu, due)) continue;
        const int pos = due ? (int)__fns(dm, 0u, k0 + pi + 1) : 0;
        // this lane's particle (lanes beyond the task take its first)
        const P e = ((const P *)b.gpos)[st + (due ? pos : (int)__fns(dm, 0u, k0 + 1))];
        const H f = ((const H *)b.gh)[st + (due ? pos : (int)__fns(dm, 0u, k0 + 1))];
        const T xi = e.x, yi = e.y, zi = e.z, hi = f.x, hinv = f.y;
        // the query's box and largest h: the leaf's, or the task's
        T blo[3], bhi[3], hleaf;
        if (blk) {
            blo[0] = warp_min(xi);
            blo[1] = warp_min(yi);
            blo[2] = warp_min(zi);
            bhi[0] = warp_max(xi);
            bhi[1] = warp_max(yi);
            bhi[2] = warp_max(zi);
            hleaf = warp_max(hi);
        } else {
            const V4 *gl = (const V4 *)b.gnode[0] + 5LL * leaf;
            const V4 GL = gl[3], GH = gl[4];
            blo[0] = GL.x;
            blo[1] = GL.y;
            blo[2] = GL.z;
            bhi[0] = GH.x;
            bhi[1] = GH.y;
            bhi[2] = GH.z;
            hleaf = gl[2].w;
        }
        long long npair = 0, nnode = 0;  // terms this lane summed
        const T th2 = (T)(ps.ph.grav_theta * ps.ph.grav_theta);
        TwoSumAcc<T> ax{T(0), T(0)}, ay{T(0), T(0)}, az{T(0), T(0)};  // pair terms
        T mx = T(0), my = T(0), mz = T(0);                              // multipole terms
        // classify node g of level `lvl`, stage it when it is used; returns 1 used, 2 opened
        auto visit = [&](const V4 *nodes, int count, unsigned filter) -> unsigned {
            int cls = 0;
            V4 A, B, C;
            if (lane < count && ((filter >> lane) & 1u)) {
                const V4 *g = nodes + 5LL * lane;
                A = g[0];
                B = g[1];
                C = g[2];
                const V4 L = g[3], U = g[4];
                const T cm[3] = {A.x, A.y, A.z}, nl[3] = {L.x, L.y, L.z}, nh[3] = {U.x, U.y, U.z};
                T d2 = T(0), g2 = T(0);
                for (int a = 0; a < 3; ++a) {
                    const T da = fmax(fmax(blo[a] - cm[a], cm[a] - bhi[a]), T(0));
                    const T ga = fmax(fmax(nl[a] - bhi[a], blo[a] - nh[a]), T(0));
                    d2 += da * da;
                    g2 += ga * ga;
                }
                const T soft = T(2) * fmax(hleaf, C.w);
                cls = (th2 > T(0) && d2 * th2 >= C.z && g2 >= soft * soft) ? 1 : 2;
            }
            const unsigned um = __ballot_sync(0xffffffffu, cls == 1);
            if (um) {  // sum the used nodes
                if (cls == 1) {
                    const int slot = __popc(um & ((1u << lane) - 1u));
                    P e;
                    e.x = A.x;
                    e.y = A.y;
                    e.z = A.z;
                    e.w = A.w;
                    s_p[wi][slot] = e;
                    s_q[wi][slot][0] = B.x;
                    s_q[wi][slot][1] = B.y;
                    s_q[wi][slot][2] = B.z;
                    s_q[wi][slot][3] = B.w;
                    s_q[wi][slot][4] = C.x;
                    s_q[wi][slot][5] = C.y;
                }
                __syncwarp();
                const int nu = __popc(um);
                if (pi < cnt) nnode += (nu - sub + lpp - 1) / lpp;
                for (int e = sub; e < nu; e += lpp) {
                    const P q = s_p[wi][e];
                    const T Q[6] = {s_q[wi][e][0], s_q[wi][e][1], s_q[wi][e][2],
                                    s_q[wi][e][3], s_q[wi][e][4], s_q[wi][e][5]};
                    multipole_acc(xi - q.x, yi - q.y, zi - q.z, q.w, Q, mx, my, mz);
                }
                __syncwarp();
            }
            return __ballot_sync(0xffffffffu, cls == 2);
        };
        // sum the particles of the opened leaves first + bits of om pair by
        // pair, staged kTreeStage at a time across leaves
        auto direct = [&](unsigned om, int first) {
            if (!om) return;
            const bool op = (om >> lane) & 1u;
            const int ls = op ? b.leaf_start[first + lane] : 0;
            const int lc = op ? b.leaf_start[first + lane + 1] - ls : 0;
            const int inc = warp_incl_scan<int>(lc);
            const int total = __shfl_sync(0xffffffffu, inc, 31);
            s_off[wi][lane] = inc - lc;
            s_st[wi][lane] = ls;
            __syncwarp();
            for (int cb = 0; cb < total; cb += kTreeStage) {
                const int nst = min(kTreeStage, total - cb);
                for (int e = lane; e < nst; e += 32) {
                    const int f = cb + e;
                    int lo = 0, hi2 = 31;  // last opened leaf whose first entry is <= f
                    while (lo < hi2) {
                        const int mid = (lo + hi2 + 1) >> 1;
                        if (s_off[wi][mid] <= f) lo = mid;
                        else hi2 = mid - 1;
                    }
                    const int j = s_st[wi][lo] + (f - s_off[wi][lo]);
                    s_p[wi][e] = ((const P *)b.gpos)[j];
                    s_h[wi][e] = ((const H *)b.gh)[j];
                }
                __syncwarp();
                if (pi < cnt) npair += (nst - sub + lpp - 1) / lpp;
                for (int e = sub; e < nst; e += lpp) grav_pair(xi, yi, zi, T(1), hi, hinv, s_p[wi][e], s_h[wi][e], ax, ay, az);
                __syncwarp();
            }
        };
        const int top = d.top_level;
        unsigned mask[kMaxLevels + 1];
        int base[kMaxLevels + 1];
        {
            const unsigned om = visit((const V4 *)b.gnode[top] + 5LL * d.node_off[top], d.node_cnt[top], ~0u);
            if (top == 0) direct(om, d.node_off[0]);
            mask[top] = om;
            base[top] = 0;
        }
        int lvl = top;
        while (top > 0) {
            const unsigned m = mask[lvl];
            if (m == 0u) {
                if (++lvl > top) break;
                continue;
            }
            const int c = __ffs(m) - 1;
            mask[lvl] = m & (m - 1u);
            const int node = base[lvl] + c;
            const int cnt_ch = min(kBranch, d.node_cnt[lvl - 1] - node * kBranch);
            if (lvl == 1) {
                // a level-1 node's leaves: its groups of four first (used
                // whole where the criterion allows), then the leaves of the
                // groups it opens
                const unsigned og = visit((const V4 *)b.ggrp + 40LL * (d.node_off[1] + node), (cnt_ch + 3) >> 2, ~0u);
                unsigned lf = 0u;
                for (unsigned m = og; m; m &= m - 1u) lf |= 0xfu << (4 * (__ffs(m) - 1));
                const unsigned om =
                    lf ? visit((const V4 *)b.gnode[0] + 5LL * (d.node_off[0] + node * kBranch), cnt_ch, lf) : 0u;
                direct(om, d.node_off[0] + node * kBranch);
                continue;
            }
            const unsigned om = visit((const V4 *)b.gnode[lvl - 1] + 5LL * (d.node_off[lvl - 1] + node * kBranch), cnt_ch, ~0u);
            --lvl;
            base[lvl] = node * kBranch;
            mask[lvl] = om;
        }
        // the lanes of each particle add their sums in a fixed order
        double gx = (double)ax.s + (double)ax.c + (double)mx, gy = (double)ay.s + (double)ay.c + (double)my,
               gz = (double)az.s + (double)az.c + (double)mz;
        for (int o = S; o < kBranch; o <<= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if (sub == 0 && due) {
            const long long io = (long long)b.perm[st + pos] - ps.base;
            ps.ax[io] += ps.ph.G * gx;
            ps.ay[io] += ps.ph.G * gy;
            ps.az[io] += ps.ph.G * gz;
        }
        // self pairs (r = 0) add nothing and are not counted
        npair = warp_sum(npair) - cnt;
        nnode = warp_sum(nnode);
        if (lane == 0) {
            atomicAdd((unsigned long long *)&ps.diag->grav_pairs, (unsigned long long)npair);
            atomicAdd((unsigned long long *)&ps.diag->grav_nodes, (unsigned long long)nnode);
        }
    }
}

// Acceleration condition of Eq. SPH_DTACCEL for the problems with gravity,
// once the long-range part has been added: dt_i = c_grav sqrt(h_i / |a_i|)
// joins the CFL minimum of the force pass.
__global__ void __launch_bounds__(256) k_grav_dt(BatchView b)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int p = -1;
    double dt = INFINITY;
    if (g < b.ntot) {
        p = find_problem(b.prob_base, b.nprob, g);
        const ProbStatic &ps = b.prob[p];
        if (ps.ph.gravity) {
            const long long i = g - ps.base;
            const double a2 = ps.ax[i] * ps.ax[i] + ps.ay[i] * ps.ay[i] + ps.az[i] * ps.az[i];
            if (a2 > 0) dt = ps.ph.c_grav * sqrt(ps.h[i] / sqrt(a2));
        }
    }
    // one atomic per warp when the warp lies in one problem
    const int p0 = __shfl_sync(0xffffffffu, p, 0);
    if (__all_sync(0xffffffffu, p == p0)) {
        dt = warp_min(dt);
        if ((threadIdx.x & 31) == 0 && p0 >= 0 && dt < INFINITY)
            atomicMin(&b.prob[p0].diag->dt_min_bits, (unsigned long long)__double_as_longlong(dt));
    } else if (p >= 0 && dt < INFINITY) {
        atomicMin(&b.prob[p].diag->dt_min_bits, (unsigned long long)__double_as_longlong(dt));
    }
}

}  // namespace

// C partner ranges for N particles: enough blocks to fill the GPU (about 8 per
// SM), at most 16 ranges and at least 4096 partners per range.
int gravity_chunks(long long n, double theta)
{
    if (theta > 0) return 0;  // the tree walk serves this problem
    const long long ib = (n + 2 * kGravThreads - 1) / (2 * kGravThreads);
    long long c = ib > 0 ? (1216 + ib - 1) / ib : 1;
    if (c > 16) c = 16;
    if (c > n / 4096) c = n / 4096;
    return c < 1 ? 1 : (int)c;
}

long long gravity_blocks(long long n, double theta)
{
    return (n + 2 * kGravThreads - 1) / (2 * kGravThreads) * gravity_chunks(n, theta);
}

void launch_gravity(const BatchView &b, int precision, cudaStream_t st)
{
    if (!b.any_gravity) return;
    if (b.grav_blocks > 0) {
        if (precision == SPH_PREC_FP64) k_gravity<double><<<(unsigned)b.grav_blocks, kGravThreads, 0, st>>>(b);
        else k_gravity<float><<<(unsigned)b.grav_blocks, kGravThreads, 0, st>>>(b);
    }
    if (b.grav_split) {
        if (precision == SPH_PREC_FP64) k_gravity_reduce<double><<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b);
        else k_gravity_reduce<float><<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b);
    }
    if (b.any_grav_tree) {
        static int sms = 0;
        if (!sms) sms = dev_info().sm_count;
        if (precision == SPH_PREC_FP64) {
            k_grav_moments<double><<<sms * 8, 256, 0, st>>>(b);
            k_gravity_tree<double><<<sms * 8, kTreeThreads, 0, st>>>(b);
        } else {
            k_grav_moments<float><<<sms * 8, 256, 0, st>>>(b);
            k_gravity_tree<float><<<sms * 8, kTreeThreads, 0, st>>>(b);
        }
    }
    if (b.ntot > 0) k_grav_dt<<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b);
}

}  // namespace sph
