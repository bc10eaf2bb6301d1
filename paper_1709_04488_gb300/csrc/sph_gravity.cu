// Self-gravity, long-range part of Eq. SPHSELFGRAV (Sec. 2.1.2): the
// kernel-softened attraction
//   g_i = -G sum_{j != i} m_j (phi'(r_ij,h_i) + phi'(r_ij,h_j))/2 r_hat_ij,
// phi'(r,h) = M(r/h)/r^2 (Eq. GRAVFORCEKERNEL), by direct summation over every
// particle of the problem.  The zeta term of the same equation runs in the
// force pass with the neighbours.
//
// Two particles per thread, sorted order; the blocks of a problem cover only
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
__global__ void __launch_bounds__(256) k_gravity_reduce(BatchView b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.ntot) return;
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

}  // namespace

// C partner ranges for N particles: enough blocks to fill the GPU (about 8 per
// SM), at most 16 ranges and at least 4096 partners per range.
int gravity_chunks(long long n)
{
    const long long ib = (n + 2 * kGravThreads - 1) / (2 * kGravThreads);
    long long c = ib > 0 ? (1216 + ib - 1) / ib : 1;
    if (c > 16) c = 16;
    if (c > n / 4096) c = n / 4096;
    return c < 1 ? 1 : (int)c;
}

long long gravity_blocks(long long n)
{
    return (n + 2 * kGravThreads - 1) / (2 * kGravThreads) * gravity_chunks(n);
}

void launch_gravity(const BatchView &b, int precision, cudaStream_t st)
{
    if (!b.any_gravity || b.grav_blocks <= 0) return;
    if (precision == SPH_PREC_FP64) k_gravity<double><<<(unsigned)b.grav_blocks, kGravThreads, 0, st>>>(b);
    else k_gravity<float><<<(unsigned)b.grav_blocks, kGravThreads, 0, st>>>(b);
    if (b.grav_split)
        k_gravity_reduce<<<(unsigned)((b.ntot + 255) / 256), 256, 0, st>>>(b);
}

}  // namespace sph
