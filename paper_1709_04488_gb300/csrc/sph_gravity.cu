// Self-gravity, long-range part of Eq. SPHSELFGRAV (Sec. 2.1.2): the
// kernel-softened attraction
//   g_i = -G sum_{j != i} m_j (phi'(r_ij,h_i) + phi'(r_ij,h_j))/2 r_hat_ij,
// phi'(r,h) = M(r/h)/r^2 (Eq. GRAVFORCEKERNEL), by direct summation over every
// particle of the problem.  The zeta term of the same equation runs in the
// force pass with the neighbours.
//
// One thread per particle, sorted order; the blocks of a problem cover only
// that problem's particles (each problem's first block is precomputed on the
// host), and the partner particles stream through shared memory in tiles.
// Positions are taken relative to the problem's key-domain corner in FP64 and
// cast, like the leaf offsets of the pair kernels.  Each pair term is formed
// from the same staged values on both sides with explicit rounding, so
// F_ij = -F_ji bit for bit, and F_i is accumulated with TwoSum; a_i = G F_i / m_i
// in FP64 is added to the accelerations the force pass wrote.
#include "sph_pairs.cuh"

namespace sph {

namespace {

constexpr int kGravThreads = 256;

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

template <typename T>
__global__ void __launch_bounds__(kGravThreads) k_gravity(BatchView b)
{
    __shared__ T tx[kGravThreads], ty[kGravThreads], tz[kGravThreads], tm[kGravThreads], th[kGravThreads],
        thv[kGravThreads];
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
    const long long base = b.prob_base[p], n = ps.n;
    const long long i = base + (long long)(blockIdx.x - ps.gblk0) * kGravThreads + threadIdx.x;
    const bool on = i < base + n;
    const double *ref = b.dyn[p].dom_lo;
    T xi = T(0), yi = T(0), zi = T(0), mi = T(0), hinv_i = T(1), hi = T(1);
    if (on) {
        xi = (T)(b.sx[i] - ref[0]);
        yi = (T)(b.sy[i] - ref[1]);
        zi = (T)(b.sz[i] - ref[2]);
        mi = (T)b.sm[i];
        hi = (T)b.sh[i];
        hinv_i = T(1) / hi;
    }
    TwoSumAcc<T> ax{T(0), T(0)}, ay{T(0), T(0)}, az{T(0), T(0)};
    for (long long j0 = 0; j0 < n; j0 += kGravThreads) {
        __syncthreads();  // the previous tile is consumed
        const long long j = base + j0 + threadIdx.x;
        if (j < base + n) {
            tx[threadIdx.x] = (T)(b.sx[j] - ref[0]);
            ty[threadIdx.x] = (T)(b.sy[j] - ref[1]);
            tz[threadIdx.x] = (T)(b.sz[j] - ref[2]);
            tm[threadIdx.x] = (T)b.sm[j];
            th[threadIdx.x] = (T)b.sh[j];
            thv[threadIdx.x] = T(1) / (T)b.sh[j];  // the same 1/h the particle's own thread forms
        }
        __syncthreads();
        const int jn = (int)(n - j0 < kGravThreads ? n - j0 : kGravThreads);
        if (!on) continue;
        const int self = (int)(i - base - j0);  // this particle's slot in the tile, if there
#pragma unroll 4
        for (int k = 0; k < jn; ++k) {
            if (k == self) continue;
            const T rx = sub_rn(xi, tx[k]), ry = sub_rn(yi, ty[k]), rz = sub_rn(zi, tz[k]);
            const T r2 = fma_rn(rz, rz, fma_rn(ry, ry, mul_rn(rx, rx)));
            const T rinv = rsqrt_t(r2);
            const T rinv2 = mul_rn(rinv, rinv);
            const T hj = th[k];
            const T r = mul_rn(r2, rinv);
            // mean force kernel of the pair: 1/r^2 beyond both supports
            T fbar = rinv2;
            if (r < T(2) * (hi > hj ? hi : hj))
                fbar = mul_rn(mul_rn(T(0.5), add_rn(grav_mass_rn(mul_rn(r, hinv_i)), grav_mass_rn(mul_rn(r, thv[k])))),
                              rinv2);
            const T w = mul_rn(mul_rn(mul_rn(mi, tm[k]), fbar), rinv);  // symmetric in (i, j)
            ax.add(-mul_rn(w, rx));
            ay.add(-mul_rn(w, ry));
            az.add(-mul_rn(w, rz));
        }
    }
    if (!on) return;
    const long long g = b.perm[i];
    const long long io = g - ps.base;
    const double minv = ps.uniform_m ? ps.inv_m_uniform : 1.0 / ps.m[io];
    const double Gm = ps.ph.G * minv;
    ps.ax[io] += Gm * ((double)ax.s + (double)ax.c);
    ps.ay[io] += Gm * ((double)ay.s + (double)ay.c);
    ps.az[io] += Gm * ((double)az.s + (double)az.c);
}

}  // namespace

long long gravity_blocks(long long n) { return (n + kGravThreads - 1) / kGravThreads; }

void launch_gravity(const BatchView &b, int precision, cudaStream_t st)
{
    if (!b.any_gravity || b.grav_blocks <= 0) return;
    if (precision == SPH_PREC_FP64) k_gravity<double><<<(unsigned)b.grav_blocks, kGravThreads, 0, st>>>(b);
    else k_gravity<float><<<(unsigned)b.grav_blocks, kGravThreads, 0, st>>>(b);
}

}  // namespace sph
