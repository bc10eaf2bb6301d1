// Pair kernels of the grad-h SPH neighbour loop.
//
// Work unit: one warp per leaf cell (the paper's OpenMP unit of work is an
// active leaf cell, Sec. 5.2.1, and neighbours are gathered per leaf, not per
// particle, Sec. 4.2).  LPP lanes serve each particle of the leaf; the warp
// walks the tree over the leaves once per leaf, stages candidate particles in
// shared memory (positions relative to the query leaf: leaf reference points
// differenced in FP64, then cast), and each lane keeps its own list of
// in-range candidates so that the arithmetic runs without divergence.
//
//  k_density   Eqs. SPHRHO, HRHO, OMEGA: Newton-Raphson on
//              F(h) = rho(h) - m (eta/h)^3 over the cached list of (r, m_j)
//              with the same bracketing fallback as the oracle; the list is
//              rebuilt if h outgrows it.  Particles whose list overflows, or
//              that need too many rebuilds, go to k_density_fallback, which
//              re-walks the tree in every iteration.
//  k_forces    Eqs. GRADHMOMEQN, GRADHENEQN, MON97ARTVISC, MON97ENERGYDISS
//              and the signal speed of Eq. SPH_DT.  Every pair term is formed
//              from an exactly antisymmetric pair vector with order-independent
//              FP32 operations, so that F_ij = -F_ji bit for bit; m_i a_i is
//              accumulated with
//              error-free (TwoSum) compensated FP32 sums combined in FP64,
//              which keeps sum_i m_i a_i near FP64 round-off.
#include "sph_internal.cuh"
#include "sph_tuned.h"

namespace sph {

namespace {

constexpr unsigned FULL = 0xffffffffu;
__host__ __device__ constexpr int lpp_log2(int l) { return l == 1 ? 0 : l == 2 ? 1 : l == 4 ? 2 : 3; }
constexpr double kListMargin = 1.03;  // list radius = 2 h * margin

constexpr int kMaxRebuild = 6;

template <typename T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ float tinf<float>() { return INFINITY; }
template <>
__device__ __forceinline__ double tinf<double>() { return INFINITY; }

// M4 cubic spline: f(q) and f'(q), support q < 2 (W = f / (pi h^3)).
template <typename T>
__device__ __forceinline__ void m4(T q, T &f, T &df)
{
    T t = q < T(2) ? T(2) - q : T(0);
    T t2 = t * t;
    T f2 = T(0.25) * t2 * t, df2 = T(-0.75) * t2;
    T q2 = q * q;
    T f1 = T(1) + q2 * (T(0.75) * q - T(1.5));
    T df1 = q * (T(2.25) * q - T(3));
    bool in = q < T(1);
    f = in ? f1 : f2;
    df = in ? df1 : df2;
}

template <typename T>
__device__ __forceinline__ T m4_df(T q)
{
    T t = q < T(2) ? T(2) - q : T(0);
    T df2 = T(-0.75) * t * t;
    T df1 = q * (T(2.25) * q - T(3));
    return q < T(1) ? df1 : df2;
}

template <typename T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <typename T>
__device__ __forceinline__ T mul_rn(T a, T b);
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T>
__device__ __forceinline__ T add_rn(T a, T b);
template <>
__device__ __forceinline__ float add_rn<float>(float a, float b) { return __fadd_rn(a, b); }
template <>
__device__ __forceinline__ double add_rn<double>(double a, double b) { return __dadd_rn(a, b); }

// 2/(rho_i + rho_j): a deterministic function of the commutative sum, so
// both sides of a pair get the same bits (fast reciprocal in FP32)
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

__device__ __forceinline__ float to_float_ru(float v) { return v; }
__device__ __forceinline__ float to_float_ru(double v) { return __double2float_ru(v); }

// sorted particle index carried in the w slot of a staged vector: bit
// pattern in FP32 staging (only ever copied), exact value in FP64 staging
__device__ __forceinline__ float bits_as_t(int v, float) { return __int_as_float(v); }
__device__ __forceinline__ double bits_as_t(int v, double) { return (double)v; }
__device__ __forceinline__ int t_as_bits(float v) { return __float_as_int(v); }
__device__ __forceinline__ int t_as_bits(double v) { return (int)v; }

// Separating-axis test of two boxes grown by R, periodic aware, conservative
// for the FP32 rounding of the box coordinates.
__device__ __forceinline__ bool axis_overlap(float alo, float ahi, float blo, float bhi, float R,
                                             int periodic, float L)
{
    float ca = 0.5f * (alo + ahi), ha = 0.5f * (ahi - alo);
    float cb = 0.5f * (blo + bhi), hb = 0.5f * (bhi - blo);
    float reach = ha + hb + R;
    reach += 2e-6f * (fabsf(ca) + fabsf(cb) + reach) + 1e-30f;
    float d = fabsf(ca - cb);
    if (periodic) {
        if (reach >= 0.5f * L) return true;
        if (d > L) d -= L;
        d = fminf(d, L - d);
    }
    return d <= reach;
}

__device__ __forceinline__ bool box_overlap(const float4 &alo, const float4 &ahi, const float4 &blo,
                                            const float4 &bhi, float R, const PhysParams &ph)
{
    return axis_overlap(alo.x, ahi.x, blo.x, bhi.x, R, ph.periodic, ph.box_len_f[0]) &&
           axis_overlap(alo.y, ahi.y, blo.y, bhi.y, R, ph.periodic, ph.box_len_f[1]) &&
           axis_overlap(alo.z, ahi.z, blo.z, bhi.z, R, ph.periodic, ph.box_len_f[2]);
}

// Gap between the two boxes' extents along one axis (minimum image if
// periodic), shrunk for the FP32 rounding of the box coordinates.
__device__ __forceinline__ float axis_gap(float alo, float ahi, float blo, float bhi, int periodic, float L)
{
    float ca = 0.5f * (alo + ahi), ha = 0.5f * (ahi - alo);
    float cb = 0.5f * (blo + bhi), hb = 0.5f * (bhi - blo);
    float reach = ha + hb;
    reach += 2e-6f * (fabsf(ca) + fabsf(cb) + reach) + 1e-30f;
    float d = fabsf(ca - cb);
    if (periodic) {
        if (reach >= 0.5f * L) return 0.f;
        if (d > L) d -= L;
        d = fminf(d, L - d);
    }
    return fmaxf(d - reach, 0.f);
}

// Do two boxes come within (Euclidean) distance R of each other?  Tighter
// than growing one box by R along each axis: the grown box's corners, where
// no point is within R, are left out.
__device__ __forceinline__ bool box_within(const float4 &alo, const float4 &ahi, const float4 &blo,
                                           const float4 &bhi, float R, const PhysParams &ph)
{
    const float gx = axis_gap(alo.x, ahi.x, blo.x, bhi.x, ph.periodic, ph.box_len_f[0]);
    const float gy = axis_gap(alo.y, ahi.y, blo.y, bhi.y, ph.periodic, ph.box_len_f[1]);
    const float gz = axis_gap(alo.z, ahi.z, blo.z, bhi.z, ph.periodic, ph.box_len_f[2]);
    return gx * gx + gy * gy + gz * gz <= R * R * 1.00001f;
}

// Warp-cooperative depth-first walk of one problem's tree.  At the leaf level
// visit(mask, first) is called (warp-uniformly) with the ballot of the up to
// 32 sibling leaves first..first+31 whose boxes pass test(box), so that a
// whole group of candidate leaves is staged in one round of memory accesses.
template <class Test, class Visit>
__device__ __forceinline__ void walk(const BatchView &b, const ProbDyn &d, Test &&test, Visit &&visit)
{
    const int lane = threadIdx.x & 31;
    const int top = d.top_level;
    unsigned mask[kMaxLevels + 1];
    int base[kMaxLevels + 1];
    {
        bool ok = lane < d.node_cnt[top] && test(b.nodes[top][d.node_off[top] + lane]);
        unsigned m = __ballot_sync(FULL, ok);
        if (top == 0) {
            if (m) visit(m, d.node_off[0]);
            return;
        }
        mask[top] = m;
        base[top] = 0;
    }
    int lvl = top;
    for (;;) {
        unsigned m = mask[lvl];
        if (m == 0u) {
            if (++lvl > top) break;
            continue;
        }
        int c = __ffs(m) - 1;
        mask[lvl] = m & (m - 1u);
        int node = base[lvl] + c;
        int ch = node * kBranch + lane;
        bool ok = ch < d.node_cnt[lvl - 1] && test(b.nodes[lvl - 1][d.node_off[lvl - 1] + ch]);
        unsigned cm = __ballot_sync(FULL, ok);
        if (lvl == 1) {
            if (cm) visit(cm, d.node_off[0] + node * kBranch);
            continue;
        }
        --lvl;
        base[lvl] = node * kBranch;
        mask[lvl] = cm;
    }
}

template <typename T>
__device__ __forceinline__ int warp_incl_scan(int v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int w = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += w;
    }
    return v;
}

// Per-warp scratch for staging one group of up to 32 candidate leaves.
template <typename T>
struct StageScratch {
    int first[32];             // group element index of each candidate leaf's first particle
    int start[32];             // sorted index of each candidate leaf's first particle
    T dx[32], dy[32], dz[32];  // leaf shift (FP64 difference of reference points, cast)
};

// candidate leaf (lane of the group) holding group element e: the last lane
// whose first element is <= e (lanes without particles share the next
// lane's first element and are passed over)
template <typename T>
__device__ __forceinline__ int owner_of(const StageScratch<T> &sc, int e)
{
    int k = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (sc.first[k + step] <= e) k += step;
    return k;
}

// Squared distance from point q to the box [lo, hi] (zero inside).
template <typename T, typename V>
__device__ __forceinline__ T box_dist2(const V &q, const V &lo, const V &hi)
{
    T dx = fmax(fmax(lo.x - q.x, q.x - hi.x), T(0));
    T dy = fmax(fmax(lo.y - q.y, q.y - hi.y), T(0));
    T dz = fmax(fmax(lo.z - q.z, q.z - hi.z), T(0));
    return dx * dx + dy * dy + dz * dz;
}

// Stage the particles of the leaves first + k (bit k of mask) that keep()
// accepts, compacted into slots [nbuf, ...) of the warp's candidate buffer of
// capacity CH; flush() runs first whenever fewer than 32 slots are free.
// The particles are read 32 at a time, one per lane, through load(j) (j the
// sorted index) and moved into the query leaf A's frame by the leaf shift
// (FP64 difference of the reference points, minimum image, cast) before
// keep(q) sees them.  group(has, B, stB, D) runs on every lane once per call
// (lane k: candidate leaf first + k if has); store(slot, q, k, idx) writes a
// kept particle (k: its leaf's lane, idx: its index within that leaf).
template <typename T, int CH, class Group, class Load, class Keep, class Store, class Flush>
__device__ __forceinline__ void stage_group(const BatchView &b, int A, unsigned mask, int first, const PhysParams &ph,
                                            int &nbuf, StageScratch<T> &sc, Group &&group, Load &&load,
                                            Keep &&keep, Store &&store, Flush &&flush)
{
    using V = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const bool has = (mask >> lane) & 1u;
    int stB = 0, nB = 0;
    T Dx = T(0), Dy = T(0), Dz = T(0);
    if (has) {
        const int B = first + lane;
        stB = b.leaf_start[B];
        nB = b.leaf_start[B + 1] - stB;
        const double *cb = b.leaf_c + 3LL * B, *ca = b.leaf_c + 3LL * A;
        Dx = (T)min_image(cb[0] - ca[0], ph.box_len[0], ph.periodic);
        Dy = (T)min_image(cb[1] - ca[1], ph.box_len[1], ph.periodic);
        Dz = (T)min_image(cb[2] - ca[2], ph.box_len[2], ph.periodic);
    }
    group(has, first + lane, stB, Dx, Dy, Dz);
    const int incl = warp_incl_scan<T>(nB);
    const int tot = __shfl_sync(FULL, incl, 31);
    __syncwarp();  // earlier readers of the scratch are done
    sc.first[lane] = incl - nB;
    sc.start[lane] = stB;
    sc.dx[lane] = Dx;
    sc.dy[lane] = Dy;
    sc.dz[lane] = Dz;
    __syncwarp();
    const unsigned below = (1u << lane) - 1u;
    for (int e0 = 0; e0 < tot; e0 += 32) {
        if (nbuf > CH - 32) flush();
        const int e = e0 + lane;
        bool ok = false;
        V q;
        int k = 0, idx = 0;
        if (e < tot) {
            k = owner_of(sc, e);
            idx = e - sc.first[k];
            q = load(sc.start[k] + idx);
            q.x += sc.dx[k];
            q.y += sc.dy[k];
            q.z += sc.dz[k];
            ok = keep(q);
        }
        const unsigned bal = __ballot_sync(FULL, ok);
        if (ok) store(nbuf + __popc(bal & below), q, k, idx);
        nbuf += __popc(bal);
    }
}

// Box of the query leaf's particles in its own frame (offsets from the
// reference point), over the lanes with on set.
template <typename V, typename T>
__device__ __forceinline__ void frame_box(const V &x, bool on, V &lo, V &hi)
{
    lo.x = warp_min(on ? x.x : tinf<T>());
    lo.y = warp_min(on ? x.y : tinf<T>());
    lo.z = warp_min(on ? x.z : tinf<T>());
    hi.x = warp_max(on ? x.x : -tinf<T>());
    hi.y = warp_max(on ? x.y : -tinf<T>());
    hi.z = warp_max(on ? x.z : -tinf<T>());
}

// sum over the LPP lanes that serve one particle
template <int LPP, typename T>
__device__ __forceinline__ T group_sum(T v)
{
#pragma unroll
    for (int o = 1; o < LPP; o <<= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
template <int LPP, typename T>
__device__ __forceinline__ T group_max(T v)
{
#pragma unroll
    for (int o = 1; o < LPP; o <<= 1) {
        T w = __shfl_xor_sync(FULL, v, o);
        v = w > v ? w : v;
    }
    return v;
}
template <int LPP>
__device__ __forceinline__ bool group_any(bool v)
{
    int x = v ? 1 : 0;
#pragma unroll
    for (int o = 1; o < LPP; o <<= 1) x |= __shfl_xor_sync(FULL, x, o);
    return x != 0;
}

// One Newton-Raphson update of the h-rho solve with the oracle's bracketing
// (Eqs. SPHRHO, HRHO).  Returns true when |h_new - h| < tol h; h then stays
// (it is within the tolerance of the root, and the caller's sums at h stay
// valid), else h becomes h_new.
template <typename T>
__device__ __forceinline__ bool nr_update(T &h, T &lo, T &hi, T rho, T drho, T m, T eta3, T tol)
{
    T hinv = T(1) / h;
    T hinv3 = hinv * hinv * hinv;
    T F = rho - m * eta3 * hinv3;
    T dF = drho + T(3) * m * eta3 * hinv3 * hinv;
    if (F < T(0)) lo = h;
    else hi = h;
    T hn = dF > T(0) ? h - F / dF : T(-1);
    bool bad = !(hn >= lo) || !(hn <= hi) || !(hn >= T(0.5) * h) || !(hn <= T(2) * h) || !(dF > T(0));
    if (bad) hn = (hi == tinf<T>()) ? T(2) * h : T(0.5) * (lo + hi);
    const bool conv = fabs(hn - h) < tol * h;
    if (!conv) h = hn;
    return conv;
}

template <typename T, int LPP, bool UM>
struct DCfg {
    using V = typename Vec4<T>::type;
    // list entries per lane: room for ~2x the mean neighbour count of 58 per particle
    static constexpr int LCAP = LPP == 1 ? SPH_DENS_LCAP1 : LPP == 2 ? 64 : LPP == 4 ? 40 : 24;
    static constexpr int CH = SPH_DENS_CH;
    static constexpr int WPB = 4;
    static constexpr int LW = UM ? 1 : 2;  // list words per entry: r (and m_j unless masses are equal)
    static constexpr size_t scratch = (sizeof(StageScratch<T>) + 31) & ~(size_t)31;
    static constexpr size_t per_warp = CH * sizeof(V) + (size_t)LCAP * 32 * LW * sizeof(T) + scratch;
    static constexpr size_t smem = WPB * per_warp;
};

// Outputs of the density solve for sorted particle s (one lane per particle).
template <typename T>
__device__ __forceinline__ void density_epilogue(const BatchView &b, const ProbStatic &ps, long long s,
                                                 typename Vec4<T>::type pi, T h, T S0, T S1, int use_pred)
{
    using V = typename Vec4<T>::type;
    const PhysParams &ph = ps.ph;
    T hinv = T(1) / h;
    T hinv3 = hinv * hinv * hinv;
    T rho = T(1.0 / kPi) * S0 * hinv3;
    T drho = -T(1.0 / kPi) * hinv3 * hinv * (T(3) * S0 + S1);
    T omega = T(1) + h / (T(3) * rho) * drho;
    long long g = b.perm[s];
    long long i = g - ps.base;
    double u = use_pred ? b.up[g] : ps.u[i];
    double v[3] = {use_pred ? b.vpx[g] : ps.vx[i], use_pred ? b.vpy[g] : ps.vy[i],
                   use_pred ? b.vpz[g] : ps.vz[i]};
    T P, c;
    if (ph.eos == SPH_EOS_ISOTHERMAL) {
        c = (T)ph.cs_iso;
        P = c * c * rho;
    } else {
        P = (T)(ph.gamma - 1.0) * rho * (T)u;
        c = sqrt((T)ph.gamma * P / rho);
    }
    T A = P / (omega * rho * rho);
    b.sh[s] = (double)h;
    b.hf[s] = to_float_ru(h);
    b.srho[s] = (double)rho;
    b.somega[s] = (double)omega;
    b.sP[s] = (double)P;
    b.sc[s] = (double)c;
    ps.h[i] = (double)h;
    ps.rho[i] = (double)rho;
    ps.omega[i] = (double)omega;
    ps.P[i] = (double)P;
    ps.c[i] = (double)c;
    V q;
    q.x = pi.x;
    q.y = pi.y;
    q.z = pi.z;
    q.w = hinv;
    ((V *)b.ph)[s] = q;
    q.x = (T)v[0];
    q.y = (T)v[1];
    q.z = (T)v[2];
    q.w = c;
    ((V *)b.vc)[s] = q;
    q.x = A;
    q.y = rho;
    q.z = pi.w;
    q.w = (T)u;
    ((V *)b.th)[s] = q;
    if (!(isfinite((double)rho) && isfinite((double)omega) && isfinite((double)P)))
        atomicOr(&ps.diag->status, ST_NONFINITE);
}

template <typename T, int LPP, bool UM>
__global__ void __launch_bounds__(DCfg<T, LPP, UM>::WPB * 32, SPH_DENS_MINB) k_density(BatchView b, int use_pred)
{
    using C = DCfg<T, LPP, UM>;
    using V = typename C::V;
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem + wib * C::per_warp;
    V *cand = reinterpret_cast<V *>(mine);
    T *lr = reinterpret_cast<T *>(mine + C::CH * sizeof(V));
    T *lm = lr + C::LCAP * 32;  // used only when masses differ
    StageScratch<T> &sc = *reinterpret_cast<StageScratch<T> *>(lr + C::LCAP * 32 * C::LW);
    const int pp = lane / LPP, sub = lane % LPP;
    const int nleaf = b.counters[0];
    const V *pm = (const V *)b.pm;

    for (;;) {
        int leaf = 0;
        if (lane == 0) leaf = atomicAdd(&b.counters[kDensityCounter + lpp_log2(LPP) + (UM ? 4 : 0)], 1);
        leaf = __shfl_sync(FULL, leaf, 0);
        if (leaf >= nleaf) break;
        const int p = b.leaf_pid[leaf];
        const ProbStatic &ps = b.prob[p];
        if (ps.lpp != LPP || (ps.uniform_m != 0) != UM) continue;  // served by another launch
        const T mu_all = (T)ps.m_uniform;
        const int st = b.leaf_start[leaf], nA = b.leaf_start[leaf + 1] - st;
        const ProbDyn &dy = b.dyn[p];
        const PhysParams &ph = ps.ph;
        const NodeBox boxA = b.nodes[0][leaf];
        const bool active = pp < nA;
        const long long s = st + (active ? pp : 0);
        const V pi = pm[s];
        const T mi = pi.w;
        V flo, fhi;
        frame_box<V, T>(pi, active, flo, fhi);
        const T eta3 = (T)(ph.eta * ph.eta * ph.eta);
        const T tol = (T)ph.h_tol;
        const int maxit = ph.h_max_iter;
        const double Lmin = ph.periodic ? fmin(ph.box_len[0], fmin(ph.box_len[1], ph.box_len[2])) : INFINITY;
        const T hbox = (T)(0.25 * Lmin);  // h beyond a quarter of the box: SPH_EBOX
        T h = active ? (T)b.sh[s] : T(1);
        // the leaf pass predicted this particle's sphere from the same start
        const float hpred = active ? __fmul_ru(kHPredict, __double2float_ru(b.sh[s])) : 0.f;
        if (active && !(h > T(0))) {
            double ext = ph.periodic ? fmax(ph.box_len[0], fmax(ph.box_len[1], ph.box_len[2])) : 1.0 / dy.dom_inv;
            h = (T)(ph.eta * cbrt(ext * ext * ext / (double)(ps.n > 0 ? ps.n : 1)));
        }
        T lo = T(0), hi = tinf<T>();
        int it = 0;
        bool conv = !active, fail = false, need = false, noconv = false;
        bool kept = false;  // converged by tolerance: the sums at the returned h are kS0, kS1
        T kS0 = T(0), kS1 = T(0);
        int knn = 0;
        int cnt = 0;
        long long pairs = 0, tested = 0;
        // bal: in-range candidates are dealt to the particle's LPP lanes by
        // their rank among the group's hits instead of by slot, so that the
        // lists fill evenly; taken after a slot-dealt list overflowed
        bool bal = false;
        // candidate-leaf groups of the last walk (lane k holds group k) and
        // the walk radius they cover, kept for the force pass unless the
        // recent records outgrew their h (then the force pass walks)
        const bool record = ps.diag->reuse_hold == 0;
        int ng = 0, g_first = 0;
        unsigned g_mask = 0u;
        float Rq_last = 0.f;
        for (int attempt = 0;; ++attempt) {
            const T hs = h * (T)kListMargin;
            float Rq = warp_max((active && !fail) ? __fmul_ru(2.0f, (float)hs) : 0.f) * 1.0001f;
            const T R2 = (T(2) * hs) * (T(2) * hs);
            Rq_last = Rq;
            ng = 0;
            cnt = 0;
            int gcnt = 0;
            bool ovf = false;
            int nbuf = 0;
            auto flush = [&]() {
                __syncwarp();  // staged candidates visible to every lane
                if (LPP == 1 || !bal) {
#pragma unroll 4
                    for (int k = sub; k < nbuf; k += LPP) {
                        V c = cand[k];
                        T dx = pi.x - c.x, dyy = pi.y - c.y, dz = pi.z - c.z;
                        T r2 = dx * dx + dyy * dyy + dz * dz;
                        if (active && !fail && r2 < R2) {
                            if (cnt < C::LCAP) {
                                lr[cnt * 32 + lane] = sqrt(r2);
                                if (!UM) lm[cnt * 32 + lane] = c.w;
                                ++cnt;
                            } else {
                                ovf = true;
                            }
                        }
                    }
                } else {
                    const unsigned below = (1u << sub) - 1u;
                    for (int k0 = 0; k0 < nbuf; k0 += LPP) {
                        const int k = k0 + sub;
                        bool hit = false;
                        T r = T(0), mj = T(0);
                        if (k < nbuf) {
                            V c = cand[k];
                            T dx = pi.x - c.x, dyy = pi.y - c.y, dz = pi.z - c.z;
                            T r2 = dx * dx + dyy * dyy + dz * dz;
                            hit = active && !fail && r2 < R2;
                            r = sqrt(r2);
                            mj = c.w;
                        }
                        const unsigned gm = (__ballot_sync(FULL, hit) >> (pp * LPP)) & ((1u << LPP) - 1u);
                        if (hit) {
                            const int e = gcnt + __popc(gm & below);
                            if (e < C::LCAP * LPP) {
                                const int o = (e / LPP) * 32 + pp * LPP + e % LPP;
                                lr[o] = r;
                                if (!UM) lm[o] = mj;
                            } else {
                                ovf = true;
                            }
                        }
                        gcnt += __popc(gm);
                    }
                }
                tested += (nbuf - sub + LPP - 1) / LPP;
                __syncwarp();
                nbuf = 0;
            };
            const T Rq2 = (T)Rq * (T)Rq;
            // visit leaves within Rq (gather) or whose predicted smoothing
            // spheres reach this leaf (what the force pass will need); stage
            // only the former
            bool near = false;  // this lane's last tested node is within Rq
            walk(
                b, dy,
                [&](const NodeBox &nb) {
                    near = box_within(boxA.plo, boxA.phi, nb.plo, nb.phi, Rq, ph);
                    return near || (record && box_overlap(boxA.plo, boxA.phi, nb.slo, nb.shi, 0.f, ph));
                },
                [&](unsigned mask, int first) {
                    if (lane == ng) {
                        g_first = first;
                        g_mask = mask;
                    }
                    ++ng;
                    // the leaf-level tests just made: stage the leaves within Rq
                    const unsigned gm = __ballot_sync(FULL, near && ((mask >> lane) & 1u));
                    if (gm == 0u) return;
                    stage_group<T, C::CH>(
                        b, leaf, gm, first, ph, nbuf, sc, [](bool, int, int, T, T, T) {},
                        [&](int j) { return pm[j]; },
                        [&](const V &q) { return box_dist2<T>(q, flo, fhi) < Rq2; },
                        [&](int slot, const V &q, int, int) { cand[slot] = q; }, flush);
                });
            flush();
            if (LPP > 1 && bal) {
                const int mine_n = gcnt > sub ? (gcnt - sub - 1) / LPP + 1 : 0;
                cnt = mine_n < C::LCAP ? mine_n : C::LCAP;
            }
            if (LPP > 1 && !bal && __any_sync(FULL, ovf)) {
                bal = true;  // same radius again, dealt by rank
                --attempt;
                continue;
            }
            if (group_any<LPP>(ovf) && active && !fail) fail = true;
            // Newton-Raphson on the cached lists
            for (;;) {
                bool go = active && !conv && !fail && !need;
                if (!__any_sync(FULL, go)) break;
                T S0 = T(0), S1 = T(0);
                int nn = 0;
                if (go) {
                    const T hinv = T(1) / h;
                    for (int e = 0; e < cnt; ++e) {
                        T q = lr[e * 32 + lane] * hinv;
                        T mj = UM ? mu_all : lm[e * 32 + lane];
                        T f, df;
                        m4(q, f, df);
                        S0 += mj * f;
                        S1 += mj * q * df;
                        nn += q < T(2);
                    }
                }
                S0 = group_sum<LPP>(S0);
                S1 = group_sum<LPP>(S1);
                nn = group_sum<LPP>(nn);
                if (go) {
                    ++it;
                    if (sub == 0) pairs += nn;
                    T hinv = T(1) / h;
                    T hinv3 = hinv * hinv * hinv;
                    T rho = T(1.0 / kPi) * S0 * hinv3;
                    T drho = -T(1.0 / kPi) * hinv3 * hinv * (T(3) * S0 + S1);
                    bool c = nr_update(h, lo, hi, rho, drho, mi, eta3, tol);
                    if (c) {
                        kept = true;
                        kS0 = S0;
                        kS1 = S1;
                        knn = nn;
                    }
                    if (h > hbox) {
                        atomicOr(&ps.diag->status, ST_BOX);
                        c = true;
                        kept = false;
                    }
                    if (!c && it >= maxit) {
                        noconv = true;
                        c = true;
                    }
                    conv = c;
                    if (h > hs) need = true;
                }
            }
            if (!__any_sync(FULL, need)) break;
            if (attempt + 1 >= kMaxRebuild) {
                if (need) fail = true;
                break;
            }
            need = false;
        }
        // record the last walk's groups for the force pass (lane 0 reserves
        // pool space); not recorded: the force pass walks for this leaf
        {
            int base = 0;
            if (lane == 0) {
                base = record && ng <= kMaxLeafGroups ? atomicAdd(&b.counters[kPoolCounter], ng) : -1;
                const bool fits = base >= 0 && (long long)base + ng <= b.group_cap;
                b.leaf_gofs[leaf] = fits ? base : 0;
                b.leaf_ngroups[leaf] = fits ? ng : -1;
                b.leaf_hcap[leaf] = Rq_last / 2.0002f;
                base = fits ? base : -1;
            }
            base = __shfl_sync(FULL, base, 0);
            if (base >= 0 && lane < ng) b.group_pool[base + lane] = make_int2(g_first, (int)g_mask);
        }
        // final evaluation at the returned h, unless the sums there are kept
        T S0 = kS0, S1 = kS1;
        int nn = knn;
        const bool fin = active && !fail;
        const bool redo = fin && !kept;
        if (__any_sync(FULL, redo)) {
            T R0 = T(0), R1 = T(0);
            int rn = 0;
            if (redo) {
                const T hinv = T(1) / h;
                for (int e = 0; e < cnt; ++e) {
                    T q = lr[e * 32 + lane] * hinv;
                    T mj = UM ? mu_all : lm[e * 32 + lane];
                    T f, df;
                    m4(q, f, df);
                    R0 += mj * f;
                    R1 += mj * q * df;
                    rn += q < T(2);
                }
            }
            R0 = group_sum<LPP>(R0);
            R1 = group_sum<LPP>(R1);
            rn = group_sum<LPP>(rn);
            if (redo) {
                S0 = R0;
                S1 = R1;
                nn = rn;
                if (sub == 0) pairs += rn;
            }
        }
        if (fin && sub == 0) {
            density_epilogue<T>(b, ps, s, pi, h, S0, S1, use_pred);
            if (noconv) {
                atomicOr(&ps.diag->status, ST_NOCONV);
                atomicAdd(&ps.diag->unconverged, 1);
            }
            // the recorded candidate groups cover this particle's pairs only
            // if its final h stays within the walk radius and its prediction
            const float hf = to_float_ru(h);
            if (hf > hpred || hf > Rq_last / 2.0002f) atomicOr(&b.dyn[p].lists_stale, 1);
        }
        if (active && fail && sub == 0) {
            int k = atomicAdd(&b.counters[kSlowCounter], 1);
            b.fallback_list[k] = (int)s;
            b.sh[s] = (double)h;  // best guess so far
            b.hf[s] = hpred;      // for the slow path's coverage check
        }
        // statistics (one atomic per warp per quantity)
        long long tp = warp_sum(pairs), tt = warp_sum(tested);
        int itn = (fin && sub == 0) ? it : 0;
        long long its = warp_sum((long long)itn);
        int itmax = warp_max(itn);
        int nmin = warp_min((fin && sub == 0) ? nn : 0x7fffffff);
        int nmax = warp_max((fin && sub == 0) ? nn : 0);
        long long nsum = warp_sum((long long)((fin && sub == 0) ? nn : 0));
        if (lane == 0) {
            ProbDiag *dg = ps.diag;
            atomicAdd((unsigned long long *)&dg->density_pairs, (unsigned long long)tp);
            atomicAdd((unsigned long long *)&dg->candidates, (unsigned long long)tt);
            atomicAdd((unsigned long long *)&dg->nr_iter, (unsigned long long)its);
            atomicAdd((unsigned long long *)&dg->ngb_sum, (unsigned long long)nsum);
            atomicMax(&dg->nr_max, itmax);
            if (nmax > 0) {
                atomicMin(&dg->ngb_min, nmin);
                atomicMax(&dg->ngb_max, nmax);
            }
        }
    }
}

// Slow path: one warp per particle for the particles whose per-lane lists in
// k_density overflowed or outgrew their radius.  The warp stages the leaf's
// candidate leaves in groups, as k_density does, gathers the particle's
// neighbours (within 2 h x 1.1) into a list spread over its 32 lanes (up to
// kFbPerLane each) and iterates on it, walking the tree again only when h
// outgrows the list; if even that list overflows, every iteration walks the
// tree and sums the staged candidates directly.
constexpr int kFbPerLane = 24;
constexpr int kFbCH = 128;
constexpr double kFbMargin = 1.1;

template <typename T>
struct FbCfg {
    using V = typename Vec4<T>::type;
    static constexpr int WPB = 4;
    static constexpr size_t scratch = (sizeof(StageScratch<T>) + 31) & ~(size_t)31;
    static constexpr size_t per_warp = kFbCH * sizeof(V) + (size_t)2 * kFbPerLane * 32 * sizeof(T) + scratch;
    static constexpr size_t smem = WPB * per_warp;
};

template <typename T>
__global__ void __launch_bounds__(FbCfg<T>::WPB * 32) k_density_fallback(BatchView b, int use_pred)
{
    using C = FbCfg<T>;
    using V = typename C::V;
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem + wib * C::per_warp;
    V *cand = reinterpret_cast<V *>(mine);
    T *fr = reinterpret_cast<T *>(mine + kFbCH * sizeof(V));
    T *fm = fr + kFbPerLane * 32;
    StageScratch<T> &sc = *reinterpret_cast<StageScratch<T> *>(fm + kFbPerLane * 32);
    const int nf = b.counters[kSlowCounter];
    const V *pm = (const V *)b.pm;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int k = w; k < nf; k += nw) {
        const long long s = b.fallback_list[k];
        const int leaf = (int)b.flag[s] - 1;
        const int p = b.leaf_pid[leaf];
        const ProbStatic &ps = b.prob[p];
        const ProbDyn &dy = b.dyn[p];
        const PhysParams &ph = ps.ph;
        const NodeBox boxA = b.nodes[0][leaf];
        const V pi = pm[s];
        const T eta3 = (T)(ph.eta * ph.eta * ph.eta);
        const T tol = (T)ph.h_tol;
        double Lmin = ph.periodic ? fmin(ph.box_len[0], fmin(ph.box_len[1], ph.box_len[2])) : INFINITY;
        T h = (T)b.sh[s];
        T lo = T(0), hi = tinf<T>();
        int it = 0;
        bool conv = false, noconv = false;
        long long pairs = 0;
        T S0, S1;
        int nn;
        // every particle within Rq of particle s, staged in groups of
        // leaves; fn(r2, m_j) sees one candidate per lane
        auto visit_all = [&](float Rq, auto &&fn) {
            const T Rq2 = (T)Rq * (T)Rq;
            int nbuf = 0;
            auto flush = [&]() {
                __syncwarp();
                for (int e = lane; e < nbuf; e += 32) {
                    const V c = cand[e];
                    T dx = pi.x - c.x, dyy = pi.y - c.y, dz = pi.z - c.z;
                    fn(dx * dx + dyy * dyy + dz * dz, c.w);
                }
                __syncwarp();
                nbuf = 0;
            };
            walk(
                b, dy, [&](const NodeBox &nb) { return box_within(boxA.plo, boxA.phi, nb.plo, nb.phi, Rq, ph); },
                [&](unsigned mask, int first) {
                    stage_group<T, kFbCH>(
                        b, leaf, mask, first, ph, nbuf, sc, [](bool, int, int, T, T, T) {},
                        [&](int j) { return pm[j]; }, [&](const V &q) { return box_dist2<T>(q, pi, pi) < Rq2; },
                        [&](int slot, const V &q, int, int) { cand[slot] = q; }, flush);
                });
            flush();
        };
        bool direct = false;
        T hs = T(0);
        int cnt = 0;
        auto build = [&]() {
            hs = h * (T)kFbMargin;
            const T R2 = T(4) * hs * hs;
            cnt = 0;
            bool ovf = false;
            visit_all(__fmul_ru(2.0f, (float)hs) * 1.0001f, [&](T r2, T mj) {
                if (r2 < R2) {
                    if (cnt < kFbPerLane) {
                        fr[cnt * 32 + lane] = sqrt(r2);
                        fm[cnt * 32 + lane] = mj;
                        ++cnt;
                    } else {
                        ovf = true;
                    }
                }
            });
            direct = __any_sync(FULL, ovf);
            __syncwarp();
        };
        auto sums = [&](T hh) {
            S0 = T(0);
            S1 = T(0);
            nn = 0;
            const T hinv = T(1) / hh;
            if (!direct) {
                for (int e = 0; e < cnt; ++e) {
                    T f, df, qq = fr[e * 32 + lane] * hinv;
                    m4(qq, f, df);
                    T mj = fm[e * 32 + lane];
                    S0 += mj * f;
                    S1 += mj * qq * df;
                    nn += qq < T(2);
                }
            } else {
                const T R2 = T(4) * hh * hh;
                visit_all(__fmul_ru(2.0f, (float)hh) * 1.0001f, [&](T r2, T mj) {
                    if (r2 < R2) {
                        T f, df, qq = sqrt(r2) * hinv;
                        m4(qq, f, df);
                        S0 += mj * f;
                        S1 += mj * qq * df;
                        ++nn;
                    }
                });
            }
            S0 = warp_sum(S0);
            S1 = warp_sum(S1);
            nn = warp_sum(nn);
        };
        build();
        while (!conv) {
            if (!direct && h > hs) build();
            sums(h);
            ++it;
            pairs += nn;
            T hinv = T(1) / h;
            T hinv3 = hinv * hinv * hinv;
            T rho = T(1.0 / kPi) * S0 * hinv3;
            T drho = -T(1.0 / kPi) * hinv3 * hinv * (T(3) * S0 + S1);
            bool c = nr_update(h, lo, hi, rho, drho, pi.w, eta3, tol);
            if ((double)h > 0.25 * Lmin) {
                if (lane == 0) atomicOr(&ps.diag->status, ST_BOX);
                c = true;
            }
            if (!c && it >= ph.h_max_iter) {
                noconv = true;
                c = true;
            }
            conv = c;
        }
        if (!direct && h > hs) build();
        sums(h);
        pairs += nn;
        if (lane == 0) {
            const float hf = to_float_ru(h);
            if (hf > b.hf[s] || hf > b.leaf_hcap[leaf]) atomicOr(&b.dyn[p].lists_stale, 1);
            density_epilogue<T>(b, ps, s, pi, h, S0, S1, use_pred);
            if (noconv) {
                atomicOr(&ps.diag->status, ST_NOCONV);
                atomicAdd(&ps.diag->unconverged, 1);
            }
            ProbDiag *dg = ps.diag;
            atomicAdd((unsigned long long *)&dg->density_pairs, (unsigned long long)pairs);
            atomicAdd((unsigned long long *)&dg->nr_iter, (unsigned long long)it);
            atomicAdd((unsigned long long *)&dg->fallback, 1ull);
            atomicAdd((unsigned long long *)&dg->ngb_sum, (unsigned long long)nn);
            atomicMax(&dg->nr_max, it);
            atomicMin(&dg->ngb_min, nn);
            atomicMax(&dg->ngb_max, nn);
        }
    }
}

// ---------------------------------------------------------------------------
// forces
// ---------------------------------------------------------------------------
// Force walk: the staged candidates (CH per chunk) are tested against the
// lane's particle and each pair found is appended to the lane's list as a
// 16-bit code (slot of its leaf in the warp's table of candidate leaves << 5 |
// index within that leaf); the lists are evaluated, reading the partner's
// data from global memory, when one of them or the table fills and at the end,
// so that every lane evaluates about the same number of pairs.
template <typename T, int LPP>
struct FCfg {
    using V = typename Vec4<T>::type;
    static constexpr int CH = SPH_FORCE_CH;
    // list entries per lane, and candidates tested per list-room check: at
    // one lane per particle a lane holds all of its particle's ~60 pairs
    static constexpr int LC = LPP == 1 ? SPH_FORCE_LC1 : SPH_FORCE_LC;
    static constexpr int SB = LPP == 1 ? SPH_FORCE_SB1 : SPH_FORCE_SB;
    static constexpr int TAB = SPH_FORCE_TAB;  // candidate leaves per table fill (<= 2048)
    static constexpr int WPB = 4;
    static_assert(TAB <= 2048 && LC >= 2 * SB / LPP, "force list layout");
    static constexpr size_t scratch = (sizeof(StageScratch<T>) + 31) & ~(size_t)31;
    static constexpr size_t codes = ((size_t)(CH + LC * 32) * 2 + 31) & ~(size_t)31;
    static constexpr size_t per_warp = (CH + TAB) * sizeof(V) + scratch + codes;
    static constexpr size_t smem = WPB * per_warp;
};

// Compensated sum with an error-free transformation per addition (Knuth's
// branch-free TwoSum): s + c carries the exact running sum to O(n eps^2),
// whatever the signs and magnitudes of the terms.
template <typename T>
struct TwoSumAcc {
    T s, c;
    __device__ __forceinline__ void add(T x)
    {
        T t = add_rn(s, x);
        T xp = t - s;
        T sp = t - xp;
        T e = (s - sp) + (x - xp);
        c = c + e;
        s = t;
    }
};

template <typename V>
__device__ __forceinline__ V ld_ro(const V *p);
template <>
__device__ __forceinline__ float4 ld_ro<float4>(const float4 *p) { return __ldg(p); }
template <>
__device__ __forceinline__ dbl4 ld_ro<dbl4>(const dbl4 *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 c = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    dbl4 v;
    v.x = a.x;
    v.y = a.y;
    v.z = c.x;
    v.w = c.y;
    return v;
}

template <typename T, int LPP>
__global__ void __launch_bounds__(FCfg<T, LPP>::WPB * 32, SPH_FORCE_MINB) k_forces(BatchView b)
{
    using C = FCfg<T, LPP>;
    using V = typename C::V;
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem + wib * C::per_warp;
    V *cand = reinterpret_cast<V *>(mine);  // staged (offset + leaf shift, 1/h)
    V *table = cand + C::CH;                // per candidate leaf: (leaf shift, first sorted index)
    StageScratch<T> &sc = *reinterpret_cast<StageScratch<T> *>(table + C::TAB);
    unsigned short *code = reinterpret_cast<unsigned short *>(mine + (C::CH + C::TAB) * sizeof(V) + C::scratch);
    unsigned short *lst = code + C::CH;
    const int pp = lane / LPP, sub = lane % LPP;
    const unsigned below = (1u << lane) - 1u;
    const int nleaf = b.counters[0];
    const V *gph = (const V *)b.ph, *gvc = (const V *)b.vc, *gth = (const V *)b.th;

    for (;;) {
        int leaf = 0;
        if (lane == 0) leaf = atomicAdd(&b.counters[kForceCounter + lpp_log2(LPP)], 1);
        leaf = __shfl_sync(FULL, leaf, 0);
        if (leaf >= nleaf) break;
        const int p = b.leaf_pid[leaf];
        const ProbStatic &ps = b.prob[p];
        if (ps.lpp != LPP) continue;  // leaf of a problem served by another launch
        const int st = b.leaf_start[leaf], nA = b.leaf_start[leaf + 1] - st;
        const ProbDyn &dy = b.dyn[p];
        const PhysParams &ph = ps.ph;
        const NodeBox boxA = b.nodes[0][leaf];
        const bool active = pp < nA;
        const int s = st + (active ? pp : 0);
        const V xi = gph[s], vi = gvc[s], ti = gth[s];
        const T alpha = (T)ph.alpha_av, beta = (T)ph.beta_av, aac = (T)ph.alpha_ac;
        const bool adi = ph.eos == SPH_EOS_ADIABATIC;
        const T sigma = T(1.0 / kPi);
        const T hi2 = xi.w * xi.w, hi4 = hi2 * hi2;
        TwoSumAcc<T> ax{T(0), T(0)}, ay{T(0), T(0)}, az{T(0), T(0)};
        T du = T(0), vs = T(-1);
        int pairs = 0, tested = 0;
        const float R = __fmul_ru(2.0f, boxA.plo.w) * 1.0001f;
        const T RA2 = (T)R * (T)R;
        V flo, fhi;
        frame_box<V, T>(xi, active, flo, fhi);
        int nbuf = 0, cnt = 0, ntab = 0, tA = -1;
        unsigned gmask = 0u;
        auto fetch = [&](int e, V &tb, V &a0, V &a1, V &a2) {
            const unsigned cd = lst[e * 32 + lane];
            tb = table[cd >> 5];
            const int j = t_as_bits(tb.w) + (int)(cd & 31u);
            a0 = ld_ro(gph + j);
            a1 = ld_ro(gvc + j);
            a2 = ld_ro(gth + j);
        };
        auto eval_lists = [&]() {
            __syncwarp();
            for (int e = 0; e < cnt; ++e) {
                V tb, a0, a1, a2;
                fetch(e, tb, a0, a1, a2);
                // r_ij = (o_i - o_j) - D_AB: IEEE subtraction is sign-symmetric and
                // D_BA = -D_AB exactly, so particle j forms exactly -r_ij
                T rx = (xi.x - a0.x) - tb.x, ry = (xi.y - a0.y) - tb.y, rz = (xi.z - a0.z) - tb.z;
                T r2 = rx * rx + ry * ry + rz * rz;
                T rinv = rsqrt_t(r2);
                T r = r2 * rinv;
                T qi = r * xi.w, qj = r * a0.w;
                T hj2 = a0.w * a0.w;
                T gi = sigma * m4_df(qi) * hi4;
                T gj = sigma * m4_df(qj) * (hj2 * hj2);
                T pterm = add_rn(mul_rn(ti.x, gi), mul_rn(a2.x, gj));
                T vx = vi.x - a1.x, vy = vi.y - a1.y, vz = vi.z - a1.z;
                T vdr = (vx * rx + vy * ry + vz * rz) * rinv;
                T mu = vdr < T(0) ? vdr : T(0);
                T rhob_inv = fast_div(T(2), add_rn(ti.y, a2.y));
                T gbar = T(0.5) * add_rn(gi, gj);
                T vsig = add_rn(vi.w, a1.w) - beta * mu;
                T visc = alpha * vsig * mu * rhob_inv;
                T S = visc * gbar - pterm;
                T wgt = mul_rn(ti.z, a2.z) * S * rinv;
                ax.add(mul_rn(wgt, rx));
                ay.add(mul_rn(wgt, ry));
                az.add(mul_rn(wgt, rz));
                if (adi)
                    du += a2.z * (ti.x * vdr * gi +
                                  rhob_inv * gbar * (T(-0.5) * alpha * vsig * mu * mu + aac * fabs(vdr) * (ti.w - a2.w)));
                vs = vsig > vs ? vsig : vs;
            }
            pairs += cnt;
            cnt = 0;
            __syncwarp();  // table and lists free for reuse
        };
        // membership: r_ij < 2 max(h_i, h_j), decided on the staged
        // (offset + shift) difference; where its rounding differs from the
        // pair vector's the pair sits at q = 2, where f' and the force vanish
        auto test = [&]() {
            __syncwarp();  // staged candidates visible to every lane
            const int self = tA >= 0 ? ((tA << 5) | pp) : -1;
            for (int k0 = 0; k0 < nbuf; k0 += C::SB) {
                if (__any_sync(FULL, cnt > C::LC - C::SB / LPP)) eval_lists();
                const int ke = k0 + C::SB < nbuf ? k0 + C::SB : nbuf;
#pragma unroll 4
                for (int k = k0 + sub; k < ke; k += LPP) {
                    const V c = cand[k];
                    T rx = xi.x - c.x, ry = xi.y - c.y, rz = xi.z - c.z;
                    T r2 = rx * rx + ry * ry + rz * rz;
                    T hm = xi.w < c.w ? xi.w : c.w;
                    const int cd = code[k];
                    if (active && cd != self && r2 * hm * hm < T(4)) lst[cnt++ * 32 + lane] = (unsigned short)cd;
                }
            }
            tested += (nbuf - sub + LPP - 1) / LPP;
            __syncwarp();
            nbuf = 0;
        };
        auto node_test = [&](const NodeBox &nb) {
            return box_within(boxA.plo, boxA.phi, nb.plo, nb.phi, R, ph) ||
                   box_overlap(boxA.plo, boxA.phi, nb.slo, nb.shi, 0.f, ph);
        };
        auto visit = [&](unsigned mask, int first) {
                if (ntab + __popc(mask) > C::TAB) {
                    test();
                    eval_lists();
                    ntab = 0;
                    tA = -1;
                }
                stage_group<T, C::CH>(
                    b, leaf, mask, first, ph, nbuf, sc,
                    [&](bool has, int B, int stB, T Dx, T Dy, T Dz) {
                        gmask = mask;
                        if (has) {
                            V t;
                            t.x = Dx;
                            t.y = Dy;
                            t.z = Dz;
                            t.w = bits_as_t(stB, T(0));
                            table[ntab + __popc(mask & below)] = t;
                        }
                        const unsigned am = __ballot_sync(FULL, has && B == leaf);
                        if (am) tA = ntab + __popc(mask & ((1u << (__ffs(am) - 1)) - 1u));
                    },
                    [&](int j) { return gph[j]; },
                    [&](const V &q) {
                        const T d2 = box_dist2<T>(q, flo, fhi);
                        return d2 < RA2 || d2 * q.w * q.w < T(4.0004);
                    },
                    [&](int slot, const V &q, int k, int idx) {
                        cand[slot] = q;
                        code[slot] = (unsigned short)(((ntab + __popc(gmask & ((1u << k) - 1u))) << 5) | idx);
                    },
                    test);
                ntab += __popc(mask);
        };
        // the candidate groups the density walk recorded cover every pair
        // unless some final h outgrew them (then walk the tree again)
        const int ngl = b.leaf_ngroups[leaf];
        if (!dy.lists_stale && ngl >= 0) {
            const int gofs = b.leaf_gofs[leaf];
            for (int g = 0; g < ngl; ++g) {
                const int2 e = b.group_pool[gofs + g];
                const unsigned mask = (unsigned)e.y;
                bool ok = false;
                if ((mask >> lane) & 1u) ok = node_test(b.nodes[0][e.x + lane]);
                const unsigned fm = __ballot_sync(FULL, ok);
                if (fm) visit(fm, e.x);
            }
        } else {
            walk(b, dy, node_test, visit);
        }
        test();
        eval_lists();
        // combine the lanes of each particle; FP64 for the compensated sums
        double Fx = (double)ax.s + (double)ax.c, Fy = (double)ay.s + (double)ay.c, Fz = (double)az.s + (double)az.c;
        Fx = group_sum<LPP>(Fx);
        Fy = group_sum<LPP>(Fy);
        Fz = group_sum<LPP>(Fz);
        du = group_sum<LPP>(du);
        vs = group_max<LPP>(vs);
        // a = F / m in FP64 (m a stays F to FP64 round-off), one reciprocal
        // per particle (none for equal masses); the CFL step C h / v_sig of
        // Eq. SPH_DT in the pair precision (FP32: the FP64 pipe is much
        // narrower than the FP32 one on this part)
        T dti = tinf<T>();
        if (active && sub == 0) {
            long long g = b.perm[s];
            long long i = g - ps.base;
            const double minv = ps.uniform_m ? ps.inv_m_uniform : 1.0 / ps.m[i];
            double a[3] = {Fx * minv, Fy * minv, Fz * minv};
            const T vsig_t = vs < T(0) ? T(2) * vi.w : vs;
            ps.ax[i] = a[0];
            ps.ay[i] = a[1];
            ps.az[i] = a[2];
            ps.du[i] = adi ? (double)du : 0.0;
            ps.vsig[i] = (double)vsig_t;
            dti = (T)ph.c_cfl * (T)b.sh[s] / vsig_t;
            if (!(isfinite(a[0]) && isfinite(a[1]) && isfinite(a[2]) && isfinite(du)))
                atomicOr(&ps.diag->status, ST_NONFINITE);
        }
        const T dmin = warp_min(dti);
        long long tp = warp_sum((long long)pairs), tt = warp_sum((long long)tested);
        if (lane == 0) {
            if (dmin < INFINITY)
                atomicMin(&ps.diag->dt_min_bits, (unsigned long long)__double_as_longlong((double)dmin));
            atomicAdd((unsigned long long *)&ps.diag->force_pairs, (unsigned long long)tp);
            atomicAdd((unsigned long long *)&ps.diag->candidates, (unsigned long long)tt);
        }
    }
}

template <typename Kern>
void set_smem(Kern k, size_t bytes)
{
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int LPP, bool UM>
cudaError_t run_density(const BatchView &b, int use_pred, cudaStream_t st)
{
    using C = DCfg<T, LPP, UM>;
    static int per_sm = 0;
    if (!per_sm) {
        set_smem(k_density<T, LPP, UM>, C::smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_density<T, LPP, UM>, C::WPB * 32, C::smem);
        if (per_sm < 1) per_sm = 1;
    }
    k_density<T, LPP, UM><<<dev_info().sm_count * per_sm, C::WPB * 32, C::smem, st>>>(b, use_pred);
    return cudaGetLastError();
}

template <typename T>
void run_density_fallback(const BatchView &b, int use_pred, cudaStream_t st)
{
    using C = FbCfg<T>;
    static bool init = false;
    if (!init) {
        set_smem(k_density_fallback<T>, C::smem);
        init = true;
    }
    k_density_fallback<T><<<dev_info().sm_count * 4, C::WPB * 32, C::smem, st>>>(b, use_pred);
}

void density_fallback_launch(const BatchView &b, int precision, int use_pred, cudaStream_t st)
{
    if (precision == SPH_PREC_FP64) run_density_fallback<double>(b, use_pred, st);
    else run_density_fallback<float>(b, use_pred, st);
}

template <typename T, int LPP>
cudaError_t run_forces(const BatchView &b, cudaStream_t st)
{
    using C = FCfg<T, LPP>;
    static bool init = false;
    if (!init) {
        set_smem(k_forces<T, LPP>, C::smem);
        init = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forces<T, LPP>, C::WPB * 32, C::smem);
    if (per_sm < 1) per_sm = 1;
    int grid = dev_info().sm_count * per_sm;
    k_forces<T, LPP><<<grid, C::WPB * 32, C::smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_density(const BatchView &b, int precision, int use_pred, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    for (int cls = 0; cls < 8; ++cls) {
        if (!(b.dens_mask & (1 << cls))) continue;
        const int k = cls & 3;
        const bool um = cls >= 4;
        cudaError_t e;
        if (precision == SPH_PREC_FP64) {
            if (k == 2) e = um ? run_density<double, 4, true>(b, use_pred, st) : run_density<double, 4, false>(b, use_pred, st);
            else e = um ? run_density<double, 2, true>(b, use_pred, st) : run_density<double, 2, false>(b, use_pred, st);
        } else {
            switch (k) {
            case 0: e = um ? run_density<float, 1, true>(b, use_pred, st) : run_density<float, 1, false>(b, use_pred, st); break;
            case 1: e = um ? run_density<float, 2, true>(b, use_pred, st) : run_density<float, 2, false>(b, use_pred, st); break;
            case 2: e = um ? run_density<float, 4, true>(b, use_pred, st) : run_density<float, 4, false>(b, use_pred, st); break;
            default: e = um ? run_density<float, 8, true>(b, use_pred, st) : run_density<float, 8, false>(b, use_pred, st); break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    density_fallback_launch(b, precision, use_pred, st);
    return cudaGetLastError();
}

cudaError_t launch_forces(const BatchView &b, int precision, cudaStream_t st)
{
    if (b.ntot == 0) return cudaSuccess;
    for (int k = 0; k < 4; ++k) {
        if (!(b.lpp_mask & (1 << k))) continue;
        cudaError_t e;
        if (precision == SPH_PREC_FP64) {
            if (k == 2) e = run_forces<double, 4>(b, st);
            else e = run_forces<double, 2>(b, st);
        } else {
            switch (k) {
            case 0: e = run_forces<float, 1>(b, st); break;
            case 1: e = run_forces<float, 2>(b, st); break;
            case 2: e = run_forces<float, 4>(b, st); break;
            default: e = run_forces<float, 8>(b, st); break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace sph
