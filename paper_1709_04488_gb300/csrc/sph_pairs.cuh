// Pair kernels of the grad-h SPH neighbour loop (templates; the translation
// units sph_pairs.cu and sph_pairs_m6.cu instantiate them for the M4 and M6
// kernels).
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
//              F(h) = rho(h) - m (eta/h)^3 over the cached list of (r^2, m_j)
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
#pragma once
#include "sph_internal.cuh"
#include "sph_leaf.cuh"
#include "sph_tuned.h"

namespace sph {

namespace {

constexpr unsigned FULL = 0xffffffffu;
// class index of a lanes-per-particle count; 32 (block-step tasks, one
// particle per warp) shares 8's slot: a tick launches only its tasks' class
__host__ __device__ constexpr int lpp_log2(int l) { return l == 1 ? 0 : l == 2 ? 1 : l == 4 ? 2 : 3; }
constexpr double kListMargin = 1.03;  // list radius = R_K h * margin (R_K: support in units of h)

constexpr int kMaxRebuild = 6;

template <typename T>
__device__ __forceinline__ T tinf();
template <>
__device__ __forceinline__ float tinf<float>() { return INFINITY; }
template <>
__device__ __forceinline__ double tinf<double>() { return INFINITY; }

// Smoothing kernels of Sec. 2, W(r, h) = sigma f(q) / h^3 with q = r / h and
// support q < R: fdf(q) gives f and f', df(q) f' alone.
template <int K>
struct Kern;

// M4 cubic spline: sigma = 1/pi, R = 2.
template <>
struct Kern<SPH_KERNEL_M4> {
    static constexpr double R = 2.0;
    static constexpr double sigma = 1.0 / kPi;
    template <typename T>
    static __device__ __forceinline__ void fdf(T q, T &f, T &df)
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
    static __device__ __forceinline__ T df(T q);  // rounding fixed operation by operation (force pass)
};

// M6 quintic spline: f = (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5 (each term while
// its bracket is positive), sigma = 1/(120 pi), R = 3.  Inside q < 1 the
// three terms are summed as their expanded polynomial 66 - 60 q^2 + 30 q^4
// - 10 q^5 (f' = -120 q + 120 q^3 - 50 q^4), which avoids the cancellation
// of f' -> 0 at q -> 0; beyond q = 1 the brackets are used directly.
template <>
struct Kern<SPH_KERNEL_M6> {
    static constexpr double R = 3.0;
    static constexpr double sigma = 1.0 / (120.0 * kPi);
    template <typename T>
    static __device__ __forceinline__ void fdf(T q, T &f, T &df)
    {
        T a = q < T(3) ? T(3) - q : T(0);
        T c = q < T(2) ? T(2) - q : T(0);
        T a4 = (a * a) * (a * a), c4 = (c * c) * (c * c);
        T f2 = a4 * a - T(6) * (c4 * c), df2 = T(30) * c4 - T(5) * a4;
        T q2 = q * q;
        T f1 = T(66) + q2 * (T(-60) + q2 * (T(30) - T(10) * q));
        T df1 = q * (T(-120) + q2 * (T(120) - T(50) * q));
        bool in = q < T(1);
        f = in ? f1 : f2;
        df = in ? df1 : df2;
    }
    template <typename T>
    static __device__ __forceinline__ T df(T q);  // rounding fixed operation by operation (force pass)
};

// f, f' and sigma of the kernel a problem selects (warp-uniform; for the
// slow path, which serves particles of any problem)
template <typename T>
__device__ __forceinline__ void kern_fdf(int k, T q, T &f, T &df)
{
    if (k == SPH_KERNEL_M6) Kern<SPH_KERNEL_M6>::fdf(q, f, df);
    else Kern<SPH_KERNEL_M4>::fdf(q, f, df);
}
__device__ __forceinline__ double kern_sigma(int k)
{
    return k == SPH_KERNEL_M6 ? Kern<SPH_KERNEL_M6>::sigma : Kern<SPH_KERNEL_M4>::sigma;
}

// Softened gravity of the M4 kernel (Eqs. GRAVFORCEKERNEL, GRADHZETA): the
// enclosed mass fraction M(q) = 4 int_0^q f s^2 ds of a unit-mass kernel
// (phi' = M / r^2) and the potential shape psi (phi = psi(q)/h, psi' = M/q^2,
// -1/q from q = 2 on).  zeta needs psi + M/q (= -h^2 dphi/dh), which vanishes
// from q = 2 on and is psi(0) = -7/5 at q = 0.
template <typename T>
__device__ __forceinline__ T grav_mass(T q)
{
    const T q3 = q * q * q;
    if (q >= T(2)) return T(1);
    if (q < T(1)) return T(4) * q3 * (T(1.0 / 3.0) + q * q * (T(-0.3) + T(0.125) * q));
    return T(4) * (q3 * (T(2.0 / 3.0) + q * (T(-0.75) + q * (T(0.3) - q * T(1.0 / 24.0)))) - T(1.0 / 60.0));
}
template <typename T>
__device__ __forceinline__ T grav_psi_plus_mq(T q)
{
    if (q >= T(2)) return T(0);
    const T q2 = q * q;
    T psi;
    if (q < T(1)) psi = q2 * (T(2.0 / 3.0) + q2 * (T(-0.3) + T(0.1) * q)) - T(1.4);
    else psi = q2 * (T(4.0 / 3.0) + q * (T(-1) + q * (T(0.3) - q * T(1.0 / 30.0)))) + T(1.0 / 15.0) / q - T(1.6);
    return psi + (q > T(0) ? grav_mass(q) / q : T(0));
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
template <typename T>
__device__ __forceinline__ T sub_rn(T a, T b);
template <>
__device__ __forceinline__ float sub_rn<float>(float a, float b) { return __fsub_rn(a, b); }
template <>
__device__ __forceinline__ double sub_rn<double>(double a, double b) { return __dsub_rn(a, b); }
template <typename T>
__device__ __forceinline__ T fma_rn(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
// (The force pass evaluates a pair's terms at several inlined call sites;
// spelling every operation that feeds m_i a_i with these intrinsics keeps the
// compiler from contracting them differently at different sites, so both
// particles of a pair get the same bits.)

template <typename T>
__device__ __forceinline__ T Kern<SPH_KERNEL_M4>::df(T q)
{
    const T t = q < T(2) ? sub_rn(T(2), q) : T(0);
    const T df2 = mul_rn(mul_rn(T(-0.75), t), t);
    const T df1 = mul_rn(q, fma_rn(T(2.25), q, T(-3)));
    return q < T(1) ? df1 : df2;
}

template <typename T>
__device__ __forceinline__ T Kern<SPH_KERNEL_M6>::df(T q)
{
    const T a = q < T(3) ? sub_rn(T(3), q) : T(0);
    const T c = q < T(2) ? sub_rn(T(2), q) : T(0);
    const T a2 = mul_rn(a, a), c2 = mul_rn(c, c);
    const T df2 = fma_rn(T(30), mul_rn(c2, c2), mul_rn(T(-5), mul_rn(a2, a2)));
    const T df1 = mul_rn(q, fma_rn(mul_rn(q, q), fma_rn(T(-50), q, T(120)), T(-120)));
    return q < T(1) ? df1 : df2;
}

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
    T L[3], Li[3];             // box lengths and their inverses (periodic wraps)
    T C[3];                    // centre of the query leaf's box (in its frame)
    float ihl[3];              // 2 / box length
    float thr[3];              // candidate extents (packed units) from which a leaf pair is ambiguous
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

// Periodic minimum images.  A pair vector is formed as (o_i - o_j) - D from
// the particles' offsets o from their leaves' reference points (at most E_A,
// E_B in magnitude) and the minimum-image shift D of the two reference
// points, so it is the minimum image of every pair within R unless
// E_A + E_B + R >= L/2 ("ambiguous" leaf pairs: few particles per box length,
// or leaves that span much of a thin box).  The particles of an ambiguous
// candidate leaf are moved, as they are staged, to their image nearest to
// the centre of the query leaf's box; the staged vectors are then minimum
// images unless W_A/2 + R >= L/2 (W_A the query box's width), in which case
// each pair vector is wrapped as well.  The force pass wraps the pair
// vectors of ambiguous leaf pairs it evaluates, r - L rint(r / L), which is
// odd in r: the vectors of i-j and j-i stay exact negatives.  The box
// lengths sit in the warp's scratch.  All of this runs in the launches that
// serve the wrap list: the common launches test each candidate leaf as they
// walk (per axis, from the extents the leaf pass packs into the leaves'
// boxes) and at the first ambiguous pair put the query leaf, with nothing
// written yet, on that list.
__device__ __forceinline__ float half_box(const PhysParams &ph)
{
    return 0.5f * fminf(ph.box_len_f[0], fminf(ph.box_len_f[1], ph.box_len_f[2])) * 0.99999f;
}

template <typename T>
__device__ __forceinline__ T box_L(const PhysParams &ph, int a);
template <>
__device__ __forceinline__ float box_L<float>(const PhysParams &ph, int a) { return ph.box_len_f[a]; }
template <>
__device__ __forceinline__ double box_L<double>(const PhysParams &ph, int a) { return ph.box_len[a]; }
template <typename T>
__device__ __forceinline__ T box_Li(const PhysParams &ph, int a);
template <>
__device__ __forceinline__ float box_Li<float>(const PhysParams &ph, int a) { return ph.box_inv_f[a]; }
template <>
__device__ __forceinline__ double box_Li<double>(const PhysParams &ph, int a) { return ph.box_inv[a]; }

// lanes 0..2 copy the box lengths and the query box's centre into the
// warp's scratch
template <typename T, typename V>
__device__ __forceinline__ void load_box(StageScratch<T> &sc, const PhysParams &ph, const V &lo, const V &hi)
{
    const int lane = threadIdx.x & 31;
    if (lane < 3) {
        sc.L[lane] = box_L<T>(ph, lane);
        sc.Li[lane] = box_Li<T>(ph, lane);
        sc.C[lane] = T(0.5) * (lane == 0 ? lo.x + hi.x : lane == 1 ? lo.y + hi.y : lo.z + hi.z);
        sc.ihl[lane] = 2.f * ph.box_inv_f[lane];
    }
    __syncwarp();
}

// A leaf pair (A, B) is ambiguous for pairs within R when on some axis
// E_A + E_B + R >= L/2, from the leaves' packed offset extents (slo.w, in
// units of L/2046).  set_thr (lanes 0..2) stores, for query leaf A and reach
// R, the extent of B from which that holds; ambiguous(E_B) tests it.
template <typename T>
__device__ __forceinline__ void set_thr(StageScratch<T> &sc, float ea, float R)
{
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (lane < 3)
        sc.thr[lane] = 1023.f * (0.99999f - R * sc.ihl[lane]) - (float)((__float_as_uint(ea) >> (10 * lane)) & 1023u);
    __syncwarp();
}
template <typename T>
__device__ __forceinline__ bool ambiguous(float eb, const StageScratch<T> &sc)
{
    const unsigned b = __float_as_uint(eb);
    return (float)(b & 1023u) >= sc.thr[0] || (float)((b >> 10) & 1023u) >= sc.thr[1] ||
           (float)((b >> 20) & 1023u) >= sc.thr[2];
}

// largest h (plo.w) and largest leaf offset extent (slo.w) of a problem,
// carried up to its top nodes
__device__ __forceinline__ void problem_top_max(const BatchView &b, const ProbDyn &dy, float &hmax, float &extmax)
{
    const int lane = threadIdx.x & 31, top = dy.top_level;
    float h = 0.f, e = 0.f;
    if (lane < dy.node_cnt[top]) {
        const NodeBox &nb = b.nodes[top][dy.node_off[top] + lane];
        h = nb.plo.w;
        e = nb.slo.w;
    }
    hmax = warp_max(h);
    extmax = warp_max(e);
}

// half of the query box's largest width
template <typename V>
__device__ __forceinline__ float half_width(const V &lo, const V &hi)
{
    return 0.5f * (float)fmax(hi.x - lo.x, fmax(hi.y - lo.y, hi.z - lo.z)) * 1.00001f;
}

// minimum image of a pair vector
template <typename T>
__device__ __forceinline__ void wrap3s(const StageScratch<T> &sc, T &x, T &y, T &z)
{
    x = fma_rn(-sc.L[0], rint(mul_rn(x, sc.Li[0])), x);
    y = fma_rn(-sc.L[1], rint(mul_rn(y, sc.Li[1])), y);
    z = fma_rn(-sc.L[2], rint(mul_rn(z, sc.Li[2])), z);
}

// move staged point q to its periodic image nearest to c (unchanged when q
// is already that image)
template <typename T, typename V>
__device__ __forceinline__ void wrap_near(const StageScratch<T> &sc, V &q, T cx, T cy, T cz)
{
    q.x = fma_rn(-sc.L[0], rint(mul_rn(sub_rn(q.x, cx), sc.Li[0])), q.x);
    q.y = fma_rn(-sc.L[1], rint(mul_rn(sub_rn(q.y, cy), sc.Li[1])), q.y);
    q.z = fma_rn(-sc.L[2], rint(mul_rn(sub_rn(q.z, cz), sc.Li[2])), q.z);
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
// keep(q, k) sees them (k: the lane of the particle's leaf; keep may move q
// to another periodic image).  group(has, B, stB, D) runs on every lane once
// per call (lane k: candidate leaf first + k if has); store(slot, q, k, idx)
// writes a kept particle (idx: its index within its leaf).
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
    // the particles are loaded one chunk of 32 ahead: a chunk's load (an L2
    // round trip) overlaps the filtering, storing and flushing of the chunk
    // before it (flush() leaves the scratch and the loaded arrays alone)
    V qn{};
    int kn = 0, idxn = 0;
    if (lane < tot) {
        kn = owner_of(sc, lane);
        idxn = lane - sc.first[kn];
        qn = load(sc.start[kn] + idxn);
    }
    for (int e0 = 0; e0 < tot; e0 += 32) {
        const int e = e0 + lane;
        V q = qn;
        const int k = kn, idx = idxn;
        if (e + 32 < tot) {
            kn = owner_of(sc, e + 32);
            idxn = e + 32 - sc.first[kn];
            qn = load(sc.start[kn] + idxn);
        }
        if (nbuf > CH - 32) flush();
        bool ok = false;
        if (e < tot) {
            q.x += sc.dx[k];
            q.y += sc.dy[k];
            q.z += sc.dz[k];
            ok = keep(q, k);
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

template <typename T, int LPP, bool UM, int K>
struct DCfg {
    using V = typename Vec4<T>::type;
    // list entries per lane: room for ~2x the mean neighbour count per
    // particle within the list radius (M4 at eta = 1.2: ~63; M6 at eta = 1.0:
    // ~123, served by 2 or more lanes per particle)
    static constexpr int LCAP = K == SPH_KERNEL_M6 ? (LPP <= 2 ? 96 : LPP == 4 ? 64 : 32)
                                                   : LPP == 1 ? SPH_DENS_LCAP1 : LPP == 2 ? 64 : LPP == 4 ? 40 : 24;
    static constexpr int CH = SPH_DENS_CH;
    static constexpr int WPB = 4;
    static constexpr int MINB = LPP == 1 ? SPH_DENS_MINB1 : SPH_DENS_MINB;  // blocks per SM the registers allow
    static constexpr int LW = UM ? 1 : 2;  // list words per entry: r^2 (and m_j unless masses are equal)
    static constexpr size_t scratch = (sizeof(StageScratch<T>) + 31) & ~(size_t)31;
    static constexpr size_t per_warp = CH * sizeof(V) + (size_t)LCAP * 32 * LW * sizeof(T) + scratch;
    static constexpr size_t smem = WPB * per_warp;
};

// Block-step tasks (k0 >= 0): the lane group pp serves the (k0 + pp)-th
// particle of the leaf whose step ends now; returns its position in the
// leaf and whether there is one.  k0 < 0: the whole leaf, position pp.
template <typename T>
__device__ __forceinline__ bool task_member(const BatchView &b, int st, int nA, int k0, int pp, int &pos)
{
    const int lane = threadIdx.x & 31;
    if (k0 < 0) {
        pos = pp;
        return pp < nA;
    }
    const unsigned dm = __ballot_sync(FULL, lane < nA && ((const T *)b.slev)[st + (lane < nA ? lane : 0)] > T(0));
    const int ord = k0 + pp;
    const bool on = ord < __popc(dm);
    pos = on ? (int)__fns(dm, 0u, ord + 1) : 0;
    return on;
}

// A task's position box (its particles only) in absolute float coordinates,
// from their offsets x (staged, leaf frame) as the leaf build forms the
// leaf's: each offset widened for its one rounding, plus the leaf's
// reference point rounded down (up).  w of plo: hmax.
__device__ __forceinline__ float task_widen_dn(float v) { return __fsub_rd(v, fabsf(v) * 2.4e-7f); }
__device__ __forceinline__ float task_widen_up(float v) { return __fadd_ru(v, fabsf(v) * 2.4e-7f); }

template <typename V>
__device__ __forceinline__ void task_box(const BatchView &b, int leaf, const V &x, bool on, float hmax, NodeBox &box)
{
    const float o[3] = {(float)x.x, (float)x.y, (float)x.z};
    float lo[3], hi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = warp_min(on ? task_widen_dn(o[a]) : INFINITY);
        hi[a] = warp_max(on ? task_widen_up(o[a]) : -INFINITY);
    }
    const float *cf = b.leaf_cf + 6LL * leaf;  // reference point rounded down (0..2) and up (3..5)
    box.plo = make_float4(__fadd_rd(cf[0], lo[0]), __fadd_rd(cf[1], lo[1]), __fadd_rd(cf[2], lo[2]), hmax);
    box.phi = make_float4(__fadd_ru(cf[3], hi[0]), __fadd_ru(cf[4], hi[1]), __fadd_ru(cf[5], hi[2]), box.phi.w);
}

// Outputs of the density solve for sorted particle s (one lane per particle).
template <typename T>
__device__ __forceinline__ void density_epilogue(const BatchView &b, const ProbStatic &ps, long long s,
                                                 typename Vec4<T>::type pi, T h, T S0, T S1, int use_pred,
                                                 T sigma, T Z = T(0))
{
    using V = typename Vec4<T>::type;
    const PhysParams &ph = ps.ph;
    long long g = b.perm[s];
    long long i = g - ps.base;
    double u = use_pred ? b.up[g] : ps.u[i];
    double v[3] = {use_pred ? b.vpx[g] : ps.vx[i], use_pred ? b.vpy[g] : ps.vy[i],
                   use_pred ? b.vpz[g] : ps.vz[i]};
    T hinv, rho, omega, P, c;
    // block time-steps: a particle whose step does not end now keeps the h,
    // rho, Omega, P and c of its last solve (restaged here for the force pass)
    const bool keep = b.block_on && ((const T *)b.slev)[s] < T(0);
    if (keep) {
        h = (T)ps.h[i];
        hinv = T(1) / h;
        rho = (T)ps.rho[i];
        omega = (T)ps.omega[i];
        P = (T)ps.P[i];
        c = (T)ps.c[i];
    } else {
        hinv = T(1) / h;
        T hinv3 = hinv * hinv * hinv;
        rho = sigma * S0 * hinv3;
        T drho = -sigma * hinv3 * hinv * (T(3) * S0 + S1);
        omega = T(1) + h / (T(3) * rho) * drho;
        if (ph.eos == SPH_EOS_ISOTHERMAL) {
            c = (T)ph.cs_iso;
            P = c * c * rho;
        } else {
            P = (T)(ph.gamma - 1.0) * rho * (T)u;
            c = sqrt((T)ph.gamma * P / rho);
        }
    }
    T A = P / (omega * rho * rho);
    b.sh[s] = (double)h;
    b.hf[s] = to_float_ru(h);
    b.srho[s] = (double)rho;
    b.somega[s] = (double)omega;
    b.sP[s] = (double)P;
    b.sc[s] = (double)c;
    if (!keep) {
        ps.h[i] = (double)h;
        ps.rho[i] = (double)rho;
        ps.omega[i] = (double)omega;
        ps.P[i] = (double)P;
        ps.c[i] = (double)c;
    }
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
    if (ph.av_switch)  // viscosity switch (Morris & Monaghan's alpha is kicked and predicted like u)
        ((T *)b.sal)[s] = (T)(use_pred && ph.av_switch == SPH_AV_MORRIS_MONAGHAN ? b.ap[g] : ps.alpha[i]);
    if (ph.av_switch == SPH_AV_CULLEN_DEHNEN) ((T *)b.scd)[s] = (T)ps.dalpha[i];  // the previous div v
    // gravity: zeta = dh/drho sum_j m_j dphi/dh = Z / (3 rho h) (Z = sum_j m_j (psi + M/q)),
    // kept as the weight G zeta / (2 Omega) of the force pass's zeta term
    if (ph.gravity) {
        if (keep) {
            ((T *)b.szg)[s] = (T)b.bzeta[g];
        } else {
            const T wz = (T)(0.5 * ph.G) * Z / (T(3) * rho * h * omega);
            ((T *)b.szg)[s] = wz;
            if (b.bzeta) b.bzeta[g] = (double)wz;  // block-step contexts keep it for the ticks that do not solve
        }
    }
    if (!(isfinite((double)rho) && isfinite((double)omega) && isfinite((double)P)))
        atomicOr(&ps.diag->status, ST_NONFINITE);
}

// One query leaf of the density pass.  WRAP: pair vectors are wrapped to
// the minimum image where they may miss it (see the wrap helpers).  Returns
// false, having written nothing, when the plain variant meets an ambiguous
// leaf pair.
template <typename T, int LPP, bool UM, int K, bool WRAP>
__device__ __forceinline__ bool density_leaf(const BatchView &b, int leaf, int k0, unsigned char *mine, int use_pred)
{
    using C = DCfg<T, LPP, UM, K>;
    using KF = Kern<K>;
    constexpr float KR_f = (float)KF::R;        // support radius in units of h
    constexpr float KR_cap = KR_f * 1.0001f;    // walk radius -> largest h it covers
    const T sigma = T(KF::sigma);
    using V = typename C::V;
    const int lane = threadIdx.x & 31;
    V *cand = reinterpret_cast<V *>(mine);
    T *lr = reinterpret_cast<T *>(mine + C::CH * sizeof(V));  // r_ij^2 per entry
    T *lm = lr + C::LCAP * 32;  // used only when masses differ
    StageScratch<T> &sc = *reinterpret_cast<StageScratch<T> *>(lr + C::LCAP * 32 * C::LW);
    const int pp = lane / LPP, sub = lane % LPP;
    const V *pm = (const V *)b.pm;
    const int p = b.leaf_pid[leaf];
    const ProbStatic &ps = b.prob[p];
    const T mu_all = (T)ps.m_uniform;
    const int st = b.leaf_start[leaf], nA = b.leaf_start[leaf + 1] - st;
    const ProbDyn &dy = b.dyn[p];
    const PhysParams &ph = ps.ph;
    NodeBox boxA = b.nodes[0][leaf];
    int pos;
    const bool active = task_member<T>(b, st, nA, k0, pp, pos);
    const long long s = st + (active ? pos : 0);
    const V pi = pm[s];
    const T mi = pi.w;
    // a block-step task walks from the box of its own particles (the others
    // of the leaf keep their last solve, restaged by k_block_restage)
    if (k0 >= 0) task_box(b, leaf, pi, active, boxA.plo.w, boxA);
    V flo, fhi;
    frame_box<V, T>(pi, active, flo, fhi);
    const float halfL = ph.periodic ? half_box(ph) : INFINITY;
    const T eta3 = (T)(ph.eta * ph.eta * ph.eta);
    const T tol = (T)ph.h_tol;
    const int maxit = ph.h_max_iter;
    const double Lmin = ph.periodic ? fmin(ph.box_len[0], fmin(ph.box_len[1], ph.box_len[2])) : INFINITY;
    const T hbox = (T)(Lmin / (2.0 * KF::R));  // support beyond half the box: SPH_EBOX
    T h = active ? (T)b.sh[s] : T(1);
    // the leaf pass predicted this particle's sphere from the same start
    const float hpred = active ? __fmul_ru(kHPredict, __double2float_ru(b.sh[s])) : 0.f;
    if (active && !(h > T(0))) {
        double ext = ph.periodic ? fmax(ph.box_len[0], fmax(ph.box_len[1], ph.box_len[2])) : 1.0 / dy.dom_inv;
        h = (T)(ph.eta * cbrt(ext * ext * ext / (double)(ps.n > 0 ? ps.n : 1)));
    }
    if (ph.periodic) load_box(sc, ph, flo, fhi);
    bool to_wrap = false;  // (plain variant) met an ambiguous leaf pair: the wrapping variant takes the leaf
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
    const bool record = k0 < 0 && ps.diag->reuse_hold == 0;
    int ng = 0, g_first = 0;
    unsigned g_mask = 0u;
    float Rq_last = 0.f;
    for (int attempt = 0;; ++attempt) {
        const T hs = h * (T)kListMargin;
        float Rq = warp_max((active && !fail) ? __fmul_ru(KR_f, (float)hs) : 0.f) * 1.0001f;
        const T R2 = (T(KF::R) * hs) * (T(KF::R) * hs);
        Rq_last = Rq;
        if (ph.periodic) set_thr(sc, boxA.slo.w, Rq);
        const bool wrap2 = WRAP && half_width(flo, fhi) + Rq >= halfL;  // staged vectors may still need a wrap
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
                    if (wrap2) wrap3s<T>(sc, dx, dyy, dz);
                    T r2 = dx * dx + dyy * dyy + dz * dz;
                    if (active && !fail && r2 < R2) {
                        if (cnt < C::LCAP) {
                            lr[cnt * 32 + lane] = r2;  // (its root where the lists are read: off the append path)
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
                    T r = T(0), mj = T(0);  // (r: r_ij^2)
                    if (k < nbuf) {
                        V c = cand[k];
                        T dx = pi.x - c.x, dyy = pi.y - c.y, dz = pi.z - c.z;
                        if (wrap2) wrap3s<T>(sc, dx, dyy, dz);
                        T r2 = dx * dx + dyy * dyy + dz * dz;
                        hit = active && !fail && r2 < R2;
                        r = r2;
                        mj = c.w;
                    }
                    const unsigned gm = (__ballot_sync(FULL, hit) >> (pp * LPP)) & (LPP == 32 ? FULL : (1u << (LPP & 31)) - 1u);
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
                // candidate leaves that form an ambiguous pair with A (periodic)
                const unsigned am =
                    ph.periodic ? __ballot_sync(FULL, ((gm >> lane) & 1u) && ambiguous(b.nodes[0][first + lane].slo.w, sc))
                                : 0u;
                if (!WRAP && am) to_wrap = true;
                if (!WRAP && to_wrap) return;
                stage_group<T, C::CH>(
                    b, leaf, gm, first, ph, nbuf, sc, [](bool, int, int, T, T, T) {},
                    [&](int j) { return pm[j]; },
                    [&](V &q, int k) {
                        if (WRAP && ((am >> k) & 1u)) wrap_near<T>(sc, q, sc.C[0], sc.C[1], sc.C[2]);
                        return box_dist2<T>(q, flo, fhi) < Rq2;
                    },
                    [&](int slot, const V &q, int, int) { cand[slot] = q; }, flush);
            });
        flush();
        if (!WRAP && to_wrap) break;
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
                    T q = sqrt(lr[e * 32 + lane]) * hinv;
                    T mj = UM ? mu_all : lm[e * 32 + lane];
                    T f, df;
                    KF::fdf(q, f, df);
                    S0 += mj * f;
                    S1 += mj * q * df;
                    nn += q < T(KF::R);
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
                T rho = sigma * S0 * hinv3;
                T drho = -sigma * hinv3 * hinv * (T(3) * S0 + S1);
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
    if (!WRAP && to_wrap) return false;  // nothing written yet
    // record the last walk's groups for the force pass (lane 0 reserves
    // pool space); not recorded: the force pass walks for this leaf (a
    // block-step task records nothing: its force pass always walks)
    if (k0 < 0) {
        int base = 0;
        if (lane == 0) {
            base = record && ng <= kMaxLeafGroups ? atomicAdd(&b.counters[kPoolCounter], ng) : -1;
            const bool fits = base >= 0 && (long long)base + ng <= b.group_cap;
            b.leaf_gofs[leaf] = fits ? base : 0;
            b.leaf_ngroups[leaf] = fits ? ng : -1;
            b.leaf_hcap[leaf] = Rq_last / KR_cap;
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
                T q = sqrt(lr[e * 32 + lane]) * hinv;
                T mj = UM ? mu_all : lm[e * 32 + lane];
                T f, df;
                KF::fdf(q, f, df);
                R0 += mj * f;
                R1 += mj * q * df;
                rn += q < T(KF::R);
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
    T Z = T(0);  // gravity (wrap-list launch): sum_j m_j (psi + M/q) at the final h
    if (WRAP && ph.gravity) {
        if (fin) {
            const T hinv = T(1) / h;
            for (int e = 0; e < cnt; ++e)
                Z += (UM ? mu_all : lm[e * 32 + lane]) * grav_psi_plus_mq(sqrt(lr[e * 32 + lane]) * hinv);
        }
        Z = group_sum<LPP>(Z);
    }
    if (fin && sub == 0) {
        density_epilogue<T>(b, ps, s, pi, h, S0, S1, use_pred, sigma, Z);
        if (noconv && !(b.block_on && ((const T *)b.slev)[s] < T(0))) {  // (a kept solve is not this one)
            atomicOr(&ps.diag->status, ST_NOCONV);
            atomicAdd(&ps.diag->unconverged, 1);
        }
        // the recorded candidate groups cover this particle's pairs only
        // if its final h stays within the walk radius and its prediction
        const float hf = to_float_ru(h);
        if (hf > hpred || hf > Rq_last / KR_cap) atomicOr(&b.dyn[p].lists_stale, 1);
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
    return true;
}

// WRAP: the launch that serves the wrap list (leaves whose pair vectors may
// miss the minimum image); the other launch puts them there.
template <typename T, int LPP, bool UM, int K, bool WRAP>
__global__ void __launch_bounds__(DCfg<T, LPP, UM, K>::WPB * 32, DCfg<T, LPP, UM, K>::MINB) k_density(BatchView b, int use_pred)
{
    using C = DCfg<T, LPP, UM, K>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem + wib * C::per_warp;
    // block-step ticks: the wrap-list launch serves the tick's tasks (leaf <<
    // 5 | first due ordinal) directly; the common launch does not run
    const bool tasks = WRAP && b.block_on && b.block_tasks;
    const int nleaf = tasks ? b.counters[kBlockTasks] : WRAP ? b.counters[kDensWrapList] : b.counters[0];
    const int cls = lpp_log2(LPP) + (UM ? 4 : 0) + 8 * K;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[(WRAP ? kDensityWrapCounter : kDensityCounter) + cls], 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nleaf) break;
        if (WRAP) item = tasks ? b.btask[item] : b.wrap_list[item];
        const int leaf = tasks ? item >> 5 : item, k0 = tasks ? item & 31 : -1;
        const ProbStatic &ps = b.prob[b.leaf_pid[leaf]];
        if ((tasks ? b.block_lanes : ps.lpp) != LPP || (ps.uniform_m != 0) != UM || ps.ph.kernel != K) continue;
        if (!WRAP && ps.ph.gravity) {  // gravity's zeta runs in the wrap-list launch only
            if (lane == 0) b.wrap_list[atomicAdd(&b.counters[kDensWrapList], 1)] = item;
            continue;
        }
        if (!density_leaf<T, LPP, UM, K, WRAP>(b, leaf, k0, mine, use_pred) && lane == 0) {
            b.wrap_list[atomicAdd(&b.counters[kDensWrapList], 1)] = item;
            atomicAdd(&ps.diag->wrap_leaves, 1);
        }
    }
}

// Slow path: one warp per particle for the particles whose per-lane lists in
// k_density overflowed or outgrew their radius.  The warp stages the leaf's
// candidate leaves in groups, as k_density does, gathers the particle's
// neighbours (within R_K h x 1.1) into a list spread over its 32 lanes (up to
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
        const int kk = ph.kernel;
        const T KR = (T)ph.kr, sigma = (T)kern_sigma(kk);
        const bool per = ph.periodic != 0;  // (every staged candidate moves to its image nearest s)
        if (per) load_box(sc, ph, pi, pi);
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
                        [&](int j) { return pm[j]; },
                        [&](V &q, int) {
                            if (per) wrap_near<T>(sc, q, pi.x, pi.y, pi.z);  // then pi - q is the minimum image
                            return box_dist2<T>(q, pi, pi) < Rq2;
                        },
                        [&](int slot, const V &q, int, int) { cand[slot] = q; }, flush);
                });
            flush();
        };
        bool direct = false;
        T hs = T(0);
        int cnt = 0;
        auto build = [&]() {
            hs = h * (T)kFbMargin;
            const T R2 = (KR * hs) * (KR * hs);
            cnt = 0;
            bool ovf = false;
            visit_all(__fmul_ru(ph.kr_f, (float)hs) * 1.0001f, [&](T r2, T mj) {
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
        T Z = T(0);  // gravity: sum_j m_j (psi + M/q)
        auto sums = [&](T hh) {
            S0 = T(0);
            S1 = T(0);
            Z = T(0);
            nn = 0;
            const T hinv = T(1) / hh;
            if (!direct) {
                for (int e = 0; e < cnt; ++e) {
                    T f, df, qq = fr[e * 32 + lane] * hinv;
                    kern_fdf(kk, qq, f, df);
                    T mj = fm[e * 32 + lane];
                    S0 += mj * f;
                    S1 += mj * qq * df;
                    if (ph.gravity) Z += mj * grav_psi_plus_mq(qq);
                    nn += qq < KR;
                }
            } else {
                const T R2 = (KR * hh) * (KR * hh);
                visit_all(__fmul_ru(ph.kr_f, (float)hh) * 1.0001f, [&](T r2, T mj) {
                    if (r2 < R2) {
                        T f, df, qq = sqrt(r2) * hinv;
                        kern_fdf(kk, qq, f, df);
                        S0 += mj * f;
                        S1 += mj * qq * df;
                        if (ph.gravity) Z += mj * grav_psi_plus_mq(qq);
                        ++nn;
                    }
                });
            }
            S0 = warp_sum(S0);
            S1 = warp_sum(S1);
            Z = warp_sum(Z);
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
            T rho = sigma * S0 * hinv3;
            T drho = -sigma * hinv3 * hinv * (T(3) * S0 + S1);
            bool c = nr_update(h, lo, hi, rho, drho, pi.w, eta3, tol);
            if ((double)h > Lmin / (2.0 * ph.kr)) {
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
            density_epilogue<T>(b, ps, s, pi, h, S0, S1, use_pred, sigma, Z);
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
    static constexpr int MINB = LPP == 1 ? SPH_FORCE_MINB1 : SPH_FORCE_MINB;  // blocks per SM the registers allow
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

// conductivity signal speed (Sec. 2.1.1): Wadsley |v_ij . r_hat| (gm1 = 0)
// or Price sqrt(|P_i - P_j| / rho_bar), P = gm1 rho u from the staged
// (A, rho, m, u) vectors
template <typename T, typename V>
__device__ __forceinline__ T ac_speed(T vdr, const V &ti, const V &tj, T gm1, T rhob_inv)
{
    if (gm1 > T(0)) return sqrt(gm1 * fabs(ti.y * ti.w - tj.y * tj.w) * rhob_inv);
    return fabs(vdr);
}

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

// One query leaf of the force pass.  Rall: the reach of the problem's pairs,
// R_K x its largest h (periodic problems); WRAP: the leaf is on the wrap
// list and its pair vectors are wrapped where they may miss the minimum
// image.  Returns false (writing nothing) when the plain launch meets an
// ambiguous leaf pair.
template <typename T, int LPP, int K, bool WRAP, bool CD>
__device__ __forceinline__ bool force_leaf(const BatchView &b, int leaf, int k0, unsigned char *mine, float Rall)
{
    using C = FCfg<T, LPP>;
    using KF = Kern<K>;
    constexpr float KR_f = (float)KF::R;
    using V = typename C::V;
    const int lane = threadIdx.x & 31;
    V *cand = reinterpret_cast<V *>(mine);  // staged (offset + leaf shift, 1/h)
    V *table = cand + C::CH;                // per candidate leaf: (leaf shift, first sorted index)
    StageScratch<T> &sc = *reinterpret_cast<StageScratch<T> *>(table + C::TAB);
    unsigned short *code = reinterpret_cast<unsigned short *>(mine + (C::CH + C::TAB) * sizeof(V) + C::scratch);
    unsigned short *lst = code + C::CH;
    const int pp = lane / LPP, sub = lane % LPP;
    const unsigned below = (1u << lane) - 1u;
    const V *gph = (const V *)b.ph, *gvc = (const V *)b.vc, *gth = (const V *)b.th;
    const int p = b.leaf_pid[leaf];
    const ProbStatic &ps = b.prob[p];
    const int st = b.leaf_start[leaf], nA = b.leaf_start[leaf + 1] - st;
    const ProbDyn &dy = b.dyn[p];
    const PhysParams &ph = ps.ph;
    NodeBox boxA = b.nodes[0][leaf];
    int pos;
    const bool active = task_member<T>(b, st, nA, k0, pp, pos);
    const int s = st + (active ? pos : 0);
    const V xi = gph[s], vi = gvc[s], ti = gth[s];
    // a block-step task walks from the box of its own particles, whose
    // largest h sets the gather reach
    if (k0 >= 0) task_box(b, leaf, xi, active, warp_max(active ? b.hf[s] : 0.f), boxA);
    const T alpha = (T)ph.alpha_av, beta = (T)ph.beta_av, aac = (T)ph.alpha_ac;
    // Price conductivity: v'_sig = sqrt(|P_i - P_j| / rho_bar) with P = (gamma - 1) rho u
    // (adiabatic); 0 selects Wadsley's |v_ij . r_hat|
    const T gm1_price = WRAP && ph.ac_signal == SPH_AC_PRICE ? (T)(ph.gamma - 1.0) : T(0);
    const bool adi = ph.eos == SPH_EOS_ADIABATIC;
    const T sigma = T(KF::sigma);
    const T hi2 = mul_rn(xi.w, xi.w), hi4 = mul_rn(hi2, hi2);
    // viscosity switch (served by the wrap-list launch): alpha_ij = (alpha_i + alpha_j)/2,
    // beta_ij = beta/alpha_max alpha_ij
    const bool sw = WRAP && ph.av_switch != 0;
    const T* __restrict__ sal = (const T *)b.sal;
    const T alpha_i = sw ? sal[s] : alpha, bratio = (T)ph.beta_ratio;
    T dvs = T(0);  // sum_j m_j v_ij . grad_i W(h_i) (switch: div v)
    // Cullen & Dehnen (its own launch, so that the other options keep their
    // registers): the gradient sums G_ab = sum_j m_j v_ij,a grad_i,b W(h_i)
    // and the signed density sum_j sign(D_j) m_j W(r_ij, h_i)
    constexpr bool cdw = CD;
    const T* __restrict__ scd = (const T *)b.scd;
    T cg[9] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    T cr = T(0);
    // gravity (wrap-list launch): the zeta term of Eq. SPHSELFGRAV has the pressure
    // term's form, with P/(Omega rho^2) + G zeta/(2 Omega) per particle
    const bool grav = WRAP && ph.gravity != 0;
    const T* __restrict__ szg = (const T *)b.szg;
    const T Ai_g = grav ? add_rn(ti.x, szg[s]) : ti.x;
    // block time-steps (wrap-list launch): only the particles whose step ends
    // now (staged level + 1 > 0) take forces; they record the largest level
    // among their neighbours and lift inactive neighbours more than
    // block_gap levels below them (Saitoh & Makino's limiter)
    const bool blk = WRAP && b.block_on;
    const T* __restrict__ slev = (const T *)b.slev;
    const T li1 = blk ? slev[s] : T(0);
    const bool due = blk ? (active && li1 > T(0)) : active;
    if (blk && !__any_sync(FULL, due)) return true;  // no particle of this leaf ends its step now
    const T lgap = (T)ph.block_gap;
    T mlev = T(0);
    TwoSumAcc<T> ax{T(0), T(0)}, ay{T(0), T(0)}, az{T(0), T(0)};
    T du = T(0), vs = T(-1);
    int pairs = 0, tested = 0;
    const float R = __fmul_ru(KR_f, boxA.plo.w) * 1.0001f;
    const T RA2 = (T)R * (T)R;
    V flo, fhi;
    frame_box<V, T>(xi, active, flo, fhi);
    const float halfL = ph.periodic ? half_box(ph) : INFINITY;
    if (ph.periodic) {
        load_box(sc, ph, flo, fhi);
        set_thr(sc, boxA.slo.w, Rall);
    }
    const bool wrap2 = WRAP && half_width(flo, fhi) + Rall >= halfL;  // staged vectors may still need a wrap
    bool to_wrap = false;  // (plain variant) met an ambiguous leaf pair: the wrapping variant takes the leaf
    int nbuf = 0, cnt = 0, ntab = 0, tA = -1;
    unsigned gmask = 0u, am = 0u;
    // table entry of a candidate leaf: its shift and first sorted index,
    // stored as ~index for an ambiguous leaf pair (whose pair vectors the
    // evaluation wraps)
    auto fetch = [&](int e, V &tb, V &a0, V &a1, V &a2, int &j) {
        const unsigned cd = lst[e * 32 + lane];
        tb = table[cd >> 5];
        const int tv = t_as_bits(tb.w);
        j = (WRAP && tv < 0 ? ~tv : tv) + (int)(cd & 31u);
        a0 = ld_ro(gph + j);
        a1 = ld_ro(gvc + j);
        a2 = ld_ro(gth + j);
    };
    auto eval_lists = [&]() {
        __syncwarp();
        for (int e = 0; e < cnt; ++e) {
            V tb, a0, a1, a2;
            int j;
            fetch(e, tb, a0, a1, a2, j);
            // r_ij = (o_i - o_j) - D_AB: IEEE subtraction is sign-symmetric and
            // D_BA = -D_AB exactly, so particle j forms exactly -r_ij
            T rx = sub_rn(sub_rn(xi.x, a0.x), tb.x), ry = sub_rn(sub_rn(xi.y, a0.y), tb.y),
              rz = sub_rn(sub_rn(xi.z, a0.z), tb.z);
            if (WRAP && t_as_bits(tb.w) < 0) wrap3s<T>(sc, rx, ry, rz);
            // every operation below up to m_i a_i with fixed rounding (odd
            // in r where it must be: particle j forms exactly the negatives)
            const T r2 = fma_rn(rz, rz, fma_rn(ry, ry, mul_rn(rx, rx)));
            const T rinv = rsqrt_t(r2);
            const T r = mul_rn(r2, rinv);
            const T qi = mul_rn(r, xi.w), qj = mul_rn(r, a0.w);
            const T hj2 = mul_rn(a0.w, a0.w);
            const T gi = mul_rn(mul_rn(sigma, KF::df(qi)), hi4);
            const T gj = mul_rn(mul_rn(sigma, KF::df(qj)), mul_rn(hj2, hj2));
            const T pterm = add_rn(mul_rn(Ai_g, gi), mul_rn(grav ? add_rn(a2.x, szg[j]) : a2.x, gj));
            const T vx = sub_rn(vi.x, a1.x), vy = sub_rn(vi.y, a1.y), vz = sub_rn(vi.z, a1.z);
            const T vdr = mul_rn(fma_rn(vz, rz, fma_rn(vy, ry, mul_rn(vx, rx))), rinv);
            const T mu = vdr < T(0) ? vdr : T(0);
            const T rhob_inv = fast_div(T(2), add_rn(ti.y, a2.y));
            const T gbar = mul_rn(T(0.5), add_rn(gi, gj));
            T al = alpha, be = beta;
            if (sw) {
                al = mul_rn(T(0.5), add_rn(alpha_i, sal[j]));
                be = mul_rn(bratio, al);
            }
            dvs += a2.z * vdr * gi;  // (div v: the switch's source, and the next step's h prediction)
            if (cdw) {
                const T mg = a2.z * gi * rinv;
                cg[0] += mg * vx * rx;
                cg[1] += mg * vx * ry;
                cg[2] += mg * vx * rz;
                cg[3] += mg * vy * rx;
                cg[4] += mg * vy * ry;
                cg[5] += mg * vy * rz;
                cg[6] += mg * vz * rx;
                cg[7] += mg * vz * ry;
                cg[8] += mg * vz * rz;
                if (qi < T(KF::R)) {
                    T f, df;
                    KF::fdf(qi, f, df);
                    cr += (scd[j] < T(0) ? -a2.z : a2.z) * f;
                }
            }
            const T vsig = fma_rn(-be, mu, add_rn(vi.w, a1.w));
            const T visc = mul_rn(mul_rn(mul_rn(al, vsig), mu), rhob_inv);
            const T S = fma_rn(visc, gbar, -pterm);
            const T wgt = mul_rn(mul_rn(mul_rn(ti.z, a2.z), S), rinv);
            ax.add(mul_rn(wgt, rx));
            ay.add(mul_rn(wgt, ry));
            az.add(mul_rn(wgt, rz));
            if (adi)
                du += a2.z * (ti.x * vdr * gi +
                              rhob_inv * gbar * (T(-0.5) * al * vsig * mu * mu + aac * ac_speed(vdr, ti, a2, gm1_price, rhob_inv) * (ti.w - a2.w)));
            vs = vsig > vs ? vsig : vs;
            if (blk) {
                const T lj = slev[j], aj = fabs(lj);
                mlev = aj > mlev ? aj : mlev;
                if (due && lj < T(0) && aj < li1 - lgap) atomicMax(&b.breq[b.perm[j]], (int)(li1 - lgap) - 1);
            }
        }
        pairs += cnt;
        cnt = 0;
        __syncwarp();  // table and lists free for reuse
    };
    // membership: r_ij < R_K max(h_i, h_j), decided on the staged
    // (offset + shift) difference; where its rounding differs from the
    // pair vector's the pair sits at q = R_K, where f' and the force vanish
    auto test = [&]() {
        __syncwarp();  // staged candidates visible to every lane
        const int self = tA >= 0 ? ((tA << 5) | pos) : -1;
        for (int k0 = 0; k0 < nbuf; k0 += C::SB) {
            if (__any_sync(FULL, cnt > C::LC - C::SB / LPP)) eval_lists();
            const int ke = k0 + C::SB < nbuf ? k0 + C::SB : nbuf;
#pragma unroll 4
            for (int k = k0 + sub; k < ke; k += LPP) {
                const V c = cand[k];
                T rx = xi.x - c.x, ry = xi.y - c.y, rz = xi.z - c.z;
                if (wrap2) wrap3s<T>(sc, rx, ry, rz);
                T r2 = rx * rx + ry * ry + rz * rz;
                T hm = xi.w < c.w ? xi.w : c.w;
                const int cd = code[k];
                if (active && cd != self && r2 * hm * hm < T(KF::R * KF::R))
                    lst[cnt++ * 32 + lane] = (unsigned short)cd;
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
            // candidate leaves that form an ambiguous pair with A (periodic)
            am = ph.periodic ? __ballot_sync(FULL, ((mask >> lane) & 1u) && ambiguous(b.nodes[0][first + lane].slo.w, sc))
                             : 0u;
            if (!WRAP && am) to_wrap = true;
            if (!WRAP && to_wrap) return;
            stage_group<T, C::CH>(
                b, leaf, mask, first, ph, nbuf, sc,
                [&](bool has, int B, int stB, T Dx, T Dy, T Dz) {
                    gmask = mask;
                    if (has) {
                        V t;
                        t.x = Dx;
                        t.y = Dy;
                        t.z = Dz;
                        t.w = bits_as_t((am >> lane) & 1u ? ~stB : stB, T(0));
                        table[ntab + __popc(mask & below)] = t;
                    }
                    const unsigned sm = __ballot_sync(FULL, has && B == leaf);
                    if (sm) tA = ntab + __popc(mask & ((1u << (__ffs(sm) - 1)) - 1u));
                },
                [&](int j) { return gph[j]; },
                [&](V &q, int k) {
                    if (WRAP && ((am >> k) & 1u)) wrap_near<T>(sc, q, sc.C[0], sc.C[1], sc.C[2]);
                    const T d2 = box_dist2<T>(q, flo, fhi);
                    return d2 < RA2 || d2 * q.w * q.w < T(KF::R * KF::R * 1.0001);
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
    const int ngl = k0 < 0 ? b.leaf_ngroups[leaf] : -1;
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
    if (!WRAP && to_wrap) return false;
    // combine the lanes of each particle; FP64 for the compensated sums
    double Fx = (double)ax.s + (double)ax.c, Fy = (double)ay.s + (double)ay.c, Fz = (double)az.s + (double)az.c;
    Fx = group_sum<LPP>(Fx);
    Fy = group_sum<LPP>(Fy);
    Fz = group_sum<LPP>(Fz);
    du = group_sum<LPP>(du);
    vs = group_max<LPP>(vs);
    dvs = group_sum<LPP>(dvs);
    if (cdw) {
#pragma unroll
        for (int k = 0; k < 9; ++k) cg[k] = group_sum<LPP>(cg[k]);
        cr = group_sum<LPP>(cr);
    }
    if (blk) mlev = group_max<LPP>(mlev);
    // a = F / m in FP64 (m a stays F to FP64 round-off), one reciprocal
    // per particle (none for equal masses); the CFL step C h / v_sig of
    // Eq. SPH_DT in the pair precision (FP32: the FP64 pipe is much
    // narrower than the FP32 one on this part)
    T dti = tinf<T>();
    if (due && sub == 0) {
        long long g = b.perm[s];
        long long i = g - ps.base;
        if (blk) b.bnml[g] = (int)mlev - 1;
        const double minv = ps.uniform_m ? ps.inv_m_uniform : 1.0 / ps.m[i];
        double a[3] = {Fx * minv, Fy * minv, Fz * minv};
        const T vsig_t = vs < T(0) ? T(2) * vi.w : vs;
        ps.ax[i] = a[0];
        ps.ay[i] = a[1];
        ps.az[i] = a[2];
        ps.du[i] = adi ? (double)du : 0.0;
        ps.vsig[i] = (double)vsig_t;
        // div v = -(1/(Omega rho)) sum_j m_j v_ij . grad_i W(h_i): the next
        // step starts its h iteration from h exp(div v dt / 3) (continuity,
        // with h ~ rho^-1/3)
        b.divv[g] = (float)(-(double)dvs / (b.somega[s] * b.srho[s]));
        if (sw && !cdw) {  // Morris & Monaghan: decay towards alpha_min, growth where compressed
            const double divv = -(double)dvs / (b.somega[s] * b.srho[s]);
            const double ai = (double)alpha_i;
            ps.dalpha[i] = -(ai - ph.alpha_min) * ph.av_decay * (double)vi.w / b.sh[s] +
                           (divv < 0.0 ? -divv * (ph.alpha_av - ai) : 0.0);
        }
        if (cdw) {  // Cullen & Dehnen: velocity gradient, shear, signed density, limiter
            const double rho_i = b.srho[s], f = -1.0 / (b.somega[s] * rho_i);
            double V[9];
            for (int k = 0; k < 9; ++k) V[k] = f * (double)cg[k];
            const double dv = V[0] + V[4] + V[8];
            double ss = 0.0;
            for (int p2 = 0; p2 < 3; ++p2)
                for (int q2 = 0; q2 < 3; ++q2) {
                    const double sab = 0.5 * (V[3 * p2 + q2] + V[3 * q2 + p2]) - (p2 == q2 ? dv / 3.0 : 0.0);
                    ss += sab * sab;
                }
            const double hinv_i = (double)xi.w, w0 = Kern<K>::sigma * hinv_i * hinv_i * hinv_i;
            T f0, df0;
            KF::fdf(T(0), f0, df0);
            const double self = (ps.dalpha[i] < 0.0 ? -1.0 : 1.0) * (double)ti.z * (double)f0;
            const double R = ((double)cr + self) * w0 / rho_i;
            const double om = 1.0 - R, qq = 2.0 * om * om * om * om * dv;
            b.cdold[g] = ps.dalpha[i];
            b.cdxi[g] = (qq * qq + ss) > 0.0 ? qq * qq / (qq * qq + ss) : 0.0;
            ps.dalpha[i] = dv;
        }
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
    return true;
}

// WRAP: the launch that serves the wrap list (leaves whose pair vectors may
// miss the minimum image); the other launch puts them there.
template <typename T, int LPP, int K, bool WRAP, bool CD>
__global__ void __launch_bounds__(FCfg<T, LPP>::WPB * 32, FCfg<T, LPP>::MINB) k_forces(BatchView b)
{
    using C = FCfg<T, LPP>;
    extern __shared__ __align__(32) unsigned char smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    unsigned char *mine = smem + wib * C::per_warp;
    // block-step ticks: the wrap-list launch serves the tick's tasks (leaf
    // << 5 | first due ordinal) directly; the common launch does not run
    const bool tasks = WRAP && b.block_on && b.block_tasks;
    const int nleaf = tasks ? b.counters[kBlockTasks] : WRAP ? b.counters[kForceWrapList] : b.counters[0];
    const int cls = lpp_log2(LPP) + 4 * K;
    int last_p = -1;
    float Rall = 0.f;  // periodic: pairs reach R_K x the problem's largest h
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(&b.counters[(CD ? kForceCdCounter : WRAP ? kForceWrapCounter : kForceCounter) + cls], 1);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nleaf) break;
        if (WRAP) item = tasks ? b.btask[item] : b.wrap_list[item];
        const int leaf = tasks ? item >> 5 : item, k0 = tasks ? item & 31 : -1;
        const int p = b.leaf_pid[leaf];
        const ProbStatic &ps = b.prob[p];
        if ((tasks ? b.block_lanes : ps.lpp) != LPP || ps.ph.kernel != K) continue;  // served by another launch
        if (WRAP && (ps.ph.av_switch == SPH_AV_CULLEN_DEHNEN) != CD) continue;  // (the switch's own launch)
        if (!WRAP && (ps.ph.av_switch || ps.ph.ac_signal || ps.ph.gravity || b.block_on)) {
            // the viscosity switch, Price's conductivity and gravity's zeta term run in the
            // wrap-list launch only, which keeps the common path's registers for the default scheme
            if (lane == 0) b.wrap_list[atomicAdd(&b.counters[kForceWrapList], 1)] = leaf;
            continue;
        }
        if (ps.ph.periodic && p != last_p) {  // (consecutive leaves mostly share a problem)
            float extmax;
            problem_top_max(b, b.dyn[p], Rall, extmax);
            Rall = __fmul_ru((float)Kern<K>::R, Rall) * 1.0001f;
            last_p = p;
        }
        if (!force_leaf<T, LPP, K, WRAP, CD>(b, leaf, k0, mine, Rall) && lane == 0) {
            b.wrap_list[atomicAdd(&b.counters[kForceWrapList], 1)] = leaf;
            atomicAdd(&ps.diag->wrap_leaves, 1);
        }
    }
}

template <typename KernFn>
void set_smem(KernFn k, size_t bytes)
{
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int LPP, bool UM, int K, bool WRAP>
cudaError_t run_density(const BatchView &b, int use_pred, cudaStream_t st)
{
    using C = DCfg<T, LPP, UM, K>;
    static int per_sm = 0;
    if (!per_sm) {
        set_smem(k_density<T, LPP, UM, K, WRAP>, C::smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_density<T, LPP, UM, K, WRAP>, C::WPB * 32, C::smem);
        if (per_sm < 1) per_sm = 1;
    }
    // the wrap-list launch serves few leaves (mostly none) unless a problem
    // has gravity or the launch is a block-step tick's
    k_density<T, LPP, UM, K, WRAP><<<dev_info().sm_count * (WRAP && !b.any_gravity && !(b.block_on && b.block_tasks) ? 1 : per_sm),
                                     C::WPB * 32, C::smem, st>>>(b, use_pred);
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

// Block-step ticks, after the leaves: each leaf with particles whose step
// ends now gives one task per 32 / block_lanes of them (in sorted order), so
// that a task's block_lanes lanes per particle and its box (of those
// particles only) keep the pair kernels' latency short when few particles of
// a leaf are due; the leaf's other particles keep the h, rho, Omega, P and c
// of their last solve and are restaged (with their drifted offsets and
// predicted v, u) for the force pass.  One warp per leaf (<= 32 particles),
// lane = position in the leaf.
template <typename T>
__device__ __forceinline__ void block_tasks_one(const BatchView &b, int leaf, int n, long long s, bool due, int use_pred)
{
    using V = typename Vec4<T>::type;
    const int lane = threadIdx.x & 31;
    const int d = __popc(__ballot_sync(FULL, due));
    const int size = 32 / b.block_lanes, nt = (d + size - 1) / size;
    int base = 0;
    if (lane == 0 && nt > 0) base = atomicAdd(&b.counters[kBlockTasks], nt);
    base = __shfl_sync(FULL, base, 0);
    if (lane < nt) b.btask[base + lane] = (leaf << 5) | (lane * size);
    if (lane < n && !due) density_epilogue<T>(b, b.prob[0], s, ((const V *)b.pm)[s], T(1), T(0), T(0), use_pred, T(0));
}

// the tasks of a tick that built its leaves
template <typename T>
__global__ void __launch_bounds__(256) k_block_tasks(BatchView b, int use_pred)
{
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) {
        const int st = b.leaf_start[leaf], n = b.leaf_start[leaf + 1] - st;
        const long long s = st + (lane < n ? lane : 0);
        const bool due = lane < n && ((const T *)b.slev)[s] > T(0);
        block_tasks_one<T>(b, leaf, n, s, due, use_pred);
    }
}

// A tick that keeps the order and the leaves (tree reuse, Sec. 4.2), one
// warp per leaf: the drift of its particles, their gather into sorted order
// and the staging of their levels, the leaf's offsets and boxes and the tree
// above it (as the leaf pass does for kept leaves), then its tasks and the
// restaging of its particles that keep their solve: one pass instead of four.
template <typename T, typename T4>
__global__ void __launch_bounds__(256) k_block_leaf_tick(BatchView b, int use_pred)
{
    const int lane = threadIdx.x & 31;
    const int nleaf = b.counters[0];
    if (blockIdx.x == 0)
        for (int p = threadIdx.x; p < b.nprob; p += blockDim.x) b.dyn[p].lists_stale = 0;
    const long long k0 = b.scratch64[4], k1 = b.scratch64[5];
    const double tau = __longlong_as_double(b.scratch64[7]);
    const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int leaf = w; leaf < nleaf; leaf += nw) {
        const int st = b.leaf_start[leaf], n = b.leaf_start[leaf + 1] - st;
        const long long s = st + (lane < n ? lane : 0);
        bool due = false;
        if (lane < n) {
            const ProbStatic &ps = b.prob[0];
            const long long g = b.perm[s], i = g - ps.base;
            const double m = ps.m[i], h = ps.h[i];  // (read with the drift's inputs, not after its stores)
            const int lv = b.blev[g];
            double x[3];
            due = drift_one(b, g, k0, k1, tau, x);
            b.sx[s] = x[0];
            b.sy[s] = x[1];
            b.sz[s] = x[2];
            b.sm[s] = m;
            b.sh[s] = h;
            const T v = (T)(lv + 1);
            ((T *)b.slev)[s] = due ? v : -v;
        }
        const unsigned dm = __ballot_sync(FULL, due);
        if (lane == 0 && dm) atomicAdd((unsigned long long *)&b.scratch64[3], (unsigned long long)__popc(dm));
        __syncwarp();  // the leaf's gathered particles visible to the whole warp
        leaf_props_one<T4, true>(b, leaf);
        __syncwarp();
        block_tasks_one<T>(b, leaf, n, s, due, use_pred);
    }
}

template <typename T, int LPP, int K, bool WRAP, bool CD = false>
cudaError_t run_forces(const BatchView &b, cudaStream_t st)
{
    using C = FCfg<T, LPP>;
    static bool init = false;
    if (!init) {
        set_smem(k_forces<T, LPP, K, WRAP, CD>, C::smem);
        init = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_forces<T, LPP, K, WRAP, CD>, C::WPB * 32, C::smem);
    if (per_sm < 1) per_sm = 1;
    // the wrap list is short unless a problem uses the viscosity switch or Price's conductivity
    int grid = dev_info().sm_count * (WRAP && !b.any_general ? 1 : per_sm);
    k_forces<T, LPP, K, WRAP, CD><<<grid, C::WPB * 32, C::smem, st>>>(b);
    cudaError_t e = cudaGetLastError();
    // the Cullen & Dehnen problems' leaves on the wrap list: their own launch
    // (never with block steps, the only users of whole-warp particles)
    if constexpr (WRAP && !CD && LPP != 32)
        if (e == cudaSuccess && b.any_cd) e = run_forces<T, LPP, K, true, true>(b, st);
    return e;
}

// The density launches of kernel K: one per class (lanes per particle, equal
// masses) present in the batch; class bit lanes_index + 4 u + 8 K.  FP64
// runs 2 or 4 lanes per particle, M6 at least 2 (the host never selects
// fewer).  WRAP: the launches that serve the wrap list.
template <int K, bool WRAP>
cudaError_t density_classes(const BatchView &b, int precision, int use_pred, cudaStream_t st)
{
    for (int cls = 0; cls < 8; ++cls) {
        if (!(b.dens_mask & (1 << (cls + 8 * K)))) continue;
        const int k = cls & 3;
        const bool um = cls >= 4;
        cudaError_t e;
        if (precision == SPH_PREC_FP64) {
            if (k == 2) e = um ? run_density<double, 4, true, K, WRAP>(b, use_pred, st) : run_density<double, 4, false, K, WRAP>(b, use_pred, st);
            else e = um ? run_density<double, 2, true, K, WRAP>(b, use_pred, st) : run_density<double, 2, false, K, WRAP>(b, use_pred, st);
        } else {
            switch (k) {
            case 0:
                if constexpr (K == SPH_KERNEL_M4) {
                    e = um ? run_density<float, 1, true, K, WRAP>(b, use_pred, st) : run_density<float, 1, false, K, WRAP>(b, use_pred, st);
                    break;
                }
                [[fallthrough]];  // (M6 never runs one lane per particle)
            case 1: e = um ? run_density<float, 2, true, K, WRAP>(b, use_pred, st) : run_density<float, 2, false, K, WRAP>(b, use_pred, st); break;
            case 2: e = um ? run_density<float, 4, true, K, WRAP>(b, use_pred, st) : run_density<float, 4, false, K, WRAP>(b, use_pred, st); break;
            default:
                // block-step tasks of one particle with a whole warp (M4, FP32)
                if constexpr (K == SPH_KERNEL_M4 && WRAP) {
                    if (b.block_on && b.block_tasks && b.block_lanes == 32) {
                        e = um ? run_density<float, 32, true, K, WRAP>(b, use_pred, st) : run_density<float, 32, false, K, WRAP>(b, use_pred, st);
                        break;
                    }
                }
                e = um ? run_density<float, 8, true, K, WRAP>(b, use_pred, st) : run_density<float, 8, false, K, WRAP>(b, use_pred, st);
                break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The force launches of kernel K, one per lanes-per-particle class present
// (class bit lanes_index + 4 K).
template <int K, bool WRAP>
cudaError_t force_classes(const BatchView &b, int precision, cudaStream_t st)
{
    for (int k = 0; k < 4; ++k) {
        if (!(b.lpp_mask & (1 << (k + 4 * K)))) continue;
        cudaError_t e;
        if (precision == SPH_PREC_FP64) {
            if (k == 2) e = run_forces<double, 4, K, WRAP>(b, st);
            else e = run_forces<double, 2, K, WRAP>(b, st);
        } else {
            switch (k) {
            case 0:
                if constexpr (K == SPH_KERNEL_M4) {
                    e = run_forces<float, 1, K, WRAP>(b, st);
                    break;
                }
                [[fallthrough]];
            case 1: e = run_forces<float, 2, K, WRAP>(b, st); break;
            case 2: e = run_forces<float, 4, K, WRAP>(b, st); break;
            default:
                if constexpr (K == SPH_KERNEL_M4 && WRAP) {
                    if (b.block_on && b.block_tasks && b.block_lanes == 32) {
                        e = run_forces<float, 32, K, WRAP>(b, st);
                        break;
                    }
                }
                e = run_forces<float, 8, K, WRAP>(b, st);
                break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

// the launches of one kernel (M4, M6) and kind (common, wrap list), each
// instantiated in a translation unit of its own so that they compile in
// parallel
cudaError_t density_launches_m4(const BatchView &b, int precision, int use_pred, cudaStream_t st);
cudaError_t density_launches_m6(const BatchView &b, int precision, int use_pred, cudaStream_t st);
cudaError_t density_launches_m4_wrap(const BatchView &b, int precision, int use_pred, cudaStream_t st);
cudaError_t density_launches_m6_wrap(const BatchView &b, int precision, int use_pred, cudaStream_t st);
cudaError_t force_launches_m4(const BatchView &b, int precision, cudaStream_t st);
cudaError_t force_launches_m6(const BatchView &b, int precision, cudaStream_t st);
cudaError_t force_launches_m4_wrap(const BatchView &b, int precision, cudaStream_t st);
cudaError_t force_launches_m6_wrap(const BatchView &b, int precision, cudaStream_t st);

}  // namespace sph
