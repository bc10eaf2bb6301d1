// Leaf boxes and the bottom-up tree pass over them, shared by the leaf build
// (sph_build.cu) and the block-step tick that keeps its leaves (sph_pairs.cu).
#pragma once
#include "sph_internal.cuh"

namespace sph {

__device__ __forceinline__ NodeBox ld_node(const NodeBox *p)
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
    NodeBox nb;
    nb.plo = __ldcg(q);
    nb.phi = __ldcg(q + 1);
    nb.slo = __ldcg(q + 2);
    nb.shi = __ldcg(q + 3);
    return nb;
}

// Union of the (up to 32) child boxes held by the lanes with on set, written
// by lane 0 to *out.
__device__ __forceinline__ void union_children(const NodeBox &c, bool on, NodeBox *out)
{
    float v[12];
    v[0] = on ? c.plo.x : INFINITY;
    v[1] = on ? c.plo.y : INFINITY;
    v[2] = on ? c.plo.z : INFINITY;
    v[3] = on ? c.phi.x : -INFINITY;
    v[4] = on ? c.phi.y : -INFINITY;
    v[5] = on ? c.phi.z : -INFINITY;
    v[6] = on ? c.slo.x : INFINITY;
    v[7] = on ? c.slo.y : INFINITY;
    v[8] = on ? c.slo.z : INFINITY;
    v[9] = on ? c.shi.x : -INFINITY;
    v[10] = on ? c.shi.y : -INFINITY;
    v[11] = on ? c.shi.z : -INFINITY;
    float hm = warp_max(on ? c.plo.w : 0.f);
    float cnt = warp_sum(on ? c.phi.w : 0.f);
    for (int a = 0; a < 3; ++a) {
        v[a] = warp_min(v[a]);
        v[3 + a] = warp_max(v[3 + a]);
        v[6 + a] = warp_min(v[6 + a]);
        v[9 + a] = warp_max(v[9 + a]);
    }
    if ((threadIdx.x & 31) == 0) {
        NodeBox nb;
        nb.plo = make_float4(v[0], v[1], v[2], hm);
        nb.phi = make_float4(v[3], v[4], v[5], cnt);
        nb.slo = make_float4(v[6], v[7], v[8], 0.f);
        nb.shi = make_float4(v[9], v[10], v[11], 0.f);
        *out = nb;
    }
}

// After lane 0 wrote the box of `leaf`: the warp that completes the last
// child of a node (arrival counter per node, cleared again by that warp)
// forms the node's box from its children and carries on upwards.
__device__ __forceinline__ void tree_up(const BatchView &b, int leaf)
{
    const int lane = threadIdx.x & 31;
    const ProbDyn &d = b.dyn[b.leaf_pid[leaf]];
    const int top = d.top_level;
    int k = leaf - d.node_off[0];
    for (int lvl = 0; lvl < top; ++lvl) {
        const int parent = k / kBranch;
        const int nch = min(kBranch, d.node_cnt[lvl] - parent * kBranch);
        int *ctr = b.node_ctr[lvl + 1] + d.node_off[lvl + 1] + parent;
        int old = 0;
        if (lane == 0) {
            __threadfence();  // this warp's child box before its arrival
            old = atomicAdd(ctr, 1);
        }
        old = __shfl_sync(0xffffffffu, old, 0);
        if (old != nch - 1) return;
        if (lane == 0) *ctr = 0;
        __threadfence();
        const bool on = lane < nch;
        NodeBox c;
        if (on) c = ld_node(b.nodes[lvl] + d.node_off[lvl] + parent * kBranch + lane);
        union_children(c, on, b.nodes[lvl + 1] + d.node_off[lvl + 1] + parent);
        k = parent;
    }
}

// Float bounds of an offset known to within one rounding (|v| 2^-24) of the
// exact FP64 difference, widened by four times that.
__device__ __forceinline__ float widen_dn(float v, float mag) { return __fsub_rd(v, mag * 2.4e-7f); }
__device__ __forceinline__ float widen_up(float v, float mag) { return __fadd_ru(v, mag * 2.4e-7f); }

// lane a (< 3) gets v[a]
__device__ __forceinline__ float axis_of(const float *v, int lane)
{
    return lane == 0 ? v[0] : lane == 1 ? v[1] : v[2];
}

__device__ __forceinline__ float offset_f(float v) { return v; }
__device__ __forceinline__ float offset_f(double v) { return (float)v; }

// Per-axis extents of a leaf's offsets from its reference point (e: this
// lane's |offset| per axis), packed for the minimum-image test of the pair
// kernels: 10 bits per axis in units of L_a / 2046, rounded up (1023: half
// the box or more), as the bits of a float; 0 for isolated problems.
__device__ __forceinline__ float leaf_ext_bits(const float (&e)[3], const PhysParams &ph)
{
    unsigned bits = 0u;
    for (int a = 0; a < 3; ++a) {
        const float m = warp_max(e[a]);
        if (ph.periodic) {
            const unsigned q = (unsigned)ceilf(m * (2.f * ph.box_inv_f[a]) * 1023.f * 1.00001f) + 1u;
            bits |= (q < 1023u ? q : 1023u) << (10 * a);
        }
    }
    return __uint_as_float(bits);
}

// Leaf reference point, position box and the offsets of its particles from
// that point.  The reference point is the leaf's first particle (FP64); the
// FP64 difference is taken before the cast to the staging precision.  The
// box is formed in FP32 from the offsets, widened for their rounding, plus
// the reference point rounded down (up): only these two conversions per axis
// and leaf, by lanes 0..2, run on the FP64 pipe besides the offsets.
// One warp per leaf; WRAP: a kept leaf (its particles may have wrapped).
template <typename T4, bool WRAP>
__device__ __forceinline__ void leaf_props_one(const BatchView &b, int leaf)
{
    const int lane = threadIdx.x & 31;
    {
        const int st = b.leaf_start[leaf], cnt = b.leaf_start[leaf + 1] - st;
        const ProbStatic &ps = b.prob[b.leaf_pid[leaf]];
        const bool on = lane < cnt;
        // reference point: the centre of the leaf's box (its first particle
        // shifted by the float midpoint of the offsets from it), so that the
        // offsets stay within half the leaf's width
        double c[3] = {b.sx[st], b.sy[st], b.sz[st]};
        double d[3] = {0.0, 0.0, 0.0};
        if (on) {
            const double x[3] = {b.sx[st + lane], b.sy[st + lane], b.sz[st + lane]};
            for (int a = 0; a < 3; ++a)
                d[a] = WRAP ? min_image(x[a] - c[a], ps.ph.box_len[a], ps.ph.periodic)  // (kept leaf: may
                            : x[a] - c[a];                                               // have wrapped)
        }
        for (int a = 0; a < 3; ++a) {
            const float mid = 0.5f * (warp_max(on ? (float)d[a] : -INFINITY) + warp_min(on ? (float)d[a] : INFINITY));
            c[a] += (double)mid;
            d[a] -= (double)mid;
        }
        float lo[3], hi[3], slo_[3], shi_[3], hp = 0.f, ex[3] = {0.f, 0.f, 0.f};
        if (on) {
            T4 v;
            v.x = (decltype(v.x))d[0];
            v.y = (decltype(v.y))d[1];
            v.z = (decltype(v.z))d[2];
            v.w = ps.uniform_m ? (decltype(v.w))ps.m_uniform : (decltype(v.w))b.sm[st + lane];
            ((T4 *)b.pm)[st + lane] = v;
            const float o[3] = {offset_f(v.x), offset_f(v.y), offset_f(v.z)};
            for (int a = 0; a < 3; ++a) ex[a] = fabsf(o[a]);
            // predicted smoothing spheres: 1.1 x the guessed h (the h the
            // density solve starts from); the force pass reuses the density
            // walk's candidates when no final h exceeds its prediction
            hp = __fmul_ru(kHPredict, __double2float_ru(b.sh[st + lane]));
            const float h2 = __fmul_ru(ps.ph.kr_f, hp);  // support radius R_K h
            for (int a = 0; a < 3; ++a) {
                lo[a] = widen_dn(o[a], fabsf(o[a]));
                hi[a] = widen_up(o[a], fabsf(o[a]));
                const float mag = __fadd_ru(fabsf(o[a]), h2);
                slo_[a] = widen_dn(__fsub_rd(o[a], h2), mag);
                shi_[a] = widen_up(__fadd_ru(o[a], h2), mag);
            }
        } else {
            for (int a = 0; a < 3; ++a) {
                lo[a] = slo_[a] = INFINITY;
                hi[a] = shi_[a] = -INFINITY;
            }
        }
        for (int a = 0; a < 3; ++a) {
            lo[a] = warp_min(lo[a]);
            hi[a] = warp_max(hi[a]);
            slo_[a] = warp_min(slo_[a]);
            shi_[a] = warp_max(shi_[a]);
        }
        hp = warp_max(hp);
        const float ext = leaf_ext_bits(ex, ps.ph);
        float bl = 0.f, bh = 0.f, sl = 0.f, sh = 0.f;
        if (lane < 3) {
            const double ca = lane == 0 ? c[0] : lane == 1 ? c[1] : c[2];
            const float cd = __double2float_rd(ca), cu = __double2float_ru(ca);
            b.leaf_c[3 * (long long)leaf + lane] = ca;
            b.leaf_cf[6 * (long long)leaf + lane] = cd;
            b.leaf_cf[6 * (long long)leaf + 3 + lane] = cu;
            bl = __fadd_rd(cd, axis_of(lo, lane));
            bh = __fadd_ru(cu, axis_of(hi, lane));
            sl = __fadd_rd(cd, axis_of(slo_, lane));
            sh = __fadd_ru(cu, axis_of(shi_, lane));
        }
        const float l0 = __shfl_sync(0xffffffffu, bl, 0), l1 = __shfl_sync(0xffffffffu, bl, 1),
                    l2 = __shfl_sync(0xffffffffu, bl, 2);
        const float h0 = __shfl_sync(0xffffffffu, bh, 0), h1 = __shfl_sync(0xffffffffu, bh, 1),
                    h2 = __shfl_sync(0xffffffffu, bh, 2);
        const float s0 = __shfl_sync(0xffffffffu, sl, 0), s1 = __shfl_sync(0xffffffffu, sl, 1),
                    s2 = __shfl_sync(0xffffffffu, sl, 2);
        const float t0 = __shfl_sync(0xffffffffu, sh, 0), t1 = __shfl_sync(0xffffffffu, sh, 1),
                    t2 = __shfl_sync(0xffffffffu, sh, 2);
        if (lane == 0) {
            NodeBox nb;
            nb.plo = make_float4(l0, l1, l2, hp);  // h_max predicted until the refit
            nb.phi = make_float4(h0, h1, h2, (float)cnt);
            nb.slo = make_float4(s0, s1, s2, ext);
            nb.shi = make_float4(t0, t1, t2, 0.f);
            b.nodes[0][leaf] = nb;
        }
        tree_up(b, leaf);
    }
}

// ---- block-step ticks ------------------------------------------------------
// v + a d with explicit rounding (the block step's kicks and predictions)
__device__ __forceinline__ double block_kick(double v, double a, double d) { return __dadd_rn(v, __dmul_rn(a, d)); }

// drift particle g (original order) from tick k0 to tick k1 and predict
// its v, u and alpha at k1 for the force pass; true if its step ends at k1.
// Every input is read before the first store (which the compiler must
// otherwise assume may alias the next input: one memory round trip per
// axis); xo, if given, receives the drifted position.
__device__ __forceinline__ bool drift_one(const BatchView &b, long long g, long long k0, long long k1, double tau,
                                          double *xo = nullptr)
{
    const ProbStatic &ps = b.prob[0];
    const PhysParams &ph = ps.ph;
    const long long i = g - ps.base, n = b.ntot;
    const bool adi = ph.eos == SPH_EOS_ADIABATIC, sw = ph.av_switch != 0;
    const int t0 = b.bt0[g], t1 = b.bt1[g];
    const double x0[3] = {ps.x[i], ps.y[i], ps.z[i]};
    const double vh[3] = {b.bvh[g], b.bvh[n + g], b.bvh[2 * n + g]};
    const double acc[3] = {ps.ax[i], ps.ay[i], ps.az[i]};
    const double uh = adi ? b.bvh[3 * n + g] : 0.0, du = adi ? ps.du[i] : 0.0, u = adi ? 0.0 : ps.u[i];
    const double ah = sw ? b.bvh[4 * n + g] : 0.0, da = sw ? ps.dalpha[i] : 0.0;
    const double dk = __dmul_rn((double)(k1 - k0), tau);
    const double dp = __dmul_rn(__dmul_rn((double)(2 * k1 - t0 - t1), 0.5), tau);  // t - t_mid
    double *X[3] = {ps.x, ps.y, ps.z};
    double *VP[3] = {b.vpx, b.vpy, b.vpz};
    for (int a = 0; a < 3; ++a) {
        double x = __dadd_rn(x0[a], __dmul_rn(vh[a], dk));
        if (ph.periodic) {
            const double lo = ph.box_lo[a], Lb = ph.box_len[a];
            if (x >= lo + Lb) x -= Lb;
            else if (x < lo) x += Lb;
        }
        X[a][i] = x;
        if (xo) xo[a] = x;
        VP[a][g] = block_kick(vh[a], acc[a], dp);
    }
    b.up[g] = adi ? block_kick(uh, du, dp) : u;
    if (sw) b.ap[g] = block_kick(ah, da, dp);
    b.breq[g] = -1;
    return t1 == k1;
}

}  // namespace sph
