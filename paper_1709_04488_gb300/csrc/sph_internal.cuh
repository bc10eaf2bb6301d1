// Internal declarations of the GB300 SPH library: device-side problem
// descriptors, workspace views and small device helpers shared by the kernels.
// Nothing here is part of the public ABI (include/sph.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sph.h"

namespace sph {

constexpr int kMaxLevels = 6;       // tree levels above the leaves (32^6 leaves)
constexpr int kBranch = 32;         // children per tree node (one per warp lane)
constexpr int kMortonBits = 10;     // bits per axis of the Morton key
constexpr int kMortonTotal = 3 * kMortonBits;
constexpr double kPi = 3.14159265358979323846;
// slots of BatchView::counters: 0 leaves, 1..7 nodes per level, 8 slow-path
// count, 9 groups used in the candidate-group pool, 10 (11) leaves on the
// density (force) wrap list, 15 look-back timeout, 16..31 density leaf
// tickets (per class: lanes, equal masses, kernel), 32..39 force leaf
// tickets (per lanes per particle and kernel), 40..55 and 56..63 the same
// for the launches that serve the wrap lists, 64..71 the force tickets of the
// Cullen & Dehnen launches; the step's first kernel clears 8..11 and 15..71,
// a forces-only call 11, 15, 32..39 and 56..71
constexpr int kNumCounters = 72;
constexpr int kSlowCounter = 8, kPoolCounter = 9, kDensWrapList = 10, kForceWrapList = 11, kTimeoutCounter = 15;
// block-step ticks: counter 12 holds the number of tasks (a leaf and up to
// 32 / block_lanes of its particles whose step ends now, served with
// block_lanes lanes each by the pair kernels); cleared by each tick's first
// kernel.  block_lanes: a whole warp per particle in FP32 pairs with the M4
// kernel (the tick's time is its slowest task's, and a warp shares that
// particle's candidates 32 ways); 8 with M6 or self-gravity (whose tree walk
// per task costs more than the lanes save); 4 in FP64 (the lanes the FP64
// kernels are built for)
constexpr int kBlockTasks = 12, kBlockLanesF32 = 32, kBlockLanesF32Walk = 8, kBlockLanesF64 = 4;
constexpr int kDensityCounter = 16, kForceCounter = 32, kDensityWrapCounter = 40, kForceWrapCounter = 56,
              kForceCdCounter = 64;
constexpr int kDensityClasses = 16, kForceClasses = 8;
static_assert(kDensityCounter + kDensityClasses <= kForceCounter && kForceCounter + kForceClasses <= kDensityWrapCounter &&
                  kDensityWrapCounter + kDensityClasses <= kForceWrapCounter &&
                  kForceWrapCounter + kForceClasses <= kForceCdCounter &&
                  kForceCdCounter + kForceClasses <= kNumCounters,
              "counter slots");
constexpr int kMaxLeafGroups = 32;  // candidate-leaf groups recorded per leaf (one per lane)
#ifndef SPH_HPREDICT
#define SPH_HPREDICT 1.1f
#endif
constexpr float kHPredict = SPH_HPREDICT;  // predicted sphere boxes use this x the guessed h
constexpr int kReuseHold = 8;  // first hold after a step whose final h outgrew the records

// Status bits kept on the device per problem (mapped to SPH_E* on the host).
enum : unsigned {
    ST_NOCONV = 1u,
    ST_BOX = 2u,
    ST_NONFINITE = 4u,
    ST_TIMEOUT = 8u,
    ST_OVERFLOW = 16u,  // internal capacity exceeded (e.g. neighbour export)
    ST_SCHEDULE = 32u,  // block step: the next event tick is not after the current one
};

// Physics parameters of one problem as the kernels read them.
struct PhysParams {
    int periodic;
    int eos;
    double box_lo[3];
    double box_len[3];
    double gamma, cs_iso, eta;
    double alpha_av, beta_av, alpha_ac, c_cfl;
    double h_tol;
    int h_max_iter;
    int kernel;          // SPH_KERNEL_M4 or SPH_KERNEL_M6
    float box_len_f[3];  // box_len as float (node tests run in FP32)
    float kr_f;          // support radius in units of h: 2 (M4) or 3 (M6)
    double kr;
    double box_inv[3];   // 1 / box_len (periodic), for minimum-image wraps
    float box_inv_f[3];
    int ac_signal;       // SPH_AC_WADSLEY or SPH_AC_PRICE
    int av_switch;       // SPH_AV_CONSTANT or SPH_AV_MORRIS_MONAGHAN
    double alpha_min, av_decay, beta_ratio;  // switch: floor, decay rate (c/h), beta_av / alpha_av
    int gravity;         // self-gravity (isolated, M4)
    int pad3_;
    double G;
    double grav_theta;   // gravity: tree opening angle (0: direct summation)
    double c_grav;       // gravity: acceleration time-step condition's multiplier
    int block;           // hierarchical block time-steps: largest level L (0: global steps)
    int block_gap;       // block steps: limiter gap dl in levels
};

// Per-problem diagnostics and persistent scalars; lives in the context's own
// workspace so that it survives between single and batched calls.
struct ProbDiag {
    double dt_next;      // CFL step from the last force evaluation
    double dt_cur;       // step in use by the current sph_step
    double time;
    double mass, mom[3], energy, fsum[3], dEdt;
    unsigned long long dt_min_bits;  // atomicMin target (positive doubles order as integers)
    long long steps;
    long long nr_iter;
    long long density_pairs, force_pairs, candidates, fallback, leaves;
    long long ngb_sum;
    int nr_max, ngb_min, ngb_max;
    unsigned status;
    int unconverged;
    int walk_reused;     // the last force pass reused the density walk's candidates
    int reuse_hold;      // steps left before the density walk records candidates again
    int reuse_backoff;   // length of the next hold (doubles while the records keep failing)
    int wrap_leaves;     // leaves of the last passes put on the wrap list
    int pad_;
    long long grav_pairs, grav_nodes;  // gravity tree walk: pair and multipole terms
};

// Host-written description of one problem inside a batch.
struct ProbStatic {
    // caller state arrays (original particle order)
    double *x, *y, *z, *vx, *vy, *vz, *u, *m, *h;
    double *rho, *omega, *P, *c, *ax, *ay, *az, *du, *vsig;
    double *alpha, *dalpha;  // viscosity switch (NULL without it)
    long long n;
    long long base;  // offset of this problem in the batch-global particle index space
    ProbDiag *diag;
    int lpp;         // lanes per particle in the pair kernels (leaf size = 32 / lpp)
    int uniform_m;   // all masses equal (m_uniform): neighbour lists keep distances only
    int gblk0;       // gravity: the problem's first block of the direct-sum launch
    int gchunks;     // gravity: ranges the partners are split into (one block per range and 256 particles)
    double m_uniform;
    double inv_m_uniform;  // 1 / m_uniform (0 unless uniform_m)
    PhysParams ph;
};

// Device-written per-step description (domain normalisation, leaves, tree).
struct ProbDyn {
    double dom_lo[3];
    double dom_inv;      // 1 / (largest extent of the key domain)
    unsigned long long bbox_bits[6];  // ordered-int min x,y,z and max x,y,z (isolated)
    int leaf_base, nleaf;
    int top_level;       // highest tree level (0 = the leaves themselves)
    int node_off[kMaxLevels + 1];  // global index of this problem's first node per level
    int node_cnt[kMaxLevels + 1];  // nodes per level (level 0 = leaves)
    int lists_stale;     // some leaf's final h exceeds what its recorded candidate groups cover
    int pad_;
};

// 32-byte vector of four doubles (FP64 staging)
struct __align__(32) dbl4 {
    double x, y, z, w;
};

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = dbl4;
};

// Box of a leaf or tree node: positions and smoothing spheres (pos +- R_K h,
// R_K the kernel's support in units of h), rounded outwards to float.
struct __align__(16) NodeBox {
    float4 plo;  // xyz = min position, w = h_max
    float4 phi;  // xyz = max position, w = particle count (as float)
    float4 slo;  // xyz = min (x - R_K h); w (leaves, periodic) = packed offset extents (leaf_ext_bits)
    float4 shi;  // xyz = max (x + R_K h)
};

// Batch-global scratch arrays (all carved from one workspace).
struct BatchView {
    int nprob;
    int lpp_mask;                // bit (k + 4 K): some problem uses 2^k lanes per particle and kernel K
    int dens_mask;               // bit (k + 4 u + 8 K): density class (2^k lanes, uniform masses u, kernel K)
    long long ntot;              // particles over all problems
    int max_leaves;              // capacity of the leaf arrays
    int key_bits;                // bits the radix sort must order
    int key_lo;                  // lowest key bit that is sorted (the bits below are cleared)
    int any_isolated;            // some problem is isolated (needs a bounding box)
    int any_periodic;            // some problem is periodic (wrap-list launches)
    int any_general;             // some problem uses the viscosity switch, Price's conductivity or
                                 // gravity (served by the wrap-list launches)
    int any_gravity;             // some problem has self-gravity (direct-sum launch)
    int any_cd;                  // some problem uses the Cullen & Dehnen switch (its own force launches)
    long long grav_blocks;       // blocks of the direct-sum launch (all gravity problems)
    int grav_split;              // some gravity problem splits its partners (partial sums to reduce)
    int any_grav_tree;           // some gravity problem walks the tree (grav_theta > 0)
    double *gpart;               // gravity: partial forces [chunk][ntot][3] of split problems
    // gravity tree: five Vec4 per node of each level (centre of mass relative
    // to the key-domain corner and mass; Q_xx, Q_xy, Q_xz, Q_yy; Q_yz, Q_zz,
    // l^2, h_max; box min; box max), element type float4 or dbl4
    void *gnode[kMaxLevels + 1];
    void *ggrp;                  // gravity tree: per level-1 node, its 8 groups of 4 leaves (five Vec4 each)
    // block time-steps (single problem): per particle, original order
    int block_on;                // this launch set is a tick of a block step
    int block_tasks;             // the pair kernels serve the tick's tasks (else whole leaves: the block's last tick)
    int block_lanes;             // lanes per particle of the tick's pair kernels (tasks)
    int *blev;                   // level
    int *bnml;                   // largest level among the force neighbours at the last force pass (-1: none)
    int *breq;                   // reactive limiter: level asked of an inactive particle (-1: none)
    int *bt0, *bt1;              // current step's first and last tick
    double *bvh;                 // half-step velocity x, y, z, u and alpha ([5][n])
    double *bzeta;               // gravity: the zeta term's weight G zeta / (2 Omega) of the last solve
    void *slev;                  // sorted: +(level + 1) if the particle ends its step now, else -(level + 1)
    int *btask;                  // tasks of this tick: leaf << 5 | ordinal of its first due particle
    void *gpos;                  // gravity tree: (x - corner, m) per sorted particle, Vec4
    void *gh;                    // gravity tree: (h, 1/h) per sorted particle, float2 or double2
    ProbStatic *prob;            // [nprob]
    ProbDyn *dyn;                // [nprob]
    long long *prob_base;        // [nprob + 1] base offsets (for searches)
    // sort
    unsigned long long *keys[2];
    unsigned *vals[2];
    unsigned *hist;              // sort: digit histograms, tile counters, look-back status
    int *perm;                   // sorted position -> batch-global original index
    // sorted FP64 copies
    double *sx, *sy, *sz, *sh, *sm;
    double *srho, *somega, *sP, *sc;
    // predicted velocity / internal energy (original order, batch-global)
    double *vpx, *vpy, *vpz, *up;
    double *ap;  // predicted alpha of the viscosity switch (original order)
    // staging for the pair kernels (sorted order); element type float4 or double4
    void *pm;   // (offset xyz, m)
    void *ph;   // (offset xyz, h)
    void *vc;   // (v xyz, c)
    void *th;   // (P/(Omega rho^2), rho, m, u)
    void *sal;  // alpha of the viscosity switch (T per particle)
    void *scd;  // Cullen & Dehnen: div v of the previous force evaluation (T per sorted particle)
    float *divv;  // div v of the last force pass (original order, batch-global): the h prediction
    double *cdold, *cdxi;  // Cullen & Dehnen (original order, batch-global): div v before this
                           // evaluation and the limiter xi of this one, for the step's alpha update
    void *szg;  // gravity: G zeta / (2 Omega) (T per particle), the zeta term's weight
    // leaves
    unsigned *flag;              // [ntot] leaf start flags, then leaf index (scan)
    int *leaf_start;             // [max_leaves + 1]
    int *leaf_pid;               // [max_leaves]
    double *leaf_c;              // [3 * max_leaves] leaf reference points (FP64)
    float *leaf_cf;              // [6 * max_leaves] the same rounded down (xyz) and up (xyz)
    float *hf;                   // [ntot] h after the density solve, float rounded up
    NodeBox *nodes[kMaxLevels + 1];  // level 0 = leaves
    int node_cap[kMaxLevels + 1];
    // state that must be zero before a build; the kernels clear what they use
    unsigned *tile_state;        // leaf scan: ticket, finished tiles, look-back status per tile
    int *node_ctr[kMaxLevels + 1];  // arrival counters of the nodes of levels 1..
    char *zero_lo;               // [zero_lo, zero_lo + zero_bytes) holds the two above
    size_t zero_bytes;
    int *fallback_list;          // [ntot] sorted indices needing the slow path
    int *wrap_list;              // [ntot] leaves served by the minimum-image (wrap) launches
    // candidate-leaf groups (first leaf, ballot of the 32 siblings) the
    // density walk visited per leaf, for the force pass to reuse
    int2 *group_pool;            // [group_cap]
    long long group_cap;
    int *leaf_gofs;              // [max_leaves] first pool entry of the leaf's groups
    int *leaf_ngroups;           // [max_leaves] group count, -1: not recorded (walk)
    float *leaf_hcap;            // [max_leaves] largest h the recorded groups cover
    int *counters;               // [kNumCounters], slots as listed at kSlowCounter
    long long *scratch64;        // [16]
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double min_image(double d, double L, int periodic)
{
    if (periodic) {
        if (d > 0.5 * L) d -= L;
        else if (d < -0.5 * L) d += L;
    }
    return d;
}

__device__ __forceinline__ unsigned long long ordered_bits(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double from_ordered_bits(unsigned long long b)
{
    b = (b & 0x8000000000000000ull) ? (b & 0x7fffffffffffffffull) : ~b;
    return __longlong_as_double((long long)b);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// index of the problem owning batch-global index g (prob_base ascending)
__device__ __forceinline__ int find_problem(const long long *base, int nprob, long long g)
{
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= g) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// host-side launch helpers (defined in the .cu files)
// ---------------------------------------------------------------------------
struct DevInfo {
    int sm_count;
};
DevInfo dev_info();

// sort / build / pair / integrate stages, each enqueued on `st`
cudaError_t launch_domain_and_keys(const BatchView &b, cudaStream_t st);
cudaError_t launch_radix_sort(const BatchView &b, cudaStream_t st);
cudaError_t launch_gather(const BatchView &b, cudaStream_t st);
cudaError_t launch_set_sorted_h(const BatchView &b, const double *h_in, cudaStream_t st);
cudaError_t launch_build_leaves(const BatchView &b, int precision, cudaStream_t st);
cudaError_t launch_update_leaves(const BatchView &b, int precision, cudaStream_t st);  // tree reuse
cudaError_t launch_refit(const BatchView &b, int precision, cudaStream_t st);
cudaError_t launch_density(const BatchView &b, int precision, int use_pred, cudaStream_t st);
cudaError_t launch_forces(const BatchView &b, int precision, cudaStream_t st);
void launch_gravity(const BatchView &b, int precision, cudaStream_t st);  // direct-sum self-gravity
// direct-sum launch of one problem (none when it walks the tree, theta > 0):
long long gravity_blocks(long long n, double theta);  // blocks (particle blocks x partner ranges)
int gravity_chunks(long long n, double theta);        // partner ranges
cudaError_t launch_kick_drift(const BatchView &b, double dt_host, cudaStream_t st);  // also selects dt, resets diagnostics
// block time-steps (sph_block.cu).  Every quantity a tick needs lives on the
// device, so that the ticks can run as a loop of a captured graph; scratch64:
// [0] smallest and [1] largest step (ordered bits), [2] next tick where a
// step ends, [3] force evaluations, [4] the current tick k0, [5] the tick k1
// being advanced to, [6] Delta t_MAX and [7] the tick length (bits), [8]
// ticks taken, [9] 1 while another tick of the loop follows, [10] blocks of
// the kick launch done, [11] 1 when the block's last tick (every particle
// due, at 2^L) follows.  `cond`/`fin` are the graph's loop and last-tick
// condition handles, set only when `use_cond` is true.
cudaError_t launch_block_dt(const BatchView &b, int L, cudaStream_t st);  // also plans Delta t_MAX
cudaError_t launch_block_open(const BatchView &b, int L, cudaStream_t st);
cudaError_t launch_block_gate(const BatchView &b, int L, bool use_cond, cudaGraphConditionalHandle cond,
                              cudaGraphConditionalHandle fin, cudaStream_t st);  // (opens the first tick)
// graph form with tree reuse: sets the branch condition (rebuild this tick)
cudaError_t launch_block_tick_begin(const BatchView &b, int every, cudaGraphConditionalHandle cond,
                                    cudaStream_t st);
cudaError_t launch_block_drift(const BatchView &b, cudaStream_t st);  // ahead of a sort
// after a new sort: the sorted gather and the staging of the levels
cudaError_t launch_block_gather(const BatchView &b, int precision, cudaStream_t st);
cudaError_t launch_block_tasks(const BatchView &b, int precision, cudaStream_t st);  // after the leaves (sph_pairs.cu)
// a tick that keeps the order and the leaves: drift, gather, leaf boxes and tasks in one pass (sph_pairs.cu)
cudaError_t launch_block_leaf_tick(const BatchView &b, int precision, cudaStream_t st);
// the tick's kicks; its last block ends the tick (flags [9], [11], the
// conditions when use_cond) and opens the next one
cudaError_t launch_block_kick(const BatchView &b, int L, bool use_cond, cudaGraphConditionalHandle cond,
                             cudaGraphConditionalHandle fin, cudaStream_t st);
cudaError_t launch_block_finish(const BatchView &b, cudaStream_t st);
cudaError_t launch_kick_close(const BatchView &b, int do_kick, int forces_ran, cudaStream_t st);
cudaError_t launch_reset_step(const BatchView &b, int mode, cudaStream_t st);  // mode 1 full, 2 forces only
cudaError_t launch_neighbour_export(const BatchView &b, int kind, const double *h_in, long long *offsets,
                                    int *idx, long long cap, long long *total_dev, cudaStream_t st);

// Reset of one problem's per-call diagnostics: mode 1 a whole step's, mode 2
// those of a forces-only call.
__device__ __forceinline__ void reset_diag(const BatchView &b, int p, int mode)
{
    ProbDiag *d = b.prob[p].diag;
    d->dt_min_bits = 0x7ff0000000000000ull;  // +inf
    d->force_pairs = 0;
    d->grav_pairs = d->grav_nodes = 0;
    if (mode == 2) return;
    d->wrap_leaves = 0;
    d->mass = 0;
    for (int a = 0; a < 3; ++a) {
        d->mom[a] = 0;
        d->fsum[a] = 0;
    }
    d->energy = 0;
    d->dEdt = 0;
    d->nr_iter = d->density_pairs = d->candidates = d->fallback = 0;
    d->ngb_sum = 0;
    d->nr_max = 0;
    d->ngb_min = 0x7fffffff;
    d->ngb_max = 0;
    d->status = 0;
    d->unconverged = 0;
}

// Clear per-call counter k (k < kNumCounters): mode 1 all of a step's,
// mode 2 those of a forces-only call.
__device__ __forceinline__ void reset_counter(const BatchView &b, int mode, int k)
{
    const bool all = (k >= kSlowCounter && k <= kForceWrapList) || k >= kTimeoutCounter;
    const bool forces = k == kForceWrapList || k == kTimeoutCounter ||
                        (k >= kForceCounter && k < kForceCounter + kForceClasses) ||
                        (k >= kForceWrapCounter && k < kForceWrapCounter + kForceClasses) ||
                        (k >= kForceCdCounter && k < kForceCdCounter + kForceClasses);
    if (mode == 1 ? all : forces) b.counters[k] = 0;
}

// the counters of a step or forces-only call (block 0, its first kNumCounters threads)
__device__ __forceinline__ void reset_counters(const BatchView &b, int mode)
{
    if (blockIdx.x == 0 && threadIdx.x < kNumCounters) reset_counter(b, mode, threadIdx.x);
}

// ---- host helpers shared by the entry points (sph_api.cu) -----------------
// Bump allocator over a workspace (base == nullptr measures the size).
struct Carver {
    char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += sizeof(T) * (count > 0 ? count : 1);
        return p;
    }
};
int fail(int code, const char *fmt, ...);  // records the thread's error message, returns code
void carve_arrays(Carver &c, BatchView &b, long long ntot, int nprob, int precision, int grav_chunks = 0,
                  int grav_tree = 0, int block = 0);
void carve_tables(Carver &c, BatchView &b, int nprob);
int key_bits_for(int nprob);
int key_low_bits(long long ntot);  // Morton bits left unsorted (cleared) for ntot particles
int mask_of(int lpp, int kernel);
int dens_class_bit(int lpp, int uniform_m, int kernel);
int validate(const sph_params *p);
PhysParams phys_of(const sph_params *p);
int lpp_of(const sph_params *p, long long n);
int status_to_code(unsigned st);

// upper bounds used to size grids and workspaces
long long leaves_upper_bound(long long n);
long long leaf_tiles(long long n);  // tiles of the leaf scan
long long sort_tiles(long long n);  // tiles of one radix-sort pass
int levels_needed(long long max_leaves);

}  // namespace sph
