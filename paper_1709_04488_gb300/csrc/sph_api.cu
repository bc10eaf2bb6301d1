// Host side of the C ABI (include/sph.h): parameter validation, workspace
// layout, context and batch bookkeeping, launch sequences, CUDA-graph capture
// of the step and status reporting.  No device memory is allocated here; every
// array lives in caller-owned workspaces.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "sph_internal.cuh"

namespace sph {

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(SPH_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                           __FILE__, __LINE__);                                      \
    } while (0)

DevInfo dev_info()
{
    static int cached_dev = -1, cached_sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cached_sms = sms > 0 ? sms : 1;
        cached_dev = dev;
    }
    return DevInfo{cached_sms};
}

// ---- workspace layout -------------------------------------------------------
// Carve the per-step scratch arrays for `ntot` particles over `nprob` problems.
void carve_arrays(Carver &c, BatchView &b, long long ntot, int nprob, int precision, int grav_chunks, int grav_tree,
                  int block)
{
    const long long n = ntot > 0 ? ntot : 1;
    const size_t v4 = precision == SPH_PREC_FP64 ? sizeof(dbl4) : sizeof(float4);
    const long long nblk = sort_tiles(n);
    const long long passes = (key_bits_for(nprob) + 7) / 8;
    b.keys[0] = c.take<unsigned long long>(n);
    b.keys[1] = c.take<unsigned long long>(n);
    b.vals[0] = c.take<unsigned>(n);
    b.vals[1] = c.take<unsigned>(n);
    b.hist = c.take<unsigned>(passes * 256 + 8 + passes * nblk * 256);
    b.perm = c.take<int>(n);
    double **sd[] = {&b.sx, &b.sy, &b.sz, &b.sh, &b.sm, &b.srho, &b.somega, &b.sP, &b.sc,
                     &b.vpx, &b.vpy, &b.vpz, &b.up, &b.ap};
    for (double **p : sd) *p = c.take<double>(n);
    void **st[] = {&b.pm, &b.ph, &b.vc, &b.th};
    for (void **p : st) *p = c.take<char>(v4 * n);
    b.sal = c.take<char>(v4 / 4 * n);
    b.scd = c.take<char>(v4 / 4 * n);
    b.divv = c.take<float>(n);
    b.cdold = c.take<double>(n);
    b.cdxi = c.take<double>(n);
    b.szg = c.take<char>(v4 / 4 * n);
    b.gpart = grav_chunks > 1 ? c.take<double>(3LL * grav_chunks * n) : nullptr;
    b.gpos = grav_tree ? (void *)c.take<char>(v4 * n) : nullptr;
    b.gh = grav_tree ? (void *)c.take<char>(v4 / 2 * n) : nullptr;
    int **bi[] = {&b.blev, &b.bnml, &b.breq, &b.bt0, &b.bt1};
    for (int **p : bi) *p = block ? c.take<int>(n) : nullptr;
    b.bvh = block ? c.take<double>(5 * n) : nullptr;
    b.bzeta = block ? c.take<double>(n) : nullptr;
    b.slev = block ? (void *)c.take<char>(v4 / 4 * n) : nullptr;
    b.btask = block ? c.take<int>(n) : nullptr;
    b.flag = c.take<unsigned>(n);
    const long long ml = leaves_upper_bound(n);
    b.max_leaves = (int)ml;
    b.leaf_start = c.take<int>(ml + 1);
    b.leaf_pid = c.take<int>(ml);
    b.leaf_c = c.take<double>(3 * ml);
    b.leaf_cf = c.take<float>(6 * ml);
    b.hf = c.take<float>(n);
    long long cap = ml;
    for (int l = 0; l <= kMaxLevels; ++l) {
        b.node_cap[l] = (int)cap;
        b.nodes[l] = c.take<NodeBox>(cap);
        b.gnode[l] = grav_tree ? (void *)c.take<char>(5 * v4 * cap) : nullptr;
        cap = cap / kBranch + nprob + 1;
    }
    b.ggrp = grav_tree ? (void *)c.take<char>(5 * v4 * 8 * (long long)b.node_cap[1]) : nullptr;
    b.fallback_list = c.take<int>(n);
    b.wrap_list = c.take<int>(n);
    b.group_cap = 2 * n;
    b.group_pool = c.take<int2>(b.group_cap);
    b.leaf_gofs = c.take<int>(ml);
    b.leaf_ngroups = c.take<int>(ml);
    b.leaf_hcap = c.take<float>(ml);
    b.counters = c.take<int>(kNumCounters);
    b.scratch64 = c.take<long long>(16);
    // zero region (kept zero by the kernels that use it)
    b.tile_state = c.take<unsigned>(leaf_tiles(n) + 2);
    b.zero_lo = (char *)b.tile_state;
    b.node_ctr[0] = nullptr;
    for (int l = 1; l <= kMaxLevels; ++l) b.node_ctr[l] = c.take<int>(b.node_cap[l]);
    b.zero_bytes = c.base ? (size_t)((char *)(b.node_ctr[kMaxLevels] + b.node_cap[kMaxLevels]) - b.zero_lo) : 0;
}

void carve_tables(Carver &c, BatchView &b, int nprob)
{
    b.nprob = nprob;
    b.prob = c.take<ProbStatic>(nprob);
    b.dyn = c.take<ProbDyn>(nprob);
    b.prob_base = c.take<long long>(nprob + 1);
}

// Up to 2^20 particles the finest two of the ten Morton levels are left
// unsorted: the 8-level cells (1/256 of the box per axis) already hold under
// one particle on average for such sizes, and the sort needs one pass fewer.
int key_low_bits(long long ntot) { return ntot <= (1ll << 20) ? 6 : 0; }

int key_bits_for(int nprob)
{
    int bits = 0;
    while ((1 << bits) < nprob) ++bits;
    return kMortonTotal + bits;
}

int mask_of(int lpp, int kernel)
{
    return (lpp == 1 ? 1 : lpp == 2 ? 2 : lpp == 4 ? 4 : 8) << (kernel == SPH_KERNEL_M6 ? 4 : 0);
}

int dens_class_bit(int lpp, int uniform_m, int kernel)
{
    return (lpp == 1 ? 1 : lpp == 2 ? 2 : lpp == 4 ? 4 : 8) << ((uniform_m ? 4 : 0) + (kernel == SPH_KERNEL_M6 ? 8 : 0));
}

// Lanes per particle by problem size: a table of (largest n, lanes) rows
// installed with sph_set_launch_table (the package's autotuner measures one
// and installs it when the library is loaded), else the built-in rule.
// Small problems spread a particle over more lanes so that the GPU stays full.
constexpr int kMaxTableRows = 32;
static std::mutex g_table_mu;
static int g_table_rows = 0;
static long long g_table_n[kMaxTableRows];
static int g_table_lpp[kMaxTableRows];

// The table and the rule are for the M4 kernel; the M6 kernel (support 3h,
// about twice the neighbours) takes twice the lanes, at least 2 and at most 8.
static int choose_lpp(long long n, int precision, int requested, int kernel)
{
    int l = requested;
    if (l == 0) {
        l = n <= 67023 ? 2 : 1;  // (the table the autotuner measured on GB300, for C callers without one)
        std::lock_guard<std::mutex> g(g_table_mu);
        for (int k = 0; k < g_table_rows; ++k)
            if (n <= g_table_n[k]) {
                l = g_table_lpp[k];
                break;
            }
    }
    if (l != 1 && l != 2 && l != 4 && l != 8) l = 4;
    if (kernel == SPH_KERNEL_M6 && requested == 0) l = l >= 4 ? 8 : 2 * l;
    if (kernel == SPH_KERNEL_M6 && l < 2) l = 2;
    if (precision == SPH_PREC_FP64) l = (l >= 4) ? 4 : 2;
    return l;
}

}  // namespace sph

using namespace sph;

struct sph_ctx {
    sph_params prm;
    long long n;
    sph_state st;
    void *ws;
    size_t ws_bytes;
    cudaStream_t stream;
    int lpp;
    BatchView bv;
    ProbDiag *diag;
    ProbStatic host_ps;
    bool have_forces;
    int since_build;              // steps since the leaves were last built
    cudaGraphExec_t graph;        // one step that rebuilds the leaves
    cudaGraphExec_t graph_reuse;  // one step that keeps them
    cudaGraphExec_t block_graph;  // one block step, its ticks a device-driven loop
    int graph_kernels;
    cudaEvent_t ev[SPH_NSTAGES + 1];
    bool timing;
    bool stage_ran[SPH_NSTAGES];
};

static void clear_ran(sph_ctx *c)
{
    for (int k = 0; k < SPH_NSTAGES; ++k) c->stage_ran[k] = false;
}

namespace sph {

int validate(const sph_params *p)
{
    if (!p) return fail(SPH_EINVAL, "params is NULL");
    if (p->av_switch != SPH_AV_CONSTANT && p->av_switch != SPH_AV_MORRIS_MONAGHAN &&
        p->av_switch != SPH_AV_CULLEN_DEHNEN)
        return fail(SPH_EINVAL, "av_switch %d not supported (0 = constant, 1 = Morris & Monaghan, 2 = Cullen & Dehnen)",
                    p->av_switch);
    if (p->av_switch == SPH_AV_MORRIS_MONAGHAN &&
        !(p->alpha_av > 0 && p->alpha_min >= 0 && p->alpha_min <= p->alpha_av && p->av_decay > 0))
        return fail(SPH_EINVAL, "viscosity switch needs alpha_av > 0, 0 <= alpha_min <= alpha_av, av_decay > 0");
    if (p->av_switch == SPH_AV_CULLEN_DEHNEN && !(p->alpha_av > 0 && p->av_decay > 0))
        return fail(SPH_EINVAL, "the Cullen & Dehnen switch needs alpha_av > 0 and av_decay > 0");
    if (p->av_switch == SPH_AV_CULLEN_DEHNEN && p->block_levels > 0)
        return fail(SPH_EINVAL, "the Cullen & Dehnen switch is not combined with block time-steps");
    if (p->gravity != 0 && p->gravity != 1) return fail(SPH_EINVAL, "gravity must be 0 or 1");
    if (p->gravity && !(p->grav_theta >= 0.0 && p->grav_theta <= 1.0))
        return fail(SPH_EINVAL, "grav_theta must lie in [0, 1]");
    if (p->gravity && !(p->c_grav > 0)) return fail(SPH_EINVAL, "c_grav must be > 0");
    if (p->block_levels < 0 || p->block_levels > 20) return fail(SPH_EINVAL, "block_levels must lie in [0, 20]");
    if (p->block_levels > 0 && (p->block_gap < 1 || p->block_gap > 20))
        return fail(SPH_EINVAL, "block_gap must lie in [1, 20]");
    if (p->gravity && (p->periodic || p->kernel != SPH_KERNEL_M4 || !(p->G > 0)))
        return fail(SPH_EINVAL, "self-gravity needs an isolated problem, the M4 kernel and G > 0");
    if (p->ac_signal != SPH_AC_WADSLEY && p->ac_signal != SPH_AC_PRICE)
        return fail(SPH_EINVAL, "ac_signal %d not supported (0 = Wadsley, 1 = Price)", p->ac_signal);
    if (p->kernel != SPH_KERNEL_M4 && p->kernel != SPH_KERNEL_M6)
        return fail(SPH_EINVAL, "kernel %d not supported (0 = M4 cubic spline, 1 = M6 quintic spline)", p->kernel);
    if (p->periodic != 0 && p->periodic != 1) return fail(SPH_EINVAL, "periodic must be 0 or 1");
    if (p->periodic)
        for (int a = 0; a < 3; ++a)
            if (!(p->box_len[a] > 0) || !std::isfinite(p->box_len[a]) || !std::isfinite(p->box_lo[a]))
                return fail(SPH_EINVAL, "periodic box_len[%d] must be positive and finite", a);
    if (p->eos != SPH_EOS_ADIABATIC && p->eos != SPH_EOS_ISOTHERMAL) return fail(SPH_EINVAL, "unknown eos %d", p->eos);
    if (p->eos == SPH_EOS_ADIABATIC && !(p->gamma > 1.0)) return fail(SPH_EINVAL, "gamma must exceed 1");
    if (p->eos == SPH_EOS_ISOTHERMAL && !(p->cs_iso > 0)) return fail(SPH_EINVAL, "cs_iso must be positive");
    if (!(p->eta > 0) || !std::isfinite(p->eta)) return fail(SPH_EINVAL, "eta must be positive");
    if (!(p->alpha_av >= 0) || !(p->beta_av >= 0) || !(p->alpha_ac >= 0))
        return fail(SPH_EINVAL, "dissipation coefficients must be non-negative");
    if (!(p->c_cfl > 0)) return fail(SPH_EINVAL, "c_cfl must be positive");
    if (!(p->h_tol >= 0) || p->h_max_iter < 0) return fail(SPH_EINVAL, "bad h_tol / h_max_iter");
    if (p->precision != SPH_PREC_FP64 && p->precision != SPH_PREC_MIXED)
        return fail(SPH_EINVAL, "unknown precision %d", p->precision);
    if (p->lanes_per_particle != 0 && p->lanes_per_particle != 1 && p->lanes_per_particle != 2 &&
        p->lanes_per_particle != 4 && p->lanes_per_particle != 8)
        return fail(SPH_EINVAL, "lanes_per_particle must be 0, 1, 2, 4 or 8");
    if (p->leaf_size != 0 && p->leaf_size != 4 && p->leaf_size != 8 && p->leaf_size != 16 && p->leaf_size != 32)
        return fail(SPH_EINVAL, "leaf_size must be 0, 4, 8, 16 or 32");
    return SPH_OK;
}

PhysParams phys_of(const sph_params *p)
{
    PhysParams ph;
    memset(&ph, 0, sizeof ph);
    ph.periodic = p->periodic;
    ph.eos = p->eos;
    for (int a = 0; a < 3; ++a) {
        ph.box_lo[a] = p->box_lo[a];
        ph.box_len[a] = p->periodic ? p->box_len[a] : 0.0;
        ph.box_len_f[a] = (float)ph.box_len[a];
        ph.box_inv[a] = p->periodic ? 1.0 / ph.box_len[a] : 0.0;
        ph.box_inv_f[a] = p->periodic ? 1.0f / ph.box_len_f[a] : 0.f;
    }
    ph.gamma = p->gamma;
    ph.cs_iso = p->cs_iso;
    ph.eta = p->eta;
    ph.alpha_av = p->alpha_av;
    ph.beta_av = p->beta_av;
    ph.alpha_ac = p->alpha_ac;
    ph.c_cfl = p->c_cfl;
    ph.h_tol = p->h_tol > 0 ? p->h_tol : (p->precision == SPH_PREC_FP64 ? 1e-13 : 1e-6);
    ph.h_max_iter = p->h_max_iter > 0 ? p->h_max_iter : 50;
    ph.kernel = p->kernel;
    ph.ac_signal = p->ac_signal;
    ph.av_switch = p->av_switch;
    ph.alpha_min = p->alpha_min;
    ph.av_decay = p->av_decay;
    ph.beta_ratio = p->alpha_av > 0 ? p->beta_av / p->alpha_av : 0.0;
    ph.gravity = p->gravity;
    ph.G = p->G;
    ph.grav_theta = p->grav_theta;
    ph.c_grav = p->c_grav;
    ph.block = p->block_levels;
    ph.block_gap = p->block_gap;
    ph.kr = p->kernel == SPH_KERNEL_M6 ? 3.0 : 2.0;
    ph.kr_f = (float)ph.kr;
    return ph;
}

int lpp_of(const sph_params *p, long long n)
{
    int req = p->lanes_per_particle;
    if (req == 0 && p->leaf_size != 0) req = 32 / p->leaf_size;
    return choose_lpp(n, p->precision, req, p->kernel);
}

int status_to_code(unsigned st)
{
    if (st & ST_NONFINITE) return fail(SPH_ENONFINITE, "non-finite value in the results");
    if (st & ST_BOX) return fail(SPH_EBOX, "kernel support (R_K h) reached half the periodic box");
    if (st & ST_TIMEOUT) return fail(SPH_ETIMEOUT, "a bounded device wait gave up");
    if (st & ST_OVERFLOW) return fail(SPH_ENOSPACE, "an internal capacity was exceeded");
    if (st & ST_SCHEDULE) return fail(SPH_ECUDA, "block step: the next event tick does not follow the current one");
    if (st & ST_NOCONV) return fail(SPH_ENOCONV, "h-rho iteration did not converge for some particles");
    return SPH_OK;
}

}  // namespace sph

extern "C" {

const char *sph_last_error(void) { return g_err.c_str(); }

const char *sph_version(void) { return "gb300-sph 0.1 (sm_103a)"; }

int sph_set_launch_table(const int64_t *n_max, const int32_t *lanes, int rows)
{
    if (rows < 0 || rows > kMaxTableRows) return fail(SPH_EINVAL, "rows must be in [0, %d]", kMaxTableRows);
    if (rows > 0 && (!n_max || !lanes)) return fail(SPH_EINVAL, "NULL table");
    for (int k = 0; k < rows; ++k) {
        if (lanes[k] != 1 && lanes[k] != 2 && lanes[k] != 4 && lanes[k] != 8)
            return fail(SPH_EINVAL, "row %d: lanes per particle must be 1, 2, 4 or 8", k);
        if (k > 0 && n_max[k] <= n_max[k - 1]) return fail(SPH_EINVAL, "row %d: n_max must increase", k);
    }
    std::lock_guard<std::mutex> g(g_table_mu);
    for (int k = 0; k < rows; ++k) {
        g_table_n[k] = (long long)n_max[k];
        g_table_lpp[k] = lanes[k];
    }
    g_table_rows = rows;
    return SPH_OK;
}

int sph_params_default(sph_params *p)
{
    if (!p) return fail(SPH_EINVAL, "params is NULL");
    memset(p, 0, sizeof *p);
    p->periodic = 1;
    for (int a = 0; a < 3; ++a) {
        p->box_lo[a] = 0.0;
        p->box_len[a] = 1.0;
    }
    p->eos = SPH_EOS_ADIABATIC;
    p->gamma = 5.0 / 3.0;
    p->cs_iso = 1.0;
    p->eta = 1.2;
    p->alpha_av = 1.0;
    p->beta_av = 2.0;
    p->alpha_ac = 1.0;
    p->c_cfl = 0.2;
    p->h_tol = 0.0;
    p->h_max_iter = 50;
    p->precision = SPH_PREC_MIXED;
    p->alpha_min = 0.1;
    p->c_grav = 0.5;
    p->block_gap = 2;
    p->av_decay = 0.1;
    return SPH_OK;
}

size_t sph_workspace_bytes(int64_t n, const sph_params *p)
{
    if (n < 0 || validate(p) != SPH_OK) return 0;
    Carver c{nullptr};
    c.take<ProbDiag>(1);
    BatchView b;
    memset(&b, 0, sizeof b);
    carve_tables(c, b, 1);
    carve_arrays(c, b, n, 1, p->precision, p->gravity ? gravity_chunks(n, p->grav_theta) : 0,
                 p->gravity && p->grav_theta > 0, p->block_levels > 0);
    return c.off + 256;
}

int sph_setup(sph_ctx **out, const sph_params *p, int64_t n, const sph_state *state, void *workspace,
              size_t ws_bytes, void *stream)
{
    if (!out) return fail(SPH_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    if (n < 0 || n > (int64_t)1 << 30) return fail(SPH_EINVAL, "n = %lld out of range", (long long)n);
    if (!state) return fail(SPH_EINVAL, "state is NULL");
    if (n > 0) {
        const double *req[] = {state->x, state->y, state->z, state->vx, state->vy, state->vz, state->u,
                               state->m, state->h, state->rho, state->omega, state->P, state->c,
                               state->ax, state->ay, state->az, state->du, state->vsig};
        for (const double *q : req)
            if (!q) return fail(SPH_EINVAL, "a state array is NULL");
        if (p->av_switch && (!state->alpha || !state->dalpha))
            return fail(SPH_EINVAL, "the viscosity switch needs state.alpha and state.dalpha");
    }
    size_t need = sph_workspace_bytes(n, p);
    if (!workspace || ws_bytes < need)
        return fail(SPH_ENOSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
    if (((uintptr_t)workspace) & 255) return fail(SPH_EINVAL, "workspace must be 256-byte aligned");
    sph_ctx *c = new sph_ctx();
    c->prm = *p;
    c->n = n;
    c->st = *state;
    c->ws = workspace;
    c->ws_bytes = ws_bytes;
    c->stream = (cudaStream_t)stream;
    c->lpp = lpp_of(p, n);
    c->have_forces = false;
    c->since_build = 0;
    c->graph = nullptr;
    c->graph_reuse = nullptr;
    c->block_graph = nullptr;
    c->graph_kernels = 0;
    c->timing = (p->flags & SPH_FLAG_TIMING) != 0;
    for (int k = 0; k <= SPH_NSTAGES; ++k) c->ev[k] = nullptr;
    clear_ran(c);
    if (c->timing)
        for (int k = 0; k <= SPH_NSTAGES; ++k)
            if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
                delete c;
                return fail(SPH_ECUDA, "cudaEventCreate failed");
            }
    Carver cv{(char *)workspace};
    c->diag = cv.take<ProbDiag>(1);
    memset(&c->bv, 0, sizeof c->bv);
    carve_tables(cv, c->bv, 1);
    carve_arrays(cv, c->bv, n, 1, p->precision, p->gravity ? gravity_chunks(n, p->grav_theta) : 0,
                 p->gravity && p->grav_theta > 0, p->block_levels > 0);
    c->bv.ntot = n;
    c->bv.key_bits = key_bits_for(1);
    c->bv.key_lo = key_low_bits(n);
    c->bv.lpp_mask = mask_of(c->lpp, p->kernel);
    c->bv.any_isolated = p->periodic ? 0 : 1;
    c->bv.any_periodic = p->periodic ? 1 : 0;
    c->bv.any_general = (p->av_switch || p->ac_signal || p->gravity) ? 1 : 0;
    c->bv.any_gravity = p->gravity ? 1 : 0;
    c->bv.any_cd = p->av_switch == SPH_AV_CULLEN_DEHNEN ? 1 : 0;
    c->bv.grav_blocks = p->gravity ? gravity_blocks(n, p->grav_theta) : 0;
    c->bv.grav_split = p->gravity && gravity_chunks(n, p->grav_theta) > 1;
    c->bv.any_grav_tree = p->gravity && p->grav_theta > 0;
    ProbStatic &ps = c->host_ps;
    memset(&ps, 0, sizeof ps);
    ps.x = state->x;
    ps.y = state->y;
    ps.z = state->z;
    ps.vx = state->vx;
    ps.vy = state->vy;
    ps.vz = state->vz;
    ps.u = state->u;
    ps.m = state->m;
    ps.h = state->h;
    ps.rho = state->rho;
    ps.omega = state->omega;
    ps.P = state->P;
    ps.c = state->c;
    ps.ax = state->ax;
    ps.ay = state->ay;
    ps.az = state->az;
    ps.du = state->du;
    ps.vsig = state->vsig;
    ps.alpha = state->alpha;
    ps.dalpha = state->dalpha;
    ps.n = n;
    ps.base = 0;
    ps.diag = c->diag;
    ps.lpp = c->lpp;
    ps.ph = phys_of(p);
    ps.gchunks = p->gravity ? gravity_chunks(n, p->grav_theta) : 0;
    // equal masses (the usual SPH set-up; masses never change) let the
    // density lists keep distances only
    if (n > 0) {
        std::vector<double> mh((size_t)n);
        cudaError_t me = cudaMemcpyAsync(mh.data(), state->m, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                                         c->stream);
        if (me == cudaSuccess) me = cudaStreamSynchronize(c->stream);
        if (me != cudaSuccess) {
            delete c;
            return fail(SPH_ECUDA, "reading the masses failed: %s", cudaGetErrorString(me));
        }
        bool uni = true;
        for (long long k = 1; k < n && uni; ++k) uni = mh[(size_t)k] == mh[0];
        ps.uniform_m = uni ? 1 : 0;
        ps.m_uniform = mh[0];
        ps.inv_m_uniform = uni && mh[0] != 0.0 ? 1.0 / mh[0] : 0.0;
    }
    c->bv.dens_mask = dens_class_bit(c->lpp, ps.uniform_m, p->kernel);
    ProbDiag d0;
    memset(&d0, 0, sizeof d0);
    d0.dt_next = 0.0;
    long long bases[2] = {0, n};
    cudaError_t e = cudaMemcpyAsync(c->bv.prob, &ps, sizeof ps, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->diag, &d0, sizeof d0, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->bv.prob_base, bases, sizeof bases, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bv.dyn, 0, sizeof(ProbDyn), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bv.counters, 0, kNumCounters * sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->bv.zero_lo, 0, c->bv.zero_bytes, c->stream);
    if (e == cudaSuccess && c->bv.blev) {  // block steps: level 0, no neighbour levels yet
        e = cudaMemsetAsync(c->bv.blev, 0, sizeof(int) * (size_t)(n > 0 ? n : 1), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->bv.bnml, 0, sizeof(int) * (size_t)(n > 0 ? n : 1), c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete c;
        return fail(SPH_ECUDA, "setup copies failed: %s", cudaGetErrorString(e));
    }
    *out = c;
    return SPH_OK;
}

}  // extern "C"

// ---- launch sequences (shared by single contexts and batches) --------------
// Optional stage events: ev[k] is recorded before stage k, ev[k+1] after it.
struct Marks {
    cudaEvent_t *ev = nullptr;
    bool *ran = nullptr;
    void at(int k, cudaStream_t st) const
    {
        if (!ev) return;
        // inside stream capture the record must become a graph node of its own
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev[k], st, cudaEventRecordExternal);
        else cudaEventRecord(ev[k], st);
    }
    void done(int k) const
    {
        if (ran) ran[k] = true;
    }
};

// rebuild: new keys, sort and leaves; otherwise the leaves of the last build
// keep their particles (gathered again by the last permutation) and only
// their offsets and boxes, and the nodes above them, are recomputed
static int enqueue_density(const BatchView &b, int precision, int use_pred, cudaStream_t st, const Marks &mk,
                           bool rebuild = true)
{
    mk.at(SPH_STAGE_SORT, st);
    if (rebuild) {
        CU(launch_domain_and_keys(b, st));
        CU(launch_radix_sort(b, st));
    }
    CU(launch_gather(b, st));
    mk.at(SPH_STAGE_TREE, st);
    mk.done(SPH_STAGE_SORT);
    if (rebuild) CU(launch_build_leaves(b, precision, st));
    else CU(launch_update_leaves(b, precision, st));
    mk.at(SPH_STAGE_DENSITY, st);
    mk.done(SPH_STAGE_TREE);
    CU(launch_density(b, precision, use_pred, st));
    mk.at(SPH_STAGE_REFIT, st);
    mk.done(SPH_STAGE_DENSITY);
    CU(launch_refit(b, precision, st));
    mk.at(SPH_STAGE_FORCES, st);
    mk.done(SPH_STAGE_REFIT);
    return SPH_OK;
}

static int enqueue_step(const BatchView &b, int precision, double dt, cudaStream_t st, const Marks &mk,
                        bool rebuild = true)
{
    mk.at(SPH_STAGE_KICK_DRIFT, st);
    CU(launch_kick_drift(b, dt, st));
    mk.done(SPH_STAGE_KICK_DRIFT);
    int rc = enqueue_density(b, precision, 1, st, mk, rebuild);
    if (rc) return rc;
    CU(launch_forces(b, precision, st));
    mk.at(SPH_STAGE_GRAVITY, st);
    mk.done(SPH_STAGE_FORCES);
    launch_gravity(b, precision, st);  // adds the long-range attraction to a
    CU(cudaGetLastError());
    mk.at(SPH_STAGE_CLOSE, st);
    if (b.any_gravity) mk.done(SPH_STAGE_GRAVITY);
    CU(launch_kick_close(b, 1, 1, st));
    mk.at(SPH_NSTAGES, st);
    mk.done(SPH_STAGE_CLOSE);
    return SPH_OK;
}

static Marks marks_of(sph_ctx *c)
{
    Marks m;
    if (c->timing) {
        m.ev = c->ev;
        m.ran = c->stage_ran;
    }
    return m;
}



// tree reuse cadence (sph_params.tree_rebuild_every)
static bool next_is_rebuild(const sph_ctx *c)
{
    const int every = c->prm.tree_rebuild_every;
    return every <= 1 || c->since_build + 1 >= every;
}

static void count_step(sph_ctx *c, bool rebuild) { c->since_build = rebuild ? 0 : c->since_build + 1; }

static int finish_call(sph_ctx *c)
{
    if (c->prm.flags & SPH_FLAG_ASYNC) return SPH_OK;
    return sph_sync(c);
}

// ---- block time-steps (Sec. 2.1.4) -----------------------------------------
// One block step: Delta t_MAX and the opening kicks, then one tick per event
// (a tick where some particle's step ends) before 2^L, then the last tick at
// 2^L (every particle due), then the conservation sums.  The schedule lives
// on the device; on a capturable stream the ticks before 2^L are the body of
// a graph loop (a conditional while node) and the last tick a conditional
// branch, whose conditions the last block of each tick's kick sets, so no
// host round trip separates the ticks.

// tasks: the ticks before 2^L, whose pair kernels serve tasks of up to 32 /
// block_lanes particles whose step ends, block_lanes lanes each; else the
// last tick, whose pair kernels serve whole leaves (as a global step's do)
static BatchView block_view(const sph_ctx *c, bool tasks = true)
{
    BatchView b = c->bv;
    b.block_on = 1;
    b.block_tasks = tasks ? 1 : 0;
    b.any_general = 1;  // the active particles' forces run in the wrap-list launch
    b.block_lanes = c->prm.precision == SPH_PREC_FP64                    ? kBlockLanesF64
                    : c->prm.kernel == SPH_KERNEL_M6 || c->prm.gravity ? kBlockLanesF32Walk
                                                                       : kBlockLanesF32;
    if (tasks) {
        b.lpp_mask = mask_of(b.block_lanes, c->prm.kernel);
        b.dens_mask = dens_class_bit(b.block_lanes, c->host_ps.uniform_m, c->prm.kernel);
    }
    return b;
}

static int block_every(const sph_ctx *c) { return c->prm.tree_rebuild_every > 1 ? c->prm.tree_rebuild_every : 1; }

// With tree reuse the block starts from the context's leaves (those of the
// last build or refit: the previous block's last tick, a global step, the
// density solve), and the ticks k > 0 with k a multiple of
// tree_rebuild_every sort and build afresh; every tick does without reuse.
// A cadence of at least 2^L ticks never rebuilds inside the loop.
static bool block_loop_rebuilds(const sph_ctx *c) { return block_every(c) < (1 << c->prm.block_levels); }
static bool block_tick_rebuilds(const sph_ctx *c, long long tick)
{
    const int every = block_every(c);
    return every == 1 || (tick > 0 && tick % every == 0 && block_loop_rebuilds(c));
}

// the tick's drift and leaves.  Tree reuse (Sec. 4.2) between ticks as
// between global steps: sort and build on every tree_rebuild_every-th tick;
// between, the order and the leaves are kept (the drift runs in sorted order
// with the gather) and the leaves refitted
static int enqueue_block_leaves(const BatchView &b, int prec, bool rebuild, cudaStream_t st)
{
    if (rebuild) {
        CU(launch_block_drift(b, st));
        CU(launch_domain_and_keys(b, st));
        CU(launch_radix_sort(b, st));
        CU(launch_block_gather(b, prec, st));  // (also which particles end their step now)
        CU(launch_build_leaves(b, prec, st));
        CU(launch_block_tasks(b, prec, st));  // (and the restaging of the particles that keep their solve)
    } else {
        CU(launch_block_leaf_tick(b, prec, st));  // drift, gather, leaf boxes, tasks and restaging
    }
    return SPH_OK;
}

static int enqueue_block_passes(const BatchView &b, int prec, int L, bool use_cond, cudaGraphConditionalHandle loop,
                                cudaGraphConditionalHandle fin, cudaStream_t st)
{
    CU(launch_density(b, prec, 1, st));  // solves the particles whose step ends
    CU(launch_refit(b, prec, st));
    CU(launch_forces(b, prec, st));
    launch_gravity(b, prec, st);  // the long range of the active particles
    CU(cudaGetLastError());
    CU(launch_block_kick(b, L, use_cond, loop, fin, st));  // (its last block ends the tick, opens the next)
    return SPH_OK;
}

// the last tick (2^L, every particle due): sort and leaves built afresh (the
// next block starts from them), whole leaves in the pair kernels
static int enqueue_block_last(const BatchView &bl, int prec, int L, cudaStream_t st)
{
    CU(launch_block_drift(bl, st));
    CU(launch_domain_and_keys(bl, st));
    CU(launch_radix_sort(bl, st));
    CU(launch_block_gather(bl, prec, st));
    CU(launch_build_leaves(bl, prec, st));
    return enqueue_block_passes(bl, prec, L, false, 0, 0, st);
}

// the legacy default stream: the host reads the flags after every tick
static int block_step_eager(sph_ctx *c, const BatchView &b, const BatchView &bl)
{
    const int L = c->prm.block_levels, prec = c->prm.precision;
    cudaStream_t st = c->stream;
    CU(launch_block_dt(b, L, st));
    CU(launch_block_open(b, L, st));
    CU(launch_block_gate(b, L, false, 0, 0, st));
    long long fl[3] = {0, 0, 0};  // [9] loop, [10], [11] last tick
    for (long long tick = 0;; ++tick) {
        CU(cudaMemcpyAsync(fl, b.scratch64 + 9, sizeof fl, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        if (!fl[0]) break;
        if (tick >= (1LL << L)) return fail(SPH_ECUDA, "block step: more than 2^L ticks");
        int rc = enqueue_block_leaves(b, prec, block_tick_rebuilds(c, tick), st);
        if (rc) return rc;
        rc = enqueue_block_passes(b, prec, L, false, 0, 0, st);
        if (rc) return rc;
    }
    if (fl[2]) {
        int rc = enqueue_block_last(bl, prec, L, st);
        if (rc) return rc;
    }
    CU(launch_kick_close(b, 0, 1, st));  // conservation sums of the synchronised state
    CU(launch_block_finish(b, st));
    return SPH_OK;
}

// adds a conditional node of `type` after the capture's current dependencies
// and makes it the stream's only dependency; returns its body graphs
static int add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                           unsigned size, cudaGraph_t **bodies)
{
    cudaStreamCaptureStatus cs;
    unsigned long long id = 0;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CU(cudaStreamGetCaptureInfo(s, &cs, &id, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = size;
    cudaGraphNode_t node = nullptr;
    CU(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    CU(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    *bodies = np.conditional.phGraph_out;
    return SPH_OK;
}

static int capture_graph(cudaStream_t s, cudaGraph_t *g_out)
{
    cudaStreamCaptureStatus cs;
    unsigned long long id = 0;
    CU(cudaStreamGetCaptureInfo(s, &cs, &id, g_out, nullptr, nullptr, nullptr));
    return SPH_OK;
}

// ends a capture into a conditional body (the graph stays its node's)
static int end_body_capture(cudaStream_t s, int rc)
{
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &g);
    if (rc) return rc;
    CU(e);
    return SPH_OK;
}

// one tick into the loop body (stream s2; s3 captures the branches)
static int capture_tick(const sph_ctx *c, const BatchView &b, cudaGraphConditionalHandle loop,
                        cudaGraphConditionalHandle fin, cudaStream_t s2, cudaStream_t s3)
{
    const int L = c->prm.block_levels, prec = c->prm.precision, every = block_every(c);
    const bool branch = every > 1 && block_loop_rebuilds(c);  // some ticks rebuild, others keep
    cudaGraphConditionalHandle rb = 0;
    if (branch) {
        cudaGraph_t body = nullptr;
        int rc = capture_graph(s2, &body);
        if (rc) return rc;
        CU(cudaGraphConditionalHandleCreate(&rb, body, 0, 0));
        CU(launch_block_tick_begin(b, every, rb, s2));
    }
    if (branch) {
        cudaGraph_t *br = nullptr;
        int rc = add_conditional(s2, rb, cudaGraphCondTypeIf, 2, &br);  // [0] rebuild, [1] keep the leaves
        if (rc) return rc;
        for (int k = 0; k < 2; ++k) {
            CU(cudaStreamBeginCaptureToGraph(s3, br[k], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
            rc = end_body_capture(s3, enqueue_block_leaves(b, prec, k == 0, s3));
            if (rc) return rc;
        }
    } else {
        int rc = enqueue_block_leaves(b, prec, every == 1, s2);
        if (rc) return rc;
    }
    return enqueue_block_passes(b, prec, L, true, loop, fin, s2);
}

static int capture_block(const sph_ctx *c, const BatchView &b, const BatchView &bl, cudaStream_t s2, cudaStream_t s3)
{
    const int L = c->prm.block_levels, prec = c->prm.precision;
    cudaStream_t st = c->stream;
    cudaGraph_t g = nullptr;
    int rc = capture_graph(st, &g);
    if (rc) return rc;
    cudaGraphConditionalHandle loop = 0, fin = 0;
    CU(cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault));
    CU(cudaGraphConditionalHandleCreate(&fin, g, 0, cudaGraphCondAssignDefault));
    CU(launch_block_dt(b, L, st));
    CU(launch_block_open(b, L, st));
    CU(launch_block_gate(b, L, true, loop, fin, st));
    cudaGraph_t *body = nullptr;
    rc = add_conditional(st, loop, cudaGraphCondTypeWhile, 1, &body);
    if (rc) return rc;
    CU(cudaStreamBeginCaptureToGraph(s2, body[0], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    rc = end_body_capture(s2, capture_tick(c, b, loop, fin, s2, s3));
    if (rc) return rc;
    rc = add_conditional(st, fin, cudaGraphCondTypeIf, 1, &body);  // the last tick
    if (rc) return rc;
    CU(cudaStreamBeginCaptureToGraph(s2, body[0], nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    rc = end_body_capture(s2, enqueue_block_last(bl, prec, L, s2));
    if (rc) return rc;
    CU(launch_kick_close(b, 0, 1, st));  // conservation sums of the synchronised state
    CU(launch_block_finish(b, st));
    return SPH_OK;
}

static int build_block_graph(sph_ctx *c, const BatchView &b, const BatchView &bl)
{
    cudaStream_t s2 = nullptr, s3 = nullptr;
    CU(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamCreateWithFlags(&s3, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s2);
        return fail(SPH_ECUDA, "stream creation failed: %s", cudaGetErrorString(e));
    }
    int rc = SPH_OK;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = capture_block(c, b, bl, s2, s3);
        for (cudaStream_t s : {s3, s2}) {  // a capture left open by a failure
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t gb = nullptr;
                cudaStreamEndCapture(s, &gb);
            }
        }
        e = cudaStreamEndCapture(c->stream, &g);
    }
    cudaStreamDestroy(s2);
    cudaStreamDestroy(s3);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(SPH_ECUDA, "block-step graph capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(&c->block_graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->block_graph = nullptr;
        return fail(SPH_ECUDA, "block-step graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return SPH_OK;
}

extern "C" {

int sph_sync(sph_ctx *c)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    CU(cudaStreamSynchronize(c->stream));
    unsigned st = 0;
    CU(cudaMemcpy(&st, &c->diag->status, sizeof st, cudaMemcpyDeviceToHost));
    return status_to_code(st);
}

int sph_block_step(sph_ctx *c, double *dtmax_out, int64_t *evals_out)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    const int L = c->prm.block_levels;
    if (L <= 0 || !c->bv.blev) return fail(SPH_EINVAL, "the context was set up without block_levels");
    if (!c->have_forces) return fail(SPH_EINVAL, "sph_block_step needs a force evaluation first");
    if (c->n == 0) return SPH_OK;
    clear_ran(c);
    const BatchView b = block_view(c), bl = block_view(c, false);
    cudaStream_t st = c->stream;
    if (block_every(c) > 1 && c->since_build >= block_every(c)) {
        // the context's leaves do not hold its particles (a batch moved them): build them first
        CU(launch_domain_and_keys(c->bv, st));
        CU(launch_radix_sort(c->bv, st));
        CU(launch_gather(c->bv, st));
        CU(launch_build_leaves(c->bv, c->prm.precision, st));
    }
    if (st == nullptr) {
        int rc = block_step_eager(c, b, bl);  // the legacy default stream cannot be captured
        if (rc) return rc;
    } else {
        if (!c->block_graph) {
            int rc = build_block_graph(c, b, bl);
            if (rc) return rc;
        }
        CU(cudaGraphLaunch(c->block_graph, st));
    }
    long long evals = 0, dbits = 0;
    CU(cudaMemcpyAsync(&evals, b.scratch64 + 3, sizeof evals, cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&dbits, b.scratch64 + 6, sizeof dbits, cudaMemcpyDeviceToHost, st));
    int rc = sph_sync(c);
    double dtmax;
    memcpy(&dtmax, &dbits, sizeof dtmax);
    if (dtmax_out) *dtmax_out = dtmax;
    if (evals_out) *evals_out = evals;
    c->have_forces = true;
    c->since_build = 0;  // the last tick built the leaves
    return rc;
}

int sph_block_prepare(sph_ctx *c)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    if (c->prm.block_levels <= 0 || !c->bv.blev) return fail(SPH_EINVAL, "the context was set up without block_levels");
    if (c->stream == nullptr || c->block_graph || c->n == 0) return SPH_OK;
    return build_block_graph(c, block_view(c), block_view(c, false));
}

int sph_block_levels(sph_ctx *c, int32_t *levels)
{
    if (!c || !levels) return fail(SPH_EINVAL, "NULL argument");
    if (!c->bv.blev) return fail(SPH_EINVAL, "the context was set up without block_levels");
    if (c->n == 0) return SPH_OK;
    CU(cudaMemcpyAsync(levels, c->bv.blev, sizeof(int32_t) * (size_t)c->n, cudaMemcpyDeviceToDevice, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return SPH_OK;
}

int sph_density_h(sph_ctx *c)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    clear_ran(c);
    CU(launch_reset_step(c->bv, 1, c->stream));
    int rc = enqueue_density(c->bv, c->prm.precision, 0, c->stream, marks_of(c));
    if (rc) return rc;
    CU(launch_kick_close(c->bv, 0, 0, c->stream));
    c->have_forces = false;
    c->since_build = 0;
    return finish_call(c);
}

int sph_forces(sph_ctx *c)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    clear_ran(c);
    Marks mk = marks_of(c);
    CU(launch_reset_step(c->bv, 2, c->stream));
    mk.at(SPH_STAGE_FORCES, c->stream);
    CU(launch_forces(c->bv, c->prm.precision, c->stream));
    mk.at(SPH_STAGE_GRAVITY, c->stream);
    mk.done(SPH_STAGE_FORCES);
    launch_gravity(c->bv, c->prm.precision, c->stream);
    CU(cudaGetLastError());
    mk.at(SPH_STAGE_CLOSE, c->stream);
    if (c->bv.any_gravity) mk.done(SPH_STAGE_GRAVITY);
    CU(launch_kick_close(c->bv, 0, 1, c->stream));
    c->have_forces = true;
    return finish_call(c);
}

int sph_step(sph_ctx *c, double dt, double *dt_used)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    if (!(dt > 0) && !c->have_forces)
        return fail(SPH_EINVAL, "no CFL step yet: call sph_density_h and sph_forces first, or pass dt > 0");
    if (!std::isfinite(dt)) return fail(SPH_EINVAL, "dt must be finite");
    clear_ran(c);
    const bool rebuild = next_is_rebuild(c);
    int rc = enqueue_step(c->bv, c->prm.precision, dt, c->stream, marks_of(c), rebuild);
    if (rc) return rc;
    count_step(c, rebuild);
    c->have_forces = true;
    if (dt_used) {
        CU(cudaMemcpyAsync(dt_used, &c->diag->dt_cur, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CU(cudaStreamSynchronize(c->stream));
    }
    return finish_call(c);
}

static int build_graph(sph_ctx *c, bool rebuild = true)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    clear_ran(c);
    int rc = enqueue_step(c->bv, c->prm.precision, -1.0, c->stream, marks_of(c), rebuild);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(SPH_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int kern = 0;
    for (size_t k = 0; k < nn; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
    }
    cudaGraphExec_t *slot = rebuild ? &c->graph : &c->graph_reuse;
    if (rebuild) c->graph_kernels = kern;
    e = cudaGraphInstantiate(slot, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        *slot = nullptr;
        return fail(SPH_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    return SPH_OK;
}

int sph_run(sph_ctx *c, int nsteps)
{
    if (!c) return fail(SPH_EINVAL, "ctx is NULL");
    if (nsteps < 0) return fail(SPH_EINVAL, "nsteps must be >= 0");
    if (!c->have_forces) return fail(SPH_EINVAL, "no CFL step yet: call sph_density_h and sph_forces first");
    if (nsteps == 0) return SPH_OK;
    for (int k = 0; k < nsteps; ++k) {
        const bool rebuild = next_is_rebuild(c);
        cudaGraphExec_t *slot = rebuild ? &c->graph : &c->graph_reuse;
        if (c->stream == nullptr || !*slot) {
            // the legacy default stream cannot be captured: enqueue eagerly;
            // otherwise one eager step first so that lazily set kernel
            // attributes are in place, then capture this kind of step
            clear_ran(c);
            int rc = enqueue_step(c->bv, c->prm.precision, -1.0, c->stream, marks_of(c), rebuild);
            if (rc) return rc;
            if (c->stream != nullptr) {
                rc = build_graph(c, rebuild);
                if (rc) return rc;
            }
        } else {
            CU(cudaGraphLaunch(*slot, c->stream));
        }
        count_step(c, rebuild);
    }
    return finish_call(c);
}

int sph_stage_times(sph_ctx *c, double *ms)
{
    if (!c || !ms) return fail(SPH_EINVAL, "NULL argument");
    if (!c->timing) return fail(SPH_EINVAL, "context was created without SPH_FLAG_TIMING");
    CU(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < SPH_NSTAGES; ++k) {
        ms[k] = 0.0;
        if (!c->stage_ran[k]) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, c->ev[k], c->ev[k + 1]) == cudaSuccess) ms[k] = t;
        else cudaGetLastError();
    }
    return SPH_OK;
}

int sph_step_kernel_count(sph_ctx *c, int *kernels)
{
    if (!c || !kernels) return fail(SPH_EINVAL, "NULL argument");
    if (!c->graph) {
        if (c->stream == nullptr) return fail(SPH_EINVAL, "needs a non-default stream");
        int rc = sph_run(c, 1);
        if (rc) return rc;
        if (!c->graph) {
            rc = build_graph(c);
            if (rc) return rc;
        }
    }
    *kernels = c->graph_kernels;
    return SPH_OK;
}

int sph_diagnostics(sph_ctx *c, sph_diag *out)
{
    if (!c || !out) return fail(SPH_EINVAL, "NULL argument");
    CU(cudaStreamSynchronize(c->stream));
    ProbDiag d;
    CU(cudaMemcpy(&d, c->diag, sizeof d, cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof *out);
    out->mass = d.mass;
    for (int a = 0; a < 3; ++a) {
        out->momentum[a] = d.mom[a];
        out->force_sum[a] = d.fsum[a];
    }
    out->energy = d.energy;
    out->dEdt = d.dEdt;
    out->dt_next = d.dt_next;
    out->time = d.time;
    out->steps = d.steps;
    out->nr_iterations = d.nr_iter;
    out->nr_max = d.nr_max;
    out->ngb_min = d.ngb_min == 0x7fffffff ? 0 : d.ngb_min;
    out->ngb_max = d.ngb_max;
    out->ngb_mean = c->n > 0 ? (double)d.ngb_sum / (double)c->n : 0.0;
    out->density_pairs = d.density_pairs;
    out->force_pairs = d.force_pairs;
    out->candidates = d.candidates;
    out->fallback = d.fallback;
    out->leaves = d.leaves;
    out->status = status_to_code(d.status);
    out->unconverged = d.unconverged;
    out->walk_reused = d.walk_reused;
    out->wrap_leaves = d.wrap_leaves;
    out->grav_pairs = d.grav_pairs;
    out->grav_nodes = d.grav_nodes;
    return SPH_OK;
}

int sph_neighbours(sph_ctx *c, int kind, const double *h_in, int64_t *offsets, int32_t *idx, int64_t cap,
                   int64_t *total)
{
    if (!c || !offsets || (!idx && cap > 0) || !total) return fail(SPH_EINVAL, "NULL argument");
    if (kind != 0 && kind != 1) return fail(SPH_EINVAL, "kind must be 0 or 1");
    if (cap < 0) return fail(SPH_EINVAL, "cap must be >= 0");
    const BatchView &b = c->bv;
    cudaStream_t st = c->stream;
    CU(launch_reset_step(b, 1, st));
    CU(launch_domain_and_keys(b, st));
    CU(launch_radix_sort(b, st));
    CU(launch_gather(b, st));
    CU(launch_build_leaves(b, c->prm.precision, st));
    CU(launch_set_sorted_h(b, h_in, st));
    CU(launch_refit(b, c->prm.precision, st));
    CU(launch_neighbour_export(b, kind, h_in, (long long *)offsets, (int *)idx, (long long)cap, b.scratch64, st));
    CU(cudaStreamSynchronize(st));
    long long tot = 0;
    CU(cudaMemcpy(&tot, b.scratch64, sizeof tot, cudaMemcpyDeviceToHost));
    *total = tot;
    unsigned s = 0;
    CU(cudaMemcpy(&s, &c->diag->status, sizeof s, cudaMemcpyDeviceToHost));
    if (s & ST_OVERFLOW) return fail(SPH_ENOSPACE, "a particle has more than 1024 neighbours");
    if (tot > cap) return fail(SPH_ENOSPACE, "%lld neighbour entries, capacity %lld", tot, (long long)cap);
    return SPH_OK;
}

int sph_destroy(sph_ctx *c)
{
    if (!c) return SPH_OK;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->graph_reuse) cudaGraphExecDestroy(c->graph_reuse);
    if (c->block_graph) cudaGraphExecDestroy(c->block_graph);
    for (int k = 0; k <= SPH_NSTAGES; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    delete c;
    return SPH_OK;
}

// ---- batching ---------------------------------------------------------------
static int batch_check(sph_ctx *const *ctxs, int nctx)
{
    if (!ctxs || nctx <= 0) return fail(SPH_EINVAL, "empty batch");
    for (int k = 0; k < nctx; ++k) {
        if (!ctxs[k]) return fail(SPH_EINVAL, "batch context %d is NULL", k);
        if (ctxs[k]->prm.precision != ctxs[0]->prm.precision)
            return fail(SPH_EINVAL, "all batch contexts must share the precision");
        if (ctxs[k]->stream != ctxs[0]->stream) return fail(SPH_EINVAL, "all batch contexts must share the stream");
    }
    return SPH_OK;
}

size_t sph_batch_workspace_bytes(sph_ctx *const *ctxs, int nctx)
{
    if (batch_check(ctxs, nctx) != SPH_OK) return 0;
    long long ntot = 0;
    int gch = 0, gtree = 0;
    for (int k = 0; k < nctx; ++k) {
        const sph_params &q = ctxs[k]->prm;
        ntot += ctxs[k]->n;
        if (q.gravity && gravity_chunks(ctxs[k]->n, q.grav_theta) > gch) gch = gravity_chunks(ctxs[k]->n, q.grav_theta);
        if (q.gravity && q.grav_theta > 0) gtree = 1;
    }
    Carver c{nullptr};
    BatchView b;
    memset(&b, 0, sizeof b);
    carve_tables(c, b, nctx);
    carve_arrays(c, b, ntot, nctx, ctxs[0]->prm.precision, gch, gtree);
    return c.off + 256;
}

// The batch-global view of nctx contexts laid out in workspace: problem
// tables (uploaded on st), scratch arrays, launch classes.
static int batch_view(sph_ctx *const *ctxs, int nctx, void *workspace, size_t ws_bytes, BatchView &b)
{
    int rc = batch_check(ctxs, nctx);
    if (rc) return rc;
    for (int k = 0; k < nctx; ++k)
        if (!ctxs[k]->have_forces)
            return fail(SPH_EINVAL, "batch context %d has no force evaluation yet", k);
    size_t need = sph_batch_workspace_bytes(ctxs, nctx);
    if (!workspace || ws_bytes < need) return fail(SPH_ENOSPACE, "batch workspace of %zu bytes needed", need);
    if (((uintptr_t)workspace) & 255) return fail(SPH_EINVAL, "workspace must be 256-byte aligned");
    const int prec = ctxs[0]->prm.precision;
    cudaStream_t st = ctxs[0]->stream;
    long long ntot = 0;
    std::vector<ProbStatic> tab(nctx);
    std::vector<long long> bases(nctx + 1);
    int mask = 0, dmask = 0, b_any_isolated = 0, b_any_periodic = 0, b_any_general = 0, b_any_gravity = 0;
    int b_any_cd = 0;
    long long grav_blocks = 0;
    int gch = 0, gtree = 0;
    for (int k = 0; k < nctx; ++k) {
        tab[k] = ctxs[k]->host_ps;
        tab[k].base = ntot;
        bases[k] = ntot;
        ntot += ctxs[k]->n;
        mask |= mask_of(tab[k].lpp, tab[k].ph.kernel);
        dmask |= dens_class_bit(tab[k].lpp, tab[k].uniform_m, tab[k].ph.kernel);
        if (!tab[k].ph.periodic) b_any_isolated = 1;
        else b_any_periodic = 1;
        if (tab[k].ph.av_switch || tab[k].ph.ac_signal || tab[k].ph.gravity) b_any_general = 1;
        if (tab[k].ph.gravity) b_any_gravity = 1;
        if (tab[k].ph.av_switch == SPH_AV_CULLEN_DEHNEN) b_any_cd = 1;
        tab[k].gblk0 = (int)grav_blocks;
        tab[k].gchunks = tab[k].ph.gravity ? gravity_chunks(ctxs[k]->n, tab[k].ph.grav_theta) : 0;
        if (tab[k].ph.gravity) grav_blocks += gravity_blocks(ctxs[k]->n, tab[k].ph.grav_theta);
        if (tab[k].ph.gravity && tab[k].ph.grav_theta > 0) gtree = 1;
        if (tab[k].gchunks > gch) gch = tab[k].gchunks;
    }
    bases[nctx] = ntot;
    Carver cv{(char *)workspace};
    memset(&b, 0, sizeof b);
    carve_tables(cv, b, nctx);
    carve_arrays(cv, b, ntot, nctx, prec, gch, gtree);
    b.ntot = ntot;
    b.key_bits = key_bits_for(nctx);
    b.key_lo = key_low_bits(ntot);
    b.lpp_mask = mask;
    b.dens_mask = dmask;
    b.any_isolated = b_any_isolated;
    b.any_periodic = b_any_periodic;
    b.any_general = b_any_general;
    b.any_gravity = b_any_gravity;
    b.any_cd = b_any_cd;
    b.grav_blocks = grav_blocks;
    b.grav_split = gch > 1;
    b.any_grav_tree = gtree;
    CU(cudaMemcpyAsync(b.prob, tab.data(), sizeof(ProbStatic) * nctx, cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(b.prob_base, bases.data(), sizeof(long long) * (nctx + 1), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(b.dyn, 0, sizeof(ProbDyn) * nctx, st));
    CU(cudaMemsetAsync(b.counters, 0, kNumCounters * sizeof(int), st));
    CU(cudaMemsetAsync(b.zero_lo, 0, b.zero_bytes, st));
    // each problem's div v from its last force pass (the next step's h
    // prediction) moves into the batch's layout
    for (int k = 0; k < nctx; ++k)
        if (ctxs[k]->n > 0)
            CU(cudaMemcpyAsync(b.divv + bases[k], ctxs[k]->bv.divv, sizeof(float) * ctxs[k]->n,
                               cudaMemcpyDeviceToDevice, st));
    // (copies from pageable host memory are staged before cudaMemcpyAsync
    // returns, so the local tables may go out of scope)
    return SPH_OK;
}

// the contexts' own step bookkeeping after batched steps: their particles
// were sorted in the batch's layout, so a later step of one context alone
// must rebuild its leaves first; div v (the h prediction) goes back to each
// context
static void after_batch_steps(sph_ctx *const *ctxs, int nctx, const BatchView &b, cudaStream_t st)
{
    long long base = 0;
    for (int k = 0; k < nctx; ++k) {
        ctxs[k]->since_build = ctxs[k]->prm.tree_rebuild_every;
        if (ctxs[k]->n > 0)
            cudaMemcpyAsync(ctxs[k]->bv.divv, b.divv + base, sizeof(float) * ctxs[k]->n, cudaMemcpyDeviceToDevice, st);
        base += ctxs[k]->n;
    }
}

// each context's device status, and the first error among them
static int batch_statuses(sph_ctx *const *ctxs, int nctx, int *status)
{
    int worst = SPH_OK;
    for (int k = 0; k < nctx; ++k) {
        unsigned s = 0;
        CU(cudaMemcpy(&s, &ctxs[k]->diag->status, sizeof s, cudaMemcpyDeviceToHost));
        const int code = status_to_code(s);
        if (status) status[k] = code;
        if (code != SPH_OK && worst == SPH_OK) worst = code;
    }
    return worst;
}

int sph_batch_step(sph_ctx *const *ctxs, int nctx, int nsteps, void *workspace, size_t ws_bytes)
{
    if (nsteps < 0) return fail(SPH_EINVAL, "nsteps must be >= 0");
    BatchView b;
    int rc = batch_view(ctxs, nctx, workspace, ws_bytes, b);
    if (rc) return rc;
    const int prec = ctxs[0]->prm.precision;
    cudaStream_t st = ctxs[0]->stream;
    for (int s = 0; s < nsteps; ++s) {
        rc = enqueue_step(b, prec, -1.0, st, Marks());
        if (rc) return rc;
    }
    if (nsteps > 0) after_batch_steps(ctxs, nctx, b, st);
    CU(cudaStreamSynchronize(st));
    return batch_statuses(ctxs, nctx, nullptr);
}

}  // extern "C"

// ---- resident batch: tables uploaded once, the step captured as a graph ----
struct sph_batch {
    std::vector<sph_ctx *> ctxs;
    BatchView b;
    int prec = SPH_PREC_MIXED;
    cudaStream_t st = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_kernels = 0;
    int eager = 0;  // steps enqueued before the capture
    bool timing = false;
    cudaEvent_t ev[SPH_NSTAGES + 1] = {};
    bool stage_ran[SPH_NSTAGES] = {};
};

static Marks marks_of(sph_batch *bt)
{
    Marks m;
    if (bt->timing) {
        m.ev = bt->ev;
        m.ran = bt->stage_ran;
    }
    return m;
}

static int batch_build_graph(sph_batch *bt)
{
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(bt->st, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(bt->b, bt->prec, -1.0, bt->st, marks_of(bt));
    cudaError_t e = cudaStreamEndCapture(bt->st, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return fail(SPH_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(e));
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    int kern = 0;
    for (size_t k = 0; k < nn; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[k], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
    }
    e = cudaGraphInstantiate(&bt->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        bt->graph = nullptr;
        return fail(SPH_ECUDA, "batch graph instantiation failed: %s", cudaGetErrorString(e));
    }
    bt->graph_kernels = kern;
    return SPH_OK;
}

extern "C" {

int sph_batch_create(sph_batch **out, sph_ctx *const *ctxs, int nctx, void *workspace, size_t ws_bytes,
                     unsigned flags)
{
    if (!out) return fail(SPH_EINVAL, "out is NULL");
    *out = nullptr;
    BatchView b;
    int rc = batch_view(ctxs, nctx, workspace, ws_bytes, b);
    if (rc) return rc;
    if (ctxs[0]->stream == nullptr)
        return fail(SPH_EINVAL, "a resident batch needs a non-default stream (its step is captured as a graph)");
    sph_batch *bt = new sph_batch();
    bt->ctxs.assign(ctxs, ctxs + nctx);
    bt->b = b;
    bt->prec = ctxs[0]->prm.precision;
    bt->st = ctxs[0]->stream;
    bt->timing = (flags & SPH_FLAG_TIMING) != 0;
    if (bt->timing)
        for (int k = 0; k <= SPH_NSTAGES; ++k)
            if (cudaEventCreate(&bt->ev[k]) != cudaSuccess) {
                for (int j = 0; j < k; ++j) cudaEventDestroy(bt->ev[j]);
                delete bt;
                return fail(SPH_ECUDA, "cudaEventCreate failed");
            }
    *out = bt;
    return SPH_OK;
}

int sph_batch_run(sph_batch *bt, int nsteps)
{
    if (!bt) return fail(SPH_EINVAL, "batch is NULL");
    if (nsteps < 0) return fail(SPH_EINVAL, "nsteps must be >= 0");
    for (int s = 0; s < nsteps; ++s) {
        if (!bt->graph && bt->eager == 0) {
            // the first step runs eagerly (it sets the kernels' lazily set
            // attributes); a batch that takes one step only is never captured
            int rc = enqueue_step(bt->b, bt->prec, -1.0, bt->st, marks_of(bt));
            if (rc) return rc;
            ++bt->eager;
            continue;
        }
        if (!bt->graph) {
            int rc = batch_build_graph(bt);
            if (rc) return rc;
        }
        CU(cudaGraphLaunch(bt->graph, bt->st));
    }
    if (nsteps > 0) after_batch_steps(bt->ctxs.data(), (int)bt->ctxs.size(), bt->b, bt->st);
    return SPH_OK;
}

int sph_batch_sync(sph_batch *bt, int *status)
{
    if (!bt) return fail(SPH_EINVAL, "batch is NULL");
    CU(cudaStreamSynchronize(bt->st));
    return batch_statuses(bt->ctxs.data(), (int)bt->ctxs.size(), status);
}

int sph_batch_stage_times(sph_batch *bt, double *ms)
{
    if (!bt || !ms) return fail(SPH_EINVAL, "NULL argument");
    if (!bt->timing) return fail(SPH_EINVAL, "batch was created without SPH_FLAG_TIMING");
    CU(cudaStreamSynchronize(bt->st));
    for (int k = 0; k < SPH_NSTAGES; ++k) {
        ms[k] = 0.0;
        if (!bt->stage_ran[k]) continue;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, bt->ev[k], bt->ev[k + 1]) == cudaSuccess) ms[k] = t;
        else cudaGetLastError();
    }
    return SPH_OK;
}

int sph_batch_kernel_count(sph_batch *bt, int *kernels)
{
    if (!bt || !kernels) return fail(SPH_EINVAL, "NULL argument");
    if (!bt->graph) return fail(SPH_EINVAL, "no step captured yet: call sph_batch_run first");
    *kernels = bt->graph_kernels;
    return SPH_OK;
}

int sph_batch_destroy(sph_batch *bt)
{
    if (!bt) return SPH_OK;
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    if (bt->timing)
        for (int k = 0; k <= SPH_NSTAGES; ++k)
            if (bt->ev[k]) cudaEventDestroy(bt->ev[k]);
    delete bt;
    return SPH_OK;
}

}  // extern "C"
