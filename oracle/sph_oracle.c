/*
 * Plain, slow FP64 CPU oracle for the grad-h SPH neighbour loop of GANDALF
 * (Hubber, Rosotti & Booth 2018, arXiv:1709.04488).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) links, imports or calls this file; only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark do.  It shares no code,
 * header or constant with the CUDA implementation.
 *
 * What it computes, in the paper's order and notation:
 *   - M4 cubic-spline kernel, support 2h, or the quintic M6 spline, support
 *     3h (Sec. 2, the two kernel functions).  The paper defers the formulas to
 *     an earlier paper; we use the standard Monaghan & Lattanzio (1985) M4
 *     spline with 3D normalisation 1/pi and the standard M6 quintic spline
 *     with 3D normalisation 1/(120 pi).
 *   - Density sum, Eq. SPHRHO, and the h-rho relation, Eq. HRHO (eta = 1.2 by
 *     default), iterated to convergence by Newton-Raphson with a bisection
 *     fallback (Sec. 2.1.1; Newton-Raphson is named in Sec. 4.1 for the same
 *     solve).
 *   - The grad-h correction Omega, Eq. OMEGA; pressure and sound speed from the
 *     adiabatic or isothermal EOS (Sec. 2.1.1, Sec. 6.2).
 *   - Grad-h momentum equation, Eq. GRADHMOMEQN; energy equation, Eq.
 *     GRADHENEQN; Monaghan (1997) artificial viscosity and Wadsley (2008)
 *     conductivity, Eqs. MON97ARTVISC and MON97ENERGYDISS.
 *   - CFL time-step, Eq. SPH_DT with its signal speed; leapfrog KDK, Eqs.
 *     LFKDK1/LFKDK2, with a predictor for the velocity-dependent forces.
 *
 * Neighbour search is brute force O(N^2) over all particles, with the periodic
 * minimum image.  A uniform-grid prefilter (use_grid=1) returns exactly the
 * same candidate set, sorted by particle id, so every sum is taken in the same
 * order and the two modes give identical bits; it only makes large inputs
 * affordable.  All sums run over j in ascending particle id with Kahan
 * compensation.  Squared distances are formed as dx*dx + dy*dy + dz*dz, left to
 * right; the file must be compiled with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

typedef struct {
    int periodic;            /* 1 = periodic box [lo, lo+L) on every axis */
    double box_lo[3];
    double box_len[3];
    int eos;                 /* 0 = adiabatic, 1 = isothermal */
    double gamma;
    double cs_iso;
    double eta;              /* h = eta (m/rho)^(1/3), Eq. HRHO */
    double alpha_av;
    double beta_av;
    double alpha_ac;
    double c_cfl;
    double h_tol;            /* stop when |dh|/h < h_tol */
    int h_max_iter;
    int use_grid;            /* 0 = brute force, 1 = grid prefilter (same result) */
    int kernel;              /* 0 = M4 cubic spline (support 2h), 1 = M6 quintic (3h) */
    int ac_signal;           /* conductivity signal speed: 0 = Wadsley |v_ij . r_hat|,
                                1 = Price sqrt(|P_i - P_j| / rho_bar) (Sec. 2.1.1) */
    int av_switch;           /* 0: constant alpha_av; 1: Morris & Monaghan (1997) switch,
                                one alpha per particle (Sec. 2.1.1); 2: Cullen & Dehnen
                                (2010) switch (Sec. 2.1.1 names both) */
    double alpha_min;        /* switch: floor the viscosity decays to */
    double av_decay;         /* switch: decay time tau = h / (av_decay c) */
    int gravity;             /* 1: self-gravity, Eq. SPHSELFGRAV (isolated, M4 kernel) */
    double G;                /* gravitational constant */
    double grav_theta;       /* gravity: opening angle theta_MAX of the tree walk (Sec. 4.2);
                                0 = direct summation over every pair */
    int grav_leaf;           /* gravity tree: N_LEAF, most particles in a leaf cell */
    double c_grav;           /* gravity: acceleration condition multiplier, Eq. SPH_DTACCEL */
} orc_params;

typedef struct {
    double *x, *y, *z;
    double *vx, *vy, *vz;
    double *u, *m, *h;
    double *rho, *omega, *P, *c;
    double *ax, *ay, *az, *du, *vsig;
    int32_t *nngb, *iters;
    double *alpha, *dalpha;  /* switch: viscosity parameter per particle and its rate */
    double *zeta;            /* gravity: zeta of Eq. GRADHZETA (written by the density solve) */
    double *cd_divv;         /* Cullen & Dehnen: div v of the last force evaluation (in: the one before) */
    double *cd_xi;           /* Cullen & Dehnen: the limiter xi of the last force evaluation */
} orc_state;

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_EBOX = -2, ORC_ENOCONV = -3, ORC_ENOMEM = -9 };

/* ------------------------------------------------------------------------ */
/* M4 cubic spline (Monaghan & Lattanzio 1985), 3D, support radius 2h.       */
/* f(q) is the dimensionless shape: W(r,h) = f(r/h) / (pi h^3).              */
/* ------------------------------------------------------------------------ */
double orc_f(double q)
{
    if (q < 0.0) q = -q;
    if (q < 1.0) return 1.0 - 1.5 * q * q + 0.75 * q * q * q;
    if (q < 2.0) {
        double t = 2.0 - q;
        return 0.25 * t * t * t;
    }
    return 0.0;
}

/* df/dq */
double orc_df(double q)
{
    if (q < 1.0) return -3.0 * q + 2.25 * q * q;
    if (q < 2.0) {
        double t = 2.0 - q;
        return -0.75 * t * t;
    }
    return 0.0;
}

double orc_W(double r, double h) { return orc_f(r / h) / (ORC_PI * h * h * h); }

/* dW/dr: magnitude of the kernel gradient along r_hat (negative inside 2h). */
double orc_dWdr(double r, double h)
{
    return orc_df(r / h) / (ORC_PI * h * h * h * h);
}

/* dW/dh at fixed r: -(3 f + q f') / (pi h^4). */
double orc_dWdh(double r, double h)
{
    double q = r / h;
    return -(3.0 * orc_f(q) + q * orc_df(q)) / (ORC_PI * h * h * h * h);
}

/* ------------------------------------------------------------------------ */
/* M6 quintic spline, 3D, support radius 3h: W(r,h) = g(r/h) / (120 pi h^3)  */
/* with g(q) = (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5, each term present only      */
/* while its bracket is positive.                                            */
/* ------------------------------------------------------------------------ */
static double pow5(double t) { return t * t * t * t * t; }
static double pow4(double t) { return t * t * t * t; }

double orc_g6(double q)
{
    if (q < 0.0) q = -q;
    if (q >= 3.0) return 0.0;
    double g = pow5(3.0 - q);
    if (q < 2.0) g -= 6.0 * pow5(2.0 - q);
    if (q < 1.0) g += 15.0 * pow5(1.0 - q);
    return g;
}

/* dg/dq */
double orc_dg6(double q)
{
    if (q >= 3.0) return 0.0;
    double d = -5.0 * pow4(3.0 - q);
    if (q < 2.0) d += 30.0 * pow4(2.0 - q);
    if (q < 1.0) d -= 75.0 * pow4(1.0 - q);
    return d;
}

/* Kernel k (0 = M4, 1 = M6): support radius in units of h, normalised shape
   F = sigma f(q) with W = F / h^3, and dF/dq. */
static double kernel_R(int k) { return k == 1 ? 3.0 : 2.0; }
static double kernel_F(int k, double q) { return k == 1 ? orc_g6(q) / (120.0 * ORC_PI) : orc_f(q) / ORC_PI; }
static double kernel_dF(int k, double q) { return k == 1 ? orc_dg6(q) / (120.0 * ORC_PI) : orc_df(q) / ORC_PI; }

double orc_Wk(int k, double r, double h) { return kernel_F(k, r / h) / (h * h * h); }
double orc_dWdrk(int k, double r, double h) { return kernel_dF(k, r / h) / (h * h * h * h); }
double orc_dWdhk(int k, double r, double h)
{
    double q = r / h;
    return -(3.0 * kernel_F(k, q) + q * kernel_dF(k, q)) / (h * h * h * h);
}

/* ------------------------------------------------------------------------ */
/* Softened gravity of the M4 kernel (Eqs. GRAVFORCEKERNEL, GRADHZETA).      */
/* The enclosed mass fraction of a unit-mass kernel, M(q) = 4 int_0^q f s^2 ds,*/
/* gives phi'(r,h) = M(q)/r^2; the potential phi(r,h) = psi(q)/h with        */
/* psi' = M/q^2 and psi = -1/q beyond q = 2; dphi/dh = -(psi + M/q)/h^2.     */
/* (Integrals of the cubic spline, written out piecewise.)                   */
/* ------------------------------------------------------------------------ */
double orc_gmass(double q)
{
    if (q >= 2.0) return 1.0;
    double q3 = q * q * q;
    if (q < 1.0) return 4.0 * (q3 / 3.0 - 0.3 * q3 * q * q + 0.125 * q3 * q3);
    return 4.0 * (2.0 * q3 / 3.0 - 0.75 * q3 * q + 0.3 * q3 * q * q - q3 * q3 / 24.0 - 1.0 / 60.0);
}

double orc_gpsi(double q)
{
    if (q >= 2.0) return -1.0 / q;
    double q2 = q * q;
    if (q < 1.0) return 2.0 * q2 / 3.0 - 0.3 * q2 * q2 + 0.1 * q2 * q2 * q - 1.4;
    return 4.0 * q2 / 3.0 - q2 * q + 0.3 * q2 * q2 - q2 * q2 * q / 30.0 + 1.0 / (15.0 * q) - 1.6;
}

/* phi'(r,h), phi(r,h) and dphi/dh at fixed r (G = 1) */
double orc_gforce(double r, double h) { return orc_gmass(r / h) / (r * r); }
double orc_gpot(double r, double h) { return orc_gpsi(r / h) / h; }
double orc_gdphidh(double r, double h)
{
    double q = r / h;
    double mq = q > 0 ? orc_gmass(q) / q : 0.0; /* M(q)/q -> 0 as q -> 0 */
    return -(orc_gpsi(q) + mq) / (h * h);
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */
static double min_image(double d, double L, int periodic)
{
    if (!periodic) return d;
    if (d > 0.5 * L) d -= L;
    else if (d < -0.5 * L) d += L;
    return d;
}

typedef struct {
    double dx, dy, dz, r2;
} sep_t;

static sep_t separation(const orc_params *p, const orc_state *s, int64_t i, int64_t j)
{
    sep_t o;
    o.dx = min_image(s->x[i] - s->x[j], p->box_len[0], p->periodic);
    o.dy = min_image(s->y[i] - s->y[j], p->box_len[1], p->periodic);
    o.dz = min_image(s->z[i] - s->z[j], p->box_len[2], p->periodic);
    /* left to right, no contraction (compiled with -ffp-contract=off) */
    o.r2 = o.dx * o.dx + o.dy * o.dy + o.dz * o.dz;
    return o;
}

/* Kahan-compensated accumulator */
typedef struct {
    double s, c;
} kahan_t;

static void kadd(kahan_t *k, double v)
{
    double y = v - k->c;
    double t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* ------------------------------------------------------------------------ */
/* Uniform-grid prefilter.  Only narrows the candidate set; the membership    */
/* test below is the same expression as in brute-force mode, and candidate    */
/* lists are sorted by id before use.                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nc[3];
    double lo[3], cs[3];
    int64_t *cell_start; /* ncell + 1 */
    int64_t *ids;        /* particle ids grouped by cell, ascending within a cell */
} grid_t;

static int cell_coord(const grid_t *g, int a, double x)
{
    int c = (int)floor((x - g->lo[a]) / g->cs[a]);
    if (c < 0) c = 0;
    if (c >= g->nc[a]) c = g->nc[a] - 1;
    return c;
}

static int grid_build(grid_t *g, const orc_params *p, const orc_state *s, int64_t n, double cell)
{
    double lo[3], hi[3];
    const double *X[3] = {s->x, s->y, s->z};
    for (int a = 0; a < 3; ++a) {
        if (p->periodic) {
            lo[a] = p->box_lo[a];
            hi[a] = p->box_lo[a] + p->box_len[a];
        } else {
            lo[a] = hi[a] = X[a][0];
            for (int64_t i = 1; i < n; ++i) {
                if (X[a][i] < lo[a]) lo[a] = X[a][i];
                if (X[a][i] > hi[a]) hi[a] = X[a][i];
            }
        }
        double ext = hi[a] - lo[a];
        int nc = (ext > 0 && cell > 0) ? (int)floor(ext / cell) : 1;
        if (nc < 1) nc = 1;
        if (nc > 512) nc = 512;
        g->nc[a] = nc;
        g->lo[a] = lo[a];
        g->cs[a] = ext > 0 ? ext / nc : 1.0;
    }
    int64_t ncell = (int64_t)g->nc[0] * g->nc[1] * g->nc[2];
    g->cell_start = (int64_t *)calloc((size_t)ncell + 1, sizeof(int64_t));
    g->ids = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *cid = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!g->cell_start || !g->ids || !cid) {
        free(cid);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        int cx = cell_coord(g, 0, s->x[i]), cy = cell_coord(g, 1, s->y[i]), cz = cell_coord(g, 2, s->z[i]);
        cid[i] = ((int64_t)cz * g->nc[1] + cy) * g->nc[0] + cx;
        g->cell_start[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell; ++c) g->cell_start[c + 1] += g->cell_start[c];
    int64_t *fill = (int64_t *)malloc((size_t)ncell * sizeof(int64_t));
    if (!fill) {
        free(cid);
        return ORC_ENOMEM;
    }
    memcpy(fill, g->cell_start, (size_t)ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->ids[fill[cid[i]]++] = i; /* ascending id within each cell */
    free(fill);
    free(cid);
    return ORC_OK;
}

static void grid_free(grid_t *g)
{
    free(g->cell_start);
    free(g->ids);
    g->cell_start = NULL;
    g->ids = NULL;
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Growable list of ids */
typedef struct {
    int64_t *v;
    int64_t n, cap;
} idlist_t;

static int push(idlist_t *l, int64_t j)
{
    if (l->n == l->cap) {
        int64_t nc = l->cap ? 2 * l->cap : 256;
        int64_t *nv = (int64_t *)realloc(l->v, (size_t)nc * sizeof(int64_t));
        if (!nv) return ORC_ENOMEM;
        l->v = nv;
        l->cap = nc;
    }
    l->v[l->n++] = j;
    return ORC_OK;
}

/*
 * All j (including i itself) with r_ij^2 < R^2, ascending in j.
 * mode "rmax_of_j": when hj != NULL the radius for pair (i,j) is
 * R_K max(h_i, h_j) (the force list, R_K the kernel's support in units of
 * h); otherwise the fixed radius R.
 */
static int gather(const orc_params *p, const orc_state *s, int64_t n, const grid_t *g,
                  int64_t i, double R, const double *hforce, idlist_t *out)
{
    out->n = 0;
    if (!g) {
        for (int64_t j = 0; j < n; ++j) {
            sep_t d = separation(p, s, i, j);
            double Rj = R;
            if (hforce) {
                double hm = hforce[i] > hforce[j] ? hforce[i] : hforce[j];
                Rj = kernel_R(p->kernel) * hm;
            }
            if (d.r2 < Rj * Rj)
                if (push(out, j)) return ORC_ENOMEM;
        }
        return ORC_OK;
    }
    /* grid: the query radius must cover the largest pair radius; for force
       lists the caller passes R = R_K max_j h_j */
    const double Rq = R;
    const double X[3] = {s->x[i], s->y[i], s->z[i]};
    int c0[3], c1[3], full[3];
    for (int a = 0; a < 3; ++a) {
        int span = (int)ceil(Rq / g->cs[a]) + 1;
        int cc = cell_coord(g, a, X[a]);
        c0[a] = cc - span;
        c1[a] = cc + span;
        full[a] = 0;
        if (p->periodic) {
            if (c1[a] - c0[a] + 1 >= g->nc[a]) {
                c0[a] = 0;
                c1[a] = g->nc[a] - 1;
                full[a] = 1;
            }
        } else {
            if (c0[a] < 0) c0[a] = 0;
            if (c1[a] >= g->nc[a]) c1[a] = g->nc[a] - 1;
        }
    }
    for (int cz = c0[2]; cz <= c1[2]; ++cz)
        for (int cy = c0[1]; cy <= c1[1]; ++cy)
            for (int cx = c0[0]; cx <= c1[0]; ++cx) {
                int w[3] = {cx, cy, cz};
                for (int a = 0; a < 3; ++a)
                    if (p->periodic && !full[a]) w[a] = ((w[a] % g->nc[a]) + g->nc[a]) % g->nc[a];
                int64_t cid = ((int64_t)w[2] * g->nc[1] + w[1]) * g->nc[0] + w[0];
                for (int64_t k = g->cell_start[cid]; k < g->cell_start[cid + 1]; ++k) {
                    int64_t j = g->ids[k];
                    sep_t d = separation(p, s, i, j);
                    double Rj = R;
                    if (hforce) {
                        double hm = hforce[i] > hforce[j] ? hforce[i] : hforce[j];
                        Rj = kernel_R(p->kernel) * hm;
                    }
                    if (d.r2 < Rj * Rj)
                        if (push(out, j)) return ORC_ENOMEM;
                }
            }
    qsort(out->v, (size_t)out->n, sizeof(int64_t), cmp_i64);
    return ORC_OK;
}

static int params_ok(const orc_params *p, int64_t n)
{
    if (n < 0 || !p) return 0;
    if (!(p->eta > 0) || !(p->h_tol > 0) || p->h_max_iter < 1) return 0;
    if (p->periodic)
        for (int a = 0; a < 3; ++a)
            if (!(p->box_len[a] > 0)) return 0;
    if (p->eos == 0 && !(p->gamma > 1.0)) return 0;
    if (p->eos == 1 && !(p->cs_iso > 0)) return 0;
    if (p->kernel != 0 && p->kernel != 1) return 0;
    if (p->ac_signal != 0 && p->ac_signal != 1) return 0;
    if (p->av_switch < 0 || p->av_switch > 2) return 0;
    if (p->av_switch && !(p->alpha_av > 0 && p->alpha_min >= 0 && p->alpha_min <= p->alpha_av && p->av_decay > 0))
        return 0;
    if (p->gravity != 0 && p->gravity != 1) return 0;
    if (p->gravity && (p->periodic || p->kernel != 0 || !(p->G > 0))) return 0;
    if (p->gravity && !(p->grav_theta >= 0.0 && p->grav_theta <= 1.0)) return 0;
    if (p->gravity && p->grav_theta > 0 && p->grav_leaf < 1) return 0;
    if (p->gravity && !(p->c_grav > 0)) return 0;
    return 1;
}

static double median_spacing_guess(const orc_params *p, const orc_state *s, int64_t n)
{
    /* cell size for the grid prefilter: a few mean spacings */
    double vol;
    if (p->periodic) vol = p->box_len[0] * p->box_len[1] * p->box_len[2];
    else {
        double lo[3] = {s->x[0], s->y[0], s->z[0]}, hi[3] = {s->x[0], s->y[0], s->z[0]};
        for (int64_t i = 1; i < n; ++i) {
            double X[3] = {s->x[i], s->y[i], s->z[i]};
            for (int a = 0; a < 3; ++a) {
                if (X[a] < lo[a]) lo[a] = X[a];
                if (X[a] > hi[a]) hi[a] = X[a];
            }
        }
        vol = (hi[0] - lo[0] + 1e-300) * (hi[1] - lo[1] + 1e-300) * (hi[2] - lo[2] + 1e-300);
    }
    return cbrt(vol / (double)(n > 0 ? n : 1));
}

/* ------------------------------------------------------------------------ */
/* Density at a fixed h: rho = sum_j m_j W(r_ij, h) (Eq. SPHRHO, j includes  */
/* i) and drho/dh = sum_j m_j dW/dh (r_ij, h).                               */
/* ------------------------------------------------------------------------ */
static int density_at(const orc_params *p, const orc_state *s, int64_t n, const grid_t *g,
                      int64_t i, double h, idlist_t *buf, double *rho, double *drho, int32_t *nn)
{
    int rc = gather(p, s, n, g, i, kernel_R(p->kernel) * h, NULL, buf);
    if (rc) return rc;
    kahan_t r = {0, 0}, d = {0, 0};
    for (int64_t k = 0; k < buf->n; ++k) {
        int64_t j = buf->v[k];
        sep_t sp = separation(p, s, i, j);
        double rr = sqrt(sp.r2);
        kadd(&r, s->m[j] * orc_Wk(p->kernel, rr, h));
        kadd(&d, s->m[j] * orc_dWdhk(p->kernel, rr, h));
    }
    *rho = r.s;
    *drho = d.s;
    if (nn) *nn = (int32_t)buf->n;
    return ORC_OK;
}

/* Exported for the pins: rho(h) and drho/dh(h) of particle i at a given h. */
int orc_density_at_h(const orc_params *p, int64_t n, const orc_state *s, int64_t i, double h,
                     double *rho, double *drho)
{
    if (!params_ok(p, n) || i < 0 || i >= n || !(h > 0)) return ORC_EINVAL;
    idlist_t buf = {0, 0, 0};
    int rc = density_at(p, s, n, NULL, i, h, &buf, rho, drho, NULL);
    free(buf.v);
    return rc;
}

static double initial_h(const orc_params *p, const orc_state *s, int64_t n, int64_t i)
{
    if (p->periodic) {
        double M = 0;
        for (int64_t j = 0; j < n; ++j) M += s->m[j];
        double rhobar = M / (p->box_len[0] * p->box_len[1] * p->box_len[2]);
        return p->eta * cbrt(s->m[i] / rhobar);
    }
    /* isolated: half the distance to the 58th nearest particle (brute force) */
    int64_t k = n < 58 ? n : 58;
    double *d2 = (double *)malloc((size_t)n * sizeof(double));
    if (!d2) return 1.0;
    for (int64_t j = 0; j < n; ++j) d2[j] = separation(p, s, i, j).r2;
    /* partial selection of the k-th smallest */
    for (int64_t a = 0; a < k; ++a) {
        int64_t best = a;
        for (int64_t b = a + 1; b < n; ++b)
            if (d2[b] < d2[best]) best = b;
        double t = d2[a];
        d2[a] = d2[best];
        d2[best] = t;
    }
    double r = sqrt(d2[k - 1]);
    free(d2);
    return r > 0 ? 0.5 * r : 1.0;
}

/*
 * h-rho solve for one particle (Eqs. SPHRHO, HRHO).
 * F(h) = rho_sum(h) - m (eta/h)^3,  F'(h) = drho/dh + 3 m eta^3 / h^4.
 * The sign of F equals that of G(h) = h^3 rho_sum(h) - m eta^3, which is
 * non-decreasing in h, so [lo, hi] brackets the unique root.  A Newton step
 * that leaves the bracket, leaves [h/2, 2h] or meets F' <= 0 is replaced by
 * bisection (or doubling while no upper bound is known).
 * On return h holds the last iterate and rho, drho are evaluated at it.
 */
static int solve_h(const orc_params *p, const orc_state *s, int64_t n, const grid_t *g, int64_t i,
                   idlist_t *buf, double *h_io, double *rho_o, double *drho_o, int32_t *nn_o,
                   int32_t *it_o)
{
    double h = *h_io;
    if (!(h > 0)) h = initial_h(p, s, n, i);
    double lo = 0.0, hi = INFINITY;
    const double m = s->m[i], eta3 = p->eta * p->eta * p->eta;
    double rho = 0, drho = 0;
    int32_t nn = 0;
    int conv = 0, it;
    for (it = 1; it <= p->h_max_iter; ++it) {
        int rc = density_at(p, s, n, g, i, h, buf, &rho, &drho, &nn);
        if (rc) return rc;
        double h3 = h * h * h;
        double F = rho - m * eta3 / h3;
        double dF = drho + 3.0 * m * eta3 / (h3 * h);
        if (F < 0) lo = h;
        else hi = h;
        double hn = (dF > 0) ? h - F / dF : NAN;
        int bad = !(hn >= lo) || !(hn <= hi) || !(hn >= 0.5 * h) || !(hn <= 2.0 * h);
        if (bad) hn = isinf(hi) ? 2.0 * h : 0.5 * (lo + hi);
        if (p->periodic) {
            /* the support 2h must stay below half the box for the minimum image */
            double Lmin = p->box_len[0];
            if (p->box_len[1] < Lmin) Lmin = p->box_len[1];
            if (p->box_len[2] < Lmin) Lmin = p->box_len[2];
            if (hn > Lmin / (2.0 * kernel_R(p->kernel))) { /* the support exceeds half the box */
                *h_io = h;
                *it_o = it;
                return ORC_EBOX;
            }
        }
        if (fabs(hn - h) < p->h_tol * h) {
            h = hn;
            conv = 1;
            break;
        }
        h = hn;
    }
    int rc = density_at(p, s, n, g, i, h, buf, &rho, &drho, &nn);
    if (rc) return rc;
    *h_io = h;
    *rho_o = rho;
    *drho_o = drho;
    *nn_o = nn;
    *it_o = it > p->h_max_iter ? p->h_max_iter : it;
    return conv ? ORC_OK : ORC_ENOCONV;
}

static void eos(const orc_params *p, double rho, double u, double *P, double *c)
{
    if (p->eos == 1) {
        *P = p->cs_iso * p->cs_iso * rho;
        *c = p->cs_iso;
    } else {
        *P = (p->gamma - 1.0) * rho * u;
        *c = sqrt(p->gamma * (*P) / rho);
    }
}

/*
 * Density, smoothing length, Omega (Eq. OMEGA), P and c for every particle.
 * h is read as the starting guess (<= 0: a default guess) and overwritten.
 * Returns ORC_ENOCONV if any particle failed to converge.
 */
/* zeta_i of Eq. GRADHZETA: (dh/drho) sum_j m_j dphi/dh (r_ij, h_i) over the
   gather list at the final h (self included), dh/drho = -h/(3 rho). */
static double gravity_zeta(const orc_params *p, const orc_state *s, int64_t i, const idlist_t *buf, double rho)
{
    kahan_t z = {0, 0};
    for (int64_t k = 0; k < buf->n; ++k) {
        int64_t j = buf->v[k];
        sep_t sp = separation(p, s, i, j);
        kadd(&z, s->m[j] * orc_gdphidh(sqrt(sp.r2), s->h[i]));
    }
    return -s->h[i] / (3.0 * rho) * z.s;
}

/* One term of the long-range part of Eq. SPHSELFGRAV: the acceleration of i
   by j, -G m_j (phi'(r_ij,h_i) + phi'(r_ij,h_j))/2 r_hat_ij. */
static void gravity_pair(const orc_params *p, const orc_state *s, int64_t i, int64_t j, kahan_t *ax, kahan_t *ay,
                         kahan_t *az)
{
    sep_t sp = separation(p, s, i, j);
    double r = sqrt(sp.r2);
    double f = -p->G * s->m[j] * 0.5 * (orc_gforce(r, s->h[i]) + orc_gforce(r, s->h[j])) / r;
    kadd(ax, f * sp.dx);
    kadd(ay, f * sp.dy);
    kadd(az, f * sp.dz);
}

/* The long-range part for particle i by direct summation over every particle
   (isolated problems). */
static void gravity_direct(const orc_params *p, const orc_state *s, int64_t n, int64_t i, kahan_t *ax, kahan_t *ay,
                           kahan_t *az)
{
    for (int64_t j = 0; j < n; ++j)
        if (j != i) gravity_pair(p, s, i, j, ax, ay, az);
}

/* ------------------------------------------------------------------------ */
/* Gravity tree (Sec. 4.2): a KD tree built top-down, each cell split at the */
/* median particle position along its most elongated axis until a cell holds */
/* at most N_LEAF particles.  Each cell keeps its mass, centre of mass,      */
/* quadrupole moment about the centre of mass, particle box, largest h and   */
/* size l_c.  The walk from the root uses a cell's multipole (monopole plus  */
/* quadrupole) when the geometric criterion |r_i - r_c|^2 >= l_c^2/theta^2   */
/* holds and no pair with the cell is softened; otherwise the cell is opened, */
/* and a leaf that is opened contributes its particles by the pair term.     */
/* Readings: r_c is the centre of mass (the expansion centre) and l_c the    */
/* largest distance from it to a corner of the cell's particle box; a cell is */
/* also opened while r_i is within 2 max(h_i, h_max of the cell) of its box, */
/* since the expansion is of the unsoftened 1/r.                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t first, count; /* particles idx[first, first + count) */
    int left, right;      /* children, -1 for a leaf */
    double mass, com[3];
    double quad[6];       /* Q_xx, Q_xy, Q_xz, Q_yy, Q_yz, Q_zz: sum m (3 d_a d_b - |d|^2 delta_ab) */
    double lo[3], hi[3], hmax, lc2;
} kdcell_t;

typedef struct {
    kdcell_t *cell;
    int ncell, cap;
    int64_t *idx;
} kdtree_t;

/* mass, centre of mass and quadrupole of the points idx[first, first+count)
   (idx NULL: the points first .. first+count-1) */
static void point_moments(const double *x, const double *y, const double *z, const double *m, const int64_t *idx,
                          int64_t first, int64_t count, double *mass, double com[3], double q[6])
{
    kahan_t M = {0, 0}, cx = {0, 0}, cy = {0, 0}, cz = {0, 0};
    for (int64_t k = first; k < first + count; ++k) {
        int64_t j = idx ? idx[k] : k;
        kadd(&M, m[j]);
        kadd(&cx, m[j] * x[j]);
        kadd(&cy, m[j] * y[j]);
        kadd(&cz, m[j] * z[j]);
    }
    *mass = M.s;
    com[0] = cx.s / M.s;
    com[1] = cy.s / M.s;
    com[2] = cz.s / M.s;
    kahan_t Q[6];
    memset(Q, 0, sizeof Q);
    for (int64_t k = first; k < first + count; ++k) {
        int64_t j = idx ? idx[k] : k;
        double d[3] = {x[j] - com[0], y[j] - com[1], z[j] - com[2]};
        double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        kadd(&Q[0], m[j] * (3.0 * d[0] * d[0] - d2));
        kadd(&Q[1], m[j] * (3.0 * d[0] * d[1]));
        kadd(&Q[2], m[j] * (3.0 * d[0] * d[2]));
        kadd(&Q[3], m[j] * (3.0 * d[1] * d[1] - d2));
        kadd(&Q[4], m[j] * (3.0 * d[1] * d[2]));
        kadd(&Q[5], m[j] * (3.0 * d[2] * d[2] - d2));
    }
    for (int a = 0; a < 6; ++a) q[a] = Q[a].s;
}

/* Acceleration at r (relative to the centre of mass) of mass M with
   quadrupole Q: the potential -G (M/|r| + r.Q.r / (2|r|^5)) gives
   -G M r/|r|^3 + G (Q r/|r|^5 - (5/2)(r.Q.r) r/|r|^7); quad = 0 keeps the
   monopole only. */
static void multipole_accel(double G, double M, const double q[6], const double r[3], int quad, double out[3])
{
    double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
    double rinv = 1.0 / sqrt(r2);
    double rinv3 = rinv * rinv * rinv;
    for (int a = 0; a < 3; ++a) out[a] = -G * M * r[a] * rinv3;
    if (!quad) return;
    double Qr[3] = {q[0] * r[0] + q[1] * r[1] + q[2] * r[2], q[1] * r[0] + q[3] * r[1] + q[4] * r[2],
                    q[2] * r[0] + q[4] * r[1] + q[5] * r[2]};
    double rQr = r[0] * Qr[0] + r[1] * Qr[1] + r[2] * Qr[2];
    double rinv5 = rinv3 * rinv * rinv, rinv7 = rinv5 * rinv * rinv;
    for (int a = 0; a < 3; ++a) out[a] += G * (Qr[a] * rinv5 - 2.5 * rQr * r[a] * rinv7);
}

/* the acceleration that points (x, y, z, m)[0..n) exert at (px, py, pz) by
   their multipole expansion about their centre of mass (G = 1) */
void orc_multipole_accel(int64_t n, const double *x, const double *y, const double *z, const double *m, double px,
                         double py, double pz, int quad, double *out)
{
    double M, com[3], q[6];
    point_moments(x, y, z, m, NULL, 0, n, &M, com, q);
    double r[3] = {px - com[0], py - com[1], pz - com[2]};
    multipole_accel(1.0, M, q, r, quad, out);
}

static const double *kd_sort_coord; /* the tree is built by one thread */
static int kd_cmp(const void *a, const void *b)
{
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    double u = kd_sort_coord[i], v = kd_sort_coord[j];
    if (u < v) return -1;
    if (u > v) return 1;
    return (i > j) - (i < j); /* equal coordinates: by particle id */
}

static int kd_build(kdtree_t *t, const orc_state *s, int64_t first, int64_t count, int nleaf)
{
    if (t->ncell == t->cap) {
        int cap = t->cap ? 2 * t->cap : 64;
        kdcell_t *c = (kdcell_t *)realloc(t->cell, sizeof(kdcell_t) * cap);
        if (!c) return -1;
        t->cell = c;
        t->cap = cap;
    }
    int id = t->ncell++;
    kdcell_t *c = &t->cell[id];
    c->first = first;
    c->count = count;
    c->left = c->right = -1;
    const double *X[3] = {s->x, s->y, s->z};
    c->hmax = 0.0;
    for (int a = 0; a < 3; ++a) c->lo[a] = c->hi[a] = X[a][t->idx[first]];
    for (int64_t k = first; k < first + count; ++k) {
        int64_t j = t->idx[k];
        for (int a = 0; a < 3; ++a) {
            if (X[a][j] < c->lo[a]) c->lo[a] = X[a][j];
            if (X[a][j] > c->hi[a]) c->hi[a] = X[a][j];
        }
        if (s->h[j] > c->hmax) c->hmax = s->h[j];
    }
    point_moments(s->x, s->y, s->z, s->m, t->idx, first, count, &c->mass, c->com, c->quad);
    c->lc2 = 0.0;
    for (int k = 0; k < 8; ++k) {
        double d2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = ((k >> a) & 1 ? c->hi[a] : c->lo[a]) - c->com[a];
            d2 += d * d;
        }
        if (d2 > c->lc2) c->lc2 = d2;
    }
    if (count <= nleaf) return 0;
    int ax = 0; /* most elongated axis */
    for (int a = 1; a < 3; ++a)
        if (c->hi[a] - c->lo[a] > c->hi[ax] - c->lo[ax]) ax = a;
    kd_sort_coord = X[ax];
    qsort(t->idx + first, (size_t)count, sizeof(int64_t), kd_cmp);
    int64_t nl = count / 2; /* the median splits the cell */
    int l = t->ncell;
    if (kd_build(t, s, first, nl, nleaf)) return -1;
    int r = t->ncell;
    if (kd_build(t, s, first + nl, count - nl, nleaf)) return -1;
    t->cell[id].left = l; /* (t->cell may have moved) */
    t->cell[id].right = r;
    return 0;
}

static void kd_free(kdtree_t *t)
{
    free(t->cell);
    free(t->idx);
    memset(t, 0, sizeof *t);
}

static int gravity_tree_build(const orc_params *p, const orc_state *s, int64_t n, kdtree_t *t)
{
    memset(t, 0, sizeof *t);
    if (!(p->gravity && p->grav_theta > 0) || n == 0) return 0;
    t->idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    if (!t->idx) return -1;
    for (int64_t i = 0; i < n; ++i) t->idx[i] = i;
    if (kd_build(t, s, 0, n, p->grav_leaf)) {
        kd_free(t);
        return -1;
    }
    return 0;
}

static void gravity_tree_walk(const orc_params *p, const orc_state *s, const kdtree_t *t, int c, int64_t i,
                              kahan_t *ax, kahan_t *ay, kahan_t *az)
{
    const kdcell_t *C = &t->cell[c];
    const double ri[3] = {s->x[i], s->y[i], s->z[i]};
    double r[3], d2 = 0.0, g2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        r[a] = ri[a] - C->com[a];
        d2 += r[a] * r[a];
        double g = ri[a] < C->lo[a] ? C->lo[a] - ri[a] : (ri[a] > C->hi[a] ? ri[a] - C->hi[a] : 0.0);
        g2 += g * g;
    }
    const double soft = 2.0 * (s->h[i] > C->hmax ? s->h[i] : C->hmax);
    if (d2 >= C->lc2 / (p->grav_theta * p->grav_theta) && g2 >= soft * soft) {
        double acc[3];
        multipole_accel(p->G, C->mass, C->quad, r, 1, acc);
        kadd(ax, acc[0]);
        kadd(ay, acc[1]);
        kadd(az, acc[2]);
        return;
    }
    if (C->left < 0) {
        for (int64_t k = C->first; k < C->first + C->count; ++k)
            if (t->idx[k] != i) gravity_pair(p, s, i, t->idx[k], ax, ay, az);
        return;
    }
    gravity_tree_walk(p, s, t, C->left, i, ax, ay, az);
    gravity_tree_walk(p, s, t, C->right, i, ax, ay, az);
}

/* long-range gravity of particle i: the tree walk when theta_MAX > 0, else
   the direct sum */
static void gravity_long_range(const orc_params *p, const orc_state *s, int64_t n, const kdtree_t *t, int64_t i,
                               kahan_t *ax, kahan_t *ay, kahan_t *az)
{
    if (p->grav_theta > 0) gravity_tree_walk(p, s, t, 0, i, ax, ay, az);
    else gravity_direct(p, s, n, i, ax, ay, az);
}

/* The long-range accelerations alone (no zeta term, no hydrodynamics) for
   every particle, with the current h. */
int orc_gravity_accel(const orc_params *p, int64_t n, const orc_state *s, double *gx, double *gy, double *gz)
{
    if (!params_ok(p, n) || !p->gravity) return ORC_EINVAL;
    kdtree_t t;
    if (gravity_tree_build(p, s, n, &t)) return ORC_ENOMEM;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
        kahan_t ax = {0, 0}, ay = {0, 0}, az = {0, 0};
        gravity_long_range(p, s, n, &t, i, &ax, &ay, &az);
        gx[i] = ax.s;
        gy[i] = ay.s;
        gz[i] = az.s;
    }
    kd_free(&t);
    return ORC_OK;
}

/* Gravitational potential energy (G/2) sum_i sum_j m_i m_j (phi(r_ij,h_i) +
   phi(r_ij,h_j))/2, self terms included, with the current h. */
double orc_gravity_energy(const orc_params *p, int64_t n, const orc_state *s)
{
    kahan_t e = {0, 0};
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) {
            double r = i == j ? 0.0 : sqrt(separation(p, s, i, j).r2);
            kadd(&e, s->m[i] * s->m[j] * 0.5 * (orc_gpot(r, s->h[i]) + orc_gpot(r, s->h[j])));
        }
    return 0.5 * p->G * e.s;
}

int orc_density(const orc_params *p, int64_t n, orc_state *s)
{
    if (!params_ok(p, n)) return ORC_EINVAL;
    if (p->gravity && !s->zeta) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    grid_t g;
    memset(&g, 0, sizeof g);
    const grid_t *gp = NULL;
    if (p->use_grid) {
        if (grid_build(&g, p, s, n, 2.0 * median_spacing_guess(p, s, n))) return ORC_ENOMEM;
        gp = &g;
    }
    int status = ORC_OK;
#pragma omp parallel
    {
        idlist_t buf = {0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            double rho = 0, drho = 0;
            int32_t nn = 0, it = 0;
            int rc = solve_h(p, s, n, gp, i, &buf, &s->h[i], &rho, &drho, &nn, &it);
            s->rho[i] = rho;
            /* Omega = 1 - (dh/drho) sum m dW/dh with dh/drho = -h/(3 rho) */
            s->omega[i] = 1.0 + s->h[i] / (3.0 * rho) * drho;
            if (p->gravity) s->zeta[i] = gravity_zeta(p, s, i, &buf, rho);
            eos(p, rho, s->u[i], &s->P[i], &s->c[i]);
            if (s->nngb) s->nngb[i] = nn;
            if (s->iters) s->iters[i] = it;
            if (rc) {
#pragma omp critical
                status = rc;
            }
        }
        free(buf.v);
    }
    if (gp) grid_free(&g);
    return status;
}

/* Viscosity parameters of pair (i,j): alpha_AV and beta_AV = (beta/alpha)
   alpha_AV, the latter the pair mean of the particles' alphas under the
   Morris & Monaghan switch. */
static void av_pair(const orc_params *p, const orc_state *s, int64_t i, int64_t j, double *a, double *b)
{
    if (p->av_switch) {
        *a = 0.5 * (s->alpha[i] + s->alpha[j]);
        *b = p->beta_av / p->alpha_av * (*a);
    } else {
        *a = p->alpha_av;
        *b = p->beta_av;
    }
}

/* Morris & Monaghan (1997) switch: d alpha_i/dt = -(alpha_i - alpha_min)/tau_i
   + max(-div v_i, 0) (alpha_max - alpha_i), tau_i = h_i / (av_decay c_i),
   alpha_max = alpha_av; div v_i = -(1/(Omega_i rho_i)) sum_j m_j v_ij . grad_i W(r_ij, h_i)
   (sumv: the sum). */
static double av_rate(const orc_params *p, const orc_state *s, int64_t i, double sumv)
{
    const double divv = -sumv / (s->omega[i] * s->rho[i]);
    const double src = divv < 0 ? -divv * (p->alpha_av - s->alpha[i]) : 0.0;
    return -(s->alpha[i] - p->alpha_min) * p->av_decay * s->c[i] / s->h[i] + src;
}

/* Cullen & Dehnen (2010) switch, as stated here (Sec. 2.1.1 names it; the
   equations are the published ones, with two readings marked):
   - the velocity gradient V_i = -(1/(Omega_i rho_i)) sum_j m_j v_ij (x) grad_i W(r_ij, h_i),
     D_i = tr V_i = div v_i, S_i = sym(V_i) - D_i/3 I, the traceless shear;
   - R_i = (1/rho_i) sum_j sign(D_j) m_j W(r_ij, h_i), self included, with the
     signs of the previous force evaluation (reading: one pass), sign(0) = +1;
   - xi_i = q^2 / (q^2 + tr(S_i S_i^T)), q = 2 (1 - R_i)^4 D_i (0 when both vanish);
   - the step applies, with dD/dt = (D_new - D_old)/dt (reading: the time
     derivative by finite differences between force evaluations),
     A_i = xi_i max(-dD/dt, 0), alpha_loc = alpha_max h^2 A / (v_sig^2 + h^2 A),
     alpha <- alpha_loc if alpha < alpha_loc, else alpha_loc + (alpha - alpha_loc)
     exp(-dt/tau) with tau = h / (2 av_decay v_sig); alpha_max = alpha_av. */
typedef struct {
    kahan_t g[9]; /* sum_j m_j v_ij,a grad_b W */
    kahan_t r;    /* sum_j sign(D_j) m_j W */
} cd_sums_t;

static void cd_finish(const orc_params *p, const orc_state *s, int64_t i, const cd_sums_t *c, double *D, double *xi)
{
    const double f = -1.0 / (s->omega[i] * s->rho[i]);
    double V[9];
    for (int k = 0; k < 9; ++k) V[k] = f * c->g[k].s;
    const double d = V[0] + V[4] + V[8];
    double ss = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double sab = 0.5 * (V[3 * a + b] + V[3 * b + a]) - (a == b ? d / 3.0 : 0.0);
            ss += sab * sab;
        }
    const double R = c->r.s / s->rho[i];
    const double om = 1.0 - R, q = 2.0 * om * om * om * om * d;
    *D = d;
    *xi = (q * q + ss) > 0 ? q * q / (q * q + ss) : 0.0;
    (void)p;
}

/* the Cullen & Dehnen update of alpha after a step of dt (D_old: div v at the step's start) */
void orc_cd_update(const orc_params *p, int64_t n, orc_state *s, const double *d_old, double dt)
{
    for (int64_t i = 0; i < n; ++i) {
        const double ddot = (s->cd_divv[i] - d_old[i]) / dt;
        const double A = s->cd_xi[i] * (ddot < 0 ? -ddot : 0.0);
        const double h2A = s->h[i] * s->h[i] * A;
        const double vs = s->vsig[i];
        const double aloc = h2A > 0 ? p->alpha_av * h2A / (vs * vs + h2A) : 0.0;
        if (s->alpha[i] < aloc) s->alpha[i] = aloc;
        else s->alpha[i] = aloc + (s->alpha[i] - aloc) * exp(-dt * 2.0 * p->av_decay * vs / s->h[i]);
    }
}

/* Signal speed of the artificial conductivity (Sec. 2.1.1): Wadsley's
   |v_ij . r_hat_ij| by default, or Price's sqrt(|P_i - P_j| / rho_bar_ij). */
static double ac_signal_speed(const orc_params *p, const orc_state *s, int64_t i, int64_t j, double vdr,
                              double rhobar)
{
    if (p->ac_signal == 1) return sqrt(fabs(s->P[i] - s->P[j]) / rhobar);
    return fabs(vdr);
}

/* Block time-steps (Sec. 2.1.4): the level of every particle, the largest
   level among each particle's force neighbours (recorded by the force pass),
   and, during a block step, which particles end their step now. */
typedef struct {
    int32_t *level;
    int32_t *ngb_maxlev;
    const uint8_t *active; /* NULL: every particle */
} orc_block_t;

static int forces_impl(const orc_params *p, int64_t n, orc_state *s, const orc_block_t *blk);

/*
 * Accelerations and energy rates (Eqs. GRADHMOMEQN, GRADHENEQN, MON97ARTVISC,
 * MON97ENERGYDISS) and the signal speed of Eq. SPH_DT, over j != i with
 * r_ij < 2 max(h_i, h_j).  Needs h, rho, Omega, P, c from orc_density.
 */
int orc_forces(const orc_params *p, int64_t n, orc_state *s) { return forces_impl(p, n, s, NULL); }

/* With block time-steps only the active particles (blk->active) get new
   accelerations and rates; each of them also records the largest level
   among its force neighbours. */
static int forces_impl(const orc_params *p, int64_t n, orc_state *s, const orc_block_t *blk)
{
    if (p && p->av_switch == 1 && (!s->alpha || !s->dalpha)) return ORC_EINVAL;
    if (p && p->av_switch == 2 && (!s->alpha || !s->cd_divv || !s->cd_xi)) return ORC_EINVAL;
    if (p && p->gravity && !s->zeta) return ORC_EINVAL;
    if (!params_ok(p, n)) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    double hmax = 0;
    for (int64_t j = 0; j < n; ++j) hmax = s->h[j] > hmax ? s->h[j] : hmax;
    grid_t g;
    memset(&g, 0, sizeof g);
    const grid_t *gp = NULL;
    if (p->use_grid) {
        if (grid_build(&g, p, s, n, 2.0 * median_spacing_guess(p, s, n))) return ORC_ENOMEM;
        gp = &g;
    }
    kdtree_t kt;
    if (gravity_tree_build(p, s, n, &kt)) {
        if (gp) grid_free(&g);
        return ORC_ENOMEM;
    }
    const double aac = p->alpha_ac;
    int status = ORC_OK;
    /* Cullen & Dehnen: the previous div v (its signs enter R) and the new one */
    double *dprev = NULL, *dnew = NULL;
    if (p->av_switch == 2) {
        dprev = (double *)malloc(sizeof(double) * (size_t)n);
        dnew = (double *)malloc(sizeof(double) * (size_t)n);
        if (!dprev || !dnew) {
            free(dprev);
            free(dnew);
            kd_free(&kt);
            grid_free(&g);
            return ORC_ENOMEM;
        }
        memcpy(dprev, s->cd_divv, sizeof(double) * (size_t)n);
        memcpy(dnew, s->cd_divv, sizeof(double) * (size_t)n);
    }
#pragma omp parallel
    {
        idlist_t buf = {0, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < n; ++i) {
            if (blk && blk->active && !blk->active[i]) continue;
            int rc = gather(p, s, n, gp, i, kernel_R(p->kernel) * hmax, s->h, &buf);
            if (rc) {
#pragma omp critical
                status = rc;
                continue;
            }
            const double Ai = s->P[i] / (s->omega[i] * s->rho[i] * s->rho[i]);
            kahan_t ax = {0, 0}, ay = {0, 0}, az = {0, 0}, du = {0, 0}, dv = {0, 0};
            cd_sums_t cds;
            memset(&cds, 0, sizeof cds);
            double vsig = 2.0 * s->c[i]; /* no neighbour: c_i + c_i */
            int have = 0;
            int32_t maxlev = -1; /* no neighbour */
            for (int64_t k = 0; k < buf.n; ++k) {
                int64_t j = buf.v[k];
                if (j == i) continue;
                if (blk && blk->level[j] > maxlev) maxlev = blk->level[j];
                sep_t sp = separation(p, s, i, j);
                double r = sqrt(sp.r2);
                double rx = sp.dx / r, ry = sp.dy / r, rz = sp.dz / r; /* r_hat_ij */
                double gi = orc_dWdrk(p->kernel, r, s->h[i]);           /* grad_i W(h_i) = gi r_hat */
                double gj = orc_dWdrk(p->kernel, r, s->h[j]);           /* grad_i W(h_j) = gj r_hat */
                double Aj = s->P[j] / (s->omega[j] * s->rho[j] * s->rho[j]);
                double mj = s->m[j];
                /* pressure term, Eq. GRADHMOMEQN */
                double fp = -mj * (Ai * gi + Aj * gj);
                if (p->gravity) /* zeta term of Eq. SPHSELFGRAV */
                    fp -= 0.5 * p->G * mj * (s->zeta[i] / s->omega[i] * gi + s->zeta[j] / s->omega[j] * gj);
                double vxij = s->vx[i] - s->vx[j], vyij = s->vy[i] - s->vy[j], vzij = s->vz[i] - s->vz[j];
                double vdr = vxij * rx + vyij * ry + vzij * rz; /* v_ij . r_hat_ij */
                double gbar = 0.5 * (gi + gj);                   /* r_hat . mean grad W */
                double rhobar = 0.5 * (s->rho[i] + s->rho[j]);
                double fav = 0.0, duav = 0.0, alpha, beta;
                av_pair(p, s, i, j, &alpha, &beta);
                kadd(&dv, mj * vdr * gi); /* sum_j m_j v_ij . grad_i W(h_i) */
                if (p->av_switch == 2) {
                    const double vv[3] = {vxij, vyij, vzij}, rh[3] = {rx, ry, rz};
                    for (int a2 = 0; a2 < 3; ++a2)
                        for (int b2 = 0; b2 < 3; ++b2) kadd(&cds.g[3 * a2 + b2], mj * vv[a2] * rh[b2] * gi);
                    kadd(&cds.r, (dprev[j] < 0 ? -1.0 : 1.0) * mj * orc_Wk(p->kernel, r, s->h[i]));
                }
                double vs = s->c[i] + s->c[j] - beta * (vdr < 0 ? vdr : 0.0);
                if (!have || vs > vsig) vsig = vs;
                have = 1;
                if (vdr < 0) {
                    double mu = vdr; /* MIN(0, v_ij . r_hat_ij) */
                    double vsig_av = s->c[i] + s->c[j] - beta * vdr;
                    fav = mj / rhobar * alpha * vsig_av * mu * gbar;            /* Eq. MON97ARTVISC */
                    duav = -mj / rhobar * 0.5 * alpha * vsig_av * mu * mu * gbar; /* Eq. MON97ENERGYDISS */
                }
                double f = fp + fav;
                kadd(&ax, f * rx);
                kadd(&ay, f * ry);
                kadd(&az, f * rz);
                if (p->eos == 0) {
                    double dui = Ai * mj * vdr * gi; /* Eq. GRADHENEQN */
                    double duac = mj / rhobar * aac * ac_signal_speed(p, s, i, j, vdr, rhobar) * (s->u[i] - s->u[j]) * gbar;
                    kadd(&du, dui + duav + duac);
                }
            }
            if (p->gravity) gravity_long_range(p, s, n, &kt, i, &ax, &ay, &az);
            s->ax[i] = ax.s;
            s->ay[i] = ay.s;
            s->az[i] = az.s;
            s->du[i] = (p->eos == 0) ? du.s : 0.0;
            s->vsig[i] = vsig;
            if (p->av_switch == 1) s->dalpha[i] = av_rate(p, s, i, dv.s);
            if (p->av_switch == 2) {
                kadd(&cds.r, (dprev[i] < 0 ? -1.0 : 1.0) * s->m[i] * orc_Wk(p->kernel, 0.0, s->h[i])); /* self */
                cd_finish(p, s, i, &cds, &dnew[i], &s->cd_xi[i]);
            }
            if (blk) blk->ngb_maxlev[i] = maxlev;
        }
        free(buf.v);
    }
    if (gp) grid_free(&g);
    kd_free(&kt);
    if (dnew) memcpy(s->cd_divv, dnew, sizeof(double) * (size_t)n);
    free(dprev);
    free(dnew);
    return status;
}

/* Global time-step: the CFL condition of Eq. SPH_DT, C_CFL * min_i h_i /
   v_sig,i, and with gravity the acceleration condition of Eq. SPH_DTACCEL,
   read as C_GRAV sqrt(h_i / |a_i|) (the printed h_i / sqrt(|a_i|) is not a
   time). */
double orc_cfl_dt(const orc_params *p, int64_t n, const orc_state *s)
{
    double dt = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        double d = p->c_cfl * s->h[i] / s->vsig[i];
        if (d < dt) dt = d;
        if (p->gravity) {
            double a = sqrt(s->ax[i] * s->ax[i] + s->ay[i] * s->ay[i] + s->az[i] * s->az[i]);
            if (a > 0) {
                double g = p->c_grav * sqrt(s->h[i] / a);
                if (g < dt) dt = g;
            }
        }
    }
    return dt;
}

static double wrap(double x, double lo, double L)
{
    double t = x - lo;
    t -= L * floor(t / L);
    if (t >= L) t -= L; /* guard rounding at the upper edge */
    return lo + t;
}

/*
 * One global-step kick-drift-kick (Eqs. LFKDK1, LFKDK2).  The state must hold
 * a and du/dt from the previous force evaluation.  Velocity- and u-dependent
 * forces are evaluated at the predicted v^ = v^(n+1/2) + a^n dt/2 and
 * u^ = u^(n+1/2) + du^n dt/2; the closing kick uses the new rates.
 */
int orc_step(const orc_params *p, int64_t n, orc_state *s, double dt)
{
    if (!params_ok(p, n) || !(dt > 0)) return ORC_EINVAL;
    if (p->av_switch == 1 && (!s->alpha || !s->dalpha)) return ORC_EINVAL;
    if (p->av_switch == 2 && (!s->alpha || !s->cd_divv || !s->cd_xi)) return ORC_EINVAL;
    double *vh = (double *)malloc((size_t)(n > 0 ? n : 1) * 5 * sizeof(double));
    if (!vh) return ORC_ENOMEM;
    double *vhx = vh, *vhy = vh + n, *vhz = vh + 2 * n, *uh = vh + 3 * n, *ah = vh + 4 * n;
    const int adi = (p->eos == 0);
    for (int64_t i = 0; i < n; ++i) {
        vhx[i] = s->vx[i] + 0.5 * s->ax[i] * dt;
        vhy[i] = s->vy[i] + 0.5 * s->ay[i] * dt;
        vhz[i] = s->vz[i] + 0.5 * s->az[i] * dt;
        uh[i] = adi ? s->u[i] + 0.5 * s->du[i] * dt : s->u[i];
        if (p->av_switch == 1) { /* the switch's alpha is kicked and predicted like u */
            ah[i] = s->alpha[i] + 0.5 * s->dalpha[i] * dt;
            s->alpha[i] = ah[i] + 0.5 * s->dalpha[i] * dt;
        }
        s->x[i] += vhx[i] * dt;
        s->y[i] += vhy[i] * dt;
        s->z[i] += vhz[i] * dt;
        if (p->periodic) {
            s->x[i] = wrap(s->x[i], p->box_lo[0], p->box_len[0]);
            s->y[i] = wrap(s->y[i], p->box_lo[1], p->box_len[1]);
            s->z[i] = wrap(s->z[i], p->box_lo[2], p->box_len[2]);
        }
        /* predictor */
        s->vx[i] = vhx[i] + 0.5 * s->ax[i] * dt;
        s->vy[i] = vhy[i] + 0.5 * s->ay[i] * dt;
        s->vz[i] = vhz[i] + 0.5 * s->az[i] * dt;
        if (adi) s->u[i] = uh[i] + 0.5 * s->du[i] * dt;
    }
    double *d_old = NULL; /* Cullen & Dehnen: div v at the step's start */
    if (p->av_switch == 2) {
        d_old = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        if (!d_old) {
            free(vh);
            return ORC_ENOMEM;
        }
        memcpy(d_old, s->cd_divv, sizeof(double) * (size_t)n);
    }
    int rc = orc_density(p, n, s);
    int rc2 = (rc == ORC_OK || rc == ORC_ENOCONV) ? orc_forces(p, n, s) : rc;
    if (d_old) {
        if (rc2 == ORC_OK) orc_cd_update(p, n, s, d_old, dt);
        free(d_old);
    }
    for (int64_t i = 0; i < n; ++i) {
        s->vx[i] = vhx[i] + 0.5 * s->ax[i] * dt;
        s->vy[i] = vhy[i] + 0.5 * s->ay[i] * dt;
        s->vz[i] = vhz[i] + 0.5 * s->az[i] * dt;
        if (adi) s->u[i] = uh[i] + 0.5 * s->du[i] * dt;
        if (p->av_switch == 1) s->alpha[i] = ah[i] + 0.5 * s->dalpha[i] * dt;
    }
    free(vh);
    return rc2 ? rc2 : rc;
}

/* ------------------------------------------------------------------------ */
/* Hierarchical block time-steps (Sec. 2.1.4) with the Saitoh & Makino       */
/* (2009) limiter in its predictive and reactive parts.                      */
/*                                                                           */
/* One call advances every particle from one synchronisation point to the   */
/* next, Delta t_MAX later.  Levels l = 0 .. L give steps Delta t_MAX / 2^l;  */
/* time is counted in ticks of Delta t_MAX / 2^L.  Readings of the paper:    */
/*  - Delta t_MAX = min(max_i dt_i, 2^L min_i dt_i), dt_i the step of Eq.     */
/*    SPH_DT (and Eq. SPH_DTACCEL with gravity), so that every particle fits  */
/*    a level; a particle takes the lowest level whose step is <= its dt_i.   */
/*  - Each particle runs its own kick-drift-kick: a half kick with its       */
/*    acceleration when its step starts, every particle drifts with its half */
/*    step velocity at every tick where some particle ends its step, and     */
/*    the particles whose step ends there (active) get a new h, density and  */
/*    forces from the positions of all particles and the predicted           */
/*    v = v_half + a (t - t_mid) and u of all particles, then the closing    */
/*    half kick.  Inactive particles keep the h, rho, Omega, P and c of      */
/*    their last solve (only the active particles' density is solved).      */
/*  - A new step's level may rise freely but fall by one level only, and    */
/*    only where the tick is a multiple of the longer step (Sec. 2.1.4).     */
/*  - Predictive limiter: a new level is at least (largest level among the  */
/*    force neighbours at the last force pass) - dl, i.e. a step at most     */
/*    2^dl times the shortest neighbour's.  Reactive limiter: an active      */
/*    particle on level l lifts every inactive force neighbour below l - dl  */
/*    to l - dl; that neighbour's step then ends at the next tick that is a  */
/*    multiple of its new step, and its opening half kick is corrected to    */
/*    the shortened step (v_half += a (dt' - dt)/2).                         */
/* ------------------------------------------------------------------------ */
int orc_density_subset(const orc_params *p, int64_t n, orc_state *s, int64_t nsub, const int64_t *idx);

static int level_of(double dt, double dtmax, int L)
{
    int l = 0;
    while (l < L && ldexp(dtmax, -l) > dt) ++l;
    return l;
}

static double particle_dt(const orc_params *p, const orc_state *s, int64_t i)
{
    double d = p->c_cfl * s->h[i] / s->vsig[i];
    if (p->gravity) {
        double a = sqrt(s->ax[i] * s->ax[i] + s->ay[i] * s->ay[i] + s->az[i] * s->az[i]);
        if (a > 0) {
            double g = p->c_grav * sqrt(s->h[i] / a);
            if (g < d) d = g;
        }
    }
    return d;
}

/* The lifted level l - dl that active particle i asks of each inactive
   force neighbour below it (the reactive part), as a maximum per particle. */
static int reactive_requests(const orc_params *p, int64_t n, const orc_state *s, const int32_t *level,
                             const uint8_t *active, int dl, int32_t *req)
{
    double hmax = 0;
    for (int64_t j = 0; j < n; ++j) hmax = s->h[j] > hmax ? s->h[j] : hmax;
    grid_t g;
    memset(&g, 0, sizeof g);
    const grid_t *gp = NULL;
    if (p->use_grid) {
        if (grid_build(&g, p, s, n, 2.0 * median_spacing_guess(p, s, n))) return ORC_ENOMEM;
        gp = &g;
    }
    idlist_t buf = {0, 0, 0};
    int rc = ORC_OK;
    for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
        if (!active[i]) continue;
        rc = gather(p, s, n, gp, i, kernel_R(p->kernel) * hmax, s->h, &buf);
        for (int64_t k = 0; rc == ORC_OK && k < buf.n; ++k) {
            int64_t j = buf.v[k];
            if (j == i || active[j]) continue;
            if (level[j] < level[i] - dl && level[i] - dl > req[j]) req[j] = level[i] - dl;
        }
    }
    free(buf.v);
    if (gp) grid_free(&g);
    return rc;
}

/*
 * One block step of the whole system.  Needs a, du/dt, v_sig (and h) from a
 * force evaluation of every particle at the start, as orc_step does;
 * level[] and ngb_maxlev[] carry the levels and the neighbours' largest
 * levels from one call to the next (zero before the first).  L = largest
 * level, dl = limiter gap in levels (steps within a factor 2^dl of the
 * neighbours').  Writes Delta t_MAX to *dtmax_out, and to counts[0] the
 * force passes and to counts[1] the particle force evaluations they made.
 */
int orc_block_step(const orc_params *p, int64_t n, orc_state *s, int32_t *level, int32_t *ngb_maxlev, int L, int dl,
                   double *dtmax_out, int64_t *counts)
{
    if (!params_ok(p, n) || L < 0 || L > 30 || dl < 1) return ORC_EINVAL;
    if (p->av_switch == 2) return ORC_EINVAL; /* (not combined with block steps) */
    if (p->av_switch == 1 && (!s->alpha || !s->dalpha)) return ORC_EINVAL;
    if (p->av_switch == 2 && (!s->alpha || !s->cd_divv || !s->cd_xi)) return ORC_EINVAL;
    if (p->gravity && !s->zeta) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    const int adi = (p->eos == 0);
    const int64_t N = (int64_t)1 << L;
    double dmin = INFINITY, dmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = particle_dt(p, s, i);
        if (d < dmin) dmin = d;
        if (d > dmax) dmax = d;
    }
    const double dtmax = dmax < ldexp(dmin, L) ? dmax : ldexp(dmin, L);
    const double tau = ldexp(dtmax, -L);
    *dtmax_out = dtmax;
    double *w = (double *)malloc((size_t)n * 5 * sizeof(double));
    int64_t *t0 = (int64_t *)malloc((size_t)n * 2 * sizeof(int64_t));
    uint8_t *act = (uint8_t *)malloc((size_t)n);
    int32_t *req = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int64_t *aidx = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!w || !t0 || !act || !req || !aidx) {
        free(w);
        free(t0);
        free(act);
        free(req);
        free(aidx);
        return ORC_ENOMEM;
    }
    double *vhx = w, *vhy = w + n, *vhz = w + 2 * n, *uh = w + 3 * n, *ah = w + 4 * n;
    int64_t *t1 = t0 + n;
    /* levels of the new steps and the opening half kicks */
    for (int64_t i = 0; i < n; ++i) {
        int l = level_of(particle_dt(p, s, i), dtmax, L);
        if (l < ngb_maxlev[i] - dl) l = ngb_maxlev[i] - dl; /* predictive limiter */
        level[i] = l;
        t0[i] = 0;
        t1[i] = N >> l;
        const double hd = 0.5 * (double)t1[i] * tau;
        vhx[i] = s->vx[i] + s->ax[i] * hd;
        vhy[i] = s->vy[i] + s->ay[i] * hd;
        vhz[i] = s->vz[i] + s->az[i] * hd;
        uh[i] = adi ? s->u[i] + s->du[i] * hd : s->u[i];
        ah[i] = p->av_switch == 1 ? s->alpha[i] + s->dalpha[i] * hd : 0.0;
    }
    int64_t k = 0, npass = 0, nevals = 0;
    int rc = ORC_OK;
    orc_block_t blk = {level, ngb_maxlev, act};
    while (k < N) {
        int64_t kn = N;
        for (int64_t i = 0; i < n; ++i)
            if (t1[i] < kn) kn = t1[i];
        const double dk = (double)(kn - k) * tau;
        for (int64_t i = 0; i < n; ++i) { /* drift every particle to tick kn */
            s->x[i] += vhx[i] * dk;
            s->y[i] += vhy[i] * dk;
            s->z[i] += vhz[i] * dk;
            if (p->periodic) {
                s->x[i] = wrap(s->x[i], p->box_lo[0], p->box_len[0]);
                s->y[i] = wrap(s->y[i], p->box_lo[1], p->box_len[1]);
                s->z[i] = wrap(s->z[i], p->box_lo[2], p->box_len[2]);
            }
        }
        k = kn;
        for (int64_t i = 0; i < n; ++i) { /* active set and the predicted v, u, alpha */
            act[i] = t1[i] == k;
            nevals += act[i];
            const double dp = (double)(2 * k - t0[i] - t1[i]) * 0.5 * tau; /* t - t_mid */
            s->vx[i] = vhx[i] + s->ax[i] * dp;
            s->vy[i] = vhy[i] + s->ay[i] * dp;
            s->vz[i] = vhz[i] + s->az[i] * dp;
            if (adi) s->u[i] = uh[i] + s->du[i] * dp;
            if (p->av_switch == 1) s->alpha[i] = ah[i] + s->dalpha[i] * dp;
            req[i] = -1;
        }
        int64_t na = 0;
        for (int64_t i = 0; i < n; ++i)
            if (act[i]) aidx[na++] = i;
        rc = orc_density_subset(p, n, s, na, aidx);
        if (rc != ORC_OK && rc != ORC_ENOCONV) break;
        int rc2 = forces_impl(p, n, s, &blk);
        if (rc2 == ORC_OK) rc2 = reactive_requests(p, n, s, level, act, dl, req);
        if (rc2) {
            rc = rc2;
            break;
        }
        ++npass;
        for (int64_t i = 0; i < n; ++i) {
            if (act[i]) { /* closing half kick, then the next step */
                const double hd = 0.5 * (double)(t1[i] - t0[i]) * tau;
                s->vx[i] = vhx[i] + s->ax[i] * hd;
                s->vy[i] = vhy[i] + s->ay[i] * hd;
                s->vz[i] = vhz[i] + s->az[i] * hd;
                if (adi) s->u[i] = uh[i] + s->du[i] * hd;
                if (p->av_switch == 1) s->alpha[i] = ah[i] + s->dalpha[i] * hd;
                if (k == N) continue;
                int l = level_of(particle_dt(p, s, i), dtmax, L);
                if (l < ngb_maxlev[i] - dl) l = ngb_maxlev[i] - dl;
                if (l < level[i]) /* down one level, and only where synchronised */
                    l = (k % (N >> (level[i] - 1)) == 0) ? level[i] - 1 : level[i];
                level[i] = l;
                t0[i] = k;
                t1[i] = k + (N >> l);
                const double hn = 0.5 * (double)(N >> l) * tau;
                vhx[i] = s->vx[i] + s->ax[i] * hn;
                vhy[i] = s->vy[i] + s->ay[i] * hn;
                vhz[i] = s->vz[i] + s->az[i] * hn;
                uh[i] = adi ? s->u[i] + s->du[i] * hn : s->u[i];
                if (p->av_switch == 1) ah[i] = s->alpha[i] + s->dalpha[i] * hn;
            } else if (req[i] > level[i]) { /* reactive limiter: end the step early */
                const int64_t st = N >> req[i];
                const int64_t ke = (k / st + 1) * st; /* next tick on the new level's grid */
                if (ke < t1[i]) {
                    const double corr = 0.5 * (double)(ke - t1[i]) * tau;
                    vhx[i] += s->ax[i] * corr;
                    vhy[i] += s->ay[i] * corr;
                    vhz[i] += s->az[i] * corr;
                    if (adi) uh[i] += s->du[i] * corr;
                    if (p->av_switch == 1) ah[i] += s->dalpha[i] * corr;
                    t1[i] = ke;
                    level[i] = req[i];
                }
            }
        }
    }
    counts[0] = npass;
    counts[1] = nevals;
    free(w);
    free(t0);
    free(act);
    free(req);
    free(aidx);
    return rc;
}

/*
 * Neighbour lists in CSR form, ids ascending.
 * kind 0: gather list {j : r_ij^2 < (2 h_i)^2} (includes i);
 * kind 1: force list  {j != i : r_ij^2 < (2 max(h_i,h_j))^2}.
 * offsets has n+1 entries.  Returns the total count (may exceed cap, in which
 * case idx holds only the first cap entries), or a negative error.
 */
int64_t orc_neighbours(const orc_params *p, int64_t n, const orc_state *s, int kind,
                       int64_t *offsets, int32_t *idx, int64_t cap)
{
    if (!params_ok(p, n) || (kind != 0 && kind != 1)) return ORC_EINVAL;
    double hmax = 0;
    for (int64_t j = 0; j < n; ++j) hmax = s->h[j] > hmax ? s->h[j] : hmax;
    grid_t g;
    memset(&g, 0, sizeof g);
    const grid_t *gp = NULL;
    if (p->use_grid && n > 0) {
        if (grid_build(&g, p, s, n, 2.0 * median_spacing_guess(p, s, n))) return ORC_ENOMEM;
        gp = &g;
    }
    offsets[0] = 0;
    idlist_t buf = {0, 0, 0};
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        int rc = kind == 0 ? gather(p, s, n, gp, i, kernel_R(p->kernel) * s->h[i], NULL, &buf)
                           : gather(p, s, n, gp, i, kernel_R(p->kernel) * hmax, s->h, &buf);
        if (rc) {
            free(buf.v);
            if (gp) grid_free(&g);
            return rc;
        }
        for (int64_t k = 0; k < buf.n; ++k) {
            if (kind == 1 && buf.v[k] == i) continue;
            if (total < cap) idx[total] = (int32_t)buf.v[k];
            total++;
        }
        offsets[i + 1] = total;
    }
    free(buf.v);
    if (gp) grid_free(&g);
    return total;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/*
 * Density / h solve (Eqs. SPHRHO, HRHO, OMEGA) for the listed particles only,
 * with the grid prefilter; every other particle is left untouched.  Each
 * particle's solve depends only on positions and masses, so the results equal
 * those of orc_density for these particles.
 */
int orc_density_subset(const orc_params *p, int64_t n, orc_state *s, int64_t nsub, const int64_t *idx)
{
    if (!params_ok(p, n) || nsub < 0) return ORC_EINVAL;
    if (n == 0 || nsub == 0) return ORC_OK;
    grid_t g;
    memset(&g, 0, sizeof g);
    if (grid_build(&g, p, s, n, 2.0 * median_spacing_guess(p, s, n))) return ORC_ENOMEM;
    int status = ORC_OK;
#pragma omp parallel
    {
        idlist_t buf = {0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < nsub; ++k) {
            int64_t i = idx[k];
            double rho = 0, drho = 0;
            int32_t nn = 0, it = 0;
            int rc = solve_h(p, s, n, &g, i, &buf, &s->h[i], &rho, &drho, &nn, &it);
            s->rho[i] = rho;
            s->omega[i] = 1.0 + s->h[i] / (3.0 * rho) * drho;
            if (p->gravity) s->zeta[i] = gravity_zeta(p, s, i, &buf, rho);
            eos(p, rho, s->u[i], &s->P[i], &s->c[i]);
            if (s->nngb) s->nngb[i] = nn;
            if (s->iters) s->iters[i] = it;
            if (rc) {
#pragma omp critical
                status = rc;
            }
        }
        free(buf.v);
    }
    grid_free(&g);
    return status;
}

/*
 * Forces (Eqs. GRADHMOMEQN, GRADHENEQN, MON97ARTVISC, MON97ENERGYDISS, SPH_DT)
 * for the listed particles only.  h, rho, Omega, P, c must be valid for these
 * particles and for all their force neighbours.  hmax bounds the smoothing
 * lengths of the particles that can reach a listed one (the grid query
 * radius is 2 hmax).
 */
int orc_forces_subset(const orc_params *p, int64_t n, orc_state *s, int64_t nsub, const int64_t *idx,
                      double hmax)
{
    if (!params_ok(p, n) || nsub < 0 || !(hmax > 0)) return ORC_EINVAL;
    if (p->av_switch == 1 && (!s->alpha || !s->dalpha)) return ORC_EINVAL;
    if (p->av_switch == 2 && (!s->alpha || !s->cd_divv || !s->cd_xi)) return ORC_EINVAL;
    if (n == 0 || nsub == 0) return ORC_OK;
    grid_t g;
    memset(&g, 0, sizeof g);
    if (grid_build(&g, p, s, n, 2.0 * median_spacing_guess(p, s, n))) return ORC_ENOMEM;
    kdtree_t kt;
    if (gravity_tree_build(p, s, n, &kt)) {
        grid_free(&g);
        return ORC_ENOMEM;
    }
    const double aac = p->alpha_ac;
    int status = ORC_OK;
    /* Cullen & Dehnen: the previous div v (its signs enter R) and the new one */
    double *dprev = NULL, *dnew = NULL;
    if (p->av_switch == 2) {
        dprev = (double *)malloc(sizeof(double) * (size_t)n);
        dnew = (double *)malloc(sizeof(double) * (size_t)n);
        if (!dprev || !dnew) {
            free(dprev);
            free(dnew);
            kd_free(&kt);
            grid_free(&g);
            return ORC_ENOMEM;
        }
        memcpy(dprev, s->cd_divv, sizeof(double) * (size_t)n);
        memcpy(dnew, s->cd_divv, sizeof(double) * (size_t)n);
    }
#pragma omp parallel
    {
        idlist_t buf = {0, 0, 0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t k = 0; k < nsub; ++k) {
            int64_t i = idx[k];
            int rc = gather(p, s, n, &g, i, kernel_R(p->kernel) * hmax, s->h, &buf);
            if (rc) {
#pragma omp critical
                status = rc;
                continue;
            }
            const double Ai = s->P[i] / (s->omega[i] * s->rho[i] * s->rho[i]);
            kahan_t ax = {0, 0}, ay = {0, 0}, az = {0, 0}, du = {0, 0}, dv = {0, 0};
            cd_sums_t cds;
            memset(&cds, 0, sizeof cds);
            double vsig = 2.0 * s->c[i];
            int have = 0;
            for (int64_t q = 0; q < buf.n; ++q) {
                int64_t j = buf.v[q];
                if (j == i) continue;
                sep_t sp = separation(p, s, i, j);
                double r = sqrt(sp.r2);
                double rx = sp.dx / r, ry = sp.dy / r, rz = sp.dz / r;
                double gi = orc_dWdrk(p->kernel, r, s->h[i]);
                double gj = orc_dWdrk(p->kernel, r, s->h[j]);
                double Aj = s->P[j] / (s->omega[j] * s->rho[j] * s->rho[j]);
                double mj = s->m[j];
                double fp = -mj * (Ai * gi + Aj * gj);
                if (p->gravity) /* zeta term of Eq. SPHSELFGRAV */
                    fp -= 0.5 * p->G * mj * (s->zeta[i] / s->omega[i] * gi + s->zeta[j] / s->omega[j] * gj);
                double vxij = s->vx[i] - s->vx[j], vyij = s->vy[i] - s->vy[j], vzij = s->vz[i] - s->vz[j];
                double vdr = vxij * rx + vyij * ry + vzij * rz;
                double gbar = 0.5 * (gi + gj);
                double rhobar = 0.5 * (s->rho[i] + s->rho[j]);
                double fav = 0.0, duav = 0.0, alpha, beta;
                av_pair(p, s, i, j, &alpha, &beta);
                kadd(&dv, mj * vdr * gi); /* sum_j m_j v_ij . grad_i W(h_i) */
                if (p->av_switch == 2) {
                    const double vv[3] = {vxij, vyij, vzij}, rh[3] = {rx, ry, rz};
                    for (int a2 = 0; a2 < 3; ++a2)
                        for (int b2 = 0; b2 < 3; ++b2) kadd(&cds.g[3 * a2 + b2], mj * vv[a2] * rh[b2] * gi);
                    kadd(&cds.r, (dprev[j] < 0 ? -1.0 : 1.0) * mj * orc_Wk(p->kernel, r, s->h[i]));
                }
                double vs = s->c[i] + s->c[j] - beta * (vdr < 0 ? vdr : 0.0);
                if (!have || vs > vsig) vsig = vs;
                have = 1;
                if (vdr < 0) {
                    double mu = vdr;
                    double vsig_av = s->c[i] + s->c[j] - beta * vdr;
                    fav = mj / rhobar * alpha * vsig_av * mu * gbar;
                    duav = -mj / rhobar * 0.5 * alpha * vsig_av * mu * mu * gbar;
                }
                double f = fp + fav;
                kadd(&ax, f * rx);
                kadd(&ay, f * ry);
                kadd(&az, f * rz);
                if (p->eos == 0) {
                    double dui = Ai * mj * vdr * gi;
                    double duac = mj / rhobar * aac * ac_signal_speed(p, s, i, j, vdr, rhobar) * (s->u[i] - s->u[j]) * gbar;
                    kadd(&du, dui + duav + duac);
                }
            }
            if (p->gravity) gravity_long_range(p, s, n, &kt, i, &ax, &ay, &az);
            s->ax[i] = ax.s;
            s->ay[i] = ay.s;
            s->az[i] = az.s;
            s->du[i] = (p->eos == 0) ? du.s : 0.0;
            s->vsig[i] = vsig;
            if (p->av_switch == 1) s->dalpha[i] = av_rate(p, s, i, dv.s);
            if (p->av_switch == 2) {
                kadd(&cds.r, (dprev[i] < 0 ? -1.0 : 1.0) * s->m[i] * orc_Wk(p->kernel, 0.0, s->h[i])); /* self */
                cd_finish(p, s, i, &cds, &dnew[i], &s->cd_xi[i]);
            }
        }
        free(buf.v);
    }
    grid_free(&g);
    kd_free(&kt);
    if (dnew) memcpy(s->cd_divv, dnew, sizeof(double) * (size_t)n);
    free(dprev);
    free(dnew);
    return status;
}
