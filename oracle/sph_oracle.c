/*
 * sph_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle of the SPH
 * particle step of relativistic viscous BSQ hydrodynamics (arXiv 2511.22852,
 * Sec. "Numerical solver: Smoothed particle hydrodynamics (SPH)").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library, and the
 * product path never calls it.
 *
 * Everything is written the plain way, in the paper's order:
 *   1. neighbour pairs r_ab < 2h (brute force O(N^2) and a uniform cell list;
 *      both must give the same set)                      -- Sec. "Kokkos and Cabana" (VerletList)
 *   2. kernel sums sigma*_a = sum_b W_ab, s*_a = sum_b S_b W_ab,
 *      n*_qa = sum_b N_qb W_ab; rest frame q = (q*) / (u^0 sqrt(-g))  -- eqs. refconv, sigmastar
 *   3. EoS inversion (s, n_B, n_S, n_Q) -> (T, mu_B, mu_S, mu_Q) by Newton on the
 *      quadrilinear table interpolant, with the closed-form EoS as backup  -- Sec. "EoS inverter"
 *   4. SPH gradients: du^j/dx^k with the n = 0 form, the stress divergence with
 *      the n = -1 form                                   -- eqs. sphderivativerel, generalsphderivative
 *   5. equations of motion: the acceleration from the linear system
 *      M du/dx0 = F, entropy production, minimal Israel-Stewart relaxation
 *                                                        -- eqs. genform, unugeneral, dsdnrewr,
 *                                                           min_bul_rel, min_she_rel
 *   6. Heun (RK2) update.
 *   7. totals: energy, entropy, charges, longitudinal work.
 *
 * The equations of motion are evaluated with generic 4x4 tensor algebra in a
 * diagonal metric with explicit Christoffel symbols (Sec. "Notation"), i.e. the
 * covariant formulas written out, not a specialised closed form.
 *
 * Compile with -ffp-contract=off so that the neighbour-acceptance test
 * r^2 = dx*dx + dy*dy (+ dz*dz) < (2h)^2 rounds each product separately.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HBARC 0.1973269804
#define NAUX 18

/* per-particle status bits */
#define ST_FALLBACK 1u     /* table Newton failed, closed-form EoS used */
#define ST_OUT_OF_TABLE 2u /* closed-form solution outside the table domain */
#define ST_NOCONV 4u       /* no EoS solution */
#define ST_NONFINITE 8u
#define ST_CS2_CAPPED 16u
#define ST_SOLVE_FAIL 32u  /* acceleration system singular */
#define ST_BACKUP 64u      /* no closed-form solution: the conformal-diagonal backup EoS used */

typedef struct {
    int dim;     /* SPH dimensions: 2 (x, y) or 3 (x, y, eta|z) */
    int milne;   /* 1: coordinates (tau, x, y, eta); 0: (t, x, y, z) */
    int viscous; /* 0: ideal; 1: minimal Israel-Stewart shear + bulk */
    int has_table;
    double h;
    /* closed-form EoS: p = T^4 [a0 + a1 (1 + tanh((T hc - Tc)/w))/2] + T^2 sum chi mu^2 / 2 */
    double a0, a1, Tc_GeV, w_GeV;
    double chi[3];
    /* table: regular grid, row-major [T][muB][muS][muQ] */
    int nT;
    int nmu[3];
    double T0, dT;
    double mu0[3], dmu[3];
    const double *tp, *ts, *tnB, *tnS, *tnQ;
    /* transport */
    double eta_over_s, zeta_peak, zeta_T_GeV, zeta_w_GeV;
    double tau_pi_coef, tau_Pi_ratio, cs2_cap;
    /* Newton */
    double newton_tol;
    int newton_maxit;
    int newton_no_polish; /* 1: stop at the first iterate that meets the tolerance (no polishing step) */
    /* energy-momentum source I^nu of straight jet tracks (Cartesian coordinates only):
       tracks[8 k ..]: x0, y0, z0, direction n (unit), start time t0, dE/dx (fm^-2) */
    int ntrack;
    int pad2;
    const double *tracks;
    double track_sigma;
    /* offline inverter (NULL: online Newton): (T, mu_B, mu_S, mu_Q) on the grid of s (log
       decades: node i at s_i = p10[i / K] (1 + 9 (i % K) / K), i <= K nd, p10[d] = 10^(d0 + d))
       times the charge ratios x_q = n_q / s (inv_nx nodes uniform on [-xmax, xmax]);
       node [i][jB][jS][jQ][4] */
    const double *inv;
    const double *inv_p10;
    int inv_K, inv_nd, inv_nx, pad3;
    double inv_xmax;
    /* viscous equations of motion: 0 minimal Israel-Stewart (eqs. min_bul_rel, min_she_rel);
       1 DNMR without K terms and diffusion couplings (eq. dnmr, with the shear-bulk J terms and
       the R term phi_7), coefficients as ratios: dnmr[0] = delta_PiPi / tau_Pi,
       dnmr[1] = lambda_Pipi / (tau_Pi (1/3 - c_s^2)), dnmr[2] = delta_pipi / tau_pi,
       dnmr[3] = tau_pipi / tau_pi, dnmr[4] = lambda_piPi / tau_pi, dnmr[5] = phi_7 p */
    int eom_model, pad4;
    double dnmr[6];
    /* dynamical-initialisation sources (Sec. "Dynamical initialization"): partons[8 k ..] =
       formation time x^0_k, position (x, y, z|eta), four-momentum p^mu (contravariant, the
       event's coordinates); a parton formed in (x^0 - dt, x^0] deposits
       N p^mu W(r - r_k, h_src) / (sqrt(-g) dt) at the stage evaluated at x^0 */
    int nparton, pad5;
    const double *partons;
    double parton_norm, parton_h, parton_dt;
    /* backup EoS (Sec. "Equation of state", backup EoS): where neither the table nor the closed
       form inverts, the conformal-diagonal EoS p = A0 [T^4 + sum_q (mu_q / mu_q0)^4] (T_0 = 1/fm),
       which inverts (s, n) in closed form; backup = 0: none (the particle has no solution) */
    int backup, pad6;
    double cd_A0, cd_mu0[3];
    /* charges of the dynamical-initialisation partons (eq. charge_conservation with I_q != 0):
       parton_q[3 k ..] = (B, S, Q) of parton k, smeared like its four-momentum (NULL: none) */
    const double *parton_q;
    /* temperature (GeV) below which a particle has left the fluid: it streams freely
       (dx/dx0 = v, its other variables and charges constant) while its neighbours still see its
       kernel sums and pressure (0: off) */
    double T_stop_GeV;
    /* BSQ diffusion (eq. min_dif_rel, minimal Israel-Stewart): tau_q Delta^mu_nu D J^nu_q + J^mu_q
       = kappa_{qq'} nabla^<mu> alpha_{q'} (metric (+,-,-,-)), alpha_q = mu_q / T, with
       kappa_{qq'} = kappaT2[3 q + q'] T^2
       and the diagonal relaxation times tau_q = tauJT[q] / T (constant kappa/T^2 and tau T, Sec.
       "Transport coefficients").  The state then carries J^i_q / sigma (contravariant spatial
       components, charge major) after the shear rows, and the charges Nq are the particles' lab
       charges sqrt(-g) N^0_q / sigma* = N_q + J^0_q / (sigma u^0) (see oc_stage). */
    int diffusion;
    int pad8;
    double kappaT2[9];
    double tauJT[3];
} oc_params;

/* ------------------------------------------------------------------------ */
/* cubic spline kernel (Sec. "Kernel function")                              */
/* ------------------------------------------------------------------------ */
static double sigma_d(int dim, double h)
{
    if (dim == 1) return 2.0 / (3.0 * h);
    if (dim == 2) return 10.0 / (7.0 * M_PI * h * h);
    return 1.0 / (M_PI * h * h * h);
}

double oc_W(double r, double h, int dim)
{
    double q = r / h;
    double sd = sigma_d(dim, h);
    if (q <= 1.0) return sd * (1.0 - 1.5 * q * q + 0.75 * q * q * q);
    if (q <= 2.0) return sd * 0.25 * (2.0 - q) * (2.0 - q) * (2.0 - q);
    return 0.0;
}

/* dW/dr: the gradient formula of the paper is (dW/dr) (r_a - r_b)/r */
double oc_dWdr(double r, double h, int dim)
{
    double q = r / h;
    double sd = sigma_d(dim, h);
    if (q <= 1.0) return sd / h * (-3.0 * q + 2.25 * q * q);
    if (q <= 2.0) return sd / h * (-0.75 * (2.0 - q) * (2.0 - q));
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* cells, Morton keys, neighbour pairs                                       */
/* ------------------------------------------------------------------------ */
static double r2_of(int dim, const double *x, long n, long a, long b)
{
    double r2 = 0.0;
    for (int d = 0; d < dim; ++d) {
        double dx = x[d * n + a] - x[d * n + b];
        double sq = dx * dx;
        r2 = r2 + sq;
    }
    return r2;
}

/* cell coordinates c_d = floor((x_d - min_a x_d) * (1/(2h))) */
void oc_cell_coords(long n, int dim, const double *x, double h, int *cc, double *xmin_out)
{
    double inv_cell = 1.0 / (2.0 * h);
    for (int d = 0; d < dim; ++d) {
        double m = INFINITY;
        for (long a = 0; a < n; ++a)
            if (x[d * n + a] < m) m = x[d * n + a];
        xmin_out[d] = m;
        for (long a = 0; a < n; ++a) cc[d * n + a] = (int)floor((x[d * n + a] - m) * inv_cell);
    }
}

/* Morton key: bit (dim*b + d) of the key is bit b of c_d */
uint64_t oc_morton(int dim, const int *c)
{
    uint64_t key = 0;
    int bits = dim == 2 ? 32 : 21;
    for (int b = 0; b < bits; ++b)
        for (int d = 0; d < dim; ++d) key |= (uint64_t)(((unsigned)c[d] >> b) & 1u) << (dim * b + d);
    return key;
}

typedef struct {
    uint64_t key;
    long id;
} keyid;

static int cmp_keyid(const void *pa, const void *pb)
{
    const keyid *a = (const keyid *)pa, *b = (const keyid *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* Morton keys and the permutation that sorts particles by (key, id) */
void oc_sort_by_cell(long n, int dim, const double *x, double h, int *cc, uint64_t *keys, long *perm)
{
    double xmin[3];
    oc_cell_coords(n, dim, x, h, cc, xmin);
    keyid *t = (keyid *)malloc(sizeof(keyid) * (size_t)(n > 0 ? n : 1));
    for (long a = 0; a < n; ++a) {
        int c[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) c[d] = cc[d * n + a];
        keys[a] = oc_morton(dim, c);
        t[a].key = keys[a];
        t[a].id = a;
    }
    qsort(t, (size_t)n, sizeof(keyid), cmp_keyid);
    for (long j = 0; j < n; ++j) perm[j] = t[j].id;
    free(t);
}

/* all ordered pairs (a, b) with r_ab^2 < (2h)^2, self pairs included, sorted by (a, b) */
long oc_neighbors_brute(long n, int dim, const double *x, double h, long cap, int *pa, int *pb)
{
    double two_h = 2.0 * h;
    double supp2 = two_h * two_h;
    long cnt = 0;
    for (long a = 0; a < n; ++a)
        for (long b = 0; b < n; ++b)
            if (r2_of(dim, x, n, a, b) < supp2) {
                if (cnt < cap) {
                    pa[cnt] = (int)a;
                    pb[cnt] = (int)b;
                }
                ++cnt;
            }
    return cnt;
}

/* uniform cell list: cells of side 2h, particles bucketed in id order */
typedef struct {
    int dim;
    long n;
    int nc[3];
    long ncell;
    int *cc;      /* [dim][n] */
    long *start;  /* [ncell + 1] */
    long *items;  /* [n] */
} grid_t;

static long lin_cell(const grid_t *g, const int *c)
{
    long l = 0;
    for (int d = g->dim - 1; d >= 0; --d) l = l * g->nc[d] + c[d];
    return l;
}

static void grid_build(grid_t *g, long n, int dim, const double *x, double h)
{
    double xmin[3];
    g->dim = dim;
    g->n = n;
    g->cc = (int *)malloc(sizeof(int) * (size_t)(dim * (n > 0 ? n : 1)));
    oc_cell_coords(n, dim, x, h, g->cc, xmin);
    g->ncell = 1;
    for (int d = 0; d < 3; ++d) g->nc[d] = 1;
    for (int d = 0; d < dim; ++d) {
        int m = 0;
        for (long a = 0; a < n; ++a)
            if (g->cc[d * n + a] > m) m = g->cc[d * n + a];
        g->nc[d] = m + 1;
        g->ncell *= g->nc[d];
    }
    g->start = (long *)calloc((size_t)g->ncell + 1, sizeof(long));
    g->items = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long *cell_of = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (long a = 0; a < n; ++a) {
        int c[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) c[d] = g->cc[d * n + a];
        cell_of[a] = lin_cell(g, c);
        g->start[cell_of[a] + 1]++;
    }
    for (long c = 0; c < g->ncell; ++c) g->start[c + 1] += g->start[c];
    long *fill = (long *)malloc(sizeof(long) * (size_t)g->ncell);
    memcpy(fill, g->start, sizeof(long) * (size_t)g->ncell);
    for (long a = 0; a < n; ++a) g->items[fill[cell_of[a]]++] = a;
    free(fill);
    free(cell_of);
}

static void grid_free(grid_t *g)
{
    free(g->cc);
    free(g->start);
    free(g->items);
}

/* visit every candidate b in the 3^dim cells around a's cell, in increasing b */
typedef void (*pair_fn)(long a, long b, double r2, void *ctx);

static int cmp_long(const void *pa, const void *pb)
{
    long a = *(const long *)pa, b = *(const long *)pb;
    return (a > b) - (a < b);
}

static long grid_neighbors(const grid_t *g, const double *x, double supp2, long a, long *buf)
{
    long n = g->n, cnt = 0;
    int dim = g->dim;
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
        lo[d] = g->cc[d * n + a] - 1;
        hi[d] = g->cc[d * n + a] + 1;
        if (lo[d] < 0) lo[d] = 0;
        if (hi[d] > g->nc[d] - 1) hi[d] = g->nc[d] - 1;
    }
    int c[3];
    for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
        for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
            for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) {
                long l = lin_cell(g, c);
                for (long k = g->start[l]; k < g->start[l + 1]; ++k) {
                    long b = g->items[k];
                    if (r2_of(dim, x, n, a, b) < supp2) buf[cnt++] = b;
                }
            }
    qsort(buf, (size_t)cnt, sizeof(long), cmp_long);
    return cnt;
}

long oc_neighbors_cells(long n, int dim, const double *x, double h, long cap, int *pa, int *pb)
{
    grid_t g;
    grid_build(&g, n, dim, x, h);
    double two_h = 2.0 * h;
    double supp2 = two_h * two_h;
    long *buf = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    long cnt = 0;
    for (long a = 0; a < n; ++a) {
        long m = grid_neighbors(&g, x, supp2, a, buf);
        for (long k = 0; k < m; ++k) {
            if (cnt < cap) {
                pa[cnt] = (int)a;
                pb[cnt] = (int)buf[k];
            }
            ++cnt;
        }
    }
    free(buf);
    grid_free(&g);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* equation of state                                                         */
/* ------------------------------------------------------------------------ */
static void an_f(const oc_params *P, double T, double *f, double *fp, double *fpp)
{
    double x = T * HBARC;
    double th = tanh((x - P->Tc_GeV) / P->w_GeV);
    double sech2 = 1.0 - th * th;
    double k = HBARC / P->w_GeV;
    *f = P->a0 + P->a1 * (1.0 + th) / 2.0;
    *fp = P->a1 / 2.0 * sech2 * k;
    *fpp = -P->a1 * sech2 * th * k * k;
}

/* closed form: p, (s, n) and H = d(s, n)/d(T, mu) */
void oc_eos_analytic(const oc_params *P, double T, const double *mu, double *p, double *sn, double *H)
{
    double f, fp, fpp;
    an_f(P, T, &f, &fp, &fpp);
    double cm2 = 0.0;
    for (int q = 0; q < 3; ++q) cm2 += P->chi[q] * mu[q] * mu[q];
    *p = T * T * T * T * f + T * T * cm2 / 2.0;
    sn[0] = 4.0 * T * T * T * f + T * T * T * T * fp + T * cm2;
    for (int q = 0; q < 3; ++q) sn[1 + q] = P->chi[q] * T * T * mu[q];
    if (H) {
        memset(H, 0, sizeof(double) * 16);
        H[0] = 12.0 * T * T * f + 8.0 * T * T * T * fp + T * T * T * T * fpp + cm2;
        for (int q = 0; q < 3; ++q) {
            H[0 * 4 + 1 + q] = 2.0 * P->chi[q] * T * mu[q];
            H[(1 + q) * 4 + 0] = 2.0 * P->chi[q] * T * mu[q];
            H[(1 + q) * 4 + 1 + q] = P->chi[q] * T * T;
        }
    }
}

/* closed-form inversion: mu_q = n_q/(chi_q T^2) reduces it to one equation in T,
   g(T) = 4 T^3 f + T^4 f' + sum_q n_q^2/(chi_q T^3) - s = 0, solved on its upper
   branch by a bracketed, bisection-safeguarded Newton iteration. */
static void an_g(const oc_params *P, double T, double s, const double *n, double *g, double *gp)
{
    double f, fp, fpp;
    an_f(P, T, &f, &fp, &fpp);
    double c = 0.0;
    for (int q = 0; q < 3; ++q)
        if (P->chi[q] > 0.0) c += n[q] * n[q] / P->chi[q];
    *g = 4.0 * T * T * T * f + T * T * T * T * fp + c / (T * T * T) - s;
    *gp = 12.0 * T * T * f + 8.0 * T * T * T * fp + T * T * T * T * fpp - 3.0 * c / (T * T * T * T);
}

int oc_eos_invert_analytic(const oc_params *P, double s, const double *n, double *T_out, double *mu_out)
{
    if (!(s > 0.0) || !isfinite(s)) return ST_NOCONV;
    for (int q = 0; q < 3; ++q) {
        if (!isfinite(n[q])) return ST_NONFINITE;
        if (!(P->chi[q] > 0.0) && n[q] != 0.0) return ST_NOCONV;
    }
    double Thi = cbrt(s / (4.0 * P->a0));
    double g, gp;
    an_g(P, Thi, s, n, &g, &gp);
    double Tlo = Thi, gprev = g;
    int found = (g <= 0.0);
    if (found) Tlo = Thi;
    for (int k = 0; k < 400 && !found; ++k) {
        Tlo = 0.8 * Tlo;
        double gl, gpl;
        an_g(P, Tlo, s, n, &gl, &gpl);
        if (gl <= 0.0) {
            found = 1;
            break;
        }
        if (gl > gprev) return ST_NOCONV; /* passed the minimum of g: no root */
        gprev = gl;
    }
    if (!found) return ST_NOCONV;
    double T = Thi;
    if (g == 0.0) {
        Tlo = Thi;
    }
    for (int it = 0; it < 200; ++it) {
        an_g(P, T, s, n, &g, &gp);
        if (g == 0.0) break;
        if (g > 0.0) Thi = T;
        else Tlo = T;
        double Tn = T - g / gp;
        if (!(gp > 0.0) || !(Tn > Tlo && Tn < Thi)) Tn = 0.5 * (Tlo + Thi);
        if (fabs(Tn - T) <= 4e-16 * T) {
            T = Tn;
            break;
        }
        T = Tn;
    }
    *T_out = T;
    for (int q = 0; q < 3; ++q) mu_out[q] = P->chi[q] > 0.0 ? n[q] / (P->chi[q] * T * T) : 0.0;
    return 0;
}

/* quadrilinear interpolation of the table (value and gradient), plain 16-corner sum */
static long tab_node(const oc_params *P, int iT, int iB, int iS, int iQ)
{
    return (((long)iT * P->nmu[0] + iB) * P->nmu[1] + iS) * P->nmu[2] + iQ;
}

static void tab_locate(double v, double v0, double dv, int nv, int *i, double *t)
{
    double r = (v - v0) / dv;
    int k = (int)floor(r);
    if (k < 0) k = 0;
    if (k > nv - 2) k = nv - 2;
    *i = k;
    *t = r - (double)k;
}

/* out: value of p, s, nB, nS, nQ at x; J[4][4] = d(s,nB,nS,nQ)/d(T,muB,muS,muQ) */
void oc_eos_table(const oc_params *P, const double *x, double *pv, double *sn, double *J)
{
    int idx[4];
    double t[4], inv[4];
    tab_locate(x[0], P->T0, P->dT, P->nT, &idx[0], &t[0]);
    inv[0] = 1.0 / P->dT;
    for (int q = 0; q < 3; ++q) {
        tab_locate(x[1 + q], P->mu0[q], P->dmu[q], P->nmu[q], &idx[1 + q], &t[1 + q]);
        inv[1 + q] = 1.0 / P->dmu[q];
    }
    const double *fld[5] = {P->ts, P->tnB, P->tnS, P->tnQ, P->tp};
    double val[5] = {0, 0, 0, 0, 0};
    double der[4][4];
    memset(der, 0, sizeof(der));
    for (int c = 0; c < 16; ++c) {
        int bit[4] = {(c >> 3) & 1, (c >> 2) & 1, (c >> 1) & 1, c & 1};
        double w[4], dw[4];
        for (int k = 0; k < 4; ++k) {
            w[k] = bit[k] ? t[k] : 1.0 - t[k];
            dw[k] = (bit[k] ? 1.0 : -1.0) * inv[k];
        }
        long node = tab_node(P, idx[0] + bit[0], idx[1] + bit[1], idx[2] + bit[2], idx[3] + bit[3]);
        double wall = w[0] * w[1] * w[2] * w[3];
        for (int f = 0; f < 5; ++f) val[f] += wall * fld[f][node];
        for (int k = 0; k < 4; ++k) {
            double wk = dw[k];
            for (int m = 0; m < 4; ++m)
                if (m != k) wk *= w[m];
            for (int f = 0; f < 4; ++f) der[f][k] += wk * fld[f][node];
        }
    }
    if (pv) *pv = val[4];
    for (int f = 0; f < 4; ++f) sn[f] = val[f];
    if (J)
        for (int f = 0; f < 4; ++f)
            for (int k = 0; k < 4; ++k) J[f * 4 + k] = der[f][k];
}

/* Gaussian elimination with partial pivoting, A (m x m, row major) x = b; returns 0 on success */
static int gauss_solve(int m, double *A, double *b)
{
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(A[r * m + c]) > fabs(A[piv * m + c])) piv = r;
        if (!(fabs(A[piv * m + c]) > 0.0) || !isfinite(A[piv * m + c])) return -1;
        if (piv != c) {
            for (int k = 0; k < m; ++k) {
                double tmp = A[c * m + k];
                A[c * m + k] = A[piv * m + k];
                A[piv * m + k] = tmp;
            }
            double tmp = b[c];
            b[c] = b[piv];
            b[piv] = tmp;
        }
        for (int r = c + 1; r < m; ++r) {
            double f = A[r * m + c] / A[c * m + c];
            for (int k = c; k < m; ++k) A[r * m + k] -= f * A[c * m + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = m - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < m; ++k) acc -= A[r * m + k] * b[k];
        b[r] = acc / A[r * m + r];
    }
    return 0;
}

static int in_table(const oc_params *P, const double *x)
{
    if (!(x[0] >= P->T0 && x[0] <= P->T0 + (P->nT - 1) * P->dT)) return 0;
    for (int q = 0; q < 3; ++q)
        if (!(x[1 + q] >= P->mu0[q] && x[1 + q] <= P->mu0[q] + (P->nmu[q] - 1) * P->dmu[q])) return 0;
    return 1;
}

static void clamp_table(const oc_params *P, double *x)
{
    double hiT = P->T0 + (P->nT - 1) * P->dT;
    if (x[0] < P->T0) x[0] = P->T0;
    if (x[0] > hiT) x[0] = hiT;
    for (int q = 0; q < 3; ++q) {
        double lo = P->mu0[q], hi = P->mu0[q] + (P->nmu[q] - 1) * P->dmu[q];
        if (x[1 + q] < lo) x[1 + q] = lo;
        if (x[1 + q] > hi) x[1 + q] = hi;
    }
}

static double resid_inf(const oc_params *P, const double *x, double s, const double *n, double *r, double *J)
{
    double sn[4];
    oc_eos_table(P, x, NULL, sn, J);
    double tgt[4] = {s, n[0], n[1], n[2]};
    double m = 0.0;
    for (int k = 0; k < 4; ++k) {
        r[k] = (sn[k] - tgt[k]) / s;
        if (fabs(r[k]) > m || !isfinite(r[k])) m = isfinite(r[k]) ? fabs(r[k]) : INFINITY;
    }
    if (J)
        for (int k = 0; k < 16; ++k) J[k] /= s;
    return m;
}

/* damped Newton on the table interpolant, started from x; 0 = converged */
static int table_newton(const oc_params *P, double s, const double *n, double *x)
{
    double r[4], J[16];
    double rn = resid_inf(P, x, s, n, r, J);
    for (int it = 0; it < P->newton_maxit; ++it) {
        if (rn <= P->newton_tol) {
            /* one polishing step, kept when its point still meets the tolerance: both points are
               solutions under the stopping rule; the polished one lies at the interpolant's root to
               rounding (quadratic convergence), so the result no longer depends on which iterate
               first crossed the tolerance */
            if (P->newton_no_polish) return 0;
            double A[16], d[4], xn[4], rr[4];
            memcpy(A, J, sizeof(A));
            for (int k = 0; k < 4; ++k) d[k] = -r[k];
            if (gauss_solve(4, A, d) == 0) {
                for (int k = 0; k < 4; ++k) xn[k] = x[k] + d[k];
                clamp_table(P, xn);
                double rnn = resid_inf(P, xn, s, n, rr, NULL);
                if (rnn <= P->newton_tol) memcpy(x, xn, sizeof(xn));
            }
            return 0;
        }
        double A[16], d[4];
        memcpy(A, J, sizeof(A));
        for (int k = 0; k < 4; ++k) d[k] = -r[k];
        if (gauss_solve(4, A, d) != 0) return -1;
        double lam = 1.0, xn[4], rr[4], Jn[16], rnn = INFINITY;
        for (int ls = 0; ls <= 8; ++ls) {
            for (int k = 0; k < 4; ++k) xn[k] = x[k] + lam * d[k];
            clamp_table(P, xn);
            rnn = resid_inf(P, xn, s, n, rr, Jn);
            if (rnn < rn) break;
            lam *= 0.5;
        }
        /* no decrease along the Newton direction (e.g. the root lies beyond a clamped table
           edge): the iteration has stalled and ends unconverged */
        if (!(rnn < rn)) return -1;
        memcpy(x, xn, sizeof(xn));
        memcpy(r, rr, sizeof(rr));
        memcpy(J, Jn, sizeof(Jn));
        rn = rnn;
    }
    return rn <= P->newton_tol ? 0 : -1;
}

/* out[0..10]: T, muB, muS, muQ, p, e, p_s, p_nB, p_nS, p_nQ, cs2 (after the cap).
   guess: the previous stage's table solution (T, muB, muS, muQ) of this particle, T <= 0
   for none (may be NULL).  The EoS-inversion passage does not fix the root finder's starting
   point; this reading starts from the particle's previous solution.  Order of attempts:
     1. table Newton warm-started from the guess, if the guess lies in the table;
     2. otherwise (or if 1. does not converge) the closed-form solution, then table Newton
        started there if it lies in the table; else the closed form (flagged).
   used_table (may be NULL) receives 1 when the table produced the result. */
/* Offline inverter (Sec. "Equation of state", offline inversion onto a grid in (s, n)): the
   quadrilinear interpolant of the inverted table at (s, n_q / s); -1 outside the grid or where a
   corner holds no solution. */
int oc_inverse_lookup(const oc_params *P, double s, const double *n, double *x)
{
    if (!(s > 0.0)) return -1;
    const int K = P->inv_K, nd = P->inv_nd, nx = P->inv_nx;
    int d = (int)floor(log10(s / P->inv_p10[0]));
    if (d < 0 || d >= nd + 1) return -1;
    double m = s / P->inv_p10[d];
    if (m >= 10.0 && d < nd) {
        m /= 10.0;
        d += 1;
    }
    if (m < 1.0 && d > 0) {
        m *= 10.0;
        d -= 1;
    }
    double r = (m - 1.0) * K / 9.0;
    int j = (int)floor(r);
    if (j > K - 1) j = K - 1;
    if (j < 0) j = 0;
    long i = (long)d * K + j;
    double t[4];
    int ix[4];
    if (i < 0 || i > (long)K * nd - 1) return -1;
    ix[0] = (int)i;
    t[0] = r - j;
    if (t[0] < 0.0 || t[0] > 1.0) return -1;
    const double dxr = 2.0 * P->inv_xmax / (nx - 1);
    for (int q = 0; q < 3; ++q) {
        double rr = (n[q] / s + P->inv_xmax) / dxr;
        if (!(rr >= 0.0 && rr <= (double)(nx - 1))) return -1;
        int k = (int)floor(rr);
        if (k > nx - 2) k = nx - 2;
        ix[1 + q] = k;
        t[1 + q] = rr - k;
    }
    for (int c = 0; c < 4; ++c) x[c] = 0.0;
    for (int corner = 0; corner < 16; ++corner) {
        long node = 0;
        double w = 1.0;
        const long dims[4] = {(long)K * nd + 1, nx, nx, nx};
        for (int a = 0; a < 4; ++a) {
            int bit = (corner >> (3 - a)) & 1;
            node = node * dims[a] + ix[a] + bit;
            w *= bit ? t[a] : 1.0 - t[a];
        }
        const double *v = P->inv + 4 * node;
        if (!isfinite(v[0])) return -1;
        for (int c = 0; c < 4; ++c) x[c] += w * v[c];
    }
    return 0;
}

unsigned oc_eos_invert_ws(const oc_params *P, double s, const double *n, const double *guess, double *out,
                          int *used_table);

/* builds the inverted table: every node (s_i, x_j) inverted by the online root finder started
   cold (closed form, then table Newton); NaN where no solution exists */
void oc_inverse_build(const oc_params *P, double *inv)
{
    const int K = P->inv_K, nd = P->inv_nd, nx = P->inv_nx;
    const long ns = (long)K * nd + 1;
    const double dxr = 2.0 * P->inv_xmax / (nx - 1);
#pragma omp parallel for schedule(dynamic, 64)
    for (long node = 0; node < ns * nx * nx * nx; ++node) {
        long r = node;
        int jQ = (int)(r % nx);
        r /= nx;
        int jS = (int)(r % nx);
        r /= nx;
        int jB = (int)(r % nx);
        long i = r / nx;
        double s = P->inv_p10[i / K] * (1.0 + 9.0 * (double)(i % K) / K);
        double nq[3] = {(-P->inv_xmax + jB * dxr) * s, (-P->inv_xmax + jS * dxr) * s, (-P->inv_xmax + jQ * dxr) * s};
        double out[11];
        int used = 0;
        unsigned st = oc_eos_invert_ws(P, s, nq, NULL, out, &used);
        for (int c = 0; c < 4; ++c) inv[4 * node + c] = (st & ST_NOCONV) ? NAN : out[c];
    }
}

unsigned oc_eos_invert_ws(const oc_params *P, double s, const double *n, const double *guess, double *out,
                          int *used_table)
{
    unsigned st = 0;
    for (int k = 0; k < 11; ++k) out[k] = 0.0;
    if (used_table) *used_table = 0;
    if (!isfinite(s) || !isfinite(n[0]) || !isfinite(n[1]) || !isfinite(n[2])) return ST_NONFINITE | ST_NOCONV;
    double x[4];
    double p, H[16], sn[4];
    int use_table = 0;
    /* offline inverter: interpolate (T, mu) from the inverted table (no root finding) */
    if (P->inv && P->has_table && oc_inverse_lookup(P, s, n, x) == 0 && in_table(P, x)) use_table = 1;
    if (!use_table && P->has_table && guess && guess[0] > 0.0 && in_table(P, guess)) {
        double xt[4];
        memcpy(xt, guess, sizeof(xt));
        if (table_newton(P, s, n, xt) == 0) {
            memcpy(x, xt, sizeof(xt));
            use_table = 1;
        }
    }
    if (!use_table) {
        int r = oc_eos_invert_analytic(P, s, n, &x[0], &x[1]);
        if (r != 0 && P->backup && s > 0.0) {
            /* conformal diagonal: s = 4 A0 T^3, n_q = 4 A0 mu_q^3 / mu_q0^4; e = 3 p;
               p_s = dp/ds|_n = T/3, p_{n_q} = dp/dn_q|_s = mu_q/3 (T and mu_q decouple) */
            const double A0 = P->cd_A0;
            out[0] = cbrt(s / (4.0 * A0));
            double pq = 0.0;
            for (int q = 0; q < 3; ++q) {
                const double m0 = P->cd_mu0[q];
                out[1 + q] = cbrt(n[q] * m0 * m0 * m0 * m0 / (4.0 * A0));
                pq += pow(out[1 + q] / m0, 4.0);
            }
            out[4] = A0 * (pow(out[0], 4.0) + pq);
            out[5] = 3.0 * out[4];
            out[6] = out[0] / 3.0;
            for (int q = 0; q < 3; ++q) out[7 + q] = out[1 + q] / 3.0;
            out[10] = 1.0 / 3.0;
            return ST_BACKUP;
        }
        if (r != 0) return (unsigned)r | ST_NOCONV;
        if (P->has_table) {
            if (in_table(P, x)) {
                double xt[4];
                memcpy(xt, x, sizeof(xt));
                if (table_newton(P, s, n, xt) == 0) {
                    memcpy(x, xt, sizeof(xt));
                    use_table = 1;
                } else {
                    st |= ST_FALLBACK;
                }
            } else {
                st |= ST_OUT_OF_TABLE;
            }
        }
    }
    if (used_table) *used_table = use_table;
    if (use_table) {
        oc_eos_table(P, x, &p, sn, H);
    } else {
        oc_eos_analytic(P, x[0], &x[1], &p, sn, H);
    }
    double e = x[0] * s + x[1] * n[0] + x[2] * n[1] + x[3] * n[2] - p;
    /* (p_s, p_n) = H^{-T} (s, n): dp = s dT + n.dmu with (dT, dmu) = H^{-1} (ds, dn) */
    /* only the charge directions the EoS couples to take part (chi_q = 0 and no table:
       n_q = 0 identically and p_{n_q} = 0) */
    int act[4], m = 0;
    for (int k = 0; k < 4; ++k)
        if (k == 0 || use_table || P->chi[k - 1] > 0.0) act[m++] = k;
    double A[16], zr[4], z[4] = {0, 0, 0, 0}, tgt[4] = {s, n[0], n[1], n[2]};
    for (int i = 0; i < m; ++i) {
        zr[i] = tgt[act[i]];
        for (int j = 0; j < m; ++j) A[i * m + j] = H[act[j] * 4 + act[i]];
    }
    if (gauss_solve(m, A, zr) != 0) return st | ST_NOCONV;
    for (int i = 0; i < m; ++i) z[act[i]] = zr[i];
    double cs2 = (s * z[0] + n[0] * z[1] + n[1] * z[2] + n[2] * z[3]) / (e + p);
    if (cs2 > P->cs2_cap) {
        double f = P->cs2_cap / cs2;
        for (int k = 0; k < 4; ++k) z[k] *= f;
        cs2 = P->cs2_cap;
        st |= ST_CS2_CAPPED;
    }
    out[0] = x[0];
    out[1] = x[1];
    out[2] = x[2];
    out[3] = x[3];
    out[4] = p;
    out[5] = e;
    for (int k = 0; k < 4; ++k) out[6 + k] = z[k];
    out[10] = cs2;
    return st;
}

unsigned oc_eos_invert(const oc_params *P, double s, const double *n, double *out)
{
    return oc_eos_invert_ws(P, s, n, NULL, out, NULL);
}

/* ------------------------------------------------------------------------ */
/* geometry: diagonal metric, Christoffel symbols (Sec. "Notation")          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double g[4], gi[4], dg[4]; /* g_mu mu, g^mu mu, d g_mu mu / dx0 */
    double G[4][4][4];         /* Gamma^a_{bc} */
    double sqrtg;
} geom_t;

static void make_geom(int milne, double tau, geom_t *G)
{
    memset(G, 0, sizeof(*G));
    G->g[0] = 1.0;
    G->g[1] = G->g[2] = G->g[3] = -1.0;
    G->sqrtg = 1.0;
    if (milne) {
        G->g[3] = -tau * tau;
        G->dg[3] = -2.0 * tau;
        G->G[0][3][3] = tau;
        G->G[3][0][3] = 1.0 / tau;
        G->G[3][3][0] = 1.0 / tau;
        G->sqrtg = tau;
    }
    for (int m = 0; m < 4; ++m) G->gi[m] = 1.0 / G->g[m];
}

/* stored independent shear components, 4D index pairs (1 = x, 2 = y, 3 = eta|z) */
static int npi_of(int dim) { return dim == 2 ? 3 : 5; }
static const int PI2[3][2] = {{1, 1}, {1, 2}, {2, 2}};
static const int PI3[5][2] = {{1, 1}, {1, 2}, {1, 3}, {2, 2}, {2, 3}};

/* full contravariant pi^{mu nu} from the stored spatial components using
   transversality u_mu pi^{mu nu} = 0 and tracelessness g_mu nu pi^{mu nu} = 0 */
static void pi_full(int dim, const geom_t *G, const double *u, const double *stored, double pi[4][4])
{
    memset(pi, 0, sizeof(double) * 16);
    int np = npi_of(dim);
    for (int k = 0; k < np; ++k) {
        int i = dim == 2 ? PI2[k][0] : PI3[k][0], j = dim == 2 ? PI2[k][1] : PI3[k][1];
        pi[i][j] = pi[j][i] = stored[k];
    }
    double ul[4];
    for (int m = 0; m < 4; ++m) ul[m] = G->g[m] * u[m];
    /* pi^{33}: unknown in the trace; pi^{00} = sum_jk u_j u_k pi^{jk} / u_0^2 */
    double known = 0.0;
    for (int j = 1; j < 4; ++j)
        for (int k = 1; k < 4; ++k)
            if (!(j == 3 && k == 3)) known += ul[j] * ul[k] * pi[j][k];
    known /= ul[0] * ul[0];
    for (int i = 1; i < 3; ++i) known += G->g[i] * pi[i][i];
    double coef = ul[3] * ul[3] / (ul[0] * ul[0]) + G->g[3];
    pi[3][3] = -known / coef;
    for (int i = 1; i < 4; ++i) {
        double acc = 0.0;
        for (int j = 1; j < 4; ++j) acc += ul[j] * pi[j][i];
        pi[0][i] = pi[i][0] = -acc / ul[0];
    }
    double acc = 0.0;
    for (int j = 1; j < 4; ++j) acc += ul[j] * pi[j][0];
    pi[0][0] = -acc / ul[0];
}

/* ------------------------------------------------------------------------ */
/* source term I^nu of jet tracks (eq. conservation_source with I^nu != 0)   */
/* ------------------------------------------------------------------------ */
/* Each track moves at the speed of light from x0 along n from time t0 and deposits energy
   dE/dx per unit path length, spread over a normalised 3D Gaussian of width sigma around its
   current position, with the momentum of light moving along n:
     I^nu(t, x) = sum_k dEdx_k G_sigma(x - x0_k - n_k (t - t0_k)) (1, n_k)   for t >= t0_k.
   x has dim components (z = 0 in 2D); Cartesian coordinates, I^nu contravariant. */
static void jet_source(const oc_params *P, int dim, double t, const double *x, double *I)
{
    for (int mu = 0; mu < 4; ++mu) I[mu] = 0.0;
    const double sg = P->track_sigma;
    const double norm = 1.0 / (pow(2.0 * M_PI, 1.5) * sg * sg * sg);
    for (int k = 0; k < P->ntrack; ++k) {
        const double *tr = P->tracks + 8 * k;
        double dt = t - tr[6];
        if (dt < 0.0) continue;
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            double xd = d < dim ? x[d] : 0.0;
            double c = xd - (tr[d] + tr[3 + d] * dt);
            r2 += c * c;
        }
        double dep = tr[7] * norm * exp(-r2 / (2.0 * sg * sg));
        I[0] += dep;
        for (int d = 0; d < 3; ++d) I[1 + d] += dep * tr[3 + d];
    }
}

/* I^mu of the partons formed in (t - dt, t], smeared with the SPH kernel of width h_src in the
   event's dimensions (distances Euclidean in the event's spatial coordinates) */
static void parton_source(const oc_params *P, int dim, int milne, double t, const double *x, double *I, double *Iq)
{
    for (int mu = 0; mu < 4; ++mu) I[mu] = 0.0;
    for (int c = 0; c < 3; ++c) Iq[c] = 0.0;
    const double sqrtg = milne ? t : 1.0;
    for (int k = 0; k < P->nparton; ++k) {
        const double *q = P->partons + 8 * k;
        if (!(q[0] > t - P->parton_dt && q[0] <= t)) continue;
        double r2 = 0.0;
        for (int d = 0; d < dim; ++d) r2 += (x[d] - q[1 + d]) * (x[d] - q[1 + d]);
        const double f = P->parton_norm * oc_W(sqrt(r2), P->parton_h, dim) / (sqrtg * P->parton_dt);
        for (int mu = 0; mu < 4; ++mu) I[mu] += f * q[4 + mu];
        /* the charge source I_q: the parton's (B, S, Q) smeared with the same weight */
        if (P->parton_q)
            for (int c = 0; c < 3; ++c) Iq[c] += f * P->parton_q[3 * k + c];
    }
}

/* ------------------------------------------------------------------------ */
/* equations of motion at one particle                                       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int dim, viscous;
    double u[4];        /* contravariant, u[0] = u^0 */
    double dudx[4][4];  /* dudx[k][j] = d_k u^j (spatial k, j) */
    double s, n[3], sigma, T, mu[3], p, e, ps, pn[3];
    double Pi, Bv;
    double pi[4][4], Pv[4][4]; /* pi^{mu nu} and pi^{mu nu}/sigma */
    double eta, zeta, taupi, tauPi;
    double uI; /* u_nu I^nu: energy deposited in the local rest frame per unit time and volume */
    double dN[3]; /* d N_q / dx0 of the particle's charges (charge sources; else 0) */
    int model;      /* viscous equations of motion (oc_params.eom_model) */
    double cs2;     /* speed of sound squared (DNMR lambda_Pipi) */
    double dnmr[6]; /* DNMR coefficient ratios (oc_params.dnmr) */
    /* BSQ diffusion */
    int diff;
    double Jc[3][4];  /* J^mu_q, contravariant (J^0 from transversality) */
    double Jh[3][4];  /* J^i_q / sigma, the stored variables */
    double ga[3][4];  /* d_i alpha_q */
    double kap[3][3]; /* kappa_{qq'} */
    double tJ[3];     /* tau_q */
    double dNt[3];    /* rate of the lab charge from the flux divergence of the currents */
    double dal[3][4]; /* d alpha_q / d(s, n_B, n_S, n_Q) */
} ppart;

typedef struct {
    double dP[4];       /* d/dx0 of P^i = sqrt(-g) T^{0i} / sigma* */
    double dS, dBv;
    double dPv[4][4];
    double theta;
    double dJ[3][4];    /* d/dx0 of J^i_q / sigma */
    double dNl[3];      /* d/dx0 of the lab charges */
} prates;

/* The diffusion rates for a given D alpha_q (the comoving derivative of alpha_q = mu_q / T),
   at a trial acceleration: from eq. min_dif_rel, tau_q Delta^i_nu D J^nu_q + J^i_q =
   kappa_{qq'} nabla^<i> alpha_{q'} (the sign for the metric (+,-,-,-): the current runs down the
   gradient of mu/T, and the entropy production kappa (nabla alpha)^2 is non-negative), with
   Delta^i_nu D J^nu = D J^i + u^i J^nu Du_nu (u_nu J^nu = 0) and
   nabla^<i> alpha = g^{ii} d_i alpha - u^i D alpha:
     D J^i = (-J^i + kappa nabla^<i> alpha) / tau - u^i J^nu Du_nu,
     dJ^i/dx0 = (D J^i - u^mu Gamma^i_{mu lambda} J^lambda) / u^0,  d(J^i/sigma) = dJ^i/sigma - J^i dsigma/sigma^2;
   the rest-frame charge N_q = lab charge - Z_q with Z_q = J^0_q / (sigma u^0), so
   dN_q = dNt_q - dZ_q; the entropy rate gains -mu_q dN_q / T (eq. dsdnrewr); and D alpha_q
   implied by those rates, u^0 (alpha_{q,s} ds + alpha_{q,n} . dn) with s = sigma S and
   n = sigma N, is returned in Dal_out (the caller solves for its fixed point). */
static void diff_chain(const ppart *q, const geom_t *G, const double *a, double du0, const double *alow, double dsig,
                       double dS0, const double *Dal_in, double dJh[3][4], double *dNd, double *Dal_out)
{
    const double *u = q->u;
    const int dim = q->dim;
    double dN[3];
    for (int c = 0; c < 3; ++c) {
        double jDu = 0.0;
        for (int nu = 0; nu < 4; ++nu) jDu += q->Jc[c][nu] * alow[nu];
        double dZ = 0.0;
        for (int i = 1; i <= dim; ++i) {
            double src = 0.0; /* kappa_{qq'} nabla^<i> alpha_{q'} */
            for (int c2 = 0; c2 < 3; ++c2)
                src += q->kap[c][c2] * (G->gi[i] * q->ga[c2][i] - u[i] * Dal_in[c2]);
            const double DJ = (-q->Jc[c][i] + src) / q->tJ[c] - u[i] * jDu;
            double chr = 0.0;
            for (int m = 0; m < 4; ++m)
                for (int l = 0; l < 4; ++l) chr += u[m] * G->G[i][m][l] * q->Jc[c][l];
            const double dJ = (DJ - chr) / u[0];
            const double dj = dJ / q->sigma - q->Jc[c][i] * dsig / (q->sigma * q->sigma);
            if (dJh) dJh[c][i] = dj;
            dZ += -(G->dg[i] * u[i] * q->Jh[c][i] + G->g[i] * a[i] * q->Jh[c][i] + G->g[i] * u[i] * dj) / (u[0] * u[0]) +
                  2.0 * G->g[i] * u[i] * q->Jh[c][i] * du0 / (u[0] * u[0] * u[0]);
        }
        dN[c] = q->dNt[c] - dZ;
        if (dNd) dNd[c] = dN[c];
    }
    double dS = dS0;
    for (int c = 0; c < 3; ++c) dS -= q->mu[c] * dN[c] / q->T;
    const double ds = q->sigma * dS + (q->s / q->sigma) * dsig;
    double dn[3];
    for (int c = 0; c < 3; ++c) dn[c] = q->sigma * (q->dN[c] + dN[c]) + (q->n[c] / q->sigma) * dsig;
    for (int c = 0; c < 3; ++c) {
        double d = q->dal[c][0] * ds;
        for (int r = 0; r < 3; ++r) d += q->dal[c][1 + r] * dn[r];
        Dal_out[c] = u[0] * d;
    }
}

/* every rate as a function of a trial acceleration a^i = du^i/dx0 (linear in a) */
static void lhs_of(const ppart *q, const geom_t *G, const double *a, prates *R)
{
    const double *u = q->u;
    double u0 = u[0];
    double v[4] = {1.0, u[1] / u0, u[2] / u0, u[3] / u0};
    /* du^0/dx0 from u.u = 1 (paper's eq. unu) */
    double acc = 0.0;
    for (int i = 1; i < 4; ++i) acc += 2.0 * G->g[i] * u[i] * a[i] + u[i] * u[i] * G->dg[i];
    double du0 = -acc / (2.0 * u0);
    double dudt[4] = {du0, a[1], a[2], a[3]};
    /* partial derivatives d[mu][nu] = d_mu u^nu */
    double d[4][4];
    memset(d, 0, sizeof(d));
    for (int k = 1; k < 4; ++k) {
        double s0 = 0.0;
        for (int j = 1; j < 4; ++j) {
            d[k][j] = q->dudx[k][j];
            s0 += G->g[j] * u[j] * q->dudx[k][j];
        }
        d[k][0] = -s0 / u0;
    }
    for (int nu = 0; nu < 4; ++nu) {
        double conv = 0.0;
        for (int k = 1; k < 4; ++k) conv += v[k] * d[k][nu];
        d[0][nu] = dudt[nu] - conv;
    }
    double nab[4][4];
    for (int m = 0; m < 4; ++m)
        for (int nu = 0; nu < 4; ++nu) {
            double c = 0.0;
            for (int l = 0; l < 4; ++l) c += G->G[nu][m][l] * u[l];
            nab[m][nu] = d[m][nu] + c;
        }
    double theta = 0.0;
    for (int m = 0; m < 4; ++m) theta += nab[m][m];
    double Du[4];
    for (int nu = 0; nu < 4; ++nu) {
        double c = 0.0;
        for (int m = 0; m < 4; ++m) c += u[m] * nab[m][nu];
        Du[nu] = c;
    }
    double sig[4][4];
    for (int m = 0; m < 4; ++m)
        for (int nu = 0; nu < 4; ++nu) {
            double Delta = (m == nu ? G->gi[m] : 0.0) - u[m] * u[nu];
            sig[m][nu] = 0.5 * (G->gi[m] * nab[m][nu] + G->gi[nu] * nab[nu][m]) - 0.5 * (u[m] * Du[nu] + u[nu] * Du[m]) -
                         Delta * theta / 3.0;
        }
    R->theta = theta;
    double dsig = -q->sigma * theta / u0;
    memset(R->dPv, 0, sizeof(R->dPv));
    if (q->viscous) {
        double pisig = 0.0;
        for (int m = 0; m < 4; ++m)
            for (int nu = 0; nu < 4; ++nu) pisig += q->pi[m][nu] * G->g[m] * G->g[nu] * sig[m][nu];
        R->dS = (-q->Pi * theta + pisig + q->uI) / (u0 * q->sigma * q->T);
        if (q->model == 1) {
            /* DNMR bulk: tau_Pi D Pi + Pi = -zeta theta - delta_PiPi Pi theta + lambda_Pipi pi:sigma;
               the stored Pi/sigma obeys u^0 d(Pi/sigma)/dx^0 = (D Pi + Pi theta)/sigma (D sigma = -sigma theta) */
            double dPP = q->dnmr[0] * q->tauPi, lPp = q->dnmr[1] * q->tauPi * (1.0 / 3.0 - q->cs2);
            double DPi = (-q->Pi - q->zeta * theta - dPP * q->Pi * theta + lPp * pisig) / q->tauPi;
            R->dBv = (DPi + q->Pi * theta) / (u0 * q->sigma);
        } else {
            R->dBv = -(q->Pi + q->zeta * theta) / (q->tauPi * u0 * q->sigma);
        }
        /* DNMR shear: the symmetric, traceless, transverse parts of pi^mu_lambda sigma^{nu lambda}
           and pi^mu_lambda pi^{nu lambda}, with Delta^mu_alpha = delta^mu_alpha - u^mu u_alpha */
        double Ppis[4][4], Ppipi[4][4];
        memset(Ppis, 0, sizeof(Ppis));
        memset(Ppipi, 0, sizeof(Ppipi));
        if (q->model == 1) {
            double ulow[4], Dm[4][4], A[4][4], Bm[4][4], trA = 0.0, trB = 0.0;
            for (int al = 0; al < 4; ++al) ulow[al] = G->g[al] * u[al];
            for (int m = 0; m < 4; ++m)
                for (int al = 0; al < 4; ++al) Dm[m][al] = (m == al ? 1.0 : 0.0) - u[m] * ulow[al];
            for (int al = 0; al < 4; ++al)
                for (int be = 0; be < 4; ++be) {
                    double sa = 0.0, sb = 0.0;
                    for (int l = 0; l < 4; ++l) {
                        sa += q->pi[al][l] * G->g[l] * sig[be][l];
                        sb += q->pi[al][l] * G->g[l] * q->pi[be][l];
                    }
                    A[al][be] = sa;
                    Bm[al][be] = sb;
                }
            for (int al = 0; al < 4; ++al)
                for (int be = 0; be < 4; ++be) {
                    double Dl = (al == be ? G->g[al] : 0.0) - ulow[al] * ulow[be]; /* Delta_{alpha beta} */
                    trA += Dl * A[al][be];
                    trB += Dl * Bm[al][be];
                }
            for (int m = 0; m < 4; ++m)
                for (int nu = 0; nu < 4; ++nu) {
                    double pa = 0.0, pb = 0.0;
                    for (int al = 0; al < 4; ++al)
                        for (int be = 0; be < 4; ++be) {
                            double w2 = 0.5 * (Dm[m][al] * Dm[nu][be] + Dm[m][be] * Dm[nu][al]);
                            pa += w2 * A[al][be];
                            pb += w2 * Bm[al][be];
                        }
                    double Du_up = (m == nu ? G->gi[m] : 0.0) - u[m] * u[nu]; /* Delta^{mu nu} */
                    Ppis[m][nu] = pa - Du_up * trA / 3.0;
                    Ppipi[m][nu] = pb - Du_up * trB / 3.0;
                }
        }
        double alow[4];
        for (int al = 0; al < 4; ++al) alow[al] = G->g[al] * Du[al];
        for (int i = 1; i < 4; ++i)
            for (int j = 1; j < 4; ++j) {
                double chr = 0.0;
                for (int m = 0; m < 4; ++m)
                    for (int l = 0; l < 4; ++l) chr += u[m] * (G->G[i][m][l] * q->pi[l][j] + G->G[j][m][l] * q->pi[i][l]);
                double pja = 0.0, pia = 0.0;
                for (int al = 0; al < 4; ++al) {
                    pja += q->pi[j][al] * alow[al];
                    pia += q->pi[i][al] * alow[al];
                }
                double coup = u[i] * pja + u[j] * pia;
                double rhs;
                if (q->model == 1) {
                    /* tau_pi D pi + pi = 2 eta sigma - delta_pipi pi theta - tau_pipi <pi sigma>
                       + phi_7 <pi pi> + lambda_piPi Pi sigma */
                    double dpp = q->dnmr[2] * q->taupi, tpp = q->dnmr[3] * q->taupi;
                    double lpP = q->dnmr[4] * q->taupi, ph7 = q->dnmr[5] / q->p;
                    rhs = (-q->pi[i][j] + 2.0 * q->eta * sig[i][j] - dpp * q->pi[i][j] * theta - tpp * Ppis[i][j] +
                           ph7 * Ppipi[i][j] + lpP * q->Pi * sig[i][j]) /
                          q->taupi;
                } else {
                    rhs = (-q->pi[i][j] + 2.0 * q->eta * sig[i][j] - 4.0 / 3.0 * q->taupi * q->pi[i][j] * theta) / q->taupi;
                }
                double dpi = (rhs - chr - coup) / u0;
                R->dPv[i][j] = dpi / q->sigma - q->pi[i][j] * dsig / (q->sigma * q->sigma);
            }
    } else {
        R->dS = q->uI / (u0 * q->sigma * q->T);
        R->dBv = 0.0;
    }
    /* rest-frame charge rates: the charge sources', plus the diffusion currents' */
    double dNq[3] = {q->dN[0], q->dN[1], q->dN[2]};
    memset(R->dJ, 0, sizeof(R->dJ));
    for (int c = 0; c < 3; ++c) R->dNl[c] = q->dN[c];
    if (q->diff) {
        double alow_d[4];
        for (int al = 0; al < 4; ++al) alow_d[al] = G->g[al] * Du[al];
        /* the chain is affine in D alpha: its fixed point from the chain at 0 and the unit vectors */
        const double z3[3] = {0.0, 0.0, 0.0};
        double f0[3], Fm[9], rhs[3];
        diff_chain(q, G, a, du0, alow_d, dsig, R->dS, z3, NULL, NULL, f0);
        for (int k = 0; k < 3; ++k) {
            double e[3] = {0.0, 0.0, 0.0}, fk[3];
            e[k] = 1.0;
            diff_chain(q, G, a, du0, alow_d, dsig, R->dS, e, NULL, NULL, fk);
            for (int c = 0; c < 3; ++c) Fm[c * 3 + k] = (c == k ? 1.0 : 0.0) - (fk[c] - f0[c]);
        }
        for (int c = 0; c < 3; ++c) rhs[c] = f0[c];
        double Dal[3] = {0.0, 0.0, 0.0};
        if (gauss_solve(3, Fm, rhs) == 0)
            for (int c = 0; c < 3; ++c) Dal[c] = rhs[c];
        double dNd[3], Dchk[3];
        diff_chain(q, G, a, du0, alow_d, dsig, R->dS, Dal, R->dJ, dNd, Dchk);
        for (int c = 0; c < 3; ++c) {
            R->dS -= q->mu[c] * dNd[c] / q->T;
            dNq[c] += dNd[c];
            R->dNl[c] += q->dNt[c];
        }
    }
    double ds = q->sigma * R->dS + (q->s / q->sigma) * dsig;
    double dPi = q->sigma * R->dBv + q->Bv * dsig;
    double dw = (q->T + q->ps) * ds + dPi;
    /* dn_q = N_q dsigma + sigma dN_q with N_q = n_q / sigma (dN_q != 0 under charge sources and
       diffusion) */
    for (int c = 0; c < 3; ++c) dw += (q->mu[c] + q->pn[c]) * ((q->n[c] / q->sigma) * dsig + q->sigma * dNq[c]);
    double w = q->e + q->p + q->Pi;
    for (int i = 1; i < 4; ++i) {
        double t1 = 0.0, t2 = 0.0;
        for (int j = 1; j < 4; ++j) {
            t1 += G->dg[j] * u[j] * q->Pv[j][i] + G->g[j] * a[j] * q->Pv[j][i] + G->g[j] * u[j] * R->dPv[j][i];
            t2 += G->g[j] * u[j] * q->Pv[j][i];
        }
        double dpi0 = -t1 / (u0 * u0) + 2.0 * t2 * du0 / (u0 * u0 * u0);
        R->dP[i] = (u[i] / q->sigma) * dw + (w / q->sigma) * a[i] - (w * u[i] / (q->sigma * q->sigma)) * dsig + dpi0;
    }
}

/* ------------------------------------------------------------------------ */
/* one stage: neighbours, densities, EoS, gradients, rates                   */
/* ------------------------------------------------------------------------ */
static int nv_of(int dim) { return 2 * dim + 2 + npi_of(dim); }
/* state rows: the diffusion currents J^i_q / sigma follow the shear rows */
static int nvp_of(const oc_params *P) { return nv_of(P->dim) + (P->diffusion ? 3 * P->dim : 0); }
static int jrow(const oc_params *P, int q, int i) { return nv_of(P->dim) + q * P->dim + i; }

/* J^0 of a transverse current from its spatial components: u_mu J^mu = 0 with g_00 = 1 */
static double j0_of(const geom_t *G, int dim, const double *u, const double *J)
{
    double acc = 0.0;
    for (int i = 1; i <= dim; ++i) acc += G->g[i] * u[i] * J[i];
    return -acc / u[0];
}

/* y layout [nv][n]: x^1..x^dim, u^1..u^dim, S, Pi/sigma, pi^{ij}/sigma (stored comps)
   aux layout [NAUX][n]: sigma*, s, nB, nS, nQ, T, muB, muS, muQ, p, e, cs2, theta, Pi,
                         u0, neighbour count, sigma, status
   grad layout [dim*dim + dim][n]: d_k u^j (k major), F^i                              */
static void densities_eos(const oc_params *P, long n, double tau, const double *y, const double *Nq, grid_t *g,
                          double *aux, unsigned *status, const double *guess_in, double *guess_out)
{
    int dim = P->dim;
    double two_h = 2.0 * P->h;
    double supp2 = two_h * two_h;
    geom_t G;
    make_geom(P->milne, tau, &G);
#pragma omp parallel
    {
        long *buf = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 64)
        for (long a = 0; a < n; ++a) {
            long m = grid_neighbors(g, y, supp2, a, buf);
            double sig = 0.0, ss = 0.0, nn[3] = {0, 0, 0};
            for (long k = 0; k < m; ++k) {
                long b = buf[k];
                double r = sqrt(r2_of(dim, y, n, a, b));
                double W = oc_W(r, P->h, dim);
                sig += W;
                ss += y[(2 * dim) * n + b] * W;
                for (int c = 0; c < 3; ++c) nn[c] += Nq[c * n + b] * W;
            }
            double uu = 0.0;
            for (int i = 0; i < dim; ++i) {
                double ui = y[(dim + i) * n + a];
                uu += -G.g[1 + i] * ui * ui;
            }
            double u0 = sqrt(1.0 + uu);
            double vol = u0 * G.sqrtg;
            aux[0 * n + a] = sig;
            aux[1 * n + a] = ss / vol;
            for (int c = 0; c < 3; ++c) aux[(2 + c) * n + a] = nn[c] / vol;
            if (P->diffusion) {
                /* the kernel sum of the lab charges is the lab density sqrt(-g) N^0 = sqrt(-g)
                   (n u^0 + J^0): the rest-frame n_q = (sum / sqrt(-g) - J^0_q) / u^0 */
                double u[4] = {u0, 0, 0, 0}, J[4] = {0, 0, 0, 0};
                for (int i = 0; i < dim; ++i) u[1 + i] = y[(dim + i) * n + a];
                for (int c = 0; c < 3; ++c) {
                    for (int i = 0; i < dim; ++i) J[1 + i] = (sig / vol) * y[jrow(P, c, i) * n + a];
                    aux[(2 + c) * n + a] = (nn[c] / G.sqrtg - j0_of(&G, dim, u, J)) / u0;
                }
            }
            aux[14 * n + a] = u0;
            aux[15 * n + a] = (double)m;
            aux[16 * n + a] = sig / vol;
            double out[11];
            double nr[3] = {aux[2 * n + a], aux[3 * n + a], aux[4 * n + a]};
            double gs[4] = {0, 0, 0, 0};
            if (guess_in)
                for (int k = 0; k < 4; ++k) gs[k] = guess_in[k * n + a];
            int used = 0;
            unsigned st = oc_eos_invert_ws(P, aux[1 * n + a], nr, gs, out, &used);
            if (guess_out)
                for (int k = 0; k < 4; ++k) guess_out[k * n + a] = used ? out[k] : 0.0;
            for (int k = 0; k < 4; ++k) aux[(5 + k) * n + a] = out[k];
            aux[9 * n + a] = out[4];
            aux[10 * n + a] = out[5];
            aux[11 * n + a] = out[10];
            status[a] = st;
            aux[17 * n + a] = (double)st;
        }
        free(buf);
    }
}

/* EoS derivative outputs are kept aside for the rates */
typedef struct {
    double ps, pn[3], cs2;
} eosder_t;

/* d alpha_q / d(s, n_B, n_S, n_Q), alpha_q = mu_q / T, at an inversion's solution x = (T, mu):
   (dT, dmu) = H^-1 (ds, dn) with H = d(s, n)/d(T, mu) of the EoS that produced it (the table,
   the closed form, or the conformal-diagonal backup); charge directions the closed form does
   not couple (chi_q = 0, no table) get zero derivatives.  Returns -1 for a singular H. */
static int dalpha_of(const oc_params *P, const double *x, int used_table, unsigned st, double dal[3][4])
{
    double H[16], p, sn[4];
    memset(dal, 0, sizeof(double) * 12);
    if (st & ST_BACKUP) {
        memset(H, 0, sizeof(H));
        H[0] = 12.0 * P->cd_A0 * x[0] * x[0];
        for (int q = 0; q < 3; ++q) {
            const double m0 = P->cd_mu0[q];
            H[(1 + q) * 4 + 1 + q] = 12.0 * P->cd_A0 * x[1 + q] * x[1 + q] / (m0 * m0 * m0 * m0);
        }
    } else if (used_table) {
        oc_eos_table(P, x, &p, sn, H);
    } else {
        oc_eos_analytic(P, x[0], &x[1], &p, sn, H);
    }
    int act[4], m = 0;
    for (int k = 0; k < 4; ++k)
        if (k == 0 || used_table || (st & ST_BACKUP) || P->chi[k - 1] > 0.0) act[m++] = k;
    double Hi[16];
    memset(Hi, 0, sizeof(Hi));
    for (int f = 0; f < m; ++f) { /* column f of the inverse over the active directions */
        double A[16], b[4];
        for (int i = 0; i < m; ++i) {
            b[i] = i == f ? 1.0 : 0.0;
            for (int j = 0; j < m; ++j) A[i * m + j] = H[act[i] * 4 + act[j]];
        }
        if (gauss_solve(m, A, b) != 0) return -1;
        for (int i = 0; i < m; ++i) Hi[act[i] * 4 + act[f]] = b[i];
    }
    for (int q = 0; q < 3; ++q)
        for (int f = 0; f < 4; ++f) dal[q][f] = (Hi[(1 + q) * 4 + f] - (x[1 + q] / x[0]) * Hi[0 * 4 + f]) / x[0];
    return 0;
}

int oc_stage(const oc_params *P, long n, double tau, const double *y, const double *Nq, double *dydt, double *aux,
             double *grad, unsigned *status, double *work_rate, const double *guess_in, double *guess_out,
             double *dNq)
{
    int dim = P->dim, np = npi_of(dim), nv = nvp_of(P);
    double two_h = 2.0 * P->h;
    double supp2 = two_h * two_h;
    geom_t G;
    make_geom(P->milne, tau, &G);
    grid_t g;
    grid_build(&g, n, dim, y, P->h);
    densities_eos(P, n, tau, y, Nq, &g, aux, status, guess_in, guess_out);
    /* diffusion: per particle alpha_q, d alpha_q / d(s, n), J^mu_q, and the flux
       (J^k - v^k J^0) / sigma*^2 of the lab charge; per particle from the gradient pass
       d_k alpha_q and the flux divergence */
    const size_t nz = (size_t)(n > 0 ? n : 1);
    double *alph = P->diffusion ? (double *)calloc(3 * nz, sizeof(double)) : NULL;
    double *dalp = P->diffusion ? (double *)calloc(12 * nz, sizeof(double)) : NULL;
    double *Jmu = P->diffusion ? (double *)calloc(12 * nz, sizeof(double)) : NULL;
    double *Fls = P->diffusion ? (double *)calloc(9 * nz, sizeof(double)) : NULL;
    double *galp = P->diffusion ? (double *)calloc(9 * nz, sizeof(double)) : NULL;
    double *dNt = P->diffusion ? (double *)calloc(3 * nz, sizeof(double)) : NULL;

    /* EoS derivatives again (kept out of aux), transport, full pi, X^{ji}/sigma*^2 */
    eosder_t *ed = (eosder_t *)malloc(sizeof(eosder_t) * (size_t)(n > 0 ? n : 1));
    double *Xs = (double *)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
    double *us = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *pif = (double *)malloc(sizeof(double) * 16 * (size_t)(n > 0 ? n : 1));
    double *Tfull = (double *)malloc(sizeof(double) * 16 * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
    for (long a = 0; a < n; ++a) {
        double out[11];
        double nr[3] = {aux[2 * n + a], aux[3 * n + a], aux[4 * n + a]};
        double gs[4] = {0, 0, 0, 0};
        if (guess_in)
            for (int k = 0; k < 4; ++k) gs[k] = guess_in[k * n + a];
        int used = 0;
        unsigned est = oc_eos_invert_ws(P, aux[1 * n + a], nr, gs, out, &used);
        if (P->diffusion) {
            double dal[3][4];
            if (!(est & (ST_NOCONV | ST_NONFINITE)) && out[0] > 0.0 && dalpha_of(P, out, used, est, dal) == 0)
                memcpy(&dalp[12 * a], dal, sizeof(dal));
            for (int c = 0; c < 3; ++c) alph[3 * a + c] = out[0] > 0.0 ? out[1 + c] / out[0] : 0.0;
        }
        ed[a].ps = out[6];
        for (int c = 0; c < 3; ++c) ed[a].pn[c] = out[7 + c];
        ed[a].cs2 = out[10];
        double u[4] = {aux[14 * n + a], 0, 0, 0};
        for (int i = 0; i < dim; ++i) u[1 + i] = y[(dim + i) * n + a];
        double sigma = aux[16 * n + a];
        double Pi = P->viscous ? sigma * y[(2 * dim + 1) * n + a] : 0.0;
        double st[5] = {0, 0, 0, 0, 0};
        if (P->viscous)
            for (int k = 0; k < np; ++k) st[k] = sigma * y[(2 * dim + 2 + k) * n + a];
        double pi[4][4];
        pi_full(dim, &G, u, st, pi);
        memcpy(&pif[16 * a], pi, sizeof(pi));
        aux[13 * n + a] = Pi;
        double p = aux[9 * n + a], e = aux[10 * n + a];
        double sstar = aux[0 * n + a];
        for (int j = 0; j < 3; ++j)
            for (int i = 0; i < 3; ++i) {
                double X = -(p + Pi) * (j == i ? G.gi[1 + j] : 0.0) + pi[1 + j][1 + i] - (u[1 + j] / u[0]) * pi[0][1 + i];
                Xs[9 * a + 3 * j + i] = X / (sstar * sstar);
            }
        for (int j = 0; j < 3; ++j) us[3 * a + j] = u[1 + j] / sstar;
        if (P->diffusion)
            for (int c = 0; c < 3; ++c) {
                double J[4] = {0, 0, 0, 0};
                for (int i = 0; i < dim; ++i) J[1 + i] = sigma * y[jrow(P, c, i) * n + a];
                J[0] = j0_of(&G, dim, u, J);
                for (int m = 0; m < 4; ++m) Jmu[12 * a + 4 * c + m] = J[m];
                for (int k = 0; k < 3; ++k) Fls[9 * a + 3 * c + k] = (J[1 + k] - (u[1 + k] / u[0]) * J[0]) / (sstar * sstar);
            }
        for (int m = 0; m < 4; ++m)
            for (int l = 0; l < 4; ++l) {
                double Delta = (m == l ? G.gi[m] : 0.0) - u[m] * u[l];
                Tfull[16 * a + 4 * m + l] = e * u[m] * u[l] - (p + Pi) * Delta + pi[m][l];
            }
    }

    /* gradients */
#pragma omp parallel
    {
        long *buf = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 64)
        for (long a = 0; a < n; ++a) {
            long m = grid_neighbors(&g, y, supp2, a, buf);
            double du[3][3], F[3], ga[3][3], dv[3];
            memset(du, 0, sizeof(du));
            memset(F, 0, sizeof(F));
            memset(ga, 0, sizeof(ga));
            memset(dv, 0, sizeof(dv));
            for (long k = 0; k < m; ++k) {
                long b = buf[k];
                double r2 = r2_of(dim, y, n, a, b);
                if (r2 == 0.0) continue; /* grad W = 0 at r = 0 */
                double r = sqrt(r2);
                double dWdr = oc_dWdr(r, P->h, dim);
                double gw[3] = {0, 0, 0};
                for (int d = 0; d < dim; ++d) gw[d] = dWdr * (y[d * n + a] - y[d * n + b]) / r;
                for (int kk = 0; kk < dim; ++kk)
                    for (int j = 0; j < dim; ++j) du[kk][j] += us[3 * b + j] * gw[kk];
                for (int i = 0; i < dim; ++i)
                    for (int j = 0; j < dim; ++j) F[i] += (Xs[9 * a + 3 * j + i] + Xs[9 * b + 3 * j + i]) * gw[j];
                if (P->diffusion)
                    for (int c = 0; c < 3; ++c) {
                        /* d_k alpha: the difference form (the general SPH derivative with n = 1,
                           zero for a uniform alpha); the flux divergence: the n = -1 form */
                        const double da = alph[3 * b + c] - alph[3 * a + c];
                        for (int kk = 0; kk < dim; ++kk) {
                            ga[c][kk] += da * gw[kk];
                            dv[c] += (Fls[9 * a + 3 * c + kk] + Fls[9 * b + 3 * c + kk]) * gw[kk];
                        }
                    }
            }
            if (P->diffusion)
                for (int c = 0; c < 3; ++c) {
                    for (int kk = 0; kk < dim; ++kk) galp[9 * a + 3 * c + kk] = ga[c][kk] / aux[0 * n + a];
                    dNt[3 * a + c] = -G.sqrtg * dv[c];
                }
            for (int kk = 0; kk < dim; ++kk)
                for (int j = 0; j < dim; ++j) grad[(kk * dim + j) * n + a] = du[kk][j];
            for (int i = 0; i < dim; ++i) grad[(dim * dim + i) * n + a] = -G.sqrtg * F[i];
        }
        free(buf);
    }

    /* equations of motion */
#pragma omp parallel for schedule(static)
    for (long a = 0; a < n; ++a) {
        if (dNq)
            for (int c = 0; c < 3; ++c) dNq[c * n + a] = 0.0;
        if ((status[a] & (ST_NOCONV | ST_NONFINITE)) ||
            (P->T_stop_GeV > 0.0 && aux[5 * n + a] * HBARC < P->T_stop_GeV)) {
            /* no EoS solution, or below the stop temperature: the particle is frozen for this
               stage, moving ballistically (its charges too stay as they are) */
            double u0 = aux[14 * n + a];
            for (int k = 0; k < nv; ++k) dydt[k * n + a] = 0.0;
            for (int i = 0; i < dim; ++i) dydt[i * n + a] = y[(dim + i) * n + a] / u0;
            continue;
        }
        ppart q;
        memset(&q, 0, sizeof(q));
        q.dim = dim;
        q.viscous = P->viscous;
        q.u[0] = aux[14 * n + a];
        for (int i = 0; i < dim; ++i) q.u[1 + i] = y[(dim + i) * n + a];
        for (int k = 0; k < dim; ++k)
            for (int j = 0; j < dim; ++j) q.dudx[1 + k][1 + j] = grad[(k * dim + j) * n + a];
        q.s = aux[1 * n + a];
        for (int c = 0; c < 3; ++c) q.n[c] = aux[(2 + c) * n + a];
        q.sigma = aux[16 * n + a];
        q.T = aux[5 * n + a];
        for (int c = 0; c < 3; ++c) q.mu[c] = aux[(6 + c) * n + a];
        q.p = aux[9 * n + a];
        q.e = aux[10 * n + a];
        q.ps = ed[a].ps;
        for (int c = 0; c < 3; ++c) q.pn[c] = ed[a].pn[c];
        q.cs2 = ed[a].cs2;
        q.model = P->eom_model;
        for (int k = 0; k < 6; ++k) q.dnmr[k] = P->dnmr[k];
        q.Pi = aux[13 * n + a];
        q.Bv = P->viscous ? y[(2 * dim + 1) * n + a] : 0.0;
        memcpy(q.pi, &pif[16 * a], sizeof(q.pi));
        for (int m = 0; m < 4; ++m)
            for (int l = 0; l < 4; ++l) q.Pv[m][l] = q.pi[m][l] / q.sigma;
        if (P->viscous) {
            q.eta = P->eta_over_s * q.s;
            double dTg = q.T * HBARC - P->zeta_T_GeV;
            q.zeta = P->zeta_peak * exp(-dTg * dTg / (2.0 * P->zeta_w_GeV * P->zeta_w_GeV)) * q.s;
            q.taupi = P->tau_pi_coef * q.eta / (q.e + q.p);
            q.tauPi = P->tau_Pi_ratio * q.taupi;
        }
        /* F^i: minus the SPH stress divergence, plus the Christoffel source */
        double F[4] = {0, 0, 0, 0};
        for (int i = 0; i < dim; ++i) {
            double src = 0.0;
            for (int m = 0; m < 4; ++m)
                for (int l = 0; l < 4; ++l) src += G.G[1 + i][m][l] * Tfull[16 * a + 4 * m + l];
            F[1 + i] = grad[(dim * dim + i) * n + a] - G.sqrtg * src / aux[0 * n + a];
        }
        /* jet and parton sources: dP^i/dx0 gains sqrt(-g) I^i / sigma*, dS/dx0 gains
           u_nu I^nu / (u^0 sigma T); parton charges: dN_q/dx0 = sqrt(-g) I_q / sigma* (the lab
           charge of the particle's volume 1/sigma*), and dS/dx0 gains R^S_q dN_q/dx0 with
           R^S_q = -mu_q / T (eq. dsdnrewr), i.e. -mu_q I_q / (u^0 sigma T) */
        if (P->ntrack > 0 || P->nparton > 0) {
            double xa[3] = {0, 0, 0}, I[4] = {0, 0, 0, 0}, Ik[4], Iq[3] = {0, 0, 0};
            for (int d = 0; d < dim; ++d) xa[d] = y[d * n + a];
            if (P->ntrack > 0) {
                jet_source(P, dim, tau, xa, Ik);
                for (int mu = 0; mu < 4; ++mu) I[mu] += Ik[mu];
            }
            if (P->nparton > 0) {
                parton_source(P, dim, P->milne, tau, xa, Ik, Iq);
                for (int mu = 0; mu < 4; ++mu) I[mu] += Ik[mu];
            }
            for (int i = 0; i < dim; ++i) F[1 + i] += G.sqrtg * I[1 + i] / aux[0 * n + a];
            for (int mu = 0; mu < 4; ++mu) q.uI += G.g[mu] * q.u[mu] * I[mu];
            if (P->parton_q) {
                for (int c = 0; c < 3; ++c) q.uI -= q.mu[c] * Iq[c];
                for (int c = 0; c < 3; ++c) q.dN[c] = G.sqrtg * Iq[c] / aux[0 * n + a];
                if (dNq)
                    for (int c = 0; c < 3; ++c) dNq[c * n + a] = q.dN[c];
            }
        }
        if (P->diffusion) {
            q.diff = 1;
            const double T = q.T;
            for (int c = 0; c < 3; ++c) {
                for (int m = 0; m < 4; ++m) q.Jc[c][m] = Jmu[12 * a + 4 * c + m];
                for (int i = 0; i < dim; ++i) {
                    q.Jh[c][1 + i] = y[jrow(P, c, i) * n + a];
                    q.ga[c][1 + i] = galp[9 * a + 3 * c + i];
                }
                for (int c2 = 0; c2 < 3; ++c2) q.kap[c][c2] = P->kappaT2[3 * c + c2] * T * T;
                q.tJ[c] = P->tauJT[c] / T;
                q.dNt[c] = dNt[3 * a + c];
                for (int f = 0; f < 4; ++f) q.dal[c][f] = dalp[12 * a + 4 * c + f];
            }
        }
        /* M_ij = dP^i(e_j) - dP^i(0), c^i = dP^i(0); solve M a = F - c */
        double zero[4] = {0, 0, 0, 0};
        prates R0;
        lhs_of(&q, &G, zero, &R0);
        double M[9], rhs[3];
        for (int j = 0; j < dim; ++j) {
            double ej[4] = {0, 0, 0, 0};
            ej[1 + j] = 1.0;
            prates Rj;
            lhs_of(&q, &G, ej, &Rj);
            for (int i = 0; i < dim; ++i) M[i * dim + j] = Rj.dP[1 + i] - R0.dP[1 + i];
        }
        for (int i = 0; i < dim; ++i) rhs[i] = F[1 + i] - R0.dP[1 + i];
        double acc4[4] = {0, 0, 0, 0};
        if (gauss_solve(dim, M, rhs) == 0) {
            for (int i = 0; i < dim; ++i) acc4[1 + i] = rhs[i];
        } else {
            status[a] |= ST_SOLVE_FAIL;
            aux[17 * n + a] = (double)status[a];
        }
        prates R;
        lhs_of(&q, &G, acc4, &R);
        aux[12 * n + a] = R.theta;
        for (int i = 0; i < dim; ++i) dydt[i * n + a] = q.u[1 + i] / q.u[0];
        for (int i = 0; i < dim; ++i) dydt[(dim + i) * n + a] = acc4[1 + i];
        dydt[(2 * dim) * n + a] = R.dS;
        dydt[(2 * dim + 1) * n + a] = P->viscous ? R.dBv : 0.0;
        for (int k = 0; k < np; ++k) {
            int i = dim == 2 ? PI2[k][0] : PI3[k][0], j = dim == 2 ? PI2[k][1] : PI3[k][1];
            dydt[(2 * dim + 2 + k) * n + a] = P->viscous ? R.dPv[i][j] : 0.0;
        }
        if (P->diffusion) {
            for (int c = 0; c < 3; ++c)
                for (int i = 0; i < dim; ++i) dydt[jrow(P, c, i) * n + a] = R.dJ[c][1 + i];
            if (dNq)
                for (int c = 0; c < 3; ++c) dNq[c * n + a] = R.dNl[c];
        }
    }
    /* longitudinal work rate: sum_a sqrt(-g) Gamma^0_{mu nu} T^{mu nu} / sigma* (serial, fixed order) */
    double wr = 0.0;
    for (long a = 0; a < n; ++a) {
        double src = 0.0;
        for (int m = 0; m < 4; ++m)
            for (int l = 0; l < 4; ++l) src += G.G[0][m][l] * Tfull[16 * a + 4 * m + l];
        wr += G.sqrtg * src / aux[0 * n + a];
    }
    *work_rate = wr;
    free(ed);
    free(Xs);
    free(us);
    free(pif);
    free(Tfull);
    free(alph);
    free(dalp);
    free(Jmu);
    free(Fls);
    free(galp);
    free(dNt);
    grid_free(&g);
    return 0;
}

/* densities and EoS only, at the current state (for read-out) */
void oc_observe(const oc_params *P, long n, double tau, const double *y, const double *Nq, double *aux, unsigned *status,
                const double *guess)
{
    grid_t g;
    grid_build(&g, n, P->dim, y, P->h);
    densities_eos(P, n, tau, y, Nq, &g, aux, status, guess, NULL);
    for (long a = 0; a < n; ++a) aux[13 * n + a] = P->viscous ? aux[16 * n + a] * y[(2 * P->dim + 1) * n + a] : 0.0;
    grid_free(&g);
}

/* Heun: y1 = y0 + dt f(t, y0); y = ((y0 + y1) + dt f(t + dt, y1)) / 2.
   work accumulates the longitudinal work integral with the same quadrature. */
int oc_heun(const oc_params *P, long n, double *tau, double dtau, int nsteps, double *y, double *Nq, double *aux,
            double *grad, unsigned *status, unsigned *status_or, double *work, double *guess)
{
    int nv = nvp_of(P);
    size_t sz = sizeof(double) * (size_t)nv * (size_t)(n > 0 ? n : 1);
    double *k = (double *)malloc(sz);
    double *y1 = (double *)malloc(sz);
    double *g1 = (double *)calloc((size_t)4 * (size_t)(n > 0 ? n : 1), sizeof(double));
    /* charges change only under charge sources or diffusion; then they take the same Heun steps */
    const int charged = (P->parton_q != NULL && P->nparton > 0) || P->diffusion;
    size_t szq = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
    double *kq = charged ? (double *)malloc(szq) : NULL;
    double *Nq1 = charged ? (double *)malloc(szq) : NULL;
    unsigned acc = 0;
    for (int step = 0; step < nsteps; ++step) {
        double wr0, wr1;
        oc_stage(P, n, *tau, y, Nq, k, aux, grad, status, &wr0, guess, g1, kq);
        for (long a = 0; a < n; ++a) acc |= status[a];
        for (long i = 0; i < (long)nv * n; ++i) y1[i] = y[i] + dtau * k[i];
        if (charged)
            for (long i = 0; i < 3 * n; ++i) Nq1[i] = Nq[i] + dtau * kq[i];
        oc_stage(P, n, *tau + dtau, y1, charged ? Nq1 : Nq, k, aux, grad, status, &wr1, g1, guess, kq);
        for (long a = 0; a < n; ++a) acc |= status[a];
        for (long i = 0; i < (long)nv * n; ++i) y[i] = 0.5 * ((y[i] + y1[i]) + dtau * k[i]);
        if (charged)
            for (long i = 0; i < 3 * n; ++i) Nq[i] = 0.5 * ((Nq[i] + Nq1[i]) + dtau * kq[i]);
        *work += 0.5 * dtau * (wr0 + wr1);
        *tau = *tau + dtau;
    }
    *status_or = acc;
    free(k);
    free(y1);
    free(g1);
    free(kq);
    free(Nq1);
    return 0;
}

/* totals at the current state: [0] E = sum sqrt(-g) T^{00}/sigma*, [1] sum S, [2..4] sum N_q
   (serial sums in particle order); needs aux from oc_observe */
void oc_totals(const oc_params *P, long n, double tau, const double *y, const double *Nq, const double *aux, double *tot)
{
    int dim = P->dim, np = npi_of(dim);
    geom_t G;
    make_geom(P->milne, tau, &G);
    double E = 0.0, S = 0.0, N[3] = {0, 0, 0};
    for (long a = 0; a < n; ++a) {
        double u[4] = {aux[14 * n + a], 0, 0, 0};
        for (int i = 0; i < dim; ++i) u[1 + i] = y[(dim + i) * n + a];
        double sigma = aux[16 * n + a];
        double st[5] = {0, 0, 0, 0, 0};
        if (P->viscous)
            for (int k = 0; k < np; ++k) st[k] = sigma * y[(2 * dim + 2 + k) * n + a];
        double pi[4][4];
        pi_full(dim, &G, u, st, pi);
        double Pi = aux[13 * n + a];
        double p = aux[9 * n + a], e = aux[10 * n + a];
        double T00 = (e + p + Pi) * u[0] * u[0] - (p + Pi) * G.gi[0] + pi[0][0];
        E += G.sqrtg * T00 / aux[0 * n + a];
        S += y[(2 * dim) * n + a];
        for (int c = 0; c < 3; ++c) N[c] += Nq[c * n + a];
    }
    tot[0] = E;
    tot[1] = S;
    for (int c = 0; c < 3; ++c) tot[2 + c] = N[c];
}

/* the stored-shear index pairs, for the Python side */
int oc_pi_pairs(int dim, int *ij)
{
    int np = npi_of(dim);
    for (int k = 0; k < np; ++k) {
        ij[2 * k] = dim == 2 ? PI2[k][0] : PI3[k][0];
        ij[2 * k + 1] = dim == 2 ? PI2[k][1] : PI3[k][1];
    }
    return np;
}

/* full pi^{mu nu} reconstruction, exported for tests (transversality, trace) */
void oc_pi_full(int dim, int milne, double tau, const double *u4, const double *stored, double *out16)
{
    geom_t G;
    make_geom(milne, tau, &G);
    double pi[4][4];
    pi_full(dim, &G, u4, stored, pi);
    memcpy(out16, pi, sizeof(pi));
}

/* ------------------------------------------------------------------------ */
/* Freeze-out hypersurface (Sec. "Freeze-out hypersurface construction")      */
/* Elements of the surface of constant energy density e_fo.  aux: oc_observe at the current
   state (time tau); eprev[n]: each particle's e at the previous observation, tau - dtau
   (NaN: none).  A particle whose e fell through e_fo (eprev > e_fo >= e) yields one
   element, evaluated at the current state (the end of the step in which it crossed):
     d_i e_a = sum_b (e_b / sigma*_b) d_i W_ab        (SPH derivative, n = 0 form),
     d_tau e = (e - eprev) / dtau - v^i d_i e          (the particle's rate minus advection),
     N_mu = -d_mu e, n_mu = N_mu / sqrt(|N_mu N^mu|)   (covariant, "outward"),
     |dsigma| = m / (sigma |u^mu n_mu|)                 (m = 1, sigma the rest-frame density),
     dsigma_mu = |dsigma| n_mu.
   Record of FO_NREC doubles: tau, x^1..3, u^0..3, T, mu_B, mu_S, mu_Q, e, p, s, n_0..3,
   |dsigma|, dsigma_0..3 (the third spatial entries are 0 in 2+1D).  Particles in index
   order; at most cap records are written; the number of crossings is returned. */
#define FO_NREC 24
long oc_freezeout(const oc_params *P, long n, double tau, double dtau, const double *y, const double *aux,
                  const double *eprev, double e_fo, long cap, double *out, long *ids)
{
    int dim = P->dim;
    geom_t G;
    make_geom(P->milne, tau, &G);
    grid_t g;
    grid_build(&g, n, dim, y, P->h);
    long *buf = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    double supp2 = 4.0 * P->h * P->h;
    long cnt = 0;
    for (long a = 0; a < n; ++a) {
        double e = aux[10 * n + a];
        if (!(eprev[a] > e_fo && e <= e_fo)) continue;
        /* spatial gradient of e */
        double de[3] = {0.0, 0.0, 0.0};
        long m = grid_neighbors(&g, y, supp2, a, buf);
        for (long k = 0; k < m; ++k) {
            long b = buf[k];
            double r2 = r2_of(dim, y, n, a, b);
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            double dWdr = oc_dWdr(r, P->h, dim);
            double eb = aux[10 * n + b] / aux[0 * n + b];
            for (int d = 0; d < dim; ++d) de[d] += eb * dWdr * (y[d * n + a] - y[d * n + b]) / r;
        }
        /* four-velocity, particle rate, covariant normal */
        double u[4] = {aux[14 * n + a], 0.0, 0.0, 0.0};
        for (int i = 0; i < dim; ++i) u[1 + i] = y[(dim + i) * n + a];
        double adv = 0.0;
        for (int i = 0; i < dim; ++i) adv += (u[1 + i] / u[0]) * de[i];
        double N[4] = {-((e - eprev[a]) / dtau - adv), 0.0, 0.0, 0.0};
        for (int i = 0; i < dim; ++i) N[1 + i] = -de[i];
        double NN = 0.0; /* N_mu N^mu = g^{mu mu} N_mu^2 (diagonal metric) */
        for (int mu = 0; mu < 4; ++mu) NN += N[mu] * N[mu] / G.g[mu];
        double norm = sqrt(fabs(NN));
        double nv[4];
        for (int mu = 0; mu < 4; ++mu) nv[mu] = N[mu] / norm;
        double un = 0.0;
        for (int mu = 0; mu < 4; ++mu) un += u[mu] * nv[mu];
        double dsig = 1.0 / (aux[16 * n + a] * fabs(un));
        if (cnt < cap) {
            double *r = out + (size_t)cnt * FO_NREC;
            r[0] = tau;
            for (int d = 0; d < 3; ++d) r[1 + d] = d < dim ? y[d * n + a] : 0.0;
            for (int mu = 0; mu < 4; ++mu) r[4 + mu] = u[mu];
            r[8] = aux[5 * n + a];
            for (int c = 0; c < 3; ++c) r[9 + c] = aux[(6 + c) * n + a];
            r[12] = e;
            r[13] = aux[9 * n + a];
            r[14] = aux[1 * n + a];
            for (int mu = 0; mu < 4; ++mu) r[15 + mu] = nv[mu];
            r[19] = dsig;
            for (int mu = 0; mu < 4; ++mu) r[20 + mu] = dsig * nv[mu];
            ids[cnt] = a;
        }
        ++cnt;
    }
    free(buf);
    grid_free(&g);
    return cnt;
}
