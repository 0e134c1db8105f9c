/*
 * sph_gb300.h -- C ABI of the GB300 (sm_103a) SPH particle step for relativistic
 * viscous BSQ hydrodynamics, following arXiv 2511.22852 (CCAKE 2.0).
 *
 * What the library computes, per Runge-Kutta stage (Sec. "Numerical solver:
 * Smoothed particle hydrodynamics (SPH)"):
 *   a1/a2  Morton-sorted cell list with cells of side 2h (the kernel support) and a
 *          stable sort of the particles by (cell key, original id);
 *   a3     kernel sums sigma*_a = sum_b W_ab, s*_a = sum_b S_b W_ab,
 *          n*_qa = sum_b N_qb W_ab (eqs. sigmastar, refconv), rest-frame
 *          densities q = q* / (u^0 sqrt(-g));
 *   a4     EoS inversion (s, n_B, n_S, n_Q) -> (T, mu_B, mu_S, mu_Q) by Newton
 *          iteration on the tabulated 4D EoS, the closed-form EoS as backup
 *          (Sec. "Equation of state", "EoS inverter");
 *   a5     SPH gradients (eqs. sphderivativerel, generalsphderivative);
 *   a6     the acceleration from the linear system M du/dx0 = F (eq. unugeneral),
 *          entropy production (eq. dsdnrewr), minimal Israel-Stewart bulk and
 *          shear relaxation (eqs. min_bul_rel, min_she_rel);
 *   a7     Heun (RK2) update;
 *   a8     conservation totals (energy, entropy, charges, longitudinal work).
 * All of it runs in hand-written CUDA kernels on one GPU; nothing falls back to
 * the CPU.
 *
 * Units: lengths and times in fm (eta dimensionless), T and mu in fm^-1,
 * densities s, n_q in fm^-3, p and e in fm^-4 (hbar c = 0.1973269804 GeV fm).
 *
 * Conventions for every call:
 *   - the return value is an sph_status, SPH_OK = 0; nothing throws across the ABI;
 *   - on an error, sph_last_error() returns a message for the calling thread;
 *   - handles are opaque; one event handle is used by one host thread at a time;
 *   - the library owns all device memory it allocates; the caller owns every
 *     buffer it passes in and may free it as soon as the call returns.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SPH_OK = 0,
    SPH_ERR_ARG = 1,        /* invalid argument (null pointer, bad size, unsupported option) */
    SPH_ERR_OOM = 2,        /* device allocation failed */
    SPH_ERR_CUDA = 3,       /* a CUDA runtime call failed */
    SPH_ERR_EOS_RANGE = 4,  /* a particle outside the table when the policy makes that fatal */
    SPH_ERR_EOS_NOCONV = 5, /* no EoS solution for a particle, policy fatal */
    SPH_ERR_NONFINITE = 6,  /* a non-finite state value, policy fatal */
    SPH_ERR_TIMEOUT = 7,    /* a bounded host wait on the device gave up */
    SPH_ERR_STATE = 8       /* call out of order, or the particles outgrew the cell table */
} sph_status;

/* per-particle status bits (read with SPH_F_STATUS; OR-ed over an event in sph_totals) */
#define SPH_PST_FALLBACK 1u     /* table Newton did not converge: closed-form EoS used */
#define SPH_PST_OUT_OF_TABLE 2u /* the solution lies outside the table: closed-form EoS used */
#define SPH_PST_NOCONV 4u       /* no EoS solution at all */
#define SPH_PST_NONFINITE 8u    /* non-finite density or state */
#define SPH_PST_CS2_CAPPED 16u  /* c_s^2 > cap: dp/ds, dp/dn scaled down in the acceleration system */
#define SPH_PST_BACKUP 64u      /* neither table nor closed form inverts: the conformal-diagonal backup EoS used */
#define SPH_PST_SOLVE_FAIL 32u  /* the acceleration system was singular */
/* A particle with NOCONV or NONFINITE from the EoS is frozen for that stage: it moves
 * ballistically (dx/dt = v), every other rate is zero, and it contributes p = e = 0 to its
 * neighbours' pressure gradient. */

/* ---------------------------------------------------------------------------
 * Equation of state (Sec. "Equation of state"; closed forms of the kind of
 * Sec. "Modified EoS to permit lower eps_min").
 *
 * Closed form, always present (and the backup when a table is given):
 *   p(T, mu) = T^4 [a0 + a1 (1 + tanh((T hbar c - Tc)/w)) / 2] + T^2 sum_q chi_q mu_q^2 / 2,
 * Tc and w in GeV.  a1 = 0, chi = 0 is the conformal EoS p = e/3.
 *
 * Optional table (has_table = 1): p, s, n_B, n_S, n_Q on the regular grid
 * T_i = T0 + i dT (i < nT), mu_q,j = mu0[q] + j dmu[q] (j < nmu[q]); each array
 * holds nT*nmu[0]*nmu[1]*nmu[2] doubles, row-major [T][mu_B][mu_S][mu_Q]
 * (mu_Q fastest), in HOST memory.  The library copies them to the device,
 * interleaved per node; the caller keeps ownership of its arrays.
 * ------------------------------------------------------------------------- */
typedef struct {
    double a0, a1, Tc_GeV, w_GeV;
    double chi[3];
    int32_t has_table;
    int32_t nT;
    int32_t nmu[3];
    int32_t newton_maxit; /* table Newton iterations (<= 0: 30) */
    double T0, dT;
    double mu0[3], dmu[3];
    const double *p, *s, *nB, *nS, *nQ;
    double newton_tol; /* max |residual| / s for convergence (<= 0: 1e-12) */
} sph_eos_desc;

typedef struct sph_eos sph_eos;
typedef struct sph_event sph_event;

/* Creates an EoS handle.  Errors: SPH_ERR_ARG (null pointers, a table dimension
 * < 2, non-positive spacing, a0 <= 0), SPH_ERR_OOM, SPH_ERR_CUDA.  The handle is
 * reference counted: events keep it alive; sph_free_eos drops the caller's reference. */
sph_status sph_set_eos_table(sph_eos **out, const sph_eos_desc *desc);
void sph_free_eos(sph_eos *eos);

/* ---------------------------------------------------------------------------
 * Event: N SPH particles with unit SPH mass (Sec. "SPH interpretation of a
 * fluid element": m_b = 1, sigma* = 1/V*), dynamical variables of eq.
 * dynamicalvariables: position x^i, u^i, S = s/sigma, Pi/sigma, pi^{ij}/sigma,
 * N_q = n_q/sigma.
 *
 * Coordinates: milne = 1 is (tau, x, y, eta) with sqrt(-g) = tau, milne = 0 is
 * Cartesian (t, x, y, z).  dim = 2 is transverse (x, y) only (with milne = 1:
 * boost-invariant 2+1D); dim = 3 adds eta (Milne, distances Euclidean in (x, y, eta))
 * or z.  Other values return SPH_ERR_ARG.
 *
 * Arrays (SoA, doubles): x[dim*n] (x^1 for all particles, then x^2, ...),
 * u[dim*n] (contravariant u^i), S[n], Nq[3*n] (B, S, Q), Bv[n] = Pi/sigma (may be
 * NULL: zero), Pv[npi*n] = pi^{ij}/sigma for (xx, xy, yy) when dim = 2 (npi = 3) and
 * (xx, xy, x3, yy, y3) when dim = 3 (npi = 5; pi^{33} follows from tracelessness) (may be
 * NULL: zero).  Host pointers, or device pointers when on_device = 1 (for example
 * torch tensors' data_ptr()).  The library copies them; the caller keeps them.
 *
 * Transport: eta = eta_over_s * s; zeta = zeta_peak exp(-(T hbar c - zeta_T)^2 /
 * (2 zeta_w^2)) s; tau_pi = tau_pi_coef eta / (e + p); tau_Pi = tau_Pi_ratio tau_pi.
 * viscous = 0 evolves an ideal fluid.  cs2_cap bounds c_s^2 inside the
 * acceleration system (<= 0: 1).  fatal_mask: per-particle status bits that
 * make sph_step fail (0: none).  stream: a cudaStream_t, or NULL to let the
 * library create one.
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t dim, milne, viscous, on_device;
    int64_t n;
    double h, tau0, dtau;
    const double *x, *u, *S, *Nq, *Bv, *Pv;
    double eta_over_s, zeta_peak, zeta_T_GeV, zeta_w_GeV;
    double tau_pi_coef, tau_Pi_ratio, cs2_cap;
    uint32_t fatal_mask;
    int32_t use_graph; /* 1: replay sph_step through a captured CUDA graph */
    void *stream;
    int32_t profile;   /* 1: time every kernel group with CUDA events (no graph; see sph_kernel_times) */
    int32_t precision; /* SPH_FP64 or SPH_MIXED (see below) */
    double T_stop_GeV; /* > 0: a particle whose temperature is below it has left the fluid (the matter
                          below the freeze-out surface of Sec. "Freeze-out hypersurface construction"):
                          in that stage it streams freely (dx/dx0 = v, its other variables and charges
                          unchanged) while its neighbours still see its kernel sums and pressure;
                          0: off */
    /* BSQ diffusion (Sec. "Equations of motion", eq. min_dif_rel; constant kappa/T^2 and tau T,
     * Sec. "Transport coefficients"), dim = 2 only, single-event forms: with kappaT2 != NULL
     * (kappaT2[3 q + q'] = kappa_{qq'} / T^2, q = B, S, Q; tauJT[q] = tau_q T > 0) the charges
     * diffuse: tau_q Delta^mu_nu D J^nu_q + J^mu_q = kappa_{qq'} nabla^<mu> (mu_{q'} / T) (metric
     * (+,-,-,-): the current runs down the gradient of mu/T); the state gains J^i_q / sigma
     * (Jv[6 n]: (x, y) of B, then S, then Q; NULL: zero) and Nq becomes the particles' lab charge
     * N_q + J^0_q / (sigma u^0), whose sum over the particles is conserved (read with SPH_F_JV,
     * SPH_F_NQ).  kappaT2 = NULL: no diffusion (the charges are constant). */
    const double *kappaT2, *tauJT, *Jv;
} sph_event_desc;

/* Precision of the step.  SPH_FP64: every operation in double precision.  SPH_MIXED (dim 2 or 3):
 * the neighbour passes (kernel sums and gradients) run in single precision with positions
 * relative to their cell's origin and compensated (two-sum) accumulation, combined per particle
 * without loss (2+1D: cell-tiled, two candidates per packed FP32 instruction); the neighbour set
 * stays exactly that of the FP64 test (a proven float error band, the FP64 test inside it); the
 * EoS inversion (to max(newton_tol, 1e-10) without the polishing step, as its inputs carry the
 * single-precision sums' rounding), equations of motion, Heun update and reductions stay FP64.
 * Results differ from SPH_FP64 at the ~1e-7 relative level. */
#define SPH_FP64 0
#define SPH_MIXED 1

/* Copies the particles to device memory (sorted by cell on the first stage) and
 * binds the EoS.  Errors: SPH_ERR_ARG (n < 0, h <= 0, dtau <= 0, dim not 2 or 3, null
 * arrays for n > 0), SPH_ERR_OOM, SPH_ERR_CUDA.  n = 0 gives an empty event on
 * which every call succeeds and does nothing. */
sph_status sph_init_event(sph_event **out, const sph_event_desc *desc, const sph_eos *eos);
void sph_free_event(sph_event *ev);

/* Advances nsteps full Heun steps (2 stages each) of size dtau on the event's
 * stream.  Asynchronous unless flags & SPH_SYNC; with SPH_SYNC the call waits
 * (bounded by the event's timeout, SPH_ERR_TIMEOUT if exceeded) and checks the
 * per-particle status against fatal_mask.  nsteps < 0: SPH_ERR_ARG. */
#define SPH_SYNC 1u
sph_status sph_step(sph_event *ev, int32_t nsteps, uint32_t flags);

/* ---------------------------------------------------------------------------
 * Read-out, in the ORIGINAL particle order of sph_init_event.  A field is copied
 * when its mask bit is set; its destination must then be non-NULL and hold the
 * stated number of doubles (or uint32/int32).  Derived fields (SIGMA_STAR ...
 * STATUS) are evaluated at the current state (cell list, kernel sums and EoS
 * inversion are rerun if the state changed since the last read).
 * Destinations are host memory unless on_device = 1.  The call synchronises the
 * event's stream.
 * ------------------------------------------------------------------------- */
#define SPH_F_X (1ull << 0)          /* x[dim*n] */
#define SPH_F_U (1ull << 1)          /* u[dim*n] */
#define SPH_F_S (1ull << 2)          /* S[n] */
#define SPH_F_NQ (1ull << 3)         /* Nq[3*n] */
#define SPH_F_BV (1ull << 4)         /* Bv[n] */
#define SPH_F_PV (1ull << 5)         /* Pv[npi*n] */
#define SPH_F_SIGMA_STAR (1ull << 6) /* sigstar[n] */
#define SPH_F_S_DENS (1ull << 7)     /* s[n] (rest frame) */
#define SPH_F_N_DENS (1ull << 8)     /* nq[3*n] (rest frame) */
#define SPH_F_T (1ull << 9)          /* T[n] */
#define SPH_F_MU (1ull << 10)        /* mu[3*n] */
#define SPH_F_P (1ull << 11)         /* p[n] */
#define SPH_F_E (1ull << 12)         /* e[n] */
#define SPH_F_PI_BULK (1ull << 13)   /* Pi[n] */
#define SPH_F_STATUS (1ull << 14)    /* status[n] (uint32) */
#define SPH_F_NNB (1ull << 15)       /* neighbour count including self, nnb[n] (int32) */
#define SPH_F_CELL (1ull << 16)      /* cell coordinates cell[dim*n] (int32) */
#define SPH_F_JV (1ull << 18)        /* diffusion currents Jv[6*n]: J^i_q / sigma (x, y of B, S, Q) */
#define SPH_F_GUESS (1ull << 17)     /* EoS warm start guess[4*n]: the previous stage's table solution
                                        (T, mu_B, mu_S, mu_Q), T = 0 where the table was not used;
                                        part of the evolved state (read it and write it back for a
                                        bitwise resume) */

typedef struct {
    double *x, *u, *S, *Nq, *Bv, *Pv;
    double *sigstar, *s, *nq, *T, *mu, *p, *e, *Pi;
    uint32_t *status;
    int32_t *nnb, *cell;
    double *guess;
    int32_t on_device;
    double *Jv; /* SPH_F_JV */
} sph_field_bufs;

typedef struct {
    double tau;
    double E;      /* sum_a sqrt(-g) T^{00}_a / sigma*_a */
    double S;      /* sum_a S_a */
    double N[3];   /* sum_a N_qa (fixed-order sums: bitwise constant) */
    double work;   /* int dtau sum_a sqrt(-g) Gamma^0_{mu nu} T^{mu nu} / sigma* (Milne) */
    uint32_t status_or;
    int32_t pair_overflows; /* plain 2D: stages (and read-out evaluations) whose neighbour pair
                               lists overflowed their capacity and ran the per-particle passes
                               instead (the lists then grow before the next step) */
    int64_t steps;
    int64_t pairs;          /* accepted neighbour pairs (self pairs included) summed over all stages */
    int64_t kernel_launches; /* kernels launched by sph_step so far (graph replays included) */
    int64_t eos_work[3];     /* EoS work done: table residual+Jacobian evaluations, 4x4 solves,
                                closed-form evaluations (all stages and read-outs) */
    int64_t shell_tests;     /* SPH_MIXED: candidates decided by the exact FP64 test */
} sph_totals;

sph_status sph_read_fields(sph_event *ev, uint64_t mask, const sph_field_bufs *out, sph_totals *tot);

/* Overwrites the evolved state (x, u, S, Bv, Pv, the EoS warm start; Nq unchanged) from
 * buffers in the original particle order (mask bits SPH_F_X .. SPH_F_PV and SPH_F_GUESS;
 * others ignored), e.g. to resume from a checkpoint read with sph_read_fields.  Fields not
 * in the mask keep their values.  Errors: SPH_ERR_ARG. */
sph_status sph_write_state(sph_event *ev, uint64_t mask, const sph_field_bufs *in);

/* Per-kernel-group device time of an event created with profile = 1: for group k < *count
 * (count <= max), names[32*k ..] gets a NUL-terminated name, ms[k] the summed milliseconds and
 * launches[k] the number of launches since creation.  Groups: cells, permute, density, eos,
 * gradient, eom, work.  SPH_ERR_STATE if profiling is off. */
sph_status sph_kernel_times(sph_event *ev, int32_t max, char *names, double *ms, int64_t *launches, int32_t *count);

/* ---------------------------------------------------------------------------
 * Offline EoS inverter (Sec. "Equation of state": the EoS converted once onto a grid in
 * (s, n) with s on logarithmic decades, uniform within each decade; interpolation instead of
 * root finding).  sph_eos_build_inverse inverts the handle's table at every node by the
 * online root finder (closed form, then table Newton; NaN where no solution exists): s at
 * 10^d (1 + 9 j / per_decade) for d = decade_lo .. decade_lo + decades - 1, j < per_decade,
 * plus 10^(decade_lo + decades); the charge ratios n_q / s on nx uniform nodes in [-xmax, xmax]
 * (4 doubles per node; at most 2^28 nodes).  An event in SPH_EOS_OFFLINE mode takes (T, mu)
 * from the quadrilinear interpolant of that table, then p, e and the derivatives from the
 * forward table there; points off the grid, or whose interpolated (T, mu) leave the forward
 * table, use the online inversion.  Faster, less accurate (first order in the grid spacing
 * for T: the inverse of the piecewise-multilinear forward table has kinks).
 * Errors: SPH_ERR_ARG (no table, bad grid), SPH_ERR_OOM; sph_set_eos_mode: SPH_ERR_STATE when
 * the handle has no inverted table. */
#define SPH_EOS_ONLINE 0
#define SPH_EOS_OFFLINE 1
sph_status sph_eos_build_inverse(sph_eos *eos, int32_t per_decade, int32_t decade_lo, int32_t decades, int32_t nx,
                                 double xmax);
sph_status sph_set_eos_mode(sph_event *ev, int32_t mode);

/* ---------------------------------------------------------------------------
 * Backup EoS (Sec. "Equation of state": backup EoS tried in turn when a point lies outside the
 * others' reach): with enable = 1, a particle that neither the table Newton nor the closed-form
 * EoS inverts takes the conformal-diagonal EoS p = A0 [T^4 + sum_q (mu_q / mu_q0)^4] (T_0 =
 * 1/fm), which inverts (s, n) in closed form for every s > 0: T = (s / 4 A0)^(1/3),
 * mu_q = (n_q mu_q0^4 / 4 A0)^(1/3), e = 3 p, c_s^2 = 1/3; flagged SPH_PST_BACKUP.  A0 and
 * mu_q0 match the closed form at T_scale: p equal at (T_scale, 0) and at (T_scale, mu_q = mu_max)
 * (T_scale = 1.1 T_FO in the paper).  enable = 0 (the default): no backup; such particles have
 * no solution (SPH_PST_NOCONV) and are frozen for the stage.  Errors: SPH_ERR_ARG for
 * non-positive T_scale or mu_max; SPH_ERR_TIMEOUT if the event's stream does not drain.
 * ------------------------------------------------------------------------- */
sph_status sph_set_eos_backup(sph_event *ev, int32_t enable, double T_scale_GeV, double mu_max_GeV);

/* ---------------------------------------------------------------------------
 * Dynamical-initialisation sources (Sec. "Dynamical initialization": the source j^mu of the
 * partons formed during the evolution): partons[8 k ..] = formation time x^0_k, position
 * (x, y, z) (Cartesian) or (x, y, eta) (Milne; 2D uses x, y), four-momentum p^mu (fm^-1,
 * contravariant, the event's coordinates).  The stage evaluated at x^0 gains
 *   I^mu(r) = sum over partons with x^0 - dtau < x^0_k <= x^0 of
 *             norm p^mu_k W(|r - r_k|, h_src) / (sqrt(-g) dtau)
 * with W the cubic spline of the event's dimension and width h_src (distances Euclidean in the
 * event's coordinates); I^mu enters the equations of motion as the jet tracks' source does
 * (sph_set_jets).  charges (may be NULL): charges[3 k ..] = (B, S, Q) of parton k, smeared with
 * the same weight into the charge source I_q of eq. charge_conservation (the paper prints the
 * smearing for p^mu; the charges take the same kernel).  The particles' charges then evolve,
 * dN_q/dx0 = sqrt(-g) I_q / sigma* with the step's Heun quadrature, the entropy rate gains
 * -mu_q/T dN_q/dx0 (eq. dsdnrewr) and the momentum equation's enthalpy rate the charges'
 * (mu_q + dp/dn_q) sigma dN_q; without charges they stay constant.  Host arrays, copied (sorted
 * by formation time); nparton = 0 removes the sources.  Errors: SPH_ERR_ARG (nparton outside
 * 0..2^24, null partons, h_src <= 0, non-finite entries), SPH_ERR_OOM; SPH_ERR_TIMEOUT if the
 * event's stream does not drain.
 * ------------------------------------------------------------------------- */
sph_status sph_set_partons(sph_event *ev, int64_t nparton, const double *partons, const double *charges, double norm,
                           double h_src);

/* ---------------------------------------------------------------------------
 * Viscous equations of motion (Sec. "Equations of motion": eqs. min_bul_rel, min_she_rel and
 * eq. dnmr).  SPH_EOM_MIN_IS (the default): minimal Israel-Stewart.  SPH_EOM_DNMR: DNMR without
 * the K terms and the couplings to diffusion, with the shear-bulk J terms and the R term phi_7
 * (phi_1 = phi_3 = phi_6 = 0):
 *   tau_Pi D Pi + Pi = -zeta theta - delta_PiPi Pi theta + lambda_Pipi pi:sigma,
 *   tau_pi D pi^<mu nu> + pi^{mu nu} = 2 eta sigma^{mu nu} - delta_pipi pi^{mu nu} theta
 *       - tau_pipi pi_lambda^<mu sigma^nu>lambda + phi_7 pi_alpha^<mu pi^nu>alpha
 *       + lambda_piPi Pi sigma^{mu nu};
 * coeffs[6] (host, copied): delta_PiPi / tau_Pi, lambda_Pipi / (tau_Pi (1/3 - c_s^2)),
 * delta_pipi / tau_pi, tau_pipi / tau_pi, lambda_piPi / tau_pi, phi_7 p (the 14-moment values
 * for a massless gas are 2/3, 8/5, 4/3, 10/7, 6/5, 9/70).  coeffs is ignored for
 * SPH_EOM_MIN_IS.  Applies to the plain and mixed single-event forms, 2D and 3D (the serving
 * form runs minimal Israel-Stewart).  Errors: SPH_ERR_ARG for an unknown model, missing or
 * non-finite coefficients; SPH_ERR_TIMEOUT if the event's stream does not drain.
 * ------------------------------------------------------------------------- */
#define SPH_EOM_MIN_IS 0
#define SPH_EOM_DNMR 1
sph_status sph_set_viscous_eom(sph_event *ev, int32_t model, const double *coeffs);

/* ---------------------------------------------------------------------------
 * Energy-momentum source of jet tracks (eq. conservation_source with I^nu != 0, Sec.
 * "Equations of motion"; Cartesian events).  Track k (tracks[8 k ..] = x0, y0, z0, n_x, n_y,
 * n_z, t0, dE/dx, host memory, n a unit vector, dE/dx in fm^-2) moves at the speed of light
 * from x0 along n from time t0 and deposits dE/dx per unit path length into a normalised
 * Gaussian of width sigma (fm) around its current position, with the momentum of light moving
 * along n: I^nu(t, x) = sum_k dE/dx_k G_sigma(x - x0_k - n_k (t - t0_k)) (1, n_k) for t >= t0_k
 * (z = 0 for dim = 2).  In the equations of motion dP^i/dt gains I^i/sigma* and dS/dt gains
 * u_nu I^nu / (u^0 sigma T).  ntrack = 0 removes the source.  Errors: SPH_ERR_ARG (Milne
 * coordinates, ntrack outside 0..4096, sigma <= 0, non-finite parameters), SPH_ERR_OOM. */
sph_status sph_set_jets(sph_event *ev, int64_t ntrack, const double *tracks, double sigma);

/* ---------------------------------------------------------------------------
 * Freeze-out hypersurface (Sec. "Freeze-out hypersurface construction"), dim = 2 or 3.
 * After sph_freezeout_setup, the first stage of every step finds the particles whose energy
 * density fell through e_fo since the previous step's first stage and records one surface
 * element each, evaluated at the current state (the end of the step in which it crossed):
 *   n_mu = N_mu / sqrt(|N_mu N^mu|), N_mu = -d_mu e (covariant, pointing outwards; in 3+1D
 *   Milne coordinates N_mu N^mu = N_0^2 - N_x^2 - N_y^2 - N_eta^2/tau^2), with the
 *   spatial derivatives by the SPH sum d_i e_a = sum_b (e_b/sigma*_b) d_i W_ab and
 *   d_tau e = (e - e_prev)/dtau - v^i d_i e (the particle's rate minus advection);
 *   |dsigma| = m/(sigma |u^mu n_mu|) with unit SPH mass and the rest-frame density sigma;
 *   dsigma_mu = |dsigma| n_mu.
 * A record holds SPH_FO_NREC doubles: tau, x^1..3, u^0..3, T, mu_B, mu_S, mu_Q, e, p, s,
 * n_0..3, |dsigma|, dsigma_0..3 (entries of the third spatial axis are 0 in 2+1D; in 3+1D Milne
 * coordinates x^3 = eta_s, u^3 = u^eta, n_3 = n_eta).  The
 * crossings of the step that ends at tau are found by the next step's first stage.
 * Setup (again) clears the recorded elements; the first step after it only records e.
 * Errors: SPH_ERR_ARG (e_fo <= 0, capacity < 1), SPH_ERR_OOM. */
#define SPH_FO_NREC 24
sph_status sph_freezeout_setup(sph_event *ev, double e_fo, int64_t capacity);
/* Elements recorded so far, sorted by (tau, particle id): min(count, capacity, cap) records to
 * elems[SPH_FO_NREC * cap] and their original particle indices to ids[cap] (host buffers);
 * *count receives the number of crossings found.  SPH_ERR_STATE if recording is off or more
 * crossings than the capacity occurred (the surplus was dropped). */
sph_status sph_read_freezeout(sph_event *ev, int64_t cap, double *elems, int64_t *ids, int64_t *count);

/* ---------------------------------------------------------------------------
 * Densities without device allocation.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory -- a serving loop that has
 * handed all free HBM to its own pool, or code running while another thread captures a
 * CUDA graph in global mode (where cudaMalloc is illegal).  It runs the cell list and the
 * kernel sums (rows a1-a3) exactly as the stepping path does and returns, in the input
 * order, out[0*n..] = sigma*, out[1*n..] = s, out[2..4 *n..] = n_B, n_S, n_Q (rest frame,
 * divided by u^0 sqrt(-g), sqrt(-g) = tau if milne else 1).
 * x[2*n], u[2*n], S[n], Nq[3*n], out[5*n] are DEVICE buffers owned by the caller; dim = 2.
 * Every temporary lives in one fixed file-scope device array (10,223,872 bytes, held by
 * every GPU that loads the library until exit); the call allocates nothing and frees
 * nothing.  Limits: n <= SPH_NOALLOC_MAX_PARTICLES (else SPH_ERR_ARG) and at most 256
 * cells of side 2h per axis (else SPH_ERR_STATE).  Work runs on `stream` and the call
 * returns after it finished; the wait is bounded (SPH_WAIT_LIMIT_S seconds, default 600,
 * then SPH_ERR_TIMEOUT).  stream = NULL is the legacy default stream, which synchronises with
 * every other stream of the device and may not be used while any thread captures a CUDA
 * graph in global mode: such callers pass a stream they created.  A launch failure returns
 * SPH_ERR_CUDA.  All calls share the array: calls that overlap on the GPU race and must be
 * serialised by the caller.  The first call on a device (and the first after its context
 * was destroyed and recreated, e.g. by cudaDeviceReset) looks up the array's address; make
 * it before any stream capture. */
#define SPH_NOALLOC_MAX_PARTICLES 65536
sph_status sph_density_noalloc(const double *x, const double *u, const double *S, const double *Nq, int64_t n,
                               double h, double tau, int32_t milne, double *out, void *stream);

/* ---------------------------------------------------------------------------
 * Serving form: event-by-event simulation (the paper runs one hydrodynamic evolution per
 * collision event, Sec. "Hydrodynamic evolution"; experiments average observables over
 * many events) with continuous batching.  A server owns one particle arena carved from
 * free HBM; submitted 2+1D events wait in a FIFO queue and are admitted while a slot and a
 * contiguous arena range are free; every batch step advances all admitted events by one
 * Heun step together (one CUDA graph, the same for every batch composition); an event that
 * has finished its steps is evaluated once more at its final state (cell list, densities,
 * EoS) and its fields are copied to pinned host memory, after which its slot and range are
 * reused.  Arithmetic: the mixed form (SPH_MIXED above, with cell-tiled neighbour passes);
 * EoS inversion, equations of motion and totals in FP64.  An event's results do not depend
 * on the other events in the batch (bitwise).
 *
 * Threading: one host thread drives a server at a time.  Ownership: sph_submit copies the
 * caller's arrays; sph_collect writes into caller-owned host buffers.
 * ------------------------------------------------------------------------- */
typedef struct sph_server sph_server;

typedef struct {
    int32_t max_events;    /* slots: events advanced together, 1..256 */
    int32_t max_inflight;  /* batch steps enqueued ahead of the device, 1..8 (0: 2) */
    int64_t max_particles; /* arena capacity in particles (0: hbm_fraction of free HBM) */
    double hbm_fraction;   /* share of free HBM for the arena when max_particles = 0, <= 0.9 (0: 0.25) */
    int64_t pinned_bytes;  /* pinned host staging pool (0: 256 bytes per arena particle) */
    void *stream;          /* cudaStream_t of all server work, NULL: library-created */
    int32_t polish;        /* 1: a Newton polishing step after convergence, as the plain form */
    int32_t groups;        /* 1: every pass over all events in turn; 0 or 2: the events split into
                              two groups of about equal particle counts, the second group's passes
                              one pass behind the first's on a second branch of the step graph,
                              so that the passes of one group fill the tails of the other's (the
                              FP64-bound EoS and equations of motion beside the FP32 neighbour
                              passes); results are bitwise the same either way */
    double newton_tol;     /* EoS Newton tolerance on max |residual|/s (<= 0: 1e-10; the plain form
                              uses the EoS handle's, 1e-12 by default) */
} sph_server_desc;

#define SPH_TICKET_QUEUED 0
#define SPH_TICKET_RUNNING 1
#define SPH_TICKET_DONE 2

typedef struct {
    int64_t queued, running, done; /* tickets by state (done: results not yet collected) */
    int64_t batch_steps;           /* batch steps launched */
    int64_t particle_steps;        /* sum over batch steps of the particles advanced */
    int64_t arena_capacity, arena_in_use; /* particles */
    int64_t kernel_launches;       /* kernels launched by the server (graph replays included) */
    int32_t slots_in_use, max_events;
    double device_ms;              /* device time of the batch steps completed so far (CUDA events
                                      around each step's graph launch) */
    int64_t steps_timed;           /* batch steps included in device_ms */
    int64_t failed;                /* events ended early because their state or rates became
                                      non-finite (their tickets are DONE; see sph_server_pump) */
} sph_server_stats;

/* Errors: SPH_ERR_ARG (max_events outside 1..256, bad fractions), SPH_ERR_OOM (arena
 * allocation), SPH_ERR_CUDA.  The server holds a reference to eos. */
sph_status sph_server_create(sph_server **out, const sph_server_desc *desc, const sph_eos *eos);
/* Waits for the server's stream and frees everything, uncollected results included. */
void sph_server_free(sph_server *srv);
/* Queues an event that is to advance nsteps Heun steps.  desc as for sph_init_event with
 * dim = 2 and n >= 1 (precision, use_graph, profile, stream and fatal_mask are ignored);
 * the arrays are copied before the call returns.  *ticket identifies the request.
 * Errors: SPH_ERR_ARG (as sph_init_event; dim != 2, n < 1, nsteps < 0), SPH_ERR_OOM (n
 * larger than the arena). */
sph_status sph_submit(sph_server *srv, const sph_event_desc *desc, int32_t nsteps, int64_t *ticket);
/* Runs up to max_steps batch steps: before each, admits queued events that fit; after
 * each, retires events that finished.  Returns early when nothing is admitted or running.
 * At most max_inflight steps run ahead of the device (bounded waits: SPH_ERR_TIMEOUT).
 * *running (may be NULL) receives the number of events in the batch.  An event whose state
 * or rates become non-finite is ended early, within max_inflight + 2 batch steps, so that it
 * does not slow the others down: its ticket becomes DONE with its last state, the
 * non-finite bit (8) in the totals' status_or and totals.steps below the requested count;
 * the other events' results do not change (sph_server_stats.failed counts such events). */
sph_status sph_server_pump(sph_server *srv, int32_t max_steps, int32_t *running);
/* State of a ticket (SPH_TICKET_*); for a DONE ticket, *latency_s (may be NULL) receives
 * the seconds from sph_submit until its results were readable in host memory (device
 * completion time of the copy).  Errors: SPH_ERR_ARG (unknown ticket). */
sph_status sph_poll(sph_server *srv, int64_t ticket, int32_t *state, double *latency_s);
/* Copies the fields in mask of a DONE ticket to host buffers (original particle order; the
 * state fields X .. PV at the final time, the derived fields SIGMA_STAR .. NNB evaluated at
 * the final state) and its totals (tot may be NULL), then releases the ticket.  Fields
 * available: X, U, S, NQ, BV, PV, SIGMA_STAR, S_DENS, N_DENS, T, MU, P, E, PI_BULK, STATUS,
 * NNB.  Errors: SPH_ERR_STATE (not done), SPH_ERR_ARG (unknown ticket, other fields, NULL
 * destinations, on_device). */
sph_status sph_collect(sph_server *srv, int64_t ticket, uint64_t mask, const sph_field_bufs *out, sph_totals *tot);
sph_status sph_server_stats_get(sph_server *srv, sph_server_stats *out);
/* Pumps until every submitted ticket is DONE (timeout_s <= 0: no limit). */
sph_status sph_server_drain(sph_server *srv, double timeout_s);
/* Autotuner of the tiled neighbour passes' shape: times them on the running batch (the state of
 * its last step) for every pair of block size (64, 96, 128, 192, 256 threads) and lane split (a
 * cell's particles shared by the lanes of 2, 4 or 8 warps: the lanes per particle follow from it
 * and the cell's occupancy), trials runs each, and keeps the fastest for the following steps
 * (*chosen: threads per block, *chosen_lanes: warps of the lane split; either may be NULL).  The
 * lane split sets the summation order of the kernel sums (results differ at the rounding level
 * between splits; for a fixed shape they stay bitwise independent of the batch composition).
 * Errors: SPH_ERR_STATE (no batch has run a step). */
sph_status sph_server_autotune(sph_server *srv, int32_t trials, int32_t *chosen, int32_t *chosen_lanes);
/* Sets the tiled neighbour passes' shape by hand (threads per block: 64, 96, 128, 192 or 256;
 * lane split: 2, 4 or 8 warps), e.g. to repeat a run bitwise with a shape an earlier
 * autotuning chose.  Waits for the server's stream; the following steps use the shape.
 * Errors: SPH_ERR_ARG (a value outside those lists). */
sph_status sph_server_set_shape(sph_server *srv, int32_t threads, int32_t lane_warps);

/* Sampled per-kernel-group timing of the batch step (measurement support): with every > 0,
 * every every-th batch step launches the same kernels eagerly instead of through the step graph,
 * with CUDA events between its kernel groups (per stage: sort = bounding boxes, cell keys, scans
 * and permutation; density; eos; gradient; eom; work), on the server's stream.  every = 0 turns
 * the sampling off (the sums are kept).  sph_server_kernel_times: for group k < *count (count <=
 * max), names[32*k ..] gets its name, ms[k] the summed milliseconds of the sampled stages and
 * launches[k] their number (two per sampled step).  Errors: SPH_ERR_ARG; SPH_ERR_STATE when
 * sampling was never enabled. */
sph_status sph_server_profile(sph_server *srv, int32_t every);
sph_status sph_server_kernel_times(sph_server *srv, int32_t max, char *names, double *ms, int64_t *launches,
                                   int32_t *count);

/* Measurement support (not part of the stepping interface): the device's fused multiply-add
 * rate in FP64 (fp64 = 1) or FP32 (fp64 = 0), the denominator of the arithmetic rooflines of the
 * step's kernels.  Eight independent multiply-add chains per thread, eight resident blocks of 256
 * threads on every SM, about 40 ms per launch; *gflops = 2 x multiply-adds / the best of reps
 * launches timed with CUDA events (*best_ms, may be NULL, its duration).  Allocates a small
 * buffer and a stream, freed before returning.  Errors: SPH_ERR_ARG (null gflops, reps < 1),
 * SPH_ERR_OOM, SPH_ERR_CUDA. */
sph_status sph_measure_fma_peak(int32_t fp64, int32_t reps, double *gflops, double *best_ms);

/* Message of the calling thread's last error ("" if none). */
const char *sph_last_error(void);

/* Test support (not part of the stepping interface): all ordered neighbour pairs
 * (a, b) with r_ab < 2h at the current positions, in original ids, sorted by
 * (a, b), self pairs included.  Writes min(count, cap) pairs; *count gets the total. */
sph_status sph_debug_neighbors(sph_event *ev, int64_t cap, int32_t *pa, int32_t *pb, int64_t *count);

/* Test support: one right-hand-side evaluation at the current state, without
 * advancing it.  rates[nv*n] (nv = 2 dim + 2 + npi, plus 6 with diffusion) and grad[(dim*dim + dim)*n]
 * (d_k u^j with k major, then F^i) in original order, host buffers; either may be NULL. */
sph_status sph_debug_rates(sph_event *ev, double *rates, double *grad);

#ifdef __cplusplus
}
#endif
#endif /* SPH_GB300_H */
