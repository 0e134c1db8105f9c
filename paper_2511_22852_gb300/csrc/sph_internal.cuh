// sph_internal.cuh -- device-side data layout and helpers of the GB300 SPH step.
//
// Layout in HBM (structure of arrays, FP64, particles in Morton-sorted cell
// order, ping-pong buffers for the per-stage permutation):
//   y[nv][n]      state: x^i, u^i, S, Pi/sigma, pi^{ij}/sigma (xx, xy, yy)
//   Nq[3][n]      charges per particle (constant without diffusion)
//   id[n]         original particle index of each sorted slot
//   dens[6][n]    sigma*, s, n_B, n_S, n_Q, u^0                 (density pass)
//   eos[11][n]    T, mu_B, mu_S, mu_Q, p, e, p_s, p_nB, p_nS, p_nQ, c_s^2
//   gin[6][n]     X^{ji}/sigma*^2 (xx, xy, yx, yy), u^x/sigma*, u^y/sigma*
//   gout[6][n]    d_x u^x, d_x u^y, d_y u^x, d_y u^y, F^x, F^y  (gradient pass)
//   guess[4][n]   warm start of the EoS Newton: the particle's previous table solution
//                 (T, mu_B, mu_S, mu_Q), T = 0 when the table was not used
// The bucket table of the cell list is indexed by the Morton key of the cell
// coordinates (B bits per dimension, fixed at event creation).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct sph_eos;

namespace sphg {

constexpr double kHbarc = 0.1973269804;  // GeV fm
constexpr double kPi = 3.14159265358979323846;

// per-particle status bits (same values as SPH_PST_* in the public header)
constexpr uint32_t PST_FALLBACK = 1u, PST_OUT_OF_TABLE = 2u, PST_NOCONV = 4u, PST_NONFINITE = 8u,
                   PST_CS2_CAPPED = 16u, PST_SOLVE_FAIL = 32u, PST_BACKUP = 64u;
// event-level device error bits
constexpr uint32_t ERR_CELL_OVERFLOW = 1u;
constexpr uint32_t ERR_PAIR_LIST = 2u;  // a backward pair missing from its partner's forward list

constexpr int kNDens = 6, kNEos = 11, kNGin = 6, kNGout = 6;

// scalars that change while stepping live in device memory, so a captured
// CUDA graph can be replayed without re-instantiation
struct DevScalars {
    double tau;
    double work;       // accumulated longitudinal work integral
    double wr[2];      // work rate of stage 1 and stage 2 of the current step
    long long xmin_enc[3];
    unsigned int status_or;
    unsigned int err_flags;
    long long steps;
    unsigned long long pairs;  // accepted neighbour pairs (self included), summed over stages
    // EoS work actually done, summed over stages: table residual+Jacobian evaluations,
    // 4x4 solves, closed-form g(T) evaluations
    unsigned long long eos_resid, eos_solve, eos_g;
    unsigned long long shell_tests;  // mixed form: candidates that needed the exact FP64 test
    // pair-list neighbour passes (plain 2D): set when a particle's neighbours exceeded the list
    // capacity in this stage (reset with the bounding box; the stage then runs the per-particle
    // passes), and the number of stages that did so
    unsigned int pair_flag;
    unsigned int pair_ovf;
    unsigned int eos_claim;  // particle counter of the lane-refill EoS pass (reset with the bounding box)
    unsigned int pad_;
};

struct EosDev {
    // closed form
    double a0, a1, Tc_GeV, w_GeV, chi[3];
    // table: sn[node] = {s, nB, nS, nQ}, p[node]; node = ((iT*n1 + iB)*n2 + iS)*n3 + iQ
    int has_table, nT, nmu[3], maxit;
    int polish;  // 1: one Newton step after convergence (the plain form); 0: stop at the tolerance
    // backup EoS where neither the table nor the closed form inverts: the conformal diagonal
    // p = cd_A0 [T^4 + sum_q (mu_q / cd_mu0[q])^4] (backup = 0: none)
    int backup;
    double cd_A0, cd_mu0[3];
    double T0, dT, mu0[3], dmu[3], inv_dT, inv_dmu[3], Tmax, mumax[3];
    const double *sn;
    const double *p;
    double tol;
    // offline inverter (Sec. "Equation of state"): (T, mu) on a grid in s (log decades,
    // node i at s_i = inv_p10[i / inv_K] (1 + 9 (i % inv_K) / inv_K)) times the charge ratios
    // n_q / s (inv_nx nodes on [-inv_xmax, inv_xmax]); used when offline = 1
    const double *inv;
    const double *inv_p10;
    int inv_K, inv_nd, inv_nx, offline;
    double inv_xmax;
};

struct TransportDev {
    int viscous;
    double eta_over_s, zeta_peak, zeta_T_GeV, zeta_w_GeV, tau_pi_coef, tau_Pi_ratio, cs2_cap;
    // temperature (GeV) below which a particle leaves the fluid and streams freely (0: off)
    double T_stop_GeV;
    // viscous equations of motion: 0 minimal Israel-Stewart, 1 DNMR (shear and bulk J terms,
    // phi_7) with the ratios delta_PiPi/tau_Pi, lambda_Pipi/(tau_Pi (1/3 - c_s^2)),
    // delta_pipi/tau_pi, tau_pipi/tau_pi, lambda_piPi/tau_pi, phi_7 p
    int model;
    double dnmr[6];
};

// everything a kernel of one event needs, passed by value
struct EvView {
    int n, dim, milne, nv, B;
    int B3[3];                // 3D: bits of the cell coordinate per axis
    const uint32_t *spread;   // 3D: spread[d * 1024 + c] = key bits of cell coordinate c on axis d
    double h, inv_h, supp2, inv_cell, sigma_d, dtau;
    float supp2_hi;  // single-precision prefilter bound, >= (2h)^2 plus the worst rounding error
    float supp2_lo;  // below it the float r^2 proves r < 2h: the exact FP64 test is skipped
    int mixed;                 // 1: neighbour passes in FP32 with compensated sums (2D)
    float cell_f;              // mixed: cell side 2h in single precision
    float shell_lo, shell_hi;  // mixed: float r^2 below lo is inside, above hi outside, else FP64 test
    DevScalars *sc;
    EosDev eos;
    TransportDev tr;
    // energy-momentum source of jet tracks (Cartesian events; ntrack = 0: none): tracks[8 k ..]
    // = x0, y0, z0, n_x, n_y, n_z, t0, dE/dx; the Gaussian's 1/((2 pi)^{3/2} sigma^3), 1/(2 sigma^2)
    int ntrack;
    const double *tracks;
    double track_norm, track_i2s2;
    // dynamical-initialisation partons (nparton = 0: none), sorted by formation time:
    // partons[8 k ..] = x^0_k, position (x, y, z|eta), p^mu; the kernel of width parton_h
    int nparton;
    const double *partons;
    double parton_norm, parton_h, parton_sd, parton_dt;  // parton_sd: the kernel normalisation
    // charge sources: the partons' (B, S, Q) in the partons' order (nullptr: none; the
    // particles' charges then stay constant).  With them the equations of motion integrate the
    // charges: nq_cur (the stage state's) -> nq_out, stage 1 nq_out = nq_cur + dt dN_q/dx0,
    // stage 2 nq_out = ((nq_out + nq_cur) + dt dN_q/dx0) / 2 (nq_out holding the step's start)
    const double *parton_q;
    const double *nq_cur;
    double *nq_out;
    // BSQ diffusion (2+1D; diff = 0: none): kappa_{qq'} / T^2 (row q), tau_q T; per stage, in the
    // stage's sorted order: dinp[9][n] = alpha_q = mu_q / T (rows 0-2) and the lab-charge flux
    // (J^i_q - v^i J^0_q) / sigma*^2 (rows 3 + 2 q + i); dal[12][n] = d alpha_q / d(s, n_B, n_S,
    // n_Q) (row 4 q + k); dout[9][n] = d_i alpha_q (rows 2 q + i, the SPH difference form) and
    // the lab-charge rate of the flux divergence (rows 6 + q).  The state carries J^i_q / sigma
    // in rows 9 + 2 q + i.
    int diff;
    double kapT2[9], tauJT[3];
    double *dinp, *dal, *dout;
};
constexpr int kJRow = 9;  // first state row of the diffusion currents (2+1D)

// I^nu of the jet tracks at time t and position (x, y, z): every track moves at the speed of
// light from x0 along n from t0 and deposits dE/dx per unit path length into a normalised
// Gaussian around its current position, with the momentum of light moving along n
// (eq. conservation_source with I^nu != 0)
__device__ __forceinline__ void jet_deposit(const EvView &v, double t, double x, double y, double z, double I[4])
{
    I[0] = I[1] = I[2] = I[3] = 0.0;
    for (int k = 0; k < v.ntrack; ++k) {
        const double *tr = v.tracks + 8 * k;
        const double dt = t - tr[6];
        if (dt < 0.0) continue;
        const double cx = x - (tr[0] + tr[3] * dt), cy = y - (tr[1] + tr[4] * dt), cz = z - (tr[2] + tr[5] * dt);
        const double dep = tr[7] * v.track_norm * exp(-(cx * cx + cy * cy + cz * cz) * v.track_i2s2);
        I[0] += dep;
        I[1] += dep * tr[3];
        I[2] += dep * tr[4];
        I[3] += dep * tr[5];
    }
}

// ---------------------------------------------------------------------------
// order-preserving map of doubles to signed 64-bit integers (for atomicMin)
__device__ __forceinline__ long long enc_double(double x)
{
    long long i = __double_as_longlong(x);
    return i >= 0 ? i : (i ^ 0x7FFFFFFFFFFFFFFFLL);
}
__host__ __device__ __forceinline__ double dec_double(long long i)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(i >= 0 ? i : (i ^ 0x7FFFFFFFFFFFFFFFLL));
#else
    long long j = i >= 0 ? i : (i ^ 0x7FFFFFFFFFFFFFFFLL);
    double d;
    memcpy(&d, &j, 8);
    return d;
#endif
}

// Morton key: bit (2b + d) of the key is bit b of coordinate d
__host__ __device__ __forceinline__ uint32_t spread2(uint32_t v)
{
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ __forceinline__ uint32_t morton2(uint32_t cx, uint32_t cy) { return spread2(cx) | (spread2(cy) << 1); }

// cell coordinate floor((x - xmin) * (1/(2h))): a single rounded subtraction and
// product, the same two operations on every platform
__device__ __forceinline__ int cell_coord(double x, double xmin, double inv_cell)
{
    return (int)floor(__dmul_rn(__dsub_rn(x, xmin), inv_cell));
}

// r^2 with each product rounded separately (no fused multiply-add), so the
// neighbour decision r^2 < (2h)^2 is bit-for-bit reproducible
__device__ __forceinline__ double dist2_2d(double dx, double dy) { return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)); }

// the same in three dimensions
__device__ __forceinline__ double dist2_3d(double dx, double dy, double dz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// 3D cell key: the generalized Morton interleave of the per-axis bits (spread tables)
__device__ __forceinline__ uint32_t key3(const EvView &v, int cx, int cy, int cz)
{
    return v.spread[cx] | v.spread[1024 + cy] | v.spread[2048 + cz];
}

// 1/sqrt(x) for x > 0 in double precision: CUDA's rsqrt (at most 1 ulp of error)
__device__ __forceinline__ double inv_sqrt(double x) { return rsqrt(x); }

// Single-precision square root and reciprocal square root as the approximate PTX instructions
// with denormal inputs flushed to zero: one MUFU operation each, relative error about 2^-22
// (the FP32 neighbour passes, whose kernel values carry that error anyway)
__device__ __forceinline__ float sqrt_apx(float x)
{
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_apx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Exact bit-level helpers that keep work off the FP64 pipe (1/64 of the FP32 rate on GB300):
// x != 0 for x >= 0 (true when any bit is set; +0 is all zero bits)
__device__ __forceinline__ bool nonzero_nonneg(double x) { return __double_as_longlong(x) != 0LL; }
// max(x, 0) for finite x, from the sign bit
__device__ __forceinline__ double pos_part(double x)
{
    const long long b = __double_as_longlong(x);
    return __longlong_as_double(b & ~(b >> 63));
}
// x / 4 for x = 0 or x >= 2^-1020, by lowering the exponent field by 2 (exact)
__device__ __forceinline__ double quarter_nonneg(double x)
{
    return __hiloint2double(max(__double2hiint(x) - 0x00200000, 0), __double2loint(x));
}

// Warp sum of up to 8 per-lane values by recursive halving (a reduce-scatter): at each of the
// first three levels a lane keeps half of its values and adds its partner's copy of them, then
// two butterfly levels finish one value.  9 additions per lane instead of 5 per value for a full
// butterfly -- on the 1:64 FP64 pipe a warp-wide addition costs as much as 32 lanes of pair
// work.  Returns, in lanes 4k .. 4k+3, the warp total of v[k]; the order of the additions is
// fixed, so results are reproducible.
__device__ __forceinline__ double warp_reduce_scatter8(const double (&v)[8], int lane)
{
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    double h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const double keep = b4 ? v[4 + i] : v[i], give = b4 ? v[i] : v[4 + i];
        h[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, give, 16);
    }
    double g[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const double keep = b3 ? h[2 + i] : h[i], give = b3 ? h[i] : h[2 + i];
        g[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, give, 8);
    }
    double f = (b2 ? g[1] : g[0]) + __shfl_xor_sync(0xFFFFFFFFu, b2 ? g[0] : g[1], 4);
    f += __shfl_xor_sync(0xFFFFFFFFu, f, 2);
    f += __shfl_xor_sync(0xFFFFFFFFu, f, 1);
    return f;
}

// cubic spline kernel (Sec. "Kernel function") as functions of q = r/h:
// W = sigma_d w(q), dW/dr = sigma_d/h w'(q)
__device__ __forceinline__ double kernel_w(double q)
{
    if (q <= 1.0) return fma(q * q, fma(0.75, q, -1.5), 1.0);
    double t = 2.0 - q;
    return 0.25 * t * t * t;
}
__device__ __forceinline__ double kernel_dw(double q)
{
    if (q <= 1.0) return q * fma(2.25, q, -3.0);
    double t = 2.0 - q;
    return -0.75 * t * t;
}

// I^mu (and I_q) of the partons formed in (t - dt, t] (Sec. "Dynamical initialization"):
// N p^mu W(r - r_k, h_src) / (sqrt(-g) dt), distances in the event's dim coordinates; the
// window is found by binary search in the formation times
__device__ __forceinline__ void parton_deposit(const EvView &v, double t, double sqrtg, const double *x,
                                               double I[4], double Iq[3])
{
    I[0] = I[1] = I[2] = I[3] = 0.0;
    Iq[0] = Iq[1] = Iq[2] = 0.0;
    const double lo_t = t - v.parton_dt;
    int lo = 0, hi = v.nparton;  // first parton with x^0 > t - dt
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v.partons[8 * mid] > lo_t) hi = mid;
        else lo = mid + 1;
    }
    const double f0 = v.parton_norm * v.parton_sd / (sqrtg * v.parton_dt), ih = 1.0 / v.parton_h;
    for (int k = lo; k < v.nparton; ++k) {
        const double *q = v.partons + 8 * k;
        if (q[0] > t) break;
        double r2 = 0.0;
        for (int d = 0; d < v.dim; ++d) r2 += (x[d] - q[1 + d]) * (x[d] - q[1 + d]);
        const double qq = sqrt(r2) * ih;
        if (!(qq < 2.0)) continue;
        const double w = f0 * kernel_w(qq);
        I[0] += w * q[4];
        I[1] += w * q[5];
        I[2] += w * q[6];
        I[3] += w * q[7];
        if (v.parton_q) {  // the charge source I_q: the parton's (B, S, Q) with the same weight
            const double *c = v.parton_q + 3 * k;
            Iq[0] += w * c[0];
            Iq[1] += w * c[1];
            Iq[2] += w * c[2];
        }
    }
}

// Heun step of the particle's charges under charge sources (v.nq_out set): stage 1 (mode 0)
// nq_out = nq_cur + dt dN, stage 2 (mode 1) nq_out = ((nq_out + nq_cur) + dt dN) / 2
__device__ __forceinline__ void heun_charges(const EvView &v, int mode, size_t n, size_t a, const double dN[3])
{
    if (!v.nq_out || mode > 1) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double cur = v.nq_cur[c * n + a];
        double *o = v.nq_out + c * n + a;
        *o = mode == 0 ? cur + v.dtau * dN[c] : 0.5 * ((*o + cur) + v.dtau * dN[c]);
    }
}

// affine form c + ax*a_x + ay*a_y in the unknown acceleration (a_x, a_y)
struct Aff {
    double c, x, y;
};
__device__ __forceinline__ Aff aff(double c) { return {c, 0.0, 0.0}; }
__device__ __forceinline__ Aff operator+(Aff a, Aff b) { return {a.c + b.c, a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ Aff operator-(Aff a, Aff b) { return {a.c - b.c, a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ Aff operator-(Aff a) { return {-a.c, -a.x, -a.y}; }
__device__ __forceinline__ Aff operator*(double s, Aff a) { return {s * a.c, s * a.x, s * a.y}; }
__device__ __forceinline__ Aff operator*(Aff a, double s) { return {s * a.c, s * a.x, s * a.y}; }
__device__ __forceinline__ Aff operator+(Aff a, double s) { return {a.c + s, a.x, a.y}; }
__device__ __forceinline__ double at(Aff a, double ax, double ay) { return fma(a.x, ax, fma(a.y, ay, a.c)); }

// warp-aggregated OR into a global word
__device__ __forceinline__ void warp_or(unsigned int *dst, unsigned int v)
{
    unsigned int m = __reduce_or_sync(__activemask(), v);
    if (m && (threadIdx.x & 31) == (__ffs(__activemask()) - 1)) atomicOr(dst, m);
}

// ---------------------------------------------------------------------------
// launchers (implemented in cells.cu, density_eos.cu, gradient_eom.cu)
// Half-pair lists of the plain 2D neighbour passes, rebuilt in every stage's density pass.
// Particle a (sorted index) owns entries [off[a], off[a+1]) of L, P, W, FAC, sized by its
// neighbour count of the previous stage plus a margin (a prefix scan per stage):
//   from the row start: its accepted neighbours b > a, ascending (L), with W(r)/sigma_d of the
//      pair (W) and grad_a W_ab h/sigma_d = (dW/dr)/r (x_a - x_b) h/sigma_d (G); both are
//      computed once per pair (W is symmetric in a, b; grad_b W_ba = -grad_a W_ab);
//   from the row end, downwards: its accepted neighbours b < a, ascending (L), with the slot of
//      the pair (b, a) in b's row (P).
// A particle whose neighbours exceed its row (or rows beyond the allocation) flags the stage,
// which then runs the per-particle passes; the counts it records size the next stage's rows.
// total = 0: lists off (the per-particle passes run).
struct PairBufs {
    long long total;              // entries allocated
    int margin;                   // entries added to each particle's previous count
    const int *cnt_src;           // previous counts (self included), state order (read through perm)
    int *cnt_dst;                 // this stage's counts, sorted order (NULL: not recorded)
    long long *off;               // [n + 1] row offsets of this stage
    unsigned long long *part;     // scan partial sums
    int *L, *P, *cntF, *cntB;
    double *W;
    double2 *G;   // 2D
    double *G3;   // 3D: three components per entry
};

struct CellBufs {
    uint32_t *key, *cnt, *start, *cursor, *tmp, *perm;
    float2 *fpos;   // 2D: sorted positions relative to the bounding-box minimum, single precision
    float4 *fpos3;  // 3D: the same with three coordinates
    uint32_t *part; // scan partial sums (multi-block scan of large bucket tables)
    int nb;         // number of buckets: 1 << (2 B) in 2D, 1 << (B3[0] + B3[1] + B3[2]) in 3D
    PairBufs pl;    // plain 2D: half-pair lists (pl.total = 0: off)
};

// Bound for the single-precision candidate prefilter of the neighbour passes.  With
// positions p = fl(x - xmin) in [0, L], L = 2^B * 2h (beyond it the cell table overflows
// and the step fails), |fl(p) - p| <= L u and |fl(pa - pb) - (pa - pb)| <= 2 L u + 4h u
// (u = 2^-24); for a true neighbour (|dx_d| <= 2h) the squared distance summed over two
// axes then errs by at most 4 (2h) e + 2 e^2 + 4 u (2h)^2 with e the difference error.
// Twice that margin is added, so the prefilter never rejects a pair the exact
// double-precision test r^2 < (2h)^2 accepts; the exact test decides every pair.
// The same margin below (2h)^2 gives the lower bound: a float r^2 under it proves r < 2h (for
// |dx_d| near 2h the error is at most err; farther candidates have r^2 - (2h)^2 much larger
// than their error), so those pairs skip the exact test and the neighbour set is unchanged.
inline void prefilter_bounds(double h, int B, int dim, float &lo_out, float &hi_out)
{
    const double u = 1.0 / 16777216.0;
    const double two_h = 2.0 * h;
    const double L = (double)(1 << B) * two_h;
    const double e = 2.0 * L * u + 2.0 * two_h * u + L * u;
    const double err = 2.0 * dim * two_h * e + dim * e * e + (dim + 2) * u * two_h * two_h;
    const double hi = two_h * two_h + 2.0 * err, lo = two_h * two_h - 2.0 * err;
    float f = (float)hi;
    while ((double)f < hi) f = nextafterf(f, 1e30f);
    float g = (float)lo;
    while ((double)g > lo) g = nextafterf(g, 0.0f);
    hi_out = f;
    lo_out = g;
}
inline float prefilter_bound(double h, int B, int dim = 2)
{
    float lo, hi;
    prefilter_bounds(h, B, dim, lo, hi);
    return hi;
}

void launch_bbox(const EvView &v, const double *y, cudaStream_t st);
void launch_cells(const EvView &v, const double *y, const int *id, CellBufs cb, cudaStream_t st);
void launch_permute(const EvView &v, const uint32_t *perm, const double *const *src, double *const *dst,
                    const int *nrows, int ngroups, const int *id_in, int *id_out, cudaStream_t st);
// plain 2D neighbour passes over the half-pair lists (cb.pl.total > 0): row offsets from the
// previous counts, then the forward and backward density passes
void launch_pairs_density(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                          cudaStream_t st);
void launch_pairs_gradient(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb,
                           double *gout, cudaStream_t st);
// the per-stage row offsets of the pair lists (prefix scan of the carried counts)
void launch_pair_rows(const EvView &v, CellBufs cb, cudaStream_t st);
// plain 3D neighbour passes over the half-pair lists (after k_fpos3 and the row offsets)
void launch_pairs3_density(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                           cudaStream_t st);
void launch_pairs3_gradient(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb,
                            double *gout, cudaStream_t st);
void launch_density(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                    cudaStream_t st);
void launch_eos(const EvView &v, int stage, const double *y, const double *dens, double *eos, double *gin,
                uint32_t *status, double *wpart, const double *guess_in, double *guess_out, cudaStream_t st);
void launch_gradient(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                     cudaStream_t st);
// mode 0: y1 = y + dt f(y); mode 1: y0 = ((y0 + y1) + dt f(y1)) / 2 in place; mode 2: rates only
void launch_eom(const EvView &v, int stage, int mode, const double *ys, const double *dens, const double *eos,
                const double *gout, double *yout, double *rates, uint32_t *status, cudaStream_t st);
void launch_work_finish(const EvView &v, int stage, const double *wpart, int nblk, cudaStream_t st);
void launch_neighbors_list(const EvView &v, const double *y, const int *id, CellBufs cb, const long long *offs,
                           int *pa, int *pb, cudaStream_t st);
void launch_scan_counts(const int *cnt, long long *offs, int n, cudaStream_t st);
void launch_totals(const EvView &v, const double *y, const double *Nq, const int *id, const double *dens,
                   const double *eos, double *contrib, cudaStream_t st);
void launch_sum_fixed(const double *vals, int n, int nfield, double *out, cudaStream_t st);
void launch_scatter_orig(const double *src, double *dst, const int *id, int n, int nrows, cudaStream_t st);
void launch_scatter_orig_u32(const uint32_t *src, uint32_t *dst, const int *id, int n, cudaStream_t st);
void launch_cell_coords(const EvView &v, const double *y, const int *id, int *cell_orig, cudaStream_t st);
int device_sm_count();  // SMs of the current device (cached after the first call)
int eos_block_count(int n, int dim);  // blocks of the EoS pass (entries of its work-rate partials)

// mixed-precision 2D neighbour passes (mixed2d.cu); dispatched when v.mixed
void launch_density2m(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                      cudaStream_t st);
void launch_gradient2m(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                       cudaStream_t st);

// Shell of the mixed-form neighbour decision.  Cell-relative positions are floats in
// [0, 2h] (error <= 2h u each, u = 2^-24); the separation (r_a - r_b) - o 2h (|o| <= 1,
// 2h itself rounded) errs by e <= 6 (2h) u per axis; for |dx_d| <= 2h the float r^2
// (fmaf) errs by at most 2 dim (2h) e + dim e^2 + 2 u (2h)^2 <= 26 (2h)^2 u in 2D.  Twice
// that margin on each side: outside [lo, hi] the float decision equals the exact one.
inline void mixed_shell(double h, float &lo, float &hi)
{
    const double u = 1.0 / 16777216.0;
    const double s2 = 4.0 * h * h;
    const double err = 52.0 * s2 * u;
    float l = (float)(s2 - err), g = (float)(s2 + err);
    while ((double)l > s2 - err) l = nextafterf(l, 0.0f);
    while ((double)g < s2 + err) g = nextafterf(g, 1e30f);
    lo = l;
    hi = g;
}

// The same for 3+1D: three axes, so the float r^2 (nested fmaf) errs by at most
// 2 dim (2h) e + dim e^2 + 6 u (2h)^2 <= 42 (2h)^2 u with e <= 6 (2h) u; the shell is
// +-96 (2h)^2 u.
inline void mixed_shell3(double h, float &lo, float &hi)
{
    const double u = 1.0 / 16777216.0;
    const double s2 = 4.0 * h * h;
    const double err = 96.0 * s2 * u;
    float l = (float)(s2 - err), g = (float)(s2 + err);
    while ((double)l > s2 - err) l = nextafterf(l, 0.0f);
    while ((double)g < s2 + err) g = nextafterf(g, 1e30f);
    lo = l;
    hi = g;
}
void launch_density3m(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                      cudaStream_t st);
void launch_gradient3m(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                       cudaStream_t st);

// 3D versions (step3d.cu); the launchers above dispatch to them when v.dim == 3
void launch_cells3(const EvView &v, const double *y, const int *id, CellBufs cb, cudaStream_t st);
void launch_density3(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                     cudaStream_t st);
void launch_eos3(const EvView &v, int stage, const double *y, const double *dens, double *eos, double *gin,
                 uint32_t *status, double *wpart, const double *guess_in, double *guess_out, cudaStream_t st);
void launch_gradient3(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                      cudaStream_t st);
void launch_eom3(const EvView &v, int stage, int mode, const double *ys, const double *dens, const double *eos,
                 const double *gout, double *yout, double *rates, uint32_t *status, cudaStream_t st);
void launch_totals3(const EvView &v, const double *y, const int *id, const double *dens, const double *eos,
                    double *contrib, cudaStream_t st);
void launch_neighbors_list3(const EvView &v, const double *y, const int *id, CellBufs cb, const long long *offs,
                            int *pa, int *pb, cudaStream_t st);
void launch_cell_coords3(const EvView &v, const double *y, const int *id, int *cell_orig, cudaStream_t st);
// exclusive scan of cnt into start and cursor, any number of buckets
void launch_scan_buckets(CellBufs cb, cudaStream_t st);

// ---------------------------------------------------------------------------
// Serving form (serve.cu): many 2+1D events advance together in one segmented particle
// arena.  Each admitted event owns the range [off, off + cap) of every per-particle row
// (row stride P, the arena capacity); off and cap are multiples of kSegAlign, so a warp
// (and a 256-particle chunk) never straddles two events.  Every kernel reads the slot
// table from device memory and loops over the arena with a fixed grid, so one captured
// CUDA graph serves every batch composition.
constexpr int kSegAlign = 256;
constexpr int kMaxSlots = 256;
constexpr int kMaxCellsAxis = 256;  // an event's cell grid clamps here (neighbour sets stay complete)
constexpr int SLOT_FREE = 0, SLOT_STEP = 1, SLOT_OBSERVE = 2;

struct SegSlot {  // host-written at step boundaries
    int mode;     // SLOT_FREE, SLOT_STEP (advance one step), SLOT_OBSERVE (stage-1 evaluation only)
    int off, n, cap;
};
struct SegGrid {  // device-written, per slot and stage: bounding box and cell grid
    long long bb[4];  // order-preserving encodings of x_min, y_min, x_max, y_max
    double x0, y0;    // grid origin (the bounding-box minimum)
    int nx, ny, base, ncell;
};
struct BatchTable {  // host-written
    int hi;          // arena high-water mark: every kernel loops over [0, hi)
    int nslots;      // slots in use (table length)
    int split;       // first slot of event group 1 (groups: slots [0, split) and [split, nslots))
    int pad;
    SegSlot slots[kMaxSlots];
};
struct Arena {
    int P, cmax;  // particle and cell capacity
    int lane_warps;  // tiled neighbour passes: warps whose lanes share a cell's particles (the tuned shape)
    unsigned int *hflags;  // mapped pinned host words: per slot, its status OR after each batch step
    double *wchunk;        // per slot, partial sums of the work rates over fixed chunks of its range
    double *Y[2], *Y1[2], *Nq[2];
    int *id[2];
    double *wguess, *guess_in;
    double *xs1[2];  // the previous step's stage-1 table solution (T = 0: none), ping-pong with the sorts
    int *segid;  // slot of every arena position of an event's range (padding included)
    double *dens, *eosf, *gin, *gout;
    uint32_t *status;
    int *nnb;
    double *wpart;  // per particle: work rate of the EoS pass (summed per event in a fixed order)
    uint32_t *key, *rnk, *tmp, *perm;
    uint32_t *cnt, *start, *scan_part;
    // single-precision copies for the neighbour passes, written once per particle and stage:
    // position relative to the origin of the particle's cell, (S, N_B, N_S, N_Q), and the
    // gradient-pass inputs X^{xx}, X^{xy}, X^{yx}, X^{yy} and u^x/sigma*, u^y/sigma*
    float2 *fpos;
    float4 *fq, *fX;
    float2 *fU;
    int *ncells;  // device-written: [0] the active slots' cells, [1] those of event group 0
    unsigned int *claim;  // work counters of the dynamically scheduled passes (reset per stage)
    BatchTable *tab;
    SegGrid *grid;
    EvView *segv;
    DevScalars *sc;
};
// work counters of the dynamically scheduled passes; event group g (0 or 1) uses index + 4 g
constexpr int CLAIM_EOS = 0, CLAIM_DENSITY = 1, CLAIM_GRADIENT = 2, kClaims = 8;
__device__ __forceinline__ int claim_of(int which, int grp) { return which + (grp > 0 ? 4 : 0); }
// slot s in event group grp (grp < 0: every slot)
__device__ __forceinline__ bool in_group(const BatchTable *t, int s, int grp)
{
    return grp < 0 || ((s >= t->split) == (grp > 0));
}
// slot s takes part in this stage's pass: stage 1 evaluates STEP and OBSERVE slots, stage 2
// and the rate passes (gradient, equations of motion, work) only STEP slots
__device__ __forceinline__ bool seg_active(const BatchTable *t, int s, int stage, bool rates)
{
    const int m = t->slots[s].mode;
    return m == SLOT_STEP || (m == SLOT_OBSERVE && stage == 1 && !rates);
}

// Shell of the cell-tiled mixed-form decision (cells of side h, a 5x5 search block).  A
// particle's position relative to its own cell's origin, in [0, h) per axis, is rounded to
// float (error <= h u, u = 2^-24); a candidate k cells away (|k| <= 2) adds k times the
// float cell side (error <= 2h u) in one float addition (result <= 3h: error <= 3h u).  So
// x_a carries <= h u, x_b <= 6h u, and the float separation of a pair with |dx_d| <= 2h errs
// by e <= 9h u = 4.5 (2h) u per axis (the subtraction included).  The float r^2 (fmaf) then
// errs by at most 4 (2h) e + 2 e^2 + 3 u (2h)^2 <= 22 (2h)^2 u near r = 2h, and the margin
// r^2 - (2h)^2 grows faster than the error beyond it.  The shell is +-64 (2h)^2 u: outside it
// the float decision equals the exact one.  A grid clamped at kMaxCellsAxis cells puts far
// particles into its edge cells, where the bound does not hold; such cells use the FP64 test
// for every candidate.
inline void tiled_shell(double h, float &lo, float &hi)
{
    const double u = 1.0 / 16777216.0;
    const double s2 = 4.0 * h * h;
    const double err = 64.0 * s2 * u;
    float l = (float)(s2 - err), g = (float)(s2 + err);
    while ((double)l > s2 - err) l = nextafterf(l, 0.0f);
    while ((double)g < s2 + err) g = nextafterf(g, 1e30f);
    lo = l;
    hi = g;
}

// offline inverter: fills the inverted table of E's grid (density_eos.cu)
void launch_inverse_build(const EosDev &E, double *inv, long long nnodes, cudaStream_t st);

// EoS handle accessors (api.cu)
EosDev eos_params(const ::sph_eos *e);
void eos_retain(::sph_eos *e);

// grp: the event group the pass covers (-1: every event)
void launch_eos2_seg(const Arena &A, const EosDev &E, int stage, const double *y, int grid, cudaStream_t st,
                     int grp = -1);
int eos_seg_grid(int sms);  // persistent grid of the serving EoS pass
// BSQ diffusion inputs and neighbour sums of a stage (2+1D; after the EoS pass)
void launch_diffusion(const EvView &v, int stage, const double *y, const double *dens, const double *eos,
                      const uint32_t *status, CellBufs cb, cudaStream_t st);
void launch_eom2_seg(const Arena &A, int stage, int mode, const double *ys, double *yout, int grid,
                     cudaStream_t st, int grp = -1);

// freeze-out surface elements (freezeout.cu): records of kFoRec doubles
// (tau, x^1..3, u^0..3, T, mu_B, mu_S, mu_Q, e, p, s, n_0..3, |dsigma|, dsigma_0..3)
constexpr int kFoRec = 24;
struct FoBuf {
    double *rec;
    long long *ids;
    unsigned long long *count;
    unsigned long long cap;
};
void launch_freezeout(const EvView &v, double e_fo, const double *y, const int *id, const double *dens,
                      const double *eosf, double *eprev, CellBufs cb, FoBuf fo, cudaStream_t st);

// sets the message returned by sph_last_error() for the calling thread
void set_last_error(const char *msg);

}  // namespace sphg
