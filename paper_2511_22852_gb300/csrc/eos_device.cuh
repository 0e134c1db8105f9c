// eos_device.cuh -- device code of the EoS inversion (row a4), shared by the 2+1D and
// 3+1D EoS passes: closed-form EoS, quadrilinear table interpolation with derivatives,
// the damped table Newton, and the warm-started inversion (Sec. "EoS inverter").
#pragma once
#include "sph_internal.cuh"

namespace sphg {
namespace {

// closed-form EoS
__device__ __forceinline__ void an_shape(const EosDev &E, double T, double &f, double &fp, double &fpp)
{
    double k = kHbarc / E.w_GeV;
    double th = tanh((T * kHbarc - E.Tc_GeV) / E.w_GeV);
    double sech2 = fma(-th, th, 1.0);
    f = E.a0 + 0.5 * E.a1 * (1.0 + th);
    fp = 0.5 * E.a1 * sech2 * k;
    fpp = -E.a1 * sech2 * th * k * k;
}

__device__ void an_eval(const EosDev &E, double T, const double *mu, double &p, double sn[4], double H[4][4])
{
    double f, fp, fpp;
    an_shape(E, T, f, fp, fpp);
    double cm2 = E.chi[0] * mu[0] * mu[0] + E.chi[1] * mu[1] * mu[1] + E.chi[2] * mu[2] * mu[2];
    double T2 = T * T, T3 = T2 * T, T4 = T2 * T2;
    p = T4 * f + 0.5 * T2 * cm2;
    sn[0] = 4.0 * T3 * f + T4 * fp + T * cm2;
    for (int q = 0; q < 3; ++q) sn[1 + q] = E.chi[q] * T2 * mu[q];
    H[0][0] = 12.0 * T2 * f + 8.0 * T3 * fp + T4 * fpp + cm2;
    for (int q = 0; q < 3; ++q) {
        double c = 2.0 * E.chi[q] * T * mu[q];
        H[0][1 + q] = c;
        H[1 + q][0] = c;
        for (int r = 0; r < 3; ++r) H[1 + q][1 + r] = (q == r) ? E.chi[q] * T2 : 0.0;
    }
}

// work counters of one inversion (reported as algorithmic work by the benchmark)
struct EosWork {
    unsigned resid, solve, g;
};

// g(T) = s(T, mu(T)) - s_target with mu_q(T) = n_q/(chi_q T^2)
__device__ __forceinline__ void an_g(const EosDev &E, double T, double s, double c, double &g, double &gp)
{
    double f, fp, fpp;
    an_shape(E, T, f, fp, fpp);
    double T2 = T * T, T3 = T2 * T, T4 = T2 * T2;
    g = 4.0 * T3 * f + T4 * fp + c / T3 - s;
    gp = 12.0 * T2 * f + 8.0 * T3 * fp + T4 * fpp - 3.0 * c / T4;
}

// Tguess > 0: the particle's closed-form T of its previous stage (warm start of the bracket and of
// the Newton iteration; the root is the same)
__device__ uint32_t an_invert(const EosDev &E, double s, const double *n, double &T, double *mu, EosWork &w,
                              double Tguess = 0.0)
{
    if (!isfinite(s) || !isfinite(n[0]) || !isfinite(n[1]) || !isfinite(n[2])) return PST_NONFINITE | PST_NOCONV;
    if (!(s > 0.0)) return PST_NOCONV;
    double c = 0.0;
    for (int q = 0; q < 3; ++q) {
        if (E.chi[q] > 0.0) c += n[q] * n[q] / E.chi[q];
        else if (n[q] != 0.0) return PST_NOCONV;
    }
    double Thi = cbrt(s / (4.0 * E.a0));
    // start: the bound cbrt(s / 4 a0) >= T, or a warm start below it
    const bool warm = Tguess > 0.0 && Tguess < Thi;
    const double t0 = warm ? Tguess : Thi;
    double g, gp;
    an_g(E, t0, s, c, g, gp);
    ++w.g;
    double Tlo = t0;
    if (g > 0.0) {  // the root lies below t0: step down to a lower bracket
        Thi = t0;
        const double f = warm ? 0.99 : 0.8;  // fine steps from a warm start
        double gprev = g;
        bool found = false;
        for (int k = 0; k < 400; ++k) {
            Tlo *= f;
            double gl, gpl;
            an_g(E, Tlo, s, c, gl, gpl);
            ++w.g;
            if (gl <= 0.0) {
                found = true;
                break;
            }
            if (gl > gprev) return PST_NOCONV;
            gprev = gl;
        }
        if (!found) return PST_NOCONV;
    }
    double t = t0;
    for (int it = 0; it < 200; ++it) {
        an_g(E, t, s, c, g, gp);
        ++w.g;
        if (g == 0.0) break;
        if (g > 0.0) Thi = t;
        else Tlo = t;
        double tn = t - g / gp;
        if (!(gp > 0.0) || !(tn > Tlo && tn < Thi)) tn = 0.5 * (Tlo + Thi);
        if (fabs(tn - t) <= 4e-16 * t) {
            t = tn;
            break;
        }
        t = tn;
    }
    T = t;
    for (int q = 0; q < 3; ++q) mu[q] = E.chi[q] > 0.0 ? n[q] / (E.chi[q] * t * t) : 0.0;
    return 0u;
}

// ---------------------------------------------------------------------------
// table: the quadrilinear interpolant reduced one axis at a time (mu_Q, mu_S inside each of the
// four (T, mu_B) corner patches, then mu_B, then T), carrying the partial derivatives along
__device__ __forceinline__ void locate(double x, double x0, double inv, int nx, int &i, double &t)
{
    const double r = (x - x0) * inv;
    // the cell below r: truncation toward zero is the floor for r >= 0, and the clamp to
    // [0, nx - 2] takes every r < 0 to cell 0 as the floor would (no rounding instruction)
    const int k = max(0, min(__double2int_rz(r), nx - 2));
    i = k;
    t = r - (double)k;
}

// sn: interpolated (s, nB, nS, nQ); J[f][k] = d sn_f / d x_k per grid step of axis k (times
// inv_dT, inv_dmu[k-1] for the derivative per unit of x_k); p optional
__device__ void tab_eval_steps(const EosDev &E, const double *x, double sn[4], double J[4][4], double *p)
{
    int iT, iB, iS, iQ;
    double tT, tB, tS, tQ;
    locate(x[0], E.T0, E.inv_dT, E.nT, iT, tT);
    locate(x[1], E.mu0[0], E.inv_dmu[0], E.nmu[0], iB, tB);
    locate(x[2], E.mu0[1], E.inv_dmu[1], E.nmu[1], iS, tS);
    locate(x[3], E.mu0[2], E.inv_dmu[2], E.nmu[2], iQ, tQ);
    const int n3 = E.nmu[2], n23 = E.nmu[1] * E.nmu[2], n123 = E.nmu[0] * n23;
    const size_t node0 = (size_t)iT * n123 + (size_t)iB * n23 + (size_t)iS * n3 + iQ;
    // a node's four fields are 32 contiguous bytes: (s, n_B) and (n_S, n_Q) as two 16-byte loads
    // (the table is a cudaMalloc allocation, 256-byte aligned)
    const double2 *sn2 = reinterpret_cast<const double2 *>(E.sn);
#pragma unroll
    for (int fp = 0; fp < 2; ++fp) {  // a pair of fields at a time: their 16 corner values
        double lv[2][2], lb[2][2], ls[2][2], lq[2][2];  // [field][bT]: after the mu_B reduction
#pragma unroll
        for (int bT = 0; bT < 2; ++bT) {
            double pv[2][2], ps[2][2], pq[2][2];  // [field][bB]: (mu_S, mu_Q) patch value, d/dS, d/dQ
#pragma unroll
            for (int bB = 0; bB < 2; ++bB) {
                const size_t base = node0 + (size_t)bT * n123 + (size_t)bB * n23;
                const double2 q00 = __ldg(sn2 + 2 * base + fp), q01 = __ldg(sn2 + 2 * (base + 1) + fp);
                const double2 q10 = __ldg(sn2 + 2 * (base + n3) + fp), q11 = __ldg(sn2 + 2 * (base + n3 + 1) + fp);
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const double c00 = g ? q00.y : q00.x, c01 = g ? q01.y : q01.x;
                    const double c10 = g ? q10.y : q10.x, c11 = g ? q11.y : q11.x;
                    const double d0 = c01 - c00, d1 = c11 - c10;  // along mu_Q
                    const double a0 = fma(tQ, d0, c00), a1 = fma(tQ, d1, c10);
                    const double ds = a1 - a0;  // along mu_S
                    pv[g][bB] = fma(tS, ds, a0);
                    ps[g][bB] = ds;
                    pq[g][bB] = fma(tS, d1 - d0, d0);
                }
            }
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                const double db = pv[g][1] - pv[g][0];  // along mu_B
                lv[g][bT] = fma(tB, db, pv[g][0]);
                lb[g][bT] = db;
                ls[g][bT] = fma(tB, ps[g][1] - ps[g][0], ps[g][0]);
                lq[g][bT] = fma(tB, pq[g][1] - pq[g][0], pq[g][0]);
            }
        }
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            const int f = 2 * fp + g;
            const double dt = lv[g][1] - lv[g][0];  // along T
            sn[f] = fma(tT, dt, lv[g][0]);
            J[f][0] = dt;
            J[f][1] = fma(tT, lb[g][1] - lb[g][0], lb[g][0]);
            J[f][2] = fma(tT, ls[g][1] - ls[g][0], ls[g][0]);
            J[f][3] = fma(tT, lq[g][1] - lq[g][0], lq[g][0]);
        }
    }
    if (p) {
        double lp[2];
#pragma unroll
        for (int bT = 0; bT < 2; ++bT) {
            double pb[2];
#pragma unroll
            for (int bB = 0; bB < 2; ++bB) {
                const size_t base = node0 + (size_t)bT * n123 + (size_t)bB * n23;
                const double p00 = __ldg(E.p + base), p01 = __ldg(E.p + base + 1);
                const double p10 = __ldg(E.p + base + n3), p11 = __ldg(E.p + base + n3 + 1);
                const double a0 = fma(tQ, p01 - p00, p00), a1 = fma(tQ, p11 - p10, p10);
                pb[bB] = fma(tS, a1 - a0, a0);
            }
            lp[bT] = fma(tB, pb[1] - pb[0], pb[0]);
        }
        *p = fma(tT, lp[1] - lp[0], lp[0]);
    }
}

// the same with the derivatives per unit of (T, mu_B, mu_S, mu_Q)
__device__ void tab_eval(const EosDev &E, const double *x, double sn[4], double J[4][4], double *p)
{
    tab_eval_steps(E, x, sn, J, p);
    const double sc[4] = {E.inv_dT, E.inv_dmu[0], E.inv_dmu[1], E.inv_dmu[2]};
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int k = 0; k < 4; ++k) J[f][k] *= sc[k];
}

// 4x4 Gaussian elimination with partial pivoting, fully unrolled so every index is a
// compile-time constant and the system stays in registers.  Row swaps are conditional
// moves; each pivot is inverted once (FP64 division is a multi-instruction sequence on
// the 1:64 FP64 pipe) and the back substitution multiplies by it.  Returns false on a
// zero or non-finite pivot.
// magnitude of a double as an integer: for non-negative doubles the IEEE bit patterns order as
// the values do (NaN above infinity), so the pivot search compares integers
__device__ __forceinline__ long long mag_bits(double v) { return __double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFLL; }
constexpr long long kInfBits = 0x7FF0000000000000LL;

__device__ __forceinline__ bool solve4(double A[4][4], double b[4])
{
    double ipv[4];  // reciprocal pivots, reused by the back substitution
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        long long best = mag_bits(A[c][c]);
#pragma unroll
        for (int r = c + 1; r < 4; ++r) {
            const long long v = mag_bits(A[r][c]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (best == 0 || best >= kInfBits) return false;  // zero, infinite or NaN pivot
#pragma unroll
        for (int r = c + 1; r < 4; ++r) {
            if (piv == r) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    double t = A[c][k];
                    A[c][k] = A[r][k];
                    A[r][k] = t;
                }
                double t = b[c];
                b[c] = b[r];
                b[r] = t;
            }
        }
        double inv = 1.0 / A[c][c];
        ipv[c] = inv;
#pragma unroll
        for (int r = c + 1; r < 4; ++r) {
            double f = A[r][c] * inv;
#pragma unroll
            for (int k = c; k < 4; ++k) A[r][k] = fma(-f, A[c][k], A[r][k]);
            b[r] = fma(-f, b[c], b[r]);
        }
    }
#pragma unroll
    for (int r = 3; r >= 0; --r) {
        double acc = b[r];
#pragma unroll
        for (int k = r + 1; k < 4; ++k) acc = fma(-A[r][k], b[k], acc);
        b[r] = acc * ipv[r];
    }
    return true;
}

// order-preserving integer key of a double (its own inverse): negative values have their
// magnitude bits flipped, so signed integer comparisons order keys as the values
__device__ __forceinline__ long long okey(double v)
{
    const long long b = __double_as_longlong(v);
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}
__device__ __forceinline__ double clamp_key(double v, double lo, double hi)
{
    const long long k = min(max(okey(v), okey(lo)), okey(hi));
    return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL));
}

// the point into the table's box (exact: a comparison and a selection per bound, on integers)
__device__ __forceinline__ void clamp4(const EosDev &E, double *x)
{
    x[0] = clamp_key(x[0], E.T0, E.Tmax);
#pragma unroll
    for (int q = 0; q < 3; ++q) x[1 + q] = clamp_key(x[1 + q], E.mu0[q], E.mumax[q]);
}

__device__ double resid(const EosDev &E, const double *x, double s, double inv_s, const double *n, double r[4],
                        double J[4][4])
{
    double sn[4];
    tab_eval_steps(E, x, sn, J, nullptr);
    // J / s per unit of x: the grid-step scaling folded into the 1/s scaling
    const double sc[4] = {E.inv_dT * inv_s, E.inv_dmu[0] * inv_s, E.inv_dmu[1] * inv_s, E.inv_dmu[2] * inv_s};
    double tgt[4] = {s, n[0], n[1], n[2]};
    double m = 0.0;
    for (int k = 0; k < 4; ++k) {
        r[k] = (sn[k] - tgt[k]) * inv_s;
        m = isfinite(r[k]) ? fmax(m, fabs(r[k])) : __longlong_as_double(0x7FF0000000000000LL);
        for (int j = 0; j < 4; ++j) J[k][j] *= sc[j];
    }
    return m;
}

// Damped Newton on the table interpolant.  The Jacobian is factorised in place (it is
// not needed after the step); each line-search trial overwrites r and J with their values
// at the trial point, so the accepted point's residual and Jacobian are ready for the
// next iteration (the same sequence as a copy-on-accept scheme, with fewer registers).
// On convergence J holds d(s, n)/d(T, mu) / s at the returned x when *jx is set (the
// caller then needs only p there); otherwise it is stale.
__device__ bool tab_newton(const EosDev &E, double s, const double *n, double *x, EosWork &w, double J[4][4],
                           bool *jx)
{
    double r[4];
    *jx = false;
    const double inv_s = 1.0 / s;
    double rn = resid(E, x, s, inv_s, n, r, J);
    ++w.resid;
    for (int it = 0; it < E.maxit; ++it) {
        double d[4] = {-r[0], -r[1], -r[2], -r[3]};
        if (rn <= E.tol) {
            if (!E.polish) {
                *jx = true;
                return true;
            }
            ++w.solve;
            if (solve4(J, d)) {  // one polishing step, kept when its point still meets the tolerance
                double xn[4] = {x[0] + d[0], x[1] + d[1], x[2] + d[2], x[3] + d[3]};
                clamp4(E, xn);
                ++w.resid;
                if (resid(E, xn, s, inv_s, n, r, J) <= E.tol) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) x[k] = xn[k];
                    *jx = true;
                }
            }
            return true;
        }
        ++w.solve;
        if (!solve4(J, d)) return false;
        double lam = 1.0, xn[4], rnn = 0.0;
        for (int ls = 0; ls <= 8; ++ls) {
#pragma unroll
            for (int k = 0; k < 4; ++k) xn[k] = fma(lam, d[k], x[k]);
            clamp4(E, xn);
            rnn = resid(E, xn, s, inv_s, n, r, J);
            ++w.resid;
            if (rnn < rn) break;
            lam *= 0.5;
        }
        // no decrease along the Newton direction (the root lies beyond a clamped table
        // edge, or the interpolant is flat): the iteration has stalled and ends unconverged
        if (!(rnn < rn)) return false;
#pragma unroll
        for (int k = 0; k < 4; ++k) x[k] = xn[k];
        rn = rnn;
    }
    return rn <= E.tol;
}

// quadrilinear interpolant of p alone
__device__ double tab_p(const EosDev &E, const double *x)
{
    int iT, iB, iS, iQ;
    double tT, tB, tS, tQ;
    locate(x[0], E.T0, E.inv_dT, E.nT, iT, tT);
    locate(x[1], E.mu0[0], E.inv_dmu[0], E.nmu[0], iB, tB);
    locate(x[2], E.mu0[1], E.inv_dmu[1], E.nmu[1], iS, tS);
    locate(x[3], E.mu0[2], E.inv_dmu[2], E.nmu[2], iQ, tQ);
    const int n3 = E.nmu[2], n23 = E.nmu[1] * E.nmu[2], n123 = E.nmu[0] * n23;
    double pv = 0.0;
    for (int bT = 0; bT < 2; ++bT)
        for (int bB = 0; bB < 2; ++bB) {
            double wT = bT ? tT : 1.0 - tT, wB = bB ? tB : 1.0 - tB;
            size_t base = (size_t)(iT + bT) * n123 + (size_t)(iB + bB) * n23 + (size_t)iS * n3 + iQ;
            double p00 = __ldg(E.p + base), p01 = __ldg(E.p + base + 1), p10 = __ldg(E.p + base + n3),
                   p11 = __ldg(E.p + base + n3 + 1);
            double a0 = p00 + tQ * (p01 - p00), a1 = p10 + tQ * (p11 - p10);
            pv = fma(wT * wB, a0 + tS * (a1 - a0), pv);
        }
    return pv;
}

// Offline inverter: the quadrilinear interpolant of the inverted table at (s, n_q / s); false
// outside the grid or where a corner holds no solution
__device__ bool inv_lookup(const EosDev &E, double s, const double *n, double *x)
{
    if (!(s > 0.0)) return false;
    const int K = E.inv_K, nd = E.inv_nd, nx = E.inv_nx;
    int d = (int)floor(log10(s / E.inv_p10[0]));
    if (d < 0 || d > nd) return false;
    double m = s / E.inv_p10[d];
    if (m >= 10.0 && d < nd) {
        m /= 10.0;
        d += 1;
    }
    if (m < 1.0 && d > 0) {
        m *= 10.0;
        d -= 1;
    }
    const double r = (m - 1.0) * K / 9.0;
    int j = (int)floor(r);
    j = max(0, min(j, K - 1));
    const long long i = (long long)d * K + j;
    if (i < 0 || i > (long long)K * nd - 1) return false;
    int ix[4];
    double t[4];
    ix[0] = (int)i;
    t[0] = r - j;
    if (!(t[0] >= 0.0 && t[0] <= 1.0)) return false;
    const double dxr = 2.0 * E.inv_xmax / (nx - 1);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double rr = (n[q] / s + E.inv_xmax) / dxr;
        if (!(rr >= 0.0 && rr <= (double)(nx - 1))) return false;
        const int k = min((int)floor(rr), nx - 2);
        ix[1 + q] = k;
        t[1 + q] = rr - k;
    }
    x[0] = x[1] = x[2] = x[3] = 0.0;
    const long long ns = (long long)K * nd + 1;
    for (int corner = 0; corner < 16; ++corner) {
        const int b0 = (corner >> 3) & 1, b1 = (corner >> 2) & 1, b2 = (corner >> 1) & 1, b3 = corner & 1;
        const long long node = (((long long)(ix[0] + b0) * nx + ix[1] + b1) * nx + ix[2] + b2) * nx + ix[3] + b3;
        const double w = (b0 ? t[0] : 1.0 - t[0]) * (b1 ? t[1] : 1.0 - t[1]) * (b2 ? t[2] : 1.0 - t[2]) *
                         (b3 ? t[3] : 1.0 - t[3]);
        const double2 *v = reinterpret_cast<const double2 *>(E.inv + 4 * node);
        const double2 a = __ldg(v), b = __ldg(v + 1);
        if (!isfinite(a.x)) return false;
        x[0] = fma(w, a.x, x[0]);
        x[1] = fma(w, a.y, x[1]);
        x[2] = fma(w, b.x, x[2]);
        x[3] = fma(w, b.y, x[3]);
    }
    (void)ns;
    return true;
}

struct EosOut {
    double T, mu[3], p, e, ps, pn[3], cs2;
    uint32_t st;
};

// the conformal-diagonal backup EoS (Sec. "Equation of state", backup EoS) inverted in closed
// form: s = 4 A0 T^3, n_q = 4 A0 mu_q^3 / mu_q0^4; e = 3 p; p_s = T/3, p_{n_q} = mu_q/3
__device__ __forceinline__ EosOut backup_eos(const EosDev &E, double s, const double *n)
{
    EosOut o;
    const double A0 = E.cd_A0;
    o.T = cbrt(s / (4.0 * A0));
    double pq = 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double m0 = E.cd_mu0[q], m02 = m0 * m0;
        o.mu[q] = cbrt(n[q] * m02 * m02 / (4.0 * A0));
        const double r = o.mu[q] / m0, r2 = r * r;
        pq += r2 * r2;
        o.pn[q] = o.mu[q] / 3.0;
    }
    const double T2 = o.T * o.T;
    o.p = A0 * (T2 * T2 + pq);
    o.e = 3.0 * o.p;
    o.ps = o.T / 3.0;
    o.cs2 = 1.0 / 3.0;
    o.st = PST_BACKUP;
    return o;
}

__device__ __forceinline__ bool inside_table(const EosDev &E, const double *x)
{
    bool in = x[0] >= E.T0 && x[0] <= E.Tmax;
#pragma unroll
    for (int q = 0; q < 3; ++q) in = in && x[1 + q] >= E.mu0[q] && x[1 + q] <= E.mumax[q];
    return in;
}

// guess: this particle's table solution of the previous stage (T <= 0: none).  Attempts:
// table Newton from the guess; else the closed form, then table Newton from it; else the
// closed form (flagged).  used_table tells whether the table produced the result.
__device__ EosOut eos_invert(const EosDev &E, double cs2_cap, double s, const double *n, const double *guess,
                             bool &used_table, EosWork &w)
{
    EosOut o;
    o.T = 0.0;
    for (int q = 0; q < 3; ++q) o.mu[q] = 0.0, o.pn[q] = 0.0;
    o.p = o.e = o.ps = o.cs2 = 0.0;
    o.st = 0u;
    used_table = false;
    if (!isfinite(s) || !isfinite(n[0]) || !isfinite(n[1]) || !isfinite(n[2])) {
        o.st = PST_NONFINITE | PST_NOCONV;
        return o;
    }
    double x[4];
    double H[4][4];
    bool use_table = false, hx = false;
    if (E.offline && E.has_table && inv_lookup(E, s, n, x) && inside_table(E, x)) use_table = true;
    if (!use_table && E.has_table && guess[0] > 0.0 && inside_table(E, guess)) {
        double xt[4] = {guess[0], guess[1], guess[2], guess[3]};
        if (tab_newton(E, s, n, xt, w, H, &hx)) {
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = xt[k];
            use_table = true;
        }
    }
    if (!use_table) {
        // a negative guess is the particle's previous closed-form T
        o.st = an_invert(E, s, n, x[0], x + 1, w, guess[0] < 0.0 ? -guess[0] : 0.0);
        if (o.st && E.backup && s > 0.0) return backup_eos(E, s, n);
        if (o.st) return o;
        if (E.has_table) {
            if (inside_table(E, x)) {
                double xt[4] = {x[0], x[1], x[2], x[3]};
                if (tab_newton(E, s, n, xt, w, H, &hx)) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) x[k] = xt[k];
                    use_table = true;
                } else {
                    o.st |= PST_FALLBACK;
                }
            } else {
                o.st |= PST_OUT_OF_TABLE;
            }
        }
    }
    used_table = use_table;
    double p, sn[4];
    if (use_table && hx) {  // the Newton's last Jacobian is the one at the solution
        p = tab_p(E, x);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) H[i][j] *= s;
    } else if (use_table) {
        tab_eval(E, x, sn, H, &p);
        ++w.resid;
    } else {
        an_eval(E, x[0], x + 1, p, sn, H);
    }
    double e = x[0] * s + x[1] * n[0] + x[2] * n[1] + x[3] * n[2] - p;
    // (p_s, p_n) = H^-T (s, n) over the directions the EoS couples to; an uncoupled charge
    // direction (no table, chi_q = 0) becomes an identity row with zero right-hand side
    double A[4][4], z[4] = {s, n[0], n[1], n[2]};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool act_i = i == 0 || use_table || E.chi[i - 1] > 0.0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool act_j = j == 0 || use_table || E.chi[j - 1] > 0.0;
            A[i][j] = (act_i && act_j) ? H[j][i] : (i == j ? 1.0 : 0.0);
        }
        if (!act_i) z[i] = 0.0;
    }
    ++w.solve;
    if (!solve4(A, z)) {
        o.st |= PST_NOCONV;
        return o;
    }
    double cs2 = (s * z[0] + n[0] * z[1] + n[1] * z[2] + n[2] * z[3]) / (e + p);
    if (cs2 > cs2_cap) {
        double f = cs2_cap / cs2;
#pragma unroll
        for (int k = 0; k < 4; ++k) z[k] *= f;
        cs2 = cs2_cap;
        o.st |= PST_CS2_CAPPED;
    }
    o.T = x[0];
    for (int q = 0; q < 3; ++q) o.mu[q] = x[1 + q], o.pn[q] = z[1 + q];
    o.p = p;
    o.e = e;
    o.ps = z[0];
    o.cs2 = cs2;
    return o;
}

// ---------------------------------------------------------------------------
// Lane-refill EoS pass.  The table Newton's work varies from particle to particle (iterations,
// line-search trials, the polishing step), so a warp that inverts 32 particles together leaves
// its finished lanes idle until the slowest is done, and every FP64 instruction of the 1:64 pipe
// costs the whole warp.  Here each lane holds its own particle and claims the next one as soon
// as its own is done.  One trip through the loop is, for every lane that holds a particle, one
// table evaluation at its trial point (s, n_q, their Jacobian and p) and at most one 4x4 solve:
// the Newton step, the polishing step, or, once converged, the transposed system of the EoS
// derivatives (p_s, p_n) = H^-T (s, n) -- so the warp's lanes evaluate and solve together
// whatever stage of the iteration their particles are at.  The iteration per particle is the
// damped Newton of tab_newton (the same iterates, with the residual and the step in grid-step
// units: the scaling changes rounding only) followed by the derivative solve of eos_invert.
// Particles whose warm start is not a table solution inside the table, whose table Newton
// fails, or when the offline inverter is on, take eos_invert inline (a divergent, rarer path).
//
// Ctx supplies  __device__ bool load(int a, double &s, double n[3], double g[4], double &cs2_cap)
// (false: not a particle of this pass), and  __device__ void store(int a, const EosOut &o, bool
// used_table).
// claim: the pass's particle counter (indices 0 .. limit-1, claimed one lane at a time).
enum { LANE_NONE = 0, LANE_NEWTON = 1, LANE_POLISH = 2, LANE_REEVAL = 3 };

// the general inversion as a call of its own: the lane loop keeps its registers for the table
// Newton, the common path
__device__ __noinline__ EosOut eos_invert_call(const EosDev &E, double cs2_cap, double s, const double *n,
                                               const double *guess, bool &used_table, EosWork &w)
{
    return eos_invert(E, cs2_cap, s, n, guess, used_table, w);
}

template <class Ctx>
__device__ void eos_lanes(const EosDev &E, unsigned int *claim, int limit, Ctx &ctx, EosWork &w)
{
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    // grid steps of the table axes: the iteration works in grid-step units with the residual
    // unscaled (the Newton step is the same: scaling the residual and the Jacobian's rows by
    // 1/s, or its columns by the steps, does not change it), and converges when
    // max |residual| <= tol s
    const double step[4] = {E.dT, E.dmu[0], E.dmu[1], E.dmu[2]};
    const double istep[4] = {E.inv_dT, E.inv_dmu[0], E.inv_dmu[1], E.inv_dmu[2]};
    int a = -1, phase = LANE_NONE, it = 0, ls = 0;
    bool more = true, first = false;
    long long rn = 0, tolb = 0;  // max-norms of the residual as integer magnitudes
    double x[4], xt[4], d[4], r[4], J[4][4], p = 0.0, lam = 1.0, s = 0.0, nq[3];
    double cs2_cap = 1.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = xt[k] = d[k] = r[k] = 0.0;
    nq[0] = nq[1] = nq[2] = 0.0;
    for (;;) {
        // lanes without a particle claim the next ones (one atomic per warp)
        const unsigned need = __ballot_sync(FULL, a < 0 && more);
        if (need) {
            const int leader = __ffs(need) - 1;
            unsigned base = 0u;
            if (lane == leader) base = atomicAdd(claim, (unsigned)__popc(need));
            base = __shfl_sync(FULL, base, leader);
            if (a < 0 && more) {
                const long long idx = (long long)base + __popc(need & ((1u << lane) - 1u));
                if (idx >= limit) more = false;
                else a = (int)idx;
            }
        }
        if (__ballot_sync(FULL, a >= 0 || more) == 0u) break;
        // a new particle: the table Newton from its warm start, or the general inversion
        if (a >= 0 && phase == LANE_NONE) {
            double g[4];
            if (!ctx.load(a, s, nq, g, cs2_cap)) {
                a = -1;
            } else if (E.has_table && !E.offline && g[0] > 0.0 && inside_table(E, g) && isfinite(s) && s > 0.0 &&
                       isfinite(nq[0]) && isfinite(nq[1]) && isfinite(nq[2])) {
#pragma unroll
                for (int k = 0; k < 4; ++k) xt[k] = g[k];
                phase = LANE_NEWTON;
                first = true;
                it = 0;
                ls = 0;
                tolb = __double_as_longlong(E.tol * s);
            } else {
                bool used = false;
                const EosOut o = eos_invert_call(E, cs2_cap, s, nq, g, used, w);
                ctx.store(a, o, used);
                a = -1;
            }
        }
        // one table evaluation at the trial point: (s, n) - target and the Jacobian per grid
        // step, and p
        const bool evl = a >= 0 && phase != LANE_NONE;
        long long rnn = 0;
        if (evl) {
            double sn[4];
            tab_eval_steps(E, xt, sn, J, &p);
            const double tgt[4] = {s, nq[0], nq[1], nq[2]};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                r[k] = sn[k] - tgt[k];
                rnn = max(rnn, min(mag_bits(r[k]), kInfBits));  // a non-finite residual counts as infinite
            }
            ++w.resid;
        }
        // what this trip solves: 0 nothing, 1 a Newton step (J d = -r, also the polishing
        // step), 2 the EoS derivatives at the converged point (H^T z = (s, n), H = d(s, n)/d(T, mu))
        int act = 0;
        bool fail = false;
        if (evl) {
            bool accepted = false;
            if (phase == LANE_NEWTON) {
                if (first || rnn < rn) {
                    accepted = true;
                    if (!first) ++it;
                    first = false;
#pragma unroll
                    for (int k = 0; k < 4; ++k) x[k] = xt[k];
                    rn = rnn;
                } else if (++ls > 8) {
                    fail = true;  // no decrease along the Newton direction: stalled
                } else {
                    lam *= 0.5;
#pragma unroll
                    for (int k = 0; k < 4; ++k) xt[k] = fma(lam, d[k], x[k]);
                    clamp4(E, xt);
                }
                if (accepted) {
                    if (it >= E.maxit) {
                        if (rn <= tolb) act = 2;
                        else fail = true;
                    } else if (rn <= tolb) {
                        act = E.polish ? 1 : 2;
                        if (E.polish) phase = LANE_POLISH;
                    } else {
                        act = 1;
                    }
                }
            } else if (phase == LANE_POLISH) {
                if (rnn <= tolb) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) x[k] = xt[k];
                    act = 2;
                } else {  // the polished point is refused: J and p again at the kept point
#pragma unroll
                    for (int k = 0; k < 4; ++k) xt[k] = x[k];
                    phase = LANE_REEVAL;
                }
            } else {  // LANE_REEVAL
                act = 2;
            }
        }
        double b[4];
        if (act == 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) b[k] = -r[k];
        } else if (act == 2) {  // A = H^T, H[f][j] = J[f][j] / step_j
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = i + 1; j < 4; ++j) {
                    const double t = J[i][j];
                    J[i][j] = J[j][i];
                    J[j][i] = t;
                }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) J[i][j] *= istep[i];
            b[0] = s;
            b[1] = nq[0];
            b[2] = nq[1];
            b[3] = nq[2];
        }
        bool ok = true;
        if (act) {
            ++w.solve;
            ok = solve4(J, b);
        }
        if (act == 1) {
            if (phase == LANE_POLISH) {
                if (ok) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) xt[k] = fma(b[k], step[k], x[k]);
                    clamp4(E, xt);
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) xt[k] = x[k];
                    phase = LANE_REEVAL;
                }
            } else if (!ok) {
                fail = true;
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    d[k] = b[k] * step[k];
                    xt[k] = x[k] + d[k];
                }
                clamp4(E, xt);
                lam = 1.0;
                ls = 0;
            }
        } else if (act == 2) {
            EosOut o;
            o.st = 0u;
            if (!ok) {
                o.T = o.p = o.e = o.ps = o.cs2 = 0.0;
#pragma unroll
                for (int q = 0; q < 3; ++q) o.mu[q] = o.pn[q] = 0.0;
                o.st = PST_NOCONV;
            } else {
                const double e = x[0] * s + x[1] * nq[0] + x[2] * nq[1] + x[3] * nq[2] - p;
                double cs2 = (s * b[0] + nq[0] * b[1] + nq[1] * b[2] + nq[2] * b[3]) / (e + p);
                if (cs2 > cs2_cap) {
                    const double f = cs2_cap / cs2;
#pragma unroll
                    for (int k = 0; k < 4; ++k) b[k] *= f;
                    cs2 = cs2_cap;
                    o.st |= PST_CS2_CAPPED;
                }
                o.T = x[0];
#pragma unroll
                for (int q = 0; q < 3; ++q) o.mu[q] = x[1 + q], o.pn[q] = b[1 + q];
                o.p = p;
                o.e = e;
                o.ps = b[0];
                o.cs2 = cs2;
            }
            ctx.store(a, o, true);
            a = -1;
            phase = LANE_NONE;
        }
        if (fail) {  // the table Newton from the warm start failed: the general inversion
            const double g0[4] = {0.0, 0.0, 0.0, 0.0};
            bool used = false;
            const EosOut o = eos_invert_call(E, cs2_cap, s, nq, g0, used, w);
            ctx.store(a, o, used);
            a = -1;
            phase = LANE_NONE;
        }
    }
}

}  // namespace
}  // namespace sphg
