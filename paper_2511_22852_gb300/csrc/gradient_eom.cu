// gradient_eom.cu -- SPH gradients (row a5), equations of motion with minimal
// Israel-Stewart sources (row a6), Heun update (row a7) and the reductions of
// the conservation totals (row a8).
//
// Gradient pass (eqs. sphderivativerel, generalsphderivative with the sigma
// exponents of the n-form corrected so that n = 0 reproduces eq.
// sphderivativerel): per particle a
//   d_k u^j  = sum_b (u^j_b / sigma*_b) d_k W_ab                        (n = 0)
//   F^i      = -sqrt(-g) sum_b sum_j (X^{ji}_a/sigma*_a^2 + X^{ji}_b/sigma*_b^2) d_j W_ab   (n = -1)
// where X^{ji} = T^{ji} - v^j T^{0i} = (p + Pi) delta^{ji} + pi^{ji} - v^j pi^{0i}
// (2+1D), so that F^i is the rate of the lab momentum per particle
// P^i = sqrt(-g) T^{0i} / sigma*.  The a-part of the n = -1 sum factorises:
// X_a sum_b dW_ab, so each pair costs 8 fused multiply-adds.
//
// Equations of motion, 2+1D Milne (boost invariant) or Cartesian: every rate is
// affine in the unknown acceleration a^i = du^i/dx^0 (entropy production eq.
// dsdnrewr, bulk eq. min_bul_rel, shear eq. min_she_rel, continuity
// D sigma = -sigma theta), so dP^i/dx^0 = M^i_j a^j + c^i is assembled with
// affine arithmetic (exact coefficients, no differencing) and M a = F - c is
// solved per particle by Cramer's rule -- the D x D system of eq. unugeneral.
#include <algorithm>

#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kWarps = 4;  // warps (particles in flight) per block

// Gradient pass, one warp per particle: single-precision prefilter of the candidates in
// the 3x3 cells, ballot-compaction of the survivors into a per-warp queue, the exact FP64
// test and the pair arithmetic 32 pairs at a time on full warps, then a fixed-order
// butterfly reduction of the per-lane partial sums.
__global__ void __launch_bounds__(32 * kWarps) k_gradient2(EvView v, int stage, const double *__restrict__ y,
                                                           const float2 *__restrict__ fpos,
                                                           const double *__restrict__ gin,
                                                           const uint32_t *__restrict__ start,
                                                           const uint32_t *__restrict__ cnt, double *__restrict__ gout,
                                                           int fallback)
{
    if (fallback && !v.sc->pair_flag) return;  // the pair-list pass did the work
    __shared__ int queue[kWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // grid-stride over particles (one warp each): launched at a few blocks per SM when it is
    // only the fallback of the pair-list passes
    for (int a = blockIdx.x * kWarps + wid; a < v.n; a += gridDim.x * kWarps) {  // warp-uniform
        int *q = queue[wid];
        const int n = v.n;
        const double *X = y, *Y = y + n;
        const double *Xxx = gin, *Xxy = gin + n, *Xyx = gin + 2 * (size_t)n, *Xyy = gin + 3 * (size_t)n;
        const double *Ux = gin + 4 * (size_t)n, *Uy = gin + 5 * (size_t)n;
        const double xa = X[a], ya = Y[a];
        const float2 fa = fpos[a];
        const double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
        const int cx = cell_coord(xa, xmin0, v.inv_cell), cy = cell_coord(ya, xmin1, v.inv_cell);
        const int lim = 1 << v.B;
        const unsigned lt = (1u << lane) - 1u;
        double Gx = 0.0, Gy = 0.0, Hx = 0.0, Hy = 0.0;
        double dxux = 0.0, dxuy = 0.0, dyux = 0.0, dyuy = 0.0;
        int qn = 0;
        // queued index with bit 31 set: the float test left the pair undecided (exact test needed)
        auto pair = [&](int qb) {
            const int b = qb & 0x7FFFFFFF;
            const double dx = xa - X[b], dy = ya - Y[b];
            if (qb < 0 && !(dist2_2d(dx, dy) < v.supp2)) return;
            const double r2 = fma(dx, dx, dy * dy);
            if (r2 > 0.0) {
                const double ir = inv_sqrt(r2);
                const double fac = kernel_dw(r2 * ir * v.inv_h) * ir;  // (dW/dr)/r without sigma_d/h
                const double gx = fac * dx, gy = fac * dy;
                Gx += gx;
                Gy += gy;
                Hx = fma(Xxx[b], gx, fma(Xyx[b], gy, Hx));
                Hy = fma(Xxy[b], gx, fma(Xyy[b], gy, Hy));
                const double ubx = Ux[b], uby = Uy[b];
                dxux = fma(ubx, gx, dxux);
                dxuy = fma(uby, gx, dxuy);
                dyux = fma(ubx, gy, dyux);
                dyuy = fma(uby, gy, dyuy);
            }
        };
        for (int oy = -1; oy <= 1; ++oy) {
            const int ny = cy + oy;
            if (ny < 0 || ny >= lim) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int nx = cx + ox;
                if (nx < 0 || nx >= lim) continue;
                const uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
                const uint32_t b0 = start[k], b1 = b0 + cnt[k];
                for (uint32_t base = b0; base < b1; base += 32) {
                    const uint32_t b = base + lane;
                    bool cand = false, sure = false;
                    if (b < b1) {
                        const float2 fb = fpos[b];
                        const float dx = fa.x - fb.x, dy = fa.y - fb.y;
                        const float r2f = fmaf(dx, dx, dy * dy);
                        cand = r2f <= v.supp2_hi;
                        sure = r2f < v.supp2_lo;
                    }
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
                    if (cand) q[qn + __popc(m & lt)] = sure ? (int)b : (int)(b | 0x80000000u);
                    qn += __popc(m);
                    __syncwarp();
                    if (qn >= 32) {
                        pair(q[lane]);
                        qn -= 32;
                        __syncwarp();
                        if (lane < qn) q[lane] = q[32 + lane];
                        __syncwarp();
                    }
                }
            }
        }
        if (lane < qn) pair(q[lane]);
        for (int o = 16; o > 0; o >>= 1) {
            Gx += __shfl_xor_sync(0xFFFFFFFFu, Gx, o);
            Gy += __shfl_xor_sync(0xFFFFFFFFu, Gy, o);
            Hx += __shfl_xor_sync(0xFFFFFFFFu, Hx, o);
            Hy += __shfl_xor_sync(0xFFFFFFFFu, Hy, o);
            dxux += __shfl_xor_sync(0xFFFFFFFFu, dxux, o);
            dxuy += __shfl_xor_sync(0xFFFFFFFFu, dxuy, o);
            dyux += __shfl_xor_sync(0xFFFFFFFFu, dyux, o);
            dyuy += __shfl_xor_sync(0xFFFFFFFFu, dyuy, o);
        }
        if (lane == 0) {
            const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
            const double sqrtg = v.milne ? tau : 1.0;
            const double c = v.sigma_d * v.inv_h;
            gout[a] = c * dxux;
            gout[(size_t)n + a] = c * dxuy;
            gout[2 * (size_t)n + a] = c * dyux;
            gout[3 * (size_t)n + a] = c * dyuy;
            const double Fx = Xxx[a] * Gx + Xyx[a] * Gy + Hx;
            const double Fy = Xxy[a] * Gx + Xyy[a] * Gy + Hy;
            gout[4 * (size_t)n + a] = -sqrtg * c * Fx;
            gout[5 * (size_t)n + a] = -sqrtg * c * Fy;
        }
    }
}

// equations of motion of one particle (rows n apart): mode 0 writes y1 = y + dt f(y),
// mode 1 closes Heun in place, mode 2 writes the rates
__device__ __forceinline__ void eom2_particle(const EvView &v, int stage, int mode, size_t n, size_t a,
                                              const double *__restrict__ ys, const double *__restrict__ dens,
                                              const double *__restrict__ eos, const double *__restrict__ gout,
                                              double *__restrict__ yout, double *__restrict__ rates,
                                              uint32_t *__restrict__ status)
{
    double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
    double hub = v.milne ? 1.0 / tau : 0.0;      // Gamma^eta_{eta tau}
    double sqrtg = v.milne ? tau : 1.0;
    double ux = ys[2 * n + a], uy = ys[3 * n + a];
    double sig_star = dens[a], s = dens[n + a], nq0 = dens[2 * n + a], nq1 = dens[3 * n + a], nq2 = dens[4 * n + a];
    double g = dens[5 * n + a];
    double T = eos[a], mu0 = eos[n + a], mu1 = eos[2 * n + a], mu2 = eos[3 * n + a];
    double p = eos[4 * n + a], e = eos[5 * n + a], ps = eos[6 * n + a];
    double pn0 = eos[7 * n + a], pn1 = eos[8 * n + a], pn2 = eos[9 * n + a];
    double dxux = gout[a], dxuy = gout[n + a], dyux = gout[2 * n + a], dyuy = gout[3 * n + a];
    double Fx = gout[4 * n + a], Fy = gout[5 * n + a];
    // one reciprocal per denominator (an FP64 division is a multi-instruction sequence):
    // sigma = sig_star / (u0 sqrt(-g)) and 1 / sigma from 1/u0 and 1/sig_star
    double ig = 1.0 / g, isig = 1.0 / sig_star;
    double sigma = sig_star * ig * (v.milne ? hub : 1.0);
    double isg = g * sqrtg * isig;
    double vx = ux * ig, vy = uy * ig;
    const bool visc = v.tr.viscous != 0;
    double Bv = 0.0, Pvxx = 0.0, Pvxy = 0.0, Pvyy = 0.0;
    if (visc) {
        Bv = ys[5 * n + a];
        Pvxx = ys[6 * n + a];
        Pvxy = ys[7 * n + a];
        Pvyy = ys[8 * n + a];
    }
    double Pi = sigma * Bv, pxx = sigma * Pvxx, pxy = sigma * Pvxy, pyy = sigma * Pvyy;
    const double dt = v.dtau;
    const int nv = v.nv;
    if ((status[a] & (PST_NOCONV | PST_NONFINITE)) || (v.tr.T_stop_GeV > 0.0 && eos[a] * kHbarc < v.tr.T_stop_GeV)) {
        // no EoS solution, or below the stop temperature: the particle is frozen for this stage
        // (ballistic motion only)
        for (int k = 0; k < nv; ++k) {
            double fk = k == 0 ? vx : (k == 1 ? vy : 0.0);
            if (mode == 0) yout[k * n + a] = ys[k * n + a] + dt * fk;
            else if (mode == 1) yout[k * n + a] = 0.5 * ((yout[k * n + a] + ys[k * n + a]) + dt * fk);
            else rates[k * n + a] = fk;
        }
        const double dN0[3] = {0.0, 0.0, 0.0};  // frozen: the charges stay as they are
        heun_charges(v, mode, n, a, dN0);
        return;
    }

    const Aff ax = {0.0, 1.0, 0.0}, ay = {0.0, 0.0, 1.0};
    Aff dg = vx * ax + vy * ay;                                  // d u^0 / dx^0
    double dgx = (ux * dxux + uy * dxuy) * ig;                   // d_x u^0
    double dgy = (ux * dyux + uy * dyuy) * ig;                   // d_y u^0
    Aff th = dg + (dxux + dyuy + g * hub - (vx * dgx + vy * dgy));  // theta = nabla_mu u^mu
    Aff dsg = (-sigma * ig) * th;                                // d sigma / dx^0

    Aff dS = aff(0.0), dBv = aff(0.0), dPxx = aff(0.0), dPxy = aff(0.0), dPyy = aff(0.0);
    if (visc) {
        const double third = 1.0 / 3.0;
        // sigma^{ij} = -(d_i u^j + d_j u^i)/2 - u^0 (u^i a^j + u^j a^i)/2 + (delta^{ij} + u^i u^j) theta/3
        Aff sxx = aff(-dxux) - (g * ux) * ax + (third * (1.0 + ux * ux)) * th;
        Aff sxy = aff(-0.5 * (dxuy + dyux)) - (0.5 * g) * (ux * ay + uy * ax) + (third * ux * uy) * th;
        Aff syy = aff(-dyuy) - (g * uy) * ay + (third * (1.0 + uy * uy)) * th;
        Aff see = aff(-g * hub) + third * th;                    // tau^2 sigma^{eta eta} (z z if Cartesian)
        Aff svx = vx * sxx + vy * sxy, svy = vx * sxy + vy * syy;
        Aff vsv = vx * svx + vy * svy;
        double pvx = vx * pxx + vy * pxy, pvy = vx * pxy + vy * pyy;  // pi^{0i}
        double vpv = vx * pvx + vy * pvy;                             // pi^{00}
        double pee = vpv - pxx - pyy;                                 // tau^2 pi^{eta eta}
        Aff pisig = vpv * vsv - 2.0 * (pvx * svx + pvy * svy) + pxx * sxx + 2.0 * pxy * sxy + pyy * syy + pee * see;
        double eta = v.tr.eta_over_s * s;
        double dTg = T * kHbarc - v.tr.zeta_T_GeV;
        double zeta = v.tr.zeta_peak * exp(-dTg * dTg / (2.0 * v.tr.zeta_w_GeV * v.tr.zeta_w_GeV)) * s;
        // 1/tau_pi = (e + p) / (c eta), tau_pi = c eta / (e + p); tau_Pi = ratio tau_pi
        double itp = (e + p) / (v.tr.tau_pi_coef * eta);
        double itPi = itp / v.tr.tau_Pi_ratio;
        double iT = 1.0 / T;
        const bool dnmr = v.tr.model == 1;
        dS = (ig * isg * iT) * (pisig - Pi * th);
        if (dnmr) {
            // tau_Pi D Pi + Pi = -zeta theta - delta_PiPi Pi theta + lambda_Pipi pi:sigma; the stored
            // Pi/sigma obeys u0 d(Pi/sigma)/dtau = (D Pi + Pi theta)/sigma
            const double cs2 = eos[10 * n + a];
            dBv = (ig * isg) * ((-itPi) * (zeta * th + Pi) + ((1.0 - v.tr.dnmr[0]) * Pi) * th +
                                (v.tr.dnmr[1] * (1.0 / 3.0 - cs2)) * pisig);
        } else {
            dBv = (-ig * isg * itPi) * (zeta * th + Pi);
        }
        // pi^{j alpha} a_alpha with the lowered four-acceleration (u^0 du^0/dx^0, -u^0 a^i)
        Aff pax = g * (pvx * dg - (pxx * ax + pxy * ay));
        Aff pay = g * (pvy * dg - (pxy * ax + pyy * ay));
        // d pi^{ij}/d tau = [(2 eta sigma^{ij} - pi^{ij}) / tau_pi - 4/3 pi^{ij} theta - coupling] / u0
        const double f43 = 4.0 / 3.0;
        Aff dpxx, dpxy, dpyy;
        if (dnmr) {
            // DNMR: - delta_pipi pi theta - tau_pipi <pi sigma> + phi_7 <pi pi> + lambda_piPi Pi sigma,
            // <A>^{ij} = (A^{ij} + A^{ji})/2 - Delta^{ij} tr A / 3 for transverse pi and sigma;
            // A^{ij} = pi^{i0} sigma^{j0} - pi^{ix} sigma^{jx} - pi^{iy} sigma^{jy} (pi^{i eta} = 0)
            const double c2 = v.tr.dnmr[2], c3 = v.tr.dnmr[3], c4 = v.tr.dnmr[4], f7 = itp * v.tr.dnmr[5] / p;
            const Aff Axx = pvx * svx - pxx * sxx - pxy * sxy, Axy = pvx * svy - pxx * sxy - pxy * syy;
            const Aff Ayx = pvy * svx - pxy * sxx - pyy * sxy, Ayy = pvy * svy - pxy * sxy - pyy * syy;
            const double dxx = (1.0 + ux * ux) / 3.0, dxy = ux * uy / 3.0, dyy = (1.0 + uy * uy) / 3.0;  // -Delta^{ij}/3
            const Aff PAxx = Axx + dxx * pisig, PAxy = 0.5 * (Axy + Ayx) + dxy * pisig, PAyy = Ayy + dyy * pisig;
            const double trB = vpv * vpv - 2.0 * (pvx * pvx + pvy * pvy) + pxx * pxx + 2.0 * pxy * pxy + pyy * pyy + pee * pee;
            const double PBxx = pvx * pvx - pxx * pxx - pxy * pxy + dxx * trB;
            const double PBxy = pvx * pvy - pxx * pxy - pxy * pyy + dxy * trB;
            const double PByy = pvy * pvy - pxy * pxy - pyy * pyy + dyy * trB;
            dpxx = ig * (itp * (2.0 * eta * sxx + (-pxx)) + aff(f7 * PBxx) - (c2 * pxx) * th - c3 * PAxx + (c4 * Pi) * sxx -
                         2.0 * ux * pax);
            dpxy = ig * (itp * (2.0 * eta * sxy + (-pxy)) + aff(f7 * PBxy) - (c2 * pxy) * th - c3 * PAxy + (c4 * Pi) * sxy -
                         (ux * pay + uy * pax));
            dpyy = ig * (itp * (2.0 * eta * syy + (-pyy)) + aff(f7 * PByy) - (c2 * pyy) * th - c3 * PAyy + (c4 * Pi) * syy -
                         2.0 * uy * pay);
        } else {
            dpxx = ig * (itp * (2.0 * eta * sxx + (-pxx)) - (f43 * pxx) * th - 2.0 * ux * pax);
            dpxy = ig * (itp * (2.0 * eta * sxy + (-pxy)) - (f43 * pxy) * th - (ux * pay + uy * pax));
            dpyy = ig * (itp * (2.0 * eta * syy + (-pyy)) - (f43 * pyy) * th - 2.0 * uy * pay);
        }
        double isg2 = isg * isg;
        dPxx = isg * dpxx - (pxx * isg2) * dsg;
        dPxy = isg * dpxy - (pxy * isg2) * dsg;
        dPyy = isg * dpyy - (pyy * isg2) * dsg;
    }
    double dN[3] = {0.0, 0.0, 0.0};  // charge rates dN_q/dx0 (charge sources only)
    if (v.ntrack > 0 || v.nparton > 0) {
        // jet tracks (Cartesian) and partons: dP^i/dx0 gains sqrt(-g) I^i/sigma*, dS/dx0 gains
        // u_nu I^nu/(u^0 sigma T); parton charges: dN_q/dx0 = sqrt(-g) I_q/sigma*, and dS/dx0
        // gains -mu_q/T dN_q/dx0 (eq. dsdnrewr, R^S_q = -mu_q/T)
        double I[4] = {0.0, 0.0, 0.0, 0.0}, Ik[4], Iq[3] = {0.0, 0.0, 0.0};
        if (v.ntrack > 0) {
            jet_deposit(v, tau, ys[a], ys[n + a], 0.0, Ik);
            for (int k = 0; k < 4; ++k) I[k] += Ik[k];
        }
        if (v.nparton > 0) {
            const double xa[3] = {ys[a], ys[n + a], 0.0};
            parton_deposit(v, tau, sqrtg, xa, Ik, Iq);
            for (int k = 0; k < 4; ++k) I[k] += Ik[k];
        }
        Fx += sqrtg * I[1] * isig;
        Fy += sqrtg * I[2] * isig;
        // no eta component in 2+1D
        const double uI = g * I[0] - ux * I[1] - uy * I[2] - (mu0 * Iq[0] + mu1 * Iq[1] + mu2 * Iq[2]);
        dS = dS + aff((ig * isg / T) * uI);
        for (int c = 0; c < 3; ++c) dN[c] = sqrtg * Iq[c] * isig;
    }
    // BSQ diffusion (eq. min_dif_rel, metric (+,-,-,-)): tau_q Delta^i_nu D J^nu_q + J^i_q =
    // kappa_{qq'} nabla^<i> alpha_{q'}, with Delta^i_nu D J^nu = D J^i + u^i J^nu Du_nu and
    // nabla^<i> alpha = -d_i alpha - u^i D alpha (no Christoffel terms for the transverse
    // components).  The particle's lab charge N_q + Z_q, Z_q = J^0_q / (sigma u^0), changes by the
    // flux divergence (dout); the rest-frame charge rate dN_q = d(lab) - dZ_q enters the entropy
    // rate (-mu_q/T dN_q, eq. dsdnrewr) and the enthalpy rate.  D alpha_q = u^0 (alpha_{q,s} ds +
    // alpha_{q,n} . dn) depends on those rates, linearly: its fixed point is solved exactly (the
    // coefficient matrix is the state's; the right-hand side is affine in the acceleration).
    Aff dNd[3] = {aff(0.0), aff(0.0), aff(0.0)}, dJhx[3], dJhy[3];
    double dNt[3] = {0.0, 0.0, 0.0};
    if (v.diff) {
        const double qn[3] = {nq0, nq1, nq2}, qmu[3] = {mu0, mu1, mu2};
        double Jhx[3], Jhy[3], Jx[3], Jy[3], kap[3][3], itJ[3], gax[3], gay[3], dal[3][4];
        Aff jDu[3];
        for (int q = 0; q < 3; ++q) {
            Jhx[q] = ys[(kJRow + 2 * q) * n + a];
            Jhy[q] = ys[(kJRow + 2 * q + 1) * n + a];
            Jx[q] = sigma * Jhx[q];
            Jy[q] = sigma * Jhy[q];
            const double J0 = (ux * Jx[q] + uy * Jy[q]) * ig;
            jDu[q] = g * (J0 * dg - (Jx[q] * ax + Jy[q] * ay));  // J^nu Du_nu
            for (int q2 = 0; q2 < 3; ++q2) kap[q][q2] = v.kapT2[3 * q + q2] * T * T;
            itJ[q] = T / v.tauJT[q];
            gax[q] = v.dout[(2 * q) * n + a];
            gay[q] = v.dout[(2 * q + 1) * n + a];
            dNt[q] = v.dout[(6 + q) * n + a];
            for (int f = 0; f < 4; ++f) dal[q][f] = v.dal[(4 * q + f) * n + a];
        }
        const double ig2 = ig * ig, ig3 = ig2 * ig, isg2 = isg * isg;
        // the rates for a given D alpha; returns D alpha implied by them
        auto chain = [&](const Aff *Dal, Aff *dNq_o, Aff &dS_o, Aff *Dal_o) {
            Aff ds_l = aff(0.0);
            for (int q = 0; q < 3; ++q) {
                Aff sx = aff(0.0), sy = aff(0.0);  // kappa nabla^<i> alpha
                for (int q2 = 0; q2 < 3; ++q2) {
                    sx = sx + kap[q][q2] * (aff(-gax[q2]) - ux * Dal[q2]);
                    sy = sy + kap[q][q2] * (aff(-gay[q2]) - uy * Dal[q2]);
                }
                const Aff DJx = itJ[q] * (sx + (-Jx[q])) - ux * jDu[q];
                const Aff DJy = itJ[q] * (sy + (-Jy[q])) - uy * jDu[q];
                dJhx[q] = (ig * isg) * DJx - (Jx[q] * isg2) * dsg;
                dJhy[q] = (ig * isg) * DJy - (Jy[q] * isg2) * dsg;
                const Aff dZ = ig2 * (Jhx[q] * ax + Jhy[q] * ay + ux * dJhx[q] + uy * dJhy[q]) -
                               (2.0 * (ux * Jhx[q] + uy * Jhy[q]) * ig3) * dg;
                dNq_o[q] = aff(dNt[q]) - dZ;
            }
            dS_o = dS;
            for (int q = 0; q < 3; ++q) dS_o = dS_o - (qmu[q] / T) * dNq_o[q];
            ds_l = sigma * dS_o + (s * isg) * dsg;
            for (int q = 0; q < 3; ++q) {
                Aff d = dal[q][0] * ds_l;
                for (int r = 0; r < 3; ++r) d = d + dal[q][1 + r] * (sigma * (dNq_o[r] + aff(dN[r])) + (qn[r] * isg) * dsg);
                Dal_o[q] = g * d;
            }
        };
        const Aff z3[3] = {aff(0.0), aff(0.0), aff(0.0)};
        Aff f0[3], dNq0[3], dS0;
        chain(z3, dNq0, dS0, f0);
        // d dN_q / d D alpha_{q2} = kappa_{qq2} |u|^2 / (tau_q u0^3 sigma), through dZ
        const double uu = ux * ux + uy * uy;
        double K[3][3], Fm[3][3];
        for (int q = 0; q < 3; ++q)
            for (int q2 = 0; q2 < 3; ++q2) K[q][q2] = itJ[q] * kap[q][q2] * uu * ig3 * isg;
        for (int c = 0; c < 3; ++c)
            for (int q2 = 0; q2 < 3; ++q2) {
                double dSd = 0.0;
                for (int q = 0; q < 3; ++q) dSd -= (qmu[q] / T) * K[q][q2];
                double d = dal[c][0] * sigma * dSd;
                for (int r = 0; r < 3; ++r) d += dal[c][1 + r] * sigma * K[r][q2];
                Fm[c][q2] = (c == q2 ? 1.0 : 0.0) - g * d;  // I - F
            }
        // (I - F) D alpha = f0 by Cramer's rule, component by component of the affine forms
        const double det = Fm[0][0] * (Fm[1][1] * Fm[2][2] - Fm[1][2] * Fm[2][1]) -
                           Fm[0][1] * (Fm[1][0] * Fm[2][2] - Fm[1][2] * Fm[2][0]) +
                           Fm[0][2] * (Fm[1][0] * Fm[2][1] - Fm[1][1] * Fm[2][0]);
        const double id = 1.0 / det;
        double Mi[3][3];
        Mi[0][0] = (Fm[1][1] * Fm[2][2] - Fm[1][2] * Fm[2][1]) * id;
        Mi[0][1] = (Fm[0][2] * Fm[2][1] - Fm[0][1] * Fm[2][2]) * id;
        Mi[0][2] = (Fm[0][1] * Fm[1][2] - Fm[0][2] * Fm[1][1]) * id;
        Mi[1][0] = (Fm[1][2] * Fm[2][0] - Fm[1][0] * Fm[2][2]) * id;
        Mi[1][1] = (Fm[0][0] * Fm[2][2] - Fm[0][2] * Fm[2][0]) * id;
        Mi[1][2] = (Fm[0][2] * Fm[1][0] - Fm[0][0] * Fm[1][2]) * id;
        Mi[2][0] = (Fm[1][0] * Fm[2][1] - Fm[1][1] * Fm[2][0]) * id;
        Mi[2][1] = (Fm[0][1] * Fm[2][0] - Fm[0][0] * Fm[2][1]) * id;
        Mi[2][2] = (Fm[0][0] * Fm[1][1] - Fm[0][1] * Fm[1][0]) * id;
        Aff Dal[3], Dchk[3];
        for (int c = 0; c < 3; ++c) Dal[c] = Mi[c][0] * f0[0] + Mi[c][1] * f0[1] + Mi[c][2] * f0[2];
        chain(Dal, dNd, dS, Dchk);
    }
    Aff ds = sigma * dS + (s * isg) * dsg;
    Aff dPi = sigma * dBv + Bv * dsg;
    // dn_q = N_q dsigma + sigma dN_q
    Aff dw = (T + ps) * ds + (((mu0 + pn0) * nq0 + (mu1 + pn1) * nq1 + (mu2 + pn2) * nq2) * isg) * dsg + dPi +
             aff(sigma * ((mu0 + pn0) * dN[0] + (mu1 + pn1) * dN[1] + (mu2 + pn2) * dN[2])) +
             sigma * ((mu0 + pn0) * dNd[0] + (mu1 + pn1) * dNd[1] + (mu2 + pn2) * dNd[2]);
    double w = e + p + Pi;
    double ig2 = ig * ig, ig3 = ig2 * ig;
    double Px0 = ux * Pvxx + uy * Pvxy, Py0 = ux * Pvxy + uy * Pvyy;
    Aff dPx = (ux * isg) * dw + (w * isg) * ax - (w * ux * isg * isg) * dsg +
              ig2 * (Pvxx * ax + Pvxy * ay + ux * dPxx + uy * dPxy) - (2.0 * Px0 * ig3) * dg;
    Aff dPy = (uy * isg) * dw + (w * isg) * ay - (w * uy * isg * isg) * dsg +
              ig2 * (Pvxy * ax + Pvyy * ay + ux * dPxy + uy * dPyy) - (2.0 * Py0 * ig3) * dg;
    double r0 = Fx - dPx.c, r1 = Fy - dPy.c;
    double det = dPx.x * dPy.y - dPx.y * dPy.x;
    uint32_t st = 0;
    double acx = 0.0, acy = 0.0;
    if (isfinite(det) && det != 0.0) {
        double idet = 1.0 / det;
        acx = (r0 * dPy.y - dPx.y * r1) * idet;
        acy = (dPx.x * r1 - dPy.x * r0) * idet;
    } else {
        st |= PST_SOLVE_FAIL;
    }
    double f[kJRow + 6];
    f[0] = vx;
    f[1] = vy;
    f[2] = acx;
    f[3] = acy;
    f[4] = at(dS, acx, acy);
    f[5] = at(dBv, acx, acy);
    f[6] = at(dPxx, acx, acy);
    f[7] = at(dPxy, acx, acy);
    f[8] = at(dPyy, acx, acy);
    if (v.diff) {
        for (int q = 0; q < 3; ++q) {
            f[kJRow + 2 * q] = at(dJhx[q], acx, acy);
            f[kJRow + 2 * q + 1] = at(dJhy[q], acx, acy);
            dN[q] += dNt[q];  // the lab charges: sources and the flux divergence
        }
    }
    bool fin = true;
    for (int k = 0; k < nv; ++k) fin = fin && isfinite(f[k]);
    if (!fin) st |= PST_NONFINITE;
    if (st) {
        status[a] |= st;
        atomicOr(&v.sc->status_or, st);
    }
    if (mode == 0) {
        for (int k = 0; k < nv; ++k) yout[k * n + a] = ys[k * n + a] + dt * f[k];
    } else if (mode == 1) {
        for (int k = 0; k < nv; ++k) yout[k * n + a] = 0.5 * ((yout[k * n + a] + ys[k * n + a]) + dt * f[k]);
    } else {
        for (int k = 0; k < nv; ++k) rates[k * n + a] = f[k];
    }
    heun_charges(v, mode, n, a, dN);
}

__global__ void __launch_bounds__(128) k_eom2(EvView v, int stage, int mode, const double *__restrict__ ys,
                                              const double *__restrict__ dens, const double *__restrict__ eos,
                                              const double *__restrict__ gout, double *__restrict__ yout,
                                              double *__restrict__ rates, uint32_t *__restrict__ status)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    eom2_particle(v, stage, mode, (size_t)v.n, (size_t)a, ys, dens, eos, gout, yout, rates, status);
}

// Serving form: the equations of motion over the segmented arena (persistent grid)
__global__ void __launch_bounds__(128) k_eom2_seg(Arena A, int stage, int mode, const double *__restrict__ ys,
                                                  double *__restrict__ yout, int grp)
{
    const BatchTable *T = A.tab;
    const int hi = T->hi;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < hi; a += gridDim.x * blockDim.x) {
        const int s = A.segid[a];
        if (s < 0 || !seg_active(T, s, stage, true) || !in_group(T, s, grp)) continue;
        if (a - T->slots[s].off >= T->slots[s].n) continue;
        eom2_particle(A.segv[s], stage, mode, (size_t)A.P, (size_t)a, ys, A.dens, A.eosf, A.gout, yout, nullptr,
                      A.status);
    }
}

// stage work rate: fixed-order tree sum of the per-block partials; stage 2
// closes the step (Heun quadrature of the work integral, tau += dtau)
__global__ void __launch_bounds__(256) k_work_finish(EvView v, int stage, const double *__restrict__ wpart, int nblk)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += 256) acc += wpart[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
        (void)tau;
        v.sc->wr[stage - 1] = v.milne ? sh[0] : 0.0;
        if (stage == 2) {
            v.sc->work += 0.5 * v.dtau * (v.sc->wr[0] + v.sc->wr[1]);
            v.sc->tau = v.sc->tau + v.dtau;
            v.sc->steps += 1;
        }
    }
}

// per-particle totals contributions in ORIGINAL order: [0] sqrt(-g) T^{00}/sigma*, [1] S
__global__ void k_totals2(EvView v, const double *__restrict__ y, const int *__restrict__ id,
                          const double *__restrict__ dens, const double *__restrict__ eos, double *__restrict__ contrib)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    double tau = v.sc->tau;
    double sqrtg = v.milne ? tau : 1.0;
    double sig_star = dens[a], g = dens[5 * n + a];
    double sigma = sig_star / (g * sqrtg);
    double ux = y[2 * n + a], uy = y[3 * n + a];
    double vx = ux / g, vy = uy / g;
    double Pi = 0.0, ptt = 0.0;
    if (v.tr.viscous) {
        Pi = sigma * y[5 * n + a];
        double pxx = sigma * y[6 * n + a], pxy = sigma * y[7 * n + a], pyy = sigma * y[8 * n + a];
        ptt = vx * (vx * pxx + vy * pxy) + vy * (vx * pxy + vy * pyy);
    }
    double p = eos[4 * n + a], e = eos[5 * n + a];
    double T00 = (e + p + Pi) * g * g - (p + Pi) + ptt;
    int o = id[a];
    contrib[o] = sqrtg * T00 / sig_star;
    contrib[n + o] = y[4 * n + a];
}

// fixed-order sums of nfield rows of n values: block partials over fixed chunks,
// then one block sums the partials in order
__global__ void __launch_bounds__(256) k_sum_rows(const double *__restrict__ vals, int n, int nfield,
                                                  double *__restrict__ part, int chunk)
{
    __shared__ double sh[256];
    int f = blockIdx.y;
    int b = blockIdx.x;
    double acc = 0.0;
    int lo = b * chunk, hi = min(lo + chunk, n);
    for (int i = lo + threadIdx.x; i < hi; i += 256) acc += vals[(size_t)f * n + i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)f * gridDim.x + b] = sh[0];
}

__global__ void k_sum_final(const double *__restrict__ part, int nb, int nfield, double *out)
{
    int f = threadIdx.x;
    if (f >= nfield) return;
    double acc = 0.0;
    for (int b = 0; b < nb; ++b) acc += part[(size_t)f * nb + b];
    out[f] = acc;
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_gradient(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                     cudaStream_t st)
{
    if (v.dim == 3) {
        launch_gradient3(v, stage, y, gin, cb, gout, st);
        return;
    }
    if (v.mixed) {
        launch_gradient2m(v, stage, y, gin, cb, gout, st);
        return;
    }
    const int lists = cb.pl.total > 0;
    if (lists) launch_pairs_gradient(v, stage, y, gin, cb, gout, st);
    const int grid = lists ? std::min(nblk(v.n, kWarps), 8 * device_sm_count()) : nblk(v.n, kWarps);
    k_gradient2<<<grid, 32 * kWarps, 0, st>>>(v, stage, y, cb.fpos, gin, cb.start, cb.cnt, gout, lists);
}

void launch_eom(const EvView &v, int stage, int mode, const double *ys, const double *dens, const double *eos,
                const double *gout, double *yout, double *rates, uint32_t *status, cudaStream_t st)
{
    if (v.dim == 3) {
        launch_eom3(v, stage, mode, ys, dens, eos, gout, yout, rates, status, st);
        return;
    }
    k_eom2<<<nblk(v.n, 128), 128, 0, st>>>(v, stage, mode, ys, dens, eos, gout, yout, rates, status);
}

void launch_eom2_seg(const Arena &A, int stage, int mode, const double *ys, double *yout, int grid,
                     cudaStream_t st, int grp)
{
    k_eom2_seg<<<grid, 128, 0, st>>>(A, stage, mode, ys, yout, grp);
}

void launch_work_finish(const EvView &v, int stage, const double *wpart, int nb, cudaStream_t st)
{
    k_work_finish<<<1, 256, 0, st>>>(v, stage, wpart, nb);
}

void launch_totals(const EvView &v, const double *y, const double *Nq, const int *id, const double *dens,
                   const double *eos, double *contrib, cudaStream_t st)
{
    (void)Nq;
    if (v.dim == 3) {
        launch_totals3(v, y, id, dens, eos, contrib, st);
        return;
    }
    k_totals2<<<nblk(v.n, 256), 256, 0, st>>>(v, y, id, dens, eos, contrib);
}

// out[f] = fixed-order sum of vals[f*n .. f*n + n); scratch after out (needs nfield*256 doubles)
void launch_sum_fixed(const double *vals, int n, int nfield, double *out, cudaStream_t st)
{
    int chunk = 4096;
    int nb = max(1, min(256, nblk(n, chunk)));
    chunk = max(1, nblk(n, nb));
    nb = max(1, nblk(n, chunk));
    double *part = out + 8;
    dim3 grid(nb, nfield);
    k_sum_rows<<<grid, 256, 0, st>>>(vals, n, nfield, part, chunk);
    k_sum_final<<<1, 32, 0, st>>>(part, nb, nfield, out);
}

}  // namespace sphg
