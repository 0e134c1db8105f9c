// diffusion.cu -- BSQ diffusion in 2+1D (Sec. "Equations of motion", eq. min_dif_rel, with the
// constant kappa_{qq'}/T^2 and tau_q T of Sec. "Transport coefficients"): the per-particle inputs
// and the neighbour sums of a stage.  The equations of motion (gradient_eom.cu) take them.
//
// Per particle a (sorted order of the stage):
//   alpha_q = mu_q / T; the flux of the lab charge relative to the particle, F^i_q = J^i_q -
//   v^i J^0_q (J^0 = u.J / u^0 from u_mu J^mu = 0), as F^i_q / sigma*^2; and d alpha_q / d(s, n)
//   = (d mu_q - alpha_q dT) / T with (dT, dmu) = H^-1 (ds, dn), H = d(s, n)/d(T, mu) of the EoS
//   branch that gave the particle's (T, mu) (the table, the closed form or the backup);
//   d_i alpha_q = (1 / sigma*_a) sum_b (alpha_qb - alpha_qa) d_i W_ab  (the SPH derivative with
//   n = 1: zero for a uniform alpha, so a uniform mu/T drives no current);
//   d(lab charge)/dx0 = -sqrt(-g) sum_b (F_a / sigma*_a^2 + F_b / sigma*_b^2) . grad W_ab (n = -1:
//   each pair moves charge from one particle to the other, so the total is conserved).
#include "sph_internal.cuh"
#include "eos_device.cuh"

namespace sphg {

namespace {

constexpr int kDiffWarps = 4;

__global__ void __launch_bounds__(128) k_diff_prep(EvView v, int stage, const double *__restrict__ y,
                                                   const double *__restrict__ dens, const double *__restrict__ eos,
                                                   const uint32_t *__restrict__ status)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
    const double sqrtg = v.milne ? tau : 1.0;
    const double sig_star = dens[a], u0 = dens[5 * n + a];
    const double sigma = sig_star / (u0 * sqrtg);
    const double ux = y[2 * n + a], uy = y[3 * n + a];
    const double vx = ux / u0, vy = uy / u0;
    const double T = eos[a];
    const uint32_t st = status[a];
    const bool ok = !(st & (PST_NOCONV | PST_NONFINITE)) && T > 0.0;
    const double i2 = 1.0 / (sig_star * sig_star);
    double al[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double Jx = sigma * y[(kJRow + 2 * q) * n + a], Jy = sigma * y[(kJRow + 2 * q + 1) * n + a];
        const double J0 = (ux * Jx + uy * Jy) / u0;
        al[q] = ok ? eos[(1 + q) * n + a] / T : 0.0;
        v.dinp[q * n + a] = al[q];
        v.dinp[(3 + 2 * q) * n + a] = (Jx - vx * J0) * i2;
        v.dinp[(4 + 2 * q) * n + a] = (Jy - vy * J0) * i2;
    }
    double dal[3][4];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < 4; ++k) dal[q][k] = 0.0;
    if (ok) {
        const EosDev &E = v.eos;
        const double x[4] = {T, eos[n + a], eos[2 * n + a], eos[3 * n + a]};
        double H[4][4];
        const bool backup = (st & PST_BACKUP) != 0;
        const bool table = !backup && E.has_table && !(st & (PST_FALLBACK | PST_OUT_OF_TABLE));
        if (backup) {
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) H[i][j] = 0.0;
            H[0][0] = 12.0 * E.cd_A0 * T * T;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const double m0 = E.cd_mu0[q];
                H[1 + q][1 + q] = 12.0 * E.cd_A0 * x[1 + q] * x[1 + q] / (m0 * m0 * m0 * m0);
            }
        } else if (table) {
            double sn[4];
            tab_eval(E, x, sn, H, nullptr);
        } else {
            double p, sn[4];
            an_eval(E, x[0], x + 1, p, sn, H);
        }
        bool act[4];
        act[0] = true;
#pragma unroll
        for (int q = 0; q < 3; ++q) act[1 + q] = table || backup || E.chi[q] > 0.0;
        // H^-1 over the active directions, one column at a time (inactive rows and columns of H
        // replaced by the identity, their entries of the inverse then set to zero)
        double Hi[4][4];
        bool good = true;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            double A[4][4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                b[i] = i == f ? 1.0 : 0.0;
#pragma unroll
                for (int j = 0; j < 4; ++j) A[i][j] = (act[i] && act[j]) ? H[i][j] : (i == j ? 1.0 : 0.0);
            }
            good = good && solve4(A, b);
#pragma unroll
            for (int i = 0; i < 4; ++i) Hi[i][f] = (act[i] && act[f]) ? b[i] : 0.0;
        }
        if (good)
#pragma unroll
            for (int q = 0; q < 3; ++q)
#pragma unroll
                for (int f = 0; f < 4; ++f) dal[q][f] = (Hi[1 + q][f] - al[q] * Hi[0][f]) / T;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int f = 0; f < 4; ++f) v.dal[(4 * q + f) * n + a] = dal[q][f];
}

// the sums of particle a (lane 0 of its warp writes them): S = sum grad W, ga = sum (alpha_b -
// alpha_a) grad W, dv = sum F_b . grad W, lane partials reduced in a fixed butterfly order
__device__ __forceinline__ void diff_finish(const EvView &v, int stage, const double *__restrict__ dens, int a,
                                            int lane, double Gx, double Gy, double (&ga)[3][2], double (&dv)[3])
{
    const size_t n = (size_t)v.n;
    const double *F = v.dinp + 3 * n;
    for (int o = 16; o > 0; o >>= 1) {
        Gx += __shfl_xor_sync(0xFFFFFFFFu, Gx, o);
        Gy += __shfl_xor_sync(0xFFFFFFFFu, Gy, o);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            ga[q][0] += __shfl_xor_sync(0xFFFFFFFFu, ga[q][0], o);
            ga[q][1] += __shfl_xor_sync(0xFFFFFFFFu, ga[q][1], o);
            dv[q] += __shfl_xor_sync(0xFFFFFFFFu, dv[q], o);
        }
    }
    if (lane == 0) {
        const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
        const double sqrtg = v.milne ? tau : 1.0;
        const double c = v.sigma_d * v.inv_h;
        const double isig = 1.0 / dens[a];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            v.dout[(2 * q) * n + a] = c * ga[q][0] * isig;
            v.dout[(2 * q + 1) * n + a] = c * ga[q][1] * isig;
            const double div = F[(2 * q) * n + a] * Gx + F[(2 * q + 1) * n + a] * Gy + dv[q];
            v.dout[(6 + q) * n + a] = -sqrtg * c * div;
        }
    }
}

// pair-list form (plain 2D events): one warp per particle over its accepted pairs, with the
// kernel gradient the density pass stored per pair (grad_a W_ab h / sigma_d: b > a forward in
// a's row, b < a as minus the entry in b's row), so no distance or kernel is evaluated again
__global__ void __launch_bounds__(32 * kDiffWarps) k_diff_pairs(EvView v, int stage, const double *__restrict__ dens,
                                                                PairBufs pl)
{
    if (v.sc->pair_flag) return;  // a list overflowed: the cell pass runs instead
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kDiffWarps + wid;
    if (a >= v.n) return;  // warp-uniform
    const size_t n = (size_t)v.n;
    const double *al = v.dinp, *F = v.dinp + 3 * n;
    const double aa[3] = {al[a], al[n + a], al[2 * n + a]};
    const long long r0 = pl.off[a], rend = pl.off[a + 1] - 1;
    const int nf = pl.cntF[a], nt = nf + pl.cntB[a];
    double ga[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}}, dv[3] = {0.0, 0.0, 0.0}, Gx = 0.0, Gy = 0.0;
    for (int j = lane; j < nt; j += 32) {
        int b;
        double gx, gy;
        if (j < nf) {
            b = pl.L[r0 + j];
            const double2 g = pl.G[r0 + j];
            gx = g.x;
            gy = g.y;
        } else {
            b = pl.L[rend - (j - nf)];
            const double2 g = pl.G[pl.off[b] + pl.P[rend - (j - nf)]];
            gx = -g.x;
            gy = -g.y;
        }
        Gx += gx;
        Gy += gy;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double da = al[q * n + b] - aa[q];
            ga[q][0] = fma(da, gx, ga[q][0]);
            ga[q][1] = fma(da, gy, ga[q][1]);
            dv[q] = fma(F[(2 * q) * n + b], gx, fma(F[(2 * q + 1) * n + b], gy, dv[q]));
        }
    }
    diff_finish(v, stage, dens, a, lane, Gx, Gy, ga, dv);
}

// one warp per particle: the 3x3 cells of side 2h around its own, the exact FP64 test r < 2h on
// every candidate (the neighbour set of the other passes).  The mixed-precision form's pass,
// and the plain form's when a pair list overflowed (fallback: it returns at once otherwise).
__global__ void __launch_bounds__(32 * kDiffWarps) k_diff2(EvView v, int stage, const double *__restrict__ y,
                                                           const double *__restrict__ dens,
                                                           const uint32_t *__restrict__ start,
                                                           const uint32_t *__restrict__ cnt, int fallback)
{
    if (fallback && !v.sc->pair_flag) return;  // the pair-list pass did the work
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const size_t n = (size_t)v.n;
    const double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
    const int lim = 1 << v.B;
    const double *al = v.dinp, *F = v.dinp + 3 * n;
    for (int a = blockIdx.x * kDiffWarps + wid; a < v.n; a += gridDim.x * kDiffWarps) {  // warp-uniform
        const double xa = y[a], ya = y[n + a];
        const int cx = cell_coord(xa, xmin0, v.inv_cell), cy = cell_coord(ya, xmin1, v.inv_cell);
        const double aa[3] = {al[a], al[n + a], al[2 * n + a]};
        double ga[3][2] = {{0.0, 0.0}, {0.0, 0.0}, {0.0, 0.0}}, dv[3] = {0.0, 0.0, 0.0}, Gx = 0.0, Gy = 0.0;
        for (int oy = -1; oy <= 1; ++oy) {
            const int ny = cy + oy;
            if (ny < 0 || ny >= lim) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int nx = cx + ox;
                if (nx < 0 || nx >= lim) continue;
                const uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
                const uint32_t b1 = start[k] + cnt[k];
                for (uint32_t b = start[k] + lane; b < b1; b += 32) {
                    const double dx = xa - y[b], dy = ya - y[n + b];
                    if (!(dist2_2d(dx, dy) < v.supp2)) continue;
                    const double r2 = fma(dx, dx, dy * dy);
                    if (!(r2 > 0.0)) continue;  // grad W = 0 at r = 0
                    const double ir = inv_sqrt(r2);
                    const double fac = kernel_dw(r2 * ir * v.inv_h) * ir;  // (dW/dr)/r without sigma_d/h
                    const double gx = fac * dx, gy = fac * dy;
                    Gx += gx;
                    Gy += gy;
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const double da = al[q * n + b] - aa[q];
                        ga[q][0] = fma(da, gx, ga[q][0]);
                        ga[q][1] = fma(da, gy, ga[q][1]);
                        dv[q] = fma(F[(2 * q) * n + b], gx, fma(F[(2 * q + 1) * n + b], gy, dv[q]));
                    }
                }
            }
        }
        diff_finish(v, stage, dens, a, lane, Gx, Gy, ga, dv);
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_diffusion(const EvView &v, int stage, const double *y, const double *dens, const double *eos,
                      const uint32_t *status, CellBufs cb, cudaStream_t st)
{
    if (!v.diff || v.n <= 0) return;
    k_diff_prep<<<nblk(v.n, 128), 128, 0, st>>>(v, stage, y, dens, eos, status);
    // the plain form keeps pair lists: the pass over them, with the cell pass standing by (at a
    // few blocks per SM) for a stage whose lists overflowed
    const int lists = !v.mixed && cb.pl.total > 0;
    if (lists) k_diff_pairs<<<nblk(v.n, kDiffWarps), 32 * kDiffWarps, 0, st>>>(v, stage, dens, cb.pl);
    const int grid = lists ? std::min(nblk(v.n, kDiffWarps), 8 * device_sm_count()) : nblk(v.n, kDiffWarps);
    k_diff2<<<grid, 32 * kDiffWarps, 0, st>>>(v, stage, y, dens, cb.start, cb.cnt, lists);
}

}  // namespace sphg
