// freezeout.cu -- freeze-out hypersurface elements at constant energy density (Sec.
// "Freeze-out hypersurface construction"), 2+1D and 3+1D (Milne or Cartesian), run in the first
// stage of every step on the stage's sorted particles, after the EoS pass:
//   a particle whose e fell through e_fo since the previous step's first stage (eprev > e_fo >= e)
//   yields one element at the current state:
//     d_i e_a = sum_b (e_b / sigma*_b) d_i W_ab                    (SPH derivative, n = 0 form)
//     d_tau e = (e - eprev) / dtau - v^i d_i e                      (particle rate minus advection)
//     n_mu = N_mu / sqrt(|N_mu N^mu|), N_mu = -d_mu e               (covariant, "outward";
//                                     N_mu N^mu = N_0^2 - N_1^2 - N_2^2 - N_3^2 / tau^2 in Milne)
//     |dsigma| = 1 / (sigma |u^mu n_mu|), dsigma_mu = |dsigma| n_mu (unit SPH mass)
// One warp per particle; a warp whose particle did not cross only updates eprev, so the pass
// costs little; crossing particles sum over their 3x3 cells in FP64 with the exact neighbour
// test (the oracle's neighbour set; 3x3x3 cells in 3+1D, distances Euclidean in (x, y, eta)).
// Records go to a fixed-capacity buffer through an atomic counter; the read-out sorts them by
// (tau, particle id).
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kFoWarps = 4;

__global__ void __launch_bounds__(32 * kFoWarps) k_freezeout2(EvView v, double e_fo, const double *__restrict__ y,
                                                              const int *__restrict__ id,
                                                              const double *__restrict__ dens,
                                                              const double *__restrict__ eosf,
                                                              double *__restrict__ eprev,
                                                              const uint32_t *__restrict__ start,
                                                              const uint32_t *__restrict__ cnt, FoBuf fo)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kFoWarps + wid;
    if (a >= v.n) return;  // warp-uniform
    const size_t n = (size_t)v.n;
    const double e = eosf[5 * n + a];
    const double ep = eprev[a];
    __syncwarp();
    if (lane == 0) eprev[a] = e;
    if (!(ep > e_fo && e <= e_fo)) return;
    const double xa = y[a], ya = y[n + a];
    const int cx = cell_coord(xa, dec_double(v.sc->xmin_enc[0]), v.inv_cell);
    const int cy = cell_coord(ya, dec_double(v.sc->xmin_enc[1]), v.inv_cell);
    const int lim = 1 << v.B;
    double dx_e = 0.0, dy_e = 0.0;
    for (int oy = -1; oy <= 1; ++oy) {
        const int ny = cy + oy;
        if (ny < 0 || ny >= lim) continue;
        for (int ox = -1; ox <= 1; ++ox) {
            const int nx = cx + ox;
            if (nx < 0 || nx >= lim) continue;
            const uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
            const uint32_t b1 = start[k] + cnt[k];
            for (uint32_t b = start[k] + lane; b < b1; b += 32) {
                const double ddx = xa - y[b], ddy = ya - y[n + b];
                const double r2 = dist2_2d(ddx, ddy);
                if (r2 < v.supp2 && r2 > 0.0) {
                    const double ir = inv_sqrt(r2);
                    const double fac = kernel_dw(r2 * ir * v.inv_h) * ir;  // (dW/dr)/r without sigma_d/h
                    const double eb = eosf[5 * n + b] / dens[b];
                    dx_e = fma(eb * fac, ddx, dx_e);
                    dy_e = fma(eb * fac, ddy, dy_e);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        dx_e += __shfl_xor_sync(0xFFFFFFFFu, dx_e, o);
        dy_e += __shfl_xor_sync(0xFFFFFFFFu, dy_e, o);
    }
    if (lane != 0) return;
    const double c = v.sigma_d * v.inv_h;
    dx_e *= c;
    dy_e *= c;
    const double tau = v.sc->tau;
    const double sqrtg = v.milne ? tau : 1.0;
    const double u0 = dens[5 * n + a], ux = y[2 * n + a], uy = y[3 * n + a];
    const double adv = (ux / u0) * dx_e + (uy / u0) * dy_e;
    const double N0 = -((e - ep) / v.dtau - adv), N1 = -dx_e, N2 = -dy_e;
    const double norm = sqrt(fabs(N0 * N0 - N1 * N1 - N2 * N2));  // N_mu N^mu, diagonal metric
    const double n0 = N0 / norm, n1 = N1 / norm, n2 = N2 / norm;
    const double un = u0 * n0 + ux * n1 + uy * n2;
    const double sigma = dens[a] / (u0 * sqrtg);
    const double dsig = 1.0 / (sigma * fabs(un));
    const unsigned long long slot = atomicAdd(fo.count, 1ull);
    if (slot >= fo.cap) return;
    double *r = fo.rec + slot * kFoRec;
    r[0] = tau;
    r[1] = xa;
    r[2] = ya;
    r[3] = 0.0;
    r[4] = u0;
    r[5] = ux;
    r[6] = uy;
    r[7] = 0.0;
    for (int k = 0; k < 4; ++k) r[8 + k] = eosf[(size_t)k * n + a];  // T, mu_B, mu_S, mu_Q
    r[12] = e;
    r[13] = eosf[4 * n + a];
    r[14] = dens[n + a];  // rest-frame s (the EoS pass converted it)
    r[15] = n0;
    r[16] = n1;
    r[17] = n2;
    r[18] = 0.0;
    r[19] = dsig;
    r[20] = dsig * n0;
    r[21] = dsig * n1;
    r[22] = dsig * n2;
    r[23] = 0.0;
    fo.ids[slot] = id[a];
}

// 3+1D: the same element with the gradient over the 27 neighbouring cells (generalized Morton
// keys) and the third components: x^3 = eta (Milne, in fm) or z, u^3 = u^eta or u^z, and the
// covariant n_3 normalised with g^{33} = -1/tau^2 (Milne) or -1
__global__ void __launch_bounds__(32 * kFoWarps) k_freezeout3(EvView v, double e_fo, const double *__restrict__ y,
                                                              const int *__restrict__ id,
                                                              const double *__restrict__ dens,
                                                              const double *__restrict__ eosf,
                                                              double *__restrict__ eprev,
                                                              const uint32_t *__restrict__ start,
                                                              const uint32_t *__restrict__ cnt, FoBuf fo)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kFoWarps + wid;
    if (a >= v.n) return;  // warp-uniform
    const size_t n = (size_t)v.n;
    const double e = eosf[5 * n + a];
    const double ep = eprev[a];
    __syncwarp();
    if (lane == 0) eprev[a] = e;
    if (!(ep > e_fo && e <= e_fo)) return;
    const double xa[3] = {y[a], y[n + a], y[2 * n + a]};
    int c[3], lim[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = cell_coord(xa[d], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
        lim[d] = 1 << v.B3[d];
    }
    double de[3] = {0.0, 0.0, 0.0};
    for (int oz = -1; oz <= 1; ++oz) {
        const int nz = c[2] + oz;
        if (nz < 0 || nz >= lim[2]) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            const int ny = c[1] + oy;
            if (ny < 0 || ny >= lim[1]) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int nx = c[0] + ox;
                if (nx < 0 || nx >= lim[0]) continue;
                const uint32_t k = key3(v, nx, ny, nz);
                const uint32_t b1 = start[k] + cnt[k];
                for (uint32_t b = start[k] + lane; b < b1; b += 32) {
                    const double d0 = xa[0] - y[b], d1 = xa[1] - y[n + b], d2 = xa[2] - y[2 * n + b];
                    const double r2 = dist2_3d(d0, d1, d2);
                    if (r2 < v.supp2 && r2 > 0.0) {
                        const double ir = inv_sqrt(r2);
                        const double f = kernel_dw(r2 * ir * v.inv_h) * ir * (eosf[5 * n + b] / dens[b]);
                        de[0] = fma(f, d0, de[0]);
                        de[1] = fma(f, d1, de[1]);
                        de[2] = fma(f, d2, de[2]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) de[d] += __shfl_xor_sync(0xFFFFFFFFu, de[d], o);
    if (lane != 0) return;
    const double cg = v.sigma_d * v.inv_h;
    const double tau = v.sc->tau;
    const double sqrtg = v.milne ? tau : 1.0;
    const double g33 = v.milne ? 1.0 / (tau * tau) : 1.0;  // -g^{33}
    const double u0 = dens[5 * n + a];
    const double u[3] = {y[3 * n + a], y[4 * n + a], y[5 * n + a]};
    double adv = 0.0;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        de[d] *= cg;
        adv += (u[d] / u0) * de[d];
    }
    const double N[4] = {-((e - ep) / v.dtau - adv), -de[0], -de[1], -de[2]};
    const double norm = sqrt(fabs(N[0] * N[0] - N[1] * N[1] - N[2] * N[2] - N[3] * N[3] * g33));
    double nv[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) nv[m] = N[m] / norm;
    const double un = u0 * nv[0] + u[0] * nv[1] + u[1] * nv[2] + u[2] * nv[3];
    const double sigma = dens[a] / (u0 * sqrtg);
    const double dsig = 1.0 / (sigma * fabs(un));
    const unsigned long long slot = atomicAdd(fo.count, 1ull);
    if (slot >= fo.cap) return;
    double *r = fo.rec + slot * kFoRec;
    r[0] = tau;
    for (int d = 0; d < 3; ++d) r[1 + d] = xa[d];
    r[4] = u0;
    for (int d = 0; d < 3; ++d) r[5 + d] = u[d];
    for (int k = 0; k < 4; ++k) r[8 + k] = eosf[(size_t)k * n + a];  // T, mu_B, mu_S, mu_Q
    r[12] = e;
    r[13] = eosf[4 * n + a];
    r[14] = dens[n + a];  // rest-frame s (the EoS pass converted it)
    for (int m = 0; m < 4; ++m) r[15 + m] = nv[m];
    r[19] = dsig;
    for (int m = 0; m < 4; ++m) r[20 + m] = dsig * nv[m];
    fo.ids[slot] = id[a];
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_freezeout(const EvView &v, double e_fo, const double *y, const int *id, const double *dens,
                      const double *eosf, double *eprev, CellBufs cb, FoBuf fo, cudaStream_t st)
{
    if (v.dim == 3)
        k_freezeout3<<<nblk(v.n, kFoWarps), 32 * kFoWarps, 0, st>>>(v, e_fo, y, id, dens, eosf, eprev, cb.start,
                                                                    cb.cnt, fo);
    else
        k_freezeout2<<<nblk(v.n, kFoWarps), 32 * kFoWarps, 0, st>>>(v, e_fo, y, id, dens, eosf, eprev, cb.start,
                                                                    cb.cnt, fo);
}

}  // namespace sphg
