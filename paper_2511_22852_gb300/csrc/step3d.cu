// step3d.cu -- the SPH step in three spatial dimensions: 3+1D Milne (tau, x, y, eta_s)
// and 3+1D Cartesian (t, x, y, z).  Same rows as the 2+1D kernels (a1-a8):
//   cells      generalized Morton key of the cell (per-axis bit counts, spread tables)
//   density    27-cell kernel sums, one warp per particle, single-precision prefilter
//   eos        u^0 = sqrt(1 - g_ij u^i u^j), rest-frame densities, inversion, X^{ji}/sigma*^2
//   gradient   27-cell n = 0 velocity gradients and n = -1 stress divergence
//   eom        covariant minimal Israel-Stewart equations with explicit Christoffel
//              symbols (Milne: Gamma^tau_{eta eta} = tau, Gamma^eta_{tau eta} = 1/tau),
//              every rate affine in the three acceleration components
// Distances are Euclidean in (x, y, eta) with eta taken in fm (Sec. "Kernel function").
// State rows (nv = 13): x^1..3, u^1..3, S, Pi/sigma, pi^{ij}/sigma for (11, 12, 13, 22, 23);
// pi^{33} follows from tracelessness, pi^{0 mu} from transversality.
#include "eos_device.cuh"
#include <algorithm>

#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kWarps3 = 4;

// ---------------------------------------------------------------------------
// a1: cell coordinates, keys and bucket counts
__global__ void k_cells3(EvView v, const double *__restrict__ y, uint32_t *key, uint32_t *cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n) return;
    int c[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = cell_coord(y[(size_t)d * v.n + i], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
        const int lim = 1 << v.B3[d];
        if (c[d] < 0 || c[d] >= lim) {
            bad = true;
            c[d] = min(max(c[d], 0), lim - 1);
        }
    }
    if (bad) atomicOr(&v.sc->err_flags, ERR_CELL_OVERFLOW);
    uint32_t k = key3(v, c[0], c[1], c[2]);
    key[i] = k;
    atomicAdd(&cnt[k], 1u);
}

__global__ void k_fpos3(EvView v, const double *__restrict__ y, float4 *__restrict__ fpos)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= v.n) return;
    float f[3];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        f[d] = __double2float_rn(__dsub_rn(y[(size_t)d * v.n + j], dec_double(v.sc->xmin_enc[d])));
    fpos[j] = make_float4(f[0], f[1], f[2], 0.0f);
}

// the 27-cell candidate walk of one warp: prefilter, compaction, then `pair` on full warps
template <class Pair>
__device__ __forceinline__ void walk27(const EvView &v, const uint32_t *__restrict__ start,
                                       const uint32_t *__restrict__ cnt, const float4 *__restrict__ fpos, int a,
                                       const double *xa, int *q, Pair &pair)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const float4 fa = fpos[a];
    int c[3], lim[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = cell_coord(xa[d], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
        lim[d] = 1 << v.B3[d];
    }
    int qn = 0;
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
                const uint32_t b0 = start[k], b1 = b0 + cnt[k];
                for (uint32_t base = b0; base < b1; base += 32) {
                    const uint32_t b = base + lane;
                    bool cand = false, sure = false;
                    if (b < b1) {
                        const float4 fb = fpos[b];
                        const float dx = fa.x - fb.x, dy = fa.y - fb.y, dz = fa.z - fb.z;
                        const float r2f = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        cand = r2f <= v.supp2_hi;
                        sure = r2f < v.supp2_lo;
                    }
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
                    // bit 31 set: the float test left the pair undecided (exact test needed)
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
    }
    if (lane < qn) pair(q[lane]);
}

__device__ __forceinline__ double warp_sum(double x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// ---------------------------------------------------------------------------
// a3: kernel sums (lab frame); u^0 and the rest-frame division happen in the EoS pass
__global__ void __launch_bounds__(32 * kWarps3) k_density3(EvView v, const double *__restrict__ y,
                                                           const float4 *__restrict__ fpos,
                                                           const double *__restrict__ Nq,
                                                           const uint32_t *__restrict__ start,
                                                           const uint32_t *__restrict__ cnt, double *__restrict__ dens,
                                                           int *__restrict__ nnb, int fallback, int *__restrict__ cnt_dst)
{
    // fallback = 1: the pair-list passes ran first; this pass only runs if one of their lists
    // overflowed (and counts such stages)
    if (fallback) {
        if (!v.sc->pair_flag) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&v.sc->pair_ovf, 1u);
    }
    __shared__ int queue[kWarps3][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // grid-stride over particles (one warp each): launched at a few blocks per SM when it is
    // only the fallback of the pair-list passes
    for (int a = blockIdx.x * kWarps3 + wid; a < v.n; a += gridDim.x * kWarps3) {  // warp-uniform
        const size_t n = (size_t)v.n;
        const double *X = y, *Y = y + n, *Z = y + 2 * n, *S = y + 6 * n;
        const double xa[3] = {X[a], Y[a], Z[a]};
        double sg = 0.0, ss = 0.0, sb = 0.0, sS = 0.0, sq = 0.0;
        int c = 0;
        auto pair = [&](int qb) {
            const int b = qb & 0x7FFFFFFF;
            const double dx = xa[0] - X[b], dy = xa[1] - Y[b], dz = xa[2] - Z[b];
            if (qb < 0 && !(dist2_3d(dx, dy, dz) < v.supp2)) return;
            {
                const double r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                double q = r2 > 0.0 ? r2 * inv_sqrt(r2) * v.inv_h : 0.0;
                double w = kernel_w(q);
                sg += w;
                ss = fma(S[b], w, ss);
                sb = fma(Nq[b], w, sb);
                sS = fma(Nq[n + b], w, sS);
                sq = fma(Nq[2 * n + b], w, sq);
                ++c;
            }
        };
        walk27(v, start, cnt, fpos, a, xa, queue[wid], pair);
        sg = warp_sum(sg);
        ss = warp_sum(ss);
        sb = warp_sum(sb);
        sS = warp_sum(sS);
        sq = warp_sum(sq);
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if (lane == 0) {
            const double sd = v.sigma_d;
            dens[a] = sd * sg;
            dens[n + a] = sd * ss;
            dens[2 * n + a] = sd * sb;
            dens[3 * n + a] = sd * sS;
            dens[4 * n + a] = sd * sq;
            nnb[a] = c;
            if (cnt_dst) cnt_dst[a] = c;  // sizes the pair-list rows of the next stage
            atomicAdd(&v.sc->pairs, (unsigned long long)c);
        }
    }
}

// ---------------------------------------------------------------------------
// geometry of the stage: metric diag(1, -1, -1, g3), g3 = -tau^2 (Milne) or -1
struct Geo3 {
    double tau, g[4], gi[4], dg3, sqrtg;
    bool milne;
};
__device__ __forceinline__ Geo3 geo3(const EvView &v, int stage)
{
    Geo3 G;
    G.milne = v.milne != 0;
    G.tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
    G.g[0] = 1.0;
    G.g[1] = G.g[2] = -1.0;
    G.g[3] = G.milne ? -G.tau * G.tau : -1.0;
    for (int m = 0; m < 4; ++m) G.gi[m] = 1.0 / G.g[m];
    G.dg3 = G.milne ? -2.0 * G.tau : 0.0;
    G.sqrtg = G.milne ? G.tau : 1.0;
    return G;
}
// Christoffel symbols Gamma^a_{bc} of the Milne metric (zero in Cartesian coordinates)
__device__ __forceinline__ double gam(const Geo3 &G, int a, int b, int c)
{
    if (!G.milne) return 0.0;
    if (a == 0 && b == 3 && c == 3) return G.tau;
    if (a == 3 && ((b == 0 && c == 3) || (b == 3 && c == 0))) return 1.0 / G.tau;
    return 0.0;
}

// full contravariant pi^{mu nu} from the stored (11, 12, 13, 22, 23) components:
// pi^{33} from g_{mu nu} pi^{mu nu} = 0, pi^{0 nu} from u_mu pi^{mu nu} = 0
__device__ __forceinline__ void pi_full3(const Geo3 &G, const double *u, const double *st, double pi[4][4])
{
    double ul[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) ul[m] = G.g[m] * u[m];
    pi[1][1] = st[0];
    pi[1][2] = pi[2][1] = st[1];
    pi[1][3] = pi[3][1] = st[2];
    pi[2][2] = st[3];
    pi[2][3] = pi[3][2] = st[4];
    const double iu02 = 1.0 / (ul[0] * ul[0]);
    double known = (ul[1] * ul[1] * pi[1][1] + ul[2] * ul[2] * pi[2][2] + 2.0 * ul[1] * ul[2] * pi[1][2] +
                    2.0 * ul[1] * ul[3] * pi[1][3] + 2.0 * ul[2] * ul[3] * pi[2][3]) * iu02 +
                   G.g[1] * pi[1][1] + G.g[2] * pi[2][2];
    pi[3][3] = -known / (ul[3] * ul[3] * iu02 + G.g[3]);
#pragma unroll
    for (int i = 1; i < 4; ++i) {
        double acc = ul[1] * pi[1][i] + ul[2] * pi[2][i] + ul[3] * pi[3][i];
        pi[0][i] = pi[i][0] = -acc / ul[0];
    }
    pi[0][0] = -(ul[1] * pi[1][0] + ul[2] * pi[2][0] + ul[3] * pi[3][0]) / ul[0];
}

// a4: u^0, rest-frame densities, EoS, stress inputs of the gradient pass, work rate
__global__ void __launch_bounds__(64, 6) k_eos3(EvView v, int stage, const double *__restrict__ y,
                                                double *__restrict__ dens, double *__restrict__ eos,
                                                double *__restrict__ gin, uint32_t *__restrict__ status,
                                                double *__restrict__ wpart, const double *__restrict__ guess_in,
                                                double *__restrict__ guess_out)
{
    __shared__ double red[2];
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n = (size_t)v.n;
    double wcontrib = 0.0;
    unsigned wres = 0u, wsol = 0u, wg = 0u;
    if (a < v.n) {
        const Geo3 G = geo3(v, stage);
        double u[4] = {0.0, y[3 * n + a], y[4 * n + a], y[5 * n + a]};
        u[0] = sqrt(1.0 - (G.g[1] * u[1] * u[1] + G.g[2] * u[2] * u[2] + G.g[3] * u[3] * u[3]));
        const double sig_star = dens[a];
        const double vol = u[0] * G.sqrtg;
        const double s = dens[n + a] / vol;
        double nq[3] = {dens[2 * n + a] / vol, dens[3 * n + a] / vol, dens[4 * n + a] / vol};
        dens[n + a] = s;
        for (int q = 0; q < 3; ++q) dens[(2 + q) * n + a] = nq[q];
        dens[5 * n + a] = u[0];
        double gs[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) gs[k] = guess_in[(size_t)k * n + a];
        bool used = false;
        EosWork w = {0u, 0u, 0u};
        EosOut o = eos_invert(v.eos, v.tr.cs2_cap, s, nq, gs, used, w);
        wres = w.resid;
        wsol = w.solve;
        wg = w.g;
        guess_out[a] = used ? o.T : ((o.st & (PST_NOCONV | PST_NONFINITE | PST_BACKUP)) ? 0.0 : -o.T);
        for (int q = 0; q < 3; ++q) guess_out[(size_t)(1 + q) * n + a] = used ? o.mu[q] : 0.0;
        status[a] = o.st;
        warp_or(&v.sc->status_or, o.st);
        eos[a] = o.T;
        for (int q = 0; q < 3; ++q) eos[(1 + q) * n + a] = o.mu[q];
        eos[4 * n + a] = o.p;
        eos[5 * n + a] = o.e;
        eos[6 * n + a] = o.ps;
        for (int q = 0; q < 3; ++q) eos[(7 + q) * n + a] = o.pn[q];
        eos[10 * n + a] = o.cs2;
        const double sigma = sig_star / vol;
        double Pi = 0.0, st[5] = {0, 0, 0, 0, 0};
        if (v.tr.viscous) {
            Pi = sigma * y[7 * n + a];
#pragma unroll
            for (int k = 0; k < 5; ++k) st[k] = sigma * y[(8 + k) * n + a];
        }
        double pi[4][4];
        pi_full3(G, u, st, pi);
        const double inv2 = 1.0 / (sig_star * sig_star);
        const double P = o.p + Pi;
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                double X = (j == i ? -P * G.gi[1 + j] : 0.0) + pi[1 + j][1 + i] - (u[1 + j] / u[0]) * pi[0][1 + i];
                gin[(size_t)(3 * j + i) * n + a] = X * inv2;
            }
        for (int j = 0; j < 3; ++j) gin[(size_t)(9 + j) * n + a] = u[1 + j] / sig_star;
        if (G.milne) {
            // sqrt(-g) Gamma^0_{33} T^{33} / sigma* = tau^2 T^{eta eta} / sigma*
            const double T33 = (o.e + P) * u[3] * u[3] - P * G.gi[3] + pi[3][3];
            wcontrib = G.tau * G.tau * T33 / sig_star;
        }
    }
    wres = __reduce_add_sync(0xFFFFFFFFu, wres);
    wsol = __reduce_add_sync(0xFFFFFFFFu, wsol);
    wg = __reduce_add_sync(0xFFFFFFFFu, wg);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&v.sc->eos_resid, (unsigned long long)wres);
        atomicAdd(&v.sc->eos_solve, (unsigned long long)wsol);
        atomicAdd(&v.sc->eos_g, (unsigned long long)wg);
    }
    wcontrib = warp_sum(wcontrib);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = wcontrib;
    __syncthreads();
    if (threadIdx.x == 0) wpart[blockIdx.x] = red[0] + red[1];
}

// ---------------------------------------------------------------------------
// a5: gradients.  gin rows: X^{ji}/sigma*^2 at 3 j + i, u^j/sigma* at 9 + j.
// gout rows: d_k u^j at 3 k + j, then F^i at 9 + i.
__global__ void __launch_bounds__(32 * kWarps3) k_gradient3(EvView v, int stage, const double *__restrict__ y,
                                                            const float4 *__restrict__ fpos,
                                                            const double *__restrict__ gin,
                                                            const uint32_t *__restrict__ start,
                                                            const uint32_t *__restrict__ cnt,
                                                            double *__restrict__ gout, int fallback)
{
    if (fallback && !v.sc->pair_flag) return;  // the pair-list pass did the work
    __shared__ int queue[kWarps3][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // grid-stride over particles (one warp each): launched at a few blocks per SM when it is
    // only the fallback of the pair-list passes
    for (int a = blockIdx.x * kWarps3 + wid; a < v.n; a += gridDim.x * kWarps3) {  // warp-uniform
        const size_t n = (size_t)v.n;
        const double *X = y, *Y = y + n, *Z = y + 2 * n;
        const double xa[3] = {X[a], Y[a], Z[a]};
        double G[3] = {0, 0, 0}, H[3] = {0, 0, 0}, du[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        auto pair = [&](int qb) {
            const int b = qb & 0x7FFFFFFF;
            const double d[3] = {xa[0] - X[b], xa[1] - Y[b], xa[2] - Z[b]};
            if (qb < 0 && !(dist2_3d(d[0], d[1], d[2]) < v.supp2)) return;
            const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
            if (r2 > 0.0) {
                const double ir = inv_sqrt(r2);
                const double fac = kernel_dw(r2 * ir * v.inv_h) * ir;
                double gw[3];
    #pragma unroll
                for (int k = 0; k < 3; ++k) {
                    gw[k] = fac * d[k];
                    G[k] += gw[k];
                }
    #pragma unroll
                for (int i = 0; i < 3; ++i) {
                    double h = H[i];
    #pragma unroll
                    for (int j = 0; j < 3; ++j) h = fma(gin[(size_t)(3 * j + i) * n + b], gw[j], h);
                    H[i] = h;
                }
    #pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const double ub = gin[(size_t)(9 + j) * n + b];
    #pragma unroll
                    for (int k = 0; k < 3; ++k) du[k][j] = fma(ub, gw[k], du[k][j]);
                }
            }
        };
        walk27(v, start, cnt, fpos, a, xa, queue[wid], pair);
    #pragma unroll
        for (int k = 0; k < 3; ++k) {
            G[k] = warp_sum(G[k]);
            H[k] = warp_sum(H[k]);
    #pragma unroll
            for (int j = 0; j < 3; ++j) du[k][j] = warp_sum(du[k][j]);
        }
        if (lane == 0) {
            const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
            const double sqrtg = v.milne ? tau : 1.0;
            const double c = v.sigma_d * v.inv_h;
    #pragma unroll
            for (int k = 0; k < 3; ++k)
    #pragma unroll
                for (int j = 0; j < 3; ++j) gout[(size_t)(3 * k + j) * n + a] = c * du[k][j];
    #pragma unroll
            for (int i = 0; i < 3; ++i) {
                double F = H[i];
    #pragma unroll
                for (int j = 0; j < 3; ++j) F = fma(gin[(size_t)(3 * j + i) * n + a], G[j], F);
                gout[(size_t)(9 + i) * n + a] = -sqrtg * c * F;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// a6/a7: equations of motion.  A3 = c + x a^1 + y a^2 + z a^3, affine in the acceleration.
struct A3 {
    double c, x, y, z;
};
__device__ __forceinline__ A3 k3(double c) { return {c, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ A3 operator+(A3 a, A3 b) { return {a.c + b.c, a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ A3 operator-(A3 a, A3 b) { return {a.c - b.c, a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ A3 operator*(double s, A3 a) { return {s * a.c, s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ A3 operator+(A3 a, double s) { return {a.c + s, a.x, a.y, a.z}; }
__device__ __forceinline__ double at3(A3 a, const double *acc) { return fma(a.x, acc[0], fma(a.y, acc[1], fma(a.z, acc[2], a.c))); }

__global__ void __launch_bounds__(64) k_eom3(EvView v, int stage, int mode, const double *__restrict__ ys,
                                             const double *__restrict__ dens, const double *__restrict__ eos,
                                             const double *__restrict__ gout, double *__restrict__ yout,
                                             double *__restrict__ rates, uint32_t *__restrict__ status)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const Geo3 G = geo3(v, stage);
    double u[4] = {dens[5 * n + a], ys[3 * n + a], ys[4 * n + a], ys[5 * n + a]};
    const double sig_star = dens[a], s = dens[n + a];
    const double nq[3] = {dens[2 * n + a], dens[3 * n + a], dens[4 * n + a]};
    const double T = eos[a], p = eos[4 * n + a], e = eos[5 * n + a], ps = eos[6 * n + a];
    const double mu[3] = {eos[n + a], eos[2 * n + a], eos[3 * n + a]};
    const double pn[3] = {eos[7 * n + a], eos[8 * n + a], eos[9 * n + a]};
    const double sigma = sig_star / (u[0] * G.sqrtg);
    const double ig = 1.0 / u[0], isg = 1.0 / sigma;
    const double vv[4] = {1.0, u[1] * ig, u[2] * ig, u[3] * ig};
    const bool visc = v.tr.viscous != 0;
    const double dt = v.dtau;
    const int nv = v.nv;
    if ((status[a] & (PST_NOCONV | PST_NONFINITE)) || (v.tr.T_stop_GeV > 0.0 && eos[a] * kHbarc < v.tr.T_stop_GeV)) {
        // no EoS solution, or below the stop temperature: ballistic motion only
        for (int k = 0; k < nv; ++k) {
            double fk = k < 3 ? vv[1 + k] : 0.0;
            if (mode == 0) yout[k * n + a] = ys[k * n + a] + dt * fk;
            else if (mode == 1) yout[k * n + a] = 0.5 * ((yout[k * n + a] + ys[k * n + a]) + dt * fk);
            else rates[k * n + a] = fk;
        }
        const double dN0[3] = {0.0, 0.0, 0.0};  // frozen: the charges stay as they are
        heun_charges(v, mode, n, a, dN0);
        return;
    }
    double Bv = 0.0, stv[5] = {0, 0, 0, 0, 0};
    if (visc) {
        Bv = ys[7 * n + a];
        for (int k = 0; k < 5; ++k) stv[k] = ys[(8 + k) * n + a];
    }
    const double Pi = sigma * Bv;
    double st[5];
    for (int k = 0; k < 5; ++k) st[k] = sigma * stv[k];
    double pi[4][4];
    pi_full3(G, u, st, pi);
    // d_k u^j (spatial k, j) and d_k u^0
    double dku[4][4];
    for (int k = 1; k < 4; ++k) {
        double s0 = 0.0;
        for (int j = 1; j < 4; ++j) {
            dku[k][j] = gout[(size_t)(3 * (k - 1) + (j - 1)) * n + a];
            s0 += G.g[j] * u[j] * dku[k][j];
        }
        dku[k][0] = -s0 * ig;
    }
    const A3 acc[4] = {k3(0.0), {0.0, 1.0, 0.0, 0.0}, {0.0, 0.0, 1.0, 0.0}, {0.0, 0.0, 0.0, 1.0}};
    // du^0/dx^0 from u.u = 1
    A3 du0 = (-ig) * (G.g[1] * u[1] * acc[1] + G.g[2] * u[2] * acc[2] + G.g[3] * u[3] * acc[3] + 0.5 * G.dg3 * u[3] * u[3]);
    A3 dudt[4] = {du0, acc[1], acc[2], acc[3]};
    // nabla_0 u^nu (affine) and nabla_k u^nu (constant)
    A3 nab0[4];
    double nabk[4][4];
    for (int nu = 0; nu < 4; ++nu) {
        double conv = 0.0, chr = 0.0;
        for (int k = 1; k < 4; ++k) conv += vv[k] * dku[k][nu];
        for (int l = 0; l < 4; ++l) chr += gam(G, nu, 0, l) * u[l];
        nab0[nu] = dudt[nu] + (chr - conv);
        for (int k = 1; k < 4; ++k) {
            double c2 = 0.0;
            for (int l = 0; l < 4; ++l) c2 += gam(G, nu, k, l) * u[l];
            nabk[k][nu] = dku[k][nu] + c2;
        }
    }
    A3 th = nab0[0] + (nabk[1][1] + nabk[2][2] + nabk[3][3]);
    A3 Du[4];
    for (int nu = 0; nu < 4; ++nu) Du[nu] = u[0] * nab0[nu] + (u[1] * nabk[1][nu] + u[2] * nabk[2][nu] + u[3] * nabk[3][nu]);
    const A3 dsg = (-sigma * ig) * th;
    A3 dS = k3(0.0), dBv = k3(0.0), dPv[4][4];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) dPv[i][j] = k3(0.0);
    if (visc) {
        // spatial shear tensor; the 0-components from transversality
        A3 sg[4][4];
        for (int i = 1; i < 4; ++i)
            for (int j = i; j < 4; ++j) {
                double sym = 0.5 * (G.gi[i] * nabk[i][j] + G.gi[j] * nabk[j][i]);
                double Delta = (i == j ? G.gi[i] : 0.0) - u[i] * u[j];
                A3 x = k3(sym) - 0.5 * (u[i] * Du[j] + u[j] * Du[i]) - (Delta / 3.0) * th;
                sg[i][j] = x;
                sg[j][i] = x;
            }
        for (int j = 1; j < 4; ++j) {
            A3 acc0 = k3(0.0);
            for (int k = 1; k < 4; ++k) acc0 = acc0 + (G.g[k] * u[k]) * sg[k][j];
            sg[0][j] = (-ig) * acc0;
            sg[j][0] = sg[0][j];
        }
        {
            A3 acc0 = k3(0.0);
            for (int k = 1; k < 4; ++k) acc0 = acc0 + (G.g[k] * u[k]) * sg[k][0];
            sg[0][0] = (-ig) * acc0;
        }
        A3 pisig = k3(0.0);
        for (int m = 0; m < 4; ++m)
            for (int l = 0; l < 4; ++l) pisig = pisig + (pi[m][l] * G.g[m] * G.g[l]) * sg[m][l];
        const double eta = v.tr.eta_over_s * s;
        const double dTg = T * kHbarc - v.tr.zeta_T_GeV;
        const double zeta = v.tr.zeta_peak * exp(-dTg * dTg / (2.0 * v.tr.zeta_w_GeV * v.tr.zeta_w_GeV)) * s;
        const double taupi = v.tr.tau_pi_coef * eta / (e + p);
        const double tauPi = v.tr.tau_Pi_ratio * taupi;
        dS = (ig * isg / T) * (pisig - Pi * th);
        const bool dnmr = v.tr.model == 1;
        if (dnmr) {  // DNMR bulk (see the 2+1D equations of motion)
            const double cs2 = eos[10 * n + a];
            dBv = (ig * isg) * ((-1.0 / tauPi) * (zeta * th + Pi) + ((1.0 - v.tr.dnmr[0]) * Pi) * th +
                                (v.tr.dnmr[1] * (1.0 / 3.0 - cs2)) * pisig);
        } else {
            dBv = (-ig * isg / tauPi) * (zeta * th + Pi);
        }
        double trB = 0.0;  // pi:pi
        if (dnmr)
            for (int m = 0; m < 4; ++m)
                for (int l = 0; l < 4; ++l) trB += pi[m][l] * G.g[m] * G.g[l] * pi[m][l];
        A3 alow[4];
        for (int al = 0; al < 4; ++al) alow[al] = G.g[al] * Du[al];
        const double itp = 1.0 / taupi;
        for (int i = 1; i < 4; ++i)
            for (int j = i; j < 4; ++j) {
                double chr = 0.0;
                for (int m = 0; m < 4; ++m)
                    for (int l = 0; l < 4; ++l) chr += u[m] * (gam(G, i, m, l) * pi[l][j] + gam(G, j, m, l) * pi[i][l]);
                A3 pja = k3(0.0), pia = k3(0.0);
                for (int al = 0; al < 4; ++al) {
                    pja = pja + pi[j][al] * alow[al];
                    pia = pia + pi[i][al] * alow[al];
                }
                A3 rhs;
                if (dnmr) {
                    // - delta_pipi pi theta - tau_pipi <pi sigma> + phi_7 <pi pi> + lambda_piPi Pi sigma with
                    // <A>^{ij} = (A^{ij} + A^{ji})/2 - Delta^{ij} tr A / 3 (pi, sigma transverse)
                    A3 Aij = k3(0.0), Aji = k3(0.0);
                    double Bij = 0.0;
                    for (int l = 0; l < 4; ++l) {
                        Aij = Aij + (pi[i][l] * G.g[l]) * sg[j][l];
                        Aji = Aji + (pi[j][l] * G.g[l]) * sg[i][l];
                        Bij += pi[i][l] * G.g[l] * pi[j][l];
                    }
                    const double Dij = (i == j ? G.gi[i] : 0.0) - u[i] * u[j];
                    const A3 PA = 0.5 * (Aij + Aji) - (Dij / 3.0) * pisig;
                    const double PB = Bij - Dij * trB / 3.0;
                    rhs = itp * (2.0 * eta * sg[i][j] + (-pi[i][j]) + k3(v.tr.dnmr[5] / p * PB)) -
                          (v.tr.dnmr[2] * pi[i][j]) * th - v.tr.dnmr[3] * PA + (v.tr.dnmr[4] * Pi) * sg[i][j];
                } else {
                    rhs = itp * (2.0 * eta * sg[i][j] - (4.0 / 3.0 * taupi * pi[i][j]) * th + (-pi[i][j]));
                }
                A3 dpi = ig * (rhs + (-chr) - (u[i] * pja + u[j] * pia));
                A3 x = isg * dpi - (pi[i][j] * isg * isg) * dsg;
                dPv[i][j] = x;
                dPv[j][i] = x;
            }
    }
    double Isrc[4] = {0.0, 0.0, 0.0, 0.0};
    double dN[3] = {0.0, 0.0, 0.0};  // charge rates dN_q/dx0 (charge sources only)
    if (v.ntrack > 0 || v.nparton > 0) {
        // jet tracks (Cartesian) and partons: dP^i/dx0 gains sqrt(-g) I^i/sigma*, dS/dx0 gains
        // u_nu I^nu/(u^0 sigma T); parton charges: dN_q/dx0 = sqrt(-g) I_q/sigma*, and dS/dx0
        // gains -mu_q/T dN_q/dx0 (eq. dsdnrewr, R^S_q = -mu_q/T)
        double Ik[4], Iq[3] = {0.0, 0.0, 0.0};
        if (v.ntrack > 0) {
            jet_deposit(v, G.tau, ys[a], ys[n + a], ys[2 * n + a], Ik);
            for (int k = 0; k < 4; ++k) Isrc[k] += Ik[k];
        }
        if (v.nparton > 0) {
            const double xa[3] = {ys[a], ys[n + a], ys[2 * n + a]};
            parton_deposit(v, G.tau, G.sqrtg, xa, Ik, Iq);
            for (int k = 0; k < 4; ++k) Isrc[k] += Ik[k];
        }
        double uI = 0.0;
        for (int k = 0; k < 4; ++k) uI += G.g[k] * u[k] * Isrc[k];
        uI -= mu[0] * Iq[0] + mu[1] * Iq[1] + mu[2] * Iq[2];
        dS = dS + k3((ig * isg / T) * uI);
        for (int c = 0; c < 3; ++c) dN[c] = G.sqrtg * Iq[c] / sig_star;
    }
    const A3 ds = sigma * dS + (s * isg) * dsg;
    const A3 dPi = sigma * dBv + Bv * dsg;
    // dn_q = N_q dsigma + sigma dN_q
    const A3 dw = (T + ps) * ds + (((mu[0] + pn[0]) * nq[0] + (mu[1] + pn[1]) * nq[1] + (mu[2] + pn[2]) * nq[2]) * isg) * dsg + dPi +
                  k3(sigma * ((mu[0] + pn[0]) * dN[0] + (mu[1] + pn[1]) * dN[1] + (mu[2] + pn[2]) * dN[2]));
    const double w = e + p + Pi;
    const double ig2 = ig * ig, ig3 = ig2 * ig;
    // T^{mu nu} for the Christoffel source of the momentum rate (i = eta in Milne)
    A3 M[3];
    double F[3], cvec[3];
    for (int i = 1; i < 4; ++i) {
        A3 t1 = k3(0.0);
        double t2 = 0.0;
        for (int j = 1; j < 4; ++j) {
            double Pvji = isg * pi[j][i];
            double dgj = (j == 3) ? G.dg3 : 0.0;
            t1 = t1 + k3(dgj * u[j] * Pvji) + (G.g[j] * Pvji) * acc[j] + (G.g[j] * u[j]) * dPv[j][i];
            t2 += G.g[j] * u[j] * Pvji;
        }
        A3 dpi0 = (-ig2) * t1 + (2.0 * t2 * ig3) * du0;
        A3 dP = (u[i] * isg) * dw + (w * isg) * acc[i] - (w * u[i] * isg * isg) * dsg + dpi0;
        double src = 0.0;
        for (int m = 0; m < 4; ++m)
            for (int l = 0; l < 4; ++l) {
                double gml = gam(G, i, m, l);
                if (gml != 0.0) {
                    double Delta = (m == l ? G.gi[m] : 0.0) - u[m] * u[l];
                    src += gml * (e * u[m] * u[l] - (p + Pi) * Delta + pi[m][l]);
                }
            }
        F[i - 1] = gout[(size_t)(9 + i - 1) * n + a] - G.sqrtg * src / sig_star + G.sqrtg * Isrc[i] / sig_star;
        M[i - 1] = dP;
        cvec[i - 1] = dP.c;
    }
    // solve M a = F - c (3x3, partial pivoting)
    double A[3][3] = {{M[0].x, M[0].y, M[0].z}, {M[1].x, M[1].y, M[1].z}, {M[2].x, M[2].y, M[2].z}};
    double b[3] = {F[0] - cvec[0], F[1] - cvec[1], F[2] - cvec[2]};
    uint32_t stt = 0;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int piv = c;
        double best = fabs(A[c][c]);
#pragma unroll
        for (int r = c + 1; r < 3; ++r)
            if (fabs(A[r][c]) > best) {
                best = fabs(A[r][c]);
                piv = r;
            }
        if (!(best > 0.0) || !isfinite(best)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int r = c + 1; r < 3; ++r)
            if (piv == r) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    double t = A[c][k];
                    A[c][k] = A[r][k];
                    A[r][k] = t;
                }
                double t = b[c];
                b[c] = b[r];
                b[r] = t;
            }
#pragma unroll
        for (int r = c + 1; r < 3; ++r) {
            double f = A[r][c] / A[c][c];
#pragma unroll
            for (int k = c; k < 3; ++k) A[r][k] = fma(-f, A[c][k], A[r][k]);
            b[r] = fma(-f, b[c], b[r]);
        }
    }
    double av[3] = {0.0, 0.0, 0.0};
    if (ok) {
#pragma unroll
        for (int r = 2; r >= 0; --r) {
            double t = b[r];
#pragma unroll
            for (int k = r + 1; k < 3; ++k) t = fma(-A[r][k], av[k], t);
            av[r] = t / A[r][r];
        }
    } else {
        stt |= PST_SOLVE_FAIL;
    }
    double f[13];
    for (int k = 0; k < 3; ++k) f[k] = vv[1 + k];
    for (int k = 0; k < 3; ++k) f[3 + k] = av[k];
    f[6] = at3(dS, av);
    f[7] = at3(dBv, av);
    f[8] = at3(dPv[1][1], av);
    f[9] = at3(dPv[1][2], av);
    f[10] = at3(dPv[1][3], av);
    f[11] = at3(dPv[2][2], av);
    f[12] = at3(dPv[2][3], av);
    bool fin = true;
    for (int k = 0; k < 13; ++k) fin = fin && isfinite(f[k]);
    if (!fin) stt |= PST_NONFINITE;
    if (stt) {
        status[a] |= stt;
        atomicOr(&v.sc->status_or, stt);
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

// a8: totals contributions in original order: [0] sqrt(-g) T^{00}/sigma*, [1] S
__global__ void k_totals3(EvView v, const double *__restrict__ y, const int *__restrict__ id,
                          const double *__restrict__ dens, const double *__restrict__ eos, double *__restrict__ contrib)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const Geo3 G = geo3(v, 1);
    double u[4] = {dens[5 * n + a], y[3 * n + a], y[4 * n + a], y[5 * n + a]};
    const double sig_star = dens[a];
    const double sigma = sig_star / (u[0] * G.sqrtg);
    double Pi = 0.0, st[5] = {0, 0, 0, 0, 0};
    if (v.tr.viscous) {
        Pi = sigma * y[7 * n + a];
        for (int k = 0; k < 5; ++k) st[k] = sigma * y[(8 + k) * n + a];
    }
    double pi[4][4];
    pi_full3(G, u, st, pi);
    const double p = eos[4 * n + a], e = eos[5 * n + a];
    const double T00 = (e + p + Pi) * u[0] * u[0] - (p + Pi) + pi[0][0];
    const int o = id[a];
    contrib[o] = G.sqrtg * T00 / sig_star;
    contrib[n + o] = y[6 * n + a];
}

// test support: neighbour pairs (pass 1 counts with offs == nullptr, pass 2 writes)
__global__ void k_neighbors3(EvView v, const double *__restrict__ y, const int *__restrict__ id,
                             const uint32_t *__restrict__ start, const uint32_t *__restrict__ cnt,
                             const long long *__restrict__ offs, int *count_out, int *pa, int *pb)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const double xa[3] = {y[a], y[n + a], y[2 * n + a]};
    int c[3], lim[3];
    for (int d = 0; d < 3; ++d) {
        c[d] = cell_coord(xa[d], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
        lim[d] = 1 << v.B3[d];
    }
    long long w = offs ? offs[a] : 0;
    int m = 0;
    for (int oz = -1; oz <= 1; ++oz)
        for (int oy = -1; oy <= 1; ++oy)
            for (int ox = -1; ox <= 1; ++ox) {
                const int nx = c[0] + ox, ny = c[1] + oy, nz = c[2] + oz;
                if (nx < 0 || ny < 0 || nz < 0 || nx >= lim[0] || ny >= lim[1] || nz >= lim[2]) continue;
                const uint32_t k = key3(v, nx, ny, nz);
                for (uint32_t b = start[k]; b < start[k] + cnt[k]; ++b) {
                    double r2 = dist2_3d(xa[0] - y[b], xa[1] - y[n + b], xa[2] - y[2 * n + b]);
                    if (r2 < v.supp2) {
                        if (offs) {
                            pa[w + m] = id[a];
                            pb[w + m] = id[b];
                        }
                        ++m;
                    }
                }
            }
    if (!offs) count_out[a] = m;
}

__global__ void k_cell_coords3(EvView v, const double *__restrict__ y, const int *__restrict__ id, int *cell_orig)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= v.n) return;
    const int o = id[j];
    for (int d = 0; d < 3; ++d)
        cell_orig[(size_t)d * v.n + o] = cell_coord(y[(size_t)d * v.n + j], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_cells3(const EvView &v, const double *y, const int *id, CellBufs cb, cudaStream_t st)
{
    (void)id;
    k_cells3<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.key, cb.cnt);
}

void launch_density3(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                     cudaStream_t st)
{
    if (v.mixed) {
        launch_density3m(v, y, Nq, cb, dens, nnb, st);
        return;
    }
    k_fpos3<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.fpos3);
    const int lists = cb.pl.total > 0;
    if (lists) launch_pairs3_density(v, y, Nq, cb, dens, nnb, st);
    // as the fallback of the pair-list passes it usually exits at once: a few blocks per SM
    const int grid = lists ? std::min(nblk(v.n, kWarps3), 8 * device_sm_count()) : nblk(v.n, kWarps3);
    k_density3<<<grid, 32 * kWarps3, 0, st>>>(v, y, cb.fpos3, Nq, cb.start, cb.cnt, dens, nnb, lists,
                                              lists ? cb.pl.cnt_dst : nullptr);
}

void launch_eos3(const EvView &v, int stage, const double *y, const double *dens, double *eos, double *gin,
                 uint32_t *status, double *wpart, const double *guess_in, double *guess_out, cudaStream_t st)
{
    k_eos3<<<nblk(v.n, 64), 64, 0, st>>>(v, stage, y, const_cast<double *>(dens), eos, gin, status, wpart, guess_in,
                                         guess_out);
}

void launch_gradient3(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                      cudaStream_t st)
{
    if (v.mixed) {
        launch_gradient3m(v, stage, y, gin, cb, gout, st);
        return;
    }
    const int lists = cb.pl.total > 0;
    if (lists) launch_pairs3_gradient(v, stage, y, gin, cb, gout, st);
    const int grid = lists ? std::min(nblk(v.n, kWarps3), 8 * device_sm_count()) : nblk(v.n, kWarps3);
    k_gradient3<<<grid, 32 * kWarps3, 0, st>>>(v, stage, y, cb.fpos3, gin, cb.start, cb.cnt, gout, lists);
}

void launch_eom3(const EvView &v, int stage, int mode, const double *ys, const double *dens, const double *eos,
                 const double *gout, double *yout, double *rates, uint32_t *status, cudaStream_t st)
{
    k_eom3<<<nblk(v.n, 64), 64, 0, st>>>(v, stage, mode, ys, dens, eos, gout, yout, rates, status);
}

void launch_totals3(const EvView &v, const double *y, const int *id, const double *dens, const double *eos,
                    double *contrib, cudaStream_t st)
{
    k_totals3<<<nblk(v.n, 256), 256, 0, st>>>(v, y, id, dens, eos, contrib);
}

void launch_neighbors_list3(const EvView &v, const double *y, const int *id, CellBufs cb, const long long *offs,
                            int *pa, int *pb, cudaStream_t st)
{
    k_neighbors3<<<nblk(v.n, 128), 128, 0, st>>>(v, y, id, cb.start, cb.cnt, offs, offs ? nullptr : pa, pa, pb);
}

void launch_cell_coords3(const EvView &v, const double *y, const int *id, int *cell_orig, cudaStream_t st)
{
    k_cell_coords3<<<nblk(v.n, 256), 256, 0, st>>>(v, y, id, cell_orig);
}

}  // namespace sphg
