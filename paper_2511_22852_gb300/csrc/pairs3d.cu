// pairs3d.cu -- plain 3D neighbour passes over half-pair lists: the 3D counterpart of the plain
// 2D passes (the same rows, ordering and fallback), over the 27 cells of the generalized Morton
// table.  Per accepted pair the forward density pass evaluates W and grad W once (both depend on
// r_ab only; grad_b W_ba = -grad_a W_ab) and keeps them with the pair; the backward pass and the
// gradient pass add every pair to both of its particles.  Sums in a fixed order: reproducible.
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kWarps = 4;
constexpr unsigned kFull = 0xFFFFFFFFu;

// the cells of the 3x3x3 block inside the grid, in ascending key (their particles then come in
// ascending sorted index)
__device__ __forceinline__ int block27_ascending(const EvView &v, const int c[3], uint32_t keys[27])
{
    int nk = 0;
    for (int oz = -1; oz <= 1; ++oz) {
        const int nz = c[2] + oz;
        if (nz < 0 || nz >= (1 << v.B3[2])) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            const int ny = c[1] + oy;
            if (ny < 0 || ny >= (1 << v.B3[1])) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int nx = c[0] + ox;
                if (nx < 0 || nx >= (1 << v.B3[0])) continue;
                const uint32_t k = key3(v, nx, ny, nz);
                int j = nk++;
                while (j > 0 && keys[j - 1] > k) {
                    keys[j] = keys[j - 1];
                    --j;
                }
                keys[j] = k;
            }
        }
    }
    return nk;
}

// Forward density pass, one warp per particle a: candidates of the 27 cells through the
// single-precision prefilter; neighbours b < a decided at once and listed from the row end;
// candidates b > a queued and, 32 at a time, put through the exact test, W and grad W on full
// warps, listed from the row start with W and grad W, and summed for a.  a's unscaled partial
// sums (self pair and pairs b > a) are left in the density rows.
__global__ void __launch_bounds__(32 * kWarps) k_pairs3_density_fwd(EvView v, const double *__restrict__ y,
                                                                    const float4 *__restrict__ fpos,
                                                                    const double *__restrict__ Nq,
                                                                    const uint32_t *__restrict__ start,
                                                                    const uint32_t *__restrict__ cnt, PairBufs pl,
                                                                    double *__restrict__ dpart)
{
    __shared__ int queue[kWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarps + wid;
    if (a >= v.n) return;  // warp-uniform
    int *q = queue[wid];
    const size_t n = (size_t)v.n;
    const double *X = y, *Y = y + n, *Z = y + 2 * n, *S = y + 6 * n;
    const double *NB = Nq, *NS = Nq + n, *NQ = Nq + 2 * n;
    const double xa[3] = {X[a], Y[a], Z[a]};
    const float4 fa = fpos[a];
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) c[d] = cell_coord(xa[d], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
    uint32_t keys[27];
    const int nk = block27_ascending(v, c, keys);
    const unsigned lt = (1u << lane) - 1u;
    const long long r0 = pl.off[a], r1 = pl.off[a + 1];
    const int cap = r1 <= pl.total ? (int)(r1 - r0) : 0;  // rows beyond the allocation: no writes
    int *F = pl.L + r0, *Bl = pl.L + (r1 - 1);
    double *Wr = pl.W + r0, *Gr = pl.G3 + 3 * r0;
    double sg = 0.0, ss = 0.0, sb = 0.0, sS = 0.0, sq = 0.0;
    if (lane == 0) {  // the self pair, W(0)
        const double w0 = kernel_w(0.0);
        sg = w0;
        ss = S[a] * w0;
        sb = NB[a] * w0;
        sS = NS[a] * w0;
        sq = NQ[a] * w0;
    }
    int nf = 0, nbk = 0, qn = 0;
    auto forward = [&](int qb, bool valid) {
        const int b = qb & 0x7FFFFFFF;
        double d[3] = {0.0, 0.0, 0.0};
        bool acc = false;
        if (valid) {
            d[0] = xa[0] - X[b];
            d[1] = xa[1] - Y[b];
            d[2] = xa[2] - Z[b];
            acc = qb >= 0 || dist2_3d(d[0], d[1], d[2]) < v.supp2;
        }
        const unsigned m = __ballot_sync(kFull, acc);
        if (acc) {
            const double r2 = fma(d[0], d[0], fma(d[1], d[1], d[2] * d[2]));
            double w = kernel_w(0.0), fac = 0.0;  // coincident particles: W(0), no gradient
            if (nonzero_nonneg(r2)) {
                // the cubic spline without a branch on q (see the 2D forward pass)
                const double ir = inv_sqrt(r2);
                const double qq = r2 * ir * v.inv_h;
                const double t = 2.0 - qq, u = pos_part(1.0 - qq);
                const double t2 = t * t, u2 = u * u;
                w = fma(quarter_nonneg(t2), t, -(u2 * u));
                fac = fma(-0.75, t2, 3.0 * u2) * ir;
            }
            const int slot = nf + __popc(m & lt);
            if (slot < cap) {
                F[slot] = b;
                Wr[slot] = w;
                Gr[3 * slot] = fac * d[0];
                Gr[3 * slot + 1] = fac * d[1];
                Gr[3 * slot + 2] = fac * d[2];
            }
            sg += w;
            ss = fma(S[b], w, ss);
            sb = fma(NB[b], w, sb);
            sS = fma(NS[b], w, sS);
            sq = fma(NQ[b], w, sq);
        }
        nf += __popc(m);
    };
    for (int kc = 0; kc < nk; ++kc) {
        const uint32_t k = keys[kc];
        const uint32_t b0 = start[k], b1 = b0 + cnt[k];
        for (uint32_t base = b0; base < b1; base += 32) {
            const uint32_t b = base + lane;
            bool cand = false, sure = false;
            if (b < b1 && b != (uint32_t)a) {
                const float4 fb = fpos[b];
                const float dx = fa.x - fb.x, dy = fa.y - fb.y, dz = fa.z - fb.z;
                const float r2f = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                cand = r2f <= v.supp2_hi;
                sure = r2f < v.supp2_lo;
            }
            bool accB = false;  // b < a: its pair values come from b's own forward pass
            if (cand && (int)b < a) accB = sure || dist2_3d(xa[0] - X[b], xa[1] - Y[b], xa[2] - Z[b]) < v.supp2;
            const unsigned mb = __ballot_sync(kFull, accB);
            if (accB) {
                const int slot = nbk + __popc(mb & lt);
                if (slot < cap) Bl[-slot] = (int)b;
            }
            nbk += __popc(mb);
            const bool fw = cand && (int)b > a;
            const unsigned m = __ballot_sync(kFull, fw);
            if (fw) q[qn + __popc(m & lt)] = sure ? (int)b : (int)(b | 0x80000000u);
            qn += __popc(m);
            __syncwarp();
            if (qn >= 32) {
                forward(q[lane], true);
                qn -= 32;
                __syncwarp();
                if (lane < qn) q[lane] = q[32 + lane];
                __syncwarp();
            }
        }
    }
    if (qn > 0) forward(lane < qn ? q[lane] : 0, lane < qn);
    const double vals[8] = {sg, ss, sb, sS, sq, 0.0, 0.0, 0.0};
    const double tot = warp_reduce_scatter8(vals, lane);
    const int kk = lane >> 2;
    if ((lane & 3) == 0 && kk < 5) dpart[(size_t)kk * n + a] = tot;
    if (lane == 0) {
        pl.cntF[a] = nf;
        pl.cntB[a] = nbk;
        if (nf + nbk > cap) atomicOr(&v.sc->pair_flag, 1u);
    }
}

// Backward density pass (as in 2D): W of the pairs (b, a), b < a, from b's row after a binary
// search; the slot kept in P; completes the density rows (the 3D EoS pass forms u0 itself).
__global__ void __launch_bounds__(32 * kWarps) k_pairs3_density_bwd(EvView v, const double *__restrict__ y,
                                                                    const double *__restrict__ Nq, PairBufs pl,
                                                                    double *__restrict__ dens, int *__restrict__ nnb)
{
    if (v.sc->pair_flag) return;  // a list overflowed: the per-particle pass runs instead
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarps + wid;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const double *S = y + 6 * n;
    const double *NB = Nq, *NS = Nq + n, *NQ = Nq + 2 * n;
    const long long rend = pl.off[a + 1] - 1;
    const int nb = pl.cntB[a];
    double sg = 0.0, ss = 0.0, sb = 0.0, sS = 0.0, sq = 0.0;
    for (int j0 = 0; j0 < nb; j0 += 32) {
        const int j = j0 + lane;
        if (j < nb) {
            const int b = pl.L[rend - j];
            const long long rb = pl.off[b];
            const int *Fb = pl.L + rb;
            const int nfb = pl.cntF[b];
            int lo = 0, hi = nfb;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (Fb[mid] < a) lo = mid + 1;
                else hi = mid;
            }
            if (lo >= nfb || Fb[lo] != a) {  // both sides decide alike; checked all the same
                atomicOr(&v.sc->err_flags, ERR_PAIR_LIST);
                lo = 0;
            }
            pl.P[rend - j] = lo;
            const double w = nfb > 0 ? pl.W[rb + lo] : 0.0;
            sg += w;
            ss = fma(S[b], w, ss);
            sb = fma(NB[b], w, sb);
            sS = fma(NS[b], w, sS);
            sq = fma(NQ[b], w, sq);
        }
    }
    const double vals[8] = {sg, ss, sb, sS, sq, 0.0, 0.0, 0.0};
    const double tot = warp_reduce_scatter8(vals, lane);
    const int k = lane >> 2;
    if ((lane & 3) == 0 && k < 5) {
        double *d = dens + (size_t)k * n + a;
        *d = v.sigma_d * (*d + tot);
    }
    if (lane == 0) {
        const int c = 1 + pl.cntF[a] + nb;
        nnb[a] = c;
        if (pl.cnt_dst) pl.cnt_dst[a] = c;
        atomicAdd(&v.sc->pairs, (unsigned long long)c);
    }
}

// Gradient pass, one warp per particle a, over its pairs b > a (stored grad_a W_ab) and b < a
// (minus the stored grad_b W_ba): sum grad W (3), sum X_b^{j i} grad_j W (3), sum u_b^j grad_k W (9),
// 15 sums reduced by two reduce-scatters; the epilogue as the per-particle pass.
__global__ void __launch_bounds__(32 * kWarps) k_pairs3_gradient(EvView v, int stage, const double *__restrict__ y,
                                                                 const double *__restrict__ gin, PairBufs pl,
                                                                 double *__restrict__ gout)
{
    if (v.sc->pair_flag) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarps + wid;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const long long r0 = pl.off[a], rend = pl.off[a + 1] - 1;
    const int nf = pl.cntF[a], nt = nf + pl.cntB[a];
    double G[3] = {0, 0, 0}, H[3] = {0, 0, 0}, du[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int j0 = 0; j0 < nt; j0 += 32) {
        const int jj = j0 + lane;
        if (jj < nt) {
            int b;
            double gw[3];
            if (jj < nf) {
                b = pl.L[r0 + jj];
                const double *g = pl.G3 + 3 * (r0 + jj);
                gw[0] = g[0];
                gw[1] = g[1];
                gw[2] = g[2];
            } else {
                b = pl.L[rend - (jj - nf)];
                const double *g = pl.G3 + 3 * (pl.off[b] + pl.P[rend - (jj - nf)]);
                gw[0] = -g[0];
                gw[1] = -g[1];
                gw[2] = -g[2];
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) G[k] += gw[k];
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
    }
    const double v1[8] = {G[0], G[1], G[2], H[0], H[1], H[2], du[0][0], du[0][1]};
    const double v2[8] = {du[0][2], du[1][0], du[1][1], du[1][2], du[2][0], du[2][1], du[2][2], 0.0};
    const double t1 = warp_reduce_scatter8(v1, lane), t2 = warp_reduce_scatter8(v2, lane);
    const double G0 = __shfl_sync(kFull, t1, 0), G1 = __shfl_sync(kFull, t1, 4), G2 = __shfl_sync(kFull, t1, 8);
    const int k = lane >> 2;
    if ((lane & 3) == 0) {
        const double c = v.sigma_d * v.inv_h;
        // du[k][j] -> row 3 k + j: t1 holds du00, du01 (lanes 24, 28); t2 du02 .. du22 (lanes 0..24)
        if (k >= 6) gout[(size_t)(k - 6) * n + a] = c * t1;
        if (k < 7) gout[(size_t)(2 + k) * n + a] = c * t2;
        if (k >= 3 && k < 6) {
            // minus the stress divergence: H_i + sum_j X_a^{j i} G_j, times sqrt(-g)
            const int i = k - 3;
            const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
            const double sqrtg = v.milne ? tau : 1.0;
            double F = t1;
            F = fma(gin[(size_t)(0 + i) * n + a], G0, F);
            F = fma(gin[(size_t)(3 + i) * n + a], G1, F);
            F = fma(gin[(size_t)(6 + i) * n + a], G2, F);
            gout[(size_t)(9 + i) * n + a] = -sqrtg * c * F;
        }
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_pairs3_density(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                           cudaStream_t st)
{
    launch_pair_rows(v, cb, st);
    k_pairs3_density_fwd<<<nblk(v.n, kWarps), 32 * kWarps, 0, st>>>(v, y, cb.fpos3, Nq, cb.start, cb.cnt, cb.pl,
                                                                    dens);
    k_pairs3_density_bwd<<<nblk(v.n, kWarps), 32 * kWarps, 0, st>>>(v, y, Nq, cb.pl, dens, nnb);
}

void launch_pairs3_gradient(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb,
                            double *gout, cudaStream_t st)
{
    k_pairs3_gradient<<<nblk(v.n, kWarps), 32 * kWarps, 0, st>>>(v, stage, y, gin, cb.pl, gout);
}

}  // namespace sphg
