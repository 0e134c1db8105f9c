// mixed2d.cu -- the neighbour passes (rows a3, a5) in the mixed-precision form, 2+1D.
//
// The pair arithmetic runs on the FP32 pipe (64x the FP64 rate on GB300):
//   * positions are stored relative to the origin of their cell, so a pair separation
//     dx = (r_a - r_b) - o * (2h) (o the cell offset, -1..1) is formed from numbers of
//     size <= 2h and its single-precision error is ~1e-7 fm regardless of where the
//     event sits;
//   * the neighbour decision stays exact: a proven bound err on the float r^2 classifies
//     candidates as certainly inside (r2f < (2h)^2 - err), certainly outside
//     (r2f > (2h)^2 + err), or in the thin shell between, where the FP64 test r^2 < (2h)^2
//     with separately rounded products decides -- the same set as the FP64 path;
//   * candidates are staged per cell in shared memory and evaluated two per packed two-wide
//     FP32 instruction; sums are compensated (Neumaier two-sum) per lane in float, and a
//     particle's lanes are combined with error-free FP32 additions in a fixed tree order.
// The EoS inversion, equations of motion and conservation reductions stay FP64.
#include <algorithm>

#include "sph_internal.cuh"
#include "tiled_common.cuh"

namespace sphg {

namespace {

// cell-relative single-precision positions of the sorted particles
__global__ void k_relpos2(EvView v, const double *__restrict__ y, float2 *__restrict__ rel)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= v.n) return;
    const double cs = 2.0 * v.h;
    double r[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        double xm = dec_double(v.sc->xmin_enc[d]);
        double x = y[(size_t)d * v.n + j];
        int c = cell_coord(x, xm, v.inv_cell);
        r[d] = __dsub_rn(__dsub_rn(x, xm), (double)c * cs);
    }
    rel[j] = make_float2(__double2float_rn(r[0]), __double2float_rn(r[1]));
}

// Cell-tiled passes: one block per occupied cell (grid-stride over the cell grid) stages the
// candidates of the 3x3 block of 2h-cells around it -- nine runs of the Morton-sorted order --
// in shared memory, in tiles of kTile2, two candidates per float4 entry (packed two-wide FP32
// arithmetic), and every particle of the cell scans them with L lanes (lanes_per_particle).  A
// candidate carries its own-cell-relative position and its cell's offset separately, so the
// separation (r_a - r_b) - o (2h) rounds exactly as the shell bound assumes.
constexpr int kTT2 = 256;      // threads of a tiled block; all its warps share a cell's particles
constexpr int kTile2 = 896;    // candidates staged at a time (about the 3x3 block of a C2 cell)

struct Runs9 {
    int rs[9];     // first sorted index of each neighbour cell (row-major over (oy, ox))
    int cum[10];   // candidates before run o
    float ox[9], oy[9];  // the run's cell offset times the float cell side
};

// the runs of cell (cx, cy), built by the first nine threads; thread 0 scans the lengths
__device__ __forceinline__ void runs9_setup(const EvView &v, const uint32_t *__restrict__ start,
                                            const uint32_t *__restrict__ cnt, int cx, int cy, Runs9 &R)
{
    const int t = threadIdx.x, lim = 1 << v.B;
    if (t < 9) {
        const int dy = t / 3 - 1, dx = t % 3 - 1, nx = cx + dx, ny = cy + dy;
        int len = 0, st = 0;
        if (nx >= 0 && nx < lim && ny >= 0 && ny < lim) {
            const uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
            st = (int)start[k];
            len = (int)cnt[k];
        }
        R.rs[t] = st;
        R.cum[t + 1] = len;
        R.ox[t] = (float)dx * v.cell_f;
        R.oy[t] = (float)dy * v.cell_f;
    }
    __syncthreads();
    if (t == 0) {
        R.cum[0] = 0;
        for (int o = 0; o < 9; ++o) R.cum[o + 1] += R.cum[o];
    }
    __syncthreads();
}

// sorted index of candidate q and its run
__device__ __forceinline__ int run_of(const Runs9 &R, int q)
{
    int o = 0;
#pragma unroll
    for (int k = 1; k < 9; ++k) o += q >= R.cum[k];
    return o;
}

template <int TT>
__global__ void __launch_bounds__(TT) k_tiled_density2m(EvView v, const double *__restrict__ y,
                                                          const float2 *__restrict__ rel,
                                                          const double *__restrict__ Nq,
                                                          const uint32_t *__restrict__ start,
                                                          const uint32_t *__restrict__ cnt,
                                                          double *__restrict__ dens, int *__restrict__ nnb)
{
    __shared__ float4 cP[kTile2 / 2];   // (-x_0, -x_1, -y_0, -y_1): own-cell-relative positions
    __shared__ float4 cO[kTile2 / 2];   // (-ox_0, -ox_1, -oy_0, -oy_1): their cells' offsets
    __shared__ float4 cQa[kTile2 / 2];  // (S_0, S_1, N_B0, N_B1)
    __shared__ float4 cQb[kTile2 / 2];  // (N_S0, N_S1, N_Q0, N_Q1)
    __shared__ Runs9 R;
    __shared__ unsigned long long s_acc[2];
    const size_t n = (size_t)v.n;
    const int lim = 1 << v.B, ncell = lim * lim;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = TT / 32;
    const float ih = (float)v.inv_h, slo = v.shell_lo, shi = v.shell_hi;
    const double supp2 = v.supp2, sd = v.sigma_d;
    if (tid == 0) s_acc[0] = s_acc[1] = 0ull;
    for (int ci = blockIdx.x; ci < ncell; ci += gridDim.x) {  // block-uniform
        const int cx = ci % lim, cy = ci / lim;
        const uint32_t kc = morton2((uint32_t)cx, (uint32_t)cy);
        const int na = (int)cnt[kc];
        if (na == 0) continue;
        __syncthreads();  // the previous cell's runs and tiles are no longer read
        runs9_setup(v, start, cnt, cx, cy, R);
        const int M = R.cum[9], first = (int)start[kc];
        const int L = lanes_per_particle(na, NW), ppw = 32 / L;
        const int pl = lane / L, l = lane - pl * L;
        unsigned pairs = 0u, shell = 0u;
        for (int g0 = 0; g0 < na; g0 += NW * ppw) {
            const int my = g0 + warp * ppw + pl;
            const bool valid = pl < ppw && my < na;
            const int a = first + (valid ? my : 0);
            const double xa = y[a], ya = y[n + a];
            const float2 ra = rel[a];
            CSum sg = {0.f, 0.f}, ss = {0.f, 0.f}, sb = {0.f, 0.f}, sS = {0.f, 0.f}, sq = {0.f, 0.f};
            int nacc = 0;
            for (int t0 = 0; t0 < M; t0 += kTile2) {
                const int mt = min(kTile2, M - t0);
                if (g0 == 0 || M > kTile2) {  // one tile serves every pass of the cell
                    if (t0 > 0 || g0 > 0) __syncthreads();
                    for (int i = tid; i < mt; i += TT) {
                        const int q = t0 + i, o = run_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                        const float2 rb = rel[b];
                        put_pair(cP, i, -rb.x, -rb.y);
                        put_pair(cO, i, -R.ox[o], -R.oy[o]);
                        put_pair(cQa, i, (float)y[4 * n + b], (float)Nq[b]);
                        put_pair(cQb, i, (float)Nq[n + b], (float)Nq[2 * n + b]);
                    }
                    if ((mt & 1) && tid == 0) {
                        put_pair(cP, mt, kFar, kFar);
                        put_pair(cO, mt, 0.0f, 0.0f);
                        put_pair(cQa, mt, 0.0f, 0.0f);
                        put_pair(cQb, mt, 0.0f, 0.0f);
                    }
                    __syncthreads();
                }
                if (valid) {
                    const float2 fx = make_float2(ra.x, ra.x), fy = make_float2(ra.y, ra.y), ih2 = make_float2(ih, ih);
                    const int np = (mt + 1) >> 1;
                    for (int kb = l; kb < np; kb += (kRun / 2) * L) {
                        const int ke = min(np, kb + (kRun / 2) * L);
                        float2 pg = make_float2(0.f, 0.f), ps = pg, pB = pg, pS = pg, pQ = pg;
#pragma unroll 2
                        for (int k = kb; k < ke; k += L) {
                            const float4 pk = cP[k], po = cO[k];
                            // (r_a - r_b) - o (2h), rounded step by step as the shell bound assumes
                            const float2 dx = __fadd2_rn(__fadd2_rn(fx, lo2(pk)), lo2(po));
                            const float2 dy = __fadd2_rn(__fadd2_rn(fy, hi2(pk)), hi2(po));
                            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                            bool a0 = r2.x < slo, a1 = r2.y < slo;
                            if (r2.x >= slo && r2.x <= shi) {  // thin shell: the exact FP64 decision
                                const int q = t0 + 2 * k, o = run_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a0 = dist2_2d(xa - y[b], ya - y[n + b]) < supp2;
                                ++shell;
                            }
                            if (r2.y >= slo && r2.y <= shi) {
                                const int q = t0 + 2 * k + 1, o = run_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a1 = dist2_2d(xa - y[b], ya - y[n + b]) < supp2;
                                ++shell;
                            }
                            const float2 qq = __fmul2_rn(make_float2(sqrt_apx(r2.x), sqrt_apx(r2.y)), ih2);
                            float2 t2, t, u2, u;
                            spline_terms2(qq, t2, t, u2, u);
                            float2 w = __ffma2_rn(__fmul2_rn(make_float2(0.25f, 0.25f), t2), t,
                                                  __fmul2_rn(u2, make_float2(-u.x, -u.y)));
                            w.x = a0 ? w.x : 0.0f;
                            w.y = a1 ? w.y : 0.0f;
                            const float4 qa = cQa[k], qb = cQb[k];
                            pg = __fadd2_rn(pg, w);
                            ps = __ffma2_rn(lo2(qa), w, ps);
                            pB = __ffma2_rn(hi2(qa), w, pB);
                            pS = __ffma2_rn(lo2(qb), w, pS);
                            pQ = __ffma2_rn(hi2(qb), w, pQ);
                            nacc += (int)a0 + (int)a1;
                        }
                        cadd(sg, pg.x + pg.y);
                        cadd(ss, ps.x + ps.y);
                        cadd(sb, pB.x + pB.y);
                        cadd(sS, pS.x + pS.y);
                        cadd(sq, pQ.x + pQ.y);
                    }
                }
            }
            sg = seg_csum(sg, l, L);
            ss = seg_csum(ss, l, L);
            sb = seg_csum(sb, l, L);
            sS = seg_csum(sS, l, L);
            sq = seg_csum(sq, l, L);
            for (int o = 1; o < L; o <<= 1) {  // the neighbour count, in the same tree
                const int t = __shfl_down_sync(0xFFFFFFFFu, nacc, o);
                if ((l & (2 * o - 1)) == 0 && l + o < L) nacc += t;
            }
            if (valid && l == 0) {
                const double ux = y[2 * n + a], uy = y[3 * n + a];
                dens[a] = sd * cval(sg);
                dens[n + a] = sd * cval(ss);
                dens[2 * n + a] = sd * cval(sb);
                dens[3 * n + a] = sd * cval(sS);
                dens[4 * n + a] = sd * cval(sq);
                dens[5 * n + a] = sqrt(fma(ux, ux, fma(uy, uy, 1.0)));
                nnb[a] = nacc;
                pairs += (unsigned)nacc;
            }
        }
        pairs = __reduce_add_sync(0xFFFFFFFFu, pairs);
        shell = __reduce_add_sync(0xFFFFFFFFu, shell);
        if (lane == 0) {
            if (pairs) atomicAdd(&s_acc[0], (unsigned long long)pairs);
            if (shell) atomicAdd(&s_acc[1], (unsigned long long)shell);
        }
    }
    __syncthreads();
    if (tid == 0) {
        if (s_acc[0]) atomicAdd(&v.sc->pairs, s_acc[0]);
        if (s_acc[1]) atomicAdd(&v.sc->shell_tests, s_acc[1]);
    }
}

template <int TT>
__global__ void __launch_bounds__(TT) k_tiled_gradient2m(EvView v, int stage, const double *__restrict__ y,
                                                           const float2 *__restrict__ rel,
                                                           const double *__restrict__ gin,
                                                           const uint32_t *__restrict__ start,
                                                           const uint32_t *__restrict__ cnt, double *__restrict__ gout)
{
    __shared__ float4 cP[kTile2 / 2];
    __shared__ float4 cO[kTile2 / 2];
    __shared__ float4 cXa[kTile2 / 2];  // (X^xx_0, X^xx_1, X^xy_0, X^xy_1) / sigma*^2
    __shared__ float4 cXb[kTile2 / 2];  // (X^yx_0, X^yx_1, X^yy_0, X^yy_1) / sigma*^2
    __shared__ float4 cU2[kTile2 / 2];  // (u^x_0, u^x_1, u^y_0, u^y_1) / sigma*
    __shared__ Runs9 R;
    const size_t n = (size_t)v.n;
    const double *Xxx = gin, *Xxy = gin + n, *Xyx = gin + 2 * n, *Xyy = gin + 3 * n;
    const double *Ux = gin + 4 * n, *Uy = gin + 5 * n;
    const int lim = 1 << v.B, ncell = lim * lim;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = TT / 32;
    const float ih = (float)v.inv_h, slo = v.shell_lo, shi = v.shell_hi;
    const double supp2 = v.supp2;
    for (int ci = blockIdx.x; ci < ncell; ci += gridDim.x) {  // block-uniform
        const int cx = ci % lim, cy = ci / lim;
        const uint32_t kc = morton2((uint32_t)cx, (uint32_t)cy);
        const int na = (int)cnt[kc];
        if (na == 0) continue;
        __syncthreads();
        runs9_setup(v, start, cnt, cx, cy, R);
        const int M = R.cum[9], first = (int)start[kc];
        const int L = lanes_per_particle(na, NW), ppw = 32 / L;
        const int pl = lane / L, l = lane - pl * L;
        for (int g0 = 0; g0 < na; g0 += NW * ppw) {
            const int my = g0 + warp * ppw + pl;
            const bool valid = pl < ppw && my < na;
            const int a = first + (valid ? my : 0);
            const double xa = y[a], ya = y[n + a];
            const float2 ra = rel[a];
            CSum Gx = {0.f, 0.f}, Gy = {0.f, 0.f}, Hx = {0.f, 0.f}, Hy = {0.f, 0.f};
            CSum xx = {0.f, 0.f}, xy = {0.f, 0.f}, yx = {0.f, 0.f}, yy = {0.f, 0.f};
            for (int t0 = 0; t0 < M; t0 += kTile2) {
                const int mt = min(kTile2, M - t0);
                if (g0 == 0 || M > kTile2) {
                    if (t0 > 0 || g0 > 0) __syncthreads();
                    for (int i = tid; i < mt; i += TT) {
                        const int q = t0 + i, o = run_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                        const float2 rb = rel[b];
                        put_pair(cP, i, -rb.x, -rb.y);
                        put_pair(cO, i, -R.ox[o], -R.oy[o]);
                        put_pair(cXa, i, (float)Xxx[b], (float)Xxy[b]);
                        put_pair(cXb, i, (float)Xyx[b], (float)Xyy[b]);
                        put_pair(cU2, i, (float)Ux[b], (float)Uy[b]);
                    }
                    if ((mt & 1) && tid == 0) {
                        put_pair(cP, mt, kFar, kFar);
                        put_pair(cO, mt, 0.0f, 0.0f);
                        put_pair(cXa, mt, 0.0f, 0.0f);
                        put_pair(cXb, mt, 0.0f, 0.0f);
                        put_pair(cU2, mt, 0.0f, 0.0f);
                    }
                    __syncthreads();
                }
                if (valid) {
                    const float2 fx = make_float2(ra.x, ra.x), fy = make_float2(ra.y, ra.y), ih2 = make_float2(ih, ih);
                    const int np = (mt + 1) >> 1;
                    for (int kb = l; kb < np; kb += (kRun / 2) * L) {
                        const int ke = min(np, kb + (kRun / 2) * L);
                        float2 pGx = make_float2(0.f, 0.f), pGy = pGx, pHx = pGx, pHy = pGx;
                        float2 pxx = pGx, pxy = pGx, pyx = pGx, pyy = pGx;
#pragma unroll 2
                        for (int k = kb; k < ke; k += L) {
                            const float4 pk = cP[k], po = cO[k];
                            const float2 dx = __fadd2_rn(__fadd2_rn(fx, lo2(pk)), lo2(po));
                            const float2 dy = __fadd2_rn(__fadd2_rn(fy, hi2(pk)), hi2(po));
                            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                            bool a0 = r2.x < slo, a1 = r2.y < slo;
                            if (r2.x >= slo && r2.x <= shi) {  // thin shell: the exact FP64 decision
                                const int q = t0 + 2 * k, o = run_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a0 = dist2_2d(xa - y[b], ya - y[n + b]) < supp2;
                            }
                            if (r2.y >= slo && r2.y <= shi) {
                                const int q = t0 + 2 * k + 1, o = run_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a1 = dist2_2d(xa - y[b], ya - y[n + b]) < supp2;
                            }
                            // r = 0 (the particle itself) gives dw/dq = 0: a zero term
                            const float2 ir = make_float2(rsqrt_apx(fmaxf(r2.x, 1e-30f)), rsqrt_apx(fmaxf(r2.y, 1e-30f)));
                            float2 t2, t, u2, u;
                            spline_terms2(__fmul2_rn(__fmul2_rn(r2, ir), ih2), t2, t, u2, u);
                            float2 fac = __fmul2_rn(__ffma2_rn(make_float2(-0.75f, -0.75f), t2,
                                                               __fmul2_rn(make_float2(3.0f, 3.0f), u2)), ir);
                            fac.x = a0 ? fac.x : 0.0f;
                            fac.y = a1 ? fac.y : 0.0f;
                            const float2 gx = __fmul2_rn(fac, dx), gy = __fmul2_rn(fac, dy);
                            const float4 xa4 = cXa[k], xb4 = cXb[k], u4 = cU2[k];
                            pGx = __fadd2_rn(pGx, gx);
                            pGy = __fadd2_rn(pGy, gy);
                            pHx = __ffma2_rn(lo2(xa4), gx, __ffma2_rn(lo2(xb4), gy, pHx));
                            pHy = __ffma2_rn(hi2(xa4), gx, __ffma2_rn(hi2(xb4), gy, pHy));
                            pxx = __ffma2_rn(lo2(u4), gx, pxx);
                            pxy = __ffma2_rn(hi2(u4), gx, pxy);
                            pyx = __ffma2_rn(lo2(u4), gy, pyx);
                            pyy = __ffma2_rn(hi2(u4), gy, pyy);
                        }
                        cadd(Gx, pGx.x + pGx.y);
                        cadd(Gy, pGy.x + pGy.y);
                        cadd(Hx, pHx.x + pHx.y);
                        cadd(Hy, pHy.x + pHy.y);
                        cadd(xx, pxx.x + pxx.y);
                        cadd(xy, pxy.x + pxy.y);
                        cadd(yx, pyx.x + pyx.y);
                        cadd(yy, pyy.x + pyy.y);
                    }
                }
            }
            Gx = seg_csum(Gx, l, L);
            Gy = seg_csum(Gy, l, L);
            Hx = seg_csum(Hx, l, L);
            Hy = seg_csum(Hy, l, L);
            xx = seg_csum(xx, l, L);
            xy = seg_csum(xy, l, L);
            yx = seg_csum(yx, l, L);
            yy = seg_csum(yy, l, L);
            if (valid && l == 0) {
                const double tGx = cval(Gx), tGy = cval(Gy), tHx = cval(Hx), tHy = cval(Hy);
                const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
                const double sqrtg = v.milne ? tau : 1.0;
                const double c = v.sigma_d * v.inv_h;
                gout[a] = c * cval(xx);
                gout[n + a] = c * cval(xy);
                gout[2 * n + a] = c * cval(yx);
                gout[3 * n + a] = c * cval(yy);
                const double Fx = Xxx[a] * tGx + Xyx[a] * tGy + tHx;
                const double Fy = Xxy[a] * tGx + Xyy[a] * tGy + tHy;
                gout[4 * n + a] = -sqrtg * c * Fx;
                gout[5 * n + a] = -sqrtg * c * Fy;
            }
        }
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

// blocks of the tiled passes: one per cell of the 2^B x 2^B grid, at most 8 per SM (the rest
// grid-stride)
inline int tiled_grid2(const EvView &v)
{
    const long long ncell = 1ll << (2 * v.B);
    return (int)std::min<long long>(ncell, 8ll * device_sm_count());
}

}  // namespace

void launch_density2m(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                      cudaStream_t st)
{
    k_relpos2<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.fpos);
    k_tiled_density2m<kTT2><<<tiled_grid2(v), kTT2, 0, st>>>(v, y, cb.fpos, Nq, cb.start, cb.cnt, dens, nnb);
}

void launch_gradient2m(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                       cudaStream_t st)
{
    k_tiled_gradient2m<kTT2><<<tiled_grid2(v), kTT2, 0, st>>>(v, stage, y, cb.fpos, gin, cb.start, cb.cnt, gout);
}

}  // namespace sphg
