// mixed3d.cu -- the neighbour passes (rows a3, a5) of the 3+1D step in the mixed-precision
// form: cell-tiled over the 27 neighbouring 2h-cells, positions relative to the origin of their
// cell in single precision, separations (r_a - r_b) - o (2h) formed from numbers of size <= 2h,
// a proven float error band around (2h)^2 inside which the FP64 test r^2 < (2h)^2 (separately
// rounded products) decides -- the neighbour sets are those of the FP64 form -- and sums
// accumulated in float in short runs folded into Neumaier-compensated sums, a particle's lanes
// combined with error-free FP32 additions.  The EoS inversion, equations of motion and
// reductions stay FP64 (step3d.cu).
#include <algorithm>

#include "sph_internal.cuh"
#include "tiled_common.cuh"

namespace sphg {

namespace {

__device__ __forceinline__ double dist2_3e(double dx, double dy, double dz)
{
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}
__device__ __forceinline__ uint32_t key3m(const EvView &v, int cx, int cy, int cz)
{
    return v.spread[cx] | v.spread[1024 + cy] | v.spread[2048 + cz];
}

// cell-relative single-precision positions of the sorted particles
__global__ void k_relpos3(EvView v, const double *__restrict__ y, float4 *__restrict__ rel)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= v.n) return;
    const double cs = 2.0 * v.h;
    float r[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double xm = dec_double(v.sc->xmin_enc[d]);
        const double x = y[(size_t)d * v.n + j];
        const int c = cell_coord(x, xm, v.inv_cell);
        r[d] = __double2float_rn(__dsub_rn(__dsub_rn(x, xm), (double)c * cs));
    }
    rel[j] = make_float4(r[0], r[1], r[2], 0.0f);
}

// Cell-tiled passes (the 3+1D counterpart of the 2+1D ones): one block per occupied cell
// (grid-stride over the cell grid) stages the candidates of the 3x3x3 block of 2h-cells -- 27
// runs of the sorted order -- in shared memory, two candidates per float4 entry (packed
// two-wide FP32 arithmetic), and the cell's particles scan them with L lanes each.  A candidate
// carries its own-cell-relative position and its cell's offset separately, and r^2 is nested
// as fmaf(dx, dx, fmaf(dy, dy, dz dz)), the rounding the 3+1D shell bound assumes.
constexpr int kTT3 = 256;    // threads of a tiled block; all its warps share a cell's particles
constexpr int kTile3 = 512;  // candidates staged at a time

struct Runs27 {
    int rs[27];
    int cum[28];
    float o[3][27];  // the run's cell offset times the float cell side, per axis
};

__device__ __forceinline__ void runs27_setup(const EvView &v, const uint32_t *__restrict__ start,
                                             const uint32_t *__restrict__ cnt, const int c[3], Runs27 &R)
{
    const int t = threadIdx.x;
    if (t < 27) {
        const int d[3] = {t % 3 - 1, (t / 3) % 3 - 1, t / 9 - 1};
        int nc[3];
        bool in = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            nc[k] = c[k] + d[k];
            in = in && nc[k] >= 0 && nc[k] < (1 << v.B3[k]);
        }
        int st = 0, len = 0;
        if (in) {
            const uint32_t k = key3m(v, nc[0], nc[1], nc[2]);
            st = (int)start[k];
            len = (int)cnt[k];
        }
        R.rs[t] = st;
        R.cum[t + 1] = len;
#pragma unroll
        for (int k = 0; k < 3; ++k) R.o[k][t] = (float)d[k] * v.cell_f;
    }
    __syncthreads();
    if (t == 0) {
        R.cum[0] = 0;
        for (int o = 0; o < 27; ++o) R.cum[o + 1] += R.cum[o];
    }
    __syncthreads();
}

__device__ __forceinline__ int run27_of(const Runs27 &R, int q)
{
    int lo = 0, hi = 26;  // the last run whose start is <= q
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (R.cum[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// the candidate's staged geometry: (-x, -y) and (-z, -o_z) pairs, and the (-o_x, -o_y) offsets
__device__ __forceinline__ void stage_geom(float4 *cP, float4 *cPz, float4 *cO, int i, float4 rb, const Runs27 &R,
                                           int o)
{
    put_pair(cP, i, -rb.x, -rb.y);
    put_pair(cPz, i, -rb.z, -R.o[2][o]);
    put_pair(cO, i, -R.o[0][o], -R.o[1][o]);
}
__device__ __forceinline__ void stage_far(float4 *cP, float4 *cPz, float4 *cO, int i)
{
    put_pair(cP, i, kFar, kFar);
    put_pair(cPz, i, kFar, 0.0f);
    put_pair(cO, i, 0.0f, 0.0f);
}

// separations and r^2 of a candidate pair, (r_a - r_b) - o (2h) per axis
__device__ __forceinline__ void sep2(float4 ra, float4 pk, float4 pz, float4 po, float2 &dx, float2 &dy, float2 &dz,
                                     float2 &r2)
{
    dx = __fadd2_rn(__fadd2_rn(make_float2(ra.x, ra.x), lo2(pk)), lo2(po));
    dy = __fadd2_rn(__fadd2_rn(make_float2(ra.y, ra.y), hi2(pk)), hi2(po));
    dz = __fadd2_rn(__fadd2_rn(make_float2(ra.z, ra.z), lo2(pz)), hi2(pz));
    r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
}

__global__ void __launch_bounds__(kTT3) k_tiled_density3m(EvView v, const double *__restrict__ y,
                                                          const float4 *__restrict__ rel,
                                                          const double *__restrict__ Nq,
                                                          const uint32_t *__restrict__ start,
                                                          const uint32_t *__restrict__ cnt,
                                                          double *__restrict__ dens, int *__restrict__ nnb)
{
    __shared__ float4 cP[kTile3 / 2], cPz[kTile3 / 2], cO[kTile3 / 2];
    __shared__ float4 cQa[kTile3 / 2];  // (S_0, S_1, N_B0, N_B1)
    __shared__ float4 cQb[kTile3 / 2];  // (N_S0, N_S1, N_Q0, N_Q1)
    __shared__ Runs27 R;
    __shared__ unsigned long long s_acc[2];
    const size_t n = (size_t)v.n;
    const double *S = y + 6 * n;
    const int l0 = 1 << v.B3[0], l1 = 1 << v.B3[1];
    const long long ncell = (long long)l0 * l1 * (1 << v.B3[2]);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kTT3 / 32;
    const float ih = (float)v.inv_h, slo = v.shell_lo, shi = v.shell_hi;
    const double supp2 = v.supp2, sd = v.sigma_d;
    if (tid == 0) s_acc[0] = s_acc[1] = 0ull;
    for (long long ci = blockIdx.x; ci < ncell; ci += gridDim.x) {  // block-uniform
        const int c[3] = {(int)(ci % l0), (int)((ci / l0) % l1), (int)(ci / ((long long)l0 * l1))};
        const uint32_t kc = key3m(v, c[0], c[1], c[2]);
        const int na = (int)cnt[kc];
        if (na == 0) continue;
        __syncthreads();
        runs27_setup(v, start, cnt, c, R);
        const int M = R.cum[27], first = (int)start[kc];
        const int L = lanes_per_particle(na, NW), ppw = 32 / L;
        const int pl = lane / L, l = lane - pl * L;
        unsigned pairs = 0u, shell = 0u;
        for (int g0 = 0; g0 < na; g0 += NW * ppw) {
            const int my = g0 + warp * ppw + pl;
            const bool valid = pl < ppw && my < na;
            const int a = first + (valid ? my : 0);
            const double xa[3] = {y[a], y[n + a], y[2 * n + a]};
            const float4 ra = rel[a];
            CSum sg = {0.f, 0.f}, ss = {0.f, 0.f}, sb = {0.f, 0.f}, sS = {0.f, 0.f}, sq = {0.f, 0.f};
            int nacc = 0;
            for (int t0 = 0; t0 < M; t0 += kTile3) {
                const int mt = min(kTile3, M - t0);
                if (g0 == 0 || M > kTile3) {
                    if (t0 > 0 || g0 > 0) __syncthreads();
                    for (int i = tid; i < mt; i += kTT3) {
                        const int q = t0 + i, o = run27_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                        stage_geom(cP, cPz, cO, i, rel[b], R, o);
                        put_pair(cQa, i, (float)S[b], (float)Nq[b]);
                        put_pair(cQb, i, (float)Nq[n + b], (float)Nq[2 * n + b]);
                    }
                    if ((mt & 1) && tid == 0) {
                        stage_far(cP, cPz, cO, mt);
                        put_pair(cQa, mt, 0.0f, 0.0f);
                        put_pair(cQb, mt, 0.0f, 0.0f);
                    }
                    __syncthreads();
                }
                if (valid) {
                    const float2 ih2 = make_float2(ih, ih);
                    const int np = (mt + 1) >> 1;
                    for (int kb = l; kb < np; kb += (kRun / 2) * L) {
                        const int ke = min(np, kb + (kRun / 2) * L);
                        float2 pg = make_float2(0.f, 0.f), ps = pg, pB = pg, pS = pg, pQ = pg;
#pragma unroll 2
                        for (int k = kb; k < ke; k += L) {
                            float2 dx, dy, dz, r2;
                            sep2(ra, cP[k], cPz[k], cO[k], dx, dy, dz, r2);
                            bool a0 = r2.x < slo, a1 = r2.y < slo;
                            if (r2.x >= slo && r2.x <= shi) {  // thin shell: the exact FP64 decision
                                const int q = t0 + 2 * k, o = run27_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a0 = dist2_3e(xa[0] - y[b], xa[1] - y[n + b], xa[2] - y[2 * n + b]) < supp2;
                                ++shell;
                            }
                            if (r2.y >= slo && r2.y <= shi) {
                                const int q = t0 + 2 * k + 1, o = run27_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a1 = dist2_3e(xa[0] - y[b], xa[1] - y[n + b], xa[2] - y[2 * n + b]) < supp2;
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
            for (int o = 1; o < L; o <<= 1) {
                const int t = __shfl_down_sync(0xFFFFFFFFu, nacc, o);
                if ((l & (2 * o - 1)) == 0 && l + o < L) nacc += t;
            }
            if (valid && l == 0) {
                dens[a] = sd * cval(sg);
                dens[n + a] = sd * cval(ss);
                dens[2 * n + a] = sd * cval(sb);
                dens[3 * n + a] = sd * cval(sS);
                dens[4 * n + a] = sd * cval(sq);
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

// gin rows: X^{ji}/sigma*^2 at 3 j + i, u^j/sigma* at 9 + j; gout rows: d_k u^j at 3 k + j, then
// F^i at 9 + i (the layout of the FP64 3+1D gradient pass).  Candidate rows r = 0..11 are staged
// as six pair arrays (row 2m in the low, 2m + 1 in the high half of entry m).
__global__ void __launch_bounds__(kTT3) k_tiled_gradient3m(EvView v, int stage, const double *__restrict__ y,
                                                           const float4 *__restrict__ rel,
                                                           const double *__restrict__ gin,
                                                           const uint32_t *__restrict__ start,
                                                           const uint32_t *__restrict__ cnt, double *__restrict__ gout)
{
    __shared__ float4 cP[kTile3 / 2], cPz[kTile3 / 2], cO[kTile3 / 2];
    __shared__ float4 cV[6][kTile3 / 2];
    __shared__ Runs27 R;
    const size_t n = (size_t)v.n;
    const int l0 = 1 << v.B3[0], l1 = 1 << v.B3[1];
    const long long ncell = (long long)l0 * l1 * (1 << v.B3[2]);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kTT3 / 32;
    const float ih = (float)v.inv_h, slo = v.shell_lo, shi = v.shell_hi;
    const double supp2 = v.supp2;
    for (long long ci = blockIdx.x; ci < ncell; ci += gridDim.x) {  // block-uniform
        const int c[3] = {(int)(ci % l0), (int)((ci / l0) % l1), (int)(ci / ((long long)l0 * l1))};
        const uint32_t kc = key3m(v, c[0], c[1], c[2]);
        const int na = (int)cnt[kc];
        if (na == 0) continue;
        __syncthreads();
        runs27_setup(v, start, cnt, c, R);
        const int M = R.cum[27], first = (int)start[kc];
        const int L = lanes_per_particle(na, NW), ppw = 32 / L;
        const int pl = lane / L, l = lane - pl * L;
        for (int g0 = 0; g0 < na; g0 += NW * ppw) {
            const int my = g0 + warp * ppw + pl;
            const bool valid = pl < ppw && my < na;
            const int a = first + (valid ? my : 0);
            const double xa[3] = {y[a], y[n + a], y[2 * n + a]};
            const float4 ra = rel[a];
            CSum G[3], H[3], du[3][3];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                G[i] = H[i] = CSum{0.f, 0.f};
#pragma unroll
                for (int j = 0; j < 3; ++j) du[i][j] = CSum{0.f, 0.f};
            }
            for (int t0 = 0; t0 < M; t0 += kTile3) {
                const int mt = min(kTile3, M - t0);
                if (g0 == 0 || M > kTile3) {
                    if (t0 > 0 || g0 > 0) __syncthreads();
                    for (int i = tid; i < mt; i += kTT3) {
                        const int q = t0 + i, o = run27_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                        stage_geom(cP, cPz, cO, i, rel[b], R, o);
#pragma unroll
                        for (int m = 0; m < 6; ++m)
                            put_pair(cV[m], i, (float)gin[(size_t)(2 * m) * n + b], (float)gin[(size_t)(2 * m + 1) * n + b]);
                    }
                    if ((mt & 1) && tid == 0) {
                        stage_far(cP, cPz, cO, mt);
#pragma unroll
                        for (int m = 0; m < 6; ++m) put_pair(cV[m], mt, 0.0f, 0.0f);
                    }
                    __syncthreads();
                }
                if (valid) {
                    const float2 ih2 = make_float2(ih, ih);
                    const int np = (mt + 1) >> 1;
                    for (int kb = l; kb < np; kb += (kRun / 2) * L) {
                        const int ke = min(np, kb + (kRun / 2) * L);
                        float2 pG[3], pH[3], pdu[3][3];
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            pG[i] = pH[i] = make_float2(0.f, 0.f);
#pragma unroll
                            for (int j = 0; j < 3; ++j) pdu[i][j] = make_float2(0.f, 0.f);
                        }
                        for (int k = kb; k < ke; k += L) {
                            float2 dx, dy, dz, r2;
                            sep2(ra, cP[k], cPz[k], cO[k], dx, dy, dz, r2);
                            bool a0 = r2.x < slo, a1 = r2.y < slo;
                            if (r2.x >= slo && r2.x <= shi) {  // thin shell: the exact FP64 decision
                                const int q = t0 + 2 * k, o = run27_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a0 = dist2_3e(xa[0] - y[b], xa[1] - y[n + b], xa[2] - y[2 * n + b]) < supp2;
                            }
                            if (r2.y >= slo && r2.y <= shi) {
                                const int q = t0 + 2 * k + 1, o = run27_of(R, q), b = R.rs[o] + (q - R.cum[o]);
                                a1 = dist2_3e(xa[0] - y[b], xa[1] - y[n + b], xa[2] - y[2 * n + b]) < supp2;
                            }
                            // r = 0 (the particle itself) gives dw/dq = 0: a zero term
                            const float2 ir = make_float2(rsqrt_apx(fmaxf(r2.x, 1e-30f)), rsqrt_apx(fmaxf(r2.y, 1e-30f)));
                            float2 t2, t, u2, u;
                            spline_terms2(__fmul2_rn(__fmul2_rn(r2, ir), ih2), t2, t, u2, u);
                            float2 fac = __fmul2_rn(__ffma2_rn(make_float2(-0.75f, -0.75f), t2,
                                                               __fmul2_rn(make_float2(3.0f, 3.0f), u2)), ir);
                            fac.x = a0 ? fac.x : 0.0f;
                            fac.y = a1 ? fac.y : 0.0f;
                            const float2 g[3] = {__fmul2_rn(fac, dx), __fmul2_rn(fac, dy), __fmul2_rn(fac, dz)};
                            float2 row[12];
#pragma unroll
                            for (int m = 0; m < 6; ++m) {
                                const float4 e = cV[m][k];
                                row[2 * m] = lo2(e);
                                row[2 * m + 1] = hi2(e);
                            }
#pragma unroll
                            for (int i = 0; i < 3; ++i) {
                                pG[i] = __fadd2_rn(pG[i], g[i]);
                                // sum_j X^{ji} g_j, j = 0, 1, 2 in turn
                                pH[i] = __ffma2_rn(row[6 + i], g[2],
                                                   __ffma2_rn(row[3 + i], g[1], __ffma2_rn(row[i], g[0], pH[i])));
                            }
#pragma unroll
                            for (int j = 0; j < 3; ++j)
#pragma unroll
                                for (int kk = 0; kk < 3; ++kk) pdu[kk][j] = __ffma2_rn(row[9 + j], g[kk], pdu[kk][j]);
                        }
#pragma unroll
                        for (int i = 0; i < 3; ++i) {
                            cadd(G[i], pG[i].x + pG[i].y);
                            cadd(H[i], pH[i].x + pH[i].y);
#pragma unroll
                            for (int j = 0; j < 3; ++j) cadd(du[i][j], pdu[i][j].x + pdu[i][j].y);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                G[i] = seg_csum(G[i], l, L);
                H[i] = seg_csum(H[i], l, L);
#pragma unroll
                for (int j = 0; j < 3; ++j) du[i][j] = seg_csum(du[i][j], l, L);
            }
            if (valid && l == 0) {
                const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
                const double sqrtg = v.milne ? tau : 1.0;
                const double cf = v.sigma_d * v.inv_h;
                double tG[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) tG[i] = cval(G[i]);
#pragma unroll
                for (int kk = 0; kk < 3; ++kk)
#pragma unroll
                    for (int j = 0; j < 3; ++j) gout[(size_t)(3 * kk + j) * n + a] = cf * cval(du[kk][j]);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    double F = cval(H[i]);
#pragma unroll
                    for (int j = 0; j < 3; ++j) F = fma(gin[(size_t)(3 * j + i) * n + a], tG[j], F);
                    gout[(size_t)(9 + i) * n + a] = -sqrtg * cf * F;
                }
            }
        }
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

// blocks of the tiled passes: one per cell of the grid, at most 8 per SM (the rest grid-stride)
inline int tiled_grid3(const EvView &v)
{
    const long long ncell = 1ll << (v.B3[0] + v.B3[1] + v.B3[2]);
    return (int)std::min<long long>(ncell, 8ll * device_sm_count());
}

}  // namespace

void launch_density3m(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                      cudaStream_t st)
{
    k_relpos3<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.fpos3);
    k_tiled_density3m<<<tiled_grid3(v), kTT3, 0, st>>>(v, y, cb.fpos3, Nq, cb.start, cb.cnt, dens, nnb);
}

void launch_gradient3m(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                       cudaStream_t st)
{
    k_tiled_gradient3m<<<tiled_grid3(v), kTT3, 0, st>>>(v, stage, y, cb.fpos3, gin, cb.start, cb.cnt, gout);
}

}  // namespace sphg
