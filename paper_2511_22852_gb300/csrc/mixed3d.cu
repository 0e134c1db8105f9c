// mixed3d.cu -- the neighbour passes (rows a3, a5) of the 3+1D step in the mixed-precision
// form: one warp per particle over the 27 neighbouring cells, positions relative to the
// origin of their cell in single precision, separations (r_a - r_b) - o (2h) formed from
// numbers of size <= 2h, a proven float error band around (2h)^2 inside which the FP64 test
// r^2 < (2h)^2 (separately rounded products) decides -- the neighbour sets are those of the
// FP64 form -- and sums accumulated in float in short runs folded into Neumaier-compensated
// sums, combined across the warp in FP64 in a fixed order.  The EoS inversion, equations of
// motion and reductions stay FP64 (step3d.cu).
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kW3 = 4;      // warps (particles) per block
constexpr int kFold = 4;    // pair calls (32 pairs each per warp) summed in plain float per run

struct CSum {
    float hi, lo;
};
__device__ __forceinline__ void cadd(CSum &s, float x)
{
    float t = s.hi + x;
    if (fabsf(s.hi) >= fabsf(x)) s.lo += (s.hi - t) + x;
    else s.lo += (x - t) + s.hi;
    s.hi = t;
}
__device__ __forceinline__ double cwarp(CSum s)
{
    double v = (double)s.hi + (double)s.lo;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ __forceinline__ float kernel_wf(float q)
{
    if (q <= 1.0f) return fmaf(q * q, fmaf(0.75f, q, -1.5f), 1.0f);
    float t = 2.0f - q;
    return 0.25f * t * t * t;
}
__device__ __forceinline__ float kernel_dwf(float q)
{
    if (q <= 1.0f) return q * fmaf(2.25f, q, -3.0f);
    float t = 2.0f - q;
    return -0.75f * t * t;
}
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

// the 27-cell walk of one warp with the three-way classification; accepted candidates and
// their float separations go to the per-warp queue; `pair` runs on full warps, then `fold`
// after every kFold full-warp calls (and once at the end)
template <class Pair, class Fold>
__device__ __forceinline__ void walk27m(const EvView &v, const uint32_t *__restrict__ start,
                                        const uint32_t *__restrict__ cnt, const float4 *__restrict__ rel,
                                        const double *__restrict__ y, int a, int *qb, float4 *qd, Pair &pair,
                                        Fold &fold, unsigned &shell)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const size_t n = (size_t)v.n;
    const double xa[3] = {y[a], y[n + a], y[2 * n + a]};
    const float4 ra = rel[a];
    int c[3], lim[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        c[d] = cell_coord(xa[d], dec_double(v.sc->xmin_enc[d]), v.inv_cell);
        lim[d] = 1 << v.B3[d];
    }
    const float cs = v.cell_f;
    int qn = 0, calls = 0;
    for (int oz = -1; oz <= 1; ++oz) {
        const int nz = c[2] + oz;
        if (nz < 0 || nz >= lim[2]) continue;
        for (int oy = -1; oy <= 1; ++oy) {
            const int ny = c[1] + oy;
            if (ny < 0 || ny >= lim[1]) continue;
            for (int ox = -1; ox <= 1; ++ox) {
                const int nx = c[0] + ox;
                if (nx < 0 || nx >= lim[0]) continue;
                const uint32_t k = key3m(v, nx, ny, nz);
                const uint32_t b0 = start[k], b1 = b0 + cnt[k];
                const float offx = (float)ox * cs, offy = (float)oy * cs, offz = (float)oz * cs;
                for (uint32_t base = b0; base < b1; base += 32) {
                    const uint32_t b = base + lane;
                    bool acc = false;
                    float dx = 0.0f, dy = 0.0f, dz = 0.0f, r2 = 0.0f;
                    if (b < b1) {
                        const float4 rb = rel[b];
                        dx = (ra.x - rb.x) - offx;
                        dy = (ra.y - rb.y) - offy;
                        dz = (ra.z - rb.z) - offz;
                        r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                        if (r2 < v.shell_lo) {
                            acc = true;
                        } else if (r2 <= v.shell_hi) {  // thin shell: the exact FP64 decision
                            acc = dist2_3e(xa[0] - y[b], xa[1] - y[n + b], xa[2] - y[2 * n + b]) < v.supp2;
                            ++shell;
                        }
                    }
                    const unsigned m = __ballot_sync(0xFFFFFFFFu, acc);
                    if (acc) {
                        const int slot = qn + __popc(m & lt);
                        qb[slot] = (int)b;
                        qd[slot] = make_float4(dx, dy, dz, r2);
                    }
                    qn += __popc(m);
                    __syncwarp();
                    if (qn >= 32) {
                        pair(qb[lane], qd[lane], true);
                        if (++calls == kFold) {
                            fold();
                            calls = 0;
                        }
                        qn -= 32;
                        __syncwarp();
                        if (lane < qn) {
                            qb[lane] = qb[32 + lane];
                            qd[lane] = qd[32 + lane];
                        }
                        __syncwarp();
                    }
                }
            }
        }
    }
    pair(lane < qn ? qb[lane] : 0, lane < qn ? qd[lane] : make_float4(0.f, 0.f, 0.f, 0.f), lane < qn);
    fold();
}

__global__ void __launch_bounds__(32 * kW3) k_density3m(EvView v, const double *__restrict__ y,
                                                        const float4 *__restrict__ rel,
                                                        const double *__restrict__ Nq,
                                                        const uint32_t *__restrict__ start,
                                                        const uint32_t *__restrict__ cnt, double *__restrict__ dens,
                                                        int *__restrict__ nnb)
{
    __shared__ int qb_s[kW3][64];
    __shared__ float4 qd_s[kW3][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kW3 + wid;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const double *S = y + 6 * n;
    const float ih = (float)v.inv_h;
    CSum sg = {0, 0}, ss = {0, 0}, sb = {0, 0}, sS = {0, 0}, sq = {0, 0};
    float pg = 0.f, ps = 0.f, pB = 0.f, pS = 0.f, pQ = 0.f;
    int c = 0;
    unsigned shell = 0;
    auto pair = [&](int b, float4 d, bool ok) {
        if (!ok) return;
        const float q = sqrt_apx(d.w) * ih;
        const float w = kernel_wf(q);
        pg += w;
        ps = fmaf((float)S[b], w, ps);
        pB = fmaf((float)Nq[b], w, pB);
        pS = fmaf((float)Nq[n + b], w, pS);
        pQ = fmaf((float)Nq[2 * n + b], w, pQ);
        ++c;
    };
    auto fold = [&]() {
        cadd(sg, pg);
        cadd(ss, ps);
        cadd(sb, pB);
        cadd(sS, pS);
        cadd(sq, pQ);
        pg = ps = pB = pS = pQ = 0.f;
    };
    walk27m(v, start, cnt, rel, y, a, qb_s[wid], qd_s[wid], pair, fold, shell);
    const double tsg = cwarp(sg), tss = cwarp(ss), tsb = cwarp(sb), tsS = cwarp(sS), tsq = cwarp(sq);
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        shell += __shfl_xor_sync(0xFFFFFFFFu, shell, o);
    }
    if (lane == 0) {
        const double sd = v.sigma_d;
        dens[a] = sd * tsg;
        dens[n + a] = sd * tss;
        dens[2 * n + a] = sd * tsb;
        dens[3 * n + a] = sd * tsS;
        dens[4 * n + a] = sd * tsq;
        nnb[a] = c;
        atomicAdd(&v.sc->pairs, (unsigned long long)c);
        if (shell) atomicAdd(&v.sc->shell_tests, (unsigned long long)shell);
    }
}

// gin rows: X^{ji}/sigma*^2 at 3 j + i, u^j/sigma* at 9 + j; gout rows: d_k u^j at 3 k + j,
// then F^i at 9 + i (the layout of the FP64 3+1D gradient pass)
__global__ void __launch_bounds__(32 * kW3) k_gradient3m(EvView v, int stage, const double *__restrict__ y,
                                                         const float4 *__restrict__ rel,
                                                         const double *__restrict__ gin,
                                                         const uint32_t *__restrict__ start,
                                                         const uint32_t *__restrict__ cnt,
                                                         double *__restrict__ gout)
{
    __shared__ int qb_s[kW3][64];
    __shared__ float4 qd_s[kW3][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kW3 + wid;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const float ih = (float)v.inv_h;
    CSum G[3], H[3], du[3][3];
    float pG[3], pH[3], pdu[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        G[i] = H[i] = CSum{0.f, 0.f};
        pG[i] = pH[i] = 0.f;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            du[i][j] = CSum{0.f, 0.f};
            pdu[i][j] = 0.f;
        }
    }
    unsigned shell = 0;
    auto pair = [&](int b, float4 d, bool ok) {
        if (!ok || !(d.w > 0.0f)) return;
        const float ir = rsqrt_apx(fmaxf(d.w, 1e-30f));  // a denormal r2 flushed to 0 would give inf
        const float fac = kernel_dwf(d.w * ir * ih) * ir;
        const float gw[3] = {fac * d.x, fac * d.y, fac * d.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) pG[k] += gw[k];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            float h = pH[i];
#pragma unroll
            for (int j = 0; j < 3; ++j) h = fmaf((float)gin[(size_t)(3 * j + i) * n + b], gw[j], h);
            pH[i] = h;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float ub = (float)gin[(size_t)(9 + j) * n + b];
#pragma unroll
            for (int k = 0; k < 3; ++k) pdu[k][j] = fmaf(ub, gw[k], pdu[k][j]);
        }
    };
    auto fold = [&]() {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            cadd(G[i], pG[i]);
            cadd(H[i], pH[i]);
            pG[i] = pH[i] = 0.f;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                cadd(du[i][j], pdu[i][j]);
                pdu[i][j] = 0.f;
            }
        }
    };
    walk27m(v, start, cnt, rel, y, a, qb_s[wid], qd_s[wid], pair, fold, shell);
    double tG[3], tH[3], tdu[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        tG[i] = cwarp(G[i]);
        tH[i] = cwarp(H[i]);
#pragma unroll
        for (int j = 0; j < 3; ++j) tdu[i][j] = cwarp(du[i][j]);
    }
    if (lane == 0) {
        const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
        const double sqrtg = v.milne ? tau : 1.0;
        const double cf = v.sigma_d * v.inv_h;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int j = 0; j < 3; ++j) gout[(size_t)(3 * k + j) * n + a] = cf * tdu[k][j];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            double F = tH[i];
#pragma unroll
            for (int j = 0; j < 3; ++j) F = fma(gin[(size_t)(3 * j + i) * n + a], tG[j], F);
            gout[(size_t)(9 + i) * n + a] = -sqrtg * cf * F;
        }
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_density3m(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                      cudaStream_t st)
{
    k_relpos3<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.fpos3);
    k_density3m<<<nblk(v.n, kW3), 32 * kW3, 0, st>>>(v, y, cb.fpos3, Nq, cb.start, cb.cnt, dens, nnb);
}

void launch_gradient3m(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                       cudaStream_t st)
{
    k_gradient3m<<<nblk(v.n, kW3), 32 * kW3, 0, st>>>(v, stage, y, cb.fpos3, gin, cb.start, cb.cnt, gout);
}

}  // namespace sphg
