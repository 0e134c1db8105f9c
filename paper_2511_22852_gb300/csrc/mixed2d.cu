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
//   * sums are compensated (Neumaier two-sum) per lane in float, then each lane's
//     (hi + lo) is combined across the warp in FP64 in a fixed butterfly order.
// The EoS inversion, equations of motion and conservation reductions stay FP64.
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kWarpsM = 4;

// Neumaier compensated accumulation in single precision
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

// candidate walk of one warp over the 3x3 cells with the three-way classification;
// accepted candidates (with their float separation) go to the per-warp queue
template <class Pair>
__device__ __forceinline__ void walk9m(const EvView &v, const uint32_t *__restrict__ start,
                                      const uint32_t *__restrict__ cnt, const float2 *__restrict__ rel,
                                      const double *__restrict__ y, int a, int *qb, float2 *qd, Pair &pair,
                                      unsigned &shell)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int n = v.n;
    const double xa = y[a], ya = y[n + a];
    const float2 ra = rel[a];
    const int cx = cell_coord(xa, dec_double(v.sc->xmin_enc[0]), v.inv_cell);
    const int cy = cell_coord(ya, dec_double(v.sc->xmin_enc[1]), v.inv_cell);
    const int lim = 1 << v.B;
    const float cs = v.cell_f;
    int qn = 0;
    for (int oy = -1; oy <= 1; ++oy) {
        const int ny = cy + oy;
        if (ny < 0 || ny >= lim) continue;
        for (int ox = -1; ox <= 1; ++ox) {
            const int nx = cx + ox;
            if (nx < 0 || nx >= lim) continue;
            const uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
            const uint32_t b0 = start[k], b1 = b0 + cnt[k];
            const float offx = (float)ox * cs, offy = (float)oy * cs;
            for (uint32_t base = b0; base < b1; base += 32) {
                const uint32_t b = base + lane;
                bool acc = false;
                float dx = 0.0f, dy = 0.0f;
                if (b < b1) {
                    const float2 rb = rel[b];
                    dx = (ra.x - rb.x) - offx;
                    dy = (ra.y - rb.y) - offy;
                    const float r2 = fmaf(dx, dx, dy * dy);
                    if (r2 < v.shell_lo) {
                        acc = true;
                    } else if (r2 <= v.shell_hi) {  // thin shell: the exact FP64 decision
                        acc = dist2_2d(xa - y[b], ya - y[n + b]) < v.supp2;
                        ++shell;
                    }
                }
                const unsigned m = __ballot_sync(0xFFFFFFFFu, acc);
                if (acc) {
                    const int slot = qn + __popc(m & lt);
                    qb[slot] = (int)b;
                    qd[slot] = make_float2(dx, dy);
                }
                qn += __popc(m);
                __syncwarp();
                if (qn >= 32) {
                    pair(qb[lane], qd[lane]);
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
    if (lane < qn) pair(qb[lane], qd[lane]);
}

__global__ void __launch_bounds__(32 * kWarpsM) k_density2m(EvView v, const double *__restrict__ y,
                                                            const float2 *__restrict__ rel,
                                                            const double *__restrict__ Nq,
                                                            const uint32_t *__restrict__ start,
                                                            const uint32_t *__restrict__ cnt,
                                                            double *__restrict__ dens, int *__restrict__ nnb)
{
    __shared__ int qb_s[kWarpsM][64];
    __shared__ float2 qd_s[kWarpsM][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarpsM + wid;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const double *S = y + 4 * n;
    const float ih = (float)v.inv_h;
    CSum sg = {0, 0}, ss = {0, 0}, sb = {0, 0}, sS = {0, 0}, sq = {0, 0};
    int c = 0;
    unsigned shell = 0;
    auto pair = [&](int b, float2 d) {
        const float r2 = fmaf(d.x, d.x, d.y * d.y);
        const float q = sqrt_apx(r2) * ih;
        const float w = kernel_wf(q);
        cadd(sg, w);
        cadd(ss, (float)S[b] * w);
        cadd(sb, (float)Nq[b] * w);
        cadd(sS, (float)Nq[n + b] * w);
        cadd(sq, (float)Nq[2 * n + b] * w);
        ++c;
    };
    walk9m(v, start, cnt, rel, y, a, qb_s[wid], qd_s[wid], pair, shell);
    const double tsg = cwarp(sg), tss = cwarp(ss), tsb = cwarp(sb), tsS = cwarp(sS), tsq = cwarp(sq);
    for (int o = 16; o > 0; o >>= 1) {
        c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        shell += __shfl_xor_sync(0xFFFFFFFFu, shell, o);
    }
    if (lane == 0) {
        const double ux = y[2 * n + a], uy = y[3 * n + a];
        const double sd = v.sigma_d;
        dens[a] = sd * tsg;
        dens[n + a] = sd * tss;
        dens[2 * n + a] = sd * tsb;
        dens[3 * n + a] = sd * tsS;
        dens[4 * n + a] = sd * tsq;
        dens[5 * n + a] = sqrt(fma(ux, ux, fma(uy, uy, 1.0)));
        nnb[a] = c;
        atomicAdd(&v.sc->pairs, (unsigned long long)c);
        if (shell) atomicAdd(&v.sc->shell_tests, (unsigned long long)shell);
    }
}

__global__ void __launch_bounds__(32 * kWarpsM) k_gradient2m(EvView v, int stage, const double *__restrict__ y,
                                                             const float2 *__restrict__ rel,
                                                             const double *__restrict__ gin,
                                                             const uint32_t *__restrict__ start,
                                                             const uint32_t *__restrict__ cnt,
                                                             double *__restrict__ gout)
{
    __shared__ int qb_s[kWarpsM][64];
    __shared__ float2 qd_s[kWarpsM][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarpsM + wid;
    if (a >= v.n) return;
    const size_t n = (size_t)v.n;
    const double *Xxx = gin, *Xxy = gin + n, *Xyx = gin + 2 * n, *Xyy = gin + 3 * n;
    const double *Ux = gin + 4 * n, *Uy = gin + 5 * n;
    const float ih = (float)v.inv_h;
    CSum Gx = {0, 0}, Gy = {0, 0}, Hx = {0, 0}, Hy = {0, 0}, dxux = {0, 0}, dxuy = {0, 0}, dyux = {0, 0}, dyuy = {0, 0};
    unsigned shell = 0;
    auto pair = [&](int b, float2 d) {
        const float r2 = fmaf(d.x, d.x, d.y * d.y);
        if (r2 > 0.0f) {
            const float ir = rsqrt_apx(fmaxf(r2, 1e-30f));  // a denormal r2 flushed to 0 would give inf
            const float fac = kernel_dwf(r2 * ir * ih) * ir;
            const float gx = fac * d.x, gy = fac * d.y;
            cadd(Gx, gx);
            cadd(Gy, gy);
            cadd(Hx, fmaf((float)Xxx[b], gx, (float)Xyx[b] * gy));
            cadd(Hy, fmaf((float)Xxy[b], gx, (float)Xyy[b] * gy));
            const float ubx = (float)Ux[b], uby = (float)Uy[b];
            cadd(dxux, ubx * gx);
            cadd(dxuy, uby * gx);
            cadd(dyux, ubx * gy);
            cadd(dyuy, uby * gy);
        }
    };
    walk9m(v, start, cnt, rel, y, a, qb_s[wid], qd_s[wid], pair, shell);
    const double tGx = cwarp(Gx), tGy = cwarp(Gy), tHx = cwarp(Hx), tHy = cwarp(Hy);
    const double t00 = cwarp(dxux), t01 = cwarp(dxuy), t10 = cwarp(dyux), t11 = cwarp(dyuy);
    if (lane == 0) {
        const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
        const double sqrtg = v.milne ? tau : 1.0;
        const double c = v.sigma_d * v.inv_h;
        gout[a] = c * t00;
        gout[n + a] = c * t01;
        gout[2 * n + a] = c * t10;
        gout[3 * n + a] = c * t11;
        const double Fx = Xxx[a] * tGx + Xyx[a] * tGy + tHx;
        const double Fy = Xxy[a] * tGx + Xyy[a] * tGy + tHy;
        gout[4 * n + a] = -sqrtg * c * Fx;
        gout[5 * n + a] = -sqrtg * c * Fy;
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_density2m(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                      cudaStream_t st)
{
    k_relpos2<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.fpos);
    k_density2m<<<nblk(v.n, kWarpsM), 32 * kWarpsM, 0, st>>>(v, y, cb.fpos, Nq, cb.start, cb.cnt, dens, nnb);
}

void launch_gradient2m(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb, double *gout,
                       cudaStream_t st)
{
    k_gradient2m<<<nblk(v.n, kWarpsM), 32 * kWarpsM, 0, st>>>(v, stage, y, cb.fpos, gin, cb.start, cb.cnt, gout);
}

}  // namespace sphg
