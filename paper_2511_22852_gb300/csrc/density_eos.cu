// density_eos.cu -- kernel-sum densities (row a3) and the EoS inversion (row a4).
//
// Density pass (eqs. sigmastar, refconv): one warp per particle (sorted order)
// walks the 3x3 cells around its own; a single-precision prefilter with a proven
// error margin discards far candidates, the survivors are compacted so the FP64
// work runs on full warps.  The acceptance test r^2 < (2h)^2 is evaluated in FP64
// with every product rounded separately, so the neighbour set is identical to a
// plain FP64 evaluation on any platform.
//
// EoS pass (Sec. "EoS inverter", online inversion done on the device):
//   0. damped Newton on the quadrilinear table interpolant warm-started from this
//      particle's previous-stage table solution, when there is one in the table;
//   1. otherwise: closed-form EoS solved for T on its upper branch
//      (mu_q = n_q/(chi_q T^2)), bracketed Newton with bisection safeguard;
//   2. if that point lies in the table, damped Newton on the quadrilinear
//      interpolant of (s, n_B, n_S, n_Q), residual scaled by s, 4x4 Jacobian from
//      the same 16-corner stencil, one polishing step after convergence;
//      otherwise (or without convergence) the closed form is kept and flagged;
//   3. p, e = T s + mu.n - p, and (dp/ds, dp/dn_q) = H^-T (s, n) with H the
//      Jacobian d(s, n)/d(T, mu) of the EoS used; c_s^2 above the cap scales
//      them down (flagged).
#include <algorithm>

#include "sph_internal.cuh"
#include "eos_device.cuh"

namespace sphg {

namespace {

// single-precision positions relative to the bounding-box minimum (prefilter input), and
// u0 = sqrt(1 + u.u) (density row 5), one thread per particle
__global__ void k_fpos(EvView v, const double *__restrict__ y, float2 *__restrict__ fpos, double *__restrict__ dens)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= v.n) return;
    double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
    fpos[j] = make_float2(__double2float_rn(__dsub_rn(y[j], xmin0)), __double2float_rn(__dsub_rn(y[v.n + j], xmin1)));
    const size_t N = (size_t)v.n;
    const double ux = y[2 * N + j], uy = y[3 * N + j];
    dens[5 * N + j] = sqrt(fma(ux, ux, fma(uy, uy, 1.0)));
}

constexpr int kWarps = 4;  // warps (particles in flight) per block of the neighbour passes

// Density pass, one warp per particle.  For each of the 3x3 cells the lanes take 32
// candidates at a time through a single-precision prefilter; survivors are compacted
// (ballot) into a per-warp queue and, 32 at a time, go through the exact FP64 test
// r^2 < (2h)^2 and the kernel sum with every lane busy.  Per-lane partial sums are
// combined by a butterfly reduction: the order is fixed, so results are reproducible.
__global__ void __launch_bounds__(32 * kWarps) k_density2(EvView v, const double *__restrict__ y,
                                                          const float2 *__restrict__ fpos,
                                                          const double *__restrict__ Nq,
                                                          const uint32_t *__restrict__ start,
                                                          const uint32_t *__restrict__ cnt,
                                                          double *__restrict__ dens, int *__restrict__ nnb,
                                                          int fallback, int *__restrict__ cnt_dst)
{
    // fallback = 1: the pair-list passes ran first; this pass only runs if one of their lists
    // overflowed (and counts such stages)
    if (fallback) {
        if (!v.sc->pair_flag) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&v.sc->pair_ovf, 1u);
    }
    __shared__ int queue[kWarps][64];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // grid-stride over particles (one warp each): launched at a few blocks per SM when it is
    // only the fallback of the pair-list passes
    for (int a = blockIdx.x * kWarps + wid; a < v.n; a += gridDim.x * kWarps) {  // warp-uniform
        int *q = queue[wid];
        const int n = v.n;
        const double *X = y, *Y = y + n, *S = y + 4 * (size_t)n;
        const double *NB = Nq, *NS = Nq + n, *NQ = Nq + 2 * (size_t)n;
        const double xa = X[a], ya = Y[a];
        const float2 fa = fpos[a];
        const double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
        const int cx = cell_coord(xa, xmin0, v.inv_cell), cy = cell_coord(ya, xmin1, v.inv_cell);
        const int lim = 1 << v.B;
        const unsigned lt = (1u << lane) - 1u;
        double sg = 0.0, ss = 0.0, sb = 0.0, sS = 0.0, sq = 0.0;
        int c = 0, qn = 0;
        // queued index with bit 31 set: the float test left the pair undecided (exact test needed)
        auto pair = [&](int qb) {
            const int b = qb & 0x7FFFFFFF;
            const double dx = xa - X[b], dy = ya - Y[b];
            if (qb < 0 && !(dist2_2d(dx, dy) < v.supp2)) return;
            {
                const double r2 = fma(dx, dx, dy * dy);
                double q = r2 > 0.0 ? r2 * inv_sqrt(r2) * v.inv_h : 0.0;
                double w = kernel_w(q);
                sg += w;
                ss = fma(S[b], w, ss);
                sb = fma(NB[b], w, sb);
                sS = fma(NS[b], w, sS);
                sq = fma(NQ[b], w, sq);
                ++c;
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
            sg += __shfl_xor_sync(0xFFFFFFFFu, sg, o);
            ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
            sb += __shfl_xor_sync(0xFFFFFFFFu, sb, o);
            sS += __shfl_xor_sync(0xFFFFFFFFu, sS, o);
            sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
            c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        }
        if (lane == 0) {
            const double ux = y[2 * (size_t)n + a], uy = y[3 * (size_t)n + a];
            const double sd = v.sigma_d;
            dens[a] = sd * sg;
            dens[(size_t)n + a] = sd * ss;  // lab-frame s*, divided by u0 sqrt(-g) in the EoS pass
            dens[2 * (size_t)n + a] = sd * sb;
            dens[3 * (size_t)n + a] = sd * sS;
            dens[4 * (size_t)n + a] = sd * sq;
            dens[5 * (size_t)n + a] = sqrt(fma(ux, ux, fma(uy, uy, 1.0)));
            nnb[a] = c;
            if (cnt_dst) cnt_dst[a] = c;  // sizes the pair-list rows of the next stage
            atomicAdd(&v.sc->pairs, (unsigned long long)c);
        }
    }
}

// EoS pass, 2+1D, one particle, in two halves around the inversion.
// eos2_load: the rest-frame densities (written back to dens) and the warm start of the Newton
// iteration: this particle's previous-stage table solution; with gprev (an earlier table
// solution, one step before guess_in) both table solutions extrapolate linearly to
// 2 guess_in - gprev (kept if inside the table).  keep receives guess_in as read.
__device__ __forceinline__ void eos2_load(const EvView &v, const EosDev &E, int stage, size_t n, size_t a,
                                          double *__restrict__ dens, const double *__restrict__ guess_in,
                                          const double *__restrict__ gprev, double &s, double nq[3], double gs[4],
                                          double keep[4], const double *__restrict__ y)
{
    const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
    const double sqrtg = v.milne ? tau : 1.0;
    const double vol = dens[5 * n + a] * sqrtg;
    const double ivol = 1.0 / vol;
    s = dens[n + a] * ivol;
#pragma unroll
    for (int q = 0; q < 3; ++q) nq[q] = dens[(2 + q) * n + a] * ivol;
    if (v.diff) {
        // the kernel sums of the lab charges give the lab density sqrt(-g) (n u^0 + J^0): the rest
        // frame n_q = (sum / sqrt(-g) - J^0_q) / u^0 with J^0 = u.J / u^0 and J^i = sigma J^i/sigma
        const double u0 = dens[5 * n + a], sigma = dens[a] * ivol;
        const double ux = y[2 * n + a], uy = y[3 * n + a];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const double J0 = (ux * sigma * y[(kJRow + 2 * q) * n + a] + uy * sigma * y[(kJRow + 2 * q + 1) * n + a]) / u0;
            nq[q] = (dens[(2 + q) * n + a] / sqrtg - J0) / u0;
        }
    }
    dens[n + a] = s;
#pragma unroll
    for (int q = 0; q < 3; ++q) dens[(2 + q) * n + a] = nq[q];
#pragma unroll
    for (int k = 0; k < 4; ++k) keep[k] = gs[k] = guess_in[k * n + a];
    if (gprev && gs[0] > 0.0 && gprev[a] > 0.0) {
        double ge[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ge[k] = 2.0 * gs[k] - gprev[k * n + a];
        if (inside_table(E, ge))
#pragma unroll
            for (int k = 0; k < 4; ++k) gs[k] = ge[k];
    }
}

// eos2_store: the EoS outputs, the next stage's warm start (the table solution, or minus the
// closed-form T; none after the backup EoS or without a solution), and the per-particle inputs
// of the gradient pass: X^{ji} / sigma*^2 with X^{ji} = (p + Pi) delta^{ji} + pi^{ji} -
// v^j pi^{tau i}, and u^j / sigma*.  Returns the particle's longitudinal work rate
// (p + Pi + tau^2 pi^{eta eta}) / sigma*.
__device__ __forceinline__ double eos2_store(const EvView &v, int stage, size_t n, size_t a,
                                             const double *__restrict__ y, const double *__restrict__ dens,
                                             double *__restrict__ eos, double *__restrict__ gin,
                                             uint32_t *__restrict__ status, double *__restrict__ guess_out,
                                             const EosOut &o, bool used)
{
    const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
    const double sqrtg = v.milne ? tau : 1.0;
    const double sig_star = dens[a];
    const double u0 = dens[5 * n + a];
    const double ivol = 1.0 / (u0 * sqrtg), isig = 1.0 / sig_star;
    guess_out[a] = used ? o.T : ((o.st & (PST_NOCONV | PST_NONFINITE | PST_BACKUP)) ? 0.0 : -o.T);
#pragma unroll
    for (int q = 0; q < 3; ++q) guess_out[(1 + q) * n + a] = used ? o.mu[q] : 0.0;
    status[a] = o.st;
    eos[a] = o.T;
    for (int q = 0; q < 3; ++q) eos[(1 + q) * n + a] = o.mu[q];
    eos[4 * n + a] = o.p;
    eos[5 * n + a] = o.e;
    eos[6 * n + a] = o.ps;
    for (int q = 0; q < 3; ++q) eos[(7 + q) * n + a] = o.pn[q];
    eos[10 * n + a] = o.cs2;
    const double ux = y[2 * n + a], uy = y[3 * n + a];
    const double iu0 = ivol * sqrtg;
    const double vx = ux * iu0, vy = uy * iu0;
    const double sigma = sig_star * ivol;
    double Pi = 0.0, pxx = 0.0, pxy = 0.0, pyy = 0.0;
    if (v.tr.viscous) {
        Pi = sigma * y[5 * n + a];
        pxx = sigma * y[6 * n + a];
        pxy = sigma * y[7 * n + a];
        pyy = sigma * y[8 * n + a];
    }
    const double ptx = vx * pxx + vy * pxy;  // pi^{tau x}
    const double pty = vx * pxy + vy * pyy;  // pi^{tau y}
    const double inv2 = isig * isig;
    const double P = o.p + Pi;
    gin[a] = (P + pxx - vx * ptx) * inv2;          // X^{xx}
    gin[n + a] = (pxy - vx * pty) * inv2;          // X^{xy}  (j = x, i = y)
    gin[2 * n + a] = (pxy - vy * ptx) * inv2;      // X^{yx}  (j = y, i = x)
    gin[3 * n + a] = (P + pyy - vy * pty) * inv2;  // X^{yy}
    gin[4 * n + a] = ux * isig;
    gin[5 * n + a] = uy * isig;
    double wcontrib = 0.0;
    if (v.milne) {
        const double ptt = vx * ptx + vy * pty;
        const double t2pee = ptt - pxx - pyy;  // tau^2 pi^{eta eta} from tracelessness
        wcontrib = (P + t2pee) * isig;
    }
    return wcontrib;
}

// Plain and mixed single-event forms: persistent blocks of kEosWarps warps run the lane-refill
// pass (eos_lanes) over the event's particles; the work rate goes to wpart[a] (summed in a fixed
// order by the work kernel), the work counters and the status bits are warp-aggregated.
constexpr int kEosWarps = 4;
#ifndef SPH_EOS_BLOCKS_PER_SM
#define SPH_EOS_BLOCKS_PER_SM 3
#endif
constexpr int kEosBlocksPerSM = SPH_EOS_BLOCKS_PER_SM;  // resident blocks per SM (the register budget)

struct Eos2Ctx {
    const EvView &v;
    int stage;
    size_t n;
    const double *__restrict__ y;
    double *__restrict__ dens, *__restrict__ eos, *__restrict__ gin, *__restrict__ wpart, *__restrict__ guess_out;
    uint32_t *__restrict__ status;
    const double *__restrict__ guess_in;
    unsigned st_or;
    __device__ bool load(int a, double &s, double nq[3], double g[4], double &cap)
    {
        double keep[4];
        cap = v.tr.cs2_cap;
        eos2_load(v, v.eos, stage, n, (size_t)a, dens, guess_in, nullptr, s, nq, g, keep, y);
        return true;
    }
    __device__ void store(int a, const EosOut &o, bool used)
    {
        wpart[a] = eos2_store(v, stage, n, (size_t)a, y, dens, eos, gin, status, guess_out, o, used);
        st_or |= o.st;
    }
};

__global__ void __launch_bounds__(32 * kEosWarps, kEosBlocksPerSM) k_eos2(EvView v, int stage, const double *__restrict__ y,
                                                         double *__restrict__ dens, double *__restrict__ eos,
                                                         double *__restrict__ gin, uint32_t *__restrict__ status,
                                                         double *__restrict__ wpart,
                                                         const double *__restrict__ guess_in,
                                                         double *__restrict__ guess_out)
{
    Eos2Ctx ctx{v, stage, (size_t)v.n, y, dens, eos, gin, wpart, guess_out, status, guess_in, 0u};
    EosWork w = {0u, 0u, 0u};
    eos_lanes(v.eos, &v.sc->eos_claim, v.n, ctx, w);
    const unsigned wres = __reduce_add_sync(0xFFFFFFFFu, w.resid);
    const unsigned wsol = __reduce_add_sync(0xFFFFFFFFu, w.solve);
    const unsigned wg = __reduce_add_sync(0xFFFFFFFFu, w.g);
    const unsigned sor = __reduce_or_sync(0xFFFFFFFFu, ctx.st_or);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&v.sc->eos_resid, (unsigned long long)wres);
        atomicAdd(&v.sc->eos_solve, (unsigned long long)wsol);
        atomicAdd(&v.sc->eos_g, (unsigned long long)wg);
        if (sor) atomicOr(&v.sc->status_or, sor);
    }
}

// Serving form: the same pass over the segmented arena (particles of every event active in this
// stage; padding and inactive slots are skipped).  A lane's particles may belong to different
// events: the per-event work counters and status bits are gathered per block in shared memory
// and flushed once.  Stage 2 starts from the stage-1 solutions of this and the previous step,
// extrapolated to the later time, and keeps this step's for the next.
struct SegEosCtx {
    const Arena &A;
    const BatchTable *T;
    int stage;
    int grp;  // event group (-1: every event)
    size_t P;
    const double *__restrict__ y;
    unsigned int *sh;  // [kMaxSlots][4]: table evaluations, solves, closed-form evaluations, status bits
    EosWork *w;
    EosWork w0;
    int slot;
    double keep[4];
    __device__ bool load(int a, double &s, double nq[3], double g[4], double &cap)
    {
        const int sl = A.segid[a];
        if (sl < 0 || !seg_active(T, sl, stage, false) || !in_group(T, sl, grp)) return false;
        const SegSlot q = T->slots[sl];
        if (a - q.off >= q.n) return false;
        slot = sl;
        w0 = *w;
        cap = A.segv[sl].tr.cs2_cap;
        eos2_load(A.segv[sl], A.segv[sl].eos, stage, P, (size_t)a, A.dens, A.guess_in,
                  stage == 2 ? A.xs1[0] : nullptr, s, nq, g, keep, y);
        return true;
    }
    __device__ void store(int a, const EosOut &o, bool used)
    {
        A.wpart[a] = eos2_store(A.segv[slot], stage, P, (size_t)a, y, A.dens, A.eosf, A.gin, A.status, A.wguess, o,
                                used);
        if (stage == 2)
#pragma unroll
            for (int k = 0; k < 4; ++k) A.xs1[0][k * P + a] = keep[k];
        if (T->slots[slot].mode == SLOT_STEP) {  // float copies of the gradient-pass inputs
            const double *g = A.gin;
            A.fX[a] = make_float4((float)g[a], (float)g[P + a], (float)g[2 * P + a], (float)g[3 * P + a]);
            A.fU[a] = make_float2((float)g[4 * P + a], (float)g[5 * P + a]);
        }
        unsigned int *c = sh + 4 * slot;
        atomicAdd_block(c, w->resid - w0.resid);
        atomicAdd_block(c + 1, w->solve - w0.solve);
        atomicAdd_block(c + 2, w->g - w0.g);
        if (o.st) atomicOr_block(c + 3, o.st);
    }
};

__global__ void __launch_bounds__(32 * kEosWarps, kEosBlocksPerSM) k_eos2_seg(Arena A, EosDev E, int stage, const double *__restrict__ y,
                                                                             int grp)
{
    __shared__ unsigned int sh[kMaxSlots * 4];
    for (int i = threadIdx.x; i < kMaxSlots * 4; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const BatchTable *T = A.tab;
    EosWork w = {0u, 0u, 0u};
    SegEosCtx ctx{A, T, stage, grp, (size_t)A.P, y, sh, &w, w, -1, {0.0, 0.0, 0.0, 0.0}};
    // E is the server's EoS (every event's view carries the same)
    eos_lanes(E, &A.claim[claim_of(CLAIM_EOS, grp)], T->hi, ctx, w);
    __syncthreads();
    const int ns = T->nslots;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        const unsigned int *c = sh + 4 * s;
        if (c[0]) atomicAdd(&A.sc[s].eos_resid, (unsigned long long)c[0]);
        if (c[1]) atomicAdd(&A.sc[s].eos_solve, (unsigned long long)c[1]);
        if (c[2]) atomicAdd(&A.sc[s].eos_g, (unsigned long long)c[2]);
        if (c[3]) atomicOr(&A.sc[s].status_or, c[3]);
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_density(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                    cudaStream_t st)
{
    if (v.dim == 3) {
        launch_density3(v, y, Nq, cb, dens, nnb, st);
        return;
    }
    if (v.mixed) {
        launch_density2m(v, y, Nq, cb, dens, nnb, st);
        return;
    }
    k_fpos<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.fpos, dens);
    const int lists = cb.pl.total > 0;
    if (lists) launch_pairs_density(v, y, Nq, cb, dens, nnb, st);
    // as the fallback of the pair-list passes it usually exits at once: a few blocks per SM
    const int grid = lists ? std::min(nblk(v.n, kWarps), 8 * device_sm_count()) : nblk(v.n, kWarps);
    k_density2<<<grid, 32 * kWarps, 0, st>>>(v, y, cb.fpos, Nq, cb.start, cb.cnt, dens, nnb, lists,
                                             lists ? cb.pl.cnt_dst : nullptr);
}

void launch_eos(const EvView &v, int stage, const double *y, const double *dens, double *eos, double *gin,
                uint32_t *status, double *wpart, const double *guess_in, double *guess_out, cudaStream_t st)
{
    if (v.dim == 3) {
        launch_eos3(v, stage, y, dens, eos, gin, status, wpart, guess_in, guess_out, st);
        return;
    }
    // persistent: resident blocks on every SM; an event with fewer particles than that many lanes
    // takes a whole number of blocks per SM (the lanes claim the rest, so no SM holds a block
    // more than another), or a lane per particle when it is smaller than one block per SM
    const int sms = device_sm_count(), need = nblk(v.n, 32 * kEosWarps);
    const int grid = need >= kEosBlocksPerSM * sms ? kEosBlocksPerSM * sms : (need >= sms ? (need / sms) * sms : std::max(1, need));
    k_eos2<<<grid, 32 * kEosWarps, 0, st>>>(v, stage, y, const_cast<double *>(dens), eos, gin, status, wpart,
                                              guess_in, guess_out);
}

// entries of the work-rate partials: one per particle in 2D (the lane-refill pass), one per
// 64-particle block in 3D
int eos_block_count(int n, int dim) { return dim == 2 ? n : nblk(n, 64); }

int device_sm_count()
{
    static int sms = 0;
    if (sms <= 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms <= 0) {
            cudaGetLastError();
            sms = 152;
        }
    }
    return sms;
}

// Offline inverter: every node (s_i, x_j) of the inverted table solved by the online inversion
// started cold (closed form, then table Newton), as the offline procedure uses the existing
// root finder; NaN where no solution exists
__global__ void k_inverse_build(EosDev E, double *__restrict__ inv, long long nnodes)
{
    const int K = E.inv_K, nx = E.inv_nx;
    const double dxr = 2.0 * E.inv_xmax / (nx - 1);
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < nnodes;
         node += (long long)gridDim.x * blockDim.x) {
        long long r = node;
        const int jQ = (int)(r % nx);
        r /= nx;
        const int jS = (int)(r % nx);
        r /= nx;
        const int jB = (int)(r % nx);
        const long long i = r / nx;
        const double s = E.inv_p10[i / K] * (1.0 + 9.0 * (double)(i % K) / K);
        const double n[3] = {(-E.inv_xmax + jB * dxr) * s, (-E.inv_xmax + jS * dxr) * s, (-E.inv_xmax + jQ * dxr) * s};
        const double g[4] = {0.0, 0.0, 0.0, 0.0};
        bool used = false;
        EosWork w = {0u, 0u, 0u};
        const EosOut o = eos_invert(E, 1.0, s, n, g, used, w);
        const bool ok = !(o.st & PST_NOCONV);
        const double nan = __longlong_as_double(0x7FF8000000000000LL);
        inv[4 * node] = ok ? o.T : nan;
        for (int q = 0; q < 3; ++q) inv[4 * node + 1 + q] = ok ? o.mu[q] : nan;
    }
}

void launch_inverse_build(const EosDev &E, double *inv, long long nnodes, cudaStream_t st)
{
    EosDev online = E;
    online.offline = 0;
    const int grid = (int)std::min<long long>((nnodes + 127) / 128, 152LL * 16);
    k_inverse_build<<<grid, 128, 0, st>>>(online, inv, nnodes);
}

void launch_eos2_seg(const Arena &A, const EosDev &E, int stage, const double *y, int grid, cudaStream_t st, int grp)
{
    k_eos2_seg<<<grid, 32 * kEosWarps, 0, st>>>(A, E, stage, y, grp);
}

int eos_seg_grid(int sms) { return kEosBlocksPerSM * sms; }

}  // namespace sphg
