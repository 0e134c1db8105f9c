// pairs2d.cu -- plain 2D neighbour passes over half-pair lists.
//
// The density sums (Sec. "SPH formalism": sigma*, s*, n*_q as kernel sums) and the gradient sums
// (Sec. "SPH formalism", the n = 0 and n = -1 derivative forms) use W(r_ab) and dW/dr(r_ab) / r_ab
// of every accepted pair; both depend on r_ab only, so they are the same for (a, b) and (b, a).
// Each stage's forward density pass evaluates them once per unordered pair -- on the pairs
// b > a of particle a (sorted index) -- and keeps them with the pair; the backward pass and the
// gradient pass then add every pair's contribution to both of its particles without evaluating
// the kernel again.  All sums run in a fixed order (a warp per particle, lanes over its list in
// ascending neighbour index, then a fixed butterfly), so results are reproducible run to run; they
// differ from the per-particle passes only in the order of the additions.
//
// Per pair the FP64 work of the two passes drops from about 126 operations (two kernel
// evaluations with the sums of each side, in each of the two passes) to about 67.
//
// Rows: a particle's row holds its previous neighbour count plus a margin (a prefix scan per
// stage); forward entries fill it from the start, backward entries from the end.
#include "sph_internal.cuh"

namespace sphg {

namespace {

constexpr int kWarps = 4;  // particles (warps) per block
constexpr unsigned kFull = 0xFFFFFFFFu;

// cells of the 3x3 block around (cx, cy) inside the grid, in ascending Morton key, so that their
// particles come in ascending sorted index
__device__ __forceinline__ int block_cells_ascending(int cx, int cy, int lim, uint32_t keys[9])
{
    int nk = 0;
    for (int oy = -1; oy <= 1; ++oy) {
        const int ny = cy + oy;
        if (ny < 0 || ny >= lim) continue;
        for (int ox = -1; ox <= 1; ++ox) {
            const int nx = cx + ox;
            if (nx < 0 || nx >= lim) continue;
            const uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
            int j = nk++;
            while (j > 0 && keys[j - 1] > k) {
                keys[j] = keys[j - 1];
                --j;
            }
            keys[j] = k;
        }
    }
    return nk;
}

// ---------------------------------------------------------------------------
// Row offsets: row j (sorted order) holds cnt_src[perm[j]] - 1 + margin entries (the previous
// neighbour count without the self pair); off = exclusive prefix sums, off[n] = entries needed.
constexpr int kScanThreads = 256, kScanPer = 8, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ long long row_size(const PairBufs &pl, const uint32_t *perm, int j)
{
    const int c = pl.cnt_src[perm[j]];
    return (long long)(c > 1 ? c - 1 : 0) + pl.margin;
}

__global__ void __launch_bounds__(kScanThreads) k_rows_part(int n, const uint32_t *__restrict__ perm, PairBufs pl)
{
    __shared__ long long ws[kScanThreads / 32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    long long t = 0;
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) t += row_size(pl, perm, base + k);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long b = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) b += ws[w];
        pl.part[blockIdx.x] = (unsigned long long)b;
    }
}

// exclusive scan of the block sums (one block); off[n] = total; rows beyond the allocation flag
// the stage (the per-particle passes run)
__global__ void __launch_bounds__(1024) k_rows_top(int n, int nparts, PairBufs pl, DevScalars *sc)
{
    __shared__ unsigned long long tot[1024];
    const int t = threadIdx.x, per = (nparts + 1023) / 1024;
    const int b0 = min(t * per, nparts), b1 = min(b0 + per, nparts);
    unsigned long long s = 0;
    for (int i = b0; i < b1; ++i) s += pl.part[i];
    tot[t] = s;
    __syncthreads();
    if (t == 0) {
        unsigned long long run = 0;
        for (int k = 0; k < 1024; ++k) {
            const unsigned long long x = tot[k];
            tot[k] = run;
            run += x;
        }
        pl.off[n] = (long long)run;
        if ((long long)run > pl.total) atomicOr(&sc->pair_flag, 1u);
    }
    __syncthreads();
    unsigned long long run = tot[t];
    for (int i = b0; i < b1; ++i) {
        const unsigned long long x = pl.part[i];
        pl.part[i] = run;
        run += x;
    }
}

__global__ void __launch_bounds__(kScanThreads) k_rows_apply(int n, const uint32_t *__restrict__ perm, PairBufs pl)
{
    __shared__ long long ws[kScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    long long v[kScanPer], t = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = base + k < n ? row_size(pl, perm, base + k) : 0;
        t += v[k];
    }
    long long incl = t;  // inclusive scan over the warp
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    long long wbase = 0;
    for (int w = 0; w < wid; ++w) wbase += ws[w];
    long long run = (long long)pl.part[blockIdx.x] + wbase + incl - t;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) pl.off[base + k] = run;
        run += v[k];
    }
}

// Forward density pass, one warp per particle a.  Candidates of the 3x3 cells pass the
// single-precision prefilter; a neighbour b < a is decided at once (exact FP64 test when the
// float test left it undecided) and listed in B; a candidate b > a is queued, and 32 at a time
// the exact test, W and dW/dr / r run on full warps, are listed (L, W, G) and summed for a.
// dpart receives a's unscaled partial sums (self pair and pairs b > a): sigma*, S, N_B, N_S, N_Q.
__global__ void __launch_bounds__(32 * kWarps) k_pairs_density_fwd(EvView v, const double *__restrict__ y,
                                                                   const float2 *__restrict__ fpos,
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
    const int n = v.n;
    const double *X = y, *Y = y + n, *S = y + 4 * (size_t)n;
    const double *NB = Nq, *NS = Nq + n, *NQ = Nq + 2 * (size_t)n;
    const double xa = X[a], ya = Y[a];
    const float2 fa = fpos[a];
    const double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
    const int cx = cell_coord(xa, xmin0, v.inv_cell), cy = cell_coord(ya, xmin1, v.inv_cell);
    uint32_t keys[9];
    const int nk = block_cells_ascending(cx, cy, 1 << v.B, keys);
    const unsigned lt = (1u << lane) - 1u;
    const long long r0 = pl.off[a], r1 = pl.off[a + 1];
    // rows beyond the allocation write nothing (the scan has flagged the stage)
    const int cap = r1 <= pl.total ? (int)(r1 - r0) : 0;
    int *F = pl.L + r0, *Bl = pl.L + (r1 - 1);  // forward up from the start, backward down from the end
    double *Wr = pl.W + r0;
    double2 *Gr = pl.G + r0;
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
    // queued index with bit 31 set: the float test left the pair undecided (exact test needed)
    auto forward = [&](int qb, bool valid) {
        const int b = qb & 0x7FFFFFFF;
        double dx = 0.0, dy = 0.0;
        bool acc = false;
        if (valid) {
            dx = xa - X[b];
            dy = ya - Y[b];
            acc = qb >= 0 || dist2_2d(dx, dy) < v.supp2;
        }
        const unsigned m = __ballot_sync(kFull, acc);
        if (acc) {
            const double r2 = fma(dx, dx, dy * dy);
            double w = kernel_w(0.0), fac = 0.0;  // coincident particles: W(0), no gradient
            if (nonzero_nonneg(r2)) {
                // the cubic spline without a branch on q: w = (2-q)^3/4 - max(1-q, 0)^3,
                // w' = -3/4 (2-q)^2 + 3 max(1-q, 0)^2 (the same polynomials on both pieces)
                // (the sign tests and the factor 1/4 on the integer pipe: t^2 is 0 or >= 2^-104)
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
                Gr[slot] = make_double2(fac * dx, fac * dy);
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
                const float2 fb = fpos[b];
                const float dx = fa.x - fb.x, dy = fa.y - fb.y;
                const float r2f = fmaf(dx, dx, dy * dy);
                cand = r2f <= v.supp2_hi;
                sure = r2f < v.supp2_lo;
            }
            // b < a: decided here and listed; its pair values come from b's own forward pass
            bool accB = false;
            if (cand && (int)b < a) accB = sure || dist2_2d(xa - X[b], ya - Y[b]) < v.supp2;
            const unsigned mb = __ballot_sync(kFull, accB);
            if (accB) {
                const int slot = nbk + __popc(mb & lt);
                if (slot < cap) Bl[-slot] = (int)b;
            }
            nbk += __popc(mb);
            // b > a: queued in arrival (ascending) order for the FP64 pair arithmetic
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
    const int k = lane >> 2;
    if ((lane & 3) == 0 && k < 5) dpart[(size_t)k * n + a] = tot;
    if (lane == 0) {
        pl.cntF[a] = nf;
        pl.cntB[a] = nbk;
        if (nf + nbk > cap) atomicOr(&v.sc->pair_flag, 1u);  // the two ends met: lists unusable
    }
}

// Backward density pass, one warp per particle a: the pairs (b, a) with b < a, whose W the
// forward pass of b stored; the slot is found by binary search of a in b's ascending list and
// kept in P for the gradient pass.  Completes a's sums (forward partial + backward partial) and
// writes the density rows as the per-particle pass does.
__global__ void __launch_bounds__(32 * kWarps) k_pairs_density_bwd(EvView v, const double *__restrict__ y,
                                                                   const double *__restrict__ Nq, PairBufs pl,
                                                                   double *__restrict__ dens, int *__restrict__ nnb)
{
    if (v.sc->pair_flag) return;  // a list overflowed: the per-particle pass runs instead
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarps + wid;
    if (a >= v.n) return;  // warp-uniform
    const int n = v.n;
    const double *S = y + 4 * (size_t)n;
    const double *NB = Nq, *NS = Nq + n, *NQ = Nq + 2 * (size_t)n;
    const long long rend = pl.off[a + 1] - 1;  // backward entries: rend, rend - 1, ...
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
            // both sides take the same acceptance decision (the float and the exact test see
            // exactly negated differences), so a is in b's list; checked all the same
            if (lo >= nfb || Fb[lo] != a) {
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
        // rows sigma*, lab-frame s* (divided by u0 sqrt(-g) in the EoS pass), n*_B, n*_S, n*_Q:
        // the forward partials were left in the density rows; u0 (row 5) is written by k_fpos
        double *d = dens + (size_t)k * n + a;
        *d = v.sigma_d * (*d + tot);
    }
    if (lane == 0) {
        const int c = 1 + pl.cntF[a] + nb;
        nnb[a] = c;
        if (pl.cnt_dst) pl.cnt_dst[a] = c;  // sizes this particle's row in the next stage
        atomicAdd(&v.sc->pairs, (unsigned long long)c);
    }
}

// Gradient pass, one warp per particle a, over its pairs b > a (forward entries of a's row, with
// G = grad_a W_ab h / sigma_d) and then b < a (backward entries: -G of the pair in b's row, slot
// P), forming the sums of the per-particle pass: sum grad W, sum X_b grad W, sum u_b grad W.
__global__ void __launch_bounds__(32 * kWarps) k_pairs_gradient(EvView v, int stage, const double *__restrict__ y,
                                                                const double *__restrict__ gin, PairBufs pl,
                                                                double *__restrict__ gout)
{
    if (v.sc->pair_flag) return;  // a list overflowed: the per-particle pass runs instead
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int a = blockIdx.x * kWarps + wid;
    if (a >= v.n) return;  // warp-uniform
    const int n = v.n;
    const double *Xxx = gin, *Xxy = gin + n, *Xyx = gin + 2 * (size_t)n, *Xyy = gin + 3 * (size_t)n;
    const double *Ux = gin + 4 * (size_t)n, *Uy = gin + 5 * (size_t)n;
    const long long r0 = pl.off[a], rend = pl.off[a + 1] - 1;
    const int nf = pl.cntF[a], nt = nf + pl.cntB[a];
    double Gx = 0.0, Gy = 0.0, Hx = 0.0, Hy = 0.0;
    double dxux = 0.0, dxuy = 0.0, dyux = 0.0, dyuy = 0.0;
    for (int j0 = 0; j0 < nt; j0 += 32) {
        const int j = j0 + lane;
        if (j < nt) {
            int b;
            double gx, gy;
            if (j < nf) {
                b = pl.L[r0 + j];
                const double2 g = pl.G[r0 + j];
                gx = g.x;
                gy = g.y;
            } else {  // grad_a W_ab = -grad_b W_ba, stored with b's forward pair
                b = pl.L[rend - (j - nf)];
                const double2 g = pl.G[pl.off[b] + pl.P[rend - (j - nf)]];
                gx = -g.x;
                gy = -g.y;
            }
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
    }
    const double vals[8] = {Gx, Gy, Hx, Hy, dxux, dxuy, dyux, dyuy};
    const double tot = warp_reduce_scatter8(vals, lane);
    // totals: lanes 0, 4: sum grad W (x, y); 8, 12: sum X_b grad W (x, y); 16..28: sum u_b grad W
    const double Sx = __shfl_sync(kFull, tot, 0), Sy = __shfl_sync(kFull, tot, 4);
    const int k = lane >> 2;
    if ((lane & 3) == 0 && k >= 2) {
        const double c = v.sigma_d * v.inv_h;
        if (k >= 4) {
            gout[(size_t)(k - 4) * n + a] = c * tot;  // d_x u^x, d_x u^y, d_y u^x, d_y u^y
        } else {
            // minus the stress divergence: X_a . sum grad W + sum X_b grad W, times sqrt(-g)
            const double tau = v.sc->tau + (stage == 2 ? v.dtau : 0.0);
            const double sqrtg = v.milne ? tau : 1.0;
            const double X0 = k == 2 ? Xxx[a] : Xxy[a], X1 = k == 2 ? Xyx[a] : Xyy[a];
            gout[(size_t)(k + 2) * n + a] = -sqrtg * c * (X0 * Sx + X1 * Sy + tot);
        }
    }
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_pair_rows(const EvView &v, CellBufs cb, cudaStream_t st)
{
    const int nparts = (v.n + kScanTile - 1) / kScanTile;
    k_rows_part<<<nparts, kScanThreads, 0, st>>>(v.n, cb.perm, cb.pl);
    k_rows_top<<<1, 1024, 0, st>>>(v.n, nparts, cb.pl, v.sc);
    k_rows_apply<<<nparts, kScanThreads, 0, st>>>(v.n, cb.perm, cb.pl);
}

void launch_pairs_density(const EvView &v, const double *y, const double *Nq, CellBufs cb, double *dens, int *nnb,
                          cudaStream_t st)
{
    launch_pair_rows(v, cb, st);
    // the forward partials go to the density rows, which the backward pass completes in place
    k_pairs_density_fwd<<<nblk(v.n, kWarps), 32 * kWarps, 0, st>>>(v, y, cb.fpos, Nq, cb.start, cb.cnt, cb.pl,
                                                                   dens);
    k_pairs_density_bwd<<<nblk(v.n, kWarps), 32 * kWarps, 0, st>>>(v, y, Nq, cb.pl, dens, nnb);
}

void launch_pairs_gradient(const EvView &v, int stage, const double *y, const double *gin, CellBufs cb,
                           double *gout, cudaStream_t st)
{
    k_pairs_gradient<<<nblk(v.n, kWarps), 32 * kWarps, 0, st>>>(v, stage, y, gin, cb.pl, gout);
}

}  // namespace sphg
