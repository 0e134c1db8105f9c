// serve.cu -- the serving form: continuous batching of 2+1D events in one segmented
// particle arena, neighbour passes in single precision (the mixed form), EoS inversion,
// equations of motion and reductions in double precision.
//
// Device side.  Every per-particle row of the arena has stride P (the capacity).  An
// admitted event owns [off, off + cap) of every row (off, cap multiples of 256); its
// particles sit in [off, off + n) in (cell, id) order after each stage's sort.  Per slot
// the device holds the event's parameters (EvView), its evolving scalars (DevScalars:
// tau, work integral, counters) and, per stage, its bounding box and cell grid (SegGrid).
// One batch step = two Heun stages over all admitted events:
//   bbox -> grid -> count -> scan -> scatter -> rank -> permute -> density (tiled, FP32)
//   -> EoS (FP64) -> gradient (tiled, FP32) -> equations of motion (FP64) -> work integral
// with the same buffer rotation as a single event (stage 1: A -> B, C = B + dt f(B);
// stage 2: C -> D, B -> A, A = ((A + D) + dt f(D)) / 2).  The kernels read the slot table
// from device memory and loop over the arena (or its cells) with a fixed grid, so the
// whole step is captured once as a CUDA graph and replayed for every composition.
//
// The neighbour passes are cell-tiled over cells of side h: one block per cell stages the
// particles of the 5x5 neighbouring cells (five contiguous runs of the sorted arena, one per
// cell row; every pair closer than 2h lies in it) in shared memory as positions relative to
// the centre cell's origin, and every particle of the cell scans them with L lanes (by the
// cell's occupancy, up to 16).  A proven
// bound on the float r^2 decides all but a thin shell of candidates; inside the shell the
// FP64 test r^2 < (2h)^2 with separately rounded products decides, so the neighbour sets
// are exactly those of the FP64 form.  A lane evaluates two candidates per packed two-wide
// FP32 instruction.  Sums are Neumaier-compensated per lane and combined across a particle's
// lanes with error-free FP32 additions in a fixed order: an event's results do not depend on
// what else is in the batch or where its range lies.
//
// Host side.  sph_submit copies an event into pinned staging and queues it; each
// sph_server_pump step admits queued events while a slot and an arena range are free
// (the arena is carved from free HBM at creation), replays the step graph, and retires
// events that finished their steps: a finished event takes one more stage-1 evaluation
// (observe mode: cells, densities, EoS at the final state), then its fields are scattered
// to the original order and copied to its pinned block; a CUDA event marks them readable.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sph_gb300.h"
#include "sph_internal.cuh"
#include "tiled_common.cuh"

using namespace sphg;

namespace {

constexpr int kScanBlocks = 256;
constexpr int kTTDefault = 128;  // threads of a tiled neighbour block (the autotuner may pick another)
constexpr int kTile = 640;  // candidates staged in shared memory at a time (a 5x5 block of ~23-particle cells)
constexpr int kRows = 5;    // cell rows (and columns) of the search block: cells of side h, pairs closer than 2h
__device__ __forceinline__ double inf_d() { return __longlong_as_double(0x7FF0000000000000LL); }

// ---------------------------------------------------------------------------
// cell list of every active event (rows a1, a2)
__global__ void k_seg_reset(Arena A)
{
    const int ns = A.tab->nslots;
    for (int s = threadIdx.x; s < ns; s += blockDim.x) {
        SegGrid &g = A.grid[s];
        g.bb[0] = g.bb[1] = enc_double(inf_d());
        g.bb[2] = g.bb[3] = enc_double(-inf_d());
    }
}

// bounding box per event: warp-reduced, one atomic per warp (a warp lies in one range)
__global__ void k_seg_bbox(Arena A, int stage, const double *__restrict__ y)
{
    const BatchTable *T = A.tab;
    const int hi = T->hi;
    const size_t P = (size_t)A.P;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < hi; a += gridDim.x * blockDim.x) {
        const int s = A.segid[a];
        if (s < 0 || !seg_active(T, s, stage, false)) continue;
        const bool v = a - T->slots[s].off < T->slots[s].n;
        double mnx = v ? y[a] : inf_d(), mny = v ? y[P + a] : inf_d();
        double mxx = v ? y[a] : -inf_d(), mxy = v ? y[P + a] : -inf_d();
        for (int o = 16; o > 0; o >>= 1) {
            mnx = fmin(mnx, __shfl_xor_sync(0xFFFFFFFFu, mnx, o));
            mny = fmin(mny, __shfl_xor_sync(0xFFFFFFFFu, mny, o));
            mxx = fmax(mxx, __shfl_xor_sync(0xFFFFFFFFu, mxx, o));
            mxy = fmax(mxy, __shfl_xor_sync(0xFFFFFFFFu, mxy, o));
        }
        if ((threadIdx.x & 31) == 0 && mnx <= mxx && mny <= mxy) {
            atomicMin(&A.grid[s].bb[0], enc_double(mnx));
            atomicMin(&A.grid[s].bb[1], enc_double(mny));
            atomicMax(&A.grid[s].bb[2], enc_double(mxx));
            atomicMax(&A.grid[s].bb[3], enc_double(mxy));
        }
    }
}

// number of cells of side h from the minimum to v, clamped to [1, kMaxCellsAxis]
__device__ __forceinline__ int cells_to(double v, double v0, double inv_cell)
{
    if (!(v >= v0)) return 1;
    const double f = floor(__dmul_rn(__dsub_rn(v, v0), inv_cell));
    return f >= (double)(kMaxCellsAxis - 1) ? kMaxCellsAxis : (int)f + 1;
}

// cell grid per event and the offset of its cells in the shared bucket table
__global__ void __launch_bounds__(kMaxSlots) k_seg_grid(Arena A, int stage)
{
    __shared__ int sh[kMaxSlots];
    const BatchTable *T = A.tab;
    const int s = threadIdx.x;
    int nc = 0;
    if (s < T->nslots && seg_active(T, s, stage, false)) {
        SegGrid &g = A.grid[s];
        const double ic = A.segv[s].inv_h;  // cells of side h
        const double x0 = dec_double(g.bb[0]), y0 = dec_double(g.bb[1]);
        const int nx = cells_to(dec_double(g.bb[2]), x0, ic), ny = cells_to(dec_double(g.bb[3]), y0, ic);
        g.x0 = x0;
        g.y0 = y0;
        g.nx = nx;
        g.ny = ny;
        nc = nx * ny;
    }
    sh[s] = nc;
    __syncthreads();
    for (int o = 1; o < kMaxSlots; o <<= 1) {  // inclusive Hillis-Steele scan
        int v = s >= o ? sh[s - o] : 0;
        __syncthreads();
        sh[s] += v;
        __syncthreads();
    }
    if (s < T->nslots) {
        A.grid[s].base = sh[s] - nc;
        A.grid[s].ncell = nc;
        if (s == T->split) A.ncells[1] = sh[s] - nc;  // group 1's cells start at its first slot's
    }
    if (s == kMaxSlots - 1) {
        A.ncells[0] = sh[s];
        if (T->split >= T->nslots) A.ncells[1] = sh[s];  // group 1 is empty
    }
    if (s < kClaims) A.claim[s] = 0u;
}

__global__ void k_seg_zero(Arena A)
{
    const int nc = *A.ncells;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) A.cnt[c] = 0u;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__global__ void k_seg_keys(Arena A, int stage, const double *__restrict__ y)
{
    const BatchTable *T = A.tab;
    const int hi = T->hi;
    const size_t P = (size_t)A.P;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < hi; a += gridDim.x * blockDim.x) {
        const int s = A.segid[a];
        if (s < 0 || !seg_active(T, s, stage, false) || a - T->slots[s].off >= T->slots[s].n) continue;
        const SegGrid &g = A.grid[s];
        const double ic = A.segv[s].inv_h;
        const int cx = clampi(cell_coord(y[a], g.x0, ic), 0, g.nx - 1);
        const int cy = clampi(cell_coord(y[P + a], g.y0, ic), 0, g.ny - 1);
        const uint32_t k = (uint32_t)(g.base + cy * g.nx + cx);
        A.key[a] = k;
        A.rnk[a] = atomicAdd(&A.cnt[k], 1u);
    }
}

// exclusive scan of the bucket counts (device-sized: the total is read on the device)
__device__ __forceinline__ uint32_t block_sum_256(uint32_t v, uint32_t *sh)
{
    v = __reduce_add_sync(0xFFFFFFFFu, v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += sh[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(256) k_seg_scan_part(Arena A)
{
    __shared__ uint32_t sh[8];
    const int nc = *A.ncells;
    const int chunk = (nc + kScanBlocks - 1) / kScanBlocks;
    const int lo = blockIdx.x * chunk, hi = min(nc, lo + chunk);
    uint32_t acc = 0u;
    for (int i = lo + threadIdx.x; i < hi; i += 256) acc += A.cnt[i];
    const uint32_t t = block_sum_256(acc, sh);
    if (threadIdx.x == 0) A.scan_part[blockIdx.x] = t;
}

// exclusive scan of 256 values held one per thread; returns this thread's prefix, *total the sum
__device__ __forceinline__ uint32_t block_exscan_256(uint32_t v, uint32_t *sh, uint32_t *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    uint32_t wp = 0, tot = 0;
    for (int k = 0; k < 8; ++k) {
        if (k < w) wp += sh[k];
        tot += sh[k];
    }
    __syncthreads();
    *total = tot;
    return wp + x - v;
}

__global__ void __launch_bounds__(256) k_seg_scan_top(Arena A)
{
    __shared__ uint32_t sh[8];
    uint32_t tot;
    const uint32_t v = A.scan_part[threadIdx.x];
    const uint32_t ex = block_exscan_256(v, sh, &tot);
    A.scan_part[threadIdx.x] = ex;
}

__global__ void __launch_bounds__(256) k_seg_scan_apply(Arena A)
{
    __shared__ uint32_t sh[8];
    const int nc = *A.ncells;
    const int chunk = (nc + kScanBlocks - 1) / kScanBlocks;
    const int lo = blockIdx.x * chunk, hi = min(nc, lo + chunk);
    uint32_t carry = A.scan_part[blockIdx.x];
    for (int t0 = lo; t0 < hi; t0 += 256) {
        const int i = t0 + threadIdx.x;
        const uint32_t v = i < hi ? A.cnt[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exscan_256(v, sh, &tot);
        if (i < hi) A.start[i] = carry + ex;
        carry += tot;
    }
}

// bucket slot of every particle, then the deterministic order inside a cell: rank by id
__global__ void k_seg_scatter(Arena A, int stage)
{
    const BatchTable *T = A.tab;
    const int hi = T->hi;
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < hi; a += gridDim.x * blockDim.x) {
        const int s = A.segid[a];
        if (s < 0 || !seg_active(T, s, stage, false)) continue;
        const SegSlot sl = T->slots[s];
        if (a - sl.off >= sl.n) continue;
        const uint32_t k = A.key[a];
        const int j = sl.off + (int)(A.start[k] - A.start[A.grid[s].base]) + (int)A.rnk[a];
        A.tmp[j] = (uint32_t)a;
    }
}

__global__ void k_seg_rank(Arena A, int stage, const int *__restrict__ id)
{
    const BatchTable *T = A.tab;
    const int hi = T->hi;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < hi; j += gridDim.x * blockDim.x) {
        const int s = A.segid[j];
        if (s < 0 || !seg_active(T, s, stage, false)) continue;
        const SegSlot sl = T->slots[s];
        if (j - sl.off >= sl.n) continue;
        const uint32_t p = A.tmp[j];
        const uint32_t k = A.key[p];
        const int c0 = sl.off + (int)(A.start[k] - A.start[A.grid[s].base]);
        const int c1 = c0 + (int)A.cnt[k];
        const int my = id[p];
        int r = 0;
        for (int m = c0; m < c1; ++m) r += id[A.tmp[m]] < my;
        A.perm[c0 + r] = p;
    }
}

struct SegPerm {
    const double *src[6];
    double *dst[6];
    int rows[6];
    int ng;
    const int *id_in;
    int *id_out;
    const double *nq;  // the charges' source rows (group 0 holds the positions and S)
};

// Gathers the state into sorted order and writes the single-precision copies of the
// neighbour passes: position relative to the origin of the particle's cell (the same FP64
// expression as the centre-cell origin of the tiled passes) and (S, N_B, N_S, N_Q).
__global__ void k_seg_permute(Arena A, int stage, SegPerm pa)
{
    const BatchTable *T = A.tab;
    const int hi = T->hi;
    const size_t P = (size_t)A.P;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < hi; j += gridDim.x * blockDim.x) {
        const int s = A.segid[j];
        if (s < 0 || !seg_active(T, s, stage, false) || j - T->slots[s].off >= T->slots[s].n) continue;
        const size_t p = A.perm[j];
        for (int g = 0; g < pa.ng; ++g)
            for (int r = 0; r < pa.rows[g]; ++r) pa.dst[g][r * P + j] = pa.src[g][r * P + p];
        pa.id_out[j] = pa.id_in[p];
        const SegGrid &g = A.grid[s];
        const int lc = (int)A.key[p] - g.base;
        const int cx = lc % g.nx, cy = lc / g.nx;
        const double cs = A.segv[s].h;
        const double *X = pa.src[0];
        A.fpos[j] = make_float2((float)(X[p] - (g.x0 + (double)cx * cs)), (float)(X[P + p] - (g.y0 + (double)cy * cs)));
        A.fq[j] = make_float4((float)X[4 * P + p], (float)pa.nq[p], (float)pa.nq[P + p], (float)pa.nq[2 * P + p]);
    }
}

// ---------------------------------------------------------------------------
// cell-tiled neighbour passes (rows a3, a5)
struct CellCtx {
    int s, first, na, M, clamped;
    int rs[kRows];       // the candidate run of each cell row: its first arena position
    int cum[kRows + 1];  // candidates of the rows before: row o holds candidates [cum[o], cum[o + 1])
    int bnd[kRows][4];   // arena positions where the row's columns cx-1, cx, cx+1, cx+2 begin
    float cs;            // cell side h in single precision
};

// last slot whose first cell is <= c (slots without cells share the next slot's base)
__device__ __forceinline__ int find_slot(const int *base, int ns, int c)
{
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base[mid] <= c) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The context of cell c, built by one warp: every lane reads the cell's scalars (broadcast
// loads), lanes 0..4 the bounds of one cell row each; the row lengths are scanned across lanes.
// Rows and columns outside the grid are empty runs.
__device__ void cell_setup(const Arena &A, const int *s_base, int ns, int c, CellCtx &cc, int lane)
{
    const int s = find_slot(s_base, ns, c);
    const SegGrid &g = A.grid[s];
    const int nx = g.nx, ny = g.ny, base = g.base;
    const int off = A.tab->slots[s].off;
    const uint32_t S0 = A.start[base];
    const int lc = c - base, cx = lc % nx, cy = lc / nx;
    const int r = cy - 2 + lane;
    int st = 0, ln = 0, e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    if (lane < kRows && r >= 0 && r < ny) {
        const int row = base + r * nx;
        const int cl = max(cx - 2, 0), cr = min(cx + 2, nx - 1);
        st = off + (int)(A.start[row + cl] - S0);
        const int en = off + (int)(A.start[row + cr] + A.cnt[row + cr] - S0);
        ln = en - st;
        // start of column col of the row; before the grid: the run's start, past it: its end
        auto col0 = [&](int col) { return col < 0 ? st : (col >= nx ? en : off + (int)(A.start[row + col] - S0)); };
        e0 = col0(cx - 1);
        e1 = col0(cx);
        e2 = col0(cx + 1);
        e3 = col0(cx + 2);
    }
    int inc = ln;  // inclusive scan of the row lengths over lanes 0..4
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane < kRows) {
        cc.rs[lane] = st;
        cc.cum[lane + 1] = inc;
        cc.bnd[lane][0] = e0;
        cc.bnd[lane][1] = e1;
        cc.bnd[lane][2] = e2;
        cc.bnd[lane][3] = e3;
    }
    const int M = __shfl_sync(0xFFFFFFFFu, inc, kRows - 1);
    if (lane == 0) {
        cc.cum[0] = 0;
        cc.s = s;
        cc.clamped = nx >= kMaxCellsAxis || ny >= kMaxCellsAxis;
        cc.first = off + (int)(A.start[c] - S0);
        cc.na = (int)A.cnt[c];
        cc.cs = (float)A.segv[s].h;
        cc.M = M;
    }
}

// arena position of candidate q of the 5x5 block
__device__ __forceinline__ int cand_arena(const CellCtx &cc, int q)
{
    int o = 0;
#pragma unroll
    for (int k = 1; k < kRows; ++k) o += q >= cc.cum[k];
    return cc.rs[o] + (q - cc.cum[o]);
}

// candidate q of the 5x5 block: its arena position and its position relative to the
// centre cell's origin (own-cell-relative float position + the cell offset, an exact
// multiple of the float cell side)
__device__ __forceinline__ int cand_index(const CellCtx &cc, int q, const float2 *__restrict__ fpos, float2 &rel)
{
    int o = 0;
#pragma unroll
    for (int k = 1; k < kRows; ++k) o += q >= cc.cum[k];
    const int b = cc.rs[o] + (q - cc.cum[o]);
    const int dc = (b >= cc.bnd[o][0]) + (b >= cc.bnd[o][1]) + (b >= cc.bnd[o][2]) + (b >= cc.bnd[o][3]) - 2;
    const float2 f = fpos[b];
    rel = make_float2(f.x + (float)dc * cc.cs, f.y + (float)(o - 2) * cc.cs);
    return b;
}

// lane splits of the tuned shape (warps sharing a cell's particles, lanes_per_particle)
constexpr int kLaneWarpsDefault = 4;
constexpr int kLaneWarpChoices[] = {2, 4, 8};

// Inner loops of the tiled passes: every candidate of a lane's run is evaluated without
// branches (the accept decision zeroes its terms; adding +0 is exact), since the lanes of a
// warp accept different candidates and a branch would cost the same issue slots.  Only the
// thin shell takes a branch, to the exact FP64 test.
template <int TT>
__global__ void __launch_bounds__(TT) k_seg_density(Arena A, const double *__restrict__ y,
                                                     const double *__restrict__ Nq, int grp)
{
    __shared__ int s_base[kMaxSlots];
    __shared__ float4 cP[kTile / 2];   // (-x_0, -x_1, -y_0, -y_1) relative to the centre cell
    __shared__ float4 cQa[kTile / 2];  // (S_0, S_1, N_B0, N_B1)
    __shared__ float4 cQb[kTile / 2];  // (N_S0, N_S1, N_Q0, N_Q1)
    __shared__ CellCtx cc;
    __shared__ int s_cell, s_cur;
    __shared__ unsigned long long s_acc[2];  // pairs and shell tests of slot s_cur, flushed when it changes
    const BatchTable *T = A.tab;
    const int ns = T->nslots;
    for (int i = threadIdx.x; i < ns; i += TT) s_base[i] = A.grid[i].base;
    if (threadIdx.x == 0) {
        s_cur = -1;
        s_acc[0] = s_acc[1] = 0ull;
    }
    // the cells of the event group (grp < 0: all): group 0's come first
    const int c_lo = grp > 0 ? A.ncells[1] : 0, c_hi = grp == 0 ? A.ncells[1] : A.ncells[0];
    const size_t P = (size_t)A.P;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = TT / 32;
    for (;;) {
        __syncthreads();  // the previous cell's context and tile are no longer read
        if (warp == 0) {
            int c = lane == 0 ? c_lo + (int)atomicAdd(&A.claim[claim_of(CLAIM_DENSITY, grp)], 1u) : 0;
            c = __shfl_sync(0xFFFFFFFFu, c, 0);
            if (lane == 0) s_cell = c;
            if (c < c_hi && A.cnt[c] > 0u) cell_setup(A, s_base, ns, c, cc, lane);
            else if (lane == 0) cc.na = 0;
            const int snew = c < c_hi ? (cc.na > 0 ? cc.s : s_cur) : -1;
            if (lane == 0 && snew != s_cur) {
                if (s_cur >= 0) {
                    if (s_acc[0]) atomicAdd(&A.sc[s_cur].pairs, s_acc[0]);
                    if (s_acc[1]) atomicAdd(&A.sc[s_cur].shell_tests, s_acc[1]);
                }
                s_acc[0] = s_acc[1] = 0ull;
                s_cur = snew;
            }
        }
        __syncthreads();
        if (s_cell >= c_hi) break;
        const int na = cc.na;
        if (na == 0) continue;
        const EvView &V = A.segv[cc.s];
        const float ih = (float)V.inv_h;
        const float slo = cc.clamped ? -1.0f : V.shell_lo, shi = cc.clamped ? 3.0e38f : V.shell_hi;
        const double supp2 = V.supp2, sd = V.sigma_d;
        const int L = lanes_per_particle(na, A.lane_warps), ppw = 32 / L;
        const int pl = lane / L, l = lane - pl * L;
        const int M = cc.M;
        unsigned pairs = 0u, shell = 0u;
        for (int g0 = 0; g0 < na; g0 += NW * ppw) {
            const int my = g0 + warp * ppw + pl;
            const bool valid = pl < ppw && my < na;
            const int a = cc.first + (valid ? my : 0);
            const double xa = y[a], ya = y[P + a];
            const float2 fa = A.fpos[a];
            CSum sg = {0.f, 0.f}, ss = {0.f, 0.f}, sb = {0.f, 0.f}, sS = {0.f, 0.f}, sq = {0.f, 0.f};
            int nacc = 0;
            for (int t0 = 0; t0 < M; t0 += kTile) {
                const int mt = min(kTile, M - t0);
                if (g0 == 0 || M > kTile) {  // one tile serves every pass of the cell
                    if (t0 > 0 || g0 > 0) __syncthreads();
                    for (int i = tid; i < mt; i += TT) {
                        float2 rel;
                        const int b = cand_index(cc, t0 + i, A.fpos, rel);
                        put_pair(cP, i, -rel.x, -rel.y);
                        const float4 q = A.fq[b];
                        put_pair(cQa, i, q.x, q.y);
                        put_pair(cQb, i, q.z, q.w);
                    }
                    if ((mt & 1) && tid == 0) {
                        put_pair(cP, mt, kFar, kFar);
                        put_pair(cQa, mt, 0.0f, 0.0f);
                        put_pair(cQb, mt, 0.0f, 0.0f);
                    }
                    __syncthreads();
                }
                if (valid) {
                    // runs of kRun candidates (kRun / 2 pairs) summed in plain FP32, each half of a
                    // packed sum over kRun / 2 terms, each run folded into the compensated sums
                    const float2 fx = make_float2(fa.x, fa.x), fy = make_float2(fa.y, fa.y), ih2 = make_float2(ih, ih);
                    const int np = (mt + 1) >> 1;
                    for (int kb = l; kb < np; kb += (kRun / 2) * L) {
                        const int ke = min(np, kb + (kRun / 2) * L);
                        float2 pg = make_float2(0.f, 0.f), ps = pg, pB = pg, pS = pg, pQ = pg;
#pragma unroll 2
                        for (int k = kb; k < ke; k += L) {
                            const float4 pk = cP[k];
                            const float2 dx = __fadd2_rn(fx, lo2(pk)), dy = __fadd2_rn(fy, hi2(pk));
                            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                            bool a0 = r2.x < slo, a1 = r2.y < slo;
                            if (r2.x >= slo && r2.x <= shi) {  // thin shell: the exact FP64 decision
                                const int b = cand_arena(cc, t0 + 2 * k);
                                a0 = dist2_2d(xa - y[b], ya - y[P + b]) < supp2;
                                ++shell;
                            }
                            if (r2.y >= slo && r2.y <= shi) {
                                const int b = cand_arena(cc, t0 + 2 * k + 1);
                                a1 = dist2_2d(xa - y[b], ya - y[P + b]) < supp2;
                                ++shell;
                            }
                            // r = 0 (the particle itself): q = 0
                            const float2 qq = __fmul2_rn(make_float2(sqrt_apx(r2.x), sqrt_apx(r2.y)), ih2);
                            float2 t2, t, u2, u;
                            spline_terms2(qq, t2, t, u2, u);
                            // w = t^3 / 4 - u^3, rounded as fmaf(0.25 t2, t, -(u2 u))
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
                const double tg = cval(sg), ts = cval(ss), tb = cval(sb), tS = cval(sS), tq = cval(sq);
                const double ux = y[2 * P + a], uy = y[3 * P + a];
                A.dens[a] = sd * tg;
                A.dens[P + a] = sd * ts;
                A.dens[2 * P + a] = sd * tb;
                A.dens[3 * P + a] = sd * tS;
                A.dens[4 * P + a] = sd * tq;
                A.dens[5 * P + a] = sqrt(fma(ux, ux, fma(uy, uy, 1.0)));
                A.nnb[a] = nacc;
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
}

template <int TT>
__global__ void __launch_bounds__(TT) k_seg_gradient(Arena A, int stage, const double *__restrict__ y, int grp)
{
    __shared__ int s_base[kMaxSlots];
    __shared__ float4 cP[kTile / 2];   // (-x_0, -x_1, -y_0, -y_1) relative to the centre cell
    __shared__ float4 cXa[kTile / 2];  // (X^xx_0, X^xx_1, X^xy_0, X^xy_1) / sigma*^2
    __shared__ float4 cXb[kTile / 2];  // (X^yx_0, X^yx_1, X^yy_0, X^yy_1) / sigma*^2
    __shared__ float4 cU2[kTile / 2];  // (u^x_0, u^x_1, u^y_0, u^y_1) / sigma*
    __shared__ CellCtx cc;
    __shared__ int s_cell;
    const BatchTable *T = A.tab;
    const int ns = T->nslots;
    for (int i = threadIdx.x; i < ns; i += TT) s_base[i] = A.grid[i].base;
    const int c_lo = grp > 0 ? A.ncells[1] : 0, c_hi = grp == 0 ? A.ncells[1] : A.ncells[0];
    const size_t P = (size_t)A.P;
    const double *gin = A.gin;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = TT / 32;
    for (;;) {
        __syncthreads();
        if (warp == 0) {
            int c = lane == 0 ? c_lo + (int)atomicAdd(&A.claim[claim_of(CLAIM_GRADIENT, grp)], 1u) : 0;
            c = __shfl_sync(0xFFFFFFFFu, c, 0);
            if (lane == 0) s_cell = c;
            bool work = c < c_hi && A.cnt[c] > 0u;
            if (work) work = T->slots[find_slot(s_base, ns, c)].mode == SLOT_STEP;
            if (work) cell_setup(A, s_base, ns, c, cc, lane);
            else if (lane == 0) cc.na = 0;
        }
        __syncthreads();
        if (s_cell >= c_hi) break;
        const int na = cc.na;
        if (na == 0) continue;
        const EvView &V = A.segv[cc.s];
        const float ih = (float)V.inv_h;
        const float slo = cc.clamped ? -1.0f : V.shell_lo, shi = cc.clamped ? 3.0e38f : V.shell_hi;
        const double supp2 = V.supp2;
        const int L = lanes_per_particle(na, A.lane_warps), ppw = 32 / L;
        const int pl = lane / L, l = lane - pl * L;
        const int M = cc.M;
        for (int g0 = 0; g0 < na; g0 += NW * ppw) {
            const int my = g0 + warp * ppw + pl;
            const bool valid = pl < ppw && my < na;
            const int a = cc.first + (valid ? my : 0);
            const double xa = y[a], ya = y[P + a];
            const float2 fa = A.fpos[a];
            CSum Gx = {0.f, 0.f}, Gy = {0.f, 0.f}, Hx = {0.f, 0.f}, Hy = {0.f, 0.f};
            CSum xx = {0.f, 0.f}, xy = {0.f, 0.f}, yx = {0.f, 0.f}, yy = {0.f, 0.f};
            for (int t0 = 0; t0 < M; t0 += kTile) {
                const int mt = min(kTile, M - t0);
                if (g0 == 0 || M > kTile) {  // one tile serves every pass of the cell
                    if (t0 > 0 || g0 > 0) __syncthreads();
                    for (int i = tid; i < mt; i += TT) {
                        float2 rel;
                        const int b = cand_index(cc, t0 + i, A.fpos, rel);
                        put_pair(cP, i, -rel.x, -rel.y);
                        const float4 X = A.fX[b];
                        const float2 U = A.fU[b];
                        put_pair(cXa, i, X.x, X.y);
                        put_pair(cXb, i, X.z, X.w);
                        put_pair(cU2, i, U.x, U.y);
                    }
                    if ((mt & 1) && tid == 0) {
                        put_pair(cP, mt, kFar, kFar);
                        put_pair(cXa, mt, 0.0f, 0.0f);
                        put_pair(cXb, mt, 0.0f, 0.0f);
                        put_pair(cU2, mt, 0.0f, 0.0f);
                    }
                    __syncthreads();
                }
                if (valid) {
                    const float2 fx = make_float2(fa.x, fa.x), fy = make_float2(fa.y, fa.y), ih2 = make_float2(ih, ih);
                    const int np = (mt + 1) >> 1;
                    for (int kb = l; kb < np; kb += (kRun / 2) * L) {
                        const int ke = min(np, kb + (kRun / 2) * L);
                        float2 pGx = make_float2(0.f, 0.f), pGy = pGx, pHx = pGx, pHy = pGx;
                        float2 pxx = pGx, pxy = pGx, pyx = pGx, pyy = pGx;
#pragma unroll 2
                        for (int k = kb; k < ke; k += L) {
                            const float4 pk = cP[k];
                            const float2 dx = __fadd2_rn(fx, lo2(pk)), dy = __fadd2_rn(fy, hi2(pk));
                            const float2 r2 = __ffma2_rn(dx, dx, __fmul2_rn(dy, dy));
                            bool a0 = r2.x < slo, a1 = r2.y < slo;
                            if (r2.x >= slo && r2.x <= shi) {  // thin shell: the exact FP64 decision
                                const int b = cand_arena(cc, t0 + 2 * k);
                                a0 = dist2_2d(xa - y[b], ya - y[P + b]) < supp2;
                            }
                            if (r2.y >= slo && r2.y <= shi) {
                                const int b = cand_arena(cc, t0 + 2 * k + 1);
                                a1 = dist2_2d(xa - y[b], ya - y[P + b]) < supp2;
                            }
                            // r = 0 (the particle itself) gives dw/dq = 0: a zero term
                            const float2 ir = make_float2(rsqrt_apx(fmaxf(r2.x, 1e-30f)), rsqrt_apx(fmaxf(r2.y, 1e-30f)));
                            float2 t2, t, u2, u;
                            spline_terms2(__fmul2_rn(__fmul2_rn(r2, ir), ih2), t2, t, u2, u);
                            // fac = (3 u^2 - 3 t^2 / 4) / r, rounded as fmaf(-0.75, t2, 3 u2) * ir
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
                const double t00 = cval(xx), t01 = cval(xy), t10 = cval(yx), t11 = cval(yy);
                const double tau = A.sc[cc.s].tau + (stage == 2 ? V.dtau : 0.0);
                const double sqrtg = V.milne ? tau : 1.0;
                const double cf = V.sigma_d * V.inv_h;
                double *go = A.gout;
                go[a] = cf * t00;
                go[P + a] = cf * t01;
                go[2 * P + a] = cf * t10;
                go[3 * P + a] = cf * t11;
                const double Fx = gin[a] * tGx + gin[2 * P + a] * tGy + tHx;
                const double Fy = gin[P + a] * tGx + gin[3 * P + a] * tGy + tHy;
                go[4 * P + a] = -sqrtg * cf * Fx;
                go[5 * P + a] = -sqrtg * cf * Fy;
            }
        }
    }
}

// launch shapes of the tiled passes the autotuner chooses among (threads per block; the
// results do not depend on the choice)
constexpr int kTTChoices[] = {64, 96, 128, 192, 256};

// persistent grids of the two tiled passes: each fills every SM with as many blocks as its own
// registers and shared memory allow (the cells are claimed dynamically, so the grid size does
// not change the results)
struct TiledGrid {
    int d = 0, g = 0;  // density, gradient
};

template <int TT>
TiledGrid tiled_grid(int sms)
{
    int o1 = 0, o2 = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_seg_density<TT>, TT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_seg_gradient<TT>, TT, 0);
    return TiledGrid{sms * std::max(1, o1), sms * std::max(1, o2)};
}

TiledGrid tiled_grid_for(int tt, int sms)
{
    switch (tt) {
    case 64: return tiled_grid<64>(sms);
    case 96: return tiled_grid<96>(sms);
    case 192: return tiled_grid<192>(sms);
    case 256: return tiled_grid<256>(sms);
    default: return tiled_grid<128>(sms);
    }
}

void tiled_density(int tt, int grid, cudaStream_t st, const Arena &A, const double *ys, const double *nq, int grp = -1)
{
    switch (tt) {
    case 64: k_seg_density<64><<<grid, 64, 0, st>>>(A, ys, nq, grp); break;
    case 96: k_seg_density<96><<<grid, 96, 0, st>>>(A, ys, nq, grp); break;
    case 192: k_seg_density<192><<<grid, 192, 0, st>>>(A, ys, nq, grp); break;
    case 256: k_seg_density<256><<<grid, 256, 0, st>>>(A, ys, nq, grp); break;
    default: k_seg_density<128><<<grid, 128, 0, st>>>(A, ys, nq, grp); break;
    }
}

void tiled_gradient(int tt, int grid, cudaStream_t st, const Arena &A, int stage, const double *ys, int grp = -1)
{
    switch (tt) {
    case 64: k_seg_gradient<64><<<grid, 64, 0, st>>>(A, stage, ys, grp); break;
    case 96: k_seg_gradient<96><<<grid, 96, 0, st>>>(A, stage, ys, grp); break;
    case 192: k_seg_gradient<192><<<grid, 192, 0, st>>>(A, stage, ys, grp); break;
    case 256: k_seg_gradient<256><<<grid, 256, 0, st>>>(A, stage, ys, grp); break;
    default: k_seg_gradient<128><<<grid, 128, 0, st>>>(A, stage, ys, grp); break;
    }
}

// The work integral's rate per event: the sum of its particles' (p + Pi + tau^2 pi^{eta eta}) /
// sigma* in a fixed order that depends on the event alone.  Its range splits into kWorkChunks
// chunks of a size set by its particle count (a multiple of 256); block (c, s) sums chunk c of
// slot s, and k_seg_work adds the chunks in order.
constexpr int kWorkChunks = 16;

__device__ __forceinline__ double block_sum_fixed(double acc, double *sh)
{
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    return sh[0];
}

__global__ void __launch_bounds__(256) k_seg_work_part(Arena A)
{
    __shared__ double sh[256];
    const int s = blockIdx.y, c = blockIdx.x;
    const BatchTable *T = A.tab;
    if (s >= T->nslots || T->slots[s].mode != SLOT_STEP) return;
    const SegSlot sl = T->slots[s];
    const int cs = ((sl.n + kWorkChunks - 1) / kWorkChunks + 255) & ~255;
    const int b0 = c * cs, b1 = min(sl.n, b0 + cs);
    double acc = 0.0;
    for (int i = b0 + (int)threadIdx.x; i < b1; i += 256) acc += A.wpart[sl.off + i];
    acc = block_sum_fixed(acc, sh);  // every block reaches it: the return above is block-uniform
    if (threadIdx.x == 0) A.wchunk[s * kWorkChunks + c] = acc;
}

__global__ void k_seg_work(Arena A, int stage)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const BatchTable *T = A.tab;
    if (s >= T->nslots || T->slots[s].mode != SLOT_STEP) return;
    double acc = 0.0;
    for (int c = 0; c < kWorkChunks; ++c) acc += A.wchunk[s * kWorkChunks + c];
    DevScalars &sc = A.sc[s];
    const EvView &V = A.segv[s];
    sc.wr[stage - 1] = V.milne ? acc : 0.0;
    if (stage == 2) {
        sc.work += 0.5 * V.dtau * (sc.wr[0] + sc.wr[1]);
        sc.tau = sc.tau + V.dtau;
        sc.steps += 1;
        // the host's view of the event's health (read before later launches)
        if (A.hflags) *(volatile unsigned int *)(A.hflags + s) = sc.status_or;
    }
}

// ---------------------------------------------------------------------------
// admission and retirement
__global__ void k_seg_admit(Arena A, int slot, int off, int n, int cap)
{
    const size_t P = (size_t)A.P;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) {
        const int a = off + i;
        A.segid[a] = slot;
        A.id[0][a] = i < n ? i : 0;
        for (int k = 0; k < 4; ++k) A.wguess[k * P + a] = A.xs1[0][k * P + a] = 0.0;
    }
}

__global__ void k_seg_release(Arena A, int off, int cap)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) A.segid[off + i] = -1;
}

// rows of a retired event's result block (original particle order)
constexpr int kResRows = 23;  // 9 state, 3 N_q, T, mu x3, p, e, sigma*, s, n_q x3
constexpr int R_STATE = 0, R_NQ = 9, R_T = 12, R_MU = 13, R_P = 16, R_E = 17, R_SIG = 18, R_S = 19, R_N = 20;

// observe-mode results: the stage-1 buffers (sorted) to the original order, plus the
// per-particle contributions to the event totals: sqrt(-g) T^{00}/sigma*, S, N_q
__global__ void k_seg_unsort(Arena A, int slot, double *__restrict__ res, int *__restrict__ ires,
                             double *__restrict__ contrib)
{
    const SegSlot sl = A.tab->slots[slot];
    const EvView &V = A.segv[slot];
    const size_t P = (size_t)A.P, n = (size_t)sl.n;
    const double tau = A.sc[slot].tau;
    const double sqrtg = V.milne ? tau : 1.0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < sl.n; j += gridDim.x * blockDim.x) {
        const size_t a = (size_t)sl.off + j;
        const size_t o = (size_t)A.id[1][a];
        const double *Y = A.Y[1], *N = A.Nq[1];
        for (int r = 0; r < 9; ++r) res[(R_STATE + r) * n + o] = Y[r * P + a];
        for (int q = 0; q < 3; ++q) res[(R_NQ + q) * n + o] = N[q * P + a];
        for (int r = 0; r < 6; ++r) res[(R_T + r) * n + o] = A.eosf[r * P + a];
        res[R_SIG * n + o] = A.dens[a];
        for (int r = 0; r < 4; ++r) res[(R_S + r) * n + o] = A.dens[(1 + r) * P + a];
        ires[o] = A.nnb[a];
        ires[n + o] = (int)A.status[a];
        const double sig = A.dens[a], g = A.dens[5 * P + a];
        const double sigma = sig / (g * sqrtg);
        const double ux = Y[2 * P + a], uy = Y[3 * P + a];
        const double vx = ux / g, vy = uy / g;
        double Pi = 0.0, ptt = 0.0;
        if (V.tr.viscous) {
            Pi = sigma * Y[5 * P + a];
            const double pxx = sigma * Y[6 * P + a], pxy = sigma * Y[7 * P + a], pyy = sigma * Y[8 * P + a];
            ptt = vx * (vx * pxx + vy * pxy) + vy * (vx * pxy + vy * pyy);
        }
        const double p = A.eosf[4 * P + a], e = A.eosf[5 * P + a];
        const double T00 = (e + p + Pi) * g * g - (p + Pi) + ptt;
        contrib[o] = sqrtg * T00 / sig;
        contrib[n + o] = Y[4 * P + a];
        for (int q = 0; q < 3; ++q) contrib[(2 + q) * n + o] = N[q * P + a];
    }
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
namespace {

thread_local std::string s_err;

sph_status sfail(sph_status s, const std::string &m)
{
    set_last_error(m.c_str());
    return s;
}

#define SCK(call)                                                                                         \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return sfail(SPH_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

double now_s() { return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count(); }

// first-fit allocator over [0, size) in units of `align`
struct RangeAlloc {
    std::map<long long, long long> fr;  // offset -> length of free ranges
    long long align = 1;
    void init(long long size, long long al)
    {
        align = al;
        fr.clear();
        if (size > 0) fr[0] = size;
    }
    long long alloc(long long len)
    {
        len = (len + align - 1) / align * align;
        for (auto it = fr.begin(); it != fr.end(); ++it)
            if (it->second >= len) {
                long long off = it->first, rest = it->second - len;
                fr.erase(it);
                if (rest > 0) fr[off + len] = rest;
                return off;
            }
        return -1;
    }
    void release(long long off, long long len)
    {
        len = (len + align - 1) / align * align;
        auto it = fr.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != fr.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            fr.erase(nx);
        }
        if (it != fr.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                fr.erase(it);
            }
        }
    }
};

enum { TK_QUEUED = 0, TK_RUNNING = 1, TK_RETIRING = 2, TK_DONE = 3 };

// kernel groups of a stage for the sampled timing, and the events that delimit them
constexpr int kProfGroups = 6;
constexpr int kProfMarks = 2 * (kProfGroups + 1);
const char *const kProfNames[kProfGroups] = {"sort", "density", "eos", "gradient", "eom", "work"};

struct Ticket {
    int64_t id = 0;
    int state = TK_QUEUED;
    int n = 0, nsteps = 0, steps_left = 0, slot = -1, off = -1, cap = 0;
    double t_submit = 0.0, t_done = 0.0;
    unsigned char *pin = nullptr;  // pinned block (or heap when the pool is exhausted)
    long long pin_off = -1;        // offset in the pool (-1: heap)
    size_t pin_bytes = 0;
    bool viscous = false;
    bool failed = false;  // ended early: its state or rates became non-finite
    cudaEvent_t done = nullptr;
    EvView view{};
    DevScalars sc0{};
    // layout of the block: inputs (12 n doubles) overlaid by results afterwards
    double *in_rows() { return reinterpret_cast<double *>(pin); }
    double *res() { return reinterpret_cast<double *>(pin); }
    int *ires() { return reinterpret_cast<int *>(pin + (size_t)kResRows * n * 8); }
    double *tot() { return reinterpret_cast<double *>(pin + (size_t)kResRows * n * 8 + (size_t)8 * n); }
    DevScalars *sc_out() { return reinterpret_cast<DevScalars *>(pin + (size_t)kResRows * n * 8 + (size_t)8 * n + 64); }
    static size_t bytes_for(int n) { return (size_t)kResRows * n * 8 + (size_t)8 * n + 64 + sizeof(DevScalars) + 256; }
};

}  // namespace

struct sph_server {
    sph_eos *eos = nullptr;
    bool eos_held = false;
    EosDev E{};
    Arena A{};
    std::vector<void *> allocs;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int max_events = 0, inflight = 2, grid_p = 0, grid_e = 0, sms = 1;
    TiledGrid grid_c;  // persistent grids of the tiled passes
    // Two-group schedule: the events split into two groups of about equal particle counts
    // (contiguous slot ranges); group 1's passes run on a second branch of the step graph one
    // pass behind group 0's, so that one group's FP64-bound passes (EoS, equations of motion)
    // and the other's FP32 neighbour passes fill each other's tails.  Each pass keeps its full
    // persistent grid: splitting the register file between a FP64 and a FP32 pass (fewer
    // blocks for each) measured slower, since both need most of it.
    int groups = 2;
    cudaStream_t st2 = nullptr;
    cudaEvent_t fk[2] = {nullptr, nullptr};
    int tt = kTTDefault;  // threads per block of the tiled passes
    int polish = 0;
    // pinned staging pool
    unsigned char *pool = nullptr;
    size_t pool_bytes = 0;
    RangeAlloc pool_alloc, arena_alloc;
    // tickets and slots
    int64_t next_id = 1;
    std::deque<Ticket *> queue;
    std::unordered_map<int64_t, Ticket *> tickets;
    std::vector<Ticket *> slot_owner;
    std::vector<SegSlot> slots;  // host mirror of the slot table
    int hi = 0, nslots = 0;
    bool table_dirty = true;
    BatchTable *tab_ring = nullptr;  // pinned snapshots of the table
    int tab_ring_n = 16, tab_ring_i = 0;
    // device scratch of retirement
    double *res_d = nullptr, *contrib_d = nullptr, *tot_d = nullptr;
    int *ires_d = nullptr;
    int res_cap = 0;
    // step graph and pacing
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};  // the step graph: [0] all events in turn, [1] overlapped groups
    cudaGraph_t graph[2] = {nullptr, nullptr};
    bool split_ok = false;  // the current table has two non-empty event groups
    std::vector<cudaEvent_t> step_ev;
    std::vector<cudaEvent_t> step_t0;  // timing events at the start of each batch step (same ring)
    long long steps_launched = 0, steps_timed = 0;
    double device_ms = 0.0;            // device time of the completed batch steps
    cudaEvent_t ref_ev = nullptr;
    double ref_host = 0.0;
    // per-slot status words the device writes after each batch step (mapped pinned memory)
    unsigned int *hflags = nullptr;
    // statistics
    long long particle_steps = 0, launches = 0, failed = 0;
    double timeout_s = 60.0;
    // sampled per-kernel-group timing: every prof_every-th batch step runs eagerly with CUDA
    // events between its kernel groups (same kernels, same stream); prof_step[i] is the batch
    // step whose marks ring entry i holds (-1: none)
    int prof_every = 0;
    std::vector<cudaEvent_t> prof_ev;  // ring of kProfMarks events per entry
    std::vector<long long> prof_step;
    double prof_ms[kProfGroups] = {};
    long long prof_n[kProfGroups] = {};
};

namespace {

sph_status dmalloc(sph_server *S, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(SPH_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    S->allocs.push_back(*p);
    return SPH_OK;
}

// kernels a batch step launches: per stage 11 for the cell list and permutation, then the
// density, EoS, gradient and equations-of-motion passes and the two of the work sum
constexpr int kKernelsPerBatchStep = 2 * 17;

// one batch step (both stages) on the server's stream; captured once into a graph.  marks (the
// sampled timing, eager launches only): kProfMarks events recorded between the kernel groups
void enqueue_batch_step(sph_server *S, const cudaEvent_t *marks = nullptr, bool overlap = false)
{
    const Arena &A = S->A;
    cudaStream_t st = S->st;
    const size_t P = (size_t)A.P;
    auto mark = [&](int stage, int j) {
        if (marks) cudaEventRecord(marks[(stage - 1) * (kProfGroups + 1) + j], st);
    };
    for (int stage = 1; stage <= 2; ++stage) {
        const double *ysrc = stage == 1 ? A.Y[0] : A.Y1[0];
        const int *idsrc = stage == 1 ? A.id[0] : A.id[1];
        mark(stage, 0);
        k_seg_reset<<<1, 256, 0, st>>>(A);
        k_seg_bbox<<<S->grid_p, 256, 0, st>>>(A, stage, ysrc);
        k_seg_grid<<<1, kMaxSlots, 0, st>>>(A, stage);
        k_seg_zero<<<S->grid_p, 256, 0, st>>>(A);
        k_seg_keys<<<S->grid_p, 256, 0, st>>>(A, stage, ysrc);
        k_seg_scan_part<<<kScanBlocks, 256, 0, st>>>(A);
        k_seg_scan_top<<<1, 256, 0, st>>>(A);
        k_seg_scan_apply<<<kScanBlocks, 256, 0, st>>>(A);
        k_seg_scatter<<<S->grid_p, 256, 0, st>>>(A, stage);
        k_seg_rank<<<S->grid_p, 256, 0, st>>>(A, stage, idsrc);
        SegPerm pa{};
        if (stage == 1) {
            pa.ng = 4;
            pa.src[0] = A.Y[0], pa.dst[0] = A.Y[1], pa.rows[0] = 9;
            pa.src[1] = A.Nq[0], pa.dst[1] = A.Nq[1], pa.rows[1] = 3;
            pa.src[2] = A.wguess, pa.dst[2] = A.guess_in, pa.rows[2] = 4;
            pa.src[3] = A.xs1[0], pa.dst[3] = A.xs1[1], pa.rows[3] = 4;
            pa.id_in = A.id[0], pa.id_out = A.id[1];
            pa.nq = A.Nq[0];
        } else {
            pa.ng = 5;
            pa.src[0] = A.Y1[0], pa.dst[0] = A.Y1[1], pa.rows[0] = 9;
            pa.src[1] = A.Y[1], pa.dst[1] = A.Y[0], pa.rows[1] = 9;
            pa.src[2] = A.Nq[1], pa.dst[2] = A.Nq[0], pa.rows[2] = 3;
            pa.src[3] = A.wguess, pa.dst[3] = A.guess_in, pa.rows[3] = 4;
            pa.src[4] = A.xs1[1], pa.dst[4] = A.xs1[0], pa.rows[4] = 4;
            pa.id_in = A.id[1], pa.id_out = A.id[0];
            pa.nq = A.Nq[1];
        }
        k_seg_permute<<<S->grid_p, 256, 0, st>>>(A, stage, pa);
        mark(stage, 1);
        const double *ys = stage == 1 ? A.Y[1] : A.Y1[1];
        const double *nq = stage == 1 ? A.Nq[1] : A.Nq[0];
        double *yout = stage == 1 ? A.Y1[0] : A.Y[0];
        const int mode = stage == 1 ? 0 : 1;
        if (overlap && !marks) {
            // group 0 on st; group 1 on st2 from the end of group 0's densities, so its density
            // pass meets group 0's EoS, its EoS group 0's gradient, its gradient group 0's
            // equations of motion; then st waits for group 1
            tiled_density(S->tt, S->grid_c.d, st, A, ys, nq, 0);
            cudaEventRecord(S->fk[0], st);
            cudaStreamWaitEvent(S->st2, S->fk[0], 0);
            launch_eos2_seg(A, S->E, stage, ys, S->grid_e, st, 0);
            tiled_density(S->tt, S->grid_c.d, S->st2, A, ys, nq, 1);
            tiled_gradient(S->tt, S->grid_c.g, st, A, stage, ys, 0);
            launch_eos2_seg(A, S->E, stage, ys, S->grid_e, S->st2, 1);
            launch_eom2_seg(A, stage, mode, ys, yout, S->grid_p, st, 0);
            tiled_gradient(S->tt, S->grid_c.g, S->st2, A, stage, ys, 1);
            launch_eom2_seg(A, stage, mode, ys, yout, S->grid_p, S->st2, 1);
            cudaEventRecord(S->fk[1], S->st2);
            cudaStreamWaitEvent(st, S->fk[1], 0);
        } else {
            tiled_density(S->tt, S->grid_c.d, st, A, ys, nq);
            mark(stage, 2);
            launch_eos2_seg(A, S->E, stage, ys, S->grid_e, st);
            mark(stage, 3);
            tiled_gradient(S->tt, S->grid_c.g, st, A, stage, ys);
            mark(stage, 4);
            launch_eom2_seg(A, stage, mode, ys, yout, S->grid_p, st);
            mark(stage, 5);
        }
        k_seg_work_part<<<dim3(kWorkChunks, S->max_events), 256, 0, st>>>(A);
        k_seg_work<<<(S->max_events + 127) / 128, 128, 0, st>>>(A, stage);
        mark(stage, 6);
    }
    (void)P;
}

sph_status wait_event(sph_server *S, cudaEvent_t ev)
{
    const double t0 = now_s();
    for (;;) {
        cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return SPH_OK;
        if (e != cudaErrorNotReady) return sfail(SPH_ERR_CUDA, std::string("event: ") + cudaGetErrorString(e));
        const double el = now_s() - t0;
        if (el > S->timeout_s) return sfail(SPH_ERR_TIMEOUT, "device did not finish within the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 20 : 200));
    }
}

// completion time of a recorded event on the host clock (device timestamps against the
// reference event, whose host time was taken when it completed)
double event_host_time(sph_server *S, cudaEvent_t ev)
{
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, S->ref_ev, ev) != cudaSuccess) {
        cudaGetLastError();
        return now_s();
    }
    return S->ref_host + 1e-3 * (double)ms;
}

void poll_retiring(sph_server *S)
{
    for (auto &kv : S->tickets) {
        Ticket *t = kv.second;
        if (t->state != TK_RETIRING) continue;
        cudaError_t e = cudaEventQuery(t->done);
        if (e == cudaSuccess) {
            t->t_done = event_host_time(S, t->done);
            t->state = TK_DONE;
        } else if (e != cudaErrorNotReady) {
            cudaGetLastError();
        }
    }
}

sph_status upload_table(sph_server *S)
{
    if (!S->table_dirty) return SPH_OK;
    BatchTable &b = S->tab_ring[S->tab_ring_i];
    S->tab_ring_i = (S->tab_ring_i + 1) % S->tab_ring_n;
    b.hi = S->hi;
    b.nslots = S->nslots;
    // the event groups: the slot boundary closest to half the particles (group 1 empty with one
    // schedule or a single event)
    b.split = S->nslots;
    if (S->groups == 2) {
        long long tot = 0, cum = 0, best = -1;
        for (int s = 0; s < S->nslots; ++s)
            if (S->slots[s].mode != SLOT_FREE) tot += S->slots[s].n;
        for (int s = 1; s < S->nslots; ++s) {
            if (S->slots[s - 1].mode != SLOT_FREE) cum += S->slots[s - 1].n;
            const long long d = std::llabs(2 * cum - tot);
            if (cum > 0 && cum < tot && (best < 0 || d < best)) {
                best = d;
                b.split = s;
            }
        }
    }
    S->split_ok = b.split < S->nslots;
    for (int s = 0; s < S->nslots; ++s) b.slots[s] = S->slots[s];
    const size_t bytes = offsetof(BatchTable, slots) + sizeof(SegSlot) * (size_t)std::max(S->nslots, 1);
    SCK(cudaMemcpyAsync(S->A.tab, &b, bytes, cudaMemcpyHostToDevice, S->st));
    S->table_dirty = false;
    return SPH_OK;
}

void recompute_hi(sph_server *S)
{
    int hi = 0, ns = 0;
    for (int s = 0; s < S->max_events; ++s)
        if (S->slots[s].mode != SLOT_FREE) {
            hi = std::max(hi, S->slots[s].off + S->slots[s].cap);
            ns = s + 1;
        }
    S->hi = hi;
    S->nslots = ns;
}

sph_status admit(sph_server *S, Ticket *t)
{
    int slot = -1;
    for (int s = 0; s < S->max_events; ++s)
        if (S->slots[s].mode == SLOT_FREE && !S->slot_owner[s]) {
            slot = s;
            break;
        }
    if (slot < 0) return SPH_ERR_STATE;
    const long long off = S->arena_alloc.alloc(t->cap);
    if (off < 0) return SPH_ERR_OOM;
    const Arena &A = S->A;
    const size_t P = (size_t)A.P;
    const int n = t->n;
    t->slot = slot;
    t->off = (int)off;
    t->view.sc = A.sc + slot;
    // initial state rows (x, y, u^x, u^y, S, Bv, Pv x3) and charges
    const double *rows = t->in_rows();
    for (int r = 0; r < 9; ++r)
        SCK(cudaMemcpyAsync(A.Y[0] + r * P + off, rows + (size_t)r * n, sizeof(double) * n, cudaMemcpyHostToDevice,
                            S->st));
    for (int q = 0; q < 3; ++q)
        SCK(cudaMemcpyAsync(A.Nq[0] + q * P + off, rows + (size_t)(9 + q) * n, sizeof(double) * n,
                            cudaMemcpyHostToDevice, S->st));
    unsigned char *tail = t->pin + t->pin_bytes - 256 - sizeof(EvView) - sizeof(DevScalars);
    std::memcpy(tail, &t->view, sizeof(EvView));
    std::memcpy(tail + sizeof(EvView), &t->sc0, sizeof(DevScalars));
    SCK(cudaMemcpyAsync(A.segv + slot, tail, sizeof(EvView), cudaMemcpyHostToDevice, S->st));
    SCK(cudaMemcpyAsync(A.sc + slot, tail + sizeof(EvView), sizeof(DevScalars), cudaMemcpyHostToDevice, S->st));
    k_seg_admit<<<nblk(t->cap, 256), 256, 0, S->st>>>(A, slot, (int)off, n, t->cap);
    SCK(cudaGetLastError());
    S->launches += 1;
    S->slot_owner[slot] = t;
    S->slots[slot] = SegSlot{t->nsteps > 0 ? SLOT_STEP : SLOT_OBSERVE, (int)off, n, t->cap};
    t->steps_left = t->nsteps;
    t->state = TK_RUNNING;
    S->table_dirty = true;
    recompute_hi(S);
    return SPH_OK;
}

// after the step that ran slot s in observe mode: results to the ticket's pinned block
sph_status retire(sph_server *S, int slot)
{
    Ticket *t = S->slot_owner[slot];
    const Arena &A = S->A;
    const int n = t->n;
    k_seg_unsort<<<nblk(n, 256), 256, 0, S->st>>>(A, slot, S->res_d, S->ires_d, S->contrib_d);
    launch_sum_fixed(S->contrib_d, n, 5, S->tot_d, S->st);
    S->launches += 3;
    SCK(cudaMemcpyAsync(t->res(), S->res_d, sizeof(double) * kResRows * n, cudaMemcpyDeviceToHost, S->st));
    SCK(cudaMemcpyAsync(t->ires(), S->ires_d, sizeof(int) * 2 * n, cudaMemcpyDeviceToHost, S->st));
    SCK(cudaMemcpyAsync(t->tot(), S->tot_d, sizeof(double) * 5, cudaMemcpyDeviceToHost, S->st));
    SCK(cudaMemcpyAsync(t->sc_out(), A.sc + slot, sizeof(DevScalars), cudaMemcpyDeviceToHost, S->st));
    k_seg_release<<<nblk(t->cap, 256), 256, 0, S->st>>>(A, t->off, t->cap);
    S->launches += 1;
    SCK(cudaEventCreate(&t->done));
    SCK(cudaEventRecord(t->done, S->st));
    SCK(cudaGetLastError());
    S->arena_alloc.release(t->off, t->cap);
    S->slots[slot] = SegSlot{SLOT_FREE, 0, 0, 0};
    S->slot_owner[slot] = nullptr;
    t->state = TK_RETIRING;
    S->table_dirty = true;
    recompute_hi(S);
    return SPH_OK;
}

void release_ticket(sph_server *S, Ticket *t)
{
    if (t->done) cudaEventDestroy(t->done);
    if (t->pin_off >= 0) S->pool_alloc.release(t->pin_off, (long long)t->pin_bytes);
    else std::free(t->pin);
    S->tickets.erase(t->id);
    delete t;
}

// adds the device time of completed batch steps (their start/end events) to device_ms
void account_steps(sph_server *S)
{
    const long long R = (long long)S->step_ev.size();
    while (S->steps_timed < S->steps_launched) {
        const size_t i = (size_t)(S->steps_timed % R);
        if (cudaEventQuery(S->step_ev[i]) != cudaSuccess) {
            cudaGetLastError();
            break;
        }
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, S->step_t0[i], S->step_ev[i]) == cudaSuccess) S->device_ms += ms;
        else cudaGetLastError();
        if (!S->prof_step.empty() && S->prof_step[i] == S->steps_timed) {
            const cudaEvent_t *mk = S->prof_ev.data() + i * kProfMarks;
            for (int stage = 0; stage < 2; ++stage)
                for (int g = 0; g < kProfGroups; ++g) {
                    float gm = 0.0f;
                    const int b = stage * (kProfGroups + 1) + g;
                    if (cudaEventElapsedTime(&gm, mk[b], mk[b + 1]) == cudaSuccess) {
                        S->prof_ms[g] += gm;
                        S->prof_n[g] += 1;
                    } else {
                        cudaGetLastError();
                    }
                }
            S->prof_step[i] = -1;
        }
        ++S->steps_timed;
    }
}

sph_status batch_step(sph_server *S)
{
    // pacing: at most `inflight` steps ahead of the device
    const long long k = S->steps_launched;
    cudaEvent_t ev = S->step_ev[(size_t)(k % (long long)S->step_ev.size())];
    cudaEvent_t ev0 = S->step_t0[(size_t)(k % (long long)S->step_ev.size())];
    if (k >= (long long)S->step_ev.size()) {
        sph_status s = wait_event(S, ev);
        if (s != SPH_OK) return s;
    }
    account_steps(S);
    if (k >= S->inflight) {
        cudaEvent_t back = S->step_ev[(size_t)((k - S->inflight) % (long long)S->step_ev.size())];
        sph_status s = wait_event(S, back);
        if (s != SPH_OK) return s;
    }
    // an event whose state or rates became non-finite ends here, with its last state, instead of
    // slowing the batch down (its particles would crowd one cell).  The status word of a slot is
    // this ticket's own once it has run more than `inflight` steps: the step k - inflight waited
    // for above has then run it and written the word.
    for (int sl = 0; sl < S->max_events; ++sl) {
        if (S->slots[sl].mode != SLOT_STEP) continue;
        Ticket *t = S->slot_owner[sl];
        if (!t || t->nsteps - t->steps_left <= S->inflight) continue;
        if (*(volatile unsigned int *)(S->hflags + sl) & PST_NONFINITE) {
            t->failed = true;
            S->failed += 1;
            sph_status r = retire(S, sl);
            if (r != SPH_OK) return r;
        }
    }
    sph_status s = upload_table(S);
    if (s != SPH_OK) return s;
    // the overlapped graph when the table has two non-empty event groups
    const int gi = (S->groups == 2 && S->split_ok) ? 1 : 0;
    if (!S->gexec[gi]) {
        SCK(cudaStreamBeginCapture(S->st, cudaStreamCaptureModeThreadLocal));
        enqueue_batch_step(S, nullptr, gi == 1);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(S->st, &g);
        if (e != cudaSuccess) return sfail(SPH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        S->graph[gi] = g;
        SCK(cudaGraphInstantiate(&S->gexec[gi], g, 0));
    }
    SCK(cudaEventRecord(ev0, S->st));
    const size_t ring_i = (size_t)(k % (long long)S->step_ev.size());
    if (S->prof_every > 0 && k % S->prof_every == 0 && !S->prof_step.empty()) {
        // a sampled step: the same kernels launched eagerly, with events between the groups
        enqueue_batch_step(S, S->prof_ev.data() + ring_i * kProfMarks);
        S->prof_step[ring_i] = k;
    } else {
        if (!S->prof_step.empty()) S->prof_step[ring_i] = -1;
        SCK(cudaGraphLaunch(S->gexec[gi], S->st));
    }
    SCK(cudaEventRecord(ev, S->st));
    S->steps_launched += 1;
    S->launches += kKernelsPerBatchStep;
    // host bookkeeping of what that step did
    std::vector<int> observed;
    for (int sl = 0; sl < S->max_events; ++sl) {
        SegSlot &q = S->slots[sl];
        if (q.mode == SLOT_STEP) {
            Ticket *t = S->slot_owner[sl];
            S->particle_steps += q.n;
            if (--t->steps_left <= 0) {
                q.mode = SLOT_OBSERVE;
                S->table_dirty = true;
            }
        } else if (q.mode == SLOT_OBSERVE) {
            observed.push_back(sl);
        }
    }
    for (int sl : observed) {
        s = retire(S, sl);
        if (s != SPH_OK) return s;
    }
    return SPH_OK;
}

void admit_queued(sph_server *S)
{
    while (!S->queue.empty()) {
        Ticket *t = S->queue.front();
        if (admit(S, t) != SPH_OK) break;  // FIFO: the head waits for a slot and a range
        S->queue.pop_front();
    }
}

bool any_running(const sph_server *S)
{
    for (int s = 0; s < S->max_events; ++s)
        if (S->slots[s].mode != SLOT_FREE) return true;
    return false;
}

// the tiled passes' shape for the following steps; the step graph holds it, so a change drops
// the graph (captured again by the next step)
void apply_shape(sph_server *S, int tt, int lw)
{
    if (tt == S->tt && lw == S->A.lane_warps) return;
    S->tt = tt;
    S->A.lane_warps = lw;
    S->grid_c = tiled_grid_for(tt, S->sms);
    for (int i = 0; i < 2; ++i) {
        if (S->gexec[i]) cudaGraphExecDestroy(S->gexec[i]);
        if (S->graph[i]) cudaGraphDestroy(S->graph[i]);
        S->gexec[i] = nullptr;
        S->graph[i] = nullptr;
    }
}

}  // namespace

extern "C" {

sph_status sph_server_create(sph_server **out, const sph_server_desc *d, const sph_eos *eos)
{
    if (!out || !d || !eos) return sfail(SPH_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->max_events < 1 || d->max_events > kMaxSlots) return sfail(SPH_ERR_ARG, "max_events must be in 1..256");
    if (d->max_particles < 0 || d->hbm_fraction < 0.0 || d->hbm_fraction > 0.9)
        return sfail(SPH_ERR_ARG, "max_particles >= 0 and 0 <= hbm_fraction <= 0.9");
    sph_server *S = new (std::nothrow) sph_server();
    if (!S) return sfail(SPH_ERR_OOM, "host allocation");
    auto bail = [&](sph_status s) {
        std::string keep = sph_last_error();
        sph_server_free(S);
        set_last_error(keep.c_str());
        return s;
    };
    S->eos = const_cast<sph_eos *>(eos);
    S->E = eos_params(eos);
    S->polish = d->polish ? 1 : 0;
    S->E.polish = S->polish;
    S->E.tol = d->newton_tol > 0.0 ? d->newton_tol : 1e-10;
    S->max_events = d->max_events;
    S->inflight = d->max_inflight > 0 ? std::min(d->max_inflight, 8) : 2;
    if (const char *tl = getenv("SPH_WAIT_LIMIT_S")) S->timeout_s = atof(tl);
    if (d->stream) {
        S->st = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(sfail(SPH_ERR_CUDA, "cudaStreamCreate failed"));
        }
        S->own_stream = true;
    }
    // arena capacity: requested, or a share of free HBM
    const size_t per_particle = sizeof(double) * (9 * 4 + 3 * 2 + 4 * 4 + kNDens + kNEos + kNGin + kNGout) +
                                sizeof(int) * (2 + 1 + 1 + 1) + sizeof(uint32_t) * (1 + 4) + 8 + 48;
    long long P = d->max_particles;
    if (P == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            return bail(sfail(SPH_ERR_CUDA, "cudaMemGetInfo failed"));
        }
        const double f = d->hbm_fraction > 0.0 ? d->hbm_fraction : 0.25;
        P = (long long)(f * (double)fr / (double)per_particle);
    }
    P = std::min<long long>(P, 0x7FFFFF00LL) / kSegAlign * kSegAlign;
    if (P < kSegAlign) return bail(sfail(SPH_ERR_OOM, "arena smaller than one segment"));
    Arena &A = S->A;
    A.P = (int)P;
    A.lane_warps = kLaneWarpsDefault;
    A.cmax = S->max_events * kMaxCellsAxis * kMaxCellsAxis;
    const size_t Pz = (size_t)P;
    sph_status s;
#define SAL(ptr, bytes)                                                      \
    do {                                                                     \
        s = dmalloc(S, reinterpret_cast<void **>(&(ptr)), (bytes));          \
        if (s != SPH_OK) return bail(s);                                     \
    } while (0)
    for (int k = 0; k < 2; ++k) {
        SAL(A.Y[k], sizeof(double) * 9 * Pz);
        SAL(A.Y1[k], sizeof(double) * 9 * Pz);
        SAL(A.Nq[k], sizeof(double) * 3 * Pz);
        SAL(A.id[k], sizeof(int) * Pz);
    }
    SAL(A.wguess, sizeof(double) * 4 * Pz);
    SAL(A.xs1[0], sizeof(double) * 4 * Pz);
    SAL(A.xs1[1], sizeof(double) * 4 * Pz);
    SAL(A.guess_in, sizeof(double) * 4 * Pz);
    SAL(A.segid, sizeof(int) * Pz);
    SAL(A.dens, sizeof(double) * kNDens * Pz);
    SAL(A.eosf, sizeof(double) * kNEos * Pz);
    SAL(A.gin, sizeof(double) * kNGin * Pz);
    SAL(A.gout, sizeof(double) * kNGout * Pz);
    SAL(A.status, sizeof(uint32_t) * Pz);
    SAL(A.nnb, sizeof(int) * Pz);
    SAL(A.wpart, sizeof(double) * Pz);
    SAL(A.wchunk, sizeof(double) * kMaxSlots * kWorkChunks);
    SAL(A.key, sizeof(uint32_t) * Pz);
    SAL(A.rnk, sizeof(uint32_t) * Pz);
    SAL(A.tmp, sizeof(uint32_t) * Pz);
    SAL(A.perm, sizeof(uint32_t) * Pz);
    SAL(A.fpos, sizeof(float2) * Pz);
    SAL(A.fq, sizeof(float4) * Pz);
    SAL(A.fX, sizeof(float4) * Pz);
    SAL(A.fU, sizeof(float2) * Pz);
    SAL(A.cnt, sizeof(uint32_t) * (size_t)A.cmax);
    SAL(A.start, sizeof(uint32_t) * (size_t)A.cmax);
    SAL(A.scan_part, sizeof(uint32_t) * kScanBlocks);
    SAL(A.ncells, sizeof(int) * 2);
    SAL(A.claim, sizeof(unsigned int) * kClaims);
    SAL(A.tab, sizeof(BatchTable));
    SAL(A.grid, sizeof(SegGrid) * kMaxSlots);
    SAL(A.segv, sizeof(EvView) * kMaxSlots);
    SAL(A.sc, sizeof(DevScalars) * kMaxSlots);
    if (cudaMemsetAsync(A.segid, 0xFF, sizeof(int) * Pz, S->st) != cudaSuccess ||
        cudaMemsetAsync(A.tab, 0, sizeof(BatchTable), S->st) != cudaSuccess ||
        cudaMemsetAsync(A.grid, 0, sizeof(SegGrid) * kMaxSlots, S->st) != cudaSuccess ||
        cudaMemsetAsync(A.ncells, 0, sizeof(int) * 2, S->st) != cudaSuccess ||
        cudaMemsetAsync(A.claim, 0, sizeof(unsigned int) * kClaims, S->st) != cudaSuccess) {
        cudaGetLastError();
        return bail(sfail(SPH_ERR_CUDA, "cudaMemsetAsync failed"));
    }
    // retirement scratch: the largest event the arena can hold
    S->res_cap = (int)P;
    SAL(S->res_d, sizeof(double) * kResRows * Pz);
    SAL(S->ires_d, sizeof(int) * 2 * Pz);
    SAL(S->contrib_d, sizeof(double) * 5 * Pz);
    SAL(S->tot_d, sizeof(double) * (8 + 5 * 256));
#undef SAL
    // pinned staging pool
    S->pool_bytes = d->pinned_bytes > 0 ? (size_t)d->pinned_bytes : Ticket::bytes_for(1) + (size_t)256 * Pz;
    if (cudaHostAlloc(reinterpret_cast<void **>(&S->pool), S->pool_bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        S->pool = nullptr;
        S->pool_bytes = 0;
    }
    S->pool_alloc.init((long long)S->pool_bytes, 256);
    S->arena_alloc.init(P, kSegAlign);
    if (cudaHostAlloc(reinterpret_cast<void **>(&S->tab_ring), sizeof(BatchTable) * S->tab_ring_n,
                      cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        S->tab_ring = nullptr;
        return bail(sfail(SPH_ERR_OOM, "pinned table ring"));
    }
    if (cudaHostAlloc(reinterpret_cast<void **>(&S->hflags), sizeof(unsigned int) * kMaxSlots, cudaHostAllocMapped) !=
            cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void **>(&A.hflags), S->hflags, 0) != cudaSuccess) {
        cudaGetLastError();
        return bail(sfail(SPH_ERR_OOM, "mapped status words"));
    }
    std::memset(S->hflags, 0, sizeof(unsigned int) * kMaxSlots);
    S->slots.assign(S->max_events, SegSlot{SLOT_FREE, 0, 0, 0});
    S->slot_owner.assign(S->max_events, nullptr);
    S->step_ev.resize(16, nullptr);
    S->step_t0.resize(16, nullptr);
    for (auto *ring : {&S->step_ev, &S->step_t0})
        for (auto &e : *ring)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
                return bail(sfail(SPH_ERR_CUDA, "cudaEventCreate failed"));
            }
    // launch shapes: persistent grids of resident blocks on every SM
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(sms, 1);
    S->sms = sms;
    S->grid_p = sms * 8;
    S->grid_c = tiled_grid_for(S->tt, sms);
    S->grid_e = eos_seg_grid(sms);
    S->groups = d->groups == 1 ? 1 : 2;
    if (S->groups == 2) {
        if (cudaStreamCreateWithFlags(&S->st2, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->fk[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&S->fk[1], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(sfail(SPH_ERR_CUDA, "second stream of the overlapped schedule"));
        }
    }
    // host/device clock reference for completion times
    if (cudaEventCreate(&S->ref_ev) != cudaSuccess || cudaEventRecord(S->ref_ev, S->st) != cudaSuccess ||
        cudaEventSynchronize(S->ref_ev) != cudaSuccess) {
        cudaGetLastError();
        return bail(sfail(SPH_ERR_CUDA, "reference event"));
    }
    S->ref_host = now_s();
    eos_retain(S->eos);
    S->eos_held = true;
    *out = S;
    return SPH_OK;
}

void sph_server_free(sph_server *S)
{
    if (!S) return;
    if (S->st) cudaStreamSynchronize(S->st);
    for (auto &kv : S->tickets) {
        Ticket *t = kv.second;
        if (t->done) cudaEventDestroy(t->done);
        if (t->pin_off < 0) std::free(t->pin);
        delete t;
    }
    S->tickets.clear();
    for (int i = 0; i < 2; ++i) {
        if (S->gexec[i]) cudaGraphExecDestroy(S->gexec[i]);
        if (S->graph[i]) cudaGraphDestroy(S->graph[i]);
    }
    for (auto e : S->step_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : S->step_t0)
        if (e) cudaEventDestroy(e);
    for (auto e : S->prof_ev)
        if (e) cudaEventDestroy(e);
    if (S->ref_ev) cudaEventDestroy(S->ref_ev);
    for (void *p : S->allocs) cudaFree(p);
    if (S->pool) cudaFreeHost(S->pool);
    if (S->tab_ring) cudaFreeHost(S->tab_ring);
    if (S->hflags) cudaFreeHost(S->hflags);
    if (S->own_stream && S->st) cudaStreamDestroy(S->st);
    if (S->st2) cudaStreamDestroy(S->st2);
    for (cudaEvent_t e : S->fk)
        if (e) cudaEventDestroy(e);
    if (S->eos_held) sph_free_eos(S->eos);  // drops the server's reference
    delete S;
}

sph_status sph_submit(sph_server *S, const sph_event_desc *d, int32_t nsteps, int64_t *ticket)
{
    if (!S || !d || !ticket) return sfail(SPH_ERR_ARG, "null argument");
    *ticket = 0;
    if (d->dim != 2) return sfail(SPH_ERR_ARG, "the serving form runs 2+1D events (dim = 2)");
    if (d->kappaT2) return sfail(SPH_ERR_ARG, "the serving form runs without diffusion currents");
    if (nsteps < 0) return sfail(SPH_ERR_ARG, "nsteps < 0");
    if (d->n < 1 || d->n > S->A.P) return sfail(d->n < 1 ? SPH_ERR_ARG : SPH_ERR_OOM,
                                                d->n < 1 ? "the serving form needs n >= 1"
                                                         : "event larger than the arena");
    if (!(d->h > 0.0) || !(d->dtau > 0.0)) return sfail(SPH_ERR_ARG, "h and dtau must be positive");
    if (d->milne && !(d->tau0 > 0.0)) return sfail(SPH_ERR_ARG, "Milne coordinates need tau0 > 0");
    if (!d->x || !d->u || !d->S || !d->Nq) return sfail(SPH_ERR_ARG, "null particle array");
    if (d->viscous && (!(d->tau_pi_coef > 0.0) || !(d->tau_Pi_ratio > 0.0) || !(d->eta_over_s > 0.0)))
        return sfail(SPH_ERR_ARG, "viscous run needs eta_over_s, tau_pi_coef, tau_Pi_ratio > 0");
    const int n = (int)d->n;
    Ticket *t = new (std::nothrow) Ticket();
    if (!t) return sfail(SPH_ERR_OOM, "host allocation");
    t->n = n;
    t->nsteps = nsteps;
    t->cap = (n + kSegAlign - 1) / kSegAlign * kSegAlign;
    t->viscous = d->viscous != 0;
    t->pin_bytes = Ticket::bytes_for(n) + sizeof(EvView) + sizeof(DevScalars) + 256;
    t->pin_bytes = (t->pin_bytes + 255) / 256 * 256;
    long long po = S->pool ? S->pool_alloc.alloc((long long)t->pin_bytes) : -1;
    if (po >= 0) {
        t->pin = S->pool + po;
        t->pin_off = po;
    } else {
        t->pin = static_cast<unsigned char *>(std::malloc(t->pin_bytes));
        t->pin_off = -1;
        if (!t->pin) {
            delete t;
            return sfail(SPH_ERR_OOM, "host staging");
        }
    }
    // inputs: rows x, y, u^x, u^y, S, Bv, Pv (xx, xy, yy), then N_q (B, S, Q)
    double *rows = t->in_rows();
    const cudaMemcpyKind kind = d->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    const size_t nb = sizeof(double) * n;
    bool ok = cudaMemcpy(rows, d->x, 2 * nb, kind) == cudaSuccess &&
              cudaMemcpy(rows + 2 * (size_t)n, d->u, 2 * nb, kind) == cudaSuccess &&
              cudaMemcpy(rows + 4 * (size_t)n, d->S, nb, kind) == cudaSuccess &&
              cudaMemcpy(rows + 9 * (size_t)n, d->Nq, 3 * nb, kind) == cudaSuccess;
    if (ok && d->Bv) ok = cudaMemcpy(rows + 5 * (size_t)n, d->Bv, nb, kind) == cudaSuccess;
    else std::memset(rows + 5 * (size_t)n, 0, nb);
    if (ok && d->Pv) ok = cudaMemcpy(rows + 6 * (size_t)n, d->Pv, 3 * nb, kind) == cudaSuccess;
    else std::memset(rows + 6 * (size_t)n, 0, 3 * nb);
    if (!ok) {
        cudaGetLastError();
        if (t->pin_off >= 0) S->pool_alloc.release(t->pin_off, (long long)t->pin_bytes);
        else std::free(t->pin);
        delete t;
        return sfail(SPH_ERR_ARG, "cannot read the particle arrays");
    }
    // per-event parameters
    EvView &v = t->view;
    v = EvView{};
    v.n = n;
    v.dim = 2;
    v.milne = d->milne ? 1 : 0;
    v.nv = 9;
    v.h = d->h;
    v.inv_h = 1.0 / d->h;
    v.supp2 = 4.0 * d->h * d->h;
    v.inv_cell = 1.0 / (2.0 * d->h);
    v.mixed = 1;
    v.cell_f = (float)(2.0 * d->h);
    tiled_shell(d->h, v.shell_lo, v.shell_hi);
    v.sigma_d = 10.0 / (7.0 * kPi * d->h * d->h);
    v.dtau = d->dtau;
    v.eos = S->E;
    v.tr.viscous = d->viscous ? 1 : 0;
    v.tr.eta_over_s = d->eta_over_s;
    v.tr.zeta_peak = d->zeta_peak;
    v.tr.zeta_T_GeV = d->zeta_T_GeV;
    v.tr.zeta_w_GeV = d->zeta_w_GeV > 0.0 ? d->zeta_w_GeV : 1.0;
    v.tr.tau_pi_coef = d->tau_pi_coef;
    v.tr.tau_Pi_ratio = d->tau_Pi_ratio;
    v.tr.cs2_cap = d->cs2_cap > 0.0 ? d->cs2_cap : 1.0;
    v.tr.T_stop_GeV = d->T_stop_GeV > 0.0 ? d->T_stop_GeV : 0.0;
    t->sc0 = DevScalars{};
    t->sc0.tau = d->tau0;
    t->id = S->next_id++;
    t->t_submit = now_s();
    S->tickets[t->id] = t;
    S->queue.push_back(t);
    *ticket = t->id;
    return SPH_OK;
}

sph_status sph_server_pump(sph_server *S, int32_t max_steps, int32_t *running)
{
    if (!S || max_steps < 0) return sfail(SPH_ERR_ARG, "bad argument");
    for (int k = 0; k < max_steps; ++k) {
        poll_retiring(S);
        admit_queued(S);
        if (!any_running(S)) break;
        sph_status s = batch_step(S);
        if (s != SPH_OK) return s;
    }
    poll_retiring(S);
    if (running) {
        int r = 0;
        for (int s = 0; s < S->max_events; ++s) r += S->slots[s].mode != SLOT_FREE;
        *running = r;
    }
    return SPH_OK;
}

sph_status sph_poll(sph_server *S, int64_t ticket, int32_t *state, double *latency_s)
{
    if (!S || !state) return sfail(SPH_ERR_ARG, "null argument");
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return sfail(SPH_ERR_ARG, "unknown ticket");
    poll_retiring(S);
    Ticket *t = it->second;
    *state = t->state == TK_DONE ? SPH_TICKET_DONE : (t->state == TK_QUEUED ? SPH_TICKET_QUEUED : SPH_TICKET_RUNNING);
    if (latency_s) *latency_s = t->state == TK_DONE ? t->t_done - t->t_submit : 0.0;
    return SPH_OK;
}

sph_status sph_collect(sph_server *S, int64_t ticket, uint64_t mask, const sph_field_bufs *o, sph_totals *tot)
{
    if (!S) return sfail(SPH_ERR_ARG, "null argument");
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return sfail(SPH_ERR_ARG, "unknown ticket");
    poll_retiring(S);
    Ticket *t = it->second;
    if (t->state != TK_DONE) return sfail(SPH_ERR_STATE, "ticket not done");
    const uint64_t known = SPH_F_X | SPH_F_U | SPH_F_S | SPH_F_NQ | SPH_F_BV | SPH_F_PV | SPH_F_SIGMA_STAR |
                           SPH_F_S_DENS | SPH_F_N_DENS | SPH_F_T | SPH_F_MU | SPH_F_P | SPH_F_E | SPH_F_PI_BULK |
                           SPH_F_STATUS | SPH_F_NNB;
    if (mask & ~known) return sfail(SPH_ERR_ARG, "field not available from the serving form");
    if (mask && !o) return sfail(SPH_ERR_ARG, "null field buffers");
    if (mask && o->on_device) return sfail(SPH_ERR_ARG, "the serving form returns host buffers");
    const size_t n = (size_t)t->n;
    const double *res = t->res();
    const int *ires = t->ires();
    auto rows = [&](uint64_t bit, void *dst, int r0, int nr) -> bool {
        if (!(mask & bit)) return true;
        if (!dst) return false;
        std::memcpy(dst, res + (size_t)r0 * n, sizeof(double) * nr * n);
        return true;
    };
    bool ok = true;
    if (mask) {
        ok = ok && rows(SPH_F_X, o->x, R_STATE, 2) && rows(SPH_F_U, o->u, R_STATE + 2, 2) &&
             rows(SPH_F_S, o->S, R_STATE + 4, 1) && rows(SPH_F_BV, o->Bv, R_STATE + 5, 1) &&
             rows(SPH_F_PV, o->Pv, R_STATE + 6, 3) && rows(SPH_F_NQ, o->Nq, R_NQ, 3) &&
             rows(SPH_F_SIGMA_STAR, o->sigstar, R_SIG, 1) && rows(SPH_F_S_DENS, o->s, R_S, 1) &&
             rows(SPH_F_N_DENS, o->nq, R_N, 3) && rows(SPH_F_T, o->T, R_T, 1) && rows(SPH_F_MU, o->mu, R_MU, 3) &&
             rows(SPH_F_P, o->p, R_P, 1) && rows(SPH_F_E, o->e, R_E, 1);
        if (ok && (mask & SPH_F_PI_BULK)) {
            if (!o->Pi) ok = false;
            else
                for (size_t a = 0; a < n; ++a) {  // Pi = sigma Bv, sigma = sigma* / (u^0 sqrt(-g))
                    const double ux = res[(R_STATE + 2) * n + a], uy = res[(R_STATE + 3) * n + a];
                    const double g = std::sqrt(std::fma(ux, ux, std::fma(uy, uy, 1.0)));
                    const double sg = t->view.milne ? t->sc_out()->tau : 1.0;
                    o->Pi[a] = t->viscous ? res[R_SIG * n + a] / (g * sg) * res[(R_STATE + 5) * n + a] : 0.0;
                }
        }
        if (ok && (mask & SPH_F_NNB)) {
            if (!o->nnb) ok = false;
            else std::memcpy(o->nnb, ires, sizeof(int) * n);
        }
        if (ok && (mask & SPH_F_STATUS)) {
            if (!o->status) ok = false;
            else std::memcpy(o->status, ires + n, sizeof(uint32_t) * n);
        }
        if (!ok) return sfail(SPH_ERR_ARG, "null destination for a requested field");
    }
    if (tot) {
        const DevScalars *sc = t->sc_out();
        const double *tt = t->tot();
        std::memset(tot, 0, sizeof(*tot));
        tot->tau = sc->tau;
        tot->E = tt[0];
        tot->S = tt[1];
        for (int q = 0; q < 3; ++q) tot->N[q] = tt[2 + q];
        tot->work = sc->work;
        tot->status_or = sc->status_or;
        tot->steps = sc->steps;
        tot->pairs = (int64_t)sc->pairs;
        tot->kernel_launches = 0;
        tot->eos_work[0] = (int64_t)sc->eos_resid;
        tot->eos_work[1] = (int64_t)sc->eos_solve;
        tot->eos_work[2] = (int64_t)sc->eos_g;
        tot->shell_tests = (int64_t)sc->shell_tests;
    }
    release_ticket(S, t);
    return SPH_OK;
}

sph_status sph_server_stats_get(sph_server *S, sph_server_stats *o)
{
    if (!S || !o) return sfail(SPH_ERR_ARG, "null argument");
    poll_retiring(S);
    std::memset(o, 0, sizeof(*o));
    for (auto &kv : S->tickets) {
        const int st = kv.second->state;
        if (st == TK_QUEUED) o->queued++;
        else if (st == TK_DONE) o->done++;
        else o->running++;
    }
    o->batch_steps = S->steps_launched;
    o->particle_steps = S->particle_steps;
    o->arena_capacity = S->A.P;
    long long used = 0;
    for (int s = 0; s < S->max_events; ++s)
        if (S->slots[s].mode != SLOT_FREE) {
            used += S->slots[s].cap;
            o->slots_in_use++;
        }
    o->arena_in_use = used;
    o->kernel_launches = S->launches;
    o->max_events = S->max_events;
    account_steps(S);
    o->device_ms = S->device_ms;
    o->steps_timed = S->steps_timed;
    o->failed = S->failed;
    return SPH_OK;
}

sph_status sph_server_autotune(sph_server *S, int32_t trials, int32_t *chosen, int32_t *chosen_lanes)
{
    if (!S) return sfail(SPH_ERR_ARG, "null argument");
    if (trials < 1) trials = 3;
    if (!any_running(S) || S->steps_launched == 0)
        return sfail(SPH_ERR_STATE, "the autotuner times the running batch: pump a step first");
    SCK(cudaStreamSynchronize(S->st));
    // The last batch step's second stage left a consistent sorted state, cell list and
    // gradient inputs.  Each candidate re-runs that stage's tiled passes; their outputs are
    // recomputed by the next step, and the counters they add to are restored afterwards.
    const int ns = std::max(S->nslots, 1);
    std::vector<DevScalars> save((size_t)ns);
    SCK(cudaMemcpy(save.data(), S->A.sc, sizeof(DevScalars) * (size_t)ns, cudaMemcpyDeviceToHost));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SCK(cudaEventCreate(&e0));
    SCK(cudaEventCreate(&e1));
    Arena A = S->A;
    float best = 1e30f;
    int best_tt = S->tt, best_lw = S->A.lane_warps;
    for (int lw : kLaneWarpChoices)
        for (int tt : kTTChoices) {
            A.lane_warps = lw;
            const TiledGrid grid = tiled_grid_for(tt, S->sms);
            float tot = 0.0f;
            for (int r = 0; r <= trials; ++r) {  // r = 0: warm-up
                SCK(cudaMemsetAsync(A.claim, 0, sizeof(unsigned int) * kClaims, S->st));
                SCK(cudaEventRecord(e0, S->st));
                tiled_density(tt, grid.d, S->st, A, A.Y1[1], A.Nq[0]);
                tiled_gradient(tt, grid.g, S->st, A, 2, A.Y1[1]);
                SCK(cudaEventRecord(e1, S->st));
                SCK(cudaGetLastError());
                sph_status s = wait_event(S, e1);
                if (s != SPH_OK) return s;
                float ms = 0.0f;
                SCK(cudaEventElapsedTime(&ms, e0, e1));
                if (r > 0) tot += ms;
            }
            if (tot < best) {
                best = tot;
                best_tt = tt;
                best_lw = lw;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SCK(cudaMemcpy(S->A.sc, save.data(), sizeof(DevScalars) * (size_t)ns, cudaMemcpyHostToDevice));
    apply_shape(S, best_tt, best_lw);
    if (chosen) *chosen = S->tt;
    if (chosen_lanes) *chosen_lanes = S->A.lane_warps;
    return SPH_OK;
}

sph_status sph_server_set_shape(sph_server *S, int32_t threads, int32_t lane_warps)
{
    if (!S) return sfail(SPH_ERR_ARG, "null argument");
    bool ok_tt = false, ok_lw = false;
    for (int tt : kTTChoices) ok_tt = ok_tt || tt == threads;
    for (int lw : kLaneWarpChoices) ok_lw = ok_lw || lw == lane_warps;
    if (!ok_tt || !ok_lw) return sfail(SPH_ERR_ARG, "threads must be 64, 96, 128, 192 or 256 and lane_warps 2, 4 or 8");
    SCK(cudaStreamSynchronize(S->st));
    apply_shape(S, threads, lane_warps);
    return SPH_OK;
}

sph_status sph_server_profile(sph_server *S, int32_t every)
{
    if (!S || every < 0) return sfail(SPH_ERR_ARG, "bad argument");
    if (every > 0 && S->prof_ev.empty()) {
        // the ring of marks follows the step ring (its entries are read when a step completes)
        SCK(cudaStreamSynchronize(S->st));
        S->prof_ev.assign(S->step_ev.size() * kProfMarks, nullptr);
        for (auto &e : S->prof_ev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
                return sfail(SPH_ERR_CUDA, "cudaEventCreate failed");
            }
        S->prof_step.assign(S->step_ev.size(), -1);
    }
    S->prof_every = every;
    return SPH_OK;
}

sph_status sph_server_kernel_times(sph_server *S, int32_t max, char *names, double *ms, int64_t *launches,
                                   int32_t *count)
{
    if (!S || !count || (max > 0 && (!names || !ms || !launches))) return sfail(SPH_ERR_ARG, "null argument");
    if (S->prof_ev.empty()) return sfail(SPH_ERR_STATE, "sampled timing is off (sph_server_profile)");
    account_steps(S);
    const int m = std::min<int>(max, kProfGroups);
    for (int g = 0; g < m; ++g) {
        std::snprintf(names + 32 * g, 32, "%s", kProfNames[g]);
        ms[g] = S->prof_ms[g];
        launches[g] = S->prof_n[g];
    }
    *count = kProfGroups;
    return SPH_OK;
}

sph_status sph_server_drain(sph_server *S, double timeout_s)
{
    if (!S) return sfail(SPH_ERR_ARG, "null argument");
    const double t0 = now_s();
    for (;;) {
        sph_status s = sph_server_pump(S, 64, nullptr);
        if (s != SPH_OK) return s;
        bool pending = false;
        for (auto &kv : S->tickets) pending = pending || kv.second->state != TK_DONE;
        if (!pending) return SPH_OK;
        if (!any_running(S) && S->queue.empty()) {
            // only retiring tickets left: wait for their copies
            cudaError_t e = cudaStreamQuery(S->st);
            if (e != cudaSuccess && e != cudaErrorNotReady) return sfail(SPH_ERR_CUDA, cudaGetErrorString(e));
            std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        if (timeout_s > 0.0 && now_s() - t0 > timeout_s) return sfail(SPH_ERR_TIMEOUT, "drain timed out");
    }
}

}  // extern "C"
