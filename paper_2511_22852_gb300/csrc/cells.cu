// cells.cu -- Morton-sorted cell list (rows a1, a2 of the step).
//
// Cells have side 2h, the support of the cubic spline kernel, so every
// neighbour of a particle lies in the 3^dim cells around its own (the binning
// of Sec. "Kokkos and Cabana", O(N) instead of O(N^2)).  Per stage:
//   bbox      min over particles of each coordinate (order-preserving integer
//             atomics: exact and order independent)
//   cells     cell coordinates floor((x - xmin)/(2h)), Morton key, bucket counts
//   scan      exclusive prefix sum of the bucket counts (one block)
//   scatter   particle -> provisional slot inside its bucket (atomic cursor)
//   rank      final slot = bucket start + number of bucket members with a smaller
//             original id: the order is (key, id), deterministic and stable
//   permute   gather of every per-particle array into the new order
#include "sph_internal.cuh"

namespace sphg {

namespace {

__global__ void k_bbox_init(DevScalars *sc)
{
    if (threadIdx.x < 3) sc->xmin_enc[threadIdx.x] = 0x7FF0000000000000LL;  // +inf
    if (threadIdx.x == 0) {
        sc->pair_flag = 0u;
        sc->eos_claim = 0u;
    }
}

__global__ void k_bbox(EvView v, const double *__restrict__ y)
{
    for (int d = 0; d < v.dim; ++d) {
        double m = __longlong_as_double(0x7FF0000000000000LL);
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += gridDim.x * blockDim.x)
            m = fmin(m, y[(size_t)d * v.n + i]);
        for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMin(&v.sc->xmin_enc[d], enc_double(m));
    }
}

__global__ void k_cells(EvView v, const double *__restrict__ y, uint32_t *key, uint32_t *cnt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= v.n) return;
    double xmin0 = dec_double(v.sc->xmin_enc[0]);
    double xmin1 = dec_double(v.sc->xmin_enc[1]);
    int cx = cell_coord(y[i], xmin0, v.inv_cell);
    int cy = cell_coord(y[(size_t)v.n + i], xmin1, v.inv_cell);
    int lim = 1 << v.B;
    if (cx >= lim || cy >= lim || cx < 0 || cy < 0) {
        atomicOr(&v.sc->err_flags, ERR_CELL_OVERFLOW);
        cx = min(max(cx, 0), lim - 1);
        cy = min(max(cy, 0), lim - 1);
    }
    uint32_t k = morton2((uint32_t)cx, (uint32_t)cy);
    key[i] = k;
    atomicAdd(&cnt[k], 1u);
}

// exclusive scan of nb counts with one block of 1024 threads, in tiles of 4096 buckets: thread t
// takes buckets 4t .. 4t + 3 of a tile (one 16-byte load and store when the arrays are 16-byte
// aligned), a warp-shuffle scan of the thread sums, and a carry from tile to tile
__global__ void __launch_bounds__(1024) k_scan(const uint32_t *__restrict__ cnt, uint32_t *start, uint32_t *cursor, int nb)
{
    __shared__ uint32_t warp_tot[32];
    __shared__ uint32_t tile_tot;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const bool vec = ((reinterpret_cast<uintptr_t>(cnt) | reinterpret_cast<uintptr_t>(start) |
                       reinterpret_cast<uintptr_t>(cursor)) & 15u) == 0;
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += 4096) {
        const int i0 = base + 4 * t;
        uint32_t v[4];
        if (vec && i0 + 3 < nb) {
            const uint4 q = *reinterpret_cast<const uint4 *>(cnt + i0);
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = i0 + k < nb ? cnt[i0 + k] : 0u;
        }
        const uint32_t local = v[0] + v[1] + v[2] + v[3];
        uint32_t incl = local;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t up = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += up;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (t < 32) {
            const uint32_t w = warp_tot[t];
            uint32_t wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t up = __shfl_up_sync(0xFFFFFFFFu, wi, o);
                if (t >= o) wi += up;
            }
            warp_tot[t] = wi - w;
            if (t == 31) tile_tot = wi;
        }
        __syncthreads();
        uint32_t r[4];
        r[0] = carry + warp_tot[wid] + incl - local;
        r[1] = r[0] + v[0];
        r[2] = r[1] + v[1];
        r[3] = r[2] + v[2];
        if (vec && i0 + 3 < nb) {
            const uint4 q = make_uint4(r[0], r[1], r[2], r[3]);
            *reinterpret_cast<uint4 *>(start + i0) = q;
            *reinterpret_cast<uint4 *>(cursor + i0) = q;
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (i0 + k < nb) start[i0 + k] = cursor[i0 + k] = r[k];
        }
        carry += tile_tot;
        __syncthreads();  // warp_tot and tile_tot are rewritten by the next tile
    }
}

// multi-block exclusive scan of large bucket tables: chunk sums, a scan of the chunk sums
// (one block), then each chunk rescanned with its offset
constexpr int kScanChunk = 4096;  // 256 threads x 16 buckets

__global__ void __launch_bounds__(256) k_scan_part(const uint32_t *__restrict__ cnt, uint32_t *part, int nb)
{
    __shared__ uint32_t sh[256];
    const int base = blockIdx.x * kScanChunk + threadIdx.x * 16;
    uint32_t acc = 0;
    for (int k = 0; k < 16; ++k)
        if (base + k < nb) acc += cnt[base + k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *part, int np)
{
    // np <= 4096: four consecutive values per thread, then a block scan of the thread sums
    __shared__ uint32_t warp_tot[32];
    const int t = threadIdx.x;
    uint32_t v[4], local = 0;
    for (int k = 0; k < 4; ++k) {
        int i = 4 * t + k;
        v[k] = i < np ? part[i] : 0u;
        local += v[k];
    }
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t up = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((t & 31) >= o) incl += up;
    }
    if ((t & 31) == 31) warp_tot[t >> 5] = incl;
    __syncthreads();
    if (t < 32) {
        uint32_t w = warp_tot[t], wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t up = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (t >= o) wi += up;
        }
        warp_tot[t] = wi - w;
    }
    __syncthreads();
    uint32_t run = warp_tot[t >> 5] + incl - local;
    for (int k = 0; k < 4; ++k) {
        int i = 4 * t + k;
        if (i < np) part[i] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(256) k_scan_apply(const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ part,
                                                    uint32_t *start, uint32_t *cursor, int nb)
{
    __shared__ uint32_t warp_tot[8];
    const int t = threadIdx.x;
    const int base = blockIdx.x * kScanChunk + t * 16;
    uint32_t local = 0;
    for (int k = 0; k < 16; ++k)
        if (base + k < nb) local += cnt[base + k];
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t up = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if ((t & 31) >= o) incl += up;
    }
    if ((t & 31) == 31) warp_tot[t >> 5] = incl;
    __syncthreads();
    if (t < 32) {
        uint32_t w = t < 8 ? warp_tot[t] : 0u, wi = w;
        for (int o = 1; o < 8; o <<= 1) {
            uint32_t up = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (t >= o) wi += up;
        }
        if (t < 8) warp_tot[t] = wi - w;
    }
    __syncthreads();
    uint32_t run = part[blockIdx.x] + warp_tot[t >> 5] + incl - local;
    for (int k = 0; k < 16; ++k)
        if (base + k < nb) {
            start[base + k] = run;
            cursor[base + k] = run;
            run += cnt[base + k];
        }
}

__global__ void k_scatter(int n, const uint32_t *__restrict__ key, uint32_t *cursor, uint32_t *tmp)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t slot = atomicAdd(&cursor[key[i]], 1u);
    tmp[slot] = (uint32_t)i;
}

__global__ void k_rank(int n, const uint32_t *__restrict__ key, const uint32_t *__restrict__ start,
                       const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ tmp, const int *__restrict__ id,
                       uint32_t *perm)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t i = tmp[j];
    uint32_t k = key[i];
    uint32_t s0 = start[k], c = cnt[k];
    int myid = id[i];
    uint32_t r = 0;
    for (uint32_t m = 0; m < c; ++m) r += (id[tmp[s0 + m]] < myid) ? 1u : 0u;
    perm[s0 + r] = i;
}

struct PermArgs {
    const double *src[8];
    double *dst[8];
    int rows[8];
    int ngroups;
};

__global__ void k_permute(int n, const uint32_t *__restrict__ perm, PermArgs a, const int *__restrict__ id_in,
                          int *id_out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t s = perm[j];
    for (int g = 0; g < a.ngroups; ++g)
        for (int r = 0; r < a.rows[g]; ++r) a.dst[g][(size_t)r * n + j] = a.src[g][(size_t)r * n + s];
    id_out[j] = id_in[s];
}

// neighbour pairs for the test interface: pass 1 counts (offs == nullptr), pass 2 writes
__global__ void k_neighbors(EvView v, const double *__restrict__ y, const int *__restrict__ id,
                            const uint32_t *__restrict__ start, const uint32_t *__restrict__ cnt,
                            const long long *__restrict__ offs, int *count_out, int *pa, int *pb)
{
    int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= v.n) return;
    const int n = v.n;
    double xa = y[a], ya = y[n + a];
    double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
    int cx = cell_coord(xa, xmin0, v.inv_cell), cy = cell_coord(ya, xmin1, v.inv_cell);
    int lim = 1 << v.B;
    long long w = offs ? offs[a] : 0;
    int c = 0;
    for (int oy = -1; oy <= 1; ++oy)
        for (int ox = -1; ox <= 1; ++ox) {
            int nx = cx + ox, ny = cy + oy;
            if (nx < 0 || ny < 0 || nx >= lim || ny >= lim) continue;
            uint32_t k = morton2((uint32_t)nx, (uint32_t)ny);
            uint32_t b0 = start[k], b1 = b0 + cnt[k];
            for (uint32_t b = b0; b < b1; ++b) {
                double r2 = dist2_2d(xa - y[b], ya - y[n + b]);
                if (r2 < v.supp2) {
                    if (offs) {
                        pa[w + c] = id[a];
                        pb[w + c] = id[b];
                    }
                    ++c;
                }
            }
        }
    if (!offs) count_out[a] = c;
}

__global__ void k_scan_counts(const int *__restrict__ cnt, long long *offs, int n)
{
    // one block; sequential chunks per thread, then a block scan of chunk sums
    __shared__ long long part[1024];
    int t = threadIdx.x, T = blockDim.x;
    int per = (n + T - 1) / T;
    int b0 = min(t * per, n), b1 = min(b0 + per, n);
    long long s = 0;
    for (int i = b0; i < b1; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        long long run = 0;
        for (int k = 0; k < T; ++k) {
            long long x = part[k];
            part[k] = run;
            run += x;
        }
    }
    __syncthreads();
    long long run = part[t];
    for (int i = b0; i < b1; ++i) {
        offs[i] = run;
        run += cnt[i];
    }
    if (t == T - 1) offs[n] = run;
}

__global__ void k_scatter_orig(const double *__restrict__ src, double *dst, const int *__restrict__ id, int n, int rows)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int o = id[j];
    for (int r = 0; r < rows; ++r) dst[(size_t)r * n + o] = src[(size_t)r * n + j];
}

__global__ void k_scatter_orig_u32(const uint32_t *__restrict__ src, uint32_t *dst, const int *__restrict__ id, int n)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    dst[id[j]] = src[j];
}

__global__ void k_cell_coords(EvView v, const double *__restrict__ y, const int *__restrict__ id, int *cell_orig)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= v.n) return;
    double xmin0 = dec_double(v.sc->xmin_enc[0]), xmin1 = dec_double(v.sc->xmin_enc[1]);
    int o = id[j];
    cell_orig[o] = cell_coord(y[j], xmin0, v.inv_cell);
    cell_orig[v.n + o] = cell_coord(y[v.n + j], xmin1, v.inv_cell);
}

inline int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

void launch_bbox(const EvView &v, const double *y, cudaStream_t st)
{
    k_bbox_init<<<1, 32, 0, st>>>(v.sc);
    int blocks = min(nblk(v.n, 256), 152 * 8);
    k_bbox<<<blocks, 256, 0, st>>>(v, y);
}

void launch_scan_buckets(CellBufs cb, cudaStream_t st)
{
    if (cb.nb <= 65536 || !cb.part) {
        k_scan<<<1, 1024, 0, st>>>(cb.cnt, cb.start, cb.cursor, cb.nb);
    } else {
        const int np = (cb.nb + kScanChunk - 1) / kScanChunk;
        k_scan_part<<<np, 256, 0, st>>>(cb.cnt, cb.part, cb.nb);
        k_scan_top<<<1, 1024, 0, st>>>(cb.part, np);
        k_scan_apply<<<np, 256, 0, st>>>(cb.cnt, cb.part, cb.start, cb.cursor, cb.nb);
    }
}

void launch_cells(const EvView &v, const double *y, const int *id, CellBufs cb, cudaStream_t st)
{
    cudaMemsetAsync(cb.cnt, 0, sizeof(uint32_t) * (size_t)cb.nb, st);
    if (v.dim == 3) launch_cells3(v, y, id, cb, st);
    else k_cells<<<nblk(v.n, 256), 256, 0, st>>>(v, y, cb.key, cb.cnt);
    launch_scan_buckets(cb, st);
    k_scatter<<<nblk(v.n, 256), 256, 0, st>>>(v.n, cb.key, cb.cursor, cb.tmp);
    k_rank<<<nblk(v.n, 128), 128, 0, st>>>(v.n, cb.key, cb.start, cb.cnt, cb.tmp, id, cb.perm);
}

void launch_permute(const EvView &v, const uint32_t *perm, const double *const *src, double *const *dst,
                    const int *nrows, int ngroups, const int *id_in, int *id_out, cudaStream_t st)
{
    PermArgs a;
    a.ngroups = ngroups;
    for (int g = 0; g < ngroups; ++g) {
        a.src[g] = src[g];
        a.dst[g] = dst[g];
        a.rows[g] = nrows[g];
    }
    k_permute<<<nblk(v.n, 256), 256, 0, st>>>(v.n, perm, a, id_in, id_out);
}

void launch_neighbors_list(const EvView &v, const double *y, const int *id, CellBufs cb, const long long *offs,
                           int *pa, int *pb, cudaStream_t st)
{
    // offs == nullptr: pa receives the per-particle counts
    if (v.dim == 3) {
        launch_neighbors_list3(v, y, id, cb, offs, pa, pb, st);
        return;
    }
    k_neighbors<<<nblk(v.n, 128), 128, 0, st>>>(v, y, id, cb.start, cb.cnt, offs, offs ? nullptr : pa, pa, pb);
}

void launch_scan_counts(const int *cnt, long long *offs, int n, cudaStream_t st)
{
    k_scan_counts<<<1, 1024, 0, st>>>(cnt, offs, n);
}

void launch_scatter_orig(const double *src, double *dst, const int *id, int n, int nrows, cudaStream_t st)
{
    k_scatter_orig<<<nblk(n, 256), 256, 0, st>>>(src, dst, id, n, nrows);
}

void launch_scatter_orig_u32(const uint32_t *src, uint32_t *dst, const int *id, int n, cudaStream_t st)
{
    k_scatter_orig_u32<<<nblk(n, 256), 256, 0, st>>>(src, dst, id, n);
}

void launch_cell_coords(const EvView &v, const double *y, const int *id, int *cell_orig, cudaStream_t st)
{
    if (v.dim == 3) {
        launch_cell_coords3(v, y, id, cell_orig, st);
        return;
    }
    k_cell_coords<<<nblk(v.n, 256), 256, 0, st>>>(v, y, id, cell_orig);
}

}  // namespace sphg
