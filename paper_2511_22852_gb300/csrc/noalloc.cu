// noalloc.cu -- sph_density_noalloc: the cell list and kernel-sum densities
// (rows a1-a3) for callers that cannot allocate device memory.
//
// Who needs it: a caller that owns all of the GPU's free memory (for example a
// serving loop that admits events by free HBM and has handed the rest to its own
// pool), or code that runs while another thread captures a CUDA graph in global
// mode, where cudaMalloc is an illegal call.  Such a caller passes its own input
// and output buffers; every temporary this entry point needs lives in one
// file-scope device array of fixed size, set aside when the library is loaded.
//
// Limits and sharing rules:
//   * at most kMaxParticles particles and 2^kMaxBits cells of side 2h per axis;
//     larger inputs are rejected with SPH_ERR_ARG / SPH_ERR_STATE, never truncated;
//   * every GPU that loads the library holds the array (10,223,872 bytes) until exit;
//   * all calls share the one array: calls that overlap on the GPU (two streams,
//     two host threads) race on it -- serialise them;
//   * the first call on a device looks up the array's device address (once per
//     device, and again after the device's context was destroyed and recreated);
//     make that first call before any stream capture begins;
//   * the waits for the device are bounded (SPH_WAIT_LIMIT_S seconds, default 600):
//     a stream that does not drain gives SPH_ERR_TIMEOUT instead of blocking.
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>

#include "sph_gb300.h"
#include "sph_internal.cuh"

using namespace sphg;

namespace {

constexpr int kMaxParticles = SPH_NOALLOC_MAX_PARTICLES;
constexpr int kMaxBits = 8;                       // 256 x 256 cells
constexpr int kBuckets = 1 << (2 * kMaxBits);

constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// layout of the scratch array (byte offsets)
constexpr size_t kOffSc = 0;
constexpr size_t kOffKey = align256(kOffSc + sizeof(DevScalars));
constexpr size_t kOffTmp = align256(kOffKey + sizeof(uint32_t) * kMaxParticles);
constexpr size_t kOffPerm = align256(kOffTmp + sizeof(uint32_t) * kMaxParticles);
constexpr size_t kOffIdIn = align256(kOffPerm + sizeof(uint32_t) * kMaxParticles);
constexpr size_t kOffIdOut = align256(kOffIdIn + sizeof(int) * kMaxParticles);
constexpr size_t kOffNnb = align256(kOffIdOut + sizeof(int) * kMaxParticles);
constexpr size_t kOffCnt = align256(kOffNnb + sizeof(int) * kMaxParticles);
constexpr size_t kOffStart = align256(kOffCnt + sizeof(uint32_t) * kBuckets);
constexpr size_t kOffCursor = align256(kOffStart + sizeof(uint32_t) * kBuckets);
constexpr size_t kOffY = align256(kOffCursor + sizeof(uint32_t) * kBuckets);      // 5 rows: x, y, ux, uy, S
constexpr size_t kOffNq = align256(kOffY + sizeof(double) * 5 * kMaxParticles);    // 3 rows
constexpr size_t kOffDens = align256(kOffNq + sizeof(double) * 3 * kMaxParticles); // 6 rows
constexpr size_t kOffFpos = align256(kOffDens + sizeof(double) * 6 * kMaxParticles);
constexpr size_t kScratchBytes = align256(kOffFpos + sizeof(float2) * kMaxParticles);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// per device: the array's device address and the id of the context it was looked up in
void *g_base[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};
std::mutex g_mu;

sph_status nfail(sph_status s, const char *msg)
{
    sphg::set_last_error(msg);
    return s;
}

// Id of the calling thread's current context (driver entry points reached through the
// runtime, so the library needs no link-time dependence on the driver library).  A context
// that is destroyed and recreated (cudaDeviceReset) gets a new id; 0 when unavailable.
unsigned long long current_context_id()
{
    typedef int (*get_current_t)(void **);
    typedef int (*get_id_t)(void *, unsigned long long *);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<get_current_t>(f1);
            get_id = reinterpret_cast<get_id_t>(f2);
        }
        cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// waits for the stream with the library's bound on host waits
sph_status bounded_wait(cudaStream_t st)
{
    double limit = 600.0;
    if (const char *t = getenv("SPH_WAIT_LIMIT_S")) limit = atof(t);
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(st);
        if (e == cudaSuccess) return SPH_OK;
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            return nfail(SPH_ERR_CUDA, cudaGetErrorString(e));
        }
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > limit) return nfail(SPH_ERR_TIMEOUT, "device did not finish within the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 20 : 500));
    }
}

__global__ void k_iota(int *id, int n)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) id[i] = i;
}

// rest-frame densities back in input order: sigma*, s, n_B, n_S, n_Q
__global__ void k_unsort(const double *__restrict__ dens, const int *__restrict__ id, int n, double sqrtg,
                         double *__restrict__ out)
{
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double vol = dens[5 * (size_t)n + j] * sqrtg;
    int o = id[j];
    out[o] = dens[j];
    for (int r = 1; r < 5; ++r) out[(size_t)r * n + o] = dens[(size_t)r * n + j] / vol;
}

}  // namespace

extern "C" sph_status sph_density_noalloc(const double *x, const double *u, const double *S, const double *Nq,
                                          int64_t n, double h, double tau, int32_t milne, double *out, void *stream)
{
    if (n < 0 || n > kMaxParticles) return nfail(SPH_ERR_ARG, "n outside [0, SPH_NOALLOC_MAX_PARTICLES]");
    if (!(h > 0.0)) return nfail(SPH_ERR_ARG, "h must be positive");
    if (milne && !(tau > 0.0)) return nfail(SPH_ERR_ARG, "Milne coordinates need tau > 0");
    if (n == 0) return SPH_OK;
    if (!x || !u || !S || !Nq || !out) return nfail(SPH_ERR_ARG, "null buffer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return nfail(SPH_ERR_CUDA, "no current CUDA device");
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        unsigned long long ctx = current_context_id();
        if (!g_base[dev] || ctx != g_ctx_id[dev]) {
            // the array's name is a host-side stand-in: its device address comes from the runtime
            // (looked up again when the device's context was recreated)
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return nfail(SPH_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_base[dev] = p;
            g_ctx_id[dev] = ctx;
        }
        base = g_base[dev];
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t st = (cudaStream_t)stream;
    const int nn = (int)n;
    DevScalars *sc = reinterpret_cast<DevScalars *>(b + kOffSc);
    CellBufs cb{};
    cb.key = reinterpret_cast<uint32_t *>(b + kOffKey);
    cb.tmp = reinterpret_cast<uint32_t *>(b + kOffTmp);
    cb.perm = reinterpret_cast<uint32_t *>(b + kOffPerm);
    cb.cnt = reinterpret_cast<uint32_t *>(b + kOffCnt);
    cb.start = reinterpret_cast<uint32_t *>(b + kOffStart);
    cb.cursor = reinterpret_cast<uint32_t *>(b + kOffCursor);
    cb.fpos = reinterpret_cast<float2 *>(b + kOffFpos);
    cb.nb = kBuckets;
    int *id_in = reinterpret_cast<int *>(b + kOffIdIn);
    int *id_out = reinterpret_cast<int *>(b + kOffIdOut);
    int *nnb = reinterpret_cast<int *>(b + kOffNnb);
    double *ys = reinterpret_cast<double *>(b + kOffY);
    double *nqs = reinterpret_cast<double *>(b + kOffNq);
    double *dens = reinterpret_cast<double *>(b + kOffDens);

    EvView v;
    memset(&v, 0, sizeof(v));
    v.n = nn;
    v.dim = 2;
    v.milne = milne ? 1 : 0;
    v.nv = 5;
    v.B = kMaxBits;
    v.h = h;
    v.inv_h = 1.0 / h;
    double two_h = 2.0 * h;
    v.supp2 = two_h * two_h;
    v.inv_cell = 1.0 / (2.0 * h);
    prefilter_bounds(h, kMaxBits, 2, v.supp2_lo, v.supp2_hi);
    v.sigma_d = 10.0 / (7.0 * kPi * h * h);
    v.sc = sc;

    // the array keeps the previous call's contents: reset the flags and counters
    cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(SPH_ERR_CUDA, cudaGetErrorString(e));
    }
    k_iota<<<(nn + 255) / 256, 256, 0, st>>>(id_in, nn);
    launch_bbox(v, x, st);
    launch_cells(v, x, id_in, cb, st);
    {
        const double *src[4] = {x, u, S, Nq};
        double *dst[4] = {ys, ys + 2 * (size_t)nn, ys + 4 * (size_t)nn, nqs};
        int rows[4] = {2, 2, 1, 3};
        launch_permute(v, cb.perm, src, dst, rows, 4, id_in, id_out, st);
    }
    launch_density(v, ys, nqs, cb, dens, nnb, st);
    k_unsort<<<(nn + 255) / 256, 256, 0, st>>>(dens, id_out, nn, milne ? tau : 1.0, out);
    if ((e = cudaGetLastError()) != cudaSuccess) return nfail(SPH_ERR_CUDA, cudaGetErrorString(e));
    // the copy below goes to pageable memory, which blocks the host until the stream drained:
    // wait first, with the bound
    sph_status ws = bounded_wait(st);
    if (ws != SPH_OK) return ws;
    DevScalars hs;
    e = cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nfail(SPH_ERR_CUDA, cudaGetErrorString(e));
    }
    if ((ws = bounded_wait(st)) != SPH_OK) return ws;
    if (hs.err_flags & ERR_CELL_OVERFLOW)
        return nfail(SPH_ERR_STATE, "particles span more than 256 cells of side 2h along an axis");
    return SPH_OK;
}
