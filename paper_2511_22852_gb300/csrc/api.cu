// api.cu -- the C ABI of include/sph_gb300.h: EoS and event handles, the
// per-stage launch sequence, CUDA-graph replay of whole steps, and read-out in
// the original particle order.
//
// One Heun step (two stages) on device buffers A/B (state), C/D (stage state):
//   stage 1: bbox(A) -> cells -> permute A -> B -> density(B) -> eos(B) ->
//            gradient(B) -> eom: C = B + dt f(B)
//   stage 2: bbox(C) -> cells -> permute C -> D and B -> A -> density(D) ->
//            eos(D) -> gradient(D) -> eom: A = ((A + D) + dt f(D)) / 2
// so the state is back in A after every step and the whole step can be captured
// once as a CUDA graph and replayed; tau and the work integral live in device
// memory and are advanced by the last kernel of the step.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sph_gb300.h"
#include "sph_internal.cuh"

using namespace sphg;

static thread_local std::string g_err;

static sph_status fail(sph_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

void sphg::set_last_error(const char *msg) { g_err = msg; }

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(SPH_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

struct sph_eos {
    EosDev dev;
    double *d_sn = nullptr, *d_p = nullptr;
    double *d_inv = nullptr, *d_p10 = nullptr;  // offline inverter (sph_eos_build_inverse)
    int refs = 1;
};

EosDev sphg::eos_params(const sph_eos *e) { return e->dev; }
void sphg::eos_retain(sph_eos *e) { e->refs++; }

struct sph_event {
    sph_eos *eos = nullptr;
    int n = 0, dim = 2, milne = 1, viscous = 0, npi = 3, nv = 9, B = 6;
    int B3[3] = {0, 0, 0};          // 3D: cell-coordinate bits per axis
    int ngin = kNGin, ngout = kNGout;  // rows of the gradient-pass inputs and outputs
    std::vector<uint32_t> spread_host;
    uint32_t *spread = nullptr;     // 3D: generalized Morton spread tables (3 x 1024)
    double h = 0.3, dtau = 0.01, tau0 = 0.0;
    int eos_offline = 0;            // 1: invert through the EoS handle's offline table
    int ntrack = 0;                 // jet tracks (sph_set_jets): device copy and Gaussian constants
    double *d_tracks = nullptr;
    double track_norm = 0.0, track_i2s2 = 0.0;
    int backup = 0;                 // conformal-diagonal backup EoS (sph_set_eos_backup)
    double cd_A0 = 0.0, cd_mu0[3] = {0.0, 0.0, 0.0};
    int nparton = 0;                // dynamical-initialisation partons (sph_set_partons), sorted by time
    double *d_partons = nullptr;
    long long parton_cap = 0;
    double parton_norm = 0.0, parton_h = 0.0;
    // charge sources of the partons (sph_set_partons with charges): their (B, S, Q) in the
    // partons' order, and the charges of the stage state (ping-pong with the sorts)
    bool charges = false;
    double *d_parton_q = nullptr;
    double *NqS[2] = {nullptr, nullptr};
    // BSQ diffusion (2+1D): kappa/T^2, tau T, and the per-stage scratch of the diffusion passes
    int diff = 0;
    double kapT2[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, tauJT[3] = {0, 0, 0};
    double *dinp = nullptr, *dal = nullptr, *dout = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevScalars *sc = nullptr;
    double *Y[2] = {nullptr, nullptr}, *Y1[2] = {nullptr, nullptr}, *Nq[2] = {nullptr, nullptr};
    int *id[2] = {nullptr, nullptr};
    double *Nq_orig = nullptr;
    CellBufs cb{};
    double *dens = nullptr, *eosf = nullptr, *gin = nullptr, *gout = nullptr;
    // EoS warm start: wguess (state order, carried across stages), guess_in (this stage's
    // sorted order), wguess_obs (written by read-out evaluations, which leave wguess alone)
    double *wguess = nullptr, *guess_in = nullptr, *wguess_obs = nullptr;
    // freeze-out surface (off until sph_freezeout_setup): e at the previous step's first stage
    // (ping-pong, permuted with the particles) and the element buffer
    bool fo_on = false;
    double e_fo = 0.0;
    double *eprev[2] = {nullptr, nullptr};
    FoBuf fo{};
    uint32_t *status = nullptr;
    int *nnb = nullptr;
    double *wpart = nullptr;
    int nwblk = 1;
    double *scratch = nullptr;  // read-out staging, rates, totals contributions
    double *ntot = nullptr;     // fixed-order sums of the charges (constant), + scratch
    double *tot = nullptr;      // totals scratch
    TransportDev tr{};
    uint32_t fatal_mask = 0;
    int mixed = 0;
    bool use_graph = false, graph_ready = false, observed = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    long long host_steps = 0;
    long long launches = 0;
    double timeout_s = 600.0;
    std::vector<void *> allocs;
    // half-pair lists of the plain 2D neighbour passes (cb.pl): sized on the first step from the
    // neighbour counts, grown after a stage whose lists overflowed (pair_ovf rose)
    int kernels_per_step = 0;  // kernel nodes of one captured step (0: not counted yet)
    bool pairs_off = false, pairs_grow = false;
    unsigned int pair_ovf_seen = 0;
    void *pair_mem = nullptr;
    int *pcnt[2] = {nullptr, nullptr};  // neighbour counts carried with the state (Y[0], Y1[0] order)
    // pinned copy of the device's overflow counter, refreshed after every sph_step call and read
    // (without a sync) at the next: the lists grow within a call of their first overflow
    volatile unsigned int *pair_ovf_host = nullptr;
    // profile mode: CUDA events around every kernel group of a step
    bool profile = false;
    std::vector<cudaEvent_t> pev;  // 2 per (group, stage)
    double prof_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    long long prof_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// kernel groups timed in profile mode
enum { G_CELLS = 0, G_PERMUTE, G_DENSITY, G_EOS, G_GRADIENT, G_EOM, G_WORK, G_COUNT };
static const char *kGroupNames[G_COUNT] = {"cells", "permute", "density", "eos", "gradient", "eom", "work"};

static inline void mark(sph_event *ev, int group, int stage, int end)
{
    if (!ev->profile) return;
    cudaEventRecord(ev->pev[(size_t)((group * 2 + (stage - 1)) * 2 + end)], ev->stream);
}

static EvView make_view(const sph_event *ev)
{
    EvView v;
    v.n = ev->n;
    v.dim = ev->dim;
    v.milne = ev->milne;
    v.nv = ev->nv;
    v.B = ev->B;
    for (int d = 0; d < 3; ++d) v.B3[d] = ev->B3[d];
    v.spread = ev->spread;
    v.h = ev->h;
    v.inv_h = 1.0 / ev->h;
    double two_h = 2.0 * ev->h;
    v.supp2 = two_h * two_h;
    v.inv_cell = 1.0 / (2.0 * ev->h);
    prefilter_bounds(ev->h, ev->B, ev->dim, v.supp2_lo, v.supp2_hi);
    v.mixed = ev->mixed;
    v.cell_f = (float)(2.0 * ev->h);
    if (ev->dim == 3) mixed_shell3(ev->h, v.shell_lo, v.shell_hi);
    else mixed_shell(ev->h, v.shell_lo, v.shell_hi);
    v.sigma_d = ev->dim == 2 ? 10.0 / (7.0 * kPi * ev->h * ev->h) : 1.0 / (kPi * ev->h * ev->h * ev->h);
    v.dtau = ev->dtau;
    v.sc = ev->sc;
    v.eos = ev->eos->dev;
    v.eos.offline = ev->eos_offline && ev->eos->dev.inv ? 1 : 0;
    if (ev->mixed) {
        // the mixed form's densities carry the FP32 sums' rounding (about 1e-7 of s): its
        // inversion stops at the serving form's tolerance, without the polishing step
        v.eos.polish = 0;
        v.eos.tol = std::max(v.eos.tol, 1e-10);
    }
    v.tr = ev->tr;
    v.eos.backup = ev->backup;
    v.eos.cd_A0 = ev->cd_A0;
    for (int q = 0; q < 3; ++q) v.eos.cd_mu0[q] = ev->cd_mu0[q];
    v.nparton = ev->nparton;
    v.partons = ev->d_partons;
    v.parton_norm = ev->parton_norm;
    v.parton_h = ev->parton_h;
    v.parton_sd = ev->parton_h > 0.0 ? (ev->dim == 2 ? 10.0 / (7.0 * kPi * ev->parton_h * ev->parton_h)
                                                     : 1.0 / (kPi * ev->parton_h * ev->parton_h * ev->parton_h))
                                     : 0.0;
    v.parton_dt = ev->dtau;
    v.parton_q = ev->charges ? ev->d_parton_q : nullptr;
    v.nq_cur = nullptr;  // set for the equations-of-motion launches under charge sources
    v.nq_out = nullptr;
    v.ntrack = ev->ntrack;
    v.tracks = ev->d_tracks;
    v.track_norm = ev->track_norm;
    v.track_i2s2 = ev->track_i2s2;
    v.diff = ev->diff;
    for (int k = 0; k < 9; ++k) v.kapT2[k] = ev->kapT2[k];
    for (int q = 0; q < 3; ++q) v.tauJT[q] = ev->tauJT[q];
    v.dinp = ev->dinp;
    v.dal = ev->dal;
    v.dout = ev->dout;
    return v;
}

static sph_status dalloc(sph_event *ev, void **p, size_t bytes)
{
    if (bytes == 0) bytes = 8;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SPH_ERR_OOM, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    ev->allocs.push_back(*p);
    return SPH_OK;
}

// ---------------------------------------------------------------------------
// launch sequences
static void enqueue_sort(sph_event *ev, const EvView &v, const double *ysrc, const int *idsrc)
{
    launch_bbox(v, ysrc, ev->stream);
    launch_cells(v, ysrc, idsrc, ev->cb, ev->stream);
}

// the cell buffers of a density pass: its pair-list rows are sized by the counts carried in
// pcnt[src]; it records its own counts in pcnt[dst] (dst < 0: not recorded, read-outs)
static CellBufs stage_cb(const sph_event *ev, int src, int dst)
{
    CellBufs cb = ev->cb;
    cb.pl.cnt_src = ev->pcnt[src];
    cb.pl.cnt_dst = dst >= 0 ? ev->pcnt[dst] : nullptr;
    return cb;
}

static void enqueue_step(sph_event *ev)
{
    EvView v = make_view(ev);
    cudaStream_t st = ev->stream;
    // stage 1
    mark(ev, G_CELLS, 1, 0);
    enqueue_sort(ev, v, ev->Y[0], ev->id[0]);
    mark(ev, G_CELLS, 1, 1);
    mark(ev, G_PERMUTE, 1, 0);
    {
        const double *src[4] = {ev->Y[0], ev->Nq[0], ev->wguess, ev->eprev[0]};
        double *dst[4] = {ev->Y[1], ev->Nq[1], ev->guess_in, ev->eprev[1]};
        int rows[4] = {ev->nv, 3, 4, 1};
        launch_permute(v, ev->cb.perm, src, dst, rows, ev->fo_on ? 4 : 3, ev->id[0], ev->id[1], st);
    }
    mark(ev, G_PERMUTE, 1, 1);
    mark(ev, G_DENSITY, 1, 0);
    launch_density(v, ev->Y[1], ev->Nq[1], stage_cb(ev, 0, 1), ev->dens, ev->nnb, st);
    mark(ev, G_DENSITY, 1, 1);
    mark(ev, G_EOS, 1, 0);
    launch_eos(v, 1, ev->Y[1], ev->dens, ev->eosf, ev->gin, ev->status, ev->wpart, ev->guess_in, ev->wguess, st);
    if (ev->fo_on)
        launch_freezeout(v, ev->e_fo, ev->Y[1], ev->id[1], ev->dens, ev->eosf, ev->eprev[1], ev->cb, ev->fo, st);
    launch_diffusion(v, 1, ev->Y[1], ev->dens, ev->eosf, ev->status, ev->cb, st);
    mark(ev, G_EOS, 1, 1);
    mark(ev, G_GRADIENT, 1, 0);
    launch_gradient(v, 1, ev->Y[1], ev->gin, ev->cb, ev->gout, st);
    mark(ev, G_GRADIENT, 1, 1);
    mark(ev, G_EOM, 1, 0);
    {
        EvView ve = v;  // under charge sources the stage-1 charges: NqS = Nq + dt dN
        if (ev->charges) ve.nq_cur = ev->Nq[1], ve.nq_out = ev->NqS[0];
        launch_eom(ve, 1, 0, ev->Y[1], ev->dens, ev->eosf, ev->gout, ev->Y1[0], nullptr, ev->status, st);
    }
    mark(ev, G_EOM, 1, 1);
    mark(ev, G_WORK, 1, 0);
    launch_work_finish(v, 1, ev->wpart, ev->nwblk, st);
    mark(ev, G_WORK, 1, 1);
    // stage 2
    mark(ev, G_CELLS, 2, 0);
    enqueue_sort(ev, v, ev->Y1[0], ev->id[1]);
    mark(ev, G_CELLS, 2, 1);
    mark(ev, G_PERMUTE, 2, 0);
    {
        const double *src[6] = {ev->Y1[0], ev->Y[1], ev->Nq[1], ev->wguess};
        double *dst[6] = {ev->Y1[1], ev->Y[0], ev->Nq[0], ev->guess_in};
        int rows[6] = {ev->nv, ev->nv, 3, 4};
        int ng = 4;
        if (ev->charges) src[ng] = ev->NqS[0], dst[ng] = ev->NqS[1], rows[ng++] = 3;
        if (ev->fo_on) src[ng] = ev->eprev[1], dst[ng] = ev->eprev[0], rows[ng++] = 1;
        launch_permute(v, ev->cb.perm, src, dst, rows, ng, ev->id[1], ev->id[0], st);
    }
    mark(ev, G_PERMUTE, 2, 1);
    mark(ev, G_DENSITY, 2, 0);
    // the stage state's charges: the stage-1 update under charge sources, else the constant ones
    launch_density(v, ev->Y1[1], ev->charges ? ev->NqS[1] : ev->Nq[0], stage_cb(ev, 1, 0), ev->dens, ev->nnb, st);
    mark(ev, G_DENSITY, 2, 1);
    mark(ev, G_EOS, 2, 0);
    launch_eos(v, 2, ev->Y1[1], ev->dens, ev->eosf, ev->gin, ev->status, ev->wpart, ev->guess_in, ev->wguess, st);
    launch_diffusion(v, 2, ev->Y1[1], ev->dens, ev->eosf, ev->status, ev->cb, st);
    mark(ev, G_EOS, 2, 1);
    mark(ev, G_GRADIENT, 2, 0);
    launch_gradient(v, 2, ev->Y1[1], ev->gin, ev->cb, ev->gout, st);
    mark(ev, G_GRADIENT, 2, 1);
    mark(ev, G_EOM, 2, 0);
    {
        EvView ve = v;  // under charge sources: Nq = ((Nq + NqS) + dt dN) / 2 in the stage-2 order
        if (ev->charges) ve.nq_cur = ev->NqS[1], ve.nq_out = ev->Nq[0];
        launch_eom(ve, 2, 1, ev->Y1[1], ev->dens, ev->eosf, ev->gout, ev->Y[0], nullptr, ev->status, st);
    }
    mark(ev, G_EOM, 2, 1);
    mark(ev, G_WORK, 2, 0);
    launch_work_finish(v, 2, ev->wpart, ev->nwblk, st);
    mark(ev, G_WORK, 2, 1);
}

// profile mode: wait for the step and add the group times
static sph_status collect_profile(sph_event *ev)
{
    CK(cudaStreamSynchronize(ev->stream));
    for (int g = 0; g < G_COUNT; ++g)
        for (int s = 0; s < 2; ++s) {
            float ms = 0.0f;
            size_t k = (size_t)((g * 2 + s) * 2);
            CK(cudaEventElapsedTime(&ms, ev->pev[k], ev->pev[k + 1]));
            ev->prof_ms[g] += ms;
            ev->prof_n[g] += 1;
        }
    return SPH_OK;
}

// cell list, densities and EoS at the current state, into the B buffers (sorted)
static void enqueue_observe(sph_event *ev)
{
    EvView v = make_view(ev);
    cudaStream_t st = ev->stream;
    enqueue_sort(ev, v, ev->Y[0], ev->id[0]);
    const double *src[3] = {ev->Y[0], ev->Nq[0], ev->wguess};
    double *dst[3] = {ev->Y[1], ev->Nq[1], ev->guess_in};
    int rows[3] = {ev->nv, 3, 4};
    launch_permute(v, ev->cb.perm, src, dst, rows, 3, ev->id[0], ev->id[1], st);
    launch_density(v, ev->Y[1], ev->Nq[1], stage_cb(ev, 0, -1), ev->dens, ev->nnb, st);
    launch_eos(v, 1, ev->Y[1], ev->dens, ev->eosf, ev->gin, ev->status, ev->wpart, ev->guess_in, ev->wguess_obs, st);
}

static sph_status wait_stream(sph_event *ev)
{
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery(ev->stream);
        if (e == cudaSuccess) return SPH_OK;
        if (e != cudaErrorNotReady) return fail(SPH_ERR_CUDA, std::string("stream: ") + cudaGetErrorString(e));
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > ev->timeout_s) return fail(SPH_ERR_TIMEOUT, "device did not finish within the wait limit");
        std::this_thread::sleep_for(std::chrono::microseconds(el < 0.01 ? 20 : 500));
    }
}

// device-to-host copy behind a bounded wait: a copy into pageable memory blocks the host until
// the stream has drained, so the stream is waited on (with the event's limit) before the copy
static sph_status fetch(sph_event *ev, void *dst, const void *src, size_t bytes)
{
    sph_status s = wait_stream(ev);
    if (s != SPH_OK) return s;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, ev->stream));
    return wait_stream(ev);
}

static sph_status check_device_flags(sph_event *ev, DevScalars *hs)
{
    sph_status s = fetch(ev, hs, ev->sc, sizeof(DevScalars));
    if (s != SPH_OK) return s;
    if (hs->pair_ovf > ev->pair_ovf_seen) {  // a stage overflowed the pair lists: grow them
        ev->pair_ovf_seen = hs->pair_ovf;
        ev->pairs_grow = true;
    }
    if (hs->err_flags & ERR_PAIR_LIST) return fail(SPH_ERR_STATE, "inconsistent neighbour pair lists");
    if (hs->err_flags & ERR_CELL_OVERFLOW)
        return fail(SPH_ERR_STATE, "particles spread beyond the cell table fixed at sph_init_event");
    uint32_t bad = hs->status_or & ev->fatal_mask;
    if (bad & PST_NONFINITE) return fail(SPH_ERR_NONFINITE, "non-finite state or rate");
    if (bad & PST_NOCONV) return fail(SPH_ERR_EOS_NOCONV, "EoS inversion without solution");
    if (bad & (PST_OUT_OF_TABLE | PST_FALLBACK)) return fail(SPH_ERR_EOS_RANGE, "particle outside the EoS table");
    if (bad) return fail(SPH_ERR_STATE, "fatal per-particle status");
    return SPH_OK;
}

// ---------------------------------------------------------------------------
extern "C" {

const char *sph_last_error(void) { return g_err.c_str(); }

sph_status sph_set_eos_table(sph_eos **out, const sph_eos_desc *d)
{
    if (!out || !d) return fail(SPH_ERR_ARG, "null argument");
    *out = nullptr;
    if (!(d->a0 > 0.0) || !(d->w_GeV > 0.0) || d->a1 < 0.0) return fail(SPH_ERR_ARG, "closed-form EoS needs a0 > 0, w > 0, a1 >= 0");
    for (int q = 0; q < 3; ++q)
        if (d->chi[q] < 0.0) return fail(SPH_ERR_ARG, "chi must be >= 0");
    sph_eos *e = new (std::nothrow) sph_eos();
    if (!e) return fail(SPH_ERR_OOM, "host allocation");
    EosDev &E = e->dev;
    memset(&E, 0, sizeof(E));
    E.a0 = d->a0;
    E.a1 = d->a1;
    E.Tc_GeV = d->Tc_GeV;
    E.w_GeV = d->w_GeV;
    for (int q = 0; q < 3; ++q) E.chi[q] = d->chi[q];
    E.tol = d->newton_tol > 0.0 ? d->newton_tol : 1e-12;
    E.maxit = d->newton_maxit > 0 ? d->newton_maxit : 30;
    E.polish = 1;
    E.has_table = d->has_table ? 1 : 0;
    if (E.has_table) {
        if (!d->p || !d->s || !d->nB || !d->nS || !d->nQ) {
            delete e;
            return fail(SPH_ERR_ARG, "table arrays must be non-null");
        }
        if (d->nT < 2 || d->nmu[0] < 2 || d->nmu[1] < 2 || d->nmu[2] < 2 || !(d->dT > 0.0) || !(d->dmu[0] > 0.0) ||
            !(d->dmu[1] > 0.0) || !(d->dmu[2] > 0.0)) {
            delete e;
            return fail(SPH_ERR_ARG, "table needs >= 2 nodes per axis and positive spacings");
        }
        E.nT = d->nT;
        E.T0 = d->T0;
        E.dT = d->dT;
        E.inv_dT = 1.0 / d->dT;
        E.Tmax = d->T0 + (d->nT - 1) * d->dT;
        for (int q = 0; q < 3; ++q) {
            E.nmu[q] = d->nmu[q];
            E.mu0[q] = d->mu0[q];
            E.dmu[q] = d->dmu[q];
            E.inv_dmu[q] = 1.0 / d->dmu[q];
            E.mumax[q] = d->mu0[q] + (d->nmu[q] - 1) * d->dmu[q];
        }
        size_t nn = (size_t)d->nT * d->nmu[0] * d->nmu[1] * d->nmu[2];
        std::vector<double> sn(4 * nn);
        for (size_t i = 0; i < nn; ++i) {
            sn[4 * i] = d->s[i];
            sn[4 * i + 1] = d->nB[i];
            sn[4 * i + 2] = d->nS[i];
            sn[4 * i + 3] = d->nQ[i];
        }
        cudaError_t c1 = cudaMalloc(&e->d_sn, sizeof(double) * 4 * nn);
        cudaError_t c2 = cudaMalloc(&e->d_p, sizeof(double) * nn);
        if (c1 != cudaSuccess || c2 != cudaSuccess) {
            cudaGetLastError();
            if (e->d_sn) cudaFree(e->d_sn);
            if (e->d_p) cudaFree(e->d_p);
            delete e;
            return fail(SPH_ERR_OOM, "cudaMalloc of the EoS table failed");
        }
        cudaError_t c3 = cudaMemcpy(e->d_sn, sn.data(), sizeof(double) * 4 * nn, cudaMemcpyHostToDevice);
        cudaError_t c4 = cudaMemcpy(e->d_p, d->p, sizeof(double) * nn, cudaMemcpyHostToDevice);
        if (c3 != cudaSuccess || c4 != cudaSuccess) {
            cudaFree(e->d_sn);
            cudaFree(e->d_p);
            delete e;
            return fail(SPH_ERR_CUDA, "copy of the EoS table failed");
        }
        E.sn = e->d_sn;
        E.p = e->d_p;
    }
    *out = e;
    return SPH_OK;
}

void sph_free_eos(sph_eos *e)
{
    if (!e) return;
    if (--e->refs > 0) return;
    if (e->d_sn) cudaFree(e->d_sn);
    if (e->d_p) cudaFree(e->d_p);
    if (e->d_inv) cudaFree(e->d_inv);
    if (e->d_p10) cudaFree(e->d_p10);
    delete e;
}

void sph_free_event(sph_event *ev)
{
    if (!ev) return;
    if (ev->stream) cudaStreamSynchronize(ev->stream);
    if (ev->gexec) cudaGraphExecDestroy(ev->gexec);
    if (ev->graph) cudaGraphDestroy(ev->graph);
    for (cudaEvent_t e : ev->pev) cudaEventDestroy(e);
    for (void *p : ev->allocs) cudaFree(p);
    if (ev->pair_mem) cudaFree(ev->pair_mem);
    if (ev->pair_ovf_host) cudaFreeHost((void *)ev->pair_ovf_host);
    if (ev->own_stream && ev->stream) cudaStreamDestroy(ev->stream);
    sph_free_eos(ev->eos);
    delete ev;
}

sph_status sph_init_event(sph_event **out, const sph_event_desc *d, const sph_eos *eos)
{
    if (!out || !d || !eos) return fail(SPH_ERR_ARG, "null argument");
    *out = nullptr;
    if (d->dim != 2 && d->dim != 3) return fail(SPH_ERR_ARG, "dim must be 2 or 3");
    if (d->n < 0 || d->n > 0x7FFFFFFF) return fail(SPH_ERR_ARG, "n out of range");
    if (!(d->h > 0.0) || !(d->dtau > 0.0)) return fail(SPH_ERR_ARG, "h and dtau must be positive");
    if (d->milne && !(d->tau0 > 0.0)) return fail(SPH_ERR_ARG, "Milne coordinates need tau0 > 0");
    if (d->n > 0 && (!d->x || !d->u || !d->S || !d->Nq)) return fail(SPH_ERR_ARG, "null particle array");
    if (d->viscous && (!(d->tau_pi_coef > 0.0) || !(d->tau_Pi_ratio > 0.0) || !(d->eta_over_s > 0.0)))
        return fail(SPH_ERR_ARG, "viscous run needs eta_over_s, tau_pi_coef, tau_Pi_ratio > 0");
    sph_event *ev = new (std::nothrow) sph_event();
    if (!ev) return fail(SPH_ERR_OOM, "host allocation");
    ev->eos = const_cast<sph_eos *>(eos);
    ev->eos->refs++;
    ev->n = (int)d->n;
    ev->dim = d->dim;
    ev->milne = d->milne ? 1 : 0;
    ev->viscous = d->viscous ? 1 : 0;
    ev->npi = ev->dim == 2 ? 3 : 5;
    ev->nv = 2 * ev->dim + 2 + ev->npi;
    if (d->kappaT2) {
        bool ok = ev->dim == 2 && d->tauJT != nullptr;
        for (int k = 0; ok && k < 9; ++k) ok = std::isfinite(d->kappaT2[k]);
        for (int q = 0; ok && q < 3; ++q) ok = std::isfinite(d->tauJT[q]) && d->tauJT[q] > 0.0;
        if (!ok) {
            sph_free_event(ev);
            return fail(SPH_ERR_ARG, "diffusion needs dim = 2, finite kappa/T^2 and positive tau T");
        }
        ev->diff = 1;
        for (int k = 0; k < 9; ++k) ev->kapT2[k] = d->kappaT2[k];
        for (int q = 0; q < 3; ++q) ev->tauJT[q] = d->tauJT[q];
        ev->nv += 6;  // J^i_q / sigma
    }
    ev->ngin = ev->dim == 2 ? kNGin : 12;
    ev->ngout = ev->dim == 2 ? kNGout : 12;
    ev->h = d->h;
    ev->dtau = d->dtau;
    ev->tau0 = d->tau0;
    ev->fatal_mask = d->fatal_mask;
    if (d->precision != SPH_FP64 && d->precision != SPH_MIXED) {
        sph_free_event(ev);
        return fail(SPH_ERR_ARG, "precision must be SPH_FP64 or SPH_MIXED");
    }
    ev->mixed = d->precision == SPH_MIXED ? 1 : 0;
    ev->profile = d->profile != 0;
    ev->use_graph = d->use_graph != 0 && !ev->profile;
    if (ev->profile) {
        ev->pev.resize(G_COUNT * 2 * 2);
        for (auto &e : ev->pev)
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
                sph_free_event(ev);
                return fail(SPH_ERR_CUDA, "cudaEventCreate failed");
            }
    }
    ev->tr.viscous = ev->viscous;
    ev->tr.eta_over_s = d->eta_over_s;
    ev->tr.zeta_peak = d->zeta_peak;
    ev->tr.zeta_T_GeV = d->zeta_T_GeV;
    ev->tr.zeta_w_GeV = d->zeta_w_GeV > 0.0 ? d->zeta_w_GeV : 1.0;
    ev->tr.tau_pi_coef = d->tau_pi_coef;
    ev->tr.tau_Pi_ratio = d->tau_Pi_ratio;
    ev->tr.cs2_cap = d->cs2_cap > 0.0 ? d->cs2_cap : 1.0;
    ev->tr.T_stop_GeV = d->T_stop_GeV > 0.0 ? d->T_stop_GeV : 0.0;
    if (const char *t = getenv("SPH_WAIT_LIMIT_S")) ev->timeout_s = atof(t);
    auto bail = [&](sph_status s) {
        std::string keep = g_err;
        sph_free_event(ev);
        g_err = keep;
        return s;
    };
    if (d->stream) {
        ev->stream = (cudaStream_t)d->stream;
    } else {
        if (cudaStreamCreateWithFlags(&ev->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(SPH_ERR_CUDA, "cudaStreamCreate failed"));
        }
        ev->own_stream = true;
    }
    const int n = ev->n;
    const size_t N = (size_t)(n > 0 ? n : 1);
    // cell table: 2^B cells per axis, four times the initial extent
    std::vector<double> hx((size_t)ev->dim * N, 0.0);
    if (n > 0) {
        cudaMemcpyKind k = d->on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        if (cudaMemcpy(hx.data(), d->x, sizeof(double) * ev->dim * n, k) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(SPH_ERR_ARG, "cannot read positions"));
        }
    }
    int ncmax = 1, nc[3] = {1, 1, 1};
    for (int dd = 0; dd < ev->dim; ++dd) {
        double lo = INFINITY, hi = -INFINITY;
        for (int i = 0; i < n; ++i) {
            double xv = hx[(size_t)dd * n + i];
            if (!std::isfinite(xv)) return bail(fail(SPH_ERR_NONFINITE, "non-finite position"));
            lo = std::min(lo, xv);
            hi = std::max(hi, xv);
        }
        if (n > 0) nc[dd] = (int)std::floor((hi - lo) / (2.0 * ev->h)) + 1;
        ncmax = std::max(ncmax, nc[dd]);
    }
    if (ev->dim == 2) {
        int B = 3;
        while ((1 << B) < 4 * ncmax && B < 15) ++B;
        if ((1 << B) < ncmax) return bail(fail(SPH_ERR_ARG, "domain too large for the cell table"));
        ev->B = B;
        ev->cb.nb = 1 << (2 * B);
    } else {
        // per-axis bits: room for 4x the initial extent (2x when that exceeds 2^24 buckets)
        for (int margin = 4; margin >= 1; margin /= 2) {
            int tot = 0;
            for (int dd = 0; dd < 3; ++dd) {
                int b = 2;
                while ((1 << b) < margin * nc[dd] && b < 10) ++b;
                ev->B3[dd] = b;
                tot += b;
            }
            if (tot <= 24 || margin == 1) break;
        }
        int tot = ev->B3[0] + ev->B3[1] + ev->B3[2];
        for (int dd = 0; dd < 3; ++dd)
            if ((1 << ev->B3[dd]) < nc[dd] || tot > 24) return bail(fail(SPH_ERR_ARG, "domain too large for the cell table"));
        ev->B = std::max(ev->B3[0], std::max(ev->B3[1], ev->B3[2]));
        ev->cb.nb = 1 << tot;
        // generalized Morton key: bit b of axis d goes to the next free key bit, axes in turn
        ev->spread_host.assign(3 * 1024, 0u);
        int pos = 0;
        for (int b = 0; b < 10; ++b)
            for (int dd = 0; dd < 3; ++dd)
                if (b < ev->B3[dd]) {
                    for (int c = 0; c < (1 << ev->B3[dd]); ++c)
                        if ((c >> b) & 1) ev->spread_host[(size_t)dd * 1024 + c] |= 1u << pos;
                    ++pos;
                }
    }
    sph_status s;
#define AL(ptr, bytes)                                                    \
    do {                                                                  \
        if ((s = dalloc(ev, (void **)&(ptr), (bytes))) != SPH_OK) return bail(s); \
    } while (0)
    const size_t dv = sizeof(double) * N;
    AL(ev->sc, sizeof(DevScalars));
    for (int b = 0; b < 2; ++b) {
        AL(ev->Y[b], dv * ev->nv);
        AL(ev->Y1[b], dv * ev->nv);
        AL(ev->Nq[b], dv * 3);
        AL(ev->id[b], sizeof(int) * N);
    }
    AL(ev->Nq_orig, dv * 3);
    AL(ev->cb.key, sizeof(uint32_t) * N);
    AL(ev->cb.tmp, sizeof(uint32_t) * N);
    AL(ev->cb.perm, sizeof(uint32_t) * N);
    if (ev->dim == 2) AL(ev->cb.fpos, sizeof(float2) * N);
    else AL(ev->cb.fpos3, sizeof(float4) * N);
    AL(ev->cb.part, sizeof(uint32_t) * (size_t)(ev->cb.nb / 4096 + 2));
    if (ev->dim == 3) AL(ev->spread, sizeof(uint32_t) * 3 * 1024);
    AL(ev->cb.cnt, sizeof(uint32_t) * (size_t)ev->cb.nb);
    AL(ev->cb.start, sizeof(uint32_t) * (size_t)ev->cb.nb);
    AL(ev->cb.cursor, sizeof(uint32_t) * (size_t)ev->cb.nb);
    AL(ev->dens, dv * kNDens);
    AL(ev->eosf, dv * kNEos);
    AL(ev->gin, dv * ev->ngin);
    AL(ev->gout, dv * ev->ngout);
    AL(ev->wguess, dv * 4);
    AL(ev->guess_in, dv * 4);
    AL(ev->wguess_obs, dv * 4);
    AL(ev->status, sizeof(uint32_t) * N);
    AL(ev->nnb, sizeof(int) * N);
    ev->nwblk = eos_block_count(n > 0 ? n : 1, ev->dim);
    AL(ev->wpart, sizeof(double) * (size_t)ev->nwblk);
    AL(ev->scratch, dv * std::max(std::max(ev->nv, kNEos), ev->ngout));
    if (ev->diff) {  // the charges evolve (the lab charges); the diffusion passes' scratch
        for (int k = 0; k < 2; ++k) AL(ev->NqS[k], dv * 3);
        AL(ev->dinp, dv * 9);
        AL(ev->dal, dv * 12);
        AL(ev->dout, dv * 9);
        ev->charges = true;
    }
    AL(ev->ntot, sizeof(double) * (8 + 3 * 256));
    AL(ev->tot, sizeof(double) * (8 + 3 * 256));
#undef AL
    cudaStream_t st = ev->stream;
    if (n > 0) {
        cudaMemcpyKind k = d->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        size_t dn = sizeof(double) * n;
        CK(cudaMemcpyAsync(ev->Y[0], d->x, dn * ev->dim, k, st));
        CK(cudaMemcpyAsync(ev->Y[0] + (size_t)ev->dim * n, d->u, dn * ev->dim, k, st));
        CK(cudaMemcpyAsync(ev->Y[0] + (size_t)2 * ev->dim * n, d->S, dn, k, st));
        if (d->Bv) CK(cudaMemcpyAsync(ev->Y[0] + (size_t)(2 * ev->dim + 1) * n, d->Bv, dn, k, st));
        else CK(cudaMemsetAsync(ev->Y[0] + (size_t)(2 * ev->dim + 1) * n, 0, dn, st));
        if (d->Pv) CK(cudaMemcpyAsync(ev->Y[0] + (size_t)(2 * ev->dim + 2) * n, d->Pv, dn * ev->npi, k, st));
        else CK(cudaMemsetAsync(ev->Y[0] + (size_t)(2 * ev->dim + 2) * n, 0, dn * ev->npi, st));
        if (ev->diff) {
            if (d->Jv) CK(cudaMemcpyAsync(ev->Y[0] + (size_t)kJRow * n, d->Jv, dn * 6, k, st));
            else CK(cudaMemsetAsync(ev->Y[0] + (size_t)kJRow * n, 0, dn * 6, st));
        }
        CK(cudaMemcpyAsync(ev->Nq[0], d->Nq, dn * 3, k, st));
        CK(cudaMemcpyAsync(ev->Nq_orig, d->Nq, dn * 3, k, st));
        CK(cudaMemsetAsync(ev->wguess, 0, dn * 4, st));
        std::vector<int> iota(n);
        for (int i = 0; i < n; ++i) iota[i] = i;
        CK(cudaMemcpyAsync(ev->id[0], iota.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
        if (!ev->viscous) {  // an ideal fluid carries no dissipative state
            CK(cudaMemsetAsync(ev->Y[0] + (size_t)(2 * ev->dim + 1) * n, 0, dn * (1 + ev->npi), st));
        }
        launch_sum_fixed(ev->Nq_orig, n, 3, ev->ntot, st);
    }
    if (ev->dim == 3)
        CK(cudaMemcpyAsync(ev->spread, ev->spread_host.data(), sizeof(uint32_t) * 3 * 1024, cudaMemcpyHostToDevice, st));
    DevScalars hs;
    memset(&hs, 0, sizeof(hs));
    hs.tau = d->tau0;
    CK(cudaMemcpyAsync(ev->sc, &hs, sizeof(hs), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    *out = ev;
    return SPH_OK;
}

// Sizes (or grows) the half-pair lists of the plain passes (2D and 3D).  Each stage gives particle a a row
// of (its previous neighbour count - 1 + margin) entries; the allocation holds 1.5 x those rows
// for the current state (at least 1.5 x the old allocation when growing), margin = 32.  Counts
// are carried from stage to stage in the state order (pcnt[0] with Y[0], pcnt[1] with Y1[0]);
// here they are taken from a read-out evaluation of the current state.  The lists stay off (the
// per-particle passes run) for other forms, when SPH_PAIR_LISTS=0, or when they would take more
// than a quarter of the free device memory.  SPH_PAIR_MARGIN and SPH_PAIR_TOTAL override the
// margin and the first allocation (tests of the overflow paths).
static sph_status size_pair_lists(sph_event *ev)
{
    if (ev->pairs_off || ev->mixed || ev->n == 0) return SPH_OK;
    if (ev->cb.pl.total > 0 && ev->pair_ovf_host && *ev->pair_ovf_host > ev->pair_ovf_seen) {
        ev->pair_ovf_seen = *ev->pair_ovf_host;
        ev->pairs_grow = true;
    }
    if (ev->cb.pl.total > 0 && !ev->pairs_grow) return SPH_OK;
    if (const char *t = getenv("SPH_PAIR_LISTS"))
        if (atoi(t) == 0) {
            ev->pairs_off = true;
            return SPH_OK;
        }
    const int n = ev->n;
    int margin = 32;
    if (const char *t = getenv("SPH_PAIR_MARGIN")) margin = std::max(0, atoi(t));
    // neighbour counts of the current state, moved from the evaluation's sorted order to the state
    // order (the sort's gather map: sorted j <- state perm[j])
    enqueue_observe(ev);
    CK(cudaGetLastError());
    ev->observed = true;
    std::vector<int> cnt(n), perm(n), state(n);
    sph_status s = fetch(ev, cnt.data(), ev->nnb, sizeof(int) * (size_t)n);
    if (s != SPH_OK) return s;
    if ((s = fetch(ev, perm.data(), ev->cb.perm, sizeof(int) * (size_t)n)) != SPH_OK) return s;
    long long rows = 0;
    for (int j = 0; j < n; ++j) {
        state[perm[j]] = cnt[j];
        rows += std::max(cnt[j] - 1, 0) + margin;
    }
    long long total = rows * 3 / 2 + 1024;
    if (ev->pairs_grow) total = std::max<long long>(total, ev->cb.pl.total * 3 / 2);
    else if (const char *t = getenv("SPH_PAIR_TOTAL")) total = std::max<long long>(1, atoll(t));
    const int nparts = (n + 2047) / 2048;
    // per entry: L, P (int), W and the kernel gradient (2 or 3 doubles)
    const size_t per_entry = 2 * sizeof(int) + (1 + (size_t)ev->dim) * sizeof(double);
    const size_t bytes = (size_t)total * per_entry + (size_t)(n + 1) * sizeof(long long) +
                         (size_t)nparts * sizeof(unsigned long long) + 4 * sizeof(int) * (size_t)n + 1024;
    size_t fr = 0, tot = 0;
    CK(cudaMemGetInfo(&fr, &tot));
    if (bytes > fr / 4) {
        ev->pairs_off = true;
        ev->pairs_grow = false;
        return SPH_OK;
    }
    if ((s = wait_stream(ev)) != SPH_OK) return s;  // the old lists may still be in use
    if (ev->pair_mem) {
        cudaFree(ev->pair_mem);
        ev->pair_mem = nullptr;
        ev->cb.pl = PairBufs{};
    }
    void *m = nullptr;
    if (cudaMalloc(&m, bytes) != cudaSuccess) {
        cudaGetLastError();
        ev->pairs_off = true;
        ev->pairs_grow = false;
        return SPH_OK;
    }
    ev->pair_mem = m;
    PairBufs pl{};
    pl.total = total;
    pl.margin = margin;
    double *gbuf = static_cast<double *>(m);  // the kernel gradients first (16-byte aligned)
    if (ev->dim == 2) pl.G = reinterpret_cast<double2 *>(gbuf);
    else pl.G3 = gbuf;
    pl.W = gbuf + (size_t)ev->dim * total;
    pl.off = reinterpret_cast<long long *>(pl.W + total);
    pl.part = reinterpret_cast<unsigned long long *>(pl.off + (n + 1));
    pl.L = reinterpret_cast<int *>(pl.part + nparts);
    pl.P = pl.L + total;
    pl.cntF = pl.P + total;
    pl.cntB = pl.cntF + n;
    ev->pcnt[0] = pl.cntB + n;
    ev->pcnt[1] = ev->pcnt[0] + n;
    CK(cudaMemcpyAsync(ev->pcnt[0], state.data(), sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, ev->stream));
    if ((s = wait_stream(ev)) != SPH_OK) return s;
    pl.cnt_src = ev->pcnt[0];
    ev->cb.pl = pl;
    ev->pairs_grow = false;
    ev->kernels_per_step = 0;
    if (!ev->pair_ovf_host) {
        void *hp = nullptr;
        if (cudaHostAlloc(&hp, sizeof(unsigned int), cudaHostAllocDefault) == cudaSuccess) {
            ev->pair_ovf_host = static_cast<volatile unsigned int *>(hp);
            *ev->pair_ovf_host = ev->pair_ovf_seen;
        } else {
            cudaGetLastError();
        }
    }
    // the captured step holds the old buffers
    if (ev->gexec) cudaGraphExecDestroy(ev->gexec);
    if (ev->graph) cudaGraphDestroy(ev->graph);
    ev->gexec = nullptr;
    ev->graph = nullptr;
    ev->graph_ready = false;
    return SPH_OK;
}

static int kernel_nodes(cudaGraph_t g)
{
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return 0;
    int k = 0;
    for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// kernels launched by one step: counted on a capture of the step's launch sequence
static sph_status count_step_kernels(sph_event *ev)
{
    if (ev->kernels_per_step > 0) return SPH_OK;
    if (ev->graph) {
        ev->kernels_per_step = kernel_nodes(ev->graph);
        return SPH_OK;
    }
    CK(cudaStreamBeginCapture(ev->stream, cudaStreamCaptureModeThreadLocal));
    const bool prof = ev->profile;
    ev->profile = false;  // no event records in the counting capture
    enqueue_step(ev);
    ev->profile = prof;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ev->stream, &g);
    if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    ev->kernels_per_step = kernel_nodes(g);
    cudaGraphDestroy(g);
    return SPH_OK;
}

sph_status sph_step(sph_event *ev, int32_t nsteps, uint32_t flags)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (nsteps < 0) return fail(SPH_ERR_ARG, "nsteps < 0");
    if (ev->n == 0 || nsteps == 0) return SPH_OK;
    {
        sph_status s = size_pair_lists(ev);
        if (s != SPH_OK) return s;
    }
    if (ev->use_graph && !ev->graph_ready) {
        CK(cudaStreamBeginCapture(ev->stream, cudaStreamCaptureModeThreadLocal));
        enqueue_step(ev);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(ev->stream, &g);
        if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        ev->graph = g;
        CK(cudaGraphInstantiate(&ev->gexec, g, 0));
        ev->graph_ready = true;
    }
    for (int k = 0; k < nsteps; ++k) {
        if (ev->use_graph) {
            CK(cudaGraphLaunch(ev->gexec, ev->stream));
        } else {
            enqueue_step(ev);
            if (ev->profile) {
                sph_status s = collect_profile(ev);
                if (s != SPH_OK) return s;
            }
        }
    }
    CK(cudaGetLastError());
    if (ev->cb.pl.total > 0 && ev->pair_ovf_host)  // picked up by the next call
        CK(cudaMemcpyAsync((void *)ev->pair_ovf_host, &ev->sc->pair_ovf, sizeof(unsigned int),
                           cudaMemcpyDeviceToHost, ev->stream));
    ev->host_steps += nsteps;
    {
        sph_status s = count_step_kernels(ev);
        if (s != SPH_OK) return s;
    }
    ev->launches += (long long)nsteps * ev->kernels_per_step;
    ev->observed = false;
    if (flags & SPH_SYNC) {
        DevScalars hs;
        return check_device_flags(ev, &hs);
    }
    return SPH_OK;
}

static sph_status copy_out(sph_event *ev, void *dst, const void *src, size_t bytes, int on_device)
{
    if (!on_device) return fetch(ev, dst, src, bytes);
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, ev->stream));
    return wait_stream(ev);
}

sph_status sph_read_fields(sph_event *ev, uint64_t mask, const sph_field_bufs *o, sph_totals *tot)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (mask && !o) return fail(SPH_ERR_ARG, "null buffers");
    const int n = ev->n;
    const size_t dn = sizeof(double) * (size_t)n;
    cudaStream_t st = ev->stream;
    const uint64_t derived = SPH_F_SIGMA_STAR | SPH_F_S_DENS | SPH_F_N_DENS | SPH_F_T | SPH_F_MU | SPH_F_P | SPH_F_E |
                             SPH_F_PI_BULK | SPH_F_STATUS | SPH_F_NNB | SPH_F_CELL;
    if (n > 0 && ((mask & derived) || tot) && !ev->observed) {
        enqueue_observe(ev);
        CK(cudaGetLastError());
        ev->observed = true;
    }
    struct Row {
        uint64_t bit;
        double *dst;
        const double *src;
        int rows;
        int state;  // 1: from the state buffer (id[0]); 0: derived (id[1])
    };
    double *dens = ev->dens, *eo = ev->eosf;
    const size_t N = (size_t)n;
    std::vector<Row> rows = {
        {SPH_F_X, o ? o->x : nullptr, ev->Y[0], ev->dim, 1},
        {SPH_F_U, o ? o->u : nullptr, ev->Y[0] + ev->dim * N, ev->dim, 1},
        {SPH_F_S, o ? o->S : nullptr, ev->Y[0] + 2 * ev->dim * N, 1, 1},
        {SPH_F_NQ, o ? o->Nq : nullptr, ev->Nq[0], 3, 1},
        {SPH_F_BV, o ? o->Bv : nullptr, ev->Y[0] + (2 * ev->dim + 1) * N, 1, 1},
        {SPH_F_PV, o ? o->Pv : nullptr, ev->Y[0] + (2 * ev->dim + 2) * N, ev->npi, 1},
        {SPH_F_GUESS, o ? o->guess : nullptr, ev->wguess, 4, 1},
        {SPH_F_JV, o ? o->Jv : nullptr, ev->Y[0] + (size_t)kJRow * N, ev->diff ? 6 : 0, 1},
        {SPH_F_SIGMA_STAR, o ? o->sigstar : nullptr, dens, 1, 0},
        {SPH_F_S_DENS, o ? o->s : nullptr, dens + N, 1, 0},
        {SPH_F_N_DENS, o ? o->nq : nullptr, dens + 2 * N, 3, 0},
        {SPH_F_T, o ? o->T : nullptr, eo, 1, 0},
        {SPH_F_MU, o ? o->mu : nullptr, eo + N, 3, 0},
        {SPH_F_P, o ? o->p : nullptr, eo + 4 * N, 1, 0},
        {SPH_F_E, o ? o->e : nullptr, eo + 5 * N, 1, 0},
    };
    if ((mask & SPH_F_JV) && !ev->diff) return fail(SPH_ERR_ARG, "the event has no diffusion currents");
    for (auto &r : rows) {
        if (!(mask & r.bit)) continue;
        if (!r.dst) return fail(SPH_ERR_ARG, "requested field has a null destination");
        if (n == 0) continue;
        launch_scatter_orig(r.src, ev->scratch, r.state ? ev->id[0] : ev->id[1], n, r.rows, st);
        sph_status s = copy_out(ev, r.dst, ev->scratch, dn * r.rows, o->on_device);
        if (s != SPH_OK) return s;
    }
    if (mask & SPH_F_PI_BULK) {
        if (!o->Pi) return fail(SPH_ERR_ARG, "requested field has a null destination");
        if (n > 0) {
            // Pi = sigma * (Pi/sigma) with sigma = sigma* / (u^0 sqrt(-g)), on the host side of the copy
            std::vector<double> bv(n), sg(n), u0(n);
            launch_scatter_orig(ev->Y[1] + (2 * ev->dim + 1) * N, ev->scratch, ev->id[1], n, 1, st);
            sph_status s = copy_out(ev, bv.data(), ev->scratch, dn, 0);
            if (s != SPH_OK) return s;
            launch_scatter_orig(dens, ev->scratch, ev->id[1], n, 1, st);
            if ((s = copy_out(ev, sg.data(), ev->scratch, dn, 0)) != SPH_OK) return s;
            launch_scatter_orig(dens + 5 * N, ev->scratch, ev->id[1], n, 1, st);
            if ((s = copy_out(ev, u0.data(), ev->scratch, dn, 0)) != SPH_OK) return s;
            DevScalars hs;
            if ((s = fetch(ev, &hs, ev->sc, sizeof(hs))) != SPH_OK) return s;
            double sqrtg = ev->milne ? hs.tau : 1.0;
            std::vector<double> Pi(n);
            for (int i = 0; i < n; ++i) Pi[i] = ev->viscous ? sg[i] / (u0[i] * sqrtg) * bv[i] : 0.0;
            CK(cudaMemcpy(o->Pi, Pi.data(), dn, o->on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost));
        }
    }
    if (mask & SPH_F_STATUS) {
        if (!o->status) return fail(SPH_ERR_ARG, "requested field has a null destination");
        if (n > 0) {
            launch_scatter_orig_u32(ev->status, (uint32_t *)ev->scratch, ev->id[1], n, st);
            sph_status s = copy_out(ev, o->status, ev->scratch, sizeof(uint32_t) * n, o->on_device);
            if (s != SPH_OK) return s;
        }
    }
    if (mask & SPH_F_NNB) {
        if (!o->nnb) return fail(SPH_ERR_ARG, "requested field has a null destination");
        if (n > 0) {
            launch_scatter_orig_u32((const uint32_t *)ev->nnb, (uint32_t *)ev->scratch, ev->id[1], n, st);
            sph_status s = copy_out(ev, o->nnb, ev->scratch, sizeof(int) * n, o->on_device);
            if (s != SPH_OK) return s;
        }
    }
    if (mask & SPH_F_CELL) {
        if (!o->cell) return fail(SPH_ERR_ARG, "requested field has a null destination");
        if (n > 0) {
            EvView v = make_view(ev);
            launch_cell_coords(v, ev->Y[1], ev->id[1], (int *)ev->scratch, st);
            sph_status s = copy_out(ev, o->cell, ev->scratch, sizeof(int) * ev->dim * n, o->on_device);
            if (s != SPH_OK) return s;
        }
    }
    if (tot) {
        memset(tot, 0, sizeof(*tot));
        DevScalars hs;
        if (n > 0) {
            EvView v = make_view(ev);
            launch_totals(v, ev->Y[1], ev->Nq[1], ev->id[1], dens, eo, ev->scratch, st);
            launch_sum_fixed(ev->scratch, n, 2, ev->tot, st);
            double h2[2], hn[3];
            sph_status s = fetch(ev, h2, ev->tot, sizeof(h2));
            if (s != SPH_OK) return s;
            if (ev->charges) {  // the charges evolve: their current fixed-order sums (original order)
                launch_scatter_orig(ev->Nq[0], ev->scratch, ev->id[0], n, 3, st);
                launch_sum_fixed(ev->scratch, n, 3, ev->ntot, st);
            }
            if ((s = fetch(ev, hn, ev->ntot, sizeof(hn))) != SPH_OK) return s;
            s = check_device_flags(ev, &hs);
            if (s != SPH_OK && s != SPH_ERR_EOS_RANGE && s != SPH_ERR_EOS_NOCONV && s != SPH_ERR_NONFINITE) return s;
            tot->E = h2[0];
            tot->S = h2[1];
            for (int q = 0; q < 3; ++q) tot->N[q] = hn[q];
        } else {
            sph_status s = fetch(ev, &hs, ev->sc, sizeof(hs));
            if (s != SPH_OK) return s;
        }
        tot->tau = hs.tau;
        tot->work = hs.work;
        tot->status_or = hs.status_or;
        tot->pair_overflows = (int32_t)hs.pair_ovf;
        tot->steps = hs.steps;
        tot->pairs = (int64_t)hs.pairs;
        tot->eos_work[0] = (int64_t)hs.eos_resid;
        tot->eos_work[1] = (int64_t)hs.eos_solve;
        tot->eos_work[2] = (int64_t)hs.eos_g;
        tot->shell_tests = (int64_t)hs.shell_tests;
        tot->kernel_launches = ev->launches;
    }
    return wait_stream(ev);
}

sph_status sph_eos_build_inverse(sph_eos *e, int32_t per_decade, int32_t decade_lo, int32_t decades, int32_t nx,
                                 double xmax)
{
    if (!e) return fail(SPH_ERR_ARG, "null EoS");
    if (!e->dev.has_table) return fail(SPH_ERR_ARG, "the offline inverter inverts a tabulated EoS");
    if (per_decade < 1 || decades < 1 || nx < 2 || !(xmax > 0.0) || decade_lo < -30 || decade_lo + decades > 30)
        return fail(SPH_ERR_ARG, "per_decade >= 1, decades >= 1, nx >= 2, xmax > 0 required");
    const long long ns = (long long)per_decade * decades + 1;
    const long long nnodes = ns * nx * nx * nx;
    if (nnodes > (1LL << 28)) return fail(SPH_ERR_ARG, "inverted table too large (more than 2^28 nodes)");
    std::vector<double> p10((size_t)decades + 1);
    for (int d = 0; d <= decades; ++d) p10[(size_t)d] = std::pow(10.0, (double)(decade_lo + d));
    double *inv = nullptr, *dp = nullptr;
    if (cudaMalloc(reinterpret_cast<void **>(&inv), sizeof(double) * 4 * (size_t)nnodes) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void **>(&dp), sizeof(double) * p10.size()) != cudaSuccess) {
        cudaGetLastError();
        if (inv) cudaFree(inv);
        return fail(SPH_ERR_OOM, "cudaMalloc failed for the inverted table");
    }
    CK(cudaMemcpy(dp, p10.data(), sizeof(double) * p10.size(), cudaMemcpyHostToDevice));
    EosDev E = e->dev;
    E.inv = inv;
    E.inv_p10 = dp;
    E.inv_K = per_decade;
    E.inv_nd = decades;
    E.inv_nx = nx;
    E.inv_xmax = xmax;
    launch_inverse_build(E, inv, nnodes, 0);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    if (e->d_inv) cudaFree(e->d_inv);
    if (e->d_p10) cudaFree(e->d_p10);
    e->d_inv = inv;
    e->d_p10 = dp;
    E.offline = 0;
    e->dev = E;
    return SPH_OK;
}

sph_status sph_set_eos_mode(sph_event *ev, int32_t mode)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (mode != SPH_EOS_ONLINE && mode != SPH_EOS_OFFLINE) return fail(SPH_ERR_ARG, "unknown EoS mode");
    if (mode == SPH_EOS_OFFLINE && !ev->eos->dev.inv)
        return fail(SPH_ERR_STATE, "the EoS handle has no inverted table (sph_eos_build_inverse)");
    CK(cudaStreamSynchronize(ev->stream));
    ev->eos_offline = mode == SPH_EOS_OFFLINE ? 1 : 0;
    if (ev->gexec) {  // the EoS parameters are part of the captured step: capture it again
        cudaGraphExecDestroy(ev->gexec);
        ev->gexec = nullptr;
    }
    if (ev->graph) {
        cudaGraphDestroy(ev->graph);
        ev->graph = nullptr;
    }
    ev->graph_ready = false;
    ev->kernels_per_step = 0;
    ev->observed = false;
    return SPH_OK;
}

sph_status sph_set_jets(sph_event *ev, int64_t ntrack, const double *tracks, double sigma)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (ntrack < 0 || ntrack > 4096) return fail(SPH_ERR_ARG, "ntrack must be in 0..4096");
    if (ntrack > 0 && (!tracks || !(sigma > 0.0))) return fail(SPH_ERR_ARG, "tracks and sigma > 0 required");
    if (ntrack > 0 && ev->milne) return fail(SPH_ERR_ARG, "jet sources are defined in Cartesian coordinates");
    for (int64_t k = 0; k < 8 * ntrack; ++k)
        if (!std::isfinite(tracks[k])) return fail(SPH_ERR_ARG, "non-finite track parameter");
    {
        sph_status ws = wait_stream(ev);  // bounded: the buffers below may be in use
        if (ws != SPH_OK) return ws;
    }
    if (ntrack > ev->ntrack || !ev->d_tracks) {
        sph_status s = dalloc(ev, reinterpret_cast<void **>(&ev->d_tracks), sizeof(double) * 8 * (size_t)(ntrack > 0 ? ntrack : 1));
        if (s != SPH_OK) return s;
    }
    if (ntrack > 0) CK(cudaMemcpy(ev->d_tracks, tracks, sizeof(double) * 8 * (size_t)ntrack, cudaMemcpyHostToDevice));
    ev->ntrack = (int)ntrack;
    ev->track_norm = ntrack > 0 ? 1.0 / (std::pow(2.0 * kPi, 1.5) * sigma * sigma * sigma) : 0.0;
    ev->track_i2s2 = ntrack > 0 ? 1.0 / (2.0 * sigma * sigma) : 0.0;
    if (ev->gexec) {  // the parameters are part of the captured step: capture it again
        cudaGraphExecDestroy(ev->gexec);
        ev->gexec = nullptr;
    }
    if (ev->graph) {
        cudaGraphDestroy(ev->graph);
        ev->graph = nullptr;
    }
    ev->graph_ready = false;
    ev->kernels_per_step = 0;
    ev->observed = false;
    return SPH_OK;
}

sph_status sph_set_eos_backup(sph_event *ev, int32_t enable, double T_scale_GeV, double mu_max_GeV)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (enable && (!(T_scale_GeV > 0.0) || !(mu_max_GeV > 0.0)))
        return fail(SPH_ERR_ARG, "T_scale and mu_max must be positive");
    {
        sph_status ws = wait_stream(ev);
        if (ws != SPH_OK) return ws;
    }
    ev->backup = enable ? 1 : 0;
    if (enable) {
        // matched to the closed form at T_scale (T_0 = 1/fm): A0 = p(T_scale, 0) / T_scale^4,
        // mu_q0 = mu_max (A0 / (p(T_scale, mu_q = mu_max) - p(T_scale, 0)))^(1/4)
        const EosDev &E = ev->eos->dev;
        const double Ts = T_scale_GeV / kHbarc, mm = mu_max_GeV / kHbarc;
        ev->cd_A0 = E.a0 + E.a1 * (1.0 + std::tanh((T_scale_GeV - E.Tc_GeV) / E.w_GeV)) / 2.0;
        for (int q = 0; q < 3; ++q) {
            const double dp = E.chi[q] * Ts * Ts * mm * mm / 2.0;
            ev->cd_mu0[q] = dp > 0.0 ? mm * std::pow(ev->cd_A0 / dp, 0.25) : mm;
        }
    }
    if (ev->gexec) {  // the parameters are part of the captured step: capture it again
        cudaGraphExecDestroy(ev->gexec);
        ev->gexec = nullptr;
    }
    if (ev->graph) {
        cudaGraphDestroy(ev->graph);
        ev->graph = nullptr;
    }
    ev->graph_ready = false;
    ev->kernels_per_step = 0;
    ev->observed = false;
    return SPH_OK;
}

sph_status sph_set_partons(sph_event *ev, int64_t nparton, const double *partons, const double *charges, double norm,
                           double h_src)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (nparton < 0 || nparton > (1 << 24)) return fail(SPH_ERR_ARG, "nparton must be in 0..2^24");
    if (nparton > 0 && (!partons || !(h_src > 0.0) || !std::isfinite(norm)))
        return fail(SPH_ERR_ARG, "partons, h_src > 0 and a finite norm required");
    for (int64_t k = 0; k < 8 * nparton; ++k)
        if (!std::isfinite(partons[k])) return fail(SPH_ERR_ARG, "non-finite parton entry");
    if (charges)
        for (int64_t k = 0; k < 3 * nparton; ++k)
            if (!std::isfinite(charges[k])) return fail(SPH_ERR_ARG, "non-finite parton charge");
    // sorted by formation time (stable), so a stage finds its window by binary search
    std::vector<int64_t> ord((size_t)nparton);
    for (int64_t k = 0; k < nparton; ++k) ord[(size_t)k] = k;
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t p, int64_t q) { return partons[8 * p] < partons[8 * q]; });
    std::vector<double> sorted((size_t)(8 * nparton)), sq(charges ? (size_t)(3 * nparton) : 0);
    for (int64_t k = 0; k < nparton; ++k) {
        for (int c = 0; c < 8; ++c) sorted[(size_t)(8 * k + c)] = partons[8 * ord[(size_t)k] + c];
        if (charges)
            for (int c = 0; c < 3; ++c) sq[(size_t)(3 * k + c)] = charges[3 * ord[(size_t)k] + c];
    }
    {
        sph_status ws = wait_stream(ev);  // bounded: the buffer below may be in use
        if (ws != SPH_OK) return ws;
    }
    if (nparton > ev->parton_cap || !ev->d_partons) {
        sph_status s = dalloc(ev, reinterpret_cast<void **>(&ev->d_partons),
                              sizeof(double) * 8 * (size_t)(nparton > 0 ? nparton : 1));
        if (s != SPH_OK) return s;
        s = dalloc(ev, reinterpret_cast<void **>(&ev->d_parton_q), sizeof(double) * 3 * (size_t)(nparton > 0 ? nparton : 1));
        if (s != SPH_OK) return s;
        ev->parton_cap = nparton > 0 ? nparton : 1;
    }
    const bool charged = charges && nparton > 0;
    if (charged && !ev->NqS[0]) {
        const size_t N = (size_t)(ev->n > 0 ? ev->n : 1);
        for (int k = 0; k < 2; ++k) {
            sph_status s = dalloc(ev, reinterpret_cast<void **>(&ev->NqS[k]), sizeof(double) * 3 * N);
            if (s != SPH_OK) return s;
        }
    }
    if (nparton > 0) {
        CK(cudaMemcpyAsync(ev->d_partons, sorted.data(), sizeof(double) * sorted.size(), cudaMemcpyHostToDevice,
                           ev->stream));
        if (charged)
            CK(cudaMemcpyAsync(ev->d_parton_q, sq.data(), sizeof(double) * sq.size(), cudaMemcpyHostToDevice,
                               ev->stream));
        sph_status ws = wait_stream(ev);
        if (ws != SPH_OK) return ws;
    }
    ev->charges = charged;
    ev->nparton = (int)nparton;
    ev->parton_norm = nparton > 0 ? norm : 0.0;
    ev->parton_h = nparton > 0 ? h_src : 0.0;
    if (ev->gexec) {  // the parameters are part of the captured step: capture it again
        cudaGraphExecDestroy(ev->gexec);
        ev->gexec = nullptr;
    }
    if (ev->graph) {
        cudaGraphDestroy(ev->graph);
        ev->graph = nullptr;
    }
    ev->graph_ready = false;
    ev->kernels_per_step = 0;
    ev->observed = false;
    return SPH_OK;
}

sph_status sph_set_viscous_eom(sph_event *ev, int32_t model, const double *coeffs)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (model != SPH_EOM_MIN_IS && model != SPH_EOM_DNMR) return fail(SPH_ERR_ARG, "unknown equations of motion");
    if (model == SPH_EOM_DNMR) {
        if (!coeffs) return fail(SPH_ERR_ARG, "DNMR needs its six coefficient ratios");
        for (int k = 0; k < 6; ++k)
            if (!std::isfinite(coeffs[k])) return fail(SPH_ERR_ARG, "non-finite DNMR coefficient");
    }
    {
        sph_status ws = wait_stream(ev);
        if (ws != SPH_OK) return ws;
    }
    ev->tr.model = model;
    for (int k = 0; k < 6; ++k) ev->tr.dnmr[k] = model == SPH_EOM_DNMR ? coeffs[k] : 0.0;
    if (ev->gexec) {  // the parameters are part of the captured step: capture it again
        cudaGraphExecDestroy(ev->gexec);
        ev->gexec = nullptr;
    }
    if (ev->graph) {
        cudaGraphDestroy(ev->graph);
        ev->graph = nullptr;
    }
    ev->graph_ready = false;
    ev->kernels_per_step = 0;
    ev->observed = false;
    return SPH_OK;
}

sph_status sph_freezeout_setup(sph_event *ev, double e_fo, int64_t capacity)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    if (!(e_fo > 0.0) || capacity < 1) return fail(SPH_ERR_ARG, "e_fo > 0 and capacity >= 1 required");
    {
        sph_status ws = wait_stream(ev);  // bounded: the buffers below may be in use
        if (ws != SPH_OK) return ws;
    }
    const size_t N = (size_t)(ev->n > 0 ? ev->n : 1);
    sph_status s;
    if (!ev->eprev[0]) {
        for (int k = 0; k < 2; ++k) {
            s = dalloc(ev, reinterpret_cast<void **>(&ev->eprev[k]), sizeof(double) * N);
            if (s != SPH_OK) return s;
        }
        s = dalloc(ev, reinterpret_cast<void **>(&ev->fo.count), sizeof(unsigned long long));
        if (s != SPH_OK) return s;
    }
    if ((unsigned long long)capacity > ev->fo.cap) {
        s = dalloc(ev, reinterpret_cast<void **>(&ev->fo.rec), sizeof(double) * kFoRec * (size_t)capacity);
        if (s != SPH_OK) return s;
        s = dalloc(ev, reinterpret_cast<void **>(&ev->fo.ids), sizeof(long long) * (size_t)capacity);
        if (s != SPH_OK) return s;
    }
    ev->fo.cap = (unsigned long long)capacity;
    // NaN: no previous value, so the first step after setup only records e
    CK(cudaMemsetAsync(ev->eprev[0], 0xFF, sizeof(double) * N, ev->stream));
    CK(cudaMemsetAsync(ev->fo.count, 0, sizeof(unsigned long long), ev->stream));
    {
        sph_status ws = wait_stream(ev);  // bounded: the buffers below may be in use
        if (ws != SPH_OK) return ws;
    }
    ev->e_fo = e_fo;
    ev->fo_on = true;
    if (ev->gexec) {  // the step graph changes: capture it again
        cudaGraphExecDestroy(ev->gexec);
        ev->gexec = nullptr;
    }
    if (ev->graph) {
        cudaGraphDestroy(ev->graph);
        ev->graph = nullptr;
    }
    ev->graph_ready = false;
    ev->kernels_per_step = 0;
    return SPH_OK;
}

sph_status sph_read_freezeout(sph_event *ev, int64_t cap, double *elems, int64_t *ids, int64_t *count)
{
    if (!ev || !count) return fail(SPH_ERR_ARG, "null argument");
    *count = 0;
    if (!ev->fo_on) return fail(SPH_ERR_STATE, "freeze-out recording is off (sph_freezeout_setup)");
    if (cap > 0 && (!elems || !ids)) return fail(SPH_ERR_ARG, "null destination");
    unsigned long long total = 0;
    sph_status s = fetch(ev, &total, ev->fo.count, sizeof(total));
    if (s != SPH_OK) return s;
    *count = (int64_t)total;
    const size_t m = (size_t)std::min<unsigned long long>(total, ev->fo.cap);
    if (cap <= 0 || m == 0) return total > ev->fo.cap ? fail(SPH_ERR_STATE, "freeze-out buffer overflowed") : SPH_OK;
    std::vector<double> rec(m * kFoRec);
    std::vector<long long> idv(m);
    if ((s = fetch(ev, rec.data(), ev->fo.rec, sizeof(double) * rec.size())) != SPH_OK) return s;
    if ((s = fetch(ev, idv.data(), ev->fo.ids, sizeof(long long) * m)) != SPH_OK) return s;
    std::vector<size_t> ord(m);
    for (size_t k = 0; k < m; ++k) ord[k] = k;
    std::sort(ord.begin(), ord.end(), [&](size_t p, size_t q) {
        const double tp = rec[p * kFoRec], tq = rec[q * kFoRec];
        return tp != tq ? tp < tq : idv[p] < idv[q];
    });
    const size_t w = std::min<size_t>(m, (size_t)cap);
    for (size_t k = 0; k < w; ++k) {
        std::memcpy(elems + k * kFoRec, rec.data() + ord[k] * kFoRec, sizeof(double) * kFoRec);
        ids[k] = (int64_t)idv[ord[k]];
    }
    return total > ev->fo.cap ? fail(SPH_ERR_STATE, "freeze-out buffer overflowed") : SPH_OK;
}

sph_status sph_kernel_times(sph_event *ev, int32_t max, char *names, double *ms, int64_t *launches, int32_t *count)
{
    if (!ev || !count) return fail(SPH_ERR_ARG, "null argument");
    if (!ev->profile) return fail(SPH_ERR_STATE, "event was not created with profile = 1");
    int m = std::min<int>(max, G_COUNT);
    for (int g = 0; g < m; ++g) {
        if (names) {
            strncpy(names + 32 * g, kGroupNames[g], 31);
            names[32 * g + 31] = 0;
        }
        if (ms) ms[g] = ev->prof_ms[g];
        if (launches) launches[g] = ev->prof_n[g];
    }
    *count = m;
    return SPH_OK;
}

sph_status sph_write_state(sph_event *ev, uint64_t mask, const sph_field_bufs *in)
{
    if (!ev || !in) return fail(SPH_ERR_ARG, "null argument");
    const int n = ev->n;
    if (n == 0) return SPH_OK;
    const size_t N = (size_t)n;
    // the state buffer is in sorted order; bring it back to the original order first
    cudaStream_t st = ev->stream;
    launch_scatter_orig(ev->Y[0], ev->scratch, ev->id[0], n, ev->nv, st);
    CK(cudaMemcpyAsync(ev->Y[0], ev->scratch, sizeof(double) * ev->nv * N, cudaMemcpyDeviceToDevice, st));
    launch_scatter_orig(ev->Nq[0], ev->scratch, ev->id[0], n, 3, st);
    CK(cudaMemcpyAsync(ev->Nq[0], ev->scratch, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, st));
    launch_scatter_orig(ev->wguess, ev->scratch, ev->id[0], n, 4, st);
    CK(cudaMemcpyAsync(ev->wguess, ev->scratch, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, st));
    if (ev->cb.pl.total > 0) {  // the neighbour counts carried with the state follow it
        launch_scatter_orig_u32((const uint32_t *)ev->pcnt[0], (uint32_t *)ev->pcnt[1], ev->id[0], n, st);
        CK(cudaMemcpyAsync(ev->pcnt[0], ev->pcnt[1], sizeof(int) * N, cudaMemcpyDeviceToDevice, st));
    }
    std::vector<int> iota(n);
    for (int i = 0; i < n; ++i) iota[i] = i;
    CK(cudaMemcpyAsync(ev->id[0], iota.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    cudaMemcpyKind k = in->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    struct Row {
        uint64_t bit;
        const double *src;
        size_t off;
        int rows;
    } rows[] = {
        {SPH_F_X, in->x, 0, ev->dim},
        {SPH_F_U, in->u, (size_t)ev->dim, ev->dim},
        {SPH_F_S, in->S, (size_t)2 * ev->dim, 1},
        {SPH_F_BV, in->Bv, (size_t)2 * ev->dim + 1, 1},
        {SPH_F_PV, in->Pv, (size_t)2 * ev->dim + 2, ev->npi},
        {SPH_F_JV, in->Jv, (size_t)kJRow, ev->diff ? 6 : 0},
    };
    if ((mask & SPH_F_JV) && !ev->diff) return fail(SPH_ERR_ARG, "the event has no diffusion currents");
    for (auto &r : rows) {
        if (!(mask & r.bit)) continue;
        if (!r.src) return fail(SPH_ERR_ARG, "masked field has a null source");
        CK(cudaMemcpyAsync(ev->Y[0] + r.off * N, r.src, sizeof(double) * r.rows * N, k, st));
    }
    if (mask & SPH_F_GUESS) {
        if (!in->guess) return fail(SPH_ERR_ARG, "masked field has a null source");
        CK(cudaMemcpyAsync(ev->wguess, in->guess, sizeof(double) * 4 * N, k, st));
    }
    ev->observed = false;
    return wait_stream(ev);
}

sph_status sph_debug_neighbors(sph_event *ev, int64_t cap, int32_t *pa, int32_t *pb, int64_t *count)
{
    if (!ev || !count) return fail(SPH_ERR_ARG, "null argument");
    const int n = ev->n;
    *count = 0;
    if (n == 0) return SPH_OK;
    enqueue_observe(ev);
    ev->observed = true;
    EvView v = make_view(ev);
    cudaStream_t st = ev->stream;
    int *d_cnt = nullptr;
    long long *d_off = nullptr;
    CK(cudaMalloc(&d_cnt, sizeof(int) * n));
    CK(cudaMalloc(&d_off, sizeof(long long) * (n + 1)));
    launch_neighbors_list(v, ev->Y[1], ev->id[1], ev->cb, nullptr, d_cnt, nullptr, st);
    launch_scan_counts(d_cnt, d_off, n, st);
    long long total = 0;
    // on a timed-out wait the scratch stays allocated: freeing it would block until the device is idle
    sph_status s = fetch(ev, &total, d_off + n, sizeof(long long));
    if (s != SPH_OK) return s;
    int *d_pa = nullptr, *d_pb = nullptr;
    CK(cudaMalloc(&d_pa, sizeof(int) * (total > 0 ? total : 1)));
    CK(cudaMalloc(&d_pb, sizeof(int) * (total > 0 ? total : 1)));
    launch_neighbors_list(v, ev->Y[1], ev->id[1], ev->cb, d_off, d_pa, d_pb, st);
    std::vector<int> ha(total), hb(total);
    if (total > 0) {
        if ((s = fetch(ev, ha.data(), d_pa, sizeof(int) * total)) != SPH_OK) return s;
        if ((s = fetch(ev, hb.data(), d_pb, sizeof(int) * total)) != SPH_OK) return s;
    }
    s = wait_stream(ev);
    cudaFree(d_cnt);
    cudaFree(d_off);
    cudaFree(d_pa);
    cudaFree(d_pb);
    if (s != SPH_OK) return s;
    std::vector<long long> key(total);
    for (long long i = 0; i < total; ++i) key[i] = ((long long)ha[i] << 32) | (unsigned)hb[i];
    std::sort(key.begin(), key.end());
    long long m = std::min<long long>(total, cap);
    for (long long i = 0; i < m; ++i) {
        pa[i] = (int)(key[i] >> 32);
        pb[i] = (int)(key[i] & 0xFFFFFFFFLL);
    }
    *count = total;
    return SPH_OK;
}

sph_status sph_debug_rates(sph_event *ev, double *rates, double *grad)
{
    if (!ev) return fail(SPH_ERR_ARG, "null event");
    const int n = ev->n;
    if (n == 0) return SPH_OK;
    enqueue_observe(ev);
    ev->observed = true;
    EvView v = make_view(ev);
    cudaStream_t st = ev->stream;
    launch_gradient(v, 1, ev->Y[1], ev->gin, ev->cb, ev->gout, st);
    const size_t N = (size_t)n;
    // rates go to Y1[1] (unused outside a step), then to the original order
    launch_eom(v, 1, 2, ev->Y[1], ev->dens, ev->eosf, ev->gout, nullptr, ev->Y1[1], ev->status, st);
    if (rates) {
        launch_scatter_orig(ev->Y1[1], ev->scratch, ev->id[1], n, ev->nv, st);
        sph_status s = copy_out(ev, rates, ev->scratch, sizeof(double) * ev->nv * N, 0);
        if (s != SPH_OK) return s;
    }
    if (grad) {
        launch_scatter_orig(ev->gout, ev->scratch, ev->id[1], n, ev->ngout, st);
        sph_status s = copy_out(ev, grad, ev->scratch, sizeof(double) * ev->ngout * N, 0);
        if (s != SPH_OK) return s;
    }
    return SPH_OK;
}

}  // extern "C"
