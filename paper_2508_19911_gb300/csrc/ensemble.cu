// Batched ensemble of independent CGKS-5th instances of uneven size.
//
// The instances' states are concatenated in caller-owned arenas (instance
// i's Q block [5][cells_i] starts at 5*off_i, its gradQ block [5][3][cells_i]
// at 15*off_i). The library splits every instance into work items of
// `tile` cells, each instance with its own dt, time and physics. A time
// step is, in mode 1 (the default), ONE persistent launch whose blocks
// stride over the work items of all instances phase by phase (dt,
// reconstruction, flux, update; ensemble_step.cu), separated by grid-wide
// barriers; in mode 0, one persistent launch per phase (8 launches; 12 in
// mixed precision, which adds the two views of the state per stage). The
// step is captured once into a CUDA graph and replayed; the autotuner times
// the graph for a set of tile sizes on a scratch copy of the state and
// keeps the fastest. The same work items serve the learned indicator's
// training dumps from all instances.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "basis.h"
#include "common.cuh"
#include "../../include/gks.h"

using namespace gks;

struct gks_ensemble {
    int device = 0;
    cudaStream_t user = nullptr;
    cudaStream_t s = nullptr;  // internal non-blocking stream (capturable)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int ninst = 0;
    std::vector<EnsInst> inst;
    EnsInst *dinst = nullptr;
    long long total = 0;
    int mixed = 0, indicator_on = 0;
    int tile = 1024;
    int mode = 1;                    // 1: one launch per step; 0: one per phase
    StepSync *sync = nullptr;        // the single-launch step's grid barrier
    std::vector<EnsItem> items;
    EnsItem *ditems = nullptr;
    int nitems = 0, items_cap = 0;
    int sms = 152;
    void *fs = nullptr;
    // FP32 gradients [15 total] and float-float averages (hi, lo: [5 total]
    // each) for the mixed kernels and the indicator dump
    float *Gf = nullptr, *Qv = nullptr;
    double *frec = nullptr, *Qs = nullptr, *Gs = nullptr, *Acc = nullptr, *S1 = nullptr;
    double *dt = nullptr, *t = nullptr, *red = nullptr;
    int *status = nullptr;
    unsigned long long *skips = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const double *gQ = nullptr, *gG = nullptr;
    int g_tile = 0, g_ind = 0, g_mode = -1;
    double g_tstop = 0.0;
};

namespace {

template <typename T>
int ealloc(T **p, size_t count) {
    *p = nullptr;
    if (cudaMalloc((void **)p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return GKS_ERR_NOMEM;
    }
    return GKS_OK;
}

void drop_graph(gks_ensemble *e) {
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->graph) cudaGraphDestroy(e->graph);
    e->exec = nullptr;
    e->graph = nullptr;
}

int build_items(gks_ensemble *e, int tile) {
    // the persistent kernels of earlier steps may still be reading the old
    // item list on e->s (a non-blocking stream, which the synchronous copy
    // below does not order against): let them finish first
    if (e->s && cudaStreamSynchronize(e->s) != cudaSuccess) return GKS_ERR_CUDA;
    e->items.clear();
    for (int i = 0; i < e->ninst; ++i)
        for (long long c0 = 0; c0 < e->inst[i].g.n; c0 += tile) {
            EnsItem it;
            it.inst = i;
            it.pad = 0;
            it.c0 = c0;
            it.c1 = std::min<long long>(c0 + tile, e->inst[i].g.n);
            e->items.push_back(it);
        }
    e->nitems = (int)e->items.size();
    if (e->nitems > e->items_cap) {
        cudaFree(e->ditems);
        e->ditems = nullptr;
        if (ealloc(&e->ditems, e->nitems)) return GKS_ERR_NOMEM;
        e->items_cap = e->nitems;
    }
    if (cudaMemcpy(e->ditems, e->items.data(), sizeof(EnsItem) * e->nitems,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return GKS_ERR_CUDA;
    e->tile = tile;
    drop_graph(e);
    return GKS_OK;
}

// wall-clock limit of a grid-barrier wait in the single-launch step: far
// above any phase's duration (the largest ensembles' flux phase takes well
// under a second), short enough that a stuck launch returns
constexpr double kStepWaitLimitS = 20.0;

// one time step of every instance on stream e->s (one launch, or 8 / 12)
int enqueue_step(gks_ensemble *e, double *Q, double *G, double t_stop) {
    if (e->mode == 1 && !e->indicator_on)
        return launch_ens_step(e->dinst, e->ninst, e->ditems, e->nitems, e->total, e->mixed, Q, G,
                               e->Qs, e->Gs, e->Acc, e->S1, e->fs, e->Gf, e->Qv, e->frec, e->dt,
                               e->t, e->red, t_stop, e->sync, kStepWaitLimitS, e->status, e->s)
                   ? GKS_ERR_CUDA
                   : GKS_OK;
    const int heavy = std::min(e->nitems, 2 * e->sms);  // 128-thread, register-heavy kernels
    const int light = std::min(e->nitems, 4 * e->sms);  // 256-thread kernels
    if (launch_dt_ens(e->dinst, e->ninst, e->ditems, e->nitems, light, Q, e->red, e->dt, e->t,
                      t_stop, e->s))
        return GKS_ERR_CUDA;
    const long long N = e->total;
    for (int stage = 1; stage <= 2; ++stage) {
        const double *Qi = stage == 1 ? Q : e->Qs;
        const double *Gi = stage == 1 ? G : e->Gs;
        if (e->mixed && (launch_g_to_f32(15 * N, Gi, e->Gf, e->s) ||
                         launch_q_to_ff(5 * N, Qi, e->Qv, e->Qv + 5 * N, e->s)))
            return GKS_ERR_CUDA;
        if (launch_recon5_ens(e->dinst, e->ditems, e->nitems, heavy, e->mixed, e->indicator_on, Qi,
                              Gi, e->Gf, e->Qv, e->Qv + 5 * N, e->fs, e->skips, e->s) ||
            launch_flux_ens(e->dinst, e->ditems, e->nitems, heavy, e->mixed, e->fs, e->Qv,
                            e->Qv + 5 * N, e->dt, e->frec, e->status, e->s) ||
            launch_update_ens(e->dinst, e->ditems, e->nitems, light, stage, e->frec, e->dt, Q, G,
                              e->Qs, e->Gs, e->Acc, e->S1, e->status, e->s))
            return GKS_ERR_CUDA;
    }
    return GKS_OK;
}

int run_steps(gks_ensemble *e, double *Q, double *G, int nsteps, double t_stop, int use_graph) {
    if (!use_graph) {
        for (int k = 0; k < nsteps; ++k) {
            const int rc = enqueue_step(e, Q, G, t_stop);
            if (rc) return rc;
        }
        return GKS_OK;
    }
    if (!e->exec || e->gQ != Q || e->gG != G || e->g_tile != e->tile ||
        e->g_tstop != t_stop || e->g_ind != e->indicator_on || e->g_mode != e->mode) {
        drop_graph(e);
        if (cudaStreamBeginCapture(e->s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return GKS_ERR_CUDA;
        const int rc = enqueue_step(e, Q, G, t_stop);
        cudaGraph_t g = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(e->s, &g);
        if (rc || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return GKS_ERR_CUDA;
        }
        e->graph = g;
        if (cudaGraphInstantiate(&e->exec, e->graph, 0) != cudaSuccess) {
            drop_graph(e);
            return GKS_ERR_CUDA;
        }
        e->gQ = Q;
        e->gG = G;
        e->g_tile = e->tile;
        e->g_tstop = t_stop;
        e->g_ind = e->indicator_on;
        e->g_mode = e->mode;
    }
    for (int k = 0; k < nsteps; ++k)
        if (cudaGraphLaunch(e->exec, e->s) != cudaSuccess) return GKS_ERR_CUDA;
    return GKS_OK;
}

}  // namespace

extern "C" {

void gks_ensemble_destroy(gks_ensemble *e) {
    if (!e) return;
    cudaSetDevice(e->device);
    if (e->s) cudaStreamSynchronize(e->s);
    drop_graph(e);
    cudaFree(e->dinst);
    cudaFree(e->ditems);
    cudaFree(e->fs);
    cudaFree(e->Gf);
    cudaFree(e->Qv);
    cudaFree(e->frec);
    cudaFree(e->Qs);
    cudaFree(e->Gs);
    cudaFree(e->Acc);
    cudaFree(e->S1);
    cudaFree(e->dt);
    cudaFree(e->t);
    cudaFree(e->red);
    cudaFree(e->status);
    cudaFree(e->sync);
    cudaFree(e->skips);
    if (e->ev_in) cudaEventDestroy(e->ev_in);
    if (e->ev_out) cudaEventDestroy(e->ev_out);
    if (e->s) cudaStreamDestroy(e->s);
    delete e;
}

int gks_ensemble_create(gks_ensemble **out, int n, const int *dims, const double *lengths,
                        const double *phys, const gks_options *opt, void *cuda_stream) {
    if (!out || n <= 0 || !dims || !lengths || !phys) return GKS_ERR_ARG;
    *out = nullptr;
    gks_options o;
    if (opt) o = *opt; else gks_default_options(&o);
    if (o.scheme != GKS_SCHEME_CGKS5) return GKS_ERR_ARG;
    if (o.precision != GKS_PREC_FP64 && o.precision != GKS_PREC_MIXED) return GKS_ERR_ARG;
    if (o.indicator && o.precision != GKS_PREC_MIXED) return GKS_ERR_ARG;
    if (!(o.T_ref > 0.0)) return GKS_ERR_ARG;
    gks_ensemble *e = new (std::nothrow) gks_ensemble;
    if (!e) return GKS_ERR_NOMEM;
    if (cudaGetDevice(&e->device) != cudaSuccess) { delete e; return GKS_ERR_CUDA; }
    cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, e->device);
    e->user = (cudaStream_t)cuda_stream;
    e->ninst = n;
    e->mixed = o.precision == GKS_PREC_MIXED;
    long long off = 0;
    for (int i = 0; i < n; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        const double *L = lengths + 3 * i, *ph = phys + 8 * i;
        if (nx < 1 || ny < 1 || nz < 1 || !(L[0] > 0 && L[1] > 0 && L[2] > 0)) { delete e; return GKS_ERR_ARG; }
        // phys: gamma, Pr, mu, cfl, mu_law, inviscid, C_tau, eps_tau
        if (!(ph[0] > 1.0) || !(ph[1] > 0.0) || !(ph[2] >= 0.0) || !(ph[3] > 0.0 && ph[3] <= 1.0) ||
            !(ph[4] == 0.0 || ph[4] == 1.0) || !(ph[5] == 0.0 || ph[5] == 1.0) ||
            !(ph[6] >= 0.0) || !(ph[7] >= 0.0)) {
            delete e;
            return GKS_ERR_ARG;
        }
        EnsInst I;
        std::memset(&I, 0, sizeof(I));
        I.g.nx = nx; I.g.ny = ny; I.g.nz = nz; I.g.n = (long long)nx * ny * nz;
        I.g.h[0] = L[0] / nx; I.g.h[1] = L[1] / ny; I.g.h[2] = L[2] / nz;
        I.P.gamma = ph[0]; I.P.Pr = ph[1]; I.P.mu0 = ph[2]; I.P.cfl = ph[3];
        I.P.mu_law = (int)ph[4]; I.P.inviscid = (int)ph[5];
        I.P.C_tau = ph[6]; I.P.eps_tau = ph[7]; I.P.T_ref = o.T_ref;
        I.P.Nint = (5.0 - 3.0 * ph[0]) / (ph[0] - 1.0);
        I.P.nonlinear = o.nonlinear ? 1 : 0;
        I.P.scheme = GKS_SCHEME_CGKS5;
        I.off = off;
        off += I.g.n;
        e->inst.push_back(I);
    }
    e->total = off;
    if (e->total > (1LL << 31)) { delete e; return GKS_ERR_ARG; }
    int rc = GKS_OK;
    if (upload_recon_tables()) { gks_ensemble_destroy(e); return GKS_ERR_CUDA; }
    if (cudaStreamCreateWithFlags(&e->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev_out, cudaEventDisableTiming) != cudaSuccess) {
        gks_ensemble_destroy(e);
        return GKS_ERR_CUDA;
    }
    const size_t N = (size_t)e->total;
    if ((rc = ealloc(&e->dinst, n)) ||
        (rc = ealloc((char **)&e->fs, 480 * N * (e->mixed ? 4 : 8))) ||
        (rc = ealloc(&e->Gf, 15 * N)) || (rc = ealloc(&e->Qv, 10 * N)) ||
        (rc = ealloc(&e->frec, 90 * N)) || (rc = ealloc(&e->Qs, 5 * N)) ||
        (rc = ealloc(&e->Gs, 15 * N)) || (rc = ealloc(&e->Acc, 5 * N)) ||
        (rc = ealloc(&e->S1, 15 * N)) || (rc = ealloc(&e->dt, n)) || (rc = ealloc(&e->t, n)) ||
        (rc = ealloc(&e->red, 2 * n)) || (rc = ealloc(&e->status, 1)) || (rc = ealloc(&e->sync, 1)) ||
        (rc = ealloc(&e->skips, 1))) {
        gks_ensemble_destroy(e);
        return rc;
    }
    if (cudaMemcpy(e->dinst, e->inst.data(), sizeof(EnsInst) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(e->t, 0, sizeof(double) * n) != cudaSuccess ||
        cudaMemset(e->red, 0, sizeof(double) * 2 * n) != cudaSuccess ||
        cudaMemset(e->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(e->skips, 0, sizeof(unsigned long long)) != cudaSuccess) {
        gks_ensemble_destroy(e);
        return GKS_ERR_CUDA;
    }
    if ((rc = build_items(e, 1024))) {
        gks_ensemble_destroy(e);
        return rc;
    }
    *out = e;
    return GKS_OK;
}

long long gks_ensemble_offset(const gks_ensemble *e, int i) {
    if (!e || i < 0 || i > e->ninst) return -1;
    return i == e->ninst ? e->total : e->inst[i].off;
}

int gks_ensemble_set_tile(gks_ensemble *e, int tile_cells) {
    if (!e || tile_cells < 32 || tile_cells > (1 << 22)) return GKS_ERR_ARG;
    return build_items(e, tile_cells);
}

int gks_ensemble_step(gks_ensemble *e, double *Q, double *G, int nsteps, double t_stop,
                      int use_graph) {
    if (!e || !Q || !G || nsteps < 0) return GKS_ERR_ARG;
    if (nsteps == 0) return GKS_OK;
    if (cudaEventRecord(e->ev_in, e->user) != cudaSuccess ||
        cudaStreamWaitEvent(e->s, e->ev_in, 0) != cudaSuccess)
        return GKS_ERR_CUDA;
    const int rc = run_steps(e, Q, G, nsteps, t_stop, use_graph);
    if (cudaEventRecord(e->ev_out, e->s) != cudaSuccess ||
        cudaStreamWaitEvent(e->user, e->ev_out, 0) != cudaSuccess)
        return GKS_ERR_CUDA;
    return rc;
}

int gks_ensemble_times(gks_ensemble *e, double *t_host, int *status) {
    if (!e || !t_host) return GKS_ERR_ARG;
    int st = 0;
    if (cudaStreamSynchronize(e->s) != cudaSuccess ||
        cudaMemcpy(t_host, e->t, sizeof(double) * e->ninst, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&st, e->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return GKS_ERR_CUDA;
    if (status) *status = st;
    if (st & kStatusTimeout) return GKS_ERR_TIMEOUT;
    return st ? GKS_ERR_NONPHYSICAL : GKS_OK;
}

int gks_ensemble_set_mode(gks_ensemble *e, int mode) {
    if (!e || (mode != 0 && mode != 1)) return GKS_ERR_ARG;
    if (e->s && cudaStreamSynchronize(e->s) != cudaSuccess) return GKS_ERR_CUDA;
    e->mode = mode;
    drop_graph(e);
    return GKS_OK;
}

int gks_ensemble_mode(const gks_ensemble *e) { return e ? e->mode : -1; }

int gks_barrier_timeout_check(double limit_s, void *cuda_stream) {
    if (!(limit_s > 0.0 && limit_s <= 10.0)) return GKS_ERR_ARG;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    StepSync *sync = nullptr;
    int *st = nullptr;
    if (ealloc(&sync, 1) || ealloc(&st, 1)) {
        cudaFree(sync);
        return GKS_ERR_NOMEM;
    }
    int host = 0;
    int rc = GKS_OK;
    if (cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess ||
        launch_barrier_timeout(sync, 2, limit_s, st, s) ||
        cudaMemcpyAsync(&host, st, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = GKS_ERR_CUDA;
    cudaStreamSynchronize(s);  // no copy into host left in flight
    cudaFree(sync);
    cudaFree(st);
    if (rc) return rc;
    return (host & kStatusTimeout) ? GKS_ERR_TIMEOUT : GKS_OK;
}

int gks_ensemble_autotune(gks_ensemble *e, const double *Q, const double *G, int *tile_out,
                          float *best_ms) {
    if (!e || !Q || !G) return GKS_ERR_ARG;
    static const int cands[] = {256, 512, 1024, 2048, 4096, 8192};
    const size_t N = (size_t)e->total;
    double *Qw = nullptr, *Gw = nullptr, *tsave = nullptr;
    int rc = GKS_OK;
    if ((rc = ealloc(&Qw, 5 * N)) || (rc = ealloc(&Gw, 15 * N)) || (rc = ealloc(&tsave, e->ninst))) {
        cudaFree(Qw); cudaFree(Gw); cudaFree(tsave);
        return rc;
    }
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaStreamSynchronize(e->user);
    cudaMemcpyAsync(tsave, e->t, sizeof(double) * e->ninst, cudaMemcpyDeviceToDevice, e->s);
    const int old_tile = e->tile;
    int best = old_tile;
    float bms = 1e30f;
    for (int tile : cands) {
        if ((rc = build_items(e, tile))) break;
        cudaMemcpyAsync(Qw, Q, sizeof(double) * 5 * N, cudaMemcpyDeviceToDevice, e->s);
        cudaMemcpyAsync(Gw, G, sizeof(double) * 15 * N, cudaMemcpyDeviceToDevice, e->s);
        if ((rc = run_steps(e, Qw, Gw, 1, INFINITY, 1))) break;  // capture + warm-up
        cudaEventRecord(a, e->s);
        if ((rc = run_steps(e, Qw, Gw, 3, INFINITY, 1))) break;
        cudaEventRecord(b, e->s);
        if (cudaEventSynchronize(b) != cudaSuccess) { rc = GKS_ERR_CUDA; break; }
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= 3.0f;
        if (ms < bms) { bms = ms; best = tile; }
    }
    cudaMemcpyAsync(e->t, tsave, sizeof(double) * e->ninst, cudaMemcpyDeviceToDevice, e->s);
    cudaMemsetAsync(e->status, 0, sizeof(int), e->s);
    cudaStreamSynchronize(e->s);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(Qw);
    cudaFree(Gw);
    cudaFree(tsave);
    const int rc2 = build_items(e, rc ? old_tile : best);
    if (rc) return rc;
    if (rc2) return rc2;
    if (tile_out) *tile_out = best;
    if (best_ms) *best_ms = bms;
    return GKS_OK;
}

int gks_ensemble_dump(gks_ensemble *e, const double *Q, const double *G, float label_eps, float *x,
                      float *chi, float *y) {
    if (!e || !Q || !G || !x || !chi || !y || !(label_eps >= 0.0f)) return GKS_ERR_ARG;
    if (cudaEventRecord(e->ev_in, e->user) != cudaSuccess ||
        cudaStreamWaitEvent(e->s, e->ev_in, 0) != cudaSuccess)
        return GKS_ERR_CUDA;
    const int heavy = std::min(e->nitems, 2 * e->sms);
    const long long N = e->total;
    if (launch_g_to_f32(15 * N, G, e->Gf, e->s) ||
        launch_q_to_ff(5 * N, Q, e->Qv, e->Qv + 5 * N, e->s) ||
        launch_indicator_dump_ens(e->dinst, e->ditems, e->nitems, heavy, e->Gf, e->Qv,
                                  e->Qv + 5 * N, x, chi, e->total, e->s) ||
        launch_labels(chi, y, 5 * e->total, label_eps, e->s))
        return GKS_ERR_CUDA;
    if (cudaEventRecord(e->ev_out, e->s) != cudaSuccess ||
        cudaStreamWaitEvent(e->user, e->ev_out, 0) != cudaSuccess)
        return GKS_ERR_CUDA;
    return GKS_OK;
}

int gks_ensemble_set_indicator(gks_ensemble *e, const float *params, float theta) {
    if (!e || !params || !(theta > 0.0f && theta <= 1.0f)) return GKS_ERR_ARG;
    if (!e->mixed) return GKS_ERR_STATE;
    if (upload_indicator(params, theta)) return GKS_ERR_CUDA;
    e->indicator_on = 1;
    return GKS_OK;
}

}  // extern "C"
