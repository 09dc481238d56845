// C-ABI of the CGKS-5th / GKS-2nd hot path (declared in include/gks.h).
// Owns the device workspace of one grid and enqueues the kernels of
// recon.cu, flux.cu and update.cu on the caller's stream.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "basis.h"
#include "common.cuh"
#include "../../include/gks.h"

using namespace gks;

struct gks_ctx {
    int device;
    cudaStream_t stream;
    GridDesc g;
    PhysParams P;
    gks_options opt;
    int K;                 // Gauss points per face
    void *fs;              // face states [6][K][20][n], FP64 or (mixed) FP32
    int mixed;             // precision == GKS_PREC_MIXED
    int indicator_on;      // learned indicator active (CGKS-5th, mixed)
    unsigned long long *skips;  // (cell, variable) pairs that skipped GENO
    double *frec;          // face records [3][30][n]
    double *Qs, *Gs, *Acc, *S1;  // CGKS-5th stage buffers
    float *Gf;             // mixed CGKS-5th: FP32 copy of the gradients [15][n]
    float *Qv;             // mixed: float-float split of the averages, hi [5][n] then lo [5][n]
    int slab_planes;       // 0: fs holds the whole grid; > 0: z-slabs of this many planes
    double *scal;          // [0] dt, [1..2] dt reduction words, [3] diagnostics out (12)
    int *status;
    double *partials;
    int diag_blocks;
    double *hQ, *hG, *hT;  // device state of gks_step_host (allocated on its first call)
    double *hsz;           // stretched mesh: the nx + ny + nz cell sizes (device)
    double *lrec, *Ls, *LS1;  // gks_step_lines: records [3][90][n], lines [60][n] x 2
    int timing;            // gks_kernel_timing: record events around the step's launches
    cudaEvent_t t_open;    // event before the launch being timed
    std::vector<struct KernelRec> *t_recs;  // (kind, start, end) of the timed launches
};

struct KernelRec {
    int kind;
    cudaEvent_t e0, e1;
};

namespace {

int cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return GKS_ERR_NOMEM;
    return GKS_ERR_CUDA;
}

template <typename T>
int dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) return GKS_OK;
    const cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return cuda_fail(e);
    }
    return GKS_OK;
}

double *dt_slot(gks_ctx *c) { return c->scal; }
double *red_slot(gks_ctx *c) { return c->scal + 1; }
double *diag_slot(gks_ctx *c) { return c->scal + 3; }

int launch_ok(int rc) { return rc == 0 ? GKS_OK : (rc == -1 ? GKS_ERR_ARG : GKS_ERR_CUDA); }

// kernel timing (gks_kernel_timing): an event on the context's stream
// before and after each timed launch; no synchronisation
enum { kTimeRecon = 0, kTimeFlux = 1, kTimeUpdate = 2, kTimeDt = 3 };
void time_open(gks_ctx *c) {
    if (!c->timing) return;
    if (cudaEventCreate(&c->t_open) != cudaSuccess) { c->t_open = nullptr; return; }
    cudaEventRecord(c->t_open, c->stream);
}
void time_close(gks_ctx *c, int kind) {
    if (!c->timing || !c->t_open) return;
    cudaEvent_t e1;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(c->t_open);
        c->t_open = nullptr;
        return;
    }
    cudaEventRecord(e1, c->stream);
    c->t_recs->push_back(KernelRec{kind, c->t_open, e1});
    c->t_open = nullptr;
}
void time_clear(gks_ctx *c) {
    if (!c->t_recs) return;
    for (const KernelRec &r : *c->t_recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    c->t_recs->clear();
}

}  // namespace

extern "C" {

void gks_default_options(gks_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->scheme = GKS_SCHEME_CGKS5;
    opt->nonlinear = 1;
    opt->precision = GKS_PREC_FP64;
    opt->indicator = 0;
    opt->mu_law = 0;
    opt->inviscid = 0;
    opt->C_tau = 10.0;
    opt->eps_tau = 0.05;
    opt->T_ref = 1.0;
    opt->theta = 0.9;
}

const char *gks_strerror(int code) {
    switch (code) {
        case GKS_OK: return "ok";
        case GKS_ERR_ARG: return "invalid argument";
        case GKS_ERR_CUDA: return "CUDA runtime error";
        case GKS_ERR_NONPHYSICAL: return "non-physical or non-finite state";
        case GKS_ERR_TIMEOUT: return "device wait timed out";
        case GKS_ERR_STATE: return "call out of order or wrong scheme";
        case GKS_ERR_NOMEM: return "device allocation failed";
        default: return "unknown error";
    }
}

void gks_destroy(gks_ctx *c) {
    if (!c) return;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    cudaFree(c->fs);
    cudaFree(c->frec);
    cudaFree(c->Qs);
    cudaFree(c->Gs);
    cudaFree(c->Acc);
    cudaFree(c->S1);
    cudaFree(c->Gf);
    cudaFree(c->Qv);
    cudaFree(c->scal);
    cudaFree(c->status);
    cudaFree(c->partials);
    cudaFree(c->skips);
    cudaFree(c->hQ);
    cudaFree(c->hG);
    cudaFree(c->hT);
    cudaFree(c->hsz);
    cudaFree(c->lrec);
    cudaFree(c->Ls);
    cudaFree(c->LS1);
    time_clear(c);
    delete c->t_recs;
    if (prev >= 0) cudaSetDevice(prev);
    delete c;
}

int gks_init(gks_ctx **out, double gamma, double Pr, double mu, double cfl, int nx, int ny,
             int nz, double Lx, double Ly, double Lz, const gks_options *opt,
             void *cuda_stream) {
    if (!out) return GKS_ERR_ARG;
    *out = nullptr;
    gks_options o;
    if (opt) o = *opt; else gks_default_options(&o);
    if (!(gamma > 1.0) || !(Pr > 0.0) || !(mu >= 0.0) || !(cfl > 0.0 && cfl <= 1.0)) return GKS_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || !(Lx > 0.0) || !(Ly > 0.0) || !(Lz > 0.0)) return GKS_ERR_ARG;
    if (o.scheme != GKS_SCHEME_GKS2 && o.scheme != GKS_SCHEME_CGKS5) return GKS_ERR_ARG;
    if (o.precision != GKS_PREC_FP64 && o.precision != GKS_PREC_MIXED) return GKS_ERR_ARG;
    if (o.indicator && !(o.scheme == GKS_SCHEME_CGKS5 && o.precision == GKS_PREC_MIXED))
        return GKS_ERR_ARG;
    if (o.indicator && !(o.theta > 0.0 && o.theta <= 1.0)) return GKS_ERR_ARG;
    if (o.mu_law < 0 || o.mu_law > 1 || !(o.C_tau >= 0.0) || !(o.eps_tau >= 0.0) ||
        !(o.T_ref > 0.0) || o.slab_planes < 0)
        return GKS_ERR_ARG;
    const int len[3] = {nx, ny, nz};
    bool general = false;
    for (int a = 0; a < 3; ++a) {
        if (o.bc[a] < GKS_BC_PERIODIC || o.bc[a] > GKS_BC_OUTFLOW) return GKS_ERR_ARG;
        if (o.bc[a] != GKS_BC_PERIODIC || o.h[a]) general = true;
        if (o.h[a])
            for (int i = 0; i < len[a]; ++i)
                if (!(o.h[a][i] > 0.0) || !std::isfinite(o.h[a][i])) return GKS_ERR_ARG;
    }
    if (general && o.indicator) return GKS_ERR_ARG;
    const long long n = (long long)nx * ny * nz;
    if (n > (1LL << 31)) return GKS_ERR_ARG;

    gks_ctx *c = new (std::nothrow) gks_ctx;
    if (!c) return GKS_ERR_NOMEM;
    std::memset(c, 0, sizeof(*c));
    if (cudaGetDevice(&c->device) != cudaSuccess) { delete c; return GKS_ERR_CUDA; }
    c->stream = (cudaStream_t)cuda_stream;
    c->opt = o;
    c->g.nx = nx; c->g.ny = ny; c->g.nz = nz; c->g.n = n;
    c->g.h[0] = Lx / nx; c->g.h[1] = Ly / ny; c->g.h[2] = Lz / nz;
    if (general) {
        c->g.general = 1;
        c->g.np = std::max((long long)ny * nz, std::max((long long)nx * nz, (long long)nx * ny));
        double hmin = INFINITY, ext[3];
        for (int a = 0; a < 3; ++a) {
            c->g.bc[a] = o.bc[a];
            ext[a] = 0.0;
            for (int i = 0; i < len[a]; ++i) {
                const double hh = o.h[a] ? o.h[a][i] : c->g.h[a];
                hmin = std::min(hmin, hh);
                ext[a] += hh;
            }
        }
        c->g.hmin = hmin;
        const bool stretched = o.h[0] || o.h[1] || o.h[2];
        c->g.volume = stretched ? ext[0] * ext[1] * ext[2]
                                : c->g.h[0] * c->g.h[1] * c->g.h[2] * (double)n;
    }
    c->P.gamma = gamma; c->P.Pr = Pr; c->P.mu0 = mu; c->P.cfl = cfl;
    c->P.C_tau = o.C_tau; c->P.eps_tau = o.eps_tau; c->P.T_ref = o.T_ref;
    c->P.Nint = (5.0 - 3.0 * gamma) / (gamma - 1.0);
    c->P.mu_law = o.mu_law; c->P.inviscid = o.inviscid; c->P.nonlinear = o.nonlinear ? 1 : 0;
    c->P.scheme = o.scheme;
    c->K = o.scheme == GKS_SCHEME_CGKS5 ? 4 : 1;
    c->mixed = o.precision == GKS_PREC_MIXED;

    int rc = GKS_OK;
    if (o.scheme == GKS_SCHEME_CGKS5) {
        const int t = upload_recon_tables();
        if (t) { gks_destroy(c); return t == -1 ? GKS_ERR_ARG : GKS_ERR_CUDA; }
    }
    c->diag_blocks = diagnostics_blocks(c->g);
    // face-state buffer: the whole grid, or z-slabs (+1 plane below each)
    const size_t fs_per_cell = (size_t)6 * c->K * 20 * (c->mixed ? 4 : 8);
    const long long nxy = (long long)nx * ny;
    long long planes = nz;
    if (o.slab_planes > 0) {
        planes = o.slab_planes;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (double)fs_per_cell * n > 0.4 * fr) {
            planes = (long long)(0.25 * fr / ((double)fs_per_cell * nxy)) - 1;
            if (planes < 1) planes = 1;
        }
    }
    c->slab_planes = planes >= nz ? 0 : (int)planes;
    const long long fs_cells = c->slab_planes ? nxy * (c->slab_planes + 1) : n;
    const size_t nrec = (size_t)90 * n + (c->g.general ? (size_t)90 * c->g.np : 0);
    if ((rc = dalloc((char **)&c->fs, fs_per_cell * fs_cells)) ||
        (rc = dalloc(&c->frec, nrec)) ||
        (rc = dalloc(&c->scal, (size_t)3 + 12)) ||
        (rc = dalloc(&c->status, 1)) ||
        (rc = dalloc(&c->skips, 1)) ||
        (rc = dalloc(&c->partials, (size_t)12 * c->diag_blocks)) ||
        (c->mixed && (rc = dalloc(&c->Qv, (size_t)10 * n)))) {
        gks_destroy(c);
        return rc;
    }
    if (o.scheme == GKS_SCHEME_CGKS5) {
        if ((rc = dalloc(&c->Qs, (size_t)5 * n)) || (rc = dalloc(&c->Gs, (size_t)15 * n)) ||
            (rc = dalloc(&c->Acc, (size_t)5 * n)) || (rc = dalloc(&c->S1, (size_t)15 * n)) ||
            (c->mixed && (rc = dalloc(&c->Gf, (size_t)15 * n)))) {
            gks_destroy(c);
            return rc;
        }
    }
    if (cudaMemsetAsync(c->scal, 0, sizeof(double) * 15, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->status, 0, sizeof(int), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->skips, 0, sizeof(unsigned long long), c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->frec, 0, sizeof(double) * nrec, c->stream) != cudaSuccess) {
        gks_destroy(c);
        return GKS_ERR_CUDA;
    }
    if (o.h[0] || o.h[1] || o.h[2]) {
        // the cell sizes, copied synchronously (the host arrays need not
        // outlive this call)
        std::vector<double> hh;
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < len[a]; ++i) hh.push_back(o.h[a] ? o.h[a][i] : c->g.h[a]);
        if ((rc = dalloc(&c->hsz, hh.size()))) {
            gks_destroy(c);
            return rc;
        }
        if (cudaMemcpy(c->hsz, hh.data(), sizeof(double) * hh.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
            gks_destroy(c);
            return GKS_ERR_CUDA;
        }
        c->g.hs[0] = c->hsz;
        c->g.hs[1] = c->hsz + nx;
        c->g.hs[2] = c->hsz + nx + ny;
    }
    *out = c;
    return GKS_OK;
}

size_t gks_face_state_bytes(const gks_ctx *c) {
    return c ? (size_t)6 * c->K * 20 * c->g.n * (c->mixed ? 4 : 8) : 0;
}

int gks_slab_planes(const gks_ctx *c) { return c ? c->slab_planes : -1; }

size_t gks_face_flux_bytes(const gks_ctx *c) {
    if (!c) return 0;
    return ((size_t)90 * c->g.n + (c->g.general ? (size_t)90 * c->g.np : 0)) * sizeof(double);
}

int gks_compute_dt(gks_ctx *c, const double *Q, double *dt_dev) {
    if (!c || !Q || !dt_dev) return GKS_ERR_ARG;
    return launch_ok(launch_dt(c->g, c->P, Q, red_slot(c), dt_dev, nullptr, 0.0, c->stream));
}

namespace {
// reconstruction and flux of one face-state buffer S (the FP32 gradient
// copy of the mixed CGKS-5th reconstruction is made by the caller)
// mixed: the views of Q, G (make_views) must be current
int make_views(gks_ctx *c, const double *Q, const double *G) {
    int rc;
    if (c->mixed && c->P.scheme == GKS_SCHEME_CGKS5 && G &&
        (rc = launch_g_to_f32(15 * c->g.n, G, c->Gf, c->stream)))
        return rc;
    if (c->mixed && (rc = launch_q_to_ff(5 * c->g.n, Q, c->Qv, c->Qv + 5 * c->g.n, c->stream)))
        return rc;
    return 0;
}
int recon_any(gks_ctx *c, const Slab &S, const double *Q, const double *G, void *fs) {
    const bool cg = c->P.scheme == GKS_SCHEME_CGKS5;
    if (c->mixed)
        return cg ? launch_recon5_mixed(c->g, S, c->P, c->Gf, c->Qv, c->Qv + 5 * c->g.n,
                                        (float *)fs, c->stream, c->indicator_on, c->skips)
                  : launch_recon2_mixed(c->g, S, c->P, Q, (float *)fs, c->stream);
    return cg ? launch_recon5(c->g, S, c->P, Q, G, (double *)fs, c->stream)
              : launch_recon2(c->g, S, c->P, Q, (double *)fs, c->stream);
}
// mixed: c->Qv must hold the split of the averages the face states came from
int flux_any(gks_ctx *c, const Slab &S, const double *Q, const void *fs, const double *dt,
             double *fr) {
    (void)Q;
    if (c->mixed)
        return launch_flux_faces_mixed(c->g, S, c->P, (const float *)fs, c->Qv,
                                       c->Qv + 5 * c->g.n, dt, fr, c->status, c->stream);
    return launch_flux_faces(c->g, S, c->P, (const double *)fs, dt, fr, c->status, c->stream);
}
// one stage's face records: reconstruction + flux over the whole grid or
// slab by slab into the context's buffer
int stage_faces(gks_ctx *c, const double *Q, const double *G, const double *dt) {
    int rc;
    if ((rc = make_views(c, Q, G))) return rc;
    if (!c->slab_planes) {
        const Slab S = whole_grid(c->g);
        time_open(c);
        if ((rc = recon_any(c, S, Q, G, c->fs))) return rc;
        time_close(c, kTimeRecon);
        time_open(c);
        if ((rc = flux_any(c, S, Q, c->fs, dt, c->frec))) return rc;
        time_close(c, kTimeFlux);
        return 0;
    }
    const int nz = c->g.nz;
    const long long nxy = (long long)c->g.nx * c->g.ny;
    for (int z0 = 0; z0 < nz; z0 += c->slab_planes) {
        const int nzs = nz - z0 < c->slab_planes ? nz - z0 : c->slab_planes;
        Slab S;
        S.zb = (z0 - 1 + nz) % nz;
        S.nzb = nzs + 1;
        S.p0 = 1;
        S.pad = 0;
        S.nb = nxy * S.nzb;
        time_open(c);
        if ((rc = recon_any(c, S, Q, G, c->fs))) return rc;
        time_close(c, kTimeRecon);
        time_open(c);
        if ((rc = flux_any(c, S, Q, c->fs, dt, c->frec))) return rc;
        time_close(c, kTimeFlux);
    }
    return 0;
}
}  // namespace

int gks_reconstruct(gks_ctx *c, const double *Q, const double *G, void *face_states) {
    if (!c || !Q) return GKS_ERR_ARG;
    if (c->P.scheme == GKS_SCHEME_CGKS5 && !G) return GKS_ERR_ARG;
    if (!face_states && c->slab_planes) return GKS_ERR_STATE;  // own buffer holds a slab only
    if (make_views(c, Q, G)) return GKS_ERR_CUDA;
    return launch_ok(recon_any(c, whole_grid(c->g), Q, G, face_states ? face_states : c->fs));
}

int gks_flux(gks_ctx *c, const double *Q, const void *face_states, const double *dt_dev,
             double *face_flux) {
    if (!c || !dt_dev) return GKS_ERR_ARG;
    if (c->mixed && !Q) return GKS_ERR_ARG;
    if (!face_states && c->slab_planes) return GKS_ERR_STATE;
    const void *fs = face_states ? face_states : c->fs;
    double *fr = face_flux ? face_flux : c->frec;
    if (c->mixed && launch_q_to_ff(5 * c->g.n, Q, c->Qv, c->Qv + 5 * c->g.n, c->stream))
        return GKS_ERR_CUDA;
    return launch_ok(flux_any(c, whole_grid(c->g), Q, fs, dt_dev, fr));
}

int gks_flux_points(gks_ctx *c, const double *s_l, const double *s_r, int n,
                    const double *dt_dev, double *out) {
    if (!c || n < 0) return GKS_ERR_ARG;
    if (n == 0) return GKS_OK;  // no points: nothing is read or written
    if (!s_l || !s_r || !dt_dev || !out) return GKS_ERR_ARG;
    return launch_ok(launch_flux_points(c->P, s_l, s_r, n, dt_dev, out, c->status, c->stream));
}

int gks_step(gks_ctx *c, double *Q, double *G, int nsteps, double t_stop, double *t_dev,
             double *dt_host_last) {
    if (!c || !Q || nsteps < 0) return GKS_ERR_ARG;
    const bool cgks = c->P.scheme == GKS_SCHEME_CGKS5;
    if (cgks && !G) return GKS_ERR_ARG;
    double *dt = dt_slot(c);
    for (int s = 0; s < nsteps; ++s) {
        time_open(c);
        int rc = launch_dt(c->g, c->P, Q, red_slot(c), dt, t_dev, t_stop, c->stream);
        if (rc) return GKS_ERR_CUDA;
        time_close(c, kTimeDt);
        if (!cgks) {
            if ((rc = stage_faces(c, Q, nullptr, dt))) return GKS_ERR_CUDA;
            time_open(c);
            if ((rc = launch_update(c->g, c->P, 0, c->frec, dt, Q, nullptr, nullptr, nullptr,
                                    nullptr, nullptr, c->status, c->stream)))
                return GKS_ERR_CUDA;
            time_close(c, kTimeUpdate);
        } else {
            if ((rc = stage_faces(c, Q, G, dt))) return GKS_ERR_CUDA;
            time_open(c);
            if ((rc = launch_update(c->g, c->P, 1, c->frec, dt, Q, G, c->Qs, c->Gs, c->Acc, c->S1,
                                    c->status, c->stream)))
                return GKS_ERR_CUDA;
            time_close(c, kTimeUpdate);
            if ((rc = stage_faces(c, c->Qs, c->Gs, dt))) return GKS_ERR_CUDA;
            time_open(c);
            if ((rc = launch_update(c->g, c->P, 2, c->frec, dt, Q, G, c->Qs, c->Gs, c->Acc, c->S1,
                                    c->status, c->stream)))
                return GKS_ERR_CUDA;
            time_close(c, kTimeUpdate);
        }
    }
    if (dt_host_last) {
        int st = 0;
        // an enqueued copy into st must finish before st goes out of scope
        if (cudaMemcpyAsync(dt_host_last, dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            return GKS_ERR_CUDA;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GKS_ERR_CUDA;
        if (st) return GKS_ERR_NONPHYSICAL;
    }
    return GKS_OK;
}

int gks_step_host(gks_ctx *c, double *Q, double *G, int nsteps, double t_stop, double *t) {
    if (!c || !Q || nsteps < 0) return GKS_ERR_ARG;
    const bool cgks = c->P.scheme == GKS_SCHEME_CGKS5;
    if (cgks && !G) return GKS_ERR_ARG;
    const size_t qn = (size_t)5 * c->g.n;
    if (!c->hQ) {
        int rc;
        if ((rc = dalloc(&c->hT, 1)) || (cgks && (rc = dalloc(&c->hG, 3 * qn))) ||
            (rc = dalloc(&c->hQ, qn))) {
            cudaFree(c->hT);
            cudaFree(c->hG);
            c->hT = nullptr;
            c->hG = nullptr;
            return rc;
        }
    }
    const size_t qb = qn * sizeof(double);
    // on any failure after a copy was enqueued, wait for the stream before
    // returning: the copies read and write the caller's host buffers
    if (cudaMemcpyAsync(c->hQ, Q, qb, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        (cgks && cudaMemcpyAsync(c->hG, G, 3 * qb, cudaMemcpyHostToDevice, c->stream) !=
                     cudaSuccess) ||
        (t && cudaMemcpyAsync(c->hT, t, sizeof(double), cudaMemcpyHostToDevice, c->stream) !=
                  cudaSuccess)) {
        cudaStreamSynchronize(c->stream);
        return GKS_ERR_CUDA;
    }
    const int rc = gks_step(c, c->hQ, cgks ? c->hG : nullptr, nsteps, t_stop, t ? c->hT : nullptr,
                            nullptr);
    if (rc) {
        cudaStreamSynchronize(c->stream);
        return rc;
    }
    int st = 0;
    if (cudaMemcpyAsync(Q, c->hQ, qb, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        (cgks && cudaMemcpyAsync(G, c->hG, 3 * qb, cudaMemcpyDeviceToHost, c->stream) !=
                     cudaSuccess) ||
        (t && cudaMemcpyAsync(t, c->hT, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
                  cudaSuccess) ||
        cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        return GKS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GKS_ERR_CUDA;
    return st ? GKS_ERR_NONPHYSICAL : GKS_OK;
}

namespace {
// the line-averaged-derivative form needs the FP64 CGKS-5th on a periodic
// grid (uniform or stretched); its buffers and tables are set up on first
// use
int lines_ready(gks_ctx *c) {
    if (c->P.scheme != GKS_SCHEME_CGKS5 || c->mixed) return GKS_ERR_STATE;
    if (c->g.bc[0] != GKS_BC_PERIODIC || c->g.bc[1] != GKS_BC_PERIODIC ||
        c->g.bc[2] != GKS_BC_PERIODIC)
        return GKS_ERR_STATE;
    if (c->lrec) return GKS_OK;
    const int t = upload_recon_tables_lines();
    if (t) return t == -1 ? GKS_ERR_ARG : GKS_ERR_CUDA;
    int rc;
    const size_t n = (size_t)c->g.n;
    if ((rc = dalloc(&c->Ls, 60 * n)) || (rc = dalloc(&c->LS1, 60 * n)) ||
        (rc = dalloc(&c->lrec, 270 * n))) {
        cudaFree(c->Ls);
        cudaFree(c->LS1);
        c->Ls = c->LS1 = nullptr;
        return rc;
    }
    return GKS_OK;
}
}  // namespace

int gks_reconstruct_lines(gks_ctx *c, const double *Q, const double *L, double *face_states) {
    if (!c || !Q || !L) return GKS_ERR_ARG;
    int rc;
    if ((rc = lines_ready(c))) return rc;
    if (!face_states && c->slab_planes) return GKS_ERR_STATE;
    return launch_ok(launch_recon5_lines(c->g, c->P, Q, L, face_states ? face_states : (double *)c->fs,
                                         c->stream));
}

int gks_step_lines(gks_ctx *c, double *Q, double *L, int nsteps, double t_stop, double *t_dev,
                   double *dt_host_last) {
    if (!c || !Q || !L || nsteps < 0) return GKS_ERR_ARG;
    int rc;
    if ((rc = lines_ready(c))) return rc;
    if (c->slab_planes) return GKS_ERR_STATE;  // the face states of the whole grid at once
    double *dt = dt_slot(c), *fs = (double *)c->fs;
    for (int s = 0; s < nsteps; ++s) {
        time_open(c);
        if (launch_dt(c->g, c->P, Q, red_slot(c), dt, t_dev, t_stop, c->stream)) return GKS_ERR_CUDA;
        time_close(c, kTimeDt);
        for (int stage = 1; stage <= 2; ++stage) {
            const double *Qx = stage == 1 ? Q : c->Qs, *Lx = stage == 1 ? L : c->Ls;
            time_open(c);
            if (launch_recon5_lines(c->g, c->P, Qx, Lx, fs, c->stream)) return GKS_ERR_CUDA;
            time_close(c, kTimeRecon);
            time_open(c);
            if (launch_flux_faces_lines(c->g, c->P, fs, dt, c->lrec, c->status, c->stream))
                return GKS_ERR_CUDA;
            time_close(c, kTimeFlux);
            time_open(c);
            if (launch_update_lines(c->g, c->P, stage, c->lrec, dt, Q, L, c->Qs, c->Ls, c->Acc,
                                    c->LS1, c->status, c->stream))
                return GKS_ERR_CUDA;
            time_close(c, kTimeUpdate);
        }
    }
    if (dt_host_last) {
        int st = 0;
        if (cudaMemcpyAsync(dt_host_last, dt, sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
                cudaSuccess) {
            cudaStreamSynchronize(c->stream);
            return GKS_ERR_CUDA;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GKS_ERR_CUDA;
        if (st) return GKS_ERR_NONPHYSICAL;
    }
    return GKS_OK;
}

int gks_lines_gradients(gks_ctx *c, const double *L, double *G) {
    if (!c || !L || !G) return GKS_ERR_ARG;
    return launch_ok(launch_lines_to_grad(c->g.n, L, G, c->stream));
}

int gks_diagnostics(gks_ctx *c, const double *Q, const double *G, double *out) {
    if (!c || !Q || !out) return GKS_ERR_ARG;
    double *od = diag_slot(c);
    if (launch_diagnostics(c->g, c->P, Q, G, c->partials, c->diag_blocks, od, c->stream))
        return GKS_ERR_CUDA;
    int st = 0;
    if (cudaMemcpyAsync(out, od, 12 * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess) {
        cudaStreamSynchronize(c->stream);
        return GKS_ERR_CUDA;
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GKS_ERR_CUDA;
    return st ? GKS_ERR_NONPHYSICAL : GKS_OK;
}

int gks_set_indicator(gks_ctx *c, const float *params, float theta) {
    if (!c || !params || !(theta > 0.0f && theta <= 1.0f)) return GKS_ERR_ARG;
    if (!(c->P.scheme == GKS_SCHEME_CGKS5 && c->mixed && c->opt.indicator)) return GKS_ERR_STATE;
    if (upload_indicator(params, theta)) return GKS_ERR_CUDA;
    c->indicator_on = 1;
    return GKS_OK;
}

int gks_indicator_skips(gks_ctx *c, unsigned long long *count) {
    if (!c || !count) return GKS_ERR_ARG;
    if (cudaMemcpyAsync(count, c->skips, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->skips, 0, sizeof(unsigned long long), c->stream) != cudaSuccess) {
        cudaStreamSynchronize(c->stream);  // no copy into *count left in flight
        return GKS_ERR_CUDA;
    }
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? GKS_OK : GKS_ERR_CUDA;
}

int gks_indicator_dump(gks_ctx *c, const double *Q, const double *G, float label_eps, float *x,
                       float *chi, float *y) {
    if (!c || !Q || !G || !x || !chi || !y || !(label_eps >= 0.0f)) return GKS_ERR_ARG;
    if (c->P.scheme != GKS_SCHEME_CGKS5) return GKS_ERR_STATE;
    if (c->mixed) {
        if (make_views(c, Q, G) ||
            launch_indicator_dump(c->g, Q, G, c->Gf, c->Qv, c->Qv + 5 * c->g.n, x, chi, c->stream))
            return GKS_ERR_CUDA;
    } else if (launch_indicator_dump(c->g, Q, G, nullptr, nullptr, nullptr, x, chi, c->stream)) {
        return GKS_ERR_CUDA;
    }
    if (launch_labels(chi, y, 5 * c->g.n, label_eps, c->stream)) return GKS_ERR_CUDA;
    return GKS_OK;
}

int gks_recon_matrix(double *R) {
    if (!R) return GKS_ERR_ARG;
    ReconTables *t = new (std::nothrow) ReconTables;
    if (!t) return GKS_ERR_NOMEM;
    const int rc = build_recon_tables(t);
    if (rc == 0) std::memcpy(R, t->R, sizeof(t->R));
    delete t;
    return rc == 0 ? GKS_OK : GKS_ERR_ARG;
}

int gks_recon_matrix_lines(double *R) {
    if (!R) return GKS_ERR_ARG;
    ReconTablesLines *t = new (std::nothrow) ReconTablesLines;
    if (!t) return GKS_ERR_NOMEM;
    const int rc = build_recon_tables_lines(t);
    if (rc == 0) std::memcpy(R, t->R, sizeof(t->R));
    delete t;
    return rc == 0 ? GKS_OK : GKS_ERR_ARG;
}

int gks_kernel_timing(gks_ctx *c, int on) {
    if (!c || (on != 0 && on != 1)) return GKS_ERR_ARG;
    if (on) {
        if (!c->t_recs) {
            c->t_recs = new (std::nothrow) std::vector<KernelRec>();
            if (!c->t_recs) return GKS_ERR_NOMEM;
        }
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GKS_ERR_CUDA;
        time_clear(c);
    }
    c->timing = on;
    return GKS_OK;
}

int gks_kernel_times(gks_ctx *c, double *ms, long long *launches) {
    if (!c || !ms || !launches) return GKS_ERR_ARG;
    for (int k = 0; k < 4; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    if (!c->t_recs) return GKS_OK;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return GKS_ERR_CUDA;
    for (const KernelRec &r : *c->t_recs) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess) return GKS_ERR_CUDA;
        ms[r.kind] += t;
        launches[r.kind] += 1;
    }
    return GKS_OK;
}

int gks_status(gks_ctx *c, int *status) {
    if (!c || !status) return GKS_ERR_ARG;
    if (cudaMemcpyAsync(status, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(c->status, 0, sizeof(int), c->stream) != cudaSuccess) {
        cudaStreamSynchronize(c->stream);  // no copy into *status left in flight
        return GKS_ERR_CUDA;
    }
    return cudaStreamSynchronize(c->stream) == cudaSuccess ? GKS_OK : GKS_ERR_CUDA;
}

}  // extern "C"
