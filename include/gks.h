/*
 * gks.h -- C-ABI of the GB300 (sm_103a) CGKS-5th / GKS-2nd hot path.
 *
 * The library advances the compressible Navier-Stokes equations on a
 * Cartesian grid (periodic or with symmetry / outflow boundaries, uniform
 * or stretched along each axis) with the gas-kinetic schemes compared in
 * Yang, Zhao & Xu, "Performance evaluation of high-order compact and
 * second-order gas-kinetic schemes in compressible flow simulations":
 * CGKS-5th (Sec. 3.2: compact fifth-order reconstruction with GENO weights,
 * two-stage fourth-order time stepping, Sec. 3.4) and GKS-2nd (Sec. 3.3:
 * least-squares linear reconstruction with the Venkatakrishnan limiter,
 * second-order time stepping). The interface flux is the time-accurate
 * gas-kinetic (BGK) flux of Sec. 2.
 *
 * Conventions shared by every entry point
 *   - Pointers to state arrays are DEVICE pointers (CUDA global memory on
 *     the context's device), 8-byte aligned, owned by the caller.
 *   - Q     : double[5][nz][ny][nx], x fastest; the cell averages of
 *             (rho, rho U, rho V, rho W, rho E).
 *   - gradQ : double[5][3][nz][ny][nx]; the cell-averaged gradient
 *             (d/dx, d/dy, d/dz) of each conserved variable (CGKS-5th
 *             only; pass NULL for GKS-2nd).
 *   - Gas constant R = 1, temperature T = p/rho.
 *   - All work is enqueued asynchronously on the CUDA stream given to
 *     gks_init (NULL = the legacy default stream); no entry point
 *     synchronises unless stated.
 *   - Return codes: GKS_OK or a negative GKS_ERR_* value; nothing throws
 *     across the ABI and no kernel traps the GPU. Arguments are checked on
 *     the host before any launch. Device-side conditions (rho <= 0, p <= 0,
 *     non-finite values) set a status word that the next synchronising
 *     call returns as GKS_ERR_NONPHYSICAL.
 */
#ifndef GKS_H
#define GKS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GKS_OK = 0,
    GKS_ERR_ARG = -1,          /* invalid argument (checked before launch) */
    GKS_ERR_CUDA = -2,         /* a CUDA runtime call failed                */
    GKS_ERR_NONPHYSICAL = -3,  /* rho <= 0, p <= 0 or non-finite state seen */
    GKS_ERR_TIMEOUT = -4,      /* a bounded device wait gave up             */
    GKS_ERR_STATE = -5,        /* call out of order / wrong scheme          */
    GKS_ERR_NOMEM = -6         /* device allocation failed                  */
};

enum { GKS_SCHEME_GKS2 = 0, GKS_SCHEME_CGKS5 = 1 };
enum { GKS_PREC_FP64 = 0, GKS_PREC_MIXED = 1 };
/* Boundary of one axis. A ghost cell beyond a non-periodic boundary is the
 * mirror image of the cell inside it: average s Q, derivative along the
 * normal -s dQ/dn, along the boundary s dQ/dt, with s = -1 for the normal
 * momentum of a symmetry plane (a free-slip, adiabatic wall) and s = +1
 * otherwise (outflow: zero normal derivative at the boundary). */
enum { GKS_BC_PERIODIC = 0, GKS_BC_SYMMETRY = 1, GKS_BC_OUTFLOW = 2 };

typedef struct gks_ctx gks_ctx; /* opaque; created by gks_init */

typedef struct {
    int scheme;      /* GKS_SCHEME_GKS2 or GKS_SCHEME_CGKS5                  */
    int nonlinear;   /* 1: GENO (CGKS-5th) / Venkatakrishnan (GKS-2nd);
                        0: the linear variants of Sec. 4 (chi = 1, phi = 1) */
    int precision;   /* GKS_PREC_FP64 or GKS_PREC_MIXED                      */
    int indicator;   /* 1: learned smoothness indicator (CGKS-5th, mixed)    */
    int mu_law;      /* 0: constant mu; 1: Sutherland law of Sec. 4.2 with
                        T normalised by T_ref                                */
    int inviscid;    /* 1: tau = eps_tau dt + C_tau |dp/sp| dt (Sec. 4)      */
    double C_tau;    /* Sec. 4 collision-time constant C (default 10)        */
    double eps_tau;  /* Sec. 4 inviscid constant epsilon (default 0.05)      */
    double T_ref;    /* Sutherland reference temperature (default 1)         */
    double theta;    /* indicator threshold in (0, 1] (default 0.9)          */
    int slab_planes; /* face-state buffer size for gks_step: 0 (default) the
                        whole grid when it fits in 40% of the free device
                        memory at gks_init, else the most z-planes that fit
                        in 25% of it; > 0: slabs of this many z-planes
                        (nz or more: the whole grid). gks_step then runs
                        reconstruction and flux slab by slab (each slab
                        also reconstructs the plane below it); the results
                        equal the whole-grid ones bit for bit.           */
    int reserved;    /* set to 0                                            */
    int bc[3];       /* GKS_BC_* per axis (x, y, z); default periodic        */
    int reserved2;   /* set to 0                                            */
    const double *h[3]; /* stretched mesh (Sec. 3.2, last paragraph): HOST
                        arrays of the nx, ny, nz cell sizes of each axis
                        (copied by gks_init; NULL: uniform L/n, and Lx, Ly,
                        Lz are then the box; an axis with sizes ignores its
                        L). Each cell is mapped to the one reference cell:
                        its stencil is taken in index coordinates, the
                        neighbours' gradients scaled by their own sizes,
                        and the derivatives mapped back with 1/h.
                        Non-periodic or stretched grids run the general
                        kernels and have no learned indicator.             */
} gks_options;

/* Fill *opt with the defaults: CGKS-5th, nonlinear, FP64, no indicator,
 * constant mu, viscous tau, C_tau = 10, eps_tau = 0.05, T_ref = 1,
 * theta = 0.9, slab_planes = 0 (automatic). */
void gks_default_options(gks_options *opt);

/* Create a context for one grid (Sec. 4 problem statement: gamma, Pr, mu,
 * grid and CFL).
 *   gamma > 1, Pr > 0, mu >= 0 (mu0 of the Sutherland law when mu_law = 1),
 *   0 < cfl <= 1, nx, ny, nz >= 1 with nx ny nz <= 2^31 cells, Lx, Ly,
 *   Lz > 0 (periodic box).
 *   opt        : NULL for gks_default_options.
 *   cuda_stream: a cudaStream_t (or NULL); the context enqueues all of its
 *                work there.
 * Allocates the library-owned device workspace (face states, face fluxes,
 * stage buffers) on the current device; freed by gks_destroy.
 * Returns GKS_ERR_ARG, GKS_ERR_NOMEM or GKS_ERR_CUDA on failure (then
 * *out = NULL). */
int gks_init(gks_ctx **out, double gamma, double Pr, double mu, double cfl,
             int nx, int ny, int nz, double Lx, double Ly, double Lz,
             const gks_options *opt, void *cuda_stream);

void gks_destroy(gks_ctx *ctx);
const char *gks_strerror(int code);

/* Bytes of the face-state buffer written by gks_reconstruct:
 * 6 faces x K Gauss points x 20 components x nx*ny*nz cells, K = 4
 * (CGKS-5th) or 1 (GKS-2nd), 8 bytes each (FP64) or 4 (mixed). */
size_t gks_face_state_bytes(const gks_ctx *ctx);
/* Bytes of the face-flux records written by gks_flux: 3 x 30 x cells x 8,
 * plus, on a grid with a non-periodic or stretched axis, 3 x 30 x np x 8
 * for the faces on the high boundary (np = max(ny nz, nx nz, nx ny)). */
size_t gks_face_flux_bytes(const gks_ctx *ctx);
/* z-planes per slab of gks_step's reconstruction + flux (see slab_planes in
 * gks_options): 0 when the context's face-state buffer holds the whole grid,
 * -1 for a NULL context. */
int gks_slab_planes(const gks_ctx *ctx);

/* a0 -- time step of Sec. 4: dt = CFL min( min_{cells,d} h_d/(|U_d| + c),
 * h_min^2/(3 nu_max) ) (the viscous bound only when the flow is viscous).
 * Writes the FP64 scalar to *dt_dev (device pointer). Asynchronous. */
int gks_compute_dt(gks_ctx *ctx, const double *Q, double *dt_dev);

/* a1/a2 -- spatial reconstruction (Sec. 3.2 CGKS-5th: S^data-5th, the
 * constrained least squares of Eq. compact-big-5, the sub-stencil
 * polynomials of Eq. compact-sub-2 and the GENO combination of
 * Eq. weno-new; Sec. 3.3 GKS-2nd: least squares + Venkatakrishnan).
 * face_states (device, gks_face_state_bytes) receives, for every cell c,
 * face f (0..5 = -x, +x, -y, +y, -z, +z), Gauss point k and component q,
 * element ((f*K + k)*20 + q)*cells + c: the reconstructed state in the
 * face frame (normal axis d = f/2, tangential axes (d+1)%3, (d+2)%3):
 *   q 0..4   (rho, rho u_n, rho u_t1, rho u_t2, rho E)
 *   q 5..9   d/dn of the same, q 10..14 d/dt1, q 15..19 d/dt2.
 * Gauss point k sits at tangential offsets (+-g, +-g) h, g = 1/(2 sqrt 3),
 * bit 0 of k choosing the sign along t1 and bit 1 along t2 (K = 1: the face
 * midpoint). Precision GKS_PREC_MIXED stores FP32 values, the components
 * q 0..4 as offsets from the reconstructing cell's own average (the flux
 * adds the FP64 average back). face_states = NULL uses the context's own
 * buffer. */
int gks_reconstruct(gks_ctx *ctx, const double *Q, const double *gradQ,
                    void *face_states);

/* a3 -- gas-kinetic flux of Sec. 2 (Eq. flux, its time integrals over
 * [0, dt] and [0, dt/2], F^n and F_t^n of Eq. deri-t-f, the collision time
 * of Sec. 4, the Prandtl correction of the energy flux, and the interface
 * values of the update model of Sec. 3.4), averaged over each face's Gauss
 * points. Q: the cell averages the face states were reconstructed from
 * (required in mixed precision, ignored in FP64); face_states: as written by
 * gks_reconstruct (NULL = the context's buffer); dt_dev: device FP64 scalar.
 * Mixed precision evaluates the Maxwellian slopes and the moments of the
 * tau-weighted terms in FP32 and everything that carries the pressure or
 * the time integration in FP64. face_flux (device,
 * gks_face_flux_bytes; NULL = the context's buffer) receives for axis d and
 * the face on the low-d side of cell c, element (d*30 + q)*cells + c:
 *   F^n(5), F_t^n(5), Q^l(5), dQ^l/dt(5), Q^r(5), dQ^r/dt(5)
 * in the global frame (the interface values only for CGKS-5th; GKS-2nd
 * leaves q 10..29 untouched). On a non-periodic axis d the face on the low
 * boundary pairs the cell with its mirror ghost, and the faces on the high
 * boundary follow the 90 x cells records: element
 * 90*cells + (d*30 + q)*np + p, p = j + ny k (d = 0), i + nx k (d = 1),
 * i + nx j (d = 2). */
int gks_flux(gks_ctx *ctx, const double *Q, const void *face_states,
             const double *dt_dev, double *face_flux);

/* The same flux (FP64 arithmetic) at n independent Gauss points:
 * s_l, s_r device double[20][n] face-frame states (layout of one Gauss point
 * of gks_reconstruct), out device double[30][n] in the face frame.
 * n = 0: returns GKS_OK without reading or writing (the pointers may then
 * be NULL). */
int gks_flux_points(gks_ctx *ctx, const double *s_l, const double *s_r,
                    int n, const double *dt_dev, double *out);

/* a0-a4 -- advance nsteps time steps (or until *t_dev reaches t_stop):
 * per step dt (a0) on the device, then for GKS-2nd one stage
 * Q += dt L + dt^2/2 dL/dt, for CGKS-5th the two-stage fourth-order update
 * of Q and of gradQ through the interface values (Sec. 3.4).
 * t_dev: device FP64 scalar, advanced in place (NULL: no time tracking and
 * t_stop is ignored). dt_host_last: if non-NULL
 * the call synchronises the stream, stores the last dt there and returns
 * GKS_ERR_NONPHYSICAL if the status word was set; if NULL the call is fully
 * asynchronous. Q and gradQ are updated in place. */
int gks_step(gks_ctx *ctx, double *Q, double *gradQ, int nsteps,
             double t_stop, double *t_dev, double *dt_host_last);

/* a0-a4 for callers that hold the state in HOST memory: copies Q (and, for
 * CGKS-5th, gradQ) host -> device into buffers the context owns, advances
 * nsteps steps exactly as gks_step, and copies the state (and *t) back.
 * Q, gradQ: caller-owned host arrays in the layouts of gks_step (pinned
 * memory for full copy bandwidth; pageable memory works); t: host scalar,
 * in/out simulation time, or NULL (no time tracking, t_stop ignored).
 * Synchronising. The device buffers (the state's size plus one double) are
 * allocated on the first call and kept until gks_destroy; GKS_ERR_NOMEM if
 * that fails. Returns GKS_ERR_NONPHYSICAL if the status word was set. */
int gks_step_host(gks_ctx *ctx, double *Q, double *gradQ, int nsteps, double t_stop,
                  double *t);

/* CGKS-5th with the target cell's own data as its 12 line-averaged
 * derivatives (the set S^0 of Sec. 3.1-3.2: per variable and axis a, the
 * derivative along a averaged over the line through the cell between the
 * face Gauss points k of its two faces normal to a) instead of its averaged
 * gradient. L: device double[5][12][n], entry (v, 4a + k, cell), line k
 * through tangential position (+-, +-) of axis (a+1)%3 (bit 0 of k) and
 * (a+2)%3 (bit 1); the averaged gradient along a is the mean of its four
 * lines. FP64 CGKS-5th contexts on periodic grids (uniform or stretched)
 * only (GKS_ERR_STATE otherwise); the first call allocates 390 doubles per cell (face records
 * [3][90][n], two line buffers) kept until gks_destroy.
 *
 * gks_reconstruct_lines: the face states of every cell, layout of
 * gks_reconstruct (FP64), into face_states (device, or NULL: the context's
 * buffer, GKS_ERR_STATE when that holds a slab only).
 *
 * gks_step_lines: nsteps two-stage steps as gks_step; Q as there, each line
 * advanced from the time-dependent interface values at its two end points
 * (Sec. 3.4 point by point): stage 1 L* = (Q^l(dt/2) at the high face -
 * Q^r(dt/2) at the low face)/h_a, stage 2 from the t = 0 values plus dt
 * times the stage-2 time derivatives. Asynchronous unless dt_host_last is
 * non-NULL (then as gks_step). GKS_ERR_STATE when the context's face-state
 * buffer holds a slab only.
 *
 * gks_lines_gradients: G[v][a][cell] (device double[15][n]) = the mean of
 * the four lines of (v, a), e.g. for gks_diagnostics. Asynchronous. */
int gks_reconstruct_lines(gks_ctx *ctx, const double *Q, const double *L, double *face_states);
int gks_step_lines(gks_ctx *ctx, double *Q, double *L, int nsteps, double t_stop, double *t_dev,
                   double *dt_host_last);
int gks_lines_gradients(gks_ctx *ctx, const double *L, double *G);

/* a5 -- diagnostics (Sec. 4.1/4.2), synchronising; out (host, 12 doubles):
 *  [0] E_k  = (1/|Omega|) sum rho |U|^2/2 h^3 (divide by rho0 U0^2 for the
 *            paper's normalisation)
 *  [1] eps_S = (1/|Omega|) sum mu |curl U|^2 h^3
 *  [2] eps_D = (4/3)(1/|Omega|) sum mu (div U)^2 h^3
 *  [3] min rho, [4] min p, [5..9] sum Q h^3, [10] count of non-physical
 *  cells, [11] max_d(|U_d| + c).
 * Velocity gradients from gradQ (CGKS-5th) or central differences of the
 * cell averages (gradQ = NULL). Returns GKS_ERR_NONPHYSICAL if the status
 * word was set. */
int gks_diagnostics(gks_ctx *ctx, const double *Q, const double *gradQ,
                    double *out);

/* Read and clear the device status word (synchronising): 0 or a bit mask
 * (1: non-physical state, 2: non-finite value). */
int gks_status(gks_ctx *ctx, int *status);

/* Host-only, no GPU needed: the CGKS-5th reconstruction matrix R (34 x 63,
 * row major) with a = R d, the least-squares solution of Eq. compact-big-5
 * (neighbour averages exact; derivative rows weighted 1, except the edge
 * neighbours' tangential derivatives, weighted 0.1 -- the paper's h2,
 * chosen near the minimum of the system's condition number)
 * for the normalised data vector d of S^data-5th (column order: the 6
 * face-neighbour differences, the 12 edge-neighbour differences, the 18
 * scaled face-neighbour gradients, the 24 scaled edge-neighbour tangential
 * derivatives, the 3 scaled own gradients) and a over the 34 monomials
 * x^a y^b z^c/(a! b! c!) minus their cell mean, ordered by degree. R is
 * caller-owned host memory of 34*63 doubles. */
int gks_recon_matrix(double *R);

/* N2 -- host-only: the least-squares matrix of the line form (the cell's
 * own data its 12 line-averaged derivatives; gks_step_lines), the same
 * weighted constrained least squares with the 3 own-gradient rows replaced
 * by the 12 line rows (weight 1; a line's row is the difference of the
 * monomial at its two end points): a = R d, d of 72 entries per variable
 * (the first 60 as for gks_recon_matrix, then line k of axis a at
 * 60 + 4a + k, scaled by h_a). R is caller-owned host memory of 34*72
 * doubles. GKS_ERR_ARG if the tables fail their own reflection-symmetry
 * check. */
int gks_recon_matrix_lines(double *R);

/* a8 -- learned smoothness indicator (an extension of the method: the
 * paper has no such component). A per-(cell, variable) network predicts
 * whether GENO's chi (Eq. weno-new) would equal 1 -- the nonlinear
 * reconstruction collapsing to the linear quartic -- so that confident
 * (cell, variable) pairs skip the nonlinear weights; all others run the
 * full reconstruction. Network: x = the 63-entry data vector of S^data-5th,
 * xh = x/(max|x| + 1e-30), h = max(W1 xh + b1, 0) (8 units),
 * logit = w2 . h + b2. Parameters (gks_mlp_nparams() floats): W1 [8][63]
 * row major, b1 [8], w2 [8], b2. */
int gks_mlp_nparams(void);

/* Training data from the method itself (CGKS-5th context, any precision):
 * for every cell c and variable v, sample s = 5 c + v: x[j*5*cells + s]
 * (j < 63) the FP32 data vector as the mixed-precision reconstruction forms
 * it, chi[s] GENO's chi, y[s] = 1 if chi >= 1 - label_eps else 0. Device
 * buffers owned by the caller. */
int gks_indicator_dump(gks_ctx *ctx, const double *Q, const double *gradQ,
                       float label_eps, float *x, float *chi, float *y);

/* Mean weighted binary cross-entropy over n samples (x: device [63][ld],
 * y: device [n]; samples of label 0 weighted by neg_weight) and its
 * gradient: *loss (device float) and grad (device, gks_mlp_nparams()).
 * Synchronises cuda_stream; allocates its own workspace. */
int gks_mlp_loss_grad(const float *params, const float *x, const float *y,
                      int n, long long ld, float neg_weight, float *loss,
                      float *grad, void *cuda_stream);

/* Adam training in place of params (device) for `epochs` passes of n/batch
 * steps over a seeded coprime-stride permutation of the samples;
 * loss_hist (device, epochs floats, nullable) receives the mean batch loss
 * of each epoch. Deterministic for a given seed. Synchronises cuda_stream;
 * allocates its own workspace. */
int gks_mlp_train(float *params, const float *x, const float *y, int n,
                  long long ld, int epochs, int batch, float lr,
                  float neg_weight, unsigned seed, float *loss_hist,
                  void *cuda_stream);

/* Activate the indicator on a context created with precision
 * GKS_PREC_MIXED, scheme CGKS-5th and options.indicator = 1: params (HOST,
 * gks_mlp_nparams() floats) become the device's network (one per device,
 * shared by all contexts on it); a (cell, variable) skips GENO when
 * sigmoid(logit) >= theta (0 < theta <= 1; theta = 1 never skips). */
int gks_set_indicator(gks_ctx *ctx, const float *params, float theta);

/* Number of (cell, variable) reconstructions that skipped GENO since the
 * last call (synchronising; resets the count). */
int gks_indicator_skips(gks_ctx *ctx, unsigned long long *count);

/* a9 -- batched ensemble of independent CGKS-5th instances of uneven size
 * (an extension of the method). Instance i has grid dims[3i..3i+2], box
 * lengths[3i..3i+2] and physics phys[8i..8i+7] = gamma, Pr, mu, CFL,
 * mu_law (0/1), inviscid (0/1), C_tau, eps_tau; opt (NULL = defaults) must
 * select CGKS-5th and gives the precision, the nonlinear switch and T_ref.
 * The caller owns the states in two concatenated device arenas:
 * Q_all[5 * total] with instance i's block [5][cells_i] at
 * 5 * gks_ensemble_offset(e, i), and gradQ_all[15 * total] with its block
 * [5][3][cells_i] at 15 * offset. The library splits the instances into
 * work items of `tile` cells; a step is one persistent launch over the
 * items of all instances whose blocks meet at grid-wide barriers between
 * the phases (dt, reconstruction, flux, update; mode 1, the default), or
 * one persistent launch per phase (mode 0, and always with the learned
 * indicator on); every instance keeps its own dt and time. Work is
 * enqueued on an internal stream ordered after and before cuda_stream. */
typedef struct gks_ensemble gks_ensemble;
int gks_ensemble_create(gks_ensemble **out, int n_instances, const int *dims,
                        const double *lengths, const double *phys,
                        const gks_options *opt, void *cuda_stream);
void gks_ensemble_destroy(gks_ensemble *e);
/* First cell of instance i in the arenas; i = n_instances: total cells;
 * -1 for an invalid argument. */
long long gks_ensemble_offset(const gks_ensemble *e, int i);
/* Work-item size in cells (32 .. 2^22); rebuilds the work list. */
int gks_ensemble_set_tile(gks_ensemble *e, int tile_cells);
/* Advance every instance nsteps steps (each stops at t_stop). use_graph:
 * capture one step into a CUDA graph (re-captured when Q, gradQ, the tile,
 * t_stop or the indicator change) and replay it nsteps times. */
int gks_ensemble_step(gks_ensemble *e, double *Q, double *gradQ, int nsteps,
                      double t_stop, int use_graph);
/* Synchronising: per-instance times (host array of n_instances) and the
 * status word; returns GKS_ERR_TIMEOUT if a barrier wait of the
 * single-launch step ran out (20 s; the launch then returned without
 * finishing the step), else GKS_ERR_NONPHYSICAL if the word is set. */
int gks_ensemble_times(gks_ensemble *e, double *t_host, int *status);
/* Step mode (an implementation choice, no counterpart in the paper): 1 one
 * launch per step (default), 0 one launch per phase. Synchronises the
 * ensemble's stream; GKS_ERR_ARG for another value. gks_ensemble_mode
 * returns the mode (-1 for NULL). */
int gks_ensemble_set_mode(gks_ensemble *e, int mode);
int gks_ensemble_mode(const gks_ensemble *e);
/* Self-check of the single-launch step's bounded barrier wait (no
 * counterpart in the paper): launches, on cuda_stream, two blocks that
 * wait for a third that never arrives; their waits must give up after
 * limit_s seconds (0 < limit_s <= 10) and report it. Returns
 * GKS_ERR_TIMEOUT when they did (the expected result), GKS_OK if the wait
 * ended otherwise, GKS_ERR_ARG, GKS_ERR_NOMEM or GKS_ERR_CUDA.
 * Synchronises cuda_stream; allocates 16 bytes of device memory. */
int gks_barrier_timeout_check(double limit_s, void *cuda_stream);
/* Autotuner: times one graph-replayed step for work-item sizes
 * 256 .. 8192 cells on a scratch copy of the state (the state and the
 * instance times are unchanged), keeps the fastest; *tile_out and *best_ms
 * (nullable) report it. Allocates and frees its scratch. */
int gks_ensemble_autotune(gks_ensemble *e, const double *Q, const double *gradQ,
                          int *tile_out, float *best_ms);
/* Indicator training data from all instances: x [63][5 total], chi and y
 * [5 total] (sample 5 (offset_i + c) + v), as gks_indicator_dump. */
int gks_ensemble_dump(gks_ensemble *e, const double *Q, const double *gradQ,
                      float label_eps, float *x, float *chi, float *y);
/* The learned indicator for a mixed-precision ensemble (see gks_set_indicator). */
int gks_ensemble_set_indicator(gks_ensemble *e, const float *params, float theta);

/* Per-kernel device time of the steps that follow (no counterpart in the
 * paper; it gives the benchmark each kernel's launch duration inside its
 * timed region). on = 1 synchronises the stream, discards earlier records
 * and starts recording a CUDA event on the context's stream before and
 * after every launch gks_step makes (time step, reconstruction, flux,
 * update; one reconstruction and one flux launch per z-slab); the events
 * add no synchronisation. on = 0 stops recording (the records are kept).
 * Do not capture gks_step in a CUDA graph while recording is on.
 * Returns GKS_ERR_ARG for a NULL context or on not 0/1, GKS_ERR_NOMEM,
 * GKS_ERR_CUDA. */
int gks_kernel_timing(gks_ctx *ctx, int on);

/* The recorded times: synchronises the stream, then ms[k] = summed
 * milliseconds and launches[k] = number of launches of kind k = 0
 * reconstruction, 1 flux, 2 update, 3 time step (host arrays of 4) since
 * the last gks_kernel_timing(ctx, 1); zeros if nothing was recorded.
 * Returns GKS_ERR_ARG for NULL arguments, GKS_ERR_CUDA. */
int gks_kernel_times(gks_ctx *ctx, double *ms, long long *launches);

/* Measured fused multiply-add throughput of this device (no counterpart in
 * the paper; it is the denominator of the FP64 and FP32 roofline fractions
 * of the ALU-bound kernels). precision: GKS_PREC_FP64 times double FMAs,
 * GKS_PREC_MIXED float FMAs. One kernel of independent FMA chains over
 * 4 x (SM count) blocks of 256 threads, best of three launches timed with
 * CUDA events on cuda_stream (NULL = legacy default stream), after one
 * warm-up launch; *flops = 2 FMAs per FMA instruction lane / second,
 * *ms = the best launch's duration (~30 ms at GB300's nominal rates).
 * Allocates and frees a 1.2 MB device buffer and synchronises the stream.
 * Returns GKS_ERR_ARG for a bad precision or NULL outputs, GKS_ERR_NOMEM,
 * GKS_ERR_CUDA. */
int gks_fma_rate(int precision, void *cuda_stream, double *flops, double *ms);

/* Diagnostics without any device allocation (the paper has no counterpart:
 * this serves callers of this library, not the method).
 * For callers that cannot allocate device memory: a monitor that samples
 * the diagnostics of a running simulation from outside the solver (another
 * thread, a checkpoint hook, code that holds only device pointers and no
 * gks_ctx). Large grids leave little free HBM, so an allocation made just to
 * sample diagnostics may fail or evict the simulation's own buffers.
 * Computes the same 12 values as gks_diagnostics (the same kernels and
 * block count: equal bit for bit) for the state Q / gradQ (gradQ may be NULL:
 * central differences) of an nx x ny x nz periodic grid of extents Lx, Ly,
 * Lz, gas constant gamma, viscosity mu (Sutherland's law when mu_law = 1,
 * temperature normalised by T_ref). out_dev: caller-owned DEVICE memory for
 * 12 doubles, written asynchronously on cuda_stream (a cudaStream_t or
 * NULL); the call does not synchronise and reads no status word.
 * Scratch: a file-scope device array of 57 KiB (12 partial results for
 * each of at most 608 reduction blocks, whatever the grid size) that every
 * GPU which loads the library holds until the process exits; grids above
 * 2^31 cells (the limit of gks_init) are rejected with GKS_ERR_ARG.
 * Every call overwrites the slots it later reads, so nothing
 * has to be cleared, but all calls on a device share the array: calls that
 * overlap on the GPU (other streams, other threads) race and must be
 * serialised by the caller. The first call on each device looks up the
 * array's device address (with that device current); make that first call
 * before any stream capture. Calls no cudaMalloc, cudaFree or allocating
 * library routine. Returns GKS_ERR_ARG for invalid arguments, GKS_ERR_CUDA
 * if the address lookup or a launch fails. */
int gks_diagnostics_noalloc(const double *Q, const double *gradQ, int nx, int ny,
                            int nz, double Lx, double Ly, double Lz, double gamma,
                            double mu, int mu_law, double T_ref, double *out_dev,
                            void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
