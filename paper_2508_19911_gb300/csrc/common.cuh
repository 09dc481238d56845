// Shared device-side definitions of the GB300 CGKS-5th / GKS-2nd path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gks {

// status word bits (gks_status)
constexpr int kStatusNonphysical = 1;
constexpr int kStatusNonfinite = 2;
constexpr int kStatusTimeout = 4;   // a bounded device wait gave up

// Grid-wide barrier of the ensemble's single-launch step (ensemble_step.cu):
// arrivals, generation, abort word; zeroed before every launch.
struct StepSync {
    unsigned int count, gen;
    int abort, pad;
};

struct GridDesc {
    int nx, ny, nz;
    long long n;     // cells
    double h[3];     // cell sizes of a uniform grid
    // General grids (general = 1; the ensemble and uniform periodic grids
    // leave it 0): per-axis cell sizes on the device (nullptr: the uniform
    // h[a]), boundary kind per axis (0 periodic, 1 symmetry plane, 2
    // outflow: a mirror ghost cell, the normal momentum negated for 1),
    // the smallest cell size, the domain's volume and the size of the
    // boundary-face planes np = max(ny nz, nx nz, nx ny). The records of
    // the faces on the high boundary of a non-periodic axis d follow the
    // [3][30][n] face records as [3][30][np], at plane position j + ny k
    // (d = 0), i + nx k (d = 1), i + nx j (d = 2).
    const double *hs[3];
    double hmin, volume;
    long long np;
    int bc[3];
    int general;
};

struct PhysParams {
    double gamma, Pr, mu0, cfl, C_tau, eps_tau, T_ref;
    double Nint;     // internal degrees of freedom (5 - 3 gamma)/(gamma - 1)
    int mu_law, inviscid, nonlinear, scheme;
};

// One instance of a batched ensemble: its grid, its physics and the index
// of its first cell in the concatenated arenas (every per-cell array of the
// ensemble stores instance i's block [components][cells_i] at component
// stride cells_i, starting at components * off).
struct EnsInst {
    GridDesc g;
    PhysParams P;
    long long off;
};
// A work item of the persistent ensemble kernels: cells [c0, c1) of one
// instance.
struct EnsItem {
    int inst;
    int pad;
    long long c0, c1;
};

__host__ __device__ __forceinline__ long long cell_index(const GridDesc &g, int i, int j, int k) {
    return ((long long)k * g.ny + j) * g.nx + i;
}

__device__ __forceinline__ int wrap(int i, int n) {
    return i < 0 ? i + n : (i >= n ? i - n : i);
}

__host__ __device__ __forceinline__ int axis_len(const GridDesc &g, int a) {
    return a == 0 ? g.nx : (a == 1 ? g.ny : g.nz);
}

// cell size along axis a at coordinate i
__device__ __forceinline__ double cell_h(const GridDesc &g, int a, int i) {
    return g.hs[a] ? __ldg(g.hs[a] + i) : g.h[a];
}

// Coordinate along axis a of the neighbour at x = i + offset: wrapped on a
// periodic axis, mirrored into the grid across a boundary (bit a of flip
// set: the neighbour is the ghost image of that cell).
__device__ __forceinline__ int nb_coord(const GridDesc &g, int a, int x, int &flip) {
    const int m = axis_len(g, a);
    if (g.bc[a] == 0) return wrap(x, m);
    if (x < 0) {
        flip |= 1 << a;
        return -1 - x;
    }
    if (x >= m) {
        flip |= 1 << a;
        return 2 * m - 1 - x;
    }
    return x;
}

// Does the average of conserved variable v change sign in a ghost mirrored
// across the axes of flip? (the momentum normal to a symmetry plane)
__device__ __forceinline__ bool ghost_neg(const GridDesc &g, int v, int flip) {
    if (v < 1 || v > 3) return false;
    return ((flip >> (v - 1)) & 1) && g.bc[v - 1] == 1;
}

// position of a cell in the boundary plane normal to axis d
__device__ __forceinline__ long long plane_pos(const GridDesc &g, int d, int i, int j, int k) {
    return d == 0 ? (long long)j + (long long)g.ny * k
                  : (d == 1 ? (long long)i + (long long)g.nx * k : (long long)i + (long long)g.nx * j);
}

// Mirror of face-frame component q (0..19: values, d/dn, d/dt1, d/dt2 of
// rho, rho u_n, rho u_t1, rho u_t2, rho E) across the face itself, for a
// boundary of kind bc: negated or not.
__host__ __device__ __forceinline__ bool mirror_neg(int q, int bc) {
    const bool normal_mom = (q % 5) == 1 && bc == 1;
    return (q / 5 == 1) != normal_mom;
}

// The face-state buffer holds nzb z-planes starting at the global plane zb
// (periodic), position l = (plane - zb) nx ny + j nx + i, stride nb =
// nx ny nzb. The reconstruction fills all its planes; the flux computes the
// faces of the cells in planes p0..nzb-1 (their low faces need the plane
// below: p0 = 1 for a slab, whose plane 0 is the plane below its first
// cell plane; p0 = 0 for the whole grid, nzb = nz, where plane 0's lower
// neighbour is plane nz - 1 of the same buffer).
struct Slab {
    int zb, nzb, p0, pad;
    long long nb;
};

__host__ __device__ __forceinline__ Slab whole_grid(const GridDesc &g) {
    Slab s;
    s.zb = 0;
    s.nzb = g.nz;
    s.p0 = 0;
    s.pad = 0;
    s.nb = g.n;
    return s;
}

// global cell of buffer position l
__device__ __forceinline__ long long slab_global(const GridDesc &g, const Slab &S, long long l) {
    const long long nxy = (long long)g.nx * g.ny;
    const long long p = l / nxy;
    const long long gz = (S.zb + p) % g.nz;
    return gz * nxy + (l - p * nxy);
}

// dynamic viscosity: constant, or the Sutherland law of Sec. 4.2 with the
// temperature T = p/rho normalised by T_ref
__device__ __forceinline__ double viscosity(const PhysParams &P, double rho, double p) {
    if (P.mu_law == 0) return P.mu0;
    const double th = (p / rho) / P.T_ref;
    return P.mu0 * 1.4042 * th * sqrt(th) / (th + 0.4042);
}

__device__ __forceinline__ void flag_status(int *status, int bits) {
    if (status) atomicOr(status, bits);
}

// Kernel launch helpers (defined in the .cu files)
// reconstruction and flux launchers take the face-state buffer's Slab
int launch_recon5(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                  const double *G, double *fs, cudaStream_t s);
int launch_recon2(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                  double *fs, cudaStream_t s);
int upload_recon_tables(void);
// the FP64 tables (recon_fp64.cu), called by upload_recon_tables
struct ReconTables;
int upload_recon_tables_fp64(const ReconTables &t);
int launch_recon5_ens_fp64(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                           const double *Qa, const double *Ga, double *fsa, cudaStream_t s);
int launch_flux_faces(const GridDesc &g, const Slab &S, const PhysParams &P, const double *fs,
                      const double *dt_dev, double *frec, int *status, cudaStream_t s);
// float-float split of m FP64 values (the averages, once per stage, for
// the mixed reconstruction and flux): hi[i] + lo[i] = x[i]
int launch_q_to_ff(long long m, const double *x, float *hi, float *lo, cudaStream_t s);
int launch_flux_faces_mixed(const GridDesc &g, const Slab &S, const PhysParams &P,
                            const float *fs, const float *Qhi, const float *Qlo,
                            const double *dt_dev, double *frec, int *status, cudaStream_t s);
// FP32 copy of m FP64 values (the cell gradients, once per stage, for the
// mixed reconstruction)
int launch_g_to_f32(long long m, const double *G, float *Gf, cudaStream_t s);
// views of one stage: Gf = FP32 gradients, Qhi/Qlo = float-float averages
int launch_recon5_mixed(const GridDesc &g, const Slab &S, const PhysParams &P, const float *Gf,
                        const float *Qhi, const float *Qlo, float *fs, cudaStream_t s,
                        int indicator, unsigned long long *skips);
// Gf/Qhi/Qlo: the views (mixed context, the caller converts first) or
// nullptr (FP64 context: the FP64 Q, G directly)
int launch_indicator_dump(const GridDesc &g, const double *Q, const double *G, const float *Gf,
                          const float *Qhi, const float *Qlo, float *x, float *chi,
                          cudaStream_t s);
int upload_indicator(const float *params, float theta);
int launch_labels(const float *chi, float *y, long long m, float eps, cudaStream_t s);
int launch_recon2_mixed(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                        float *fs, cudaStream_t s);
int launch_flux_points(const PhysParams &P, const double *sl, const double *sr, int n,
                       const double *dt_dev, double *out, int *status, cudaStream_t s);
int launch_dt(const GridDesc &g, const PhysParams &P, const double *Q, double *red,
              double *dt_dev, double *t_dev, double t_stop, cudaStream_t s);
// stage: 0 GKS-2nd single stage, 1 CGKS first stage, 2 CGKS second stage
int launch_update(const GridDesc &g, const PhysParams &P, int stage, const double *frec,
                  const double *dt_dev, double *Q, double *G, double *Qs, double *Gs,
                  double *Acc, double *S1, int *status, cudaStream_t s);
// CGKS-5th with the line-averaged derivatives as the target cell's data
// (recon_lines.cu; FP64, periodic): L [5][12][n] (line 4a + k of variable
// v along axis a), face records [3][90][n]
int upload_recon_tables_lines(void);
int launch_recon5_lines(const GridDesc &g, const PhysParams &P, const double *Q, const double *L,
                        double *fs, cudaStream_t s);
int launch_flux_faces_lines(const GridDesc &g, const PhysParams &P, const double *fs,
                            const double *dt_dev, double *frec, int *status, cudaStream_t s);
int launch_update_lines(const GridDesc &g, const PhysParams &P, int stage, const double *frec,
                        const double *dt_dev, double *Q, double *L, double *Qs, double *Ls,
                        double *Acc, double *S1, int *status, cudaStream_t s);
int launch_lines_to_grad(long long n, const double *L, double *G, cudaStream_t s);
// diagnostics: nblocks (1..kDiagMaxBlocks) blocks write kDiagSlots partial
// results each to partials, one block reduces them into out_dev
constexpr int kDiagSlots = 12;
constexpr int kDiagMaxBlocks = 152 * 4;
int launch_diagnostics(const GridDesc &g, const PhysParams &P, const double *Q,
                       const double *G, double *partials, int nblocks, double *out_dev,
                       cudaStream_t s);
int diagnostics_blocks(const GridDesc &g);

// the ensemble's time step as one persistent launch (ensemble_step.cu):
// its own copy of the reconstruction tables (FP64 tables and the FP32
// table), the grid it launches, the launch, and a barrier that cannot
// complete (its bounded wait must report kStatusTimeout)
int upload_recon_tables_step(const ReconTables &t, const float *tab, size_t tab_bytes);
int ens_step_grid(int mixed);
int launch_ens_step(const EnsInst *inst, int ninst, const EnsItem *items, int nitems,
                    long long total, int mixed, double *Q, double *G, double *Qs, double *Gs,
                    double *Acc, double *S1, void *fs, float *Gf, float *Qv, double *frec,
                    double *dt, double *t, double *red, double t_stop, StepSync *sync,
                    double limit_s, int *status, cudaStream_t s);
int launch_barrier_timeout(StepSync *sync, int blocks, double limit_s, int *status,
                           cudaStream_t s);

// persistent ensemble kernels (see ensemble.cu)
// mixed ensemble kernels read the arenas' views (Gfa, Qhia, Qloa)
int launch_recon5_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                      int mixed, int indicator, const double *Qa, const double *Ga,
                      const float *Gfa, const float *Qhia, const float *Qloa, void *fsa,
                      unsigned long long *skips, cudaStream_t s);
int launch_indicator_dump_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                              const float *Gfa, const float *Qhia, const float *Qloa, float *x,
                              float *chi, long long total_cells, cudaStream_t s);
int launch_flux_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks, int mixed,
                    const void *fsa, const float *Qhia, const float *Qloa, const double *dt_arr,
                    double *fra, int *status, cudaStream_t s);
int launch_dt_ens(const EnsInst *inst, int ninst, const EnsItem *items, int nitems, int blocks,
                  const double *Qa, double *red, double *dt_arr, double *t_arr, double t_stop,
                  cudaStream_t s);
int launch_update_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks, int stage,
                      const double *fra, const double *dt_arr, double *Qa, double *Ga, double *Qsa,
                      double *Gsa, double *Acca, double *S1a, int *status, cudaStream_t s);

}  // namespace gks
