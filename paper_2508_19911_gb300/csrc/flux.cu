// Gas-kinetic interface flux at Gauss points (Sec. 2 of the paper).
//
// For the face frame (u along the face normal) and left/right reconstructed
// states W_l, W_r with their spatial derivatives, the distribution of
// Eq. flux is integrated over [0, dt] and [0, dt/2]; F^n and F_t^n follow
// from the linearisation f = f^n + t f_t^n (Eq. deri-t-f). Moments of the
// Maxwellians are evaluated in closed form:
//   <u^n> on the full line by <u^{n+2}> = U <u^{n+1}> + (n+1)/(2 lam) <u^n>,
//   on the half lines from erfc/exp starting values and the same recursion,
//   <xi^2> = N/(2 lam), <xi^4> = (N^2 + 2N)/(4 lam^2),
// composed into the symmetric moment matrices <u^A v^B w^D psi psi^T> with
// compile-time exponents, each built once per weight and applied to every
// slope vector that meets it; the Maxwellian slopes a (<(a.psi) psi> =
// dW/rho) are solved in closed form. Where a moment of a full Maxwellian is
// an Euler flux, its contraction with slopes is the flux Jacobian applied
// to the derivatives (the compatibility sums sum_j <u_j (a_j.psi) psi> and
// term 3's flux moments).
// One thread evaluates one Gauss point; the four Gauss points of a CGKS-5th
// face are four adjacent lanes reduced with a butterfly of shuffles.
#include <cmath>

#include "flux_device.cuh"

namespace gks {
namespace {

// mixed: at most 168 registers for 3 blocks per SM (a few spills; 20%
// faster at 128^3 than 2 blocks with 255 registers and none).
// GEN (general grids): the faces of cells on the low boundary of a
// non-periodic axis pair the cell with its mirror ghost, and the high
// boundary faces of this buffer's cells follow the 3 x cells faces.
template <bool kCGKS, bool MIXED, bool GEN>
__global__ void __launch_bounds__(128, MIXED ? 3 : 1) flux_faces_kernel(GridDesc g, Slab S, PhysParams P,
                                                         const void *__restrict__ fs,
                                                         const float *__restrict__ Qhi,
                                                         const float *__restrict__ Qlo,
                                                         const double *__restrict__ dt_dev,
                                                         double *__restrict__ frec, int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;  // same for every thread of the grid
    constexpr int K = kCGKS ? 4 : 1;
    const long long nxy = (long long)g.nx * g.ny;
    const long long cnt = (long long)(S.nzb - S.p0) * nxy;  // cells whose faces are computed
    long long total = 3 * cnt * K;
    long long nbx = 0, nby = 0;
    if constexpr (GEN) {
        const long long planes = S.nzb - S.p0;
        nbx = g.bc[0] ? (long long)g.ny * planes : 0;
        nby = g.bc[1] ? (long long)g.nx * planes : 0;
        const long long nbz = (g.bc[2] && (S.zb + S.nzb - 1) % g.nz == g.nz - 1) ? nxy : 0;
        total += K * (nbx + nby + nbz);
    }
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gid < total;
    if (!valid) gid = total - 1;  // groups of K lanes are entirely in or out
    const int k = (int)(gid % K);
    const long long fc = gid / K;
    if (!GEN || fc < 3 * cnt) {
        const int d = (int)(fc / cnt);
        const long long t = fc - (long long)d * cnt;
        const long long l = S.p0 * nxy + t;
        int bmode = 0;
        if constexpr (GEN) {
            if (g.bc[d]) {
                const long long ij = l % nxy;
                const int cd = d == 0 ? (int)(ij % g.nx)
                                      : (d == 1 ? (int)(ij / g.nx) : (int)((S.zb + l / nxy) % g.nz));
                if (cd == 0) bmode = 1;
            }
        }
        flux_face_point<kCGKS, MIXED>(g, S, P, fs, Qhi, Qlo, dt, frec, status, d, l, k, valid,
                                      bmode);
    } else {
        long long e = fc - 3 * cnt, l;
        int d;
        if (e < nbx) {
            d = 0;
            l = (S.p0 + e / g.ny) * nxy + (e % g.ny) * g.nx + (g.nx - 1);
        } else if (e < nbx + nby) {
            d = 1;
            e -= nbx;
            l = (S.p0 + e / g.nx) * nxy + (long long)(g.ny - 1) * g.nx + e % g.nx;
        } else {
            d = 2;
            e -= nbx + nby;
            l = (long long)(S.nzb - 1) * nxy + e;
        }
        flux_face_point<kCGKS, MIXED>(g, S, P, fs, Qhi, Qlo, dt, frec, status, d, l, k, valid, 2);
    }
}

// Persistent ensemble flux (CGKS-5th): blocks stride over the work items
// of all instances; an item of T cells holds 3 x T faces x 4 Gauss points.
template <bool MIXED>
__global__ void __launch_bounds__(128) flux_ens_kernel(const EnsInst *__restrict__ inst,
                                                       const EnsItem *__restrict__ items,
                                                       int nitems, const void *__restrict__ fsa,
                                                       const float *__restrict__ Qhia,
                                                       const float *__restrict__ Qloa,
                                                       const double *__restrict__ dt_arr,
                                                       double *__restrict__ fra, int *status) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        const double dt = dt_arr[it.inst];
        if (!(dt > 0.0)) continue;  // uniform across the block
        const long long T = it.c1 - it.c0;
        const long long total = 12 * T;
        const void *fs = MIXED ? (const void *)((const float *)fsa + 480 * I.off)
                               : (const void *)((const double *)fsa + 480 * I.off);
        for (long long t0 = 0; t0 < total; t0 += blockDim.x) {
            long long gid = t0 + threadIdx.x;
            const bool valid = gid < total;
            if (!valid) gid = total - 1;
            const int k = (int)(gid & 3);
            const long long rem = gid >> 2;
            const int d = (int)(rem / T);
            const long long c = it.c0 + rem % T;
            flux_face_point<true, MIXED>(I.g, whole_grid(I.g), I.P, fs,
                                         MIXED ? Qhia + 5 * I.off : nullptr,
                                         MIXED ? Qloa + 5 * I.off : nullptr, dt, fra + 90 * I.off,
                                         status, d, c, k, valid);
        }
    }
}

__global__ void __launch_bounds__(128) flux_points_kernel(PhysParams P, const double *__restrict__ sl_,
                                                          const double *__restrict__ sr_, int n,
                                                          const double *__restrict__ dt_dev,
                                                          double *__restrict__ out_, int *status) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dt = *dt_dev;
    double sl[20], sr[20], out[30];
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        sl[q] = sl_[(long long)q * n + i];
        sr[q] = sr_[(long long)q * n + i];
    }
    flux_point<true>(P, sl, sr, dt, out, status);
#pragma unroll
    for (int q = 0; q < 30; ++q) out_[(long long)q * n + i] = out[q];
}

}  // namespace

// float-float split of m FP64 values: hi[i] + lo[i] = x[i] (to 2^-48)
__global__ void q_to_ff_kernel(const double *__restrict__ x, float *__restrict__ hi,
                               float *__restrict__ lo, long long m) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x) {
        const ff v = ff_from_double(x[i]);
        hi[i] = v.hi;
        lo[i] = v.lo;
    }
}

int launch_q_to_ff(long long m, const double *x, float *hi, float *lo, cudaStream_t s) {
    const long long blocks = (m + 255) / 256;
    q_to_ff_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(x, hi, lo, m);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// threads of one flux launch: K per face, 3 faces per cell of the slab's
// planes p0..nzb-1, and on a general grid the high boundary faces
static long long flux_threads(const GridDesc &g, const Slab &S, int K) {
    const long long planes = S.nzb - S.p0, nxy = (long long)g.nx * g.ny;
    long long faces = 3 * planes * nxy;
    if (g.general) {
        if (g.bc[0]) faces += (long long)g.ny * planes;
        if (g.bc[1]) faces += (long long)g.nx * planes;
        if (g.bc[2] && (S.zb + S.nzb - 1) % g.nz == g.nz - 1) faces += nxy;
    }
    return faces * K;
}

template <bool MIXED, bool GEN>
static void launch_flux_t(const GridDesc &g, const Slab &S, const PhysParams &P, const void *fs,
                          const float *Qhi, const float *Qlo, const double *dt_dev, double *frec,
                          int *status, cudaStream_t s) {
    const long long total = flux_threads(g, S, P.scheme ? 4 : 1);
    const int block = 128;
    const unsigned grid = (unsigned)((total + block - 1) / block);
    if (P.scheme)
        flux_faces_kernel<true, MIXED, GEN><<<grid, block, 0, s>>>(g, S, P, fs, Qhi, Qlo, dt_dev,
                                                                   frec, status);
    else
        flux_faces_kernel<false, MIXED, GEN><<<grid, block, 0, s>>>(g, S, P, fs, Qhi, Qlo, dt_dev,
                                                                    frec, status);
}

int launch_flux_faces_mixed(const GridDesc &g, const Slab &S, const PhysParams &P,
                            const float *fs, const float *Qhi, const float *Qlo,
                            const double *dt_dev, double *frec, int *status, cudaStream_t s) {
    if (g.general) launch_flux_t<true, true>(g, S, P, fs, Qhi, Qlo, dt_dev, frec, status, s);
    else launch_flux_t<true, false>(g, S, P, fs, Qhi, Qlo, dt_dev, frec, status, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_faces(const GridDesc &g, const Slab &S, const PhysParams &P, const double *fs,
                      const double *dt_dev, double *frec, int *status, cudaStream_t s) {
    if (g.general) launch_flux_t<false, true>(g, S, P, fs, nullptr, nullptr, dt_dev, frec, status, s);
    else launch_flux_t<false, false>(g, S, P, fs, nullptr, nullptr, dt_dev, frec, status, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// mixed: Qhia, Qloa are the float-float split of the averages' arena
int launch_flux_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks, int mixed,
                    const void *fsa, const float *Qhia, const float *Qloa, const double *dt_arr,
                    double *fra, int *status, cudaStream_t s) {
    if (mixed)
        flux_ens_kernel<true><<<blocks, 128, 0, s>>>(inst, items, nitems, fsa, Qhia, Qloa, dt_arr,
                                                     fra, status);
    else
        flux_ens_kernel<false><<<blocks, 128, 0, s>>>(inst, items, nitems, fsa, nullptr, nullptr,
                                                      dt_arr, fra, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_points(const PhysParams &P, const double *sl, const double *sr, int n,
                       const double *dt_dev, double *out, int *status, cudaStream_t s) {
    const int block = 128;
    flux_points_kernel<<<(n + block - 1) / block, block, 0, s>>>(P, sl, sr, n, dt_dev, out, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
