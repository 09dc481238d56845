// CGKS-5th with reading B of the target cell's data (the paper's S^0 of
// S^data-5th, Sec. 3.1-3.2): the state carries, per conserved variable,
// the 12 line-averaged derivatives L[4a + k] (along axis a, between the
// face Gauss points k of the cell's two faces normal to a) instead of the
// averaged gradient. FP64, periodic grids (uniform or stretched).
//
//   reconstruction: the 72-entry data vector (the neighbours' averages, the
//     face neighbours' averaged gradients and the edge neighbours'
//     tangential derivatives from their lines' means, the own 12 lines),
//     a = R d with the dense 34 x 72 matrix of the constrained least
//     squares, GENO (Eq. weno-new; the sub-stencil slopes' tangential parts
//     from the own lines' means, chi from the misfit of the 54 weighted
//     derivative rows), the quartic and its derivatives at the 24 face
//     Gauss points from tabulated monomials;
//   flux: the Gauss-point flux of flux_device.cuh; F^n and F_t^n averaged
//     over the face's 4 points, the interface values kept per point;
//   update: Q as with gradients; each line from the interface values at
//     its two face Gauss points (the two-stage update point by point).
// The dense tables fill most of this translation unit's constant memory.
#include "recon_common.cuh"
#include "flux_device.cuh"

namespace gks {
namespace {

constexpr int kNd = 72;    // data entries per variable
constexpr int kNl = 54;    // weighted derivative rows
constexpr int kRecL = 90;  // record values per face: F^n, F_t^n, then 4 x 20 interface values

__constant__ double cRL[kNumBasis][kNd];
__constant__ double cWBL[kNl][kNumBasis];
__constant__ double cWL[kNl];
__constant__ double cMeanL[kNumBasis];
__constant__ double cMptL[24][4][kNumBasis];

// averaged gradient along axis a of variable v in cell nb: the mean of its
// four lines
__device__ __forceinline__ double line_mean(const double *__restrict__ Lv, long long n, int a,
                                            long long nb) {
    return 0.25 * (__ldg(Lv + (long long)(4 * a) * n + nb) + __ldg(Lv + (long long)(4 * a + 1) * n + nb) +
                   __ldg(Lv + (long long)(4 * a + 2) * n + nb) + __ldg(Lv + (long long)(4 * a + 3) * n + nb));
}

__global__ void __launch_bounds__(128) recon5_lines_kernel(GridDesc g, int nonlinear,
                                                           const double *__restrict__ Q,
                                                           const double *__restrict__ L,
                                                           double *__restrict__ fs) {
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int v = (int)blockIdx.y;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const int c0[3] = {i, j, k};
    const double *Qv = Q + (long long)v * n;
    const double *Lv = L + (long long)v * 12 * n;
    const double q0 = __ldg(Qv + c);
    double h0[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) h0[a] = cell_h(g, a, c0[a]);

    double d[kNd];
#pragma unroll 1
    for (int m = 0; m < 6; ++m) {
        int cc[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) cc[a] = wrap(c0[a] + face_off(m, a), axis_len(g, a));
        const long long nb = cell_index(g, cc[0], cc[1], cc[2]);
        d[m] = __ldg(Qv + nb) - q0;
#pragma unroll
        for (int a = 0; a < 3; ++a) d[18 + 3 * m + a] = cell_h(g, a, cc[a]) * line_mean(Lv, n, a, nb);
    }
#pragma unroll 1
    for (int e = 0; e < 12; ++e) {
        int cc[3], o[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            o[a] = edge_off(e, a);
            cc[a] = wrap(c0[a] + o[a], axis_len(g, a));
        }
        const long long nb = cell_index(g, cc[0], cc[1], cc[2]);
        d[6 + e] = __ldg(Qv + nb) - q0;
        const int ea = edge_axis_a(e), eb = edge_axis_b(e), ee = edge_axis_e(e);
        const double da = cell_h(g, ea, cc[ea]) * line_mean(Lv, n, ea, nb);
        const double db = cell_h(g, eb, cc[eb]) * line_mean(Lv, n, eb, nb);
        d[36 + 2 * e] = (o[ea] * da - o[eb] * db) * kRs2;
        d[36 + 2 * e + 1] = cell_h(g, ee, cc[ee]) * line_mean(Lv, n, ee, nb);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) d[60 + 4 * a + kk] = h0[a] * __ldg(Lv + (long long)(4 * a + kk) * n + c);

    // a = R d
    double a[kNumBasis];
#pragma unroll
    for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = 0.0;
#pragma unroll 1
    for (int col = 0; col < kNd; ++col) {
        const double dc = d[col];
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) a[ii] = fma(cRL[ii][col], dc, a[ii]);
    }
    double K = 0.0;
#pragma unroll
    for (int ii = 0; ii < kNumBasis; ++ii) K = fma(a[ii], cMeanL[ii], K);
    const double base = q0 - K;

    double chi = 1.0, bbar[3] = {0.0, 0.0, 0.0};
    if (nonlinear) {
        const double eps = 1e-15;
        double g0[3];
#pragma unroll
        for (int q = 0; q < 3; ++q)
            g0[q] = 0.25 * (d[60 + 4 * q] + d[61 + 4 * q] + d[62 + 4 * q] + d[63 + 4 * q]);
        double w[6], wsum = 0.0;
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            const int ax = m / 2;
            const double bn = (m & 1) ? d[m] : -d[m];
            double s = bn * bn;
#pragma unroll
            for (int q = 0; q < 3; ++q)
                if (q != ax) s = fma(g0[q], g0[q], s);
            const double t = s + eps, t2 = t * t;
            w[m] = (1.0 / 6.0) / (t2 * t2 * t);
            wsum += w[m];
        }
#pragma unroll
        for (int m = 0; m < 6; ++m) w[m] /= wsum;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            bbar[q] = (1.0 - w[2 * q] - w[2 * q + 1]) * g0[q] - w[2 * q] * d[2 * q] +
                      w[2 * q + 1] * d[2 * q + 1];
        // GENO's misfit (reading R5) over the 54 weighted derivative rows
        double res2 = 0.0, norm2 = 0.0;
#pragma unroll
        for (int m = 0; m < 18; ++m) norm2 = fma(d[m], d[m], norm2);
#pragma unroll 1
        for (int q = 0; q < kNl; ++q) {
            const double wd = cWL[q] * d[18 + q];
            double r = -wd;
#pragma unroll
            for (int ii = 0; ii < kNumBasis; ++ii) r = fma(cWBL[q][ii], a[ii], r);
            res2 = fma(r, r, res2);
            norm2 = fma(wd, wd, norm2);
        }
        const double r0 = __ldg(Q + c), e0 = __ldg(Q + 4 * n + c);
        const double S = v == 0 ? r0 : (v == 4 ? e0 : sqrt(fabs(r0 * e0)));
        const double sig = res2 / (norm2 + kGenoKappa * kGenoKappa * S * S + eps);
        const double s = sig * (1.0 / kGenoSigma0);
        chi = 1.0 / (1.0 + s + s * s);
    }
    // the 24 face Gauss points
#pragma unroll 1
    for (int pt = 0; pt < 24; ++pt) {
        const int f = pt / 4, kk = pt % 4, D = f / 2, side = f & 1;
        double val = base, der[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int ii = 0; ii < kNumBasis; ++ii) {
            val = fma(a[ii], cMptL[pt][0][ii], val);
            der[0] = fma(a[ii], cMptL[pt][1][ii], der[0]);
            der[1] = fma(a[ii], cMptL[pt][2][ii], der[1]);
            der[2] = fma(a[ii], cMptL[pt][3][ii], der[2]);
        }
        if (nonlinear) {
            double x[3];
            x[D] = side ? 0.5 : -0.5;
            x[(D + 1) % 3] = (kk & 1) ? kG : -kG;
            x[(D + 2) % 3] = (kk & 2) ? kG : -kG;
            const double p1 = fma(bbar[0], x[0], fma(bbar[1], x[1], fma(bbar[2], x[2], q0)));
            val = fma(chi, val - p1, p1);
#pragma unroll
            for (int q = 0; q < 3; ++q) der[q] = fma(chi, der[q] - bbar[q], bbar[q]);
        }
        const int cmp = frame_comp(v, D);
        double *o = fs + ((long long)pt * 20) * n + c;
        o[(long long)cmp * n] = val;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const int jf = (q - D + 3) % 3;
            o[(long long)(5 + 5 * jf + cmp) * n] = der[q] / h0[q];
        }
    }
}

// The Gauss-point flux of every face (periodic): four adjacent lanes hold
// the four points of a face; F^n and F_t^n are averaged by a butterfly,
// each lane keeps its point's interface values. Records per axis d and
// cell c (the face on c's low side): [0..9] F^n, F_t^n, [10 + 20 p + 5 b +
// component] Q^l, dQ^l/dt, Q^r, dQ^r/dt (b = 0..3) of point p, global frame.
__global__ void __launch_bounds__(128, 1) flux_faces_lines_kernel(GridDesc g, PhysParams P,
                                                                 const double *__restrict__ fs,
                                                                 const double *__restrict__ dt_dev,
                                                                 double *__restrict__ frec,
                                                                 int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;  // same for every thread of the grid
    const long long n = g.n;
    const long long total = 12 * n;
    long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = gid < total;
    if (!valid) gid = total - 1;  // groups of four lanes are entirely in or out
    const int kq = (int)(gid & 3);
    const long long fc = gid >> 2;
    const int d = (int)(fc / n);
    const long long c = fc - (long long)d * n;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const long long left = cell_index(g, d == 0 ? wrap(i - 1, g.nx) : i, d == 1 ? wrap(j - 1, g.ny) : j,
                                      d == 2 ? wrap(k - 1, g.nz) : k);
    double sl[20], sr[20], out[30];
    const double *pl = fs + ((long long)((2 * d + 1) * 4 + kq) * 20) * n + left;
    const double *pr = fs + ((long long)((2 * d) * 4 + kq) * 20) * n + c;
#pragma unroll
    for (int q = 0; q < 20; ++q) {
        sl[q] = __ldg(pl + (long long)q * n);
        sr[q] = __ldg(pr + (long long)q * n);
    }
    flux_point<true>(P, sl, sr, dt, out, valid ? status : nullptr);
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        double s = out[q] + __shfl_xor_sync(0xffffffffu, out[q], 1);
        s = s + __shfl_xor_sync(0xffffffffu, s, 2);
        out[q] = 0.25 * s;
    }
    if (!valid) return;
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        if (q % 4 != kq) continue;
        const int blk = q / 5, cmp = q % 5;
        frec[((long long)d * kRecL + blk * 5 + global_var(cmp, d)) * n + c] = out[q];
    }
#pragma unroll
    for (int q = 10; q < 30; ++q) {
        const int blk = (q - 10) / 5, cmp = q % 5;
        frec[((long long)d * kRecL + 10 + 20 * kq + blk * 5 + global_var(cmp, d)) * n + c] = out[q];
    }
}

// one stage of the update with lines (see the file comment)
template <int STAGE>
__global__ void __launch_bounds__(256) update_lines_kernel(GridDesc g, PhysParams P,
                                                           const double *__restrict__ fr,
                                                           const double *__restrict__ dt_dev,
                                                           double *__restrict__ Q, double *__restrict__ L,
                                                           double *__restrict__ Qs, double *__restrict__ Ls,
                                                           double *__restrict__ Acc, double *__restrict__ S1,
                                                           int *status) {
    const double dt = *dt_dev;
    if (!(dt > 0.0)) return;
    const long long n = g.n;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    const long long hi[3] = {cell_index(g, wrap(i + 1, g.nx), j, k),
                             cell_index(g, i, wrap(j + 1, g.ny), k),
                             cell_index(g, i, j, wrap(k + 1, g.nz))};
    const double ih[3] = {1.0 / cell_h(g, 0, i), 1.0 / cell_h(g, 1, j), 1.0 / cell_h(g, 2, k)};
    const double dt2 = dt * dt;
    double out[5];
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        double Lq = 0.0, Lt = 0.0;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double *F = fr + (long long)d * kRecL * n;
            Lq += (F[(long long)v * n + hi[d]] - F[(long long)v * n + c]) * ih[d];
            Lt += (F[(long long)(5 + v) * n + hi[d]] - F[(long long)(5 + v) * n + c]) * ih[d];
        }
        Lq = -Lq;
        Lt = -Lt;
        const long long qi = (long long)v * n + c;
        if (STAGE == 1) {
            const double q = Q[qi];
            out[v] = q + 0.5 * dt * Lq + 0.125 * dt2 * Lt;
            Qs[qi] = out[v];
            Acc[qi] = q + dt * Lq + dt2 * (1.0 / 6.0) * Lt;
        } else {
            out[v] = Acc[qi] + dt2 * (1.0 / 3.0) * Lt;
            Q[qi] = out[v];
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double *F = fr + (long long)d * kRecL * n;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const double *Fp = F + (long long)(10 + 20 * p) * n;
                const long long li = ((long long)v * 12 + 4 * d + p) * n + c;
                const double qlt = Fp[(long long)(5 + v) * n + hi[d]];
                const double qrt = Fp[(long long)(15 + v) * n + c];
                if (STAGE == 1) {
                    const double ql = Fp[(long long)v * n + hi[d]];
                    const double qr = Fp[(long long)(10 + v) * n + c];
                    Ls[li] = ((ql + 0.5 * dt * qlt) - (qr + 0.5 * dt * qrt)) * ih[d];
                    S1[li] = (ql - qr) * ih[d];
                } else {
                    L[li] = S1[li] + dt * (qlt - qrt) * ih[d];
                }
            }
        }
    }
    const double rho = out[0];
    const double ke = 0.5 * (out[1] * out[1] + out[2] * out[2] + out[3] * out[3]) / rho;
    const double p = (P.gamma - 1.0) * (out[4] - ke);
    bool finite = true;
#pragma unroll
    for (int v = 0; v < 5; ++v) finite = finite && isfinite(out[v]);
    if (!finite) flag_status(status, kStatusNonfinite);
    else if (!(rho > 0.0 && p > 0.0)) flag_status(status, kStatusNonphysical);
}

// the averaged gradients [5][3][cells] of a lines state (for the diagnostics)
__global__ void lines_to_grad_kernel(long long n, const double *__restrict__ L,
                                     double *__restrict__ G) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < 15 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long c = t % n, va = t / n;  // va = 3 v + a
        const int v = (int)(va / 3), a = (int)(va % 3);
        const double *Lv = L + (long long)v * 12 * n;
        G[t] = 0.25 * (Lv[(long long)(4 * a) * n + c] + Lv[(long long)(4 * a + 1) * n + c] +
                       Lv[(long long)(4 * a + 2) * n + c] + Lv[(long long)(4 * a + 3) * n + c]);
    }
}

}  // namespace

int upload_recon_tables_lines(void) {
    static ReconTablesLines t;
    static int built = 0;
    if (!built) {
        if (build_recon_tables_lines(&t)) return -1;
        built = 1;
    }
    if (cudaMemcpyToSymbol(cRL, t.R, sizeof(t.R)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cWBL, t.WB, sizeof(t.WB)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cWL, t.w, sizeof(t.w)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMeanL, t.mean, sizeof(t.mean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMptL, t.mpt, sizeof(t.mpt)) != cudaSuccess) return -2;
    return 0;
}

int launch_recon5_lines(const GridDesc &g, const PhysParams &P, const double *Q, const double *L,
                        double *fs, cudaStream_t s) {
    const long long blocks = (g.n + 127) / 128;
    recon5_lines_kernel<<<dim3((unsigned)blocks, 5), 128, 0, s>>>(g, P.nonlinear, Q, L, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_flux_faces_lines(const GridDesc &g, const PhysParams &P, const double *fs,
                            const double *dt_dev, double *frec, int *status, cudaStream_t s) {
    const long long blocks = (12 * g.n + 127) / 128;
    flux_faces_lines_kernel<<<(unsigned)blocks, 128, 0, s>>>(g, P, fs, dt_dev, frec, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_update_lines(const GridDesc &g, const PhysParams &P, int stage, const double *frec,
                        const double *dt_dev, double *Q, double *L, double *Qs, double *Ls,
                        double *Acc, double *S1, int *status, cudaStream_t s) {
    const long long blocks = (g.n + 255) / 256;
    if (stage == 1)
        update_lines_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(g, P, frec, dt_dev, Q, L, Qs, Ls,
                                                                Acc, S1, status);
    else
        update_lines_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(g, P, frec, dt_dev, Q, L, Qs, Ls,
                                                                Acc, S1, status);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_lines_to_grad(long long n, const double *L, double *G, cudaStream_t s) {
    const long long blocks = (15 * n + 255) / 256;
    lines_to_grad_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(n, L, G);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
