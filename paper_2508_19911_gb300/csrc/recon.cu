// Mixed-precision reconstruction kernels (Sec. 3.2 CGKS-5th in FP32, Sec. 3.3
// GKS-2nd in FP32), the learned indicator's inference and training dumps,
// the ensemble's mixed reconstruction and the table upload. The FP64
// kernels are in recon_fp64.cu. This file is compiled without implicit
// multiply-add contraction (only explicit fmaf), so that every kernel that
// inlines the reconstruction rounds identically.
//
// CGKS-5th, one thread per (cell, conserved variable):
//   1. load the 63 entries of S^data-5th orbit by orbit under the axis
//      reflections, form the symmetrised combinations and accumulate
//      a = R d by parity-class blocks (basis.h: kSym, kClass);
//   2. GENO (Eq. weno-new): the six sub-stencil slopes b^m (Eq.
//      compact-sub-2), IS_m = |b^m|^2, w_m = d_m/(IS_m + eps)^5 normalised;
//      chi from the misfit of the quartic against the derivative data,
//      sigma = |W (B a - d_B)|^2 / (|d_C|^2 + |W d_B|^2 + (kappa S)^2 + eps)
//      (W B block-diagonal by parity class in the symmetrised basis, the
//      derivative columns loaded a second time), chi = 1/(1 + s + s^2),
//      s = sigma/sigma0;
//   3. evaluate P4 and its gradient at the 24 face Gauss points: the
//      monomials are summed into 8 parity classes per face axis and the 8
//      points of a face follow by a Walsh-Hadamard transform.
#include <mutex>

#include "recon_mixed_device.cuh"

namespace gks {
namespace {

// Persistent: each block stages the FP32 table once, then strides over
// tiles of 128 cells x one conserved variable (the five variables of a cell
// block are adjacent tiles). The empty asm with a memory clobber at the top
// of each tile keeps the compiler from hoisting table loads out of the tile
// loop into registers (which spills).
template <int MODE, bool VIEW, bool GEN = false>
__global__ void __launch_bounds__(128) recon5_mixed_kernel(GridDesc g, Slab S, int nonlinear,
                                                           const double *__restrict__ Q,
                                                           const double *__restrict__ G,
                                                           const float *__restrict__ Gf,
                                                           const float *__restrict__ Qhi,
                                                           const float *__restrict__ Qlo,
                                                           float *__restrict__ fs,
                                                           float *__restrict__ dump_x,
                                                           float *__restrict__ dump_chi,
                                                           unsigned long long *skips) {
    __shared__ __align__(16) float sT[kTabFloats];
    stage_tables(sT);
    const long long ntiles = 5 * ((S.nb + 127) / 128);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        asm volatile("" ::: "memory");
        const long long l = (t / 5) * 128 + threadIdx.x;
        if (l < S.nb)
            recon5_mixed_cell<MODE, VIEW, GEN>(sT, g, nonlinear, Q, G, Gf, Qhi, Qlo, fs, dump_x,
                                               dump_chi, skips, slab_global(g, S, l), 5 * g.n,
                                               0, (int)(t % 5), S.nb, l);
    }
}

// Persistent ensemble reconstruction: blocks stride over the work items of
// all instances; MIXED selects the FP32 kernel (MODE as above).
template <int MODE>
__global__ void __launch_bounds__(128) recon5_ens_kernel(const EnsInst *__restrict__ inst,
                                                         const EnsItem *__restrict__ items,
                                                         int nitems, const float *__restrict__ Gfa,
                                                         const float *__restrict__ Qhia,
                                                         const float *__restrict__ Qloa,
                                                         void *__restrict__ fsa,
                                                         float *__restrict__ dump_x,
                                                         float *__restrict__ dump_chi,
                                                         unsigned long long *skips,
                                                         long long dump_ld) {
    __shared__ __align__(16) float sT[kTabFloats];
    stage_tables(sT);
    for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
        const EnsItem it = items[w];
        const EnsInst I = inst[it.inst];
        const long long T = it.c1 - it.c0;
        for (long long t = threadIdx.x; t < 5 * T; t += blockDim.x) {
            asm volatile("" ::: "memory");
            recon5_mixed_cell<MODE, true>(sT, I.g, I.P.nonlinear, nullptr, nullptr,
                                          Gfa + 15 * I.off, Qhia + 5 * I.off, Qloa + 5 * I.off,
                                          fsa ? (float *)fsa + 480 * I.off : nullptr, dump_x,
                                          dump_chi, skips, it.c0 + t % T, dump_ld, 5 * I.off,
                                          (int)(t / T), I.g.n, it.c0 + t % T);
        }
    }
}

template <bool GEN>
__global__ void __launch_bounds__(128) recon2_mixed_kernel(GridDesc g, Slab S, int nonlinear,
                                                           float eps2, const double *__restrict__ Q,
                                                           float *__restrict__ fs) {
    const long long n = g.n;
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= S.nb) return;
    const long long c = slab_global(g, S, l);
    const int i = (int)(c % g.nx);
    const int j = (int)((c / g.nx) % g.ny);
    const int k = (int)(c / ((long long)g.nx * g.ny));
    long long nb[6];
    int fl[6];
    float ih[3] = {(float)(1.0 / g.h[0]), (float)(1.0 / g.h[1]), (float)(1.0 / g.h[2])};
    if constexpr (!GEN) {
#pragma unroll
        for (int m = 0; m < 6; ++m)
            nb[m] = cell_index(g, wrap(i + face_off(m, 0), g.nx), wrap(j + face_off(m, 1), g.ny),
                               wrap(k + face_off(m, 2), g.nz));
    } else {
        const int c0[3] = {i, j, k};
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            int cc[3];
            fl[m] = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) cc[a] = nb_coord(g, a, c0[a] + face_off(m, a), fl[m]);
            nb[m] = cell_index(g, cc[0], cc[1], cc[2]);
        }
        double h[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            h[a] = cell_h(g, a, c0[a]);
            ih[a] = (float)(1.0 / h[a]);
        }
        const double hv = cbrt(h[0] * h[1] * h[2]);
        eps2 = (float)(hv * hv * hv);
    }
#pragma unroll 1
    for (int v = 0; v < 5; ++v) {
        const double *Qv = Q + (long long)v * n;
        const double q0 = __ldg(Qv + c);
        float dn[6];  // neighbour minus own average, FP64 difference
#pragma unroll
        for (int m = 0; m < 6; ++m) {
            double x = __ldg(Qv + nb[m]);
            if constexpr (GEN) x = neg_if(x, ghost_neg(g, v, fl[m]));
            dn[m] = (float)(x - q0);
        }
        float b[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) b[d] = 0.5f * (dn[2 * d + 1] - dn[2 * d]);
        float phi = 1.0f;
        if (nonlinear) {
            float dmax = 0.0f, dmin = 0.0f;
#pragma unroll
            for (int m = 0; m < 6; ++m) {
                dmax = fmaxf(dmax, dn[m]);
                dmin = fminf(dmin, dn[m]);
            }
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                const float d2 = (f & 1) ? 0.5f * b[f / 2] : -0.5f * b[f / 2];
                if (d2 != 0.0f) {
                    const float dp = d2 > 0.0f ? dmax : dmin;
                    const float pf = (dp * dp + eps2 + 2.0f * d2 * dp) /
                                     (dp * dp + 2.0f * d2 * d2 + d2 * dp + eps2);
                    phi = fminf(phi, pf);
                }
            }
        }
#pragma unroll
        for (int f = 0; f < 6; ++f) {
            const int d = f / 2;
            const int cmp = frame_comp(v, d);
            float *o = fs + ((long long)f * 20) * S.nb + l;
            o[(long long)cmp * S.nb] = phi * ((f & 1) ? 0.5f : -0.5f) * b[d];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int jf = (q - d + 3) % 3;
                o[(long long)(5 + 5 * jf + cmp) * S.nb] = phi * b[q] * ih[q];
            }
        }
    }
}

}  // namespace

int upload_recon_tables(void) {
    // one builder at a time: contexts may be created from several threads
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    static ReconTables t;
    static int built = 0;
    if (!built) {
        if (build_recon_tables(&t)) return -1;
        built = 1;
    }
    if (upload_recon_tables_fp64(t)) return -2;
    // FP32 sections of the staged table (the network's sections are left
    // as they are)
    static float tab[kTabW1];
    for (int i = 0; i < kTabW1; ++i) tab[i] = 0.0f;
    for (int r = 0; r < kNumData; ++r)
        for (int j = 0; j < kMaxClass; ++j) {
            tab[kTabRs + r * kPadS + j] = (float)t.Rs[r][j];
            tab[kTabBs + r * kPadS + j] = (float)t.Bs[r][j];
        }
    for (int i = 0; i < kNumBasis; ++i) {
        tab[kTabMean + i] = (float)t.mean[i];
        for (int d = 0; d < 3; ++d) {
            tab[kTabMval + d * kPad + i] = (float)t.mval[d][i];
            for (int q = 0; q < 3; ++q) tab[kTabMder + (3 * d + q) * kPad + i] = (float)t.mder[d][q][i];
        }
    }
    if (cudaMemcpyToSymbol(gTabF, tab, sizeof(tab)) != cudaSuccess) return -2;
    // the single-launch ensemble step's copies
    if (upload_recon_tables_step(t, tab, sizeof(tab))) return -2;
    return 0;
}

// grid of a persistent kernel: the blocks that fit on the device at once
// (occupancy of this kernel: registers, 18 KB of shared memory), capped by
// the number of tiles
template <typename K>
static unsigned persistent_blocks(K kernel, long long tiles) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0) != cudaSuccess ||
        sms <= 0 || per_sm <= 0) {
        sms = 152;
        per_sm = 2;
    }
    const long long b = (long long)per_sm * sms;
    return (unsigned)(tiles < b ? tiles : b);
}

// FP32 copy of the cell gradients (15 per cell), read by the mixed
// reconstruction instead of converting each G value at every stencil use
__global__ void g_to_f32_kernel(const double *__restrict__ G, float *__restrict__ Gf, long long m) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (long long)gridDim.x * blockDim.x)
        Gf[i] = (float)G[i];
}

int launch_g_to_f32(long long m, const double *G, float *Gf, cudaStream_t s) {
    const long long blocks = (m + 255) / 256;
    g_to_f32_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(G, Gf, m);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// Gf, Qhi, Qlo: the views of this stage (launch_g_to_f32, launch_q_to_ff)
int launch_recon5_mixed(const GridDesc &g, const Slab &S, const PhysParams &P, const float *Gf,
                        const float *Qhi, const float *Qlo, float *fs, cudaStream_t s,
                        int indicator, unsigned long long *skips) {
    if (!Gf || !Qhi || !Qlo) return -1;
    const long long tiles = 5 * ((S.nb + 127) / 128);
    if (g.general) {
        // general grids: the plain reconstruction only (no indicator)
        if (indicator) return -1;
        recon5_mixed_kernel<kModePlain, true, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModePlain, true, true>, tiles), 128, 0, s>>>(
                g, S, P.nonlinear, nullptr, nullptr, Gf, Qhi, Qlo, fs, nullptr, nullptr, nullptr);
    } else if (indicator)
        recon5_mixed_kernel<kModeIndicator, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModeIndicator, true>, tiles), 128, 0, s>>>(
                g, S, P.nonlinear, nullptr, nullptr, Gf, Qhi, Qlo, fs, nullptr, nullptr, skips);
    else
        recon5_mixed_kernel<kModePlain, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModePlain, true>, tiles), 128, 0, s>>>(
                g, S, P.nonlinear, nullptr, nullptr, Gf, Qhi, Qlo, fs, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_indicator_dump(const GridDesc &g, const double *Q, const double *G, const float *Gf,
                          const float *Qhi, const float *Qlo, float *x, float *chi,
                          cudaStream_t s) {
    if (g.general) return -1;  // training dumps come from periodic uniform grids
    const long long tiles = 5 * ((g.n + 127) / 128);
    const Slab S = whole_grid(g);
    if (Gf && Qhi && Qlo) {
        recon5_mixed_kernel<kModeDump, true>
            <<<persistent_blocks(recon5_mixed_kernel<kModeDump, true>, tiles), 128, 0, s>>>(
                g, S, 1, nullptr, nullptr, Gf, Qhi, Qlo, nullptr, x, chi, nullptr);
    } else {
        recon5_mixed_kernel<kModeDump, false>
            <<<persistent_blocks(recon5_mixed_kernel<kModeDump, false>, tiles), 128, 0, s>>>(
                g, S, 1, Q, G, nullptr, nullptr, nullptr, nullptr, x, chi, nullptr);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_recon5_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                      int mixed, int indicator, const double *Qa, const double *Ga,
                      const float *Gfa, const float *Qhia, const float *Qloa, void *fsa,
                      unsigned long long *skips, cudaStream_t s) {
    if (!mixed) return launch_recon5_ens_fp64(inst, items, nitems, blocks, Qa, Ga, (double *)fsa, s);
    if (indicator)
        recon5_ens_kernel<kModeIndicator><<<blocks, 128, 0, s>>>(
            inst, items, nitems, Gfa, Qhia, Qloa, fsa, nullptr, nullptr, skips, 0);
    else
        recon5_ens_kernel<kModePlain><<<blocks, 128, 0, s>>>(
            inst, items, nitems, Gfa, Qhia, Qloa, fsa, nullptr, nullptr, nullptr, 0);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int launch_indicator_dump_ens(const EnsInst *inst, const EnsItem *items, int nitems, int blocks,
                              const float *Gfa, const float *Qhia, const float *Qloa, float *x,
                              float *chi, long long total_cells, cudaStream_t s) {
    recon5_ens_kernel<kModeDump><<<blocks, 128, 0, s>>>(inst, items, nitems, Gfa, Qhia, Qloa,
                                                        nullptr, x, chi, nullptr, 5 * total_cells);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

int upload_indicator(const float *params, float theta) {
    // params: W1 [kMlpHidden][63] row major, b1, w2, b2 (kMlpParams floats,
    // host); stored with W1 transposed so that one column is contiguous
    static float net[kTabFloats - kTabW1];
    for (int j = 0; j < kMlpHidden; ++j)
        for (int c = 0; c < kNumData; ++c) net[c * kMlpHidden + j] = params[j * kNumData + c];
    for (int j = 0; j < kMlpHidden; ++j) {
        net[kTabB1 - kTabW1 + j] = params[kMlpHidden * kNumData + j];
        net[kTabW2 - kTabW1 + j] = params[kMlpHidden * kNumData + kMlpHidden + j];
    }
    net[kTabB2 - kTabW1] = params[kMlpHidden * kNumData + 2 * kMlpHidden];
    // skip when sigmoid(logit) >= theta, i.e. logit >= log(theta / (1 - theta))
    net[kTabB2 - kTabW1 + 1] = theta >= 1.0f ? INFINITY : logf(theta / (1.0f - theta));
    net[kTabB2 - kTabW1 + 2] = net[kTabB2 - kTabW1 + 3] = 0.0f;
    if (cudaMemcpyToSymbol(gTabF, net, sizeof(net), sizeof(float) * kTabW1) != cudaSuccess)
        return -2;
    return 0;
}

int launch_recon2_mixed(const GridDesc &g, const Slab &S, const PhysParams &P, const double *Q,
                        float *fs, cudaStream_t s) {
    const double hv = cbrt(g.h[0] * g.h[1] * g.h[2]);
    const float eps2 = (float)(hv * hv * hv);
    const int block = 128;
    const long long grid = (S.nb + block - 1) / block;
    if (g.general)
        recon2_mixed_kernel<true><<<(unsigned)grid, block, 0, s>>>(g, S, P.nonlinear, eps2, Q, fs);
    else
        recon2_mixed_kernel<false><<<(unsigned)grid, block, 0, s>>>(g, S, P.nonlinear, eps2, Q, fs);
    return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

}  // namespace gks
