// One time step of a batched ensemble in ONE persistent launch.
//
// The blocks of a grid that fits on the device at once stride over the
// work items of all instances phase by phase -- dt reduction, dt per
// instance, then per stage (the mixed views of the state,) reconstruction,
// flux and update -- and meet at a grid-wide barrier between phases (each
// phase needs all of the previous one's output of its instance). The
// phases run the same device code as the per-phase kernels (the *_device.cuh
// headers); this translation unit keeps its own copies of the
// reconstruction tables, uploaded with the others.
//
// The barrier is a counter and a generation word in global memory. Its
// wait is bounded: a block that waits longer than the launch's limit (wall
// clock, %globaltimer) raises the abort word and the status bit
// kStatusTimeout and returns; the other blocks see the abort word at their
// next wait and return too, so no launch can hang. The launch requests
// co-residency of all its blocks (cooperative attribute) and sizes the grid
// by the kernel's occupancy.
#include <cooperative_groups.h>

#include "recon_fp64_device.cuh"
#include "recon_mixed_device.cuh"
#include "flux_device.cuh"
#include "update_device.cuh"

namespace gks {
namespace {

constexpr int kStepThreads = 128;

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of `expect` arriving blocks (gridDim.x); false if this
// launch aborted (a wait ran out of time here or in another block).
__device__ bool grid_sync(StepSync *b, unsigned long long limit_ns, int *status,
                          unsigned int expect) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *vgen = &b->gen;
        volatile int *vabort = &b->abort;
        const unsigned int g = *vgen;  // this barrier's generation (it moves on only
                                       // once every block, this one too, has arrived)
        __threadfence();
        if (atomicAdd(&b->count, 1u) + 1u == expect) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (*vgen == g) {
                if (*vabort) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > limit_ns) {
                    atomicExch(&b->abort, 1);
                    flag_status(status, kStatusTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

struct StepArgs {
    const EnsInst *inst;
    const EnsItem *items;
    int ninst, nitems;
    long long total;
    double *Q, *G, *Qs, *Gs, *Acc, *S1;
    void *fs;
    float *Gf, *Qv;
    double *frec, *dt, *t, *red;
    double t_stop;
    StepSync *sync;
    unsigned long long limit_ns;
    int *status;
};

template <bool MIXED>
__global__ void __launch_bounds__(kStepThreads) ens_step_kernel(StepArgs a) {
    __shared__ __align__(16) float sT[MIXED ? kTabFloats : 4];
    if constexpr (MIXED) stage_tables(sT);
    // dt: per-instance maxima of (|U_d| + c)/h_d and nu
    unsigned long long *red = reinterpret_cast<unsigned long long *>(a.red);
    for (int w = blockIdx.x; w < a.nitems; w += gridDim.x) {
        const EnsItem it = a.items[w];
        const EnsInst I = a.inst[it.inst];
        double rate = 0.0, numax = 0.0;
        for (long long c = it.c0 + threadIdx.x; c < it.c1; c += blockDim.x)
            cell_rates(I.g, I.P, a.Q + 5 * I.off, c, rate, numax);
        block_max_to<kStepThreads>(rate, numax, red + 2 * it.inst);
    }
    if (!grid_sync(a.sync, a.limit_ns, a.status, gridDim.x)) return;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < a.ninst; i += blockDim.x) {
            const EnsInst I = a.inst[i];
            double dt = dt_from_rates(I.g, I.P, __longlong_as_double((long long)red[2 * i]),
                                      __longlong_as_double((long long)red[2 * i + 1]));
            const double rem = a.t_stop - a.t[i];
            if (dt > rem) dt = rem;
            if (!(dt > 0.0) || !isfinite(dt)) dt = 0.0;
            a.t[i] += dt;
            a.dt[i] = dt;
            red[2 * i] = 0ull;
            red[2 * i + 1] = 0ull;
        }
    }
    if (!grid_sync(a.sync, a.limit_ns, a.status, gridDim.x)) return;
    const long long N = a.total;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll 1
    for (int stage = 1; stage <= 2; ++stage) {
        const double *Qi = stage == 1 ? a.Q : a.Qs;
        const double *Gi = stage == 1 ? a.G : a.Gs;
        if constexpr (MIXED) {
            // the views of this stage: FP32 gradients, float-float averages
            for (long long i = gtid; i < 15 * N; i += gstride) a.Gf[i] = (float)Gi[i];
            for (long long i = gtid; i < 5 * N; i += gstride) {
                const ff v = ff_from_double(Qi[i]);
                a.Qv[i] = v.hi;
                a.Qv[5 * N + i] = v.lo;
            }
            if (!grid_sync(a.sync, a.limit_ns, a.status, gridDim.x)) return;
        }
        // reconstruction
        for (int w = blockIdx.x; w < a.nitems; w += gridDim.x) {
            const EnsItem it = a.items[w];
            const EnsInst I = a.inst[it.inst];
            const long long T = it.c1 - it.c0;
            for (long long t = threadIdx.x; t < 5 * T; t += blockDim.x) {
                const long long c = it.c0 + t % T;
                const int v = (int)(t / T);
                if constexpr (MIXED) {
                    asm volatile("" ::: "memory");
                    recon5_mixed_cell<kModePlain, true>(
                        sT, I.g, I.P.nonlinear, nullptr, nullptr, a.Gf + 15 * I.off,
                        a.Qv + 5 * I.off, a.Qv + 5 * N + 5 * I.off, (float *)a.fs + 480 * I.off,
                        nullptr, nullptr, nullptr, c, 0, 0, v, I.g.n, c);
                } else {
                    recon5_cell<false>(I.g, I.P.nonlinear, Qi + 5 * I.off, Gi + 15 * I.off,
                                       (double *)a.fs + 480 * I.off, c, v, I.g.n, c);
                }
            }
        }
        if (!grid_sync(a.sync, a.limit_ns, a.status, gridDim.x)) return;
        // flux: an item of T cells holds 3 x T faces x 4 Gauss points, four
        // adjacent lanes per face (every lane of a warp takes part)
        for (int w = blockIdx.x; w < a.nitems; w += gridDim.x) {
            const EnsItem it = a.items[w];
            const EnsInst I = a.inst[it.inst];
            const double dt = a.dt[it.inst];
            if (!(dt > 0.0)) continue;  // uniform across the block
            const long long T = it.c1 - it.c0;
            const long long total = 12 * T;
            const void *fs = MIXED ? (const void *)((const float *)a.fs + 480 * I.off)
                                   : (const void *)((const double *)a.fs + 480 * I.off);
            for (long long t0 = 0; t0 < total; t0 += blockDim.x) {
                long long gid = t0 + threadIdx.x;
                const bool valid = gid < total;
                if (!valid) gid = total - 1;
                const int k = (int)(gid & 3);
                const long long rem = gid >> 2;
                const int d = (int)(rem / T);
                const long long c = it.c0 + rem % T;
                flux_face_point<true, MIXED>(I.g, whole_grid(I.g), I.P, fs,
                                             MIXED ? a.Qv + 5 * I.off : nullptr,
                                             MIXED ? a.Qv + 5 * N + 5 * I.off : nullptr, dt,
                                             a.frec + 90 * I.off, a.status, d, c, k, valid);
            }
        }
        if (!grid_sync(a.sync, a.limit_ns, a.status, gridDim.x)) return;
        // update
        for (int w = blockIdx.x; w < a.nitems; w += gridDim.x) {
            const EnsItem it = a.items[w];
            const EnsInst I = a.inst[it.inst];
            const double dt = a.dt[it.inst];
            if (!(dt > 0.0)) continue;
            const long long o = I.off;
            for (long long c = it.c0 + threadIdx.x; c < it.c1; c += blockDim.x) {
                if (stage == 1)
                    update_cell<1>(I.g, I.P, a.frec + 90 * o, dt, a.Q + 5 * o, a.G + 15 * o,
                                   a.Qs + 5 * o, a.Gs + 15 * o, a.Acc + 5 * o, a.S1 + 15 * o,
                                   a.status, c);
                else
                    update_cell<2>(I.g, I.P, a.frec + 90 * o, dt, a.Q + 5 * o, a.G + 15 * o,
                                   a.Qs + 5 * o, a.Gs + 15 * o, a.Acc + 5 * o, a.S1 + 15 * o,
                                   a.status, c);
            }
        }
        if (stage == 1 && !grid_sync(a.sync, a.limit_ns, a.status, gridDim.x)) return;
    }
}

// A launch whose barrier can never complete (it waits for one block more
// than it has): its waits must run out and report kStatusTimeout.
__global__ void __launch_bounds__(kStepThreads) barrier_timeout_kernel(StepSync *sync,
                                                                       unsigned long long limit_ns,
                                                                       int *status) {
    grid_sync(sync, limit_ns, status, gridDim.x + 1u);
}

template <typename K>
int step_blocks(K kernel) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kStepThreads, 0) !=
            cudaSuccess ||
        sms <= 0 || per_sm <= 0)
        return 0;
    return per_sm * sms;
}

template <typename K, typename... Args>
int launch_coop(K kernel, int blocks, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kStepThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...) == cudaSuccess ? 0 : -2;
}

}  // namespace

int upload_recon_tables_step(const ReconTables &t, const float *tab, size_t tab_bytes) {
    if (cudaMemcpyToSymbol(cR, t.R, sizeof(t.R)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cRs, t.Rs, sizeof(t.Rs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cBs, t.Bs, sizeof(t.Bs)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMean, t.mean, sizeof(t.mean)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMval, t.mval, sizeof(t.mval)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(cMder, t.mder, sizeof(t.mder)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(gTabF, tab, tab_bytes) != cudaSuccess) return -2;
    return 0;
}

int ens_step_grid(int mixed) {
    return mixed ? step_blocks(ens_step_kernel<true>) : step_blocks(ens_step_kernel<false>);
}

int launch_ens_step(const EnsInst *inst, int ninst, const EnsItem *items, int nitems,
                    long long total, int mixed, double *Q, double *G, double *Qs, double *Gs,
                    double *Acc, double *S1, void *fs, float *Gf, float *Qv, double *frec,
                    double *dt, double *t, double *red, double t_stop, StepSync *sync,
                    double limit_s, int *status, cudaStream_t s) {
    StepArgs a;
    a.inst = inst;
    a.items = items;
    a.ninst = ninst;
    a.nitems = nitems;
    a.total = total;
    a.Q = Q;
    a.G = G;
    a.Qs = Qs;
    a.Gs = Gs;
    a.Acc = Acc;
    a.S1 = S1;
    a.fs = fs;
    a.Gf = Gf;
    a.Qv = Qv;
    a.frec = frec;
    a.dt = dt;
    a.t = t;
    a.red = red;
    a.t_stop = t_stop;
    a.sync = sync;
    a.limit_ns = (unsigned long long)(limit_s * 1e9);
    a.status = status;
    const int blocks = ens_step_grid(mixed);
    if (blocks <= 0) return -2;
    // a fresh barrier for this launch (stream-ordered, captured with it)
    if (cudaMemsetAsync(sync, 0, sizeof(StepSync), s) != cudaSuccess) return -2;
    return mixed ? launch_coop(ens_step_kernel<true>, blocks, s, a)
                 : launch_coop(ens_step_kernel<false>, blocks, s, a);
}

int launch_barrier_timeout(StepSync *sync, int blocks, double limit_s, int *status,
                           cudaStream_t s) {
    if (cudaMemsetAsync(sync, 0, sizeof(StepSync), s) != cudaSuccess) return -2;
    return launch_coop(barrier_timeout_kernel, blocks, s, sync,
                       (unsigned long long)(limit_s * 1e9), status);
}

}  // namespace gks
