// Sweep kernels of the split shallow-water step (arXiv 1410.0753, section "Numerics").
//
//  k_step_fused  one full step (x-sweep then y-sweep) per launch. A warp owns a strip of
//                56 output columns and S output rows. It walks the rows of its strip from
//                r0-3 to r0+S+2. Each row (64 columns of eta, u, v, d and, when max-wave is
//                due, the max-wave rows three rows behind) arrives in shared memory by TMA
//                (cp.async.bulk.tensor) through a 4-slot ring per warp with one mbarrier per
//                slot; one lane keeps the ring RING rows ahead. The row is x-swept across the
//                warp with shuffles and pushed into a per-column register pipeline that
//                finishes the y-sweep three rows behind. The step reads eta, u, v, d and
//                writes eta, u, v once per cell (28 B/cell-update plus the halo), fused with
//                the max-wave update (+8 B) and the gauge / enclosed-grid sampling.
//  k_batch       the same per-warp work in a persistent cooperative kernel that loops over
//                the steps of a batch of scenarios, with a grid barrier between steps.
//  k_xsweep      x-sweep alone (1D grids along x).
//  k_ysweep      y-sweep alone (1D grids along y).
// Variants (template parameters): spherical metric (SPH), friction on (FRIC), a y-first step
// of the alternating order (YF, fused step only), eq. (solver1) (S1) and open outer edges
// (OPEN); the launchers pick one from kernel tables. The templates live in step_kernels.cuh;
// this file instantiates the reflecting-edge kernels, cliffs_step_open.cu the OPEN ones. Every mbarrier wait and the grid barrier are bounded (about a
// second of clock); on expiry the warp raises the timeout flag, drains the copies it issued
// (again bounded) and returns.
#include "step_kernels.cuh"

namespace cliffs {

// ------------------------------------------------------------------ launchers
// the ring needs more than the default 48 KB of dynamic shared memory per block
// Kernel variants, indexed by the grid's metric (spherical: +1), friction (on: +2), sweep
// order of the step (y first: +4) and solver (eq. (solver1): +8 for the fused step, +4 for
// the others); grids with open outer edges take the OPEN instantiations of the same tables.
#define CLIFFS_V2(K, ...) (const void*)K<false, false, __VA_ARGS__>, (const void*)K<true, false, __VA_ARGS__>, \
                          (const void*)K<false, true, __VA_ARGS__>, (const void*)K<true, true, __VA_ARGS__>

// the same tables for grids with open outer edges (cliffs_step_open.cu)
const void* fused_kernel_open(int v);
const void* batch_kernel_open(int v);
const void* batch_kernel_alt(int v);        // the alternating order (cliffs_step_alt.cu), v + 8 open
const void* xsweep_kernel_open(int v);
const void* ysweep_kernel_open(int v);

static const void* fused_kernel(bool sph, bool fric, bool yf, bool s1, bool open) {
    static const void* const t[16] = {CLIFFS_V2(k_step_fused, false, false, false), CLIFFS_V2(k_step_fused, true, false, false),
                                      CLIFFS_V2(k_step_fused, false, true, false), CLIFFS_V2(k_step_fused, true, true, false)};
    const int v = (sph ? 1 : 0) + (fric ? 2 : 0) + (yf ? 4 : 0) + (s1 ? 8 : 0);
    return open ? fused_kernel_open(v) : t[v];
}
static const void* batch_kernel(bool sph, bool fric, bool s1, bool open, bool alt) {
    static const void* const t[8] = {CLIFFS_V2(k_batch, false, false, false), CLIFFS_V2(k_batch, true, false, false)};
    const int v = (sph ? 1 : 0) + (fric ? 2 : 0) + (s1 ? 4 : 0);
    if (alt) return batch_kernel_alt(v + (open ? 8 : 0));
    return open ? batch_kernel_open(v) : t[v];
}
static const void* xsweep_kernel(bool sph, bool fric, bool s1, bool open) {
    static const void* const t[8] = {CLIFFS_V2(k_xsweep, false, false), CLIFFS_V2(k_xsweep, true, false)};
    const int v = (sph ? 1 : 0) + (fric ? 2 : 0) + (s1 ? 4 : 0);
    return open ? xsweep_kernel_open(v) : t[v];
}
static const void* ysweep_kernel(bool sph, bool fric, bool s1, bool open) {
    static const void* const t[8] = {CLIFFS_V2(k_ysweep, false, false), CLIFFS_V2(k_ysweep, true, false)};
    const int v = (sph ? 1 : 0) + (fric ? 2 : 0) + (s1 ? 4 : 0);
    return open ? ysweep_kernel_open(v) : t[v];
}

static bool solver1(const StepArgs& a) { return a.inv_dt2_s1 > 0.f; }

static cudaError_t fused_smem_optin() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady) {
        done = cudaSuccess;
        for (int v = 0; v < 32 && done == cudaSuccess; ++v)
            done = cudaFuncSetAttribute(fused_kernel(v & 1, v & 2, v & 4, v & 8, v & 16),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, FUSED_SMEM);
        for (int v = 0; v < 32 && done == cudaSuccess; ++v)
            done = cudaFuncSetAttribute(batch_kernel(v & 1, v & 2, v & 4, v & 8, v & 16),
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, FUSED_SMEM);
    }
    return done;
}

cudaError_t launch_step_fused(const StepArgs& a, const StepMaps& m, int batch, cudaStream_t s) {
    const cudaError_t e = fused_smem_optin();
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nitems + FUSED_WARPS - 1) / FUSED_WARPS, batch);
    StepMaps mm = m;
    StepArgs aa = a;
    void* args[] = {&mm, &aa};
    return cudaLaunchKernel(fused_kernel(a.sph, a.dt_gn2 > 0.f, a.yfirst != 0, solver1(a), a.open_edges != 0), grid,
                            dim3(FUSED_WARPS * 32), args, FUSED_SMEM, s);
}

cudaError_t launch_batch(const StepArgs& a, const StepMaps2& mm, const BatchArgs& b, int blocks, cudaStream_t s) {
    const cudaError_t e = fused_smem_optin();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(FUSED_WARPS * 32);
    cfg.dynamicSmemBytes = FUSED_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;         // all blocks resident: the grid barrier
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    StepMaps2 m2 = mm;
    StepArgs aa = a;
    BatchArgs bb = b;
    void* args[] = {&m2, &aa, &bb};
    return cudaLaunchKernelExC(&cfg, batch_kernel(a.sph, a.dt_gn2 > 0.f, solver1(a), a.open_edges != 0, b.alternate != 0), args);
}

int batch_blocks_per_sm(bool sph) {
    if (fused_smem_optin() != cudaSuccess) return 1;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_kernel(sph, true, false, false, false), FUSED_WARPS * 32, FUSED_SMEM);
    return nb;
}

int fused_blocks_per_sm(bool sph) {
    if (fused_smem_optin() != cudaSuccess) return 1;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fused_kernel(sph, true, false, false, false), FUSED_WARPS * 32,
                                                  FUSED_SMEM);
    return nb;
}

int fused_warps_per_block() { return FUSED_WARPS; }

cudaError_t launch_xsweep(const StepArgs& a, int batch, cudaStream_t s) {
    const dim3 grid((a.nstrips * a.ny + 3) / 4, batch);
    StepArgs aa = a;
    void* args[] = {&aa};
    return cudaLaunchKernel(xsweep_kernel(a.sph, a.dt_gn2 > 0.f, solver1(a), a.open_edges != 0), grid, dim3(128), args, 0, s);
}

cudaError_t launch_ysweep(const StepArgs& a, int batch, cudaStream_t s) {
    const int nw = a.nstrips * a.nseg;
    const dim3 grid((nw + 3) / 4, batch);
    StepArgs aa = a;
    void* args[] = {&aa};
    return cudaLaunchKernel(ysweep_kernel(a.sph, a.dt_gn2 > 0.f, solver1(a), a.open_edges != 0), grid, dim3(128), args, 0, s);
}

}  // namespace cliffs
