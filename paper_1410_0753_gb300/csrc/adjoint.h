// Declarations of the adjoint kernels' launchers (adjoint.cu), used by the adjoint driver in
// cliffs_api.cu; kept apart from internal.h, which the forward step kernels include.
#pragma once
#include "internal.h"

namespace cliffs {

// Adjoint of the sweeps along one direction (adjoint.cu). Lines lie along memory: line l,
// position p at l * ipitch + p; the output goes to p * opitch + l (transposed).
struct AdjLineArgs {
    const float *pe, *pw, *pt, *pd;  // primal sweep input: eta, velocity along, across, depth
    const float *ge, *gw, *gt;       // adjoint of the sweep output, same layout
    float *oe, *ow, *ot;             // adjoint of the sweep input, transposed layout
    int nlines, npos, ipitch, opitch;
    const float *xa, *xb, *xk, *xrow;  // x-sweep metric (lines are rows)
    const float4* ymet;              // y-sweep metric (lines are columns)
    const int* gxy;                  // gauge nodes (ix, iy)
    int G;
    const float* seed;               // dL/d (eta, u, v) at the gauges for this step ([G][3]), or null
    float hmin, dwall, half_dt, dt_gn2;
    int transverse;
    float inv_dt2_s1;                // 1/dt^2 with eq. (solver1), else 0
    int open_lo, open_hi;            // the line's first / last node is at an open outer edge
};

// pdl: launched with programmatic stream serialization. For k_adj_line the kernel then
// starts early and waits for its predecessor before reading anything it wrote; for
// k_adj_xfwd only right behind the x-sweep adjoint of the next step (see adjoint.cu).
cudaError_t launch_adj_line(const AdjLineArgs& A, int dir, bool sph, cudaStream_t s, bool pdl = false);
cudaError_t launch_adj_xfwd(const StepArgs& a, const float* e, const float* u, const float* v, float* te,
                            float* tu, float* tv, int tpitch, cudaStream_t s, bool pdl = false);
cudaError_t launch_transpose(const float* in, int ipitch, float* out, int opitch, int rows, int cols,
                             cudaStream_t s);
cudaError_t launch_adj_seed(float* te, int tpitch, long long tplane, const int* gxy, int G, const float* seed,
                            cudaStream_t s);
cudaError_t launch_adj_zero_edges(float* t, int tpitch, int nx, int ny, int mask, cudaStream_t s);

}  // namespace cliffs
