// Internal interface between the host runtime (cliffs_api.cu) and the kernel translation
// units. Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cliffs {

struct SweepConstH {       // mirror of SweepConst for host code
    float hmin, dwall, half_dt, dt_gn2;
    int transverse;
};

// Arguments of one sweep-kernel launch (all device pointers). Fields 2D are pitched:
// element (b, r, c) lives at b * plane + r * pitch + c.
struct StepArgs {
    const float* eta_in; const float* u_in; const float* v_in;
    float* eta_out; float* u_out; float* v_out;
    const float* d;                  // [ny][pitch], FP32 depth
    const float* xa; const float* xb; const float* xk;   // [nx] per-column x metric
    const float* xrow;               // [ny] row factor of the x metric (1 or 1/(R cos phi))
    const float4* ymet;              // [ny] (1/dy_{j-1}, 1/dy_j, dt^2/(dy_{j-1}+dy_j), dt tan(phi)/R)
    float* emax; float* smax;        // max-wave fields, or null when not due this step
    float* rec_g;                    // gauge record row of this step (scenario 0) or null
    float* rec_n;                    // enclosed-grid node record row or null
    long long rec_g_bstride;         // floats between scenarios in the gauge records
    const int* samp_ptr;             // [nwarps + 1] per-warp sample list (CSR)
    const int4* samp;                // (row, col, class 0 gauge / 1 node, slot)
    const long long* limit;          // [batch] step limits, or null
    long long step;                  // index of the step being produced (1-based)
    int* err;                        // device error flags
    int nx, ny, pitch;
    long long plane;
    int S;                           // output rows per warp (fused / y kernels)
    int nstrips, nseg;
    float hmin, dwall, half_dt, dt_gn2;
    int transverse;
    int sph;                         // geographic grid: x metric scaled per row
};

enum { ERRF_NONFINITE = 1, ERRF_TIMEOUT = 2 };

// message returned by cliffs_last_error() on the calling thread (cliffs_api.cu)
void set_last_error(const char* msg);

// launchers (cliffs_step.cu)
cudaError_t launch_step_fused(const StepArgs& a, int batch, int wpb, cudaStream_t s);
cudaError_t launch_xsweep(const StepArgs& a, int batch, cudaStream_t s);
cudaError_t launch_ysweep(const StepArgs& a, int batch, cudaStream_t s);

}  // namespace cliffs
