// Internal interface between the host runtime (cliffs_api.cu) and the kernel translation
// units. Not part of the public ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cliffs {

// Arguments of one sweep-kernel launch (all device pointers). Fields 2D are pitched:
// element (b, r, c) lives at b * plane + r * pitch + c.
struct StepArgs {
    const float* eta_in; const float* u_in; const float* v_in;
    float* eta_out; float* u_out; float* v_out;
    const float* d;                  // [ny][pitch], FP32 depth
    const float* xa; const float* xb; const float* xk;   // [nx] per-column x metric
    // per-row tables, valid for row indices -MET_PAD .. ny + MET_PAD - 1 (edge rows repeated)
    const float* xrow;               // row factor of the x metric (1 or 1/(R cos phi))
    const float4* ymet;              // (1/dy_{j-1}, 1/dy_j, dt^2/(dy_{j-1}+dy_j), dt tan(phi)/R)
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
    int S;                           // output rows per warp (y kernel)
    int nstrips, nseg;
    const int4* items;               // fused kernel: per warp (strip, first row, end row)
    int nitems;
    float hmin, dwall, half_dt, dt_gn2;
    int transverse;
    int sph;                         // geographic grid: x metric scaled per row
    int yfirst;                      // this step sweeps y, then x (alternating order)
    float inv_dt2_s1;                // 1/dt^2 with eq. (solver1), 0 with eq. (solver2)
    int open_edges;                  // open outer edges: bits W 1, E 2, S 4, N 8
    long long wait_cycles;           // limit of every mbarrier wait (clock cycles)
    unsigned tx_pad;                 // extra bytes each ring slot expects (fault injection; 0)
};

enum { ERRF_NONFINITE = 1, ERRF_TIMEOUT = 2 };
constexpr int MET_PAD = 8;
constexpr int TMA_BOX_COLS = 64;   // columns of one TMA box (a warp's window)
constexpr int TMA_BOX_ROWS = 2;    // rows of one TMA box (one ring slot)

// Depth-jump filter (section "Numerical stability", eqs. (dstab), (newdw), (newdc)), one
// node per thread; shared by cliffs_set_bathy and cliffs_depth_filter_noalloc so that both
// launch the same code. Wet nodes (0 < d < min_depth) are first raised to min_depth.
__device__ __forceinline__ void filter_minraise_node(double* d, long long i, double min_depth) {
    if (d[i] > 0.0 && d[i] < min_depth) d[i] = min_depth;
}
// One Jacobi pass along rows (dir 0) or columns (dir 1) at node i of an nx x ny grid: where a
// wet neighbour is deeper than alpha^2 d_j, d_j becomes the square of the mean square root of
// its two neighbours (open water) or the coastal neighbour's depth over alpha^2; land
// (d <= 0) and lines shorter than 3 nodes stay. Sets *changed when the node changed.
__device__ __forceinline__ void filter_pass_node(const double* in, double* out, long long i, int nx, int ny,
                                                 int dir, double a2, int* changed) {
    const int r = (int)(i / nx), c = (int)(i % nx);
    const int n = dir == 0 ? nx : ny, j = dir == 0 ? c : r;
    const long long st = dir == 0 ? 1 : nx;
    const double dj = in[i];
    double nd = dj;
    if (n >= 3 && dj > 0.0) {
        const bool lw = j > 0 && in[i - st] > 0.0;
        const bool rw = j < n - 1 && in[i + st] > 0.0;
        const bool viol = (lw && in[i - st] > a2 * dj) || (rw && in[i + st] > a2 * dj);
        if (viol) {
            if (lw && rw) {
                const double s = sqrt(in[i - st]) + sqrt(in[i + st]);
                nd = s * s / 4.0;
            } else {
                nd = (lw ? in[i - st] : in[i + st]) / a2;
            }
        }
    }
    out[i] = nd;
    if (nd != dj) *changed = 1;
}

// message returned by cliffs_last_error() on the calling thread (cliffs_api.cu)
void set_last_error(const char* msg);

// TMA descriptors of the fused step's inputs: eta, u, v, eta_max, speed_max as 3D
// [batch][ny][pitch] tensors and d as a 2D [ny][pitch] tensor, each read as 64 x 1 boxes.
struct StepMaps {
    CUtensorMap e, u, v, d, em, sm;
};

struct StepMaps2 {
    StepMaps m[2];                   // [k]: buffer k is the input
};

// The batched persistent run (k_batch). ctl lives in device memory so that one captured
// graph serves every call: ctl[0] = steps done before the launch, ctl[1] = steps done after
// it, ctl[2] = grid barrier (arrival count in the low 32 bits, generation in the high 32),
// ctl[3] = work-item ticket counters for even (low 32 bits) and odd (high 32) steps.
// Interpolation of one step's boundary input per edge: record k and weight w toward k + 1.
struct BndRow {
    long long k[4];
    double w[4];
};

struct BatchArgs {
    long long* ctl;
    const int* order;                // scenarios by decreasing step limit
    const int* nact;                 // [nact_len]: scenarios whose limit is >= the step; null: all
    long long nact_len;
    int nall;                        // the batch size
    float* eta[2]; float* u[2]; float* v[2];
    float* emax; float* smax;
    int maxout, gout, bndout;
    float* grec;                     // gauge records, row = step / gout (scenario stride in StepArgs)
    long long grec_row;              // floats per record row
    float* nrec;                     // enclosed-grid corner records, row = step / bndout
    long long nrec_row;
    int alternate;                   // y first on the odd steps (the alternating order)
    // boundary input (batch 1): before step step0 + 1 + j the edge nodes of its input take
    // record k, weight w of bnd_rows[j] (computed on the host as cliffs_step_n does)
    int bnd;
    const BndRow* bnd_rows;
    const double* bv[4];             // records [nt][3][np] per edge, or null
    int bnp[4];                      // nodes per edge
};

// Edge node q of edge e (0 W, 1 E, 2 S, 3 N) takes its input (u, v, eta) from record k with
// weight w toward k + 1 (the interpolation in FP64, non-fused, then rounded to FP32). S and
// N own the corners when they carry input. Shared by the per-step kernel and the persistent
// one, so both give the same bits.
__device__ __forceinline__ void bnd_apply(float* eta, float* u, float* v, int pitch, int nx, int ny, int e, int q,
                                          const double* const* vals, const int* np, long long k, double w) {
    if (!vals[e] || q >= np[e]) return;
    if (e < 2 && ((q == 0 && vals[2]) || (q == ny - 1 && vals[3])) && nx > 1 && ny > 1) return;
    const int ix = (e == 0) ? 0 : (e == 1) ? nx - 1 : q;
    const int iy = (e == 2) ? 0 : (e == 3) ? ny - 1 : q;
    const int n = np[e];
    const double* r0 = vals[e] + k * 3 * n;
    double val[3];
    for (int f = 0; f < 3; ++f) {
        const double a = r0[f * n + q];
        val[f] = (w > 0.0) ? __dadd_rn(__dmul_rn(__dsub_rn(1.0, w), a), __dmul_rn(w, r0[(3 + f) * n + q])) : a;
    }
    const size_t o = (size_t)iy * pitch + ix;
    u[o] = (float)val[0];
    v[o] = (float)val[1];
    eta[o] = (float)val[2];
}

// launchers (cliffs_step.cu)
cudaError_t launch_batch(const StepArgs& a, const StepMaps2& mm, const BatchArgs& b, int blocks, cudaStream_t s);
int batch_blocks_per_sm(bool sph);
cudaError_t launch_step_fused(const StepArgs& a, const StepMaps& m, int batch, cudaStream_t s);
int fused_blocks_per_sm(bool sph);
int fused_warps_per_block();
cudaError_t launch_xsweep(const StepArgs& a, int batch, cudaStream_t s);
cudaError_t launch_ysweep(const StepArgs& a, int batch, cudaStream_t s);

}  // namespace cliffs
