// Host runtime of libcliffs.so: the C ABI declared in include/cliffs.h.
//
// A grid owns its device buffers: the FP32 state eta, u, v (double-buffered, rows padded to
// a pitch of 32 floats so that the sweep kernels' 8-byte vector accesses stay aligned), the
// FP32 and FP64 depth, the max-wave fields, the per-row / per-column metric tables and the
// gauge / enclosed-grid record buffers. Every step of the method runs in a kernel: the
// sweeps (cliffs_step.cu), the depth filter, the initial-state set-up, the records and the
// reductions of the read-out calls (this file). Host code only validates arguments,
// computes the metric and interpolation tables, and sequences launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "cliffs.h"
#include "internal.h"
#include "adjoint.h"
#include "sweep.cuh"

using namespace cliffs;

namespace {

thread_local char g_err[1024] = "";

int set_err(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

#define CK(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_err(e_ == cudaErrorMemoryAllocation ? CLIFFS_ERR_NOMEM : CLIFFS_ERR_CUDA, \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

const double R_SPHERE = 6371000.0;
const double DEGR = 3.14159265358979323846 / 180.0;

// The adjoint recomputes its segments of K steps several at a time, as one batched launch
// per step: as many segments as fit in this many bytes of recomputed states, tiled to fill
// about this many waves of resident warps.
#ifndef CLIFFS_ADJ_GROUP_GIB
#define CLIFFS_ADJ_GROUP_GIB 16
#endif
#ifndef CLIFFS_ADJ_GROUP_WAVES
#define CLIFFS_ADJ_GROUP_WAVES 3
#endif
const double ADJ_GROUP_BYTES = (double)CLIFFS_ADJ_GROUP_GIB * (1 << 30);
const int ADJ_GROUP_MAX = 16;                  // and at most this many segments per launch
const int ADJ_GROUP_WAVES = CLIFFS_ADJ_GROUP_WAVES;
#ifndef CLIFFS_ADJ_PDL
#define CLIFFS_ADJ_PDL 1
#endif
const bool ADJ_PDL = CLIFFS_ADJ_PDL != 0;     // programmatic launches between the adjoint's kernels

// ----------------------------------------------------------------------------- kernels

// depth-jump filter, section "Numerical stability": eqs. (dstab), (newdw), (newdc)
__global__ void k_filter_minraise(double* d, long long n, double min_depth) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) filter_minraise_node(d, i, min_depth);
}

// One Jacobi pass along rows (dir 0) or columns (dir 1).
__global__ void k_filter_pass(const double* in, double* out, int nx, int ny, int dir, double a2,
                              int* changed) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < (long long)nx * ny) filter_pass_node(in, out, i, nx, ny, dir, a2, changed);
}

__global__ void k_depth_to_f32(const double* d64, float* d32, int nx, int ny, int pitch) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)ny * pitch) return;
    const int r = (int)(i / pitch), c = (int)(i % pitch);
    d32[i] = (c < nx) ? (float)d64[(long long)r * nx + c] : OUTSIDE_D;
}

// largest still-water Courant number sqrt(g d) dt / dx over wet nodes, both directions
__global__ void k_cfl(const double* d64, int nx, int ny, const float* xa, const float* xb,
                      const float* xrow, const float4* ymet, double dt, unsigned* out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int r = (int)(i / nx), c = (int)(i % nx);
    const double d = d64[i];
    if (!(d > 0.0)) return;
    double inv = 0.0;
    if (nx > 1) inv = fmax((double)xa[c], (double)xb[c]) * (double)xrow[r];
    if (ny > 1) inv = fmax(inv, fmax((double)ymet[r].x, (double)ymet[r].y));
    const float cour = (float)(sqrt(9.81 * d) * dt * inv);
    atomicMax(out, __float_as_uint(cour));
}

// quake = 1: the deformation zeta lifts the sea floor (d <- d - zeta) and, on nodes that
// were wet, the free surface with it (eta <- zeta); elsewhere eta = 0.
__global__ void k_quake(double* d64, const float* zeta, float* eta, float* d32, int nx, int ny,
                        int pitch, double hmin, double dwall) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int r = (int)(i / nx), c = (int)(i % nx);
    const double d = d64[i];
    const float z = zeta[i];
    const bool wet = (d >= dwall) && (d >= hmin);
    eta[(long long)r * pitch + c] = wet ? z : 0.f;
    const double nd = d - (double)z;
    d64[i] = nd;
    d32[(long long)r * pitch + c] = (float)nd;
}

// max-wave initialisation from the state of step 0 (wet nodes), batched over planes
__global__ void k_max_init(const float* eta, const float* u, const float* v, const float* d,
                           float* emax, float* smax, int nx, int ny, int pitch, long long plane,
                           int b0, int nb, float hmin, float dwall) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nb * plane) return;
    const long long o = (long long)b0 * plane + i;
    const long long p = i % plane;
    const int c = (int)(p % pitch);
    const float dd = d[p];
    const float e = eta[o];
    const bool wet = c < nx && (dd >= dwall) && (e + dd >= hmin);
    emax[o] = wet ? e : -3.402823466e38f;
    smax[o] = wet ? sqrtf(u[o] * u[o] + v[o] * v[o]) : 0.f;
    (void)ny;
}

// Diagnostics of one state plane (a monitor, not a step of the method): over wet nodes (the
// max-wave test), the displaced volume sum eta * wx_i * wy_j, the node count, max |eta| and
// max speed. FP64 sums per block, then one atomic per block; the maxima are non-negative
// floats, so their bit patterns order like unsigned integers.
__global__ void k_diag(const float* eta, const float* u, const float* v, const float* d32,
                       const double* wx, const double* wy, int nx, int ny, int pitch, float hmin,
                       float dwall, double* acc, unsigned* mx) {
    double vol = 0.0, cnt = 0.0;
    float me = 0.f, ms = 0.f;
    const long long N = (long long)nx * ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(i / nx), c = (int)(i % nx);
        const long long o = (long long)r * pitch + c;
        const float e = eta[o], dd = d32[o];
        if (!((dd >= dwall) && (e + dd >= hmin))) continue;
        vol += (double)e * wx[c] * wy[r];
        cnt += 1.0;
        me = fmaxf(me, fabsf(e));
        ms = fmaxf(ms, sqrtf(u[o] * u[o] + v[o] * v[o]));
    }
    __shared__ double sv[8], sc[8];
    __shared__ float se[8], ss[8];
    for (int k = 16; k > 0; k >>= 1) {
        vol += __shfl_down_sync(0xffffffffu, vol, k);
        cnt += __shfl_down_sync(0xffffffffu, cnt, k);
        me = fmaxf(me, __shfl_down_sync(0xffffffffu, me, k));
        ms = fmaxf(ms, __shfl_down_sync(0xffffffffu, ms, k));
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sv[w] = vol; sc[w] = cnt; se[w] = me; ss[w] = ms; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            vol += sv[k]; cnt += sc[k]; me = fmaxf(me, se[k]); ms = fmaxf(ms, ss[k]);
        }
        atomicAdd(&acc[0], vol);
        atomicAdd(&acc[1], cnt);
        atomicMax(&mx[0], __float_as_uint(me));
        atomicMax(&mx[1], __float_as_uint(ms));
    }
}

// step-0 record of the gauges / enclosed-grid nodes of scenarios [b0, b0 + nb)
__global__ void k_record0(const float* eta, const float* u, const float* v, int pitch,
                          long long plane, const int4* items, int nitems, float* rec_g,
                          long long g_bstride, float* rec_n, int b0, int nb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nitems * nb) return;
    const int k = t % nitems, b = b0 + t / nitems;
    const int4 it = items[k];
    const long long o = (long long)b * plane + (long long)it.x * pitch + it.y;
    float* out = it.z == 0 ? rec_g + (long long)b * g_bstride : (b == 0 ? rec_n : nullptr);
    if (!out) return;
    out[3 * it.w + 0] = eta[o];
    out[3 * it.w + 1] = u[o];
    out[3 * it.w + 2] = v[o];
}

// max-wave read-out: stored maxima folded with the current (last) state, dense output
__global__ void k_max_fold(const float* emax, const float* smax, const float* eta, const float* u,
                           const float* v, const float* d, float* oe, float* os, int nx, int ny,
                           int pitch, float hmin, float dwall) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int r = (int)(i / nx), c = (int)(i % nx);
    const long long o = (long long)r * pitch + c;
    float em = emax[o], sm = smax[o];
    const float e = eta[o], dd = d[o];
    if ((dd >= dwall) && (e + dd >= hmin)) {
        em = fmaxf(em, e);
        sm = fmaxf(sm, sqrtf(u[o] * u[o] + v[o] * v[o]));
    }
    if (oe) oe[i] = em;
    if (os) os[i] = sm;
}

// boundary series of one edge: bilinear combination of the recorded corner nodes, FP64,
// vals[t][q][p] with q = 0 u, 1 v, 2 eta
__global__ void k_boundary(const float* nrec, int nnodes, const int* slot, const double* wt,
                           int p0, int np, long long nt, double* vals) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nt * np) return;
    const long long t = i / np;
    const int p = (int)(i % np);
    const float* rec = nrec + t * (long long)nnodes * 3;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 4; ++k) {
        const int s = slot[4 * (p0 + p) + k];
        const double w = wt[4 * (p0 + p) + k];
        acc[0] += w * (double)rec[3 * s + 1];
        acc[1] += w * (double)rec[3 * s + 2];
        acc[2] += w * (double)rec[3 * s + 0];
    }
    for (int q = 0; q < 3; ++q) vals[(t * 3 + q) * np + p] = acc[q];
}

inline unsigned nblk(long long n, int bs = 256) { return (unsigned)((n + bs - 1) / bs); }

// Boundary input for one step: per edge the series and the two records (k, k+1) to mix
// with weight w.
struct BndStep {
    const double* vals[4];
    int np[4];
    long long k[4];
    double w[4];
};

// Edge nodes take the input (u, v, eta); S and N own the corners when they have input.
__global__ void k_bnd(float* eta, float* u, float* v, int pitch, int nx, int ny, BndStep b) {
    const int e = blockIdx.y;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    bnd_apply(eta, u, v, pitch, nx, ny, e, q, b.vals, b.np, b.k[e], b.w[e]);
}

// Bilinear interpolation of a source field [sny][snx] onto the master nodes: per master
// column the source interval and fraction (col[ix] = (i, a), i < 0 outside), per row alike;
// zero outside the source grid. FP64 arithmetic, rounded once to FP32.
struct Ax { int i; double a; };
__global__ void k_interp(const float* __restrict__ src, int snx, const Ax* __restrict__ col,
                         const Ax* __restrict__ row, int nx, int ny, float* out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nx * ny) return;
    const int ix = (int)(idx % nx), iy = (int)(idx / nx);
    const Ax c = col[ix], r = row[iy];
    if (c.i < 0 || r.i < 0) { out[idx] = 0.f; return; }
    const int i1 = c.a > 0.0 ? c.i + 1 : c.i, j1 = r.a > 0.0 ? r.i + 1 : r.i;
    const double v00 = src[(long long)r.i * snx + c.i], v01 = src[(long long)r.i * snx + i1];
    const double v10 = src[(long long)j1 * snx + c.i], v11 = src[(long long)j1 * snx + i1];
    out[idx] = (float)((1.0 - r.a) * ((1.0 - c.a) * v00 + c.a * v01) + r.a * ((1.0 - c.a) * v10 + c.a * v11));
}

}  // namespace

void cliffs::set_last_error(const char* msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
}

// ----------------------------------------------------------------------------- grid

struct cliffs_grid {
    cliffs_config cfg{};
    std::vector<int32_t> gauges;
    std::vector<cliffs_nest> nests;
    int nx = 0, ny = 0, B = 1, pitch = 0;
    long long plane = 0;
    cudaStream_t stream = nullptr;
    bool have_bathy = false, have_init = false;
    std::vector<double> hx, hy;              // node coordinates as given to set_bathy
    float* eta[2] = {nullptr, nullptr};
    float* u[2] = {nullptr, nullptr};
    float* v[2] = {nullptr, nullptr};
    float* d32 = nullptr;
    double* d64 = nullptr;
    double* d64b = nullptr;
    float* emax = nullptr;
    float* smax = nullptr;
    float *xa = nullptr, *xb = nullptr, *xk = nullptr, *xrow = nullptr;
    float4* ymet = nullptr;
    int* err = nullptr;
    long long inject_cycles = 0;             // armed by cliffs_inject_wait_expiry
    long long* limit = nullptr;
    std::vector<long long> limit_h;
    long long step = 0;
    // samples: gauges (class 0) then enclosed-grid corner nodes (class 1)
    std::vector<int4> samples;
    int G = 0, NN = 0;
    int4* items_d = nullptr;
    int* samp_ptr = nullptr;
    int4* samp = nullptr;
    // records
    float* grec = nullptr;
    long long grec_cap = 0;
    float* nrec = nullptr;
    long long nrec_cap = 0;
    // enclosed-grid boundary points
    std::vector<int> edge_off, edge_np;      // per nest * 4 + edge
    int* pt_slot = nullptr;
    double* pt_w = nullptr;
    // TMA descriptors: [k] reads buffer k as the step input
    StepMaps maps[2];
    // launch geometry
    int kind = 0;                            // 0 fused 2D, 1 x only, 2 y only
    int S = 32, nstrips = 0, nseg = 0;
    int S_hard = 32;                         // rows per warp in strips with dry nodes / edges
    std::vector<unsigned char> hard;         // per strip: dry nodes in its window, or an edge
    std::vector<int4> items;                 // fused kernel work items (strip, r0, r1, 0)
    int4* items_dev = nullptr;
    // timing
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
    double t_ms = 0.0;
    long long t_launches = 0;
    // scratch for read-outs
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    unsigned* ured = nullptr;
    // persistent batched run: scenario order and running counts (from the durations), the
    // device control block with its pinned host image, and the captured graph with the
    // launch arguments it was captured with
    int* order_d = nullptr;
    int* nact_d = nullptr;
    long long nact_len = 0;
    long long* ctl_d = nullptr;
    long long* ctl_h = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<unsigned char> gkey;
    int pblocks = 0;
    // adjoint work space: K recomputed states of up to adj_G segments ([3][adj_G][plane]
    // per state) and the checkpoints (row-major, 3 planes each), the transposed x-swept
    // state, adjoint and depth (7 planes of [nx][tpitch]), the row-major intermediate
    // adjoint (3 planes), gauge nodes and seeds; the work items of the batched segment
    // recomputation (adj_S rows per warp)
    int adj_K = 0;
    int adj_G = 0;
    // the checkpoint pass: two states to step between (3 planes each) and their TMA
    // descriptors; descriptors of single planes of the state slots (batch extent 1), made
    // when first needed: [slot * adj_G + plane]
    float* adj_pp = nullptr;
    StepMaps adj_ppmaps[2];
    std::vector<StepMaps> adj_pmaps;
    std::vector<unsigned char> adj_pmaps_ok;
    int adj_S = 0;
    std::vector<int4> adj_items;
    int4* adj_items_dev = nullptr;
    long long adj_ncap = 0;
    float* adj_slots = nullptr;
    float* adj_ckpt = nullptr;
    float* adj_t = nullptr;
    float* adj_lb = nullptr;
    std::vector<StepMaps> adj_maps;
    int* adj_gxy = nullptr;
    float* adj_seed = nullptr;
    long long adj_seed_cap = 0;
    // boundary input: per edge (W, E, S, N) the record times (host) and (u, v, eta) series
    // (device), the model clock and whether a run stops at the end of the records
    // forward checkpoints recorded by cliffs_step_n for cliffs_adjoint_recorded: spacing K
    // (0: off), state every K steps since set_initial, steps recorded
    int rec_K = 0;
    float* rec_ckpt = nullptr;
    long long rec_cap = 0;
    long long rec_n = 0;
    bool adj_done = false;                   // the adjoint state of the last adjoint call is kept
    float* adj_alt = nullptr;                // alternating order: y-swept state (3 row-major planes)
                                             // and an intermediate adjoint (3 transposed planes)
    std::vector<double> bnd_t[4];
    double* bnd_v[4] = {nullptr, nullptr, nullptr, nullptr};
    BndRow* bnd_rows = nullptr;              // per-step interpolation table of a persistent run
    long long bnd_rows_cap = 0;
    bool bnd_any = false;
    double t_start = 0.0;
    bool bnd_stop = false;
};

namespace {

int ensure_tmp(cliffs_grid* g, size_t bytes) {
    if (bytes <= g->tmp_bytes) return CLIFFS_OK;
    if (g->tmp) CK(cudaFree(g->tmp));
    g->tmp = nullptr;
    g->tmp_bytes = 0;
    CK(cudaMalloc(&g->tmp, bytes));
    g->tmp_bytes = bytes;
    return CLIFFS_OK;
}

long long cur_buf(const cliffs_grid* g, int b) {
    long long s = g->step;
    if (g->limit_h.size() && g->limit_h[b] >= 0) s = std::min(s, g->limit_h[b]);
    return s & 1;
}

long long steps_of(const cliffs_grid* g, int b) {
    long long s = g->step;
    if (g->limit_h.size() && g->limit_h[b] >= 0) s = std::min(s, g->limit_h[b]);
    return s;
}

// Strips of the fused kernels (2D grids): window s holds columns 56 s .. 56 s + 63 and
// finishes columns 56 s + 4 .. 56 s + 59, the first from column 0 and the last to column
// nx - 1 (there the domain's edge is the window's, or past it lie dry ghost columns).
int fused_strips(int nx) { return nx <= XWIN ? 1 : (nx - XWIN + XOUT - 1) / XOUT + 1; }
int fused_strip_of(int c, int nstrips) { return c < XOUT + 4 ? 0 : std::min((c - 4) / XOUT, nstrips - 1); }

// per-warp sample lists for the current launch geometry
int build_samples(cliffs_grid* g) {
    // a warp owns output columns [W * strip, W * strip + W): 56 for the x-sweep alone, 64 for
    // the y-sweep alone; the fused kernels' strips are those of fused_strips
    const int W = (g->kind == 2) ? XWIN : XOUT;
    const int S = g->kind == 1 ? 1 : g->S;
    const int nseg = g->kind == 1 ? g->ny : g->nseg;
    long long nw = (long long)g->nstrips * nseg;
    // kind 0: warp index of (row, strip) from the item table
    std::vector<std::vector<int>> seg_start;
    std::vector<std::vector<int>> seg_item;
    if (g->kind == 0) {
        nw = (long long)g->items.size();
        seg_start.assign(g->nstrips, {});
        seg_item.assign(g->nstrips, {});
        for (size_t i = 0; i < g->items.size(); ++i) {
            seg_start[g->items[i].x].push_back(g->items[i].y);
            seg_item[g->items[i].x].push_back((int)i);
        }
    }
    std::vector<std::vector<int4>> per(nw);
    for (const int4& it : g->samples) {
        long long w;
        if (g->kind == 0) {
            const int st = fused_strip_of(it.y, g->nstrips);
            const auto& v = seg_start[st];
            const int k = (int)(std::upper_bound(v.begin(), v.end(), it.x) - v.begin()) - 1;
            w = seg_item[st][k];
        } else {
            w = (long long)(it.x / S) * g->nstrips + it.y / W;
        }
        per[w].push_back(it);
    }
    std::vector<int> ptr(nw + 1, 0);
    std::vector<int4> flat;
    for (long long w = 0; w < nw; ++w) {
        std::stable_sort(per[w].begin(), per[w].end(),
                         [](const int4& a, const int4& b) { return a.x < b.x; });
        ptr[w] = (int)flat.size();
        flat.insert(flat.end(), per[w].begin(), per[w].end());
    }
    ptr[nw] = (int)flat.size();
    if (g->samp_ptr) CK(cudaFree(g->samp_ptr));
    if (g->samp) CK(cudaFree(g->samp));
    g->samp_ptr = nullptr;
    g->samp = nullptr;
    CK(cudaMalloc(&g->samp_ptr, sizeof(int) * (nw + 1)));
    CK(cudaMemcpy(g->samp_ptr, ptr.data(), sizeof(int) * (nw + 1), cudaMemcpyHostToDevice));
    if (!flat.empty()) {
        CK(cudaMalloc(&g->samp, sizeof(int4) * flat.size()));
        CK(cudaMemcpy(g->samp, flat.data(), sizeof(int4) * flat.size(), cudaMemcpyHostToDevice));
    }
    return CLIFFS_OK;
}

// Work items of the fused kernel: every strip is cut into segments of S rows, or S_hard
// rows in strips whose window holds dry nodes or reaches past the domain edge (their warps
// take the wet/dry correction paths on every row, so shorter segments even out the time
// the warps of one launch take).
int set_rows_per_warp(cliffs_grid* g, int S, int S_hard) {
    g->S = S;
    g->S_hard = S_hard;
    g->nseg = (g->ny + S - 1) / S;
    if (g->kind == 0) {
        g->items.clear();
        for (int st = 0; st < g->nstrips; ++st) {
            const int h = g->hard.empty() ? 0 : g->hard[st];
            const int seg = h ? S_hard : S;
            for (int r0 = 0; r0 < g->ny; r0 += seg)
                g->items.push_back(make_int4(st, r0, std::min(r0 + seg, g->ny), 0));
        }
        cudaFree(g->items_dev);
        g->items_dev = nullptr;
        CK(cudaMalloc(&g->items_dev, sizeof(int4) * g->items.size()));
        CK(cudaMemcpy(g->items_dev, g->items.data(), sizeof(int4) * g->items.size(), cudaMemcpyHostToDevice));
    }
    return build_samples(g);
}

int hard_rows(int S) { return std::max(8, (S * 3 / 4) & ~1); }

// warps of one fused launch with S rows per warp, and the warps resident at once
long long fused_warps(const cliffs_grid* g, int S) {
    int nhard = 0;
    for (int st = 0; st < g->nstrips; ++st) nhard += g->hard.empty() ? 0 : g->hard[st];
    const int Sh = hard_rows(S);
    return ((long long)(g->nstrips - nhard) * ((g->ny + S - 1) / S) +
            (long long)nhard * ((g->ny + Sh - 1) / Sh)) * g->B;
}

long long resident_warps(const cliffs_grid* g) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return (long long)std::max(1, nsm) * std::max(1, fused_blocks_per_sm(g->cfg.coords != 1)) *
           fused_warps_per_block();
}

// the smallest even S whose launch fits in `waves` waves of resident warps (0 if none does)
int wave_rows(const cliffs_grid* g, int waves) {
    const long long cap = resident_warps(g) * waves;
    for (int S = 8; S <= std::max(8, g->ny); S += 2)
        if (fused_warps(g, S) <= cap) return S;
    return 0;
}

int choose_geometry(cliffs_grid* g) {
    if (g->ny == 1) {
        g->kind = 1;
        g->nstrips = (g->nx + XOUT - 1) / XOUT;
        g->S = 1;
        g->nseg = g->ny;
    } else if (g->nx == 1) {
        g->kind = 2;
        g->nstrips = (g->nx + XWIN - 1) / XWIN;
        g->S = 64;
        g->nseg = (g->ny + g->S - 1) / g->S;
    } else {
        g->kind = 0;
        g->nstrips = fused_strips(g->nx);
        // rows per warp S: each warp walks S + 6 rows (3-row halo above and below), so the
        // cost of one wave of warps is ~ S + 6; pick the even S minimising waves * (S + 6)
        // with the resident warps the occupancy calculator reports (ties go to the larger S)
        const long long resident = resident_warps(g);
        double best = 1e300;
        int bestS = 32;
        for (int S = 8; S <= 1024; S += (S < 128 ? 2 : 32)) {
            if (S > 2 * g->ny && S != 8) break;
            const long long warps = fused_warps(g, S);
            const double cost = (double)((warps + resident - 1) / resident) * (S + 6);
            if (cost <= best) { best = cost; bestS = S; }
        }
        return set_rows_per_warp(g, bestS, hard_rows(bestS));
    }
    return build_samples(g);
}

int grow_records(cliffs_grid* g, long long need_g, long long need_n) {
    if (g->G > 0 && need_g > g->grec_cap) {
        const long long cap = std::max(need_g, 2 * g->grec_cap);
        float* nb = nullptr;
        const size_t rec = (size_t)g->G * 3 * sizeof(float);
        CK(cudaMalloc(&nb, (size_t)g->B * cap * rec));
        if (g->grec) {
            CK(cudaMemcpy2DAsync(nb, cap * rec, g->grec, g->grec_cap * rec, g->grec_cap * rec, g->B,
                                 cudaMemcpyDeviceToDevice, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            CK(cudaFree(g->grec));
        }
        g->grec = nb;
        g->grec_cap = cap;
    }
    if (g->NN > 0 && need_n > g->nrec_cap) {
        const long long cap = std::max(need_n, 2 * g->nrec_cap);
        float* nb = nullptr;
        const size_t rec = (size_t)g->NN * 3 * sizeof(float);
        CK(cudaMalloc(&nb, cap * rec));
        if (g->nrec) {
            CK(cudaMemcpyAsync(nb, g->nrec, g->nrec_cap * rec, cudaMemcpyDeviceToDevice, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            CK(cudaFree(g->nrec));
        }
        g->nrec = nb;
        g->nrec_cap = cap;
    }
    return CLIFFS_OK;
}

bool locate(const std::vector<double>& c, double xp, int* i, double* a) {
    const int n = (int)c.size();
    if (n == 1) { *i = 0; *a = 0.0; return xp == c[0]; }
    if (xp < c[0] || xp > c[n - 1]) return false;
    int k = (int)(std::upper_bound(c.begin(), c.end(), xp) - c.begin()) - 1;
    k = std::min(std::max(k, 0), n - 2);
    *i = k;
    *a = (xp - c[k]) / (c[k + 1] - c[k]);
    return true;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// a [batch][ny][pitch] FP32 tensor (batch 1 for the depth) read in 64 x 2 x 1 boxes;
// out-of-range boxes fill with zeros
int make_map(CUtensorMap* m, const float* base, int rank, int pitch, int ny, int batch) {
    auto fn = encode_fn();
    if (!fn) return set_err(CLIFFS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, (cuuint64_t)batch};
    cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * ny * 4};
    cuuint32_t box[3] = {(cuuint32_t)TMA_BOX_COLS, (cuuint32_t)TMA_BOX_ROWS, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, const_cast<float*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_err(CLIFFS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return CLIFFS_OK;
}

int make_maps(cliffs_grid* g) {
    for (int k = 0; k < 2; ++k) {
        StepMaps& M = g->maps[k];
        int rc = make_map(&M.e, g->eta[k], 3, g->pitch, g->ny, g->B);
        if (!rc) rc = make_map(&M.u, g->u[k], 3, g->pitch, g->ny, g->B);
        if (!rc) rc = make_map(&M.v, g->v[k], 3, g->pitch, g->ny, g->B);
        if (!rc) rc = make_map(&M.d, g->d32, 3, g->pitch, g->ny, 1);
        if (!rc) rc = make_map(&M.em, g->emax, 3, g->pitch, g->ny, g->B);
        if (!rc) rc = make_map(&M.sm, g->smax, 3, g->pitch, g->ny, g->B);
        if (rc) return rc;
    }
    return CLIFFS_OK;
}

void fill_step_args(cliffs_grid* g, StepArgs& a, int in, int out) {
    a.eta_in = g->eta[in]; a.u_in = g->u[in]; a.v_in = g->v[in];
    a.eta_out = g->eta[out]; a.u_out = g->u[out]; a.v_out = g->v[out];
    a.d = g->d32;
    a.xa = g->xa; a.xb = g->xb; a.xk = g->xk; a.xrow = g->xrow + MET_PAD; a.ymet = g->ymet + MET_PAD;
    a.emax = nullptr; a.smax = nullptr; a.rec_g = nullptr; a.rec_n = nullptr;
    a.rec_g_bstride = g->grec_cap * g->G * 3;
    a.samp_ptr = g->samp_ptr; a.samp = g->samp;
    a.limit = g->limit;
    a.err = g->err;
    a.nx = g->nx; a.ny = g->ny; a.pitch = g->pitch; a.plane = g->plane;
    a.S = g->S; a.nstrips = g->nstrips; a.nseg = g->nseg;
    a.items = g->items_dev; a.nitems = (int)g->items.size();
    a.hmin = (float)g->cfg.h_min;
    a.dwall = g->cfg.itopo ? -3.402823466e38f : (float)g->cfg.dwall;
    a.half_dt = (float)(0.5 * g->cfg.dt);
    a.dt_gn2 = (float)(g->cfg.dt * 9.81 * g->cfg.manning_n2);
    a.transverse = g->cfg.transverse ? 1 : 0;
    a.sph = g->cfg.coords != 1;
    a.wait_cycles = 2000000000LL;            // about a second at the GB300's clocks
    a.tx_pad = 0;
    a.yfirst = 0;
    a.inv_dt2_s1 = g->cfg.solver == 1 ? (float)(1.0 / (g->cfg.dt * g->cfg.dt)) : 0.f;
    a.open_edges = g->cfg.open_edges;
}

// dst[3][n] = (a, b, c): the three state planes into one checkpoint in one launch (n a
// multiple of 4; all pointers 16-byte aligned)
__global__ void k_copy3(float* __restrict__ dst, const float* __restrict__ a, const float* __restrict__ b,
                        const float* __restrict__ c, long long n) {
    const long long n4 = n / 4;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n4;
         i += (long long)gridDim.x * blockDim.x) {
        const long long f = i / n4, k = i - f * n4;
        const float4* src = reinterpret_cast<const float4*>(f == 0 ? a : f == 1 ? b : c);
        reinterpret_cast<float4*>(dst)[i] = __ldg(src + k);
    }
}

// Keep the current state of a recorded run as checkpoint `idx` (grows the store by doubling).
int record_checkpoint(cliffs_grid* g, long long idx) {
    const size_t st = sizeof(float) * 3 * g->B * g->plane;         // [3][batch][plane]
    if (idx >= g->rec_cap) {
        const long long cap = std::max<long long>(idx + 1, 2 * g->rec_cap);
        float* nb = nullptr;
        CK(cudaMalloc(&nb, st * cap));
        if (g->rec_ckpt) {
            CK(cudaMemcpyAsync(nb, g->rec_ckpt, st * g->rec_cap, cudaMemcpyDeviceToDevice, g->stream));
            CK(cudaStreamSynchronize(g->stream));
            CK(cudaFree(g->rec_ckpt));
        }
        g->rec_ckpt = nb;
        g->rec_cap = cap;
    }
    const int cb = (int)(g->step & 1);
    float* dst = g->rec_ckpt + (size_t)3 * g->B * g->plane * idx;
    k_copy3<<<1216, 256, 0, g->stream>>>(dst, g->eta[cb], g->u[cb], g->v[cb], (long long)g->B * g->plane);
    const cudaError_t le = cudaGetLastError();
    if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "checkpoint copy: %s", cudaGetErrorString(le));
    return CLIFFS_OK;
}

// Boundary input at model time t into the edge nodes of a state (batch 1).
// The record and weight of every edge's input at model time t (the first or last record
// outside their span).
static BndRow bnd_row(const cliffs_grid* g, double t) {
    BndRow r{};
    for (int e = 0; e < 4; ++e) {
        const std::vector<double>& T = g->bnd_t[e];
        if (T.empty()) continue;
        long long i = 0;
        double w = 0.0;
        if (t <= T.front() || T.size() == 1) i = 0;
        else if (t >= T.back()) i = (long long)T.size() - 1;
        else {
            i = (long long)(std::upper_bound(T.begin(), T.end(), t) - T.begin()) - 1;
            w = (t - T[i]) / (T[i + 1] - T[i]);
        }
        r.k[e] = i;
        r.w[e] = w;
    }
    return r;
}

// Model time of the state after `step` steps, and the end of the shortest record.
static double bnd_time(const cliffs_grid* g, long long step) { return g->t_start + (double)step * g->cfg.dt; }
static double bnd_end(const cliffs_grid* g) {
    double t_end = 1e300;
    for (int e = 0; e < 4; ++e)
        if (!g->bnd_t[e].empty()) t_end = std::min(t_end, g->bnd_t[e].back());
    return t_end;
}
static bool bnd_stops(const cliffs_grid* g, double t, double t_end) {
    return g->bnd_stop && t + g->cfg.dt > t_end * (1.0 + 1e-12) + 1e-9 * g->cfg.dt;
}

int impose_boundary(cliffs_grid* g, float* eta, float* u, float* v, double t) {
    BndStep b{};
    int npmax = 0;
    const BndRow r = bnd_row(g, t);
    for (int e = 0; e < 4; ++e) {
        if (g->bnd_t[e].empty()) continue;
        b.vals[e] = g->bnd_v[e];
        b.np[e] = e < 2 ? g->ny : g->nx;
        b.k[e] = r.k[e];
        b.w[e] = r.w[e];
        npmax = std::max(npmax, b.np[e]);
    }
    k_bnd<<<dim3((npmax + 127) / 128, 4), 128, 0, g->stream>>>(eta, u, v, g->pitch, g->nx, g->ny, b);
    CK(cudaGetLastError());
    return CLIFFS_OK;
}

// edges with boundary input as a mask (1 W, 2 E, 4 S, 8 N)
int input_edges(const cliffs_grid* g) {
    int m = 0;
    for (int e = 0; e < 4; ++e)
        if (!g->bnd_t[e].empty()) m |= 1 << e;
    return m;
}

void free_grid(cliffs_grid* g) {
    for (int k = 0; k < 2; ++k) { cudaFree(g->eta[k]); cudaFree(g->u[k]); cudaFree(g->v[k]); }
    cudaFree(g->d32); cudaFree(g->d64); cudaFree(g->d64b);
    cudaFree(g->emax); cudaFree(g->smax);
    cudaFree(g->xa); cudaFree(g->xb); cudaFree(g->xk); cudaFree(g->xrow); cudaFree(g->ymet);
    cudaFree(g->err); cudaFree(g->limit); cudaFree(g->items_d); cudaFree(g->items_dev);
    cudaFree(g->samp_ptr); cudaFree(g->samp); cudaFree(g->grec); cudaFree(g->nrec);
    cudaFree(g->pt_slot); cudaFree(g->pt_w); cudaFree(g->tmp); cudaFree(g->ured);
    cudaFree(g->order_d); cudaFree(g->nact_d); cudaFree(g->ctl_d);
    if (g->ctl_h) cudaFreeHost(g->ctl_h);
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    cudaFree(g->adj_slots); cudaFree(g->adj_ckpt); cudaFree(g->adj_t); cudaFree(g->adj_lb);
    cudaFree(g->adj_gxy); cudaFree(g->adj_seed); cudaFree(g->adj_items_dev); cudaFree(g->adj_pp);
    for (int e = 0; e < 4; ++e) cudaFree(g->bnd_v[e]);
    cudaFree(g->bnd_rows);
    cudaFree(g->rec_ckpt);
    cudaFree(g->adj_alt);
    if (g->cap) cudaStreamDestroy(g->cap);
    for (auto& e : g->ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    delete g;
}

int collect_timing(cliffs_grid* g) {
    if (g->ev.empty()) return CLIFFS_OK;
    CK(cudaEventSynchronize(g->ev.back().second));
    for (auto& e : g->ev) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e.first, e.second));
        g->t_ms += ms;
        ++g->t_launches;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    g->ev.clear();
    return CLIFFS_OK;
}

}  // namespace

// ============================================================================ C ABI
extern "C" {

const char* cliffs_last_error(void) { return g_err; }

int cliffs_abi_version(void) { return 2; }

int cliffs_grid_create(const cliffs_config* cfg, cliffs_grid** out) {
    g_err[0] = 0;
    if (!cfg || !out) return set_err(CLIFFS_ERR_ARG, "null argument");
    *out = nullptr;
    const int nx = cfg->nx, ny = cfg->ny;
    if (nx < 1 || ny < 1 || (nx == 1 && ny == 1))
        return set_err(CLIFFS_ERR_ARG, "grid %d x %d: need nx, ny >= 1 and not both 1", nx, ny);
    if ((nx > 1 && nx < 3) || (ny > 1 && ny < 3))
        return set_err(CLIFFS_ERR_ARG, "a 2D grid needs at least 3 nodes in each direction");
    if (cfg->batch < 1) return set_err(CLIFFS_ERR_ARG, "batch must be >= 1");
    if (!(cfg->h_min > 0.0)) return set_err(CLIFFS_ERR_ARG, "h_min must be > 0");
    if (!(cfg->dt > 0.0)) return set_err(CLIFFS_ERR_ARG, "dt must be > 0");
    if (cfg->manning_n2 < 0.0) return set_err(CLIFFS_ERR_ARG, "manning_n2 must be >= 0");
    if (cfg->maxout < 1 || cfg->gout < 1 || cfg->bndout < 1)
        return set_err(CLIFFS_ERR_ARG, "maxout, gout and bndout must be >= 1");
    if (!(cfg->solver == 0 || cfg->solver == 1 || cfg->solver == 2))
        return set_err(CLIFFS_ERR_ARG, "solver must be 1 or 2 (0 means 2)");
    if (cfg->open_edges < 0 || cfg->open_edges > 15)
        return set_err(CLIFFS_ERR_ARG, "open_edges is a mask of W 1, E 2, S 4, N 8");
    if (cfg->alternate != 0 && cfg->alternate != 1) return set_err(CLIFFS_ERR_ARG, "alternate must be 0 or 1");
    if (cfg->n_gauges < 0 || (cfg->n_gauges > 0 && !cfg->gauge_ixiy))
        return set_err(CLIFFS_ERR_ARG, "bad gauge list");
    for (int k = 0; k < cfg->n_gauges; ++k) {
        const int ix = cfg->gauge_ixiy[2 * k], iy = cfg->gauge_ixiy[2 * k + 1];
        if (ix < 0 || ix >= nx || iy < 0 || iy >= ny)
            return set_err(CLIFFS_ERR_ARG, "gauge %d at (%d, %d) is outside the %d x %d grid", k, ix, iy, nx, ny);
    }
    if (cfg->n_nests < 0 || (cfg->n_nests > 0 && !cfg->nests))
        return set_err(CLIFFS_ERR_ARG, "bad nest list");
    if (cfg->n_nests > 0 && (nx < 3 || ny < 3))
        return set_err(CLIFFS_ERR_ARG, "enclosed grids need a 2D master grid");
    if (cfg->n_nests > 0 && cfg->batch != 1)
        return set_err(CLIFFS_ERR_ARG, "enclosed grids need batch == 1");
    for (int m = 0; m < cfg->n_nests; ++m)
        if (cfg->nests[m].nx < 2 || cfg->nests[m].ny < 2 || !(cfg->nests[m].dx > 0) || !(cfg->nests[m].dy > 0))
            return set_err(CLIFFS_ERR_ARG, "nest %d: need nx, ny >= 2 and dx, dy > 0", m);

    cliffs_grid* g = new cliffs_grid();
    g->cfg = *cfg;
    g->gauges.assign(cfg->gauge_ixiy, cfg->gauge_ixiy + 2 * cfg->n_gauges);
    g->nests.assign(cfg->nests, cfg->nests + cfg->n_nests);
    g->cfg.gauge_ixiy = nullptr;
    g->cfg.nests = nullptr;
    g->nx = nx; g->ny = ny; g->B = cfg->batch;
    g->pitch = (nx + 31) / 32 * 32;
    g->plane = (long long)g->pitch * ny;
    g->stream = (cudaStream_t)cfg->stream;
    g->G = cfg->n_gauges;
    auto fail = [&](int rc) { free_grid(g); return rc; };
    const size_t sb = sizeof(float) * (size_t)g->B * g->plane;
#define CKG(call) do { int rc_ = [&]() -> int { CK(call); return CLIFFS_OK; }(); if (rc_) return fail(rc_); } while (0)
    for (int k = 0; k < 2; ++k) {
        CKG(cudaMalloc(&g->eta[k], sb)); CKG(cudaMalloc(&g->u[k], sb)); CKG(cudaMalloc(&g->v[k], sb));
        CKG(cudaMemsetAsync(g->eta[k], 0, sb, g->stream));
        CKG(cudaMemsetAsync(g->u[k], 0, sb, g->stream));
        CKG(cudaMemsetAsync(g->v[k], 0, sb, g->stream));
    }
    CKG(cudaMalloc(&g->emax, sb)); CKG(cudaMalloc(&g->smax, sb));
    CKG(cudaMalloc(&g->d32, sizeof(float) * g->plane));
    CKG(cudaMalloc(&g->d64, sizeof(double) * (size_t)nx * ny));
    CKG(cudaMalloc(&g->d64b, sizeof(double) * (size_t)nx * ny));
    CKG(cudaMalloc(&g->xa, sizeof(float) * nx)); CKG(cudaMalloc(&g->xb, sizeof(float) * nx));
    CKG(cudaMalloc(&g->xk, sizeof(float) * nx)); CKG(cudaMalloc(&g->xrow, sizeof(float) * (ny + 2 * MET_PAD)));
    CKG(cudaMalloc(&g->ymet, sizeof(float4) * (ny + 2 * MET_PAD)));
    CKG(cudaMalloc(&g->err, sizeof(int) * 4));
    CKG(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, g->stream));
    CKG(cudaMalloc(&g->ured, sizeof(unsigned) * 4));
    CKG(cudaStreamSynchronize(g->stream));
#undef CKG
    if (nx >= 3 && ny >= 3) {
        int rc = make_maps(g);
        if (rc) { free_grid(g); return rc; }
    }
    *out = g;
    return CLIFFS_OK;
}

int cliffs_set_bathy(cliffs_grid* g, const double* x, const double* y, const double* depth,
                     int apply_filter, double alpha, double min_depth) {
    g_err[0] = 0;
    if (!g || !x || !y || !depth) return set_err(CLIFFS_ERR_ARG, "null argument");
    const int nx = g->nx, ny = g->ny;
    std::vector<double> hx(nx), hy(ny);
    CK(cudaMemcpy(hx.data(), x, sizeof(double) * nx, cudaMemcpyDefault));
    CK(cudaMemcpy(hy.data(), y, sizeof(double) * ny, cudaMemcpyDefault));
    g->hx = hx;
    g->hy = hy;
    for (int i = 0; i + 1 < nx; ++i)
        if (!(hx[i + 1] > hx[i])) return set_err(CLIFFS_ERR_ARG, "x must be strictly increasing (index %d)", i);
    for (int j = 0; j + 1 < ny; ++j)
        if (!(hy[j + 1] > hy[j])) return set_err(CLIFFS_ERR_ARG, "y must be strictly increasing (index %d)", j);
    const bool sph = g->cfg.coords != 1;
    if (sph)
        for (int j = 0; j < ny; ++j)
            if (!(std::fabs(hy[j]) < 90.0)) return set_err(CLIFFS_ERR_ARG, "latitude %g out of (-90, 90)", hy[j]);
    if (apply_filter && !(alpha > 1.0 && alpha < 3.0))
        return set_err(CLIFFS_ERR_ARG, "filter limit alpha must be in (1, 3)");
    const long long N = (long long)nx * ny;
    cudaStream_t s = g->stream;
    CK(cudaMemcpyAsync(g->d64, depth, sizeof(double) * N, cudaMemcpyDefault, s));
    if (apply_filter) {
        k_filter_minraise<<<nblk(N), 256, 0, s>>>(g->d64, N, min_depth);
        CK(cudaGetLastError());
        int* changed = reinterpret_cast<int*>(g->ured);
        const double a2 = alpha * alpha;
        bool conv = false;
        for (int pass = 1; pass <= 100; ++pass) {
            CK(cudaMemsetAsync(changed, 0, sizeof(int), s));
            k_filter_pass<<<nblk(N), 256, 0, s>>>(g->d64, g->d64b, nx, ny, 0, a2, changed);
            k_filter_pass<<<nblk(N), 256, 0, s>>>(g->d64b, g->d64, nx, ny, 1, a2, changed);
            CK(cudaGetLastError());
            int h = 0;
            CK(cudaMemcpyAsync(&h, changed, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            if (!h) { conv = true; break; }
        }
        if (!conv) fprintf(stderr, "cliffs: depth filter stopped after 100 passes\n");
    }
    // metric tables (section "Running Options", "Units": metres, or degrees on a sphere)
    std::vector<float> xa(nx, 0.f), xb(nx, 0.f), xk(nx, 0.f), xrow(ny, 1.f);
    std::vector<float4> ym(ny, make_float4(0.f, 0.f, 0.f, 0.f));
    const double dt = g->cfg.dt;
    if (nx > 1) {
        const double f = sph ? DEGR : 1.0;
        for (int c = 0; c < nx; ++c) {
            const double l = f * ((c > 0) ? hx[c] - hx[c - 1] : hx[1] - hx[0]);
            const double r = f * ((c < nx - 1) ? hx[c + 1] - hx[c] : hx[nx - 1] - hx[nx - 2]);
            xa[c] = (float)(1.0 / l); xb[c] = (float)(1.0 / r); xk[c] = (float)(dt * dt / (l + r));
        }
        if (sph) for (int j = 0; j < ny; ++j) xrow[j] = (float)(1.0 / (R_SPHERE * std::cos(hy[j] * DEGR)));
    }
    if (ny > 1) {
        const double f = sph ? R_SPHERE * DEGR : 1.0;
        for (int j = 0; j < ny; ++j) {
            const double l = f * ((j > 0) ? hy[j] - hy[j - 1] : hy[1] - hy[0]);
            const double r = f * ((j < ny - 1) ? hy[j + 1] - hy[j] : hy[ny - 1] - hy[ny - 2]);
            const double src = sph ? dt * std::tan(hy[j] * DEGR) / R_SPHERE : 0.0;
            ym[j] = make_float4((float)(1.0 / l), (float)(1.0 / r), (float)(dt * dt / (l + r)), (float)src);
        }
    }
    CK(cudaMemcpyAsync(g->xa, xa.data(), sizeof(float) * nx, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(g->xb, xb.data(), sizeof(float) * nx, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(g->xk, xk.data(), sizeof(float) * nx, cudaMemcpyHostToDevice, s));
    // row tables padded by MET_PAD rows on each side (edge rows repeated), so that the
    // kernels index them without clamping
    std::vector<float> xrow_p(ny + 2 * MET_PAD);
    std::vector<float4> ym_p(ny + 2 * MET_PAD);
    for (int j = 0; j < ny + 2 * MET_PAD; ++j) {
        const int jj = std::min(std::max(j - MET_PAD, 0), ny - 1);
        xrow_p[j] = xrow[jj];
        ym_p[j] = ym[jj];
    }
    CK(cudaMemcpyAsync(g->xrow, xrow_p.data(), sizeof(float) * xrow_p.size(), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(g->ymet, ym_p.data(), sizeof(float4) * ym_p.size(), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    k_depth_to_f32<<<nblk((long long)ny * g->pitch), 256, 0, s>>>(g->d64, g->d32, nx, ny, g->pitch);
    CK(cudaGetLastError());
    // CFL (section "Difference Scheme": |lambda| dt / dx <= 1)
    CK(cudaMemsetAsync(g->ured + 1, 0, sizeof(unsigned), s));
    k_cfl<<<nblk(N), 256, 0, s>>>(g->d64, nx, ny, g->xa, g->xb, g->xrow + MET_PAD, g->ymet + MET_PAD, dt, g->ured + 1);
    CK(cudaGetLastError());
    unsigned cb = 0;
    CK(cudaMemcpyAsync(&cb, g->ured + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    float cour;
    std::memcpy(&cour, &cb, sizeof(float));
    if (cour > 1.0f + 1e-6f)
        return set_err(CLIFFS_ERR_ARG, "Courant number %.4f > 1: reduce dt (section Difference Scheme)", cour);
    // samples: gauges, then the corner nodes of every enclosed-grid boundary point
    g->samples.clear();
    for (int k = 0; k < g->G; ++k) g->samples.push_back(make_int4(g->gauges[2 * k + 1], g->gauges[2 * k], 0, k));
    std::map<long long, int> slot_of;
    std::vector<int> pslot;
    std::vector<double> pw;
    g->edge_off.clear(); g->edge_np.clear();
    int npts = 0;
    for (size_t m = 0; m < g->nests.size(); ++m) {
        const cliffs_nest& n = g->nests[m];
        for (int e = 0; e < 4; ++e) {
            const int np = (e < 2) ? n.ny : n.nx;
            g->edge_off.push_back(npts);
            g->edge_np.push_back(np);
            for (int k = 0; k < np; ++k) {
                double px, py;
                if (e == 0) { px = n.x0; py = n.y0 + k * n.dy; }
                else if (e == 1) { px = n.x0 + (n.nx - 1) * n.dx; py = n.y0 + k * n.dy; }
                else if (e == 2) { px = n.x0 + k * n.dx; py = n.y0; }
                else { px = n.x0 + k * n.dx; py = n.y0 + (n.ny - 1) * n.dy; }
                int i, j; double a, b;
                if (!locate(hx, px, &i, &a) || !locate(hy, py, &j, &b))
                    return set_err(CLIFFS_ERR_ARG, "nest %d: boundary point (%g, %g) outside the master grid", (int)m, px, py);
                const int cc[4][2] = {{j, i}, {j, i + 1}, {j + 1, i}, {j + 1, i + 1}};
                const double ww[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
                for (int q = 0; q < 4; ++q) {
                    const long long key = (long long)cc[q][0] * nx + cc[q][1];
                    auto it = slot_of.find(key);
                    int sl;
                    if (it == slot_of.end()) {
                        sl = (int)slot_of.size();
                        slot_of[key] = sl;
                        g->samples.push_back(make_int4(cc[q][0], cc[q][1], 1, sl));
                    } else {
                        sl = it->second;
                    }
                    pslot.push_back(sl);
                    pw.push_back(ww[q]);
                }
                ++npts;
            }
        }
    }
    g->NN = (int)slot_of.size();
    cudaFree(g->pt_slot); cudaFree(g->pt_w); cudaFree(g->items_d);
    g->pt_slot = nullptr; g->pt_w = nullptr; g->items_d = nullptr;
    if (npts) {
        CK(cudaMalloc(&g->pt_slot, sizeof(int) * pslot.size()));
        CK(cudaMalloc(&g->pt_w, sizeof(double) * pw.size()));
        CK(cudaMemcpy(g->pt_slot, pslot.data(), sizeof(int) * pslot.size(), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(g->pt_w, pw.data(), sizeof(double) * pw.size(), cudaMemcpyHostToDevice));
    }
    if (!g->samples.empty()) {
        CK(cudaMalloc(&g->items_d, sizeof(int4) * g->samples.size()));
        CK(cudaMemcpy(g->items_d, g->samples.data(), sizeof(int4) * g->samples.size(), cudaMemcpyHostToDevice));
    }
    if (nx >= 3 && ny >= 3) {
        // strips whose 64-column window holds a node that is dry at rest (d < h_min), or
        // reaches the domain edge
        std::vector<double> hd((size_t)nx * ny);
        CK(cudaMemcpy(hd.data(), g->d64, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost));
        const int nstrips = fused_strips(nx);
        g->hard.assign(nstrips, 0);
        for (int st = 0; st < nstrips; ++st) {
            const int c0 = st * XOUT, c1 = c0 + XWIN;
            if (c0 == 0 || c1 >= nx) { g->hard[st] = 1; continue; }
            for (int j = 0; j < ny && !g->hard[st]; ++j)
                for (int c = c0; c < c1; ++c)
                    if (hd[(size_t)j * nx + c] < g->cfg.h_min) { g->hard[st] = 1; break; }
        }
    }
    int rc = choose_geometry(g);
    if (rc) return rc;
    g->have_bathy = true;
    g->have_init = false;
    return CLIFFS_OK;
}

int cliffs_read_depth(cliffs_grid* g, double* depth) {
    g_err[0] = 0;
    if (!g || !depth) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_bathy) return set_err(CLIFFS_ERR_STATE, "set_bathy first");
    CK(cudaMemcpyAsync(depth, g->d64, sizeof(double) * g->nx * g->ny, cudaMemcpyDefault, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return CLIFFS_OK;
}

int cliffs_set_initial(cliffs_grid* g, int scenario, const float* eta, const float* u,
                       const float* v, int quake) {
    g_err[0] = 0;
    if (!g || !eta) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_bathy) return set_err(CLIFFS_ERR_STATE, "set_bathy first");
    if (scenario < -1 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d out of range", scenario);
    if (quake && g->B != 1) return set_err(CLIFFS_ERR_ARG, "quake needs batch == 1");
    cudaStream_t s = g->stream;
    const int nx = g->nx, ny = g->ny;
    const size_t rowb = sizeof(float) * nx, pitchb = sizeof(float) * g->pitch;
    // scenarios not set now keep their state: move it into buffer 0
    if (g->step > 0 && scenario >= 0) {
        for (int b = 0; b < g->B; ++b) {
            if (b == scenario || cur_buf(g, b) == 0) continue;
            const size_t o = (size_t)b * g->plane * sizeof(float);
            CK(cudaMemcpyAsync((char*)g->eta[0] + o, (char*)g->eta[1] + o, g->plane * sizeof(float), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync((char*)g->u[0] + o, (char*)g->u[1] + o, g->plane * sizeof(float), cudaMemcpyDeviceToDevice, s));
            CK(cudaMemcpyAsync((char*)g->v[0] + o, (char*)g->v[1] + o, g->plane * sizeof(float), cudaMemcpyDeviceToDevice, s));
        }
    }
    const int b0 = scenario < 0 ? 0 : scenario, nb = scenario < 0 ? g->B : 1;
    const size_t off = (size_t)b0 * g->plane;
    const size_t rows = (size_t)nb * ny;
    if (quake) {
        int rc = ensure_tmp(g, sizeof(float) * (size_t)nx * ny);
        if (rc) return rc;
        CK(cudaMemcpyAsync(g->tmp, eta, sizeof(float) * (size_t)nx * ny, cudaMemcpyDefault, s));
        const double dwall = g->cfg.itopo ? -1e300 : g->cfg.dwall;
        k_quake<<<nblk((long long)nx * ny), 256, 0, s>>>(g->d64, (const float*)g->tmp, g->eta[0], g->d32, nx, ny,
                                                        g->pitch, g->cfg.h_min, dwall);
        CK(cudaGetLastError());
    } else {
        CK(cudaMemcpy2DAsync(g->eta[0] + off, pitchb, eta, rowb, rowb, rows, cudaMemcpyDefault, s));
    }
    if (u) CK(cudaMemcpy2DAsync(g->u[0] + off, pitchb, u, rowb, rowb, rows, cudaMemcpyDefault, s));
    else CK(cudaMemsetAsync(g->u[0] + off, 0, sizeof(float) * nb * g->plane, s));
    if (v) CK(cudaMemcpy2DAsync(g->v[0] + off, pitchb, v, rowb, rowb, rows, cudaMemcpyDefault, s));
    else CK(cudaMemsetAsync(g->v[0] + off, 0, sizeof(float) * nb * g->plane, s));
    g->step = 0;
    const float dwall = g->cfg.itopo ? -3.402823466e38f : (float)g->cfg.dwall;
    k_max_init<<<nblk((long long)nb * g->plane), 256, 0, s>>>(g->eta[0], g->u[0], g->v[0], g->d32, g->emax, g->smax,
                                                             nx, ny, g->pitch, g->plane, b0, nb,
                                                             (float)g->cfg.h_min, dwall);
    CK(cudaGetLastError());
    int rc = grow_records(g, 1, 1);
    if (rc) return rc;
    if (!g->samples.empty()) {
        const int ni = (int)g->samples.size();
        k_record0<<<nblk((long long)ni * nb), 256, 0, s>>>(g->eta[0], g->u[0], g->v[0], g->pitch, g->plane,
                                                          g->items_d, ni, g->grec, g->grec_cap * g->G * 3,
                                                          g->nrec, b0, nb);
        CK(cudaGetLastError());
    }
    if (quake) {
        // the deformed depth must still satisfy the CFL limit
        CK(cudaMemsetAsync(g->ured + 1, 0, sizeof(unsigned), s));
        k_cfl<<<nblk((long long)nx * ny), 256, 0, s>>>(g->d64, nx, ny, g->xa, g->xb, g->xrow + MET_PAD, g->ymet + MET_PAD, g->cfg.dt, g->ured + 1);
        unsigned cb = 0;
        CK(cudaMemcpyAsync(&cb, g->ured + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        float cour;
        std::memcpy(&cour, &cb, sizeof(float));
        if (cour > 1.0f + 1e-6f) return set_err(CLIFFS_ERR_ARG, "Courant number %.4f > 1 after deformation", cour);
    }
    g->rec_n = 0;
    if (g->rec_K > 0) {
        rc = record_checkpoint(g, 0);
        if (rc) return rc;
    }
    CK(cudaStreamSynchronize(s));
    g->have_init = true;
    return CLIFFS_OK;
}

int cliffs_set_initial_interp(cliffs_grid* g, int scenario, const double* sx, int32_t snx, const double* sy,
                              int32_t sny, const float* eta, const float* u, const float* v, int quake) {
    g_err[0] = 0;
    if (!g || !sx || !sy || !eta) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_bathy) return set_err(CLIFFS_ERR_STATE, "set_bathy first");
    if (snx < 1 || sny < 1) return set_err(CLIFFS_ERR_ARG, "empty source grid");
    if (scenario < 0 && g->B != 1) return set_err(CLIFFS_ERR_ARG, "interpolate one scenario at a time");
    std::vector<double> hsx(snx), hsy(sny);
    CK(cudaMemcpy(hsx.data(), sx, sizeof(double) * snx, cudaMemcpyDefault));
    CK(cudaMemcpy(hsy.data(), sy, sizeof(double) * sny, cudaMemcpyDefault));
    for (int i = 0; i + 1 < snx; ++i)
        if (!(hsx[i + 1] > hsx[i])) return set_err(CLIFFS_ERR_ARG, "source x must increase");
    for (int j = 0; j + 1 < sny; ++j)
        if (!(hsy[j + 1] > hsy[j])) return set_err(CLIFFS_ERR_ARG, "source y must increase");
    const int nx = g->nx, ny = g->ny;
    std::vector<Ax> col(nx), row(ny);
    for (int c = 0; c < nx; ++c) {
        int i; double a;
        col[c] = locate(hsx, g->hx[c], &i, &a) ? Ax{i, a} : Ax{-1, 0.0};
    }
    for (int r = 0; r < ny; ++r) {
        int j; double b;
        row[r] = locate(hsy, g->hy[r], &j, &b) ? Ax{j, b} : Ax{-1, 0.0};
    }
    const size_t N = (size_t)nx * ny, S = (size_t)snx * sny;
    int rc = ensure_tmp(g, sizeof(float) * (3 * N + S) + sizeof(Ax) * (nx + ny) + 256);
    if (rc) return rc;
    float* out = (float*)g->tmp;
    float* src = out + 3 * N;
    Ax* dcol = reinterpret_cast<Ax*>(reinterpret_cast<char*>(g->tmp) + ((sizeof(float) * (3 * N + S) + 15) & ~size_t(15)));
    Ax* drow = dcol + nx;
    cudaStream_t s = g->stream;
    CK(cudaMemcpyAsync(dcol, col.data(), sizeof(Ax) * nx, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(drow, row.data(), sizeof(Ax) * ny, cudaMemcpyHostToDevice, s));
    const float* fields[3] = {eta, u, v};
    for (int f = 0; f < 3; ++f) {
        if (!fields[f]) continue;
        CK(cudaMemcpyAsync(src, fields[f], sizeof(float) * S, cudaMemcpyDefault, s));
        k_interp<<<nblk((long long)N), 256, 0, s>>>(src, snx, dcol, drow, nx, ny, out + f * N);
        CK(cudaGetLastError());
    }
    CK(cudaStreamSynchronize(s));
    // the interpolated fields are copied out of the scratch by set_initial (which may reuse it)
    std::vector<float> h(3 * N);
    CK(cudaMemcpy(h.data(), out, sizeof(float) * 3 * N, cudaMemcpyDeviceToHost));
    return cliffs_set_initial(g, scenario < 0 ? -1 : scenario, h.data(), u ? h.data() + N : nullptr,
                              v ? h.data() + 2 * N : nullptr, quake);
}

int cliffs_set_durations(cliffs_grid* g, const int64_t* steps) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    cudaFree(g->order_d); cudaFree(g->nact_d);
    g->order_d = g->nact_d = nullptr;
    g->nact_len = 0;
    if (!steps) {
        g->limit_h.clear();
        cudaFree(g->limit);
        g->limit = nullptr;
        return CLIFFS_OK;
    }
    std::vector<long long> h(g->B);
    CK(cudaMemcpy(h.data(), steps, sizeof(long long) * g->B, cudaMemcpyDefault));
    for (int b = 0; b < g->B; ++b)
        if (h[b] < 0) return set_err(CLIFFS_ERR_ARG, "negative duration for scenario %d", b);
    if (!g->limit) CK(cudaMalloc(&g->limit, sizeof(long long) * g->B));
    CK(cudaMemcpy(g->limit, h.data(), sizeof(long long) * g->B, cudaMemcpyHostToDevice));
    g->limit_h = h;
    // for the persistent run: scenarios by decreasing duration (ties by index), and for each
    // step s the number of scenarios still running there (limit >= s)
    std::vector<int> order(g->B);
    for (int b = 0; b < g->B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return h[p] > h[q]; });
    const long long L = h[order[0]] + 1;
    std::vector<int> nact(L, 0);
    for (int b = 0; b < g->B; ++b) nact[h[b]] += 1;          // scenarios ending at exactly s
    for (long long t = L - 2; t >= 0; --t) nact[t] += nact[t + 1];
    CK(cudaMalloc(&g->order_d, sizeof(int) * g->B));
    CK(cudaMalloc(&g->nact_d, sizeof(int) * L));
    CK(cudaMemcpy(g->order_d, order.data(), sizeof(int) * g->B, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(g->nact_d, nact.data(), sizeof(int) * L, cudaMemcpyHostToDevice));
    g->nact_len = L;
    return CLIFFS_OK;
}

int cliffs_set_boundary_input(cliffs_grid* g, int edge, const double* times, int64_t nt, const double* vals) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (edge < 0 || edge > 3) return set_err(CLIFFS_ERR_ARG, "edge %d out of range (0 W, 1 E, 2 S, 3 N)", edge);
    if (g->B != 1) return set_err(CLIFFS_ERR_ARG, "boundary input needs batch == 1");
    if ((g->ny == 1 && edge >= 2) || (g->nx == 1 && edge < 2))
        return set_err(CLIFFS_ERR_ARG, "edge %d runs along the 1D grid", edge);
    if (nt < 0 || (nt > 0 && (!times || !vals))) return set_err(CLIFFS_ERR_ARG, "bad series");
    cudaFree(g->bnd_v[edge]);
    g->bnd_v[edge] = nullptr;
    g->bnd_t[edge].clear();
    if (nt > 0) {
        std::vector<double> t(nt);
        CK(cudaMemcpy(t.data(), times, sizeof(double) * nt, cudaMemcpyDefault));
        for (int64_t i = 0; i + 1 < nt; ++i)
            if (!(t[i + 1] > t[i])) return set_err(CLIFFS_ERR_ARG, "record times must increase");
        const int np = edge < 2 ? g->ny : g->nx;
        CK(cudaMalloc(&g->bnd_v[edge], sizeof(double) * 3 * np * nt));
        CK(cudaMemcpy(g->bnd_v[edge], vals, sizeof(double) * 3 * np * nt, cudaMemcpyDefault));
        g->bnd_t[edge] = t;
    }
    g->bnd_any = false;
    for (int e = 0; e < 4; ++e) g->bnd_any |= !g->bnd_t[e].empty();
    return CLIFFS_OK;
}

int cliffs_set_boundary_clock(cliffs_grid* g, double cuke, int stop_at_end, double* t_start) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->bnd_any) return set_err(CLIFFS_ERR_STATE, "no boundary input");
    double t0 = 1e300, tc = 1e300;
    for (int e = 0; e < 4; ++e) {
        const std::vector<double>& T = g->bnd_t[e];
        if (T.empty()) continue;
        t0 = std::min(t0, T.front());
        if (cuke > 0.0) {
            const int np = e < 2 ? g->ny : g->nx;
            std::vector<double> h((size_t)3 * np * T.size());
            CK(cudaMemcpy(h.data(), g->bnd_v[e], sizeof(double) * h.size(), cudaMemcpyDeviceToHost));
            for (size_t r = 0; r < T.size() && T[r] < tc; ++r)
                for (int q = 0; q < np; ++q)
                    if (std::fabs(h[(r * 3 + 2) * np + q]) > cuke) { tc = T[r]; break; }
        }
    }
    g->t_start = (cuke > 0.0 && tc < 1e300) ? tc : t0;
    g->bnd_stop = stop_at_end != 0;
    if (t_start) *t_start = g->t_start;
    return CLIFFS_OK;
}

int cliffs_step_n(cliffs_grid* g, int64_t n) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    if (n < 0) return set_err(CLIFFS_ERR_ARG, "negative step count");
    if (n == 0) return CLIFFS_OK;
    const long long last = g->step + n;
    int rc = grow_records(g, last / g->cfg.gout + 1, last / g->cfg.bndout + 1);
    if (rc) return rc;
    cudaStream_t s = g->stream;
    StepArgs a;
    const double t_end = g->bnd_any ? bnd_end(g) : 1e300;
    for (long long k = 0; k < n; ++k) {
        const long long st = g->step + 1;
        const int in = (int)(g->step & 1), out = 1 - in;
        if (g->bnd_any) {
            const double t = bnd_time(g, g->step);
            if (bnd_stops(g, t, t_end)) break;
            rc = impose_boundary(g, g->eta[in], g->u[in], g->v[in], t);
            if (rc) return rc;
        }
        fill_step_args(g, a, in, out);
        a.step = st;
        a.yfirst = g->cfg.alternate && ((st - 1) & 1);       // odd steps sweep y first
        if (st % g->cfg.maxout == 0) { a.emax = g->emax; a.smax = g->smax; }
        if (g->G && st % g->cfg.gout == 0) a.rec_g = g->grec + (st / g->cfg.gout) * g->G * 3;
        if (g->NN && st % g->cfg.bndout == 0) a.rec_n = g->nrec + (st / g->cfg.bndout) * g->NN * 3;
        if (g->inject_cycles > 0) {
            // fault injection: every ring slot of this launch waits for bytes that never come
            a.wait_cycles = g->inject_cycles;
            a.tx_pad = 16;
            g->inject_cycles = 0;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (g->timing) {
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventRecord(e0, s));
        }
        cudaError_t le;
        if (g->kind == 0) le = launch_step_fused(a, g->maps[in], g->B, s);
        else if (g->kind == 1) le = launch_xsweep(a, g->B, s);
        else le = launch_ysweep(a, g->B, s);
        if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "sweep launch: %s", cudaGetErrorString(le));
        if (g->timing) {
            CK(cudaEventRecord(e1, s));
            g->ev.emplace_back(e0, e1);
            if (g->ev.size() >= 4096) { rc = collect_timing(g); if (rc) return rc; }
        }
        g->step = st;
        if (g->rec_K > 0) {
            g->rec_n = st;
            if (st % g->rec_K == 0) {
                rc = record_checkpoint(g, st / g->rec_K);
                if (rc) return rc;
            }
        }
    }
    int h[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, g->err, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[0]) {
        CK(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, s));
        if (h[0] & ERRF_TIMEOUT) return set_err(CLIFFS_ERR_TIMEOUT, "a bounded device wait gave up");
        return set_err(CLIFFS_ERR_UNSTABLE, "non-finite or runaway state before step %lld", (long long)g->step);
    }
    return CLIFFS_OK;
}

int cliffs_run_persistent(cliffs_grid* g, int64_t n) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    if (n < 0) return set_err(CLIFFS_ERR_ARG, "negative step count");
    if (g->kind != 0) return set_err(CLIFFS_ERR_ARG, "the persistent run needs a 2D grid");
    if (g->rec_K > 0) return set_err(CLIFFS_ERR_ARG, "a recorded run goes through cliffs_step_n");
    if (g->bnd_any) {                             // the steps cliffs_step_n would take
        const double t_end = bnd_end(g);
        long long m = 0;
        while (m < n && !bnd_stops(g, bnd_time(g, g->step + m), t_end)) ++m;
        n = m;
    }
    if (n == 0) return CLIFFS_OK;
    const long long last = g->step + n;
    int rc = grow_records(g, last / g->cfg.gout + 1, last / g->cfg.bndout + 1);
    if (rc) return rc;
    cudaStream_t s = g->stream;
    if (!g->ctl_d) {
        CK(cudaMalloc(&g->ctl_d, 4 * sizeof(long long)));
        CK(cudaMallocHost(&g->ctl_h, 4 * sizeof(long long)));
        CK(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
        int dev = 0, sms = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        g->pblocks = sms * std::max(1, batch_blocks_per_sm(g->cfg.coords != 1));
    }
    // launch arguments; all padding zeroed so that they compare byte for byte
    struct Key { StepArgs a; BatchArgs b; } k;
    std::memset(&k, 0, sizeof(k));
    fill_step_args(g, k.a, 0, 1);
    k.a.eta_out = k.a.u_out = k.a.v_out = nullptr;
    k.a.eta_in = k.a.u_in = k.a.v_in = nullptr;
    k.a.limit = nullptr;
    if (g->inject_cycles > 0) {
        // fault injection: every ring slot of this run waits for bytes that never come
        k.a.wait_cycles = g->inject_cycles;
        k.a.tx_pad = 16;
        g->inject_cycles = 0;
    }
    BatchArgs& b = k.b;
    b.ctl = g->ctl_d;
    b.order = g->order_d;
    b.nact = g->nact_d;
    b.nact_len = g->nact_len;
    b.nall = g->B;
    for (int i = 0; i < 2; ++i) { b.eta[i] = g->eta[i]; b.u[i] = g->u[i]; b.v[i] = g->v[i]; }
    b.emax = g->emax; b.smax = g->smax;
    b.maxout = g->cfg.maxout; b.gout = g->cfg.gout; b.bndout = g->cfg.bndout;
    b.grec = g->G ? g->grec : nullptr;
    b.grec_row = (long long)g->G * 3;
    b.nrec = g->NN ? g->nrec : nullptr;
    b.nrec_row = (long long)g->NN * 3;
    b.alternate = g->cfg.alternate;
    if (g->bnd_any) {
        // the interpolation of every step of this run, computed as cliffs_step_n does
        if (g->bnd_rows_cap < n) {
            cudaFree(g->bnd_rows);
            g->bnd_rows = nullptr;
            const long long cap = std::max<long long>(n, 2 * g->bnd_rows_cap);
            CK(cudaMalloc(&g->bnd_rows, sizeof(BndRow) * cap));
            g->bnd_rows_cap = cap;
        }
        std::vector<BndRow> rows(n);
        for (long long j = 0; j < n; ++j) rows[j] = bnd_row(g, bnd_time(g, g->step + j));
        CK(cudaMemcpyAsync(g->bnd_rows, rows.data(), sizeof(BndRow) * n, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        b.bnd = 1;
        b.bnd_rows = g->bnd_rows;
        for (int e = 0; e < 4; ++e) {
            b.bv[e] = g->bnd_t[e].empty() ? nullptr : g->bnd_v[e];
            b.bnp[e] = e < 2 ? g->ny : g->nx;
        }
    }
    if (!b.order) {                               // no durations: every scenario, in index order
        std::vector<int> id(g->B);
        for (int i = 0; i < g->B; ++i) id[i] = i;
        CK(cudaMalloc(&g->order_d, sizeof(int) * g->B));
        CK(cudaMemcpy(g->order_d, id.data(), sizeof(int) * g->B, cudaMemcpyHostToDevice));
        b.order = g->order_d;
    }
    const unsigned char* kb = reinterpret_cast<const unsigned char*>(&k);
    if (!g->gexec || g->gkey.size() != sizeof(k) || std::memcmp(g->gkey.data(), kb, sizeof(k)) != 0) {
        if (g->gexec) { cudaGraphExecDestroy(g->gexec); g->gexec = nullptr; }
        // the graph: copy the control block in from its pinned host image, then the
        // cooperative launch
        StepMaps2 mm;
        mm.m[0] = g->maps[0];
        mm.m[1] = g->maps[1];
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
        cudaError_t e1 = cudaMemcpyAsync(g->ctl_d, g->ctl_h, 4 * sizeof(long long), cudaMemcpyHostToDevice, g->cap);
        cudaError_t e2 = e1 == cudaSuccess ? launch_batch(k.a, mm, b, g->pblocks, g->cap) : e1;
        cudaError_t e3 = cudaStreamEndCapture(g->cap, &graph);
        if (e2 != cudaSuccess || e3 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return set_err(CLIFFS_ERR_CUDA, "capturing the persistent run: %s",
                           cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
        }
        cudaError_t e4 = cudaGraphInstantiate(&g->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e4 != cudaSuccess) {
            g->gexec = nullptr;
            return set_err(CLIFFS_ERR_CUDA, "instantiating the persistent run: %s", cudaGetErrorString(e4));
        }
        g->gkey.assign(kb, kb + sizeof(k));
    }
    g->ctl_h[0] = g->step;
    g->ctl_h[1] = last;
    g->ctl_h[2] = 0;
    g->ctl_h[3] = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (g->timing) {
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventRecord(e0, s));
    }
    CK(cudaGraphLaunch(g->gexec, s));
    if (g->timing) {
        CK(cudaEventRecord(e1, s));
        g->ev.emplace_back(e0, e1);
    }
    g->step = last;
    int h[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, g->err, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));   // the pinned control block is free again after this
    if (h[0]) {
        CK(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, s));
        if (h[0] & ERRF_TIMEOUT) return set_err(CLIFFS_ERR_TIMEOUT, "a bounded device wait gave up");
        return set_err(CLIFFS_ERR_UNSTABLE, "non-finite or runaway state before step %lld", (long long)g->step);
    }
    return CLIFFS_OK;
}

static int adjoint_core(cliffs_grid* g, int scenario, int64_t n, int32_t checkpoint_every, const float* dL_dgauges,
                        float* dL_deta0, const float* recorded, int comps = 1);

int cliffs_adjoint_n(cliffs_grid* g, int64_t n, int32_t checkpoint_every, const float* dL_dgauges,
                     float* dL_deta0) {
    return adjoint_core(g, 0, n, checkpoint_every, dL_dgauges, dL_deta0, nullptr);
}

int cliffs_adjoint_scenario(cliffs_grid* g, int32_t scenario, int64_t n, int32_t checkpoint_every,
                            const float* dL_dgauges, float* dL_deta0) {
    return adjoint_core(g, scenario, n, checkpoint_every, dL_dgauges, dL_deta0, nullptr);
}

int cliffs_adjoint_record(cliffs_grid* g, int32_t checkpoint_every) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (checkpoint_every < 0) return set_err(CLIFFS_ERR_ARG, "checkpoint_every must be >= 0");
    if (checkpoint_every == 0) {
        cudaFree(g->rec_ckpt);
        cudaFree(g->adj_alt);
        g->adj_alt = nullptr;
        g->rec_ckpt = nullptr;
        g->rec_cap = 0;
        g->rec_K = 0;
        g->rec_n = 0;
        return CLIFFS_OK;
    }
    if (g->kind != 0) return set_err(CLIFFS_ERR_ARG, "the adjoint needs a 2D grid");
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    if (g->step != 0) return set_err(CLIFFS_ERR_STATE, "record from the initial state (no steps since set_initial)");
    g->rec_K = checkpoint_every;
    g->rec_n = 0;
    int rc = record_checkpoint(g, 0);
    if (rc) return rc;
    CK(cudaStreamSynchronize(g->stream));
    return CLIFFS_OK;
}

int cliffs_adjoint_recorded(cliffs_grid* g, const float* dL_dgauges, float* dL_deta0) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (g->rec_K <= 0 || g->rec_n < 1) return set_err(CLIFFS_ERR_STATE, "no recorded run");
    return adjoint_core(g, 0, g->rec_n, g->rec_K, dL_dgauges, dL_deta0, g->rec_ckpt);
}

int cliffs_adjoint_records(cliffs_grid* g, int32_t scenario, int64_t n, int32_t checkpoint_every,
                           const float* dL_drecords, float* dL_deta0) {
    return adjoint_core(g, scenario, n, checkpoint_every, dL_drecords, dL_deta0, nullptr, 3);
}

int cliffs_adjoint_recorded_records(cliffs_grid* g, const float* dL_drecords, float* dL_deta0) {
    return cliffs_adjoint_recorded_scenario(g, 0, 3, dL_drecords, dL_deta0);
}

int cliffs_adjoint_recorded_scenario(cliffs_grid* g, int32_t scenario, int32_t components, const float* dL,
                                     float* dL_deta0) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (components != 1 && components != 3) return set_err(CLIFFS_ERR_ARG, "components must be 1 or 3");
    if (g->rec_K <= 0 || g->rec_n < 1) return set_err(CLIFFS_ERR_STATE, "no recorded run");
    return adjoint_core(g, scenario, g->rec_n, g->rec_K, dL, dL_deta0, g->rec_ckpt, components);
}

// Adjoint of a y-first step j of the alternating order, X_{j+1} = x-sweep(y-sweep(X_j)),
// from lambda_{j+1} (transposed, in the second third of adj_t) to lambda_j in the same place:
// the y-sweep of X_j is recomputed row-major, the x-sweep adjoint runs over it, then the
// y-sweep adjoint over X_j transposed, with transposes where the layouts differ.
static int adjoint_yfirst_step(cliffs_grid* g, const StepArgs& a, const AdjLineArgs& X, const AdjLineArgs& Y,
                               const float* st, long long fst, long long j, bool seeded) {
    const int nx = g->nx, ny = g->ny, tp = (ny + 31) / 32 * 32;
    const long long P = g->plane, TPL = (long long)tp * nx;
    cudaStream_t s = g->stream;
    if (!g->adj_alt) CK(cudaMalloc(&g->adj_alt, sizeof(float) * (3 * P + 3 * TPL)));
    float* XT = g->adj_t;
    float* LT = g->adj_t + 3 * TPL;
    float* LB = g->adj_lb;
    float* XR = g->adj_alt;
    float* LT2 = g->adj_alt + 3 * P;
    cudaError_t le = cudaSuccess;
    for (int f = 0; f < 3 && le == cudaSuccess; ++f)            // lambda_{j+1} row-major
        le = launch_transpose(LT + f * TPL, tp, LB + f * P, g->pitch, nx, ny, s);
    StepArgs ay = a;                                             // y-sweep of X_j
    ay.eta_in = st; ay.u_in = st + fst; ay.v_in = st + 2 * fst;
    ay.eta_out = XR; ay.u_out = XR + P; ay.v_out = XR + 2 * P;
    ay.emax = ay.smax = nullptr; ay.rec_g = ay.rec_n = nullptr; ay.samp_ptr = nullptr; ay.limit = nullptr;
    ay.nstrips = (nx + XWIN - 1) / XWIN; ay.S = 64; ay.nseg = (ny + 63) / 64;
    if (le == cudaSuccess) le = launch_ysweep(ay, 1, s);
    AdjLineArgs X2 = X;                                          // x-sweep adjoint over it
    X2.pe = XR; X2.pw = XR + P; X2.pt = XR + 2 * P;
    X2.oe = LT2; X2.ow = LT2 + TPL; X2.ot = LT2 + 2 * TPL;
    X2.seed = nullptr;
    if (le == cudaSuccess) le = launch_adj_line(X2, 0, a.sph, s);
    for (int f = 0; f < 3 && le == cudaSuccess; ++f)            // X_j transposed
        le = launch_transpose(st + f * fst, g->pitch, XT + f * TPL, tp, ny, nx, s);
    AdjLineArgs Y2 = Y;                                          // y-sweep adjoint -> row-major
    Y2.ge = LT2; Y2.gw = LT2 + 2 * TPL; Y2.gt = LT2 + TPL;
    if (le == cudaSuccess) le = launch_adj_line(Y2, 1, a.sph, s);
    for (int f = 0; f < 3 && le == cudaSuccess; ++f)            // lambda_j transposed
        le = launch_transpose(LB + f * P, g->pitch, LT + f * TPL, tp, ny, nx, s);
    if (le == cudaSuccess && seeded && j % g->cfg.gout == 0)
        le = launch_adj_seed(LT, tp, TPL, g->adj_gxy, g->G, g->adj_seed + (j / g->cfg.gout) * 3 * g->G, s);
    if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "adjoint launch: %s", cudaGetErrorString(le));
    return CLIFFS_OK;
}

// The adjoint steps of cliffs_adjoint_n; `recorded` holds the checkpoints of a recorded run
// (X_0 included), else a checkpoint pass from the grid's current state makes them.
// comps: dL_dgauges holds dL/d eta at the gauge records ([nrec][G], comps 1) or dL/d (eta,
// u, v) ([nrec][G][3], comps 3); the seeds are kept as [nrec][G][3] either way.
static int adjoint_core(cliffs_grid* g, int scenario, int64_t n, int32_t checkpoint_every, const float* dL_dgauges,
                        float* dL_deta0, const float* recorded, int comps) {
    g_err[0] = 0;
    if (!g || !dL_deta0) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    if (g->kind != 0) return set_err(CLIFFS_ERR_ARG, "the adjoint needs a 2D grid");
    if (scenario < 0 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d outside 0..%d", scenario, g->B - 1);
    if (recorded && !g->limit_h.empty() && g->limit_h[scenario] < n)
        return set_err(CLIFFS_ERR_ARG, "scenario %d stopped after %lld of the %lld recorded steps", scenario,
                       (long long)g->limit_h[scenario], (long long)n);
    if (n < 1 || checkpoint_every < 1) return set_err(CLIFFS_ERR_ARG, "need n >= 1 and checkpoint_every >= 1");
    if (!recorded && !g->limit_h.empty() && g->step + n > g->limit_h[scenario])
        return set_err(CLIFFS_ERR_ARG, "scenario %d stops after %lld steps, before %lld more", scenario,
                       (long long)g->limit_h[scenario], (long long)n);
    cudaStream_t s = g->stream;
    const int nx = g->nx, ny = g->ny, K = (int)std::min<int64_t>(checkpoint_every, n);
    const long long P = g->plane;                          // row-major plane, floats
    const int tp = (ny + 31) / 32 * 32;                     // transposed pitch
    const long long TPL = (long long)tp * nx;               // transposed plane, floats
    const long long nseg = (n + K - 1) / K;
    const long long nrec = n / g->cfg.gout + 1;
    const int G = g->G;
    // Segments are recomputed NG at a time: one launch per step advances NG segments (the
    // fused kernel's batch dimension), which fills the GPU where one grid's launch does not.
    // NG is the number of segments whose K states fit in ADJ_GROUP_BYTES, at most
    // ADJ_GROUP_MAX (1 with boundary input or the alternating order, whose steps differ
    // between segments).
    int NG = 1;
    if (K > 1 && !g->bnd_any && !g->cfg.alternate) {
        const double seg_bytes = 12.0 * (double)P * K;
        NG = (int)std::max(1.0, std::min({(double)nseg, (double)ADJ_GROUP_MAX,
                                          std::floor((double)ADJ_GROUP_BYTES / seg_bytes)}));
    }
    // work space (kept for later calls); a smaller group if the larger one does not fit
    if (g->adj_K < K || g->adj_G < NG || !g->adj_slots) {
        cudaFree(g->adj_slots);
        g->adj_slots = nullptr;
        g->adj_maps.clear();
        const int KA = std::max(K, 2);
        for (;;) {
            const cudaError_t me = cudaMalloc(&g->adj_slots, sizeof(float) * 3 * P * (size_t)NG * KA);
            if (me == cudaSuccess) break;
            cudaGetLastError();
            if (NG == 1) return set_err(CLIFFS_ERR_CUDA, "adjoint work space: %s", cudaGetErrorString(me));
            NG = (NG + 1) / 2;
        }
        g->adj_K = KA;
        g->adj_G = NG;
        g->adj_pmaps.assign((size_t)KA * NG, StepMaps{});
        g->adj_pmaps_ok.assign((size_t)KA * NG, 0);
        g->adj_maps.resize(KA);
        for (int j = 0; j < KA; ++j) {
            StepMaps& M = g->adj_maps[j];
            M = g->maps[0];
            float* b = g->adj_slots + 3 * P * (size_t)NG * j;
            int rc = make_map(&M.e, b, 3, g->pitch, ny, NG);
            if (!rc) rc = make_map(&M.u, b + (size_t)NG * P, 3, g->pitch, ny, NG);
            if (!rc) rc = make_map(&M.v, b + (size_t)2 * NG * P, 3, g->pitch, ny, NG);
            if (rc) return rc;
        }
    }
    NG = std::min(NG, g->adj_G);
    const long long FS = (long long)g->adj_G * P;          // floats between the fields of a state
    // work items of the batched launches: rows per warp such that NG grids fill about
    // ADJ_GROUP_WAVES waves of resident warps (strips with dry nodes take shorter segments)
    if (NG > 1) {
        const long long cap = resident_warps(g) * ADJ_GROUP_WAVES;
        int Sr = 16;
        for (; Sr < ny; Sr += 2) {
            long long nw = 0;
            for (int st = 0; st < g->nstrips; ++st) {
                const int seg = (!g->hard.empty() && g->hard[st]) ? hard_rows(Sr) : Sr;
                nw += (ny + seg - 1) / seg;
            }
            if (nw * NG <= cap) break;
        }
        if (Sr != g->adj_S || g->adj_items.empty()) {
            g->adj_items.clear();
            for (int st = 0; st < g->nstrips; ++st) {
                const int seg = (!g->hard.empty() && g->hard[st]) ? hard_rows(Sr) : Sr;
                for (int r0 = 0; r0 < ny; r0 += seg) g->adj_items.push_back(make_int4(st, r0, std::min(r0 + seg, ny), 0));
            }
            cudaFree(g->adj_items_dev);
            g->adj_items_dev = nullptr;
            CK(cudaMalloc(&g->adj_items_dev, sizeof(int4) * g->adj_items.size()));
            CK(cudaMemcpy(g->adj_items_dev, g->adj_items.data(), sizeof(int4) * g->adj_items.size(),
                          cudaMemcpyHostToDevice));
            g->adj_S = Sr;
        }
    }
    if (!recorded && (g->adj_ncap < nseg || !g->adj_ckpt)) {
        cudaFree(g->adj_ckpt);
        g->adj_ckpt = nullptr;
        CK(cudaMalloc(&g->adj_ckpt, sizeof(float) * 3 * P * nseg));
        g->adj_ncap = nseg;
    }
    if (!g->adj_t) {
        CK(cudaMalloc(&g->adj_t, sizeof(float) * 7 * TPL));
        CK(cudaMalloc(&g->adj_lb, sizeof(float) * 3 * P));
        CK(cudaMemsetAsync(g->adj_t, 0, sizeof(float) * 7 * TPL, s));
        CK(cudaMemsetAsync(g->adj_lb, 0, sizeof(float) * 3 * P, s));
        if (G > 0) {
            CK(cudaMalloc(&g->adj_gxy, sizeof(int) * 2 * G));
            CK(cudaMemcpyAsync(g->adj_gxy, g->gauges.data(), sizeof(int) * 2 * G, cudaMemcpyHostToDevice, s));
        }
    }
    if (G > 0 && dL_dgauges && g->adj_seed_cap < nrec) {
        cudaFree(g->adj_seed);
        g->adj_seed = nullptr;
        CK(cudaMalloc(&g->adj_seed, sizeof(float) * 3 * G * nrec));
        g->adj_seed_cap = nrec;
    }
    const bool seeded = G > 0 && dL_dgauges;
    if (seeded) {
        if (comps == 3) {
            CK(cudaMemcpyAsync(g->adj_seed, dL_dgauges, sizeof(float) * 3 * G * nrec, cudaMemcpyDefault, s));
        } else {                                            // eta seeds into every third slot
            CK(cudaMemsetAsync(g->adj_seed, 0, sizeof(float) * 3 * G * nrec, s));
            CK(cudaMemcpy2DAsync(g->adj_seed, 3 * sizeof(float), dL_dgauges, sizeof(float), sizeof(float),
                                 (size_t)G * nrec, cudaMemcpyDefault, s));
        }
    }
    float* XT = g->adj_t;                                   // eta', u', v' transposed
    float* LT = g->adj_t + 3 * TPL;                         // adjoint (eta, u, v) transposed
    float* DT = g->adj_t + 6 * TPL;                         // depth transposed
    float* LB = g->adj_lb;                                  // adjoint (eta, u, v) row-major
    auto slot = [&](int j) { return g->adj_slots + 3 * FS * j; };
    StepArgs a;
    fill_step_args(g, a, 0, 1);
    a.limit = nullptr;
    a.step = 1;
    const long long s0 = recorded ? 0 : steps_of(g, scenario);   // steps done before X_0
    // step j of the run (y first on odd j with the alternating order) for one grid, from
    // state `in` (fields fin floats apart, read through the descriptors M) to state `out`
    // (fields fout apart)
    auto step1 = [&](float* in, long long fin, const StepMaps& M, float* out, long long fout, long long j) -> int {
        a.eta_in = in; a.u_in = in + fin; a.v_in = in + 2 * fin;
        a.eta_out = out; a.u_out = out + fout; a.v_out = out + 2 * fout;
        a.yfirst = g->cfg.alternate && ((s0 + j) & 1);     // the forward's parity: steps since set_initial
        a.items = g->items_dev;
        a.nitems = (int)g->items.size();
        if (g->bnd_any) {                                  // boundary input, as in cliffs_step_n
            const int rci = impose_boundary(g, in, in + fin, in + 2 * fin, g->t_start + (double)(s0 + j) * g->cfg.dt);
            if (rci) return rci;
        }
        const cudaError_t le = launch_step_fused(a, M, 1, s);
        if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "adjoint forward launch: %s", cudaGetErrorString(le));
        return CLIFFS_OK;
    };
    // step j from slot `from` to slot `to`, for nb segments at once (their steps then have the
    // same parity and no boundary input: NG is 1 otherwise)
    auto fwd = [&](int from, int to, long long j, int nb) -> int {
        if (nb == 1) return step1(slot(from), FS, g->adj_maps[from], slot(to), FS, j);
        a.eta_in = slot(from); a.u_in = slot(from) + FS; a.v_in = slot(from) + 2 * FS;
        a.eta_out = slot(to); a.u_out = slot(to) + FS; a.v_out = slot(to) + 2 * FS;
        a.yfirst = 0;
        a.items = g->adj_items_dev;
        a.nitems = (int)g->adj_items.size();
        const cudaError_t le = launch_step_fused(a, g->adj_maps[from], nb, s);
        if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "adjoint forward launch: %s", cudaGetErrorString(le));
        return CLIFFS_OK;
    };
    const float* ckpt = recorded ? recorded : g->adj_ckpt;
    const long long cfield = recorded ? (long long)g->B * P : P;      // floats between fields
    const long long cstride = 3 * cfield;                             // floats between checkpoints
    const long long coff = recorded ? (long long)scenario * P : 0;    // the scenario's plane
    // Groups of segments [sb, se), from the last, each recomputed in one batched run. Without
    // a recorded run and with K > 1 the checkpoint pass itself keeps every state of the first
    // group (the last segments: NG of them, the shorter last one included), which then needs
    // no recomputation. Otherwise a shorter last segment is recomputed alone, then NG at a
    // time.
    const bool keep_first = !recorded && K > 1;
    std::vector<std::pair<long long, long long>> groups;
    for (long long se = nseg; se > 0;) {
        const long long sb = (keep_first && se == nseg) ? std::max<long long>(0, se - NG)
                             : (n % K != 0 && se == nseg) ? se - 1 : std::max<long long>(0, se - NG);
        groups.push_back({sb, se});
        se = sb;
    }
    // X_0: the grid's current state (or the recorded run's first checkpoint)
    const int cb = (int)cur_buf(g, scenario);
    const size_t so = (size_t)scenario * P;                 // the scenario's plane
    if (!recorded && !keep_first) {
        CK(cudaMemcpyAsync(slot(0), g->eta[cb] + so, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(slot(0) + FS, g->u[cb] + so, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(slot(0) + 2 * FS, g->v[cb] + so, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        // checkpoint pass with every state kept (K = 1): X_j for every step j
        for (long long j = 0; j <= (nseg - 1) * K; ++j) {
            const int cur = (int)(j & 1);
            if (j % K == 0)
                for (int f = 0; f < 3; ++f)
                    CK(cudaMemcpyAsync(g->adj_ckpt + 3 * P * (j / K) + f * P, slot(cur) + f * FS, sizeof(float) * P,
                                       cudaMemcpyDeviceToDevice, s));
            if (j < (nseg - 1) * K) {
                int rc = fwd(cur, 1 - cur, j, 1);
                if (rc) return rc;
            }
        }
    }
    if (keep_first) {
        // checkpoint pass X_0 .. X_{n-1}: up to the first group's first step jk between two
        // states of its own (a checkpoint every K steps), from there in the first group's
        // slots (segment sb0 + p in plane p)
        const long long sb0 = groups[0].first, jk = sb0 * K;
        if (!g->adj_pp) {
            CK(cudaMalloc(&g->adj_pp, sizeof(float) * 6 * P));
            for (int k = 0; k < 2; ++k) {
                StepMaps& M = g->adj_ppmaps[k];
                M = g->maps[0];
                float* b = g->adj_pp + 3 * P * k;
                int rc = make_map(&M.e, b, 3, g->pitch, ny, 1);
                if (!rc) rc = make_map(&M.u, b + P, 3, g->pitch, ny, 1);
                if (!rc) rc = make_map(&M.v, b + 2 * P, 3, g->pitch, ny, 1);
                if (rc) return rc;
            }
        }
        // where X_j is kept during the pass, its field stride and its descriptors
        auto at = [&](long long j) -> float* {
            if (j < jk) return g->adj_pp + 3 * P * (j & 1);
            return slot((int)(j % K)) + (j / K - sb0) * P;
        };
        auto maps_of = [&](long long j, const StepMaps*& M) -> int {
            if (j < jk) { M = &g->adj_ppmaps[j & 1]; return CLIFFS_OK; }
            const size_t q = (size_t)(j % K) * g->adj_G + (size_t)(j / K - sb0);
            if (!g->adj_pmaps_ok[q]) {
                StepMaps& Mq = g->adj_pmaps[q];
                Mq = g->maps[0];
                float* b = at(j);
                int rc = make_map(&Mq.e, b, 3, g->pitch, ny, 1);
                if (!rc) rc = make_map(&Mq.u, b + FS, 3, g->pitch, ny, 1);
                if (!rc) rc = make_map(&Mq.v, b + 2 * FS, 3, g->pitch, ny, 1);
                if (rc) return rc;
                g->adj_pmaps_ok[q] = 1;
            }
            M = &g->adj_pmaps[q];
            return CLIFFS_OK;
        };
        auto fs_of = [&](long long j) -> long long { return j < jk ? P : FS; };
        float* x0 = at(0);
        CK(cudaMemcpyAsync(x0, g->eta[cb] + so, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(x0 + fs_of(0), g->u[cb] + so, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(x0 + 2 * fs_of(0), g->v[cb] + so, sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        for (long long j = 0; j + 1 < n; ++j) {
            if (j % K == 0 && j < jk)                         // checkpoints of the later groups
                for (int f = 0; f < 3; ++f)
                    CK(cudaMemcpyAsync(g->adj_ckpt + 3 * P * (j / K) + f * P, at(j) + f * P, sizeof(float) * P,
                                       cudaMemcpyDeviceToDevice, s));
            const StepMaps* M = nullptr;
            int rc = maps_of(j, M);
            if (!rc) rc = step1(at(j), fs_of(j), *M, at(j + 1), fs_of(j + 1), j);
            if (rc) return rc;
        }
    }
    cudaError_t le = launch_transpose(g->d32, g->pitch, DT, tp, ny, nx, s);
    if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "transpose: %s", cudaGetErrorString(le));
    // lambda_n: the seed of the last record
    CK(cudaMemsetAsync(LT, 0, sizeof(float) * 3 * TPL, s));
    if (seeded && n % g->cfg.gout == 0) {
        le = launch_adj_seed(LT, tp, TPL, g->adj_gxy, G, g->adj_seed + (n / g->cfg.gout) * 3 * G, s);
        if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "seed: %s", cudaGetErrorString(le));
    }
    AdjLineArgs Y{};                                        // y-sweep adjoint: lines are columns
    Y.pe = XT; Y.pw = XT + 2 * TPL; Y.pt = XT + TPL; Y.pd = DT;
    Y.ge = LT; Y.gw = LT + 2 * TPL; Y.gt = LT + TPL;
    Y.oe = LB; Y.ow = LB + 2 * P; Y.ot = LB + P;
    Y.nlines = nx; Y.npos = ny; Y.ipitch = tp; Y.opitch = g->pitch;
    Y.ymet = a.ymet;
    AdjLineArgs X{};                                        // x-sweep adjoint: lines are rows
    X.pd = g->d32;
    X.ge = LB; X.gw = LB + P; X.gt = LB + 2 * P;
    X.oe = LT; X.ow = LT + TPL; X.ot = LT + 2 * TPL;
    X.nlines = ny; X.npos = nx; X.ipitch = g->pitch; X.opitch = tp;
    X.xa = a.xa; X.xb = a.xb; X.xk = a.xk; X.xrow = a.xrow;
    X.gxy = g->adj_gxy; X.G = G;
    for (AdjLineArgs* A : {&X, &Y}) {
        A->hmin = a.hmin; A->dwall = a.dwall; A->half_dt = a.half_dt; A->dt_gn2 = a.dt_gn2;
        A->transverse = a.transverse;
        A->inv_dt2_s1 = a.inv_dt2_s1;
    }
    X.open_lo = g->cfg.open_edges & 1; X.open_hi = (g->cfg.open_edges >> 1) & 1;     // W, E
    Y.open_lo = (g->cfg.open_edges >> 2) & 1; Y.open_hi = (g->cfg.open_edges >> 3) & 1;   // S, N
    bool after_xadj = false;                   // the last launch was an x-sweep adjoint
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const long long sb = groups[gi].first, se = groups[gi].second;
        const int nb = (int)(se - sb);
        const bool pass_kept = keep_first && gi == 0;        // states from the checkpoint pass
        // a one-step segment (every state kept: K = 1) is read where it is stored, with no
        // copy and no recomputation
        // a checkpoint holds [3][batch][plane] (recorded) or [3][plane]: this scenario's fields
        const bool kept = !pass_kept && nb == 1 && std::min<long long>(sb * K + K, n) - sb * K == 1 && cfield == P;
        if (!kept && !pass_kept)
            for (int b = 0; b < nb; ++b)
                for (int f = 0; f < 3; ++f)
                    CK(cudaMemcpyAsync(slot(0) + f * FS + b * P, ckpt + cstride * (sb + b) + coff + f * cfield,
                                       sizeof(float) * P, cudaMemcpyDeviceToDevice, s));
        if (!kept) after_xadj = false;                     // the checkpoint copies and the recomputation
        const long long len = std::min<long long>(sb * K + K, n) - sb * K;   // steps of each segment
        for (long long i = 0; i + 1 < len && !pass_kept; ++i) {
            int rc = fwd((int)i, (int)(i + 1), sb * K + i, nb);
            if (rc) return rc;
        }
        for (long long sg = se - 1; sg >= sb; --sg) {
            const long long j0 = sg * K, j1 = std::min<long long>(j0 + K, n);
            for (long long j = j1 - 1; j >= j0; --j) {
                const float* st = kept ? ckpt + cstride * sg + coff : slot((int)(j - j0)) + (sg - sb) * P;
                const long long fst = kept ? cfield : FS;     // floats between the fields of st
                // with boundary input the stored state is imposed again first (the step ran on
                // the imposed state), and the seed goes in after the input edges of lambda_j are
                // zeroed
                if (g->bnd_any) {
                    const int rci = impose_boundary(g, const_cast<float*>(st), const_cast<float*>(st) + fst,
                                                    const_cast<float*>(st) + 2 * fst,
                                                    g->t_start + (double)(s0 + j) * g->cfg.dt);
                    if (rci) return rci;
                }
                const float* seed_j =
                    (seeded && j % g->cfg.gout == 0) ? g->adj_seed + (j / g->cfg.gout) * 3 * G : nullptr;
                if (g->cfg.alternate && ((s0 + j) & 1)) {
                    int rc2 = adjoint_yfirst_step(g, a, X, Y, st, fst, j, g->bnd_any ? false : seeded);
                    if (rc2) return rc2;
                    after_xadj = false;
                } else {
                    // Without boundary input or the alternating order the three launches of a
                    // step follow one another as programmatic launches: each may start in the
                    // last wave of the one before; the x-sweep recomputation only right behind
                    // the previous step's x-sweep adjoint (not behind the copies and the
                    // recomputation that write its state).
                    const bool pdl = ADJ_PDL && !g->bnd_any && !g->cfg.alternate;
                    le = launch_adj_xfwd(a, st, st + fst, st + 2 * fst, XT, XT + TPL, XT + 2 * TPL, tp, s,
                                         pdl && after_xadj);
                    if (le == cudaSuccess) le = launch_adj_line(Y, 1, a.sph, s, pdl);
                    X.pe = st; X.pw = st + fst; X.pt = st + 2 * fst;
                    X.seed = g->bnd_any ? nullptr : seed_j;
                    if (le == cudaSuccess) le = launch_adj_line(X, 0, a.sph, s, pdl);
                    after_xadj = true;
                    if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "adjoint launch: %s", cudaGetErrorString(le));
                }
                if (g->bnd_any) {
                    after_xadj = false;
                    le = launch_adj_zero_edges(LT, tp, nx, ny, input_edges(g), s);
                    if (le == cudaSuccess && seed_j) le = launch_adj_seed(LT, tp, TPL, g->adj_gxy, G, seed_j, s);
                    if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "adjoint launch: %s", cudaGetErrorString(le));
                }
            }
        }
    }
    // dL/d eta_0 = the eta part of lambda_0, back to [ny][nx]; the u and v parts stay for
    // cliffs_adjoint_velocity
    g->adj_done = false;
    int rc = ensure_tmp(g, sizeof(float) * (size_t)nx * ny);
    if (rc) return rc;
    le = launch_transpose(LT, tp, (float*)g->tmp, nx, nx, ny, s);
    if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "transpose: %s", cudaGetErrorString(le));
    CK(cudaMemcpyAsync(dL_deta0, g->tmp, sizeof(float) * (size_t)nx * ny, cudaMemcpyDefault, s));
    int h[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(h, g->err, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h[0]) {
        CK(cudaMemsetAsync(g->err, 0, sizeof(int) * 4, s));
        if (h[0] & ERRF_TIMEOUT) return set_err(CLIFFS_ERR_TIMEOUT, "a bounded device wait gave up");
        return set_err(CLIFFS_ERR_UNSTABLE, "non-finite or runaway state in the forward recomputation");
    }
    g->adj_done = true;
    return CLIFFS_OK;
}

int cliffs_adjoint_velocity(cliffs_grid* g, float* dL_du0, float* dL_dv0) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->adj_done) return set_err(CLIFFS_ERR_STATE, "no adjoint has run");
    const int nx = g->nx, ny = g->ny, tp = (ny + 31) / 32 * 32;
    const long long TPL = (long long)tp * nx;
    const float* LT = g->adj_t + 3 * TPL;
    cudaStream_t s = g->stream;
    int rc = ensure_tmp(g, sizeof(float) * (size_t)nx * ny);
    if (rc) return rc;
    float* outs[2] = {dL_du0, dL_dv0};
    for (int f = 0; f < 2; ++f) {
        if (!outs[f]) continue;
        const cudaError_t le = launch_transpose(LT + (1 + f) * TPL, tp, (float*)g->tmp, nx, nx, ny, s);
        if (le != cudaSuccess) return set_err(CLIFFS_ERR_CUDA, "transpose: %s", cudaGetErrorString(le));
        CK(cudaMemcpyAsync(outs[f], g->tmp, sizeof(float) * (size_t)nx * ny, cudaMemcpyDefault, s));
    }
    CK(cudaStreamSynchronize(s));
    return CLIFFS_OK;
}

int cliffs_set_rows_per_warp(cliffs_grid* g, int32_t rows) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_bathy) return set_err(CLIFFS_ERR_STATE, "set_bathy first (it chooses the geometry)");
    if (g->kind != 0) return set_err(CLIFFS_ERR_ARG, "a 1D grid has no tile shape");
    if (rows < 1 || rows > 8192) return set_err(CLIFFS_ERR_ARG, "rows per warp %d outside 1..8192", rows);
    return set_rows_per_warp(g, rows, hard_rows(rows));
}

int cliffs_autotune(cliffs_grid* g, int trials, int32_t* cand, double* us, int32_t* ncand) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    if (g->kind != 0) {                       // 1D grids have no tile shape to choose
        if (ncand) *ncand = 0;
        return CLIFFS_OK;
    }
    if (trials < 1) trials = 3;
    cudaStream_t s = g->stream;
    // scratch output planes: the trial steps read the current state and write elsewhere,
    // with max-wave and records off, so the grid's state and outputs are untouched; before
    // each trial a write larger than L2 evicts the inputs, as in a long run
    const size_t pb = sizeof(float) * (size_t)g->B * g->plane;
    const size_t flush_bytes = (size_t)192 << 20;
    float* scratch = nullptr;
    CK(cudaMalloc(&scratch, 3 * pb + flush_bytes));
    unsigned char* flush = reinterpret_cast<unsigned char*>(scratch + 3 * (pb / sizeof(float)));
    const int cur = (int)(g->step & 1);
    StepArgs a;
    fill_step_args(g, a, cur, 1 - cur);
    a.eta_out = scratch;
    a.u_out = scratch + (size_t)g->B * g->plane;
    a.v_out = scratch + 2 * (size_t)g->B * g->plane;
    a.step = g->step + 1;
    // fixed shapes, and those that just fit one, two or three waves of resident warps
    std::vector<int> list = {16, 24, 32, 48, 64, 96, 128};
    for (int wv = 1; wv <= 3; ++wv) {
        const int S1 = wave_rows(g, wv);
        if (S1 > 0)
            for (int d : {0, 2, 4}) list.push_back(S1 + d);
    }
    std::sort(list.begin(), list.end());
    list.erase(std::unique(list.begin(), list.end()), list.end());
    if (list.size() > 16) list.resize(16);
    const int oldS = g->S;
    int bestS = oldS, n = 0;
    double best = 1e300;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int rc = CLIFFS_OK;
    for (int S : list) {
        if (S > 2 * g->ny && S != list[0]) break;
        rc = set_rows_per_warp(g, S, hard_rows(S));
        if (rc) break;
        a.S = g->S; a.nseg = g->nseg; a.samp_ptr = g->samp_ptr; a.samp = g->samp;
        a.items = g->items_dev; a.nitems = (int)g->items.size();
        float tbest = 1e30f;
        for (int t = 0; t <= trials; ++t) {             // the first launch warms up
            cudaMemsetAsync(flush, t & 0xff, flush_bytes, s);
            cudaEventRecord(e0, s);
            cudaError_t le = launch_step_fused(a, g->maps[cur], g->B, s);
            cudaEventRecord(e1, s);
            if (le != cudaSuccess) { rc = set_err(CLIFFS_ERR_CUDA, "autotune launch: %s", cudaGetErrorString(le)); break; }
            if (cudaEventSynchronize(e1) != cudaSuccess) { rc = set_err(CLIFFS_ERR_CUDA, "autotune sync"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (t > 0) tbest = std::min(tbest, ms);
        }
        if (rc) break;
        if (cand) cand[n] = S;
        if (us) us[n] = 1e3 * tbest;
        ++n;
        if (tbest < best) { best = tbest; bestS = S; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(scratch);
    int h[4] = {0, 0, 0, 0};
    cudaMemcpy(h, g->err, sizeof(h), cudaMemcpyDeviceToHost);
    cudaMemset(g->err, 0, sizeof(h));
    const int rc2 = set_rows_per_warp(g, rc ? oldS : bestS, hard_rows(rc ? oldS : bestS));
    if (ncand) *ncand = n;
    if (rc) return rc;
    if (rc2) return rc2;
    if (h[0] & ERRF_TIMEOUT) return set_err(CLIFFS_ERR_TIMEOUT, "a bounded device wait gave up during autotuning");
    return CLIFFS_OK;
}

int cliffs_inject_wait_expiry(cliffs_grid* g, int64_t cycles) {
    g_err[0] = 0;
    if (!g || cycles <= 0) return set_err(CLIFFS_ERR_ARG, "need a grid and a positive cycle limit");
    if (g->kind != 0) return set_err(CLIFFS_ERR_ARG, "the bounded waits belong to the 2D step kernel");
    g->inject_cycles = cycles;
    return CLIFFS_OK;
}

int cliffs_steps_done(cliffs_grid* g, int64_t* steps) {
    if (!g || !steps) return set_err(CLIFFS_ERR_ARG, "null argument");
    *steps = g->step;
    return CLIFFS_OK;
}

int cliffs_read_gauges(cliffs_grid* g, int scenario, float* out, int64_t* nrec) {
    g_err[0] = 0;
    if (!g || !nrec) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (scenario < 0 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d out of range", scenario);
    if (!g->have_init || g->G == 0) { *nrec = 0; return CLIFFS_OK; }
    const long long n = steps_of(g, scenario) / g->cfg.gout + 1;
    *nrec = n;
    if (out) {
        CK(cudaMemcpyAsync(out, g->grec + (size_t)scenario * g->grec_cap * g->G * 3,
                           sizeof(float) * n * g->G * 3, cudaMemcpyDefault, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    return CLIFFS_OK;
}

int cliffs_read_maxwave(cliffs_grid* g, int scenario, float* eta_max, float* speed_max) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (scenario < 0 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d out of range", scenario);
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    const long long N = (long long)g->nx * g->ny;
    int rc = ensure_tmp(g, 2 * sizeof(float) * N);
    if (rc) return rc;
    float* te = (float*)g->tmp;
    float* ts = te + N;
    const int cb = (int)cur_buf(g, scenario);
    const size_t o = (size_t)scenario * g->plane;
    k_max_fold<<<nblk(N), 256, 0, g->stream>>>(g->emax + o, g->smax + o, g->eta[cb] + o, g->u[cb] + o,
                                               g->v[cb] + o, g->d32, te, ts, g->nx, g->ny, g->pitch,
                                               (float)g->cfg.h_min,
                                               g->cfg.itopo ? -3.402823466e38f : (float)g->cfg.dwall);
    CK(cudaGetLastError());
    if (eta_max) CK(cudaMemcpyAsync(eta_max, te, sizeof(float) * N, cudaMemcpyDefault, g->stream));
    if (speed_max) CK(cudaMemcpyAsync(speed_max, ts, sizeof(float) * N, cudaMemcpyDefault, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return CLIFFS_OK;
}

int cliffs_read_boundary(cliffs_grid* g, int nest, int edge, double* vals, int64_t* nt) {
    g_err[0] = 0;
    if (!g || !nt) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (nest < 0 || nest >= (int)g->nests.size() || edge < 0 || edge > 3)
        return set_err(CLIFFS_ERR_ARG, "nest %d edge %d out of range", nest, edge);
    if (!g->have_init) { *nt = 0; return CLIFFS_OK; }
    const long long n = g->step / g->cfg.bndout + 1;
    *nt = n;
    if (!vals) return CLIFFS_OK;
    const int k = nest * 4 + edge;
    const int np = g->edge_np[k];
    int rc = ensure_tmp(g, sizeof(double) * n * 3 * np);
    if (rc) return rc;
    k_boundary<<<nblk(n * np), 256, 0, g->stream>>>(g->nrec, g->NN, g->pt_slot, g->pt_w, g->edge_off[k], np, n,
                                                    (double*)g->tmp);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(vals, g->tmp, sizeof(double) * n * 3 * np, cudaMemcpyDefault, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return CLIFFS_OK;
}

int cliffs_read_state(cliffs_grid* g, int scenario, float* eta, float* u, float* v) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (scenario < 0 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d out of range", scenario);
    const int cb = (int)cur_buf(g, scenario);
    const size_t o = (size_t)scenario * g->plane;
    const size_t rowb = sizeof(float) * g->nx, pitchb = sizeof(float) * g->pitch;
    if (eta) CK(cudaMemcpy2DAsync(eta, rowb, g->eta[cb] + o, pitchb, rowb, g->ny, cudaMemcpyDefault, g->stream));
    if (u) CK(cudaMemcpy2DAsync(u, rowb, g->u[cb] + o, pitchb, rowb, g->ny, cudaMemcpyDefault, g->stream));
    if (v) CK(cudaMemcpy2DAsync(v, rowb, g->v[cb] + o, pitchb, rowb, g->ny, cudaMemcpyDefault, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return CLIFFS_OK;
}

int cliffs_state_ptrs(cliffs_grid* g, int scenario, float** eta, float** u, float** v, int64_t* pitch) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (scenario < 0 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d out of range", scenario);
    const int cb = (int)cur_buf(g, scenario);
    const size_t o = (size_t)scenario * g->plane;
    if (eta) *eta = g->eta[cb] + o;
    if (u) *u = g->u[cb] + o;
    if (v) *v = g->v[cb] + o;
    if (pitch) *pitch = g->pitch;
    return CLIFFS_OK;
}

// Node control widths along one axis: half the distance to each neighbour, the full spacing
// at an end node (the wall stands half a spacing beyond it), 1 on a one-node axis.
static void control_widths(const std::vector<double>& c, std::vector<double>& w) {
    const size_t n = c.size();
    w.assign(n, 1.0);
    if (n < 2) return;
    w[0] = c[1] - c[0];
    w[n - 1] = c[n - 1] - c[n - 2];
    for (size_t i = 1; i + 1 < n; ++i) w[i] = 0.5 * (c[i + 1] - c[i - 1]);
}

int cliffs_diagnostics(cliffs_grid* g, int scenario, double* out) {
    g_err[0] = 0;
    if (!g || !out) return set_err(CLIFFS_ERR_ARG, "null argument");
    if (scenario < 0 || scenario >= g->B) return set_err(CLIFFS_ERR_ARG, "scenario %d out of range", scenario);
    if (!g->have_init) return set_err(CLIFFS_ERR_STATE, "set_initial first");
    const int nx = g->nx, ny = g->ny;
    std::vector<double> wx, wy;
    control_widths(g->hx, wx);
    control_widths(g->hy, wy);
    if (g->cfg.coords != 1) {                    // lon/lat in degrees: R^2 cos(phi) dlambda dphi
        for (int i = 0; i < nx; ++i) wx[i] *= R_SPHERE * DEGR;
        for (int j = 0; j < ny; ++j) wy[j] *= R_SPHERE * DEGR * std::cos(g->hy[j] * DEGR);
    }
    std::vector<double> host(nx + ny + 2, 0.0);
    std::copy(wx.begin(), wx.end(), host.begin());
    std::copy(wy.begin(), wy.end(), host.begin() + nx);
    int rc = ensure_tmp(g, sizeof(double) * host.size() + 2 * sizeof(unsigned));
    if (rc) return rc;
    double* dw = (double*)g->tmp;
    unsigned* mx = (unsigned*)(dw + host.size());
    CK(cudaMemcpyAsync(dw, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemsetAsync(mx, 0, 2 * sizeof(unsigned), g->stream));
    const int cb = (int)cur_buf(g, scenario);
    const size_t o = (size_t)scenario * g->plane;
    const long long N = (long long)nx * ny;
    const unsigned blocks = std::min<unsigned>(nblk(N), 1024u);
    k_diag<<<blocks, 256, 0, g->stream>>>(g->eta[cb] + o, g->u[cb] + o, g->v[cb] + o, g->d32, dw, dw + nx,
                                          nx, ny, g->pitch, (float)g->cfg.h_min,
                                          g->cfg.itopo ? -3.402823466e38f : (float)g->cfg.dwall,
                                          dw + nx + ny, mx);
    CK(cudaGetLastError());
    double acc[2];
    unsigned m[2];
    CK(cudaMemcpyAsync(acc, dw + nx + ny, sizeof(acc), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(m, mx, sizeof(m), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    float me, ms;
    std::memcpy(&me, &m[0], sizeof(float));
    std::memcpy(&ms, &m[1], sizeof(float));
    out[0] = acc[0];
    out[1] = acc[1];
    out[2] = me;
    out[3] = ms;
    return CLIFFS_OK;
}

int cliffs_kernel_time(cliffs_grid* g, int enable, double* ms, int64_t* launches) {
    g_err[0] = 0;
    if (!g) return set_err(CLIFFS_ERR_ARG, "null argument");
    int rc = collect_timing(g);
    if (rc) return rc;
    if (enable < 0) { g->t_ms = 0.0; g->t_launches = 0; }
    else g->timing = enable != 0;
    if (ms) *ms = g->t_ms;
    if (launches) *launches = g->t_launches;
    return CLIFFS_OK;
}

void cliffs_destroy(cliffs_grid* g) {
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    free_grid(g);
}

}  // extern "C"
