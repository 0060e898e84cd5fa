// Sweep kernels of the split shallow-water step (arXiv 1410.0753, section "Numerics").
//
//  k_step_fused  one full step (x-sweep then y-sweep) per launch. A warp owns a strip of
//                56 output columns and S output rows. It walks the rows of its strip from
//                r0-3 to r0+S+2: each row is loaded once (64 columns, 2 per lane, 8-byte
//                vector loads, the next row prefetched), x-swept across the warp with
//                shuffles, and pushed into a per-column register pipeline that finishes the
//                y-sweep three rows behind. The step reads eta, u, v, d and writes eta, u, v
//                once per cell (28 B/cell-update plus the halo), fused with the max-wave
//                update and the gauge / enclosed-grid sampling of that step.
//  k_xsweep      x-sweep alone (1D grids along x).
//  k_ysweep      y-sweep alone (1D grids along y).
#include "internal.h"
#include "sweep.cuh"

namespace cliffs {

__device__ __forceinline__ SweepConst sweep_const(const StepArgs& a) {
    return SweepConst{a.hmin, a.dwall, a.half_dt, a.dt_gn2, a.transverse};
}

// Nodes (r, c) and (r, c+1) of the step input; nodes outside the domain get depth
// OUTSIDE_D (dry, never wetted) and zero state. c is even and rows are padded to an even
// pitch, so the 8-byte loads stay aligned and inside the allocation.
__device__ __forceinline__ void load_pair(const StepArgs& a, size_t boff, int r, int c,
                                          float& e0, float& u0, float& v0, float& d0,
                                          float& e1, float& u1, float& v1, float& d1) {
    e0 = u0 = v0 = e1 = u1 = v1 = 0.f;
    d0 = d1 = OUTSIDE_D;
    if (r >= 0 && r < a.ny && c >= 0 && c < a.nx) {
        const size_t o = (size_t)r * a.pitch + c;
        const float2 e = __ldg(reinterpret_cast<const float2*>(a.eta_in + boff + o));
        const float2 u = __ldg(reinterpret_cast<const float2*>(a.u_in + boff + o));
        const float2 v = __ldg(reinterpret_cast<const float2*>(a.v_in + boff + o));
        const float2 d = __ldg(reinterpret_cast<const float2*>(a.d + o));
        e0 = e.x; u0 = u.x; v0 = v.x; d0 = d.x;
        if (c + 1 < a.nx) { e1 = e.y; u1 = u.y; v1 = v.y; d1 = d.y; }
    }
}

// max-wave update of one node (section "Running Options", field maxout): wet nodes only
__device__ __forceinline__ void max_upd(float& em, float& sm, float e, float u, float v,
                                        float d, const StepArgs& a, bool& ch) {
    if (!((d >= a.dwall) && (e + d >= a.hmin))) return;
    if (e > em) { em = e; ch = true; }
    const float s2 = fmaf(u, u, v * v);
    if (s2 > sm * sm) { sm = fmaxf(sm, sqrtf(s2)); ch = true; }
}

// Store a finished pair of nodes of row r and apply the step's max-wave update.
__device__ __forceinline__ void emit_pair(const StepArgs& a, size_t boff, int r, int c,
                                          bool va, bool vb,
                                          float eA, float uA, float vA, float dA,
                                          float eB, float uB, float vB, float dB, int& bad) {
    if (!va) return;
    const size_t o = boff + (size_t)r * a.pitch + c;
    if (vb) {
        *reinterpret_cast<float2*>(a.eta_out + o) = make_float2(eA, eB);
        *reinterpret_cast<float2*>(a.u_out + o) = make_float2(uA, uB);
        *reinterpret_cast<float2*>(a.v_out + o) = make_float2(vA, vB);
    } else {
        a.eta_out[o] = eA; a.u_out[o] = uA; a.v_out[o] = vA;
    }
    bad |= !(fabsf(eA) < 1e5f && fabsf(uA) < 1e5f && fabsf(vA) < 1e5f);
    if (vb) bad |= !(fabsf(eB) < 1e5f && fabsf(uB) < 1e5f && fabsf(vB) < 1e5f);
    if (a.emax) {
        bool ch = false;
        if (vb) {
            float2 em = *reinterpret_cast<float2*>(a.emax + o);
            float2 sm = *reinterpret_cast<float2*>(a.smax + o);
            max_upd(em.x, sm.x, eA, uA, vA, dA, a, ch);
            max_upd(em.y, sm.y, eB, uB, vB, dB, a, ch);
            if (ch) {
                *reinterpret_cast<float2*>(a.emax + o) = em;
                *reinterpret_cast<float2*>(a.smax + o) = sm;
            }
        } else {
            float em = a.emax[o], sm = a.smax[o];
            max_upd(em, sm, eA, uA, vA, dA, a, ch);
            if (ch) { a.emax[o] = em; a.smax[o] = sm; }
        }
    }
}

// Gauge / enclosed-grid node samples of row r owned by this warp (sorted by row).
__device__ __forceinline__ void emit_samples(const StepArgs& a, int b, int& sp, int se, int r,
                                             int c0, int lane,
                                             float eA, float uA, float vA,
                                             float eB, float uB, float vB) {
    while (sp < se) {
        const int4 it = __ldg(a.samp + sp);
        if (it.x != r) break;
        const int rel = it.y - c0;
        if ((rel >> 1) == lane) {
            const bool isB = rel & 1;
            float* out = (it.z == 0) ? (a.rec_g ? a.rec_g + (long long)b * a.rec_g_bstride : nullptr)
                                     : a.rec_n;
            if (out) {
                out[3 * it.w + 0] = isB ? eB : eA;
                out[3 * it.w + 1] = isB ? uB : uA;
                out[3 * it.w + 2] = isB ? vB : vA;
            }
        }
        ++sp;
    }
}

template <bool SPH>
__global__ void __launch_bounds__(128) k_step_fused(const StepArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int b = blockIdx.y;
    if (gw >= a.nstrips * a.nseg) return;
    if (a.limit && a.step > a.limit[b]) return;
    const int strip = gw % a.nstrips, seg = gw / a.nstrips;
    const int c0 = strip * XOUT - 4;
    const int cA = c0 + 2 * lane;
    const int r0 = seg * a.S, r1 = min(r0 + a.S, a.ny);
    const size_t boff = (size_t)b * a.plane;
    const SweepConst K = sweep_const(a);
    XMet mA0{0.f, 0.f, 0.f}, mB0{0.f, 0.f, 0.f};
    if (cA >= 0 && cA < a.nx) mA0 = XMet{__ldg(a.xa + cA), __ldg(a.xb + cA), __ldg(a.xk + cA)};
    if (cA + 1 >= 0 && cA + 1 < a.nx)
        mB0 = XMet{__ldg(a.xa + cA + 1), __ldg(a.xb + cA + 1), __ldg(a.xk + cA + 1)};
    const bool own = lane >= 2 && lane < 30;
    const bool vA = own && cA < a.nx;
    const bool vB = own && cA + 1 < a.nx;
    int sp = 0, se = 0;
    if (a.samp_ptr && (a.rec_g || a.rec_n)) { sp = a.samp_ptr[gw]; se = a.samp_ptr[gw + 1]; }
    YMarch ya, yb;
    ya.init();
    yb.init();
    int bad = 0;
    float pe0, pu0, pv0, pd0, pe1, pu1, pv1, pd1;
    load_pair(a, boff, r0 - 3, cA, pe0, pu0, pv0, pd0, pe1, pu1, pv1, pd1);
    for (int k = r0 - 3; k < r1 + 3; ++k) {
        float eA = pe0, uA = pu0, vA_ = pv0, dA = pd0;
        float eB = pe1, uB = pu1, vB_ = pv1, dB = pd1;
        if (k + 1 < r1 + 3) load_pair(a, boff, k + 1, cA, pe0, pu0, pv0, pd0, pe1, pu1, pv1, pd1);
        if (k >= 0 && k < a.ny) {
            XMet mA = mA0, mB = mB0;
            if (SPH) {
                const float f = __ldg(a.xrow + k);
                mA.inv_l *= f; mA.inv_r *= f; mA.k2 *= f;
                mB.inv_l *= f; mB.inv_r *= f; mB.k2 *= f;
            }
            xsweep_pair(eA, uA, vA_, dA, eB, uB, vB_, dB, mA, mB, K, lane);
            // a non-finite x-sweep result would read as a dry node in the y-sweep and be
            // refilled by step (b) there, so it is checked here, before that happens
            if (own && cA < a.nx) bad |= !(fabsf(eA) < 1e5f && fabsf(uA) < 1e5f && fabsf(vA_) < 1e5f);
            if (own && cA + 1 < a.nx) bad |= !(fabsf(eB) < 1e5f && fabsf(uB) < 1e5f && fabsf(vB_) < 1e5f);
        }
        const float4 m2 = __ldg(a.ymet + min(max(k - 2, 0), a.ny - 1));
        float oeA, owA, otA, oeB, owB, otB;
        const float odA = ya.dd3, odB = yb.dd3;
        ya.push(eA, vA_, uA, dA, m2, K, oeA, owA, otA);
        yb.push(eB, vB_, uB, dB, m2, K, oeB, owB, otB);
        const int r = k - 3;
        if (r >= r0 && r < r1) {
            emit_pair(a, boff, r, cA, vA, vB, oeA, otA, owA, odA, oeB, otB, owB, odB, bad);
            if (sp < se) emit_samples(a, b, sp, se, r, c0, lane, oeA, otA, owA, oeB, otB, owB);
        }
    }
    if (bad) atomicOr(a.err, ERRF_NONFINITE);
}

// x-sweep alone: one warp per (row, strip of 56 columns).
template <bool SPH>
__global__ void __launch_bounds__(128) k_xsweep(const StepArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int b = blockIdx.y;
    if (gw >= a.nstrips * a.ny) return;
    if (a.limit && a.step > a.limit[b]) return;
    const int strip = gw % a.nstrips, r = gw / a.nstrips;
    const int c0 = strip * XOUT - 4;
    const int cA = c0 + 2 * lane;
    const size_t boff = (size_t)b * a.plane;
    const SweepConst K = sweep_const(a);
    XMet mA{0.f, 0.f, 0.f}, mB{0.f, 0.f, 0.f};
    if (cA >= 0 && cA < a.nx) mA = XMet{a.xa[cA], a.xb[cA], a.xk[cA]};
    if (cA + 1 >= 0 && cA + 1 < a.nx) mB = XMet{a.xa[cA + 1], a.xb[cA + 1], a.xk[cA + 1]};
    if (SPH) {
        const float f = a.xrow[r];
        mA.inv_l *= f; mA.inv_r *= f; mA.k2 *= f;
        mB.inv_l *= f; mB.inv_r *= f; mB.k2 *= f;
    }
    float eA, uA, vA_, dA, eB, uB, vB_, dB;
    load_pair(a, boff, r, cA, eA, uA, vA_, dA, eB, uB, vB_, dB);
    xsweep_pair(eA, uA, vA_, dA, eB, uB, vB_, dB, mA, mB, K, lane);
    const bool own = lane >= 2 && lane < 30;
    int bad = 0;
    emit_pair(a, boff, r, cA, own && cA < a.nx, own && cA + 1 < a.nx,
              eA, uA, vA_, dA, eB, uB, vB_, dB, bad);
    if (a.samp_ptr && (a.rec_g || a.rec_n)) {
        int sp = a.samp_ptr[gw];
        const int se = a.samp_ptr[gw + 1];
        if (sp < se) emit_samples(a, b, sp, se, r, c0, lane, eA, uA, vA_, eB, uB, vB_);
    }
    if (bad) atomicOr(a.err, ERRF_NONFINITE);
}

// y-sweep alone: one warp per (strip of 64 columns, S rows).
__global__ void __launch_bounds__(128) k_ysweep(const StepArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int b = blockIdx.y;
    if (gw >= a.nstrips * a.nseg) return;
    if (a.limit && a.step > a.limit[b]) return;
    const int strip = gw % a.nstrips, seg = gw / a.nstrips;
    const int c0 = strip * XWIN;
    const int cA = c0 + 2 * lane;
    const int r0 = seg * a.S, r1 = min(r0 + a.S, a.ny);
    const size_t boff = (size_t)b * a.plane;
    const SweepConst K = sweep_const(a);
    const bool vA = cA < a.nx, vB = cA + 1 < a.nx;
    int sp = 0, se = 0;
    if (a.samp_ptr && (a.rec_g || a.rec_n)) { sp = a.samp_ptr[gw]; se = a.samp_ptr[gw + 1]; }
    YMarch ya, yb;
    ya.init();
    yb.init();
    int bad = 0;
    for (int k = r0 - 3; k < r1 + 3; ++k) {
        float eA, uA, vA_, dA, eB, uB, vB_, dB;
        load_pair(a, boff, k, cA, eA, uA, vA_, dA, eB, uB, vB_, dB);
        const float4 m2 = __ldg(a.ymet + min(max(k - 2, 0), a.ny - 1));
        float oeA, owA, otA, oeB, owB, otB;
        const float odA = ya.dd3, odB = yb.dd3;
        ya.push(eA, vA_, uA, dA, m2, K, oeA, owA, otA);
        yb.push(eB, vB_, uB, dB, m2, K, oeB, owB, otB);
        const int r = k - 3;
        if (r >= r0 && r < r1) {
            emit_pair(a, boff, r, cA, vA, vB, oeA, otA, owA, odA, oeB, otB, owB, odB, bad);
            if (sp < se) emit_samples(a, b, sp, se, r, c0, lane, oeA, otA, owA, oeB, otB, owB);
        }
    }
    if (bad) atomicOr(a.err, ERRF_NONFINITE);
}

cudaError_t launch_step_fused(const StepArgs& a, int batch, int wpb, cudaStream_t s) {
    (void)wpb;
    const int nw = a.nstrips * a.nseg;
    const dim3 grid((nw + 3) / 4, batch);
    if (a.sph) k_step_fused<true><<<grid, 128, 0, s>>>(a);
    else k_step_fused<false><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_xsweep(const StepArgs& a, int batch, cudaStream_t s) {
    const int nw = a.nstrips * a.ny;
    const dim3 grid((nw + 3) / 4, batch);
    if (a.sph) k_xsweep<true><<<grid, 128, 0, s>>>(a);
    else k_xsweep<false><<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ysweep(const StepArgs& a, int batch, cudaStream_t s) {
    const int nw = a.nstrips * a.nseg;
    const dim3 grid((nw + 3) / 4, batch);
    k_ysweep<<<grid, 128, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace cliffs
