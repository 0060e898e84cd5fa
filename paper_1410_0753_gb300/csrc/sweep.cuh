// Device building blocks of the split shallow-water step (arXiv 1410.0753, "Numerics").
//
// One sweep of one line applies, in order, the inundation steps of section "Inundation
// algorithm": (a) mark dry nodes (h < h_min), (b) add a dry node to a wet neighbour's
// segment when h_j - d_j + d_i > h_min, with height h_min and the neighbour's velocities,
// (c) treat wet/dry interfaces as reflecting walls half a node from the wet node (mirror
// ghosts), (d) update every wet node by eq. (solver2), (e) limit a newly wetted node to half
// its neighbour's height and to its neighbour's speed. The readings where the paper is
// silent (tie-break in (b), ghost values, friction law and clamp, spherical terms) are the
// ones the FP64 oracle states; this file restates them for FP32.
//
// FP32 form. eq. (solver2) is written in the paper on the Riemann invariants p, q = u +- 2c
// (c = sqrt(g h)). In deep water c is ~200 m/s while a wave changes it by ~1e-4, below the
// FP32 resolution of p, so the kernels keep eta (not h) and evaluate the algebraically
// identical perturbation form of eq. (eqQ):
//   Q(b,a) dx = 1/2 (lam_b + lam_a)(w_b - w_a) +- (w_b + w_a)(c_b - c_a) + g (eta_b - eta_a),
//   c_b - c_a = g ((eta_b - eta_a) + (d_b - d_a)) / (c_b + c_a),
// and recover by increments (eqs. (stateu), (stateh)): du = (dp + dq)/2, dc = (dp - dq)/4,
// deta = dc (2c + dc)/g. At rest every term is exactly zero, so the lake at rest is kept
// bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cliffs {

constexpr float GRAV = 9.81f;
constexpr float INV_GRAV = 1.0f / 9.81f;
constexpr float OUTSIDE_D = -1.0e30f;     // depth given to nodes beyond the domain edge
constexpr unsigned FULL = 0xffffffffu;
constexpr int XWIN = 64;                  // columns a warp holds in an x-sweep (2 per lane)
constexpr int XOUT = 56;                  // columns it can finish: 4-column halo per side

struct SweepConst {
    float hmin;       // h_min ('ground')
    float dwall;      // nodes with d < dwall are permanent walls (-FLT_MAX when itopo != 0)
    float half_dt;    // dt / 2
    float dt_gn2;     // dt * g * Manning n^2 (0 disables friction)
    int   transverse; // eq. (pq3) on/off
};

// post-(b) state of a node
struct Node {
    float eta, w, t, d, c;   // c = sqrt(g h), meaningful only when wet
    bool  wet;               // wet after (b)
    int   dir;               // -1 / +1: wetted in (b) from the left / right neighbour
};

struct Flux { float p, q, t; };

__device__ __forceinline__ bool wet_mark(float eta, float d, const SweepConst& K) {
    return (d >= K.dwall) && (eta + d >= K.hmin);              // (a): dry when h < h_min
}

// (b) for a node that is dry at the start of the sweep. Neighbours: start-of-sweep eta, w,
// t and wet mark. The wetter neighbour (larger eta) wins, the left one on a tie.
__device__ __forceinline__ void flood(Node& n, float eL, float wL, float tL, bool oL,
                                      float eR, float wR, float tR, bool oR,
                                      const SweepConst& K) {
    if (n.wet) return;
    n.w = 0.f;                                                 // a dry node is at rest
    n.t = 0.f;
    if (!(n.d >= K.dwall)) return;
    const bool okL = oL && (eL + n.d > K.hmin);
    const bool okR = oR && (eR + n.d > K.hmin);
    if (okL || okR) {
        const bool useR = okR && (!okL || eR > eL);
        n.eta = K.hmin - n.d;                                  // height h_min
        n.w = useR ? wR : wL;
        n.t = useR ? tR : tL;
        n.wet = true;
        n.dir = useR ? 1 : -1;
    }
}

// eq. (eqQ) for p and q and the eq. (pq3) flux for t across the interface between node a
// (left) and node b (right), perturbation form, divided by the interval.
__device__ __forceinline__ Flux iface(const Node& a, const Node& b, float inv_ds) {
    const float deta = b.eta - a.eta;
    const float sc = b.c + a.c;
    const float dc = __fdividef(GRAV * (deta + (b.d - a.d)), sc);
    const float sw = b.w + a.w;
    const float hdw = 0.5f * (b.w - a.w);
    const float y = sw * dc;
    const float z = GRAV * deta;
    Flux F;
    F.p = fmaf(hdw, sw + sc, z + y) * inv_ds;
    F.q = fmaf(hdw, sw - sc, z - y) * inv_ds;
    F.t = 0.5f * sw * (b.t - a.t) * inv_ds;
    return F;
}

// The same fluxes when the neighbour is the mirror ghost of n (eta_g = eta, d_g = d,
// w_g = -w, t_g = t): a wall on the left of n, or on its right.
__device__ __forceinline__ Flux ghost_left(const Node& n, float inv_ds) {
    const float f = 2.f * n.w * n.c * inv_ds;
    return Flux{f, -f, 0.f};
}
__device__ __forceinline__ Flux ghost_right(const Node& n, float inv_ds) {
    const float f = 2.f * n.w * n.c * inv_ds;
    return Flux{-f, f, 0.f};
}

// (d): eq. (solver2) at a wet node given its left and right interface fluxes.
//   k2 = dt^2 / (dx_{j-1} + dx_j); sdt = dt tan(phi) / R in the spherical y-sweep, else 0.
// Friction: alpha = g n^2 w sqrt(w^2 + t^2) / h^(4/3) at time level n on both p and q,
// clamped so that |alpha dt| <= |w|.
__device__ __forceinline__ void node_update(const Node& n, const Flux& L, const Flux& R,
                                            float k2, float sdt, const SweepConst& K,
                                            float& eta2, float& w2, float& t2) {
    const float lp = n.w + n.c;
    const float lq = n.w - n.c;
    float adt = 0.f;
    if (K.dt_gn2 > 0.f) {
        const float h = n.eta + n.d;
        const float s = sqrtf(fmaf(n.w, n.w, n.t * n.t));
        adt = __fdividef(K.dt_gn2 * n.w * s, h * cbrtf(h));
        if (fabsf(adt) > fabsf(n.w)) adt = n.w;
    }
    const float src = sdt * n.c * n.w;
    const float dp = -K.half_dt * (L.p + R.p) + lp * k2 * (R.p - L.p) - adt + src;
    const float dq = -K.half_dt * (L.q + R.q) + lq * k2 * (R.q - L.q) - adt - src;
    const float du = 0.5f * (dp + dq);
    const float dc = 0.25f * (dp - dq);
    w2 = n.w + du;
    eta2 = n.eta + dc * (2.f * n.c + dc) * INV_GRAV;
    t2 = K.transverse ? n.t - K.half_dt * (L.t + R.t) + n.w * k2 * (R.t - L.t) : n.t;
}

// (e): a node wetted in (b) against its source neighbour's state after (d).
__device__ __forceinline__ void cushion(float& e, float& w, float d, float hj, float wj) {
    const float hi = e + d;
    if (hi > 0.5f * hj) e = 0.5f * hj - d;
    if (fabsf(w) > fabsf(wj)) w = wj;
}

struct XMet { float inv_l, inv_r, k2; };   // 1/dx_{j-1}, 1/dx_j, dt^2/(dx_{j-1}+dx_j)

// x-sweep of one row segment held by a warp: lane l has nodes A (window column 2l) and
// B (2l+1). Neighbours across lanes come by shuffles. On return (eA,wA,tA) and (eB,wB,tB)
// hold the sweep result; it is valid for window columns 4..59 (the outer 4 columns on each
// side lack their 3-node dependency radius).
__device__ __forceinline__ void xsweep_pair(float& eA, float& wA, float& tA, float dA,
                                            float& eB, float& wB, float& tB, float dB,
                                            const XMet& mA, const XMet& mB,
                                            const SweepConst& K, int lane) {
    const bool oA = wet_mark(eA, dA, K), oB = wet_mark(eB, dB, K);
    const unsigned bA = __ballot_sync(FULL, oA), bB = __ballot_sync(FULL, oB);
    Node nA{eA, wA, tA, dA, 0.f, oA, 0};
    Node nB{eB, wB, tB, dB, 0.f, oB, 0};
    if ((bA & bB) != FULL) {
        const float eL = __shfl_up_sync(FULL, eB, 1), wL = __shfl_up_sync(FULL, wB, 1);
        const float tL = __shfl_up_sync(FULL, tB, 1);
        const float eR = __shfl_down_sync(FULL, eA, 1), wR = __shfl_down_sync(FULL, wA, 1);
        const float tR = __shfl_down_sync(FULL, tA, 1);
        const bool oL = lane > 0 && ((bB >> (lane - 1)) & 1u);
        const bool oR = lane < 31 && ((bA >> (lane + 1)) & 1u);
        flood(nA, eL, wL, tL, oL, eB, wB, tB, oB, K);
        flood(nB, eA, wA, tA, oA, eR, wR, tR, oR, K);
    }
    nA.c = sqrtf(GRAV * (nA.eta + nA.d));
    nB.c = sqrtf(GRAV * (nB.eta + nB.d));
    // post-(b) state of the right neighbour of B (node A of lane + 1)
    Node nR;
    nR.eta = __shfl_down_sync(FULL, nA.eta, 1);
    nR.w = __shfl_down_sync(FULL, nA.w, 1);
    nR.t = __shfl_down_sync(FULL, nA.t, 1);
    nR.d = __shfl_down_sync(FULL, nA.d, 1);
    nR.c = __shfl_down_sync(FULL, nA.c, 1);
    const unsigned wA1 = __ballot_sync(FULL, nA.wet), wB1 = __ballot_sync(FULL, nB.wet);
    nR.wet = lane < 31 && ((wA1 >> (lane + 1)) & 1u);
    const bool wetL = lane > 0 && ((wB1 >> (lane - 1)) & 1u);
    const Flux fAB = iface(nA, nB, mA.inv_r);
    const Flux fBR = iface(nB, nR, mB.inv_r);
    Flux fLA;
    fLA.p = __shfl_up_sync(FULL, fBR.p, 1);
    fLA.q = __shfl_up_sync(FULL, fBR.q, 1);
    fLA.t = __shfl_up_sync(FULL, fBR.t, 1);
    float e2A = nA.eta, w2A = nA.w, t2A = nA.t;
    float e2B = nB.eta, w2B = nB.w, t2B = nB.t;
    if (nA.wet) {
        const Flux L = wetL ? fLA : ghost_left(nA, mA.inv_l);
        const Flux R = nB.wet ? fAB : ghost_right(nA, mA.inv_r);
        node_update(nA, L, R, mA.k2, 0.f, K, e2A, w2A, t2A);
    }
    if (nB.wet) {
        const Flux L = nA.wet ? fAB : ghost_left(nB, mB.inv_l);
        const Flux R = nR.wet ? fBR : ghost_right(nB, mB.inv_r);
        node_update(nB, L, R, mB.k2, 0.f, K, e2B, w2B, t2B);
    }
    if (__any_sync(FULL, (nA.dir | nB.dir) != 0)) {
        const float hA = e2A + dA, hB = e2B + dB;
        const float hL = __shfl_up_sync(FULL, hB, 1), wLn = __shfl_up_sync(FULL, w2B, 1);
        const float hR = __shfl_down_sync(FULL, hA, 1), wRn = __shfl_down_sync(FULL, w2A, 1);
        const float w2A0 = w2A, w2B0 = w2B;
        if (nA.dir < 0) cushion(e2A, w2A, dA, hL, wLn);
        else if (nA.dir > 0) cushion(e2A, w2A, dA, hB, w2B0);
        if (nB.dir < 0) cushion(e2B, w2B, dB, hA, w2A0);
        else if (nB.dir > 0) cushion(e2B, w2B, dB, hR, wRn);
    }
    eA = e2A; wA = w2A; tA = t2A;
    eB = e2B; wB = w2B; tB = t2B;
}

// y-sweep of one column as a march down the rows. Each push takes the sweep input of row k
// and returns the finished result of row k - 3: (b) runs on row k-1, the interface flux
// between rows k-2 and k-1 is formed once and shared, (d) runs on row k-2 and (e) on k-3.
struct YMarch {
    float e2, w2, t2, d2; bool o2;          // input, row k-2
    float e1, w1, t1, d1; bool o1;          // input, row k-1
    Node  b2;                               // after (b), row k-2
    Flux  f3; bool wet3;                    // flux (k-3 | k-2), wet mark of row k-3 after (b)
    float de4, dw4, dd4;                    // after (d), row k-4
    float de3, dw3, dt3, dd3; int dir3;     // after (d), row k-3

    __device__ __forceinline__ void init() {
        e2 = w2 = t2 = 0.f; d2 = OUTSIDE_D; o2 = false;
        e1 = w1 = t1 = 0.f; d1 = OUTSIDE_D; o1 = false;
        b2 = Node{0.f, 0.f, 0.f, OUTSIDE_D, 0.f, false, 0};
        f3 = Flux{0.f, 0.f, 0.f}; wet3 = false;
        de4 = dw4 = 0.f; dd4 = OUTSIDE_D;
        de3 = dw3 = dt3 = 0.f; dd3 = OUTSIDE_D; dir3 = 0;
    }

    // m2: metric of row k-2 (inv_l, inv_r, k2, sdt); returns (oe, ow, ot) of row k-3
    __device__ __forceinline__ void push(float e0, float w0, float t0, float d0, float4 m2,
                                         const SweepConst& K, float& oe, float& ow, float& ot) {
        const bool o0 = wet_mark(e0, d0, K);
        Node b1{e1, w1, t1, d1, 0.f, o1, 0};
        flood(b1, e2, w2, t2, o2, e0, w0, t0, o0, K);
        b1.c = sqrtf(GRAV * (b1.eta + b1.d));
        const Flux f2 = iface(b2, b1, m2.y);
        float ne = b2.eta, nw = b2.w, nt = b2.t;
        if (b2.wet) {
            const Flux L = wet3 ? f3 : ghost_left(b2, m2.x);
            const Flux R = b1.wet ? f2 : ghost_right(b2, m2.y);
            node_update(b2, L, R, m2.z, m2.w, K, ne, nw, nt);
        }
        float fe = de3, fw = dw3;
        if (dir3 != 0) {
            const float hj = (dir3 < 0) ? de4 + dd4 : ne + b2.d;
            const float wj = (dir3 < 0) ? dw4 : nw;
            cushion(fe, fw, dd3, hj, wj);
        }
        oe = fe; ow = fw; ot = dt3;
        de4 = de3; dw4 = dw3; dd4 = dd3;
        de3 = ne; dw3 = nw; dt3 = nt; dd3 = b2.d; dir3 = b2.dir;
        f3 = f2; wet3 = b2.wet;
        b2 = b1;
        e2 = e1; w2 = w1; t2 = t1; d2 = d1; o2 = o1;
        e1 = e0; w1 = w0; t1 = t0; d1 = d0; o1 = o0;
    }
};

}  // namespace cliffs
