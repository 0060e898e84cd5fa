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
//
// Layout of the work. Every lane owns two neighbouring nodes (columns A and B of its pair)
// and evaluates the update of both with packed FP32x2 instructions (add/mul/fma .f32x2).
// Steps (b), (c) and (e) are corrections applied per node, and only inside warp-uniform
// branches taken when some node of the warp needs them (a dry node that can flood, a wet
// node next to a dry one, a newly wetted node), so open water runs the update alone.
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
    float inv_dt2;    // 1 / dt^2 (eq. (solver1): 1/(dx_{j-1}+dx_j) = k2 / dt^2)
};

// ------------------------------------------------------------------ packed FP32x2
__device__ __forceinline__ float2 v2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, v2(-1.f), a); }

#ifndef CLIFFS_IEEE_MATH
// Hardware approximations (MUFU): one instruction each.
__device__ __forceinline__ float rsqrt_approx(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// sqrt(x) for x >= 0 (x = 0 gives 0 through the 1e-30 floor)
__device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrt_approx(fmaxf(x, 1e-30f)); }
__device__ __forceinline__ float div_pos(float a, float b) { return a * rcp_approx(b); }
// base-2 logarithm (log2(0) = -inf) and exponential (2^-inf = 0)
__device__ __forceinline__ float log2_fast(float x) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float exp2_fast(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
#else
// Build option CLIFFS_IEEE_MATH: correctly rounded square root, reciprocal and quotient
// (IEEE round-to-nearest) in place of the hardware approximations.
__device__ __forceinline__ float rsqrt_approx(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ float rcp_approx(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float sqrt_pos(float x) { return __fsqrt_rn(x); }
__device__ __forceinline__ float div_pos(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float log2_fast(float x) { return log2f(x); }
__device__ __forceinline__ float exp2_fast(float x) { return exp2f(x); }
#endif

// c = sqrt(g h) of both nodes (h > 0 for wet nodes; dry nodes give NaN and are not used)
__device__ __forceinline__ float2 wave_speed2(float2 h) {
    const float2 gh = mul2(v2(GRAV), h);
#ifndef CLIFFS_IEEE_MATH
    return mul2(gh, make_float2(rsqrt_approx(gh.x), rsqrt_approx(gh.y)));
#else
    return make_float2(__fsqrt_rn(gh.x), __fsqrt_rn(gh.y));
#endif
}
__device__ __forceinline__ float wave_speed(float h) {
    const float gh = GRAV * h;
#ifndef CLIFFS_IEEE_MATH
    return gh * rsqrt_approx(gh);
#else
    return __fsqrt_rn(gh);
#endif
}

__device__ __forceinline__ bool wet_mark(float eta, float d, const SweepConst& K) {
    return (d >= K.dwall) && (eta + d >= K.hmin);              // (a): dry when h < h_min
}

// Friction (reading 4: Manning at time level n, alpha = g n^2 w sqrt(w^2 + t^2) / h^(4/3),
// clamped so that |alpha dt| <= |w|), as alpha dt = w k with
//   k = min(dt g n^2 sqrt(s2) h^(-4/3), 1) = 2^min(ex, 0),
//   ex = log2(dt g n^2) + log2(s2) / 2 - 4/3 log2(h),   s2 = w^2 + t^2:
// one power of two carries the clamp (ex >= 0: clamped, alpha dt = w). s2 = 0 gives k = 0.
// The adjoint's recomputation calls the same function, so both take the same clamp decision.
__device__ __forceinline__ float2 fric_k2(float2 w, float2 t, float2 h, float dt_gn2, float2& s2, float2& ex) {
    s2 = fma2(w, w, mul2(t, t));
    const float2 ls = make_float2(log2_fast(s2.x), log2_fast(s2.y));
    const float2 lh = make_float2(log2_fast(h.x), log2_fast(h.y));
    ex = fma2(v2(0.5f), ls, fma2(v2(-4.0f / 3.0f), lh, v2(log2_fast(dt_gn2))));
    return make_float2(exp2_fast(fminf(ex.x, 0.f)), exp2_fast(fminf(ex.y, 0.f)));
}
__device__ __forceinline__ float fric_k(float w, float t, float h, float dt_gn2, float& s2, float& ex) {
    float2 s2p, exp_;
    const float2 k = fric_k2(v2(w), v2(t), v2(h), dt_gn2, s2p, exp_);
    s2 = s2p.x;
    ex = exp_.x;
    return k.x;
}

struct Flux2 { float2 p, q, t; };

// eq. (eqQ) for p and q and the eq. (pq3) flux for t across two interfaces at once, each
// between a left node a and a right node b, perturbation form, divided by the interval.
__device__ __forceinline__ Flux2 iface2(float2 ea, float2 wa, float2 ta, float2 da, float2 ca,
                                        float2 eb, float2 wb, float2 tb, float2 db, float2 cb,
                                        float2 inv_ds) {
    const float2 deta = sub2(eb, ea);
    const float2 sc = add2(cb, ca);
    const float2 num = mul2(v2(GRAV), add2(deta, sub2(db, da)));
#ifndef CLIFFS_IEEE_MATH
    const float2 dc = mul2(num, make_float2(rcp_approx(sc.x), rcp_approx(sc.y)));
#else
    const float2 dc = make_float2(__fdiv_rn(num.x, sc.x), __fdiv_rn(num.y, sc.y));
#endif
    const float2 sw = add2(wb, wa);
    const float2 hdw = mul2(v2(0.5f), sub2(wb, wa));
    const float2 y = mul2(sw, dc);
    const float2 z = mul2(v2(GRAV), deta);
    Flux2 F;
    F.p = mul2(fma2(hdw, add2(sw, sc), add2(z, y)), inv_ds);
    F.q = mul2(fma2(hdw, sub2(sw, sc), sub2(z, y)), inv_ds);
    F.t = mul2(mul2(mul2(v2(0.5f), sw), sub2(tb, ta)), inv_ds);
    return F;
}

// Fluxes when the neighbour is the mirror ghost of the node (eta_g = eta, d_g = d,
// w_g = -w, t_g = t): a wall on its left gives (2wc, -2wc, 0)/dx, on its right the negation.
__device__ __forceinline__ void ghost_left(float w, float c, float inv, float& p, float& q, float& t) {
    const float f = 2.f * w * c * inv;
    p = f; q = -f; t = 0.f;
}
__device__ __forceinline__ void ghost_right(float w, float c, float inv, float& p, float& q, float& t) {
    const float f = 2.f * w * c * inv;
    p = -f; q = f; t = 0.f;
}

// Open outer edge (no condition in the paper): the ghost beyond a wet edge node carries the
// node's outgoing Riemann invariant and the incoming invariant of still water at its depth,
// c0 = sqrt(g max(d, 0)). With delta = c - c0 (= g eta / (c + c0) for d > 0, else c):
//   right end (p leaves, q = -2 c0 enters): w_g = w/2 + delta, c_g = c + w/4 - delta/2;
//   left end  (q leaves, p = 2 c0 enters):  w_g = w/2 - delta, c_g = c - w/4 - delta/2;
// eta_g = eta + (c_g - c)(c_g + c)/g, the node's depth and transverse velocity. A ghost
// whose c_g would be negative is dry (c_g = 0). At rest (eta = w = 0) the ghost equals the
// node exactly, so the edge flux vanishes.
__device__ __forceinline__ void open_ghost(float e, float w, float d, float c, bool right,
                                           float& eg, float& wg, float& cg) {
    const bool deep = d > 0.f;
    const float c0 = deep ? wave_speed(d) : 0.f;
    const float delta = deep ? div_pos(GRAV * e, c + c0) : c;
    const float s = right ? 1.f : -1.f;
    wg = fmaf(0.5f, w, s * delta);
    float gam = fmaf(s * 0.25f, w, -0.5f * delta);           // c_g - c
    if (c + gam < 0.f) gam = -c;
    cg = c + gam;
    eg = fmaf(gam * (2.f * c + gam), INV_GRAV, e);
}

// Fluxes at the open edge of a node (scalar; the .x lane of the packed form). Kept out of
// line: open edges are rare, and inlined they would take registers from the sweeps.
static __device__ __noinline__ void open_flux(float e, float w, float t, float d, float c, float inv, bool right,
                                          float& p, float& q, float& tf, float& eg, float& wg, float& cg) {
    open_ghost(e, w, d, c, right, eg, wg, cg);
    const Flux2 F = right ? iface2(v2(e), v2(w), v2(t), v2(d), v2(c), v2(eg), v2(wg), v2(t), v2(d), v2(cg), v2(inv))
                          : iface2(v2(eg), v2(wg), v2(t), v2(d), v2(cg), v2(e), v2(w), v2(t), v2(d), v2(c), v2(inv));
    p = F.p.x; q = F.q.x; tf = F.t.x;
}

// (d): eq. (solver2) at two nodes given their left and right interface fluxes.
//   k2 = dt^2 / (dx_{j-1} + dx_j); sdt = dt tan(phi) / R in the spherical y-sweep (SRC).
// Friction (fric_k2) at time level n on both p and q.
// With S1, eq. (solver1): the first-order term is dt Q(j+1, j-1) over dx_{j-1} + dx_j, given
// as the flux F1 between the two neighbours (per unit length) instead of the mean of L and R.
template <bool SRC, bool FRIC, bool S1 = false>
__device__ __forceinline__ void node_update2(float2 e, float2 w, float2 t, float2 d, float2 c,
                                             const Flux2& L, const Flux2& R, float2 k2, float2 sdt,
                                             const SweepConst& K,
                                             float2& e2, float2& w2, float2& t2, const Flux2* F1 = nullptr) {
    const float2 lp = add2(w, c);
    const float2 lq = sub2(w, c);
    const float2 nh = v2(-K.half_dt);
    const float2 ndt = v2(-2.f * K.half_dt);
    float2 dp, dq;
    if (S1) {
        dp = fma2(mul2(lp, k2), sub2(R.p, L.p), mul2(ndt, F1->p));
        dq = fma2(mul2(lq, k2), sub2(R.q, L.q), mul2(ndt, F1->q));
    } else {
        dp = fma2(mul2(lp, k2), sub2(R.p, L.p), mul2(nh, add2(L.p, R.p)));
        dq = fma2(mul2(lq, k2), sub2(R.q, L.q), mul2(nh, add2(L.q, R.q)));
    }
    if (FRIC) {
        float2 s2, ex;
        const float2 adt = mul2(w, fric_k2(w, t, add2(e, d), K.dt_gn2, s2, ex));
        dp = sub2(dp, adt);
        dq = sub2(dq, adt);
    }
    if (SRC) {
        const float2 src = mul2(mul2(sdt, c), w);
        dp = add2(dp, src);
        dq = sub2(dq, src);
    }
    const float2 du = mul2(v2(0.5f), add2(dp, dq));
    const float2 dc = mul2(v2(0.25f), sub2(dp, dq));
    w2 = add2(w, du);
    e2 = fma2(mul2(dc, fma2(v2(2.f), c, dc)), v2(INV_GRAV), e);
    const float2 tn = S1 ? fma2(mul2(w, k2), sub2(R.t, L.t), fma2(ndt, F1->t, t))
                         : fma2(mul2(w, k2), sub2(R.t, L.t), fma2(nh, add2(L.t, R.t), t));
    t2 = K.transverse ? tn : t;
}

// (e): a node wetted in (b) against its source neighbour's state after (d).
__device__ __forceinline__ void cushion(float& e, float& w, float d, float hj, float wj) {
    const float hi = e + d;
    if (hi > 0.5f * hj) e = 0.5f * hj - d;
    if (fabsf(w) > fabsf(wj)) w = wj;
}

// (b) for one node i, dry at the start of the sweep and not a wall, with neighbours L and R
// (start-of-sweep eta, w, t and wet marks): the wetter neighbour (larger eta) wins, the
// left one on a tie. Returns the direction of the source (-1, +1) or 0.
__device__ __forceinline__ int flood1(float& e, float& w, float& t, float d,
                                      float eL, float wL, float tL, bool oL,
                                      float eR, float wR, float tR, bool oR, float hmin) {
    const bool okL = oL && (eL + d > hmin);
    const bool okR = oR && (eR + d > hmin);
    if (!(okL || okR)) return 0;
    const bool useR = okR && (!okL || eR > eL);
    e = hmin - d;                                              // height h_min
    w = useR ? wR : wL;
    t = useR ? tR : tL;
    return useR ? 1 : -1;
}

struct XMet2 { float2 inv_l, inv_r, k2; };   // per pair: 1/dx_{j-1}, 1/dx_j, dt^2/(dx_{j-1}+dx_j)

// x-sweep of one row segment held by a warp: lane l has nodes A = window column 2l (.x)
// and B = 2l + 1 (.y). Neighbours across lanes come by shuffles. On return (E, W, T) hold
// the sweep result; it is valid for window columns 4..59 (the outer 4 columns on each side
// lack their 3-node dependency radius), and up to the window's edge on a side where that
// edge is the domain's (bounded). W is the velocity along the row, T across it.
// ends: this lane's nodes at open outer edges, bits 1 A left, 2 A right, 4 B left, 8 B right.
template <bool FRIC, bool S1 = false, bool OPEN = false>
__device__ __forceinline__ void xsweep2(float2& E, float2& W, float2& T, float2 D, const XMet2& m,
                                        const SweepConst& K, int lane, unsigned ends = 0u, bool bounded = false) {
    const bool oA = wet_mark(E.x, D.x, K), oB = wet_mark(E.y, D.y, K);
    const unsigned bA = __ballot_sync(FULL, oA), bB = __ballot_sync(FULL, oB);
    // bounded: the window starts or ends at the domain's edge, where the first (last) lane's
    // outer neighbour is the wall's mirror ghost: the general path, which takes it so
    const bool allwet = (bA & bB) == FULL && !bounded;
    bool wA = oA, wB = oB;                 // wet after (b)
    int dirA = 0, dirB = 0;
    if (!allwet) {
        if (!oA) { W.x = 0.f; T.x = 0.f; }   // (a): a dry node is at rest
        if (!oB) { W.y = 0.f; T.y = 0.f; }
        const bool oL = lane > 0 && ((bB >> (lane - 1)) & 1u);
        const bool oR = lane < 31 && ((bA >> (lane + 1)) & 1u);
        const bool cA = !oA && D.x >= K.dwall && (oL || oB);
        const bool cB = !oB && D.y >= K.dwall && (oA || oR);
        if (__any_sync(FULL, cA || cB)) {
            const float eL = __shfl_up_sync(FULL, E.y, 1), eR = __shfl_down_sync(FULL, E.x, 1);
            const bool qA = cA && ((oL && eL + D.x > K.hmin) || (oB && E.y + D.x > K.hmin));
            const bool qB = cB && ((oA && E.x + D.y > K.hmin) || (oR && eR + D.y > K.hmin));
            if (__any_sync(FULL, qA || qB)) {
                const float wL = __shfl_up_sync(FULL, W.y, 1), tL = __shfl_up_sync(FULL, T.y, 1);
                const float wR = __shfl_down_sync(FULL, W.x, 1), tR = __shfl_down_sync(FULL, T.x, 1);
                const float eA0 = E.x, wA0 = W.x, tA0 = T.x;     // A as the source of B
                if (qA) {
                    dirA = flood1(E.x, W.x, T.x, D.x, eL, wL, tL, oL, E.y, W.y, T.y, oB, K.hmin);
                    wA = true;
                }
                if (qB) {
                    dirB = flood1(E.y, W.y, T.y, D.y, eA0, wA0, tA0, oA, eR, wR, tR, oR, K.hmin);
                    wB = true;
                }
            }
        }
    }
    const float2 C = wave_speed2(add2(E, D));
    // post-(b) state of the right neighbour of B (node A of lane + 1)
    const float eR = __shfl_down_sync(FULL, E.x, 1), wR = __shfl_down_sync(FULL, W.x, 1);
    const float tR = __shfl_down_sync(FULL, T.x, 1), dR = __shfl_down_sync(FULL, D.x, 1);
    const float cR = __shfl_down_sync(FULL, C.x, 1);
    // right interfaces of A and B: (A|B) and (B|R)
    Flux2 FR = iface2(E, W, T, D, C, make_float2(E.y, eR), make_float2(W.y, wR),
                      make_float2(T.y, tR), make_float2(D.y, dR), make_float2(C.y, cR), m.inv_r);
    // left interfaces: (B_{l-1}|A) from the lane below, and (A|B)
    Flux2 FL;
    FL.p = make_float2(__shfl_up_sync(FULL, FR.p.y, 1), FR.p.x);
    FL.q = make_float2(__shfl_up_sync(FULL, FR.q.y, 1), FR.q.x);
    FL.t = make_float2(__shfl_up_sync(FULL, FR.t.y, 1), FR.t.x);
    bool wetL = true, wetR = true;
    if (!allwet) {
        // (c): walls between wet and dry nodes
        const unsigned w1A = __ballot_sync(FULL, wA), w1B = __ballot_sync(FULL, wB);
        wetL = lane > 0 && ((w1B >> (lane - 1)) & 1u);
        wetR = lane < 31 && ((w1A >> (lane + 1)) & 1u);
        if (!wetL) ghost_left(W.x, C.x, m.inv_l.x, FL.p.x, FL.q.x, FL.t.x);
        if (!wB) ghost_right(W.x, C.x, m.inv_r.x, FR.p.x, FR.q.x, FR.t.x);
        if (!wA) ghost_left(W.y, C.y, m.inv_l.y, FL.p.y, FL.q.y, FL.t.y);
        if (!wetR) ghost_right(W.y, C.y, m.inv_r.y, FR.p.y, FR.q.y, FR.t.y);
    }
    float2 gE = v2(0.f), gW = v2(0.f), gC = v2(0.f);   // open-edge ghosts of A (.x) and B (.y)
    if (OPEN && ends) {
        if ((ends & 1u) && wA) open_flux(E.x, W.x, T.x, D.x, C.x, m.inv_l.x, false, FL.p.x, FL.q.x, FL.t.x, gE.x, gW.x, gC.x);
        if ((ends & 2u) && wA) open_flux(E.x, W.x, T.x, D.x, C.x, m.inv_r.x, true, FR.p.x, FR.q.x, FR.t.x, gE.x, gW.x, gC.x);
        if ((ends & 4u) && wB) open_flux(E.y, W.y, T.y, D.y, C.y, m.inv_l.y, false, FL.p.y, FL.q.y, FL.t.y, gE.y, gW.y, gC.y);
        if ((ends & 8u) && wB) open_flux(E.y, W.y, T.y, D.y, C.y, m.inv_r.y, true, FR.p.y, FR.q.y, FR.t.y, gE.y, gW.y, gC.y);
    }
    Flux2 F1;
    if (S1) {
        // eq. (solver1): flux between the two neighbours of each node, mirror ghosts for dry ones
        float2 le = make_float2(__shfl_up_sync(FULL, E.y, 1), E.x), lw = make_float2(__shfl_up_sync(FULL, W.y, 1), W.x);
        float2 lt = make_float2(__shfl_up_sync(FULL, T.y, 1), T.x), ld = make_float2(__shfl_up_sync(FULL, D.y, 1), D.x);
        float2 lc = make_float2(__shfl_up_sync(FULL, C.y, 1), C.x);
        float2 re = make_float2(E.y, eR), rw = make_float2(W.y, wR), rt = make_float2(T.y, tR);
        float2 rd = make_float2(D.y, dR), rc = make_float2(C.y, cR);
        if (!allwet) {
            if (!wetL) { le.x = E.x; lw.x = -W.x; lt.x = T.x; ld.x = D.x; lc.x = C.x; }
            if (!wB) { re.x = E.x; rw.x = -W.x; rt.x = T.x; rd.x = D.x; rc.x = C.x; }
            if (!wA) { le.y = E.y; lw.y = -W.y; lt.y = T.y; ld.y = D.y; lc.y = C.y; }
            if (!wetR) { re.y = E.y; rw.y = -W.y; rt.y = T.y; rd.y = D.y; rc.y = C.y; }
        }
        if (OPEN && ends) {                // an open edge's neighbour is its ghost
            if (ends & 1u) { le.x = gE.x; lw.x = gW.x; lt.x = T.x; ld.x = D.x; lc.x = gC.x; }
            if (ends & 2u) { re.x = gE.x; rw.x = gW.x; rt.x = T.x; rd.x = D.x; rc.x = gC.x; }
            if (ends & 4u) { le.y = gE.y; lw.y = gW.y; lt.y = T.y; ld.y = D.y; lc.y = gC.y; }
            if (ends & 8u) { re.y = gE.y; rw.y = gW.y; rt.y = T.y; rd.y = D.y; rc.y = gC.y; }
        }
        F1 = iface2(le, lw, lt, ld, lc, re, rw, rt, rd, rc, mul2(m.k2, v2(K.inv_dt2)));
    }
    float2 E2, W2, T2;
    node_update2<false, FRIC, S1>(E, W, T, D, C, FL, FR, m.k2, v2(0.f), K, E2, W2, T2, &F1);
    if (!allwet) {
        if (!wA) { E2.x = E.x; W2.x = W.x; T2.x = T.x; }
        if (!wB) { E2.y = E.y; W2.y = W.y; T2.y = T.y; }
        if (__any_sync(FULL, (dirA | dirB) != 0)) {
            const float hA = E2.x + D.x, hB = E2.y + D.y;
            const float hL = __shfl_up_sync(FULL, hB, 1), wLn = __shfl_up_sync(FULL, W2.y, 1);
            const float hR = __shfl_down_sync(FULL, hA, 1), wRn = __shfl_down_sync(FULL, W2.x, 1);
            const float w2A0 = W2.x, w2B0 = W2.y;
            if (dirA < 0) cushion(E2.x, W2.x, D.x, hL, wLn);
            else if (dirA > 0) cushion(E2.x, W2.x, D.x, hB, w2B0);
            if (dirB < 0) cushion(E2.y, W2.y, D.y, hA, w2A0);
            else if (dirB > 0) cushion(E2.y, W2.y, D.y, hR, wRn);
        }
    }
    E = E2; W = W2; T = T2;
}

// xsweep2 when every node of the warp is wet at the start of the sweep (eq. (solver2),
// reflecting edges): steps (a), (b), (c) and (e) change nothing then, and this is the
// sequence of operations xsweep2 takes in that case, without its warp-uniform branches, so
// that the x-sweeps of two rows can share one basic block.
template <bool FRIC>
__device__ __forceinline__ void xsweep2_open(float2& E, float2& W, float2& T, float2 D, const XMet2& m,
                                             const SweepConst& K) {
    const float2 C = wave_speed2(add2(E, D));
    const float eR = __shfl_down_sync(FULL, E.x, 1), wR = __shfl_down_sync(FULL, W.x, 1);
    const float tR = __shfl_down_sync(FULL, T.x, 1), dR = __shfl_down_sync(FULL, D.x, 1);
    const float cR = __shfl_down_sync(FULL, C.x, 1);
    const Flux2 FR = iface2(E, W, T, D, C, make_float2(E.y, eR), make_float2(W.y, wR),
                            make_float2(T.y, tR), make_float2(D.y, dR), make_float2(C.y, cR), m.inv_r);
    Flux2 FL;
    FL.p = make_float2(__shfl_up_sync(FULL, FR.p.y, 1), FR.p.x);
    FL.q = make_float2(__shfl_up_sync(FULL, FR.q.y, 1), FR.q.x);
    FL.t = make_float2(__shfl_up_sync(FULL, FR.t.y, 1), FR.t.x);
    float2 E2, W2, T2;
    node_update2<false, FRIC, false>(E, W, T, D, C, FL, FR, m.k2, v2(0.f), K, E2, W2, T2);
    E = E2; W = W2; T = T2;
}

// One row of a pair of columns in the y-sweep pipeline.
struct YRow {
    float2 e, w, t, d, c;     // w: velocity along the column (v), t: across it (u)
    bool oA, oB;              // wet at the start of the sweep (a)
    bool wA, wB;              // wet after (b)
    int dA, dB;               // (b) source direction
};

// y-sweep of a pair of columns as a march down the rows. Each push takes the sweep input of
// row k and returns the finished result of row k - 3: (b) runs on row k-1, the interface
// flux between rows k-2 and k-1 is formed once and shared, (d) runs on row k-2 and (e) on
// k-3. Rows k-2 and k-1 live in two banks whose roles swap every push (PH), so the
// pipeline advances without copying them. Row k-2 is held after (b) only: when it was wet
// at the start of the sweep its values are its start-of-sweep values, which is all step
// (b) of row k-1 needs from it.
struct YMarch2 {
    YRow bank[2];             // [PH]: row k-2 after (b); [1-PH]: row k-1 as input
    Flux2 fb[2];              // [PH]: flux (k-3 | k-2)
    bool f3A, f3B;            // row k-3 wet after (b)
    float2 e3, w3, t3, d3;    // row k-3 after (d)
    int dir3A, dir3B;
    float2 h4, w4;            // row k-4 after (d): height, velocity
    float2 pe, pw, pt, pd, pc;   // row k-3 after (b) (eq. (solver1) only)

    __device__ __forceinline__ void init() {
        for (int i = 0; i < 2; ++i) {
            bank[i].e = bank[i].w = bank[i].t = bank[i].c = v2(0.f);
            bank[i].d = v2(OUTSIDE_D);
            bank[i].oA = bank[i].oB = bank[i].wA = bank[i].wB = false;
            bank[i].dA = bank[i].dB = 0;
            fb[i].p = fb[i].q = fb[i].t = v2(0.f);
        }
        f3A = f3B = false;
        e3 = w3 = t3 = v2(0.f);
        d3 = v2(OUTSIDE_D);
        dir3A = dir3B = 0;
        h4 = w4 = v2(0.f);
        pe = pw = pt = pc = v2(0.f);
        pd = v2(OUTSIDE_D);
    }

    // eq. (solver1): flux between rows k-3 and k-1 around row k-2 (P), with mirror ghosts
    // of P for a neighbour row that is dry after (b)
    // of P for a neighbour row that is dry after (b); at an open edge (pend 1: row k-2 is the
    // first row, 2: the last) the neighbour beyond it is the open ghost (ge, gw, gc)
    __device__ __forceinline__ Flux2 f1(const YRow& P, const YRow& B1, bool open, float k2,
                                        const SweepConst& K, int pend = 0, float2 ge = v2(0.f),
                                        float2 gw = v2(0.f), float2 gc = v2(0.f)) const {
        float2 le = pe, lw = pw, lt = pt, ld = pd, lc = pc;
        float2 re = B1.e, rw = B1.w, rt = B1.t, rd = B1.d, rc = B1.c;
        if (!open) {
            if (!f3A) { le.x = P.e.x; lw.x = -P.w.x; lt.x = P.t.x; ld.x = P.d.x; lc.x = P.c.x; }
            if (!f3B) { le.y = P.e.y; lw.y = -P.w.y; lt.y = P.t.y; ld.y = P.d.y; lc.y = P.c.y; }
            if (!B1.wA) { re.x = P.e.x; rw.x = -P.w.x; rt.x = P.t.x; rd.x = P.d.x; rc.x = P.c.x; }
            if (!B1.wB) { re.y = P.e.y; rw.y = -P.w.y; rt.y = P.t.y; rd.y = P.d.y; rc.y = P.c.y; }
        }
        if (pend == 1) { le = ge; lw = gw; lt = P.t; ld = P.d; lc = gc; }
        if (pend == 2) { re = ge; rw = gw; rt = P.t; rd = P.d; rc = gc; }
        return iface2(le, lw, lt, ld, lc, re, rw, rt, rd, rc, v2(k2 * K.inv_dt2));
    }

    // m2: metric of row k-2 (1/dy_{j-1}, 1/dy_j, dt^2/(dy_{j-1}+dy_j), dt tan(phi)/R).
    // emit(e, w, t, d) receives the finished row k-3; o0A/o0B: the incoming row's wet marks.
    // careA/careB: whether this lane's columns are emitted; the others may compute anything.
    // pend: row k-2 is the first row of the grid at an open edge (1) or the last (2), else 0.
    template <int PH, bool SRC, bool FRIC, bool S1, bool OPEN, class Emit>
    __device__ __forceinline__ void push(float2 E0, float2 W0, float2 T0, float2 D0, bool o0A, bool o0B,
                                         float4 m2, const SweepConst& K, bool careA, bool careB,
                                         Emit&& emit, int pend = 0) {
        YRow& P = bank[PH];
        YRow& B1 = bank[1 - PH];
        Flux2& F3 = fb[PH];
        Flux2& F2 = fb[1 - PH];
        // rows k-3..k-1 wet in (a) and no newly wetted row k-3: no (b), no walls, no (e)
        const bool openA = B1.oA && P.wA && f3A && dir3A == 0;
        const bool openB = B1.oB && P.wB && f3B && dir3B == 0;
        if (__all_sync(FULL, (!careA || openA) && (!careB || openB))) {
            B1.wA = B1.wB = true;
            B1.dA = B1.dB = 0;
            B1.c = wave_speed2(add2(B1.e, B1.d));
            F2 = iface2(P.e, P.w, P.t, P.d, P.c, B1.e, B1.w, B1.t, B1.d, B1.c, v2(m2.y));
            emit(e3, w3, t3, d3);
            h4 = add2(e3, d3);
            w4 = w3;
            Flux2 F1;
            if (S1) F1 = f1(P, B1, true, m2.z, K);
            node_update2<SRC, FRIC, S1>(P.e, P.w, P.t, P.d, P.c, F3, F2, v2(m2.z), v2(m2.w), K, e3, w3, t3, &F1);
        } else {
            // (a)/(b) on row k-1 (input held in B1), neighbours row k-2 (P) and row k (new)
            B1.wA = B1.oA;
            B1.wB = B1.oB;
            B1.dA = B1.dB = 0;
            if (!B1.oA) {
                B1.w.x = 0.f; B1.t.x = 0.f;
                if (B1.d.x >= K.dwall) {
                    B1.dA = flood1(B1.e.x, B1.w.x, B1.t.x, B1.d.x, P.e.x, P.w.x, P.t.x, P.oA,
                                   E0.x, W0.x, T0.x, o0A, K.hmin);
                    B1.wA = B1.dA != 0;
                }
            }
            if (!B1.oB) {
                B1.w.y = 0.f; B1.t.y = 0.f;
                if (B1.d.y >= K.dwall) {
                    B1.dB = flood1(B1.e.y, B1.w.y, B1.t.y, B1.d.y, P.e.y, P.w.y, P.t.y, P.oB,
                                   E0.y, W0.y, T0.y, o0B, K.hmin);
                    B1.wB = B1.dB != 0;
                }
            }
            B1.c = wave_speed2(add2(B1.e, B1.d));
            F2 = iface2(P.e, P.w, P.t, P.d, P.c, B1.e, B1.w, B1.t, B1.d, B1.c, v2(m2.y));
            // (c): walls, then (d) on row k-2
            Flux2 L = F3, R = F2;
            if (P.wA && !f3A) ghost_left(P.w.x, P.c.x, m2.x, L.p.x, L.q.x, L.t.x);
            if (P.wA && !B1.wA) ghost_right(P.w.x, P.c.x, m2.y, R.p.x, R.q.x, R.t.x);
            if (P.wB && !f3B) ghost_left(P.w.y, P.c.y, m2.x, L.p.y, L.q.y, L.t.y);
            if (P.wB && !B1.wB) ghost_right(P.w.y, P.c.y, m2.y, R.p.y, R.q.y, R.t.y);
            float2 ge = v2(0.f), gw = v2(0.f), gc = v2(0.f);
            if (OPEN && pend) {
                // an open outer edge: the flux across it from the open ghost (wet nodes only)
                const bool right = pend == 2;
                Flux2 Fo;
                open_flux(P.e.x, P.w.x, P.t.x, P.d.x, P.c.x, right ? m2.y : m2.x, right, Fo.p.x, Fo.q.x, Fo.t.x,
                          ge.x, gw.x, gc.x);
                open_flux(P.e.y, P.w.y, P.t.y, P.d.y, P.c.y, right ? m2.y : m2.x, right, Fo.p.y, Fo.q.y, Fo.t.y,
                          ge.y, gw.y, gc.y);
                Flux2& S = right ? R : L;
                if (P.wA) { S.p.x = Fo.p.x; S.q.x = Fo.q.x; S.t.x = Fo.t.x; }
                if (P.wB) { S.p.y = Fo.p.y; S.q.y = Fo.q.y; S.t.y = Fo.t.y; }
            }
            float2 ne, nw, nt;
            Flux2 F1;
            if (S1) F1 = f1(P, B1, false, m2.z, K, pend, ge, gw, gc);
            node_update2<SRC, FRIC, S1>(P.e, P.w, P.t, P.d, P.c, L, R, v2(m2.z), v2(m2.w), K, ne, nw, nt, &F1);
            if (!P.wA) { ne.x = P.e.x; nw.x = P.w.x; nt.x = P.t.x; }
            if (!P.wB) { ne.y = P.e.y; nw.y = P.w.y; nt.y = P.t.y; }
            // (e) on row k-3, against row k-4 (h4, w4) or row k-2 (ne, nw)
            float2 oe = e3, ow = w3;
            if (dir3A != 0) cushion(oe.x, ow.x, d3.x, dir3A < 0 ? h4.x : ne.x + P.d.x, dir3A < 0 ? w4.x : nw.x);
            if (dir3B != 0) cushion(oe.y, ow.y, d3.y, dir3B < 0 ? h4.y : ne.y + P.d.y, dir3B < 0 ? w4.y : nw.y);
            emit(oe, ow, t3, d3);
            h4 = add2(e3, d3);
            w4 = w3;
            e3 = ne; w3 = nw; t3 = nt;
        }
        if (S1) { pe = P.e; pw = P.w; pt = P.t; pd = P.d; pc = P.c; }
        d3 = P.d;
        dir3A = P.dA; dir3B = P.dB;
        f3A = P.wA; f3B = P.wB;
        // row k takes the freed bank
        P.e = E0; P.w = W0; P.t = T0; P.d = D0;
        P.oA = o0A; P.oB = o0B;
    }
};

}  // namespace cliffs
