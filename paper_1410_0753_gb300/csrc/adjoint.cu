// Reverse mode of the split step: the transpose of the Jacobian of one x-sweep followed by
// one y-sweep (arXiv 1410.0753, section "Numerics", eqs. (eqQ), (solver2), (stateu),
// (stateh), (pq3) and the inundation steps (a)-(e)), with every branch taken as the forward
// pass took it: the wet/dry marks of (a), the flooding choice of (b), the mirror walls of
// (c), the friction clamp and both tests of the cushion (e). Differentiating the step is
// this library's addition; the paper has no adjoint.
//
// One adjoint step k, given the adjoint lambda_{k+1} of the state after step k:
//   k_adj_xfwd    recompute the x-sweep of the stored state X_k (the same arithmetic as
//                 the forward kernel, so the same bits) and write it transposed, so that
//                 the y-sweep's lines (columns) lie along memory;
//   k_adj_line<1> adjoint of the y-sweep, line by line over the transposed data, written
//                 back untransposed;
//   k_adj_line<0> adjoint of the x-sweep over rows, plus the gauge-misfit seed of step k,
//                 written transposed for the next step's y-sweep adjoint.
// A warp holds 64 nodes of a line (two per lane); each stage of the sweep needs its line
// neighbours once, so after the six stages (b), (d), the tests of (e), and the adjoints of
// (e), (d) and (b), the middle 52 nodes are exact. A block stages its 8 lines x 52 nodes
// in shared memory and writes them transposed (32-byte segments), so every load and store is
// coalesced; blocks this small keep the last partial wave of the grid short.
//
// Derivatives are taken on the perturbation form used by the forward kernels (eta kept,
// c_a - c_b = g (eta_a - eta_b + d_a - d_b)/(c_a + c_b)), which keeps the coefficients
// free of the cancellation that p = w + 2c would suffer in FP32. Reciprocals in the
// coefficients come from the hardware approximation (relative error ~1e-7), as in the forward.
#include "internal.h"
#include "adjoint.h"
#include "sweep.cuh"

namespace cliffs {

constexpr int AHALO = 6;                    // nodes of a window without their full dependency
constexpr int AOUT = XWIN - 2 * AHALO;      // nodes a window finishes
constexpr int ALINES = 8;                   // lines per block (one per warp: a short tail wave)
constexpr int AWARPS = 8;                   // warps per block
constexpr int TP = ALINES + 1;              // shared tile pitch (no bank conflicts)

struct ANode { float e, w, t, d, c; };      // post-(b) state of a node or of a mirror ghost
struct ABar { float e, w, t; };             // adjoints of (eta, w, t)
struct AMet { float il, ir, k2, sdt; };     // 1/ds_left, 1/ds_right, dt^2/(ds_l+ds_r), dt tan/R

// Interface between a left node b and a right node a (times the interval): the fluxes of
// p, q (eq. (eqQ)) and t (eq. (pq3)) and the differences their derivatives need.
struct AIface { float dw, dcs, sw, S, dtt, qp, qq, qt; };

__device__ __forceinline__ AIface a_iface(const ANode& b, const ANode& a) {
    AIface f;
    const float de = a.e - b.e;
    f.S = a.c + b.c;
    f.dcs = GRAV * (de + (a.d - b.d)) * rcp_approx(f.S);    // c_a - c_b
    f.dw = a.w - b.w;
    f.sw = a.w + b.w;
    f.dtt = a.t - b.t;
    const float y = f.sw * f.dcs, z = GRAV * de;
    f.qp = 0.5f * f.dw * (f.sw + f.S) + z + y;
    f.qq = 0.5f * f.dw * (f.sw - f.S) + z - y;
    f.qt = 0.5f * f.sw * f.dtt;
    return f;
}

// Friction of reading 4 as the forward step computes it (fric_k2): adt = w k with
// k = min(dt g n^2 sqrt(s2) h^(-4/3), 1); mode 2 when clamped (k = 1), else mode 1; mode 0
// without friction.
struct AFric { float adt, s2, k; int mode; };

__device__ __forceinline__ AFric a_friction(const ANode& C, const SweepConst& K) {
    AFric F{0.f, 0.f, 0.f, 0};
    if (K.dt_gn2 > 0.f) {
        float ex;
        F.k = fric_k(C.w, C.t, C.e + C.d, K.dt_gn2, F.s2, ex);
        F.adt = C.w * F.k;
        F.mode = ex >= 0.f ? 2 : 1;
    }
    return F;
}

// (d) at a wet node C with neighbours L and R (mirror ghosts already substituted): the
// new eta and w, which the tests of (e) compare.
// With S1, eq. (solver1): the first-order term is dt Q(R, L) across the double interval
// (1/(dx_{j-1} + dx_j) = k2 / dt^2) instead of dt/2 (Q_L + Q_R).
template <bool SRC, bool S1>
__device__ __forceinline__ void a_dstage(const ANode& L, const ANode& C, const ANode& R, const AMet& m,
                                         const SweepConst& K, float& e2, float& w2) {
    const AIface fl = a_iface(L, C), fr = a_iface(C, R);
    const float QpL = fl.qp * m.il, QpR = fr.qp * m.ir, QqL = fl.qq * m.il, QqR = fr.qq * m.ir;
    const float hdt = K.half_dt;
    float dp, dq;
    if (S1) {
        const AIface flr = a_iface(L, R);
        const float f = -2.f * hdt * m.k2 * K.inv_dt2;
        dp = f * flr.qp + (C.w + C.c) * m.k2 * (QpR - QpL);
        dq = f * flr.qq + (C.w - C.c) * m.k2 * (QqR - QqL);
    } else {
        dp = -hdt * (QpL + QpR) + (C.w + C.c) * m.k2 * (QpR - QpL);
        dq = -hdt * (QqL + QqR) + (C.w - C.c) * m.k2 * (QqR - QqL);
    }
    const AFric F = a_friction(C, K);
    dp -= F.adt;
    dq -= F.adt;
    if (SRC) {
        const float s = m.sdt * C.c * C.w;
        dp += s;
        dq -= s;
    }
    const float dc = 0.25f * (dp - dq);
    w2 = C.w + 0.5f * (dp + dq);
    e2 = C.e + dc * (2.f * C.c + dc) * INV_GRAV;
}

// Adjoint of (d) at a wet node: given the adjoints (ge, gw, gt) of its new (eta, w, t), add
// the adjoints of the post-(b) states of L, C and R (c folded into eta by dc/deta = g/2c).
template <bool SRC, bool S1>
__device__ __forceinline__ void a_dstage_adj(const ANode& L, const ANode& C, const ANode& R, const AMet& m,
                                             const SweepConst& K, float ge, float gw, float gt,
                                             ABar& bL, ABar& bC, ABar& bR) {
    const AIface fl = a_iface(L, C), fr = a_iface(C, R);
    const float QpL = fl.qp * m.il, QpR = fr.qp * m.ir, QqL = fl.qq * m.il, QqR = fr.qq * m.ir;
    const float QtL = fl.qt * m.il, QtR = fr.qt * m.ir;
    const float hdt = K.half_dt;
    const float lp = C.w + C.c, lq = C.w - C.c;
    AIface flr{};
    float ilr = 0.f;
    float dp, dq;
    if (S1) {
        flr = a_iface(L, R);
        ilr = m.k2 * K.inv_dt2;
        dp = -2.f * hdt * flr.qp * ilr + lp * m.k2 * (QpR - QpL);
        dq = -2.f * hdt * flr.qq * ilr + lq * m.k2 * (QqR - QqL);
    } else {
        dp = -hdt * (QpL + QpR) + lp * m.k2 * (QpR - QpL);
        dq = -hdt * (QqL + QqR) + lq * m.k2 * (QqR - QqL);
    }
    const AFric F = a_friction(C, K);
    dp -= F.adt;
    dq -= F.adt;
    if (SRC) {
        const float s = m.sdt * C.c * C.w;
        dp += s;
        dq -= s;
    }
    const float dcn = 0.25f * (dp - dq);
    // eta2 = eta + dcn (2c + dcn)/g, w2 = w + (dp + dq)/2, dcn = (dp - dq)/4
    float eC = ge, wC = gw, tC = gt, cC = ge * 2.f * dcn * INV_GRAV, cL = 0.f, cR = 0.f;
    const float gdcn = ge * 2.f * (C.c + dcn) * INV_GRAV;
    const float gdp = 0.5f * gw + 0.25f * gdcn, gdq = 0.5f * gw - 0.25f * gdcn;
    // t2 = t - dt/2 (QtL + QtR) + w k2 (QtR - QtL)   (eq. (pq3)); with S1 the first term is
    // -dt Qt(R, L) over the double interval
    const float hh = S1 ? 0.f : hdt;
    float gQtL = 0.f, gQtR = 0.f, gF1t = 0.f;
    if (K.transverse) {
        gQtL = gt * (-hh - C.w * m.k2);
        gQtR = gt * (-hh + C.w * m.k2);
        if (S1) gF1t = gt * (-2.f * hdt);
        wC += gt * m.k2 * (QtR - QtL);
    }
    // dp = -dt/2 (QpL + QpR) + (w + c) k2 (QpR - QpL) - adt + sdt c w, dq alike with w - c
    const float gQpL = gdp * (-hh - lp * m.k2), gQpR = gdp * (-hh + lp * m.k2);
    const float gQqL = gdq * (-hh - lq * m.k2), gQqR = gdq * (-hh + lq * m.k2);
    const float glp = gdp * m.k2 * (QpR - QpL), glq = gdq * m.k2 * (QqR - QqL);
    wC += glp + glq;
    cC += glp - glq;
    const float gadt = -(gdp + gdq);
    if (F.mode == 2) {
        wC += gadt;
    } else if (F.mode == 1 && F.s2 > 1e-30f) {   // below, k < 1e-15: no friction to speak of
        // adt = w k, k ~ sqrt(s2) h^(-4/3): dk/dw = k w / s2, dk/dt = k t / s2, dk/dh = -4/3 k / h
        const float G = gadt * F.k, rs2 = rcp_approx(F.s2);
        wC += G * (1.f + C.w * C.w * rs2);
        tC += G * C.w * C.t * rs2;
        eC += G * C.w * (-4.f / 3.f) * rcp_approx(C.e + C.d);
    }
    if (SRC) {
        const float gs = (gdp - gdq) * m.sdt;
        cC += gs * C.w;
        wC += gs * C.c;
    }
    // Q(a, b) ds = 1/2 (lam_a + lam_b)(r_a - r_b) - g (d_a - d_b): partials with respect to
    // w and c of both sides, for p (lam = w + c, r = w + 2c) and q (lam = w - c, r = w - 2c)
    {   // left interface: b = L, a = C
        const float A = gQpL * m.il, B = gQqL * m.il, T = gQtL * m.il;
        const float hp = 0.5f * fl.dw + fl.dcs, hq = 0.5f * fl.dw - fl.dcs;
        const float sp = fl.sw + fl.S, sq = fl.sw - fl.S;
        wC += A * (hp + 0.5f * sp) + B * (hq + 0.5f * sq) + T * 0.5f * fl.dtt;
        bL.w += A * (hp - 0.5f * sp) + B * (hq - 0.5f * sq) + T * 0.5f * fl.dtt;
        cC += A * (hp + sp) - B * (hq + sq);
        cL += A * (hp - sp) - B * (hq - sq);
        tC += T * 0.5f * fl.sw;
        bL.t -= T * 0.5f * fl.sw;
    }
    {   // right interface: b = C, a = R
        const float A = gQpR * m.ir, B = gQqR * m.ir, T = gQtR * m.ir;
        const float hp = 0.5f * fr.dw + fr.dcs, hq = 0.5f * fr.dw - fr.dcs;
        const float sp = fr.sw + fr.S, sq = fr.sw - fr.S;
        bR.w += A * (hp + 0.5f * sp) + B * (hq + 0.5f * sq) + T * 0.5f * fr.dtt;
        wC += A * (hp - 0.5f * sp) + B * (hq - 0.5f * sq) + T * 0.5f * fr.dtt;
        cR += A * (hp + sp) - B * (hq + sq);
        cC += A * (hp - sp) - B * (hq - sq);
        bR.t += T * 0.5f * fr.sw;
        tC -= T * 0.5f * fr.sw;
    }
    if (S1) {   // the flux across the double interval: b = L, a = R
        const float A = gdp * (-2.f * hdt) * ilr, B = gdq * (-2.f * hdt) * ilr, T = gF1t * ilr;
        const float hp = 0.5f * flr.dw + flr.dcs, hq = 0.5f * flr.dw - flr.dcs;
        const float sp = flr.sw + flr.S, sq = flr.sw - flr.S;
        bR.w += A * (hp + 0.5f * sp) + B * (hq + 0.5f * sq) + T * 0.5f * flr.dtt;
        bL.w += A * (hp - 0.5f * sp) + B * (hq - 0.5f * sq) + T * 0.5f * flr.dtt;
        cR += A * (hp + sp) - B * (hq + sq);
        cL += A * (hp - sp) - B * (hq - sq);
        bR.t += T * 0.5f * flr.sw;
        bL.t -= T * 0.5f * flr.sw;
    }
    bC.e += eC + cC * (0.5f * GRAV) * rcp_approx(C.c);
    bC.w += wC;
    bC.t += tC;
    bL.e += cL * (0.5f * GRAV) * rcp_approx(L.c);
    bR.e += cR * (0.5f * GRAV) * rcp_approx(R.c);
}

// ------------------------------------------------------------------ open outer edges
// The open ghost of a wet edge node C (the forward's open_ghost, as a stencil node) and the
// transpose of its map: with delta = c - c0 the ghost is w_g = w/2 + s delta,
// c_g = c/2 + s w/4 + c0/2 (s = +1 at the right end, -1 at the left; c_g = 0 when clamped),
// eta_g = c_g^2/g - d, t_g = t, so dw_g = dw/2 + s dc, dc_g = s dw/4 + dc/2 with
// dc = g/(2c) deta, and deta_g = 2 c_g/g dc_g.
__device__ __forceinline__ ANode a_open_ghost(const ANode& C, bool right) {
    float eg, wg, cg;
    open_ghost(C.e, C.w, C.d, C.c, right, eg, wg, cg);
    return ANode{eg, wg, C.t, C.d, cg};
}
__device__ __forceinline__ void a_open_ghost_adj(const ANode& C, const ANode& Gh, bool right, const ABar& bg,
                                                 ABar& bC) {
    const float s = right ? 1.f : -1.f;
    const float gcg = Gh.c > 0.f ? bg.e * 2.f * Gh.c * INV_GRAV : 0.f;   // adjoint of c_g
    const float gc = s * bg.w + 0.5f * gcg;                               // adjoint of c
    bC.w += 0.5f * bg.w + s * 0.25f * gcg;
    bC.e += gc * (0.5f * GRAV) * rcp_approx(C.c);
    bC.t += bg.t;
}

// ------------------------------------------------------------------ packed open water
// The same adjoint of (d) for the two nodes of a lane at once (packed FP32x2), for windows
// where every node is wet: real neighbours, no ghosts.
__device__ __forceinline__ float2 rcp2(float2 x) { return make_float2(rcp_approx(x.x), rcp_approx(x.y)); }

struct N2 { float2 e, w, t, d, c; };
struct AIface2 { float2 dw, dcs, sw, S, dtt, qp, qq, qt; };

__device__ __forceinline__ AIface2 a_iface2(const N2& b, const N2& a) {
    AIface2 f;
    const float2 de = sub2(a.e, b.e);
    f.S = add2(a.c, b.c);
    f.dcs = mul2(mul2(v2(GRAV), add2(de, sub2(a.d, b.d))), rcp2(f.S));
    f.dw = sub2(a.w, b.w);
    f.sw = add2(a.w, b.w);
    f.dtt = sub2(a.t, b.t);
    const float2 y = mul2(f.sw, f.dcs), z = mul2(v2(GRAV), de), hdw = mul2(v2(0.5f), f.dw);
    f.qp = fma2(hdw, add2(f.sw, f.S), add2(z, y));
    f.qq = fma2(hdw, sub2(f.sw, f.S), sub2(z, y));
    f.qt = mul2(mul2(v2(0.5f), f.sw), f.dtt);
    return f;
}

// friction part of the adjoint for one node (adt = w k, see a_friction)
__device__ __forceinline__ void fric_adj1(float gadt, float w, float t, float e, float d, float s2, float k,
                                          bool clamped, float& wC, float& tC, float& eC) {
    if (clamped) {
        wC += gadt;
    } else if (s2 > 1e-30f) {                      // below, k < 1e-15: no friction to speak of
        const float G = gadt * k, rs2 = rcp_approx(s2);
        wC += G * (1.f + w * w * rs2);
        tC += G * w * t * rs2;
        eC += G * w * (-4.f / 3.f) * rcp_approx(e + d);
    }
}

template <bool SRC>
__device__ __forceinline__ void a_dstage_adj2(const N2& L, const N2& C, const N2& R, float2 il, float2 ir,
                                              float2 k2, float2 sdt, const SweepConst& K, float2 ge, float2 gw,
                                              float2 gt, float2 (&bL)[3], float2 (&bC)[3], float2 (&bR)[3]) {
    const AIface2 fl = a_iface2(L, C), fr = a_iface2(C, R);
    const float2 QpL = mul2(fl.qp, il), QpR = mul2(fr.qp, ir), QqL = mul2(fl.qq, il), QqR = mul2(fr.qq, ir);
    const float2 QtL = mul2(fl.qt, il), QtR = mul2(fr.qt, ir);
    const float2 nh = v2(-K.half_dt);
    const float2 lp = add2(C.w, C.c), lq = sub2(C.w, C.c);
    const float2 dQp = sub2(QpR, QpL), dQq = sub2(QqR, QqL);
    float2 dp = fma2(mul2(lp, k2), dQp, mul2(nh, add2(QpL, QpR)));
    float2 dq = fma2(mul2(lq, k2), dQq, mul2(nh, add2(QqL, QqR)));
    float2 s2 = v2(0.f), kf = v2(0.f);
    bool clA = false, clB = false;
    const bool fric = K.dt_gn2 > 0.f;
    if (fric) {
        float2 ex;
        kf = fric_k2(C.w, C.t, add2(C.e, C.d), K.dt_gn2, s2, ex);
        clA = ex.x >= 0.f;
        clB = ex.y >= 0.f;
        const float2 adt = mul2(C.w, kf);
        dp = sub2(dp, adt);
        dq = sub2(dq, adt);
    }
    if (SRC) {
        const float2 sw_ = mul2(mul2(sdt, C.c), C.w);
        dp = add2(dp, sw_);
        dq = sub2(dq, sw_);
    }
    const float2 dcn = mul2(v2(0.25f), sub2(dp, dq));
    // reverse sweep
    float2 eC = ge, wC = gw, tC = gt;
    float2 cC = mul2(ge, mul2(v2(2.f * INV_GRAV), dcn));
    const float2 gdcn = mul2(ge, mul2(v2(2.f * INV_GRAV), add2(C.c, dcn)));
    const float2 gdp = fma2(v2(0.5f), gw, mul2(v2(0.25f), gdcn));
    const float2 gdq = fma2(v2(0.5f), gw, mul2(v2(-0.25f), gdcn));
    float2 gQtL = v2(0.f), gQtR = v2(0.f);
    if (K.transverse) {
        const float2 wk = mul2(C.w, k2);
        gQtL = mul2(gt, sub2(nh, wk));
        gQtR = mul2(gt, add2(nh, wk));
        wC = fma2(mul2(gt, k2), sub2(QtR, QtL), wC);
    }
    const float2 lpk = mul2(lp, k2), lqk = mul2(lq, k2);
    const float2 gQpL = mul2(gdp, sub2(nh, lpk)), gQpR = mul2(gdp, add2(nh, lpk));
    const float2 gQqL = mul2(gdq, sub2(nh, lqk)), gQqR = mul2(gdq, add2(nh, lqk));
    const float2 glp = mul2(mul2(gdp, k2), dQp), glq = mul2(mul2(gdq, k2), dQq);
    wC = add2(wC, add2(glp, glq));
    cC = add2(cC, sub2(glp, glq));
    if (fric) {
        const float2 gadt = mul2(v2(-1.f), add2(gdp, gdq));
        fric_adj1(gadt.x, C.w.x, C.t.x, C.e.x, C.d.x, s2.x, kf.x, clA, wC.x, tC.x, eC.x);
        fric_adj1(gadt.y, C.w.y, C.t.y, C.e.y, C.d.y, s2.y, kf.y, clB, wC.y, tC.y, eC.y);
    }
    if (SRC) {
        const float2 gs = mul2(sub2(gdp, gdq), sdt);
        cC = fma2(gs, C.w, cC);
        wC = fma2(gs, C.c, wC);
    }
    float2 cL, cR;
    {   // left interface: b = L, a = C
        const float2 A = mul2(gQpL, il), B = mul2(gQqL, il), T = mul2(gQtL, il);
        const float2 hp = fma2(v2(0.5f), fl.dw, fl.dcs), hq = fma2(v2(0.5f), fl.dw, mul2(v2(-1.f), fl.dcs));
        const float2 sp = add2(fl.sw, fl.S), sq = sub2(fl.sw, fl.S);
        const float2 hsp = mul2(v2(0.5f), sp), hsq = mul2(v2(0.5f), sq);
        const float2 tdt = mul2(mul2(v2(0.5f), T), fl.dtt), tsw = mul2(mul2(v2(0.5f), T), fl.sw);
        wC = add2(wC, fma2(A, add2(hp, hsp), fma2(B, add2(hq, hsq), tdt)));
        bL[1] = fma2(A, sub2(hp, hsp), fma2(B, sub2(hq, hsq), tdt));
        cC = add2(cC, sub2(mul2(A, add2(hp, sp)), mul2(B, add2(hq, sq))));
        cL = sub2(mul2(A, sub2(hp, sp)), mul2(B, sub2(hq, sq)));
        tC = add2(tC, tsw);
        bL[2] = mul2(v2(-1.f), tsw);
    }
    {   // right interface: b = C, a = R
        const float2 A = mul2(gQpR, ir), B = mul2(gQqR, ir), T = mul2(gQtR, ir);
        const float2 hp = fma2(v2(0.5f), fr.dw, fr.dcs), hq = fma2(v2(0.5f), fr.dw, mul2(v2(-1.f), fr.dcs));
        const float2 sp = add2(fr.sw, fr.S), sq = sub2(fr.sw, fr.S);
        const float2 hsp = mul2(v2(0.5f), sp), hsq = mul2(v2(0.5f), sq);
        const float2 tdt = mul2(mul2(v2(0.5f), T), fr.dtt), tsw = mul2(mul2(v2(0.5f), T), fr.sw);
        bR[1] = fma2(A, add2(hp, hsp), fma2(B, add2(hq, hsq), tdt));
        wC = add2(wC, fma2(A, sub2(hp, hsp), fma2(B, sub2(hq, hsq), tdt)));
        cR = sub2(mul2(A, add2(hp, sp)), mul2(B, add2(hq, sq)));
        cC = add2(cC, sub2(mul2(A, sub2(hp, sp)), mul2(B, sub2(hq, sq))));
        bR[2] = tsw;
        tC = sub2(tC, tsw);
    }
    const float2 hg = v2(0.5f * GRAV);
    bC[0] = fma2(mul2(cC, hg), rcp2(C.c), eC);
    bC[1] = wC;
    bC[2] = tC;
    bL[0] = mul2(mul2(cL, hg), rcp2(L.c));
    bR[0] = mul2(mul2(cR, hg), rcp2(R.c));
}

// neighbours across the window: node 0 of a lane is window node 2*lane, node 1 is 2*lane+1
__device__ __forceinline__ void nbr(const float (&x)[2], float (&l)[2], float (&r)[2]) {
    l[0] = __shfl_up_sync(FULL, x[1], 1);
    l[1] = x[0];
    r[0] = x[1];
    r[1] = __shfl_down_sync(FULL, x[0], 1);
}
__device__ __forceinline__ void nbr(const int (&x)[2], int (&l)[2], int (&r)[2]) {
    l[0] = __shfl_up_sync(FULL, x[1], 1);
    l[1] = x[0];
    r[0] = x[1];
    r[1] = __shfl_down_sync(FULL, x[0], 1);
}

// Adjoint of one sweep of a 64-node line window. In: the sweep's input (e, w, t, d) and the
// adjoint (ge, gw, gt) of its output. Out: the adjoint of its input, exact at window
// nodes 6..57.
// ends: this lane's nodes at open outer edges, bits 1 node 0 left, 2 node 0 right, 4 node 1
// left, 8 node 1 right (their outside neighbour is the open ghost instead of a mirror).
template <bool SRC, bool S1>
__device__ __forceinline__ void line_adjoint(const float (&e)[2], const float (&w)[2], const float (&t)[2],
                                             const float (&d)[2], const float (&ge)[2], const float (&gw)[2],
                                             const float (&gt)[2], const AMet (&m)[2], const SweepConst& K,
                                             float (&oe)[2], float (&ow)[2], float (&ot)[2], unsigned ends = 0u) {
    // (a) wet marks at the start of the sweep
    int o[2], fl[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        fl[i] = d[i] >= K.dwall;
        o[i] = fl[i] && (e[i] + d[i] >= K.hmin);
    }
    if (!S1 && __all_sync(FULL, o[0] && o[1])) {
        // every node of the window wet: no (b), no walls, no (e); only the stencil of (d)
        float c[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) c[i] = wave_speed(e[i] + d[i]);
        float eL[2], eR[2], wL[2], wR[2], tL[2], tR[2], dL[2], dR[2], cL[2], cR[2];
        nbr(e, eL, eR); nbr(w, wL, wR); nbr(t, tL, tR); nbr(d, dL, dR); nbr(c, cL, cR);
        auto f2 = [](const float (&x)[2]) { return make_float2(x[0], x[1]); };
        const N2 Ln{f2(eL), f2(wL), f2(tL), f2(dL), f2(cL)}, Cn{f2(e), f2(w), f2(t), f2(d), f2(c)};
        const N2 Rn{f2(eR), f2(wR), f2(tR), f2(dR), f2(cR)};
        float2 bL[3], bC[3], bR[3];
        a_dstage_adj2<SRC>(Ln, Cn, Rn, make_float2(m[0].il, m[1].il), make_float2(m[0].ir, m[1].ir),
                           make_float2(m[0].k2, m[1].k2), make_float2(m[0].sdt, m[1].sdt), K, f2(ge), f2(gw),
                           f2(gt), bL, bC, bR);
        // node A gathers from B's left part and lane-1's B's right part; B from A's right
        // part and lane+1's A's left part
        float* out[3] = {oe, ow, ot};
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            out[f][0] = bC[f].x + bL[f].y + __shfl_up_sync(FULL, bR[f].y, 1);
            out[f][1] = bC[f].y + bR[f].x + __shfl_down_sync(FULL, bL[f].x, 1);
        }
        return;
    }
    // (b) flooding from the wetter neighbour (left on a tie), start-of-sweep values
    float eL[2], eR[2], wL[2], wR[2], tL[2], tR[2];
    int oL[2], oR[2];
    nbr(e, eL, eR); nbr(w, wL, wR); nbr(t, tL, tR); nbr(o, oL, oR);
    float e1[2], w1[2], t1[2];
    int dir[2], wt[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        e1[i] = e[i]; w1[i] = w[i]; t1[i] = t[i]; dir[i] = 0; wt[i] = o[i];
        if (!o[i]) {
            w1[i] = 0.f;
            t1[i] = 0.f;
            if (fl[i]) {
                const bool okL = oL[i] && (eL[i] + d[i] > K.hmin);
                const bool okR = oR[i] && (eR[i] + d[i] > K.hmin);
                if (okL || okR) {
                    const bool useR = okR && (!okL || eR[i] > eL[i]);
                    e1[i] = K.hmin - d[i];
                    w1[i] = useR ? wR[i] : wL[i];
                    t1[i] = useR ? tR[i] : tL[i];
                    dir[i] = useR ? 1 : -1;
                    wt[i] = 1;
                }
            }
        }
    }
    // (c)+(d): the stencil of each wet node, mirror ghosts for dry neighbours
    float c1[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) c1[i] = wt[i] ? wave_speed(e1[i] + d[i]) : 1.f;
    float e1L[2], e1R[2], w1L[2], w1R[2], t1L[2], t1R[2], dL[2], dR[2], cL[2], cR[2];
    int wtL[2], wtR[2];
    nbr(e1, e1L, e1R); nbr(w1, w1L, w1R); nbr(t1, t1L, t1R); nbr(d, dL, dR); nbr(c1, cL, cR);
    nbr(wt, wtL, wtR);
    ANode Cn[2], Ln[2], Rn[2];
    float h2[2], w2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        Cn[i] = ANode{e1[i], w1[i], t1[i], d[i], c1[i]};
        const ANode G{e1[i], -w1[i], t1[i], d[i], c1[i]};
        Ln[i] = wtL[i] ? ANode{e1L[i], w1L[i], t1L[i], dL[i], cL[i]} : G;
        Rn[i] = wtR[i] ? ANode{e1R[i], w1R[i], t1R[i], dR[i], cR[i]} : G;
        if (ends && wt[i]) {
            if (ends & (1u << (2 * i))) Ln[i] = a_open_ghost(Cn[i], false);
            if (ends & (2u << (2 * i))) Rn[i] = a_open_ghost(Cn[i], true);
        }
        if (wt[i]) {
            float ee, ww;
            a_dstage<SRC, S1>(Ln[i], Cn[i], Rn[i], m[i], K, ee, ww);
            h2[i] = ee + d[i];
            w2[i] = ww;
        } else {
            h2[i] = e1[i] + d[i];
            w2[i] = w1[i];
        }
    }
    // (e) tests of each newly wetted node against its source after (d)
    float h2L[2], h2R[2], w2L[2], w2R[2];
    nbr(h2, h2L, h2R); nbr(w2, w2L, w2R);
    int ce[2], cw[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        ce[i] = cw[i] = 0;
        if (dir[i]) {
            const float hs = dir[i] < 0 ? h2L[i] : h2R[i];
            const float ws = dir[i] < 0 ? w2L[i] : w2R[i];
            ce[i] = h2[i] > 0.5f * hs;
            cw[i] = fabsf(w2[i]) > fabsf(ws);
        }
    }
    // adjoint of (e): a limited value came from the source's
    float geL[2], geR[2], gwL[2], gwR[2];
    int dirL[2], dirR[2], ceL[2], ceR[2], cwL[2], cwR[2];
    nbr(ge, geL, geR); nbr(gw, gwL, gwR);
    nbr(dir, dirL, dirR); nbr(ce, ceL, ceR); nbr(cw, cwL, cwR);
    ABar bL[2], bC[2], bR[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float De = (ce[i] ? 0.f : ge[i]) + ((dirL[i] == 1 && ceL[i]) ? 0.5f * geL[i] : 0.f) +
                         ((dirR[i] == -1 && ceR[i]) ? 0.5f * geR[i] : 0.f);
        const float Dw = (cw[i] ? 0.f : gw[i]) + ((dirL[i] == 1 && cwL[i]) ? gwL[i] : 0.f) +
                         ((dirR[i] == -1 && cwR[i]) ? gwR[i] : 0.f);
        // adjoint of (c)+(d); a dry node passes its values through
        bL[i] = bR[i] = ABar{0.f, 0.f, 0.f};
        if (wt[i]) {
            bC[i] = ABar{0.f, 0.f, 0.f};
            a_dstage_adj<SRC, S1>(Ln[i], Cn[i], Rn[i], m[i], K, De, Dw, gt[i], bL[i], bC[i], bR[i]);
            if (ends & (1u << (2 * i))) {        // the open ghost is a function of C
                a_open_ghost_adj(Cn[i], Ln[i], false, bL[i], bC[i]);
                bL[i] = ABar{0.f, 0.f, 0.f};
            } else if (!wtL[i]) {                // the ghost mirrors C: (eta, -w, t)
                bC[i].e += bL[i].e; bC[i].w -= bL[i].w; bC[i].t += bL[i].t;
                bL[i] = ABar{0.f, 0.f, 0.f};
            }
            if (ends & (2u << (2 * i))) {
                a_open_ghost_adj(Cn[i], Rn[i], true, bR[i], bC[i]);
                bR[i] = ABar{0.f, 0.f, 0.f};
            } else if (!wtR[i]) {
                bC[i].e += bR[i].e; bC[i].w -= bR[i].w; bC[i].t += bR[i].t;
                bR[i] = ABar{0.f, 0.f, 0.f};
            }
        } else {
            bC[i] = ABar{De, Dw, gt[i]};
        }
    }
    // every node gathers its own part and its neighbours' parts
    float Be[2], Bw[2], Bt[2];
    Be[0] = bC[0].e + bL[1].e + __shfl_up_sync(FULL, bR[1].e, 1);
    Bw[0] = bC[0].w + bL[1].w + __shfl_up_sync(FULL, bR[1].w, 1);
    Bt[0] = bC[0].t + bL[1].t + __shfl_up_sync(FULL, bR[1].t, 1);
    Be[1] = bC[1].e + bR[0].e + __shfl_down_sync(FULL, bL[0].e, 1);
    Bw[1] = bC[1].w + bR[0].w + __shfl_down_sync(FULL, bL[0].w, 1);
    Bt[1] = bC[1].t + bR[0].t + __shfl_down_sync(FULL, bL[0].t, 1);
    // adjoint of (b) and (a): a flooded node took its source's velocities; its height
    // h_min is a constant; a dry node keeps its eta and has no velocity
    float BwL[2], BwR[2], BtL[2], BtR[2];
    nbr(Bw, BwL, BwR); nbr(Bt, BtL, BtR);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        if (o[i]) {
            oe[i] = Be[i];
            ow[i] = Bw[i] + (dirL[i] == 1 ? BwL[i] : 0.f) + (dirR[i] == -1 ? BwR[i] : 0.f);
            ot[i] = Bt[i] + (dirL[i] == 1 ? BtL[i] : 0.f) + (dirR[i] == -1 ? BtR[i] : 0.f);
        } else {
            oe[i] = dir[i] == 0 ? Be[i] : 0.f;
            ow[i] = 0.f;
            ot[i] = 0.f;
        }
    }
}

// ------------------------------------------------------------------ kernels
// Programmatic dependent launch: a kernel launched with programmatic stream serialization
// may start before its predecessor in the stream has finished. grid_dep_wait() returns once
// the predecessor has completed and its writes are visible (at once without the attribute);
// grid_dep_release() lets the successor start (its blocks then fill the SMs this grid's last
// wave leaves idle).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// the pair of nodes pos, pos + 1 of a line (fill outside 0 .. n-1); inner: the caller knows
// both are inside
__device__ __forceinline__ void load2(const float* p, long long o, int pos, int n, float& a, float& b, float fill,
                                      bool inner = false) {
    a = b = fill;
    if (inner || (pos >= 0 && pos + 1 < n)) {
        const float2 v = *reinterpret_cast<const float2*>(p + o + pos);
        a = v.x; b = v.y;
    } else {
        if (pos >= 0 && pos < n) a = p[o + pos];
        if (pos + 1 >= 0 && pos + 1 < n) b = p[o + pos + 1];
    }
}

// Adjoint of the sweeps along one direction. DIR 0: lines are rows of row-major data and
// the output is written transposed; DIR 1: lines are rows of transposed data (columns of
// the grid) and the output is written row-major.
#ifndef CLIFFS_ADJ_LINE_BLOCKS
#define CLIFFS_ADJ_LINE_BLOCKS 3
#endif
template <int DIR, bool SPH, bool S1>
__global__ void __launch_bounds__(AWARPS * 32, SPH ? 2 : CLIFFS_ADJ_LINE_BLOCKS) k_adj_line(const AdjLineArgs A) {
    __shared__ float tile[3][AOUT][TP];
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int strip = blockIdx.x, l0 = blockIdx.y * ALINES;
    const int p0 = strip * AOUT - AHALO;
    const int pA = p0 + 2 * lane;
    const SweepConst K{A.hmin, A.dwall, A.half_dt, A.dt_gn2, A.transverse, A.inv_dt2_s1};
    AMet mb[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int p = pA + i;
        mb[i] = AMet{0.f, 0.f, 0.f, 0.f};
        if (DIR == 0) {
            if (p >= 0 && p < A.npos) mb[i] = AMet{A.xa[p], A.xb[p], A.xk[p], 0.f};
        } else {
            const float4 q = A.ymet[min(max(p, -MET_PAD), A.npos - 1 + MET_PAD)];
            mb[i] = AMet{q.x, q.y, q.z, q.w};
        }
    }
    static_assert(ALINES == AWARPS, "one line per warp");
    const int ln = wi, line = l0 + ln;
    const long long o = (long long)line * A.ipitch;
    float e[2], w[2], t[2], d[2], ge[2], gw[2], gt[2];
    const bool has = line < A.nlines;               // warp-uniform
    const bool inner = p0 >= 0 && p0 + XWIN <= A.npos;   // the window lies inside the line
    // The x-sweep adjoint's primal input (a stored state) and the depth were written before
    // the adjoint steps began: they load while the previous kernel finishes. Everything else
    // comes from the previous kernels of the adjoint step.
    if (DIR == 0 && has) {
        load2(A.pe, o, pA, A.npos, e[0], e[1], 0.f, inner);
        load2(A.pw, o, pA, A.npos, w[0], w[1], 0.f, inner);
        load2(A.pt, o, pA, A.npos, t[0], t[1], 0.f, inner);
    }
    if (has) load2(A.pd, o, pA, A.npos, d[0], d[1], OUTSIDE_D, inner);
    grid_dep_wait();
    grid_dep_release();
    if (has) {
        if (DIR == 1) {
            load2(A.pe, o, pA, A.npos, e[0], e[1], 0.f, inner);
            load2(A.pw, o, pA, A.npos, w[0], w[1], 0.f, inner);
            load2(A.pt, o, pA, A.npos, t[0], t[1], 0.f, inner);
        }
        load2(A.ge, o, pA, A.npos, ge[0], ge[1], 0.f, inner);
        load2(A.gw, o, pA, A.npos, gw[0], gw[1], 0.f, inner);
        load2(A.gt, o, pA, A.npos, gt[0], gt[1], 0.f, inner);
        AMet m[2] = {mb[0], mb[1]};
        if (DIR == 0 && SPH) {
            const float f = A.xrow[line];
#pragma unroll
            for (int i = 0; i < 2; ++i) { m[i].il *= f; m[i].ir *= f; m[i].k2 *= f; }
        }
        float oe[2], ow[2], ot[2];
        unsigned ends = 0u;
        if (A.open_lo | A.open_hi) {
            if (A.open_lo) ends |= (pA == 0 ? 1u : 0u) | (pA + 1 == 0 ? 4u : 0u);
            if (A.open_hi) ends |= (pA == A.npos - 1 ? 2u : 0u) | (pA + 1 == A.npos - 1 ? 8u : 0u);
        }
        line_adjoint<DIR == 1 && SPH, S1>(e, w, t, d, ge, gw, gt, m, K, oe, ow, ot, ends);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = 2 * lane + i - AHALO;
            if (q >= 0 && q < AOUT) {
                tile[0][q][ln] = oe[i];
                tile[1][q][ln] = ow[i];
                tile[2][q][ln] = ot[i];
            }
        }
    }
    __syncthreads();
    if (DIR == 0 && A.seed) {
        // gauge-misfit seed of this step: dL/d (eta, u, v) at each gauge node
        for (int k = threadIdx.x; k < A.G; k += blockDim.x) {
            const int q = A.gxy[2 * k] - strip * AOUT, ln = A.gxy[2 * k + 1] - l0;
            if (q >= 0 && q < AOUT && ln >= 0 && ln < ALINES) {
                atomicAdd(&tile[0][q][ln], A.seed[3 * k]);           // eta
                atomicAdd(&tile[1][q][ln], A.seed[3 * k + 1]);       // u, along the rows
                atomicAdd(&tile[2][q][ln], A.seed[3 * k + 2]);       // v
            }
        }
        __syncthreads();
    }
    // each position's 8 lines are 32 contiguous bytes of the output: two 16-byte stores (the
    // output pitch and planes are multiples of 32 floats, l0 a multiple of 8)
    static_assert(ALINES == 8, "two float4 per output position");
    const bool full = l0 + ALINES <= A.nlines;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        float* out = f == 0 ? A.oe : f == 1 ? A.ow : A.ot;
        const int k = threadIdx.x;
        if (k < 2 * AOUT) {
            const int q = k >> 1, h = (k & 1) * 4;
            const int p = strip * AOUT + q;
            if (p < A.npos) {
                float* dst = out + (long long)p * A.opitch + l0 + h;
                const float4 v = make_float4(tile[f][q][h], tile[f][q][h + 1], tile[f][q][h + 2], tile[f][q][h + 3]);
                if (full) {
                    *reinterpret_cast<float4*>(dst) = v;
                } else {
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (l0 + h + i < A.nlines) dst[i] = vv[i];
                }
            }
        }
    }
}

// The forward x-sweep of a stored state, written transposed ([nx][tpitch]): the same
// window loads, edge treatment and sweep as the fused step kernel.
template <bool SPH, bool FRIC, bool S1, bool OPEN>
__global__ void __launch_bounds__(AWARPS * 32) k_adj_xfwd(const StepArgs a, const float* __restrict__ pe,
                                                          const float* __restrict__ pu,
                                                          const float* __restrict__ pv, float* te, float* tu,
                                                          float* tv, int tpitch) {
    __shared__ float tile[3][XOUT][TP];
    // Launched right behind the x-sweep adjoint of the next step (programmatic launch), this
    // kernel reads a stored state nothing writes any more and overwrites the x-swept buffer
    // whose last reader finished before that kernel got going; it runs in that kernel's last
    // wave and holds its own completion until that kernel has completed, so that the y-sweep
    // adjoint after it sees both.
    grid_dep_release();
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int strip = blockIdx.x, r0 = blockIdx.y * ALINES;
    const int c0 = strip * XOUT - 4, cA = c0 + 2 * lane;
    const SweepConst K{a.hmin, a.dwall, a.half_dt, a.dt_gn2, a.transverse, a.inv_dt2_s1};
    const bool colA = cA >= 0 && cA < a.nx, colB = cA + 1 >= 0 && cA + 1 < a.nx;
    float2 il = v2(0.f), ir = v2(0.f), k2 = v2(0.f);
    if (colA) { il.x = a.xa[cA]; ir.x = a.xb[cA]; k2.x = a.xk[cA]; }
    if (colB) { il.y = a.xa[cA + 1]; ir.y = a.xb[cA + 1]; k2.y = a.xk[cA + 1]; }
    for (int j = 0; j < ALINES / AWARPS; ++j) {
        const int ln = wi * (ALINES / AWARPS) + j;
        const int r = r0 + ln;
        if (r >= a.ny) break;                       // warp-uniform
        const long long o = (long long)r * a.pitch;
        const bool inner = c0 >= 0 && c0 + XWIN <= a.nx;
        float2 E, U, V, D;
        load2(pe, o, cA, a.nx, E.x, E.y, 0.f, inner);
        load2(pu, o, cA, a.nx, U.x, U.y, 0.f, inner);
        load2(pv, o, cA, a.nx, V.x, V.y, 0.f, inner);
        load2(a.d, o, cA, a.nx, D.x, D.y, OUTSIDE_D, inner);
        XMet2 m{il, ir, k2};
        if (SPH) {
            const float2 f = v2(a.xrow[r]);
            m.inv_l = mul2(m.inv_l, f); m.inv_r = mul2(m.inv_r, f); m.k2 = mul2(m.k2, f);
        }
        unsigned ends = 0u;                         // open outer edges among this lane's columns
        if (OPEN) {
            if (a.open_edges & 1) ends |= (cA == 0 ? 1u : 0u) | (cA + 1 == 0 ? 4u : 0u);
            if (a.open_edges & 2) ends |= (cA == a.nx - 1 ? 2u : 0u) | (cA + 1 == a.nx - 1 ? 8u : 0u);
        }
        xsweep2<FRIC, S1, OPEN>(E, U, V, D, m, K, lane, ends);
        const float vals[3][2] = {{E.x, E.y}, {U.x, U.y}, {V.x, V.y}};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int q = 2 * lane + i - 4;
            if (q >= 0 && q < XOUT) {
                tile[0][q][ln] = vals[0][i];
                tile[1][q][ln] = vals[1][i];
                tile[2][q][ln] = vals[2][i];
            }
        }
    }
    __syncthreads();
    const bool full = r0 + ALINES <= a.ny;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        float* out = f == 0 ? te : f == 1 ? tu : tv;
        const int k = threadIdx.x;
        if (k < 2 * XOUT) {
            const int q = k >> 1, h = (k & 1) * 4;
            const int c = strip * XOUT + q;
            if (c < a.nx) {
                float* dst = out + (long long)c * tpitch + r0 + h;
                const float4 v = make_float4(tile[f][q][h], tile[f][q][h + 1], tile[f][q][h + 2], tile[f][q][h + 3]);
                if (full) {
                    *reinterpret_cast<float4*>(dst) = v;
                } else {
                    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (r0 + h + i < a.ny) dst[i] = vv[i];
                }
            }
        }
    }
    grid_dep_wait();
}

// out[c][r] = in[r][c] for r < rows, c < cols (32 x 32 tiles through shared memory)
__global__ void __launch_bounds__(256) k_transpose(const float* __restrict__ in, int ipitch, float* out,
                                                   int opitch, int rows, int cols) {
    __shared__ float t[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.x; k < 1024; k += 256) {
        const int r = r0 + k / 32, c = c0 + k % 32;
        if (r < rows && c < cols) t[k / 32][k % 32] = in[(long long)r * ipitch + c];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < 1024; k += 256) {
        const int c = c0 + k / 32, r = r0 + k % 32;
        if (r < rows && c < cols) out[(long long)c * opitch + r] = t[k % 32][k / 32];
    }
}

// lambda.eta[gauge] += seed[gauge] on transposed data
__global__ void k_adj_seed(float* te, int tpitch, long long tplane, const int* gxy, int G, const float* seed) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= G) return;
    const long long o = (long long)gxy[2 * k] * tpitch + gxy[2 * k + 1];
    atomicAdd(te + o, seed[3 * k]);                          // eta
    atomicAdd(te + tplane + o, seed[3 * k + 1]);             // u
    atomicAdd(te + 2 * tplane + o, seed[3 * k + 2]);         // v
}

// lambda = 0 on the edges whose nodes the boundary input overwrites before a step (mask:
// 1 W, 2 E, 4 S, 8 N), on the transposed adjoint ([nx][tpitch], three fields)
__global__ void k_adj_zero_edges(float* t, int tpitch, long long tplane, int nx, int ny, int mask) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int e = blockIdx.y;
    if (!((mask >> e) & 1)) return;
    const int np = e < 2 ? ny : nx;
    if (q >= np) return;
    const int ix = e == 0 ? 0 : e == 1 ? nx - 1 : q;
    const int iy = e == 2 ? 0 : e == 3 ? ny - 1 : q;
    const long long o = (long long)ix * tpitch + iy;
    t[o] = 0.f;
    t[o + tplane] = 0.f;
    t[o + 2 * tplane] = 0.f;
}

cudaError_t launch_adj_zero_edges(float* t, int tpitch, int nx, int ny, int mask, cudaStream_t s) {
    const int np = nx > ny ? nx : ny;
    k_adj_zero_edges<<<dim3((np + 127) / 128, 4), 128, 0, s>>>(t, tpitch, (long long)tpitch * nx, nx, ny, mask);
    return cudaGetLastError();
}

// a launch that may start before its predecessor in the stream has finished
static cudaError_t launch_pdl(const void* k, dim3 grid, dim3 block, void** args, cudaStream_t s, bool pdl) {
    if (!pdl) return cudaLaunchKernel(k, grid, block, args, 0, s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, k, args);
}

cudaError_t launch_adj_line(const AdjLineArgs& A, int dir, bool sph, cudaStream_t s, bool pdl) {
    const dim3 grid((A.npos + AOUT - 1) / AOUT, (A.nlines + ALINES - 1) / ALINES);
    static const void* const t[8] = {(const void*)k_adj_line<0, false, false>, (const void*)k_adj_line<0, true, false>,
                                     (const void*)k_adj_line<1, false, false>, (const void*)k_adj_line<1, true, false>,
                                     (const void*)k_adj_line<0, false, true>, (const void*)k_adj_line<0, true, true>,
                                     (const void*)k_adj_line<1, false, true>, (const void*)k_adj_line<1, true, true>};
    AdjLineArgs aa = A;
    void* args[] = {&aa};
    return launch_pdl(t[(sph ? 1 : 0) + (dir ? 2 : 0) + (A.inv_dt2_s1 > 0.f ? 4 : 0)], grid, dim3(AWARPS * 32),
                      args, s, pdl);
}

cudaError_t launch_adj_xfwd(const StepArgs& a, const float* e, const float* u, const float* v, float* te,
                            float* tu, float* tv, int tpitch, cudaStream_t s, bool pdl) {
    const dim3 grid((a.nx + XOUT - 1) / XOUT, (a.ny + ALINES - 1) / ALINES);
    static const void* const t[16] = {
        (const void*)k_adj_xfwd<false, false, false, false>, (const void*)k_adj_xfwd<true, false, false, false>,
        (const void*)k_adj_xfwd<false, true, false, false>, (const void*)k_adj_xfwd<true, true, false, false>,
        (const void*)k_adj_xfwd<false, false, true, false>, (const void*)k_adj_xfwd<true, false, true, false>,
        (const void*)k_adj_xfwd<false, true, true, false>, (const void*)k_adj_xfwd<true, true, true, false>,
        (const void*)k_adj_xfwd<false, false, false, true>, (const void*)k_adj_xfwd<true, false, false, true>,
        (const void*)k_adj_xfwd<false, true, false, true>, (const void*)k_adj_xfwd<true, true, false, true>,
        (const void*)k_adj_xfwd<false, false, true, true>, (const void*)k_adj_xfwd<true, false, true, true>,
        (const void*)k_adj_xfwd<false, true, true, true>, (const void*)k_adj_xfwd<true, true, true, true>};
    StepArgs aa = a;
    void* args[] = {&aa, (void*)&e, (void*)&u, (void*)&v, &te, &tu, &tv, &tpitch};
    return launch_pdl(t[(a.sph ? 1 : 0) + (a.dt_gn2 > 0.f ? 2 : 0) + (a.inv_dt2_s1 > 0.f ? 4 : 0) +
                        (a.open_edges ? 8 : 0)],
                      grid, dim3(AWARPS * 32), args, s, pdl);
}

cudaError_t launch_transpose(const float* in, int ipitch, float* out, int opitch, int rows, int cols,
                             cudaStream_t s) {
    const dim3 grid((cols + 31) / 32, (rows + 31) / 32);
    k_transpose<<<grid, 256, 0, s>>>(in, ipitch, out, opitch, rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_adj_seed(float* te, int tpitch, long long tplane, const int* gxy, int G, const float* seed,
                            cudaStream_t s) {
    if (G <= 0) return cudaSuccess;
    k_adj_seed<<<(G + 127) / 128, 128, 0, s>>>(te, tpitch, tplane, gxy, G, seed);
    return cudaGetLastError();
}

}  // namespace cliffs
