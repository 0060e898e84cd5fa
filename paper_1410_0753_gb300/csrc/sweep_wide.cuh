// Four-node-per-lane forms of the sweep building blocks (arXiv 1410.0753, section
// "Numerics"; steps (a)-(e) of section "Inundation algorithm"), for the wide step kernel.
//
// A lane owns four neighbouring nodes n0..n3 of a 128-column window, held as two packed
// pairs a = (n0, n1) and b = (n2, n3). Three of a lane's four interfaces are inside the lane;
// only n0's left and n3's right neighbours come from the neighbouring lanes, so a row needs
// half the shuffles and votes per node of the two-node form, and the two pairs give every
// warp two independent chains of packed arithmetic. Every node is updated by the same
// sequence of operations as in xsweep2 / YMarch2 (the same iface2, node_update2, flood1 and
// cushion calls on the same operands), so both forms give the same bits.
#pragma once
#include "sweep.cuh"

namespace cliffs {

constexpr int WWIN = 128;                 // columns a warp holds in the wide x-sweep (4 per lane)
constexpr int WOUT = 120;                 // columns it finishes: 4-column halo per side

// x-sweep of one row segment of 128 columns: lane l holds window columns 4l .. 4l+3 as pairs
// a (.x = 4l, .y = 4l+1) and b (.x = 4l+2, .y = 4l+3). On return the pairs hold the sweep
// result, valid for window columns 4..123.
template <bool FRIC>
__device__ __forceinline__ void xsweep4(float2& Ea, float2& Wa, float2& Ta, const float2 Da, const XMet2& ma,
                                        float2& Eb, float2& Wb, float2& Tb, const float2 Db, const XMet2& mb,
                                        const SweepConst& K, int lane) {
    const bool o0 = wet_mark(Ea.x, Da.x, K), o1 = wet_mark(Ea.y, Da.y, K);
    const bool o2 = wet_mark(Eb.x, Db.x, K), o3 = wet_mark(Eb.y, Db.y, K);
    const bool allwet = __all_sync(FULL, o0 && o1 && o2 && o3);
    bool w0 = o0, w1 = o1, w2 = o2, w3 = o3;   // wet after (b)
    int d0 = 0, d1 = 0, d2 = 0, d3 = 0;        // (b) source directions
    if (!allwet) {
        if (!o0) { Wa.x = 0.f; Ta.x = 0.f; }    // (a): a dry node is at rest
        if (!o1) { Wa.y = 0.f; Ta.y = 0.f; }
        if (!o2) { Wb.x = 0.f; Tb.x = 0.f; }
        if (!o3) { Wb.y = 0.f; Tb.y = 0.f; }
        const unsigned b3 = __ballot_sync(FULL, o3), b0 = __ballot_sync(FULL, o0);
        const bool oL = lane > 0 && ((b3 >> (lane - 1)) & 1u);
        const bool oR = lane < 31 && ((b0 >> (lane + 1)) & 1u);
        const bool c0 = !o0 && Da.x >= K.dwall && (oL || o1);
        const bool c1 = !o1 && Da.y >= K.dwall && (o0 || o2);
        const bool c2 = !o2 && Db.x >= K.dwall && (o1 || o3);
        const bool c3 = !o3 && Db.y >= K.dwall && (o2 || oR);
        if (__any_sync(FULL, c0 || c1 || c2 || c3)) {
            const float eL = __shfl_up_sync(FULL, Eb.y, 1), eR = __shfl_down_sync(FULL, Ea.x, 1);
            const bool q0 = c0 && ((oL && eL + Da.x > K.hmin) || (o1 && Ea.y + Da.x > K.hmin));
            const bool q1 = c1 && ((o0 && Ea.x + Da.y > K.hmin) || (o2 && Eb.x + Da.y > K.hmin));
            const bool q2 = c2 && ((o1 && Ea.y + Db.x > K.hmin) || (o3 && Eb.y + Db.x > K.hmin));
            const bool q3 = c3 && ((o2 && Eb.x + Db.y > K.hmin) || (oR && eR + Db.y > K.hmin));
            if (__any_sync(FULL, q0 || q1 || q2 || q3)) {
                const float wL = __shfl_up_sync(FULL, Wb.y, 1), tL = __shfl_up_sync(FULL, Tb.y, 1);
                const float wR = __shfl_down_sync(FULL, Wa.x, 1), tR = __shfl_down_sync(FULL, Ta.x, 1);
                // start-of-sweep values of the four nodes as sources
                const float e0 = Ea.x, e1 = Ea.y, e2 = Eb.x, e3 = Eb.y;
                const float u0 = Wa.x, u1 = Wa.y, u2 = Wb.x, u3 = Wb.y;
                const float t0 = Ta.x, t1 = Ta.y, t2 = Tb.x, t3 = Tb.y;
                if (q0) { d0 = flood1(Ea.x, Wa.x, Ta.x, Da.x, eL, wL, tL, oL, e1, u1, t1, o1, K.hmin); w0 = true; }
                if (q1) { d1 = flood1(Ea.y, Wa.y, Ta.y, Da.y, e0, u0, t0, o0, e2, u2, t2, o2, K.hmin); w1 = true; }
                if (q2) { d2 = flood1(Eb.x, Wb.x, Tb.x, Db.x, e1, u1, t1, o1, e3, u3, t3, o3, K.hmin); w2 = true; }
                if (q3) { d3 = flood1(Eb.y, Wb.y, Tb.y, Db.y, e2, u2, t2, o2, eR, wR, tR, oR, K.hmin); w3 = true; }
            }
        }
    }
    const float2 Ca = wave_speed2(add2(Ea, Da)), Cb = wave_speed2(add2(Eb, Db));
    // post-(b) state of n0 of the next lane
    const float eR = __shfl_down_sync(FULL, Ea.x, 1), wR = __shfl_down_sync(FULL, Wa.x, 1);
    const float tR = __shfl_down_sync(FULL, Ta.x, 1), dR = __shfl_down_sync(FULL, Da.x, 1);
    const float cR = __shfl_down_sync(FULL, Ca.x, 1);
    // right interfaces: a -> (n0|n1), (n1|n2); b -> (n2|n3), (n3|n0')
    Flux2 FRa = iface2(Ea, Wa, Ta, Da, Ca, make_float2(Ea.y, Eb.x), make_float2(Wa.y, Wb.x),
                       make_float2(Ta.y, Tb.x), make_float2(Da.y, Db.x), make_float2(Ca.y, Cb.x), ma.inv_r);
    Flux2 FRb = iface2(Eb, Wb, Tb, Db, Cb, make_float2(Eb.y, eR), make_float2(Wb.y, wR),
                       make_float2(Tb.y, tR), make_float2(Db.y, dR), make_float2(Cb.y, cR), mb.inv_r);
    // left interfaces: a -> (n3 of the lane below | n0), (n0|n1); b -> (n1|n2), (n2|n3)
    Flux2 FLa, FLb;
    FLa.p = make_float2(__shfl_up_sync(FULL, FRb.p.y, 1), FRa.p.x);
    FLa.q = make_float2(__shfl_up_sync(FULL, FRb.q.y, 1), FRa.q.x);
    FLa.t = make_float2(__shfl_up_sync(FULL, FRb.t.y, 1), FRa.t.x);
    FLb.p = make_float2(FRa.p.y, FRb.p.x);
    FLb.q = make_float2(FRa.q.y, FRb.q.x);
    FLb.t = make_float2(FRa.t.y, FRb.t.x);
    if (!allwet) {
        // (c): walls between wet and dry nodes
        const unsigned v3 = __ballot_sync(FULL, w3), v0 = __ballot_sync(FULL, w0);
        const bool wetL = lane > 0 && ((v3 >> (lane - 1)) & 1u);
        const bool wetR = lane < 31 && ((v0 >> (lane + 1)) & 1u);
        if (!wetL) ghost_left(Wa.x, Ca.x, ma.inv_l.x, FLa.p.x, FLa.q.x, FLa.t.x);
        if (!w1) ghost_right(Wa.x, Ca.x, ma.inv_r.x, FRa.p.x, FRa.q.x, FRa.t.x);
        if (!w0) ghost_left(Wa.y, Ca.y, ma.inv_l.y, FLa.p.y, FLa.q.y, FLa.t.y);
        if (!w2) ghost_right(Wa.y, Ca.y, ma.inv_r.y, FRa.p.y, FRa.q.y, FRa.t.y);
        if (!w1) ghost_left(Wb.x, Cb.x, mb.inv_l.x, FLb.p.x, FLb.q.x, FLb.t.x);
        if (!w3) ghost_right(Wb.x, Cb.x, mb.inv_r.x, FRb.p.x, FRb.q.x, FRb.t.x);
        if (!w2) ghost_left(Wb.y, Cb.y, mb.inv_l.y, FLb.p.y, FLb.q.y, FLb.t.y);
        if (!wetR) ghost_right(Wb.y, Cb.y, mb.inv_r.y, FRb.p.y, FRb.q.y, FRb.t.y);
    }
    float2 E2a, W2a, T2a, E2b, W2b, T2b;
    node_update2<false, FRIC, false>(Ea, Wa, Ta, Da, Ca, FLa, FRa, ma.k2, v2(0.f), K, E2a, W2a, T2a);
    node_update2<false, FRIC, false>(Eb, Wb, Tb, Db, Cb, FLb, FRb, mb.k2, v2(0.f), K, E2b, W2b, T2b);
    if (!allwet) {
        if (!w0) { E2a.x = Ea.x; W2a.x = Wa.x; T2a.x = Ta.x; }
        if (!w1) { E2a.y = Ea.y; W2a.y = Wa.y; T2a.y = Ta.y; }
        if (!w2) { E2b.x = Eb.x; W2b.x = Wb.x; T2b.x = Tb.x; }
        if (!w3) { E2b.y = Eb.y; W2b.y = Wb.y; T2b.y = Tb.y; }
        if (__any_sync(FULL, (d0 | d1 | d2 | d3) != 0)) {
            // (e) against the neighbours' state after (d)
            const float h0 = E2a.x + Da.x, h1 = E2a.y + Da.y, h2 = E2b.x + Db.x, h3 = E2b.y + Db.y;
            const float hL = __shfl_up_sync(FULL, h3, 1), wLn = __shfl_up_sync(FULL, W2b.y, 1);
            const float hR = __shfl_down_sync(FULL, h0, 1), wRn = __shfl_down_sync(FULL, W2a.x, 1);
            const float s0 = W2a.x, s1 = W2a.y, s2 = W2b.x, s3 = W2b.y;
            if (d0 < 0) cushion(E2a.x, W2a.x, Da.x, hL, wLn);
            else if (d0 > 0) cushion(E2a.x, W2a.x, Da.x, h1, s1);
            if (d1 < 0) cushion(E2a.y, W2a.y, Da.y, h0, s0);
            else if (d1 > 0) cushion(E2a.y, W2a.y, Da.y, h2, s2);
            if (d2 < 0) cushion(E2b.x, W2b.x, Db.x, h1, s1);
            else if (d2 > 0) cushion(E2b.x, W2b.x, Db.x, h3, s3);
            if (d3 < 0) cushion(E2b.y, W2b.y, Db.y, h2, s2);
            else if (d3 > 0) cushion(E2b.y, W2b.y, Db.y, hR, wRn);
        }
    }
    Ea = E2a; Wa = W2a; Ta = T2a;
    Eb = E2b; Wb = W2b; Tb = T2b;
}

// The y-sweep pipeline of one pair of columns (the state of YMarch2) with its push split in
// two, so that a warp holding two pairs decides the open-water path once for both: fast_ok
// is this pair's vote, fast and slow the two paths of YMarch2::push (the finished row k-3
// returned in oe, ow, ot, od instead of passed to an emitter). eq. (solver2) only.
struct YPair : YMarch2 {
    template <int PH>
    __device__ __forceinline__ bool fast_ok(bool careA, bool careB) const {
        const YRow& P = bank[PH];
        const YRow& B1 = bank[1 - PH];
        const bool openA = B1.oA && P.wA && f3A && dir3A == 0;
        const bool openB = B1.oB && P.wB && f3B && dir3B == 0;
        return (!careA || openA) && (!careB || openB);
    }

    template <int PH>
    __device__ __forceinline__ void advance(float2 E0, float2 W0, float2 T0, float2 D0, bool o0A, bool o0B) {
        YRow& P = bank[PH];
        d3 = P.d;
        dir3A = P.dA; dir3B = P.dB;
        f3A = P.wA; f3B = P.wB;
        P.e = E0; P.w = W0; P.t = T0; P.d = D0;
        P.oA = o0A; P.oB = o0B;
    }

    template <int PH, bool SRC, bool FRIC>
    __device__ __forceinline__ void fast(float2 E0, float2 W0, float2 T0, float2 D0, bool o0A, bool o0B,
                                         float4 m2, const SweepConst& K,
                                         float2& oe, float2& ow, float2& ot, float2& od) {
        YRow& P = bank[PH];
        YRow& B1 = bank[1 - PH];
        Flux2& F3 = fb[PH];
        Flux2& F2 = fb[1 - PH];
        B1.wA = B1.wB = true;
        B1.dA = B1.dB = 0;
        B1.c = wave_speed2(add2(B1.e, B1.d));
        F2 = iface2(P.e, P.w, P.t, P.d, P.c, B1.e, B1.w, B1.t, B1.d, B1.c, v2(m2.y));
        oe = e3; ow = w3; ot = t3; od = d3;
        h4 = add2(e3, d3);
        w4 = w3;
        node_update2<SRC, FRIC, false>(P.e, P.w, P.t, P.d, P.c, F3, F2, v2(m2.z), v2(m2.w), K, e3, w3, t3);
        advance<PH>(E0, W0, T0, D0, o0A, o0B);
    }

    template <int PH, bool SRC, bool FRIC>
    __device__ __forceinline__ void slow(float2 E0, float2 W0, float2 T0, float2 D0, bool o0A, bool o0B,
                                         float4 m2, const SweepConst& K,
                                         float2& oe, float2& ow, float2& ot, float2& od) {
        YRow& P = bank[PH];
        YRow& B1 = bank[1 - PH];
        Flux2& F3 = fb[PH];
        Flux2& F2 = fb[1 - PH];
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
        float2 ne, nw, nt;
        node_update2<SRC, FRIC, false>(P.e, P.w, P.t, P.d, P.c, L, R, v2(m2.z), v2(m2.w), K, ne, nw, nt);
        if (!P.wA) { ne.x = P.e.x; nw.x = P.w.x; nt.x = P.t.x; }
        if (!P.wB) { ne.y = P.e.y; nw.y = P.w.y; nt.y = P.t.y; }
        // (e) on row k-3, against row k-4 (h4, w4) or row k-2 (ne, nw)
        oe = e3; ow = w3;
        if (dir3A != 0) cushion(oe.x, ow.x, d3.x, dir3A < 0 ? h4.x : ne.x + P.d.x, dir3A < 0 ? w4.x : nw.x);
        if (dir3B != 0) cushion(oe.y, ow.y, d3.y, dir3B < 0 ? h4.y : ne.y + P.d.y, dir3B < 0 ? w4.y : nw.y);
        ot = t3; od = d3;
        h4 = add2(e3, d3);
        w4 = w3;
        e3 = ne; w3 = nw; t3 = nt;
        advance<PH>(E0, W0, T0, D0, o0A, o0B);
    }
};

}  // namespace cliffs
