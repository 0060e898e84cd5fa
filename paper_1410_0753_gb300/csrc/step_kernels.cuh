// Kernel templates of the split step (arXiv 1410.0753, section "Numerics"); instantiated by
// cliffs_step.cu (reflecting outer edges) and cliffs_step_open.cu (open outer edges, OPEN).
// The kernels and their work split are described at the top of cliffs_step.cu.
#pragma once
#include "internal.h"
#include "sweep.cuh"

namespace cliffs {

constexpr int RING = 4;                       // slots in flight per warp
constexpr int SLOT_ROWS = TMA_BOX_ROWS;       // rows per slot (one TMA box each array)
static_assert(TMA_BOX_COLS == XWIN, "a TMA box spans the warp's window");
constexpr int NARR = 6;                       // eta, u, v, d, eta_max, speed_max
constexpr int ARR_FLOATS = SLOT_ROWS * XWIN;
constexpr int SLOT_FLOATS = NARR * ARR_FLOATS;
constexpr int WARP_RING_BYTES = RING * SLOT_FLOATS * 4;
constexpr int FUSED_WARPS = 4;
constexpr int FUSED_SMEM = FUSED_WARPS * (WARP_RING_BYTES + RING * 8);

// ------------------------------------------------------------------ TMA / mbarrier (PTX)
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r) : "r"(smem_u32(b)), "r"(parity) : "memory");
    return r != 0;
}
// bounded wait for the phase with the given parity
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, long long limit) {
    if (mbar_test(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(b, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void tma_row3(float* dst, const CUtensorMap* m, uint64_t* b, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(m)), "r"(smem_u32(b)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// ------------------------------------------------------------------ epilogue
// Nodes (r, c) and (r, c+1) of the step input, for the kernels without TMA; nodes outside
// the domain get depth OUTSIDE_D (dry, never wetted) and zero state.
__device__ __forceinline__ void load_pair(const StepArgs& a, size_t boff, int r, int c,
                                          float2& E, float2& U, float2& V, float2& D) {
    E = U = V = make_float2(0.f, 0.f);
    D = make_float2(OUTSIDE_D, OUTSIDE_D);
    if (r >= 0 && r < a.ny && c >= 0 && c < a.nx) {
        const size_t o = (size_t)r * a.pitch + c;
        E = __ldg(reinterpret_cast<const float2*>(a.eta_in + boff + o));
        U = __ldg(reinterpret_cast<const float2*>(a.u_in + boff + o));
        V = __ldg(reinterpret_cast<const float2*>(a.v_in + boff + o));
        D = __ldg(reinterpret_cast<const float2*>(a.d + o));
        if (c + 1 >= a.nx) { E.y = U.y = V.y = 0.f; D.y = OUTSIDE_D; }
    }
}

// Open outer edges of a lane's pair of columns for xsweep2 (bits 1 A left, 2 A right, 4 B
// left, 8 B right) and of a row for the y-sweep pipeline (1 first row, 2 last row, 0 none).
__device__ __forceinline__ unsigned open_ends_x(const StepArgs& a, int cA) {
    unsigned e = 0u;
    if (a.open_edges & 1) { if (cA == 0) e |= 1u; if (cA + 1 == 0) e |= 4u; }
    if (a.open_edges & 2) { if (cA == a.nx - 1) e |= 2u; if (cA + 1 == a.nx - 1) e |= 8u; }
    return e;
}
__device__ __forceinline__ int open_end_y(const StepArgs& a, int row) {
    return (row == 0 && (a.open_edges & 4)) ? 1 : (row == a.ny - 1 && (a.open_edges & 8)) ? 2 : 0;
}

__device__ __forceinline__ int runaway(float e, float u, float v) {
    return !(fabsf(e) + fabsf(u) + fabsf(v) < 3e5f);
}
// The same test accumulated branch-free over the rows of a warp's work: the sum of
// e^2 + u^2 + v^2 over its stored nodes reaches 9e10 when any node reaches 3e5 in a component
// (no physical state sums that high over a warp's few thousand nodes), and a non-finite
// value makes it non-finite.
constexpr float RUNAWAY_SQ = 9e10f;

// What changes from one step to the next: the input state's TMA descriptors, the output
// planes, and the max-wave fields and record rows when they are due this step (else null).
struct StepOut {
    const StepMaps* M;
    float* eta_out;
    float* u_out;
    float* v_out;
    float* emax;
    float* smax;
    float* rec_g;
    float* rec_n;
};

__device__ __forceinline__ StepOut step_out(const StepMaps* M, const StepArgs& a) {
    return StepOut{M, a.eta_out, a.u_out, a.v_out, a.emax, a.smax, a.rec_g, a.rec_n};
}

// Store a finished pair of nodes of row r. With max-wave due (section "Running Options",
// field maxout), (em, sm) hold the stored maxima of the pair (loaded beforehand); on wet
// nodes they take the new eta and speed sqrt(u^2 + v^2) where these are larger and are
// written back.
// With CHECK the runaway test runs here (the fused kernels accumulate it instead, chk_out).
template <bool CHECK = true>
__device__ __forceinline__ void emit_pair(const StepArgs& a, const StepOut& O, size_t o, bool va, bool vb,
                                          float2 E, float2 U, float2 V, float2 D,
                                          float2 em, float2 sm, int& bad) {
    if (!va) return;
    if (vb) {
        *reinterpret_cast<float2*>(O.eta_out + o) = E;
        *reinterpret_cast<float2*>(O.u_out + o) = U;
        *reinterpret_cast<float2*>(O.v_out + o) = V;
        if (CHECK) bad |= runaway(E.x, U.x, V.x) | runaway(E.y, U.y, V.y);
    } else {
        O.eta_out[o] = E.x; O.u_out[o] = U.x; O.v_out[o] = V.x;
        if (CHECK) bad |= runaway(E.x, U.x, V.x);
    }
    if (O.emax) {
        // max-wave of the pair (wet nodes only), the tests in packed form
        const float2 h = add2(E, D);
        const float2 s2 = fma2(U, U, mul2(V, V));
        const float2 sm2 = mul2(sm, sm);
        const bool wA = (D.x >= a.dwall) && (h.x >= a.hmin);
        const bool wB = vb && (D.y >= a.dwall) && (h.y >= a.hmin);
        const bool eA = wA && E.x > em.x, eB = wB && E.y > em.y;
        const bool sA = wA && s2.x > sm2.x, sB = wB && s2.y > sm2.y;
        if (eA || eB || sA || sB) {
            if (eA) em.x = E.x;
            if (eB) em.y = E.y;
            if (sA) sm.x = fmaxf(sm.x, sqrt_pos(s2.x));
            if (sB) sm.y = fmaxf(sm.y, sqrt_pos(s2.y));
            if (vb) {
                *reinterpret_cast<float2*>(O.emax + o) = em;
                *reinterpret_cast<float2*>(O.smax + o) = sm;
            } else {
                O.emax[o] = em.x; O.smax[o] = sm.x;
            }
        }
    }
}

// Gauge / enclosed-grid node samples owned by this warp, sorted by row. The warp keeps 32
// consecutive sample records in registers (lane l holds record base + l). For a row with
// samples, every lane whose record belongs to that row fetches the node's values from the
// lane that owns the node by shuffle and writes the record, so all samples of a row go out
// together; `next` holds the row of the next sample so rows without samples cost a compare.
// The writer is a separate (not inlined) function: it runs on the few rows with samples,
// and kept out of the row loop it leaves the loop's code to the sweeps.
struct Samples {
    int sp, se, base, next;
    int4 mine;

    __device__ __forceinline__ void load(const int4* samp, int lane) {
        base = sp;
        mine = (sp + lane < se) ? __ldg(samp + sp + lane) : make_int4(0x7fffffff, 0, 0, 0);
    }
    __device__ __forceinline__ void init(const StepArgs& a, const StepOut& O, int gw, int lane) {
        sp = se = base = 0;
        next = 0x7fffffff;
        mine = make_int4(0x7fffffff, 0, 0, 0);
        if (a.samp_ptr && (O.rec_g || O.rec_n)) {
            sp = a.samp_ptr[gw];
            se = a.samp_ptr[gw + 1];
            if (sp < se) {
                load(a.samp, lane);
                next = __shfl_sync(FULL, mine.x, 0);
            }
        }
    }
    __device__ __forceinline__ void emit(const StepArgs& a, const StepOut& O, int b, int r, int c0,
                                         int lane, float2 E, float2 U, float2 V);
};

// the samples of row r (warp-collective); returns the updated sample cursor
static __device__ __noinline__ Samples samples_write(Samples S, const int4* samp, float* rec_g, float* rec_n, int r,
                                                     int c0, int lane, float2 E, float2 U, float2 V) {
    while (true) {
        const bool mineRow = lane >= S.sp - S.base && S.mine.x == r;
        const int rel = S.mine.y - c0;
        const int src = mineRow ? (rel >> 1) & 31 : lane;
        const float ex = __shfl_sync(FULL, E.x, src), ey = __shfl_sync(FULL, E.y, src);
        const float ux = __shfl_sync(FULL, U.x, src), uy = __shfl_sync(FULL, U.y, src);
        const float vx = __shfl_sync(FULL, V.x, src), vy = __shfl_sync(FULL, V.y, src);
        if (mineRow) {
            const bool isB = rel & 1;
            float* out = (S.mine.z == 0) ? rec_g : rec_n;
            if (out) {
                out[3 * S.mine.w + 0] = isB ? ey : ex;
                out[3 * S.mine.w + 1] = isB ? uy : ux;
                out[3 * S.mine.w + 2] = isB ? vy : vx;
            }
        }
        S.sp += __popc(__ballot_sync(FULL, mineRow));
        if (S.sp >= S.se) { S.next = 0x7fffffff; return S; }
        if (S.sp - S.base < 32) {                  // the next record is cached: a later row
            S.next = __shfl_sync(FULL, S.mine.x, S.sp - S.base);
            return S;
        }
        S.load(samp, lane);                        // the row's records run past the cache
        S.next = __shfl_sync(FULL, S.mine.x, 0);
        if (S.next != r) return S;
    }
}

__device__ __forceinline__ void Samples::emit(const StepArgs& a, const StepOut& O, int b, int r, int c0,
                                              int lane, float2 E, float2 U, float2 V) {
    if (r != next) return;
    *this = samples_write(*this, a.samp, O.rec_g ? O.rec_g + (long long)b * a.rec_g_bstride : nullptr, O.rec_n,
                          r, c0, lane, E, U, V);
}

// ------------------------------------------------------------------ fused step
// One warp of the fused step. A work item is a strip and an output row range [r0, r1); the
// warp walks rows r0-3 .. r1+2 as pairs, one pair per ring slot. The ring's slot and phase
// follow a running pair count, so a warp may process any number of items in a row. With YF
// (a y-first step of the alternating order) rows enter the y-sweep pipeline unswept and each
// finished row is x-swept across the warp on its way out; the tile geometry is the same.
template <bool SPH, bool FRIC, bool YF = false, bool S1 = false, bool OPEN = false>
struct FusedWarp {
    const StepArgs& a;
    SweepConst K;
    float* ring;
    uint64_t* bar;
    unsigned used;             // ring pairs consumed by this warp so far (2^32 is a multiple of 2 * RING)
    int lane, b, c0, cA, r0, r1, k0, npairs;
    size_t orow;               // output offset of row r0 (scenario plane + column)
    bool colA, colB, vA, vB, edge;
    bool bounded;              // the window starts or ends at the domain's edge (xsweep2)
    unsigned tx, nbox;
    unsigned ends;             // open outer edges among this lane's columns (open_ends_x)
    XMet2 m0;
    YMarch2 ym;
    Samples smp;
    StepOut O;
    int bad;
    float2 chk_x;              // sum of 0 * (x-swept eta): 0, or NaN once a value is not finite
    float2 chk_out;            // sum of e^2 + u^2 + v^2 over the stored nodes (RUNAWAY_SQ)

    __device__ __forceinline__ FusedWarp(const StepArgs& a_) : a(a_) {}

    __device__ __forceinline__ void setup(unsigned char* smem_raw, int wib) {
        lane = threadIdx.x & 31;
        K = SweepConst{a.hmin, a.dwall, a.half_dt, a.dt_gn2, a.transverse, a.inv_dt2_s1};
        ring = reinterpret_cast<float*>(smem_raw + wib * WARP_RING_BYTES);
        bar = reinterpret_cast<uint64_t*>(smem_raw + FUSED_WARPS * WARP_RING_BYTES) + wib * RING;
        used = 0;
        bad = 0;
        chk_x = chk_out = v2(0.f);
        if (lane == 0) {
            for (int s = 0; s < RING; ++s) mbar_init(&bar[s], 1);
            fence_mbar_init();
        }
        __syncwarp();
    }

    // lanes 0..nbox-1 each start one 64 x 2 box of the item's row pair j into its ring slot
    __device__ __forceinline__ void issue(int j) {
        const int slot = (int)((used + (unsigned)j) % RING);
        const int row = k0 + SLOT_ROWS * j;
        if (lane == 0) mbar_arrive_tx(&bar[slot], tx);
        if (lane < (int)nbox) {
            fence_proxy_async();
            tma_row3(ring + slot * SLOT_FLOATS + lane * ARR_FLOATS, &O.M->e + lane, &bar[slot], c0,
                     lane >= 4 ? row - 3 : row, lane == 3 ? 0 : b);
        }
    }

    // row k held at `s`: its values (zero state, dry depth outside the domain) and x metric
    __device__ __forceinline__ bool load_row(int k, const float* s, float2& E, float2& U, float2& V, float2& D,
                                             XMet2& m) {
        E = reinterpret_cast<const float2*>(s + 0 * ARR_FLOATS)[lane];
        U = reinterpret_cast<const float2*>(s + 1 * ARR_FLOATS)[lane];
        V = reinterpret_cast<const float2*>(s + 2 * ARR_FLOATS)[lane];
        D = reinterpret_cast<const float2*>(s + 3 * ARR_FLOATS)[lane];
        const bool rowin = k >= 0 && k < a.ny;
        if (edge || !rowin) {
            if (!(rowin && colA)) { E.x = U.x = V.x = 0.f; D.x = OUTSIDE_D; }
            if (!(rowin && colB)) { E.y = U.y = V.y = 0.f; D.y = OUTSIDE_D; }
        }
        m = m0;
        if (SPH && rowin) {
            const float2 f = v2(__ldg(a.xrow + k));
            m.inv_l = mul2(m.inv_l, f); m.inv_r = mul2(m.inv_r, f); m.k2 = mul2(m.k2, f);
        }
        return rowin;
    }

    // the x-swept row k into the y-sweep pipeline; the finished row k - 3 goes out
    template <int PH>
    __device__ __forceinline__ void push_row(int k, const float* s, float2 E, float2 U, float2 V, float2 D) {
        const float4 m2 = __ldg(a.ymet + k - 2);
        // y-sweep input of row k: eta, w = v, t = u
        const bool oA = wet_mark(E.x, D.x, K), oB = wet_mark(E.y, D.y, K);
        // a non-finite x-sweep result reads as a dry node in the y-sweep and would be
        // refilled by step (b) there: it is caught here (0 * NaN or 0 * inf is NaN)
        chk_x = fma2(E, v2(0.f), chk_x);
        const int r = k - 3;
        // the y-sweep results a lane must get right: its own output columns, and with YF every
        // column of the window (the x-sweep on the way out reads three columns past the outputs)
        ym.template push<PH, SPH, FRIC, S1, OPEN>(E, V, U, D, oA, oB, m2, K, YF ? colA : vA, YF ? colB : vB,
            [&](float2 oe, float2 ow, float2 ot, float2 od) {
                if (r >= r0 && r < r1) {
                    if (YF) {
                        // x-sweep of the y-swept row r: along-row velocity u (ot), across v (ow)
                        XMet2 mr = m0;
                        if (SPH) {
                            const float2 f = v2(__ldg(a.xrow + r));
                            mr.inv_l = mul2(mr.inv_l, f); mr.inv_r = mul2(mr.inv_r, f); mr.k2 = mul2(mr.k2, f);
                        }
                        xsweep2<FRIC, S1, OPEN>(oe, ot, ow, od, mr, K, lane, ends, bounded);
                    }
                    float2 em = make_float2(0.f, 0.f), sm = em;
                    if (O.emax) {
                        em = reinterpret_cast<const float2*>(s + 4 * ARR_FLOATS)[lane];
                        sm = reinterpret_cast<const float2*>(s + 5 * ARR_FLOATS)[lane];
                    }
                    emit_pair<false>(a, O, orow + (size_t)(r - r0) * a.pitch, vA, vB, oe, ot, ow, od, em, sm, bad);
                    // the stored nodes only (an unstored column past the domain edge may hold
                    // anything after an open-water y-sweep that did not need it)
                    const float2 q2 = fma2(oe, oe, fma2(ot, ot, mul2(ow, ow)));
                    if (vB) chk_out = add2(chk_out, q2);
                    else if (vA) chk_out.x += q2.x;
                    smp.emit(a, O, b, r, c0, lane, oe, ot, ow);
                }
            }, OPEN ? open_end_y(a, k - 2) : 0);
    }

    // row k of a ring slot: x-sweep, then into the y-sweep pipeline
    template <int PH>
    __device__ __forceinline__ void row(int k, const float* s) {
        float2 E, U, V, D;
        XMet2 m;
        if (load_row(k, s, E, U, V, D, m) && !YF) xsweep2<FRIC, S1, OPEN>(E, U, V, D, m, K, lane, ends, bounded);
        push_row<PH>(k, s, E, U, V, D);
    }

    // The two rows of a ring slot on Cartesian grids (x first, eq. (solver2), reflecting
    // edges): when one vote finds every node of both rows wet, their x-sweeps run in one
    // basic block as two independent chains (the same operations as row by row).
    __device__ __forceinline__ void rows2(int k, const float* s) {
        float2 E0, U0, V0, D0, E1, U1, V1, D1;
        XMet2 m0r, m1r;
        const bool in0 = load_row(k, s, E0, U0, V0, D0, m0r);
        const bool in1 = load_row(k + 1, s + XWIN, E1, U1, V1, D1, m1r);
        const bool wet = wet_mark(E0.x, D0.x, K) && wet_mark(E0.y, D0.y, K) &&
                         wet_mark(E1.x, D1.x, K) && wet_mark(E1.y, D1.y, K);
        if (in0 && in1 && !bounded && __all_sync(FULL, wet)) {
            xsweep2_open<FRIC>(E0, U0, V0, D0, m0r, K);
            xsweep2_open<FRIC>(E1, U1, V1, D1, m1r, K);
        } else {
            if (in0) xsweep2<FRIC, S1, OPEN>(E0, U0, V0, D0, m0r, K, lane, ends, bounded);
            if (in1) xsweep2<FRIC, S1, OPEN>(E1, U1, V1, D1, m1r, K, lane, ends, bounded);
        }
        push_row<0>(k, s, E0, U0, V0, D0);
        push_row<1>(k + 1, s + XWIN, E1, U1, V1, D1);
    }

    // Process work item `idx` (strip, rows) of scenario b_ for the step described by O_.
    // Returns false when a wait expired (the warp's copies have landed when it returns).
    __device__ __forceinline__ bool run_item(int idx, int b_, const StepOut& O_) {
        O = O_;
        b = b_;
        const int4 item = __ldg(a.items + idx);          // (strip, first row, end row)
        c0 = item.x * XOUT;                          // window columns c0 .. c0 + 63 (fused_strips)
        cA = c0 + 2 * lane;
        r0 = item.y;
        r1 = item.z;
        k0 = r0 - 3;
        npairs = (r1 + 3 - k0 + 1) / 2;
        orow = (size_t)b * a.plane + (size_t)r0 * a.pitch + cA;
        nbox = O.emax ? 6u : 4u;
        tx = nbox * ARR_FLOATS * 4u + a.tx_pad;
        colA = cA >= 0 && cA < a.nx;
        ends = OPEN ? open_ends_x(a, cA) : 0u;
        colB = cA + 1 >= 0 && cA + 1 < a.nx;
        // the output columns: c0 + 4 .. c0 + 59, and from the domain's first column in the
        // first window, to its last column in the window that reaches it (past it the
        // window holds dry ghost columns, or its edge is the domain's)
        const bool own = (lane >= 2 || c0 == 0) && (lane < 30 || c0 + XWIN >= a.nx);
        vA = own && colA;
        vB = own && colB;
        edge = c0 + XWIN > a.nx;
        bounded = c0 == 0 || c0 + XWIN == a.nx;
        for (int j = 0; j < min(RING, npairs); ++j) issue(j);
        float2 il = v2(0.f), ir = v2(0.f), k2 = v2(0.f);
        if (colA) { il.x = __ldg(a.xa + cA); ir.x = __ldg(a.xb + cA); k2.x = __ldg(a.xk + cA); }
        if (colB) { il.y = __ldg(a.xa + cA + 1); ir.y = __ldg(a.xb + cA + 1); k2.y = __ldg(a.xk + cA + 1); }
        m0 = XMet2{il, ir, k2};
        smp.init(a, O, idx, lane);
        ym.init();
        int j = 0;
        for (; j < npairs; ++j) {
            const int slot = (int)((used + (unsigned)j) % RING);
            const bool ok = mbar_wait(&bar[slot], ((used + (unsigned)j) / RING) & 1u, a.wait_cycles);
            if (!__all_sync(FULL, ok)) break;
            const float* s = ring + slot * SLOT_FLOATS;
            const int k = k0 + SLOT_ROWS * j;
            if (!SPH && !YF && !S1 && !OPEN) {
                rows2(k, s);
            } else {
                row<0>(k, s);
                row<1>(k + 1, s + XWIN);
            }
            __syncwarp();
            if (j + RING < npairs) issue(j + RING);
        }
        if (j < npairs) {
            // a wait expired at pair j: pairs j .. j+RING-1 may still be in flight; let
            // each land (bounded) before going on
            for (int i = j; i < min(j + RING, npairs); ++i)
                mbar_wait(&bar[(used + (unsigned)i) % RING], ((used + (unsigned)i) / RING) & 1u, a.wait_cycles);
            bad |= 2;
            return false;
        }
        used += (unsigned)npairs;
        return true;
    }

    __device__ __forceinline__ void report() {
        bad |= !(chk_x.x + chk_x.y == 0.f) | !(chk_out.x + chk_out.y < RUNAWAY_SQ);
        if (bad) atomicOr(a.err, (bad & 2) ? (ERRF_TIMEOUT | ERRF_NONFINITE) : ERRF_NONFINITE);
    }
};

template <bool SPH, bool FRIC, bool YF, bool S1, bool OPEN>
__global__ void __launch_bounds__(FUSED_WARPS * 32, 4)
k_step_fused(const __grid_constant__ StepMaps M, const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * FUSED_WARPS + wib;
    const int b = blockIdx.y;
    if (gw >= a.nitems) return;
    if (a.limit && a.step > a.limit[b]) return;
    // a wait of an earlier launch expired: do not start new copies
    if (*reinterpret_cast<volatile int*>(a.err) & ERRF_TIMEOUT) return;
    FusedWarp<SPH, FRIC, YF, S1, OPEN> W(a);
    W.setup(smem_raw, wib);
    W.run_item(gw, b, step_out(&M, a));
    W.report();
}

// ------------------------------------------------------------------ batched, persistent
// Grid-wide barrier of a cooperative launch. Thread 0 of every block adds one arrival to the
// low half of *bar; the last arrival clears the count and advances the generation in the high
// half, which the others wait on for at most `limit` cycles before setting the timeout flag.
// Returns false when the run must stop (a wait expired here or anywhere else).
__device__ __forceinline__ bool grid_sync(unsigned long long* bar, unsigned nblocks, long long limit, int* err) {
    __shared__ int go;
    asm volatile("fence.proxy.async.global;" ::: "memory");    // outputs before the next TMA reads
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        const unsigned long long old = atomicAdd(bar, 1ull);
        const unsigned gen = (unsigned)(old >> 32);
        if ((unsigned)old == nblocks - 1) {
            // last arrival: count back to zero and generation + 1, in one atomic
            atomicAdd(bar, (1ull << 32) - (unsigned long long)nblocks);
        } else {
            volatile unsigned* vgen = reinterpret_cast<volatile unsigned*>(bar) + 1;
            const long long t0 = clock64();
            while (*vgen == gen) {
                if (clock64() - t0 > limit) { ok = 0; break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        if (!ok) atomicOr(err, ERRF_TIMEOUT);
        go = ok && !(*reinterpret_cast<volatile int*>(err) & ERRF_TIMEOUT);
    }
    __syncthreads();
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return go;
}

// Steps ctl[0]+1 .. ctl[1] of a batch of scenarios in one launch. Scenarios are taken in
// decreasing order of duration, so those still running at a step are the first nact[step]
// of `order`; the step's (scenario, item) pairs are numbered scenario-major and each warp
// takes the next number from a ticket counter until none are left, then the warps meet at
// the grid barrier before the next step reads what this one wrote. Two ticket counters
// (the halves of ctl[3]) alternate by step parity; block 0 clears the one the next step
// uses while the other is in use. A scenario that has stopped keeps its last state in the
// buffer of its last step's parity.
// With ALT (the alternating order) the odd-indexed steps (st - 1 odd) sweep y first: a second
// per-warp worker of the y-first kind shares the warp's ring, barriers and ring count.
template <bool SPH, bool FRIC, bool S1, bool OPEN, bool ALT>
__global__ void __launch_bounds__(FUSED_WARPS * 32, 4)
k_batch(const __grid_constant__ StepMaps2 MM, const StepArgs a, const BatchArgs B) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const long long step0 = B.ctl[0], step_end = B.ctl[1];
    unsigned* tickets = reinterpret_cast<unsigned*>(B.ctl + 3);
    if (*reinterpret_cast<volatile int*>(a.err) & ERRF_TIMEOUT) return;
    FusedWarp<SPH, FRIC, false, S1, OPEN> W(a);
    W.setup(smem_raw, wib);
    FusedWarp<SPH, FRIC, true, S1, OPEN> WY(a);
    if (ALT) {
        WY.lane = W.lane; WY.K = W.K; WY.ring = W.ring; WY.bar = W.bar; WY.used = W.used; WY.bad = 0;
        WY.chk_x = WY.chk_out = v2(0.f);
    }
    for (long long st = step0 + 1; st <= step_end; ++st) {
        const bool yf = ALT && (((st - 1) & 1) != 0);
        if (yf) WY.used = W.used;
        if (B.bnd) {
            // boundary input: the edge nodes of this step's input take the input at its model
            // time, then every block waits so that no TMA load reads an edge before it is set
            const BndRow& R = B.bnd_rows[st - step0 - 1];
            float* ei = (st & 1) ? B.eta[0] : B.eta[1];
            float* ui = (st & 1) ? B.u[0] : B.u[1];
            float* vi = (st & 1) ? B.v[0] : B.v[1];
            const int per = 2 * a.ny + 2 * a.nx;
            for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < per; idx += gridDim.x * blockDim.x) {
                const int e = idx < a.ny ? 0 : idx < 2 * a.ny ? 1 : idx < 2 * a.ny + a.nx ? 2 : 3;
                const int q = e == 0 ? idx : e == 1 ? idx - a.ny : e == 2 ? idx - 2 * a.ny : idx - 2 * a.ny - a.nx;
                bnd_apply(ei, ui, vi, a.pitch, a.nx, a.ny, e, q, B.bv, B.bnp, R.k[e], R.w[e]);
            }
            if (!grid_sync(reinterpret_cast<unsigned long long*>(B.ctl + 2), gridDim.x, a.wait_cycles, a.err)) break;
        }
        const bool odd = (st & 1) != 0;          // odd steps read buffer 0 and write buffer 1
        const bool mx = st % B.maxout == 0;
        StepOut O{odd ? &MM.m[0] : &MM.m[1], odd ? B.eta[1] : B.eta[0], odd ? B.u[1] : B.u[0],
                  odd ? B.v[1] : B.v[0], mx ? B.emax : nullptr, mx ? B.smax : nullptr,
                  (B.grec && st % B.gout == 0) ? B.grec + (st / B.gout) * B.grec_row : nullptr,
                  (B.nrec && st % B.bndout == 0) ? B.nrec + (st / B.bndout) * B.nrec_row : nullptr};
        const int na = B.nact ? (st < B.nact_len ? __ldg(B.nact + st) : 0) : B.nall;
        const unsigned total = (unsigned)na * (unsigned)a.nitems;
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(tickets + (odd ? 0 : 1), 0u);
        bool ok = true;
        while (ok) {
            unsigned t = 0;
            if (W.lane == 0) t = atomicAdd(tickets + (odd ? 1 : 0), 1u);
            t = __shfl_sync(FULL, t, 0);
            if (t >= total) break;
            const int item = (int)(t % (unsigned)a.nitems), scen = __ldg(B.order + t / (unsigned)a.nitems);
            ok = yf ? WY.run_item(item, scen, O) : W.run_item(item, scen, O);
        }
        if (yf) W.used = WY.used;
        if (!ok && W.lane == 0) atomicOr(a.err, ERRF_TIMEOUT);
        if (!grid_sync(reinterpret_cast<unsigned long long*>(B.ctl + 2), gridDim.x, a.wait_cycles, a.err)) break;
    }
    W.report();
    if (ALT) WY.report();
}

// x-sweep alone: one warp per (row, strip of 56 columns).
template <bool SPH, bool FRIC, bool S1, bool OPEN>
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
    const SweepConst K{a.hmin, a.dwall, a.half_dt, a.dt_gn2, a.transverse, a.inv_dt2_s1};
    float2 il = v2(0.f), ir = v2(0.f), k2 = v2(0.f);
    if (cA >= 0 && cA < a.nx) { il.x = a.xa[cA]; ir.x = a.xb[cA]; k2.x = a.xk[cA]; }
    if (cA + 1 >= 0 && cA + 1 < a.nx) { il.y = a.xa[cA + 1]; ir.y = a.xb[cA + 1]; k2.y = a.xk[cA + 1]; }
    XMet2 m{il, ir, k2};
    if (SPH) {
        const float2 f = v2(a.xrow[r]);
        m.inv_l = mul2(m.inv_l, f); m.inv_r = mul2(m.inv_r, f); m.k2 = mul2(m.k2, f);
    }
    float2 E, U, V, D;
    load_pair(a, boff, r, cA, E, U, V, D);
    xsweep2<FRIC, S1, OPEN>(E, U, V, D, m, K, lane, OPEN ? open_ends_x(a, cA) : 0u);
    const bool own = lane >= 2 && lane < 30;
    const bool va = own && cA < a.nx, vb = own && cA + 1 < a.nx;
    int bad = 0;
    const size_t o = boff + (size_t)r * a.pitch + cA;
    float2 em = make_float2(0.f, 0.f), sm = em;
    const StepOut O = step_out(nullptr, a);
    if (O.emax && va) {
        em.x = a.emax[o]; sm.x = a.smax[o];
        if (vb) { em.y = a.emax[o + 1]; sm.y = a.smax[o + 1]; }
    }
    emit_pair(a, O, o, va, vb, E, U, V, D, em, sm, bad);
    Samples smp;
    smp.init(a, O, gw, lane);
    smp.emit(a, O, b, r, c0, lane, E, U, V);
    if (bad) atomicOr(a.err, ERRF_NONFINITE);
}

// y-sweep alone: one warp per (strip of 64 columns, S rows).
template <bool SPH, bool FRIC, bool S1, bool OPEN>
struct YOnly {
    const StepArgs& a;
    SweepConst K;
    int lane, b, c0, cA, r0, r1;
    size_t boff;
    bool vA, vB, withmax;
    YMarch2 ym;
    Samples smp;
    StepOut O;
    int bad;
    __device__ __forceinline__ YOnly(const StepArgs& a_) : a(a_) {}
    template <int PH>
    __device__ __forceinline__ void row(int k) {
        float2 E, U, V, D;
        load_pair(a, boff, k, cA, E, U, V, D);
        const float4 m2 = __ldg(a.ymet + k - 2);
        const bool oA = wet_mark(E.x, D.x, K), oB = wet_mark(E.y, D.y, K);
        const int r = k - 3;
        ym.template push<PH, SPH, FRIC, S1, OPEN>(E, V, U, D, oA, oB, m2, K, vA, vB,
            [&](float2 oe, float2 ow, float2 ot, float2 od) {
                if (r >= r0 && r < r1) {
                    const size_t o = boff + (size_t)r * a.pitch + cA;
                    float2 em = make_float2(0.f, 0.f), sm = em;
                    if (O.emax && vA) {
                        em.x = a.emax[o]; sm.x = a.smax[o];
                        if (vB) { em.y = a.emax[o + 1]; sm.y = a.smax[o + 1]; }
                    }
                    emit_pair(a, O, o, vA, vB, oe, ot, ow, od, em, sm, bad);
                    smp.emit(a, O, b, r, c0, lane, oe, ot, ow);
                }
            }, OPEN ? open_end_y(a, k - 2) : 0);
    }
};

template <bool SPH, bool FRIC, bool S1, bool OPEN>
__global__ void __launch_bounds__(128) k_ysweep(const StepArgs a) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int b = blockIdx.y;
    if (gw >= a.nstrips * a.nseg) return;
    if (a.limit && a.step > a.limit[b]) return;
    YOnly<SPH, FRIC, S1, OPEN> Y(a);
    Y.K = SweepConst{a.hmin, a.dwall, a.half_dt, a.dt_gn2, a.transverse, a.inv_dt2_s1};
    const int strip = gw % a.nstrips, seg = gw / a.nstrips;
    Y.lane = lane;
    Y.b = b;
    Y.c0 = strip * XWIN;
    Y.cA = Y.c0 + 2 * lane;
    Y.r0 = seg * a.S;
    Y.r1 = min(Y.r0 + a.S, a.ny);
    Y.boff = (size_t)b * a.plane;
    Y.vA = Y.cA < a.nx;
    Y.vB = Y.cA + 1 < a.nx;
    Y.withmax = a.emax != nullptr;
    Y.bad = 0;
    Y.O = step_out(nullptr, a);
    Y.smp.init(a, Y.O, gw, lane);
    Y.ym.init();
    int k = Y.r0 - 3;
    for (; k + 1 < Y.r1 + 3; k += 2) {
        Y.template row<0>(k);
        Y.template row<1>(k + 1);
    }
    if (k < Y.r1 + 3) Y.template row<0>(k);
    if (Y.bad) atomicOr(a.err, ERRF_NONFINITE);
}

}  // namespace cliffs
