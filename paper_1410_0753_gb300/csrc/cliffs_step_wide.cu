// The wide fused step (arXiv 1410.0753, section "Numerics"): one launch per step, x-sweep
// then y-sweep, for grids with reflecting outer edges and eq. (solver2), steps taken x first.
//
//  k_step_wide   a warp owns a strip of 120 output columns and S output rows; it holds a
//                128-column window, four nodes per lane (xsweep4), and walks rows r0-3 ..
//                r1+2. Rows (eta, u, v, d and, when max-wave is due, the max-wave rows
//                three rows behind) arrive in shared memory by TMA (128 x 2 boxes) through a
//                ring of 4 slots per warp, one mbarrier per slot, every wait bounded. Each row is
//                x-swept across the warp and pushed into two per-lane y-sweep pipelines (one
//                per pair of columns) that finish the y-sweep three rows behind; one vote per
//                row picks the open-water path for both. The finished row is stored as
//                128-bit vectors, with the max-wave update and the gauge / enclosed-grid
//                samples of that row.
// It computes the same bits as k_step_fused (the same per-node operations); it halves the
// per-node shuffles, votes, loads, stores and address arithmetic, narrows the column halo
// from 64/56 to 128/120, and gives each warp two independent chains of arithmetic.
#include "step_kernels.cuh"
#include "sweep_wide.cuh"

namespace cliffs {

#ifndef WIDE_MINB
#define WIDE_MINB 2                               // resident blocks per SM (registers: 65536 / (128 * 2))
#endif
constexpr int WRING = WIDE_MINB >= 3 ? 3 : 4;     // slots in flight per warp
constexpr int W_ARR = SLOT_ROWS * WWIN;           // floats of one array in a slot
constexpr int W_SLOT = NARR * W_ARR;
constexpr int W_WARP_BYTES = WRING * W_SLOT * 4;
constexpr int WIDE_WARPS = 4;
constexpr int WIDE_SMEM = WIDE_WARPS * (W_WARP_BYTES + WRING * 8);
static_assert((WIDE_SMEM + 1024) * WIDE_MINB <= 228 * 1024, "shared memory for WIDE_MINB blocks per SM");

// Gauge / enclosed-grid samples of the wide warp (the records of Samples, four nodes a lane).
struct Samples4 : Samples {
    __device__ __forceinline__ void emit4(const StepArgs& a, const StepOut& O, int b, int r, int c0, int lane,
                                          float2 Ea, float2 Eb, float2 Ua, float2 Ub, float2 Va, float2 Vb) {
        if (r != next) return;
        while (true) {
            const bool mineRow = lane >= sp - base && mine.x == r;
            const int rel = mine.y - c0;
            const int src = mineRow ? (rel >> 2) & 31 : lane;
            const int q = rel & 3;
            const float e0 = __shfl_sync(FULL, Ea.x, src), e1 = __shfl_sync(FULL, Ea.y, src);
            const float e2 = __shfl_sync(FULL, Eb.x, src), e3 = __shfl_sync(FULL, Eb.y, src);
            const float u0 = __shfl_sync(FULL, Ua.x, src), u1 = __shfl_sync(FULL, Ua.y, src);
            const float u2 = __shfl_sync(FULL, Ub.x, src), u3 = __shfl_sync(FULL, Ub.y, src);
            const float v0 = __shfl_sync(FULL, Va.x, src), v1 = __shfl_sync(FULL, Va.y, src);
            const float v2_ = __shfl_sync(FULL, Vb.x, src), v3 = __shfl_sync(FULL, Vb.y, src);
            if (mineRow) {
                float* out = (mine.z == 0) ? (O.rec_g ? O.rec_g + (long long)b * a.rec_g_bstride : nullptr)
                                           : O.rec_n;
                if (out) {
                    out[3 * mine.w + 0] = q == 0 ? e0 : q == 1 ? e1 : q == 2 ? e2 : e3;
                    out[3 * mine.w + 1] = q == 0 ? u0 : q == 1 ? u1 : q == 2 ? u2 : u3;
                    out[3 * mine.w + 2] = q == 0 ? v0 : q == 1 ? v1 : q == 2 ? v2_ : v3;
                }
            }
            sp += __popc(__ballot_sync(FULL, mineRow));
            if (sp >= se) { next = 0x7fffffff; return; }
            if (sp - base < 32) {
                next = __shfl_sync(FULL, mine.x, sp - base);
                return;
            }
            load(a, lane);
            next = __shfl_sync(FULL, mine.x, 0);
            if (next != r) return;
        }
    }
};

// max-wave of a pair of nodes (section "Running Options", field maxout), as in emit_pair:
// on wet nodes eta_max and speed_max take the new values where these are larger
__device__ __forceinline__ void maxwave_pair(const StepArgs& a, const StepOut& O, size_t o, bool va, bool vb,
                                             float2 E, float2 U, float2 V, float2 D, float2 em, float2 sm) {
    if (!va) return;
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

template <bool SPH, bool FRIC>
struct WideWarp {
    const StepArgs& a;
    SweepConst K;
    float* ring;
    uint64_t* bar;
    unsigned used;             // ring pairs consumed so far
    int lane, b, c0, cA, r0, r1, k0, npairs;
    size_t orow;
    unsigned col, val;         // bit q: column cA + q inside the domain / stored by this lane
    bool edge;
    unsigned tx, nbox;
    XMet2 ma, mb;
    YPair ya, yb;
    Samples4 smp;
    StepOut O;
    int bad;

    __device__ __forceinline__ WideWarp(const StepArgs& a_) : a(a_) {}

    __device__ __forceinline__ void setup(unsigned char* smem_raw, int wib) {
        lane = threadIdx.x & 31;
        K = SweepConst{a.hmin, a.dwall, a.half_dt, a.dt_gn2, a.transverse, 0.f};
        ring = reinterpret_cast<float*>(smem_raw + wib * W_WARP_BYTES);
        bar = reinterpret_cast<uint64_t*>(smem_raw + WIDE_WARPS * W_WARP_BYTES) + wib * WRING;
        used = 0;
        bad = 0;
        if (lane == 0) {
            for (int s = 0; s < WRING; ++s) mbar_init(&bar[s], 1);
            fence_mbar_init();
        }
        __syncwarp();
    }

    // lanes 0..nbox-1 each start one 128 x 2 box of the item's row pair j into its ring slot
    __device__ __forceinline__ void issue(int j) {
        const int slot = (int)((used + (unsigned)j) % WRING);
        const int row = k0 + SLOT_ROWS * j;
        if (lane == 0) mbar_arrive_tx(&bar[slot], tx);
        if (lane < (int)nbox) {
            fence_proxy_async();
            tma_row3(ring + slot * W_SLOT + lane * W_ARR, &O.M->e + lane, &bar[slot], c0,
                     lane >= 4 ? row - 3 : row, lane == 3 ? 0 : b);
        }
    }

    __device__ __forceinline__ void load4(const float* s, int arr, float2& A, float2& B) const {
        const float4 v = reinterpret_cast<const float4*>(s + arr * W_ARR)[lane];
        A = make_float2(v.x, v.y);
        B = make_float2(v.z, v.w);
    }

    template <int PH>
    __device__ __forceinline__ void row(int k, const float* s) {
        float2 Ea, Eb, Ua, Ub, Va, Vb, Da, Db;
        load4(s, 0, Ea, Eb);
        load4(s, 1, Ua, Ub);
        load4(s, 2, Va, Vb);
        load4(s, 3, Da, Db);
        const bool rowin = k >= 0 && k < a.ny;
        if (edge || !rowin) {
            const unsigned in = rowin ? col : 0u;
            if (!(in & 1u)) { Ea.x = Ua.x = Va.x = 0.f; Da.x = OUTSIDE_D; }
            if (!(in & 2u)) { Ea.y = Ua.y = Va.y = 0.f; Da.y = OUTSIDE_D; }
            if (!(in & 4u)) { Eb.x = Ub.x = Vb.x = 0.f; Db.x = OUTSIDE_D; }
            if (!(in & 8u)) { Eb.y = Ub.y = Vb.y = 0.f; Db.y = OUTSIDE_D; }
        }
        if (rowin) {
            XMet2 xa = ma, xb = mb;
            if (SPH) {
                const float2 f = v2(__ldg(a.xrow + k));
                xa.inv_l = mul2(xa.inv_l, f); xa.inv_r = mul2(xa.inv_r, f); xa.k2 = mul2(xa.k2, f);
                xb.inv_l = mul2(xb.inv_l, f); xb.inv_r = mul2(xb.inv_r, f); xb.k2 = mul2(xb.k2, f);
            }
            xsweep4<FRIC>(Ea, Ua, Va, Da, xa, Eb, Ub, Vb, Db, xb, K, lane);
        }
        // into the y-sweep pipelines: eta, w = v, t = u
        const float4 m2 = __ldg(a.ymet + k - 2);
        const bool o0 = wet_mark(Ea.x, Da.x, K), o1 = wet_mark(Ea.y, Da.y, K);
        const bool o2 = wet_mark(Eb.x, Db.x, K), o3 = wet_mark(Eb.y, Db.y, K);
        // a non-finite x-sweep result reads as a dry node in the y-sweep: flag it here
        if ((val & 1u) && !o0) bad |= !(fabsf(Ea.x) < 1e5f);
        if ((val & 2u) && !o1) bad |= !(fabsf(Ea.y) < 1e5f);
        if ((val & 4u) && !o2) bad |= !(fabsf(Eb.x) < 1e5f);
        if ((val & 8u) && !o3) bad |= !(fabsf(Eb.y) < 1e5f);
        float2 ea, wa, ta, da, eb, wb, tb, db;
        const bool fast = __all_sync(FULL, ya.template fast_ok<PH>(val & 1u, val & 2u) &&
                                           yb.template fast_ok<PH>(val & 4u, val & 8u));
        if (fast) {
            ya.template fast<PH, SPH, FRIC>(Ea, Va, Ua, Da, o0, o1, m2, K, ea, wa, ta, da);
            yb.template fast<PH, SPH, FRIC>(Eb, Vb, Ub, Db, o2, o3, m2, K, eb, wb, tb, db);
        } else {
            ya.template slow<PH, SPH, FRIC>(Ea, Va, Ua, Da, o0, o1, m2, K, ea, wa, ta, da);
            yb.template slow<PH, SPH, FRIC>(Eb, Vb, Ub, Db, o2, o3, m2, K, eb, wb, tb, db);
        }
        const int r = k - 3;
        if (r >= r0 && r < r1 && val) {
            // the finished row r: eta, u (= t), v (= w)
            const size_t o = orow + (size_t)(r - r0) * a.pitch;
            if (val == 15u) {
                *reinterpret_cast<float4*>(O.eta_out + o) = make_float4(ea.x, ea.y, eb.x, eb.y);
                *reinterpret_cast<float4*>(O.u_out + o) = make_float4(ta.x, ta.y, tb.x, tb.y);
                *reinterpret_cast<float4*>(O.v_out + o) = make_float4(wa.x, wa.y, wb.x, wb.y);
            } else {
                const float e4[4] = {ea.x, ea.y, eb.x, eb.y}, u4[4] = {ta.x, ta.y, tb.x, tb.y};
                const float v4[4] = {wa.x, wa.y, wb.x, wb.y};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (val & (1u << q)) { O.eta_out[o + q] = e4[q]; O.u_out[o + q] = u4[q]; O.v_out[o + q] = v4[q]; }
            }
            bad |= runaway(ea.x, ta.x, wa.x) | ((val & 2u) ? runaway(ea.y, ta.y, wa.y) : 0) |
                   ((val & 4u) ? runaway(eb.x, tb.x, wb.x) : 0) | ((val & 8u) ? runaway(eb.y, tb.y, wb.y) : 0);
            if (O.emax) {
                float2 ema, emb, sma, smb;
                load4(s, 4, ema, emb);
                load4(s, 5, sma, smb);
                maxwave_pair(a, O, o, val & 1u, val & 2u, ea, ta, wa, da, ema, sma);
                maxwave_pair(a, O, o + 2, val & 4u, val & 8u, eb, tb, wb, db, emb, smb);
            }
        }
        if (r >= r0 && r < r1) smp.emit4(a, O, b, r, c0, lane, ea, eb, ta, tb, wa, wb);
    }

    // Process work item idx (strip, rows) of scenario b_. Returns false when a wait expired
    // (the warp's copies have landed when it returns).
    __device__ __forceinline__ bool run_item(int idx, int b_, const StepOut& O_) {
        O = O_;
        b = b_;
        const int4 item = __ldg(a.items + idx);          // (strip, first row, end row)
        c0 = item.x * WOUT - 4;
        cA = c0 + 4 * lane;
        r0 = item.y;
        r1 = item.z;
        k0 = r0 - 3;
        npairs = (r1 + 3 - k0 + 1) / 2;
        orow = (size_t)b * a.plane + (size_t)r0 * a.pitch + cA;
        nbox = O.emax ? 6u : 4u;
        tx = nbox * W_ARR * 4u + a.tx_pad;
        col = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (cA + q >= 0 && cA + q < a.nx) col |= 1u << q;
        val = (lane >= 1 && lane < 31) ? col : 0u;
        edge = c0 < 0 || c0 + WWIN > a.nx;
        for (int j = 0; j < min(WRING, npairs); ++j) issue(j);
        float il[4], ir[4], k2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            il[q] = ir[q] = k2[q] = 0.f;
            if (col & (1u << q)) { il[q] = __ldg(a.xa + cA + q); ir[q] = __ldg(a.xb + cA + q); k2[q] = __ldg(a.xk + cA + q); }
        }
        ma = XMet2{make_float2(il[0], il[1]), make_float2(ir[0], ir[1]), make_float2(k2[0], k2[1])};
        mb = XMet2{make_float2(il[2], il[3]), make_float2(ir[2], ir[3]), make_float2(k2[2], k2[3])};
        smp.init(a, O, idx, lane);
        ya.init();
        yb.init();
        int j = 0;
        for (; j < npairs; ++j) {
            const int slot = (int)((used + (unsigned)j) % WRING);
            const bool ok = mbar_wait(&bar[slot], ((used + (unsigned)j) / WRING) & 1u, a.wait_cycles);
            if (!__all_sync(FULL, ok)) break;
            const float* s = ring + slot * W_SLOT;
            const int k = k0 + SLOT_ROWS * j;
            row<0>(k, s);
            row<1>(k + 1, s + WWIN);
            __syncwarp();
            if (j + WRING < npairs) issue(j + WRING);
        }
        if (j < npairs) {
            for (int i = j; i < min(j + WRING, npairs); ++i)
                mbar_wait(&bar[(used + (unsigned)i) % WRING], ((used + (unsigned)i) / WRING) & 1u, a.wait_cycles);
            bad |= 2;
            return false;
        }
        used += (unsigned)npairs;
        return true;
    }

    __device__ __forceinline__ void report() {
        if (bad) atomicOr(a.err, (bad & 2) ? (ERRF_TIMEOUT | ERRF_NONFINITE) : ERRF_NONFINITE);
    }
};

template <bool SPH, bool FRIC>
__global__ void __launch_bounds__(WIDE_WARPS * 32, WIDE_MINB)
k_step_wide(const __grid_constant__ StepMaps M, const StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * WIDE_WARPS + wib;
    const int b = blockIdx.y;
    if (gw >= a.nitems) return;
    if (a.limit && a.step > a.limit[b]) return;
    if (*reinterpret_cast<volatile int*>(a.err) & ERRF_TIMEOUT) return;
    WideWarp<SPH, FRIC> W(a);
    W.setup(smem_raw, wib);
    W.run_item(gw, b, step_out(&M, a));
    W.report();
}

// The batched persistent run (S7) with the wide warps: steps ctl[0]+1 .. ctl[1] of a batch of
// scenarios in one cooperative launch, as k_batch (work items handed out by a ticket counter
// per step, scenarios still running first, a grid barrier between steps, boundary input
// imposed by the blocks before each step), for steps swept x first.
template <bool SPH, bool FRIC>
__global__ void __launch_bounds__(WIDE_WARPS * 32, WIDE_MINB)
k_batch_wide(const __grid_constant__ StepMaps2 MM, const StepArgs a, const BatchArgs B) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int wib = threadIdx.x >> 5;
    const long long step0 = B.ctl[0], step_end = B.ctl[1];
    unsigned* tickets = reinterpret_cast<unsigned*>(B.ctl + 3);
    if (*reinterpret_cast<volatile int*>(a.err) & ERRF_TIMEOUT) return;
    WideWarp<SPH, FRIC> W(a);
    W.setup(smem_raw, wib);
    for (long long st = step0 + 1; st <= step_end; ++st) {
        if (B.bnd) {
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
            ok = W.run_item(item, scen, O);
        }
        if (!ok && W.lane == 0) atomicOr(a.err, ERRF_TIMEOUT);
        if (!grid_sync(reinterpret_cast<unsigned long long*>(B.ctl + 2), gridDim.x, a.wait_cycles, a.err)) break;
    }
    W.report();
}

static const void* batch_wide_kernel(bool sph, bool fric) {
    static const void* const t[4] = {(const void*)k_batch_wide<false, false>, (const void*)k_batch_wide<true, false>,
                                     (const void*)k_batch_wide<false, true>, (const void*)k_batch_wide<true, true>};
    return t[(sph ? 1 : 0) + (fric ? 2 : 0)];
}

static const void* wide_kernel(bool sph, bool fric) {
    static const void* const t[4] = {(const void*)k_step_wide<false, false>, (const void*)k_step_wide<true, false>,
                                     (const void*)k_step_wide<false, true>, (const void*)k_step_wide<true, true>};
    return t[(sph ? 1 : 0) + (fric ? 2 : 0)];
}

static cudaError_t wide_smem_optin() {
    static cudaError_t done = cudaErrorNotReady;
    if (done == cudaErrorNotReady) {
        done = cudaSuccess;
        for (int v = 0; v < 4 && done == cudaSuccess; ++v)
            done = cudaFuncSetAttribute(wide_kernel(v & 1, v & 2), cudaFuncAttributeMaxDynamicSharedMemorySize, WIDE_SMEM);
        for (int v = 0; v < 4 && done == cudaSuccess; ++v)
            done = cudaFuncSetAttribute(batch_wide_kernel(v & 1, v & 2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        WIDE_SMEM);
    }
    return done;
}

cudaError_t launch_batch_wide(const StepArgs& a, const StepMaps2& mm, const BatchArgs& b, int blocks, cudaStream_t s) {
    const cudaError_t e = wide_smem_optin();
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(WIDE_WARPS * 32);
    cfg.dynamicSmemBytes = WIDE_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;         // all blocks resident: the grid barrier
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    StepMaps2 m2 = mm;
    StepArgs aa = a;
    BatchArgs bb = b;
    void* args[] = {&m2, &aa, &bb};
    return cudaLaunchKernelExC(&cfg, batch_wide_kernel(a.sph, a.dt_gn2 > 0.f), args);
}

int batch_wide_blocks_per_sm(bool sph) {
    if (wide_smem_optin() != cudaSuccess) return 1;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_wide_kernel(sph, true), WIDE_WARPS * 32, WIDE_SMEM);
    return nb;
}

cudaError_t launch_step_wide(const StepArgs& a, const StepMaps& m, int batch, cudaStream_t s) {
    const cudaError_t e = wide_smem_optin();
    if (e != cudaSuccess) return e;
    const dim3 grid((a.nitems + WIDE_WARPS - 1) / WIDE_WARPS, batch);
    StepMaps mm = m;
    StepArgs aa = a;
    void* args[] = {&mm, &aa};
    return cudaLaunchKernel(wide_kernel(a.sph, a.dt_gn2 > 0.f), grid, dim3(WIDE_WARPS * 32), args, WIDE_SMEM, s);
}

int wide_blocks_per_sm(bool sph) {
    if (wide_smem_optin() != cudaSuccess) return 1;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, wide_kernel(sph, true), WIDE_WARPS * 32, WIDE_SMEM);
    return nb;
}

int wide_warps_per_block() { return WIDE_WARPS; }

}  // namespace cliffs
