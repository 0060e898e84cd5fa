// FP64 CPU oracle for the Cliffs shallow-water step (Tolkova, "Cliffs User Manual",
// arXiv 1410.0753). TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU
// baseline of the benchmark call it; the product path never does. It shares no code,
// header or table with the CUDA library.
//
// What it computes, in the paper's notation (section "Numerics"):
//   * dimensional splitting, eqs. (eq2A)/(eq2B): an x-sweep over every row, then a
//     y-sweep over every column, each a 1D problem on one line;
//   * Riemann invariants p = u + 2 sqrt(gh), q = u - 2 sqrt(gh) with eigenvalues
//     lambda = u +- sqrt(gh) and the characteristic equations (pq1), (pq2); the
//     transverse velocity is advected by (pq3);
//   * the well-balanced combination Q(k,j) of eq. (eqQ) and the update (solver2)
//     (optionally the original (solver1));
//   * the recovery u = (p+q)/2, h = (p-q)^2/16g of eqs. (stateu), (stateh);
//   * the inundation algorithm, steps (a)-(e) of section "Inundation algorithm";
//   * the depth-jump filter of section "Numerical stability", eqs. (dstab), (newdw),
//     (newdc);
//   * the outputs of section "Running Options": max-wave (field maxout), gauges
//     (gout), and boundary series for enclosed grids (bndout);
//   * boundary input on the domain edges and open (radiating) outer edges, both readings
//     where the paper gives no condition (stated where they are computed).
// Where the paper is silent, the readings are listed at the top of each function.
//
// Two algebraic forms of the same update are provided: form 0 is the literal one
// (Riemann invariants, eq. (eqQ) as printed); form 1 rewrites the same arithmetic in
// perturbation variables (eta, c_k - c_j = g(h_k - h_j)/(c_k + c_j), increments). The
// tests require the two to agree in FP64; form 0 is the oracle proper.
//
// The sweep is a template over the scalar type: instantiated with `double` it is the
// oracle; with `Dual` (value + tangent) it is the tangent-linear model, with every
// branch (wet/dry marks, flooding choice, cushion limiter, friction clamp) decided on
// the value, which is the derivative the adjoint of the step must reproduce.

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double GRAV = 9.81;
const double R_SPHERE = 6371000.0;
const double DEG = 3.14159265358979323846 / 180.0;

// ------------------------------------------------------------------ dual numbers
struct Dual {
    double v, d;
    Dual() : v(0), d(0) {}
    Dual(double a) : v(a), d(0) {}
    Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
    return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v));
}
inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
inline Dual sqrt(Dual a) {
    double s = std::sqrt(a.v);
    return Dual(s, s > 0 ? a.d / (2.0 * s) : 0.0);
}
inline Dual pow43(Dual a) {                       // a^(4/3)
    double c = std::cbrt(a.v);
    return Dual(a.v * c, (4.0 / 3.0) * c * a.d);
}
inline double pow43(double a) { return a * std::cbrt(a); }
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
using std::sqrt;

// ------------------------------------------------------------------ parameters
struct Params {
    int nx, ny, coords;        // coords: 1 Cartesian, otherwise geographic spherical
    double h_min;              // 'ground': minimal flow depth
    double manning_n2;         // 'crough' read as Manning n^2
    int itopo;                 // 0: vertical wall at depth dwall; otherwise inundation
    double dwall;
    double dt;
    int transverse;            // 1: advect the transverse velocity by eq. (pq3)
    int solver;                // 2: eq. (solver2) (current Cliffs); 1: eq. (solver1)
    int form;                  // 0: literal Riemann-invariant form; 1: perturbation form
    int alternate;             // 1: y-sweep first on odd steps (alternating splitting)
    int open_edges;            // open outer edges, bits W 1, E 2, S 4, N 8 (others walls)
};

// Per-node state as seen by the solver: a real wet node or a mirror ghost.
template <typename T> struct Node { T eta, w, t; double d; };

// Phase record of a single line, for tests of steps (a)-(e).
struct PhaseRec {
    int*    wet0;      // (a) mark, start of the sweep
    int*    wet1;      // after (b)
    int*    src;       // (b) index of the wet cell a newly wetted cell was filled from, or -1
    double* eta_b;     // state after (b)
    double* w_b;
    double* t_b;
    double* eta_d;     // state after (d)
    double* w_d;
    double* t_d;
};

template <typename T> struct Scratch {
    std::vector<int> floodable, wet0, wet1, src;
    std::vector<T> e1, w1, t1, e2, w2, t2;
    void resize(int n) {
        floodable.resize(n); wet0.resize(n); wet1.resize(n); src.resize(n);
        e1.resize(n); w1.resize(n); t1.resize(n); e2.resize(n); w2.resize(n); t2.resize(n);
    }
};

// eq. (eqQ) for the Riemann invariant r with eigenvalue lam, between node a on the right
// and node b on the left, ds = x_a - x_b > 0:
//   Q(a,b) = 1/2 (lam_a + lam_b) (r_a - r_b)/(x_a - x_b) - g (d_a - d_b)/(x_a - x_b)
template <typename T>
inline T Q_literal(T lam_a, T lam_b, T r_a, T r_b, double d_a, double d_b, double ds) {
    return 0.5 * (lam_a + lam_b) * (r_a - r_b) / ds - GRAV * (d_a - d_b) / ds;
}

// The same combination in perturbation variables. With c^2 = g h, h = eta + d:
//   1/2 (lam_a+lam_b)(r_a-r_b) - g(d_a-d_b)
//     = 1/2 (lam_a+lam_b)(w_a-w_b) + s (w_a+w_b)(c_a-c_b) + g (eta_a-eta_b),
// s = +1 for p (lam = w + c), s = -1 for q (lam = w - c), and
//   c_a - c_b = g ((eta_a-eta_b) + (d_a-d_b)) / (c_a + c_b).
template <typename T>
inline T Q_perturb(T lam_a, T lam_b, T w_a, T w_b, T dc, T deta, double s, double ds) {
    return (0.5 * (lam_a + lam_b) * (w_a - w_b) + s * (w_a + w_b) * dc + GRAV * deta) / ds;
}

// eq. (pq3)'s stencil: Q for the transverse velocity t advected with speed w, no depth term.
template <typename T>
inline T Qt(T w_a, T w_b, T t_a, T t_b, double ds) {
    return 0.5 * (w_a + w_b) * (t_a - t_b) / ds;
}

// Open outer edge (the paper gives no condition for one): the ghost beyond a wet edge node
// carries the node's outgoing Riemann invariant and the incoming invariant of still water at
// the node's depth, c0 = sqrt(g max(d, 0)); its depth and transverse velocity are the node's.
// At the right end (east, north) p leaves and q enters: p_g = w + 2c, q_g = -2 c0; at the
// left end q leaves and p enters: q_g = w - 2c, p_g = 2 c0. A ghost whose c would be
// negative (an inflow past the critical speed) is taken dry, c_g = 0.
template <typename T>
Node<T> open_ghost(const Node<T>& C, bool right, double g) {
    const T c = sqrt(g * (C.eta + C.d));
    const double c0 = std::sqrt(g * std::max(C.d, 0.0));
    const T p = right ? C.w + 2.0 * c : T(2.0 * c0);
    const T q = right ? T(-2.0 * c0) : C.w - 2.0 * c;
    T cg = 0.25 * (p - q);
    if (val(cg) < 0.0) cg = T(0.0);
    return Node<T>{cg * cg / g - C.d, 0.5 * (p + q), C.t, C.d};
}

// One sweep of one line (a row in the x-sweep, a column in the y-sweep).
//   n     nodes on the line (n >= 3)
//   ds    n-1 intervals between consecutive nodes, in metres
//   d     depth, positive down
//   src   spherical continuity factor tan(phi)/R per node, or null (see reading 7)
//   eta, w, t  free surface, along-line velocity, transverse velocity (in/out)
//   open  bit 0: the end at j = 0 is an open edge, bit 1: the end at j = n-1 (else walls)
// Readings of the paper where it is silent (binding on both the oracle and the GPU):
//  1. (a) dry means h = eta + d < h_min (the algorithm text; "at and below" in the
//     parameter list conflicts). A dry cell carries no velocity; its eta is left as is.
//     With itopo = 0, cells with d < dwall are permanent walls: never wet, never flooded.
//  2. (b) of two qualifying wet neighbours the one with the larger eta wins, the left
//     one on a tie; wetness is taken from the start of the sweep, so one ring per sweep.
//  3. (c) a dry neighbour, or a node beyond the domain edge, is a mirror ghost of the wet
//     node: eta_g = eta_j, d_g = d_j, w_g = -w_j, t_g = t_j, across the real interval
//     (the edge interval at the domain edge): the wall sits half a node from the wet node.
//  4. friction alpha = g n^2 w sqrt(w^2 + t^2) / h^(4/3) at time level n, subtracted from
//     p and q alike, with |alpha dt| <= |w| (friction never reverses the flow).
//  5. (e) "exceed" compares magnitudes; the neighbour's state is the one after (d).
//  7. spherical: ds = R cos(phi) dlambda along a row, R dphi along a column; the y-sweep
//     adds the continuity term h_t += h v tan(phi)/R, i.e. p += dt c v tan(phi)/R and
//     q -= dt c v tan(phi)/R; no Coriolis and no metric momentum terms.
template <typename T>
void sweep_line(const Params& P, int n, const double* ds, const double* d, const double* src,
                T* eta, T* w, T* t, Scratch<T>& S, PhaseRec* rec, int open = 0)
{
    const double g = GRAV, hmin = P.h_min, dt = P.dt;
    S.resize(n);
    // (a) mark dry cells
    for (int j = 0; j < n; ++j) {
        S.floodable[j] = (P.itopo != 0) || (d[j] >= P.dwall);
        S.wet0[j] = S.floodable[j] && (val(eta[j]) + d[j] >= hmin);
    }
    // (b) add a dry cell to a wet neighbour's segment when h_j - d_j + d_i > h_min,
    //     with height h_min and the neighbour's velocities
    for (int i = 0; i < n; ++i) {
        S.e1[i] = eta[i]; S.w1[i] = w[i]; S.t1[i] = t[i];
        S.src[i] = -1; S.wet1[i] = S.wet0[i];
        if (S.wet0[i]) continue;
        S.w1[i] = T(0.0); S.t1[i] = T(0.0);
        if (!S.floodable[i]) continue;
        int best = -1;
        for (int k = 0; k < 2; ++k) {
            int j = (k == 0) ? i - 1 : i + 1;
            if (j < 0 || j >= n || !S.wet0[j]) continue;
            if (!(val(eta[j]) + d[i] > hmin)) continue;
            if (best < 0 || val(eta[j]) > val(eta[best])) best = j;
        }
        if (best >= 0) {
            S.e1[i] = T(hmin - d[i]);
            S.w1[i] = w[best];
            S.t1[i] = t[best];
            S.src[i] = best;
            S.wet1[i] = 1;
        }
    }
    // (c)+(d) solver at every wet node; interfaces with dry nodes are reflecting walls
    for (int j = 0; j < n; ++j) {
        if (!S.wet1[j]) { S.e2[j] = S.e1[j]; S.w2[j] = S.w1[j]; S.t2[j] = S.t1[j]; continue; }
        const double dsL = (j > 0) ? ds[j - 1] : ds[0];
        const double dsR = (j < n - 1) ? ds[j] : ds[n - 2];
        Node<T> C{S.e1[j], S.w1[j], S.t1[j], d[j]};
        Node<T> Gh{S.e1[j], -S.w1[j], S.t1[j], d[j]};
        Node<T> L = (j > 0 && S.wet1[j - 1]) ? Node<T>{S.e1[j - 1], S.w1[j - 1], S.t1[j - 1], d[j - 1]} : Gh;
        Node<T> R = (j < n - 1 && S.wet1[j + 1]) ? Node<T>{S.e1[j + 1], S.w1[j + 1], S.t1[j + 1], d[j + 1]} : Gh;
        if (j == 0 && (open & 1)) L = open_ghost(C, false, g);
        if (j == n - 1 && (open & 2)) R = open_ghost(C, true, g);

        T hC = C.eta + C.d, hL = L.eta + L.d, hR = R.eta + R.d;
        T cC = sqrt(g * hC), cL = sqrt(g * hL), cR = sqrt(g * hR);
        T lpC = C.w + cC, lpL = L.w + cL, lpR = R.w + cR;      // lambda_p = u + sqrt(gh)
        T lqC = C.w - cC, lqL = L.w - cL, lqR = R.w - cR;      // lambda_q = u - sqrt(gh)

        // friction (reading 4)
        T adt = T(0.0);
        if (P.manning_n2 > 0.0) {
            T alpha = g * P.manning_n2 * C.w * sqrt(C.w * C.w + C.t * C.t) / pow43(hC);
            adt = alpha * dt;
            if (std::fabs(val(adt)) > std::fabs(val(C.w))) adt = C.w;
        }
        // spherical continuity term (reading 7), y-sweep only
        T sdt = T(0.0);
        if (src) sdt = dt * cC * C.w * src[j];

        const double k2 = dt * dt / (dsL + dsR);
        T pn, qn, tn;
        if (P.form == 0) {
            T pC = C.w + 2.0 * cC, pL = L.w + 2.0 * cL, pR = R.w + 2.0 * cR;
            T qC = C.w - 2.0 * cC, qL = L.w - 2.0 * cL, qR = R.w - 2.0 * cR;
            T QpL = Q_literal(lpC, lpL, pC, pL, C.d, L.d, dsL);  // Qhat_{j-1} = Q(j, j-1)
            T QpR = Q_literal(lpR, lpC, pR, pC, R.d, C.d, dsR);  // Qhat_j     = Q(j+1, j)
            T QqL = Q_literal(lqC, lqL, qC, qL, C.d, L.d, dsL);
            T QqR = Q_literal(lqR, lqC, qR, qC, R.d, C.d, dsR);
            T Fp, Fq;
            if (P.solver == 1) {                                   // eq. (solver1)
                Fp = dt * Q_literal(lpR, lpL, pR, pL, R.d, L.d, dsL + dsR);
                Fq = dt * Q_literal(lqR, lqL, qR, qL, R.d, L.d, dsL + dsR);
            } else {                                               // eq. (solver2)
                Fp = 0.5 * dt * (QpL + QpR);
                Fq = 0.5 * dt * (QqL + QqR);
            }
            pn = pC - Fp + lpC * k2 * (QpR - QpL) - adt + sdt;
            qn = qC - Fq + lqC * k2 * (QqR - QqL) - adt - sdt;
            // eqs. (stateu), (stateh)
            T un = 0.5 * (pn + qn);
            T hn = (pn - qn) * (pn - qn) / (16.0 * g);
            S.w2[j] = un;
            S.e2[j] = hn - C.d;
        } else {
            T dcL = g * ((C.eta - L.eta) + (C.d - L.d)) / (cC + cL);   // c_j - c_{j-1}
            T dcR = g * ((R.eta - C.eta) + (R.d - C.d)) / (cR + cC);   // c_{j+1} - c_j
            T QpL = Q_perturb(lpC, lpL, C.w, L.w, dcL, C.eta - L.eta, +1.0, dsL);
            T QpR = Q_perturb(lpR, lpC, R.w, C.w, dcR, R.eta - C.eta, +1.0, dsR);
            T QqL = Q_perturb(lqC, lqL, C.w, L.w, dcL, C.eta - L.eta, -1.0, dsL);
            T QqR = Q_perturb(lqR, lqC, R.w, C.w, dcR, R.eta - C.eta, -1.0, dsR);
            T Fp, Fq;
            if (P.solver == 1) {
                T dcRL = g * ((R.eta - L.eta) + (R.d - L.d)) / (cR + cL);
                Fp = dt * Q_perturb(lpR, lpL, R.w, L.w, dcRL, R.eta - L.eta, +1.0, dsL + dsR);
                Fq = dt * Q_perturb(lqR, lqL, R.w, L.w, dcRL, R.eta - L.eta, -1.0, dsL + dsR);
            } else {
                Fp = 0.5 * dt * (QpL + QpR);
                Fq = 0.5 * dt * (QqL + QqR);
            }
            T dp = -Fp + lpC * k2 * (QpR - QpL) - adt + sdt;
            T dq = -Fq + lqC * k2 * (QqR - QqL) - adt - sdt;
            T du = 0.5 * (dp + dq);
            T dc = 0.25 * (dp - dq);
            S.w2[j] = C.w + du;
            S.e2[j] = C.eta + dc * (2.0 * cC + dc) / g;
        }
        // eq. (pq3): transverse velocity, same stencil with speed w and no depth term
        if (P.transverse) {
            T QtL = Qt(C.w, L.w, C.t, L.t, dsL);
            T QtR = Qt(R.w, C.w, R.t, C.t, dsR);
            T Ft = (P.solver == 1) ? dt * Qt(R.w, L.w, R.t, L.t, dsL + dsR) : 0.5 * dt * (QtL + QtR);
            tn = C.t - Ft + C.w * k2 * (QtR - QtL);
        } else {
            tn = C.t;
        }
        S.t2[j] = tn;
    }
    if (rec) {
        for (int j = 0; j < n; ++j) {
            if (rec->wet0) rec->wet0[j] = S.wet0[j];
            if (rec->wet1) rec->wet1[j] = S.wet1[j];
            if (rec->src) rec->src[j] = S.src[j];
            if (rec->eta_b) rec->eta_b[j] = val(S.e1[j]);
            if (rec->w_b) rec->w_b[j] = val(S.w1[j]);
            if (rec->t_b) rec->t_b[j] = val(S.t1[j]);
            if (rec->eta_d) rec->eta_d[j] = val(S.e2[j]);
            if (rec->w_d) rec->w_d[j] = val(S.w2[j]);
            if (rec->t_d) rec->t_d[j] = val(S.t2[j]);
        }
    }
    // (e) cushion limiter on newly wetted cells, against the neighbour's updated state
    for (int i = 0; i < n; ++i) {
        const int j = S.src[i];
        if (j < 0) continue;
        T hi = S.e2[i] + d[i];
        T hj = S.e2[j] + d[j];
        if (val(hi) > 0.5 * val(hj)) S.e2[i] = 0.5 * hj - d[i];
        if (std::fabs(val(S.w2[i])) > std::fabs(val(S.w2[j]))) S.w2[i] = S.w2[j];
    }
    for (int j = 0; j < n; ++j) { eta[j] = S.e2[j]; w[j] = S.w2[j]; t[j] = S.t2[j]; }
}

// ------------------------------------------------------------------ grid geometry
struct Grid {
    Params P;
    const double* x;   // [nx] x (m) or longitude (deg)
    const double* y;   // [ny] y (m) or latitude (deg)
    const double* d;   // [ny*nx]
    bool sph() const { return P.coords != 1; }
    // intervals along row jy, in metres
    void row_ds(int jy, double* ds) const {
        const double f = sph() ? R_SPHERE * std::cos(y[jy] * DEG) * DEG : 1.0;
        for (int i = 0; i + 1 < P.nx; ++i) ds[i] = f * (x[i + 1] - x[i]);
    }
    void col_ds(double* ds) const {
        const double f = sph() ? R_SPHERE * DEG : 1.0;
        for (int j = 0; j + 1 < P.ny; ++j) ds[j] = f * (y[j + 1] - y[j]);
    }
};

template <typename T>
void x_sweep(const Grid& Gd, T* eta, T* u, T* v) {
    const int nx = Gd.P.nx, ny = Gd.P.ny;
    #pragma omp parallel
    {
        Scratch<T> S;
        std::vector<double> ds(nx > 1 ? nx - 1 : 1);
        #pragma omp for schedule(static)
        for (int jy = 0; jy < ny; ++jy) {
            Gd.row_ds(jy, ds.data());
            const size_t o = (size_t)jy * nx;
            sweep_line<T>(Gd.P, nx, ds.data(), Gd.d + o, nullptr, eta + o, u + o, v + o, S, nullptr,
                          Gd.P.open_edges & 3);
        }
    }
}

template <typename T>
void y_sweep(const Grid& Gd, T* eta, T* u, T* v) {
    const int nx = Gd.P.nx, ny = Gd.P.ny;
    std::vector<double> ds(ny > 1 ? ny - 1 : 1), src;
    Gd.col_ds(ds.data());
    if (Gd.sph()) {
        src.resize(ny);
        for (int j = 0; j < ny; ++j) src[j] = std::tan(Gd.y[j] * DEG) / R_SPHERE;
    }
    #pragma omp parallel
    {
        Scratch<T> S;
        std::vector<T> e(ny), a(ny), b(ny);
        std::vector<double> dd(ny);
        #pragma omp for schedule(static)
        for (int ix = 0; ix < nx; ++ix) {
            for (int j = 0; j < ny; ++j) {
                const size_t o = (size_t)j * nx + ix;
                e[j] = eta[o]; a[j] = v[o]; b[j] = u[o]; dd[j] = Gd.d[o];
            }
            sweep_line<T>(Gd.P, ny, ds.data(), dd.data(), src.empty() ? nullptr : src.data(),
                          e.data(), a.data(), b.data(), S, nullptr, (Gd.P.open_edges >> 2) & 3);
            for (int j = 0; j < ny; ++j) {
                const size_t o = (size_t)j * nx + ix;
                eta[o] = e[j]; v[o] = a[j]; u[o] = b[j];
            }
        }
    }
}

// One time step. Order (reading 6): x then y; with P.alternate, y then x on odd steps.
// A 1D grid (nx == 1 or ny == 1) runs only the sweep along its long dimension.
template <typename T>
void step(const Grid& Gd, long k, T* eta, T* u, T* v) {
    const bool dox = Gd.P.nx > 1, doy = Gd.P.ny > 1;
    const bool yfirst = Gd.P.alternate && (k & 1);
    if (yfirst) { if (doy) y_sweep(Gd, eta, u, v); if (dox) x_sweep(Gd, eta, u, v); }
    else        { if (dox) x_sweep(Gd, eta, u, v); if (doy) y_sweep(Gd, eta, u, v); }
}

// ------------------------------------------------------------------ outputs
// Bilinear interpolation weights in the master grid's index space: i is the last node
// with x_i <= xp (clamped to the last interval), a the fraction along that interval.
bool locate(const double* c, int n, double xp, int* i, double* a) {
    if (n == 1) { *i = 0; *a = 0.0; return xp == c[0]; }
    const double lo = std::min(c[0], c[n - 1]), hi = std::max(c[0], c[n - 1]);
    if (xp < lo || xp > hi) return false;
    int k = 0;
    while (k + 2 < n && c[k + 1] <= xp) ++k;
    *i = k;
    *a = (xp - c[k]) / (c[k + 1] - c[k]);
    return true;
}

struct Outputs {
    int maxout;  double* eta_max; double* speed_max;          // [ny*nx] each, or null
    int gout;    int n_gauges; const int* gauge_ixiy;         // [2*G]
    double* gauge_rec; long gauge_cap; long* n_gauge_rec;     // [cap][G][3] (eta,u,v)
    int bndout;  int n_pts; const double* pts_xy;             // [2*P] master coordinates
    double* bnd_rec; long bnd_cap; long* n_bnd_rec;           // [cap][P][3] (u,v,eta)
    std::vector<int> pi, pj;                                  // stencil corner (i, j) per point
    std::vector<double> pa, pb;                               // fractions along x and y
};

template <typename T>
void record(const Grid& Gd, long k, const T* eta, const T* u, const T* v, Outputs* O) {
    const int nx = Gd.P.nx, ny = Gd.P.ny;
    if (O->eta_max && O->maxout > 0 && k % O->maxout == 0) {
        for (size_t c = 0; c < (size_t)nx * ny; ++c) {
            const bool fl = (Gd.P.itopo != 0) || (Gd.d[c] >= Gd.P.dwall);
            if (!(fl && val(eta[c]) + Gd.d[c] >= Gd.P.h_min)) continue;
            O->eta_max[c] = std::max(O->eta_max[c], val(eta[c]));
            const double s = std::sqrt(val(u[c]) * val(u[c]) + val(v[c]) * val(v[c]));
            O->speed_max[c] = std::max(O->speed_max[c], s);
        }
    }
    if (O->gauge_rec && O->gout > 0 && k % O->gout == 0 && *O->n_gauge_rec < O->gauge_cap) {
        double* r = O->gauge_rec + (*O->n_gauge_rec) * O->n_gauges * 3;
        for (int g = 0; g < O->n_gauges; ++g) {
            const size_t c = (size_t)O->gauge_ixiy[2 * g + 1] * nx + O->gauge_ixiy[2 * g];
            r[3 * g + 0] = val(eta[c]); r[3 * g + 1] = val(u[c]); r[3 * g + 2] = val(v[c]);
        }
        ++*O->n_gauge_rec;
    }
    if (O->bnd_rec && O->bndout > 0 && k % O->bndout == 0 && *O->n_bnd_rec < O->bnd_cap) {
        double* r = O->bnd_rec + (*O->n_bnd_rec) * O->n_pts * 3;
        for (int p = 0; p < O->n_pts; ++p) {
            const int i = O->pi[p], j = O->pj[p];
            const double a = O->pa[p], b = O->pb[p];
            const int i1 = (nx > 1) ? i + 1 : i, j1 = (ny > 1) ? j + 1 : j;
            const size_t c00 = (size_t)j * nx + i, c01 = (size_t)j * nx + i1;
            const size_t c10 = (size_t)j1 * nx + i, c11 = (size_t)j1 * nx + i1;
            const double w00 = (1 - a) * (1 - b), w01 = a * (1 - b), w10 = (1 - a) * b, w11 = a * b;
            auto bil = [&](const T* f) {
                return w00 * val(f[c00]) + w01 * val(f[c01]) + w10 * val(f[c10]) + w11 * val(f[c11]);
            };
            r[3 * p + 0] = bil(u); r[3 * p + 1] = bil(v); r[3 * p + 2] = bil(eta);
        }
        ++*O->n_bnd_rec;
    }
}

int set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n; return 1;
#endif
}

}  // namespace

// ================================================================== C interface
extern "C" {

struct oracle_params {
    int32_t nx, ny, coords;
    double h_min, manning_n2;
    int32_t itopo;
    double dwall, dt;
    int32_t transverse, solver, form, alternate;
    int32_t open_edges;
};

static Params to_params(const oracle_params* p) {
    Params P;
    P.nx = p->nx; P.ny = p->ny; P.coords = p->coords; P.h_min = p->h_min;
    P.manning_n2 = p->manning_n2; P.itopo = p->itopo; P.dwall = p->dwall; P.dt = p->dt;
    P.transverse = p->transverse; P.solver = p->solver == 1 ? 1 : 2; P.form = p->form;
    P.alternate = p->alternate;
    P.open_edges = p->open_edges;
    return P;
}

int oracle_threads(int n) { return set_threads(n); }

// Depth-jump filter (section "Numerical stability", eqs. (dstab), (newdw), (newdc)).
// Readings: wet nodes with 0 < d < min_depth are first raised to min_depth (the
// "minimal water depth in wet nodes" of depth_ssl); then passes of a row-wise and a
// column-wise Jacobi update repeat until a pass changes nothing (at most max_passes).
// Land (d <= 0) is never changed. A node is "next to the coastline" when a line
// neighbour is land or lies beyond the domain edge. At a wet node j where
// max(d_{j-1}/d_j, d_{j+1}/d_j) > alpha^2 (over wet neighbours):
//   open water:   d_j = (sqrt(d_{j-1}) + sqrt(d_{j+1}))^2 / 4        (newdw)
//   next to coast: d_j = d_w / alpha^2, d_w the wet neighbour's depth  (newdc)
// Returns the number of passes made (the last one changing nothing), or -1 if the
// cap was reached while nodes were still changing.
int oracle_depth_filter(int nx, int ny, double* d, double alpha, double min_depth, int max_passes) {
    const size_t N = (size_t)nx * ny;
    for (size_t c = 0; c < N; ++c)
        if (d[c] > 0.0 && d[c] < min_depth) d[c] = min_depth;
    const double a2 = alpha * alpha;
    std::vector<double> line;
    auto pass_line = [&](int n, auto get, auto set) -> bool {
        line.resize(n);
        for (int j = 0; j < n; ++j) line[j] = get(j);
        bool changed = false;
        for (int j = 0; j < n; ++j) {
            const double dj = line[j];
            if (!(dj > 0.0)) continue;
            const bool lw = (j > 0) && line[j - 1] > 0.0;
            const bool rw = (j < n - 1) && line[j + 1] > 0.0;
            const bool viol = (lw && line[j - 1] > a2 * dj) || (rw && line[j + 1] > a2 * dj);
            if (!viol) continue;
            double nd;
            if (lw && rw) {
                const double s = std::sqrt(line[j - 1]) + std::sqrt(line[j + 1]);
                nd = s * s / 4.0;
            } else {
                nd = (lw ? line[j - 1] : line[j + 1]) / a2;
            }
            if (nd != dj) { set(j, nd); changed = true; }
        }
        return changed;
    };
    for (int pass = 1; pass <= max_passes; ++pass) {
        bool changed = false;
        if (nx >= 3) for (int jy = 0; jy < ny; ++jy) {
            double* row = d + (size_t)jy * nx;
            changed |= pass_line(nx, [&](int j) { return row[j]; }, [&](int j, double v) { row[j] = v; });
        }
        if (ny >= 3) for (int ix = 0; ix < nx; ++ix) {
            changed |= pass_line(ny, [&](int j) { return d[(size_t)j * nx + ix]; },
                                 [&](int j, double v) { d[(size_t)j * nx + ix] = v; });
        }
        if (!changed) return pass;
    }
    return -1;
}

// One sweep of one line with the phase record (tests of steps (a)-(e)).
int oracle_sweep_line(const oracle_params* p, int n, const double* ds, const double* d,
                      const double* src, double* eta, double* w, double* t,
                      int* wet0, int* wet1, int* srcidx, double* eta_b, double* w_b, double* t_b,
                      double* eta_d, double* w_d, double* t_d) {
    if (n < 3) return -1;
    Params P = to_params(p);
    Scratch<double> S;
    PhaseRec rec{wet0, wet1, srcidx, eta_b, w_b, t_b, eta_d, w_d, t_d};
    sweep_line<double>(P, n, ds, d, src, eta, w, t, S, &rec, P.open_edges & 3);
    return 0;
}

// Run nsteps time steps from step index step0. Outputs (any may be null):
//  record_initial: record the outputs of the given state as step step0 first;
//  fold_final: fold the final state into the max-wave fields (the "end of the
//  computations" update of field maxout).
int oracle_run(const oracle_params* p, const double* x, const double* y, const double* d,
               double* eta, double* u, double* v, long step0, long nsteps,
               int record_initial, int fold_final,
               int maxout, double* eta_max, double* speed_max,
               int gout, int n_gauges, const int* gauge_ixiy, double* gauge_rec, long gauge_cap,
               long* n_gauge_rec,
               int bndout, int n_pts, const double* pts_xy, double* bnd_rec, long bnd_cap,
               long* n_bnd_rec) {
    Params P = to_params(p);
    if (P.nx < 1 || P.ny < 1) return -1;
    if ((P.nx > 1 && P.nx < 3) || (P.ny > 1 && P.ny < 3)) return -1;
    Grid Gd{P, x, y, d};
    long zero1 = 0, zero2 = 0;
    Outputs O{maxout, eta_max, speed_max, gout, n_gauges, gauge_ixiy, gauge_rec, gauge_cap,
              n_gauge_rec ? n_gauge_rec : &zero1, bndout, n_pts, pts_xy, bnd_rec, bnd_cap,
              n_bnd_rec ? n_bnd_rec : &zero2, {}, {}, {}, {}};
    for (int i = 0; i + 1 < P.nx; ++i) if (!(x[i + 1] > x[i])) return -3;
    for (int j = 0; j + 1 < P.ny; ++j) if (!(y[j + 1] > y[j])) return -3;
    O.pi.resize(n_pts); O.pj.resize(n_pts); O.pa.resize(n_pts); O.pb.resize(n_pts);
    for (int q = 0; q < n_pts; ++q) {
        if (!locate(x, P.nx, pts_xy[2 * q], &O.pi[q], &O.pa[q]) ||
            !locate(y, P.ny, pts_xy[2 * q + 1], &O.pj[q], &O.pb[q])) return -2;
    }
    if (record_initial) record<double>(Gd, step0, eta, u, v, &O);
    for (long k = step0; k < step0 + nsteps; ++k) {
        step<double>(Gd, k, eta, u, v);
        record<double>(Gd, k + 1, eta, u, v, &O);
    }
    if (fold_final && eta_max) {
        Outputs F = O; F.maxout = 1; F.gauge_rec = nullptr; F.bnd_rec = nullptr;
        record<double>(Gd, 0, eta, u, v, &F);
    }
    return 0;
}

// Boundary input (section "Running Options", "The input to the computations"): time series
// of (u, v, eta) at the nodes of the W, E, S and N edges, vals[nt][3][np] at times[nt]. The
// paper does not say how the input enters the scheme; the reading taken here: before each
// step, the edge nodes take the input's values at the current model time, linearly
// interpolated between records (the first or last record outside their span); the edges
// are set in the order W, E, S, N, so S and N own the corners. An edge with no series is
// left to the scheme (a reflecting wall).
extern "C++" {
template <typename T>
static void impose_edge(const Params& P, T* eta, T* u, T* v, int edge,
                        const double* times, long nt, const double* vals, double t) {
    const int np = (edge < 2) ? P.ny : P.nx;
    long k = 0;
    double w = 0.0;
    if (t <= times[0] || nt == 1) { k = 0; w = 0.0; }
    else if (t >= times[nt - 1]) { k = nt - 1; w = 0.0; }
    else {
        while (k + 1 < nt - 1 && times[k + 1] <= t) ++k;
        w = (t - times[k]) / (times[k + 1] - times[k]);
    }
    for (int q = 0; q < np; ++q) {
        const int ix = (edge == 0) ? 0 : (edge == 1) ? P.nx - 1 : q;
        const int iy = (edge == 2) ? 0 : (edge == 3) ? P.ny - 1 : q;
        const size_t c = (size_t)iy * P.nx + ix;
        double val[3];
        for (int f = 0; f < 3; ++f) {
            const double a = vals[(k * 3 + f) * np + q];
            const double b = (w > 0.0) ? vals[((k + 1) * 3 + f) * np + q] : a;
            val[f] = (1.0 - w) * a + w * b;
        }
        u[c] = T(val[0]); v[c] = T(val[1]); eta[c] = T(val[2]);   // the input does not depend on the state
    }
}
}  // extern "C++"

// A run under boundary input from model time t0: before step k the edges are set at time
// t0 + (k - step0) dt. Gauges (eta, u, v) are recorded as in oracle_run.
int oracle_run_forced(const oracle_params* p, const double* x, const double* y, const double* d,
                      double* eta, double* u, double* v, long step0, long nsteps, double t0,
                      const double* const* times, const long* nt, const double* const* vals,
                      int gout, int n_gauges, const int* gauge_ixiy, double* gauge_rec, long gauge_cap,
                      long* n_gauge_rec) {
    Params P = to_params(p);
    if ((P.nx > 1 && P.nx < 3) || (P.ny > 1 && P.ny < 3)) return -1;
    Grid Gd{P, x, y, d};
    long zero1 = 0, zero2 = 0;
    Outputs O{0, nullptr, nullptr, gout, n_gauges, gauge_ixiy, gauge_rec, gauge_cap,
              n_gauge_rec ? n_gauge_rec : &zero1, 0, 0, nullptr, nullptr, 0, &zero2, {}, {}, {}, {}};
    record<double>(Gd, step0, eta, u, v, &O);
    for (long k = step0; k < step0 + nsteps; ++k) {
        const double t = t0 + (double)(k - step0) * P.dt;
        for (int e = 0; e < 4; ++e)
            if (times[e] && nt[e] > 0) impose_edge<double>(P, eta, u, v, e, times[e], nt[e], vals[e], t);
        step<double>(Gd, k, eta, u, v);
        record<double>(Gd, k + 1, eta, u, v, &O);
    }
    return 0;
}

static int run_tlm_impl(const oracle_params* p, const double* x, const double* y, const double* d,
                        double* eta, double* u, double* v, double* deta, double* du, double* dv,
                        long step0, long nsteps, int record_initial,
                        int gout, int n_gauges, const int* gauge_ixiy,
                        double* gauge_val, double* gauge_tan, long cap, long* nrec,
                        double t0, const double* const* times, const long* nt, const double* const* vals,
                        double* gauge_tan_uv);

// Tangent-linear run: the primal (eta,u,v) and a tangent (deta,du,dv) advance together;
// every branch is decided on the primal. Gauge tangents of eta are written to
// gauge_tan[nrec][G] at the steps where gauges are recorded.
int oracle_run_tlm(const oracle_params* p, const double* x, const double* y, const double* d,
                   double* eta, double* u, double* v, double* deta, double* du, double* dv,
                   long step0, long nsteps, int record_initial,
                   int gout, int n_gauges, const int* gauge_ixiy,
                   double* gauge_val, double* gauge_tan, long cap, long* nrec) {
    return run_tlm_impl(p, x, y, d, eta, u, v, deta, du, dv, step0, nsteps, record_initial, gout, n_gauges,
                        gauge_ixiy, gauge_val, gauge_tan, cap, nrec, 0.0, nullptr, nullptr, nullptr, nullptr);
}

// oracle_run_tlm that also writes the gauge tangents of u and v to gauge_tan_uv[nrec][G][2].
int oracle_run_tlm_uv(const oracle_params* p, const double* x, const double* y, const double* d,
                      double* eta, double* u, double* v, double* deta, double* du, double* dv,
                      long step0, long nsteps, int record_initial,
                      int gout, int n_gauges, const int* gauge_ixiy,
                      double* gauge_val, double* gauge_tan, double* gauge_tan_uv, long cap, long* nrec) {
    return run_tlm_impl(p, x, y, d, eta, u, v, deta, du, dv, step0, nsteps, record_initial, gout, n_gauges,
                        gauge_ixiy, gauge_val, gauge_tan, cap, nrec, 0.0, nullptr, nullptr, nullptr, gauge_tan_uv);
}

// The tangent-linear model of oracle_run_forced: the imposed edge values carry no tangent.
int oracle_run_tlm_forced(const oracle_params* p, const double* x, const double* y, const double* d,
                          double* eta, double* u, double* v, double* deta, double* du, double* dv,
                          long step0, long nsteps, int gout, int n_gauges, const int* gauge_ixiy,
                          double* gauge_val, double* gauge_tan, long cap, long* nrec,
                          double t0, const double* const* times, const long* nt, const double* const* vals) {
    return run_tlm_impl(p, x, y, d, eta, u, v, deta, du, dv, step0, nsteps, 1, gout, n_gauges, gauge_ixiy,
                        gauge_val, gauge_tan, cap, nrec, t0, times, nt, vals, nullptr);
}

}  // extern "C"

static int run_tlm_impl(const oracle_params* p, const double* x, const double* y, const double* d,
                        double* eta, double* u, double* v, double* deta, double* du, double* dv,
                        long step0, long nsteps, int record_initial,
                        int gout, int n_gauges, const int* gauge_ixiy,
                        double* gauge_val, double* gauge_tan, long cap, long* nrec,
                        double t0, const double* const* times, const long* nt, const double* const* vals,
                        double* gauge_tan_uv) {
    Params P = to_params(p);
    if ((P.nx > 1 && P.nx < 3) || (P.ny > 1 && P.ny < 3)) return -1;
    Grid Gd{P, x, y, d};
    const size_t N = (size_t)P.nx * P.ny;
    std::vector<Dual> E(N), U(N), V(N);
    for (size_t c = 0; c < N; ++c) { E[c] = Dual(eta[c], deta[c]); U[c] = Dual(u[c], du[c]); V[c] = Dual(v[c], dv[c]); }
    long n = 0;
    auto rec = [&](long k) {
        if (gout <= 0 || k % gout != 0 || n >= cap) return;
        for (int g = 0; g < n_gauges; ++g) {
            const size_t c = (size_t)gauge_ixiy[2 * g + 1] * P.nx + gauge_ixiy[2 * g];
            if (gauge_val) gauge_val[n * n_gauges + g] = E[c].v;
            gauge_tan[n * n_gauges + g] = E[c].d;
            if (gauge_tan_uv) {
                gauge_tan_uv[2 * (n * n_gauges + g)] = U[c].d;
                gauge_tan_uv[2 * (n * n_gauges + g) + 1] = V[c].d;
            }
        }
        ++n;
    };
    if (record_initial) rec(step0);
    for (long k = step0; k < step0 + nsteps; ++k) {
        if (times) {
            const double t = t0 + (double)(k - step0) * P.dt;
            for (int e = 0; e < 4; ++e)
                if (times[e] && nt[e] > 0) impose_edge<Dual>(P, E.data(), U.data(), V.data(), e, times[e], nt[e], vals[e], t);
        }
        step<Dual>(Gd, k, E.data(), U.data(), V.data());
        rec(k + 1);
    }
    for (size_t c = 0; c < N; ++c) {
        eta[c] = E[c].v; u[c] = U[c].v; v[c] = V[c].v;
        deta[c] = E[c].d; du[c] = U[c].d; dv[c] = V[c].d;
    }
    if (nrec) *nrec = n;
    return 0;
}


