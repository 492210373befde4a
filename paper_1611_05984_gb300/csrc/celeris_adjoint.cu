// Discrete adjoint of the time step -- the AB3 predictor with its Euler
// start-up and the AM4 corrector stages (Eq. 15-20, Sec. 2.3) -- for the
// Boussinesq model and the nonlinear shallow-water model (Sec. 3.2), and the
// gradient of a gauge misfit.  The reverse of one stage, given the adjoint
// lambda of the state after it (the host code in celeris_api.cu orders the
// stages, the checkpoints and the recomputation):
//   1. the masks of the update: the dry clamp w >= Bbar (Reading A-D1), the
//      sponge (Eq. 30), the zero discharge of dry cells;
//   2. the line solves (Eq. 21-23) transposed: the adjoint of the U* and V*
//      increments solves the transposed tridiagonal system of every line
//      (the forward's line solver in its transposed mode);
//   3. the history: the right sides R = (E, F, G) and the mixed terms F*, G*
//      collect the adjoint weighted by their AB3 / AM4 coefficients;
//   4. R's and F*'s Jacobians transposed at the stage's input state: every
//      face flux (KP07 reconstruction with the limiter and positivity
//      branches the forward took, then the central-upwind flux: a reverse
//      written by hand, checked against dual numbers), the bed slope and
//      friction (by hand), the dispersive eta terms of Eq. 10-11 and
//      F*, G* of Eq. 12-13 (linear in the neighbours, transposed in closed
//      form, ghosts mapped back to the cells they mirror).
// With the bed's gradient requested, the same Jacobians are taken with
// respect to the bed as well: the face beds of the reconstruction and the
// flux, the cell bed of the bed slope, friction and the dry clamp, the
// still-water depth d of the dispersive terms and of the line systems' rows
// (dT/dd with the transposed solves' solution and the forward's), the sine
// makers' ghost values (Eq. 25-29), summed over the run and mapped through
// d = max(w_s - Bbar, 0), Bbar = mean of 4 corners and corner = mean of 4
// cell-centre beds (Reading A-W1) to dL/dz.  Every branch is the forward's.
// Adjoints reach a cell from several faces and cells; they are summed in
// shared memory per tile and added to global memory with atomics, so the
// sums' order is not fixed.
#include "celeris_adjoint.cuh"
#include "celeris_physics.cuh"

#include <math.h>

namespace cel {
namespace {

// Forward-mode dual number: a value and its derivative along one direction.
template <typename T>
struct Dual {
    T v, d;
    __device__ __forceinline__ Dual() : v(0), d(0) {}
    __device__ __forceinline__ Dual(T x) : v(x), d(0) {}
    __device__ __forceinline__ Dual(T x, T dx) : v(x), d(dx) {}
};

template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b)
{
    return {a.v * b.v, a.d * b.v + a.v * b.d};
}
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b)
{
    const T q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <typename T> __device__ __forceinline__ bool operator<(Dual<T> a, Dual<T> b) { return a.v < b.v; }
template <typename T> __device__ __forceinline__ bool operator>(Dual<T> a, Dual<T> b) { return a.v > b.v; }
template <typename T> __device__ __forceinline__ Dual<T> fmax(Dual<T> a, Dual<T> b) { return a.v >= b.v ? a : b; }
template <typename T> __device__ __forceinline__ Dual<T> fmin(Dual<T> a, Dual<T> b) { return a.v <= b.v ? a : b; }
template <typename T> __device__ __forceinline__ Dual<T> sqrt(Dual<T> a)
{
    const T s = ::sqrt(a.v);
    return {s, s > T(0) ? a.d / (T(2) * s) : T(0)};
}
template <typename T> __device__ __forceinline__ Dual<T> rsqrt(Dual<T> a)
{
    const T r = ::rsqrt(a.v);
    return {r, T(-0.5) * r * r * r * a.d};
}
template <typename T> __device__ __forceinline__ Dual<T> cbrt_r(Dual<T> a)
{
    const T c = cel::cbrt_r(a.v);
    return {c, a.v > T(0) ? a.d / (T(3) * c * c) : T(0)};
}

// the plain-type overloads stay visible next to the dual ones
using ::fmax;
using ::fmin;
using ::sqrt;
using ::rsqrt;

// A cell a face stencil reads: its (w, P, Q) and either the interior cell it
// mirrors with the sign of each variable there (Sec. 2.4, Reading A-B1), or,
// for a sine-maker ghost, its place in the ghost table.
template <typename real>
struct Src {
    real v[3];
    int idx;          // interior cell, -1 for a sine-maker ghost
    int ci, cj;       // its coordinates
    int gs, gl, gp;   // the ghost's side, layer and table position (idx = -1)
    real sgn[3];
};

// Cell (i, j) of an interior row (x-direction ghosts only) or column
// (y-direction ghosts only).
template <typename real>
__device__ __forceinline__ Src<real> source(const AdjArgs<real> &A, int i, int j, int dir)
{
    const Geo &G = A.geo;
    Src<real> s;
    s.sgn[0] = s.sgn[1] = s.sgn[2] = real(1);
    int side = -1, layer = 0, si = i, sj = j;
    if (dir == 0 && i < 0) { side = 0; layer = -1 - i; si = -1 - i; }
    if (dir == 0 && i >= G.nx) { side = 1; layer = i - G.nx; si = 2 * G.nx - 1 - i; }
    if (dir == 1 && j < 0) { side = 2; layer = -1 - j; sj = -1 - j; }
    if (dir == 1 && j >= G.ny) { side = 3; layer = j - G.ny; sj = 2 * G.ny - 1 - j; }
    if (side >= 0 && ((A.c.sine >> side) & 1)) {
        const int pos = (dir == 0 ? j : i) + 2;
        const real *tb = A.ghost + ghost_index(A.tsel, side, layer, 0, pos, A.c.npos);
        s.v[0] = tb[0];
        s.v[1] = tb[A.c.npos];
        s.v[2] = tb[2 * A.c.npos];
        s.idx = -1;
        s.gs = side;
        s.gl = layer;
        s.gp = pos;
        return s;
    }
    if (side >= 0) s.sgn[dir == 0 ? 1 : 2] = real(-1);   // the normal discharge is negated
    s.idx = sj * G.nx + si;
    s.ci = si;
    s.cj = sj;
    s.v[0] = A.w[s.idx];
    s.v[1] = s.sgn[1] * A.P[s.idx];
    s.v[2] = s.sgn[2] * A.Q[s.idx];
    return s;
}

// Any cell of the one-cell ring around the grid, or two cells out along an
// axis, as the stencil fills it: x-side ghosts over interior rows, then
// y-side ghosts over every column, so a corner ghost is the y-mirror of an
// x-ghost (Reading A-B5).
template <typename real>
__device__ __forceinline__ Src<real> source2d(const AdjArgs<real> &A, int i, int j)
{
    const Geo &G = A.geo;
    if (j >= 0 && j < G.ny) return source(A, i, j, 0);
    const int side = j < 0 ? 2 : 3, layer = j < 0 ? -1 - j : j - G.ny;
    const int sj = j < 0 ? -1 - j : 2 * G.ny - 1 - j;
    Src<real> s;
    if ((A.c.sine >> side) & 1) {
        const real *tb = A.ghost + ghost_index(A.tsel, side, layer, 0, i + 2, A.c.npos);
        s.v[0] = tb[0];
        s.v[1] = tb[A.c.npos];
        s.v[2] = tb[2 * A.c.npos];
        s.idx = -1;
        s.gs = side;
        s.gl = layer;
        s.gp = i + 2;
        s.sgn[0] = s.sgn[1] = s.sgn[2] = real(1);
        return s;
    }
    s = source(A, i, sj, 0);   // the cell of the mirrored row (an x-ghost if i is outside)
    s.v[2] = -s.v[2];
    s.sgn[2] = -s.sgn[2];
    return s;
}

// Where a cell of the ring source2d reads comes from, without its values:
// the interior cell it mirrors and the signs, or idx = -1 for a sine-maker
// ghost (the same cases as source and source2d).
template <typename real>
__device__ __forceinline__ void mirror2d(const Geo &G, int sine, int i, int j, Src<real> &s)
{
    s.sgn[0] = s.sgn[1] = s.sgn[2] = real(1);
    s.idx = -1;
    int si = i, sj = j;
    if (j < 0 || j >= G.ny) {   // a y-ghost: the mirrored row's cell, Q negated
        if ((sine >> (j < 0 ? 2 : 3)) & 1) {
            s.gs = j < 0 ? 2 : 3;
            s.gl = j < 0 ? -1 - j : j - G.ny;
            s.gp = i + 2;
            s.sgn[2] = real(1);
            return;
        }
        sj = j < 0 ? -1 - j : 2 * G.ny - 1 - j;
        s.sgn[2] = real(-1);
    }
    if (i < 0 || i >= G.nx) {   // an x-ghost: P negated
        if ((sine >> (i < 0 ? 0 : 1)) & 1) {
            s.gs = i < 0 ? 0 : 1;
            s.gl = i < 0 ? -1 - i : i - G.nx;
            s.gp = sj + 2;
            s.sgn[0] = s.sgn[1] = s.sgn[2] = real(1);
            return;
        }
        si = i < 0 ? -1 - i : 2 * G.nx - 1 - i;
        s.sgn[1] = real(-1);
    }
    s.ci = si;
    s.cj = sj;
    s.idx = sj * G.nx + si;
}

// Flux through x-face f (dir 0: between cells f-1 and f of row `line`) or
// y-face f (dir 1: between rows f-1 and f of column `line`) from the 4 cells
// around it, in the forward's order of operations.
template <typename T>
__device__ __forceinline__ void face_flux(const Dual<T> w[4], const Dual<T> P[4], const Dual<T> Q[4], Dual<T> Bm,
                                          Dual<T> Bf, Dual<T> Bp, T th, T g, T eps, int dir, Dual<T> H[3])
{
    Dual<T> lo[3], hiL[3], loR[3], hiR[3];
    const Dual<T> w0[3] = {w[0], w[1], w[2]}, P0[3] = {P[0], P[1], P[2]}, Q0[3] = {Q[0], Q[1], Q[2]};
    const Dual<T> w1[3] = {w[1], w[2], w[3]}, P1[3] = {P[1], P[2], P[3]}, Q1[3] = {Q[1], Q[2], Q[3]};
    recon(Dual<T>(th), w0, P0, Q0, Bm, Bf, lo, hiL);
    recon(Dual<T>(th), w1, P1, Q1, Bf, Bp, loR, hiR);
    if (dir == 0)
        cu_flux(Dual<T>(g), Dual<T>(eps), hiL[0], hiL[1], hiL[2], loR[0], loR[1], loR[2], Bf, H);
    else
        cu_flux(Dual<T>(g), Dual<T>(eps), hiL[0], hiL[2], hiL[1], loR[0], loR[2], loR[1], Bf, H);
}

// The same flux's vector-Jacobian product by hand (reverse mode): one pass
// forward keeping the branch each max, min, minmod and positivity test took
// (ties resolved as the dual numbers resolve them: fmax keeps its first
// argument when equal, fmin too, sqrt has derivative 0 at 0), then the
// adjoints back through every operation.  Outputs: the adjoints of the 4
// cells' (w, P, Q) and of the three face beds (Bm, Bf, Bp), added to.
template <typename T>
__device__ __forceinline__ int minmod3_sel(T th, T qm, T q0, T qp)
{
    const T a = th * (q0 - qm), b = T(0.5) * (qp - qm), c = th * (qp - q0);
    const int ilo_bc = b <= c ? 2 : 3, ihi_bc = b >= c ? 2 : 3;
    const T lo_bc = b <= c ? b : c, hi_bc = b >= c ? b : c;
    const int ilo = a <= lo_bc ? 1 : ilo_bc, ihi = a >= hi_bc ? 1 : ihi_bc;
    const T lo = a <= lo_bc ? a : lo_bc, hi = a >= hi_bc ? a : hi_bc;
    return lo > T(0) ? ilo : (hi < T(0) ? ihi : 0);
}

template <typename T>
__device__ __forceinline__ T slope_of(int sel, T th, T qm, T q0, T qp)
{
    return sel == 1 ? th * (q0 - qm) : sel == 2 ? T(0.5) * (qp - qm) : sel == 3 ? th * (qp - q0) : T(0);
}

// adjoint ls of the selected slope into its three cells
template <typename T>
__device__ __forceinline__ void slope_vjp(int sel, T th, T ls, T &lqm, T &lq0, T &lqp)
{
    if (sel == 1) { lqm -= th * ls; lq0 += th * ls; }
    else if (sel == 2) { lqm -= T(0.5) * ls; lqp += T(0.5) * ls; }
    else if (sel == 3) { lq0 -= th * ls; lqp += th * ls; }
}

// dk/dh of desing (Eq. 14) with its branch of max(h^4, eps)
template <typename T>
__device__ __forceinline__ T desing_dh(T h, T eps)
{
    const T h2 = h * h, h4 = h2 * h2;
    const bool sel = h4 >= eps;
    const T r = rsqrt(h4 + (sel ? h4 : eps));
    return T(1.4142135623730951) * r * (T(1) - T(2) * h4 * r * r * (sel ? T(2) : T(1)));
}

template <typename T>
__device__ __forceinline__ void face_flux_vjp(const T w[4], const T P[4], const T Q[4], T Bm, T Bf, T Bp, T th, T g,
                                              T eps, int dir, const T lH[3], T lw[4], T lP[4], T lQ[4], T lB[3])
{
    // reconstruction: left cell 1 (its high face), right cell 2 (its low face)
    int sw[2], sP[2], sQ[2], fix[2];   // fix: 0 none, 1 high face clamped, 2 low face clamped
    T f[2][3];                          // hiL and loR in (w, P, Q)
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const T Blo = c == 0 ? Bm : Bf, Bhi = c == 0 ? Bf : Bp;
        sw[c] = minmod3_sel(th, w[c], w[c + 1], w[c + 2]);
        sP[c] = minmod3_sel(th, P[c], P[c + 1], P[c + 2]);
        sQ[c] = minmod3_sel(th, Q[c], Q[c + 1], Q[c + 2]);
        const T s0 = slope_of(sw[c], th, w[c], w[c + 1], w[c + 2]);
        const T lo0 = w[c + 1] - T(0.5) * s0, hi0 = w[c + 1] + T(0.5) * s0;
        fix[c] = hi0 < Bhi ? 1 : (lo0 < Blo ? 2 : 0);
        const T v0 = c == 0 ? (fix[c] == 1 ? Bhi : fix[c] == 2 ? T(2) * w[1] - Blo : hi0)
                            : (fix[c] == 1 ? T(2) * w[2] - Bhi : fix[c] == 2 ? Blo : lo0);
        const T sgn = c == 0 ? T(0.5) : T(-0.5);
        f[c][0] = v0;
        f[c][1] = P[c + 1] + sgn * slope_of(sP[c], th, P[c], P[c + 1], P[c + 2]);
        f[c][2] = Q[c + 1] + sgn * slope_of(sQ[c], th, Q[c], Q[c + 1], Q[c + 2]);
    }
    // central-upwind flux on (w, normal, tangential)
    const int nv = dir == 0 ? 1 : 2, tv = dir == 0 ? 2 : 1;
    const T wL = f[0][0], nL = f[0][nv], tL = f[0][tv], wR = f[1][0], nR = f[1][nv], tR = f[1][tv];
    const T aL = wL - Bf, aR = wR - Bf;
    const bool pL = aL >= T(0), pR = aR >= T(0);
    const T hL = pL ? aL : T(0), hR = pR ? aR : T(0);
    const T kL = desing(hL, eps), kR = desing(hR, eps);
    const T uL = kL * nL, vL = kL * tL, uR = kR * nR, vR = kR * tR;
    const T qnL = hL * uL, qtL = hL * vL, qnR = hR * uR, qtR = hR * vR;
    const T sL = sqrt(g * hL), sR = sqrt(g * hR);
    const T ap1c = uL + sL, ap2c = uR + sR, am1c = uL - sL, am2c = uR - sR;
    const bool apL = ap1c >= ap2c, amL = am1c <= am2c;
    const T ap1 = apL ? ap1c : ap2c, am1 = amL ? am1c : am2c;
    const bool apK = ap1 >= T(0), amK = am1 <= T(0);
    const T ap = apK ? ap1 : T(0), am = amK ? am1 : T(0);
    const T den = ap - am;
    if (!(den > T(0))) return;
    const T inv = T(1) / den, apam = ap * am;
    const T FL1 = qnL * uL + T(0.5) * g * hL * hL, FR1 = qnR * uR + T(0.5) * g * hR * hR;
    const T N0 = ap * qnL - am * qnR + apam * (wR - wL);
    const T N1 = ap * FL1 - am * FR1 + apam * (qnR - qnL);
    const T N2 = ap * (qnL * vL) - am * (qnR * vR) + apam * (qtR - qtL);
    // reverse
    const T lN0 = lH[0] * inv, lN1 = lH[1] * inv, lN2 = lH[2] * inv;
    const T lden = -(lH[0] * N0 + lH[1] * N1 + lH[2] * N2) * inv * inv;
    const T lapam = lN0 * (wR - wL) + lN1 * (qnR - qnL) + lN2 * (qtR - qtL);
    const T lap = lN0 * qnL + lN1 * FL1 + lN2 * (qnL * vL) + lapam * am + lden;
    const T lam = -(lN0 * qnR) - lN1 * FR1 - lN2 * (qnR * vR) + lapam * ap - lden;
    const T lFL1 = lN1 * ap, lFR1 = -(lN1 * am);
    T lqnL = lN0 * ap - lN1 * apam + lN2 * ap * vL + lFL1 * uL;
    T lqnR = -(lN0 * am) + lN1 * apam - lN2 * am * vR + lFR1 * uR;
    T lvL = lN2 * ap * qnL, lvR = -(lN2 * am * qnR);
    const T lqtL = -(lN2 * apam), lqtR = lN2 * apam;
    T lwL = -(lN0 * apam), lwR = lN0 * apam;
    T luL = lFL1 * qnL, luR = lFR1 * qnR;
    T lhL = lFL1 * g * hL, lhR = lFR1 * g * hR;
    T lsL = T(0), lsR = T(0);
    if (apK) {
        if (apL) { luL += lap; lsL += lap; }
        else { luR += lap; lsR += lap; }
    }
    if (amK) {
        if (amL) { luL += lam; lsL -= lam; }
        else { luR += lam; lsR -= lam; }
    }
    if (sL > T(0)) lhL += lsL * g / (T(2) * sL);
    if (sR > T(0)) lhR += lsR * g / (T(2) * sR);
    lhL += lqnL * uL + lqtL * vL;
    luL += lqnL * hL;
    lvL += lqtL * hL;
    lhR += lqnR * uR + lqtR * vR;
    luR += lqnR * hR;
    lvR += lqtR * hR;
    const T lkL = luL * nL + lvL * tL, lkR = luR * nR + lvR * tR;
    T lf[2][3];
    lf[0][nv] = luL * kL;
    lf[0][tv] = lvL * kL;
    lf[1][nv] = luR * kR;
    lf[1][tv] = lvR * kR;
    lhL += lkL * desing_dh(hL, eps);
    lhR += lkR * desing_dh(hR, eps);
    const T laL = pL ? lhL : T(0), laR = pR ? lhR : T(0);
    lf[0][0] = lwL + laL;
    lf[1][0] = lwR + laR;
    lB[1] -= laL + laR;
    // reconstruction reversed
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const T sgn = c == 0 ? T(0.5) : T(-0.5);
        const T lv = lf[c][0];
        const int bl = c == 0 ? 0 : 1, bh = c == 0 ? 1 : 2;   // indices of Blo, Bhi in lB
        if (c == 0) {
            if (fix[c] == 1) lB[bh] += lv;
            else if (fix[c] == 2) { lw[1] += T(2) * lv; lB[bl] -= lv; }
            else { lw[1] += lv; slope_vjp(sw[c], th, sgn * lv, lw[0], lw[1], lw[2]); }
        } else {
            if (fix[c] == 1) { lw[2] += T(2) * lv; lB[bh] -= lv; }
            else if (fix[c] == 2) lB[bl] += lv;
            else { lw[2] += lv; slope_vjp(sw[c], th, sgn * lv, lw[1], lw[2], lw[3]); }
        }
        lP[c + 1] += lf[c][1];
        slope_vjp(sP[c], th, sgn * lf[c][1], lP[c], lP[c + 1], lP[c + 2]);
        lQ[c + 1] += lf[c][2];
        slope_vjp(sQ[c], th, sgn * lf[c][2], lQ[c], lQ[c + 1], lQ[c + 2]);
    }
}

// The dual-number VJP of the same flux, one input direction at a time: the
// reference the hand-written reverse is checked against.
template <typename T>
__device__ __forceinline__ void face_flux_vjp_dual(const T w[4], const T P[4], const T Q[4], T Bm, T Bf, T Bp, T th,
                                                   T g, T eps, int dir, const T lH[3], T out[15])
{
    for (int k = 0; k < 15; k++) {
        Dual<T> dw[4], dP[4], dQ[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            dw[q] = Dual<T>(w[q], k == q ? T(1) : T(0));
            dP[q] = Dual<T>(P[q], k == 4 + q ? T(1) : T(0));
            dQ[q] = Dual<T>(Q[q], k == 8 + q ? T(1) : T(0));
        }
        Dual<T> H[3];
        face_flux(dw, dP, dQ, Dual<T>(Bm, k == 12 ? T(1) : T(0)), Dual<T>(Bf, k == 13 ? T(1) : T(0)),
                  Dual<T>(Bp, k == 14 ? T(1) : T(0)), th, g, eps, dir, H);
        out[k] = lH[0] * H[0].d + lH[1] * H[1].d + lH[2] * H[2].d;
    }
}

// Index of cell (i, j), i in [-1, nx], j in [-1, ny], in the ring arrays.
__device__ __forceinline__ size_t ring_index(const Geo &G, int i, int j)
{
    return (size_t)(j + 1) * (G.nx + 2) + (i + 1);
}

// Index of corner (ci, cj) in the corner arrays.
__device__ __forceinline__ size_t corner_index(const Geo &G, int ci, int cj)
{
    return (size_t)(cj + 1) * G.pc + (ci + 1);
}

// Step 1 of the reverse: the masks; the state's own path (w^{n+1} = w^n +
// ...) passes the masked adjoint on unchanged.  One 32 x 32 tile per block
// of 32 x 32 threads, a cell per thread; the y-lines' right side
// (column-major) is transposed in shared memory and written along columns.
template <typename real>
__global__ void __launch_bounds__(1024) k_adj_mask(AdjArgs<real> A)
{
    dependent_launch_wait_then_release();
    __shared__ real tq[32][33];
    const Geo &G = A.geo;
    const int tx = threadIdx.x, ty = threadIdx.y, bx = blockIdx.x * 32, by = blockIdx.y * 32;
    const int i = bx + tx, j = by + ty;
    real lq = real(0);
    if (i < G.nx && j < G.ny) {
        const int k = j * G.nx + i;
        const real Bb = bbar_at(A.Bc, G, i, j);
        const real ws = A.c.ws;
        const real d = fmax(ws - Bb, real(0));
        const real gam = A.final_stage ? sponge_gamma<real>(A.c, G, i, j) : real(1);
        const real wn = A.w_next[k];
        const bool dry = wn - Bb <= real(0);
        const bool spw = gam < real(1) && d > real(0);
        const real w1 = spw ? ws + (wn - ws) / gam : wn;   // before the sponge
        const real tol = (sizeof(real) == 8 ? real(1e-12) : real(1e-6)) * fmax(real(1), fabs(Bb));
        const bool clamped = w1 - Bb <= tol;
        if (clamped && A.lBb) A.lBb[ring_index(G, i, j)] += A.lw[k] * (spw ? gam : real(1));   // w = Bbar there
        A.lw[k] = clamped ? real(0) : A.lw[k] * (spw ? gam : real(1));
        const real lp = dry ? real(0) : A.lP[k] * gam;
        lq = dry ? real(0) : A.lQ[k] * gam;
        A.lP[k] = lp;
        A.lQ[k] = lq;
        if (A.packX) A.packX[(size_t)j * G.px + i] = lp;
        if (A.zero[0]) A.zero[0][k] = A.zero[1][k] = A.zero[2][k] = real(0);
    }
    if (A.packX) {
        tq[ty][tx] = lq;
        __syncthreads();
        const int ic = bx + ty, jc = by + tx;
        if (ic < G.nx && jc < G.ny) A.packY[(size_t)ic * G.py + jc] = tq[tx][ty];
    }
}

// Step 3: the history.  The increments of w, U* and V* weigh R^n, R^{n-1},
// R^{n-2} by c0, c1, c2 and (U*, V*) the mixed terms F*, G* by e0, e1, e2.
// One 32 x 32 tile per block of 32 x 32 threads, a cell per thread; the
// y-lines' solution (column-major) is read along its columns and transposed
// in shared memory.
template <typename real>
__global__ void __launch_bounds__(1024) k_adj_hist(AdjArgs<real> A)
{
    dependent_launch_wait_then_release();
    __shared__ real tq[32][33];
    const Geo &G = A.geo;
    const int tx = threadIdx.x, ty = threadIdx.y, bx = blockIdx.x * 32, by = blockIdx.y * 32;
    if (A.muY) {
        const int i = bx + ty, j = by + tx;
        tq[ty][tx] = i < G.nx && j < G.ny ? A.muY[(size_t)i * G.py + j] : real(0);
        __syncthreads();
    }
    const int i = bx + tx, j = by + ty;
    if (i >= G.nx || j >= G.ny) return;
    const int k = j * G.nx + i;
    const real mu = A.muX ? A.muX[(size_t)j * G.px + i] : A.ldU[k];
    const real mv = A.muY ? tq[tx][ty] : A.ldV[k];
    const real m[5] = {A.lw[k], mu, mv, mu, mv};
#pragma unroll
    for (int v = 0; v < 5; v++) {
        if (v >= 3 && !A.bsnq) break;
        const real c0 = v < 3 ? A.c0 : A.e0, c1 = v < 3 ? A.c1 : A.e1, c2 = v < 3 ? A.c2 : A.e2;
        A.G0[v][k] += c0 * m[v];
        if (A.G1[v]) A.G1[v][k] += c1 * m[v];
        if (A.G2[v]) A.G2[v][k] += c2 * m[v];
        if (A.H0[v]) A.H0[v][k] = (v < 3 ? A.hc : A.he) * m[v];
    }
    if (A.accw) {
        A.accw[k] += m[0];
        A.accP[k] += A.lP[k];
        A.accQ[k] += A.lQ[k];
    }
}

// Bed slope and friction (Eq. 9-10, 31-32) at cell (i, j): no neighbours.
template <typename real, typename Acc>
__device__ __forceinline__ void cell_vjp(const AdjArgs<real> &A, int i, int j, const Acc &acc)
{
    const Geo &G = A.geo;
    const int k = j * G.nx + i;
    const real lF = A.G0[1][k], lG = A.G0[2][k];
    const real c00 = acc.bed(i, j), c10 = acc.bed(i + 1, j);
    const real c01 = acc.bed(i, j + 1), c11 = acc.bed(i + 1, j + 1);
    const real Bb = cell_bbar(c00, c10, c01, c11);
    const real BxW = real(0.5) * (c00 + c01), BxE = real(0.5) * (c10 + c11);
    const real ByS = real(0.5) * (c00 + c10), ByN = real(0.5) * (c01 + c11);
    const real g = A.c.g;
    real dw = -(g * (BxE - BxW) * A.c.rdx) * lF - (g * (ByN - ByS) * A.c.rdy) * lG;
    real dP = real(0), dQ = real(0), dfw = real(0);   // dfw: friction's part of dw
    if (A.phy.friction != kFricNone) {
        // -fc |u| u / h with u = k(h) P (Eq. 31-32, Eq. 14): lF fF + lG fG =
        // -fc mag k^2 (lF P + lG Q), mag = |(P, Q)|, k = desing(max(h, 0)),
        // fc = f or g n^2 k^(1/3); its derivatives by hand, along the
        // forward's branches (max keeps h at h = 0; sqrt and cbrt have
        // derivative 0 at 0)
        const real P0 = acc.val(i, j, 1), Q0 = acc.val(i, j, 2);
        const real hb = acc.val(i, j, 0) - Bb;
        const bool hpos = hb >= real(0);
        const real hp = hpos ? hb : real(0);
        const real hinv = desing(hp, A.c.eps);
        const bool man = A.phy.friction == kFricManning;
        const real cr = man ? cel::cbrt_r(hinv) : real(1);
        const real fc = man ? A.c.fric * cr : A.c.fric;
        const real dfc = man && hinv > real(0) ? A.c.fric / (real(3) * cr * cr) : real(0);
        const real mag = sqrt(P0 * P0 + Q0 * Q0);
        const real Aq = lF * P0 + lG * Q0;
        const real k2 = hinv * hinv;
        dfw = hpos ? -mag * Aq * (dfc * k2 + real(2) * fc * hinv) * desing_dh(hp, A.c.eps) : real(0);
        const real um = mag > real(0) ? Aq / mag : real(0);
        dw += dfw;
        dP = -fc * k2 * (P0 * um + mag * lF);
        dQ = -fc * k2 * (Q0 * um + mag * lG);
    }
    if (A.lBc) {   // the bed: Bbar through h = w - Bbar, the face beds through the slope
        const real hb = acc.val(i, j, 0) - Bb;
        A.lBb[ring_index(G, i, j)] += g * (BxE - BxW) * A.c.rdx * lF + g * (ByN - ByS) * A.c.rdy * lG - dfw;
        const real lBxE = -(g * hb * A.c.rdx) * lF, lByN = -(g * hb * A.c.rdy) * lG;
        // BxW = (c00 + c01) / 2, BxE = (c10 + c11) / 2, ByS = (c00 + c10) / 2, ByN = (c01 + c11) / 2
        acc.corner(i, j, real(0.5) * (-lBxE - lByN));
        acc.corner(i + 1, j, real(0.5) * (lBxE - lByN));
        acc.corner(i, j + 1, real(0.5) * (-lBxE + lByN));
        acc.corner(i + 1, j + 1, real(0.5) * (lBxE + lByN));
    }
    acc.cell(0, i, j, dw);
    acc.cell(1, i, j, dP);
    acc.cell(2, i, j, dQ);
}

// The face fluxes' Jacobians transposed.  dir 0: x-face f of row `line`;
// dir 1: y-face f of column `line`.
template <typename real, typename Acc>
__device__ __forceinline__ void face_vjp(const AdjArgs<real> &A, int dir, int f, int line, const Acc &acc)
{
    const Geo &G = A.geo;
    const int n = dir == 0 ? G.nx : G.ny;
    auto cell = [&](int c) { return dir == 0 ? line * G.nx + c : c * G.nx + line; };
    // H enters R of the cell after the face with +1/h and the cell before with -1/h
    const real rh = dir == 0 ? A.c.rdx : A.c.rdy;
    real lR[3];
#pragma unroll
    for (int v = 0; v < 3; v++)
        lR[v] = ((f < n ? A.G0[v][cell(f)] : real(0)) - (f > 0 ? A.G0[v][cell(f - 1)] : real(0))) * rh;
    // flux components: mass, normal and tangential momentum
    const real lH[3] = {lR[0], dir == 0 ? lR[1] : lR[2], dir == 0 ? lR[2] : lR[1]};
    if (lH[0] == real(0) && lH[1] == real(0) && lH[2] == real(0)) return;
    // the values now, the mappings after the reverse (fewer live registers)
    auto at = [&](int c, int &i, int &j) {
        i = dir == 0 ? f - 2 + c : line;
        j = dir == 0 ? line : f - 2 + c;
    };
    auto face_bed = [&](int q) {   // bed of face q (dir 0: x-face q of row line)
        return dir == 0 ? real(0.5) * (acc.bed(q, line) + acc.bed(q, line + 1))
                        : real(0.5) * (acc.bed(line, q) + acc.bed(line + 1, q));
    };
    const real Bm = face_bed(f - 1), Bf = face_bed(f), Bp = face_bed(f + 1);
    real w[4], P[4], Q[4], lw[4] = {0, 0, 0, 0}, lP[4] = {0, 0, 0, 0}, lQ[4] = {0, 0, 0, 0}, lB[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < 4; q++) {
        int i, j;
        at(q, i, j);
        w[q] = acc.val(i, j, 0);
        P[q] = acc.val(i, j, 1);
        Q[q] = acc.val(i, j, 2);
    }
    face_flux_vjp(w, P, Q, Bm, Bf, Bp, A.c.theta, A.c.g, A.c.eps, dir, lH, lw, lP, lQ, lB);
#pragma unroll
    for (int c = 0; c < 4; c++) {
        int i, j;
        at(c, i, j);
        const Src<real> s = acc.map(i, j);
        if (s.idx < 0) {   // a sine-maker ghost: its values' adjoints, for the depth they follow
            acc.ghost(s, 0, lw[c]);
            acc.ghost(s, 1, lP[c]);
            acc.ghost(s, 2, lQ[c]);
            continue;
        }
        acc.cell(0, s.ci, s.cj, lw[c]);
        acc.cell(1, s.ci, s.cj, s.sgn[1] * lP[c]);
        acc.cell(2, s.ci, s.cj, s.sgn[2] * lQ[c]);
    }
    if (A.lBc) {   // the three face beds, each the mean of its two corners
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const real gsum = real(0.5) * lB[b];
            const int q = f - 1 + b;
            if (dir == 0) {
                acc.corner(q, line, gsum);
                acc.corner(q, line + 1, gsum);
            } else {
                acc.corner(line, q, gsum);
                acc.corner(line + 1, q, gsum);
            }
        }
    }
}

// Self-check of the hand-written flux VJP against the dual numbers: per
// face 22 inputs (w[4], P[4], Q[4], Bm, Bf, Bp, lH[3], theta, g, eps, dir)
// and 30 outputs (the 15 adjoints by dual numbers, then by hand).
template <typename real>
__global__ void k_face_vjp_check(const real *in, int n, real *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const real *x = in + (size_t)k * 22;
    real *o = out + (size_t)k * 30;
    const int dir = x[21] != real(0) ? 1 : 0;
    face_flux_vjp_dual(x, x + 4, x + 8, x[12], x[13], x[14], x[18], x[19], x[20], dir, x + 15, o);
    real lw[4] = {0, 0, 0, 0}, lP[4] = {0, 0, 0, 0}, lQ[4] = {0, 0, 0, 0}, lB[3] = {0, 0, 0};
    face_flux_vjp(x, x + 4, x + 8, x[12], x[13], x[14], x[18], x[19], x[20], dir, x + 15, lw, lP, lQ, lB);
    for (int q = 0; q < 4; q++) {
        o[15 + q] = lw[q];
        o[19 + q] = lP[q];
        o[23 + q] = lQ[q];
    }
    for (int b = 0; b < 3; b++) o[27 + b] = lB[b];
}

// Eq. 10-13 transposed: the dispersive eta terms of F and G and the mixed
// terms F*(Q), G*(P) are linear in the neighbouring eta, Q and P, with
// coefficients from the still-water depth; each cell adds its adjoints to
// the cells (or the cells their ghosts mirror) its stencil reads.
template <typename real, typename Acc>
__device__ __forceinline__ void disp_vjp(const AdjArgs<real> &A, int i, int j, const Acc &acc)
{
    const Geo &G = A.geo;
    const int k = j * G.nx + i;
    const real lF = A.G0[1][k], lG = A.G0[2][k], lFs = A.G0[3][k], lGs = A.G0[4][k];
    if (lF == real(0) && lG == real(0) && lFs == real(0) && lGs == real(0)) return;
    const Coef<real> &C = A.c;
    auto dcell = [&](int ii, int jj) { return fmax(C.ws - acc.bbar(ii, jj), real(0)); };
    const real dd = dcell(i, j);
    const real ddx = (dcell(i + 1, j) - dcell(i - 1, j)) * C.hrdx, ddy = (dcell(i, j + 1) - dcell(i, j - 1)) * C.hrdy;
    const real K3 = C.Bd * C.g * dd * dd * dd, K2 = C.Bd * C.g * dd * dd;
    // d F / d eta_p and d G / d eta_p over the 13 points, through exx, eyy,
    // exy, exxx, eyyy, exyy, exxy
    const real fxx = K2 * ddx * real(2) * lF + K2 * ddy * lG;          // weight of exx
    const real fyy = K2 * ddx * lF + K2 * ddy * real(2) * lG;          // eyy
    const real fxy = K2 * ddy * lF + K2 * ddx * lG;                    // exy
    const real fxxx = K3 * lF, fyyy = K3 * lG, fxyy = K3 * lF, fxxy = K3 * lG;
    const real ax = fxx * C.rdx2, ay = fyy * C.rdy2, axy = fxy * C.rdxdy4;
    const real a3x = fxxx * C.rdx3h, a3y = fyyy * C.rdy3h, bxyy = fxyy * C.rdxdy2h, bxxy = fxxy * C.rdx2dyh;
    struct Pt { int di, dj; real wgt; };
    const Pt pts[13] = {
        {0, 0, -real(2) * ax - real(2) * ay},
        {1, 0, ax - real(2) * a3x - real(2) * bxyy},
        {-1, 0, ax + real(2) * a3x + real(2) * bxyy},
        {0, 1, ay - real(2) * a3y - real(2) * bxxy},
        {0, -1, ay + real(2) * a3y + real(2) * bxxy},
        {2, 0, a3x},
        {-2, 0, -a3x},
        {0, 2, a3y},
        {0, -2, -a3y},
        {1, 1, axy + bxyy + bxxy},
        {-1, 1, -axy - bxyy + bxxy},
        {1, -1, -axy + bxyy - bxxy},
        {-1, -1, axy - bxyy - bxxy}};
#pragma unroll
    for (int q = 0; q < 13; q++) {
        if (pts[q].wgt == real(0)) continue;
        const Src<real> s = acc.map(i + pts[q].di, j + pts[q].dj);
        if (s.idx >= 0) acc.cell(0, s.ci, s.cj, pts[q].wgt);
        else acc.ghost(s, 0, pts[q].wgt);
    }
    // F* = d ddx Qy / 6 + d ddy Qx / 6 + B3 d^2 Qxy; G* the same in P with x, y exchanged
    const real qx = dd * ddy * C.sixth * C.hrdx, qy = dd * ddx * C.sixth * C.hrdy, qxy = C.B3 * dd * dd * C.rdxdy4;
    const real px = dd * ddy * C.sixth * C.hrdx, py = dd * ddx * C.sixth * C.hrdy;
    // Gs = dd ddy Px / 6 + dd ddx Py / 6 + B3 dd^2 Pxy, Fs = dd ddx Qy / 6 + dd ddy Qx / 6 + B3 dd^2 Qxy
    const Pt mq[8] = {{1, 0, qx * lFs}, {-1, 0, -qx * lFs}, {0, 1, qy * lFs}, {0, -1, -qy * lFs},
                      {1, 1, qxy * lFs}, {1, -1, -qxy * lFs}, {-1, 1, -qxy * lFs}, {-1, -1, qxy * lFs}};
    const Pt mp[8] = {{1, 0, px * lGs}, {-1, 0, -px * lGs}, {0, 1, py * lGs}, {0, -1, -py * lGs},
                      {1, 1, qxy * lGs}, {1, -1, -qxy * lGs}, {-1, 1, -qxy * lGs}, {-1, -1, qxy * lGs}};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const Src<real> s = acc.map(i + mq[q].di, j + mq[q].dj);
        if (s.idx >= 0) acc.cell(2, s.ci, s.cj, s.sgn[2] * mq[q].wgt);
        else acc.ghost(s, 2, mq[q].wgt);
        const Src<real> t = acc.map(i + mp[q].di, j + mp[q].dj);
        if (t.idx >= 0) acc.cell(1, t.ci, t.cj, t.sgn[1] * mp[q].wgt);
        else acc.ghost(t, 1, mp[q].wgt);
    }
    if (!A.ld) return;
    // the same terms with respect to d at the cell (dd) and its 4 neighbours
    // (through ddx, ddy), at the forward's eta, P and Q (ghosts included)
    auto val = [&](int di, int dj, int v) { return acc.val(i + di, j + dj, v); };
    const real e00 = val(0, 0, 0), eE = val(1, 0, 0), eW = val(-1, 0, 0), eN = val(0, 1, 0), eS = val(0, -1, 0);
    const real eNE = val(1, 1, 0), eNW = val(-1, 1, 0), eSE = val(1, -1, 0), eSW = val(-1, -1, 0);
    const real exx = (eE - real(2) * e00 + eW) * C.rdx2;
    const real eyy = (eN - real(2) * e00 + eS) * C.rdy2;
    const real exy = (eNE - eSE - eNW + eSW) * C.rdxdy4;
    const real exxx = (val(2, 0, 0) - real(2) * eE + real(2) * eW - val(-2, 0, 0)) * C.rdx3h;
    const real eyyy = (val(0, 2, 0) - real(2) * eN + real(2) * eS - val(0, -2, 0)) * C.rdy3h;
    const real exyy = ((eNE - real(2) * eE + eSE) - (eNW - real(2) * eW + eSW)) * C.rdxdy2h;
    const real exxy = ((eNE - real(2) * eN + eNW) - (eSE - real(2) * eS + eSW)) * C.rdx2dyh;
    const real Qx = (val(1, 0, 2) - val(-1, 0, 2)) * C.hrdx, Qy = (val(0, 1, 2) - val(0, -1, 2)) * C.hrdy;
    const real Qxy = (val(1, 1, 2) - val(1, -1, 2) - val(-1, 1, 2) + val(-1, -1, 2)) * C.rdxdy4;
    const real Px = (val(1, 0, 1) - val(-1, 0, 1)) * C.hrdx, Py = (val(0, 1, 1) - val(0, -1, 1)) * C.hrdy;
    const real Pxy = (val(1, 1, 1) - val(1, -1, 1) - val(-1, 1, 1) + val(-1, -1, 1)) * C.rdxdy4;
    const real Bg = C.Bd * C.g;
    // F = Bg d^3 (exxx + exyy) + Bg d^2 (ddx (2 exx + eyy) + ddy exy), G likewise,
    // Fs = d ddx Qy / 6 + d ddy Qx / 6 + B3 d^2 Qxy, Gs = d ddy Px / 6 + d ddx Py / 6 + B3 d^2 Pxy
    const real Ld = lF * (real(3) * Bg * dd * dd * (exxx + exyy) + real(2) * Bg * dd * (ddx * (real(2) * exx + eyy) + ddy * exy)) +
                    lG * (real(3) * Bg * dd * dd * (eyyy + exxy) + real(2) * Bg * dd * (ddy * (real(2) * eyy + exx) + ddx * exy)) +
                    lFs * (ddx * Qy * C.sixth + ddy * Qx * C.sixth + real(2) * C.B3 * dd * Qxy) +
                    lGs * (ddy * Px * C.sixth + ddx * Py * C.sixth + real(2) * C.B3 * dd * Pxy);
    const real Ldx = (lF * Bg * dd * dd * (real(2) * exx + eyy) + lG * Bg * dd * dd * exy + lFs * dd * Qy * C.sixth +
                      lGs * dd * Py * C.sixth) * C.hrdx;
    const real Ldy = (lF * Bg * dd * dd * exy + lG * Bg * dd * dd * (real(2) * eyy + exx) + lFs * dd * Qx * C.sixth +
                      lGs * dd * Px * C.sixth) * C.hrdy;
    acc.ring(i, j, Ld);
    acc.ring(i + 1, j, Ldx);
    acc.ring(i - 1, j, -Ldx);
    acc.ring(i, j + 1, Ldy);
    acc.ring(i, j - 1, -Ldy);
}

// The right sides' Jacobians transposed over one tile of 32 columns and TY
// rows: the cells' bed slope, friction and dispersive terms, the x-faces of
// the tile's rows and the y-faces of its columns (the east and north boundary
// faces with the last tiles).  Their adjoints reach cells up to 2 beyond the
// tile (ghosts mapped to the cells they mirror), depths 1 beyond and corners
// 2 beyond; they are summed in shared memory over that window and added to
// global memory once per window element.
constexpr int kVT = 32;              // tile width
constexpr int kVW = kVT + 4;         // cell window: x0 - 2 .. x0 + 33
constexpr int kVWS = kVW + 1;
constexpr int kVC = kVT + 5;         // corner window: x0 - 2 .. x0 + 34
constexpr int kVCS = kVC + 1;
constexpr int kVjpThreads = 256;

// The accumulator's pointers and tile position.
template <typename real>
struct TileData {
    real *sv[3], *sd, *sc;   // shared windows: lw, lP, lQ, ld, lBc
    real *gv[3], *gd, *gc;   // global arrays
    const real *xv[3], *xb;  // shared windows: the state as source2d gives it, the bed corners
    const Geo *G;
    int sine;
    int interior;            // the whole cell window lies inside the grid: no ghosts
    real *lg;                // ghost adjoints (NULL: not wanted)
    int tsel, npos;
    int x0, y0, nx, pc;
};

// kInt: a tile whose window lies inside the grid, where every source is the
// cell itself and every target lies in the shared windows (no mapping, no
// bounds checks, no global fallback).
template <typename real, int TY, bool kInt>
struct TileAcc : TileData<real> {
    using D = TileData<real>;
    static constexpr int kWH = TY + 4;   // cell window rows: y0 - 2 .. y0 + TY + 1
    static constexpr int kCH = TY + 5;   // corner window rows
    __device__ __forceinline__ void ghost(const Src<real> &s, int var, real v) const
    {
        if (D::lg && v != real(0)) atomicAdd(D::lg + ghost_index(D::tsel, s.gs, s.gl, var, s.gp, D::npos), v);
    }
    __device__ __forceinline__ real val(int i, int j, int v) const
    {
        return D::xv[v][(j - D::y0 + 2) * kVWS + (i - D::x0 + 2)];
    }
    // where the adjoint of window cell (i, j) goes: the cell it is or
    // mirrors, with the signs, or a sine-maker ghost (no values)
    __device__ __forceinline__ Src<real> map(int i, int j) const
    {
        Src<real> s;
        if (kInt || D::interior) {
            s.sgn[0] = s.sgn[1] = s.sgn[2] = real(1);
            s.ci = i;
            s.cj = j;
            s.idx = 0;   // a cell (its index is not needed here)
        } else {
            mirror2d(*D::G, D::sine, i, j, s);
        }
        return s;
    }
    __device__ __forceinline__ real bed(int ci, int cj) const
    {
        return D::xb[(cj - D::y0 + 2) * kVCS + (ci - D::x0 + 2)];
    }
    __device__ __forceinline__ real bbar(int i, int j) const
    {
        return cell_bbar(bed(i, j), bed(i + 1, j), bed(i, j + 1), bed(i + 1, j + 1));
    }
    __device__ __forceinline__ void cell(int var, int i, int j, real v) const
    {
        if (v == real(0)) return;
        const int li = i - D::x0 + 2, lj = j - D::y0 + 2;
        if (kInt || (li >= 0 && li < kVW && lj >= 0 && lj < kWH)) atomicAdd(D::sv[var] + lj * kVWS + li, v);
        else atomicAdd(D::gv[var] + (size_t)j * D::nx + i, v);
    }
    __device__ __forceinline__ void ring(int i, int j, real v) const
    {
        if (v == real(0)) return;
        const int li = i - D::x0 + 2, lj = j - D::y0 + 2;
        if (kInt || (li >= 0 && li < kVW && lj >= 0 && lj < kWH)) atomicAdd(D::sd + lj * kVWS + li, v);
        else atomicAdd(D::gd + (size_t)(j + 1) * (D::nx + 2) + (i + 1), v);
    }
    __device__ __forceinline__ void corner(int ci, int cj, real v) const
    {
        if (v == real(0)) return;
        const int li = ci - D::x0 + 2, lj = cj - D::y0 + 2;
        if (kInt || (li >= 0 && li < kVC && lj >= 0 && lj < kCH)) atomicAdd(D::sc + lj * kVCS + li, v);
        else atomicAdd(D::gc + (size_t)(cj + 1) * D::pc + (ci + 1), v);
    }
};

// The tile's cells and faces.
template <typename real, int TY, bool kInt>
__device__ __forceinline__ void vjp_tile_work(const AdjArgs<real> &A, const TileData<real> &td, int tx, int ty)
{
    TileAcc<real, TY, kInt> acc;
    static_cast<TileData<real> &>(acc) = td;
    const Geo &G = A.geo;
    const int x0 = td.x0, y0 = td.y0;
    const int xe = min(x0 + kVT, G.nx), ye = min(y0 + TY, G.ny);
    for (int j = y0 + ty; j < ye; j += kVjpThreads / 32) {
        const int i = x0 + tx;
        if (i < xe) {
            cell_vjp(A, i, j, acc);
            if (A.bsnq) disp_vjp(A, i, j, acc);
        }
    }
    const int fe = xe + (xe == G.nx ? 1 : 0);
    for (int j = y0 + ty; j < ye; j += kVjpThreads / 32)
        for (int f = x0 + tx; f < fe; f += 32) face_vjp(A, 0, f, j, acc);
    const int ge = ye + (ye == G.ny ? 1 : 0);
    for (int gq = y0 + ty; gq < ge; gq += kVjpThreads / 32) {
        const int i = x0 + tx;
        if (i < xe) face_vjp(A, 1, gq, i, acc);
    }
}

template <typename real, int TY>
constexpr size_t vjp_smem_bytes()
{
    return sizeof(real) * (size_t)(7 * (TY + 4) * kVWS + 2 * (TY + 5) * kVCS);
}

template <typename real, int TY>
__global__ void __launch_bounds__(kVjpThreads, sizeof(real) == 4 ? 4 : 2) k_adj_vjp(const __grid_constant__ AdjArgs<real> A)
{
    dependent_launch_wait_then_release();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    real *sm = reinterpret_cast<real *>(smem_raw);
    const Geo &G = A.geo;
    constexpr int kWH = TY + 4, kCH = TY + 5;
    const int x0 = blockIdx.x * kVT, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    constexpr int ntot = 4 * kWH * kVWS + kCH * kVCS;
    for (int k = tid; k < ntot; k += kVjpThreads) sm[k] = real(0);
    TileData<real> acc;
    for (int v = 0; v < 3; v++) acc.sv[v] = sm + v * kWH * kVWS;
    acc.sd = sm + 3 * kWH * kVWS;
    acc.sc = sm + 4 * kWH * kVWS;
    real *xs = sm + ntot;
    for (int v = 0; v < 3; v++) acc.xv[v] = xs + v * kWH * kVWS;
    real *xb = xs + 3 * kWH * kVWS;
    acc.xb = xb;
    acc.G = &G;
    acc.sine = A.c.sine;
    acc.interior = x0 >= 2 && y0 >= 2 && x0 + kVW - 2 <= G.nx && y0 + kWH - 2 <= G.ny;
    acc.lg = A.lg;
    acc.tsel = A.tsel;
    acc.npos = A.c.npos;
    // the state with its ghosts (source2d) on cells within 2 of the grid,
    // and the bed corners, over the windows
    for (int k = tid; k < kVW * kWH; k += kVjpThreads) {
        const int li = k % kVW, lj = k / kVW, i = x0 - 2 + li, j = y0 - 2 + lj, o = lj * kVWS + li;
        if (i >= -2 && i <= G.nx + 1 && j >= -2 && j <= G.ny + 1) {
            const Src<real> q = source2d(A, i, j);
            for (int v = 0; v < 3; v++) xs[v * kWH * kVWS + o] = q.v[v];
        }
    }
    for (int k = tid; k < kVC * kCH; k += kVjpThreads) {
        const int li = k % kVC, lj = k / kVC, ci = x0 - 2 + li, cj = y0 - 2 + lj;
        if (ci >= -1 && ci <= G.nx + 1 && cj >= -1 && cj <= G.ny + 1) xb[lj * kVCS + li] = corner(A.Bc, G, ci, cj);
    }
    acc.gv[0] = A.lw;
    acc.gv[1] = A.lP;
    acc.gv[2] = A.lQ;
    acc.gd = A.ld;
    acc.gc = A.lBc;
    acc.x0 = x0;
    acc.y0 = y0;
    acc.nx = G.nx;
    acc.pc = G.pc;
    __syncthreads();
    if (acc.interior) vjp_tile_work<real, TY, true>(A, acc, tx, ty);
    else vjp_tile_work<real, TY, false>(A, acc, tx, ty);
    __syncthreads();
    for (int k = tid; k < kVW * kWH; k += kVjpThreads) {
        const int li = k % kVW, lj = k / kVW, i = x0 - 2 + li, j = y0 - 2 + lj, o = lj * kVWS + li;
        if (i >= 0 && i < G.nx && j >= 0 && j < G.ny) {
            const size_t c = (size_t)j * G.nx + i;
            for (int v = 0; v < 3; v++)
                if (acc.sv[v][o] != real(0)) atomicAdd(acc.gv[v] + c, acc.sv[v][o]);
        }
        if (A.ld && i >= -1 && i <= G.nx && j >= -1 && j <= G.ny && acc.sd[o] != real(0))
            atomicAdd(A.ld + ring_index(G, i, j), acc.sd[o]);
    }
    if (A.lBc)
        for (int k = tid; k < kVC * kCH; k += kVjpThreads) {
            const int li = k % kVC, lj = k / kVC, ci = x0 - 2 + li, cj = y0 - 2 + lj;
            const real v = acc.sc[lj * kVCS + li];
            if (v != real(0) && ci >= -1 && ci <= G.nx + 1 && cj >= -1 && cj <= G.ny + 1)
                atomicAdd(A.lBc + corner_index(G, ci, cj), v);
        }
}

// Eq. 23's rows depend on d: a_k = s_k - r_k, b_k = 1 + 2 r_k, c_k = -s_k - r_k
// with r_k = B3 d_k^2 / h^2, s_k = d_k (d_{k+1} - d_{k-1}) / (12 h^2) (the
// ends mirrored, d_{-1} = d_0, d_n = d_{n-1}).  T x = r gives dL/dT_kl =
// -mu_k x_l with mu = T^-T (adjoint of x); a wall's boundary row folds a_0
// into b_0 (x_{-1} = -x_0), a sine maker's moves a_0 times the ghost
// increment to the right side (x_{-1} = that increment).  One thread per
// line element gathers the terms of rows k-1, k, k+1 that hold its d; all
// arrays in the line layout (x-rows [ny][px], y-columns [nx][py]), so both
// families read along their lines.  blockIdx.z: the family.
// Eq. 23's constants 1/h^2, 1/(2h), 1/(6h) of one family, rounded once on
// the host from the double spacing, as the forward's line solver gets them.
template <typename real>
struct LineConst {
    real rh2[2], hrh[2], srh[2];
};

template <typename real>
__global__ void k_adj_tri_bed(AdjArgs<real> A, const real *X, const real *Yc, const real *MUx, const real *MUy,
                              const real *dr, const real *dc, LineConst<real> K)
{
    dependent_launch_wait_then_release();
    const Geo &G = A.geo;
    const int dir = blockIdx.z;
    const int n = dir == 0 ? G.nx : G.ny, nl = dir == 0 ? G.ny : G.nx;
    const int e = blockIdx.x * blockDim.x + threadIdx.x, line = blockIdx.y;
    if (e >= n || line >= nl) return;
    const size_t base = (size_t)line * (dir == 0 ? G.px : G.py);
    const real *x = (dir == 0 ? X : Yc) + base, *mu = (dir == 0 ? MUx : MUy) + base, *d = (dir == 0 ? dr : dc) + base;
    const int lo_side = dir == 0 ? 0 : 2, hi_side = dir == 0 ? 1 : 3, gvar = dir == 0 ? 1 : 2;
    auto ghost_inc = [&](int side) {
        return A.ghost[ghost_index(1, side, 0, gvar, line + 2, A.c.npos)] -
               A.ghost[ghost_index(0, side, 0, gvar, line + 2, A.c.npos)];
    };
    const bool lo_sine = (A.c.sine >> lo_side) & 1, hi_sine = (A.c.sine >> hi_side) & 1;
    const real xlo = lo_sine ? ghost_inc(lo_side) : -x[0];
    const real xhi = hi_sine ? ghost_inc(hi_side) : -x[n - 1];
    // row k's adjoints of r_k and s_k
    auto row = [&](int k, real &Lr, real &Ls) {
        const real m = mu[k], xk = x[k];
        const real xm = k > 0 ? x[k - 1] : xlo, xp = k < n - 1 ? x[k + 1] : xhi;
        const real gA = -m * xm, gB = -m * xk, gC = -m * xp;
        Lr = -gA + real(2) * gB - gC;
        Ls = gA - gC;
    };
    const real rh2 = K.rh2[dir], hrh = K.hrh[dir], srh = K.srh[dir];
    const real sh = srh * hrh;
    real Lr, Ls;
    row(e, Lr, Ls);
    const real de = d[e], dm = d[e > 0 ? e - 1 : 0], dp = d[e < n - 1 ? e + 1 : n - 1];
    real ld = Lr * real(2) * A.c.B3 * de * rh2 + Ls * (dp - dm) * hrh * srh;
    if (e == n - 1) ld += Ls * de * sh;   // d_n = d_{n-1}
    if (e == 0) ld -= Ls * de * sh;       // d_{-1} = d_0
    real L2r, L2s;
    if (e >= 1) {   // row e-1 reads d_e as its d_{k+1}
        row(e - 1, L2r, L2s);
        ld += L2s * d[e - 1] * sh;
    }
    if (e <= n - 2) {   // row e+1 reads d_e as its d_{k-1}
        row(e + 1, L2r, L2s);
        ld -= L2s * d[e + 1] * sh;
    }
    (dir == 0 ? A.ldx : A.ldy)[base + e] += ld;
    // a maker's row: r_0 - a_0 (g^{n+1} - g^n) (and the last row with c), so
    // the ghost increments' adjoints are -+ mu a_0
    if (A.lg && ((e == 0 && lo_sine) || (e == n - 1 && hi_sine))) {
        const bool lo = e == 0 && lo_sine;
        const int side = lo ? lo_side : hi_side;
        const real r = A.c.B3 * de * de * rh2, sk = de * (dp - dm) * hrh * srh;
        const real coef = lo ? sk - r : -sk - r;
        const real gi = -mu[e] * coef;
        atomicAdd(A.lg + ghost_index(1, side, 0, gvar, line + 2, A.c.npos), gi);
        atomicAdd(A.lg + ghost_index(0, side, 0, gvar, line + 2, A.c.npos), -gi);
        if (n == 1 && lo_sine && hi_sine) {   // one row carries both ends
            const real gh = -mu[e] * (-sk - r);
            atomicAdd(A.lg + ghost_index(1, hi_side, 0, gvar, line + 2, A.c.npos), gh);
            atomicAdd(A.lg + ghost_index(0, hi_side, 0, gvar, line + 2, A.c.npos), -gh);
        }
    }
}

// The ghost values of one table entry (Eq. 25-28: eta, P, Q summed over the
// components, Eckart wave number k = k0 / sqrt(tanh(k0 d)), celerity w / k)
// differentiated with respect to the adjacent depth d, in double:
// dk/dd = -k0^2 / (2 sqrt(coth(k0 d)) sinh^2(k0 d)), d(a sin th)/dk =
// -a cos th (x cos + y sin), dc/dk = -c / k.  Their adjoints (lg) go to ld
// of the cell whose depth the entry reads; lg is zeroed.
template <typename real>
__global__ void k_adj_ghost_bed(AdjArgs<real> A, Bnd b, const double *ktab, const real *d_r, double t0, double t1)
{
    dependent_launch_wait_then_release();
    const int pos = blockIdx.x * blockDim.x + threadIdx.x, yb = blockIdx.y;
    const int time = yb & 1, layer = (yb >> 1) & 1, side = yb >> 2;
    const int npos = A.c.npos;
    if (pos >= npos || !((A.c.sine >> side) & 1)) return;
    real *l0 = A.lg + ghost_index(time, side, layer, 0, pos, npos);
    const double le = (double)l0[0], lP = (double)l0[npos], lQ = (double)l0[2 * npos];
    l0[0] = l0[npos] = l0[2 * npos] = real(0);
    double x, y, dadj;
    if (!ghost_site(A.geo, d_r, side, layer, pos, x, y, dadj)) return;
    if ((le == 0.0 && lP == 0.0 && lQ == 0.0) || !(dadj > 0.0)) return;
    const Side &S = b.s[side];
    const double t = time ? t1 : t0, g = (double)A.phy.g;
    double dd = 0.0;
    for (int m = 0; m < S.ncomp; m++) {
        const double k = ktab[((size_t)side * npos + pos) * 8 + m];
        if (!(k > 0.0)) continue;
        const double om = S.omega[m], k0 = om * om / g, kd = k0 * dadj;
        const double sh = sinh(kd);
        const double dkdd = -k0 * k0 / (2.0 * sqrt(1.0 / tanh(kd)) * sh * sh);
        const double arg = om * t - k * S.cdir[m] * x - k * S.sdir[m] * y + S.phase[m];
        const double em = S.amp[m] * sin(arg), demdk = -S.amp[m] * cos(arg) * (S.cdir[m] * x + S.sdir[m] * y);
        const double c = om / k, dcdk = -c / k;
        const double dPdk = S.cdir[m] * (dcdk * em + c * demdk), dQdk = S.sdir[m] * (dcdk * em + c * demdk);
        dd += (le * demdk + lP * dPdk + lQ * dQdk) * dkdd;
    }
    int i, j;
    ghost_adjacent(A.geo, side, pos, i, j);
    atomicAdd(A.ld + ring_index(A.geo, i, j), real(dd));
}

// ld into lBb (d = max(w_s - Bbar, 0)), the initial clamp, and lBb into the
// 4 corners of each cell (ring included).
template <typename real>
__global__ void k_adj_bed_cells(AdjArgs<real> A, const real *w0, const real *lw0)
{
    const Geo &G = A.geo;
    const int i = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1, j = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
    if (i > G.nx || j > G.ny) return;
    const size_t r = ring_index(G, i, j);
    const real Bb = bbar_at(A.Bc, G, i, j);
    real lb = A.lBb[r];
    const bool inside = i >= 0 && i < G.nx && j >= 0 && j < G.ny;
    if (A.c.ws - Bb > real(0)) {
        real ld = A.ld[r];
        if (inside && A.ldx) ld += A.ldx[(size_t)j * G.px + i] + A.ldy[(size_t)i * G.py + j];
        lb -= ld;
    }
    if (inside) {
        const size_t k = (size_t)j * G.nx + i;
        if (w0[k] - Bb <= real(0)) lb += lw0[k];   // w0 = max(w_in, Bbar) follows the bed on dry cells
    }
    if (lb == real(0)) return;
    lb *= real(0.25);
    atomicAdd(A.lBc + corner_index(G, i, j), lb);
    atomicAdd(A.lBc + corner_index(G, i + 1, j), lb);
    atomicAdd(A.lBc + corner_index(G, i, j + 1), lb);
    atomicAdd(A.lBc + corner_index(G, i + 1, j + 1), lb);
}

// Corner (ci, cj) = mean of the cell-centre beds around it, mirrored evenly
// beyond the grid: its adjoint goes to those 4 cells.
template <typename real>
__global__ void k_adj_bed_z(AdjArgs<real> A, real *grad_z)
{
    const Geo &G = A.geo;
    const int ci = (int)(blockIdx.x * blockDim.x + threadIdx.x) - 1, cj = (int)(blockIdx.y * blockDim.y + threadIdx.y) - 1;
    if (ci > G.nx + 1 || cj > G.ny + 1) return;
    const real v = real(0.25) * A.lBc[corner_index(G, ci, cj)];
    if (v == real(0)) return;
    const int i0 = mirror_index(ci - 1, G.nx), i1 = mirror_index(ci, G.nx);
    const int j0 = mirror_index(cj - 1, G.ny), j1 = mirror_index(cj, G.ny);
    atomicAdd(grad_z + (size_t)j0 * G.nx + i0, v);
    atomicAdd(grad_z + (size_t)j0 * G.nx + i1, v);
    atomicAdd(grad_z + (size_t)j1 * G.nx + i0, v);
    atomicAdd(grad_z + (size_t)j1 * G.nx + i1, v);
}

// The misfit at the gauges after step n enters the adjoint of w^n.
template <typename real>
__global__ void k_adj_misfit(AdjArgs<real> A, const int32_t *gij, int ng, const real *rec, const real *obs)
{
    dependent_launch_wait_then_release();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    atomicAdd(A.lw + gij[2 * k + 1] * A.geo.nx + gij[2 * k], rec[k] - obs[k]);
}

}  // namespace

template <typename real>
cudaError_t launch_adjoint_mask(const AdjArgs<real> &a, cudaStream_t st)
{
    dim3 b(32, 32), g((a.geo.nx + 31) / 32, (a.geo.ny + 31) / 32);
    cudaError_t e = launch_step_kernel(k_adj_mask<real>, g, b, 0, st, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_hist(const AdjArgs<real> &a, cudaStream_t st)
{
    dim3 b(32, 32), g((a.geo.nx + 31) / 32, (a.geo.ny + 31) / 32);
    cudaError_t e = launch_step_kernel(k_adj_hist<real>, g, b, 0, st, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename real, int TY>
cudaError_t launch_vjp_rows(const AdjArgs<real> &a, cudaStream_t st)
{
    constexpr size_t smem = vjp_smem_bytes<real, TY>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(k_adj_vjp<real, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dim3 g((a.geo.nx + kVT - 1) / kVT, (a.geo.ny + TY - 1) / TY);
    cudaError_t e = launch_step_kernel(k_adj_vjp<real, TY>, g, dim3(kVjpThreads), smem, st, a);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Tile rows of the Jacobian kernel: 32 while 32 x 32 tiles give every SM
// several blocks, else 16 or 8, so that small grids still fill the GPU.
static int vjp_tile_rows(int nx, int ny)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 1;
    }
    const long cols = (nx + kVT - 1) / kVT, want = 4L * nsm;
    if (cols * ((ny + 31) / 32) >= want) return 32;
    if (cols * ((ny + 15) / 16) >= want) return 16;
    return 8;
}

template <typename real>
cudaError_t launch_adjoint_vjp(const AdjArgs<real> &a, cudaStream_t st)
{
    switch (vjp_tile_rows(a.geo.nx, a.geo.ny)) {
    case 32: return launch_vjp_rows<real, 32>(a, st);
    case 16: return launch_vjp_rows<real, 16>(a, st);
    default: return launch_vjp_rows<real, 8>(a, st);
    }
}

template <typename real>
cudaError_t launch_face_vjp_check(const real *in, int n, real *out, cudaStream_t st)
{
    k_face_vjp_check<real><<<(n + 127) / 128, 128, 0, st>>>(in, n, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_tri_bed(const AdjArgs<real> &a, const real *X, const real *Yc, const real *MUx,
                                   const real *MUy, const real *dr, const real *dc, cudaStream_t st)
{
    const int n = a.geo.nx > a.geo.ny ? a.geo.nx : a.geo.ny, nl = a.geo.nx > a.geo.ny ? a.geo.nx : a.geo.ny;
    LineConst<real> K;
    for (int d = 0; d < 2; d++) {
        const double h = d == 0 ? a.geo.dx : a.geo.dy;
        K.rh2[d] = real(1.0 / (h * h));
        K.hrh[d] = real(0.5 / h);
        K.srh[d] = real(1.0 / (6.0 * h));
    }
    cudaError_t e = launch_step_kernel(k_adj_tri_bed<real>, dim3((n + 127) / 128, nl, 2), dim3(128), 0, st, a, X, Yc,
                                       MUx, MUy, dr, dc, K);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_ghost_bed(const AdjArgs<real> &a, const Bnd &b, const double *ktab, const real *d_r,
                                     double t0, double t1, cudaStream_t st)
{
    if (!a.lg || !a.c.sine) return cudaSuccess;
    cudaError_t e = launch_step_kernel(k_adj_ghost_bed<real>, dim3((a.c.npos + 127) / 128, 16), dim3(128), 0, st, a,
                                       b, ktab, d_r, t0, t1);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_bed_final(const AdjArgs<real> &a, const real *w0, const real *lw0, real *grad_z,
                                     cudaStream_t st)
{
    dim3 b(32, 8);
    k_adj_bed_cells<real><<<dim3((a.geo.nx + 2 + 31) / 32, (a.geo.ny + 2 + 7) / 8), b, 0, st>>>(a, w0, lw0);
    cudaError_t e = cudaMemsetAsync(grad_z, 0, sizeof(real) * (size_t)a.geo.nx * a.geo.ny, st);
    if (e != cudaSuccess) return e;
    k_adj_bed_z<real><<<dim3((a.geo.nx + 3 + 31) / 32, (a.geo.ny + 3 + 7) / 8), b, 0, st>>>(a, grad_z);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_misfit(const AdjArgs<real> &a, const int32_t *gij, int ng, const real *rec, const real *obs,
                                  cudaStream_t st)
{
    cudaError_t e = launch_step_kernel(k_adj_misfit<real>, dim3((ng + 127) / 128), dim3(128), 0, st, a, gij, ng, rec,
                                       obs);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

#define CEL_ADJ_INSTANTIATE(real)                                                                        \
    template cudaError_t launch_adjoint_mask<real>(const AdjArgs<real> &, cudaStream_t);                 \
    template cudaError_t launch_adjoint_hist<real>(const AdjArgs<real> &, cudaStream_t);                 \
    template cudaError_t launch_adjoint_vjp<real>(const AdjArgs<real> &, cudaStream_t);                  \
    template cudaError_t launch_face_vjp_check<real>(const real *, int, real *, cudaStream_t);            \
    template cudaError_t launch_adjoint_tri_bed<real>(const AdjArgs<real> &, const real *, const real *,   \
                                                      const real *, const real *, const real *,         \
                                                      const real *, cudaStream_t);                      \
    template cudaError_t launch_adjoint_ghost_bed<real>(const AdjArgs<real> &, const Bnd &, const double *, \
                                                        const real *, double, double, cudaStream_t);    \
    template cudaError_t launch_adjoint_bed_final<real>(const AdjArgs<real> &, const real *, const real *, \
                                                        real *, cudaStream_t);                         \
    template cudaError_t launch_adjoint_misfit<real>(const AdjArgs<real> &, const int32_t *, int,         \
                                                     const real *, const real *, cudaStream_t);

CEL_ADJ_INSTANTIATE(float)
CEL_ADJ_INSTANTIATE(double)

}  // namespace cel
