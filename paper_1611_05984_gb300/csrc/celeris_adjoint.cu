// Discrete adjoint of the time step with the AB3 predictor and the Euler
// start-up (Eq. 15-17, Sec. 2.3), for the Boussinesq model and the
// nonlinear shallow-water model (Sec. 3.2), and the gradient of a gauge
// misfit.  The reverse of one step, given the adjoint lambda of the state
// after it:
//   1. the masks of the update: the dry clamp w >= Bbar (Reading A-D1), the
//      sponge (Eq. 30), the zero discharge of dry cells;
//   2. the line solves (Eq. 21-23) transposed: the adjoint of the U* and V*
//      increments solves the transposed tridiagonal system of every line
//      (sub- and super-diagonals exchanged, boundary rows included);
//   3. the AB3 history: the right sides R^n = (E, F, G) and the mixed terms
//      F*^n, G*^n collect the adjoint weighted by their coefficients in steps
//      n, n+1 and n+2;
//   4. R^n's and F*^n's Jacobians transposed: every face flux (KP07
//      reconstruction with the limiter and positivity branches of the
//      forward state, then the central-upwind flux), the bed slope and
//      friction, the dispersive eta terms of Eq. 10-11 and F*, G* of
//      Eq. 12-13 (linear in the neighbours, ghosts mapped back to the cells
//      they mirror).
// The face and cell Jacobians are exact: the forward device functions are
// evaluated on dual numbers, one input direction at a time, so every branch
// follows the forward state.  Adjoints reach a cell through the faces around
// it, so they are added with atomics (the sums' order is not fixed).
#include "celeris_internal.cuh"
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

// A cell a face stencil reads: its (w, P, Q) and, unless it is a sine-maker
// ghost (a constant), the interior cell it mirrors and the sign of each
// variable there (Sec. 2.4, Reading A-B1).
template <typename real>
struct Src {
    real v[3];
    int idx;          // interior cell, -1 for a constant ghost
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
        return s;
    }
    if (side >= 0) s.sgn[dir == 0 ? 1 : 2] = real(-1);   // the normal discharge is negated
    s.idx = sj * G.nx + si;
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
        s.sgn[0] = s.sgn[1] = s.sgn[2] = real(1);
        return s;
    }
    s = source(A, i, sj, 0);   // the cell of the mirrored row (an x-ghost if i is outside)
    s.v[2] = -s.v[2];
    s.sgn[2] = -s.sgn[2];
    return s;
}

// Flux through x-face f (dir 0: between cells f-1 and f of row `line`) or
// y-face f (dir 1: between rows f-1 and f of column `line`) from the 4 cells
// around it, in the forward's order of operations.
template <typename T>
__device__ __forceinline__ void face_flux(const Dual<T> w[4], const Dual<T> P[4], const Dual<T> Q[4], T Bm, T Bf,
                                          T Bp, T th, T g, T eps, int dir, Dual<T> H[3])
{
    Dual<T> lo[3], hiL[3], loR[3], hiR[3];
    const Dual<T> w0[3] = {w[0], w[1], w[2]}, P0[3] = {P[0], P[1], P[2]}, Q0[3] = {Q[0], Q[1], Q[2]};
    const Dual<T> w1[3] = {w[1], w[2], w[3]}, P1[3] = {P[1], P[2], P[3]}, Q1[3] = {Q[1], Q[2], Q[3]};
    recon(Dual<T>(th), w0, P0, Q0, Dual<T>(Bm), Dual<T>(Bf), lo, hiL);
    recon(Dual<T>(th), w1, P1, Q1, Dual<T>(Bf), Dual<T>(Bp), loR, hiR);
    if (dir == 0)
        cu_flux(Dual<T>(g), Dual<T>(eps), hiL[0], hiL[1], hiL[2], loR[0], loR[1], loR[2], Dual<T>(Bf), H);
    else
        cu_flux(Dual<T>(g), Dual<T>(eps), hiL[0], hiL[2], hiL[1], loR[0], loR[2], loR[1], Dual<T>(Bf), H);
}

// Step 1 of the reverse for one cell: the masks; the state's own path
// (w^{n+1} = w^n + ...) passes the masked adjoint on unchanged.
template <typename real>
__global__ void k_adj_mask(AdjArgs<real> A)
{
    const Geo &G = A.geo;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
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
    A.lw[k] = clamped ? real(0) : A.lw[k] * (spw ? gam : real(1));
    A.lP[k] = dry ? real(0) : A.lP[k] * gam;
    A.lQ[k] = dry ? real(0) : A.lQ[k] * gam;
}

// Step 3: the history.  The increments of w, U* and V* weigh R^n, R^{n-1},
// R^{n-2} by c0, c1, c2 and (U*, V*) the mixed terms F*, G* by e0, e1, e2.
template <typename real>
__global__ void k_adj_hist(AdjArgs<real> A)
{
    const Geo &G = A.geo;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const int k = j * G.nx + i;
    const real m[5] = {A.lw[k], A.ldU[k], A.ldV[k], A.ldU[k], A.ldV[k]};
#pragma unroll
    for (int v = 0; v < 5; v++) {
        if (v >= 3 && !A.bsnq) break;
        const real c0 = v < 3 ? A.c0 : A.e0, c1 = v < 3 ? A.c1 : A.e1, c2 = v < 3 ? A.c2 : A.e2;
        A.G0[v][k] += c0 * m[v];
        if (A.G1[v]) A.G1[v][k] += c1 * m[v];
        if (A.G2[v]) A.G2[v][k] += c2 * m[v];
    }
}

template <typename real>
__global__ void k_adj_add(AdjArgs<real> A, const real *xw, const real *xP, const real *xQ)
{
    const Geo &G = A.geo;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const int k = j * G.nx + i;
    A.lw[k] += xw[k];
    A.lP[k] += xP[k];
    A.lQ[k] += xQ[k];
}

// Step 2: the transposed line solves, one thread per line (Thomas, in the
// scratch array).  The forward solves T x = r with the Eq. 23 rows
// a_k x_{k-1} + b_k x_k + c_k x_{k+1} and their boundary rows (Reading
// A-B2); here T^T y = mu, whose row k is c_{k-1} y_{k-1} + b_k y_k +
// a_{k+1} y_{k+1}.
template <typename real>
__global__ void k_adj_lines_t(AdjArgs<real> A, int dir)
{
    const Geo &G = A.geo;
    const int n = dir == 0 ? G.nx : G.ny, nl = dir == 0 ? G.ny : G.nx;
    const int line = blockIdx.x * blockDim.x + threadIdx.x;
    if (line >= nl) return;
    auto at = [&](int k) { return dir == 0 ? line * G.nx + k : k * G.nx + line; };
    auto dcell = [&](int k) {
        const int i = dir == 0 ? k : line, j = dir == 0 ? line : k;
        return fmax(A.c.ws - bbar_at(A.Bc, G, i, j), real(0));
    };
    const double h = dir == 0 ? G.dx : G.dy;   // the forward's constants, rounded once
    const real rh2 = real(1.0 / (h * h)), hrh = real(0.5 / h), srh = real(1.0 / (6.0 * h));
    const int lo_side = dir == 0 ? 0 : 2, hi_side = dir == 0 ? 1 : 3;
    const bool lo_sine = (A.c.sine >> lo_side) & 1, hi_sine = (A.c.sine >> hi_side) & 1;
    const real *mu = dir == 0 ? A.lP : A.lQ;
    real *y = dir == 0 ? A.ldU : A.ldV;
    real *cp = A.tri;   // c' of the forward sweep, then y
    // coefficients of row k of T (Eq. 23) with the ends mirrored
    auto row = [&](int k, real &a, real &b, real &c) {
        const real dk = dcell(k), dm = dcell(k > 0 ? k - 1 : 0), dp = dcell(k + 1 < n ? k + 1 : n - 1);
        const real dda = (dp - dm) * hrh, r = A.c.B3 * dk * dk * rh2, s = dk * dda * srh;
        a = s - r;
        b = real(1) + real(2) * r;
        c = -s - r;
        if (k == 0) {
            if (!lo_sine) b -= a;
            a = real(0);
        }
        if (k == n - 1) {
            if (!hi_sine) b -= c;
            c = real(0);
        }
    };
    // T^T: sub_k = c_{k-1}, diag_k = b_k, sup_k = a_{k+1}
    real a0, b0, c0v, an, bn, cn;
    row(0, a0, b0, c0v);
    real sub = real(0), diag = b0, sup = real(0);
    if (n > 1) {
        row(1, an, bn, cn);
        sup = an;
    }
    real cprev = sup / diag, dprev = mu[at(0)] / diag;
    cp[at(0)] = cprev;
    y[at(0)] = dprev;
    real ck_prev = c0v;   // c_{k-1} of T
    for (int k = 1; k < n; k++) {
        real ak, bk, ck;
        row(k, ak, bk, ck);
        sub = ck_prev;
        diag = bk;
        sup = real(0);
        if (k + 1 < n) {
            real a1, b1, c1;
            row(k + 1, a1, b1, c1);
            sup = a1;
        }
        const real den = diag - sub * cprev;
        cprev = sup / den;
        dprev = (mu[at(k)] - sub * dprev) / den;
        cp[at(k)] = cprev;
        y[at(k)] = dprev;
        ck_prev = ck;
    }
    for (int k = n - 2; k >= 0; k--) y[at(k)] = y[at(k)] - cp[at(k)] * y[at(k + 1)];
}

// Bed slope and friction (Eq. 9-10, 31-32): per cell, no neighbours.
template <typename real>
__global__ void k_adj_cells(AdjArgs<real> A)
{
    const Geo &G = A.geo;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const int k = j * G.nx + i;
    const real lF = A.G0[1][k], lG = A.G0[2][k];
    const real c00 = corner(A.Bc, G, i, j), c10 = corner(A.Bc, G, i + 1, j);
    const real c01 = corner(A.Bc, G, i, j + 1), c11 = corner(A.Bc, G, i + 1, j + 1);
    const real Bb = cell_bbar(c00, c10, c01, c11);
    const real BxW = real(0.5) * (c00 + c01), BxE = real(0.5) * (c10 + c11);
    const real ByS = real(0.5) * (c00 + c10), ByN = real(0.5) * (c01 + c11);
    const real g = A.c.g;
    real dw = -(g * (BxE - BxW) * A.c.rdx) * lF - (g * (ByN - ByS) * A.c.rdy) * lG;
    real dP = real(0), dQ = real(0);
    if (A.phy.friction != kFricNone) {
        const real x[3] = {A.w[k], A.P[k], A.Q[k]};
        real grad[3];
#pragma unroll
        for (int v = 0; v < 3; v++) {
            Dual<real> w0(x[0], v == 0 ? real(1) : real(0)), P0(x[1], v == 1 ? real(1) : real(0)),
                Q0(x[2], v == 2 ? real(1) : real(0));
            Dual<real> hb = w0 - Dual<real>(Bb);
            Dual<real> hinv = desing(fmax(hb, Dual<real>(real(0))), Dual<real>(A.c.eps));
            Dual<real> fc = A.phy.friction == kFricManning ? Dual<real>(A.c.fric) * cbrt_r(hinv) : Dual<real>(A.c.fric);
            Dual<real> mag = sqrt(P0 * P0 + Q0 * Q0);
            Dual<real> fF = -(fc * P0 * mag * hinv * hinv), fG = -(fc * Q0 * mag * hinv * hinv);
            grad[v] = lF * fF.d + lG * fG.d;
        }
        dw += grad[0];
        dP = grad[1];
        dQ = grad[2];
    }
    A.lw[k] += dw;
    A.lP[k] += dP;
    A.lQ[k] += dQ;
}

// The face fluxes' Jacobians transposed.  dir 0: x-face f of row `line`;
// dir 1: y-face f of column `line`.
template <typename real>
__global__ void k_adj_faces(AdjArgs<real> A, int dir)
{
    const Geo &G = A.geo;
    const int n = dir == 0 ? G.nx : G.ny, nl = dir == 0 ? G.ny : G.nx;
    const int f = blockIdx.x * blockDim.x + threadIdx.x, line = blockIdx.y * blockDim.y + threadIdx.y;
    if (f > n || line >= nl) return;
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
    Src<real> s[4];
#pragma unroll
    for (int c = 0; c < 4; c++) s[c] = dir == 0 ? source(A, f - 2 + c, line, 0) : source(A, line, f - 2 + c, 1);
    auto face_bed = [&](int q) {   // bed of face q (dir 0: x-face q of row line)
        return dir == 0 ? real(0.5) * (corner(A.Bc, G, q, line) + corner(A.Bc, G, q, line + 1))
                        : real(0.5) * (corner(A.Bc, G, line, q) + corner(A.Bc, G, line + 1, q));
    };
    const real Bm = face_bed(f - 1), Bf = face_bed(f), Bp = face_bed(f + 1);
    for (int c = 0; c < 4; c++) {
        if (s[c].idx < 0) continue;
        for (int v = 0; v < 3; v++) {
            Dual<real> w[4], P[4], Q[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                w[q] = Dual<real>(s[q].v[0], q == c && v == 0 ? real(1) : real(0));
                P[q] = Dual<real>(s[q].v[1], q == c && v == 1 ? real(1) : real(0));
                Q[q] = Dual<real>(s[q].v[2], q == c && v == 2 ? real(1) : real(0));
            }
            Dual<real> H[3];
            face_flux(w, P, Q, Bm, Bf, Bp, A.c.theta, A.c.g, A.c.eps, dir, H);
            const real gsum = lH[0] * H[0].d + lH[1] * H[1].d + lH[2] * H[2].d;
            if (gsum != real(0)) {
                real *dst = v == 0 ? A.lw : (v == 1 ? A.lP : A.lQ);
                atomicAdd(dst + s[c].idx, s[c].sgn[v] * gsum);
            }
        }
    }
}

// Eq. 10-13 transposed: the dispersive eta terms of F and G and the mixed
// terms F*(Q), G*(P) are linear in the neighbouring eta, Q and P, with
// coefficients from the still-water depth; each cell adds its adjoints to
// the cells (or the cells their ghosts mirror) its stencil reads.
template <typename real>
__global__ void k_adj_disp(AdjArgs<real> A)
{
    const Geo &G = A.geo;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const int k = j * G.nx + i;
    const real lF = A.G0[1][k], lG = A.G0[2][k], lFs = A.G0[3][k], lGs = A.G0[4][k];
    if (lF == real(0) && lG == real(0) && lFs == real(0) && lGs == real(0)) return;
    const Coef<real> &C = A.c;
    auto dcell = [&](int ii, int jj) { return fmax(C.ws - bbar_at(A.Bc, G, ii, jj), real(0)); };
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
        const Src<real> s = source2d(A, i + pts[q].di, j + pts[q].dj);
        if (s.idx >= 0) atomicAdd(A.lw + s.idx, pts[q].wgt);
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
        const Src<real> s = source2d(A, i + mq[q].di, j + mq[q].dj);
        if (s.idx >= 0 && mq[q].wgt != real(0)) atomicAdd(A.lQ + s.idx, s.sgn[2] * mq[q].wgt);
        const Src<real> t = source2d(A, i + mp[q].di, j + mp[q].dj);
        if (t.idx >= 0 && mp[q].wgt != real(0)) atomicAdd(A.lP + t.idx, t.sgn[1] * mp[q].wgt);
    }
}

// The adjoint of P and Q into the line solver's layouts (x-rows [ny][px],
// y-columns [nx][py]) and the transposed solves' solutions back.
template <typename real>
__global__ void k_adj_pack(Geo g, const real *lP, const real *lQ, real *X, real *Yc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const size_t k = (size_t)j * g.nx + i;
    X[(size_t)j * g.px + i] = lP[k];
    Yc[(size_t)i * g.py + j] = lQ[k];
}

template <typename real>
__global__ void k_adj_unpack(Geo g, const real *X, const real *Yc, real *ldU, real *ldV)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const size_t k = (size_t)j * g.nx + i;
    ldU[k] = X[(size_t)j * g.px + i];
    ldV[k] = Yc[(size_t)i * g.py + j];
}

// The misfit at the gauges after step n enters the adjoint of w^n.
template <typename real>
__global__ void k_adj_misfit(AdjArgs<real> A, const int32_t *gij, int ng, const real *rec, const real *obs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    atomicAdd(A.lw + gij[2 * k + 1] * A.geo.nx + gij[2 * k], rec[k] - obs[k]);
}

}  // namespace

template <typename real>
cudaError_t launch_adjoint_mask(const AdjArgs<real> &a, cudaStream_t st)
{
    dim3 b(32, 8), g((a.geo.nx + 31) / 32, (a.geo.ny + 7) / 8);
    k_adj_mask<real><<<g, b, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_solves(const AdjArgs<real> &a, cudaStream_t st)
{
    if (a.bsnq) {
        k_adj_lines_t<real><<<(a.geo.ny + 127) / 128, 128, 0, st>>>(a, 0);
        k_adj_lines_t<real><<<(a.geo.nx + 127) / 128, 128, 0, st>>>(a, 1);
        return cudaGetLastError();
    }
    const size_t bytes = sizeof(real) * (size_t)a.geo.nx * a.geo.ny;   // NLSW: P = U*, Q = V*
    cudaError_t e = cudaMemcpyAsync(a.ldU, a.lP, bytes, cudaMemcpyDeviceToDevice, st);
    return e != cudaSuccess ? e : cudaMemcpyAsync(a.ldV, a.lQ, bytes, cudaMemcpyDeviceToDevice, st);
}

template <typename real>
cudaError_t launch_adjoint_hist(const AdjArgs<real> &a, cudaStream_t st)
{
    dim3 b(32, 8), g((a.geo.nx + 31) / 32, (a.geo.ny + 7) / 8);
    k_adj_hist<real><<<g, b, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_vjp(const AdjArgs<real> &a, cudaStream_t st)
{
    dim3 b(32, 8), g((a.geo.nx + 31) / 32, (a.geo.ny + 7) / 8);
    k_adj_cells<real><<<g, b, 0, st>>>(a);
    if (a.bsnq) k_adj_disp<real><<<g, b, 0, st>>>(a);
    dim3 bf(64, 4);
    k_adj_faces<real><<<dim3((a.geo.nx + 1 + 63) / 64, (a.geo.ny + 3) / 4), bf, 0, st>>>(a, 0);
    k_adj_faces<real><<<dim3((a.geo.ny + 1 + 63) / 64, (a.geo.nx + 3) / 4), bf, 0, st>>>(a, 1);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_add(const AdjArgs<real> &a, const real *xw, const real *xP, const real *xQ,
                               cudaStream_t st)
{
    dim3 b(32, 8), g((a.geo.nx + 31) / 32, (a.geo.ny + 7) / 8);
    k_adj_add<real><<<g, b, 0, st>>>(a, xw, xP, xQ);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_pack(const AdjArgs<real> &a, real *X, real *Yc, int back, cudaStream_t st)
{
    dim3 b(32, 8), g((a.geo.nx + 31) / 32, (a.geo.ny + 7) / 8);
    if (back) k_adj_unpack<real><<<g, b, 0, st>>>(a.geo, X, Yc, a.ldU, a.ldV);
    else k_adj_pack<real><<<g, b, 0, st>>>(a.geo, a.lP, a.lQ, X, Yc);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_adjoint_step(const AdjArgs<real> &a, cudaStream_t st)
{
    cudaError_t e = launch_adjoint_mask(a, st);
    if (e == cudaSuccess) e = launch_adjoint_solves(a, st);
    if (e == cudaSuccess) e = launch_adjoint_hist(a, st);
    if (e == cudaSuccess) e = launch_adjoint_vjp(a, st);
    return e;
}

template <typename real>
cudaError_t launch_adjoint_misfit(const AdjArgs<real> &a, const int32_t *gij, int ng, const real *rec, const real *obs,
                                  cudaStream_t st)
{
    k_adj_misfit<real><<<(ng + 127) / 128, 128, 0, st>>>(a, gij, ng, rec, obs);
    return cudaGetLastError();
}

#define CEL_ADJ_INSTANTIATE(real)                                                                        \
    template cudaError_t launch_adjoint_step<real>(const AdjArgs<real> &, cudaStream_t);                 \
    template cudaError_t launch_adjoint_mask<real>(const AdjArgs<real> &, cudaStream_t);                 \
    template cudaError_t launch_adjoint_solves<real>(const AdjArgs<real> &, cudaStream_t);               \
    template cudaError_t launch_adjoint_hist<real>(const AdjArgs<real> &, cudaStream_t);                 \
    template cudaError_t launch_adjoint_vjp<real>(const AdjArgs<real> &, cudaStream_t);                  \
    template cudaError_t launch_adjoint_add<real>(const AdjArgs<real> &, const real *, const real *,      \
                                                  const real *, cudaStream_t);                          \
    template cudaError_t launch_adjoint_pack<real>(const AdjArgs<real> &, real *, real *, int, cudaStream_t); \
    template cudaError_t launch_adjoint_misfit<real>(const AdjArgs<real> &, const int32_t *, int,         \
                                                     const real *, const real *, cudaStream_t);

CEL_ADJ_INSTANTIATE(float)
CEL_ADJ_INSTANTIATE(double)

}  // namespace cel
