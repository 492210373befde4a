// Discrete adjoint of the time step, for the nonlinear shallow-water model
// (Sec. 3.2: the dispersive terms and the line solves off) with the AB3
// predictor and the Euler start-up (Eq. 15, Sec. 2.3), and the gradient of a
// gauge misfit.  The reverse of one step, given the adjoint lambda of the
// state after it:
//   1. the masks of the update: the dry clamp w >= Bbar (Reading A-D1), the
//      sponge (Eq. 30), the zero discharge of dry cells;
//   2. the AB3 history: the right side R^n = (E, F, G) collects the
//      adjoint weighted by its coefficient in steps n, n+1 and n+2;
//   3. R^n's Jacobian transposed, applied to that adjoint: every face flux
//      (KP07 reconstruction with the limiter and positivity branches of the
//      forward state, then the central-upwind flux) and the per-cell bed
//      slope and friction terms.
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
        const real *tb = A.ghost + ghost_index(0, side, layer, 0, pos, A.c.npos);
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

// Step 1 and 2 of the reverse for one cell: the masks, then the history.
template <typename real>
__global__ void k_adj_update(AdjArgs<real> A)
{
    const Geo &G = A.geo;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= G.nx || j >= G.ny) return;
    const int k = j * G.nx + i;
    const real Bb = bbar_at(A.Bc, G, i, j);
    const real ws = A.c.ws;
    const real d = fmax(ws - Bb, real(0));
    const real gam = sponge_gamma<real>(A.c, G, i, j);
    const real wn = A.w_next[k];
    const bool dry = wn - Bb <= real(0);
    const bool spw = gam < real(1) && d > real(0);
    const real w1 = spw ? ws + (wn - ws) / gam : wn;   // before the sponge
    const real tol = (sizeof(real) == 8 ? real(1e-12) : real(1e-6)) * fmax(real(1), fabs(Bb));
    const bool clamped = w1 - Bb <= tol;
    const real mw = clamped ? real(0) : A.lw[k] * (spw ? gam : real(1));
    const real mP = dry ? real(0) : A.lP[k] * gam;
    const real mQ = dry ? real(0) : A.lQ[k] * gam;
    A.lw[k] = mw;
    A.lP[k] = mP;
    A.lQ[k] = mQ;
    const real m[3] = {mw, mP, mQ};
#pragma unroll
    for (int v = 0; v < 3; v++) {
        A.G0[v][k] += A.c0 * m[v];
        A.G1[v][k] += A.c1 * m[v];
        A.G2[v][k] += A.c2 * m[v];
    }
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
cudaError_t launch_adjoint_step(const AdjArgs<real> &a, cudaStream_t st)
{
    dim3 b(32, 8), g((a.geo.nx + 31) / 32, (a.geo.ny + 7) / 8);
    k_adj_update<real><<<g, b, 0, st>>>(a);
    k_adj_cells<real><<<g, b, 0, st>>>(a);
    dim3 bf(64, 4);
    k_adj_faces<real><<<dim3((a.geo.nx + 1 + 63) / 64, (a.geo.ny + 3) / 4), bf, 0, st>>>(a, 0);
    k_adj_faces<real><<<dim3((a.geo.ny + 1 + 63) / 64, (a.geo.nx + 3) / 4), bf, 0, st>>>(a, 1);
    return cudaGetLastError();
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
    template cudaError_t launch_adjoint_misfit<real>(const AdjArgs<real> &, const int32_t *, int,         \
                                                     const real *, const real *, cudaStream_t);

CEL_ADJ_INSTANTIATE(float)
CEL_ADJ_INSTANTIATE(double)

}  // namespace cel
