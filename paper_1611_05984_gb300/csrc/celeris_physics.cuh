// Device functions of the method shared by the step kernels and the
// adjoint kernels: KP07 reconstruction and central-upwind flux (Sec. 2.2,
// Eq. 14), friction helpers, the sponge factor (Eq. 30).  They are templates
// on the arithmetic type, so the adjoint can evaluate them on dual numbers
// and get their exact derivatives along the same branches.
#pragma once
#include "celeris_internal.cuh"

namespace cel {

__device__ __forceinline__ int mirror_index(int i, int n)
{
    return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
}

// Eq. 14: u = k(h) P with k(h) = sqrt(2) h / sqrt(h^4 + max(h^4, eps)).
template <typename real>
__device__ __forceinline__ real desing(real h, real eps)
{
    real h2 = h * h;
    real h4 = h2 * h2;
    return real(1.4142135623730951) * h * rsqrt(h4 + fmax(h4, eps));
}

// KP07 step 1: generalized minmod of the three one-sided / central slopes.
template <typename real>
__device__ __forceinline__ real minmod3(real th, real qm, real q0, real qp)
{
    // the three slopes share a sign iff the two one-sided ones do (the
    // central one lies between them); then the one of least magnitude
    real a = th * (q0 - qm), b = real(0.5) * (qp - qm), c = th * (qp - q0);
    real lo = fmin(a, fmin(b, c)), hi = fmax(a, fmax(b, c));
    return lo > real(0) ? lo : (hi < real(0) ? hi : real(0));
}

// KP07 steps 1-2 for one cell along one direction: face values of (w, P, Q)
// at the low and high faces, then the positivity fix of w.
template <typename real>
__device__ __forceinline__ void recon(real th, const real wq[3], const real Pq[3],
                                      const real Qq[3], real Blo, real Bhi, real lo[3],
                                      real hi[3])
{
    real sw = minmod3(th, wq[0], wq[1], wq[2]);
    real sP = minmod3(th, Pq[0], Pq[1], Pq[2]);
    real sQ = minmod3(th, Qq[0], Qq[1], Qq[2]);
    lo[0] = wq[1] - real(0.5) * sw;
    hi[0] = wq[1] + real(0.5) * sw;
    lo[1] = Pq[1] - real(0.5) * sP;
    hi[1] = Pq[1] + real(0.5) * sP;
    lo[2] = Qq[1] - real(0.5) * sQ;
    hi[2] = Qq[1] + real(0.5) * sQ;
    if (hi[0] < Bhi) {
        hi[0] = Bhi;
        lo[0] = real(2) * wq[1] - Bhi;
    } else if (lo[0] < Blo) {
        lo[0] = Blo;
        hi[0] = real(2) * wq[1] - Blo;
    }
}

// KP07 step 3: central-upwind flux.  States are (w, normal, tangential
// discharge); H = (mass, normal momentum, tangential momentum).
template <typename real>
__device__ __forceinline__ void cu_flux(real g, real eps, real wL, real nL, real tL, real wR,
                                        real nR, real tR, real Bf, real H[3])
{
    real hL = fmax(wL - Bf, real(0)), hR = fmax(wR - Bf, real(0));
    real kL = desing(hL, eps), kR = desing(hR, eps);
    real uL = kL * nL, vL = kL * tL, uR = kR * nR, vR = kR * tR;
    real qnL = hL * uL, qtL = hL * vL, qnR = hR * uR, qtR = hR * vR;
    real sL = sqrt(g * hL), sR = sqrt(g * hR);
    real ap = fmax(fmax(uL + sL, uR + sR), real(0));
    real am = fmin(fmin(uL - sL, uR - sR), real(0));
    real den = ap - am;
    if (!(den > real(0))) {
        H[0] = H[1] = H[2] = real(0);
        return;
    }
    real inv = real(1) / den, apam = ap * am;
    real FL1 = qnL * uL + real(0.5) * g * hL * hL, FR1 = qnR * uR + real(0.5) * g * hR * hR;
    H[0] = (ap * qnL - am * qnR + apam * (wR - wL)) * inv;
    H[1] = (ap * FL1 - am * FR1 + apam * (qnR - qnL)) * inv;
    H[2] = (ap * (qnL * vL) - am * (qnR * vR) + apam * (qtR - qtL)) * inv;
}

__device__ __forceinline__ float cbrt_r(float x) { return x > 0.f ? exp2f(__log2f(x) * (1.f / 3.f)) : 0.f; }
__device__ __forceinline__ double cbrt_r(double x) { return cbrt(x); }
__device__ __forceinline__ float cospi_r(float x) { return cospif(x); }
__device__ __forceinline__ double cospi_r(double x) { return cospi(x); }

// Eq. 30 with D the distance from the absorbing face to the cell centre and
// L_s = width cells: a cell idx cells from the side (idx = i for the west) is
// inside when idx < width, with (L_s - D)/L_s = (2 (width - idx) - 1)/(2 width).
template <typename real>
__device__ __forceinline__ real sponge_eq30(int w, int idx)
{
    const real r = real(2 * (w - idx) - 1) / real(2 * w);
    return real(0.5) * (real(1) + cospi_r(r));
}

// The factor of side s for a cell idx cells from it: 1 outside its sponge;
// inside, from the solver's table when the arguments carry one (the same
// expression, evaluated once per side and position), else evaluated here.
template <typename real>
__device__ __forceinline__ real sponge_side(const Coef<real> &c, int s, int idx)
{
    const int w = c.spw[s];
    if (idx >= w) return real(1);
    return c.gam ? c.gam[(size_t)s * c.npos + idx] : sponge_eq30<real>(w, idx);
}

// The smallest gamma over the sponge sides.
template <typename real>
__device__ __forceinline__ real sponge_gamma(const Coef<real> &c, const Geo &g, int i, int j)
{
    return fmin(fmin(sponge_side(c, 0, i), sponge_side(c, 1, g.nx - 1 - i)),
                fmin(sponge_side(c, 2, j), sponge_side(c, 3, g.ny - 1 - j)));
}

// Adjacent still-water depth d and ghost coordinates of table position pos
// (Reading A-B4): west / east sides run along rows j = pos - 2, south /
// north sides along columns i = pos - 2 including the corner columns, where
// d is clamped along the side.  Returns false where the position is unused.
template <typename real>
__device__ inline bool ghost_site(const Geo &g, const real *d_r, int side, int layer, int pos, double &x,
                                  double &y, double &dadj)
{
    const int along = pos - 2;
    if (side < 2) {
        if (along < 0 || along >= g.ny) return false;
        const int gi = side == 0 ? -1 - layer : g.nx + layer;
        x = (gi + 0.5) * g.dx;
        y = (along + 0.5) * g.dy;
        dadj = (double)d_r[(size_t)along * g.px + (side == 0 ? 0 : g.nx - 1)];
    } else {
        if (along < -2 || along > g.nx + 1) return false;
        const int gj = side == 2 ? -1 - layer : g.ny + layer;
        const int ia = along < 0 ? 0 : (along > g.nx - 1 ? g.nx - 1 : along);
        x = (along + 0.5) * g.dx;
        y = (gj + 0.5) * g.dy;
        dadj = (double)d_r[(size_t)(side == 2 ? 0 : g.ny - 1) * g.px + ia];
    }
    return true;
}

// The interior cell whose depth ghost_site reads for table position pos.
__device__ __forceinline__ void ghost_adjacent(const Geo &g, int side, int pos, int &i, int &j)
{
    const int along = pos - 2;
    if (side < 2) {
        i = side == 0 ? 0 : g.nx - 1;
        j = along;
    } else {
        i = along < 0 ? 0 : (along > g.nx - 1 ? g.nx - 1 : along);
        j = side == 2 ? 0 : g.ny - 1;
    }
}

}  // namespace cel
