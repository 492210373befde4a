/*
 * celeris_oracle.c -- FP64 CPU oracle of the Celeris extended-Boussinesq step.
 *
 * TEST INFRASTRUCTURE ONLY (see celeris_oracle.h).  Plain loops in the order
 * the paper describes, one function per step of the method, no blocking or
 * fusion.  Readings of passages the paper leaves open are marked "Reading:".
 *
 * Paper: S. Tavakkol, P. Lynett, "Celeris: A GPU-accelerated open source
 * software with a Boussinesq-type wave solver ...", arXiv 1611.05984.
 *   Sec. 2.1  governing equations (Eq. 1-3)
 *   Sec. 2.2  Wei-Kirby form (Eq. 4-13), KP07 steps 1-4, Eq. 14
 *   Sec. 2.3  AB3 predictor (Eq. 15-17), AM4 corrector (Eq. 18-20),
 *             tridiagonal systems (Eq. 21-23)
 *   Sec. 2.4  boundaries: solid wall (Eq. 24), sine maker (Eq. 25-29),
 *             sponge (Eq. 30)
 *   Sec. 2.6  friction (Eq. 31-32);  Sec. 2.7 solitary wave (Eq. 33-36)
 *
 * Storage: every cell field is "extended", (nx+4) x (ny+4) with two ghost
 * layers (Sec. 2.4).  Bed corners are (nx+3) x (ny+3), corner (ci,cj) at
 * (ci*dx, cj*dy), ci in [-1, nx+1].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include "celeris_oracle.h"

#define ORC_PI 3.14159265358979323846

struct orc {
    orc_params p;
    orc_bc bc[4];
    int nx, ny, ex, ey;
    long long step;   /* steps since create: t = step * dt                  */
    long long nh;     /* steps since the last restart of the AB3 history    */
    orc_real clamp_mass;
    orc_real *z, *Bc, *Bbar, *d, *ddx, *ddy;      /* static fields           */
    orc_real *w, *P, *Q, *w1, *P1, *Q1;           /* state n and iterate n+1 */
    orc_real *U, *V, *U1, *V1;                    /* U*, V* (Eq. 7-8)        */
    orc_real *E[3], *F[3], *G[3], *Fs[3], *Gs[3]; /* [0]=n, [1]=n-1, [2]=n-2 */
    orc_real *Ec, *Fc, *Gc, *Fsc, *Gsc;           /* rhs at the AM4 iterate  */
    orc_real *Hx[3], *Hy[3];                      /* face fluxes             */
    int ng, log_every, cap, nrec, head;
    int *gij;
    orc_real *grec;
    orc_real *maxw, delta;                        /* run-up tracking         */
};

static size_t IX(const orc *o, int i, int j)
{
    return (size_t)(j + 2) * (size_t)o->ex + (size_t)(i + 2);
}
static size_t CX(const orc *o, int ci, int cj)
{
    return (size_t)(cj + 1) * (size_t)(o->nx + 3) + (size_t)(ci + 1);
}
/* Bed on the x-face f (x = f dx) of row j, and on the y-face g of column i:
 * mean of the face's two end corners (Reading A-W1). */
static orc_real Bx(const orc *o, int f, int j)
{
    return 0.5 * (o->Bc[CX(o, f, j)] + o->Bc[CX(o, f, j + 1)]);
}
static orc_real By(const orc *o, int i, int g)
{
    return 0.5 * (o->Bc[CX(o, i, g)] + o->Bc[CX(o, i + 1, g)]);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------- pieces */

/* Generalized minmod of KP07 step 1 (Sec. 2.2): the slope is
 * minmod(theta*(q0-qm), (qp-qm)/2, theta*(qp-q0)); zero unless all three
 * share a sign, else the one of least magnitude (Reading A-L1). */
orc_real orc_minmod(orc_real theta, orc_real qm, orc_real q0, orc_real qp)
{
    orc_real a = theta * (q0 - qm), b = 0.5 * (qp - qm), c = theta * (qp - q0);
    if (a > 0.0 && b > 0.0 && c > 0.0) return fmin(a, fmin(b, c));
    if (a < 0.0 && b < 0.0 && c < 0.0) return fmax(a, fmax(b, c));
    return 0.0;
}

/* Eq. 29: Eckart's approximation k = omega^2/g * sqrt(coth(omega^2 d / g)). */
orc_real orc_eckart_k(orc_real omega, orc_real d, orc_real g)
{
    orc_real k0 = omega * omega / g;
    return k0 * sqrt(1.0 / tanh(k0 * d));
}

/* Eq. 30: gamma = (1 + cos(pi (Ls - D)/Ls))/2 inside the layer, 1 outside. */
orc_real orc_sponge_gamma(orc_real D, orc_real Ls)
{
    if (!(D < Ls)) return 1.0;
    return 0.5 * (1.0 + cos(ORC_PI * (Ls - D) / Ls));
}

/* Textbook Thomas algorithm: a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = r[i]. */
static void thomas_ws(int n, const orc_real *a, const orc_real *b, const orc_real *c,
                      const orc_real *r, orc_real *x, orc_real *cp, orc_real *dp)
{
    cp[0] = c[0] / b[0];
    dp[0] = r[0] / b[0];
    for (int i = 1; i < n; i++) {
        orc_real m = b[i] - a[i] * cp[i - 1];
        cp[i] = c[i] / m;
        dp[i] = (r[i] - a[i] * dp[i - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
}

void orc_thomas(int n, const orc_real *a, const orc_real *b, const orc_real *c,
                const orc_real *r, orc_real *x)
{
    if (n <= 0) return;
    orc_real *cp = (orc_real *)malloc(sizeof(orc_real) * (size_t)n);
    orc_real *dp = (orc_real *)malloc(sizeof(orc_real) * (size_t)n);
    thomas_ws(n, a, b, c, r, x, cp, dp);
    free(cp);
    free(dp);
}

/* Eq. 14 factor: u = k(h) * P with k(h) = sqrt(2) h / sqrt(h^4 + max(h^4, eps))
 * (Reading A-G3); also the desingularised 1/h of the friction term (Sec. 2.6). */
static orc_real desing(orc_real h, orc_real eps)
{
    orc_real h4 = (h * h) * (h * h);
    return sqrt(2.0) * h / sqrt(h4 + fmax(h4, eps));
}

/* KP07 step 3 (Sec. 2.2): central-upwind flux through one face.  L/R states
 * are (w, normal discharge, tangential discharge) at the face; Bf is the bed
 * on the face.  H = (mass, normal momentum, tangential momentum). */
void orc_central_upwind(orc_real g, orc_real eps, orc_real wL, orc_real nL, orc_real tL,
                        orc_real wR, orc_real nR, orc_real tR, orc_real Bf, orc_real H[3])
{
    orc_real hL = fmax(wL - Bf, 0.0), hR = fmax(wR - Bf, 0.0);
    orc_real kL = desing(hL, eps), kR = desing(hR, eps);
    orc_real uL = kL * nL, vL = kL * tL, uR = kR * nR, vR = kR * tR;
    orc_real qnL = hL * uL, qtL = hL * vL, qnR = hR * uR, qtR = hR * vR;
    orc_real sL = sqrt(g * hL), sR = sqrt(g * hR);
    orc_real ap = fmax(fmax(uL + sL, uR + sR), 0.0);
    orc_real am = fmin(fmin(uL - sL, uR - sR), 0.0);
    orc_real den = ap - am;
    if (!(den > 0.0)) { /* both sides dry (Reading A-F1) */
        H[0] = H[1] = H[2] = 0.0;
        return;
    }
    orc_real FL0 = qnL, FL1 = qnL * uL + 0.5 * g * hL * hL, FL2 = qnL * vL;
    orc_real FR0 = qnR, FR1 = qnR * uR + 0.5 * g * hR * hR, FR2 = qnR * vR;
    H[0] = (ap * FL0 - am * FR0 + ap * am * (wR - wL)) / den;
    H[1] = (ap * FL1 - am * FR1 + ap * am * (qnR - qnL)) / den;
    H[2] = (ap * FL2 - am * FR2 + ap * am * (qtR - qtL)) / den;
}

/* Sine-wave maker, Eq. 25-28 summed over components (Reading A-B4). */
static void sine_eval(const orc *o, const orc_bc *bc, orc_real dadj, orc_real x,
                      orc_real y, orc_real t, orc_real *eta, orc_real *Pg, orc_real *Qg)
{
    *eta = *Pg = *Qg = 0.0;
    if (!(dadj > 0.0)) return;
    for (int m = 0; m < bc->ncomp; m++) {
        orc_real om = 2.0 * ORC_PI / bc->period[m];
        orc_real k = orc_eckart_k(om, dadj, o->p.g);
        orc_real c = om / k;
        orc_real cs = cos(bc->dir[m]), sn = sin(bc->dir[m]);
        orc_real em = bc->amp[m] * sin(om * t - k * cs * x - k * sn * y + bc->phase[m]);
        *eta += em;
        *Pg += c * cs * em;
        *Qg += c * sn * em;
    }
}

/* ------------------------------------------------------------ boundaries */

/* Ghost layers at time t (Sec. 2.4).  x-sides first over interior rows, then
 * y-sides over every column, so corner ghosts come by composition.
 * Solid (and the outer ghosts behind a sponge): face-centred mirror, ghost
 * -1-k <- interior k, normal discharge negated (Eq. 24, Reading A-B1). */
static void fill_ghosts(orc *o, orc_real *w, orc_real *P, orc_real *Q, orc_real t)
{
    const int nx = o->nx, ny = o->ny;
    const orc_real ws = o->p.ws;
    for (int side = ORC_W; side <= ORC_E; side++) {
        const orc_bc *bc = &o->bc[side];
        for (int j = 0; j < ny; j++)
            for (int k = 0; k < 2; k++) {
                int gi = side == ORC_W ? -1 - k : nx + k;
                int si = side == ORC_W ? k : nx - 1 - k;
                size_t gc = IX(o, gi, j), sc = IX(o, si, j);
                if (bc->type == ORC_SINE) {
                    orc_real eta, Pg, Qg;
                    orc_real dadj = o->d[IX(o, side == ORC_W ? 0 : nx - 1, j)];
                    sine_eval(o, bc, dadj, (gi + 0.5) * o->p.dx,
                              (j + 0.5) * o->p.dy, t, &eta, &Pg, &Qg);
                    w[gc] = ws + eta;
                    P[gc] = Pg;
                    Q[gc] = Qg;
                } else {
                    w[gc] = w[sc];
                    P[gc] = -P[sc];
                    Q[gc] = Q[sc];
                }
            }
    }
    for (int side = ORC_S; side <= ORC_N; side++) {
        const orc_bc *bc = &o->bc[side];
        for (int i = -2; i < nx + 2; i++)
            for (int k = 0; k < 2; k++) {
                int gj = side == ORC_S ? -1 - k : ny + k;
                int sj = side == ORC_S ? k : ny - 1 - k;
                size_t gc = IX(o, i, gj), sc = IX(o, i, sj);
                if (bc->type == ORC_SINE) {
                    orc_real eta, Pg, Qg;
                    int ic = i < 0 ? 0 : (i > nx - 1 ? nx - 1 : i);
                    orc_real dadj = o->d[IX(o, ic, side == ORC_S ? 0 : ny - 1)];
                    sine_eval(o, bc, dadj, (i + 0.5) * o->p.dx,
                              (gj + 0.5) * o->p.dy, t, &eta, &Pg, &Qg);
                    w[gc] = ws + eta;
                    P[gc] = Pg;
                    Q[gc] = Qg;
                } else {
                    w[gc] = w[sc];
                    P[gc] = P[sc];
                    Q[gc] = -Q[sc];
                }
            }
    }
}

/* Sponge coefficient of cell (i,j): Eq. 30 with D the distance from the
 * absorbing boundary face to the cell centre; the smallest gamma over all
 * sponge sides (Reading A-B3). */
static orc_real sponge_at(const orc *o, int i, int j)
{
    orc_real gmin = 1.0;
    for (int s = 0; s < 4; s++) {
        const orc_bc *bc = &o->bc[s];
        if (bc->type != ORC_SPONGE || bc->width <= 0) continue;
        orc_real D, L;
        if (s == ORC_W) { D = (i + 0.5) * o->p.dx; L = bc->width * o->p.dx; }
        else if (s == ORC_E) { D = (o->nx - i - 0.5) * o->p.dx; L = bc->width * o->p.dx; }
        else if (s == ORC_S) { D = (j + 0.5) * o->p.dy; L = bc->width * o->p.dy; }
        else { D = (o->ny - j - 0.5) * o->p.dy; L = bc->width * o->p.dy; }
        gmin = fmin(gmin, orc_sponge_gamma(D, L));
    }
    return gmin;
}

/* ------------------------------------------------------- static fields */

/* a0: bed corners from cell-centre z (Reading A-W1): ghost z mirrored evenly,
 * corner = mean of its 4 cells, cell Bbar = mean of its 4 corners,
 * d = max(w_s - Bbar, 0) (Sec. 2.1), d_x, d_y by central differences. */
static void derive_static(orc *o, const orc_real *zin)
{
    const int nx = o->nx, ny = o->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) o->z[IX(o, i, j)] = zin[(size_t)j * nx + i];
    for (int j = 0; j < ny; j++)
        for (int k = 0; k < 2; k++) {
            o->z[IX(o, -1 - k, j)] = o->z[IX(o, k, j)];
            o->z[IX(o, nx + k, j)] = o->z[IX(o, nx - 1 - k, j)];
        }
    for (int i = -2; i < nx + 2; i++)
        for (int k = 0; k < 2; k++) {
            o->z[IX(o, i, -1 - k)] = o->z[IX(o, i, k)];
            o->z[IX(o, i, ny + k)] = o->z[IX(o, i, ny - 1 - k)];
        }
    for (int cj = -1; cj <= ny + 1; cj++)
        for (int ci = -1; ci <= nx + 1; ci++)
            o->Bc[CX(o, ci, cj)] =
                0.25 * (o->z[IX(o, ci - 1, cj - 1)] + o->z[IX(o, ci, cj - 1)] +
                        o->z[IX(o, ci - 1, cj)] + o->z[IX(o, ci, cj)]);
    for (int j = -1; j <= ny; j++)
        for (int i = -1; i <= nx; i++) {
            orc_real b = 0.25 * (o->Bc[CX(o, i, j)] + o->Bc[CX(o, i + 1, j)] +
                               o->Bc[CX(o, i, j + 1)] + o->Bc[CX(o, i + 1, j + 1)]);
            o->Bbar[IX(o, i, j)] = b;
            o->d[IX(o, i, j)] = fmax(o->p.ws - b, 0.0);
        }
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            o->ddx[IX(o, i, j)] =
                (o->d[IX(o, i + 1, j)] - o->d[IX(o, i - 1, j)]) / (2.0 * o->p.dx);
            o->ddy[IX(o, i, j)] =
                (o->d[IX(o, i, j + 1)] - o->d[IX(o, i, j - 1)]) / (2.0 * o->p.dy);
        }
}

/* ------------------------------------------------------------- the rhs */

/* KP07 steps 1-2 for one cell along one direction (stride s): minmod slopes
 * of w, P, Q give the low- and high-face values; then the conservative
 * positivity fix of w against the face beds Blo, Bhi (Reading A-L2). */
static void recon_cell(orc_real theta, const orc_real *w, const orc_real *P,
                       const orc_real *Q, size_t c, size_t s, orc_real Blo,
                       orc_real Bhi, orc_real lo[3], orc_real hi[3])
{
    const orc_real *q[3] = {w, P, Q};
    for (int v = 0; v < 3; v++) {
        orc_real sig = orc_minmod(theta, q[v][c - s], q[v][c], q[v][c + s]);
        lo[v] = q[v][c] - 0.5 * sig;
        hi[v] = q[v][c] + 0.5 * sig;
    }
    if (hi[0] < Bhi) {
        hi[0] = Bhi;
        lo[0] = 2.0 * w[c] - Bhi;
    } else if (lo[0] < Blo) {
        lo[0] = Blo;
        hi[0] = 2.0 * w[c] - Blo;
    }
}

/* Eq. 9-13 at every interior cell, for state (w,P,Q) whose ghosts are set.
 * E, F, G: flux divergence of KP07 (steps 3-4) + bed slope + friction
 * (Eq. 31-32) + the dispersive eta terms of Eq. 10-11 by central FD;
 * Fs = F*(Q) (Eq. 12), Gs = G*(P) (Eq. 13, Reading A-G2). */
static void compute_rhs(orc *o, const orc_real *w, const orc_real *P,
                        const orc_real *Q, orc_real *E, orc_real *F, orc_real *G,
                        orc_real *Fs, orc_real *Gs)
{
    const int nx = o->nx, ny = o->ny;
    const orc_real dx = o->p.dx, dy = o->p.dy, g = o->p.g, eps = o->p.eps;
    const orc_real th = o->p.theta;
    const size_t ex = (size_t)o->ex;

#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int f = 0; f <= nx; f++) {
            orc_real loL[3], hiL[3], loR[3], hiR[3], H[3];
            recon_cell(th, w, P, Q, IX(o, f - 1, j), 1, Bx(o, f - 1, j), Bx(o, f, j), loL, hiL);
            recon_cell(th, w, P, Q, IX(o, f, j), 1, Bx(o, f, j), Bx(o, f + 1, j), loR, hiR);
            orc_central_upwind(g, eps, hiL[0], hiL[1], hiL[2], loR[0], loR[1],
                               loR[2], Bx(o, f, j), H);
            size_t k = (size_t)j * (size_t)(nx + 1) + (size_t)f;
            o->Hx[0][k] = H[0];
            o->Hx[1][k] = H[1];
            o->Hx[2][k] = H[2];
        }
#pragma omp parallel for schedule(static)
    for (int gq = 0; gq <= ny; gq++)
        for (int i = 0; i < nx; i++) {
            orc_real loS[3], hiS[3], loN[3], hiN[3], H[3];
            recon_cell(th, w, P, Q, IX(o, i, gq - 1), ex, By(o, i, gq - 1), By(o, i, gq), loS, hiS);
            recon_cell(th, w, P, Q, IX(o, i, gq), ex, By(o, i, gq), By(o, i, gq + 1), loN, hiN);
            /* normal discharge is Q, tangential is P */
            orc_central_upwind(g, eps, hiS[0], hiS[2], hiS[1], loN[0], loN[2],
                               loN[1], By(o, i, gq), H);
            size_t k = (size_t)gq * (size_t)nx + (size_t)i;
            o->Hy[0][k] = H[0];
            o->Hy[1][k] = H[2];
            o->Hy[2][k] = H[1];
        }

    const int bsnq = o->p.model == ORC_BSNQ;
    const orc_real Bd = o->p.Bd, ws = o->p.ws, B3 = o->p.Bd + 1.0 / 3.0;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = IX(o, i, j);
            size_t kx = (size_t)j * (size_t)(nx + 1) + (size_t)i;
            size_t ky = (size_t)j * (size_t)nx + (size_t)i;
            size_t kyn = (size_t)(j + 1) * (size_t)nx + (size_t)i;
            orc_real hb = w[c] - o->Bbar[c];
            orc_real e = -(o->Hx[0][kx + 1] - o->Hx[0][kx]) / dx -
                       (o->Hy[0][kyn] - o->Hy[0][ky]) / dy;
            orc_real f = -(o->Hx[1][kx + 1] - o->Hx[1][kx]) / dx -
                       (o->Hy[1][kyn] - o->Hy[1][ky]) / dy -
                       g * hb * (Bx(o, i + 1, j) - Bx(o, i, j)) / dx;
            orc_real gg = -(o->Hx[2][kx + 1] - o->Hx[2][kx]) / dx -
                        (o->Hy[2][kyn] - o->Hy[2][ky]) / dy -
                        g * hb * (By(o, i, j + 1) - By(o, i, j)) / dy;
            if (o->p.friction != ORC_FRIC_NONE) {
                orc_real hinv = desing(fmax(hb, 0.0), eps);
                orc_real fc = o->p.friction == ORC_FRIC_MANNING
                                ? g * o->p.fcoef * o->p.fcoef * cbrt(hinv)
                                : o->p.fcoef;
                orc_real mag = sqrt(P[c] * P[c] + Q[c] * Q[c]);
                f -= fc * P[c] * mag * hinv * hinv;
                gg -= fc * Q[c] * mag * hinv * hinv;
            }
            orc_real fs = 0.0, gs = 0.0;
            if (bsnq) {
                orc_real dd = o->d[c], dxd = o->ddx[c], dyd = o->ddy[c];
#define ETA(a, b) (w[IX(o, i + (a), j + (b))] - ws)
                orc_real exx = (ETA(1, 0) - 2.0 * ETA(0, 0) + ETA(-1, 0)) / (dx * dx);
                orc_real eyy = (ETA(0, 1) - 2.0 * ETA(0, 0) + ETA(0, -1)) / (dy * dy);
                orc_real exy = (ETA(1, 1) - ETA(1, -1) - ETA(-1, 1) + ETA(-1, -1)) / (4.0 * dx * dy);
                orc_real exxx = (ETA(2, 0) - 2.0 * ETA(1, 0) + 2.0 * ETA(-1, 0) - ETA(-2, 0)) /
                              (2.0 * dx * dx * dx);
                orc_real eyyy = (ETA(0, 2) - 2.0 * ETA(0, 1) + 2.0 * ETA(0, -1) - ETA(0, -2)) /
                              (2.0 * dy * dy * dy);
                orc_real exyy = ((ETA(1, 1) - 2.0 * ETA(1, 0) + ETA(1, -1)) -
                               (ETA(-1, 1) - 2.0 * ETA(-1, 0) + ETA(-1, -1))) /
                              (2.0 * dx * dy * dy);
                orc_real exxy = ((ETA(1, 1) - 2.0 * ETA(0, 1) + ETA(-1, 1)) -
                               (ETA(1, -1) - 2.0 * ETA(0, -1) + ETA(-1, -1))) /
                              (2.0 * dx * dx * dy);
#undef ETA
                f += Bd * g * dd * dd * dd * (exxx + exyy) +
                     Bd * g * dd * dd * (dxd * (2.0 * exx + eyy) + dyd * exy);
                gg += Bd * g * dd * dd * dd * (eyyy + exxy) +
                      Bd * g * dd * dd * (dyd * (2.0 * eyy + exx) + dxd * exy);
#define QQ(a, b) Q[IX(o, i + (a), j + (b))]
#define PP(a, b) P[IX(o, i + (a), j + (b))]
                orc_real Qx = (QQ(1, 0) - QQ(-1, 0)) / (2.0 * dx);
                orc_real Qy = (QQ(0, 1) - QQ(0, -1)) / (2.0 * dy);
                orc_real Qxy = (QQ(1, 1) - QQ(1, -1) - QQ(-1, 1) + QQ(-1, -1)) / (4.0 * dx * dy);
                orc_real Px = (PP(1, 0) - PP(-1, 0)) / (2.0 * dx);
                orc_real Py = (PP(0, 1) - PP(0, -1)) / (2.0 * dy);
                orc_real Pxy = (PP(1, 1) - PP(1, -1) - PP(-1, 1) + PP(-1, -1)) / (4.0 * dx * dy);
#undef QQ
#undef PP
                fs = dd * dxd * Qy / 6.0 + dd * dyd * Qx / 6.0 + B3 * dd * dd * Qxy;
                gs = dd * dyd * Px / 6.0 + dd * dxd * Py / 6.0 + B3 * dd * dd * Pxy;
            }
            E[c] = e;
            F[c] = f;
            G[c] = gg;
            Fs[c] = fs;
            Gs[c] = gs;
        }
}

/* Eq. 23 coefficients of the line through cell c (spacing h, d, d_alpha). */
static void coef23(orc_real Bd, orc_real h, orc_real dd, orc_real dda, orc_real *a,
                   orc_real *b, orc_real *c)
{
    orc_real r = (Bd + 1.0 / 3.0) * dd * dd / (h * h);
    orc_real s = dd * dda / (6.0 * h);
    *a = s - r;
    *b = 1.0 + 2.0 * r;
    *c = -s - r;
}

/* U*, V* of Eq. 7-8 discretised exactly as the rows of Eq. 21-23, from P, Q
 * with their ghosts (Reading A-T3).  NLSW: U* = P, V* = Q. */
static void compute_ustar(orc *o, const orc_real *P, const orc_real *Q, orc_real *U,
                          orc_real *V)
{
    const int nx = o->nx, ny = o->ny;
    const size_t ex = (size_t)o->ex;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            size_t c = IX(o, i, j);
            if (o->p.model != ORC_BSNQ) {
                U[c] = P[c];
                V[c] = Q[c];
                continue;
            }
            orc_real a, b, cc;
            coef23(o->p.Bd, o->p.dx, o->d[c], o->ddx[c], &a, &b, &cc);
            U[c] = a * P[c - 1] + b * P[c] + cc * P[c + 1];
            coef23(o->p.Bd, o->p.dy, o->d[c], o->ddy[c], &a, &b, &cc);
            V[c] = a * Q[c - ex] + b * Q[c] + cc * Q[c + ex];
        }
}

/* Eq. 21 per x-row (dir 0) or Eq. 22 per y-column (dir 1), Thomas.  Boundary
 * rows (Reading A-B2): a solid or sponge end uses the mirror P_{-1} = -P_0;
 * a sine end moves the known ghost discharge at t1 to the right side. */
static void solve_lines(orc *o, int dir, const orc_real *R, orc_real *X, orc_real t1)
{
    const int nx = o->nx, ny = o->ny;
    const int n = dir == 0 ? nx : ny, nl = dir == 0 ? ny : nx;
    const orc_real h = dir == 0 ? o->p.dx : o->p.dy;
    const orc_bc *lo = &o->bc[dir == 0 ? ORC_W : ORC_S];
    const orc_bc *hi = &o->bc[dir == 0 ? ORC_E : ORC_N];
#pragma omp parallel
    {
        orc_real *a = (orc_real *)malloc(sizeof(orc_real) * (size_t)n * 7);
        orc_real *b = a + n, *c = b + n, *r = c + n, *x = r + n, *cp = x + n, *dp = cp + n;
#pragma omp for schedule(static)
        for (int l = 0; l < nl; l++) {
            for (int k = 0; k < n; k++) {
                int i = dir == 0 ? k : l, j = dir == 0 ? l : k;
                size_t cc = IX(o, i, j);
                coef23(o->p.Bd, h, o->d[cc], dir == 0 ? o->ddx[cc] : o->ddy[cc],
                       &a[k], &b[k], &c[k]);
                r[k] = R[cc];
            }
            for (int end = 0; end < 2; end++) {
                const orc_bc *bc = end == 0 ? lo : hi;
                int k = end == 0 ? 0 : n - 1;
                orc_real *off = end == 0 ? &a[0] : &c[n - 1];
                if (bc->type == ORC_SINE) {
                    int gk = end == 0 ? -1 : n;
                    int gi = dir == 0 ? gk : l, gj = dir == 0 ? l : gk;
                    int ai = dir == 0 ? k : l, aj = dir == 0 ? l : k;
                    orc_real eta, Pg, Qg;
                    sine_eval(o, bc, o->d[IX(o, ai, aj)], (gi + 0.5) * o->p.dx,
                              (gj + 0.5) * o->p.dy, t1, &eta, &Pg, &Qg);
                    r[k] -= *off * (dir == 0 ? Pg : Qg);
                } else {
                    b[k] -= *off;
                }
                *off = 0.0;
            }
            thomas_ws(n, a, b, c, r, x, cp, dp);
            for (int k = 0; k < n; k++) {
                int i = dir == 0 ? k : l, j = dir == 0 ? l : k;
                X[IX(o, i, j)] = x[k];
            }
        }
        free(a);
    }
}

/* Reading A-D1: AB3 is not positivity preserving, so w is clamped to the
 * bed after each update and P, Q are zeroed where the depth is zero.  The
 * mass the clamp adds is recorded for the last stage only (count = 1): each
 * corrector starts again from w^n, so what an earlier stage's clamp added
 * never reaches w^{n+1}. */
static void clamp_w(orc *o, orc_real *w, int count)
{
    orc_real added = 0.0;
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j);
            if (w[c] < o->Bbar[c]) {
                added += o->Bbar[c] - w[c];
                w[c] = o->Bbar[c];
            }
        }
    if (count) o->clamp_mass += added * o->p.dx * o->p.dy;
}

static void dry_zero(orc *o, const orc_real *w, orc_real *P, orc_real *Q)
{
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j);
            if (w[c] - o->Bbar[c] <= 0.0) {
                P[c] = 0.0;
                Q[c] = 0.0;
            }
        }
}

static void record_gauges(orc *o)
{
    if (o->ng <= 0 || o->log_every <= 0 || o->cap <= 0) return;
    if (o->step % o->log_every != 0) return;
    int slot = (o->head + o->nrec) % o->cap;
    if (o->nrec == o->cap) { /* full: keep the newest capacity records */
        slot = o->head;
        o->head = (o->head + 1) % o->cap;
    } else {
        o->nrec++;
    }
    for (int gk = 0; gk < o->ng; gk++) {
        int i = o->gij[2 * gk], j = o->gij[2 * gk + 1];
        o->grec[(size_t)slot * o->ng + gk] = o->w[IX(o, i, j)] - o->p.ws;
    }
}

/* Run-up tracking (Sec. 4.1, 4.3): the highest w seen at each cell while its
 * depth w - Bbar exceeded the threshold delta; -inf where it never did.
 * start = 1 sets the field from the present state. */
static void track_runup(orc *o, int start)
{
    if (!o->maxw) return;
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j), k = (size_t)j * o->nx + i;
            int wet = o->w[c] - o->Bbar[c] > o->delta;
            if (start) o->maxw[k] = wet ? o->w[c] : -INFINITY;
            else if (wet && o->w[c] > o->maxw[k]) o->maxw[k] = o->w[c];
        }
}

/* -------------------------------------------------------------- the step */

static void swap3(orc_real **h)
{
    orc_real *t = h[2];
    h[2] = h[1];
    h[1] = h[0];
    h[0] = t;
}

int orc_step(orc *o, int nsteps)
{
    if (!o || nsteps < 0) return -1;
    const int nx = o->nx, ny = o->ny;
    const orc_real dt = o->p.dt;
    const int bsnq = o->p.model == ORC_BSNQ;
    for (int s = 0; s < nsteps; s++) {
        orc_real t0 = (orc_real)o->step * dt, t1 = (orc_real)(o->step + 1) * dt;
        fill_ghosts(o, o->w, o->P, o->Q, t0);
        compute_rhs(o, o->w, o->P, o->Q, o->E[0], o->F[0], o->G[0], o->Fs[0], o->Gs[0]);
        compute_ustar(o, o->P, o->Q, o->U, o->V);
        /* Sec. 2.3: forward Euler for the first two steps after a (re)start,
         * the AM4 corrector only once AB3 runs (Reading A-T1, A-T2). */
        const int Kn = o->nh >= 2 ? o->p.K : 0;
        for (int stage = 0; stage <= Kn; stage++) {
            if (stage == 0) {
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        size_t c = IX(o, i, j);
                        if (o->nh == 0) { /* Euler; F* increment zero */
                            o->w1[c] = o->w[c] + dt * o->E[0][c];
                            o->U1[c] = o->U[c] + dt * o->F[0][c];
                            o->V1[c] = o->V[c] + dt * o->G[0][c];
                        } else if (o->nh == 1) { /* Euler; F*^1 - F*^0 */
                            o->w1[c] = o->w[c] + dt * o->E[0][c];
                            o->U1[c] = o->U[c] + dt * o->F[0][c] + (o->Fs[0][c] - o->Fs[1][c]);
                            o->V1[c] = o->V[c] + dt * o->G[0][c] + (o->Gs[0][c] - o->Gs[1][c]);
                        } else { /* Eq. 15-17 */
                            o->w1[c] = o->w[c] + dt / 12.0 *
                                (23.0 * o->E[0][c] - 16.0 * o->E[1][c] + 5.0 * o->E[2][c]);
                            o->U1[c] = o->U[c] + dt / 12.0 *
                                (23.0 * o->F[0][c] - 16.0 * o->F[1][c] + 5.0 * o->F[2][c]) +
                                2.0 * o->Fs[0][c] - 3.0 * o->Fs[1][c] + o->Fs[2][c];
                            o->V1[c] = o->V[c] + dt / 12.0 *
                                (23.0 * o->G[0][c] - 16.0 * o->G[1][c] + 5.0 * o->G[2][c]) +
                                2.0 * o->Gs[0][c] - 3.0 * o->Gs[1][c] + o->Gs[2][c];
                        }
                    }
            } else { /* Eq. 18-20 at the previous iterate */
                fill_ghosts(o, o->w1, o->P1, o->Q1, t1);
                compute_rhs(o, o->w1, o->P1, o->Q1, o->Ec, o->Fc, o->Gc, o->Fsc, o->Gsc);
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        size_t c = IX(o, i, j);
                        o->w1[c] = o->w[c] + dt / 24.0 *
                            (9.0 * o->Ec[c] + 19.0 * o->E[0][c] - 5.0 * o->E[1][c] + o->E[2][c]);
                        o->U1[c] = o->U[c] + dt / 24.0 *
                            (9.0 * o->Fc[c] + 19.0 * o->F[0][c] - 5.0 * o->F[1][c] + o->F[2][c]) +
                            o->Fsc[c] - o->Fs[0][c];
                        o->V1[c] = o->V[c] + dt / 24.0 *
                            (9.0 * o->Gc[c] + 19.0 * o->G[0][c] - 5.0 * o->G[1][c] + o->G[2][c]) +
                            o->Gsc[c] - o->Gs[0][c];
                    }
            }
            clamp_w(o, o->w1, stage == Kn);
            if (bsnq) {
                solve_lines(o, 0, o->U1, o->P1, t1);
                solve_lines(o, 1, o->V1, o->Q1, t1);
            } else {
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        size_t c = IX(o, i, j);
                        o->P1[c] = o->U1[c];
                        o->Q1[c] = o->V1[c];
                    }
            }
            if (stage == Kn) { /* Eq. 30 once per step (Reading A-B3) */
                for (int j = 0; j < ny; j++)
                    for (int i = 0; i < nx; i++) {
                        orc_real gam = sponge_at(o, i, j);
                        if (gam >= 1.0) continue;
                        size_t c = IX(o, i, j);
                        if (o->d[c] > 0.0) o->w1[c] = o->p.ws + gam * (o->w1[c] - o->p.ws);
                        o->P1[c] *= gam;
                        o->Q1[c] *= gam;
                    }
            }
            dry_zero(o, o->w1, o->P1, o->Q1);
        }
        swap3(o->E); swap3(o->F); swap3(o->G); swap3(o->Fs); swap3(o->Gs);
        orc_real *t;
        t = o->w; o->w = o->w1; o->w1 = t;
        t = o->P; o->P = o->P1; o->P1 = t;
        t = o->Q; o->Q = o->Q1; o->Q1 = t;
        o->step++;
        o->nh++;
        record_gauges(o);
        track_runup(o, 0);
    }
    return 0;
}

/* ------------------------------------------------------------------ API */

orc *orc_create(const orc_params *p, const orc_real *z)
{
    if (!p || !z || p->nx < 2 || p->ny < 2 || !(p->dx > 0) || !(p->dy > 0) ||
        !(p->dt > 0) || p->K < 0 || !(p->eps > 0))
        return NULL;
    orc *o = (orc *)calloc(1, sizeof(orc));
    o->p = *p;
    o->nx = p->nx;
    o->ny = p->ny;
    o->ex = p->nx + 4;
    o->ey = p->ny + 4;
    size_t ne = (size_t)o->ex * (size_t)o->ey;
    orc_real **cell[] = {&o->z, &o->Bbar, &o->d, &o->ddx, &o->ddy, &o->w, &o->P,
                       &o->Q, &o->w1, &o->P1, &o->Q1, &o->U, &o->V, &o->U1,
                       &o->V1, &o->Ec, &o->Fc, &o->Gc, &o->Fsc, &o->Gsc};
    for (size_t k = 0; k < sizeof(cell) / sizeof(cell[0]); k++)
        *cell[k] = (orc_real *)calloc(ne, sizeof(orc_real));
    for (int k = 0; k < 3; k++) {
        o->E[k] = (orc_real *)calloc(ne, sizeof(orc_real));
        o->F[k] = (orc_real *)calloc(ne, sizeof(orc_real));
        o->G[k] = (orc_real *)calloc(ne, sizeof(orc_real));
        o->Fs[k] = (orc_real *)calloc(ne, sizeof(orc_real));
        o->Gs[k] = (orc_real *)calloc(ne, sizeof(orc_real));
        o->Hx[k] = (orc_real *)calloc((size_t)(p->nx + 1) * p->ny, sizeof(orc_real));
        o->Hy[k] = (orc_real *)calloc((size_t)p->nx * (p->ny + 1), sizeof(orc_real));
    }
    o->Bc = (orc_real *)calloc((size_t)(p->nx + 3) * (p->ny + 3), sizeof(orc_real));
    for (int s = 0; s < 4; s++) o->bc[s].type = ORC_SOLID;
    derive_static(o, z);
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j);
            o->w[c] = fmax(p->ws, o->Bbar[c]);
        }
    return o;
}

void orc_destroy(orc *o)
{
    if (!o) return;
    orc_real *cell[] = {o->z, o->Bbar, o->d, o->ddx, o->ddy, o->w, o->P, o->Q,
                      o->w1, o->P1, o->Q1, o->U, o->V, o->U1, o->V1, o->Ec,
                      o->Fc, o->Gc, o->Fsc, o->Gsc, o->Bc};
    for (size_t k = 0; k < sizeof(cell) / sizeof(cell[0]); k++) free(cell[k]);
    for (int k = 0; k < 3; k++) {
        free(o->E[k]); free(o->F[k]); free(o->G[k]); free(o->Fs[k]);
        free(o->Gs[k]); free(o->Hx[k]); free(o->Hy[k]);
    }
    free(o->gij);
    free(o->grec);
    free(o->maxw);
    free(o);
}

int orc_set_boundary(orc *o, int side, const orc_bc *bc)
{
    if (!o || !bc || side < 0 || side > 3 || bc->type < ORC_SOLID ||
        bc->type > ORC_SINE || bc->ncomp < 0 || bc->ncomp > 8 || bc->width < 0)
        return -1;
    o->bc[side] = *bc;
    return 0;
}

int orc_set_state(orc *o, const orc_real *w, const orc_real *P, const orc_real *Q)
{
    if (!o || !w || !P || !Q) return -1;
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j), k = (size_t)j * o->nx + i;
            o->w[c] = fmax(w[k], o->Bbar[c]);
            o->P[c] = P[k];
            o->Q[c] = Q[k];
        }
    dry_zero(o, o->w, o->P, o->Q);
    o->nh = 0;
    return 0;
}

/* Eq. 33-36 (Reading A-S1): d is the still-water depth of the cell holding
 * the crest; the wave is added where d > 0. */
int orc_add_solitary(orc *o, orc_real H, orc_real theta, orc_real x0, orc_real y0)
{
    if (!o) return -1;
    int ic = (int)floor(x0 / o->p.dx), jc = (int)floor(y0 / o->p.dy);
    ic = ic < 0 ? 0 : (ic > o->nx - 1 ? o->nx - 1 : ic);
    jc = jc < 0 ? 0 : (jc > o->ny - 1 ? o->ny - 1 : jc);
    orc_real ds = o->d[IX(o, ic, jc)];
    if (!(ds > 0.0) || !(H + ds > 0.0)) return -1;
    orc_real ks = sqrt(3.0 * fabs(H) / (4.0 * ds * ds * ds));
    orc_real cs = sqrt(o->p.g * (H + ds));
    orc_real ct = cos(theta), st = sin(theta);
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j);
            if (!(o->d[c] > 0.0)) continue;
            orc_real xi = ((i + 0.5) * o->p.dx - x0) * ct + ((j + 0.5) * o->p.dy - y0) * st;
            orc_real sh = 1.0 / cosh(ks * xi);
            orc_real es = H * sh * sh;
            o->w[c] = fmax(o->w[c] + es, o->Bbar[c]);
            o->P[c] += cs * es * ct;
            o->Q[c] += cs * es * st;
        }
    dry_zero(o, o->w, o->P, o->Q);
    o->nh = 0;
    return 0;
}

void orc_get_state(const orc *o, orc_real *w, orc_real *P, orc_real *Q)
{
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j), k = (size_t)j * o->nx + i;
            if (w) w[k] = o->w[c];
            if (P) P[k] = o->P[c];
            if (Q) Q[k] = o->Q[c];
        }
}

int orc_get_field(const orc *o, int which, orc_real *out)
{
    const orc_real *src = which == 0 ? o->Bbar : which == 1 ? o->d
                        : which == 2 ? o->U : which == 3 ? o->V : NULL;
    if (!src || !out) return -1;
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) out[(size_t)j * o->nx + i] = src[IX(o, i, j)];
    return 0;
}

void orc_get_time(const orc *o, orc_real *t, long long *step)
{
    if (t) *t = (orc_real)o->step * o->p.dt;
    if (step) *step = o->step;
}

orc_real orc_mass(const orc *o)
{
    orc_real m = 0.0;
    for (int j = 0; j < o->ny; j++)
        for (int i = 0; i < o->nx; i++) {
            size_t c = IX(o, i, j);
            m += o->w[c] - o->Bbar[c];
        }
    return m * o->p.dx * o->p.dy;
}

orc_real orc_clamp_mass(const orc *o) { return o->clamp_mass; }

int orc_set_gauges(orc *o, const int *ij, int n, int log_every, int capacity)
{
    if (!o || n < 0 || (n > 0 && !ij) || log_every < 0 || capacity < 0) return -1;
    for (int k = 0; k < n; k++)
        if (ij[2 * k] < 0 || ij[2 * k] >= o->nx || ij[2 * k + 1] < 0 || ij[2 * k + 1] >= o->ny)
            return -1;
    free(o->gij);
    free(o->grec);
    o->gij = n ? (int *)malloc(sizeof(int) * 2 * (size_t)n) : NULL;
    if (n) memcpy(o->gij, ij, sizeof(int) * 2 * (size_t)n);
    o->grec = (n && capacity) ? (orc_real *)calloc((size_t)n * capacity, sizeof(orc_real)) : NULL;
    o->ng = n;
    o->log_every = log_every;
    o->cap = capacity;
    o->nrec = 0;
    o->head = 0;
    return 0;
}

int orc_read_gauges(orc *o, orc_real *eta, int max_rec, int *n_rec)
{
    if (!o || !n_rec || max_rec < 0) return -1;
    int n = o->nrec < max_rec ? o->nrec : max_rec;
    for (int r = 0; r < n; r++) {
        int slot = (o->head + r) % (o->cap ? o->cap : 1);
        for (int gk = 0; gk < o->ng; gk++)
            eta[(size_t)r * o->ng + gk] = o->grec[(size_t)slot * o->ng + gk];
    }
    o->head = o->cap ? (o->head + n) % o->cap : 0;
    o->nrec -= n;
    *n_rec = n;
    return 0;
}

int orc_runup_enable(orc *o, orc_real delta)
{
    if (!o || !(delta >= 0.0)) return -1;
    if (!o->maxw) o->maxw = (orc_real *)malloc(sizeof(orc_real) * (size_t)o->nx * o->ny);
    o->delta = delta;
    track_runup(o, 1);
    return 0;
}

int orc_runup_read(const orc *o, orc_real *maxw)
{
    if (!o || !o->maxw || !maxw) return -1;
    memcpy(maxw, o->maxw, sizeof(orc_real) * (size_t)o->nx * o->ny);
    return 0;
}
