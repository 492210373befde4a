/*
 * celeris_oracle.h -- FP64 CPU oracle of the extended-Boussinesq time step
 * (Tavakkol & Lynett, "Celeris", arXiv 1611.05984).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA library: every formula here is written out again
 * from the paper (section / equation numbers are cited at each function).
 *
 * Conventions: SI units; interior arrays are row-major [ny][nx] doubles;
 * cell (i,j) has its centre at ((i+1/2)dx, (j+1/2)dy).
 */
#ifndef CELERIS_ORACLE_H
#define CELERIS_ORACLE_H

/* The arithmetic type: double.  The tangent-linear build (celeris_tlm.cpp)
 * compiles this same source with a forward-mode dual number in its place, so
 * its tangents are the exact derivatives of these operations. */
#ifndef ORC_REAL
#define ORC_REAL double
#endif
typedef ORC_REAL orc_real;

#if defined(__cplusplus) && !defined(ORC_NO_EXTERN_C)
extern "C" {
#endif

enum { ORC_BSNQ = 0, ORC_NLSW = 1 };                       /* model (Sec. 3.2) */
enum { ORC_FRIC_NONE = 0, ORC_FRIC_QUAD = 1, ORC_FRIC_MANNING = 2 }; /* Sec. 2.6 */
enum { ORC_SOLID = 0, ORC_SPONGE = 1, ORC_SINE = 2 };      /* Sec. 2.4 */
enum { ORC_W = 0, ORC_E = 1, ORC_S = 2, ORC_N = 3 };        /* boundary sides */

typedef struct {
    int nx, ny;          /* interior cells                                     */
    orc_real dx, dy;       /* cell sizes                                         */
    int model;           /* ORC_BSNQ | ORC_NLSW                                */
    orc_real g;            /* gravity                                            */
    orc_real Bd;           /* dispersion calibration B (Eq. 2, 1/15)             */
    orc_real theta;        /* generalized-minmod parameter (KP07 step 1)         */
    orc_real eps;          /* desingularisation tolerance (Eq. 14)               */
    orc_real dt;           /* fixed time step                                    */
    int K;               /* AM4 corrector iterations (Sec. 2.3)                */
    orc_real ws;           /* still-water elevation w_s                          */
    int friction;        /* ORC_FRIC_*                                         */
    orc_real fcoef;        /* f (quadratic) or Manning n                         */
} orc_params;

typedef struct {
    int type;            /* ORC_SOLID | ORC_SPONGE | ORC_SINE                  */
    int width;           /* sponge width in cells (Eq. 30, L_s = width * d)    */
    int ncomp;           /* sine components summed (0..8)                      */
    orc_real amp[8], period[8], dir[8], phase[8]; /* a, T, theta [rad], phase    */
} orc_bc;

typedef struct orc orc;

/* Create with cell-centre bed elevation z[ny][nx].  All sides start SOLID,
 * state starts at rest (w = max(w_s, Bbar), P = Q = 0).  NULL on bad input. */
orc *orc_create(const orc_params *p, const orc_real *z);
void orc_destroy(orc *o);
int orc_set_boundary(orc *o, int side, const orc_bc *bc);
/* Copies w,P,Q; clamps w >= Bbar; zeroes P,Q in dry cells; restarts AB3. */
int orc_set_state(orc *o, const orc_real *w, const orc_real *P, const orc_real *Q);
/* Superposes a solitary wave (Eq. 33-36); restarts AB3.  -1 if d=0 at crest. */
int orc_add_solitary(orc *o, orc_real H, orc_real theta, orc_real x0, orc_real y0);
int orc_step(orc *o, int nsteps);
void orc_get_state(const orc *o, orc_real *w, orc_real *P, orc_real *Q);
/* which: 0 = Bbar, 1 = d, 2 = U* (last step), 3 = V* (last step) */
int orc_get_field(const orc *o, int which, orc_real *out);
void orc_get_time(const orc *o, orc_real *t, long long *step);
orc_real orc_mass(const orc *o);        /* sum (w - Bbar) dx dy over interior */
orc_real orc_clamp_mass(const orc *o);  /* mass the w >= Bbar clamp added to w^{n+1} */
int orc_set_gauges(orc *o, const int *ij, int n, int log_every, int capacity);
int orc_read_gauges(orc *o, orc_real *eta, int max_rec, int *n_rec);
int orc_num_threads(void);
/* Run-up tracking (Sec. 4.1, 4.3): after every step, maxw[j][i] = the highest
 * w seen while the cell's depth w - Bbar exceeded delta (-inf if never);
 * enable starts it from the present state, read copies it out ([ny][nx]). */
int orc_runup_enable(orc *o, orc_real delta);
int orc_runup_read(const orc *o, orc_real *maxw);

/* Building blocks exported so tests can pin them one by one. */
orc_real orc_minmod(orc_real theta, orc_real qm, orc_real q0, orc_real qp);
orc_real orc_eckart_k(orc_real omega, orc_real d, orc_real g);           /* Eq. 29 */
orc_real orc_sponge_gamma(orc_real D, orc_real Ls);                    /* Eq. 30 */
void orc_thomas(int n, const orc_real *a, const orc_real *b, const orc_real *c,
                const orc_real *r, orc_real *x);                     /* textbook */
void orc_central_upwind(orc_real g, orc_real eps, orc_real wL, orc_real nL, orc_real tL,
                        orc_real wR, orc_real nR, orc_real tR, orc_real Bf,
                        orc_real H[3]);                            /* KP07 step 3 */

#if defined(__cplusplus) && !defined(ORC_NO_EXTERN_C)
}
#endif
#endif
