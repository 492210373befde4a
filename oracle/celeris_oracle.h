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

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BSNQ = 0, ORC_NLSW = 1 };                       /* model (Sec. 3.2) */
enum { ORC_FRIC_NONE = 0, ORC_FRIC_QUAD = 1, ORC_FRIC_MANNING = 2 }; /* Sec. 2.6 */
enum { ORC_SOLID = 0, ORC_SPONGE = 1, ORC_SINE = 2 };      /* Sec. 2.4 */
enum { ORC_W = 0, ORC_E = 1, ORC_S = 2, ORC_N = 3 };        /* boundary sides */

typedef struct {
    int nx, ny;          /* interior cells                                     */
    double dx, dy;       /* cell sizes                                         */
    int model;           /* ORC_BSNQ | ORC_NLSW                                */
    double g;            /* gravity                                            */
    double Bd;           /* dispersion calibration B (Eq. 2, 1/15)             */
    double theta;        /* generalized-minmod parameter (KP07 step 1)         */
    double eps;          /* desingularisation tolerance (Eq. 14)               */
    double dt;           /* fixed time step                                    */
    int K;               /* AM4 corrector iterations (Sec. 2.3)                */
    double ws;           /* still-water elevation w_s                          */
    int friction;        /* ORC_FRIC_*                                         */
    double fcoef;        /* f (quadratic) or Manning n                         */
} orc_params;

typedef struct {
    int type;            /* ORC_SOLID | ORC_SPONGE | ORC_SINE                  */
    int width;           /* sponge width in cells (Eq. 30, L_s = width * d)    */
    int ncomp;           /* sine components summed (0..8)                      */
    double amp[8], period[8], dir[8], phase[8]; /* a, T, theta [rad], phase    */
} orc_bc;

typedef struct orc orc;

/* Create with cell-centre bed elevation z[ny][nx].  All sides start SOLID,
 * state starts at rest (w = max(w_s, Bbar), P = Q = 0).  NULL on bad input. */
orc *orc_create(const orc_params *p, const double *z);
void orc_destroy(orc *o);
int orc_set_boundary(orc *o, int side, const orc_bc *bc);
/* Copies w,P,Q; clamps w >= Bbar; zeroes P,Q in dry cells; restarts AB3. */
int orc_set_state(orc *o, const double *w, const double *P, const double *Q);
/* Superposes a solitary wave (Eq. 33-36); restarts AB3.  -1 if d=0 at crest. */
int orc_add_solitary(orc *o, double H, double theta, double x0, double y0);
int orc_step(orc *o, int nsteps);
void orc_get_state(const orc *o, double *w, double *P, double *Q);
/* which: 0 = Bbar, 1 = d, 2 = U* (last step), 3 = V* (last step) */
int orc_get_field(const orc *o, int which, double *out);
void orc_get_time(const orc *o, double *t, long long *step);
double orc_mass(const orc *o);        /* sum (w - Bbar) dx dy over interior */
double orc_clamp_mass(const orc *o);  /* mass added by the w >= Bbar clamp */
int orc_set_gauges(orc *o, const int *ij, int n, int log_every, int capacity);
int orc_read_gauges(orc *o, double *eta, int max_rec, int *n_rec);
int orc_num_threads(void);
/* Run-up tracking (Sec. 4.1, 4.3): after every step, maxw[j][i] = the highest
 * w seen while the cell's depth w - Bbar exceeded delta (-inf if never);
 * enable starts it from the present state, read copies it out ([ny][nx]). */
int orc_runup_enable(orc *o, double delta);
int orc_runup_read(const orc *o, double *maxw);

/* Building blocks exported so tests can pin them one by one. */
double orc_minmod(double theta, double qm, double q0, double qp);
double orc_eckart_k(double omega, double d, double g);           /* Eq. 29 */
double orc_sponge_gamma(double D, double Ls);                    /* Eq. 30 */
void orc_thomas(int n, const double *a, const double *b, const double *c,
                const double *r, double *x);                     /* textbook */
void orc_central_upwind(double g, double eps, double wL, double nL, double tL,
                        double wR, double nR, double tR, double Bf,
                        double H[3]);                            /* KP07 step 3 */

#ifdef __cplusplus
}
#endif
#endif
