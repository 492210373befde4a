/*
 * celeris_tlm.cpp -- tangent-linear version of the FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY (like the oracle it is built from; only the test
 * suite loads it).  The oracle's own source, celeris_oracle.c, is compiled
 * here a second time with its arithmetic type set to a forward-mode dual
 * number: every value carries its derivative along one direction of the
 * inputs (the bed z and the initial state), propagated operation by
 * operation through exactly the oracle's arithmetic and branches.  So the
 * tangent of a run is the exact directional derivative of the oracle's
 * result -- the tangent-linear reference a discrete adjoint is checked
 * against: <dL/dx, v> from the adjoint must equal dL(x; v) from here.
 *
 * Branches follow the values, as the oracle takes them; at a tie, max and
 * min keep their first argument; sqrt and cbrt have derivative 0 at 0.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

struct orc_dual {
    double v, d;
    orc_dual() = default;
    constexpr orc_dual(double x) : v(x), d(0.0) {}
    constexpr orc_dual(double x, double dx) : v(x), d(dx) {}
    explicit operator int() const { return (int)v; }
    orc_dual &operator+=(orc_dual b)
    {
        v += b.v;
        d += b.d;
        return *this;
    }
    orc_dual &operator-=(orc_dual b)
    {
        v -= b.v;
        d -= b.d;
        return *this;
    }
    orc_dual &operator*=(orc_dual b)
    {
        d = d * b.v + v * b.d;
        v *= b.v;
        return *this;
    }
};

static inline orc_dual operator+(orc_dual a, orc_dual b) { return {a.v + b.v, a.d + b.d}; }
static inline orc_dual operator-(orc_dual a, orc_dual b) { return {a.v - b.v, a.d - b.d}; }
static inline orc_dual operator-(orc_dual a) { return {-a.v, -a.d}; }
static inline orc_dual operator*(orc_dual a, orc_dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
static inline orc_dual operator/(orc_dual a, orc_dual b)
{
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
static inline bool operator<(orc_dual a, orc_dual b) { return a.v < b.v; }
static inline bool operator>(orc_dual a, orc_dual b) { return a.v > b.v; }
static inline bool operator<=(orc_dual a, orc_dual b) { return a.v <= b.v; }
static inline bool operator>=(orc_dual a, orc_dual b) { return a.v >= b.v; }
static inline bool operator==(orc_dual a, orc_dual b) { return a.v == b.v; }
static inline bool operator!=(orc_dual a, orc_dual b) { return a.v != b.v; }

static inline orc_dual fmax(orc_dual a, orc_dual b) { return a.v >= b.v ? a : b; }
static inline orc_dual fmin(orc_dual a, orc_dual b) { return a.v <= b.v ? a : b; }
static inline orc_dual fabs(orc_dual a) { return a.v < 0.0 ? -a : a; }
static inline orc_dual floor(orc_dual a) { return {::floor(a.v), 0.0}; }
static inline orc_dual sqrt(orc_dual a)
{
    const double s = ::sqrt(a.v);
    return {s, s > 0.0 ? a.d / (2.0 * s) : 0.0};
}
static inline orc_dual cbrt(orc_dual a)
{
    const double c = ::cbrt(a.v);
    return {c, c != 0.0 ? a.d / (3.0 * c * c) : 0.0};
}
static inline orc_dual sin(orc_dual a) { return {::sin(a.v), ::cos(a.v) * a.d}; }
static inline orc_dual cos(orc_dual a) { return {::cos(a.v), -::sin(a.v) * a.d}; }
static inline orc_dual cosh(orc_dual a) { return {::cosh(a.v), ::sinh(a.v) * a.d}; }
static inline orc_dual tanh(orc_dual a)
{
    const double t = ::tanh(a.v);
    return {t, (1.0 - t * t) * a.d};
}

#define ORC_REAL orc_dual
#define ORC_NO_EXTERN_C
namespace tlm {
#include "celeris_oracle.c"
}

// A plain-double C ABI over the dual-number oracle: every real input comes
// as a value array and a tangent array, every real output likewise.
extern "C" {

// the layouts of orc_params and orc_bc with double fields
struct tlm_params {
    int nx, ny;
    double dx, dy;
    int model;
    double g, Bd, theta, eps, dt;
    int K;
    double ws;
    int friction;
    double fcoef;
};

struct tlm_bc {
    int type, width, ncomp;
    double amp[8], period[8], dir[8], phase[8];
};

static orc_dual *duals(const double *v, const double *d, size_t n)
{
    orc_dual *x = (orc_dual *)malloc(sizeof(orc_dual) * (n ? n : 1));
    for (size_t k = 0; k < n; k++) x[k] = orc_dual(v[k], d ? d[k] : 0.0);
    return x;
}

void *tlm_create(const tlm_params *p, const double *z, const double *dz)
{
    tlm::orc_params q;
    q.nx = p->nx;
    q.ny = p->ny;
    q.dx = p->dx;
    q.dy = p->dy;
    q.model = p->model;
    q.g = p->g;
    q.Bd = p->Bd;
    q.theta = p->theta;
    q.eps = p->eps;
    q.dt = p->dt;
    q.K = p->K;
    q.ws = p->ws;
    q.friction = p->friction;
    q.fcoef = p->fcoef;
    orc_dual *zd = duals(z, dz, (size_t)p->nx * p->ny);
    tlm::orc *o = tlm::orc_create(&q, zd);
    free(zd);
    return o;
}

void tlm_destroy(void *o) { tlm::orc_destroy((tlm::orc *)o); }

int tlm_set_boundary(void *o, int side, const tlm_bc *b)
{
    tlm::orc_bc c;
    c.type = b->type;
    c.width = b->width;
    c.ncomp = b->ncomp;
    for (int m = 0; m < 8; m++) {
        c.amp[m] = b->amp[m];
        c.period[m] = b->period[m];
        c.dir[m] = b->dir[m];
        c.phase[m] = b->phase[m];
    }
    return tlm::orc_set_boundary((tlm::orc *)o, side, &c);
}

int tlm_set_state(void *o, int n, const double *w, const double *dw, const double *P, const double *dP,
                  const double *Q, const double *dQ)
{
    orc_dual *a = duals(w, dw, (size_t)n), *b = duals(P, dP, (size_t)n), *c = duals(Q, dQ, (size_t)n);
    const int r = tlm::orc_set_state((tlm::orc *)o, a, b, c);
    free(a);
    free(b);
    free(c);
    return r;
}

int tlm_set_gauges(void *o, const int *ij, int n, int log_every, int capacity)
{
    return tlm::orc_set_gauges((tlm::orc *)o, ij, n, log_every, capacity);
}

int tlm_step(void *o, int nsteps) { return tlm::orc_step((tlm::orc *)o, nsteps); }

int tlm_read_gauges(void *o, double *eta, double *deta, int max_rec, int ng, int *n_rec)
{
    orc_dual *e = (orc_dual *)malloc(sizeof(orc_dual) * (size_t)(max_rec > 0 ? max_rec : 1) * (ng > 0 ? ng : 1));
    const int r = tlm::orc_read_gauges((tlm::orc *)o, e, max_rec, n_rec);
    if (r == 0)
        for (int k = 0; k < *n_rec * ng; k++) {
            eta[k] = e[k].v;
            deta[k] = e[k].d;
        }
    free(e);
    return r;
}

}  // extern "C"
