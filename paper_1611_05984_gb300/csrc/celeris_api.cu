// C ABI of the Celeris step library (declared in include/celeris_gb.h).
//
// The handle keeps host metadata and pointers into the caller's workspace;
// the library never allocates device memory.  Every call returns a status and
// records the text of the last error in the handle.
#include "celeris_gb.h"
#include "celeris_internal.cuh"
#include "celeris_adjoint.cuh"

#include <nvtx3/nvToolsExt.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

using namespace cel;

namespace {

constexpr double kPiD = 3.14159265358979323846;
constexpr uint64_t kCkptMagic = 0x43454c4b50543031ull;   // "CELKPT01"

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
int round_up_i(int a, int b) { return (a + b - 1) / b * b; }

struct Layout {
    size_t w[2], P[2], U, dr, a[3], b[3][2];     // carries (K = 0)
    size_t R[3][3], Ph[3][3], Y[3];              // rings and AM4 bases (K >= 1)
    size_t Qc[2], Vc, dc, Bc, mr, mc, ghost, ktab, gam, flag;
    size_t total;
    size_t row_bytes, col_bytes;
};

Geo make_geo(const cel_grid &g)
{
    Geo G;
    G.nx = g.nx;
    G.ny = g.ny;
    G.px = round_up_i(g.nx, 32);
    G.py = round_up_i(g.ny, 32);
    G.pc = round_up_i(g.nx + 3, 32);
    G.nwx = (g.nx + 31) / 32;
    G.nwy = (g.ny + 31) / 32;
    G.dx = g.dx;
    G.dy = g.dy;
    return G;
}

Layout make_layout(const Geo &G, int es, int K)
{
    Layout L;
    memset(&L, 0, sizeof(L));
    size_t cur = 0;
    auto take = [&](size_t b) {
        size_t o = cur;
        cur += align256(b);
        return o;
    };
    L.row_bytes = (size_t)G.ny * G.px * es;
    L.col_bytes = (size_t)G.nx * G.py * es;
    L.w[0] = take(L.row_bytes);
    L.w[1] = take(L.row_bytes);
    L.P[0] = take(L.row_bytes);
    L.P[1] = take(L.row_bytes);
    L.U = take(L.row_bytes);
    L.dr = take(L.row_bytes);
    if (K == 0) {
        for (int v = 0; v < 3; v++) {
            L.a[v] = take(L.row_bytes);
            L.b[v][0] = take(L.row_bytes);
            L.b[v][1] = take(L.row_bytes);
        }
    } else {
        for (int v = 0; v < 3; v++) {
            for (int k = 0; k < 3; k++) L.R[v][k] = take(L.row_bytes);
            if (v > 0)
                for (int k = 0; k < 3; k++) L.Ph[v][k] = take(L.row_bytes);
            L.Y[v] = take(L.row_bytes);
        }
    }
    L.Qc[0] = take(L.col_bytes);
    L.Qc[1] = take(L.col_bytes);
    L.Vc = take(L.col_bytes);
    L.dc = take(L.col_bytes);
    L.Bc = take((size_t)(G.ny + 3) * G.pc * es);
    L.mr = take((size_t)G.ny * G.nwx * 4);
    L.mc = take((size_t)G.nx * G.nwy * 4);
    L.ghost = take(ghost_index(2, 0, 0, 0, 0, (G.nx > G.ny ? G.nx : G.ny) + 4) * es);
    L.ktab = take((size_t)4 * ((G.nx > G.ny ? G.nx : G.ny) + 4) * 8 * sizeof(double));
    L.gam = take((size_t)4 * ((G.nx > G.ny ? G.nx : G.ny) + 4) * es);
    L.flag = take(256);
    L.total = cur;
    return L;
}

bool grid_ok(const cel_grid *g)
{
    if (!g) return false;
    if (g->real_bytes != 4 && g->real_bytes != 8) return false;
    int mx = g->real_bytes == 4 ? CEL_MAX_LINE_F32 : CEL_MAX_LINE_F64;
    if (g->nx < 2 || g->ny < 2 || g->nx > mx || g->ny > mx) return false;
    if (!(g->dx > 0) || !(g->dy > 0) || !isfinite(g->dx) || !isfinite(g->dy)) return false;
    return true;
}

bool params_ok(const cel_params *p)
{
    if (!p) return false;
    if (p->model != CEL_BSNQ && p->model != CEL_NLSW) return false;
    if (p->friction < CEL_FRIC_NONE || p->friction > CEL_FRIC_MANNING) return false;
    if (!(p->g > 0) || !(p->dt > 0) || !(p->eps > 0) || !(p->Bdisp >= 0)) return false;
    if (!(p->theta >= 0 && p->theta <= 2.0)) return false;
    if (p->corrector_iters < 0 || p->corrector_iters > 64) return false;
    if (!isfinite(p->still_water) || !(p->fric_coef >= 0)) return false;
    return true;
}

// Optional per-kernel timing: CUDA event pairs recorded around launches.
struct EventProf {
    cudaEvent_t *beg = nullptr, *end = nullptr;
    int *kind = nullptr;
    int cap = 0, used = 0;

    void release()
    {
        for (int k = 0; k < cap; k++) {
            cudaEventDestroy(beg[k]);
            cudaEventDestroy(end[k]);
        }
        delete[] beg;
        delete[] end;
        delete[] kind;
        beg = end = nullptr;
        kind = nullptr;
        cap = used = 0;
    }
    cudaError_t create(int capacity)
    {
        release();
        beg = new cudaEvent_t[capacity];
        end = new cudaEvent_t[capacity];
        kind = new int[capacity];
        for (int k = 0; k < capacity; k++) {
            cudaError_t e1 = cudaEventCreate(&beg[k]);
            cudaError_t e2 = e1 == cudaSuccess ? cudaEventCreate(&end[k]) : e1;
            if (e2 != cudaSuccess) {
                if (e1 == cudaSuccess) cudaEventDestroy(beg[k]);
                cap = k;
                release();
                return e2;
            }
        }
        cap = capacity;
        used = 0;
        return cudaSuccess;
    }
    int begin(int kd, cudaStream_t st)
    {
        if (!cap || used >= cap) return -1;
        int k = used++;
        kind[k] = kd;
        cudaEventRecord(beg[k], st);
        return k;
    }
    void finish(int k, cudaStream_t st)
    {
        if (k >= 0) cudaEventRecord(end[k], st);
    }
    // summed milliseconds and counts per kind (0..2); synchronises the stream
    cudaError_t read(cudaStream_t st, double ms[3], int64_t count[3])
    {
        for (int k = 0; k < 3; k++) {
            ms[k] = 0.0;
            count[k] = 0;
        }
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        for (int k = 0; k < used; k++) {
            float t = 0.f;
            e = cudaEventElapsedTime(&t, beg[k], end[k]);
            if (e != cudaSuccess) return e;
            ms[kind[k]] += t;
            count[kind[k]] += 1;
        }
        used = 0;
        return cudaSuccess;
    }
};

}  // namespace

struct cel_solver {
    cel_grid grid;
    cel_params params;
    Geo geo;
    Phys phy;
    Bnd bnd;
    Layout lay;
    int es;
    cudaStream_t stream;
    unsigned char *ws;
    int cur;      // w buffer of the state (w alternates per stage)
    int pcur;     // P / Q buffer of the state (alternates per step)
    int64_t step, nh;
    // gauges
    int32_t *gij;
    unsigned char *gring;
    int ng, log_every, cap, nrec, head;
    int64_t launches;
    void *runup;      // caller's [ny][nx] run-up field, or NULL
    double runup_delta;
    // adjoint recomputation: where to copy the iterate after every stage but
    // the last ([stage][w, P, Q][ny][nx] dense), or NULL
    unsigned char *capture;
    size_t capture_field;
    // and where the line solves write their solutions of every stage
    // ([stage][U*, V* increments][line layout], capture_line bytes each), or NULL
    unsigned char *capture_rhs;
    size_t capture_line;
    int ktab_dirty;   // boundaries or bed changed: rebuild the Eckart table
    int gam_dirty;    // boundaries changed: rebuild the sponge factors
    uint64_t gen;     // counts boundary and bed changes (ensembles rebuild their tables)
    std::string err;
    EventProf prof;   // optional per-kernel event timing

    template <typename T>
    T *at(size_t off) const { return reinterpret_cast<T *>(ws + off); }
};

namespace {

cel_status fail(cel_solver *s, cel_status st, const std::string &msg)
{
    if (s) s->err = msg;
    return st;
}

cel_status cuda_fail(cel_solver *s, cudaError_t e, const char *where)
{
    return fail(s, CEL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CEL_CUDA(s, expr, where)                       \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_fail(s, e_, where); \
    } while (0)

// Each kernel kind of the step is also an NVTX range (stencil, line
// solves, ghost table), for profilers that filter by range; without a tool
// attached a range costs a few host nanoseconds.
const char *const kRangeName[3] = {"cel stencil", "cel line solves", "cel ghost table"};

int prof_begin(cel_solver *s, int kind)
{
    nvtxRangePushA(kRangeName[kind]);
    return s->prof.begin(kind, s->stream);
}

void prof_end(cel_solver *s, int k)
{
    s->prof.finish(k, s->stream);
    nvtxRangePop();
}

void prof_free(cel_solver *s) { s->prof.release(); }

template <typename real>
cel_status derive_static(cel_solver *s, const void *z)
{
    CEL_CUDA(s, launch_corners<real>(s->geo, (const real *)z, s->at<real>(s->lay.Bc), s->stream), "corners");
    CEL_CUDA(s, launch_static_cells<real>(s->geo, s->phy, s->at<real>(s->lay.Bc), s->at<real>(s->lay.dr),
                                          s->at<real>(s->lay.dc), s->stream), "static cells");
    return CEL_OK;
}

template <typename real>
cel_status set_state_t(cel_solver *s, const void *w, const void *P, const void *Q, int rest)
{
    s->cur = 0;
    s->pcur = 0;
    CEL_CUDA(s, launch_set_state<real>(s->geo, s->phy, s->at<real>(s->lay.Bc), (const real *)w,
                                       (const real *)P, (const real *)Q, s->at<real>(s->lay.w[0]),
                                       s->at<real>(s->lay.P[s->pcur]), s->at<real>(s->lay.Qc[s->pcur]), rest, s->stream),
             "set_state");
    s->nh = 0;
    return CEL_OK;
}

// Arguments of the stencil launch of one stage (stage 0: the predictor or an
// Euler step; stage >= 1: AM4 corrector iterations; Kn: last stage).
template <typename real>
StencilArgs<real> stencil_args(const cel_solver *s, const Coef<real> &coef, int stage, int Kn)
{
    const Layout &L = s->lay;
    const int K = s->params.corrector_iters;
    const int kind0 = s->nh == 0 ? kEuler0 : (s->nh == 1 ? kEuler1 : kAB3);
    const int slot = (int)(s->nh & 1);
    StencilArgs<real> a;
    memset(&a, 0, sizeof(a));
    a.geo = s->geo;
    a.phy = s->phy;
    a.c = coef;
    a.c.gam = s->at<real>(L.gam);
    a.ghost = s->at<real>(L.ghost);
    a.Bc = s->at<real>(L.Bc);
    a.w_in = s->at<real>(L.w[(s->cur + stage) & 1]);
    a.w_out = s->at<real>(L.w[(s->cur + stage + 1) & 1]);
    a.P_in = s->at<real>(L.P[stage == 0 ? s->pcur : 1 - s->pcur]);
    a.Qc_in = s->at<real>(L.Qc[stage == 0 ? s->pcur : 1 - s->pcur]);
    a.U_out = s->at<real>(L.U);
    a.Vc_out = s->at<real>(L.Vc);
    // ring slots: R^n goes to slot nh % 3, R^{n-1} and R^{n-2} before it
    const int s0 = (int)(s->nh % 3), s1 = (s0 + 2) % 3, s2 = (s0 + 1) % 3;
    for (int v = 0; v < 3; v++) {
        a.a[v] = K == 0 ? s->at<real>(L.a[v]) : nullptr;
        a.b[v] = K == 0 ? s->at<real>(L.b[v][slot]) : nullptr;
        a.R0[v] = K > 0 ? s->at<real>(L.R[v][s0]) : nullptr;
        a.R1[v] = K > 0 ? s->at<real>(L.R[v][s1]) : nullptr;
        a.R2[v] = K > 0 ? s->at<real>(L.R[v][s2]) : nullptr;
        a.F0[v] = K > 0 && v > 0 ? s->at<real>(L.Ph[v][s0]) : nullptr;
        a.F1[v] = K > 0 && v > 0 ? s->at<real>(L.Ph[v][s1]) : nullptr;
        a.F2[v] = K > 0 && v > 0 ? s->at<real>(L.Ph[v][s2]) : nullptr;
        a.Y[v] = K > 0 ? s->at<real>(L.Y[v]) : nullptr;
    }
    a.mask_r = s->at<uint32_t>(L.mr);
    a.mask_c = s->at<uint32_t>(L.mc);
    a.kind = stage == 0 ? kind0 : kAM4;
    a.ring = K > 0;
    a.final_stage = stage == Kn;
    a.tsel = stage == 0 ? 0 : 1;
    return a;
}

// Arguments of the x-line (dir 0) or y-line (dir 1) solves of one stage.
template <typename real>
LineArgs<real> line_args(const cel_solver *s, const Coef<real> &coef, int dir, int stage, int Kn)
{
    const Layout &L = s->lay;
    LineArgs<real> l;
    memset(&l, 0, sizeof(l));
    l.geo = s->geo;
    l.phy = s->phy;
    l.c = coef;
    l.c.gam = s->at<real>(L.gam);
    l.ghost = s->at<real>(L.ghost);
    const double h = dir == 0 ? s->geo.dx : s->geo.dy;
    l.rh = real(1.0 / h);
    l.rh2 = real(1.0 / (h * h));
    l.hrh = real(0.5 / h);
    l.srh = real(1.0 / (6.0 * h));
    l.rhs = s->at<real>(dir == 0 ? L.U : L.Vc);
    l.d = s->at<real>(dir == 0 ? L.dr : L.dc);
    l.mask = s->at<uint32_t>(dir == 0 ? L.mr : L.mc);
    l.base = s->at<real>(dir == 0 ? L.P[s->pcur] : L.Qc[s->pcur]);
    l.sol = s->at<real>(dir == 0 ? L.P[1 - s->pcur] : L.Qc[1 - s->pcur]);
    l.dir = dir;
    l.n = dir == 0 ? s->geo.nx : s->geo.ny;
    l.nlines = dir == 0 ? s->geo.ny : s->geo.nx;
    l.pitch = dir == 0 ? s->geo.px : s->geo.py;
    l.nwords = dir == 0 ? s->geo.nwx : s->geo.nwy;
    const LineCfg lc = line_config(l.n, s->es);
    l.algo = lc.algo;
    l.nseg = lc.nseg;
    l.mshift = lc.mshift;
    l.sp = lc.sp;
    l.final_stage = stage == Kn;
    l.identity = s->params.model == CEL_NLSW;
    return l;
}

// Stages of the step about to be taken: AM4 iterations only once the AB3
// history holds two earlier steps.
int stages_of(const cel_solver *s) { return (s->nh >= 2 ? s->params.corrector_iters : 0) + 1; }

// Counters after a step of Kn + 1 stages: w alternates per stage, P / Q per step.
void finish_step(cel_solver *s, int Kn)
{
    s->cur = (s->cur + Kn + 1) & 1;
    s->pcur = 1 - s->pcur;
    s->step++;
    s->nh++;
}

// Gauge record and run-up update of the step just finished, where enabled;
// adds their launches.
template <typename real>
cel_status log_gauges(cel_solver *s, cudaStream_t st, int64_t &launches)
{
    if (s->runup) {
        CEL_CUDA(s, launch_runup<real>(s->geo, s->at<real>(s->lay.Bc), s->at<real>(s->lay.w[s->cur]),
                                       (real *)s->runup, s->runup_delta, 0, st), "run-up");
        launches += 1;
    }
    if (!(s->ng > 0 && s->log_every > 0 && s->cap > 0 && s->step % s->log_every == 0)) return CEL_OK;
    int slotg;
    if (s->nrec < s->cap) {
        slotg = (s->head + s->nrec) % s->cap;
        s->nrec++;
    } else {
        slotg = s->head;
        s->head = (s->head + 1) % s->cap;
    }
    real *dst = reinterpret_cast<real *>(s->gring) + (size_t)slotg * s->ng;
    CEL_CUDA(s, launch_gauges<real>(s->geo, s->phy, s->at<real>(s->lay.w[s->cur]), s->gij, s->ng, dst, st), "gauges");
    launches += 1;
    return CEL_OK;
}

template <typename real>
cel_status step_t(cel_solver *s, int nsteps)
{
    const Layout &L = s->lay;
    int64_t launches = 0;
    const Coef<real> coef = make_coef<real>(s->geo, s->phy, s->bnd);
    real *ghost = s->at<real>(L.ghost);
    if (s->gam_dirty) {
        if (coef.spw[0] | coef.spw[1] | coef.spw[2] | coef.spw[3]) {
            CEL_CUDA(s, launch_sponge_table<real>(coef, s->at<real>(L.gam), s->stream), "sponge table");
            launches += 1;
        }
        s->gam_dirty = 0;
    }
    for (int it = 0; it < nsteps; it++) {
        const int Kn = stages_of(s) - 1;
        const double t0 = (double)s->step * s->params.dt, t1 = (double)(s->step + 1) * s->params.dt;
        if (coef.sine) {
            int pg = prof_begin(s, 2);
            if (s->ktab_dirty) {
                CEL_CUDA(s, launch_eckart_table<real>(s->geo, s->phy, s->bnd, s->at<real>(L.dr),
                                                      s->at<double>(L.ktab), coef.npos, s->stream), "Eckart table");
                s->ktab_dirty = 0;
                launches += 1;
            }
            CEL_CUDA(s, launch_ghost_table<real>(s->geo, s->phy, s->bnd, s->at<real>(L.dr), s->at<double>(L.ktab),
                                                 t0, t1, ghost, coef.npos, s->stream), "ghost table");
            prof_end(s, pg);
            launches += 1;
        }
        for (int stage = 0; stage <= Kn; stage++) {
            const StencilArgs<real> a = stencil_args<real>(s, coef, stage, Kn);
            int pe = prof_begin(s, 0);
            CEL_CUDA(s, launch_stencil<real>(a, s->stream), "stencil");
            prof_end(s, pe);
            LinePair<real> lp;
            for (int dir = 0; dir < 2; dir++) lp.L[dir] = line_args<real>(s, coef, dir, stage, Kn);
            if (s->capture_rhs) {   // the adjoint keeps each stage's line solutions (line layout)
                unsigned char *dst = s->capture_rhs + s->capture_line * 2 * stage;
                lp.L[0].xcap = reinterpret_cast<real *>(dst);
                lp.L[1].xcap = reinterpret_cast<real *>(dst + s->capture_line);
            }
            int pl = prof_begin(s, 1);
            CEL_CUDA(s, launch_lines<real>(lp, s->stream), "line solves");
            prof_end(s, pl);
            launches += 1 + line_launches(lp.L[0].nlines, lp.L[0].n, lp.L[1].nlines, lp.L[1].n, s->es);
            if (s->capture && stage < Kn) {
                real *dst = reinterpret_cast<real *>(s->capture + s->capture_field * 3 * stage);
                const size_t f = s->capture_field / sizeof(real);
                CEL_CUDA(s, launch_get_state<real>(s->geo, s->at<real>(L.w[(s->cur + stage + 1) & 1]),
                                                   s->at<real>(L.P[1 - s->pcur]), s->at<real>(L.Qc[1 - s->pcur]), dst,
                                                   dst + f, dst + 2 * f, s->stream),
                         "iterate capture");
            }
        }
        finish_step(s, Kn);
        cel_status st = log_gauges<real>(s, s->stream, launches);
        if (st != CEL_OK) return st;
    }
    s->launches = launches;
    return CEL_OK;
}

struct CkptHeader {
    uint64_t magic;
    int32_t nx, ny, es, K;
    int64_t step, nh;
    uint64_t bytes;
    uint64_t pad[2];
};

struct CkptPart {
    size_t off_ws, bytes;
};

int ckpt_parts(const cel_solver *s, CkptPart *parts)
{
    const Layout &L = s->lay;
    int n = 0;
    parts[n++] = {L.w[s->cur], L.row_bytes};
    parts[n++] = {L.P[s->pcur], L.row_bytes};
    parts[n++] = {L.Qc[s->pcur], L.col_bytes};
    if (s->params.corrector_iters == 0) {
        for (int v = 0; v < 3; v++) {
            parts[n++] = {L.a[v], L.row_bytes};
            parts[n++] = {L.b[v][0], L.row_bytes};
            parts[n++] = {L.b[v][1], L.row_bytes};
        }
    } else {   // the rings (the AM4 bases live within one step only)
        for (int v = 0; v < 3; v++) {
            for (int k = 0; k < 3; k++) parts[n++] = {L.R[v][k], L.row_bytes};
            if (v > 0)
                for (int k = 0; k < 3; k++) parts[n++] = {L.Ph[v][k], L.row_bytes};
        }
    }
    return n;
}

size_t ckpt_total(const cel_solver *s)
{
    CkptPart parts[32];
    int n = ckpt_parts(s, parts);
    size_t t = align256(sizeof(CkptHeader));
    for (int k = 0; k < n; k++) t += align256(parts[k].bytes);
    return t;
}

}  // namespace

extern "C" {

const char *cel_status_string(cel_status st)
{
    switch (st) {
    case CEL_OK: return "ok";
    case CEL_ERR_INVALID_ARG: return "invalid argument";
    case CEL_ERR_WORKSPACE_TOO_SMALL: return "workspace too small";
    case CEL_ERR_CUDA: return "CUDA error";
    case CEL_ERR_NONFINITE: return "non-finite value in the state";
    case CEL_ERR_TIMEOUT: return "timeout";
    case CEL_ERR_NOT_IMPLEMENTED: return "not implemented";
    }
    return "unknown status";
}

const char *cel_last_error(const cel_solver *s) { return s ? s->err.c_str() : ""; }

cel_status cel_workspace_bytes(const cel_grid *grid, const cel_params *params, size_t *bytes)
{
    if (!grid_ok(grid) || !params_ok(params) || !bytes) return CEL_ERR_INVALID_ARG;
    Geo G = make_geo(*grid);
    *bytes = make_layout(G, grid->real_bytes, params->corrector_iters).total;
    return CEL_OK;
}

cel_status cel_create(const cel_grid *grid, const cel_params *params, const void *z_dev,
                      void *workspace_dev, size_t ws_bytes, void *cuda_stream, cel_solver **out)
{
    if (!out) return CEL_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid_ok(grid) || !params_ok(params) || !z_dev || !workspace_dev) return CEL_ERR_INVALID_ARG;
    if (((uintptr_t)workspace_dev & 255) != 0) return CEL_ERR_INVALID_ARG;
    Geo G = make_geo(*grid);
    Layout L = make_layout(G, grid->real_bytes, params->corrector_iters);
    if (ws_bytes < L.total) return CEL_ERR_WORKSPACE_TOO_SMALL;
    cel_solver *s = new cel_solver();
    s->grid = *grid;
    s->params = *params;
    s->geo = G;
    s->lay = L;
    s->es = grid->real_bytes;
    s->stream = (cudaStream_t)cuda_stream;
    s->ws = (unsigned char *)workspace_dev;
    s->phy.model = params->model;
    s->phy.friction = params->friction;
    s->phy.K = params->corrector_iters;
    s->phy.g = params->g;
    s->phy.Bd = params->Bdisp;
    s->phy.theta = params->theta;
    s->phy.eps = params->eps;
    s->phy.dt = params->dt;
    s->phy.ws = params->still_water;
    s->phy.fcoef = params->fric_coef;
    memset(&s->bnd, 0, sizeof(s->bnd));
    for (int k = 0; k < 4; k++) s->bnd.s[k].type = kSolid;
    s->gij = nullptr;
    s->gring = nullptr;
    s->ng = s->log_every = s->cap = s->nrec = s->head = 0;
    s->launches = 0;
    s->runup = nullptr;
    s->runup_delta = 0.0;
    s->capture = nullptr;
    s->capture_field = 0;
    s->capture_rhs = nullptr;
    s->capture_line = 0;
    s->ktab_dirty = 1;
    s->gam_dirty = 1;
    s->gen = 0;
    s->step = 0;
    s->cur = s->pcur = 0;
    cudaError_t e = cudaMemsetAsync(workspace_dev, 0, L.total, s->stream);
    if (e != cudaSuccess) {
        delete s;
        return CEL_ERR_CUDA;
    }
    cel_status st = s->es == 4 ? derive_static<float>(s, z_dev) : derive_static<double>(s, z_dev);
    if (st == CEL_OK)
        st = s->es == 4 ? set_state_t<float>(s, nullptr, nullptr, nullptr, 1)
                        : set_state_t<double>(s, nullptr, nullptr, nullptr, 1);
    if (st != CEL_OK) {
        delete s;
        return st;
    }
    *out = s;
    return CEL_OK;
}

void cel_destroy(cel_solver *s)
{
    if (!s) return;
    prof_free(s);
    delete s;
}

cel_status cel_set_boundary(cel_solver *s, int32_t side, const cel_bc *bc)
{
    if (!s || !bc || side < 0 || side > 3) return fail(s, CEL_ERR_INVALID_ARG, "bad side or NULL bc");
    if (bc->type < CEL_SOLID || bc->type > CEL_SINE || bc->ncomp < 0 || bc->ncomp > 8 || bc->width_cells < 0)
        return fail(s, CEL_ERR_INVALID_ARG, "bad boundary type, ncomp or width");
    if (bc->type == CEL_SINE)
        for (int m = 0; m < bc->ncomp; m++)
            if (!(bc->period[m] > 0) || !isfinite(bc->amp[m]) || !isfinite(bc->theta[m]) ||
                !isfinite(bc->phase[m]))
                return fail(s, CEL_ERR_INVALID_ARG, "bad sine component");
    Side &S = s->bnd.s[side];
    memset(&S, 0, sizeof(S));
    s->ktab_dirty = 1;
    s->gam_dirty = 1;
    s->gen++;
    S.type = bc->type;
    S.width = bc->width_cells;
    S.L = bc->width_cells * (side < 2 ? s->grid.dx : s->grid.dy);
    S.ncomp = bc->type == CEL_SINE ? bc->ncomp : 0;
    for (int m = 0; m < S.ncomp; m++) {
        S.amp[m] = bc->amp[m];
        S.omega[m] = 2.0 * kPiD / bc->period[m];
        S.cdir[m] = cos(bc->theta[m]);
        S.sdir[m] = sin(bc->theta[m]);
        S.phase[m] = bc->phase[m];
    }
    return CEL_OK;
}

cel_status cel_set_state(cel_solver *s, const void *w, const void *P, const void *Q)
{
    if (!s || !w || !P || !Q) return fail(s, CEL_ERR_INVALID_ARG, "NULL state array");
    return s->es == 4 ? set_state_t<float>(s, w, P, Q, 0) : set_state_t<double>(s, w, P, Q, 0);
}

cel_status cel_add_solitary(cel_solver *s, double H, double theta, double x0, double y0)
{
    if (!s || !isfinite(H) || !isfinite(theta) || !isfinite(x0) || !isfinite(y0))
        return fail(s, CEL_ERR_INVALID_ARG, "bad solitary-wave arguments");
    int ic = (int)floor(x0 / s->grid.dx), jc = (int)floor(y0 / s->grid.dy);
    ic = ic < 0 ? 0 : (ic > s->grid.nx - 1 ? s->grid.nx - 1 : ic);
    jc = jc < 0 ? 0 : (jc > s->grid.ny - 1 ? s->grid.ny - 1 : jc);
    double ds;
    const size_t off = s->lay.dr + ((size_t)jc * s->geo.px + ic) * s->es;
    if (s->es == 4) {
        float v;
        CEL_CUDA(s, cudaMemcpyAsync(&v, s->ws + off, 4, cudaMemcpyDeviceToHost, s->stream), "read depth");
        CEL_CUDA(s, cudaStreamSynchronize(s->stream), "read depth");
        ds = v;
    } else {
        CEL_CUDA(s, cudaMemcpyAsync(&ds, s->ws + off, 8, cudaMemcpyDeviceToHost, s->stream), "read depth");
        CEL_CUDA(s, cudaStreamSynchronize(s->stream), "read depth");
    }
    if (!(ds > 0.0) || !(H + ds > 0.0)) return fail(s, CEL_ERR_INVALID_ARG, "dry crest or H + d <= 0");
    double ks = sqrt(3.0 * fabs(H) / (4.0 * ds * ds * ds));
    double cs = sqrt(s->params.g * (H + ds));
    double ct = cos(theta), st = sin(theta);
    cudaError_t e;
    if (s->es == 4)
        e = launch_add_solitary<float>(s->geo, s->phy, s->at<float>(s->lay.Bc), s->at<float>(s->lay.w[s->cur]),
                                       s->at<float>(s->lay.P[s->pcur]), s->at<float>(s->lay.Qc[s->pcur]), H, ct, st, x0, y0, ks, cs,
                                       s->stream);
    else
        e = launch_add_solitary<double>(s->geo, s->phy, s->at<double>(s->lay.Bc),
                                        s->at<double>(s->lay.w[s->cur]), s->at<double>(s->lay.P[s->pcur]),
                                        s->at<double>(s->lay.Qc[s->pcur]), H, ct, st, x0, y0, ks, cs, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "add_solitary");
    s->nh = 0;
    return CEL_OK;
}

cel_status cel_set_bathymetry(cel_solver *s, const void *z_dev)
{
    if (!s || !z_dev) return fail(s, CEL_ERR_INVALID_ARG, "NULL bathymetry");
    cel_status st = s->es == 4 ? derive_static<float>(s, z_dev) : derive_static<double>(s, z_dev);
    if (st != CEL_OK) return st;
    s->ktab_dirty = 1;
    s->gen++;
    // raise w to the new bed in place, zero the discharge where now dry
    cudaError_t e = s->es == 4
                        ? launch_clamp_state<float>(s->geo, s->phy, s->at<float>(s->lay.Bc),
                                                    s->at<float>(s->lay.w[s->cur]), s->at<float>(s->lay.P[s->pcur]),
                                                    s->at<float>(s->lay.Qc[s->pcur]), s->stream)
                        : launch_clamp_state<double>(s->geo, s->phy, s->at<double>(s->lay.Bc),
                                                     s->at<double>(s->lay.w[s->cur]), s->at<double>(s->lay.P[s->pcur]),
                                                     s->at<double>(s->lay.Qc[s->pcur]), s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "set_bathymetry");
    s->nh = 0;
    return CEL_OK;
}

cel_status cel_step(cel_solver *s, int32_t nsteps)
{
    if (!s || nsteps < 0) return fail(s, CEL_ERR_INVALID_ARG, "bad step count");
    return s->es == 4 ? step_t<float>(s, nsteps) : step_t<double>(s, nsteps);
}

cel_status cel_get_state(cel_solver *s, void *w, void *P, void *Q)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    cudaError_t e;
    if (s->es == 4)
        e = launch_get_state<float>(s->geo, s->at<float>(s->lay.w[s->cur]), s->at<float>(s->lay.P[s->pcur]),
                                    s->at<float>(s->lay.Qc[s->pcur]), (float *)w, (float *)P, (float *)Q, s->stream);
    else
        e = launch_get_state<double>(s->geo, s->at<double>(s->lay.w[s->cur]), s->at<double>(s->lay.P[s->pcur]),
                                     s->at<double>(s->lay.Qc[s->pcur]), (double *)w, (double *)P, (double *)Q, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "get_state");
    return CEL_OK;
}

cel_status cel_get_field(cel_solver *s, int32_t which, void *dst)
{
    if (!s || !dst || which < 0 || which > 3) return fail(s, CEL_ERR_INVALID_ARG, "bad field");
    cudaError_t e;
    if (s->es == 4)
        e = launch_get_field<float>(s->geo, s->phy, which, s->at<float>(s->lay.Bc), s->at<float>(s->lay.dr),
                                    s->at<float>(s->lay.U), s->at<float>(s->lay.Vc), (float *)dst, s->stream);
    else
        e = launch_get_field<double>(s->geo, s->phy, which, s->at<double>(s->lay.Bc), s->at<double>(s->lay.dr),
                                     s->at<double>(s->lay.U), s->at<double>(s->lay.Vc), (double *)dst,
                                     s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "get_field");
    return CEL_OK;
}

cel_status cel_gauge_bytes(int32_t n, int32_t capacity, int32_t real_bytes, size_t *bytes)
{
    if (!bytes || n < 0 || capacity < 0 || (real_bytes != 4 && real_bytes != 8)) return CEL_ERR_INVALID_ARG;
    *bytes = align256((size_t)n * 2 * sizeof(int32_t)) + (size_t)n * capacity * real_bytes;
    return CEL_OK;
}

cel_status cel_set_gauges(cel_solver *s, const int32_t *ij_host, int32_t n, int32_t log_every, int32_t capacity,
                          void *gauge_buf_dev, size_t buf_bytes)
{
    if (!s || n < 0 || log_every < 0 || capacity < 0 || (n > 0 && (!ij_host || !gauge_buf_dev)))
        return fail(s, CEL_ERR_INVALID_ARG, "bad gauge arguments");
    for (int k = 0; k < n; k++)
        if (ij_host[2 * k] < 0 || ij_host[2 * k] >= s->grid.nx || ij_host[2 * k + 1] < 0 ||
            ij_host[2 * k + 1] >= s->grid.ny)
            return fail(s, CEL_ERR_INVALID_ARG, "gauge outside the grid");
    size_t need;
    cel_gauge_bytes(n, capacity, s->es, &need);
    if (n > 0 && buf_bytes < need) return fail(s, CEL_ERR_WORKSPACE_TOO_SMALL, "gauge buffer too small");
    if (n > 0 && ((uintptr_t)gauge_buf_dev & 255) != 0) return fail(s, CEL_ERR_INVALID_ARG, "gauge buffer alignment");
    s->ng = n;
    s->log_every = log_every;
    s->cap = capacity;
    s->nrec = s->head = 0;
    s->gij = n ? (int32_t *)gauge_buf_dev : nullptr;
    s->gring = n ? (unsigned char *)gauge_buf_dev + align256((size_t)n * 2 * sizeof(int32_t)) : nullptr;
    if (n > 0)
        CEL_CUDA(s, cudaMemcpyAsync(s->gij, ij_host, (size_t)n * 2 * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    s->stream), "gauge indices");
    return CEL_OK;
}

namespace {
// Copies of up to max_rec oldest gauge records to eta_host, queued on the
// handle's stream, and the records dropped from the ring.
cel_status queue_gauge_read(cel_solver *s, void *eta_host, int32_t max_rec, int32_t *n_rec)
{
    if (!s || !n_rec || max_rec < 0 || (max_rec > 0 && !eta_host)) return fail(s, CEL_ERR_INVALID_ARG, "bad read");
    int n = s->nrec < max_rec ? s->nrec : max_rec;
    size_t rec = (size_t)s->ng * s->es;
    for (int r = 0; r < n; r++) {
        int slot = (s->head + r) % s->cap;
        CEL_CUDA(s, cudaMemcpyAsync((unsigned char *)eta_host + (size_t)r * rec, s->gring + (size_t)slot * rec, rec,
                                    cudaMemcpyDeviceToHost, s->stream), "read gauges");
    }
    if (s->cap) s->head = (s->head + n) % s->cap;
    s->nrec -= n;
    *n_rec = n;
    return CEL_OK;
}
}  // namespace

cel_status cel_read_gauges(cel_solver *s, void *eta_host, int32_t max_rec, int32_t *n_rec)
{
    cel_status st = queue_gauge_read(s, eta_host, max_rec, n_rec);
    if (st != CEL_OK) return st;
    CEL_CUDA(s, cudaStreamSynchronize(s->stream), "read gauges");
    return CEL_OK;
}

cel_status cel_read_gauges_async(cel_solver *s, void *eta_host, int32_t max_rec, int32_t *n_rec)
{
    return queue_gauge_read(s, eta_host, max_rec, n_rec);
}

cel_status cel_get_time(cel_solver *s, double *t, int64_t *step)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    if (t) *t = (double)s->step * s->params.dt;
    if (step) *step = s->step;
    return CEL_OK;
}

cel_status cel_check_finite(cel_solver *s)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    unsigned long long *flag = s->at<unsigned long long>(s->lay.flag);
    CEL_CUDA(s, cudaMemsetAsync(flag, 0xff, sizeof(unsigned long long), s->stream), "check_finite");
    cudaError_t e = s->es == 4
                        ? launch_check_finite<float>(s->geo, s->at<float>(s->lay.w[s->cur]), s->at<float>(s->lay.P[s->pcur]),
                                                     s->at<float>(s->lay.Qc[s->pcur]), flag, s->stream)
                        : launch_check_finite<double>(s->geo, s->at<double>(s->lay.w[s->cur]),
                                                      s->at<double>(s->lay.P[s->pcur]), s->at<double>(s->lay.Qc[s->pcur]), flag,
                                                      s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "check_finite");
    unsigned long long v = 0;
    CEL_CUDA(s, cudaMemcpyAsync(&v, flag, sizeof(v), cudaMemcpyDeviceToHost, s->stream), "check_finite");
    CEL_CUDA(s, cudaStreamSynchronize(s->stream), "check_finite");
    if (v != ~0ull) {
        char buf[128];
        snprintf(buf, sizeof(buf), "non-finite value at cell i=%llu j=%llu", v % (unsigned long long)s->grid.nx,
                 v / (unsigned long long)s->grid.nx);
        return fail(s, CEL_ERR_NONFINITE, buf);
    }
    return CEL_OK;
}

cel_status cel_get_stats(cel_solver *s, cel_stats *out)
{
    if (!s || !out) return CEL_ERR_INVALID_ARG;
    unsigned long long *acc = s->at<unsigned long long>(s->lay.flag) + 8;   // 64 bytes in, beside the finite flag
    CEL_CUDA(s, cudaMemsetAsync(acc, 0, 3 * sizeof(unsigned long long), s->stream), "stats");
    const Coef<float> cf = make_coef<float>(s->geo, s->phy, s->bnd);
    const Coef<double> cd = make_coef<double>(s->geo, s->phy, s->bnd);
    cudaError_t e = s->es == 4
                        ? launch_stats<float>(s->geo, s->phy, s->at<float>(s->lay.Bc), s->at<float>(s->lay.w[s->cur]),
                                              s->at<float>(s->lay.P[s->pcur]), s->at<float>(s->lay.Qc[s->pcur]), cf.eps,
                                              acc, s->stream)
                        : launch_stats<double>(s->geo, s->phy, s->at<double>(s->lay.Bc),
                                               s->at<double>(s->lay.w[s->cur]), s->at<double>(s->lay.P[s->pcur]),
                                               s->at<double>(s->lay.Qc[s->pcur]), cd.eps, acc, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "stats");
    unsigned long long v[3];
    CEL_CUDA(s, cudaMemcpyAsync(v, acc, sizeof(v), cudaMemcpyDeviceToHost, s->stream), "stats");
    CEL_CUDA(s, cudaStreamSynchronize(s->stream), "stats");
    double mass, vmax;
    memcpy(&mass, &v[0], sizeof(double));
    memcpy(&vmax, &v[1], sizeof(double));
    out->mass = mass * s->geo.dx * s->geo.dy;
    out->max_speed = vmax;
    out->wet_cells = (int64_t)v[2];
    return CEL_OK;
}

cel_status cel_checkpoint_bytes(const cel_solver *s, size_t *bytes)
{
    if (!s || !bytes) return CEL_ERR_INVALID_ARG;
    *bytes = ckpt_total(s);
    return CEL_OK;
}

cel_status cel_save_checkpoint(cel_solver *s, void *dst_dev, size_t bytes)
{
    if (!s || !dst_dev) return fail(s, CEL_ERR_INVALID_ARG, "NULL checkpoint buffer");
    size_t need = ckpt_total(s);
    if (bytes < need) return fail(s, CEL_ERR_WORKSPACE_TOO_SMALL, "checkpoint buffer too small");
    CkptHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kCkptMagic;
    h.nx = s->grid.nx;
    h.ny = s->grid.ny;
    h.es = s->es;
    h.K = s->params.corrector_iters;
    h.step = s->step;
    h.nh = s->nh;
    h.bytes = need;
    unsigned char *dst = (unsigned char *)dst_dev;
    CEL_CUDA(s, cudaMemcpyAsync(dst, &h, sizeof(h), cudaMemcpyHostToDevice, s->stream), "checkpoint header");
    // the header copy reads pageable host memory: finish it before h goes away
    CEL_CUDA(s, cudaStreamSynchronize(s->stream), "checkpoint header");
    CkptPart parts[32];
    int np = ckpt_parts(s, parts);
    size_t off = align256(sizeof(CkptHeader));
    for (int k = 0; k < np; k++) {
        CEL_CUDA(s, cudaMemcpyAsync(dst + off, s->ws + parts[k].off_ws, parts[k].bytes, cudaMemcpyDeviceToDevice,
                                    s->stream), "checkpoint");
        off += align256(parts[k].bytes);
    }
    return CEL_OK;
}

cel_status cel_load_checkpoint(cel_solver *s, const void *src_dev, size_t bytes)
{
    if (!s || !src_dev) return fail(s, CEL_ERR_INVALID_ARG, "NULL checkpoint buffer");
    CkptHeader h;
    if (bytes < sizeof(h)) return fail(s, CEL_ERR_INVALID_ARG, "checkpoint too small");
    CEL_CUDA(s, cudaMemcpyAsync(&h, src_dev, sizeof(h), cudaMemcpyDeviceToHost, s->stream), "checkpoint header");
    CEL_CUDA(s, cudaStreamSynchronize(s->stream), "checkpoint header");
    if (h.magic != kCkptMagic || h.nx != s->grid.nx || h.ny != s->grid.ny || h.es != s->es ||
        h.K != s->params.corrector_iters)
        return fail(s, CEL_ERR_INVALID_ARG, "checkpoint does not match this solver");
    s->cur = 0;
    s->pcur = 0;
    size_t need = ckpt_total(s);
    if (bytes < need || h.bytes != need) return fail(s, CEL_ERR_INVALID_ARG, "checkpoint size mismatch");
    CkptPart parts[32];
    int np = ckpt_parts(s, parts);
    size_t off = align256(sizeof(CkptHeader));
    const unsigned char *src = (const unsigned char *)src_dev;
    for (int k = 0; k < np; k++) {
        CEL_CUDA(s, cudaMemcpyAsync(s->ws + parts[k].off_ws, src + off, parts[k].bytes, cudaMemcpyDeviceToDevice,
                                    s->stream), "checkpoint");
        off += align256(parts[k].bytes);
    }
    s->step = h.step;
    s->nh = h.nh;
    return CEL_OK;
}

cel_status cel_profile_enable(cel_solver *s, int32_t capacity)
{
    if (!s || capacity < 1 || capacity > (1 << 20)) return fail(s, CEL_ERR_INVALID_ARG, "bad profile capacity");
    CEL_CUDA(s, s->prof.create(capacity), "profile events");
    return CEL_OK;
}

cel_status cel_profile_read(cel_solver *s, double ms[3], int64_t count[3])
{
    if (!s || !ms || !count) return CEL_ERR_INVALID_ARG;
    CEL_CUDA(s, s->prof.read(s->stream, ms, count), "profile read");
    return CEL_OK;
}

cel_status cel_profile_disable(cel_solver *s)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    prof_free(s);
    return CEL_OK;
}

cel_status cel_runup_enable(cel_solver *s, void *maxw_dev, double delta)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    if (!maxw_dev) {
        s->runup = nullptr;
        return CEL_OK;
    }
    if (!(delta >= 0.0) || !isfinite(delta)) return fail(s, CEL_ERR_INVALID_ARG, "bad run-up threshold");
    s->runup = maxw_dev;
    s->runup_delta = delta;
    cudaError_t e = s->es == 4 ? launch_runup<float>(s->geo, s->at<float>(s->lay.Bc), s->at<float>(s->lay.w[s->cur]),
                                                     (float *)maxw_dev, delta, 1, s->stream)
                               : launch_runup<double>(s->geo, s->at<double>(s->lay.Bc),
                                                      s->at<double>(s->lay.w[s->cur]), (double *)maxw_dev, delta, 1,
                                                      s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "run-up");
    return CEL_OK;
}

cel_status cel_render(cel_solver *s, const cel_render_params *p, void *rgba_dev)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    if (!p || !rgba_dev) return fail(s, CEL_ERR_INVALID_ARG, "NULL render parameters or image");
    const float vals[] = {p->vmin, p->vmax, p->dry_h, p->h_min, p->zmin, p->zmax, p->grid, p->exaggeration,
                          p->view[0], p->view[1], p->view[2], p->sun[0], p->sun[1], p->sun[2], p->absorb};
    for (float v : vals)
        if (!isfinite(v)) return fail(s, CEL_ERR_INVALID_ARG, "non-finite render parameter");
    const bool view0 = p->view[0] == 0.f && p->view[1] == 0.f && p->view[2] == 0.f;
    const bool sun0 = p->sun[0] == 0.f && p->sun[1] == 0.f && p->sun[2] == 0.f;
    if (p->mode < CEL_RENDER_ETA || p->mode > CEL_RENDER_FRESNEL || !(p->vmax > p->vmin) ||
        !(p->zmax > p->zmin) || p->grid < 0.f || p->dry_h < 0.f || !(p->h_min > 0.f) || p->absorb < 0.f || view0 ||
        sun0)
        return fail(s, CEL_ERR_INVALID_ARG, "bad render parameters");
    cudaError_t e;
    if (s->es == 4) {
        RenderArgs<float> a;
        a.geo = s->geo;
        a.dx = (float)s->grid.dx;
        a.dy = (float)s->grid.dy;
        a.ws = (float)s->params.still_water;
        a.p = *p;
        a.w = s->at<float>(s->lay.w[s->cur]);
        a.P = s->at<float>(s->lay.P[s->pcur]);
        a.Qc = s->at<float>(s->lay.Qc[s->pcur]);
        a.Bc = s->at<float>(s->lay.Bc);
        a.rgba = (uchar4 *)rgba_dev;
        e = launch_render<float>(a, s->stream);
    } else {
        RenderArgs<double> a;
        a.geo = s->geo;
        a.dx = (float)s->grid.dx;
        a.dy = (float)s->grid.dy;
        a.ws = (float)s->params.still_water;
        a.p = *p;
        a.w = s->at<double>(s->lay.w[s->cur]);
        a.P = s->at<double>(s->lay.P[s->pcur]);
        a.Qc = s->at<double>(s->lay.Qc[s->pcur]);
        a.Bc = s->at<double>(s->lay.Bc);
        a.rgba = (uchar4 *)rgba_dev;
        e = launch_render<double>(a, s->stream);
    }
    if (e != cudaSuccess) return cuda_fail(s, e, "render");
    return CEL_OK;
}

cel_status cel_set_line_split(int32_t real_bytes, int32_t max_rows, int32_t rows_per_thread)
{
    return line_split_set(real_bytes, max_rows, rows_per_thread) == 0 ? CEL_OK : CEL_ERR_INVALID_ARG;
}

cel_status cel_reset_line_splits(void)
{
    line_split_reset();
    return CEL_OK;
}

cel_status cel_line_config(int32_t real_bytes, int32_t rows, int32_t *rows_per_thread, int32_t *threads)
{
    if ((real_bytes != 4 && real_bytes != 8) || rows < 2 ||
        rows > (real_bytes == 4 ? CEL_MAX_LINE_F32 : CEL_MAX_LINE_F64) || !rows_per_thread || !threads)
        return CEL_ERR_INVALID_ARG;
    const LineCfg c = line_config(rows, real_bytes);
    *rows_per_thread = 1 << c.mshift;
    *threads = c.threads;
    return CEL_OK;
}

cel_status cel_set_dependent_launch(int32_t enable)
{
    set_dependent_launch(enable != 0);
    return CEL_OK;
}

cel_status cel_get_dependent_launch(int32_t *enabled)
{
    if (!enabled) return CEL_ERR_INVALID_ARG;
    *enabled = dependent_launch();
    return CEL_OK;
}

cel_status cel_last_launch_count(const cel_solver *s, int64_t *launches)
{
    if (!s || !launches) return CEL_ERR_INVALID_ARG;
    *launches = s->launches;
    return CEL_OK;
}

// ------------------------------------------------- fixed-scratch variant

}  // extern "C"

namespace {

// The scratch of cel_advance_noalloc: one array in device memory, defined
// here so that the library never has to allocate it.  Host code must not use
// the name as an address (it is a host-side stand-in); the device address is
// looked up with cudaGetSymbolAddress once per device and CUDA context, and
// kept with the context's unique id: after cudaDeviceReset, or with another
// context current on the device, the module is loaded again at another
// address, so a changed id means a new lookup.
static __device__ __align__(256) unsigned char g_noalloc_scratch[CEL_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
struct NoallocSlot {
    unsigned long long ctx_id;   // unique id of the context the address belongs to
    void *ptr;                   // device address of g_noalloc_scratch there (null: none yet)
};
NoallocSlot g_noalloc_slot[kMaxDevices];
std::mutex g_noalloc_mutex;

// The CUDA driver API's context queries, fetched through the runtime (the
// library links no libcuda of its own).
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

// Unique id of the context current on this thread; the runtime binds the
// device's primary context first when none is current.  False with a reason
// in why on failure.
bool current_context_id(unsigned long long *id, std::string *why)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
        cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
        if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
            *why = "the CUDA driver API's context queries (cuCtxGetCurrent, cuCtxGetId) are unavailable";
            return false;
        }
        get_current = (CtxGetCurrentFn)f1;
        get_id = (CtxGetIdFn)f2;
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0) {
        *why = "cuCtxGetCurrent failed";
        return false;
    }
    if (!ctx) {
        // no context current yet: a runtime call binds the primary context
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return false;
        }
        if (get_current(&ctx) != 0 || !ctx) {
            *why = "no CUDA context is current after binding the device";
            return false;
        }
    }
    if (get_id(ctx, id) != 0) {
        *why = "cuCtxGetId failed";
        return false;
    }
    return true;
}

void put_msg(char *msg, size_t len, const std::string &text)
{
    if (!msg || len == 0) return;
    size_t n = text.size() < len - 1 ? text.size() : len - 1;
    memcpy(msg, text.data(), n);
    msg[n] = 0;
}

}  // namespace

extern "C" cel_status cel_advance_noalloc(const cel_grid *grid, const cel_params *params, const cel_bc *bcs,
                                          const void *z_dev, const void *w_in, const void *P_in,
                                          const void *Q_in, void *w_out, void *P_out, void *Q_out,
                                          int32_t nsteps, int64_t first_step, void *cuda_stream, char *msg,
                                          size_t msg_len)
{
    put_msg(msg, msg_len, "");
    if (!grid_ok(grid) || !params_ok(params) || !z_dev || !w_in || !P_in || !Q_in || !w_out || !P_out ||
        !Q_out || nsteps < 0 || first_step < 0) {
        put_msg(msg, msg_len, "invalid grid, parameters, pointers or step counts");
        return CEL_ERR_INVALID_ARG;
    }
    Geo G = make_geo(*grid);
    Layout L = make_layout(G, grid->real_bytes, params->corrector_iters);
    if (L.total > CEL_NOALLOC_SCRATCH_BYTES) {
        char buf[200];
        snprintf(buf, sizeof(buf), "this grid needs %zu bytes of scratch; the fixed scratch holds %zu bytes",
                 L.total, (size_t)CEL_NOALLOC_SCRATCH_BYTES);
        put_msg(msg, msg_len, buf);
        return CEL_ERR_WORKSPACE_TOO_SMALL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        put_msg(msg, msg_len, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return CEL_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        char buf[120];
        snprintf(buf, sizeof(buf), "device %d is beyond the %d devices this entry point serves", dev, kMaxDevices);
        put_msg(msg, msg_len, buf);
        return CEL_ERR_CUDA;
    }
    void *scratch;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        unsigned long long ctx_id = 0;
        std::string why;
        if (!current_context_id(&ctx_id, &why)) {
            put_msg(msg, msg_len, why);
            return CEL_ERR_CUDA;
        }
        NoallocSlot &slot = g_noalloc_slot[dev];
        if (!slot.ptr || slot.ctx_id != ctx_id) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                put_msg(msg, msg_len, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return CEL_ERR_CUDA;
            }
            slot.ptr = p;
            slot.ctx_id = ctx_id;
        }
        scratch = slot.ptr;
    }
    // a handle on the stack, pointing at the fixed scratch; set up as
    // cel_create does (the scratch is cleared, so nothing of an earlier call
    // is read)
    cel_solver s;
    s.grid = *grid;
    s.params = *params;
    s.geo = G;
    s.lay = L;
    s.es = grid->real_bytes;
    s.stream = (cudaStream_t)cuda_stream;
    s.ws = (unsigned char *)scratch;
    s.phy.model = params->model;
    s.phy.friction = params->friction;
    s.phy.K = params->corrector_iters;
    s.phy.g = params->g;
    s.phy.Bd = params->Bdisp;
    s.phy.theta = params->theta;
    s.phy.eps = params->eps;
    s.phy.dt = params->dt;
    s.phy.ws = params->still_water;
    s.phy.fcoef = params->fric_coef;
    memset(&s.bnd, 0, sizeof(s.bnd));
    for (int k = 0; k < 4; k++) s.bnd.s[k].type = kSolid;
    s.gij = nullptr;
    s.gring = nullptr;
    s.ng = s.log_every = s.cap = s.nrec = s.head = 0;
    s.launches = 0;
    s.runup = nullptr;
    s.runup_delta = 0.0;
    s.capture = nullptr;
    s.capture_field = 0;
    s.capture_rhs = nullptr;
    s.capture_line = 0;
    s.ktab_dirty = 1;
    s.gam_dirty = 1;
    s.gen = 0;
    s.step = first_step;
    s.nh = 0;
    s.cur = s.pcur = 0;
    cel_status st = CEL_OK;
    if (bcs)
        for (int side = 0; side < 4 && st == CEL_OK; side++) st = cel_set_boundary(&s, side, &bcs[side]);
    if (st == CEL_OK) {
        e = cudaMemsetAsync(scratch, 0, L.total, s.stream);
        if (e != cudaSuccess) st = cuda_fail(&s, e, "clear scratch");
    }
    if (st == CEL_OK) st = s.es == 4 ? derive_static<float>(&s, z_dev) : derive_static<double>(&s, z_dev);
    if (st == CEL_OK)
        st = s.es == 4 ? set_state_t<float>(&s, w_in, P_in, Q_in, 0) : set_state_t<double>(&s, w_in, P_in, Q_in, 0);
    if (st == CEL_OK) st = s.es == 4 ? step_t<float>(&s, nsteps) : step_t<double>(&s, nsteps);
    if (st == CEL_OK) st = cel_get_state(&s, w_out, P_out, Q_out);
    if (st != CEL_OK) put_msg(msg, msg_len, s.err);
    return st;
}


// ------------------------------------------------------------- ensembles
//
// An ensemble steps many solvers (members) in lockstep with one launch per
// kernel kind and stage: the stencil launch covers every member's tiles, the
// line launch every member's x- and y-lines of one segment length, the ghost
// launch every member's sine-maker table.  Each member keeps its own
// workspace; the ensemble only adds argument tables in the caller's device
// memory.  The argument blocks of a stage are the ones the member's own step
// would pass (same builders), so every member evolves bit for bit as if it
// were stepped alone.

struct cel_ensemble {
    struct Group {            // line families of one line-solver configuration
        LineCfg cfg;
        int first, nfam, blocks;
        size_t off_desc;
    };
    std::vector<cel_solver *> m;
    int es, K;
    cudaStream_t stream;
    unsigned char *tab;
    size_t tab_bytes;
    int tiles;                           // stencil blocks over all members
    size_t off_tile_desc;                // int2 per stencil block
    std::vector<std::pair<int, int>> fam;   // (member, dir) in table order
    std::vector<Group> groups;
    std::vector<int> gmem;               // members with a sine maker
    int gblocks;
    size_t off_gargs, off_gstart;
    std::vector<int64_t> gstep0;         // member steps the ghost arguments were built at
    bool gvalid;
    size_t sarg_bytes, entry_bytes, off_entries;
    int cap;
    std::vector<uint64_t> keys;          // key of each filled entry
    uint64_t gen_sum;
    int64_t launches;
    EventProf prof;
    std::string err;
    // Captured cycles: once the history is full the argument blocks repeat
    // every 6 steps, so 6 steps captured as one graph replay as they are;
    // one graph per phase of the cycle it starts at (key of member 0).
    struct Graph {
        uint64_t key;
        cudaGraphExec_t exec;
        int64_t launches;
    };
    std::vector<Graph> graphs;
    bool use_graphs = true;
    int64_t graph_steps = 0;             // steps taken by replaying a graph, since creation
    int split_gen = 0;                   // line-split table generation the plan was made with
    cudaStream_t cap_stream = nullptr;   // the library's own stream, for capture only
    size_t off_kdev = 0;                 // device step counter of the ghost tables
    int64_t kdev_val = 0;                // its value once the queued work has run
    bool kdev_known = false;
    // The persistent launch (cel_ensemble_use_persistent): one cooperative
    // launch for a call's steps once the cycle's argument blocks are in place.
    bool use_persist = false;
    double persist_timeout_ms = 1000.0;
    int64_t persist_steps = 0;           // steps taken by persistent launches, since creation
    size_t off_bar = 0;                  // the launch's barrier words
    void drop_graphs()
    {
        for (Graph &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    }
};

namespace {

struct EnsPlan {
    int tiles = 0, gblocks = 0;
    std::vector<std::pair<int, int>> fam;
    std::vector<cel_ensemble::Group> groups;
    std::vector<int> gmem;
    size_t off_tile_desc = 0, off_gargs = 0, off_gstart = 0, off_kdev = 0, off_bar = 0, sarg_bytes = 0,
           entry_bytes = 0, off_entries = 0;
    int cap = 0;
    size_t total = 0;
};

template <typename real>
void plan_t(cel_solver *const *ms, int n, EnsPlan &P)
{
    size_t cur = 0;
    auto take = [&](size_t b) {
        size_t o = cur;
        cur += align256(b);
        return o;
    };
    P.tiles = 0;
    for (int e = 0; e < n; e++)
        P.tiles += ((ms[e]->geo.nx + kTile - 1) / kTile) * ((ms[e]->geo.ny + kTile - 1) / kTile);
    P.off_tile_desc = take(sizeof(int2) * (size_t)P.tiles);
    // line families grouped by their solver configuration (one launch
    // each), longest lines first within a group
    P.fam.clear();
    P.groups.clear();
    auto len_of = [&](const std::pair<int, int> &f) { return f.second == 0 ? ms[f.first]->geo.nx : ms[f.first]->geo.ny; };
    // register-path lines of one block size share a launch whatever their
    // segment length; shared-memory ones need one segment length too
    auto same = [](const LineCfg &a, const LineCfg &b) {
        return a.algo == b.algo && a.threads == b.threads && (a.algo == 0 || a.mshift == b.mshift);
    };
    std::vector<std::pair<int, int>> all;
    for (int e = 0; e < n; e++)
        for (int dir = 0; dir < 2; dir++) all.push_back(std::pair<int, int>(e, dir));
    std::vector<char> taken(all.size(), 0);
    for (size_t a = 0; a < all.size(); a++) {
        if (taken[a]) continue;
        const LineCfg ca = line_config(len_of(all[a]), (int)sizeof(real));
        std::vector<std::pair<int, int>> g;
        for (size_t b = a; b < all.size(); b++)
            if (!taken[b] && same(ca, line_config(len_of(all[b]), (int)sizeof(real)))) {
                g.push_back(all[b]);
                taken[b] = 1;
            }
        std::stable_sort(g.begin(), g.end(), [&](const std::pair<int, int> &x, const std::pair<int, int> &y) {
            return len_of(x) > len_of(y);
        });
        cel_ensemble::Group G;
        G.cfg = ca;
        G.first = (int)P.fam.size();
        G.nfam = (int)g.size();
        G.blocks = 0;
        for (auto &f : g) {
            G.blocks += f.second == 0 ? ms[f.first]->geo.ny : ms[f.first]->geo.nx;
            G.cfg.smem = std::max(G.cfg.smem, line_config(len_of(f), (int)sizeof(real)).smem);
            P.fam.push_back(f);
        }
        G.off_desc = take(sizeof(int2) * (size_t)G.blocks);
        P.groups.push_back(G);
    }
    P.gmem.clear();
    P.gblocks = 0;
    for (int e = 0; e < n; e++) {
        bool sine = false;
        for (int k = 0; k < 4; k++) sine |= ms[e]->bnd.s[k].type == kSine;
        if (!sine) continue;
        P.gmem.push_back(e);
        const int npos = (ms[e]->geo.nx > ms[e]->geo.ny ? ms[e]->geo.nx : ms[e]->geo.ny) + 4;
        P.gblocks += ((npos + 127) / 128) * 16;
    }
    P.off_gargs = take(sizeof(GhostArgs<real>) * (size_t)n);
    P.off_gstart = take(sizeof(int) * (size_t)(n + 1));
    P.off_kdev = take(sizeof(int64_t));
    P.off_bar = take(8 * sizeof(unsigned));   // barrier words, then the work counters
    P.sarg_bytes = align256(sizeof(StencilArgs<real>) * (size_t)n);
    P.entry_bytes = P.sarg_bytes + align256(sizeof(LineArgs<real>) * P.fam.size());
    // the argument blocks repeat every 6 steps once the AB3 history is full
    // (ring slot nh % 3, carry slot nh % 2, P / Q buffers alternate), plus
    // the two Euler steps: 8 (K + 1) entries hold a run from set_state on
    P.cap = 8 * (ms[0]->params.corrector_iters + 1);
    P.off_entries = cur;
    P.total = cur + P.entry_bytes * (size_t)P.cap;
}

cel_status plan(cel_solver *const *ms, int n, EnsPlan &P, std::string &why)
{
    if (!ms || n < 1) {
        why = "an ensemble needs at least one member";
        return CEL_ERR_INVALID_ARG;
    }
    for (int e = 0; e < n; e++) {
        if (!ms[e]) {
            why = "NULL member";
            return CEL_ERR_INVALID_ARG;
        }
        if (ms[e]->es != ms[0]->es || ms[e]->params.corrector_iters != ms[0]->params.corrector_iters) {
            why = "members differ in precision or in the number of corrector iterations";
            return CEL_ERR_INVALID_ARG;
        }
    }
    // members must not share workspace memory: one launch writes all of them
    std::vector<std::pair<uintptr_t, uintptr_t>> r;
    for (int e = 0; e < n; e++) r.push_back({(uintptr_t)ms[e]->ws, (uintptr_t)ms[e]->ws + ms[e]->lay.total});
    std::sort(r.begin(), r.end());
    for (size_t k = 1; k < r.size(); k++)
        if (r[k].first < r[k - 1].second) {
            why = "two members share workspace memory (or a member is listed twice)";
            return CEL_ERR_INVALID_ARG;
        }
    if (ms[0]->es == 4) plan_t<float>(ms, n, P);
    else plan_t<double>(ms, n, P);
    return CEL_OK;
}

cel_status ens_fail(cel_ensemble *e, cel_status st, const std::string &msg)
{
    e->err = msg;
    return st;
}

#define ENS_CUDA(e, expr, where)                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (expr);                                                                   \
        if (e_ != cudaSuccess) return ens_fail(e, CEL_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e_)); \
    } while (0)

uint64_t ens_key_of(int64_t nh, int cur, int pcur, int stage)
{
    const uint64_t nhk = nh < 2 ? (uint64_t)nh : 2 + (uint64_t)((nh - 2) % 6);
    return (nhk << 16) | ((uint64_t)cur << 9) | ((uint64_t)pcur << 8) | (uint64_t)stage;
}

uint64_t ens_key(const cel_solver *s, int stage) { return ens_key_of(s->nh, s->cur, s->pcur, stage); }

// Index of the table entry holding the arguments of this stage for the
// members' present state; built and uploaded if missing (stream-ordered, so
// launches queued earlier still read the old contents).
template <typename real>
cel_status ens_entry(cel_ensemble *e, int stage, int Kn, int *idx)
{
    const uint64_t key = ens_key(e->m[0], stage);
    for (size_t k = 0; k < e->keys.size(); k++)
        if (e->keys[k] == key) {
            *idx = (int)k;
            return CEL_OK;
        }
    if ((int)e->keys.size() >= e->cap) e->keys.clear();
    e->drop_graphs();   // the captured graphs read entries by their index
    const int k = (int)e->keys.size();
    const int n = (int)e->m.size();
    std::vector<unsigned char> host(e->entry_bytes, 0);
    StencilArgs<real> *sa = reinterpret_cast<StencilArgs<real> *>(host.data());
    LineArgs<real> *la = reinterpret_cast<LineArgs<real> *>(host.data() + e->sarg_bytes);
    std::vector<Coef<real>> coef(n);
    for (int j = 0; j < n; j++) {
        const cel_solver *s = e->m[j];
        coef[j] = make_coef<real>(s->geo, s->phy, s->bnd);
        sa[j] = stencil_args<real>(s, coef[j], stage, Kn);
    }
    for (size_t f = 0; f < e->fam.size(); f++)
        la[f] = line_args<real>(e->m[e->fam[f].first], coef[e->fam[f].first], e->fam[f].second, stage, Kn);
    ENS_CUDA(e, cudaMemcpyAsync(e->tab + e->off_entries + (size_t)k * e->entry_bytes, host.data(), e->entry_bytes,
                                cudaMemcpyHostToDevice, e->stream), "ensemble arguments");
    e->keys.push_back(key);
    *idx = k;
    return CEL_OK;
}

// Before a step: the members in lockstep, the tables rebuilt after a change
// of boundary or bed, the ghost tables' arguments and Eckart tables current.
template <typename real>
cel_status ens_prepare(cel_ensemble *e, int64_t &launches)
{
    const int n = (int)e->m.size();
    const cel_solver *m0 = e->m[0];
    if (line_split_generation() != e->split_gen)
        return ens_fail(e, CEL_ERR_INVALID_ARG,
                        "the line-solver splits changed after the ensemble was created (create it again)");
    uint64_t gsum = 0;
    for (int j = 0; j < n; j++) {
        const cel_solver *s = e->m[j];
        if (s->nh != m0->nh || s->cur != m0->cur || s->pcur != m0->pcur)
            return ens_fail(e, CEL_ERR_INVALID_ARG,
                            "members are not in lockstep (set their states together, then step the ensemble)");
        gsum += s->gen;
    }
    if (gsum != e->gen_sum) {      // a boundary or bed changed: rebuild every table
        e->keys.clear();
        e->drop_graphs();
        e->gvalid = false;
        e->gen_sum = gsum;
    }
    if (e->gvalid && !e->gmem.empty()) {        // members moved on outside the ensemble?
        const int64_t k0 = e->m[e->gmem[0]]->step - e->gstep0[0];
        for (size_t g = 0; g < e->gmem.size(); g++)
            if (e->m[e->gmem[g]]->step - e->gstep0[g] != k0) e->gvalid = false;
    }
    if (!e->gvalid) {                           // members with a sine maker, their ghost arguments
        e->drop_graphs();
        e->gmem.clear();
        for (int j = 0; j < n; j++)
            if (make_coef<real>(e->m[j]->geo, e->m[j]->phy, e->m[j]->bnd).sine) e->gmem.push_back(j);
        e->gstep0.assign(e->gmem.size(), 0);
        std::vector<GhostArgs<real>> ga(e->gmem.size());
        std::vector<int> start(e->gmem.size() + 1, 0);
        for (size_t g = 0; g < e->gmem.size(); g++) {
            const cel_solver *s = e->m[e->gmem[g]];
            GhostArgs<real> &a = ga[g];
            memset(&a, 0, sizeof(a));
            a.g = s->geo;
            a.p = s->phy;
            a.b = s->bnd;
            a.d_r = s->at<real>(s->lay.dr);
            a.ktab = s->at<double>(s->lay.ktab);
            a.tab = s->at<real>(s->lay.ghost);
            a.npos = make_coef<real>(s->geo, s->phy, s->bnd).npos;
            a.step0 = s->step;
            a.dt = s->params.dt;
            e->gstep0[g] = s->step;
            start[g + 1] = start[g] + ((a.npos + 127) / 128) * 16;
        }
        e->gblocks = start.back();
        if (!ga.empty()) {
            ENS_CUDA(e, cudaMemcpyAsync(e->tab + e->off_gargs, ga.data(), sizeof(GhostArgs<real>) * ga.size(),
                                        cudaMemcpyHostToDevice, e->stream), "ensemble ghost arguments");
            ENS_CUDA(e, cudaMemcpyAsync(e->tab + e->off_gstart, start.data(), sizeof(int) * start.size(),
                                        cudaMemcpyHostToDevice, e->stream), "ensemble ghost arguments");
        }
        e->gvalid = true;
    }
    for (int j = 0; j < n; j++) {
        cel_solver *s = e->m[j];
        if (!s->gam_dirty) continue;
        const Coef<real> c = make_coef<real>(s->geo, s->phy, s->bnd);
        if (c.spw[0] | c.spw[1] | c.spw[2] | c.spw[3]) {
            ENS_CUDA(e, launch_sponge_table<real>(c, s->at<real>(s->lay.gam), e->stream), "sponge table");
            launches += 1;
        }
        s->gam_dirty = 0;
    }
    for (int j : e->gmem) {
        cel_solver *s = e->m[j];
        if (!s->ktab_dirty) continue;
        const Coef<real> c = make_coef<real>(s->geo, s->phy, s->bnd);
        ENS_CUDA(e, launch_eckart_table<real>(s->geo, s->phy, s->bnd, s->at<real>(s->lay.dr),
                                              s->at<double>(s->lay.ktab), c.npos, e->stream), "Eckart table");
        s->ktab_dirty = 0;
        launches += 1;
    }
    return CEL_OK;
}

// One step's launches on stream st: the ghost tables (their step index k,
// plus *kdev where given), then per stage the stencil over every member's
// tiles and the line solves; the members' bookkeeping moves on a step.
template <typename real>
cel_status ens_launch_step(cel_ensemble *e, cudaStream_t st, const int64_t *kdev, int64_t k, int64_t &launches)
{
    const int n = (int)e->m.size();
    const int Kn = stages_of(e->m[0]) - 1;
    if (!e->gmem.empty()) {
        const int pg = e->prof.begin(2, st);
        ENS_CUDA(e, launch_ghost_batch<real>(reinterpret_cast<const GhostArgs<real> *>(e->tab + e->off_gargs),
                                             reinterpret_cast<const int *>(e->tab + e->off_gstart),
                                             (int)e->gmem.size(), e->gblocks, k, kdev, st), "ensemble ghost tables");
        e->prof.finish(pg, st);
        launches += 1;
    }
    for (int stage = 0; stage <= Kn; stage++) {
        int idx = 0;
        cel_status cs = ens_entry<real>(e, stage, Kn, &idx);
        if (cs != CEL_OK) return cs;
        const unsigned char *ent = e->tab + e->off_entries + (size_t)idx * e->entry_bytes;
        // the members step in lockstep: member 0's stage kind is every member's
        const Coef<real> c0 = make_coef<real>(e->m[0]->geo, e->m[0]->phy, e->m[0]->bnd);
        const int spec = stencil_spec(stencil_args<real>(e->m[0], c0, stage, Kn));
        const int pe = e->prof.begin(0, st);
        ENS_CUDA(e, launch_stencil_batch<real>(reinterpret_cast<const StencilArgs<real> *>(ent),
                                               reinterpret_cast<const int2 *>(e->tab + e->off_tile_desc),
                                               e->tiles, spec, st), "ensemble stencil");
        e->prof.finish(pe, st);
        launches += 1;
        const LineArgs<real> *la = reinterpret_cast<const LineArgs<real> *>(ent + e->sarg_bytes);
        for (const cel_ensemble::Group &G : e->groups) {
            const int pl = e->prof.begin(1, st);
            ENS_CUDA(e, launch_lines_batch<real>(la + G.first, reinterpret_cast<const int2 *>(e->tab + G.off_desc),
                                                 G.blocks, G.cfg, st),
                     "ensemble line solves");
            e->prof.finish(pl, st);
            launches += 1;
        }
    }
    for (int j = 0; j < n; j++) {
        cel_solver *s = e->m[j];
        finish_step(s, Kn);
        int64_t lg = 0;
        cel_status gs = log_gauges<real>(s, st, lg);
        if (gs != CEL_OK) return ens_fail(e, gs, s->err);
        launches += lg;
    }
    return CEL_OK;
}

// Six steps as one captured graph, replayed on the ensemble's stream: only
// where nothing in those steps differs between repetitions of the cycle (the
// history full, no gauges, run-up tracking or profiling, every argument
// block of the cycle already uploaded).  *done: the six steps were taken.
template <typename real>
cel_status ens_graph_cycle(cel_ensemble *e, int64_t &launches, bool *done)
{
    *done = false;
    const int n = (int)e->m.size();
    const cel_solver *m0 = e->m[0];
    if (!e->use_graphs || m0->nh < 2 || e->prof.cap > 0) return CEL_OK;
    for (int j = 0; j < n; j++) {
        const cel_solver *s = e->m[j];
        if (s->runup || (s->ng > 0 && s->log_every > 0 && s->cap > 0)) return CEL_OK;
    }
    const int Kn = stages_of(m0) - 1;
    // the cycle's argument blocks must all be in the table already
    {
        int64_t nh = m0->nh;
        int cur = m0->cur, pcur = m0->pcur;
        for (int i = 0; i < 6; i++) {   // as finish_step moves them on
            for (int stage = 0; stage <= Kn; stage++)
                if (std::find(e->keys.begin(), e->keys.end(), ens_key_of(nh, cur, pcur, stage)) == e->keys.end())
                    return CEL_OK;
            cur = (cur + Kn + 1) & 1;
            pcur = 1 - pcur;
            nh++;
        }
    }
    const int64_t k = e->gmem.empty() ? 0 : e->m[e->gmem[0]]->step - e->gstep0[0];
    int64_t *kdev = reinterpret_cast<int64_t *>(e->tab + e->off_kdev);
    const uint64_t key = ens_key(m0, 0);
    cel_ensemble::Graph *g = nullptr;
    for (cel_ensemble::Graph &h : e->graphs)
        if (h.key == key) g = &h;
    if (!g) {
        // capture the cycle on the library's own stream (the caller's may be
        // the legacy default stream, which cannot be captured); the members'
        // bookkeeping moves on as the launches are recorded, and is put back
        // if the capture fails
        if (!e->cap_stream && cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            e->cap_stream = nullptr;
            cudaGetLastError();
            return CEL_OK;
        }
        struct Saved {
            int cur, pcur;
            int64_t step, nh;
        };
        std::vector<Saved> saved(n);
        for (int j = 0; j < n; j++) saved[j] = {e->m[j]->cur, e->m[j]->pcur, e->m[j]->step, e->m[j]->nh};
        auto restore = [&]() {
            for (int j = 0; j < n; j++) {
                e->m[j]->cur = saved[j].cur;
                e->m[j]->pcur = saved[j].pcur;
                e->m[j]->step = saved[j].step;
                e->m[j]->nh = saved[j].nh;
            }
        };
        if (cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return CEL_OK;
        }
        int64_t lc = 0;
        cel_status cs = CEL_OK;
        for (int i = 0; i < 6 && cs == CEL_OK; i++) cs = ens_launch_step<real>(e, e->cap_stream, kdev, i, lc);
        if (cs == CEL_OK && launch_counter(kdev, 6, 1, e->cap_stream) != cudaSuccess) cs = CEL_ERR_CUDA;
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(e->cap_stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (cs == CEL_OK && ce == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            cudaGraphDestroy(graph);
            e->graphs.push_back(cel_ensemble::Graph{key, exec, lc});
            g = &e->graphs.back();
            restore();   // the replay below moves the bookkeeping on
        } else {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            restore();
            e->err.clear();
            return CEL_OK;   // the steps are taken one at a time instead
        }
    }
    if (!e->kdev_known || e->kdev_val != k)
        ENS_CUDA(e, launch_counter(kdev, k, 0, e->stream), "ensemble step counter");
    ENS_CUDA(e, cudaGraphLaunch(g->exec, e->stream), "ensemble graph");
    e->kdev_val = k + 6;
    e->kdev_known = true;
    for (int i = 0; i < 6; i++)
        for (int j = 0; j < n; j++) finish_step(e->m[j], Kn);
    launches += g->launches;
    e->graph_steps += 6;
    *done = true;
    return CEL_OK;
}

// The remaining nsteps steps as one persistent cooperative launch, where the
// captured cycle's conditions hold (history full, no gauges, run-up tracking
// or profiling, every argument block of the 6-step cycle in the table) and
// every line family takes the register path in blocks of at most 256
// threads.  *done: the steps were taken.
template <typename real>
cel_status ens_persistent(cel_ensemble *e, int nsteps, int64_t &launches, bool *done)
{
    *done = false;
    const int n = (int)e->m.size();
    const cel_solver *m0 = e->m[0];
    if (!e->use_persist || nsteps < 1 || m0->nh < 2 || e->prof.cap > 0) return CEL_OK;
    for (int j = 0; j < n; j++) {
        const cel_solver *s = e->m[j];
        if (s->runup || (s->ng > 0 && s->log_every > 0 && s->cap > 0)) return CEL_OK;
    }
    const int Kn = stages_of(m0) - 1;
    if (Kn + 1 > kPersistMaxStages) return CEL_OK;
    PersistArgs<real> P;
    memset(&P, 0, sizeof(P));
    {
        int64_t nh = m0->nh;
        int cur = m0->cur, pcur = m0->pcur;
        for (int i = 0; i < 6; i++) {
            for (int stage = 0; stage <= Kn; stage++) {
                auto it = std::find(e->keys.begin(), e->keys.end(), ens_key_of(nh, cur, pcur, stage));
                if (it == e->keys.end()) return CEL_OK;
                P.ent[i][stage] = (int)(it - e->keys.begin());
            }
            cur = (cur + Kn + 1) & 1;
            pcur = 1 - pcur;
            nh++;
        }
    }
    // line runs: families of one group with one segment length and one model,
    // in table order (the solver's barriers are taken by Boussinesq lines
    // alone, so lines of both models never share a block)
    int nruns = 0;
    for (const cel_ensemble::Group &G : e->groups) {
        if (G.cfg.algo != 0 || G.cfg.threads > kStencilThreads) return CEL_OK;
        size_t off = G.off_desc;
        int prev = -1;
        for (int f = 0; f < G.nfam; f++) {
            const std::pair<int, int> &fm = e->fam[G.first + f];
            const cel_solver *s = e->m[fm.first];
            const int len = fm.second == 0 ? s->geo.nx : s->geo.ny, nl = fm.second == 0 ? s->geo.ny : s->geo.nx;
            const int ident = s->params.model == CEL_NLSW;
            const int msh = line_config(len, (int)sizeof(real)).mshift;
            if (msh * 2 + ident != prev) {
                if (nruns == kPersistMaxRuns) return CEL_OK;
                P.run_desc[nruns] = reinterpret_cast<const int2 *>(e->tab + off);
                P.run_first[nruns] = G.first;
                P.run_lines[nruns] = 0;
                P.run_threads[nruns] = G.cfg.threads;
                P.run_mshift[nruns] = msh;
                P.run_identity[nruns] = ident;
                P.run_nfam[nruns] = G.nfam;
                nruns++;
                prev = msh * 2 + ident;
            }
            P.run_lines[nruns - 1] += nl;
            off += sizeof(int2) * (size_t)nl;
        }
    }
    const int grid = persistent_grid<real>();
    if (grid <= 0) return CEL_OK;
    P.nruns = nruns;
    P.run_pass0[0] = 0;
    for (int r = 0; r < nruns; r++) {
        const int G = kStencilThreads / P.run_threads[r];
        P.run_pass0[r + 1] = P.run_pass0[r] + (P.run_lines[r] + G - 1) / G;
    }
    P.nmembers = n;
    P.nent = (int)e->keys.size();
    P.entries = e->tab + e->off_entries;
    P.entry_bytes = e->entry_bytes;
    P.sarg_bytes = e->sarg_bytes;
    for (int stage = 0; stage <= Kn; stage++) {
        StencilArgs<real> a;
        memset(&a, 0, sizeof(a));
        a.kind = stage == 0 ? kAB3 : kAM4;
        a.ring = e->K > 0;
        P.spec[stage] = stencil_spec(a);
    }
    P.nstages = Kn + 1;
    P.phase0 = 0;
    P.nsteps = nsteps;
    P.tile_desc = reinterpret_cast<const int2 *>(e->tab + e->off_tile_desc);
    P.tiles = e->tiles;
    if (!e->gmem.empty()) {
        P.gargs = reinterpret_cast<const GhostArgs<real> *>(e->tab + e->off_gargs);
        P.gstart = reinterpret_cast<const int *>(e->tab + e->off_gstart);
        P.ngm = (int)e->gmem.size();
        P.gblocks = e->gblocks;
        P.k0 = e->m[e->gmem[0]]->step - e->gstep0[0];
    }
    P.bar = reinterpret_cast<unsigned *>(e->tab + e->off_bar);
    P.work = reinterpret_cast<int *>(P.bar + 4);
    P.expect = (unsigned)grid;
    P.timeout_ns = (long long)(e->persist_timeout_ms * 1e6);
    ENS_CUDA(e, cudaMemsetAsync(P.bar, 0, 8 * sizeof(unsigned), e->stream), "persistent barrier words");
    ENS_CUDA(e, launch_persistent<real>(P, grid, e->stream), "persistent ensemble launch");
    for (int i = 0; i < nsteps; i++)
        for (int j = 0; j < n; j++) finish_step(e->m[j], Kn);
    e->kdev_known = false;   // the device step counter was not advanced
    launches += 1;
    e->persist_steps += nsteps;
    *done = true;
    return CEL_OK;
}

template <typename real>
cel_status ens_step_t(cel_ensemble *e, int nsteps)
{
    int64_t launches = 0;
    for (int it = 0; it < nsteps;) {
        cel_status st = ens_prepare<real>(e, launches);
        if (st != CEL_OK) return st;
        {
            bool done = false;
            st = ens_persistent<real>(e, nsteps - it, launches, &done);
            if (st != CEL_OK) return st;
            if (done) break;
        }
        if (nsteps - it >= 6) {
            bool done = false;
            st = ens_graph_cycle<real>(e, launches, &done);
            if (st != CEL_OK) return st;
            if (done) {
                it += 6;
                continue;
            }
        }
        const int64_t k = e->gmem.empty() ? 0 : e->m[e->gmem[0]]->step - e->gstep0[0];
        st = ens_launch_step<real>(e, e->stream, nullptr, k, launches);
        if (st != CEL_OK) return st;
        it += 1;
    }
    e->launches = launches;
    return CEL_OK;
}

}  // namespace

extern "C" {

cel_status cel_ensemble_table_bytes(cel_solver *const *members, int32_t n, size_t *bytes)
{
    if (!bytes) return CEL_ERR_INVALID_ARG;
    EnsPlan P;
    std::string why;
    cel_status st = plan(members, n, P, why);
    if (st != CEL_OK) return st;
    *bytes = P.total;
    return CEL_OK;
}

cel_status cel_ensemble_create(cel_solver *const *members, int32_t n, void *table_dev, size_t table_bytes,
                               void *cuda_stream, cel_ensemble **out, char *msg, size_t msg_len)
{
    put_msg(msg, msg_len, "");
    if (!out) return CEL_ERR_INVALID_ARG;
    *out = nullptr;
    EnsPlan P;
    std::string why;
    const int split_gen = line_split_generation();
    cel_status st = plan(members, n, P, why);
    if (st != CEL_OK) {
        put_msg(msg, msg_len, why);
        return st;
    }
    if (!table_dev || ((uintptr_t)table_dev & 255) != 0) {
        put_msg(msg, msg_len, "the table must be device memory aligned to 256 bytes");
        return CEL_ERR_INVALID_ARG;
    }
    if (table_bytes < P.total) {
        put_msg(msg, msg_len, "table smaller than cel_ensemble_table_bytes");
        return CEL_ERR_WORKSPACE_TOO_SMALL;
    }
    cel_ensemble *e = new cel_ensemble();
    e->split_gen = split_gen;
    e->m.assign(members, members + n);
    e->es = members[0]->es;
    e->K = members[0]->params.corrector_iters;
    e->stream = (cudaStream_t)cuda_stream;
    e->tab = (unsigned char *)table_dev;
    e->tab_bytes = table_bytes;
    e->tiles = P.tiles;
    e->off_tile_desc = P.off_tile_desc;
    e->fam = P.fam;
    e->groups = P.groups;
    e->gmem = P.gmem;
    e->gblocks = P.gblocks;
    e->off_gargs = P.off_gargs;
    e->off_gstart = P.off_gstart;
    e->off_kdev = P.off_kdev;
    e->off_bar = P.off_bar;
    e->gstep0.assign(P.gmem.size(), 0);
    e->gvalid = false;
    e->sarg_bytes = P.sarg_bytes;
    e->entry_bytes = P.entry_bytes;
    e->off_entries = P.off_entries;
    e->cap = P.cap;
    e->gen_sum = 0;
    for (int j = 0; j < n; j++) e->gen_sum += members[j]->gen;
    e->launches = 0;
    // block descriptors: (member, tile) of every stencil block, (family,
    // line) of every line block
    std::vector<int2> td;
    td.reserve(P.tiles);
    for (int j = 0; j < n; j++) {
        const int tx = (members[j]->geo.nx + kTile - 1) / kTile, ty = (members[j]->geo.ny + kTile - 1) / kTile;
        for (int b = 0; b < tx * ty; b++) td.push_back(make_int2(j, ((b / tx) << 16) | (b % tx)));
    }
    cudaError_t ce = cudaMemcpyAsync(e->tab + e->off_tile_desc, td.data(), sizeof(int2) * td.size(),
                                     cudaMemcpyHostToDevice, e->stream);
    for (const cel_ensemble::Group &G : e->groups) {
        if (ce != cudaSuccess) break;
        std::vector<int2> ld;
        ld.reserve(G.blocks);
        for (int f = 0; f < G.nfam; f++) {
            const std::pair<int, int> &fm = e->fam[G.first + f];
            const int nl = fm.second == 0 ? members[fm.first]->geo.ny : members[fm.first]->geo.nx;
            for (int l = 0; l < nl; l++) ld.push_back(make_int2(f, l));
        }
        ce = cudaMemcpyAsync(e->tab + G.off_desc, ld.data(), sizeof(int2) * ld.size(), cudaMemcpyHostToDevice,
                             e->stream);
    }
    if (ce != cudaSuccess) {
        put_msg(msg, msg_len, std::string("ensemble tables: ") + cudaGetErrorString(ce));
        delete e;
        return CEL_ERR_CUDA;
    }
    *out = e;
    return CEL_OK;
}

cel_status cel_ensemble_step(cel_ensemble *e, int32_t nsteps)
{
    if (!e || nsteps < 0) return CEL_ERR_INVALID_ARG;
    return e->es == 4 ? ens_step_t<float>(e, nsteps) : ens_step_t<double>(e, nsteps);
}

cel_status cel_ensemble_last_launch_count(const cel_ensemble *e, int64_t *launches)
{
    if (!e || !launches) return CEL_ERR_INVALID_ARG;
    *launches = e->launches;
    return CEL_OK;
}

cel_status cel_ensemble_profile_enable(cel_ensemble *e, int32_t capacity)
{
    if (!e || capacity < 1 || capacity > (1 << 20)) return CEL_ERR_INVALID_ARG;
    cudaError_t ce = e->prof.create(capacity);
    if (ce != cudaSuccess) return ens_fail(e, CEL_ERR_CUDA, std::string("profile events: ") + cudaGetErrorString(ce));
    return CEL_OK;
}

cel_status cel_ensemble_profile_read(cel_ensemble *e, double ms[3], int64_t count[3])
{
    if (!e || !ms || !count) return CEL_ERR_INVALID_ARG;
    cudaError_t ce = e->prof.read(e->stream, ms, count);
    if (ce != cudaSuccess) return ens_fail(e, CEL_ERR_CUDA, std::string("profile read: ") + cudaGetErrorString(ce));
    return CEL_OK;
}

cel_status cel_ensemble_profile_disable(cel_ensemble *e)
{
    if (!e) return CEL_ERR_INVALID_ARG;
    e->prof.release();
    return CEL_OK;
}

const char *cel_ensemble_last_error(const cel_ensemble *e) { return e ? e->err.c_str() : ""; }

cel_status cel_ensemble_graph_steps(const cel_ensemble *e, int64_t *steps)
{
    if (!e || !steps) return CEL_ERR_INVALID_ARG;
    *steps = e->graph_steps;
    return CEL_OK;
}

cel_status cel_ensemble_use_graphs(cel_ensemble *e, int32_t enable)
{
    if (!e) return CEL_ERR_INVALID_ARG;
    e->use_graphs = enable != 0;
    if (!e->use_graphs) e->drop_graphs();
    return CEL_OK;
}

cel_status cel_ensemble_use_persistent(cel_ensemble *e, int32_t enable, double timeout_ms)
{
    if (!e) return CEL_ERR_INVALID_ARG;
    if (!(timeout_ms > 0.0) || timeout_ms > 60000.0)
        return ens_fail(e, CEL_ERR_INVALID_ARG, "the barrier timeout must lie in (0, 60000] ms");
    if (enable && (e->es == 4 ? persistent_grid<float>() : persistent_grid<double>()) <= 0)
        return ens_fail(e, CEL_ERR_CUDA, "no block of the persistent launch fits an SM");
    e->use_persist = enable != 0;
    e->persist_timeout_ms = timeout_ms;
    return CEL_OK;
}

cel_status cel_ensemble_persistent_steps(const cel_ensemble *e, int64_t *steps)
{
    if (!e || !steps) return CEL_ERR_INVALID_ARG;
    *steps = e->persist_steps;
    return CEL_OK;
}

namespace {
// Reads the barrier status after the stream's work and clears the words.
cel_status ens_read_barrier(cel_ensemble *e, unsigned *status)
{
    unsigned w[4] = {0, 0, 0, 0};
    ENS_CUDA(e, cudaStreamSynchronize(e->stream), "ensemble stream");
    ENS_CUDA(e, cudaMemcpy(w, e->tab + e->off_bar, sizeof(w), cudaMemcpyDeviceToHost), "persistent barrier words");
    ENS_CUDA(e, cudaMemset(e->tab + e->off_bar, 0, 8 * sizeof(unsigned)), "persistent barrier words");
    *status = w[2];
    if (w[3] != 0)
        return ens_fail(e, CEL_ERR_INVALID_ARG,
                        "the persistent launch met a descriptor out of range (code " + std::to_string(w[3] >> 24) +
                            ", index " + std::to_string(w[3] & 0xffffffu) + ") and skipped its work");
    return CEL_OK;
}
}  // namespace

cel_status cel_ensemble_check(cel_ensemble *e)
{
    if (!e) return CEL_ERR_INVALID_ARG;
    unsigned status = 0;
    cel_status st = ens_read_barrier(e, &status);
    if (st != CEL_OK) return st;
    if (status != 0)
        return ens_fail(e, CEL_ERR_TIMEOUT,
                        "a wait of the persistent launch ran out: the members' states are undefined (set them again)");
    return CEL_OK;
}

cel_status cel_ensemble_barrier_check(cel_ensemble *e, int32_t missing, double timeout_ms, int32_t *timed_out)
{
    if (!e || !timed_out || missing < 0 || missing > 1024 || !(timeout_ms > 0.0) || timeout_ms > 60000.0)
        return CEL_ERR_INVALID_ARG;
    const int grid = e->es == 4 ? persistent_grid<float>() : persistent_grid<double>();
    if (grid <= 0) return ens_fail(e, CEL_ERR_CUDA, "no block of the persistent launch fits an SM");
    ENS_CUDA(e, cudaMemsetAsync(e->tab + e->off_bar, 0, 8 * sizeof(unsigned), e->stream), "persistent barrier words");
    cudaError_t ce;
    if (e->es == 4) {
        PersistArgs<float> P;
        memset(&P, 0, sizeof(P));
        P.barrier_only = 1;
        P.bar = reinterpret_cast<unsigned *>(e->tab + e->off_bar);
        P.expect = (unsigned)(grid + missing);
        P.timeout_ns = (long long)(timeout_ms * 1e6);
        ce = launch_persistent<float>(P, grid, e->stream);
    } else {
        PersistArgs<double> P;
        memset(&P, 0, sizeof(P));
        P.barrier_only = 1;
        P.bar = reinterpret_cast<unsigned *>(e->tab + e->off_bar);
        P.expect = (unsigned)(grid + missing);
        P.timeout_ns = (long long)(timeout_ms * 1e6);
        ce = launch_persistent<double>(P, grid, e->stream);
    }
    ENS_CUDA(e, ce, "persistent barrier check");
    unsigned status = 0;
    cel_status st = ens_read_barrier(e, &status);
    if (st != CEL_OK) return st;
    *timed_out = status != 0;
    return CEL_OK;
}

void cel_ensemble_destroy(cel_ensemble *e)
{
    if (!e) return;
    e->prof.release();
    e->drop_graphs();
    if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
    delete e;
}

}  // extern "C"

// ------------------------------------------------------- discrete adjoint
//
// Gradient of the gauge misfit L = 1/2 sum_{n=1..N} sum_g (eta_g^n - obs_g^n)^2
// with respect to w at the start and the bed, by the reverse of every stage
// of every step (kernels in celeris_adjoint.cu).  The forward run keeps a
// checkpoint every C steps; the reverse sweep goes through the segments
// from the last, each recomputed from its checkpoint (the resume is
// bit-exact) on the solver's stream while the segment after it is reversed
// on a stream of its own.

namespace {

struct AdjLayout {
    size_t ckpt_bytes, cells_bytes, line_bytes;
    size_t ckpt, seg, iter, lam, G, rec, gij, total;
    size_t seg_slot, iter_slot, rhs_slot;   // two slots each: one segment recomputed while the next is reversed
    size_t gtab, xy;                        // the reverse's own ghost table and line-layout scratch
    size_t rhs, lBc, lBb, ld, ldl, lg;       // the bed's gradient (bed != 0)
    size_t ghost_bytes;
    int nseg, bed;
    int keep;   // every step kept from the forward run: one segment, one slot, no recomputation
};

AdjLayout adj_layout(const cel_solver *s, int N, int C, int ng, int bed)
{
    AdjLayout L;
    L.bed = bed;
    L.keep = C == 0;
    if (L.keep) C = N;
    const int slots = L.keep ? 1 : 2;
    L.ckpt_bytes = align256(ckpt_total(s));
    L.cells_bytes = align256((size_t)s->grid.nx * s->grid.ny * s->es);
    L.line_bytes = align256(std::max((size_t)s->geo.ny * s->geo.px, (size_t)s->geo.nx * s->geo.py) * s->es);
    L.nseg = (N + C - 1) / C;
    size_t cur = 0;
    auto take = [&](size_t b) {
        size_t o = cur;
        cur += align256(b);
        return o;
    };
    L.ckpt = take(L.ckpt_bytes * (size_t)(L.nseg + 1));   // + the final state
    const int K = s->params.corrector_iters;
    L.seg_slot = L.cells_bytes * 3 * (size_t)(C + 1);
    L.seg = take(L.seg_slot * slots);
    L.iter_slot = L.cells_bytes * 3 * (size_t)K * (size_t)(C + 1);   // the iterates of every step
    L.iter = take(L.iter_slot * slots);
    L.lam = take(L.cells_bytes * 9);   // 3 sets of (w, P, Q)
    L.G = take(L.cells_bytes * 20);    // 3 steps x (E, F, G, F*, G*), and the corrector's
    L.rec = take((size_t)N * ng * s->es);
    L.gij = take((size_t)ng * 2 * sizeof(int32_t));
    L.rhs = L.lBc = L.lBb = L.ld = L.ldl = L.lg = 0;
    L.rhs_slot = 0;
    L.ghost_bytes = ghost_index(2, 0, 0, 0, 0, (s->geo.nx > s->geo.ny ? s->geo.nx : s->geo.ny) + 4) * s->es;
    L.gtab = take(L.ghost_bytes);
    L.xy = take(L.line_bytes * 2);
    if (bed) {
        const bool lines = s->params.model == CEL_BSNQ;
        L.rhs_slot = lines ? L.line_bytes * 2 * (size_t)(K + 1) * (size_t)C : 0;   // every stage's line solutions
        L.rhs = take(L.rhs_slot * slots);
        L.ldl = take(lines ? L.line_bytes * 2 : 0);                                 // ld of the line systems
        L.lBc = take((size_t)s->geo.pc * (s->grid.ny + 3) * s->es);
        L.lBb = take((size_t)(s->grid.nx + 2) * (s->grid.ny + 2) * s->es);
        L.ld = take((size_t)(s->grid.nx + 2) * (s->grid.ny + 2) * s->es);
        L.lg = take(L.ghost_bytes);   // the sine makers' ghost values
    }
    L.total = cur;
    return L;
}

// Weights of R^n, R^{n-1}, R^{n-2} (c) and of F*^n, F*^{n-1}, F*^{n-2} (e)
// in the update of step n of a fresh history, predictor only (Eq. 15-17;
// Euler for the first two steps, the second adding F*^1 - F*^0).
void adj_coefs(int64_t n, double dt, double c[3], double e[3])
{
    if (n < 2) {
        c[0] = dt;
        c[1] = c[2] = 0.0;
        e[0] = n == 1 ? 1.0 : 0.0;
        e[1] = n == 1 ? -1.0 : 0.0;
        e[2] = 0.0;
    } else {
        c[0] = 23.0 * dt / 12.0;
        c[1] = -16.0 * dt / 12.0;
        c[2] = 5.0 * dt / 12.0;
        e[0] = 2.0;
        e[1] = -3.0;
        e[2] = 1.0;
    }
}

template <typename real>
cel_status adjoint_t(cel_solver *s, int N, int C, const int32_t *gij_host, int ng, const real *obs, unsigned char *scr,
                     const AdjLayout &L, real *eta_out, real *grad, real *grad_z, double *loss)
{
    cudaStream_t st = s->stream;
    if (L.keep) C = N;
    const size_t cells = (size_t)s->grid.nx * s->grid.ny;
    int32_t *gij = reinterpret_cast<int32_t *>(scr + L.gij);
    real *rec = reinterpret_cast<real *>(scr + L.rec);
    CEL_CUDA(s, cudaMemcpyAsync(gij, gij_host, sizeof(int32_t) * 2 * ng, cudaMemcpyHostToDevice, st), "adjoint gauges");
    auto ckpt = [&](int k) { return scr + L.ckpt + L.ckpt_bytes * (size_t)k; };
    // segment sg's recomputed data live in slot sg & 1
    int slot = 0;   // the slot the reverse is reading
    auto segf_in = [&](int sl, int k, int v) {
        return reinterpret_cast<real *>(scr + L.seg + L.seg_slot * sl + L.cells_bytes * (3 * (size_t)k + v));
    };
    auto segf = [&](int k, int v) { return segf_in(slot, k, v); };
    auto lam = [&](int v) { return reinterpret_cast<real *>(scr + L.lam + L.cells_bytes * v); };
    auto Gb = [&](int sl, int v) { return reinterpret_cast<real *>(scr + L.G + L.cells_bytes * (5 * sl + v)); };
    const int K = s->params.corrector_iters;
    auto iterf_in = [&](int sl, int k, int stage, int v) {   // iterate after `stage` of step k of the segment
        return reinterpret_cast<real *>(scr + L.iter + L.iter_slot * sl +
                                        L.cells_bytes * (3 * ((size_t)k * K + stage) + v));
    };
    auto iterf = [&](int k, int stage, int v) { return iterf_in(slot, k, stage, v); };
    const bool bed = grad_z != nullptr, bed_lines = bed && s->params.model == CEL_BSNQ;
    auto rhsf_in = [&](int sl, int k, int stage) {   // line solutions of `stage` of step k of the segment
        return scr + L.rhs + L.rhs_slot * sl + L.line_bytes * 2 * ((size_t)k * (K + 1) + stage);
    };
    auto rhsf = [&](int k, int stage) { return rhsf_in(slot, k, stage); };
    const int64_t step0 = s->step;
    cel_status stt;
    // forward, with checkpoints and the gauge records
    struct Range {   // an NVTX range over a scope
        explicit Range(const char *name) { nvtxRangePushA(name); }
        ~Range() { nvtxRangePop(); }
    };
    Range whole("cel adjoint");
    // the state before step k of a segment, into slot sl
    auto keep_state = [&](int sl, int k, cudaStream_t q) {
        return launch_get_state<real>(s->geo, s->at<real>(s->lay.w[s->cur]), s->at<real>(s->lay.P[s->pcur]),
                                      s->at<real>(s->lay.Qc[s->pcur]), segf_in(sl, k, 0), segf_in(sl, k, 1),
                                      segf_in(sl, k, 2), q);
    };
    // one step, its corrector iterates and line solutions kept in slot sl
    auto kept_step = [&](int sl, int k) -> cel_status {
        s->capture = K > 0 ? reinterpret_cast<unsigned char *>(iterf_in(sl, k, 0, 0)) : nullptr;
        s->capture_field = L.cells_bytes;
        s->capture_rhs = bed_lines ? rhsf_in(sl, k, 0) : nullptr;
        s->capture_line = L.line_bytes;
        const cel_status r = step_t<real>(s, 1);
        s->capture = nullptr;
        s->capture_rhs = nullptr;
        return r;
    };
    for (int n = 0; n < N; n++) {
        if (n % C == 0 && (stt = cel_save_checkpoint(s, ckpt(n / C), L.ckpt_bytes)) != CEL_OK) return stt;
        if (L.keep) {   // the forward run keeps what the reverse reads
            CEL_CUDA(s, keep_state(0, n, st), "adjoint states");
            stt = kept_step(0, n);
        } else {
            stt = step_t<real>(s, 1);
        }
        if (stt != CEL_OK) return stt;
        CEL_CUDA(s, launch_gauges<real>(s->geo, s->phy, s->at<real>(s->lay.w[s->cur]), gij, ng, rec + (size_t)n * ng, st),
                 "adjoint gauges");
    }
    if (L.keep) CEL_CUDA(s, keep_state(0, N, st), "adjoint states");
    if ((stt = cel_save_checkpoint(s, ckpt(L.nseg), L.ckpt_bytes)) != CEL_OK) return stt;
    {
        std::vector<real> r((size_t)N * ng), o((size_t)N * ng);
        CEL_CUDA(s, cudaMemcpyAsync(r.data(), rec, sizeof(real) * r.size(), cudaMemcpyDeviceToHost, st), "adjoint loss");
        CEL_CUDA(s, cudaMemcpyAsync(o.data(), obs, sizeof(real) * o.size(), cudaMemcpyDeviceToHost, st), "adjoint loss");
        CEL_CUDA(s, cudaStreamSynchronize(st), "adjoint loss");
        double acc = 0.0;
        for (size_t k = 0; k < r.size(); k++) acc += 0.5 * ((double)r[k] - (double)o[k]) * ((double)r[k] - (double)o[k]);
        if (loss) *loss = acc;
    }
    // reverse, on a stream of its own: segment sg is reversed while segment
    // sg - 1 is recomputed on the solver's stream (the solver's workspace
    // belongs to the recomputation; the reverse has its own ghost table and
    // line scratch).  Events order the two: rec[slot] when a slot's segment
    // is recomputed, rev[slot] when its reverse is done with it.
    // The line systems' depth term (a re-solve and a gather per stage, read
    // by nothing until the end) runs on a third stream beside the stage's
    // history and Jacobian passes: it starts when the transposed solves are
    // done (event mu) and the reverse waits for it (event tri) before the
    // next mask pass rewrites their solutions, before the ghost table is
    // rewritten or its adjoints mapped, and before a segment's slot is freed.
    struct Streams {
        cudaStream_t rs = nullptr, ts = nullptr;
        cudaEvent_t rec[2] = {nullptr, nullptr}, rev[2] = {nullptr, nullptr}, fin = nullptr, mu = nullptr,
                    tri = nullptr;
        ~Streams()
        {
            for (cudaStream_t q : {rs, ts})
                if (q) {
                    cudaStreamSynchronize(q);
                    cudaStreamDestroy(q);
                }
            for (int k = 0; k < 2; k++) {
                if (rec[k]) cudaEventDestroy(rec[k]);
                if (rev[k]) cudaEventDestroy(rev[k]);
            }
            for (cudaEvent_t e : {fin, mu, tri})
                if (e) cudaEventDestroy(e);
        }
    } ss;
    CEL_CUDA(s, cudaStreamCreateWithFlags(&ss.rs, cudaStreamNonBlocking), "adjoint stream");
    CEL_CUDA(s, cudaStreamCreateWithFlags(&ss.ts, cudaStreamNonBlocking), "adjoint stream");
    for (int k = 0; k < 2; k++) {
        CEL_CUDA(s, cudaEventCreateWithFlags(&ss.rec[k], cudaEventDisableTiming), "adjoint events");
        CEL_CUDA(s, cudaEventCreateWithFlags(&ss.rev[k], cudaEventDisableTiming), "adjoint events");
    }
    CEL_CUDA(s, cudaEventCreateWithFlags(&ss.fin, cudaEventDisableTiming), "adjoint events");
    CEL_CUDA(s, cudaEventCreateWithFlags(&ss.mu, cudaEventDisableTiming), "adjoint events");
    CEL_CUDA(s, cudaEventCreateWithFlags(&ss.tri, cudaEventDisableTiming), "adjoint events");
    bool tri_pending = false;   // the depth term's stream has work the reverse must wait for
    auto wait_tri = [&]() -> cudaError_t {
        if (!tri_pending) return cudaSuccess;
        tri_pending = false;
        return cudaStreamWaitEvent(ss.rs, ss.tri, 0);
    };
    const cudaStream_t fst = st;   // forward and recomputation
    st = ss.rs;                    // the reverse
    real *gtab = reinterpret_cast<real *>(scr + L.gtab);
    real *Xr = reinterpret_cast<real *>(scr + L.xy), *Yr = reinterpret_cast<real *>(scr + L.xy + L.line_bytes);
    // lam sets 0-2: the adjoint of the state after the step (then before
    // it), of the present iterate, and the accumulator of the state before
    // the step.
    CEL_CUDA(s, cudaMemsetAsync(scr + L.lam, 0, L.cells_bytes * 9, st), "adjoint");
    CEL_CUDA(s, cudaMemsetAsync(scr + L.G, 0, L.cells_bytes * 20, st), "adjoint");
    AdjArgs<real> a;
    memset(&a, 0, sizeof(a));
    a.geo = s->geo;
    a.phy = s->phy;
    a.c = make_coef<real>(s->geo, s->phy, s->bnd);
    a.Bc = s->at<real>(s->lay.Bc);
    a.ghost = gtab;
    a.bsnq = s->params.model == CEL_BSNQ;
    if (bed) {
        a.lBc = reinterpret_cast<real *>(scr + L.lBc);
        a.lBb = reinterpret_cast<real *>(scr + L.lBb);
        a.ld = reinterpret_cast<real *>(scr + L.ld);
        CEL_CUDA(s, cudaMemsetAsync(a.lBc, 0, (size_t)s->geo.pc * (s->grid.ny + 3) * sizeof(real), st), "adjoint");
        CEL_CUDA(s, cudaMemsetAsync(a.lBb, 0, (size_t)(s->grid.nx + 2) * (s->grid.ny + 2) * sizeof(real), st), "adjoint");
        CEL_CUDA(s, cudaMemsetAsync(a.ld, 0, (size_t)(s->grid.nx + 2) * (s->grid.ny + 2) * sizeof(real), st), "adjoint");
        if (a.c.sine) {
            a.lg = reinterpret_cast<real *>(scr + L.lg);
            CEL_CUDA(s, cudaMemsetAsync(a.lg, 0, L.ghost_bytes, st), "adjoint");
        }
        if (bed_lines) {
            a.ldx = reinterpret_cast<real *>(scr + L.ldl);
            a.ldy = reinterpret_cast<real *>(scr + L.ldl + L.line_bytes);
            CEL_CUDA(s, cudaMemsetAsync(scr + L.ldl, 0, L.line_bytes * 2, st), "adjoint");
        }
    }
    int lset = 0;   // which lam set holds the adjoint of the state after the step
    auto setl = [&](AdjArgs<real> &x, int set) {
        x.lw = lam(3 * set);
        x.lP = lam(3 * set + 1);
        x.lQ = lam(3 * set + 2);
    };
    auto setG = [&](AdjArgs<real> &x, int slot0, int slot1, int slot2) {
        for (int v = 0; v < 5; v++) {
            x.G0[v] = Gb(slot0, v);
            x.G1[v] = slot1 >= 0 ? Gb(slot1, v) : nullptr;
            x.G2[v] = slot2 >= 0 ? Gb(slot2, v) : nullptr;
        }
    };
    auto coefs = [&](AdjArgs<real> &x, double c0, double c1, double c2, double e0, double e1, double e2) {
        x.c0 = real(c0);
        x.c1 = real(c1);
        x.c2 = real(c2);
        x.e0 = real(e0);
        x.e1 = real(e1);
        x.e2 = real(e2);
    };
    // the line solves' arguments for the reverse: its own ghost table
    auto rline = [&](const AdjArgs<real> &x, int dir) {
        LineArgs<real> l = line_args<real>(s, x.c, dir, 0, 0);
        l.ghost = gtab;
        l.identity = 0;
        return l;
    };
    // the transposed line solves (Boussinesq) through the forward's line
    // solver, in the reverse's line-layout scratch;
    // after it the history phase reads the U*, V* adjoints from x.muX, x.muY
    // (Boussinesq: the solutions in the line layouts) or x.ldU, x.ldV (the
    // shallow-water model, where U* = P: the masked lP, lQ themselves)
    auto solves = [&](AdjArgs<real> &x) -> cudaError_t {
        if (!x.bsnq) {
            x.ldU = x.lP;
            x.ldV = x.lQ;
            x.muX = x.muY = nullptr;
            return cudaSuccess;
        }
        x.muX = Xr;
        x.muY = Yr;
        LinePair<real> lp;   // the right sides: the mask phase wrote them to Xr, Yr
        for (int dir = 0; dir < 2; dir++) {
            lp.L[dir] = rline(x, dir);
            real *buf = dir == 0 ? Xr : Yr;
            lp.L[dir].rhs = buf;
            lp.L[dir].base = buf;
            lp.L[dir].sol = buf;
        }
        return launch_lines_transposed<real>(lp, st);
    };
    // the line systems' dependence on d: the stage's solutions again from
    // its line solutions kept by the forward run, with the transposed solves' still in Xr, Yr
    auto tri_bed = [&](const AdjArgs<real> &x, int k, int stage) -> cudaError_t {
        if (!bed_lines) return cudaSuccess;
        cudaError_t e = cudaEventRecord(ss.mu, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ss.ts, ss.mu, 0);
        if (e != cudaSuccess) return e;
        // the stage's line solutions, kept by the forward run's line solves
        const real *Xs = reinterpret_cast<const real *>(rhsf(k, stage));
        const real *Ys = reinterpret_cast<const real *>(rhsf(k, stage) + L.line_bytes);
        e = launch_adjoint_tri_bed<real>(x, Xs, Ys, Xr, Yr, s->at<real>(s->lay.dr), s->at<real>(s->lay.dc), ss.ts);
        if (e == cudaSuccess) e = cudaEventRecord(ss.tri, ss.ts);
        tri_pending = e == cudaSuccess;
        return e;
    };
    // the mask phase, writing the Boussinesq solves' right sides as well
    auto mask = [&](AdjArgs<real> &x, int zero_set) -> cudaError_t {
        cudaError_t w = wait_tri();   // it rewrites Xr, Yr
        if (w != cudaSuccess) return w;
        x.packX = x.bsnq ? Xr : nullptr;
        x.packY = x.bsnq ? Yr : nullptr;
        for (int v = 0; v < 3; v++) x.zero[v] = zero_set >= 0 ? lam(3 * zero_set + v) : nullptr;
        cudaError_t e = launch_adjoint_mask<real>(x, st);
        x.packX = x.packY = nullptr;
        for (int v = 0; v < 3; v++) x.zero[v] = nullptr;
        return e;
    };
    auto full_step = [&](AdjArgs<real> &x, int k) -> cudaError_t {
        cudaError_t e = mask(x, -1);
        if (e == cudaSuccess) e = solves(x);
        if (e == cudaSuccess) e = tri_bed(x, k, 0);
        if (e == cudaSuccess) e = launch_adjoint_hist<real>(x, st);
        if (e == cudaSuccess) e = launch_adjoint_vjp<real>(x, st);
        return e;
    };
    setl(a, lset);
    CEL_CUDA(s, launch_adjoint_misfit<real>(a, gij, ng, rec + (size_t)(N - 1) * ng, obs + (size_t)(N - 1) * ng, st),
             "adjoint misfit");
    const double dt = s->params.dt, c12 = dt / 12.0, c24 = dt / 24.0;
    bool used[2] = {false, false};
    // recompute segment sg into slot sg & 1 on the solver's stream, once the
    // reverse of the segment that held the slot is done
    auto recompute = [&](int sg) -> cel_status {
        const int sl = sg & 1;
        if (L.keep) {   // kept by the forward run, which precedes on the solver's stream
            CEL_CUDA(s, cudaEventRecord(ss.rec[sl], fst), "adjoint order");
            return CEL_OK;
        }
        Range r_("cel adjoint recompute");
        const int n0 = sg * C, n1 = n0 + C < N ? n0 + C : N;
        if (used[sl]) CEL_CUDA(s, cudaStreamWaitEvent(fst, ss.rev[sl], 0), "adjoint order");
        cel_status r = cel_load_checkpoint(s, ckpt(sg), L.ckpt_bytes);
        if (r != CEL_OK) return r;
        for (int k = 0; k <= n1 - n0; k++) {
            CEL_CUDA(s, keep_state(sl, k, fst), "adjoint states");
            if (k < n1 - n0 && (r = kept_step(sl, k)) != CEL_OK) return r;
        }
        CEL_CUDA(s, cudaEventRecord(ss.rec[sl], fst), "adjoint order");
        used[sl] = true;
        return CEL_OK;
    };
    if ((stt = recompute(L.nseg - 1)) != CEL_OK) return stt;
    for (int sg = L.nseg - 1; sg >= 0; sg--) {
        const int n0 = sg * C, n1 = n0 + C < N ? n0 + C : N;
        slot = sg & 1;
        CEL_CUDA(s, cudaStreamWaitEvent(st, ss.rec[slot], 0), "adjoint order");
        nvtxRangePushA("cel adjoint reverse");
        for (int n = n1 - 1; n >= n0; n--) {
            const int k = n - n0;
            CEL_CUDA(s, wait_tri(), "adjoint order");
            if (a.c.sine)
                CEL_CUDA(s, launch_ghost_table<real>(s->geo, s->phy, s->bnd, s->at<real>(s->lay.dr),
                                                     s->at<double>(s->lay.ktab), (double)(step0 + n) * dt,
                                                     (double)(step0 + n + 1) * dt, gtab, a.c.npos, st),
                         "adjoint ghosts");
            const int Kn = n >= 2 ? K : 0;
            const int sn = n % 3, sm1 = (n + 2) % 3, sm2 = (n + 1) % 3;
            if (Kn == 0) {
                double c[3], e[3];
                adj_coefs(n, dt, c, e);
                coefs(a, c[0], c[1], c[2], e[0], e[1], e[2]);
                setl(a, lset);
                setG(a, sn, sm1, sm2);
                a.w = segf(k, 0);
                a.P = segf(k, 1);
                a.Q = segf(k, 2);
                a.w_next = segf(k + 1, 0);
                a.final_stage = 1;
                CEL_CUDA(s, full_step(a, k), "adjoint step");
            } else {
                // corrector stages Kn..1, then the predictor; acc collects the
                // adjoint of the state before the step
                const int acc = (lset + 2) % 3;
                int cur = lset, nxt = (lset + 1) % 3;
                CEL_CUDA(s, cudaMemsetAsync(lam(3 * acc), 0, L.cells_bytes * 3, st), "adjoint");
                for (int stg = Kn; stg >= 1; stg--) {
                    AdjArgs<real> b = a;
                    setl(b, cur);
                    b.w_next = stg == Kn ? segf(k + 1, 0) : iterf(k, stg, 0);
                    b.final_stage = stg == Kn;
                    // the mask also clears the set the iterate's adjoint collects in
                    CEL_CUDA(s, mask(b, nxt), "adjoint mask");
                    CEL_CUDA(s, solves(b), "adjoint solves");
                    CEL_CUDA(s, tri_bed(b, k, stg), "adjoint solves");
                    // one pass: the AM4 base (Eq. 18-20), w^n + dt/24 (19 R^n - 5 R^{n-1}
                    // + R^{n-2}) - F*^n, into the history slots; the right side at the
                    // iterate before this stage, 9 dt/24 R + F*, written to slot 3; the
                    // masked adjoint (the state's own path) added to acc
                    coefs(b, 19.0 * c24, -5.0 * c24, c24, -1.0, 0.0, 0.0);
                    setG(b, sn, sm1, sm2);
                    for (int v = 0; v < 5; v++) b.H0[v] = Gb(3, v);
                    b.hc = real(9.0 * c24);
                    b.he = real(1.0);
                    b.accw = lam(3 * acc);
                    b.accP = lam(3 * acc + 1);
                    b.accQ = lam(3 * acc + 2);
                    CEL_CUDA(s, launch_adjoint_hist<real>(b, st), "adjoint history");
                    for (int v = 0; v < 5; v++) b.H0[v] = nullptr;
                    b.accw = b.accP = b.accQ = nullptr;
                    coefs(b, 9.0 * c24, 0.0, 0.0, 1.0, 0.0, 0.0);
                    setG(b, 3, -1, -1);
                    AdjArgs<real> v = b;
                    v.tsel = 1;   // the corrector stages read the ghosts at t^{n+1}
                    setl(v, nxt);
                    v.w = iterf(k, stg - 1, 0);
                    v.P = iterf(k, stg - 1, 1);
                    v.Q = iterf(k, stg - 1, 2);
                    CEL_CUDA(s, launch_adjoint_vjp<real>(v, st), "adjoint iterate");
                    std::swap(cur, nxt);
                }
                // the predictor (Eq. 15-17): masks without the sponge, solves, AB3 history
                AdjArgs<real> p = a;
                setl(p, cur);
                p.w_next = iterf(k, 0, 0);
                p.final_stage = 0;
                CEL_CUDA(s, mask(p, -1), "adjoint mask");
                CEL_CUDA(s, solves(p), "adjoint solves");
                CEL_CUDA(s, tri_bed(p, k, 0), "adjoint solves");
                coefs(p, 23.0 * c12, -16.0 * c12, 5.0 * c12, 2.0, -3.0, 1.0);
                setG(p, sn, sm1, sm2);
                p.accw = lam(3 * acc);
                p.accP = lam(3 * acc + 1);
                p.accQ = lam(3 * acc + 2);
                CEL_CUDA(s, launch_adjoint_hist<real>(p, st), "adjoint history");
                AdjArgs<real> x = a;
                setl(x, acc);
                // R^n and F*^n at the state before the step
                x.w = segf(k, 0);
                x.P = segf(k, 1);
                x.Q = segf(k, 2);
                setG(x, sn, -1, -1);
                CEL_CUDA(s, launch_adjoint_vjp<real>(x, st), "adjoint state");
                lset = acc;
            }
            if (a.lg) {   // the step's ghost values (t^n, t^{n+1}) follow the adjacent depth
                CEL_CUDA(s, wait_tri(), "adjoint order");
                CEL_CUDA(s, launch_adjoint_ghost_bed<real>(a, s->bnd, s->at<double>(s->lay.ktab),
                                                           s->at<real>(s->lay.dr), (double)(step0 + n) * dt,
                                                           (double)(step0 + n + 1) * dt, st),
                         "adjoint ghosts");
            }
            setl(a, lset);
            if (n >= 1)
                CEL_CUDA(s, launch_adjoint_misfit<real>(a, gij, ng, rec + (size_t)(n - 1) * ng,
                                                        obs + (size_t)(n - 1) * ng, st),
                         "adjoint misfit");
            CEL_CUDA(s, cudaMemsetAsync(Gb(sn, 0), 0, L.cells_bytes * 5, st), "adjoint");
        }
        nvtxRangePop();
        CEL_CUDA(s, wait_tri(), "adjoint order");   // the captured line solutions of this slot
        CEL_CUDA(s, cudaEventRecord(ss.rev[slot], st), "adjoint order");
        if (sg > 0 && (stt = recompute(sg - 1)) != CEL_OK) return stt;   // overlaps this segment's reverse
    }
    CEL_CUDA(s, cudaMemcpyAsync(grad, lam(3 * lset), sizeof(real) * cells, cudaMemcpyDeviceToDevice, st),
             "adjoint gradient");
    CEL_CUDA(s, wait_tri(), "adjoint order");
    if (bed)   // segment 0's first state is the initial one
        CEL_CUDA(s, launch_adjoint_bed_final<real>(a, segf(0, 0), lam(3 * lset), grad_z, st), "adjoint bed");
    if (eta_out)
        CEL_CUDA(s, cudaMemcpyAsync(eta_out, rec, sizeof(real) * (size_t)N * ng, cudaMemcpyDeviceToDevice, st),
                 "adjoint records");
    CEL_CUDA(s, cudaEventRecord(ss.fin, st), "adjoint order");
    CEL_CUDA(s, cudaStreamWaitEvent(fst, ss.fin, 0), "adjoint order");
    stt = cel_load_checkpoint(s, ckpt(L.nseg), L.ckpt_bytes);   // leave the solver after step N
    if (stt == CEL_OK) CEL_CUDA(s, cudaStreamSynchronize(fst), "adjoint");
    return stt;
}

cel_status adjoint_check(const cel_solver *, int N, int C, int ng, std::string &why)
{
    if (N < 1 || C < 0 || ng < 1) {
        why = "nsteps and the gauge count must be positive, ckpt_every positive or 0";
        return CEL_ERR_INVALID_ARG;
    }
    return CEL_OK;
}

}  // namespace

extern "C" {

cel_status cel_adjoint_face_selfcheck(int32_t real_bytes, const void *in_dev, int32_t n, void *out_dev,
                                      void *cuda_stream)
{
    if ((real_bytes != 4 && real_bytes != 8) || n < 0 || (n > 0 && (!in_dev || !out_dev))) return CEL_ERR_INVALID_ARG;
    if (n == 0) return CEL_OK;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = real_bytes == 4 ? launch_face_vjp_check<float>((const float *)in_dev, n, (float *)out_dev, st)
                                    : launch_face_vjp_check<double>((const double *)in_dev, n, (double *)out_dev, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? CEL_OK : CEL_ERR_CUDA;
}

cel_status cel_adjoint_bytes(const cel_solver *s, int32_t nsteps, int32_t ckpt_every, int32_t ngauges,
                             int32_t with_bed, size_t *bytes)
{
    if (!s || !bytes) return CEL_ERR_INVALID_ARG;
    std::string why;
    cel_status st = adjoint_check(s, nsteps, ckpt_every, ngauges, why);
    if (st != CEL_OK) return st;
    *bytes = adj_layout(s, nsteps, ckpt_every, ngauges, with_bed != 0).total;
    return CEL_OK;
}

cel_status cel_adjoint_gauge_misfit(cel_solver *s, int32_t nsteps, int32_t ckpt_every, const int32_t *gij_host,
                                    int32_t ngauges, const void *obs_dev, void *scratch_dev, size_t scratch_bytes,
                                    void *eta_dev, void *grad_w_dev, void *grad_z_dev, double *loss)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    std::string why;
    cel_status st = adjoint_check(s, nsteps, ckpt_every, ngauges, why);
    if (st != CEL_OK) return fail(s, st, why);
    if (s->nh != 0) return fail(s, CEL_ERR_INVALID_ARG, "set the initial state first (the history must be fresh)");
    if (!gij_host || !obs_dev || !scratch_dev || !grad_w_dev || ((uintptr_t)scratch_dev & 255) != 0)
        return fail(s, CEL_ERR_INVALID_ARG, "NULL argument or unaligned scratch");
    for (int k = 0; k < ngauges; k++)
        if (gij_host[2 * k] < 0 || gij_host[2 * k] >= s->grid.nx || gij_host[2 * k + 1] < 0 ||
            gij_host[2 * k + 1] >= s->grid.ny)
            return fail(s, CEL_ERR_INVALID_ARG, "gauge outside the grid");
    AdjLayout L = adj_layout(s, nsteps, ckpt_every, ngauges, grad_z_dev != nullptr);
    if (scratch_bytes < L.total) return fail(s, CEL_ERR_WORKSPACE_TOO_SMALL, "adjoint scratch too small");
    return s->es == 4 ? adjoint_t<float>(s, nsteps, ckpt_every, gij_host, ngauges, (const float *)obs_dev,
                                         (unsigned char *)scratch_dev, L, (float *)eta_dev, (float *)grad_w_dev,
                                         (float *)grad_z_dev, loss)
                      : adjoint_t<double>(s, nsteps, ckpt_every, gij_host, ngauges, (const double *)obs_dev,
                                          (unsigned char *)scratch_dev, L, (double *)eta_dev, (double *)grad_w_dev,
                                          (double *)grad_z_dev, loss);
}

cel_status cel_adjoint_input_gradient(cel_solver *s, const void *w_in_dev, void *grad_w_dev)
{
    if (!s) return CEL_ERR_INVALID_ARG;
    if (!w_in_dev || !grad_w_dev) return fail(s, CEL_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = s->es == 4 ? launch_clamp_adjoint<float>(s->geo, s->at<float>(s->lay.Bc), (const float *)w_in_dev,
                                                             (float *)grad_w_dev, s->stream)
                               : launch_clamp_adjoint<double>(s->geo, s->at<double>(s->lay.Bc),
                                                              (const double *)w_in_dev, (double *)grad_w_dev, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "adjoint input gradient");
    return CEL_OK;
}

}  // extern "C"
