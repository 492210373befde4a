// CUDA kernels of the Celeris extended-Boussinesq step for GB300 (sm_103a).
//
// Paper: Tavakkol & Lynett, "Celeris", arXiv 1611.05984.
//   Sec. 2.1  Eq. 1-3 (governing equations); Sec. 2.2 Eq. 4-14 (Wei-Kirby
//   form, KP07 steps 1-4); Sec. 2.3 Eq. 15-23 (AB3 / AM4, tridiagonal
//   systems); Sec. 2.4 Eq. 24-30 (boundaries); Sec. 2.6 Eq. 31-32 (friction);
//   Sec. 2.7 Eq. 33-36 (solitary wave).
//
// Per step and per stage (predictor, then K corrector iterations) three
// kernels run:
//   k_stencil  one 32x32 tile per thread block: stages w, P, Q (+2 ghost
//              layers produced in shared memory from the boundary rules) and
//              the bed corners, computes every face flux once, then per cell
//              E, F, G, F*, G*, friction and the time update; writes w^{n+1},
//              the increments of U* (row-major) and V* (column-major,
//              transposed through shared memory) and the dry-cell bits.
//   k_lines    one thread block per line, x-rows then y-columns: a
//              partitioned tridiagonal solve of Eq. 21/22 for the increment
//              P^{n+1} - P^n (each thread eliminates its own segment, the
//              2-per-segment interface system is solved by parallel cyclic
//              reduction), then P^n + increment, sponge and dry-cell epilogue.
#include "celeris_internal.cuh"
#include "celeris_physics.cuh"

#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include <math.h>

namespace cel {

namespace {

constexpr double kPi = 3.14159265358979323846;

__host__ __device__ inline int round_up(int a, int b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------ static fields

// a0 (Reading A-W1): corner bed = mean of the 4 cells around it, with the
// cell-centre bed mirrored evenly into the two ghost layers.
template <typename real>
__global__ void k_corners(Geo g, const real *__restrict__ z, real *__restrict__ Bc)
{
    int ci = blockIdx.x * blockDim.x + threadIdx.x - 1;
    int cj = blockIdx.y * blockDim.y + threadIdx.y - 1;
    if (ci > g.nx + 1 || cj > g.ny + 1) return;
    int i0 = mirror_index(ci - 1, g.nx), i1 = mirror_index(ci, g.nx);
    int j0 = mirror_index(cj - 1, g.ny), j1 = mirror_index(cj, g.ny);
    real z00 = z[(size_t)j0 * g.nx + i0], z10 = z[(size_t)j0 * g.nx + i1];
    real z01 = z[(size_t)j1 * g.nx + i0], z11 = z[(size_t)j1 * g.nx + i1];
    Bc[(size_t)(cj + 1) * g.pc + (ci + 1)] = real(0.25) * (((z00 + z10) + z01) + z11);
}

template <typename real>
__global__ void k_static_cells(Geo g, Phys p, const real *__restrict__ Bc, real *__restrict__ d_r,
                               real *__restrict__ d_c)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    real d = fmax(real(p.ws) - bbar_at(Bc, g, i, j), real(0));
    d_r[(size_t)j * g.px + i] = d;
    d_c[(size_t)i * g.py + j] = d;
}

// Hot start (or rest): w >= Bbar, P = Q = 0 where the depth is zero.
template <typename real>
__global__ void k_set_state(Geo g, Phys p, const real *__restrict__ Bc, const real *w_in,
                            const real *P_in, const real *Q_in, real *w, real *P, real *Qc,
                            int rest)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    size_t k = (size_t)j * g.nx + i;
    real Bb = bbar_at(Bc, g, i, j);
    real wv = rest ? real(p.ws) : w_in[k];
    real Pv = rest ? real(0) : P_in[k];
    real Qv = rest ? real(0) : Q_in[k];
    wv = fmax(wv, Bb);
    if (wv - Bb <= real(0)) {
        Pv = real(0);
        Qv = real(0);
    }
    w[(size_t)j * g.px + i] = wv;
    P[(size_t)j * g.px + i] = Pv;
    Qc[(size_t)i * g.py + j] = Qv;
}

template <typename real>
__global__ void k_clamp_state(Geo g, Phys p, const real *__restrict__ Bc, real *w, real *P, real *Qc)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    size_t kr = (size_t)j * g.px + i, kc = (size_t)i * g.py + j;
    real Bb = bbar_at(Bc, g, i, j);
    real wv = fmax(w[kr], Bb);
    w[kr] = wv;
    if (wv - Bb <= real(0)) {
        P[kr] = real(0);
        Qc[kc] = real(0);
    }
}

// Reading A-J3: w0 = max(w_in, Bbar) has derivative 1 in w_in where w_in
// lies above the cell bed and 0 where the clamp holds w0 at the bed (the
// one-sided derivative at a tie); grad ([ny][nx]) is masked in place.
template <typename real>
__global__ void k_clamp_adjoint(Geo g, const real *__restrict__ Bc, const real *__restrict__ w_in, real *grad)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    size_t k = (size_t)j * g.nx + i;
    if (!(w_in[k] > bbar_at(Bc, g, i, j))) grad[k] = real(0);
}

template <typename real>
__global__ void k_get_state(Geo g, const real *w, const real *P, const real *Qc, real *w_out,
                            real *P_out, real *Q_out)
{
    dependent_launch_wait_then_release();
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    size_t k = (size_t)j * g.nx + i;
    if (w_out) w_out[k] = w[(size_t)j * g.px + i];
    if (P_out) P_out[k] = P[(size_t)j * g.px + i];
    if (Q_out) Q_out[k] = Qc[(size_t)i * g.py + j];
}

template <typename real>
__global__ void k_get_field(Geo g, Phys p, int which, const real *Bc, const real *d_r,
                            const real *U, const real *Vc, real *out)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    real v;
    if (which == 0) v = bbar_at(Bc, g, i, j);
    else if (which == 1) v = d_r[(size_t)j * g.px + i];
    else if (which == 2) v = U[(size_t)j * g.px + i];
    else v = Vc[(size_t)i * g.py + j];
    out[(size_t)j * g.nx + i] = v;
}

// Run-up tracking (Sec. 4.1, 4.3): maxw ([ny][nx]) keeps the highest w seen
// while the cell's depth w - Bbar exceeds delta, -inf where it never did;
// start sets it from the present state.
template <typename real>
__global__ void k_runup(Geo g, const real *Bc, const real *w, real *maxw, real delta, int start)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    const real wv = w[(size_t)j * g.px + i];
    const bool wet = wv - bbar_at(Bc, g, i, j) > delta;
    real *m = maxw + (size_t)j * g.nx + i;
    if (start) *m = wet ? wv : real(-INFINITY);
    else if (wet && wv > *m) *m = wv;
}

// Eq. 33-36 (Reading A-S1), evaluated in double, added where d > 0.
template <typename real>
__global__ void k_add_solitary(Geo g, Phys p, const real *Bc, real *w, real *P, real *Qc,
                               double H, double ct, double st, double x0, double y0, double ks,
                               double cs)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.nx || j >= g.ny) return;
    size_t kr = (size_t)j * g.px + i, kc = (size_t)i * g.py + j;
    real Bb = bbar_at(Bc, g, i, j);
    real d = fmax(real(p.ws) - Bb, real(0));
    real wv = w[kr], Pv = P[kr], Qv = Qc[kc];
    if (d > real(0)) {
        double xi = ((i + 0.5) * g.dx - x0) * ct + ((j + 0.5) * g.dy - y0) * st;
        double sh = 1.0 / cosh(ks * xi);
        double es = H * sh * sh;
        wv = (real)fmax((double)wv + es, (double)Bb);
        Pv = (real)((double)Pv + cs * es * ct);
        Qv = (real)((double)Qv + cs * es * st);
    }
    if (wv - Bb <= real(0)) {
        Pv = real(0);
        Qv = real(0);
    }
    w[kr] = wv;
    P[kr] = Pv;
    Qc[kc] = Qv;
}

template <typename real>
__global__ void k_gauges(Geo g, Phys p, const real *w, const int32_t *ij, int n, real *slot)
{
    dependent_launch_wait_then_release();
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int i = ij[2 * k], j = ij[2 * k + 1];
    slot[k] = w[(size_t)j * g.px + i] - real(p.ws);
}

// Diagnostics over the interior cells: sum of the depths w - Bbar (the
// mass over dx dy), the largest speed |(P, Q)| k(h) with the Eq. 14
// velocity factor, the count of wet cells (w > Bbar).  Block sums, one
// atomic per block and quantity: out[0] double sum, out[1] the bits of the
// largest speed (non-negative doubles order as their bits), out[2] count.
template <typename real>
__global__ void k_stats(Geo g, Phys p, const real *Bc, const real *w, const real *P, const real *Qc, real eps,
                        unsigned long long *out)
{
    double mass = 0.0, vmax = 0.0;
    unsigned long long wet = 0;
    const size_t n = (size_t)g.nx * g.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(k % g.nx), j = (int)(k / g.nx);
        const real h = w[(size_t)j * g.px + i] - bbar_at(Bc, g, i, j);
        const real Pv = P[(size_t)j * g.px + i], Qv = Qc[(size_t)i * g.py + j];
        mass += (double)h;
        const real sp = desing(fmax(h, real(0)), eps) * sqrt(Pv * Pv + Qv * Qv);
        vmax = fmax(vmax, (double)sp);
        wet += h > real(0) ? 1ull : 0ull;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mass += __shfl_down_sync(0xffffffffu, mass, o);
        vmax = fmax(vmax, __shfl_down_sync(0xffffffffu, vmax, o));
        wet += __shfl_down_sync(0xffffffffu, wet, o);
    }
    __shared__ double sm[32], sv[32];
    __shared__ unsigned long long sw[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
        sm[wid] = mass;
        sv[wid] = vmax;
        sw[wid] = wet;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < nw; k++) {
            mass += sm[k];
            vmax = fmax(vmax, sv[k]);
            wet += sw[k];
        }
        atomicAdd(reinterpret_cast<double *>(out), mass);
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(vmax));
        atomicAdd(out + 2, wet);
    }
}

template <typename real>
__global__ void k_check_finite(Geo g, const real *w, const real *P, const real *Qc,
                               unsigned long long *first_bad)
{
    size_t n = (size_t)g.nx * g.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(k % g.nx), j = (int)(k / g.nx);
        real a = w[(size_t)j * g.px + i], b = P[(size_t)j * g.px + i], c = Qc[(size_t)i * g.py + j];
        if (!isfinite(a) || !isfinite(b) || !isfinite(c)) atomicMin(first_bad, (unsigned long long)k);
    }
}

// Last entry of a sorted prefix array not above b: the ensemble member (or line family) that block b belongs to.
__device__ __forceinline__ int find_owner(const int *__restrict__ start, int n, int b)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (start[mid] <= b) lo = mid;
        else hi = mid;
    }
    return lo;
}


// Eckart wave number (Eq. 29) per sine side, position and component, from
// the static depths; 0 where the adjacent cell is dry.  Rebuilt when a
// boundary or the bed changes.
template <typename real>
__global__ void k_eckart_table(Geo g, Phys p, Bnd b, const real *__restrict__ d_r, double *__restrict__ ktab,
                               int npos)
{
    int pos = blockIdx.x * blockDim.x + threadIdx.x, side = blockIdx.y;
    if (pos >= npos || b.s[side].type != kSine) return;
    double x, y, dadj;
    bool used = ghost_site(g, d_r, side, 0, pos, x, y, dadj);
    for (int m = 0; m < 8; m++) {
        double k = 0.0;
        if (used && m < b.s[side].ncomp && dadj > 0.0) {
            double om = b.s[side].omega[m];
            double k0 = om * om / p.g;
            k = k0 * sqrt(1.0 / tanh(k0 * dadj));
        }
        ktab[((size_t)side * npos + pos) * 8 + m] = k;
    }
}

// Eq. 30's factor per sponge side and position from the side ([side][pos],
// 1 beyond the sponge).  Rebuilt when a boundary changes.
template <typename real>
__global__ void k_sponge_table(const Coef<real> c, real *__restrict__ gam)
{
    const int pos = blockIdx.x * blockDim.x + threadIdx.x, side = blockIdx.y;
    if (pos >= c.npos) return;
    const int w = c.spw[side];
    gam[(size_t)side * c.npos + pos] = pos < w ? sponge_eq30<real>(w, pos) : real(1);
}

// Sine-maker ghosts (Eq. 25-28) for one step: both ghost layers of every
// sine side at t^n and t^{n+1}, summed over components.
template <typename real>
__device__ __forceinline__ void ghost_entry(const Geo &g, const Phys &p, const Bnd &b, const real *__restrict__ d_r,
                                            const double *__restrict__ ktab, double t0, double t1,
                                            real *__restrict__ tab, int npos, int pos, int yb)
{
    int time = yb & 1, layer = (yb >> 1) & 1, side = yb >> 2;
    if (pos >= npos || b.s[side].type != kSine) return;
    double x, y, dadj;
    if (!ghost_site(g, d_r, side, layer, pos, x, y, dadj)) return;
    const Side &S = b.s[side];
    const double t = time ? t1 : t0;
    if constexpr (sizeof(real) == 4) {
        // single precision: the phase in double (omega t grows without
        // bound), reduced there to [-pi, pi]; the sine and the sums in
        // single precision, which the table holds (double-precision
        // arithmetic runs at a small fraction of the single-precision rate)
        constexpr double kTwoPi = 6.283185307179586, kInvTwoPi = 0.15915494309189535;
        float eta = 0.f, Pg = 0.f, Qg = 0.f;
        for (int m = 0; m < S.ncomp; m++) {
            const double k = ktab[((size_t)side * npos + pos) * 8 + m];
            if (!(k > 0.0)) continue;
            const double ph = S.omega[m] * t - k * S.cdir[m] * x - k * S.sdir[m] * y + S.phase[m];
            const double r = ph - kTwoPi * rint(ph * kInvTwoPi);
            const float em = (float)S.amp[m] * sinf((float)r), c = (float)S.omega[m] / (float)k;
            eta += em;
            Pg += c * (float)S.cdir[m] * em;
            Qg += c * (float)S.sdir[m] * em;
        }
        tab[ghost_index(time, side, layer, 0, pos, npos)] = (float)p.ws + eta;
        tab[ghost_index(time, side, layer, 1, pos, npos)] = Pg;
        tab[ghost_index(time, side, layer, 2, pos, npos)] = Qg;
    } else {
        double eta = 0.0, Pg = 0.0, Qg = 0.0;
        for (int m = 0; m < S.ncomp; m++) {
            const double k = ktab[((size_t)side * npos + pos) * 8 + m];
            if (!(k > 0.0)) continue;
            const double om = S.omega[m], c = om / k;
            const double em = S.amp[m] * sin(om * t - k * S.cdir[m] * x - k * S.sdir[m] * y + S.phase[m]);
            eta += em;
            Pg += c * S.cdir[m] * em;
            Qg += c * S.sdir[m] * em;
        }
        tab[ghost_index(time, side, layer, 0, pos, npos)] = real(p.ws + eta);
        tab[ghost_index(time, side, layer, 1, pos, npos)] = real(Pg);
        tab[ghost_index(time, side, layer, 2, pos, npos)] = real(Qg);
    }
}

template <typename real>
__global__ void k_ghost_table(Geo g, Phys p, Bnd b, const real *__restrict__ d_r,
                              const double *__restrict__ ktab, double t0, double t1, real *__restrict__ tab,
                              int npos)
{
    dependent_launch_wait_then_release();
    ghost_entry(g, p, b, d_r, ktab, t0, t1, tab, npos, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// Ensemble: the ghost tables of every member with a sine maker; member e
// owns blocks [start[e], start[e+1]), 16 per 128 positions, and is at step
// step0 + k.
template <typename real>
__device__ __forceinline__ void ghost_batch_block(const GhostArgs<real> *__restrict__ args,
                                                  const int *__restrict__ start, int n, int blk, int t, int64_t k)
{
    const int e = find_owner(start, n, blk);
    const GhostArgs<real> &A = args[e];
    const int b = blk - start[e];
    const int nbx = (A.npos + 127) / 128;
    const int64_t step = A.step0 + k;
    ghost_entry(A.g, A.p, A.b, A.d_r, A.ktab, (double)step * A.dt, (double)(step + 1) * A.dt, A.tab, A.npos,
                (b % nbx) * 128 + t, b / nbx);
}

template <typename real>
__global__ void k_ghost_batch(const GhostArgs<real> *__restrict__ args, const int *__restrict__ start, int n,
                              int64_t k, const int64_t *__restrict__ kdev)
{
    ghost_batch_block(args, start, n, blockIdx.x, threadIdx.x, (kdev ? *kdev : 0) + k);
}

// ------------------------------------------------------------ the stencil

template <typename real>
struct StencilSmem {
    real w[kTileIn * kStride];
    real P[kTileIn * kStride];
    real Q[kTileIn * kStride];
    real Bc[kCorner * kCornerStride];
    real d[kDcell * kDStride];
    real Fx[3][kTile][kTile + 1];    // x-faces: [component][row][face]
    real Fy[3][kTile + 1][kTile];    // y-faces: [component][face][column]
    real Vout[kTile][kTile + 1];     // V*^{n+1} staged for the transposed store
    uint32_t colbits[kTile];
};

// Update of one unknown (w, U* or V*) with right side R and mixed term Phi
// (0 for w), Sec. 2.3, returned as the increment X^{n+1} - X^n.  Carries
// (per cell, row-major):
//   a = -16 (dt/12) R^{n-1} - 3 Phi^{n-1}       (in place)
//   b = 5 (dt/12) R^{n-2} + Phi^{n-2}           (two slots, by step parity)
// so that Eq. 15-17 read X^{n+1} - X^n = 23 (dt/12) R^n + 2 Phi^n + a + b.
// The first two steps are forward Euler; the second adds Phi^1 - Phi^0,
// for which `a` holds Phi^0 after the first.  With K > 0 also
//   q = (dt/24)(-5 R^{n-1} + R^{n-2}),  e = (dt/24) R^{n-1},
//   Y = X0 + 19 (dt/24) R^n - Phi^n + q         (corrector base),
// so that Eq. 18-20 read X^{n+1} - X0 = Y - X0 + 9 (dt/24) R^{n+1} + Phi^{n+1}
// (the AM4 stage returns Y + 9 (dt/24) R + Phi).  For w, X0 = w^n, so the
// corrector returns w^{n+1} itself.  U* and V* are carried as increments
// only (X0 = 0): the line solves find P^{n+1} - P^n from the increment of U*,
// which equals recomputing U*^n from P^n by Eq. 23 but keeps the rounding
// relative to the increment instead of to P.
// History of one unknown (w, U* or V*) for the update of Sec. 2.3, with R
// its right side and Phi its mixed term (0 for w); the AB3 and AM4 stages
// return the increment X^{n+1} - X^n (for the AM4 stage of w: w^{n+1}).
//
// K = 0 (predictor only): two combined carries per unknown,
//   a = -16 (dt/12) R^{n-1} - 3 Phi^{n-1}        (in place)
//   b = 5 (dt/12) R^{n-2} + Phi^{n-2}            (two slots, by step parity)
// so Eq. 15-17 read X^{n+1} - X^n = 23 (dt/12) R^n + 2 Phi^n + a + b, with
// 2 reads and 2 writes per unknown.  The first two steps are forward Euler;
// the second adds Phi^1 - Phi^0, for which `a` holds Phi^0 after the first.
//
// K >= 1: rings of R and Phi (three slots each) as Eq. 15-20 write them,
// and the corrector base
//   Y = X0 + (dt/24)(19 R^n - 5 R^{n-1} + R^{n-2}) - Phi^n
// (X0 = w^n for w, 0 for U*, V*), so that Eq. 18-20 read
// X^{n+1} - X0 = Y - X0 + 9 (dt/24) R^{n+1} + Phi^{n+1}.
//
// U* and V* are carried as increments only: the line solves find
// P^{n+1} - P^n from the increment of U*, which equals recomputing U*^n from
// P^n by Eq. 23 but keeps the rounding relative to the increment.
template <typename real>
struct Carry {
    real a, b, r1, r2, p1, p2, Y;
};

// The history a stage reads, loaded at the top of a cell's iteration so the
// loads are in flight while the cell's right side is computed.
// Stage specialisations of the stencil (kSpec): 0, any stage, its kind and
// history layout read at run time; 1, the AB3 predictor with the ring
// history (K >= 1); 2, the AM4 corrector.  The two hot stages then carry no
// branches on the stage kind.
template <int kSpec, typename real>
__device__ __forceinline__ int stage_kind(const StencilArgs<real> &A)
{
    return kSpec == 1 ? kAB3 : (kSpec == 2 ? kAM4 : A.kind);
}

template <int kSpec, typename real>
__device__ __forceinline__ bool stage_ring(const StencilArgs<real> &A)
{
    return kSpec != 0 ? true : A.ring != 0;
}

template <typename real, int kSpec>
__device__ __forceinline__ Carry<real> load_carry(const StencilArgs<real> &A, int v, size_t k)
{
    const int kind = stage_kind<kSpec>(A);
    const bool ring = stage_ring<kSpec>(A);
    Carry<real> c;
    c.a = c.b = c.r1 = c.r2 = c.p1 = c.p2 = c.Y = real(0);
    if (kind == kAM4) {
        c.Y = A.Y[v][k];
    } else if (ring) {
        if (kind == kAB3) {
            c.r1 = A.R1[v][k];
            c.r2 = A.R2[v][k];
        }
        if (v > 0 && kind != kEuler0) {
            c.p1 = A.F1[v][k];
            if (kind == kAB3) c.p2 = A.F2[v][k];
        }
    } else if (kind == kEuler1) {
        c.a = A.a[v][k];
    } else if (kind == kAB3) {
        c.a = A.a[v][k];
        c.b = A.b[v][k];
    }
    return c;
}

template <typename real, int kSpec>
__device__ __forceinline__ real advance(const StencilArgs<real> &A, int v, real X0, real R, real Phi, size_t k,
                                        const Carry<real> &c)
{
    const int kind = stage_kind<kSpec>(A);
    const bool ring = stage_ring<kSpec>(A);
    const real dt = A.c.dt, c12 = dt / real(12), c24 = dt / real(24);
    if (kind == kAM4) return c.Y + real(9) * c24 * R + Phi;
    if (ring) {
        real D;
        if (kind == kEuler0) {
            D = dt * R;
        } else if (kind == kEuler1) {
            D = dt * R + (Phi - c.p1);
        } else {
            D = c12 * (real(23) * R - real(16) * c.r1 + real(5) * c.r2) + real(2) * Phi - real(3) * c.p1 + c.p2;
            A.Y[v][k] = X0 + c24 * (real(19) * R - real(5) * c.r1 + c.r2) - Phi;
        }
        A.R0[v][k] = R;
        if (v > 0) A.F0[v][k] = Phi;
        return D;
    }
    real D;
    if (kind == kEuler0) {
        D = dt * R;
        A.a[v][k] = Phi;
    } else if (kind == kEuler1) {
        D = dt * R + (Phi - c.a);
        A.a[v][k] = real(-16) * c12 * R - real(3) * Phi;
    } else {
        D = real(23) * c12 * R + real(2) * Phi + (c.a + c.b);
        A.a[v][k] = real(-16) * c12 * R - real(3) * Phi;
    }
    A.b[v][k] = real(5) * c12 * R + Phi;
    return D;
}

template <typename real> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// One tile to stage: `rows` rows of `cols` elements starting at column gx0
// (even) of row gy0 of a field with row pitch `pitch`, elements outside
// [0, lim_x) x [0, lim_y) read as 0; `transpose` stores element (r, c) at
// dst[c * dstride + r].
template <typename real>
struct StageSpec {
    const real *src;
    size_t pitch;
    int gx0, gy0, rows, cols, lim_x, lim_y;
    real *dst;
    int dstride;
    bool transpose;
};

// Stage several tiles with every global load of a thread issued before any
// of its shared-memory stores, so the loads' latencies overlap (a load-store
// loop would pay one full latency per element pair).  Pairs are loaded as
// one aligned vector where both elements are inside the field.
template <typename real, int NT, int MAXP>
__device__ __forceinline__ void stage_tiles(const StageSpec<real> *sp, int tid)
{
    using real2 = typename Vec2<real>::type;
    real v0[NT][MAXP], v1[NT][MAXP];
#pragma unroll
    for (int t = 0; t < NT; t++) {
        const StageSpec<real> &S = sp[t];
        const int pairs = (S.cols + 1) >> 1;
#pragma unroll
        for (int u = 0; u < MAXP; u++) {
            const int k = tid + u * kStencilThreads;
            v0[t][u] = v1[t][u] = real(0);
            if (k < S.rows * pairs) {
                const int r = k / pairs, c = 2 * (k - r * pairs);
                const int gy = S.gy0 + r, gx = S.gx0 + c;
                if (gy >= 0 && gy < S.lim_y) {
                    const real *row = S.src + (size_t)gy * S.pitch;
                    if (gx >= 0 && gx + 1 < S.lim_x) {
                        real2 v = *reinterpret_cast<const real2 *>(row + gx);
                        v0[t][u] = v.x;
                        v1[t][u] = v.y;
                    } else {
                        if (gx >= 0 && gx < S.lim_x) v0[t][u] = row[gx];
                        if (gx + 1 >= 0 && gx + 1 < S.lim_x) v1[t][u] = row[gx + 1];
                    }
                }
            }
        }
    }
#pragma unroll
    for (int t = 0; t < NT; t++) {
        const StageSpec<real> &S = sp[t];
        const int pairs = (S.cols + 1) >> 1;
#pragma unroll
        for (int u = 0; u < MAXP; u++) {
            const int k = tid + u * kStencilThreads;
            if (k < S.rows * pairs) {
                const int r = k / pairs, c = 2 * (k - r * pairs);
                if (S.transpose) {
                    S.dst[c * S.dstride + r] = v0[t][u];
                    if (c + 1 < S.cols) S.dst[(c + 1) * S.dstride + r] = v1[t][u];
                } else {
                    S.dst[r * S.dstride + c] = v0[t][u];
                    if (c + 1 < S.cols) S.dst[r * S.dstride + c + 1] = v1[t][u];
                }
            }
        }
    }
}

// Tile origin of a single-grid launch: the block index, which the compiler
// re-reads where it needs it instead of keeping it in a register.
struct GridOrigin {
    __device__ __forceinline__ int x0() const { return blockIdx.x * kTile; }
    __device__ __forceinline__ int y0() const { return blockIdx.y * kTile; }
};

// Tile origin of an ensemble launch: two ints in shared memory, loaded at
// each use for the same reason.
struct SharedOrigin {
    const int *o;
    __device__ __forceinline__ int ld(int k) const
    {
        int v;
        asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"((unsigned)__cvta_generic_to_shared(o + k)));
        return v;
    }
    __device__ __forceinline__ int x0() const { return ld(0); }
    __device__ __forceinline__ int y0() const { return ld(1); }
};

// One 32 x 32 tile of one grid, at the origin O gives: the whole stencil stage.
template <typename real, int kSpec, typename Origin>
__device__ __forceinline__ void stencil_tile(const StencilArgs<real> &A, const Origin &O, unsigned char *smem_raw)
{
    StencilSmem<real> &sm = *reinterpret_cast<StencilSmem<real> *>(smem_raw);
    const Geo &G = A.geo;
    const int nx = G.nx, ny = G.ny;
    const int tid = threadIdx.x;
    const Coef<real> &C = A.c;
    const real ws = C.ws, g = C.g, eps = C.eps;
    const real th = C.theta;

    // ---- 1. stage the state tile (+2 halo) and the bed corners; Q is
    //         column-major, so its tile is staged along y and transposed.
    //         Corners: array index (corner + 1) in [0, nx + 2] x [0, ny + 2].
    {
        const StageSpec<real> spec[4] = {
            {A.w_in, (size_t)G.px, O.x0() - kHalo, O.y0() - kHalo, kTileIn, kTileIn, nx, ny, sm.w, kStride, false},
            {A.P_in, (size_t)G.px, O.x0() - kHalo, O.y0() - kHalo, kTileIn, kTileIn, nx, ny, sm.P, kStride, false},
            {A.Qc_in, (size_t)G.py, O.y0() - kHalo, O.x0() - kHalo, kTileIn, kTileIn, ny, nx, sm.Q, kStride, true},
            {A.Bc, (size_t)G.pc, O.x0(), O.y0(), kCorner, kCorner, nx + 3, ny + 3, sm.Bc, kCornerStride, false}};
        // 36 x 18 pairs per state tile: at most 3 per thread
        stage_tiles<real, 4, (kTileIn * (kTileIn / 2) + kStencilThreads - 1) / kStencilThreads>(spec, tid);
    }
    if (tid < kTile) sm.colbits[tid] = 0u;
    __syncthreads();

    auto cell_d = [&](int cx, int cy) -> real {   // cell whose SW corner is tile corner (cx,cy)
        const real *c = sm.Bc;
        real Bb = cell_bbar(c[cy * kCornerStride + cx], c[cy * kCornerStride + cx + 1],
                            c[(cy + 1) * kCornerStride + cx], c[(cy + 1) * kCornerStride + cx + 1]);
        return fmax(ws - Bb, real(0));
    };

    // ---- 2. ghost layers (Sec. 2.4): x-sides over interior rows, then
    //         y-sides over every column, so corners come by composition.
    const bool westT = O.x0() == 0, eastT = O.x0() + kTile + kHalo > nx;
    const bool southT = O.y0() == 0, northT = O.y0() + kTile + kHalo > ny;
    if (westT || eastT) {
        for (int k = tid; k < 4 * (kTileIn - 2); k += kStencilThreads) {
            int ty = 1 + k % (kTileIn - 2), which = k / (kTileIn - 2);   // ty in [1, 35)
            int gy = O.y0() - kHalo + ty;
            if (gy < 0 || gy >= ny) continue;
            int side = which < 2 ? 0 : 1, kk = which & 1;
            if ((side == 0 && !westT) || (side == 1 && !eastT)) continue;
            int gx = side == 0 ? -1 - kk : nx + kk;
            int tx = gx - O.x0() + kHalo;
            if (tx < 0 || tx >= kTileIn) continue;
            int sx = side == 0 ? kk : nx - 1 - kk;
            int stx = sx - O.x0() + kHalo;
            int gi = ty * kStride + tx, si = ty * kStride + stx;
            if ((C.sine >> side) & 1) {
                const real *tb = A.ghost + ghost_index(A.tsel, side, kk, 0, gy + 2, C.npos);
                sm.w[gi] = tb[0];
                sm.P[gi] = tb[C.npos];
                sm.Q[gi] = tb[2 * C.npos];
            } else {
                sm.w[gi] = sm.w[si];
                sm.P[gi] = -sm.P[si];
                sm.Q[gi] = sm.Q[si];
            }
        }
    }
    __syncthreads();
    if (southT || northT) {
        for (int k = tid; k < 4 * (kTileIn - 2); k += kStencilThreads) {
            int tx = 1 + k % (kTileIn - 2), which = k / (kTileIn - 2);
            int gx = O.x0() - kHalo + tx;
            int side = which < 2 ? 2 : 3, kk = which & 1;
            if ((side == 2 && !southT) || (side == 3 && !northT)) continue;
            int gy = side == 2 ? -1 - kk : ny + kk;
            int ty = gy - O.y0() + kHalo;
            if (ty < 0 || ty >= kTileIn) continue;
            int sy = side == 2 ? kk : ny - 1 - kk;
            int sty = sy - O.y0() + kHalo;
            int gi = ty * kStride + tx, si = sty * kStride + tx;
            if ((C.sine >> side) & 1) {
                const real *tb = A.ghost + ghost_index(A.tsel, side, kk, 0, gx + 2, C.npos);
                sm.w[gi] = tb[0];
                sm.P[gi] = tb[C.npos];
                sm.Q[gi] = tb[2 * C.npos];
            } else {
                sm.w[gi] = sm.w[si];
                sm.P[gi] = sm.P[si];
                sm.Q[gi] = -sm.Q[si];
            }
        }
    }
    // ---- 3. still-water depth d (Sec. 2.1) on the tile + 1 ring
    for (int k = tid; k < kDcell * kDcell; k += kStencilThreads) {
        int cy = k / kDcell, cx = k % kDcell;
        sm.d[cy * kDStride + cx] = cell_d(cx, cy);
    }
    __syncthreads();

    // ---- 4. fluxes through every face of the tile, each computed once.
    //         Warps 0-3 sweep x-faces, warps 4-7 y-faces; a lane owns one
    //         row (x) or column (y) and 8 consecutive faces of it (the last
    //         warp of each half also face 32), so every cell is reconstructed
    //         once per direction: the right cell of a face is the left cell
    //         of the next.
    {
        const int lane = tid & 31, wq = (tid >> 5) & 3;
        const int f0 = wq * 8, f1 = wq == 3 ? kTile + 1 : f0 + 8;
        real lo[3], hiL[3], hiR[3];
        // the three cells a reconstruction reads slide along the row (or
        // column) one cell per face, so each face loads one new cell and one
        // new pair of corners
        real wq3[3], Pq[3], Qq[3];
        if (tid < 4 * 32) {
            const int r = lane;
            const int rowo = (r + kHalo) * kStride;
            const real *cb = sm.Bc + (r + 1) * kCornerStride;
            real Bf;   // bed at the face about to be computed
            {
                const int o = rowo + f0 + 1;
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    wq3[u] = sm.w[o - 1 + u];
                    Pq[u] = sm.P[o - 1 + u];
                    Qq[u] = sm.Q[o - 1 + u];
                }
                Bf = real(0.5) * (cb[f0 + 1] + cb[f0 + 1 + kCornerStride]);
                recon(th, wq3, Pq, Qq, real(0.5) * (cb[f0] + cb[f0 + kCornerStride]), Bf, lo, hiL);
            }
            for (int f = f0; f < f1; f++) {
                const int o = rowo + f + 2;           // right cell of face f
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    wq3[u] = wq3[u + 1];
                    Pq[u] = Pq[u + 1];
                    Qq[u] = Qq[u + 1];
                }
                wq3[2] = sm.w[o + 1];
                Pq[2] = sm.P[o + 1];
                Qq[2] = sm.Q[o + 1];
                const real Bn = real(0.5) * (cb[f + 2] + cb[f + 2 + kCornerStride]);
                recon(th, wq3, Pq, Qq, Bf, Bn, lo, hiR);
                real H[3];
                cu_flux(g, eps, hiL[0], hiL[1], hiL[2], lo[0], lo[1], lo[2], Bf, H);
                sm.Fx[0][r][f] = H[0];
                sm.Fx[1][r][f] = H[1];
                sm.Fx[2][r][f] = H[2];
                hiL[0] = hiR[0];
                hiL[1] = hiR[1];
                hiL[2] = hiR[2];
                Bf = Bn;
            }
        } else {
            const int c = lane;
            const int tx = c + kHalo;
            const real *cb = sm.Bc + c + 1;
            real Bf;
            {
                const int o = (f0 + 1) * kStride + tx;
#pragma unroll
                for (int u = 0; u < 3; u++) {
                    wq3[u] = sm.w[o + (u - 1) * kStride];
                    Pq[u] = sm.P[o + (u - 1) * kStride];
                    Qq[u] = sm.Q[o + (u - 1) * kStride];
                }
                Bf = real(0.5) * (cb[(f0 + 1) * kCornerStride] + cb[(f0 + 1) * kCornerStride + 1]);
                recon(th, wq3, Pq, Qq, real(0.5) * (cb[f0 * kCornerStride] + cb[f0 * kCornerStride + 1]), Bf, lo,
                      hiL);
            }
            for (int gq = f0; gq < f1; gq++) {
                const int o = (gq + 2) * kStride + tx;  // north cell of face gq
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    wq3[u] = wq3[u + 1];
                    Pq[u] = Pq[u + 1];
                    Qq[u] = Qq[u + 1];
                }
                wq3[2] = sm.w[o + kStride];
                Pq[2] = sm.P[o + kStride];
                Qq[2] = sm.Q[o + kStride];
                const real Bn = real(0.5) * (cb[(gq + 2) * kCornerStride] + cb[(gq + 2) * kCornerStride + 1]);
                recon(th, wq3, Pq, Qq, Bf, Bn, lo, hiR);
                real H[3];
                // normal discharge is Q, tangential is P
                cu_flux(g, eps, hiL[0], hiL[2], hiL[1], lo[0], lo[2], lo[1], Bf, H);
                sm.Fy[0][gq][c] = H[0];
                sm.Fy[1][gq][c] = H[2];
                sm.Fy[2][gq][c] = H[1];
                hiL[0] = hiR[0];
                hiL[1] = hiR[1];
                hiL[2] = hiR[2];
                Bf = Bn;
            }
        }
    }
    __syncthreads();

    // ---- 5. per cell: Eq. 9-13, friction, U*, V*, update
    const real dt = C.dt;
    const real rdx = C.rdx, rdy = C.rdy, rdx2 = C.rdx2, rdy2 = C.rdy2, rdxdy4 = C.rdxdy4;
    const real rdx3h = C.rdx3h, rdy3h = C.rdy3h, rdxdy2h = C.rdxdy2h, rdx2dyh = C.rdx2dyh;
    const real Bd = C.Bd, B3 = C.B3, sixth = C.sixth;
    const bool bsnq = A.phy.model == kBsnq;
    const int friction = A.phy.friction;
    const int lane = tid & 31;
    // the sponge (Eq. 30) on the last stage, where the tile reaches into one
    const bool sponge_tile = A.final_stage &&
                             (O.x0() < C.spw[0] || O.x0() + kTile > nx - C.spw[1] || O.y0() < C.spw[2] ||
                              O.y0() + kTile > ny - C.spw[3]);
    constexpr int kRows = kTile / (kStencilThreads / 32);   // rows per thread
#pragma unroll 1
    for (int rr = 0; rr < kRows; rr++) {
        const int cx = lane, cy = (tid >> 5) + rr * (kStencilThreads / 32);
        const int i = O.x0() + cx, j = O.y0() + cy;
        const bool valid = i < nx && j < ny;
        const int o = (cy + kHalo) * kStride + cx + kHalo;
        const size_t kr = (size_t)j * G.px + i;
        // the history this stage reads, issued before the cell's arithmetic
        // (holding the next row's history in registers as well costs more
        // occupancy than it saves latency)
        Carry<real> cw, cu, cv;
        if (valid) {
            cw = load_carry<real, kSpec>(A, 0, kr);
            cu = load_carry<real, kSpec>(A, 1, kr);
            cv = load_carry<real, kSpec>(A, 2, kr);
        }
        const real *cb = sm.Bc + (cy + 1) * kCornerStride + cx + 1;
        real c00 = cb[0], c10 = cb[1], c01 = cb[kCornerStride], c11 = cb[kCornerStride + 1];
        real Bb = cell_bbar(c00, c10, c01, c11);
        real BxW = real(0.5) * (c00 + c01), BxE = real(0.5) * (c10 + c11);
        real ByS = real(0.5) * (c00 + c10), ByN = real(0.5) * (c01 + c11);
        real w0 = sm.w[o], P0 = sm.P[o], Q0 = sm.Q[o];
        real hb = w0 - Bb;
        real E = -(sm.Fx[0][cy][cx + 1] - sm.Fx[0][cy][cx]) * rdx - (sm.Fy[0][cy + 1][cx] - sm.Fy[0][cy][cx]) * rdy;
        real F = -(sm.Fx[1][cy][cx + 1] - sm.Fx[1][cy][cx]) * rdx - (sm.Fy[1][cy + 1][cx] - sm.Fy[1][cy][cx]) * rdy -
                 g * hb * (BxE - BxW) * rdx;
        real Gq = -(sm.Fx[2][cy][cx + 1] - sm.Fx[2][cy][cx]) * rdx - (sm.Fy[2][cy + 1][cx] - sm.Fy[2][cy][cx]) * rdy -
                  g * hb * (ByN - ByS) * rdy;
        if (friction != kFricNone) {   // Eq. 31-32 with the Eq. 14 device
            real hinv = desing(fmax(hb, real(0)), eps);
            real fc = friction == kFricManning ? C.fric * cbrt_r(hinv) : C.fric;
            real mag = sqrt(P0 * P0 + Q0 * Q0);
            F -= fc * P0 * mag * hinv * hinv;
            Gq -= fc * Q0 * mag * hinv * hinv;
        }
        real Fs = real(0), Gs = real(0);
        const int od = (cy + 1) * kDStride + cx + 1;
        const real dd = sm.d[od];
        if (bsnq) {
            const real ddx = (sm.d[od + 1] - sm.d[od - 1]) * C.hrdx;
            const real ddy = (sm.d[od + kDStride] - sm.d[od - kDStride]) * C.hrdy;
            const real *W = sm.w + o;
            const int S1 = kStride, S2 = 2 * kStride;
            // eta = w - w_s enters only through differences, where w_s cancels
            real e00 = W[0];
            real eE = W[1], eW = W[-1], eN = W[S1], eS = W[-S1];
            real eEE = W[2], eWW = W[-2], eNN = W[S2], eSS = W[-S2];
            real eNE = W[S1 + 1], eNW = W[S1 - 1], eSE = W[-S1 + 1], eSW = W[-S1 - 1];
            real exx = (eE - real(2) * e00 + eW) * rdx2;
            real eyy = (eN - real(2) * e00 + eS) * rdy2;
            real exy = (eNE - eSE - eNW + eSW) * rdxdy4;
            real exxx = (eEE - real(2) * eE + real(2) * eW - eWW) * rdx3h;
            real eyyy = (eNN - real(2) * eN + real(2) * eS - eSS) * rdy3h;
            real exyy = ((eNE - real(2) * eE + eSE) - (eNW - real(2) * eW + eSW)) * rdxdy2h;
            real exxy = ((eNE - real(2) * eN + eNW) - (eSE - real(2) * eS + eSW)) * rdx2dyh;
            F += Bd * g * dd * dd * dd * (exxx + exyy) + Bd * g * dd * dd * (ddx * (real(2) * exx + eyy) + ddy * exy);
            Gq += Bd * g * dd * dd * dd * (eyyy + exxy) + Bd * g * dd * dd * (ddy * (real(2) * eyy + exx) + ddx * exy);
            const real *Pt = sm.P + o, *Qt = sm.Q + o;
            real Qx = (Qt[1] - Qt[-1]) * C.hrdx, Qy = (Qt[S1] - Qt[-S1]) * C.hrdy;
            real Qxy = (Qt[S1 + 1] - Qt[-S1 + 1] - Qt[S1 - 1] + Qt[-S1 - 1]) * rdxdy4;
            real Px = (Pt[1] - Pt[-1]) * C.hrdx, Py = (Pt[S1] - Pt[-S1]) * C.hrdy;
            real Pxy = (Pt[S1 + 1] - Pt[-S1 + 1] - Pt[S1 - 1] + Pt[-S1 - 1]) * rdxdy4;
            Fs = dd * ddx * Qy * sixth + dd * ddy * Qx * sixth + B3 * dd * dd * Qxy;
            Gs = dd * ddy * Px * sixth + dd * ddx * Py * sixth + B3 * dd * dd * Pxy;
        }
        real w1 = w0, dU = real(0), dV = real(0);
        if (valid) {
            real dw = advance<real, kSpec>(A, 0, w0, E, real(0), kr, cw);
            w1 = stage_kind<kSpec>(A) == kAM4 ? dw : w0 + dw;   // the AM4 base of w holds w^n
            dU = advance<real, kSpec>(A, 1, real(0), F, Fs, kr, cu);
            dV = advance<real, kSpec>(A, 2, real(0), Gq, Gs, kr, cv);
            if (w1 < Bb) w1 = Bb;   // Reading A-D1
            if (sponge_tile) {
                real gam = sponge_gamma<real>(C, G, i, j);
                if (gam < real(1) && dd > real(0)) w1 = ws + gam * (w1 - ws);
            }
            A.w_out[kr] = w1;
            A.U_out[kr] = dU;
        }
        const bool dry = valid && (w1 - Bb <= real(0));
        unsigned bits = __ballot_sync(0xffffffffu, dry);
        if (lane == 0 && j < ny) A.mask_r[(size_t)j * G.nwx + (O.x0() >> 5)] = bits;
        if (dry) atomicOr(&sm.colbits[cx], 1u << cy);
        sm.Vout[cy][cx] = dV;
    }
    __syncthreads();
    for (int k = tid; k < kTile * kTile; k += kStencilThreads) {
        int c = k / kTile, r = k % kTile;
        int i = O.x0() + c, j = O.y0() + r;
        if (i < nx && j < ny) A.Vc_out[(size_t)i * G.py + j] = sm.Vout[r][c];
    }
    if (tid < kTile && O.x0() + tid < nx) A.mask_c[(size_t)(O.x0() + tid) * G.nwy + (O.y0() >> 5)] = sm.colbits[tid];
}

template <typename real, int kSpec>
__global__ void __launch_bounds__(kStencilThreads, sizeof(real) == 4 ? 4 : 2) k_stencil(const __grid_constant__ StencilArgs<real> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dependent_launch_wait_then_release();
    stencil_tile<real, kSpec>(A, GridOrigin(), smem_raw);
}

// Copy a scenario's argument block (device memory) into shared memory.
template <typename T>
__device__ __forceinline__ void load_args(T &dst, const T *src)
{
    const int nw = (int)(sizeof(T) / sizeof(int));
    int *d = reinterpret_cast<int *>(&dst);
    const int *s = reinterpret_cast<const int *>(src);
    for (int k = threadIdx.x; k < nw; k += blockDim.x) d[k] = s[k];
}

// Ensemble: the tiles of every member in one launch.  desc[b] names block
// b's member (x) and tile (y: row << 16 | column); the member's arguments
// are copied to shared memory.
template <typename real, int kSpec>
__global__ void __launch_bounds__(kStencilThreads, sizeof(real) == 4 ? 4 : 2)
    k_stencil_batch(const StencilArgs<real> *__restrict__ args, const int2 *__restrict__ desc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) StencilArgs<real> A;
    __shared__ int origin[2];
    const int2 d = desc[blockIdx.x];
    if (threadIdx.x == 0) {
        origin[0] = (d.y & 0xffff) * kTile;
        origin[1] = (d.y >> 16) * kTile;
    }
    load_args(A, args + d.x);
    __syncthreads();
    stencil_tile<real, kSpec>(A, SharedOrigin{origin}, smem_raw);
}

// ------------------------------------------------------------ line solves

// Eq. 23 coefficients of line element k.
template <typename real>
__device__ __forceinline__ void coef23(real B3, real hrh, real srh, real rh2, real dd, real dm, real dp,
                                       real &a, real &b, real &c)
{
    real dda = (dp - dm) * hrh;
    real r = B3 * dd * dd * rh2;
    real s = dd * dda * srh;
    a = s - r;
    b = real(1) + real(2) * r;
    c = -s - r;
}

// Asynchronous copy of one element from global to shared memory (zero-filled
// when !valid, reading nothing); all of a thread's copies are in flight at
// once and cost no registers.  cp_async_wait_all waits for this thread's.
template <typename real>
__device__ __forceinline__ void cp_async_elem(real *smem, const real *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if (sizeof(real) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0)
                     : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0)
                     : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared-memory slot of line element k: element j of segment t sits at
// j * sp + t (sp odd), so the threads of a warp sweeping their segments touch
// consecutive words at every step (no bank conflicts).
__device__ __forceinline__ int seg_slot(int k, int mshift, int sp)
{
    return (k & ((1 << mshift) - 1)) * sp + (k >> mshift);
}

// ------------------------------------------- line solves, segments in registers
//
// A line of n rows (Eq. 21-23) is cut into T = blockDim.x segments of M
// consecutive rows, one per thread; rows from n on are identity rows.  The
// last row of segment t is its separator s_t.  Thread t eliminates the M - 1
// rows before it by Thomas against three right sides (the data, and the
// couplings to s_{t-1} and s_t), so that each of them is y + u s_{t-1} +
// v s_t, and the separators' rows form a tridiagonal system with one row per
// thread.  Lane 31 of each warp holds the warp's separator S_w: a warp
// reduces its other 31 rows by cyclic reduction in registers (shuffles)
// against the same three right sides, and the warps' separators form a
// system of one row per warp, which warp 0 solves the same way.  Two
// barriers per line; the system is strictly diagonally dominant (|d_x| below
// about 5), so no pivoting.

constexpr unsigned kFull = 0xffffffffu;

// Cyclic reduction of a warp's 32 rows a x_{i-1} + b x_i + c x_{i+1} = r
// (rows beyond the warp decoupled), NR right sides at once: afterwards row i
// reads b x_i = r.  Where only the first `rows` rows couple (the rest are
// identity rows), ceil(log2(rows)) levels decouple them.
template <typename real, int NR>
__device__ __forceinline__ void warp_cr(real &a, real &b, real &c, real (&r)[NR], int lane, int rows = 32)
{
#pragma unroll
    for (int s = 1; s < 32; s <<= 1) {
        if (s >= rows) break;
        const real ib = real(1) / b;   // each row's reciprocal, once, to both neighbours
        const real am = __shfl_up_sync(kFull, a, s), ibm = __shfl_up_sync(kFull, ib, s);
        const real cm = __shfl_up_sync(kFull, c, s);
        const real ap = __shfl_down_sync(kFull, a, s), ibp = __shfl_down_sync(kFull, ib, s);
        const real cp = __shfl_down_sync(kFull, c, s);
        real rm[NR], rp[NR];
#pragma unroll
        for (int q = 0; q < NR; q++) {
            rm[q] = __shfl_up_sync(kFull, r[q], s);
            rp[q] = __shfl_down_sync(kFull, r[q], s);
        }
        const real k1 = lane >= s ? a * ibm : real(0);
        const real k2 = lane + s < 32 ? c * ibp : real(0);
        b = b - cm * k1 - ap * k2;
#pragma unroll
        for (int q = 0; q < NR; q++) r[q] = r[q] - rm[q] * k1 - rp[q] * k2;
        a = -am * k1;
        c = -cp * k2;
    }
}

// M consecutive reals at p (16-byte aligned when M * sizeof(real) >= 16)
template <typename real, int M>
__device__ __forceinline__ void load_run(real (&v)[M], const real *p)
{
    if constexpr (M * sizeof(real) >= 16) {
        using V = typename Vec2<real>::type;
        if constexpr (sizeof(real) == 4) {
#pragma unroll
            for (int u = 0; u < M / 4; u++) {
                const float4 q = reinterpret_cast<const float4 *>(p)[u];
                v[4 * u] = q.x;
                v[4 * u + 1] = q.y;
                v[4 * u + 2] = q.z;
                v[4 * u + 3] = q.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < M / 2; u++) {
                const V q = reinterpret_cast<const V *>(p)[u];
                v[2 * u] = q.x;
                v[2 * u + 1] = q.y;
            }
        }
    } else if constexpr (M == 2) {
        const typename Vec2<real>::type q = *reinterpret_cast<const typename Vec2<real>::type *>(p);
        v[0] = q.x;
        v[1] = q.y;
    } else {
#pragma unroll
        for (int u = 0; u < M; u++) v[u] = p[u];
    }
}

template <typename real, int M>
__device__ __forceinline__ void store_run(real *p, const real (&v)[M])
{
    if constexpr (sizeof(real) == 4 && M % 4 == 0) {
#pragma unroll
        for (int u = 0; u < M / 4; u++)
            reinterpret_cast<float4 *>(p)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
    } else if constexpr (M % 2 == 0) {
        using V = typename Vec2<real>::type;
#pragma unroll
        for (int u = 0; u < M / 2; u++) {
            V q;
            q.x = v[2 * u];
            q.y = v[2 * u + 1];
            reinterpret_cast<V *>(p)[u] = q;
        }
    } else {
#pragma unroll
        for (int u = 0; u < M; u++) p[u] = v[u];
    }
}

// Row k of the line's system T: Eq. 23 from the depths dm, dd, dp of rows
// k - 1, k, k + 1, with the boundary rows of Reading A-B2 (a solid or sponge
// end folds the mirrored neighbour into b; at a maker end the known ghost
// increment moves to the right side, *rk -= a * inc, when rk is given);
// identity rows beyond the line.
template <typename real>
__device__ __forceinline__ void t_row(const LineArgs<real> &A, int k, real dm, real dd, real dp, bool lo_sine,
                                      bool hi_sine, real lo_inc, real hi_inc, real &a, real &b, real &c,
                                      real *rk)
{
    if (k < 0 || k >= A.n) {
        a = c = real(0);
        b = real(1);
        return;
    }
    coef23(A.c.B3, A.hrh, A.srh, A.rh2, dd, dm, dp, a, b, c);
    if (k == 0) {
        if (!lo_sine) b -= a;
        else if (rk) *rk -= a * lo_inc;
        a = real(0);
    }
    if (k == A.n - 1) {
        if (!hi_sine) b -= c;
        else if (rk) *rk -= c * hi_inc;
        c = real(0);
    }
}

// The values that cross warps, per warp: lane 0's first interior row
// (y, u, v) and its separator's (Y, U, V); lane 31's row and its last
// interior row; lane 30's (Y, U, V); the warps' separators.
template <typename real>
struct LineShared {
    real sh0[32][3], sh1[32][3], sh31[32][7], sh30[32][3], shS[32];
};

// One line of one family: kMode 0, the step's solve with P^n + x, the sponge
// on the last stage and the dry mask; 1, the transposed system T^T y = r
// (row k of T^T is (c_{k-1}, b_k, a_{k+1}) of T's rows), y alone; 2, T x = r,
// x alone.  The line's own segment count A.nseg (a multiple of 32, at most
// the threads given to the line) sets the reduction, so the result does not
// depend on the block size: warps beyond it only pass the barriers.  A block
// may solve several lines side by side: tid is the thread's index among its
// line's threads and wbase the block warp its line starts at; every thread
// of the block takes the call (with `valid` false where its slot has no
// line), since the two barriers are the block's.
template <typename real, int M, int kMode>
__device__ __forceinline__ void line_solve_reg(const LineArgs<real> &A, int line, LineShared<real> &L, int tid,
                                               int wbase, bool valid)
{
    static_assert(M >= 2 && M <= 8, "rows per thread");
    constexpr int m1 = M - 1;
    real(*sh0)[3] = L.sh0 + wbase;
    real(*sh1)[3] = L.sh1 + wbase;
    real(*sh31)[7] = L.sh31 + wbase;
    real(*sh30)[3] = L.sh30 + wbase;
    real *shS = L.shS + wbase;
    const int n = A.n, lane = tid & 31, warp = tid >> 5, nw = valid ? A.nseg >> 5 : 0;
    const bool act = warp < nw;            // whole warps: the segment count is a multiple of 32
    const int f = tid * M;
    const int lo_side = A.dir == 0 ? 0 : 2, hi_side = A.dir == 0 ? 1 : 3;
    const bool lo_sine = (A.c.sine >> lo_side) & 1, hi_sine = (A.c.sine >> hi_side) & 1;
    const int gvar = A.dir == 0 ? 1 : 2;   // ghost discharge: P on x-lines, Q on y-lines
    const size_t lo = (size_t)line * A.pitch;
    real *out = A.sol + lo;
    const bool any = act && f < n;         // the segment holds rows of the line

    // What the kernel before this one on the stream does not write comes
    // first: P^n (read in the epilogue: to L1 now), the depths, the rows of
    // the system and the makers' ghost increments.  Then the wait for that
    // kernel (a stencil launch), and the right side it wrote.
    if (any && kMode == 0) {
#pragma unroll
        for (int u = 0; u < M; u += 32 / (int)sizeof(real))
            asm volatile("prefetch.global.L1 [%0];" ::"l"(A.base + lo + f + u));
    }
    real r[M];
    auto load_rhs = [&]() {
        dependent_launch_wait_then_release();
        if (any) {
            if (kMode == 0)   // the dry bits, read in the epilogue
                asm volatile("prefetch.global.L1 [%0];" ::"l"(A.mask + (size_t)line * A.nwords + (f >> 5)));
            load_run<real, M>(r, A.rhs + lo + f);
#pragma unroll
            for (int j = 0; j < M; j++)
                if (f + j >= n) r[j] = real(0);
        } else {
#pragma unroll
            for (int j = 0; j < M; j++) r[j] = real(0);
        }
    };
    real x[M];
    if (A.identity) {   // NLSW: P = U*
        load_rhs();
#pragma unroll
        for (int j = 0; j < M; j++) x[j] = r[j];
    } else {
        // depths of rows f - 2 .. f + M + 1 (mirrored at the ends)
        real dv[M + 4];
        const real *dl = A.d + lo;
        if (any) {
            real mid[M];
            load_run<real, M>(mid, dl + f);
#pragma unroll
            for (int j = 0; j < M; j++) dv[j + 2] = f + j < n ? mid[j] : dl[n - 1];
            dv[0] = dl[f >= 2 ? f - 2 : 0];
            dv[1] = dl[f >= 1 ? f - 1 : 0];
            dv[M + 2] = dl[f + M < n ? f + M : n - 1];
            dv[M + 3] = dl[f + M + 1 < n ? f + M + 1 : n - 1];
        } else {
#pragma unroll
            for (int j = 0; j < M + 4; j++) dv[j] = real(0);
        }
        // rows f .. f + M - 1 of the system solved (T, or T^T in mode 1):
        // Eq. 23 on every row, then the rows at the line's ends (Reading
        // A-B2) and beyond it (identity), in the segments that hold them
        real ra[M], rb[M], rc[M];
        const bool at_end = f + M > n - 1;   // holds row n - 1 (or lies beyond)
        if (kMode == 1) {
            real ta[M + 2], tb[M + 2], tc[M + 2];   // T's rows f - 1 .. f + M
#pragma unroll
            for (int j = 0; j < M + 2; j++)
                coef23(A.c.B3, A.hrh, A.srh, A.rh2, dv[j + 1], dv[j], dv[j + 2], ta[j], tb[j], tc[j]);
            if (f == 0 || at_end) {
#pragma unroll
                for (int j = 0; j < M + 2; j++)
                    t_row(A, f - 1 + j, dv[j], dv[j + 1], dv[j + 2], lo_sine, hi_sine, real(0), real(0), ta[j],
                          tb[j], tc[j], (real *)nullptr);
            }
#pragma unroll
            for (int j = 0; j < M; j++) {
                ra[j] = tc[j];
                rb[j] = tb[j + 1];
                rc[j] = ta[j + 2];
            }
            load_rhs();
        } else {
#pragma unroll
            for (int j = 0; j < M; j++)
                coef23(A.c.B3, A.hrh, A.srh, A.rh2, dv[j + 2], dv[j + 1], dv[j + 3], ra[j], rb[j], rc[j]);
            // the makers' ghost increments (t^{n+1} - t^n) at the line's ends
            // and the coefficients that carry them to the right side
            real lo_inc = real(0), hi_inc = real(0), a_lo = real(0), c_hi = real(0);
            if (f == 0 || at_end) {
                if (lo_sine && f == 0) {
                    lo_inc = A.ghost[ghost_index(1, lo_side, 0, gvar, line + 2, A.c.npos)] -
                             A.ghost[ghost_index(0, lo_side, 0, gvar, line + 2, A.c.npos)];
                    a_lo = ra[0];
                }
                if (hi_sine && at_end && f <= n - 1) {
                    hi_inc = A.ghost[ghost_index(1, hi_side, 0, gvar, line + 2, A.c.npos)] -
                             A.ghost[ghost_index(0, hi_side, 0, gvar, line + 2, A.c.npos)];
#pragma unroll
                    for (int j = 0; j < M; j++)
                        if (f + j == n - 1) c_hi = rc[j];
                }
#pragma unroll
                for (int j = 0; j < M; j++)
                    t_row(A, f + j, dv[j + 1], dv[j + 2], dv[j + 3], lo_sine, hi_sine, lo_inc, hi_inc, ra[j], rb[j],
                          rc[j], (real *)nullptr);
            }
            load_rhs();
            if (lo_sine && f == 0) r[0] -= a_lo * lo_inc;   // Reading A-B2: the known ghost increment moves to the right side
            if (hi_sine && at_end && f <= n - 1) {
#pragma unroll
                for (int j = 0; j < M; j++)
                    if (f + j == n - 1) r[j] -= c_hi * hi_inc;
            }
        }
        // Thomas on rows f .. f + M - 2 against (r, -a_f e_0, -c e_last)
        real g[m1], y[m1], uu[m1], vv[m1];
        real Y = real(0), U = real(0), V = real(0);
        {
            real gp = real(0), yp = real(0), up = real(0);
#pragma unroll
            for (int j = 0; j < m1; j++) {
                const real inv = real(1) / (rb[j] - ra[j] * gp);
                g[j] = j + 1 < m1 ? rc[j] * inv : real(0);
                y[j] = (r[j] - ra[j] * yp) * inv;
                uu[j] = (j == 0 ? -ra[0] : -ra[j] * up) * inv;
                vv[j] = j + 1 == m1 ? -rc[j] * inv : real(0);
                gp = g[j];
                yp = y[j];
                up = uu[j];
            }
#pragma unroll
            for (int j = m1 - 2; j >= 0; j--) {
                y[j] -= g[j] * y[j + 1];
                uu[j] -= g[j] * uu[j + 1];
                vv[j] = -g[j] * vv[j + 1];
            }
        }
        // the separator's row in (s_{t-1}, s_t, s_{t+1}): the next thread's
        // first interior row by shuffle (lane 31: later, from shared memory)
        const real al = ra[m1], bl = rb[m1], cl = rc[m1], rl = r[m1];
        if (act) {
        const real ny0 = __shfl_down_sync(kFull, y[0], 1), nu0 = __shfl_down_sync(kFull, uu[0], 1);
        const real nv0 = __shfl_down_sync(kFull, vv[0], 1);
        real a1 = al * uu[m1 - 1];
        real b1 = al * vv[m1 - 1] + bl + cl * nu0;
        real c1 = cl * nv0;
        real rr1[3] = {rl - al * y[m1 - 1] - cl * ny0, real(0), real(0)};
        // lanes 0..30 reduced against (S_{w-1}, S_w): lane 0's coupling to
        // the previous warp's separator and lane 30's to lane 31 move to the
        // right sides; lane 31 is the warp's separator
        if (lane == 0) {
            rr1[1] = -a1;
            a1 = real(0);
        }
        if (lane == 30) {
            rr1[2] = -c1;
            c1 = real(0);
        }
        if (lane == 31) {
            a1 = c1 = real(0);
            b1 = real(1);
            rr1[0] = real(0);
        }
        warp_cr<real, 3>(a1, b1, c1, rr1, lane);
        const real ib = real(1) / b1;
        Y = rr1[0] * ib;
        U = rr1[1] * ib;
        V = rr1[2] * ib;
        const real Y30 = __shfl_up_sync(kFull, Y, 1), U30 = __shfl_up_sync(kFull, U, 1);
        const real V30 = __shfl_up_sync(kFull, V, 1);
        if (lane == 0) {
            sh0[warp][0] = y[0];
            sh0[warp][1] = uu[0];
            sh0[warp][2] = vv[0];
            sh1[warp][0] = Y;
            sh1[warp][1] = U;
            sh1[warp][2] = V;
        }
        if (lane == 31) {
            sh31[warp][0] = al;
            sh31[warp][1] = bl;
            sh31[warp][2] = cl;
            sh31[warp][3] = rl;
            sh31[warp][4] = y[m1 - 1];
            sh31[warp][5] = uu[m1 - 1];
            sh31[warp][6] = vv[m1 - 1];
            sh30[warp][0] = Y30;
            sh30[warp][1] = U30;
            sh30[warp][2] = V30;
        }
        }
        __syncthreads();
        if (warp == 0) {
            // row of separator S_w in (S_{w-1}, S_w, S_{w+1})
            real A2 = real(0), B2 = real(1), C2 = real(0), R2[1] = {real(0)};
            if (lane < nw) {
                const bool nx = lane + 1 < nw;
                const real p0 = nx ? sh0[lane + 1][0] : real(0), p1 = nx ? sh0[lane + 1][1] : real(0);
                const real p2 = nx ? sh0[lane + 1][2] : real(0);
                const real q0 = nx ? sh1[lane + 1][0] : real(0), q1 = nx ? sh1[lane + 1][1] : real(0);
                const real q2 = nx ? sh1[lane + 1][2] : real(0);
                const real la = sh31[lane][0], lb = sh31[lane][1], lc = sh31[lane][2], lr = sh31[lane][3];
                const real ly = sh31[lane][4], lu = sh31[lane][5], lv = sh31[lane][6];
                // lane 31's separator row in (x_{lane 30}, S_w, x_{next warp's lane 0})
                const real A1 = la * lu, B1 = la * lv + lb + lc * p1, C1 = lc * p2, R1 = lr - la * ly - lc * p0;
                A2 = A1 * sh30[lane][1];
                B2 = A1 * sh30[lane][2] + B1 + C1 * q1;
                C2 = C1 * q2;
                R2[0] = R1 - A1 * sh30[lane][0] - C1 * q0;
            }
            warp_cr<real, 1>(A2, B2, C2, R2, lane, nw);
            if (lane < nw) shS[lane] = R2[0] / B2;
        }
        __syncthreads();
        if (!act) return;
        const real Sw = shS[warp], Sm = warp > 0 ? shS[warp - 1] : real(0);
        const real st = lane == 31 ? Sw : Y + U * Sm + V * Sw;      // this thread's separator
        const real up1 = __shfl_up_sync(kFull, st, 1);
        const real sm = lane == 0 ? Sm : up1;                          // the previous thread's
#pragma unroll
        for (int j = 0; j < m1; j++) x[j] = y[j] + uu[j] * sm + vv[j] * st;
        x[m1] = st;
    }
    if (!any) return;
    real o[M];
    if (kMode == 0 && A.xcap) {   // the solution itself, for the adjoint's depth term
        real *xc = A.xcap + lo;
        if (f + M <= n) {
            store_run<real, M>(xc + f, x);
        } else {
#pragma unroll
            for (int j = 0; j < M; j++)
                if (f + j < n) xc[f + j] = x[j];
        }
    }
    if (kMode != 0) {
#pragma unroll
        for (int j = 0; j < M; j++) o[j] = x[j];
    } else {
        // epilogue: P^n + increment, sponge (Eq. 30) on the last stage, zero
        // discharge where dry
        load_run<real, M>(o, A.base + lo + f);
        const uint32_t bits = A.mask[(size_t)line * A.nwords + (f >> 5)] >> (f & 31);
        // the sponge only where the segment reaches into one (Eq. 30): the
        // sides across the line give one factor for the whole segment, the
        // sides along it one per row
        bool sponge = false;
        real g_across = real(1);
        const int s_lo = A.dir == 0 ? 0 : 2, a_lo = A.dir == 0 ? 2 : 0;   // west/south along, across
        if (A.final_stage) {
            const int *w = A.c.spw;
            const int across = A.dir == 0 ? A.geo.ny : A.geo.nx;
            sponge = f < w[s_lo] || f + M > n - w[s_lo + 1] || line < w[a_lo] || line >= across - w[a_lo + 1];
            if (sponge)
                g_across = fmin(sponge_side(A.c, a_lo, line), sponge_side(A.c, a_lo + 1, across - 1 - line));
        }
#pragma unroll
        for (int j = 0; j < M; j++) {
            real v = o[j] + x[j];
            if (sponge) {
                const int k = f + j;
                if (k < n)
                    v *= fmin(g_across, fmin(sponge_side(A.c, s_lo, k), sponge_side(A.c, s_lo + 1, n - 1 - k)));
            }
            if ((bits >> j) & 1u) v = real(0);
            o[j] = v;
        }
    }
    if (f + M <= n) {
        store_run<real, M>(out + f, o);
    } else {
#pragma unroll
        for (int j = 0; j < M; j++)
            if (f + j < n) out[f + j] = o[j];
    }
}

// ----------------------------------------- line solves, segments in shared memory
//
// Lines too long for one segment per thread in registers (FP32 beyond 8192
// rows, FP64 beyond 4096).
//
// One line of one family, segments in shared memory (x-row or y-column): the whole solve and epilogue.
// kMode 0: the step's solve, P^n + x with the sponge and the dry mask;
// 1: the transposed system T^T y = r (the adjoint), whose row k is
// (c_{k-1}, b_k, a_{k+1}) of T's rows with T's boundary rows, y alone;
// 2: the step's system T x = r, x alone.
template <typename real, int M, int kMode = 0>
__device__ __forceinline__ void line_solve_seg(const LineArgs<real> &A, int line, unsigned char *smem_raw)
{
    const int n = A.n, S = A.nseg, N2 = 2 * S;
    constexpr int m = M;                             // rows per segment
    const int mshift = A.mshift, sp = A.sp;
    const int npad = S * m;                          // lines padded with identity rows
    real *sA = reinterpret_cast<real *>(smem_raw);   // d, then alpha / alpha-hat
    real *sC = sA + m * sp;                          // gamma / gamma-hat
    real *sR = sC + m * sp;                          // rhs -> rho -> rho-hat -> x
    real *ra = sR + m * sp, *rb = ra + N2, *rc = rb + N2, *rr = rc + N2;
    uint32_t *smask = reinterpret_cast<uint32_t *>(rr + N2);   // dry bits of the line
    const int tid = threadIdx.x, T = blockDim.x;
    const Geo &G = A.geo;
    const real rh2 = A.rh2, hrh = A.hrh, srh = A.srh;
    const real B3 = A.c.B3;
    const int lo_side = A.dir == 0 ? 0 : 2, hi_side = A.dir == 0 ? 1 : 3;
    const bool lo_sine = (A.c.sine >> lo_side) & 1, hi_sine = (A.c.sine >> hi_side) & 1;
    const int gvar = A.dir == 0 ? 1 : 2;   // ghost discharge: P on x-lines, Q on y-lines
    constexpr bool kT = kMode == 1;

    {
        const real *rhs = A.rhs + (size_t)line * A.pitch;
        const real *dl = A.d + (size_t)line * A.pitch;
        // P^n (or Q^n) of the elements this thread writes in the epilogue,
        // loaded now so the loads complete during the elimination
        constexpr int kMaxOwn = M == 32 ? 16 : (M < 8 ? M : 8);   // ceil(n / T) <= kMaxOwn (line_threads)
        real own[kMaxOwn];
        {
            const real *bs = A.base + (size_t)line * A.pitch;
#pragma unroll
            for (int u = 0; u < kMaxOwn; u++) {
                const int k = tid + u * T;
                own[u] = k < n ? bs[k] : real(0);
            }
        }
        if (kMode == 0) {   // the dry bits serve the epilogue alone
            const uint32_t *mw = A.mask + (size_t)line * A.nwords;
            for (int k = tid; k < A.nwords; k += T) smask[k] = mw[k];
        }
        // right side and depth straight into their segment-major slots
        // (d = 0 on the padding rows: a = c = 0, b = 1)
#pragma unroll
        for (int u = 0; u < M; u++) {
            const int k = tid + u * T;
            if (k < npad) {
                const int q = seg_slot(k, mshift, sp);
                const bool in = k < n;
                cp_async_elem(sR + q, rhs + (in ? k : 0), in);
                cp_async_elem(sA + q, dl + (in ? k : 0), in);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        if (!A.identity) {
        const bool act = tid < S;
        const int f = tid * m, l = f + m - 1;
        real dm = real(0), dp = real(0), dcur = real(0), dlast = real(0), dm2 = real(0), dp2 = real(0);
        if (act) {
            dlast = sA[seg_slot(n - 1, mshift, sp)];
            dm = f > 0 ? sA[seg_slot(f - 1, mshift, sp)] : sA[seg_slot(0, mshift, sp)];
            dp = l + 1 < n ? sA[seg_slot(l + 1, mshift, sp)] : dlast;   // mirrored beyond the end
            dcur = sA[tid];
            if (kT) {   // one more on each side for the neighbouring rows' coefficients
                dm2 = f > 1 ? sA[seg_slot(f - 2, mshift, sp)] : sA[seg_slot(0, mshift, sp)];
                dp2 = l + 2 < n ? sA[seg_slot(l + 2, mshift, sp)] : dlast;
            }
        }
        __syncthreads();
        real af = 0, bf = 1, cf = 0, rf = 0;
        if (act) {
            // forward: rows f+1..l as alpha x_f + x_k + gamma x_{k+1} = rho
            real dprev = dm, dprev2 = dm2, ap = 0, gp = 0, rp = 0;
#pragma unroll
            for (int j = 0; j < m; j++) {
                const int k = f + j, q = j * sp + tid;
                real dnext = j + 1 < m ? (k + 1 < n ? sA[q + sp] : dlast) : dp;
                real ak, bk, ck;
                coef23(B3, hrh, srh, rh2, dcur, dprev, dnext, ak, bk, ck);
                real rk = sR[q];
                if (kT) {
                    const real dnext2 = j + 2 < m ? (k + 2 < n ? sA[q + 2 * sp] : dlast) : (j + 2 == m ? dp : dp2);
                    if (k == 0 && !lo_sine) bk -= ak;
                    if (k == n - 1 && !hi_sine) bk -= ck;
                    real am, bm, cm, a1, b1, c1;
                    coef23(B3, hrh, srh, rh2, dprev, dprev2, dcur, am, bm, cm);    // row k - 1
                    coef23(B3, hrh, srh, rh2, dnext, dcur, dnext2, a1, b1, c1);    // row k + 1
                    ak = k >= 1 && k - 1 < n - 1 ? cm : real(0);   // c_{n-1} is 0 (boundary row)
                    ck = k + 1 <= n - 1 ? a1 : real(0);
                    if (k >= n) {   // padding: identity rows
                        ak = ck = real(0);
                        bk = real(1);
                    }
                    dprev2 = dprev;
                } else if (k == 0) {   // Reading A-B2: mirror, or the known ghost increment
                    if (lo_sine) {
                        const real *t0 = A.ghost + ghost_index(0, lo_side, 0, gvar, line + 2, A.c.npos);
                        const real *t1 = A.ghost + ghost_index(1, lo_side, 0, gvar, line + 2, A.c.npos);
                        rk -= ak * (t1[0] - t0[0]);
                    } else {
                        bk -= ak;
                    }
                    ak = real(0);
                }
                if (!kT && k == n - 1) {
                    if (hi_sine) {
                        const real *t0 = A.ghost + ghost_index(0, hi_side, 0, gvar, line + 2, A.c.npos);
                        const real *t1 = A.ghost + ghost_index(1, hi_side, 0, gvar, line + 2, A.c.npos);
                        rk -= ck * (t1[0] - t0[0]);
                    } else {
                        bk -= ck;
                    }
                    ck = real(0);
                }
                if (j == 0) {
                    af = ak;
                    bf = bk;
                    cf = ck;
                    rf = rk;
                } else {
                    real al, ga, rho;
                    if (j == 1) {
                        real inv = real(1) / bk;
                        al = ak * inv;
                        ga = ck * inv;
                        rho = rk * inv;
                    } else {
                        real inv = real(1) / (bk - ak * gp);
                        al = -ak * ap * inv;
                        ga = ck * inv;
                        rho = (rk - ak * rp) * inv;
                    }
                    sA[q] = al;
                    sC[q] = ga;
                    sR[q] = rho;
                    ap = al;
                    gp = ga;
                    rp = rho;
                }
                dprev = dcur;
                dcur = dnext;
            }
            // backward: rows l-2..f+1 as x_k = rho^ - alpha^ x_f - gamma^ x_l
            real ah = sA[(m - 2) * sp + tid], gh = sC[(m - 2) * sp + tid], rhh = sR[(m - 2) * sp + tid];
#pragma unroll
            for (int j = m - 3; j >= 1; j--) {
                const int q = j * sp + tid;
                real ga = sC[q];
                rhh = sR[q] - ga * rhh;
                ah = sA[q] - ga * ah;
                gh = -ga * gh;
                sA[q] = ah;
                sC[q] = gh;
                sR[q] = rhh;
            }
            // reduced rows: (x_{l of prev}, x_f, x_l) and (x_f, x_l, x_{f of next})
            const int q1 = sp + tid, ql = (m - 1) * sp + tid;
            ra[2 * tid] = af;
            if (m > 2) {   // x_{f+1} = rho^ - alpha^ x_f - gamma^ x_l
                rb[2 * tid] = bf - cf * sA[q1];
                rc[2 * tid] = -cf * sC[q1];
                rr[2 * tid] = rf - cf * sR[q1];
            } else {       // two rows: x_{f+1} is x_l itself
                rb[2 * tid] = bf;
                rc[2 * tid] = cf;
                rr[2 * tid] = rf;
            }
            ra[2 * tid + 1] = sA[ql];
            rb[2 * tid + 1] = real(1);
            rc[2 * tid + 1] = sC[ql];
            rr[2 * tid + 1] = sR[ql];
        }
        __syncthreads();
        // parallel cyclic reduction of the 2S interface rows until they fall
        // into P independent systems (rows r, r + P, r + 2P, ...), which one
        // thread each then solves by elimination (fewer levels and barriers)
        const int P = N2 > 64 ? 32 : N2;
        for (int s = 1; s < P; s <<= 1) {
            real na[2], nb[2], nc[2], nr[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                int e = tid + u * T;
                if (e >= N2) continue;
                real ae = ra[e], be = rb[e], ce = rc[e], re = rr[e];
                real k1 = real(0), k2 = real(0), am = 0, cm = 0, rm = 0, ap = 0, cp = 0, rp = 0;
                if (e - s >= 0) {
                    k1 = ae / rb[e - s];
                    am = ra[e - s];
                    cm = rc[e - s];
                    rm = rr[e - s];
                }
                if (e + s < N2) {
                    k2 = ce / rb[e + s];
                    ap = ra[e + s];
                    cp = rc[e + s];
                    rp = rr[e + s];
                }
                na[u] = -am * k1;
                nc[u] = -cp * k2;
                nb[u] = be - cm * k1 - ap * k2;
                nr[u] = re - rm * k1 - rp * k2;
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 2; u++) {
                int e = tid + u * T;
                if (e >= N2) continue;
                ra[e] = na[u];
                rb[e] = nb[u];
                rc[e] = nc[u];
                rr[e] = nr[u];
            }
            __syncthreads();
        }
        if (P < N2) {
            if (tid < P) {
                real cprev = real(0), rprev = real(0);
                int e = tid;
                for (; e < N2; e += P) {
                    const real ae = ra[e];
                    const real inv = real(1) / (rb[e] - ae * cprev);
                    cprev = rc[e] * inv;
                    rprev = (rr[e] - ae * rprev) * inv;
                    rc[e] = cprev;
                    rr[e] = rprev;
                    rb[e] = real(1);
                }
                real x = rprev;
                for (e -= 2 * P; e >= 0; e -= P) {
                    x = rr[e] - rc[e] * x;
                    rr[e] = x;
                }
            }
            __syncthreads();
        }
        if (act) {
            real xf = rr[2 * tid] / rb[2 * tid], xl = rr[2 * tid + 1] / rb[2 * tid + 1];
#pragma unroll
            for (int j = 1; j < m - 1; j++) {
                const int q = j * sp + tid;
                sR[q] = sR[q] - sA[q] * xf - sC[q] * xl;
            }
            sR[tid] = xf;
            sR[(m - 1) * sp + tid] = xl;
        }
        __syncthreads();
        }
        // epilogue: P^n + increment, sponge (Eq. 30) on the last stage, zero
        // discharge where dry
        real *out = A.sol + (size_t)line * A.pitch;
        if (kMode != 0) {   // the solution alone
            for (int k = tid; k < n; k += T) out[k] = sR[seg_slot(k, mshift, sp)];
            return;
        }
#pragma unroll
        for (int u = 0; u < kMaxOwn; u++) {
            const int k = tid + u * T;
            if (k >= n) continue;
            const real xk = sR[seg_slot(k, mshift, sp)];
            if (A.xcap) A.xcap[(size_t)line * A.pitch + k] = xk;
            real v = own[u] + xk;
            if (A.final_stage) {
                int i = A.dir == 0 ? k : line, j = A.dir == 0 ? line : k;
                v *= sponge_gamma<real>(A.c, G, i, j);
            }
            if ((smask[k >> 5] >> (k & 31)) & 1u) v = real(0);
            out[k] = v;
        }
    }
}

// The segment length of the line's family picks the instance.
template <typename real, int kMode>
__device__ __forceinline__ void line_solve_any(const LineArgs<real> &A, int line, LineShared<real> &L,
                                               int tid = threadIdx.x, int wbase = 0, bool valid = true)
{
    if (A.mshift == 3)
        line_solve_reg<real, 8, kMode>(A, line, L, tid, wbase, valid);
    else if (A.mshift == 2)
        line_solve_reg<real, 4, kMode>(A, line, L, tid, wbase, valid);
    else
        line_solve_reg<real, 2, kMode>(A, line, L, tid, wbase, valid);
}

// kOcc: blocks of at most 256 threads held to 48 registers, so that 5 of
// them fit an SM (the register path is latency-bound); else up to 1024
// (FP32) or 512 (FP64) threads.
template <typename real, int kMode, int kOcc = 0>
__global__ void __launch_bounds__(kOcc ? 256 : (sizeof(real) == 4 ? 1024 : 512), kOcc ? 5 : 1)
    k_lines(const __grid_constant__ LinePair<real> PA)
{
    // blocks [0, nlines of x) solve x-rows, the rest y-columns (the solve
    // waits for the kernel before this one once it has read what that
    // kernel does not write)
    __shared__ LineShared<real> L;
    const int fam = blockIdx.x < PA.L[0].nlines ? 0 : 1;
    const int line = fam == 0 ? blockIdx.x : blockIdx.x - PA.L[0].nlines;
    line_solve_any<real, kMode>(PA.L[fam], line, L);
}

template <typename real, int M, int kMode>
__global__ void __launch_bounds__(sizeof(real) == 4 ? 1024 : 512) k_lines_seg(const __grid_constant__ LinePair<real> PA)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    dependent_launch_wait_then_release();
    const int fam = blockIdx.x < PA.L[0].nlines ? 0 : 1;
    const int line = fam == 0 ? blockIdx.x : blockIdx.x - PA.L[0].nlines;
    line_solve_seg<real, M, kMode>(PA.L[fam], line, smem_raw);
}

// Ensemble: lines of many members and both families in one launch, all of
// one configuration.  desc[b] names block b's family (x) and line (y).
template <typename real, int kOcc = 0>
__global__ void __launch_bounds__(kOcc ? 256 : (sizeof(real) == 4 ? 1024 : 512), kOcc ? 5 : 1)
    k_lines_batch(const LineArgs<real> *__restrict__ args, const int2 *__restrict__ desc)
{
    __shared__ __align__(16) LineArgs<real> A;
    __shared__ LineShared<real> L;
    const int2 d = desc[blockIdx.x];
    load_args(A, args + d.x);
    __syncthreads();
    line_solve_any<real, 0>(A, d.y, L);
}

template <typename real, int M>
__global__ void __launch_bounds__(sizeof(real) == 4 ? 1024 : 512)
    k_lines_batch_seg(const LineArgs<real> *__restrict__ args, const int2 *__restrict__ desc)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) LineArgs<real> A;
    const int2 d = desc[blockIdx.x];
    load_args(A, args + d.x);
    __syncthreads();
    line_solve_seg<real, M>(A, d.y, smem_raw);
}

// ------------------------------------------------- persistent ensemble launch

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of the persistent launch (a cooperative launch: every
// block is resident).  bar[0] counts arrivals, bar[1] is the generation,
// bar[2] the status.  Each wait is bounded by timeout_ns of the global
// timer: a block that gives up sets the status to 1, and every block ends
// the launch at its next barrier.  The last block to arrive clears *reset
// (a work counter no block uses until after the next barrier) before it
// releases the others.  Returns false when the launch must end.
__device__ __noinline__ bool grid_sync(unsigned *bar, unsigned expect, long long timeout_ns, int *reset = nullptr)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vb = bar;
        int good = vb[2] == 0u;
        if (good) {
            const unsigned gen = vb[1];
            __threadfence();   // the block's writes (ordered by the block barrier) before its arrival
            if (atomicAdd(bar, 1u) + 1u == expect) {
                atomicExch(bar, 0u);
                if (reset) atomicExch(reset, 0);
                __threadfence();
                atomicAdd(bar + 1, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                while (vb[1] == gen) {
                    if (vb[2] != 0u) {
                        good = 0;
                        break;
                    }
                    if ((long long)(global_ns() - t0) > timeout_ns) {
                        atomicExch(bar + 2, 1u);
                        good = 0;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            __threadfence();   // the others' writes after the release
        }
        ok = good && vb[2] == 0u;
    }
    __syncthreads();
    return ok != 0;
}

// The phases' work as calls of their own, so that each gets the register
// file to itself instead of sharing one allocation with the launch's loops.
// The arguments sit in shared memory and nothing the work stores aliases
// them, which the compiler is told so that it keeps them in registers
// across the global stores.
template <typename real, int kSpec>
__device__ __noinline__ void persist_tile(const StencilArgs<real> &__restrict__ A, const int *origin,
                                          unsigned char *smem_raw)
{
    __builtin_assume(__isShared(&A));
    stencil_tile<real, kSpec>(A, SharedOrigin{origin}, smem_raw);
}

template <typename real, int M>
__device__ __noinline__ void persist_line(const LineArgs<real> &__restrict__ A, int line, LineShared<real> &L, int tid,
                                          int wbase, bool valid)
{
    __builtin_assume(__isShared(&A));
    line_solve_reg<real, M, 0>(A, line, L, tid, wbase, valid);
}

// A descriptor or entry index out of range: recorded once in bar[3] (code
// in the top byte, the index below), and the work it names is skipped.
__device__ __forceinline__ void persist_flag(unsigned *bar, unsigned code, unsigned info)
{
    atomicCAS(bar + 3, 0u, (code << 24) | (info & 0xffffffu));
}

// One launch for nsteps lockstep steps of an ensemble: the work of each
// batched launch (ghost tables; per stage the stencil tiles, then the line
// solves) spread over the resident blocks, a grid-wide barrier where a
// batched launch would end.  Every block runs the same loop, so each takes
// every barrier.
template <typename real>
__global__ void __launch_bounds__(kStencilThreads, sizeof(real) == 4 ? 4 : 2)
    k_ensemble_persistent(const __grid_constant__ PersistArgs<real> P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) StencilArgs<real> As;
    __shared__ int origin[2];
    __shared__ int item;
    // the line phases reuse the stencil's shared memory: a slot's arguments,
    // then the values that cross warps
    static_assert(sizeof(LineArgs<real>) * (kStencilThreads / 32) + sizeof(LineShared<real>) <=
                      sizeof(StencilSmem<real>),
                  "line phase shared memory");
    LineArgs<real> *Al = reinterpret_cast<LineArgs<real> *>(smem_raw);
    LineShared<real> &L =
        *reinterpret_cast<LineShared<real> *>(smem_raw + sizeof(LineArgs<real>) * (kStencilThreads / 32));
    if (P.barrier_only) {
        grid_sync(P.bar, P.expect, P.timeout_ns);
        return;
    }
    // Tiles and line passes go to blocks as they free up (a counter per
    // phase, three used in turn), as the hardware hands out the blocks of a
    // launch, so that a phase ends when its work does and not with its
    // slowest block's fixed share.
    int phase = 0;
    auto next_item = [&]() -> int {
        __syncthreads();   // the block is done with its previous item
        if (threadIdx.x == 0) item = atomicAdd(P.work + phase % 3, 1);
        __syncthreads();
        return item;
    };
    auto end_phase = [&]() -> bool {
        const bool ok = grid_sync(P.bar, P.expect, P.timeout_ns, P.work + (phase + 2) % 3);
        phase++;
        return ok;
    };
    for (int s = 0; s < P.nsteps; s++) {
        const int ph = (P.phase0 + s) % 6;
        if (P.gblocks > 0) {
            // ghost tables: two 128-position blocks per pass
            for (int b = 2 * blockIdx.x; b < P.gblocks; b += 2 * gridDim.x) {
                const int blk = b + (threadIdx.x >> 7);
                if (blk < P.gblocks) ghost_batch_block(P.gargs, P.gstart, P.ngm, blk, threadIdx.x & 127, P.k0 + s);
            }
            if (!end_phase()) return;
        }
        for (int stage = 0; stage < P.nstages; stage++) {
            const int ei = P.ent[ph][stage];
            if (ei < 0 || ei >= P.nent) {
                if (threadIdx.x == 0) persist_flag(P.bar, 3u, (unsigned)(ph * 16 + stage));
                return;   // every block returns here: no barrier is left waiting
            }
            const unsigned char *ent = P.entries + (size_t)ei * P.entry_bytes;
            const StencilArgs<real> *sa = reinterpret_cast<const StencilArgs<real> *>(ent);
            const int spec = P.spec[stage];
            for (int t = next_item(); t < P.tiles; t = next_item()) {
                const int2 d = P.tile_desc[t];
                if (d.x < 0 || d.x >= P.nmembers) {
                    if (threadIdx.x == 0) persist_flag(P.bar, 1u, (unsigned)t);
                    continue;
                }
                if (threadIdx.x == 0) {
                    origin[0] = (d.y & 0xffff) * kTile;
                    origin[1] = (d.y >> 16) * kTile;
                }
                load_args(As, sa + d.x);
                __syncthreads();
                if ((d.y & 0xffff) * kTile >= As.geo.nx || (d.y >> 16) * kTile >= As.geo.ny) {
                    if (threadIdx.x == 0) persist_flag(P.bar, 2u, (unsigned)t);
                    continue;
                }
                if (spec == 1)
                    persist_tile<real, 1>(As, origin, smem_raw);
                else if (spec == 2)
                    persist_tile<real, 2>(As, origin, smem_raw);
                else
                    persist_tile<real, 0>(As, origin, smem_raw);
            }
            if (!end_phase()) return;
            const LineArgs<real> *la = reinterpret_cast<const LineArgs<real> *>(ent + P.sarg_bytes);
            for (int p = next_item(); p < P.run_pass0[P.nruns]; p = next_item()) {
                int r = 0;
                while (P.run_pass0[r + 1] <= p) r++;
                const int q = p - P.run_pass0[r];
                {
                    // G lines of T threads side by side; threads past G T only pass the barriers
                    const int T = P.run_threads[r], G = kStencilThreads / T, nl = P.run_lines[r];
                    const int slot = threadIdx.x / T, tid = threadIdx.x - slot * T;
                    const int line_q = q * G + slot;
                    const bool valid = slot < G && line_q < nl;
                    const int own = valid ? slot : 0;   // a spare slot takes slot 0's arguments
                    bool bad = false;
                    if (slot < G) {
                        const int2 d = P.run_desc[r][valid ? line_q : q * G];
                        bad = d.x < 0 || d.x >= P.run_nfam[r];
                        if (bad && tid == 0) persist_flag(P.bar, 4u, (unsigned)(r * 65536 + q));
                        if ((valid || slot == 0) && !bad) {
                            const int nw = (int)(sizeof(LineArgs<real>) / sizeof(int));
                            int *dst = reinterpret_cast<int *>(&Al[slot]);
                            const int *src = reinterpret_cast<const int *>(la + P.run_first[r] + d.x);
                            for (int k = tid; k < nw; k += T) dst[k] = src[k];
                        }
                    }
                    if (__syncthreads_or(bad)) continue;   // skip the pass (the block's decision)
                    // the run's segment length picks the instance, the same
                    // for every slot, and the run's lines are all of one
                    // model: the solve's barriers are the block's, and the
                    // shallow-water model takes none
                    const int2 d = P.run_desc[r][valid ? line_q : q * G];
                    const bool bad2 = slot < G && (d.y < 0 || d.y >= Al[own].nlines || Al[own].nseg > T ||
                                                   (Al[own].nseg & 31) != 0 || Al[own].mshift != P.run_mshift[r] ||
                                                   Al[own].identity != P.run_identity[r]);
                    if (bad2 && tid == 0) persist_flag(P.bar, 5u, (unsigned)(r * 65536 + q));
                    if (__syncthreads_or(bad2)) continue;
                    const int wb = slot * (T >> 5);
                    if (P.run_mshift[r] == 3)
                        persist_line<real, 8>(Al[own], d.y, L, tid, wb, valid);
                    else if (P.run_mshift[r] == 2)
                        persist_line<real, 4>(Al[own], d.y, L, tid, wb, valid);
                    else
                        persist_line<real, 2>(Al[own], d.y, L, tid, wb, valid);
                }
            }
            if (!end_phase()) return;
        }
    }
}

}  // namespace

// ----------------------------------------------------------------- launchers

static dim3 grid2(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

namespace {
std::atomic<int> g_dependent_launch{1};
}  // namespace

void set_dependent_launch(int on) { g_dependent_launch.store(on ? 1 : 0); }
int dependent_launch() { return g_dependent_launch.load(); }

template <typename real>
cudaError_t launch_corners(const Geo &g, const real *z, real *Bc, cudaStream_t st)
{
    dim3 b(32, 8);
    k_corners<real><<<grid2(g.nx + 3, g.ny + 3, b), b, 0, st>>>(g, z, Bc);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_static_cells(const Geo &g, const Phys &p, const real *Bc, real *d_r, real *d_c,
                                cudaStream_t st)
{
    dim3 b(32, 8);
    k_static_cells<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, p, Bc, d_r, d_c);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_set_state(const Geo &g, const Phys &p, const real *Bc, const real *w_in,
                             const real *P_in, const real *Q_in, real *w, real *P, real *Qc, int rest,
                             cudaStream_t st)
{
    dim3 b(32, 8);
    k_set_state<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, p, Bc, w_in, P_in, Q_in, w, P, Qc, rest);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_clamp_state(const Geo &g, const Phys &p, const real *Bc, real *w, real *P, real *Qc,
                               cudaStream_t st)
{
    dim3 b(32, 8);
    k_clamp_state<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, p, Bc, w, P, Qc);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_clamp_adjoint(const Geo &g, const real *Bc, const real *w_in, real *grad, cudaStream_t st)
{
    dim3 b(32, 8);
    k_clamp_adjoint<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, Bc, w_in, grad);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_state(const Geo &g, const real *w, const real *P, const real *Qc, real *w_out,
                             real *P_out, real *Q_out, cudaStream_t st)
{
    dim3 b(32, 8);
    cudaError_t e = launch_step_kernel(k_get_state<real>, grid2(g.nx, g.ny, b), b, 0, st, g, w, P, Qc, w_out, P_out,
                                       Q_out);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename real>
cudaError_t launch_get_field(const Geo &g, const Phys &p, int which, const real *Bc, const real *d_r,
                             const real *U, const real *Vc, real *out, cudaStream_t st)
{
    dim3 b(32, 8);
    k_get_field<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, p, which, Bc, d_r, U, Vc, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_runup(const Geo &g, const real *Bc, const real *w, real *maxw, double delta, int start,
                         cudaStream_t st)
{
    dim3 b(32, 8);
    k_runup<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, Bc, w, maxw, real(delta), start);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_add_solitary(const Geo &g, const Phys &p, const real *Bc, real *w, real *P, real *Qc,
                                double H, double ct, double st_, double x0, double y0, double ks,
                                double cs, cudaStream_t st)
{
    dim3 b(32, 8);
    k_add_solitary<real><<<grid2(g.nx, g.ny, b), b, 0, st>>>(g, p, Bc, w, P, Qc, H, ct, st_, x0, y0, ks, cs);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_gauges(const Geo &g, const Phys &p, const real *w, const int32_t *ij, int n, real *slot,
                          cudaStream_t st)
{
    cudaError_t e = launch_step_kernel(k_gauges<real>, dim3((n + 127) / 128), dim3(128), 0, st, g, p, w, ij, n, slot);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename real>
cudaError_t launch_stats(const Geo &g, const Phys &p, const real *Bc, const real *w, const real *P, const real *Qc,
                         real eps, unsigned long long *out, cudaStream_t st)
{
    k_stats<real><<<304, 256, 0, st>>>(g, p, Bc, w, P, Qc, eps, out);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_check_finite(const Geo &g, const real *w, const real *P, const real *Qc,
                                unsigned long long *first_bad, cudaStream_t st)
{
    k_check_finite<real><<<304, 256, 0, st>>>(g, w, P, Qc, first_bad);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_eckart_table(const Geo &g, const Phys &p, const Bnd &b, const real *d_r, double *ktab, int npos,
                                cudaStream_t st)
{
    k_eckart_table<real><<<dim3((npos + 127) / 128, 4), 128, 0, st>>>(g, p, b, d_r, ktab, npos);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_sponge_table(const Coef<real> &c, real *gam, cudaStream_t st)
{
    k_sponge_table<real><<<dim3((c.npos + 127) / 128, 4), 128, 0, st>>>(c, gam);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_ghost_table(const Geo &g, const Phys &p, const Bnd &b, const real *d_r, const double *ktab,
                               double t0, double t1, real *tab, int npos, cudaStream_t st)
{
    cudaError_t e = launch_step_kernel(k_ghost_table<real>, dim3((npos + 127) / 128, 16), dim3(128), 0, st, g, p, b,
                                       d_r, ktab, t0, t1, tab, npos);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_stencil(const StencilArgs<real> &a, cudaStream_t st)
{
    static bool configured[3] = {false, false, false};
    const size_t smem = sizeof(StencilSmem<real>);
    const int spec = stencil_spec(a);
    auto *kern = spec == 1 ? k_stencil<real, 1> : spec == 2 ? k_stencil<real, 2> : k_stencil<real, 0>;
    if (!configured[spec]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[spec] = true;
    }
    dim3 grid((a.geo.nx + kTile - 1) / kTile, (a.geo.ny + kTile - 1) / kTile);
    cudaError_t e = launch_step_kernel(kern, grid, dim3(kStencilThreads), smem, st, a);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// The ensemble's batched launches are plain launches: replayed as captured
// graphs, programmatic dependent launch made the ensemble's step 3 % slower.
template <typename real>
cudaError_t launch_ghost_batch(const GhostArgs<real> *args, const int *start, int n, int nblocks, int64_t k,
                               const int64_t *kdev, cudaStream_t st)
{
    if (nblocks > 0) k_ghost_batch<real><<<nblocks, 128, 0, st>>>(args, start, n, k, kdev);
    return cudaGetLastError();
}

namespace {
__global__ void k_counter(int64_t *p, int64_t v, int add) { *p = add ? *p + v : v; }
}  // namespace

cudaError_t launch_counter(int64_t *p, int64_t v, int add, cudaStream_t st)
{
    k_counter<<<1, 1, 0, st>>>(p, v, add);
    return cudaGetLastError();
}

template <typename real>
cudaError_t launch_stencil_batch(const StencilArgs<real> *args, const int2 *desc, int nblocks, int spec,
                                 cudaStream_t st)
{
    static bool configured[3] = {false, false, false};
    if (spec < 0 || spec > 2) return cudaErrorInvalidValue;
    const size_t smem = sizeof(StencilSmem<real>);
    auto *kern = spec == 1 ? k_stencil_batch<real, 1> : spec == 2 ? k_stencil_batch<real, 2> : k_stencil_batch<real, 0>;
    if (!configured[spec]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[spec] = true;
    }
    if (nblocks > 0) kern<<<nblocks, kStencilThreads, smem, st>>>(args, desc);
    return cudaGetLastError();
}

namespace {

// The shared-memory solver's segments: 8 rows up to 1024 rows, 16 up to
// 4096, 32 above (at most 512 segments, and two 8192-row FP32 lines fit one
// SM's shared memory); fewer for short lines so that there are at least 2
// segments of >= 2 rows
int seg_shift(int n)
{
    int sh = n > 4096 ? 5 : (n > 1024 ? 4 : 3);
    while (sh > 1 && (n >> sh) < 2) sh--;
    return sh;
}

template <typename real>
size_t seg_smem_bytes(int n, int nseg)
{
    const int m = 1 << seg_shift(n);
    return sizeof(real) * ((size_t)3 * m * (nseg | 1) + (size_t)8 * nseg) + sizeof(uint32_t) * (size_t)((n + 31) / 32);
}

}  // namespace

// Rows per thread of the register path, per class of line lengths and per
// precision, as set by cel_set_line_split (an autotuner's choices); a class
// covers the lengths above the previous class's bound up to its own.
namespace {
struct SplitTable {
    std::mutex mu;
    std::vector<std::pair<int, int>> cls[2];   // (largest rows, rows per thread), ascending
    int generation = 0;
};
SplitTable &split_table()
{
    static SplitTable t;
    return t;
}
int max_line_threads(int real_bytes) { return real_bytes == 4 ? 1024 : 512; }
}  // namespace

int line_split_set(int real_bytes, int max_rows, int rows_per_thread)
{
    if ((real_bytes != 4 && real_bytes != 8) || max_rows < 2) return -1;
    if (rows_per_thread != 0 && rows_per_thread != 2 && rows_per_thread != 4 && rows_per_thread != 8) return -1;
    SplitTable &t = split_table();
    std::lock_guard<std::mutex> lock(t.mu);
    auto &v = t.cls[real_bytes == 8];
    for (size_t k = 0; k < v.size(); k++)
        if (v[k].first == max_rows) {
            v.erase(v.begin() + k);
            break;
        }
    if (rows_per_thread != 0) {
        v.push_back(std::make_pair(max_rows, rows_per_thread));
        std::sort(v.begin(), v.end());
    }
    t.generation++;
    return 0;
}

void line_split_reset()
{
    SplitTable &t = split_table();
    std::lock_guard<std::mutex> lock(t.mu);
    t.cls[0].clear();
    t.cls[1].clear();
    t.generation++;
}

int line_split_generation()
{
    SplitTable &t = split_table();
    std::lock_guard<std::mutex> lock(t.mu);
    return t.generation;
}

LineCfg line_config(int n, int real_bytes)
{
    LineCfg c;
    if (real_bytes == 4 ? n <= 8192 : n <= 4096) {
        // one segment per thread in registers: 8 rows (2 or 4 on lines of at
        // most 64 or 128 rows, which one warp then holds), a multiple of 32
        // threads, at most 1024 (FP32) or 512 (FP64); a class set by
        // cel_set_line_split overrides the rows where its block fits
        c.algo = 0;
        c.mshift = n <= 64 ? 1 : (n <= 128 ? 2 : 3);
        {
            SplitTable &t = split_table();
            std::lock_guard<std::mutex> lock(t.mu);
            for (const auto &e : t.cls[real_bytes == 8])
                if (n <= e.first) {
                    const int m = e.second, tt = round_up((n + m - 1) / m, 32);
                    if (tt <= max_line_threads(real_bytes)) c.mshift = m == 2 ? 1 : (m == 4 ? 2 : 3);
                    break;
                }
        }
        const int m = 1 << c.mshift;
        c.nseg = round_up((n + m - 1) / m, 32);
        c.threads = c.nseg;
        c.sp = 0;
        c.smem = 0;
        return c;
    }
    // segments in shared memory: a thread per segment, and at most 8
    // elements of P^n per thread held through the solve (16 with 32-row
    // segments, so that the longest lines stay within 1024 threads)
    c.algo = 1;
    c.mshift = seg_shift(n);
    const int m = 1 << c.mshift;
    c.nseg = (n + m - 1) / m;
    c.sp = c.nseg | 1;
    const int own = m == 32 ? 16 : (m < 8 ? m : 8);
    int t = c.nseg;
    if ((n + own - 1) / own > t) t = (n + own - 1) / own;
    t = round_up(t, 32);
    c.threads = t < 32 ? 32 : t;
    c.smem = real_bytes == 4 ? seg_smem_bytes<float>(n, c.nseg) : seg_smem_bytes<double>(n, c.nseg);
    return c;
}

template <typename real>
cudaError_t launch_lines_impl(const LinePair<real> &p, cudaStream_t st, int mode);

template <typename real>
cudaError_t launch_lines(const LinePair<real> &p, cudaStream_t st)
{
    return launch_lines_impl(p, st, 0);
}

template <typename real>
cudaError_t launch_lines_transposed(const LinePair<real> &p, cudaStream_t st)
{
    return launch_lines_impl(p, st, 1);
}

template <typename real>
cudaError_t launch_lines_solution(const LinePair<real> &p, cudaStream_t st)
{
    return launch_lines_impl(p, st, 2);
}

template <typename real, int kMode>
auto seg_kernel(int sh)
{
    return sh == 1 ? k_lines_seg<real, 2, kMode> : sh == 2 ? k_lines_seg<real, 4, kMode>
         : sh == 3 ? k_lines_seg<real, 8, kMode> : sh == 4 ? k_lines_seg<real, 16, kMode>
                   : k_lines_seg<real, 32, kMode>;
}

int line_launches(int nx_lines, int n_x, int ny_lines, int n_y, int real_bytes)
{
    if (nx_lines <= 0 || ny_lines <= 0) return nx_lines > 0 || ny_lines > 0 ? 1 : 0;
    const LineCfg a = line_config(n_x, real_bytes), b = line_config(n_y, real_bytes);
    if (a.algo != b.algo) return 2;
    return a.algo == 1 && (a.mshift != b.mshift || a.threads != b.threads) ? 2 : 1;
}

template <typename real>
cudaError_t launch_lines_impl(const LinePair<real> &p, cudaStream_t st, int mode)
{
    if (mode < 0 || mode > 2) return cudaErrorInvalidValue;
    LineCfg cf[2];
    for (int f = 0; f < 2; f++) {
        const LineArgs<real> &a = p.L[f];
        if (a.nlines <= 0) continue;
        cf[f] = line_config(a.n, (int)sizeof(real));
        if (a.algo != cf[f].algo || a.mshift != cf[f].mshift || a.nseg != cf[f].nseg ||
            (a.algo == 1 && a.sp != cf[f].sp))
            return cudaErrorInvalidValue;
    }
    const bool both = p.L[0].nlines > 0 && p.L[1].nlines > 0;
    // register-path families share a launch (each uses its own segment
    // length and count); shared-memory ones need one segment length
    if (both && (cf[0].algo != cf[1].algo ||
                 (cf[0].algo == 1 && (cf[0].mshift != cf[1].mshift || cf[0].threads != cf[1].threads)))) {
        LinePair<real> a = p, b = p;   // one configuration per launch
        a.L[1].nlines = 0;
        b.L[0].nlines = 0;
        cudaError_t e = launch_lines_impl<real>(a, st, mode);
        return e != cudaSuccess ? e : launch_lines_impl<real>(b, st, mode);
    }
    const int blocks = p.L[0].nlines + p.L[1].nlines;
    if (blocks <= 0) return cudaSuccess;
    const LineCfg &c = p.L[0].nlines > 0 ? cf[0] : cf[1];
    const int sh = c.mshift;
    if (c.algo == 0) {
        int threads = c.threads;
        if (both && cf[1].threads > threads) threads = cf[1].threads;
        const bool occ = sizeof(real) == 4 && threads <= 256;
        auto *kern = mode == 1 ? (occ ? k_lines<real, 1, 1> : k_lines<real, 1>)
                   : mode == 2 ? (occ ? k_lines<real, 2, 1> : k_lines<real, 2>)
                               : (occ ? k_lines<real, 0, 1> : k_lines<real, 0>);
        cudaError_t e = launch_step_kernel(kern, dim3(blocks), dim3(threads), 0, st, p);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    if (sh < 1 || sh > 5) return cudaErrorInvalidValue;
    size_t smem = c.smem;
    if (both && cf[1].smem > smem) smem = cf[1].smem;
    static int configured[3][6] = {{0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0}};
    auto *kern = mode == 1 ? seg_kernel<real, 1>(sh) : mode == 2 ? seg_kernel<real, 2>(sh) : seg_kernel<real, 0>(sh);
    if ((int)smem > configured[mode][sh]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[mode][sh] = (int)smem;
    }
    cudaError_t e = launch_step_kernel(kern, dim3(blocks), dim3(c.threads), smem, st, p);
    return e != cudaSuccess ? e : cudaGetLastError();
}

template <typename real>
cudaError_t launch_lines_batch(const LineArgs<real> *args, const int2 *desc, int nblocks, const LineCfg &cfg,
                               cudaStream_t st)
{
    const int sh = cfg.mshift, threads = cfg.threads;
    if (threads < 32 || threads % 32 || threads > (sizeof(real) == 4 ? 1024 : 512)) return cudaErrorInvalidValue;
    if (nblocks <= 0) return cudaSuccess;
    if (cfg.algo == 0) {
        if (sizeof(real) == 4 && threads <= 256)
            k_lines_batch<real, 1><<<nblocks, threads, 0, st>>>(args, desc);
        else
            k_lines_batch<real><<<nblocks, threads, 0, st>>>(args, desc);
        return cudaGetLastError();
    }
    static int configured[6] = {0, 0, 0, 0, 0, 0};
    if (sh < 1 || sh > 5) return cudaErrorInvalidValue;
    auto *kern = sh == 1 ? k_lines_batch_seg<real, 2> : sh == 2 ? k_lines_batch_seg<real, 4>
               : sh == 3 ? k_lines_batch_seg<real, 8> : sh == 4 ? k_lines_batch_seg<real, 16>
                         : k_lines_batch_seg<real, 32>;
    if ((int)cfg.smem > configured[sh]) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        if (e != cudaSuccess) return e;
        configured[sh] = (int)cfg.smem;
    }
    kern<<<nblocks, threads, cfg.smem, st>>>(args, desc);
    return cudaGetLastError();
}

template <typename real>
int persistent_grid()
{
    // per device (the SM count and the function attribute are the device's)
    constexpr int kDevices = 64;
    static std::atomic<int> grid[kDevices];
    static std::once_flag init;
    std::call_once(init, [] {
        for (auto &g : grid) g.store(-1);
    });
    const size_t smem = sizeof(StencilSmem<real>);
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) {
        cudaGetLastError();
        return 0;
    }
    const int known = grid[dev].load();
    if (known >= 0) return known;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaFuncSetAttribute(k_ensemble_persistent<real>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_ensemble_persistent<real>, kStencilThreads, smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    grid[dev].store(sms * per);
    return sms * per;
}

template <typename real>
cudaError_t launch_persistent(const PersistArgs<real> &p, int grid, cudaStream_t st)
{
    if (grid <= 0 || p.nstages > kPersistMaxStages || p.nruns > kPersistMaxRuns) return cudaErrorInvalidValue;
    const size_t smem = sizeof(StencilSmem<real>);
    void *params[] = {const_cast<PersistArgs<real> *>(&p)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(k_ensemble_persistent<real>), dim3(grid),
                                       dim3(kStencilThreads), params, smem, st);
}

#define CEL_INSTANTIATE(real)                                                                           \
    template cudaError_t launch_corners<real>(const Geo &, const real *, real *, cudaStream_t);           \
    template cudaError_t launch_static_cells<real>(const Geo &, const Phys &, const real *, real *,      \
                                                   real *, cudaStream_t);                               \
    template cudaError_t launch_set_state<real>(const Geo &, const Phys &, const real *, const real *,   \
                                                const real *, const real *, real *, real *, real *, int, \
                                                cudaStream_t);                                          \
    template cudaError_t launch_clamp_state<real>(const Geo &, const Phys &, const real *, real *, real *, \
                                                  real *, cudaStream_t);                                \
    template cudaError_t launch_clamp_adjoint<real>(const Geo &, const real *, const real *, real *,      \
                                                    cudaStream_t);                                      \
    template cudaError_t launch_get_state<real>(const Geo &, const real *, const real *, const real *,   \
                                                real *, real *, real *, cudaStream_t);                  \
    template cudaError_t launch_get_field<real>(const Geo &, const Phys &, int, const real *,            \
                                                const real *, const real *, const real *, real *,       \
                                                cudaStream_t);                                          \
    template cudaError_t launch_add_solitary<real>(const Geo &, const Phys &, const real *, real *,      \
                                                   real *, real *, double, double, double, double,      \
                                                   double, double, double, cudaStream_t);               \
    template cudaError_t launch_runup<real>(const Geo &, const real *, const real *, real *, double, int,   \
                                            cudaStream_t);                                              \
    template cudaError_t launch_gauges<real>(const Geo &, const Phys &, const real *, const int32_t *,   \
                                             int, real *, cudaStream_t);                                \
    template cudaError_t launch_stats<real>(const Geo &, const Phys &, const real *, const real *, const real *, \
                                            const real *, real, unsigned long long *, cudaStream_t);       \
    template cudaError_t launch_check_finite<real>(const Geo &, const real *, const real *, const real *, \
                                                   unsigned long long *, cudaStream_t);                 \
    template cudaError_t launch_eckart_table<real>(const Geo &, const Phys &, const Bnd &, const real *,  \
                                                   double *, int, cudaStream_t);                        \
    template cudaError_t launch_sponge_table<real>(const Coef<real> &, real *, cudaStream_t);            \
    template cudaError_t launch_ghost_table<real>(const Geo &, const Phys &, const Bnd &, const real *,   \
                                                  const double *, double, double, real *, int,          \
                                                  cudaStream_t);                                        \
    template cudaError_t launch_stencil<real>(const StencilArgs<real> &, cudaStream_t);                  \
    template cudaError_t launch_lines<real>(const LinePair<real> &, cudaStream_t);                       \
    template cudaError_t launch_lines_transposed<real>(const LinePair<real> &, cudaStream_t);            \
    template cudaError_t launch_lines_solution<real>(const LinePair<real> &, cudaStream_t);              \
    template cudaError_t launch_ghost_batch<real>(const GhostArgs<real> *, const int *, int, int, int64_t, \
                                                  const int64_t *, cudaStream_t);                                        \
    template cudaError_t launch_stencil_batch<real>(const StencilArgs<real> *, const int2 *, int, int, cudaStream_t); \
    template cudaError_t launch_lines_batch<real>(const LineArgs<real> *, const int2 *, int, const LineCfg &, \
                                                  cudaStream_t);                                          \
    template int persistent_grid<real>();                                                                  \
    template cudaError_t launch_persistent<real>(const PersistArgs<real> &, int, cudaStream_t);

CEL_INSTANTIATE(float)
CEL_INSTANTIATE(double)

}  // namespace cel
