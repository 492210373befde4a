// Internal declarations shared by the kernels and the C-ABI host code.
//
// Data layout in device memory (all arrays carved from the caller's workspace):
//   * x-family fields (w, P, dU*, and every per-cell history value) are
//     row-major [ny][px], px = nx rounded up to 32 elements, so an x-row is a
//     contiguous line (the x tridiagonal solves of Eq. 21 read whole rows);
//   * y-family fields (Q, dV*) are column-major [nx][py], py = ny rounded up
//     to 32, so a y-column is a contiguous line (the y solves of Eq. 22);
//   * the static bed is stored once, as corner values (nx+3) x (ny+3): corner
//     (ci, cj) at (ci dx, cj dy), ci in [-1, nx+1], at [(cj+1)*pc + ci+1];
//   * the still-water depth d is stored twice, row-major for the x solves and
//     column-major for the y solves (static, derived at create);
//   * dry-cell bit masks, one bit per cell, row-major words for the x solves
//     and column-major words for the y solves.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "celeris_gb.h"

namespace cel {

constexpr int kTile = 32;          // stencil tile edge (cells)
constexpr int kHalo = 2;           // ghost layers (Sec. 2.4)
constexpr int kTileIn = kTile + 2 * kHalo;   // 36
constexpr int kStride = kTileIn + 1;         // padded smem row of the state tile
constexpr int kCorner = kTile + 3;           // 35 corners per tile edge
constexpr int kCornerStride = kCorner + 2;    // odd: a warp reading one corner per row hits 32 banks
constexpr int kDcell = kTile + 2;            // 34 cells of d per tile edge
constexpr int kDStride = kDcell + 1;
constexpr int kStencilThreads = 256;

enum { kSolid = 0, kSponge = 1, kSine = 2 };
enum { kBsnq = 0, kNlsw = 1 };
enum { kFricNone = 0, kFricQuad = 1, kFricManning = 2 };
// Stage kinds of one step (Sec. 2.3).
enum { kEuler0 = 0, kEuler1 = 1, kAB3 = 2, kAM4 = 3 };

struct Side {
    int type;            // kSolid | kSponge | kSine
    int width;           // sponge width in cells
    int ncomp;
    double L;            // sponge width in metres
    double amp[8], omega[8], cdir[8], sdir[8], phase[8];
};

struct Geo {
    int nx, ny;
    int px, py, pc;      // pitches (elements): row-major, column-major, corners
    int nwx, nwy;        // mask words per row / per column
    double dx, dy;
};

struct Phys {
    int model, friction, K;
    double g, Bd, theta, eps, dt, ws, fcoef;
};

struct Bnd {
    Side s[4];           // west, east, south, north
};

// Real-typed constants of the step, computed once on the host so that the
// FP32 kernels do no double-precision arithmetic (GB300's FP64 rate is a
// small fraction of its FP32 rate).
template <typename real>
struct Coef {
    real g, eps, theta, ws, dt, Bd, B3, sixth;
    real rdx, rdy, hrdx, hrdy, rdx2, rdy2, rdxdy4, rdx3h, rdy3h, rdxdy2h, rdx2dyh;
    real fric;           // quadratic f, or g n^2 for Manning
    int spw[4];          // sponge width in cells per side (0: not a sponge)
    int sine;            // bit s set: side s is a sine maker
    int npos;            // positions per side in the ghost table
    const real *gam;     // Eq. 30 factor per side and position ([side][npos]), or null
};

template <typename real>
inline Coef<real> make_coef(const Geo &G, const Phys &p, const Bnd &b)
{
    Coef<real> c;
    c.g = real(p.g);
    c.eps = real(p.eps);
    c.theta = real(p.theta);
    c.ws = real(p.ws);
    c.dt = real(p.dt);
    c.Bd = real(p.Bd);
    c.B3 = real(p.Bd + 1.0 / 3.0);
    c.sixth = real(1.0 / 6.0);
    c.rdx = real(1.0 / G.dx);
    c.rdy = real(1.0 / G.dy);
    c.hrdx = real(0.5 / G.dx);
    c.hrdy = real(0.5 / G.dy);
    c.rdx2 = real(1.0 / (G.dx * G.dx));
    c.rdy2 = real(1.0 / (G.dy * G.dy));
    c.rdxdy4 = real(1.0 / (4.0 * G.dx * G.dy));
    c.rdx3h = real(1.0 / (2.0 * G.dx * G.dx * G.dx));
    c.rdy3h = real(1.0 / (2.0 * G.dy * G.dy * G.dy));
    c.rdxdy2h = real(1.0 / (2.0 * G.dx * G.dy * G.dy));
    c.rdx2dyh = real(1.0 / (2.0 * G.dx * G.dx * G.dy));
    c.fric = real(p.friction == kFricManning ? p.g * p.fcoef * p.fcoef : p.fcoef);
    c.sine = 0;
    for (int s = 0; s < 4; s++) {
        c.spw[s] = b.s[s].type == kSponge ? b.s[s].width : 0;
        if (b.s[s].type == kSine) c.sine |= 1 << s;
    }
    c.npos = (G.nx > G.ny ? G.nx : G.ny) + 4;
    c.gam = nullptr;
    return c;
}

// Ghost table of the sine-wave makers, one per step: [time t0|t1][side]
// [layer 0 (adjacent) | 1][w, P, Q][position along the side + 2].
__host__ __device__ inline size_t ghost_index(int time, int side, int layer, int var, int pos, int npos)
{
    return ((((size_t)time * 4 + side) * 2 + layer) * 3 + var) * (size_t)npos + pos;
}

// Reading A-W1: the cell bed Bbar is the mean of the cell's 4 corners; the
// corner array is (nx + 3) x (ny + 3) with corner (ci, cj) at [cj + 1][ci + 1].
template <typename real>
__device__ __forceinline__ real cell_bbar(real c00, real c10, real c01, real c11)
{
    return real(0.25) * (((c00 + c10) + c01) + c11);
}

template <typename real>
__device__ __forceinline__ real corner(const real *Bc, const Geo &g, int ci, int cj)
{
    return Bc[(size_t)(cj + 1) * g.pc + (ci + 1)];
}

template <typename real>
__device__ __forceinline__ real bbar_at(const real *Bc, const Geo &g, int i, int j)
{
    return cell_bbar(corner(Bc, g, i, j), corner(Bc, g, i + 1, j), corner(Bc, g, i, j + 1),
                     corner(Bc, g, i + 1, j + 1));
}

template <typename real>
struct StencilArgs {
    Geo geo;
    Phys phy;
    Coef<real> c;
    const real *ghost;                   // sine-maker ghost table of this step
    const real *Bc;
    const real *w_in, *P_in, *Qc_in;     // state (or AM4 iterate) at time t
    real *w_out, *U_out, *Vc_out;        // w^{n+1}, and the increments of U*, V*
    // K = 0: combined AB3 carries of (w, U, V), b = this step's slot
    real *a[3], *b[3];
    // K >= 1: rings of the right sides R (slots of R^n written, R^{n-1},
    // R^{n-2}), of the mixed terms F*, G* (U, V only) and the AM4 bases Y
    real *R0[3], *R1[3], *R2[3], *F0[3], *F1[3], *F2[3], *Y[3];
    uint32_t *mask_r, *mask_c;
    int kind;                            // kEuler0 | kEuler1 | kAB3 | kAM4
    int ring;                            // K >= 1: ring history (else carries)
    int final_stage;                     // last stage of the step: sponge on w
    int tsel;                            // ghost-table time: 0 = t^n, 1 = t^{n+1}
};

template <typename real>
struct LineArgs {
    Geo geo;
    Phys phy;
    Coef<real> c;
    const real *ghost;     // sine-maker ghost table of this step
    const real *rhs;       // increment of U* (x-lines) or V* (y-lines), line-major
    const real *d;         // still-water depth, line-major
    const uint32_t *mask;  // dry bits, line-major words
    const real *base;      // P^n or Q^n, line-major
    real *sol;             // P^{n+1} = P^n + solution, line-major
    real *xcap;            // or NULL: the step's solution itself as well (line-major), for the adjoint
    int dir;               // 0: x-lines (rows), 1: y-lines (columns)
    int n, nlines, pitch, nwords;
    int algo;              // 0: segments in registers, one per thread; 1: segments in shared memory
    int nseg;              // segments per line (algo 0: one per thread, the block size)
    int mshift;            // log2 of the rows per segment (lines padded to nseg << mshift)
    int sp;                // algo 1: odd shared-memory stride between rows of the segments
    int final_stage;       // apply the sponge
    int identity;          // NLSW model: no dispersive solve, P = U*, Q = V*
    real rh, rh2, hrh, srh; // 1/h, 1/h^2, 1/(2h), 1/(6h) along the line
};

// Headless rendering of the state (celeris_render.cu).
template <typename real>
struct RenderArgs {
    Geo geo;
    float dx, dy, ws;
    cel_render_params p;
    const real *w, *P, *Qc, *Bc;
    uchar4 *rgba;          // [ny][nx]
};

template <typename real>
cudaError_t launch_render(const RenderArgs<real> &a, cudaStream_t st);

// Launchers (celeris_kernels.cu).  All return cudaGetLastError().
template <typename real>
cudaError_t launch_corners(const Geo &g, const real *z, real *Bc, cudaStream_t st);
template <typename real>
cudaError_t launch_static_cells(const Geo &g, const Phys &p, const real *Bc, real *d_r,
                                real *d_c, cudaStream_t st);
template <typename real>
cudaError_t launch_set_state(const Geo &g, const Phys &p, const real *Bc, const real *w_in,
                             const real *P_in, const real *Q_in, real *w, real *P, real *Qc,
                             int rest, cudaStream_t st);
template <typename real>
cudaError_t launch_clamp_state(const Geo &g, const Phys &p, const real *Bc, real *w, real *P,
                               real *Qc, cudaStream_t st);
// dL/dw_in from dL/dw0 for w0 = max(w_in, Bbar): zero where clamped.
template <typename real>
cudaError_t launch_clamp_adjoint(const Geo &g, const real *Bc, const real *w_in, real *grad, cudaStream_t st);
template <typename real>
cudaError_t launch_get_state(const Geo &g, const real *w, const real *P, const real *Qc,
                             real *w_out, real *P_out, real *Q_out, cudaStream_t st);
template <typename real>
cudaError_t launch_get_field(const Geo &g, const Phys &p, int which, const real *Bc,
                             const real *d_r, const real *U, const real *Vc, real *out,
                             cudaStream_t st);
template <typename real>
cudaError_t launch_add_solitary(const Geo &g, const Phys &p, const real *Bc, real *w, real *P,
                                real *Qc, double H, double ct, double st_, double x0,
                                double y0, double ks, double cs, cudaStream_t st);
template <typename real>
cudaError_t launch_runup(const Geo &g, const real *Bc, const real *w, real *maxw, double delta, int start,
                         cudaStream_t st);
template <typename real>
cudaError_t launch_gauges(const Geo &g, const Phys &p, const real *w, const int32_t *ij,
                          int n, real *slot, cudaStream_t st);
// Sum of depths, largest speed (as bits), wet-cell count into out[0..2]
// (zeroed by the caller).
template <typename real>
cudaError_t launch_stats(const Geo &g, const Phys &p, const real *Bc, const real *w, const real *P, const real *Qc,
                         real eps, unsigned long long *out, cudaStream_t st);
template <typename real>
cudaError_t launch_check_finite(const Geo &g, const real *w, const real *P, const real *Qc,
                                unsigned long long *first_bad, cudaStream_t st);
template <typename real>
cudaError_t launch_eckart_table(const Geo &g, const Phys &p, const Bnd &b, const real *d_r, double *ktab,
                                int npos, cudaStream_t st);
template <typename real>
cudaError_t launch_sponge_table(const Coef<real> &c, real *gam, cudaStream_t st);
template <typename real>
cudaError_t launch_ghost_table(const Geo &g, const Phys &p, const Bnd &b, const real *d_r,
                               const double *ktab, double t0, double t1, real *tab, int npos,
                               cudaStream_t st);
template <typename real>
cudaError_t launch_stencil(const StencilArgs<real> &a, cudaStream_t st);
// The stencil kernel's stage specialisation: 1 for the AB3 predictor with
// the ring history, 2 for the AM4 corrector, 0 for the other stages.
template <typename real>
inline int stencil_spec(const StencilArgs<real> &a)
{
    return a.kind == kAM4 ? 2 : (a.ring && a.kind == kAB3 ? 1 : 0);
}
// How a line of n rows is solved: the algorithm, rows per segment, segments,
// the odd shared-memory stride (algo 1), threads per block and dynamic
// shared memory.  Lines of one launch share algo, mshift and threads.
struct LineCfg {
    int algo, mshift, nseg, sp, threads;
    size_t smem;
};
LineCfg line_config(int n, int real_bytes);
// The register path's rows per thread per class of line lengths (0: the
// built-in rule); the generation counts changes (ensembles plan with it).
int line_split_set(int real_bytes, int max_rows, int rows_per_thread);
void line_split_reset();
int line_split_generation();
// Programmatic dependent launch of the step kernels (process-wide, on by default).
void set_dependent_launch(int on);
int dependent_launch();

// A kernel launched with programmatic stream serialisation may start while
// the kernel before it on the stream drains its last blocks.  Each such
// kernel first waits for that kernel to complete (its writes visible),
// before any access to memory, then lets the kernel after it launch: the
// kernels overlap only in their launch and block scheduling, never in their
// memory accesses.  Without the launch attribute the wait returns at once.
__device__ __forceinline__ void dependent_launch_wait_then_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// A step kernel's launch, with programmatic stream serialisation where it is
// switched on (the kernel's own wait keeps its memory accesses after the
// previous kernel's).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_step_kernel(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent_launch() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
// Launches that launch_lines and its kin issue for the two families.
int line_launches(int nx_lines, int n_x, int ny_lines, int n_y, int real_bytes);

// The x-line and the y-line solves of one stage are independent (P from
// the increment of U*, Q from that of V*) and run in one launch.
template <typename real>
struct LinePair {
    LineArgs<real> L[2];
};

template <typename real>
cudaError_t launch_lines(const LinePair<real> &a, cudaStream_t st);
// The transposed systems T^T y = rhs of the same lines (the adjoint): y goes
// to sol; base, mask and the sponge are not used.
template <typename real>
cudaError_t launch_lines_transposed(const LinePair<real> &a, cudaStream_t st);
// The step's systems T x = rhs, x alone to sol (no base, sponge or mask).
template <typename real>
cudaError_t launch_lines_solution(const LinePair<real> &a, cudaStream_t st);

// Ensembles: one launch covers every member.  The argument blocks live in
// device memory, one per member (stencil, ghost table) or per line family.
// Ghost tables: start[e] is the first block of entry e (ascending, start[0]
// = 0).  Stencil and lines: desc[b] = (argument block, tile or line) of
// block b, the tile as row << 16 | column.
template <typename real>
struct GhostArgs {
    Geo g;
    Phys p;
    Bnd b;
    const real *d_r;
    const double *ktab;
    real *tab;
    int npos;
    int64_t step0;         // the member's step when the launch's k is 0
    double dt;
};

// The persistent ensemble launch: one cooperative launch runs nsteps steps
// of every member, its phases (ghost tables, then per stage the stencil
// tiles and the line solves) separated by grid-wide barriers.  The argument
// entries of the 6-step cycle are the ones the batched launches use.  Line
// solves run in runs of one block size and one segment length each, as many
// lines side by side per block as fit 256 threads.
constexpr int kPersistMaxStages = 4, kPersistMaxRuns = 48;

template <typename real>
struct PersistArgs {
    const unsigned char *entries;      // argument entries (stencil arguments, then line arguments)
    size_t entry_bytes, sarg_bytes;
    int ent[6][kPersistMaxStages];     // entry per step of the cycle and stage
    int spec[kPersistMaxStages];       // stencil instance per stage (stencil_spec)
    int nstages, phase0, nsteps;
    const int2 *tile_desc;             // as for the batched stencil launch
    int tiles;
    int nruns;
    const int2 *run_desc[kPersistMaxRuns];   // (family, line) per line, as for the batched line launch
    int run_first[kPersistMaxRuns];    // the run's first family in the entry's line arguments
    int run_lines[kPersistMaxRuns], run_threads[kPersistMaxRuns];
    int run_mshift[kPersistMaxRuns];   // log2 rows per segment of every line of the run
    int run_identity[kPersistMaxRuns]; // 1: the run's lines are shallow-water ones (P = U*, no solve)
    int run_nfam[kPersistMaxRuns];     // families of the run's group (descriptor x below it)
    int run_pass0[kPersistMaxRuns + 1];   // first pass of each run in the phase's pass order (prefix sums)
    int nmembers, nent;                // members; argument entries in the table
    const GhostArgs<real> *gargs;      // as for the batched ghost launch
    const int *gstart;
    int ngm, gblocks;
    int64_t k0;                        // lockstep step index of the first step
    unsigned *bar;                     // barrier words: arrivals, generation, status, check (0 at launch)
    int *work;                         // three work counters, used by the phases in turn (0 at launch)
    unsigned expect;                   // arrivals a barrier waits for: the grid size
    long long timeout_ns;              // bound of every wait
    int barrier_only;                  // 1: one barrier and nothing else (a check of the waits' bound)
};

// k: the lockstep step index, plus *kdev where kdev is given (a device
// counter that a captured graph advances between its replays).
template <typename real>
cudaError_t launch_ghost_batch(const GhostArgs<real> *args, const int *start, int n, int nblocks, int64_t k,
                               const int64_t *kdev, cudaStream_t st);
// *p = v (add 0) or *p += v (add 1), one thread.
cudaError_t launch_counter(int64_t *p, int64_t v, int add, cudaStream_t st);
// spec: the stencil's stage specialisation (stencil_spec of the members'
// arguments, which step in lockstep and share it).
template <typename real>
cudaError_t launch_persistent(const PersistArgs<real> &p, int grid, cudaStream_t st);
// Blocks of the persistent launch that fit the GPU at once (0 on an error).
template <typename real>
int persistent_grid();
template <typename real>
cudaError_t launch_stencil_batch(const StencilArgs<real> *args, const int2 *desc, int nblocks, int spec,
                                 cudaStream_t st);
// All families of one launch share cfg (line_config of their length): the
// algorithm, the segment length 1 << mshift and the block size.
template <typename real>
cudaError_t launch_lines_batch(const LineArgs<real> *args, const int2 *desc, int nblocks, const LineCfg &cfg,
                               cudaStream_t st);

}  // namespace cel
