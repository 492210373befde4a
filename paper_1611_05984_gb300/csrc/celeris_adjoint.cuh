// Discrete adjoint (celeris_adjoint.cu, driven from celeris_api.cu): the
// argument block of one stage's reverse and the launchers of its phases.
#pragma once
#include "celeris_internal.cuh"

namespace cel {

// Discrete adjoint of one stage (celeris_adjoint.cu).  State
// arrays are dense [ny][nx]: w, P, Q the state before the step, w_next w
// after it; lw, lP, lQ the adjoint (in: of the state after the step, out: of
// the state before it); G0, G1, G2 the adjoint of this step's right sides
// and of the two before it, per component E, F, G, F*, G*; ldU, ldV the
// adjoint of the U* and V* increments (the line solves' right sides) in the
// dense layout, where the history phase reads them (see muX, muY).
template <typename real>
struct AdjArgs {
    Geo geo;
    Phys phy;
    Coef<real> c;
    const real *Bc, *ghost;
    const real *w, *P, *Q, *w_next;
    real *lw, *lP, *lQ;
    real *G0[5], *G1[5], *G2[5];
    const real *ldU, *ldV;
    // the bed's adjoints, or NULL: lBc at the corners (Bc's layout), lBb of
    // the cell bed Bbar and ld of the still-water depth d on the cells with
    // a one-cell ring ([ny + 2][nx + 2], cell (i, j) at [j + 1][i + 1])
    real *lBc, *lBb, *ld;
    real *ldx, *ldy;       // the line systems' part of ld, in the line layouts (Boussinesq)
    real *lg;              // adjoint of the sine makers' ghost values (the ghost table's layout), or NULL
    real c0, c1, c2;       // weights of R^n, R^{n-1}, R^{n-2} in this step's update
    real e0, e1, e2;       // weights of F*^n, F*^{n-1}, F*^{n-2} (Boussinesq)
    // optional parts of the history phase: the U*, V* adjoints read from
    // the transposed solves' line layouts (muX [ny][px], muY [nx][py])
    // instead of ldU, ldV; a second right side H = (hc E, F, G; he F*, G*)
    // weights written (not added) to H0; the masked adjoint added to acc
    const real *muX, *muY;
    // optional parts of the mask phase: the masked lP, lQ also written to
    // the line layouts packX [ny][px], packY [nx][py] (the transposed solves'
    // right sides); three dense fields zero[0..2] cleared
    real *packX, *packY, *zero[3];
    real *H0[5];
    real hc, he;
    real *accw, *accP, *accQ;
    int bsnq;
    int final_stage;       // the masks include the sponge
    int tsel;              // sine-maker ghosts at t^n (0, predictor) or t^{n+1} (1, corrector)
};

// The phases of one stage's reverse: masks, the transposed solves (through
// launch_lines_transposed), history, the right sides' Jacobians transposed.
// G1 and G2 may be NULL in the history phase.
template <typename real>
cudaError_t launch_adjoint_mask(const AdjArgs<real> &a, cudaStream_t st);
template <typename real>
cudaError_t launch_adjoint_hist(const AdjArgs<real> &a, cudaStream_t st);
template <typename real>
cudaError_t launch_adjoint_vjp(const AdjArgs<real> &a, cudaStream_t st);
// The line systems' dependence on d (Eq. 23): with x the stage's solutions
// and mu the transposed solves' solutions (line layouts: x-rows [ny][px],
// y-columns [nx][py]) and dr, dc the depths in the same layouts,
// dL/dT_kl = -mu_k x_l is added to ldx, ldy.
template <typename real>
cudaError_t launch_adjoint_tri_bed(const AdjArgs<real> &a, const real *X, const real *Yc, const real *MUx,
                                   const real *MUy, const real *dr, const real *dc, cudaStream_t st);
// The sine makers' ghost values depend on the adjacent depth through the
// Eckart wave number (Eq. 25-29): lg (this step's ghost adjoints, t0 = t^n,
// t1 = t^{n+1}) into ld, then lg zeroed.
template <typename real>
cudaError_t launch_adjoint_ghost_bed(const AdjArgs<real> &a, const Bnd &b, const double *ktab, const real *d_r,
                                     double t0, double t1, cudaStream_t st);
// The end of the reverse: ld and the clamp of the initial state (cells with
// w0 <= Bbar follow the bed, weight lw0) into lBb, lBb into lBc, and lBc
// into the cell-centre bed z as dL/dz (grad_z zeroed here).
template <typename real>
cudaError_t launch_adjoint_bed_final(const AdjArgs<real> &a, const real *w0, const real *lw0, real *grad_z,
                                     cudaStream_t st);
// Self-check of the face flux's hand-written VJP against dual numbers
// (inputs [n][22], outputs [n][30]; see cel_adjoint_face_selfcheck).
template <typename real>
cudaError_t launch_face_vjp_check(const real *in, int n, real *out, cudaStream_t st);
template <typename real>
cudaError_t launch_adjoint_misfit(const AdjArgs<real> &a, const int32_t *gij, int ng, const real *rec,
                                  const real *obs, cudaStream_t st);

}  // namespace cel
