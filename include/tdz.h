/*
 * tdz.h - C ABI of the B300 Crank-Nicolson propagator for the B-spline Galerkin
 * time-dependent Schrodinger equation with a BenDaniel-Duke (position-dependent
 * mass) kinetic operator, after TDSE-Z (arXiv 2608.18472).
 *
 * Conventions shared by every entry point
 *   - Status: every function returns int; TDZ_OK (0) on success, a negative
 *     TDZ_E* code otherwise. No call aborts or exits the process.
 *   - Ownership: the caller owns every array it passes; the library copies
 *     what it keeps. Opaque handles are library-owned and freed by their
 *     *_destroy function (NULL is accepted and ignored).
 *   - Complex vectors are interleaved (re, im) doubles: element j at [2j], [2j+1].
 *   - Coefficient order: B-spline index with the two Dirichlet end functions
 *     removed (Sec. "Weak form"): DoF j <-> B-spline j+1. In 2-D/3-D the linear
 *     index is x fastest: I = i_x + n_x (i_y + n_y i_z).
 *   - Pointers documented "host or device" may be either; the library tells
 *     them apart with cudaPointerGetAttributes.
 *   - Units are atomic units throughout.
 */
#ifndef TDZ_H
#define TDZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define TDZ_OK            0
#define TDZ_EINVAL       -1   /* bad argument: null pointer, size, range, knot vector */
#define TDZ_ENOMEM       -2   /* host or device allocation failed                      */
#define TDZ_ECUDA        -3   /* a CUDA runtime call failed (message: tdz_last_error)  */
#define TDZ_ENOCONV      -4   /* an iteration reached its cap before its tolerance     */
#define TDZ_ENONFINITE   -5   /* a NaN/Inf appeared in the state or the field          */
#define TDZ_EUNSUPPORTED -6   /* valid request outside what this build implements      */

/* Human-readable description of the last error raised on the calling thread. */
const char* tdz_last_error(void);

/* ------------------------------------------------------------------ precision */
#define TDZ_FP64   0  /* binary64 everywhere: factors, solves, residuals, state              */
#define TDZ_MIXED  1  /* FP32 factors and solves; residual, correction, state and observable
                         products in double-float (hi+lo FP32 pair, 48-bit significand);
                         reductions accumulated in binary64                                   */

/* ------------------------------------------------------------------ basis
 * tdz_basis_create: B-spline basis of degree `degree` on an open knot vector
 * (Sec. "Weak form": ends repeated degree+1 times; Eq. tensor3d gives the
 * tensor product of such 1-D bases), with an `nquad`-point Gauss-Legendre
 * rule on every non-empty knot span (Sec. "Parallel assembly").
 *   knots  : host, nknots non-decreasing values, first and last repeated
 *            degree+1 times, at least one non-empty span.
 *   degree : 1..8.   nquad: 1..16.
 * Errors: TDZ_EINVAL for a malformed knot vector or out-of-range sizes.
 */
typedef struct tdz_basis tdz_basis;
int  tdz_basis_create(const double* knots, int64_t nknots, int degree, int nquad, tdz_basis** out);
/* nfun = number of B-splines (Dirichlet ends included), nelem = non-empty spans. */
int  tdz_basis_info(const tdz_basis* b, int64_t* nfun, int64_t* nelem, int* degree, int* nquad);
/* Values and first derivatives of all nfun B-splines at npts host points,
 * written to host arrays val[nfun*npts], der[nfun*npts] (function-major). */
int  tdz_basis_eval(const tdz_basis* b, const double* x, int64_t npts, double* val, double* der);
void tdz_basis_destroy(tdz_basis* b);

/* ------------------------------------------------------------------ medium */
#define TDZ_MASS_CONST    0  /* m(r) = mass_par[0]                                              */
#define TDZ_MASS_QUESNE   1  /* m(x) = (1 + x/a)^-1, a = mass_par[0] (Eq. mass)                  */
#define TDZ_MASS_LAYERS   2  /* 1-D piecewise constant: layer_mass[r] on [bounds[r], bounds[r+1]) */
#define TDZ_MASS_ELLIPSE  3  /* 2-D dot: m_in inside x^2/a^2+y^2/b^2<1, m_out outside;
                                mass_par = {a, b, m_in, m_out}                                  */
#define TDZ_POT_ZERO      0
#define TDZ_POT_SOFTCORE  1  /* V = -z / sqrt(|r|^2 + eps), pot_par = {z, eps}                   */
#define TDZ_POT_HO        2  /* V = 1/2 sum_a w_a^2 x_a^2, pot_par = {w_x, w_y, w_z}              */
#define TDZ_POT_QUESNE    3  /* V = a w^2 x^2 / (8 (x + a)) (Eq. rescaling), pot_par = {a, w}      */
#define TDZ_POT_LAYERS    4  /* 1-D piecewise constant layer_pot[r]                               */
#define TDZ_POT_ELLIPSE   5  /* 2-D dot, pot_par = {a, b, v_in, v_out}                            */
#define TDZ_POT_H2P       6  /* 1-D two-centre soft core, pot_par = {R, eps} (Sec. Molecular HHG) */

/* Absorbing boundary layer: the complex absorbing potential -i eta(r) of Sec. "Parallel assembly" (CAP
 * matrix W = <B|eta|B>), eta = sum over the axes a of a 1-D mask of |x_a| that starts at |x_a| = r0 and
 * ends at |x_a| = R, s = (|x_a| - r0)/(R - r0) in (0, 1]. The paper names a Manolopoulos-type mask and
 * prints no formula; these are the two readings this library implements:
 *   TDZ_CAP_POLY          eta = eta0 s^k,                         cap_par = {r0, R, eta0, k}
 *   TDZ_CAP_MANOLOPOULOS  eta = (1/(2m)) (2 pi/(R - r0))^2 f(c s), cap_par = {r0, R, m, 0},
 *        f(y) = a y - b y^3 + 4/(c - y)^2 - 4/(c + y)^2, a = 1 - 16/c^3, b = (1 - 17/c^3)/c^2,
 *        c = 2.62206 (D. E. Manolopoulos, J. Chem. Phys. 117, 9552 (2002): a transmission-free layer that
 *        absorbs with little reflection above E_min = (c/(2 (R - r0)))^2/(2m); it diverges at |x_a| = R,
 *        which must therefore be the edge of the domain).
 * With a layer, Eq. cn_system becomes (S + tau W + i tau H) c^{n+1} = (S - tau W - i tau H) c^n: still
 * complex symmetric, and the norm c^H S c decreases by the flux the layer absorbs. */
#define TDZ_CAP_NONE          0
#define TDZ_CAP_POLY          1
#define TDZ_CAP_MANOLOPOULOS  2

typedef struct tdz_medium {
  int mass_kind;
  int pot_kind;
  double mass_par[4];
  double pot_par[4];
  int nlayers;                 /* TDZ_*_LAYERS only                      */
  const double* layer_bounds;  /* host, nlayers+1 increasing points      */
  const double* layer_mass;    /* host, nlayers                          */
  const double* layer_pot;     /* host, nlayers                          */
  int cap_kind;                /* TDZ_CAP_*; TDZ_CAP_NONE: no absorbing layer */
  double cap_par[4];
} tdz_medium;

/* ------------------------------------------------------------------ assembly
 * tdz_assemble: Galerkin matrices of Sec. "Parallel assembly" by Gauss
 * quadrature on every element, all in one pass over the elements:
 *   S = <B|B> (Eq. mass_elem), T = 1/2 <dB| m^-1 |dB> (Eq. bdd_elem),
 *   V = <B|V|B>, D_a = <B|x_a|B> (potential/dipole element formulas),
 *   G_a = <B| m^-1 dV/dx_a |B>, K = <B| m^-1 |B>  (acceleration, Eq. pdm_acceleration),
 *   W = <B|eta|B> (the absorbing layer's mask, CAP matrix; zero without a layer),
 * with the Dirichlet end functions removed. 1-D results are symmetric band
 * matrices, half bandwidth = degree. For dim = 2, 3 the operators keep the
 * per-axis 1-D factors S_a, T1_a = 1/2 <dB|dB>, D_a, W_a (Eq. tensor3d) and the
 * quadrature tables; the non-separable terms are applied by the batch from the
 * medium (one element per knot span and equal degrees are required, else
 * TDZ_EUNSUPPORTED; layered and Quesne media are 1-D only).
 */
typedef struct tdz_ops tdz_ops;
#define TDZ_MAT_S  0
#define TDZ_MAT_T  1
#define TDZ_MAT_V  2
#define TDZ_MAT_H0 3   /* T + V */
#define TDZ_MAT_D  4
#define TDZ_MAT_G  5
#define TDZ_MAT_K  6
#define TDZ_MAT_W  7   /* absorbing-layer mask <B|eta|B> (1-D), or the axis factor <B|eta_a|B> (2-D/3-D) */
#define TDZ_MAT_VEL 8  /* 1-D velocity matrix of Eq. vel_elem as Vel = -(i/2) M: returns the real antisymmetric
                          M, M_ab = sum_q w_q J_q m^-1 (N_a N_b' - N_a' N_b), lower band M(i, i-d)       */
int  tdz_assemble(const tdz_basis* const* axes, int dim, const tdz_medium* medium, tdz_ops** out);
/* n = DoF per axis (shape[0..dim-1]); degree per axis. */
int  tdz_ops_info(const tdz_ops* ops, int* dim, int64_t* shape, int* degree);
/* Copy a 1-D band matrix to host out[n*(degree+1)]: out[i*(degree+1)+d] = M(i, i-d). */
int  tdz_ops_band(const tdz_ops* ops, int which, int axis, double* out);
void tdz_ops_destroy(tdz_ops* ops);

/* tdz_pdm_acceleration: the position-dependent-mass term a_Q of the dipole acceleration (Eq.
 * aQ_definition; Eq. pdm_acceleration adds it to the Ehrenfest term that tdz_observe records) for nstates
 * 1-D states c[nstates][2n] (host, interleaved complex), written to aq[nstates] (host). In 1-D a_Q =
 * i <[T, v]> with T = 1/2 p m^-1 p and v the velocity operator (Eq. velocity_op); in the Galerkin basis an
 * operator product A B is A S^-1 B, so a_Q = -2 Im[(T c)^H S^-1 (Vel c)]. It vanishes with the mass
 * gradient. Host arithmetic in binary64 (one banded factorisation of S per call).
 * Errors: TDZ_EINVAL (null pointers, nstates < 1, a 2-D/3-D operator), TDZ_ENOCONV. */
int  tdz_pdm_acceleration(const tdz_ops* ops, const double* c, int64_t nstates, double* aq);

/* tdz_lowest_states: the nstates lowest eigenpairs of H0 c = eps S c (Eq. gen_ev) of nops 1-D geometries
 * (one degree) at once on the GPU: subspace inverse iteration with nstates + 2 vectors, a shift below the
 * spectrum (H0 - sigma S positive definite, factored once per geometry) and Rayleigh-Ritz in binary64, one
 * warp per geometry; stops when every wanted pair has ||H0 c - eps S c|| <= 1e-11 ||eps S c||.
 *   energies : host [nops][nstates], ascending per geometry.
 *   states   : host, geometry after geometry, [nstates][2 n_g] interleaved complex (real-valued,
 *              S-normalised, largest component positive: Sec. "Wavefunction realignment").
 *   residuals: host [nops][nstates] relative residuals (may be NULL); iterations: host [nops] (may be NULL).
 *   cuda_stream: the stream of the work (NULL: legacy default); the call synchronises it.
 * Errors: TDZ_EINVAL (nstates outside 1..6, a 2-D/3-D operator, mixed degrees, fewer than nstates + 2
 * coefficients), TDZ_EUNSUPPORTED (degree > 8), TDZ_ENOCONV (some geometry did not converge within 2000
 * iterations; its best pairs are still returned), TDZ_ECUDA. */
int  tdz_lowest_states(const tdz_ops* const* ops, int nops, int nstates, double* energies, double* states,
                       double* residuals, int* iterations, void* cuda_stream);

/* tdz_populations: projections of nstates 1-D states c[nstates][2n] on nev field-free eigenstates
 * phi[nev][2n] (S-orthonormal, e.g. from tdz_lowest_states), Sec. "Currents and coherence dynamics":
 *   pop [nstates][nev] (may be NULL): |c_n|^2 with c_n = phi_n^H S c;
 *   jdec[nstates][4]   (may be NULL): J_tot = c^H Vel c, J_intra = sum_n |c_n|^2 v_nn, J_inter =
 *        sum_{m != n} conj(c_m) c_n v_mn (v_mn = phi_m^H Vel phi_n) and J_bc = J_tot - J_intra - J_inter
 *        (Eqs. Jdecomp-Jbc); for real eigenstates v_nn = 0, so J_intra = 0.
 * Host arrays, binary64 host arithmetic. Errors: TDZ_EINVAL. */
int  tdz_populations(const tdz_ops* ops, const double* phi, int nev, const double* c, int64_t nstates, double* pop,
                     double* jdec);

/* Ground state of H0 c = eps S c (Eq. gen_ev) by shifted inverse iteration on
 * the host (1-D). Output: *energy and c[2n] (interleaved complex, real-valued,
 * S-normalised, largest component positive: Sec. "Wavefunction realignment").
 * TDZ_ENOCONV if the Rayleigh quotient has not settled within the cap.       */
int  tdz_ground_state(const tdz_ops* ops, double* energy, double* c);

/* ------------------------------------------------------------------ batch
 * A batch is a set of independent runs propagated together on one GPU (1-D:
 * one persistent launch per tdz_propagate call; 2-D/3-D: preconditioned COCG per
 * step, runs of a batch on concurrent workers: host threads with their own streams and work
 * buffers, 8 by default or the environment variable TDZ_ND_WORKERS (1..64) at creation, bounded by
 * a quarter of the free device memory). Run r uses ops[ops_index[r]];
 * runs may have different sizes; all operators of a batch have the same
 * dimension and degree. precision is TDZ_FP64 or TDZ_MIXED.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream); every GPU
 * operation of the batch is enqueued on it. The batch owns its device memory
 * (allocated here with cudaMalloc, freed by tdz_batch_destroy).
 */
typedef struct tdz_batch tdz_batch;
int  tdz_batch_create(const tdz_ops* const* ops, int nops, int nruns, const int* ops_index,
                      int precision, void* cuda_stream, tdz_batch** out);
/* Device bytes held by the batch (for capacity planning). */
int  tdz_batch_info(const tdz_batch* b, int* nruns, int64_t* total_dof, size_t* device_bytes);
/* Set the state of one run: c[2n], host or device. Resets that run's
 * extrapolation history (the next mixed step refines without a predictor). */
int  tdz_set_state(tdz_batch* b, int run, const double* c);
/* Copy the state of one run to c[2n], host or device. */
int  tdz_get_state(const tdz_batch* b, int run, double* c);
/* Set the states of all runs at once: c holds every run's coefficients (re, im interleaved) in
 * run order, c[2 (off_r + i) + {0,1}] with off_r = n_0 + ... + n_{r-1}; host or device. One upload
 * for the whole batch (a host array is staged in a device buffer allocated on first use, 16 bytes
 * per coefficient, held until tdz_batch_destroy). Resets every run's history and status like
 * tdz_set_state. Errors: TDZ_EINVAL, TDZ_ENONFINITE (a non-finite coefficient; the states are then
 * undefined), TDZ_ECUDA. Synchronises the batch stream. */
int  tdz_set_state_all(tdz_batch* b, const double* c);

/* Mixed-precision refinement control: after each FP32 solve the step is accepted when
 * ||B_n c^n - A_n c^{n+1}|| <= tol ||S c^n||; at most max_solves FP32 solves per step
 * (then the run's status becomes TDZ_ENOCONV and propagation continues). A solve after the
 * first is accepted without forming its residual when the contraction measured on the first
 * solve (below 1e-2) predicts a residual at most tol/10; the predicted value then enters
 * tdz_refine_stats. Defaults: tol = 1e-11, max_solves = 6. Ignored by TDZ_FP64 batches (one
 * exact solve per step). */
int  tdz_batch_set_refinement(tdz_batch* b, double tol, int max_solves);

/* Solver options of 2-D/3-D batches (1-D batches accept and ignore them).
 * TDZ_OPT_PRECOND selects the preconditioner M of the Krylov (COCG) solve:
 *   TDZ_PRECOND_AUTO  fast diagonalisation where it was set up at tdz_batch_create, else lines;
 *   TDZ_PRECOND_LINES M = (x)_a (S_a + i tau mbar T1_a), per-axis banded LDL^T line solves;
 *   TDZ_PRECOND_FD    M = S(x)S + i tau mbar (T1(x)S + S(x)T1) (all axes), inverted exactly through
 *                     the per-axis generalised eigenvectors T1_a v = lam S_a v (dense transforms).
 *   mbar = 1/m for a constant mass, the mean of 1/m_in and 1/m_out for a dot.
 * TDZ_OPT_OPERATOR selects how the non-separable part of H (V, and the kinetic term of a
 * position-dependent mass) is applied:
 *   TDZ_OPERATOR_AUTO        stencil where it was assembled (2-D), else quadrature;
 *   TDZ_OPERATOR_QUADRATURE  sum factorisation at the Gauss points, f(r) evaluated on the fly;
 *   TDZ_OPERATOR_STENCIL     2-D only: the same quadrature assembled once into a (2p+1)^2-point
 *                            stencil per DoF.
 * Both operator choices give the same A_n up to rounding.
 * TDZ_OPT_APPLY_GROUPS selects the variant of the fused FP32 2-D operator apply of mixed batches
 * with a stencil (how many warps split the 2p+1 offsets dy of a row tile): 0 (default) = the
 * variant the autotuner chose at tdz_batch_create, or 8 or 16 to force one. Results do not depend
 * on it beyond FP32 rounding.
 * TDZ_OPT_WAIT_TEST (test aid for the bounded waits; 0 = off, the default): with 1 the fused FP32
 * 2-D apply issues no stencil copies and waits at most about 10 ms for them, so its wait runs out
 * and tdz_propagate returns TDZ_ECUDA with the run's status set; the device stays usable.
 * Errors: TDZ_EINVAL (unknown option or value), TDZ_EUNSUPPORTED (the choice was not set up for
 * this batch). */
#define TDZ_OPT_PRECOND          1
#define TDZ_OPT_OPERATOR         2
#define TDZ_OPT_APPLY_GROUPS     3
#define TDZ_OPT_WAIT_TEST        4
#define TDZ_OPT_CURRENT          5   /* 1-D: 1 = record J = c^H Vel c after every step (tdz_observe_current) */
#define TDZ_PRECOND_AUTO         0
#define TDZ_PRECOND_LINES        1
#define TDZ_PRECOND_FD           2
#define TDZ_OPERATOR_AUTO        0
#define TDZ_OPERATOR_QUADRATURE  1
#define TDZ_OPERATOR_STENCIL     2
int  tdz_batch_set_option(tdz_batch* b, int option, int value);
/* Autotuner result for geometry `geometry` (index into the ops array of tdz_batch_create) of a
 * 2-D mixed batch: at creation every variant of the fused FP32 operator apply is timed on the
 * batch's own buffers (CUDA events, best of three) and the fastest is kept. groups (host, optional):
 * the chosen variant (8 or 16; 0 when the geometry has no FP32 stencil or the batch is not 2-D
 * mixed); ms (host, optional, 2 doubles): the measured ms per apply of the variants 8 and 16.
 * Errors: TDZ_EINVAL (bad handle or geometry index). */
int  tdz_batch_tuning(const tdz_batch* b, int geometry, int* groups, double* ms);
/* Autotuner result for the fast-diagonalisation preconditioner of geometry `geometry` of a 2-D/3-D
 * mixed batch: at creation one whole preconditioner apply (the tensor-core axis transforms of
 * tdz_tc_axis_transform with the split, eigenvalue scaling and merge around them) is timed on the
 * batch's own buffers (CUDA events, best of three) in six variants and the fastest is kept: variants
 * 0-3 use 256-column transform tiles if bit 0 of v is set (else 128) and split the data into TF32 pairs
 * inside the transform, in shared memory, if bit 1 is set (else the kernels around the transforms write
 * the pairs to memory); variants 4 and 5 use 64-column tiles (more blocks on small planes) with the
 * pairs in memory and in shared memory respectively. variant (host, optional): the chosen v (-1 when
 * the geometry has no fast diagonalisation or the batch is not mixed); ms (host, optional, 6 doubles):
 * ms per preconditioner apply of variants 0..5. Errors: TDZ_EINVAL (bad handle or geometry index).
 * Autotuner cache (both autotuners): with the environment variable TDZ_TUNE_CACHE naming a file, each
 * result is appended to it as one JSON object per line, {"key": ..., "values": [...]}, keyed by what
 * was tuned, the sizes, the precision and the device name; a later batch creation with the same key
 * takes the stored result instead of timing (the ms reported are then the stored timings). */
int  tdz_batch_precond_tuning(const tdz_batch* b, int geometry, int* variant, double* ms);
/* tdz_batch_time_operator (2-D/3-D): time one apply of the inner-solve operator y = A_n x of Eq. cn_system
 * (FP32 in a mixed batch, binary64 otherwise; the batch's operator and absorbing-layer choices) for a run
 * of geometry `geometry`, on the batch's own work buffers, with CUDA events on the batch stream: *ms = the
 * best of `reps` applies after one warm-up. Run states are not touched. Synchronises the stream.
 * Errors: TDZ_EINVAL (bad handle, geometry or reps), TDZ_EUNSUPPORTED (1-D batch), TDZ_ECUDA. */
int  tdz_batch_time_operator(tdz_batch* b, int geometry, int reps, double* ms);
/* tdz_batch_ground_state (2-D/3-D): the ground state of H0 c = eps S c (Eq. gen_ev, no field) of run `run`,
 * on the GPU, by inverse iteration with the fixed shift sigma: every outer iteration solves
 * (H0 - sigma S) x = S c with the batch's preconditioned COCG (operator i tau (H0 - sigma S), fast
 * diagonalisation with the shifted eigenvalue scaling, inner tolerance tol / 10), in binary64 in a binary64
 * batch and with the FP32 operator and tensor-core preconditioner of the inner solves in a mixed batch
 * (FP32 accuracy: tol of about 1e-5 or more, inner tolerance at least 1e-6), takes the Rayleigh
 * quotient eps = sigma + c^H S x / x^H S x and sets c = x / |x|_S; it stops when the eigen-residual
 * |H0 c - eps S c|_{S^-1} <= tol |eps|. sigma must lie below the lowest eigenvalue, close enough that
 * (eps_0 - sigma) / (eps_1 - sigma) is small (the contraction per outer iteration). The run's current state
 * (tdz_set_state) is the start vector and must overlap the ground state; it is replaced by the result,
 * S-normalised. energy, iterations (outer iterations), residual (the final relative eigen-residual): host
 * outputs, each may be NULL. Synchronises the batch stream.
 * Errors: TDZ_EINVAL (bad handle, run, tol <= 0, max_outer < 1, a start vector with no S-norm),
 * TDZ_EUNSUPPORTED (1-D batch, an absorbing layer, or the line preconditioner selected),
 * TDZ_ENOCONV (not converged within max_outer; the last iterate and its residual are returned),
 * TDZ_ENONFINITE, TDZ_ECUDA. */
int  tdz_batch_ground_state(tdz_batch* b, int run, double sigma, double tol, int max_outer, double* energy,
                            int* iterations, double* residual);
/* Total Krylov iterations of all runs since the batch was created (2-D/3-D; 0 in 1-D, whose
 * solve is direct). Synchronises the batch stream. */
int  tdz_krylov_stats(const tdz_batch* b, double* iterations);

/* tdz_propagate: nsteps Crank-Nicolson steps of every run (Sec. "Time
 * propagation", Eq. cn_system), from absolute step index step0:
 *   (S + i dt/2 H_n) c^{n+1} = (S - i dt/2 H_n) c^n,  H_n = H0 + Ebar_n D,
 *   Ebar_n = (E(t_n) + E(t_{n+1}))/2,  t_n = n dt.
 * field: host or device, field[(r*(nsteps+1) + k)*dim + a] = E_a(t_{step0+k}),
 *   k = 0..nsteps, for every run r.
 * After every step the observables of Sec. "Dipoles" are recorded (see
 * tdz_observe). The call is asynchronous with respect to the host when the
 * field is a device pointer; it synchronises the stream otherwise.
 * Errors: TDZ_EINVAL (sizes), TDZ_ECUDA. Per-run numerical failures
 * (non-finite state, refinement cap) are reported by tdz_observe's status. */
int  tdz_propagate(tdz_batch* b, const double* field, double dt, int64_t step0, int64_t nsteps);

/* tdz_observe: observables of run `run` for the steps of the last
 * tdz_propagate call, out[nsteps][2+3*dim] (host or device):
 *   [t_{n+1}, E_a(t_{n+1}), d_a = c^H D_a c, a_a = -c^H G_a c - E_a c^H K c, c^H S c]
 * (raw, not divided by the norm). *status (host, may be NULL) receives the
 * run's status: TDZ_OK, TDZ_ENONFINITE or TDZ_ENOCONV (first failure wins).
 * Synchronises the batch stream. */
int  tdz_observe(const tdz_batch* b, int run, double* out, int* status);
/* Observables of all runs at once: out[nruns][nsteps][2+3*dim] (host or device, may be NULL) in the
 * layout of tdz_observe for each run, status[nruns] (host, may be NULL). Synchronises the batch
 * stream. */
int  tdz_observe_all(const tdz_batch* b, double* out, int* status);
/* tdz_observe_current: the total dipole velocity J(t_{n+1}) = c^H Vel c (Sec. "Currents and coherence
 * dynamics": the expectation of the velocity operator of Eq. velocity_op, equal to d<x>/dt) of run `run`
 * for every step of the last tdz_propagate call, out[nsteps] (host or device). Recorded by 1-D batches
 * after tdz_batch_set_option(b, TDZ_OPT_CURRENT, 1) (binary64 sums, or double-float in mixed precision).
 * Errors: TDZ_EINVAL (no current recorded), TDZ_ECUDA. Synchronises the batch stream. */
int  tdz_observe_current(const tdz_batch* b, int run, double* out);
/* Largest relative residual ||b - A c||/||b|| seen by the refinement of any run
 * (mixed precision; 0 for a 1-D TDZ_FP64 batch) and the total number of solves of
 * all runs, both since the batch was created. Synchronises the batch stream. */
int  tdz_refine_stats(const tdz_batch* b, double* max_rel_residual, double* mean_solves);
void tdz_batch_destroy(tdz_batch* b);


/* ------------------------------------------------------------------ harmonic spectrum
 * tdz_spectrum: the windowed spectrum of Sec. "Dipoles", S(w) = |dt sum_k s(t_k) W_k e^{i w t_k}|^2 with
 * t_k = k dt and the Kaiser window W_k = I0(beta sqrt(1 - (2k/(nt-1) - 1)^2)) / I0(beta), for nsig records
 * at once, at the nw frequencies w_j = w_lo + j dw; length_form = 1 multiplies by w^4 (the acceleration
 * spectrum from a dipole record), 0 leaves it (an acceleration record). Direct sums in binary64 on the GPU.
 *   signal: host or device, record s sample k at signal[s * sig_stride + k * t_stride] (e.g. the d or a
 *           column of tdz_observe_all's output: t_stride = 2 + 3 dim, sig_stride = nsteps t_stride).
 *   S     : host or device, [nsig][nw] output.
 *   cuda_stream: stream of the work (NULL: legacy default stream); the call synchronises it.
 * Errors: TDZ_EINVAL (sizes, strides, dt <= 0, beta < 0, nsig > 65535), TDZ_ECUDA.
 * tdz_harmonic_yields: per record, the yield of every odd harmonic q = 1, 3, ..., <= qmax of the
 * fundamental omega0: the trapezoid integral of S over the grid points in [(q - 1/2) omega0,
 * (q + 1/2) omega0]. S: host [nsig][nw] on the grid w_lo + j dw; Y: host [nsig][(qmax + 1)/2].
 * Errors: TDZ_EINVAL. */
int  tdz_spectrum(const double* signal, int64_t nsig, int64_t nt, int64_t sig_stride, int64_t t_stride, double dt,
                  double beta, int length_form, double w_lo, double dw, int64_t nw, double* S, void* cuda_stream);
int  tdz_harmonic_yields(const double* S, int64_t nsig, double w_lo, double dw, int64_t nw, double omega0, int qmax,
                         double* Y);

/* ------------------------------------------------------------------ device rates
 * tdz_device_rates: the FP32 and binary64 fused multiply-add throughput of the current device in flop/s
 * (eight independent FMA chains per thread, 8 blocks of 256 threads per SM, CUDA events, best of three
 * timed launches). The ratio is what makes the mixed path form its binary64-class residuals in
 * double-float on B300. No counterpart in the paper. Errors: TDZ_EINVAL, TDZ_ECUDA. */
int  tdz_device_rates(double* fp32_flops, double* fp64_flops);

/* ------------------------------------------------------------------ tensor-core axis transform
 * tdz_tc_axis_transform: one axis transform of the fast-diagonalisation preconditioner M^-1 =
 * (V_x (x) V_y ...) diag(1 / (1 + i tau mbar sum_a lam_a)) (V_x (x) V_y ...)^T (Sec. "Eigenvalue
 * problem": V_a the S_a-orthonormal eigenvectors of T1_a v = lam S_a v), as the mixed-precision 2-D/3-D
 * preconditioner runs it, on the tensor cores (tcgen05, TF32 operands, FP32 accumulation):
 *   D(m, j) = sum_kk (a_hi + a_lo)[m*k + kk] (b + b_lo)[j*k + kk]   (kk < k),   m < rows, j < ncols,
 * evaluated as a_hi b + a_lo b + a_hi b_lo (the a_lo b_lo term is dropped; without b_lo, b_lo = 0),
 * written to out_hi[p*plane_stride + j*plane_rows + r] with p = m / plane_rows, r = m mod plane_rows
 * (the contracted index moves from fastest to slowest). With out_lo non-NULL the result is stored as
 * a TF32 pair: out_hi = D rounded to TF32 (nearest, ties away), out_lo = D - out_hi; with out_lo NULL
 * out_hi = D in FP32. The hi arrays should hold TF32 values and the lo arrays the FP32 remainders
 * (every operand is read as TF32: the low 13 bits of each FP32 pattern are ignored). With a_lo NULL,
 * a_hi holds the data in FP32 and each block splits its tiles into the pair in shared memory. tile_n: 0 (the
 * library's choice: 128 or 256), 64, 128 or 256 columns per block. All pointers are device memory owned by the caller,
 * the operands 16-byte aligned; k must be a multiple of 4. Synchronises the stream. Errors:
 * TDZ_EINVAL (sizes, alignment, tile_n), TDZ_ECUDA (launch failure, or a pipeline wait that ran out
 * of time). */
int  tdz_tc_axis_transform(const float* a_hi, const float* a_lo, int64_t rows, int k, const float* b,
                           const float* b_lo, int ncols, int64_t plane_rows, int64_t plane_stride, float* out_hi,
                           float* out_lo, int tile_n, void* cuda_stream);

/* ------------------------------------------------------------------ allocation-free entry point
 * tdz_cn1d_propagate_noalloc: the binary64 1-D propagation of tdz_propagate for ONE run, for
 * callers that cannot call cudaMalloc: integrations whose host framework owns all device memory
 * through its own pool (a caching allocator or an arena reserved at start-up) and forbids side
 * allocations, and code that must not risk the implicit device synchronisation cudaMalloc and
 * cudaFree can cause. The paper has no counterpart; it exists for deployment only.
 * The caller passes inputs and outputs; the scratch lives in one fixed device array compiled
 * into this library (about 2.4 MB, held by every GPU that loads the library until exit):
 *   bands : device, [5][n][degree+1] lower bands S, H0, D, G, K: bands[(q*n + i)*(degree+1) + d]
 *           = M_q(i, i-d) (as returned by tdz_ops_band), read only.
 *   field : device, E(t_{step0+k}) for k = 0..nsteps.   state: device, [2n] complex in/out.
 *   obs   : device, [nsteps][5] = t, E, d, a, norm (as tdz_observe).
 *   status: host, optional; if given the call synchronises the stream and stores the run status.
 *           Pass NULL when the call is recorded into a stream capture (a synchronisation is not
 *           allowed there); read the status later from obs instead (non-finite norms).
 * Limits: n <= TDZ_NOALLOC_MAX_N, degree <= 8; larger sizes return TDZ_EINVAL with a message, and
 * so does a current device index of 64 or more.
 * The first call on a device resolves the array's device address with cudaGetSymbolAddress
 * (that device current); make that first call before any stream capture. Every call shares the
 * one array and overwrites it (the call initialises all of it that it reads), so calls that
 * overlap on the GPU - on different streams or host threads - race and must be serialised.
 * No cudaMalloc, cudaFree or allocating library routine is called.                           */
#define TDZ_NOALLOC_MAX_N 4096
int  tdz_cn1d_propagate_noalloc(const double* bands, int64_t n, int degree, const double* field, double dt,
                                int64_t step0, int64_t nsteps, double* state, double* obs, void* cuda_stream,
                                int* status);

#ifdef __cplusplus
}
#endif
#endif /* TDZ_H */
