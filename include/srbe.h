/*
 * srbe.h - C ABI of the GB300 (sm_103a) implementation of the symmetry-preserving
 * random batch Ewald (SRBE) method for constant-potential electrode/electrolyte
 * slabs (Gao, Zhou, Zhang, Xu, arXiv 2509.24742).
 *
 * Equation numbers count the paper's displayed equations in order: Eq. 7 the
 * potential split, Eqs. 9-11 the neutral charge solve, Eq. 13 the real-space
 * energy, Eq. 15 the structure factors, Eq. 17 the self/slab corrections,
 * Eq. 18 the matrix A, Eq. 19 the vector b, Eq. 24 the SRBE vector b, Eq. 25
 * the SRBE force, Eqs. 26-29 the sampling law and Metropolis step; Algorithm 1
 * is the MD loop.
 *
 * Units: nm, ps, amu, e, kJ/mol; potentials in volts at the interface.  Arrays of
 * vectors are row-major [n][3] doubles.  Host-pointer calls copy in and out;
 * the context owns every device buffer.  Every call returns an srbe_status;
 * srbe_last_error() gives the text of the last failure.  Calls made in the wrong
 * order return SRBE_ESTATE.  A context is used by one host thread at a time.
 */
#ifndef SRBE_H
#define SRBE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srbe_ctx srbe_ctx;

enum srbe_status {
  SRBE_OK = 0,
  SRBE_EINVAL = 1,   /* bad argument (null pointer, size, non-finite value, box) */
  SRBE_ENOMEM = 2,   /* device or host allocation failed */
  SRBE_ECUDA = 3,    /* a CUDA call failed; the message names it */
  SRBE_ESTATE = 4,   /* call out of order (e.g. forces before positions) */
  SRBE_ENOTCONV = 5, /* iterative solve did not reach its tolerance */
  SRBE_ETIMEOUT = 6, /* a bounded wait for the device gave up (srbe_synchronize) */
  SRBE_ENONFINITE = 7 /* a force or an electrode charge came out NaN or infinite */
};

/* Errors found on the device.  Kernels raise flags in a few words of host-mapped memory owned by
 * the context: an iterative charge solve that stopped at maxit (SRBE_ENOTCONV; the charges of that
 * pass then come from the direct solve instead, see srbe_set_solver) and a non-finite force or
 * charge (SRBE_ENONFINITE; checked on every force pass, on every charge update of
 * srbe_solve_electrode_charges, and in the closing half kick of every MD step).  A flag is reported,
 * and cleared, by the first of these calls that sees it: srbe_forces and
 * srbe_solve_electrode_charges (after their outputs are written, so the outputs of that call are
 * valid host copies of what the device holds), srbe_synchronize, srbe_step, which is asynchronous:
 * it reports SRBE_ENONFINITE (and a bad input) raised by earlier steps at its start and between the
 * steps it queues, as soon as the host sees them, and then steps no further, and srbe_batch_step
 * (each replica's flags, at its start).  Neither of the two stops for SRBE_ENOTCONV, since that pass
 * took the direct solve's charges: the flag stays raised for srbe_synchronize (or the next
 * srbe_forces / srbe_solve_electrode_charges).  srbe_minimize reports SRBE_ENOTCONV only: its forces may overflow where the random packing
 * put two sites on top of each other, which its capped step handles.  srbe_forces_dev is
 * asynchronous and leaves its flags to the next of these calls.  SRBE_ENONFINITE takes precedence
 * over SRBE_ENOTCONV; srbe_last_error names what was found.
 *
 * srbe_synchronize: waits for every pass queued on the context's streams, at most timeout_s seconds
 * (timeout_s < 0: without limit), then reports the device flags.  SRBE_ETIMEOUT if work is still
 * running at the limit (nothing is cancelled; the call may be repeated). */
int srbe_synchronize(srbe_ctx *ctx, double timeout_s);

enum srbe_precision {
  SRBE_FP64 = 0,  /* every sum, phase and pair term in FP64 */
  SRBE_MIXED = 1  /* FP32 phases/sums/pairs with compensated accumulation; FP64 neutrality, slab, solve */
};

enum srbe_sampler {
  SRBE_SAMPLER_METROPOLIS = 0, /* Eqs. 28-29: rounded-Gaussian proposals, Metropolis acceptance */
  SRBE_SAMPLER_EXACT = 1       /* i.i.d. inverse-CDF draws of P(k) (Eq. 26), rejecting I u {0} */
};

/* Creates a context for a slab in the box [0,Lx) x [0,Ly) x [0,Lz), periodic in x and y,
 * with Lz the Fourier period in z that already contains the vacuum padding (§2, the
 * slab-correction paragraph: L_z = lambda H).
 *   alpha      Ewald splitting parameter of Eq. 12 used for the dynamics (nm^-1)
 *   eta        width of the Gaussian electrode charges of Eq. 1, as a LENGTH (nm)
 *   rc         real-space cutoff (nm); every in-plane image within rc is summed
 *   P          sampled Fourier modes per step (Eq. 26), P >= 0
 *   kz0        M: the deterministic set I = {(0,0,2 pi m_z / Lz): 1 <= |m_z| <= M}
 *   psi_left, psi_right  electrode potentials (V); only dpsi = psi_right - psi_left enters
 *              (Eqs. 9-11, d = -1/2 on the left electrode, +1/2 on the right, Eq. 7)
 * Errors: SRBE_EINVAL for a non-positive box/alpha/eta/rc or negative P/kz0. */
int srbe_create(const double box[3], double alpha, double eta, double rc, int P, int kz0,
                double psi_left, double psi_right, srbe_ctx **out);

/* Releases every device and host resource of the context. NULL is accepted. */
int srbe_destroy(srbe_ctx *ctx);

/* Text of the last error on this context (never NULL; "" when none). */
const char *srbe_last_error(const srbe_ctx *ctx);

/* Runs the context's work on this CUDA stream (a cudaStream_t passed as void*; NULL = the
 * context's own stream).  The caller keeps ownership of the stream. */
int srbe_set_stream(srbe_ctx *ctx, void *stream);

/* Chooses the arithmetic of the hot path (enum srbe_precision). */
int srbe_set_precision(srbe_ctx *ctx, int mode);

/* Parameters of the one-time build of A (Eq. 18): A is independent of its Ewald parameter
 * up to the pi/(V alpha_A^2) e e^T background constant, which drops out under e^T Q = 0, so
 * it is built with its own alpha_A (<= 0: chosen automatically, never below 6.5 / (Lz - H)
 * so that the in-plane-only real-space sum stays exact) and truncated where
 * exp(-k^2/4 alpha_A^2) and erfc(alpha_A r) fall below tol (<= 0: 1e-17). */
int srbe_set_A_params(srbe_ctx *ctx, double alpha_A, double tol);
/* The alpha_A A was built with (after srbe_set_electrode; 0 for a NULL context). */
double srbe_get_alpha_A(const srbe_ctx *ctx);

/* Fixes the electrode: n_ele sites R [n_ele][3] and their side (0 = left, 1 = right).
 * Builds A (Eq. 18, slab term (4 pi / V) Z_i Z_j), inverts it on the GPU, and stores the
 * projected inverse J A^-1 (Eqs. 10-11) and A^-1 e.  Cost is paid once (§2: A is constant).
 * Up to 16,384 sites A is stored densely; lattice electrodes (srbe_set_lattice) also get the
 * spectral form of A, and beyond 16,384 sites (up to 4,194,304) they get only that.
 * Errors: SRBE_EINVAL (n_ele < 2 or too large, more than 16,384 sites that are not a lattice, a
 * side other than 0/1, one side empty, non-finite R), SRBE_ENOTCONV if A is not positive definite. */
int srbe_set_electrode(srbe_ctx *ctx, int64_t n_ele, const double *R, const int8_t *side);

/* Sets the n_ion electrolyte positions r [n_ion][3] (nm) and charges q (e).  0 <= n_ion <= 8,388,607.
 * Positions outside [0,L) in x or y are wrapped.  With the same ion count and the same charges as
 * the previous call (an MD engine handing in each step's positions) the Verlet lists are kept and
 * rebuilt only once an ion has moved more than half the skin since their build; otherwise they are
 * rebuilt at the next force evaluation.  Errors: SRBE_EINVAL on non-finite input. */
int srbe_set_positions(srbe_ctx *ctx, int64_t n_ion, const double *r, const double *q);

/* Copies the current ion positions and velocities out (either pointer may be NULL). */
int srbe_get_positions(srbe_ctx *ctx, double *r, double *v);

/* MD support terms for srbe_step: masses (amu), velocities (nm/ps, may be NULL = 0), a site
 * type per ion (0..ntype-2; type ntype-1 is the electrode), a molecule id per ion (LJ is
 * excluded inside a molecule), ntype x ntype LJ sigma (nm) and epsilon (kJ/mol) tables,
 * nb harmonic bonds (pairs of ion indices, rest lengths r0, force constant kb) and the time
 * step dt (ps).  1 <= ntype <= 16.  Must follow srbe_set_positions with the same n_ion. */
int srbe_set_md(srbe_ctx *ctx, const double *mass, const double *v, int ntype, const int32_t *itype,
                const int32_t *mol, const double *lj_sigma, const double *lj_eps, int64_t nb,
                const int32_t *bonds, const double *r0, double kb, double dt);

/* Chooses the sampler (enum srbe_sampler) and an optional truncation box |m_d| <= mmax[d]
 * for the sampled modes (mmax NULL or entries <= 0: the whole lattice L_k \ I). */
int srbe_set_sampler(srbe_ctx *ctx, int kind, const int32_t *mmax);

/* Draws the P modes of one step from P(k) = exp(-k^2/4 alpha^2)/G on L_k \ I (Eqs. 26-29) on
 * the host with a Philox4x64-10 stream keyed by seed and indexed by step, and computes G
 * (Eq. 27).  The same (seed, step) always gives the same list. */
int srbe_sample_k(srbe_ctx *ctx, uint64_t seed, uint64_t step);

/* The exact sampler (SRBE_SAMPLER_EXACT, inverse CDF per dimension of Eq. 26's P(k), rejection of
 * I u {0}) on the device: one kernel draws the same Philox stream as the host sampler, takes the
 * first P admissible tries in order and writes the modes and the Eq. 24-25 weights (G / P) 4 pi /
 * (V k^2) with the host's operations in the host's order, so the list is bitwise the host's.  With
 * it on, srbe_step's captured steps sample on the device (the host writes only the step and seed);
 * the batch keeps host sampling.  srbe_set_device_sampler: on = 1 needs SRBE_SAMPLER_EXACT
 * (SRBE_EINVAL otherwise); its tables follow srbe_set_sampler.  srbe_sample_k_device: like
 * srbe_sample_k through the device kernel; copies the P sampled modes m [P][3] and their weights
 * w [P] out (either may be NULL).  SRBE_ESTATE without the device sampler on; SRBE_ENOTCONV if fewer
 * than P admissible modes came out of 2^20 tries. */
int srbe_set_device_sampler(srbe_ctx *ctx, int on);
int srbe_sample_k_device(srbe_ctx *ctx, uint64_t seed, uint64_t step, int32_t *m, double *w);

/* Copies out the current sampled modes (m [P][3] integers, k = 2 pi m / L) and G. */
int srbe_get_k(const srbe_ctx *ctx, int32_t *m, double *G);

/* Sets the P sampled modes explicitly (m [P][3]); weights follow Eq. 24/25 with the
 * context's G.  P may differ from srbe_create's.  Errors: SRBE_EINVAL for a mode in I u {0} or
 * more than 2,097,120 modes in all. */
int srbe_set_k(srbe_ctx *ctx, const int32_t *m, int P);

/* Replaces the whole mode list by an explicit deterministic list m [K][3] with per-mode
 * weights w [K] (the factor c_k multiplying Re/Im terms in Eqs. 20-21; for full Ewald
 * w = 4 pi exp(-k^2/4 alpha^2) / (V k^2)).  Used to evaluate full Ewald on the same path.
 * Errors: SRBE_EINVAL for k = 0, non-finite weights or K > 2,097,120. */
int srbe_set_mode_list(srbe_ctx *ctx, const int32_t *m, const double *w, int K);

/* Electrode-charge update of Algorithm 1 ("compute b, update Q"): S1 (Eq. 15), b (Eq. 24 with
 * the near and slab parts of Eq. 19), then psi_bar and Q (Eqs. 9-10).  Outputs (host, any
 * may be NULL): Q [n_ele] (e), psi_bar (V), b [n_ele] (V).  Needs electrode, positions, modes. */
int srbe_solve_electrode_charges(srbe_ctx *ctx, double *Q, double *psi_bar, double *b);

/* One force evaluation: the charge update above, then S2, the SRBE k-space force (Eq. 25),
 * the slab force -(4 pi / V) q_i M_z, the real-space Coulomb forces of Eq. 13 and, after
 * srbe_set_md, LJ and bond forces.  Outputs (host, any may be NULL): F [n_ion][3] (kJ/mol/nm),
 * Q [n_ele] (e), psi_bar (V), energy[8] (kJ/mol): U_N ion-ion, U_N ion-electrode, U_N
 * electrode-electrode (within rc), U_F (1/2 sum_k c_k |S|^2), U_self, U_slab, U_LJ, U_bond. */
int srbe_forces(srbe_ctx *ctx, double *F, double *Q, double *psi_bar, double *energy);

/* Algorithm 1 for nsteps velocity-Verlet steps of dt: per step, draw the P modes with
 * srbe_sample_k(seed0, step_counter++), update Q, compute forces, integrate.  Electrode
 * sites stay fixed, ions wrap in x and y.  State stays on the device. */
int srbe_step(srbe_ctx *ctx, int nsteps, uint64_t seed0);

/* Relaxes the ions before MD by nsteps of displacement-capped steepest descent on the full
 * force of srbe_forces (Coulomb with the CP charges, LJ, bonds): r_i += F_i min(a, dmax / |F_i|)
 * with a in nm^2 mol/kJ and dmax in nm; the modes of iteration t are drawn with
 * srbe_sample_k(seed, t).  No counterpart in the paper (the synthetic workloads start from a
 * random packing); needs srbe_set_md.  Velocities are kept. */
int srbe_minimize(srbe_ctx *ctx, int nsteps, double a, double dmax, uint64_t seed);

/* Captured force provider for an MD engine that keeps its state in host memory (no counterpart in
 * the paper; launch- and copy-overhead removal).  srbe_set_host_io binds three caller-owned buffers of
 * page-locked host memory mapped for the device (cudaHostAlloc, or registered with cudaHostRegister;
 * the caller keeps ownership and must keep them alive while bound): r [n_ion][3] positions in,
 * F [n_ion][3] forces out, Q [n_ele] charges out (Q may be NULL).  srbe_forces_host_io then equals
 * srbe_set_positions(r, same charges) + srbe_sample_k(seed, step) + srbe_forces(F, Q, psi_bar), bitwise,
 * as one CUDA-graph replay per call: a kernel reads the positions straight from the bound buffer, the
 * force pass runs, a kernel writes F (and Q) back into the bound buffers, and the call returns once
 * they hold the result.  The first call after any state change (and after srbe_set_host_io) runs the
 * ordinary way and captures the graphs.  The charges are those of the last srbe_set_positions.
 * Errors: SRBE_ESTATE (not bound, no electrode or positions), SRBE_EINVAL (a buffer that is not mapped
 * page-locked memory; a non-finite position in r, which that pass replaced by the origin), and the
 * device flags of srbe_synchronize. */
int srbe_set_host_io(srbe_ctx *ctx, double *r, double *F, double *Q);
int srbe_forces_host_io(srbe_ctx *ctx, uint64_t seed, uint64_t step, double *psi_bar);

/* Device-resident variants: same as the host calls, with device pointers on the context's
 * stream and no host copies.  F_dev [n_ion*3], Q_dev [n_ele] may be NULL. */
int srbe_set_positions_dev(srbe_ctx *ctx, int64_t n_ion, const double *r_dev, const double *q_dev);
int srbe_forces_dev(srbe_ctx *ctx, double *F_dev, double *Q_dev);

/* Counters for benchmarking: kernels launched by this context since creation, and the
 * k-space work units (particle x mode evaluations) since creation. */
int srbe_get_counters(const srbe_ctx *ctx, int64_t *kernel_launches, int64_t *mode_evals);

/* Phase tracing (no counterpart in the paper; a measurement aid).  When on, every pass records a
 * CUDA event pair around each phase of Algorithm 1:
 *   0 mode-list upload, 1 cell lists, 2 S1 (ions), 3 b (electrode right-hand side),
 *   4 charge solve, 5 S2 (electrode), 6 ion forces, 7 integration, 8 energies,
 *   9 ion-ion forces (mixed form without energies: the ion-ion pairs and bonds run as their own
 *     pass on the context's side stream, beside phases 3-5; phase 6 is then the rest).
 * Phases 1 and 9 are timed on the side stream, the others on the context's stream.
 * srbe_get_phase_times synchronises and returns, per phase, the summed device time (ms) and the
 * number of timed intervals since tracing was switched on (arrays of 10; either may be NULL).
 * Switching tracing on resets the sums. */
int srbe_set_profiling(srbe_ctx *ctx, int on);

/* CUDA graphs for srbe_step (no counterpart in the paper; launch-overhead removal).  With graphs on
 * (the default) and tracing off, srbe_step runs its first step after any state change the ordinary
 * way, then captures the device half of a step (mode list read from one of two mapped pinned host
 * slots, kick/drift, the full force pass, kick) into one graph per slot and replays it; the host samples
 * the next step's modes into the other slot while the GPU runs.  Results are bitwise those of the
 * ordinary path.  Every call other than srbe_step and the get/stat queries drops the graphs (they
 * are captured again on the next srbe_step).  If capture fails the context keeps stepping the
 * ordinary way until srbe_set_graphs is called again.  srbe_graph_state reports captured = 1
 * (graphs live), 0 (none yet) or -1 (capture failed) and the kernels one replay runs; either
 * pointer may be NULL. */
int srbe_set_graphs(srbe_ctx *ctx, int on);
int srbe_graph_state(srbe_ctx *ctx, int *captured, int64_t *kernels_per_step);
int srbe_get_phase_times(srbe_ctx *ctx, double *ms, int64_t *count);

/* ---- iterative charge solve and the learned warm start ------------------------------------------
 * The per-step charge update can run preconditioned conjugate gradients on A y = dpsi d + b
 * (Jacobi preconditioner, one cooperative launch, convergence tested on the device) instead of the
 * direct projected inverse; Q and psi_bar then follow from Eqs. 9-10.  The starting guess is zero,
 * the previous step's solution, or the prediction of a per-site MLP (the learned form; no
 * counterpart in the paper).  tol is the relative residual ||dpsi d + b - A y|| / ||dpsi d + b||. */
/* SRBE_SOLVER_LATTICE (lattice electrodes, see srbe_set_lattice): A is block-circulant over the
 * lattice, so A^-1 acts as one nl x nl inverse per (m_x mod nx, m_y mod ny) bin between two of
 * the lattice transforms; the solve is exact (no iteration; tol, maxit and warm are ignored) and
 * needs no dense matrix.  srbe_set_electrode picks it for lattice electrodes of 8,192 sites or
 * more; beyond 16,384 sites it is the only solver (A is not stored densely), otherwise
 * SRBE_SOLVER_DIRECT is the default.  Errors: SRBE_ESTATE for a solver the electrode cannot use. */
/* In the mixed form PCG runs as iterative refinement: the FP64 residual dpsi d + b - A y decides
 * convergence (tol as above), and each correction comes from Jacobi-preconditioned CG on an FP32 copy
 * of A (formed once per electrode; half the bytes per product), in the Chronopoulos-Gear arrangement
 * (one grid-wide reduction per iteration), run until its residual has fallen by 1e-4; maxit bounds
 * these inner iterations, which srbe_get_solver_stats counts.  The inner sums are FP32, so the
 * iteration count can differ by a few between builds that group them differently; the FP64 residual
 * bar does not.
 * A PCG solve that reaches maxit above tol raises SRBE_ENOTCONV (see srbe_synchronize); the same pass
 * then takes its charges from the direct projected inverse (one extra kernel that runs only in that
 * case), so the forces and the MD step that follow use converged charges. */
enum srbe_solver { SRBE_SOLVER_DIRECT = 0, SRBE_SOLVER_PCG = 1, SRBE_SOLVER_LATTICE = 2 };
enum srbe_warm { SRBE_WARM_ZERO = 0, SRBE_WARM_PREVIOUS = 1, SRBE_WARM_MODEL = 2 };
int srbe_set_solver(srbe_ctx *ctx, int kind, double tol, int maxit, int warm);
/* Iterations and the recomputed relative residual of the last PCG solve. */
int srbe_get_solver_stats(srbe_ctx *ctx, int *iterations, double *rel_residual);

/* The MLP (80 -> 128 -> 128 -> 1, SiLU; FP32 parameters) predicts y = A^-1 (dpsi d + b) per electrode site from
 * 80 descriptors: 32 Gaussian radial densities (centres 0.25..1.25 nm, width 0.035 nm) of the
 * positive and of the negative ion charge within rc, and Re, Im of exp(-i k_z Z_j) S1(k_z) for the 8
 * lowest k_z modes.  Parameters are one float vector (srbe_mlp_get_params gives its length):
 * W1[128][80], b1, W2[128][128], b2, W3[128], b3, input mean[80], input spread[80], target mean,
 * target spread; inputs and target are standardised by the last four. */
int srbe_mlp_init(srbe_ctx *ctx, uint64_t seed);
int srbe_mlp_get_params(srbe_ctx *ctx, float *params, int64_t *count);
int srbe_mlp_set_params(srbe_ctx *ctx, const float *params, int64_t count);
/* Descriptors [n_ele][80] of the current configuration; valid after a charge update or force call. */
int srbe_descriptors(srbe_ctx *ctx, float *D);
/* The unprojected solution y = Q - psi_bar A^-1 e [n_ele] of the last charge update (the target). */
int srbe_solution(srbe_ctx *ctx, double *y);
/* srbe_mlp_predict and the learned warm start run the forward pass on the tensor cores (tcgen05
 * kind::f16): both GEMMs with operands split into BF16 (hi, lo) pairs, hi hi + hi lo + lo hi products
 * and FP32 accumulation (about 16 significand bits). */
int srbe_mlp_predict(srbe_ctx *ctx, const float *D, int64_t n, float *out);
/* The same with device pointers D_dev [n][80] and out_dev [n], queued on the context's stream. */
int srbe_mlp_predict_dev(srbe_ctx *ctx, const float *D_dev, int64_t n, float *out_dev);
/* Gradient of the mean squared standardised error over n rows (no update); grad has the length of
 * the trainable part of the parameter vector (everything before the input mean). */
int srbe_mlp_gradients(srbe_ctx *ctx, const float *D, const float *target, int64_t n, float *grad, double *loss);
/* Sets the standardisation from the data, then epochs of shuffled minibatch AdamW (lr, decoupled
 * weight decay); returns the mean loss of the last epoch. */
int srbe_mlp_train(srbe_ctx *ctx, const float *D, const float *target, int64_t n, int epochs, int batch, float lr,
                   float weight_decay, uint64_t seed, double *final_loss);

/* ---- checks, tuning and the batching form (no counterpart in the paper) ---------------------------
 * srbe_charge_residual: relative FP64 residual of the constant-potential conditions met by the
 * charges of the last pass, ||A Q - dpsi d - b - psi_bar e|| / ||dpsi d + b|| (A Q = dpsi d + b +
 * psi_bar e follows from Eqs. 9-10), with A in FP64 whatever the precision of the solve.
 * srbe_set_skin / srbe_get_skin: Verlet-list skin (nm, default 0.1); lists hold pairs within rc +
 * skin and are rebuilt on the device once an ion has moved more than skin / 2.  Results do not
 * depend on the skin beyond summation order.
 * srbe_autotune_skin: times trial_steps MD steps (after two untimed ones) for each candidate skin,
 * restores positions, velocities, forces, charges and the step counter after each trial, keeps the
 * fastest skin and writes the per-candidate ms per step to ms_per_step (n_skins entries, or NULL). */
int srbe_charge_residual(srbe_ctx *ctx, double *rel_residual);

/* Lattice electrodes (an evaluation order of Eqs. 15 and 24, not a change of the method): when every
 * electrode layer (sites of equal z, at most 8 layers) is a full nx x ny rectangular lattice whose
 * spacing divides Lx and Ly (the same nx, ny in every layer; any in-plane origin per layer),
 * srbe_set_electrode recognises it and the electrode sums run through per-layer 2D discrete Fourier
 * transforms: S2(k) = sum_l e^{i k.(x0_l, y0_l, Z_l)} Qhat_l[m_x mod nx, m_y mod ny] and the far part
 * of b from the modes binned by (m_x mod nx, m_y mod ny), in FP64 in both precision forms.  The
 * results equal the plain per-site sums up to rounding.  The transforms cost a fixed handful of small
 * launches, so they only pay for large electrodes: srbe_set_lattice(ctx, mode) with mode 0 = never,
 * 1 = when N_ele x K >= 4e6 (the default), 2 = always (whenever the lattice is recognised).
 * srbe_lattice_info gives (layers, nx, ny), or zeros when the electrode is not such a lattice. */
int srbe_set_lattice(srbe_ctx *ctx, int mode);
int srbe_lattice_info(srbe_ctx *ctx, int32_t dims[3]);

/* Thermostat of Algorithm 1's integration step: the Langevin equation of Eq. 39, read with gamma as
 * a collision rate (1/ps): friction m gamma v and noise sqrt(2 m gamma kB T) dW per ion component.
 * srbe_step applies its exact Ornstein-Uhlenbeck solution over each step after the closing half
 * kick: v <- c1 v + sqrt((1 - c1^2) kB T / m) g, c1 = exp(-gamma dt), g standard normal from
 * Philox4x64-10 with key (seed, 0x4C414E47) and counter (step, ion, 0, 0) through Box-Muller (the
 * same numbers as any other implementation of that recipe; the mixed form takes the top 24 bits of
 * the same words as FP32 uniforms and transforms them in FP32).  gamma = 0 (the default) is plain
 * velocity Verlet.  Errors: SRBE_EINVAL for negative or non-finite gamma or T. */
int srbe_set_thermostat(srbe_ctx *ctx, double gamma, double T, uint64_t seed);
int srbe_set_skin(srbe_ctx *ctx, double skin);
double srbe_get_skin(const srbe_ctx *ctx);
int srbe_autotune_skin(srbe_ctx *ctx, int trial_steps, uint64_t seed, const double *skins, int n_skins,
                       double *ms_per_step);

/* Tile shape of the structure-factor kernel (S1, S2; no counterpart in the paper): the sum over
 * particles runs in chunks of whole 128-particle batches, as long as the grid keeps at least `occ`
 * blocks per SM (longer chunks amortise each block's closing reductions, shorter ones give more
 * blocks to hide latency with).  Default occ = 8.  Results do not depend on it beyond summation
 * order.  srbe_autotune_tiles times trial_steps MD steps (after two untimed ones) for each candidate
 * occ (1..64), restores the state after each trial as srbe_autotune_skin does, keeps the fastest and
 * writes the per-candidate ms per step to ms_per_step (n_occ entries, or NULL); srbe_set_tiles sets
 * it directly and srbe_get_tiles gives the setting in use.  Errors: SRBE_EINVAL (no candidates, occ
 * out of range, trial_steps < 1), SRBE_ESTATE (no MD state, srbe_autotune_tiles only). */
int srbe_autotune_tiles(srbe_ctx *ctx, int trial_steps, uint64_t seed, const int *occ, int n_occ,
                        double *ms_per_step);
int srbe_set_tiles(srbe_ctx *ctx, int occ);
int srbe_get_tiles(const srbe_ctx *ctx);

/* A batch steps many independent replicas (contexts of any size, electrode, voltage, precision,
 * solver and mode count, each with its own seed and so its own k-sample lists) as one unit: each
 * batch step is ONE CUDA graph launch that runs Algorithm 1's step for every replica, the replicas
 * spread over `width` streams inside the graph so that small systems overlap on the GPU.  The host
 * samples every replica's next mode list (over a few host threads) into mapped pinned slots while
 * the GPU runs the current step; one kernel at the head of the graph reads them all.  A replica's trajectory is bitwise the one srbe_step gives it with the same
 * seed.  Cooperative kernels of different replicas are ordered one after another inside the graph
 * (two overlapping grid-wide barriers could starve each other of SMs).
 *   srbe_batch_create: ctxs are borrowed (the caller keeps and destroys them, after the batch);
 *     all on the current device, distinct; default width min(n, 16).
 *   srbe_batch_step: nsteps steps, seeds[n] (replica r's modes of step t come from (seeds[r], t)).
 *     The first step after creation, a width change or any state-changing call on a replica runs
 *     the ordinary way and recaptures.  residuals (n entries, or NULL) receives each replica's
 *     srbe_charge_residual after the last step: the FP64 check of the FP32 bulk of mixed replicas.
 *     The call returns once the work is queued; each replica's own stream is ordered after it.
 *   srbe_batch_set_width: streams inside the graph (0: one stream, replicas in order).
 *   srbe_batch_autotune: for each candidate width, times trial_steps batch steps (after two
 *     untimed ones), restores every replica's state (as srbe_autotune_skin does) and keeps the
 *     fastest width; ms_per_step (n_widths entries, or NULL) receives the timings.
 *   srbe_batch_autotune_tiles: the same for the structure-factor tile (srbe_autotune_tiles' occ),
 *     one setting for every replica (each replica's chunk length then follows its own size).
 * Errors: SRBE_EINVAL (bad arguments), SRBE_ESTATE (a replica without electrode, positions or MD
 * state, or with phase tracing on), SRBE_ECUDA (capture or launch failed), SRBE_ENOMEM;
 * srbe_batch_last_error gives the message. */
typedef struct srbe_batch srbe_batch;
int srbe_batch_create(int n, srbe_ctx *const *ctxs, srbe_batch **out);
int srbe_batch_destroy(srbe_batch *batch);
const char *srbe_batch_last_error(const srbe_batch *batch);
int srbe_batch_set_width(srbe_batch *batch, int width);
int srbe_batch_get_width(const srbe_batch *batch);
/* the batch's own stream (cudaStream_t as void*), on which every batch step is launched */
void *srbe_batch_stream(const srbe_batch *batch);
int srbe_batch_step(srbe_batch *batch, int nsteps, const uint64_t *seeds, double *residuals);
int srbe_batch_autotune(srbe_batch *batch, int trial_steps, const uint64_t *seeds, const int *widths, int n_widths,
                        double *ms_per_step);
int srbe_batch_autotune_tiles(srbe_batch *batch, int trial_steps, const uint64_t *seeds, const int *occ, int n_occ,
                              double *ms_per_step);

/* Test aid (no counterpart in the paper): from the next pass on, overwrite one entry of the output
 * with a NaN right after it is computed and before the non-finite check runs: what = 1 the force
 * F[0], 2 the charge Q[0], 0 stops it.  It exists so that the reporting of SRBE_ENONFINITE can be
 * tested without driving a trajectory to divergence. */
int srbe_debug_inject_nonfinite(srbe_ctx *ctx, int what);

/* Structure factor without any device allocation (the paper has no counterpart; an interface
 * for callers that cannot allocate device memory, e.g. an MD engine that hands out every byte of
 * GPU memory from its own pool, or code that must not allocate while its pipeline runs).
 * Computes S(k) = sum_j w_j exp(i k . r_j) in FP64 for
 *   box      host [3]: periodic lengths (nm), k = 2 pi m / L componentwise
 *   r_dev    device [n][3] positions, w_dev device [n] weights (charges), n >= 0
 *   m_dev    device [K][3] integer modes, 0 <= K <= 8192
 *   S_dev    device [K][2] output (re, im), overwritten
 *   stream   cudaStream_t as void* (NULL: legacy default stream); the call is asynchronous
 * Partial sums go to one fixed 2 MiB array (131072 double2) compiled into the library, next to a
 * 16 KiB sin/cos table; every GPU that loads the library holds both until the process exits.
 * The first call on each device does its set-up (looks up the arrays' device addresses, copies
 * the table in, waits for the device to finish that copy and loads the kernels, with that device
 * current), so make that first call before any stream capture; it may come on any stream.  Every call shares the array and leaves its partials there; each partial is written
 * before it is read, so nothing has to be cleared, but calls that overlap on the GPU race on it.
 * Allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 * Errors: SRBE_EINVAL (bad box, n < 0, K outside [0, 8192], null pointers), SRBE_ECUDA. */
int srbe_structure_factor_noalloc(const double box[3], int64_t n, const double *r_dev, const double *w_dev, int K,
                                  const int32_t *m_dev, double *S_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SRBE_H */
