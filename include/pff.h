/*
 * pff.h -- C ABI of the B300 (sm_103a) matrix-free phase-field fracture step.
 *
 * The library computes the hot path of the explicit-dynamic phase-field
 * method of arxiv 2606.23458: the P1 element kernel (strain, energy split,
 * degraded stress, history), deterministic internal-force accumulation, the
 * lumped-mass velocity-Verlet update, and the staggered damage solve (AT2 by
 * Jacobi-preconditioned CG with post-clamp, AT1 by projected CG), plus the
 * implicit-differentiation backward for dL/dGc.
 *
 * Conventions for every entry point:
 *  - Units are SI (m, Pa, kg/m^3, J/m^2, s); energies are per unit thickness.
 *  - Host pointers are marked "host"; all other buffers are device pointers
 *    owned by the caller, contiguous, and typed by the mesh precision:
 *      PFF_FP64       : u, v, a (N x 2, x/y interleaved), d (N) are double;
 *      PFF_FP32_MIXED : u, v, a, d are float.
 *    The history H (Ne) is always double.
 *  - Calls are ordered on the given cudaStream_t and asynchronous, except
 *    where a call returns host scalars (then it synchronises that stream).
 *  - No call throws; every call returns a pff_status.  pff_last_error()
 *    returns a thread-local message for the last failure.
 *  - Deterministic: force and damage-operator accumulation use a
 *    node-to-element gather in ascending element order (no float atomics);
 *    reductions use fixed-order block partial sums.  Two runs on the same
 *    device give bit-identical results.
 */
#ifndef PFF_H
#define PFF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *pff_stream; /* same handle as cudaStream_t */

typedef enum {
  PFF_OK = 0,
  PFF_ERR_ARG = 1,            /* invalid argument (null, size, enum) */
  PFF_ERR_MESH = 2,           /* inverted/degenerate element or bad index */
  PFF_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  PFF_ERR_OOM = 4,            /* device allocation failed */
  PFF_ERR_NOT_CONVERGED = 5,  /* CG hit its iteration/restart cap; the last
                                 iterate is still written */
  PFF_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
  PFF_ERR_NONFINITE = 7       /* NaN/Inf met in a reduction */
} pff_status;

enum { PFF_AT1 = 1, PFF_AT2 = 2 };
enum { PFF_SPLIT_SPECTRAL = 0, PFF_SPLIT_AMOR = 1, PFF_SPLIT_ISO = 2 };
enum { PFF_PLANE_STRAIN = 0, PFF_PLANE_STRESS = 1 };
enum { PFF_FP64 = 0, PFF_FP32_MIXED = 1 };
enum { PFF_LOOP_GRAPH = 0, PFF_LOOP_HOST = 1 };
enum { PFF_CG_AUTO = 0, PFF_CG_PHASES = 1, PFF_CG_PERSISTENT = 2, PFF_CG_TEST_TIMEOUT = 3,
       PFF_CG_STAGED = 4, PFF_CG_FUSED = 5, PFF_CG_FUSED_STAGED = 6, PFF_CG_RESIDENT = 7 };

typedef struct pff_mesh pff_mesh; /* opaque; owns geometry, CSR, workspaces */

/* Material (Sec. 2.1 of the paper; Table 1 gives the benchmark values).
 * model: PFF_AT1 | PFF_AT2 (crack density, Sec. 2.1);
 * split: spectral (Eq. spectral_split), volumetric-deviatoric (Eq.
 *        amor_split) or isotropic (psi+ = psi);
 * plane: PFF_PLANE_STRAIN (lambda_PE = E nu / ((1+nu)(1-2nu))) or
 *        PFF_PLANE_STRESS (lambda_PS = E nu / (1-nu^2); the
 *        volumetric-deviatoric split keeps the 3-D bulk modulus and adds
 *        e_zz = -nu/(1-nu) tr to the 3-D trace, Sec. 2.1 plane assumptions);
 * eta: residual stiffness in g(d) = (1-d)^2 + eta. */
typedef struct {
  double E, nu, rho, Gc, l0, eta;
  int32_t model, split, plane, reserved;
} pff_material;

/* Solver options.  Zero-initialise and set what you need; zero fields take
 * the defaults given in brackets. */
typedef struct {
  double cg_tol;        /* ||r||_2 <= cg_tol * ||b_eff||_2 (Sec. 2.4) [1e-8] */
  int32_t cg_max_it;    /* CG iterations per solve (all restarts) [10000] */
  int32_t max_restarts; /* AT1 projected-CG restarts [50] */
  double t_ramp;        /* traction ramp S(t), Eq. smooth_traction_ramp [5e-8 s] */
  int32_t energy_every; /* pff_run: energies every k steps, 0 = off [0] */
  int32_t ckpt_every;   /* pff_backward: checkpoint period [25] */
  int32_t block;        /* threads per block, 0 = autotuned [0] */
  int32_t loop_mode;    /* PFF_LOOP_GRAPH (device-side CG loop in a CUDA
                           graph) or PFF_LOOP_HOST (host polls) [graph] */
  int32_t variant;      /* gather schedule of the force / damage kernels:
                           0 = autotuned on first use [0]; 1 = entry-parallel
                           node blocks (force: an element pass, then a node
                           gather); 2..5 = node-centric with 1..4 gathers
                           in flight.  Every row sums in the same order:
                           bit-identical results in FP32; in FP64 the
                           mechanics are bit-identical and the damage
                           solve's FP64 dot products may differ in the
                           last bit with the summation order. */
  int32_t cg_kernel;    /* AT2 CG loop: PFF_CG_PHASES = a matvec and an
                           update kernel per iteration; PFF_CG_PERSISTENT =
                           the whole solve in one cooperative kernel (all
                           CTAs resident, grid barriers with bounded waits,
                           PFF_ERR_TIMEOUT if one gives up);
                           PFF_CG_STAGED = the same kernel with each CTA's
                           element records and history copied into shared
                           memory once per solve (FP32 meshes whose CTA
                           sets fit, else as PFF_CG_PERSISTENT);
                           PFF_CG_FUSED = one cooperative kernel running the
                           single-reduction (Chronopoulos-Gear) form of the
                           same Jacobi PCG: one pass and one grid
                           all-reduce per iteration (FP32; FP64 meshes use
                           the kernel-per-phase loop);
                           PFF_CG_FUSED_STAGED = that with the operator
                           staged in shared memory;
                           PFF_CG_RESIDENT = the single-reduction CG with
                           each CTA owning a contiguous range of rows whose
                           x, p, diagonal and fan tables stay in shared
                           memory for the whole solve, and where the rows
                           fit 108 B each their coefficients and records
                           too (FP32 element-wise operator in fan order,
                           rows fitting at least 28 B each; else as
                           PFF_CG_FUSED);
                           PFF_CG_AUTO = the fastest on this mesh, timed on
                           first use [0].
                           Same iteration arithmetic; the forms group the
                           partial sums of the dot products differently.
                           AT1 always uses the kernel-per-phase loop.
                           PFF_CG_TEST_TIMEOUT: the persistent loop awaits
                           one arrival more than it launches, so its first
                           barrier wait gives up after its 2 s limit and the
                           call reports PFF_ERR_TIMEOUT (a test of the
                           bounded wait; the result is not usable). */
  int32_t damage_every; /* pff_run: damage subcycling N_sub (Sec. 2.4): the
                           damage problem is solved only after steps n with
                           (n + 1) % N_sub == 0 (n counted from 0 at step 0,
                           not from step0); the history H is still updated
                           every step; d stays d_n in between and those
                           steps log 0 iterations.  0 or 1: every step [0].
                           See pff_subcycling_limit for the admissible value.
                           Not supported by pff_run_ckpt / pff_batch_run
                           (PFF_ERR_ARG). */
  int32_t fuse;         /* a step's internal force and damage right-hand
                           side: 0 = one fused kernel if the autotuner timed
                           it faster than the two, 1 = two kernels, 2 = the
                           fused kernel (same results either way: each
                           element's history max is taken the way the force
                           kernel stores it) [0] */
} pff_options;

/* Device state of one plate (caller-owned). */
typedef struct {
  void *u, *v, *a; /* N x 2 displacement, velocity, acceleration */
  void *d;         /* N damage */
  double *H;       /* Ne history max of psi+ (per element) */
} pff_state;

/* Builds a mesh on the current device from host arrays (copied).
 *  xy     host, N x 2 node coordinates (double);
 *  tri    host, Ne x 3 counter-clockwise P1 connectivity (int32, 0-based);
 *  notch  host, N flags (nullable): damage held at d = 1 there (Dirichlet);
 *  tedges host, M x 2 loaded boundary edges; tvec host, M x 2 traction (Pa)
 *         on each edge; the consistent P1 edge load gives half the edge
 *         force to each end node;
 *  precision: PFF_FP64 or PFF_FP32_MIXED.
 * Geometry per Eq. (grad_phi) (Sec. 2.3): areas, shape gradients, the
 * node-to-element incidence (for node i: (e << 2) | slot, ascending e) and
 * the minimum incircle diameter are computed by device kernels.
 * Errors: PFF_ERR_ARG (sizes, Ne >= 2^29), PFF_ERR_MESH (A_e <= 0 or an
 * index outside [0, N); pff_last_error names the element), PFF_ERR_OOM. */
pff_status pff_mesh_create(int64_t N, const double *xy, int64_t Ne,
                           const int32_t *tri, const uint8_t *notch, int64_t M,
                           const int32_t *tedges, const double *tvec,
                           int32_t precision, pff_mesh **out);

void pff_mesh_destroy(pff_mesh *mesh);

/* Options of the quasi-static loop.  Defaults in brackets (also taken when
 * the pointer is NULL). */
enum { PFF_QS_KRYLOV_FP32 = 0, PFF_QS_KRYLOV_MESH = 1 };
typedef struct {
  double newton_tol;  /* Newton stop: |r_free| <= newton_tol |f_int| [1e-8] */
  int32_t newton_max; /* Newton steps per increment [25] */
  int32_t krylov;     /* precision of the tangent CG (its vectors and the
                         stored element tangents): PFF_QS_KRYLOV_FP32, or
                         PFF_QS_KRYLOV_MESH for the mesh's precision.  Under
                         an FP64 mesh FP32 is mixed-precision refinement:
                         the state and the Newton residual stay FP64. [FP32] */
  double eta_min;     /* forcing term of the inexact Newton step: the CG of a */
  double eta_max;     /* step stops at |r_cg| <= eta |r|, eta = clamp(0.1
                         newton_tol |f_int| / |r|, eta_min, eta_max).  With
                         FP32 CG vectors eta_min is the attainable reduction
                         per step. [1e-4 with FP32 CG, else 0; 0.5] */
  int32_t cg_max_it;  /* CG iterations per Newton step [100000] */
  int32_t pad;
} pff_qs_options;

/* Quasi-static staggered loop (Sec. 3.5, e.g. single-edge-notched
 * tension), nincr load increments: increment k puts u_y = (incr0 + k + 1) du
 * on the loaded nodes, then solves the mechanics f_int(u; d) = 0 on the free
 * dofs by inexact Newton iterations (qopt), each linear step
 * K_T(u) du = -r by Jacobi-PCG with the tangent action of Eq.
 * matrix_free_tangent_action (the internal force's derivative along the
 * trial vector through the split's tangent; the element's A C_T is
 * evaluated once per Newton step), then H = max(H, psi+(u)) and the damage
 * solve of pff_damage_solve (opt's tolerance; d_prev = d).  state: u, d, H
 * on the device, updated in place (v, a unused).  bc (host, N bytes): 1 =
 * u_x fixed at 0, 2 = u_y fixed at 0, 4 = loaded (u_y = U).  reaction
 * (host, nincr, nullable): sum of f_int,y over the loaded nodes at the
 * converged u (per unit thickness).  iters (host, nincr x 3, nullable):
 * Newton steps, mechanics CG iterations, damage CG iterations.  Allocates
 * its workspace (N x 49 + Ne x 88 bytes with FP32 CG) and frees it before
 * returning; synchronises the stream.  PFF_ERR_ARG for options out of
 * range (eta_min < 0, eta_max < eta_min or >= 1, newton_tol <= 0);
 * PFF_ERR_NOT_CONVERGED if a Newton loop, mechanics CG or damage solve hit
 * its cap (the increments still complete). */
pff_status pff_qs_run(pff_mesh *mesh, const pff_state *state, const uint8_t *bc, int64_t incr0,
                      int32_t nincr, double du, const pff_qs_options *qopt, const pff_options *opt,
                      double *reaction, int32_t *iters, pff_stream stream);

/* Toughness field (Secs. 4.2 and 7: the field-valued inverse): per-element
 * Gc_e (host, Ne doubles, each > 0 and finite; NULL restores the material's
 * uniform Gc) in place of Gc in the damage operator, its right-hand side and
 * the fracture energy.  Call after pff_mesh_set_material; the field is kept
 * as Gc_e / Gc and follows later material changes.  While a field is set
 * the shared-memory staged CG loops are not used.  Copies synchronously.
 * PFF_ERR_ARG: null mesh, no material yet, a non-positive value. */
pff_status pff_mesh_set_gc_field(pff_mesh *mesh, const double *gc);

/* Form in which the damage operator A = sum_e [kappa_e K^e + c_e M^e]
 * (Eqs. damage_pde_at2 / damage_pde_at1 with the consistent mass, Sec. 2.4)
 * is applied by every CG product of the damage solve (and of its adjoint,
 * and by the quasi-static tangent CG for the element tangents):
 *  PFF_OP_ELEMENT (default): matrix-free in the sense of Eq.
 *    matrix_free_fe_operator -- each product gathers p on every element
 *    and applies that element's own coefficients; no two elements'
 *    coupling coefficients are ever added together.  The coefficients of
 *    an element (they depend on H, which is fixed while a solve runs) are
 *    evaluated once per solve by the right-hand-side pass and kept per
 *    incidence entry (row a of element e: the coefficients of p_b and p_c,
 *    FP32 or FP64 with the mesh; the row's own terms sum_e A^e_aa p_a are
 *    applied as diag_a p_a through the Jacobi diagonal the preconditioner
 *    needs anyway).  On conforming meshes whose vertex fans have at most six
 *    triangles the entries are stored in fan order (triangle k of a vertex
 *    couples its neighbours v_k and v_{k+1}), so a row gathers each
 *    distinct neighbour once; other meshes keep incidence order with 16-bit
 *    neighbour offsets, and FP64 meshes too wide for those one 64-byte
 *    record per element from which every product evaluates whole element
 *    rows.
 *  PFF_OP_MERGED: the two elements' coefficients of each mesh edge summed
 *    once per solve into one coefficient per distinct neighbour -- the
 *    solve's sparse operator assembled in an ELL layout and thrown away
 *    after the solve (fewer bytes per product; FP32 roundings differ).
 *    Only on meshes whose rows have at most 8 distinct neighbours and whose
 *    elements span fewer than 2^15 node ids (PFF_ERR_ARG otherwise).
 * Changing the form drops the mesh's step graphs and its CG autotuning
 * (re-timed on the next solve).  Host-only; no device work. */
enum { PFF_OP_ELEMENT = 0, PFF_OP_MERGED = 1 };
pff_status pff_mesh_set_operator(pff_mesh *mesh, int32_t form);
/* The form in use, whether PFF_OP_MERGED is available, and whether the
 * element-wise entries are stored in fan order (1) or incidence order (0)
 * (host outputs, each nullable). */
pff_status pff_mesh_get_operator(const pff_mesh *mesh, int32_t *form, int32_t *merged_available,
                                 int32_t *fan_order);

/* Sets the material: the plane model's Lame constants (Sec. 2.1), lumped mass
 * m_i = rho sum A_e / 3 and the stable step dt = cfl * h_min / c_p with
 * c_p = sqrt((lambda + 2 mu) / rho) (velocity-Verlet paragraph, Sec. 2.3).
 * dt_out (host, nullable) receives that step.  Synchronises internally. */
pff_status pff_mesh_set_material(pff_mesh *mesh, const pff_material *mat,
                                 double cfl, double *dt_out);

/* Host copies for inspection (each output nullable):
 *  N, Ne, h_min, precision; */
pff_status pff_mesh_info(const pff_mesh *mesh, int64_t *N, int64_t *Ne,
                         double *hmin, int32_t *precision);
/*  ptr (N+1) and ent (3 Ne) incidence, int32; */
pff_status pff_mesh_get_csr(const pff_mesh *mesh, int32_t *ptr, int32_t *ent);
/*  area (Ne), grad (Ne x 3 x 2), fext (N x 2 full-scale load), minv (N)
 *  converted to double (minv needs pff_mesh_set_material first). */
pff_status pff_mesh_get_geometry(const pff_mesh *mesh, double *area,
                                 double *grad, double *fext, double *minv);

/* One explicit step n -> n+1 without the damage solve (Sec. 2.2, Eqs.
 * vv_u, vv_a, vv_v): u += dt v + dt^2/2 a; f = internal force at the new u
 * with the current d; H_e = max(H_e, psi+_e); a = (S(t_next) f_ext - f)/m;
 * v += dt/2 (a_old + a_new).  In place on state.  Asynchronous. */
pff_status pff_step_explicit(pff_mesh *mesh, const pff_state *state,
                             double t_next, double dt, const pff_options *opt,
                             pff_stream stream);

/* Staggered damage solve with history H (Sec. 2.4):
 *  AT2: Eq. (damage_pde_at2) with consistent mass, notch nodes eliminated
 *       (x_D = 1), Jacobi-PCG from x0 = d_prev to cg_tol, then
 *       d_out = min(1, max(x, d_prev)), d_out = 1 on the notch;
 *  AT1: Eq. (damage_pde_at1) by projected CG on [d_prev, 1].
 * d_out may alias d_prev.  iters/relres/restarts (host, nullable) receive
 * the iteration count, ||r||/||b_eff|| and the AT1 restarts; this
 * synchronises the stream.  PFF_ERR_NOT_CONVERGED still writes d_out. */
pff_status pff_damage_solve(pff_mesh *mesh, const double *H, const void *d_prev,
                            void *d_out, const pff_options *opt, int32_t *iters,
                            double *relres, int32_t *restarts, pff_stream stream);

/* nsteps staggered steps (predictor, force, history, corrector, damage
 * solve) starting at step index step0 (t_n = n dt), in place on state.
 * The step sequence runs as one CUDA graph per step with the CG loop on
 * the device.  iters_log (device int32, nsteps x 2, nullable): per step
 * (CG iterations, AT1 restarts).  energy_log (device double, nsteps x 4,
 * nullable): E_el, E_kin, E_frac, W_ext after every opt->energy_every-th
 * step (other rows untouched).  Asynchronous; pff_sync_status() returns the
 * worst device status. */
pff_status pff_run(pff_mesh *mesh, const pff_state *state, int64_t step0,
                   int64_t nsteps, double dt, const pff_options *opt,
                   int32_t *iters_log, double *energy_log, pff_stream stream);

/* pff_run with the state resident in host memory: host holds u, v, a, d, H
 * in pinned host memory (the device layout and precision), dev the same
 * fields as device workspace (caller-owned, mesh precision).  Every step
 * copies the state in, runs the step of pff_run on dev, and copies it back
 * out; the copies of u, v, a and H back to the host start as soon as the
 * step's mechanics are done, overlapping the damage solve, and d follows
 * the clamp.  With a persistent CG loop the steps run in pipelined chunks
 * of eight (a step's copies in overlapping the previous step's solve).  The paper has no counterpart: this is the call for callers
 * whose state lives on the host between steps.  damage_every > 1 is
 * PFF_ERR_ARG.  iters_log as pff_run (device).  Asynchronous: host is
 * complete after the stream synchronises. */
pff_status pff_run_host(pff_mesh *mesh, const pff_state *host, const pff_state *dev,
                        int64_t step0, int64_t nsteps, double dt, const pff_options *opt,
                        int32_t *iters_log, pff_stream stream);

/* Checkpointed run and its adjoint (Sec. 4: implicit differentiation of the
 * damage solve, Eqs. implicit_forward_linear_system /
 * implicit_adjoint_linear_system / implicit_gc_l0_element_term, with
 * active-set masking; the reverse of the explicit mechanics; segment
 * checkpointing with recompute).
 * pff_ckpt_create: store for nsteps steps.  every = 0: full tape (Sec. 7,
 *   the whole activation tape in device memory): u, x, d (N each, mesh
 *   precision) and H (Ne doubles) of every step, about
 *   nsteps (4 sizeof(R) N + 8 Ne) bytes, and no recompute in the backward.
 *   every > 0: segments of `every` steps, device memory
 *   O(N (nsteps/every + every)) (checkpoints of u, v, a, d, H at each
 *   segment start, a per-step tape for one segment, adjoint state) for one
 *   extra forward pass in the backward.  PFF_ERR_OOM if it does not fit.
 * pff_run_ckpt: pff_run that also fills the tape or the checkpoints; nsteps
 *   must equal the store's.  iters_log as in pff_run.
 * pff_backward: given dL/dd at the final step (device, N, mesh precision),
 *   recomputes each segment from its checkpoint (bit-identical to the
 *   forward; skipped for a full tape), reverses the steps and returns
 *   dL/dGc (host) for the AT2 model.  One adjoint CG solve per step with warm start.  Synchronises
 *   the stream.  Errors: PFF_ERR_ARG (wrong mesh, unfilled store, AT1),
 *   PFF_ERR_NOT_CONVERGED / PFF_ERR_NONFINITE from an adjoint solve. */
typedef struct pff_ckpt pff_ckpt;
pff_status pff_ckpt_create(pff_mesh *mesh, int64_t nsteps, int32_t every, pff_ckpt **out);
/* pff_ckpt_create with a choice of what a checkpointed store (every > 0)
 * keeps between its segment checkpoints:
 *  PFF_CKPT_RECOMPUTE: nothing; the backward recomputes each segment in
 *    full, damage solves included (what pff_ckpt_create does);
 *  PFF_CKPT_DAMAGE_TAPE: the unclamped damage solution x_{n+1} of every
 *    step (nsteps x N values of the mesh precision, an eighth of the full
 *    tape in FP32); the backward recomputes each segment's mechanics only
 *    (predictor, force with history and corrector, then the clamp of the
 *    taped x, bit-identical to the forward) and no damage solve.
 * Ignored for every = 0 (the full tape).  PFF_ERR_ARG for another policy. */
enum { PFF_CKPT_RECOMPUTE = 0, PFF_CKPT_DAMAGE_TAPE = 1 };
pff_status pff_ckpt_create_policy(pff_mesh *mesh, int64_t nsteps, int32_t every, int32_t policy,
                                  pff_ckpt **out);
void pff_ckpt_destroy(pff_ckpt *ckpt);
/* Total adjoint CG iterations of the last pff_backward on this store. */
pff_status pff_ckpt_stats(const pff_ckpt *ckpt, int64_t *adjoint_iters);
pff_status pff_run_ckpt(pff_mesh *mesh, const pff_state *state, int64_t step0,
                        int64_t nsteps, double dt, const pff_options *opt,
                        pff_ckpt *ckpt, int32_t *iters_log, pff_stream stream);
pff_status pff_backward(pff_mesh *mesh, pff_ckpt *ckpt, const void *dL_dd,
                        const pff_options *opt, double *dL_dGc, pff_stream stream);

/* pff_backward that also returns dL/dGc_e per element (device, Ne doubles,
 * overwritten): the per-element terms of Eq. implicit_gc_l0_element_term
 * summed over the steps, the gradient of a toughness field (see
 * pff_mesh_set_gc_field); their sum is *dL_dGc. */
pff_status pff_backward_field(pff_mesh *mesh, pff_ckpt *ckpt, const void *dL_dd,
                              const pff_options *opt, double *dL_dGc, double *dL_dGc_field,
                              pff_stream stream);

/* Batches: many independent plates (uneven sizes, Gc, l0, loads and time
 * steps) advanced together, one CUDA graph launch per step for all plates,
 * with per-plate CG reductions and convergence (the CG loop of all plates
 * either as kernels per phase, a converged plate's blocks skipping the
 * remaining iterations, as one cooperative launch with a group of CTAs
 * per plate, or as a few such launches (waves of plates) with each CTA's
 * rows resident in shared memory; see pff_batch_tuning).  Plates share E, nu, rho, eta, the split
 * and the AT2 model.  The caller owns the concatenated state of
 * pff_batch_size's N nodes / Ne elements: plate p's nodes start at node0
 * (pff_batch_plate_info; a multiple of 256, padding nodes between plates
 * carry no elements and stay at rest), its elements at elem0.  Each plate's
 * dt = cfl * h_min / c_p of its own mesh.
 * pff_batch_run: nsteps staggered steps of every plate (step index step0 +
 * k of each plate's own clock); iters_log (device, nsteps x nplates,
 * nullable) receives each plate's CG iterations.  Asynchronous. */
typedef struct pff_batch pff_batch;
typedef struct {
  int64_t N;              /* nodes */
  const double *xy;       /* host N x 2 */
  int64_t Ne;             /* elements */
  const int32_t *tri;     /* host Ne x 3, 0-based within the plate */
  const uint8_t *notch;   /* host N, nullable */
  int64_t M;              /* loaded edges */
  const int32_t *tedges;  /* host M x 2 */
  const double *tvec;     /* host M x 2 traction, Pa */
  pff_material mat;
} pff_plate;
pff_status pff_batch_create(int32_t nplates, const pff_plate *plates, int32_t precision,
                            double cfl, pff_batch **out);
void pff_batch_destroy(pff_batch *batch);
/* The batch's loop configuration (host outputs, each nullable):
 * choice[6] = gathers in flight of the force kernel, of the right-hand side,
 * the CG loop form (PFF_CG_PHASES: a matvec and an update kernel per
 * iteration for all plates in a device loop; PFF_CG_PERSISTENT: one
 * cooperative launch in which each plate's group of CTAs iterates its own
 * plate to its own stop; PFF_CG_RESIDENT: the same single-reduction loop
 * as the one-mesh resident family, on FP32 batches with fan-order rows, in
 * waves of consecutive plates whose rows fit the SMs' shared memory
 * together, one cooperative launch per wave, each plate's CTAs owning
 * contiguous row ranges), that loop's gathers in flight (the resident
 * loop's CTA shape), 1 once the autotuner has run, and the persistent
 * launch's CTAs (0: unavailable).
 * ms[3 x 12]: the autotuner's timings -- force U = 1..4, right-hand side
 * U = 1..4, a right-hand side plus a whole solve for the phases loop with
 * U = 1..4, the persistent loop with U = 2..4 and the resident loop with
 * U = 1..4 (0 where not timed).  The autotuner runs at the first
 * pff_batch_run unless pff_options.variant fixes the gathers;
 * pff_options.cg_kernel PFF_CG_PHASES, PFF_CG_PERSISTENT or
 * PFF_CG_RESIDENT forces the loop form (the resident loop falls back to
 * the persistent one where it is unavailable). */
pff_status pff_batch_tuning(const pff_batch *batch, int32_t *choice, float *ms);
/* pff_mesh_set_operator for every plate of the batch (the same forms and
 * conditions; PFF_OP_ELEMENT by default); the batch is re-tuned. */
pff_status pff_batch_set_operator(pff_batch *batch, int32_t form);
pff_status pff_batch_size(const pff_batch *batch, int64_t *N, int64_t *Ne);
pff_status pff_batch_plate_info(const pff_batch *batch, int32_t plate, int64_t *node0,
                                int64_t *N, int64_t *elem0, int64_t *Ne, double *dt);
pff_status pff_batch_run(pff_batch *batch, const pff_state *state, int64_t step0, int64_t nsteps,
                         const pff_options *opt, int32_t *iters_log, pff_stream stream);

/* Synchronises the stream and returns (and clears) the worst status the
 * device recorded since the last call (not converged, non-finite, timeout). */
pff_status pff_sync_status(pff_mesh *mesh, pff_stream stream);

/* Energies per unit thickness (Sec. 3.1): out[0] = E_el = sum A_e psi,
 * out[1] = E_kin = 1/2 sum m |v|^2, out[2] = E_frac = Gc int gamma(d).
 * out is host; synchronises the stream. */
pff_status pff_energies(pff_mesh *mesh, const pff_state *state, double *out,
                        pff_stream stream);

/* Measurement helper: average device time (ms) of each kernel of the step
 * on this mesh's data, ms_out[0..6] = predictor, force/corrector, damage
 * right-hand side, CG matvec, CG update, clamp/finish, energies; when the
 * AT2 solve runs as one persistent launch (pff_mesh_cg_choice),
 * ms_out[7] = that launch after one mechanics step, ms_out[8] = its CG
 * iterations, ms_out[9] = its family (0 phases, 1 persistent, 2 staged,
 * 3 fused, 4 fused staged; ms_out[7..8] = 0 for phases); ms_out[10] = the
 * fused force and right-hand-side kernel, ms_out[11] = 1 if steps use it.
 * Every timed launch is preceded by a write larger than L2 and bracketed
 * by CUDA events on `stream`; reps launches per kernel.  It OVERWRITES the
 * state and the solve workspace (call it after the run whose numbers you
 * need).  Synchronises the stream.  ms_out holds 12 doubles. */
pff_status pff_profile_kernels(pff_mesh *mesh, const pff_state *state, double dt,
                               const pff_options *opt, int32_t reps, double *ms_out,
                               pff_stream stream);

/* Gather schedules in use for (force, damage right-hand side, CG matvec)
 * as pff_options.variant codes (1..5), and the autotuner's timings in ms
 * (3 x 5, 0 where not measured).  Host outputs, each nullable. */
pff_status pff_mesh_schedule(const pff_mesh *mesh, int32_t *variant, float *tune_ms);

/* The fused internal force and damage right-hand side (Sec. 2.2-2.4: one
 * node-centric pass computing the force of Eq. vv_a with the history update
 * and the set-up of the damage solve of Eq. damage_pde_at2/at1): *variant =
 * the pff_options.variant code in use (1..5: U = 2, 1, 2, 3, 4 entries in
 * flight; every variant gives the same bits), tune_ms[5] = the autotuner's
 * time per variant (0 where not measured).  Whether a step uses the fused
 * kernel at all is ms_out[11] of pff_profile_kernels.  Host outputs, each
 * nullable. */
pff_status pff_mesh_fused_schedule(const pff_mesh *mesh, int32_t *variant, float *tune_ms);

/* The AT2 CG loop the autotuner chose on this mesh: *cg_kernel =
 * PFF_CG_PHASES, _PERSISTENT, _STAGED, _FUSED, _FUSED_STAGED or _RESIDENT
 * (PFF_CG_AUTO while not yet timed), the chosen persistent kernel's variant
 * (1..4: gathers in flight, or the resident kernel's CTA shape; 0 for
 * phases), and ms[6]: 30 iterations of the kernel-per-phase
 * loop and of the best variant of each persistent kernel in that order (0
 * if not timed or not available).  Host outputs; each pointer nullable. */
pff_status pff_mesh_cg_choice(const pff_mesh *mesh, int32_t *cg_kernel, int32_t *gathers, float *ms);

/* Which form of the resident loop (PFF_CG_RESIDENT) each of its CTA shapes
 * U = 1..4 runs on this mesh: forms[U - 1] = -1 unavailable (no fan order,
 * FP64, or the rows do not fit shared memory), 0 partial (x, p, the
 * diagonal and the fan words resident), 1 full (the coefficients and both
 * CG record buffers resident as well).  Fixed at mesh creation and by
 * pff_mesh_set_operator.  forms is host, 4 entries. */
pff_status pff_mesh_resident_forms(const pff_mesh *mesh, int32_t *forms);

/* The damage solve of pff_damage_solve, for callers that must not allocate
 * device memory during the call.  The paper has no counterpart of this entry
 * point.  Who needs it: cudaFree synchronises the whole device and the
 * allocator may not be entered from every context, so a memory-capped
 * serving process that owns the device pool, code running inside an
 * allocator or stream callback, or a latency-critical loop cannot use the
 * regular call, whose first use per mesh allocates (autotuning, CUDA graph).
 * This call allocates nothing (no cudaMalloc / cudaFree, no allocating
 * library routine); the caller still passes H, d_prev and d_out (device),
 * and the mesh must already exist (pff_mesh_create allocates).
 *  - Workspace: a statically reserved __device__ array of about 9 MiB inside
 *    libpff.so, which every GPU that loads the library holds until the
 *    process exits.  It fits meshes of at most 131,072 nodes and 262,144
 *    elements; larger meshes return PFF_ERR_ARG with a message.
 *  - The first call on each device looks up that array's device address
 *    (cudaGetSymbolAddress) with the mesh's device current; make that first
 *    call before any stream capture.
 *  - Every call shares the one array and leaves its workspace there; calls
 *    that overlap on the GPU (unordered streams, other host threads) race
 *    and corrupt each other's results.  Like every damage solve, it also
 *    writes the mesh's own per-solve operator records and Jacobi diagonal
 *    (allocated with the mesh), so it races as well with any other solve
 *    on the same mesh (pff_damage_solve, pff_run, ...) that overlaps it on
 *    the GPU.  Order them on one stream.
 *  - The CG loop is host-polled (no CUDA graph) and uses the mesh's current
 *    gather schedule (no autotuning).  Same arguments, results and status
 *    codes as pff_damage_solve; synchronises the stream. */
pff_status pff_damage_solve_noalloc(pff_mesh *mesh, const double *H,
                                    const void *d_prev, void *d_out,
                                    const pff_options *opt, int32_t *iters,
                                    double *relres, int32_t *restarts,
                                    pff_stream stream);

/* Pre-simulation check of the damage subcycling factor (Sec. 2.4): the
 * damage front moves at most at about 0.6 c_R while the explicit step is set
 * by the dilatational wave speed c_p, so N_max = floor(c_p / (0.6 c_R)).
 * c_p = sqrt((lambda + 2 mu) / rho) with the plane model's lambda (the
 * speed of the CFL step), c_R the Rayleigh wave speed of the same plane
 * model.  Host-only (no device work); ratio and n_max nullable.
 * PFF_ERR_ARG for a non-physical material (E <= 0, rho <= 0, nu outside
 * (-1, 0.5), unknown plane). */
pff_status pff_subcycling_limit(const pff_material *mat, double *ratio, int32_t *n_max);

/* Message of the last failing call on this host thread. */
const char *pff_last_error(void);
const char *pff_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PFF_H */
