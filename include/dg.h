/*
 * dg.h -- C ABI of the GB300 matrix-free modal DG + p-multigrid FGMRES library.
 *
 * Method: Franciolini, Fidkowski & Crivellini, "Efficient discontinuous Galerkin
 * implementations and preconditioners for implicit unsteady compressible flow
 * simulations" (arXiv 1812.04789).  Every entry point cites the passage that
 * defines the operation it computes.
 *
 * Conventions for every call
 *  - Pointers named as device pointers are CUDA device memory owned by the
 *    caller, contiguous, FP64, laid out W[e][v][i]: element e (e = i0 + n0*(i1 +
 *    n1*i2)), conservative variable v = 0..m-1 (rho, rho*v_1..rho*v_d, rho*e0;
 *    m = d + 2), modal coefficient i = 0..n_m-1 of the orthonormal total-degree
 *    Legendre basis ordered by degree, then lexicographically with the first
 *    index descending.  n_m = C(p + d, d).
 *  - Host pointers (descriptors, options, statistics) are read or written
 *    during the call only; the library keeps no reference to them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Calls are asynchronous on that stream unless stated otherwise.
 *  - The return value reports argument validation and launch errors at call
 *    time.  Outcomes found on the device (non-physical states, Krylov
 *    breakdown) are recorded in a per-mesh device status word read by
 *    dg_status_sync(), and by dg_fgmres_step() in its statistics.
 *  - Handles own their device workspace (basis tables, face slots, blocks,
 *    Krylov bases); it is allocated by the create/setup calls, never during
 *    residual, JVP, apply or solve calls.  A handle is not safe for concurrent
 *    use from several host threads or several streams at once.
 *  - There is no CPU fallback: without a CUDA device every call returns
 *    DG_ERR_CUDA.
 */
#ifndef DG_H
#define DG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_INVALID = 1,        /* bad argument: null handle/pointer, bad size or option */
  DG_ERR_OOM = 2,            /* device allocation failed in a create/setup call */
  DG_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
  DG_ERR_NONPHYSICAL = 4,    /* rho <= 0 or p <= 0 met at a quadrature point */
  DG_ERR_NOT_CONVERGED = 5,  /* FGMRES stopped at its iteration limit above tolerance */
  DG_ERR_BREAKDOWN = 6,      /* singular element block, or non-finite Krylov scalar */
  DG_ERR_TIMEOUT = 7,        /* a bounded device wait ran out */
  DG_ERR_UNSUPPORTED = 8     /* valid request the library does not implement */
} dg_status;

/* Periodic structured mesh of boxes on [lo, hi] (quads for dim 2, hexes for
 * dim 3) with n[k] elements per direction, polynomial degree p (0..8) and nq1d
 * Gauss-Legendre points per direction on volumes and faces (0 => p + 2).
 * space: DG_SPACE_P, orthonormal Legendre products of total degree <= p
 * (C(p+d, d) modes), or DG_SPACE_Q, the tensor-product space of degree <= p in
 * each direction ((p+1)^d modes; the paper's quadrilateral basis, Sec. 3).
 * Modes are ordered by degree (total for P, largest one-dimensional for Q),
 * then lexicographically with the first index descending, so the leading
 * modes of a level span every lower level of the same space (Sec. 6.1).
 * Sec. 3 (broken space, eq. BSpace) and Sec. 3.1 (DG discretisation). */
#define DG_SPACE_P 0
#define DG_SPACE_Q 1
typedef struct {
  int dim;
  int n[3];
  double lo[3], hi[3];
  int p;
  int nq1d;
  int space;
} dg_mesh_desc;

/* Gas and discretisation constants (Sec. 2 closure; Sec. 3.1): ratio of specific
 * heats, Prandtl number, constant viscosity, gas constant, BR2 penalty eta_F
 * (must exceed the number of element faces; 0 => 2*dim + 1) and the Roe
 * entropy-fix fraction (|lambda| smoothed below roe_delta * c; 0 = plain Roe). */
typedef struct {
  double gamma, Pr, mu, Rgas, eta_br2, roe_delta;
} dg_physics;

typedef struct dg_mesh_s* dg_mesh;
typedef struct dg_pmg_s* dg_pmg;

/* Build the mesh handle: face-neighbour maps, basis/quadrature tables in FP64
 * and FP32 on the device, face-slot workspace.  Blocks until the tables are
 * uploaded.  Errors: DG_ERR_INVALID (dim not 2/3, n < 1, p out of range,
 * hi <= lo, nq1d < p + 1), DG_ERR_OOM, DG_ERR_CUDA.  *out is NULL on error. */
dg_status dg_mesh_create(const dg_mesh_desc* desc, const dg_physics* phys, void* stream,
                         dg_mesh* out);
dg_status dg_mesh_destroy(dg_mesh mesh);

/* A periodic triangulation of the box [lo, hi]^2 with the full-order space
 * P_p on every triangle (Sec. 3: total degree <= k on triangular grids; the
 * quadrilateral grids of Sec. 7.2 split into triangles).  Host inputs, read
 * during the call: X[n_vert][2] vertex coordinates; tri[n_tri][3] vertex ids
 * of each triangle, counter-clockwise; shift[n_tri][3][2] integer lattice
 * shifts, corner k of triangle e at X[tri[e][k]] + shift[e][k] * (hi - lo).
 * Edges are matched by their vertex pair and relative shift: every edge must
 * belong to exactly two triangles (periodic, no boundary).  Basis:
 * orthonormal Dubiner polynomials on the reference triangle (-1,-1), (1,-1),
 * (-1,1), ordered by total degree i + j, then i descending; state layout
 * W[e][v][i] as for dg_mesh_create; nq1d (0 => p + 2) points per direction of
 * the collapsed Gauss rule and per edge; the BR2 penalty eta_br2 = 0 means 4
 * (n_faces + 1).  Such a handle serves dg_residual, dg_jvp (exact modes), the
 * p-multigrid (blocks by coloured JVP probing, three neighbour blocks per
 * triangle; block Jacobi smoothers), dg_fgmres_step, the BDF2 / ESDIRK3
 * right-hand sides and steps (per-triangle mass |J_e|), dg_mesh_info and
 * dg_status_sync; the FD JVP modes, the block ILU(0) coarse option and
 * dg_residual_noalloc return DG_ERR_INVALID.
 * DG_ERR_INVALID on bad sizes, indices, a clockwise or degenerate triangle or
 * an edge not shared by exactly two triangles. */
typedef struct {
  int n_vert;
  const double* X;
  int n_tri;
  const int* tri;
  const int* shift;
  double lo[2], hi[2];
  int p;
  int nq1d;
} dg_tri_desc;
dg_status dg_mesh_create_tri(const dg_tri_desc* desc, const dg_physics* phys, void* stream, dg_mesh* out);

/* Sizes: elements, modes per variable, variables (m), total DOFs E*m*n_m. */
dg_status dg_mesh_info(dg_mesh mesh, int* n_elem, int* n_modes, int* n_vars, size_t* n_dofs);

/* R = R(W), the DG spatial residual of eq. dg_ns (M dW/dt + R(W) = 0, Sec. 3.1):
 * volume term, Roe inviscid flux, BR2 viscous flux (eq. visc_flux) with the
 * lifting of eq. re, and the dual-consistency face term.  Optional S (may be
 * NULL): a modal source, R <- R - S.  W, S, R: device, E*m*n_m FP64; R must
 * not alias W.  Sets DG_ERR_NONPHYSICAL in the status word if rho or p <= 0 at
 * a quadrature point. */
dg_status dg_residual(dg_mesh mesh, const double* W, const double* S, double* R, void* stream);

/* dg_residual for callers that must not cause any device allocation when they
 * ask for a residual (the paper has no counterpart: this is a library-usage
 * entry point).  Such callers include applications that reserve all device
 * memory at start-up and time-critical loops that must stay out of the CUDA
 * allocator.  Same arguments as dg_residual and the same result: the same
 * face kernel, while the volume term takes the direct contractions where
 * dg_residual sums it by factorisation (3-D meshes and Q_p meshes), so the
 * two agree to rounding there and bit for bit elsewhere.  The face-slot scratch is a fixed file-scope device
 * array of 2^20 doubles (8 MiB) that every GPU loading the library holds
 * until the process exits, instead of the mesh handle's workspace.
 * Limits: E * dim * 2 * m * n_m must not exceed 2^20, else DG_ERR_INVALID.
 * dg_mesh_create looks up the array on its device (the library's device code
 * may be loaded lazily, and loading it is what allocates the array), so a
 * call here, on a mesh handle that exists, allocates nothing; mesh creation
 * reports DG_ERR_OOM if the array cannot be loaded.  All calls share the array:
 * calls that may overlap on the GPU race, so order them on one stream.
 * The array keeps the last call's contents; nothing in it needs clearing,
 * since each call writes every slot it reads. */
dg_status dg_residual_noalloc(dg_mesh mesh, const double* W, const double* S, double* R, void* stream);

#define DG_JVP_EXACT 0      /* forward-mode derivative of the discrete residual */
#define DG_JVP_FD 1         /* eq. DG-mf with h = eps sqrt(1 + ||v||)/||W|| as printed */
#define DG_JVP_FD_SCALED 2  /* eq. DG-mf with h = eps sqrt(1 + ||W||)/||v|| */
#define DG_JVP_EXACT_FP32 3 /* exact linearisation evaluated in FP32 (the operator of
                               the mixed-precision smoother on the finest level) */

/* Kv = sigma M v + dR/dW(W) v: the product of the iteration matrix
 * K = M/(a_ii dt) + dR/dW of eq. ODEDG with a vector (Sec. 5.1), sigma being
 * the shift (1/(a_ii dt) for ESDIRK, 3/(2 dt) for BDF2) and M = |J| I.
 * DG_JVP_EXACT: exact linearisation (default).  DG_JVP_FD / _SCALED: the
 * matrix-free finite difference of eq. DG-mf with eps = 1e-7; R_W = R(W) must
 * then be given (device), else it may be NULL.  DG_JVP_EXACT_FP32: W and v
 * rounded to FP32, the exact linearisation in FP32, Kv widened to FP64 (Sec. 6:
 * the inexact operator the mixed-precision preconditioner uses).  The FD and
 * FP32 modes use the mesh handle's scratch: such calls on one mesh must not
 * overlap.  W, v, Kv: device FP64; Kv must not alias W or v. */
dg_status dg_jvp(dg_mesh mesh, const double* W, const double* R_W, double sigma,
                 const double* v, double* Kv, int mode, void* stream);

#define DG_CYCLE_FMG 0      /* MG_full (Algorithm 1) */
#define DG_CYCLE_V 1        /* one MG_V cycle (Algorithm 2) from a zero guess */
#define DG_CYCLE_BJ 2       /* element block Jacobi only (no multigrid) */
#define DG_PREC_FP64 0
#define DG_PREC_MIXED 1     /* FP32 smoothers, blocks and fine JVP inside the preconditioner */

#define DG_COARSE_BJ 0      /* coarsest smoother: GMRES(element block Jacobi) */
#define DG_COARSE_BILU 1    /* coarsest smoother: GMRES(element block ILU(0)) (Table MGSettings) */
#define DG_ORDER_MDF 0      /* block ILU(0) in minimum discarded fill order (Sec. 6.3) */
#define DG_ORDER_NATURAL 1  /* element index order */
#define DG_ORDER_COLOUR 2   /* greedy multicolour order (few substitution levels) */

#define DG_STORE_NATIVE 0   /* blocks stored in the handle's precision (FP64, or FP32 in mixed mode) */
#define DG_STORE_BF16 1     /* mixed mode: the smoothers stream BF16 copies of the inverse diagonal
                               blocks of every level and of the inherited coarse blocks (rounded to
                               nearest from the FP32 blocks at setup/refresh), multiplying in FP32 */

/* p-multigrid options (Sec. 6; Table MGSettings).  p_level[0] must equal the
 * mesh degree and the levels must decrease strictly.  Every smoother is GMRES
 * right-preconditioned by element block Jacobi, except the coarsest one with
 * coarse_precond = DG_COARSE_BILU (needs n_levels >= 2, the cycle FMG or V, no
 * periodic direction of exactly 3 elements, and a coarsest block of at most
 * 64 rows in FP64 / 90 in FP32); nu_pre/nu_post (0..64) per level (ignored on
 * the coarsest), nu_coarse (1..64) on the coarsest level.  A zero-initialised
 * tail (coarse_precond, coarse_order, block_storage) selects block Jacobi with
 * blocks in the handle's precision.  block_storage = DG_STORE_BF16 needs
 * precision DG_PREC_MIXED and blocks of at most 2048 rows (fine) and
 * (1 + 2 dim) * ceil(nb / 8) <= 256 on coarse levels; else DG_ERR_INVALID.
 * The FP32 blocks are kept beside the BF16 copies (the inversion and the
 * block ILU(0) use them); dg_pmg_export_blocks returns the BF16 values the
 * smoothers use for DG_BLOCKS_DIAG_INV and DG_BLOCKS_NEIGHBOUR. */
typedef struct {
  int n_levels;
  int p_level[8];
  int nu_pre[8], nu_post[8], nu_coarse;
  int cycle;
  int precision;
  int fgmres_restart;   /* size of the outer FGMRES workspace allocated here (0 => 30, <= 64) */
  int coarse_precond;   /* DG_COARSE_BJ or DG_COARSE_BILU */
  int coarse_order;     /* DG_ORDER_*: element order of the block ILU(0) */
  int block_storage;    /* DG_STORE_NATIVE or DG_STORE_BF16 */
} dg_pmg_opts;

/* Assemble the preconditioner at state W and shift sigma (once per time step:
 * lagged, Sec. 7.4): diagonal Jacobian blocks dR_e/dW_e + sigma |J| I at the fine
 * order, neighbour blocks at the first coarse order only (Sec. 6.3),
 * coarse-level blocks by subspace inheritance (Sec. 6.1: with the orthonormal
 * hierarchical basis the projection keeps the leading modes of each variable
 * pair), and the inverse of every diagonal block by Gauss-Jordan elimination
 * with partial pivoting (the element block Jacobi of Sec. 6.3).  W: device FP64.
 * Allocates the handle's workspace; DG_ERR_OOM if it does not fit.  Blocks
 * until setup is complete; a singular block gives DG_ERR_BREAKDOWN. */
dg_status dg_pmg_setup(dg_mesh mesh, const double* W, double sigma, const dg_pmg_opts* opts,
                       void* stream, dg_pmg* out);

/* Recompute the preconditioner of an existing handle at a new state W and
 * shift sigma (same mesh and options), in the handle's own buffers: the same
 * work as dg_pmg_setup without allocation, asynchronous on `stream` (a
 * singular block is reported by dg_status_sync).  This is the once-per-time-
 * step preconditioner update of a lagged (Sec. 7.4) implicit time loop. */
dg_status dg_pmg_refresh(dg_pmg pmg, const double* W, double sigma, void* stream);

/* z = P^{-1} r: one application of the preconditioner (MG_full of Algorithm 1,
 * one MG_V of Algorithm 2, or block Jacobi), r and z device FP64, may not alias. */
dg_status dg_pmg_apply(dg_pmg pmg, const double* r, double* z, void* stream);
dg_status dg_pmg_destroy(dg_pmg pmg);

/* FGMRES options: restart length (<= the pmg handle's fgmres_restart), restarts allowed after the first
 * cycle, relative tolerance on the unpreconditioned residual ||b - K dW|| /
 * ||b|| (right preconditioning, Sec. 7.4), absolute tolerance, JVP mode. */
typedef struct {
  int restart;
  int max_restarts;
  double rtol;
  double atol;
  int jvp_mode;
} dg_krylov_opts;

typedef struct {
  int iters;            /* FGMRES iterations (preconditioner applications) */
  double res0;          /* ||b|| */
  double res_final;     /* residual estimate at exit */
  double rho;           /* (res_final/res0)^(1/iters), Sec. 7.3 */
  int status;           /* dg_status of the solve */
  float ms_total;       /* device time of the call */
  float ms_setup;       /* host time spent building the cycle graph in this call (0 when reused) */
} dg_krylov_stats;

/* Solve K dW = b (eq. ODEDG: the caller passes b = -f of the Newton step,
 * eq. NEWTON) by flexible GMRES (Saad 1993; Sec. 6) from dW = 0, right
 * preconditioned by pmg (setup at the same mesh; its sigma must be the one
 * given here), Arnoldi by classical Gram-Schmidt applied twice, Givens
 * rotations.  The outer Krylov vectors and the JVP are FP64.  W, b, dW: device
 * FP64.  With the exact JVP on a structured mesh the convergence test runs on
 * the device: a restart cycle is one launch of a graph in which every
 * iteration sits behind a conditional node that the previous iteration's test
 * opens (built at the first call and again when restart or sigma changes; it
 * works on copies of W and b in the handle, so a call may pass other pointers),
 * and the host waits once per cycle; the FD modes and triangle meshes read the
 * residual estimate on the host once per iteration.  Blocks until the solve
 * ends; stats (host, may be NULL) is filled in.  Returns DG_OK,
 * DG_ERR_NOT_CONVERGED, DG_ERR_BREAKDOWN or an error of the calls above. */
dg_status dg_fgmres_step(dg_mesh mesh, dg_pmg pmg, const double* W, const double* b,
                         double sigma, const dg_krylov_opts* opts, double* dW,
                         dg_krylov_stats* stats, void* stream);

/* Newton right-hand side of ESDIRK stage i (Sec. 4, eq. NEWTON):
 *   b = -[ sigma M (Wk - Wn) + racc + R(Wk) ],  sigma = 1/(a_ii dt),  M = |J| I,
 * racc = sum_{j<i} (a_ij / a_ii) R(W^j) (device, may be NULL when i has no
 * earlier implicit terms).  Wk (current Newton iterate of the stage), Wn, b:
 * device FP64; b must not alias the inputs.  sigma > 0. */
dg_status dg_esdirk3_rhs(dg_mesh mesh, const double* Wk, const double* Wn, double sigma,
                         const double* racc, double* b, void* stream);

/* One ESDIRK3 time step of M dW/dt + R(W) = 0 (Sec. 4): the four-stage,
 * third-order, explicit-first-stage, stiffly accurate scheme the paper uses
 * (Kennedy & Carpenter's ESDIRK3(2)4L[2]SA coefficients).  The preconditioner
 * `pmg` is refreshed once at Wn with sigma = 1/(a_ii dt) and reused for every
 * stage and Newton iteration (lagging, Sec. 7.4); each of the three implicit
 * stages starts from the previous stage and takes `newton` (1..16) Newton
 * iterations, each an FGMRES solve (dg_fgmres_step with kopts) of eq. NEWTON.
 * W^{n+1} = the last stage goes to Wout (device FP64, must not alias Wn).
 * work: caller-owned device scratch of at least 6 * n_dofs doubles
 * (work_bytes), the stage residuals and the Newton vectors.  Blocks until the
 * step ends.  stats (host, may be NULL): iterations summed over the 3*newton
 * solves, ms_total summed, res0/res_final/rho of the last solve.  Returns
 * DG_OK, DG_ERR_NOT_CONVERGED if some solve stopped above tolerance (the step
 * still completes), or an error of the calls above. */
dg_status dg_esdirk3_step(dg_mesh mesh, dg_pmg pmg, const double* Wn, double dt, int newton,
                          const dg_krylov_opts* kopts, double* work, size_t work_bytes, double* Wout,
                          dg_krylov_stats* stats, void* stream);

/* Newton right-hand side of one BDF2 step (the form of eq. NEWTON with the
 * BDF2 shift 3/(2 dt) in place of 1/(a_ii dt)):
 *   b = -[ M (3 Wk - 4 Wn + Wnm1) / (2 dt) + R(Wk) ],  M = |J| I.
 * Wk (current Newton iterate), Wn, Wnm1 (previous steps), b: device FP64;
 * b must not alias the inputs.  dt > 0. */
dg_status dg_bdf2_rhs(dg_mesh mesh, const double* Wk, const double* Wn, const double* Wnm1, double dt,
                      double* b, void* stream);

/* y <- y + alpha x over the E*m*n_m DOFs (the Newton update W <- W + dW of
 * eq. NEWTON).  x, y: device FP64, may not alias. */
dg_status dg_axpy(dg_mesh mesh, double alpha, const double* x, double* y, void* stream);

/* Number of CUDA kernels this library has launched in this process so far
 * (host-side counter; for launch accounting in benchmarks). */
dg_status dg_launch_count(unsigned long long* count);

/* ---------------------------------------------------------------- serving
 * A request loop over implicit steps (no counterpart in the paper: it serves
 * many independent cases of the step above on one GPU).  A request is one BDF2
 * step of one case, solved as in dg_fgmres_step with the p-multigrid
 * preconditioner refreshed at W^n.  Requests are admitted as device memory
 * frees up: each runs in a resident slot (mesh + p-multigrid handles + Krylov
 * workspace + its own stream) that stays alive after completion and is reused
 * by later requests of the same shape (mesh descriptor, physics, options);
 * idle slots are evicted least-recently-used to stay within the byte budget.
 * `workers` requests run at a time on separate streams, so their kernels
 * overlap on the device; new requests are admitted while others run
 * (continuous batching).  The result of a request does not depend on what else
 * is in flight (deterministic kernels, private buffers). */
typedef struct dg_server_s* dg_server;

typedef struct {
  long long id;
  int status;            /* dg_status of the request */
  double latency_ms;     /* submit to completion, host clock */
  double queue_ms;       /* submit to start */
  int fgmres_iters;      /* FGMRES iterations over the step's Newton iterations */
  long long ndofs;
} dg_server_result;

/* Start `workers` (1..64) worker threads on the current device with a device
 * memory budget in bytes.  DG_ERR_INVALID on bad arguments. */
dg_status dg_server_create(size_t budget_bytes, int workers, dg_server* out);

/* Queue one request.  Wn, Wnm1 (inputs) and Wout (the step's result W^{n+1})
 * are host arrays of E*m*n_m doubles that must stay valid until the request's
 * completion has been returned by dg_server_poll.  A request whose estimated
 * footprint exceeds the whole budget completes with DG_ERR_OOM. */
dg_status dg_server_submit(dg_server server, long long id, const dg_mesh_desc* desc, const dg_physics* phys,
                           const dg_pmg_opts* opts, const double* Wn, const double* Wnm1, double dt, int newton,
                           double rtol, double* Wout);

/* Wait until at least min_done completions are pending (timeout_ms < 0: no
 * limit), then move up to cap of them (oldest first) into out; *n_out = count.
 * DG_ERR_TIMEOUT if the wait ran out first (whatever was ready is returned). */
dg_status dg_server_poll(dg_server server, int min_done, int timeout_ms, dg_server_result* out, int cap,
                         int* n_out);

/* Device bytes held by resident slots, slot count, requests submitted/completed. */
dg_status dg_server_stats(dg_server server, size_t* used_bytes, int* resident_slots, long long* submitted,
                          long long* completed);

/* Stop the workers after their current requests, free every slot. */
dg_status dg_server_destroy(dg_server server);

/* Synchronise `stream`, return the mesh's device status word (DG_OK if no
 * device-side problem was recorded since the last call) and clear it. */
dg_status dg_status_sync(dg_mesh mesh, void* stream);

/* Element order and substitution levels of a block ILU(0) (Sec. 6.3), on the
 * host.  Graph: n_elem elements with n_faces face neighbours each, nbr[e *
 * n_faces + s] (a neighbour equal to e is a self coupling and ignored; one
 * neighbour reached through several faces counts once).  kind DG_ORDER_MDF
 * takes c[e * n_faces + s] = ||A_ee^{-1} A_e,nbr||_F for the first face of each
 * distinct neighbour (other entries unread; c may be NULL for the other kinds):
 * the next element is the one whose elimination drops the least fill, weight
 * w_i = sqrt(sum (c_ji c_ik)^2) over ordered pairs (j, k) of distinct unordered
 * neighbours of i that are not neighbours of each other, ties to the lowest
 * index, the neighbours' weights updated after each step.  DG_ORDER_NATURAL:
 * index order; DG_ORDER_COLOUR: greedy colouring in index order, then sorted by
 * (colour, index).  Outputs (host, caller-owned, n_elem entries): order[p] = the
 * element at position p, level[e] = 1 + the largest level of e's neighbours
 * ordered before it (0 if none); *n_levels = number of levels.  No GPU use.
 * DG_ERR_INVALID on a bad argument or neighbour index. */
dg_status dg_bilu_order(int n_elem, int n_faces, const int* nbr, const double* c, int kind, int* order,
                        int* level, int* n_levels);

/* The element order and level count the handle's coarsest block ILU(0) uses
 * now (after the last setup or refresh; host copies, order: n_elem entries or
 * NULL).  Synchronises `stream` first.  DG_ERR_INVALID if the handle has no
 * block ILU(0). */
dg_status dg_pmg_bilu_order(dg_pmg pmg, int* order, int* n_levels, void* stream);

/* y = A_l x: the operator level `level` of the handle smooths with (Sec. 6.1):
 * level 0 the matrix-free Jacobian-vector product sigma M x + dR/dW(W) x at
 * the handle's state and shift (in mixed precision the FP32 product the
 * smoother uses, with the state's traces cached at setup/refresh), levels >= 1
 * the inherited block-sparse operator D_e x_e + sum_s O_{e,s} x_nbr(e,s) on
 * the leading n_m(p_level[level]) modes of every variable.  x, y: device FP64,
 * E * m * n_m(p_level[level]) entries, may not alias (widened from FP32 in
 * mixed mode).  For testing and inspection; uses the handle's staging
 * buffers, so it must not overlap other calls on the handle.  DG_ERR_INVALID
 * if the level does not exist. */
dg_status dg_pmg_operator(dg_pmg pmg, int level, const double* x, double* y, void* stream);

#define DG_KT_FACE_JVP 0      /* face kernel of the fine-level operator (level 0) */
#define DG_KT_VOLUME_JVP 1    /* volume kernel of the fine-level operator (level 0) */
#define DG_KT_BLOCK_JACOBI 2  /* block-Jacobi apply of the level */
#define DG_KT_OPERATOR 3      /* the level's operator (level >= 1: the block-sparse product) */
#define DG_KT_SMOOTH 4        /* one smoother call of the level (nu_pre iterations; nu_coarse on the coarsest) */

/* Mean device time in ms (*ms, host) of one kernel of the handle's solve path,
 * launched `reps` (>= 1) times back to back on `stream` between two CUDA
 * events, for benchmarks and roofline reports: the fine-level operator's face
 * or volume kernel (the FP32 smoother JVP with the state's cached traces in
 * mixed mode, the FP64 JVP in an FP64 handle), the block-Jacobi apply, the
 * operator or one smoother call of `level`.  Inputs are a fixed pattern in the
 * handle's own level vectors; the results are discarded (the vectors, not the
 * blocks, are overwritten).  The mesh must be structured.  Synchronises
 * `stream`.  DG_ERR_INVALID for a bad kernel or level (the face and volume
 * kernels belong to level 0; a block-Jacobi-only handle has no smoother). */
dg_status dg_pmg_kernel_time(dg_pmg pmg, int kernel, int level, int reps, float* ms, void* stream);

/* Sizes of the pMG workspace in bytes (blocks, vectors), for memory budgeting. */
dg_status dg_pmg_bytes(dg_pmg pmg, size_t* block_bytes, size_t* vector_bytes);

#define DG_BLOCKS_DIAG_INV 0   /* inverse diagonal blocks, E * nb * nb */
#define DG_BLOCKS_NEIGHBOUR 1  /* neighbour blocks, E * 2d * nb * nb, [e][2k+side] */
#define DG_BLOCKS_DIAG 2       /* diagonal blocks before inversion, E * nb * nb */

/* Copy the blocks of level `level` into a caller device buffer (entries of the
 * handle's precision: FP64, or FP32 in mixed mode; nb = m * n_m(p_level[level]);
 * row-major [v*n_m + i][w*n_m + j]), for testing and inspection.  Neighbour
 * blocks exist for levels >= 1 (side 0 = the xi_k = -1 face).  DG_BLOCKS_DIAG
 * (Sec. 5.1 eq. ODEDG, d R_e / d W_e + sigma |J| I): level 0 is recomputed by
 * the fine-level probe at the handle's state and shift, written straight into
 * `out`; coarser levels are the inherited (truncated) blocks.  Synchronous.
 * DG_ERR_INVALID if the level or kind does not exist or out_bytes is short. */
dg_status dg_pmg_export_blocks(dg_pmg pmg, int level, int which, void* out, size_t out_bytes,
                               void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
