/*
 * hz.h -- C ABI of the GB300 nested polarized-traces Helmholtz solver.
 *
 * Problem (Section 2, Appendix A of Zepeda-Nunez & Demanet, "Nested domain
 * decomposition with polarized traces for the 2D Helmholtz equation"):
 *     (-Laplacian - omega^2 m(x)) u = f   on the PML-extended rectangle,
 * discretised by the 5-point stencil with PML (d/dx -> alpha_x d/dx,
 * alpha = 1/(1 + i sigma/omega), sigma(d) = (C/delta)(d/delta)^2) and
 * homogeneous Dirichlet data beyond the extended grid.  The interior has
 * n_x x n_z nodes x_p = p h (p = 1..n_x), with n_pml PML nodes on every side.
 *
 * Method: the online stage of the nested polarized-traces solver
 * (Sections 3-4): L layers of C cells; GMRES on the polarized interface
 * traces (eq. integral_polarized) preconditioned by the Gauss-Seidel
 * sweeps (eq. preconditioner_GS); layer Green's integrals applied through
 * the factorization of eq. (factorization) with the inner compressed-block
 * LU of Section 4.2.2 kept dense.
 *
 * Conventions for every entry point:
 *   - Complex arrays are interleaved (re, im) doubles.
 *   - Grid arrays are row-major [n_z + 2 n_pml][n_x + 2 n_pml], x fastest;
 *     batched arrays put the batch index outermost: [B][rows][cols].
 *   - Pointers are host pointers unless opts.device_ptrs = 1 at setup, in
 *     which case every array argument (m excepted) is a device pointer.
 *   - The caller owns every array it passes.  The context owns its factors
 *     and workspaces and frees them in hz_destroy.
 *   - No entry point aborts.  Each returns a status; hz_last_error() returns
 *     a message for the last failure on that context.
 *   - Calls on one context must not overlap; distinct contexts are
 *     independent (they may share a stream).
 *   - Fault injection for tests of the failure paths (read at hz_setup from
 *     the environment variable HZ_FAULT; unset in normal use):
 *       alloc[:n]  the n-th device allocation of the context, counted from
 *                  hz_setup, fails (HZ_ENOMEM);
 *       singular   the factorization reports a zero pivot (HZ_ESINGULAR);
 *       nan        a NaN enters the polarized right-hand side of each solve
 *                  pass (the solve returns HZ_ENOTCONV, residual NaN);
 *       noconv     one GMRES iteration and one pass per solve (HZ_ENOTCONV).
 */
#ifndef HZ_H
#define HZ_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hz_ctx hz_ctx;

typedef enum {
    HZ_OK = 0,
    HZ_EINVAL = 1,      /* bad argument (sizes, partition, NULL pointer, NaN/Inf input) */
    HZ_ENOMEM = 2,      /* host or device allocation failed */
    HZ_ECUDA = 3,       /* a CUDA call failed (message in hz_last_error) */
    HZ_ESTATE = 4,      /* call out of order (solve before factor) */
    HZ_ENOTCONV = 5,    /* GMRES or refinement did not reach the tolerance; best iterate written */
    HZ_ETIMEOUT = 6,    /* a bounded device wait gave up */
    HZ_ESINGULAR = 7    /* a zero pivot in a cell or inner factorization */
} hz_status;

enum { HZ_FP64 = 0, HZ_MIXED = 1 };            /* hz_opts.precision */
enum { HZ_PGS = 0, HZ_PJAC = 1, HZ_PNONE = 2 }; /* hz_opts.precond */
enum { HZ_GMRES = 0, HZ_BICGSTAB = 1 };         /* hz_opts.krylov */
enum { HZ_INNER_LU = 0, HZ_INNER_NESTED = 1 };  /* hz_opts.inner */

typedef struct {
    int precision;      /* HZ_FP64: every online operator in FP64.
                           HZ_MIXED: operators and sweeps in complex FP32, GMRES
                           Arnoldi and the volume residual in FP64, accuracy
                           recovered by residual refinement. */
    int precond;        /* HZ_PGS (eq. preconditioner_GS), HZ_PJAC (eq.
                           preconditioner_Jac) or HZ_PNONE */
    int restart;        /* GMRES restart length (default 30) */
    int max_it;         /* GMRES iteration cap per solve (default 200) */
    double tol;         /* GMRES relative residual on the polarized system
                           (default 1e-10 FP64, 3e-5 mixed: refinement
                           passes carry the volume residual to refine_tol) */
    double refine_tol;  /* target ||H u - f|| / ||f|| on the volume; refinement
                           passes repeat the solve on the residual until it is
                           met (0: no refinement; default 1e-8) */
    int max_refine;     /* refinement pass cap (default 6) */
    double pml_C;       /* sigma amplitude C; <= 0 selects
                           1.5 * c_max * ln(1e6) (1e-6 normal-incidence
                           continuum reflection at the fastest speed) */
    const int *layer_rows; /* L interior rows per layer, sum n_z; NULL = even split */
    const int *cell_cols;  /* C interior columns per cell, sum n_x; NULL = even split */
    int device_ptrs;    /* 1: array arguments of solve/gradient/component calls are device pointers */
    void *stream;       /* cudaStream_t used by every call on the context (NULL = legacy default) */
    int time_kernels;   /* 1: time the hot kernels with CUDA events (hz_stats.kt_*) */
    int krylov;         /* outer Krylov method on the polarized traces: HZ_GMRES
                           (flexible GMRES, default) or HZ_BICGSTAB (Bi-CGstab,
                           right preconditioned, two preconditioned operator
                           applications per iteration; §5) */
    int autotune;       /* 1: time the launch configurations of the inner sweep at
                           the first use of each launch shape and keep the
                           fastest (environment HZ_TUNE_CACHE: JSON file that
                           keeps the choices across processes); 0 (default): fixed
                           rule */
    int tensor_cores;   /* HZ_MIXED only: 1 (default) runs the cell solves (a1) on
                           the tensor cores (tcgen05, 3xTF32 split, cells up to
                           128 columns wide, cell-solve error ~3e-6 against
                           ~8e-7 on the FP32 SIMT pipes); 2 also runs the
                           batched F / E / S / W products (a2-a5) with long K
                           on them (3xTF32, error ~2e-7 against ~5e-7 on the
                           SIMT pipes, at the cost of TF32 split copies of the
                           operators, twice their FP32 size in device memory);
                           0 keeps everything on the SIMT pipes */
    int rhs_lanes;      /* hz_solve with B a multiple of rhs_lanes (> 1) splits the
                           right-hand sides into rhs_lanes equal groups solved in
                           lockstep, each on its own stream with its own
                           workspaces but the context's factorization, so that
                           the latency-bound sweep chains of the groups overlap on
                           the GPU (1, the default: one group) */
    double wait_ms;     /* limit of every bounded device wait (the mbarrier waits of
                           the inner sweep, the tensor-core kernels and the
                           cluster exchange), in milliseconds; a wait that runs
                           out makes the call return HZ_ETIMEOUT with its results
                           invalid, the context staying usable (<= 0: 1000) */
    int inner;          /* solver of each layer's local problem (Section 4.2):
                           HZ_INNER_LU (default): the inner SIE over the cells by
                           block LU (exact); HZ_INNER_NESTED: the inner nested
                           polarized traces -- the layer's box with x and z
                           swapped is a problem of the same form whose layers are
                           the cells, solved by FGMRES on its polarized traces with
                           the Gauss-Seidel sweeps over the cells, to inner_tol
                           inside the preconditioner (the outer solver is then a
                           flexible GMRES, which admits it); needs C >= 2,
                           krylov HZ_GMRES and rhs_lanes 1, and hz_update_model is
                           not available with it */
    double compress;    /* compressed-block LU (Section 4.2.2, with the compression
                           of Section 4.3): > 0 stores every inner block-LU factor
                           P_j = W_j(:,a) Z_j and V_j = W_j(:,b) K_{j+1} (the cell's
                           Green's function between its two sides) as a rank-r
                           product, r the largest numerical rank at relative
                           Frobenius accuracy `compress` found by an adaptive
                           randomized range finder; the inner sweeps then run on
                           r-vectors.  0: dense factors; < 0 (the default):
                           1e-8 (the paper's accuracy for the compressed
                           operators) in HZ_MIXED, dense in HZ_FP64 */
    double inner_tol;   /* HZ_INNER_NESTED: relative GMRES tolerance of the inner
                           solves inside the preconditioner (<= 0: 1e-6); the
                           polarized operator, the Newton potentials and the
                           reconstruction use 1e-10 (HZ_FP64) or 1e-6 (HZ_MIXED) */
} hz_opts;

typedef struct {
    int iterations;        /* GMRES iterations, summed over refinement passes (max over RHS per pass) */
    int refinements;       /* solves performed (1 = no refinement pass needed) */
    double gmres_resid;    /* max over RHS of the last pass's GMRES relative residual */
    double resid;          /* max over RHS of ||H u - f||_2 / ||f||_2 (FP64, Appendix A operator) */
    double t_total_ms;     /* wall time of the call (device-synchronised) */
    double t_local_ms;     /* Newton potentials: cell solves + inner sweeps (all passes) */
    double t_gmres_ms;     /* GMRES on the traces (all passes) */
    double t_recon_ms;     /* volume reconstruction (all passes) */
    double t_resid_ms;     /* FP64 residual evaluations */
    int gpu_launches;      /* kernels launched by the call */
    /* with opts.time_kernels: launches and summed device time of the hot
       kernel classes 0 = cell chain solves (a1), 1 = inner block-LU sweeps
       (a3), 2 = batched F/E/S products (a2, a4) */
    int kt_launches[3];
    double kt_ms[3];
    double kt_bytes[3];    /* algorithmic bytes moved by those launches */
    double kt_flops[3];    /* algorithmic real flops of those launches */
    int inner_iterations;  /* HZ_INNER_NESTED: GMRES iterations of all inner solves of
                              the call (max over right-hand sides per inner solve) */
    int compress_rank;     /* opts.compress > 0: the rank r of the compressed inner
                              factors (0: dense) */
} hz_stats;

/* Fill opts with the defaults documented above (precision HZ_FP64). */
void hz_default_opts(hz_opts *opts);

/* Create a context for one medium and frequency (Section 2: H u = f on the
 * extended grid, m given on the extended grid, Appendix A footnote).
 *   m      : host array (n_z+2n_pml) x (n_x+2n_pml) of squared slowness, copied.
 *   L, C   : layers and cells per layer (Section 4; every layer and cell needs
 *            at least 1 interior row/column; L >= 2).
 *   opts   : may be NULL for defaults; copied (the partition arrays too).
 * Errors: HZ_EINVAL (sizes, partition, non-finite m/omega/h), HZ_ENOMEM, HZ_ECUDA. */
hz_status hz_setup(hz_ctx **ctx, const double *m, int n_x, int n_z, double omega,
                   double h, int n_pml, int L, int C, const hz_opts *opts);

/* Offline stage (Section 4.3.1, Table chap:nested:table:complexity): per cell
 * assembly and block-tridiagonal factorization in FP64 with pivoted inverses of
 * the diagonal Schur blocks, the cell Green's blocks of eq. (factorization)
 * (M_f, M_u split into F, E, S), and the block-LU factors of each layer's inner
 * SIE (Section 4.2.2) with inverted diagonal blocks.  Idempotent.
 * Errors: HZ_ESINGULAR (zero pivot), HZ_ENOMEM, HZ_ECUDA. */
hz_status hz_factor(hz_ctx *ctx);

/* Online solve (Alg. matrix_free_solver with the nested inner solver):
 *   f : [B][n_z+2p][n_x+2p] complex source, u : same shape, written.
 *   st: may be NULL.
 * u satisfies H u = f for the Appendix A operator.  Returns HZ_ENOTCONV (u still
 * written with the best iterate) when the GMRES or refinement target is missed.
 * Errors: HZ_ESTATE (not factored), HZ_EINVAL (B < 1, NULL, non-finite f). */
hz_status hz_solve(hz_ctx *ctx, const double *f, int B, double *u, hz_stats *st);

/* Solve of G problems at once (several frequencies or media sharing a device,
 * e.g. the frequencies of one inversion step; not in the paper).  Each member
 * is an hz_solve on its own context and stream; the members' Newton stages,
 * GMRES iterations, reconstructions and residuals are enqueued together and
 * the host waits once per step for all of them, so their kernels overlap.
 *   ctxs : G distinct factored contexts, same precision and device; give each
 *          its own stream (opts.stream) for overlap (same stream: serialised).
 *   f[i], u[i] : as hz_solve for ctxs[i] (host or device per its device_ptrs).
 *   st   : NULL or G stats, one per member.
 * Returns the worst member status (HZ_ENOTCONV if any member missed its
 * target; every u[i] written).  Errors: HZ_EINVAL (NULL, G < 1, mixed
 * precisions or devices, repeated ctx), HZ_ESTATE, and those of hz_solve;
 * the message is on ctxs[0]. */
hz_status hz_solve_group(hz_ctx **ctxs, int G, const double *const *f, int B,
                         double *const *u, hz_stats *st);

/* Receiver misfit J = 1/2 sum_s ||R u_s - d_s||^2 and its gradient with respect
 * to m on the extended grid (not in the paper; adjoint state).  One forward
 * solve per source, one adjoint solve reusing the factors (the row-scaled
 * operator is complex symmetric), then
 *   dJ/dm_i = omega^2 sum_s Re(lambda_{s,i} u_{s,i}),  H^T lambda_s = R^T conj(r_s).
 *   f      : [B][grid] sources; d : [B][n_rec] data; rec_idx: [n_rec] flat
 *            grid indices in [0, grid) (host or device per device_ptrs; read
 *            back and range-checked on the host in both modes, HZ_EINVAL
 *            beyond); an index listed twice is two receivers at one node and
 *            counts twice in J and in the gradient;
 *   J      : scalar out (host pointer always); grad_m : [grid] real out;
 *   u_out  : optional [B][grid] forward fields (may be NULL).
 * Errors as hz_solve. */
hz_status hz_gradient(hz_ctx *ctx, const double *f, int B, const double *d,
                      const int *rec_idx, int n_rec, double *J, double *grad_m,
                      double *u_out, hz_stats *st);

/* Local model update (paper, Conclusion: a medium updated locally inside an
 * inversion loop needs only a local modification of the method): replace the
 * medium by m_new and re-factor only the layers with a cell whose box reads a
 * changed value (the cell operators, their Green's blocks F / E / S and the
 * layer's inner block LU; the other layers' operators stay as they are),
 * plus the global residual coefficients.  The result is the factorization
 * hz_factor computes for m_new (same kernels on the same data); the PML
 * strength stays the one fixed at hz_setup.
 *   m_new      : [n_z+2p][n_x+2p] squared slowness, host pointer always,
 *                finite and positive;
 *   n_layers   : NULL or out: how many layers were re-factored (0 when m_new
 *                equals the current medium).
 * Errors: HZ_EINVAL (NULL, non-finite or non-positive m_new), HZ_ESTATE (before
 * hz_factor), HZ_ENOMEM, HZ_ECUDA; on an error after validation the context
 * must be destroyed. */
hz_status hz_update_model(hz_ctx *ctx, const double *m_new, int *n_layers);

/* Adjoint of hz_solve for an arbitrary real loss L(u) (not in the paper; the
 * differentiation pattern of the solver): with gu = dL/dRe(u) + i dL/dIm(u)
 * (PyTorch's gradient convention for complex tensors),
 *   mu     = H^{-T} conj(gu)                 (transposed Appendix A system,
 *                                             solved with the forward factors),
 *   grad_m = omega^2 sum_s Re(mu_s . u_s)    (dL/dm, real, [grid]),
 *   grad_f = conj(mu)                        (dL/df in the same convention; may be NULL).
 *   u, gu : [B][grid] complex (forward fields and their gradients).
 * Errors as hz_solve. */
hz_status hz_adjoint(hz_ctx *ctx, const double *u, const double *gu, int B, double *grad_m, double *grad_f,
                     hz_stats *st);

/* Checkpoint of a solve (not in the paper; used to differentiate without
 * keeping volume fields): the interface traces of a field,
 *   tr[b][k][0][x] = u[b][row_a(k)][x],  tr[b][k][1][x] = u[b][row_b(k)][x],
 * row_a(k) = last interior row of layer k, row_b(k) = first interior row of
 * layer k+1 (k = 0..L-2), x over the full extended width n_x+2p.
 *   u : [B][grid] complex; tr : [B][L-1][2][n_x+2p] complex, written.
 * Errors: HZ_EINVAL (NULL, B < 1, L < 2), HZ_ECUDA. */
hz_status hz_traces(hz_ctx *ctx, const double *u, int B, double *tr);

/* Recompute a field from its source and its interface traces: every layer's
 * field is its local solution with the interface forcing of Appendix C built
 * from the traces (the reconstruction stage of Alg. matrix_free_solver, lines
 * 10-18, with the traces given), so no GMRES runs.  With tr = hz_traces(u) of
 * a converged u it returns u to the working precision of the operators
 * (roundoff in FP64, ~1e-6 relative in HZ_MIXED).
 *   f : [B][grid]; tr : [B][L-1][2][n_x+2p]; u : [B][grid], written.
 * Errors: HZ_ESTATE (not factored), HZ_EINVAL (NULL, B < 1, L < 2, non-finite
 * f or tr), HZ_ETIMEOUT, HZ_ECUDA. */
hz_status hz_reconstruct(hz_ctx *ctx, const double *f, const double *tr, int B, double *u);

/* ---- component entry points (each runs one step of the online path on the
 * device, used to test that step alone; inputs/outputs follow the conventions
 * above, batch outermost) ---- */

/* a1: solve one cell's local problem H^{l,c} x = g (0-based l, c) on the cell's
 * extended grid [B][n_l+2p][w_c+2p]; the cell operator is the row-scaled
 * (symmetric) form of Appendix A on a box with its own PML (Section 4). */
hz_status hz_cell_solve(hz_ctx *ctx, int l, int c, const double *g, int B, double *x);

/* a5: layer Green's integrals of layer l (Def. incomplete_green in the form of
 * Appendix C, eq. pde_GRF_real) applied through eq. (factorization):
 *   tr  : [B][4][T] traces at local rows (0, 1, n_l, n_l+1), T = n_x + 2p
 *   out : [B][4][T] field sampled at the same rows.
 * in_mask bit 0: use rows (0,1); bit 1: use rows (n,n+1). */
hz_status hz_layer_green(hz_ctx *ctx, int l, const double *tr, int in_mask, int B, double *out);

/* a6: y = M x for the polarized system (eqs. jump_1..jump_4, moved to the
 * left); x, y : [B][L-1][4][T] with components (d_a, d_b, u_a, u_b) of each
 * interface k (a = last row of layer k, b = first row of layer k+1). */
hz_status hz_apply_M(hz_ctx *ctx, const double *x, int B, double *y);

/* a7-a9: which = 0: P^GS x (eq. preconditioner_GS); 1: P^Jac x;
 * 2: D_down^{-1} (Alg. downwardsSweep) on the d-part, u-part copied;
 * 3: D_up^{-1} (Alg. upwardsSweep) on the u-part, d-part copied;
 * 4: L applied to the d-part (Alg. upwardsReflections), written to the u-part,
 *    d-part zeroed.  Layout as hz_apply_M. */
hz_status hz_precond(hz_ctx *ctx, int which, const double *x, int B, double *y);

/* a12: relative residual ||H u - f|| / ||f|| per RHS in FP64 (res: [B], host
 * or device per device_ptrs). */
hz_status hz_residual(hz_ctx *ctx, const double *u, const double *f, int B, double *res);

/* Allocation-free variant of hz_residual, for callers that cannot allocate
 * device memory when they need the residual (their device memory is reserved
 * up front by another allocator, or their loop forbids allocation calls,
 * which synchronise the device).  The paper has no counterpart.
 *   u, f : device pointers, [B][n_z+2p][n_x+2p] complex (read in place);
 *   res  : device pointer, [B] relative residuals ||H u - f||_2 / ||f||_2,
 *          as hz_residual computes them.
 * Makes no cudaMalloc/cudaFree or allocating library call.  Its scratch is a
 * fixed 512 KiB device array inside the library (every GPU that loads it
 * holds it until exit), so B is limited to 256 (HZ_EINVAL beyond).  The first
 * call on each device looks up that array's device address; make that first
 * call before any stream capture.  The work is enqueued on the context's
 * stream and res is valid once the stream reaches it.  All calls share the
 * scratch array: calls whose kernels overlap on the GPU race.
 * Errors: HZ_EINVAL (NULL pointer, B out of 1..256, u/f/res not device
 * memory of the context's device, another device current), HZ_ECUDA. */
hz_status hz_residual_noalloc(hz_ctx *ctx, const double *u, const double *f, int B, double *res);

/* Check of the timeout path (not in the paper): launches one thread block that
 * waits, through the same bounded wait every kernel of the library uses, on an
 * mbarrier that nothing completes, so the wait runs out after opts.wait_ms.
 * Returns HZ_ETIMEOUT when the limit and the error report work (the context
 * stays usable; nothing else is launched), HZ_OK if the wait completed (it
 * cannot), HZ_ECUDA on a CUDA failure. */
hz_status hz_check_timeout(hz_ctx *ctx);

/* Switch the pointer mode of later calls (same meaning as opts.device_ptrs). */
hz_status hz_set_device_ptrs(hz_ctx *ctx, int device_ptrs);

/* Switch per-kernel-class CUDA-event timing of later calls (same meaning as
 * opts.time_kernels: 1 records events around every launch of the online path
 * and fills hz_stats.kt_*; 0 records none, so that consecutive launches may
 * overlap their prologues).  HZ_EINVAL if ctx is NULL. */
hz_status hz_set_time_kernels(hz_ctx *ctx, int time_kernels);

/* Bytes of device memory held by the context (factors + workspaces). */
long long hz_device_bytes(const hz_ctx *ctx);

void hz_destroy(hz_ctx *ctx);
const char *hz_last_error(const hz_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H */
