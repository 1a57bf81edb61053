/*
 * lsgpu.h -- C ABI of the B300 (sm_103a) Lippmann-Schwinger Nystrom hot path.
 *
 * Method: arXiv 2608.17615, "Fast high-order solvers for the Lippmann-Schwinger
 * equation in piecewise-smooth heterogeneous media".  The library solves the
 * Nystrom system L u = b of Eq. nystrom_linear_system,
 *
 *     L = I + k^2 V M                         (Eq. linear_system_matrix)
 *     (V f)_j = sum_{n != j} G(y_j, y_n) w_n f_n + sum_q dV_jq f_q
 *     G(x, y) = (i/4) H0^(1)(k |x - y|),     M = diag(m(y_j)),  m = 1 - n
 *
 * on the quadrature nodes y_j of a curved triangle mesh: a dense pair sum plus
 * the sparse VDIM near/self correction dV (Eq. DIM_decomp, local-patch form),
 * by unrestarted GMRES (Section 6) with optional left preconditioning by
 * P = I + T_C^Q (S - I) T_Q^C (Eq. preconditioner_factored, Approach II
 * transfers Eq. T_H^C_def, sparsifying preconditioner S = C^{-1} A, Eq. LC_def).
 *
 * Conventions
 *  - Complex numbers are interleaved pairs of doubles (re, im) (complex128).
 *  - Host arrays passed in are copied; the caller keeps ownership.  Device
 *    arrays (suffix _dev) are borrowed for the duration of the call, must hold
 *    the stated number of elements, and are read/written on the operator's
 *    stream; the call returns after the work is enqueued and synchronised.
 *  - Every function returns an ls_status; on failure ls_last_error() returns
 *    a thread-local message.  No function aborts the process.
 *  - Handles are not thread-safe: one thread uses one ls_op at a time.
 */
#ifndef LSGPU_H
#define LSGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LS_OK = 0,
    LS_EINVAL = 1,      /* bad argument (null pointer, size, mesh inconsistency, NaN input) */
    LS_ENOMEM = 2,      /* device or host allocation failed */
    LS_ECUDA = 3,       /* a CUDA runtime / library call failed */
    LS_ESINGULAR = 4,   /* a block of the Cartesian matrix C could not be factored */
    LS_ENOCONV = 5,     /* GMRES hit max_iter; outputs hold the last iterate */
    LS_ETIMEOUT = 6     /* a bounded device wait ran out (tensor-core pipeline); the context stays usable */
} ls_status;

typedef struct ls_mesh ls_mesh;
typedef struct ls_op ls_op;

/* Pair-sum arithmetic of an operator (ls_params.prec). */
enum {
    LS_PREC_FP64_TABLE = 0,   /* FP64, H0 from a per-operator table of polynomials in t = r^2 on
                                 octave-graded cells (each table validated to 2e-15 against the
                                 long-double routine at setup; degree chosen by timing at setup) */
    LS_PREC_FP64_DIRECT = 1,  /* FP64 direct evaluation of H0 (series / fitted asymptotic form)  */
    LS_PREC_FP32 = 2,         /* precision form: FP32 table (degree 6, validated to 2e-8),
                                 double-float coordinate differences, Kahan-compensated FP32 sums */
    LS_PREC_FP64_DF = 3,      /* FP64-accurate: the FP64 table evaluated in double-float (pairs of
                                 FP32) arithmetic and accumulated on the FP32 pipe                */
    LS_PREC_MIXED = 4         /* mixed precision: every GMRES solve runs with the FP32 pair sum
                                 (as LS_PREC_FP32) and is refined against the double-float
                                 operator (as LS_PREC_FP64_DF): r = b - L u with the accurate L,
                                 an FP32 GMRES correction d, u += d, r -= L d (the product of the
                                 small correction in FP32: its error, eps32 cond(L) ||r||, is far
                                 below tol ||b||), until ||P r|| <= tol ||P b|| (at most 4
                                 corrections).  Single applies (ls_apply*) use the accurate
                                 operator; iters_out counts every inner iteration, hist_out holds
                                 the first FP32 solve's history; ls_op_last_residual is the
                                 refinement's final residual.  The batched solves are not
                                 affected (they refine on their own).                           */
};

/* Build parameters of an operator. */
typedef struct {
    double  tol;          /* GMRES stop: ||P(b - L u_k)|| / ||P b|| <= tol          */
    int32_t max_iter;     /* GMRES iteration cap (the paper stops at 600)            */
    int32_t use_precond;  /* 1: left-precondition with P; 0: plain GMRES             */
    double  kappa;        /* VDIM patch radius in units of the target element size   */
    double  box[4];       /* Cartesian grid box xmin, xmax, ymin, ymax (Section 4)    */
    int32_t nx, ny;       /* grid nodes per direction, endpoints included; the step
                             (xmax - xmin)/(nx - 1) must equal (ymax - ymin)/(ny - 1) */
    int32_t prec;         /* LS_PREC_* above                                          */
    int32_t approach;     /* transfer T_Q^C of the preconditioner: 2 = Approach II, the
                             renormalised transpose D^{-1} (T_C^Q)^T (Eq. T_H^C_def);
                             1 = Approach I, the element-wise L^2 projection
                             E_C (M^tri)^{-1} E_Q^T W (Eq. T_HC_proj_def)             */
    int32_t setup_on_device; /* 1: the correction dV is built on the GPU in double-double
                             arithmetic (blocks out of its series range on the host);
                             0: entirely on the host in long double                  */
} ls_params;

/* Defaults: tol 1e-8, max_iter 600, use_precond 1, kappa 3, box [-1.2,1.2]^2, 256 x 256,
   prec LS_PREC_FP64_DF, approach 2, setup_on_device 1. */
void ls_params_default(ls_params* p);

/*
 * Mesh of N_T curved triangles with 15 quadrature nodes each (Section 3:
 * conforming curved mesh of every subdomain Omega_l; the meshes of different
 * subdomains need not match across an interface).
 *   vert_xy     [n_vert][2]     vertex coordinates
 *   elem_vert   [n_elem][3]     vertex ids, counter-clockwise; edge e runs from
 *                               elem_vert[t][e] to elem_vert[t][(e+1)%3]
 *   elem_domain [n_elem]        subdomain id l >= 0 (contrast smooth on each)
 *   edge_curve  [n_elem][3]     -1: straight edge; c >= 0: arc of curve c
 *   edge_theta  [n_elem][3][2]  arc parameter range (theta_start, theta_end)
 *   curves      [n_curve][6]    polar curves (cx, cy, R, a, m, phi):
 *                               gamma(t) = c + R (1 + a cos(m t + phi)) (cos t, sin t)
 *   nodes_xy    [15 n_elem][2]  quadrature nodes, element-major (node j lies in
 *                               element j / 15); all interior to their element
 *   weights     [15 n_elem]     quadrature weights (Jacobian included)
 * Elements of one subdomain must share edges exactly (same vertex ids).
 * Errors: LS_EINVAL for null pointers, n_elem < 1, ids out of range, or a
 * clockwise/degenerate element.
 */
ls_status ls_mesh_create(int32_t n_vert, const double* vert_xy,
                         int32_t n_elem, const int32_t* elem_vert, const int32_t* elem_domain,
                         const int32_t* edge_curve, const double* edge_theta,
                         int32_t n_curve, const double* curves,
                         const double* nodes_xy, const double* weights,
                         ls_mesh** out);
void ls_mesh_destroy(ls_mesh* mesh);
int32_t ls_mesh_num_nodes(const ls_mesh* mesh);

/*
 * Operator L = I + k^2 V M on a mesh (Eq. linear_system_matrix) and, when
 * params->use_precond, the preconditioner P (Eq. preconditioner_factored).
 *   k        wavenumber > 0
 *   m        [N_Q] complex contrast m(y_j) = 1 - n(y_j) at the nodes
 *   m_grid   [nx * ny] complex contrast at the grid nodes (x fastest), zero
 *            outside the scatterer; required when use_precond, else may be NULL
 *   stream   cudaStream_t (NULL = default stream) for all device work
 * Setup builds the VDIM correction dV in extended precision (on the GPU in
 * double-double arithmetic, or on the host in long double, see setup_on_device)
 * and the preconditioner factors on the device; it is not part of the timed
 * solve.  The mesh may be destroyed afterwards.
 * Errors: LS_EINVAL (k <= 0, NaN contrast, bad grid), LS_ENOMEM, LS_ECUDA,
 * LS_ESINGULAR (a Schur block of C is singular).
 */
ls_status ls_operator_create(const ls_mesh* mesh, double k, const double* m, const double* m_grid,
                             const ls_params* params, void* stream, ls_op** out);
/*
 * Purely Cartesian operator (Section 6, comparison with a purely Cartesian discretization;
 * Eq. LS_eq_on_cartesian_points): the unknowns are the nx x ny grid nodes of params->box
 * (x fastest), L^(C) = I + k^2 V^(C) M^(C) with V^(C)_il = G(z_i - z_l) h^2 off the diagonal
 * and the integral of G over the disc of area h^2 on it, applied by zero-padded FFT
 * convolution (cuFFT, 2 nx x 2 ny); preconditioner (params->use_precond) the sparsifying
 * S^(C) = C^{-1} A of the same grid (Eq. sparsifying_min, Eq. LC_def).  The returned ls_op
 * works with ls_apply[_dev], ls_apply_precond[_dev], ls_apply_transpose[_dev],
 * ls_solve[_dev] (plane waves and far field use the grid nodes with weights h^2),
 * ls_solve_adjoint and ls_residual_dev; the quadrature-node calls (pair sums, batched
 * forms, correction) return LS_EINVAL.
 *   m_grid [nx * ny] complex contrast at the grid nodes
 * Errors: LS_EINVAL (k <= 0, bad grid, non-finite contrast), LS_ENOMEM, LS_ECUDA, LS_ESINGULAR.
 */
ls_status ls_cartesian_create(double k, const double* m_grid, const ls_params* params, void* stream, ls_op** out);

void ls_op_destroy(ls_op* op);
int32_t ls_op_num_nodes(const ls_op* op);

/* y = L x on device buffers x_dev, y_dev of N_Q complex (they may not alias). */
ls_status ls_apply_dev(ls_op* op, const void* x_dev, void* y_dev);
/* Same with host buffers; includes the host<->device copies. */
ls_status ls_apply(ls_op* op, const double* x, double* y);
/* y = P x (Eq. preconditioner_factored) on device buffers; LS_EINVAL without a preconditioner. */
ls_status ls_apply_precond_dev(ls_op* op, const void* x_dev, void* y_dev);
/* y_r = P x_r for R right-hand sides x_dev, y_dev [R][N_Q] complex (no aliasing) with the
   batched preconditioner kernels of ls_solve_batch_dev: FP64 block-LU sweeps under batch
   kernel 0, FP32 sweeps under kernel 1 (ls_op_set_batch_kernel).  LS_EINVAL without a
   preconditioner. */
ls_status ls_apply_precond_batch_dev(ls_op* op, int32_t R, const void* x_dev, void* y_dev);

/*
 * Plain pair sum y_j = sum_{n != j} G(y_j, y_n) w_n f_n (the naive Nystrom
 * quadrature of V_Omega[f], Eq. vol_pot) on device buffers of N_Q complex.
 */
ls_status ls_pairsum_dev(ls_op* op, const void* f_dev, void* y_dev);

/*
 * Full solve for R right-hand sides with host buffers (Eq. nystrom_linear_system):
 *   b          [R][N_Q] complex right-hand sides, or NULL for the plane waves
 *              b_j = u_inc(y_j) = exp(i k d . y_j), d = (cos a, sin a), a = dir_angles[r]
 *   dir_angles [R] (unused when b is given, may then be NULL);  ff_angles [n_ff]
 *   u_out    [R][N_Q] complex total field at the nodes (may be NULL)
 *   uinf_out [R][n_ff] complex far-field pattern
 *            u_inf(t) = -k^2 e^{i pi/4} / sqrt(8 pi k) sum_j w_j m_j u_j e^{-i k (cos t, sin t) . y_j}
 *            (may be NULL)
 *   hist_out [R][max_iter + 1] relative residual estimates (may be NULL)
 *   iters_out [R] iterations taken (may be NULL)
 * Every GMRES solve ends with an explicit residual check: ||P b - sum_i y_i P L v_i|| /
 * ||P b|| from the stored operator products (independent of the orthogonality of the
 * Krylov basis that the Givens estimate assumes); ls_op_last_residual returns the largest
 * of the last call.  Returns LS_ENOCONV when any right-hand side hit max_iter or its
 * explicit residual exceeds 10 tol (outputs are still written).
 */
ls_status ls_solve(ls_op* op, int32_t R, const double* dir_angles, const double* b, int32_t n_ff,
                   const double* ff_angles, double* u_out, double* uinf_out, double* hist_out, int32_t* iters_out);

/* y = P x (Eq. preconditioner_factored) and y = L^T x with host buffers of N_Q complex
   (the copies included); LS_EINVAL without a preconditioner for ls_apply_precond. */
ls_status ls_apply_precond(ls_op* op, const double* x, double* y);
ls_status ls_apply_transpose(ls_op* op, const double* x, double* y);

/* Adjoint solves L^T lambda_r = g_r (GMRES left-preconditioned by P^T when built) with host
   buffers g, lambda_out [R][N_Q] complex; iters_out [R] (may be NULL).  LS_ENOCONV as ls_solve. */
ls_status ls_solve_adjoint(ls_op* op, int32_t R, const double* g, double* lambda_out, int32_t* iters_out);

/* ||P (b - L u)|| / ||P b|| (without P: ||b - L u|| / ||b||) by full applies of L and P, for
   device buffers b_dev, u_dev of N_Q complex. */
ls_status ls_residual_dev(ls_op* op, const void* b_dev, const void* u_dev, double* rel);
/*
 * Ritz values of the last single-system GMRES solve on this operator (Section 6: the
 * eigenvalues of the square Hessenberg matrix H_k of k Arnoldi steps on P L, the matrix
 * whose spectrum the preconditioner clusters around 1; Figure ritz_spectrum uses 80 steps,
 * e.g. tol tiny and max_iter 80).  *count = k; with ritz [cap >= k][2] non-null the k
 * values are written (order unspecified).  Errors: LS_EINVAL (cap < k), LS_ENOCONV (the
 * QR iteration did not converge).
 */
ls_status ls_op_ritz(ls_op* op, int32_t cap, int32_t* count, double* ritz);
/* Eigenvalues of an upper Hessenberg matrix H [n][n] complex, column-major (host utility of
   ls_op_ritz: shifted QR iteration with Wilkinson shifts); eig [n] complex out. */
ls_status ls_hessenberg_eigenvalues(int32_t n, const double* H, double* eig);

/*
 * Invertibility diagnostic of the Approach II preconditioner (appendix on invertibility in
 * practice, Eq. rho_def): for R grid vectors x_dev [R][nx * ny] complex (the caller draws them,
 * e.g. standard complex normal), w = R_II x = D^{-1} (T_C^Q)^T T_C^Q x and
 *   rho = <S^(C) w, w>_D / <w, w>_D,   <x, y>_D = x^* D y (Eq. D_inner_product),
 * S^(C) w = C^{-1} A w; rho [R][2] (re, im) on the host.  Errors: LS_EINVAL without a
 * preconditioner (or on a purely Cartesian operator).
 */
ls_status ls_precond_rho_dev(ls_op* op, int32_t R, const void* x_dev, double* rho);

/* Largest explicit residual (see ls_solve) of the last single-system solve call. */
ls_status ls_op_last_residual(const ls_op* op, double* rel);

/*
 * Device-buffer solve for R right-hand sides b_dev [R][N_Q] complex; writes
 * u_dev [R][N_Q] and, if n_ff > 0, uinf_dev [R][n_ff] (ff_angles on the host).
 * iters_out [R] on the host (may be NULL).
 */
ls_status ls_solve_dev(ls_op* op, int32_t R, const void* b_dev, void* u_dev,
                       int32_t n_ff, const double* ff_angles, void* uinf_dev, int32_t* iters_out);

/*
 * Batching form: R right-hand sides of one operator advanced together.
 *   ls_pairsum_batch_dev  y_r = (i/4) sum_{n != j} H0 w_n f_r,n for f_dev, y_dev [R][N]
 *   ls_solve_batch_dev    R independent GMRES solves in lock step (each system
 *                         keeps its own Krylov space, Hessenberg matrix and stop),
 *                         b_dev, u_dev [R][N]; far field as ls_solve_dev
 * The pair sum of all R systems is one launch per iteration on the kernel chosen
 * by ls_op_set_batch_kernel.  Kinds 0 and 1 take each H(j, n) from an FP32 table
 * (degree 6, validated to 2e-8) with double-float t.  On the CUDA cores (kind 0) it
 * is applied to blocks of 8 right-hand sides with Kahan-compensated FP32 sums over
 * runs of 64 sources and FP64 across runs; on the tensor cores (kind 1, the default)
 * the sum over sources is a tcgen05 GEMM over up to 64 right-hand sides.  Kind 2 is
 * the double-float (FP64-accurate) CUDA-core kernel.  Solves on kind 1 (and on kind 0
 * under ls_op_set_batch_refine(op, 1)) are followed by iterative refinement: against
 * the batched double-float operator by default on operators in the double-float or
 * mixed form (solutions FP64-accurate to tol), else against the kind 0 operator (~1e-6,
 * the per-entry FP32 rounding of H0).  The batching form's target is <= 1e-6 relative
 * solution error.  The preconditioner sweeps and the Arnoldi kernels are batched over
 * r as well.  Workspace grows on first use with a larger R.
 */
ls_status ls_pairsum_batch_dev(ls_op* op, int32_t R, const void* f_dev, void* y_dev);
ls_status ls_solve_batch_dev(ls_op* op, int32_t R, const void* b_dev, void* u_dev, int32_t n_ff,
                             const double* ff_angles, void* uinf_dev, int32_t* iters_out);

/*
 * Several scatterers (operators of uneven size, own k and mesh) with R right-hand
 * sides each, advanced in lock step; every iteration runs ONE persistent pair-sum
 * launch over all (scatterer, target block, source chunk[, RHS block]) work units,
 * followed by each operator's batched epilogue, preconditioner and Arnoldi kernels.
 * Kernel as set on ops[0] by ls_op_set_batch_kernel (0 or 1): tensor cores (one CTA
 * per SM taking units round-robin) or CUDA cores (units fetched from an atomic
 * counter, grid size autotuned on the first iteration); afterwards each operator's
 * iterative refinement as ls_solve_batch_dev runs it (ls_op_set_batch_refine).
 *   ops [S]; b_devs[s], u_devs[s]: [R][N_s] complex; iters_out [S][R] (may be NULL)
 * All operators must share one stream and max_iter.  LS_ENOCONV if any system
 * hit max_iter.
 */
ls_status ls_solve_multi_dev(int32_t S, ls_op* const* ops, int32_t R, const void* const* b_devs,
                             void* const* u_devs, int32_t* iters_out);

/*
 * Differentiation form (the paper has no adjoint; this follows from
 * Eq. linear_system_matrix: L(m) = I + k^2 V diag(m), V independent of m).
 *   ls_apply_transpose_dev          y = L^T x = x + k^2 diag(m) V^T x
 *   ls_potential_transpose_dev      y = V^T x (the pair sum is symmetric up to
 *                                   the weights: (K^T x)_n = w_n sum_j G(y_n, y_j) x_j)
 *   ls_apply_precond_transpose_dev  y = P^T x = x + T_Q^C^T (A^T C^{-T} - I) T_C^Q^T x
 *   ls_solve_transpose_dev          L^T lambda = g for R right-hand sides g_dev [R][N],
 *                                   GMRES left-preconditioned by P^T when built
 * Device buffers of N complex (R x N for the solve); x and y may not alias.
 */
ls_status ls_apply_transpose_dev(ls_op* op, const void* x_dev, void* y_dev);
ls_status ls_potential_transpose_dev(ls_op* op, const void* x_dev, void* y_dev);
ls_status ls_apply_precond_transpose_dev(ls_op* op, const void* x_dev, void* y_dev);
ls_status ls_solve_transpose_dev(ls_op* op, int32_t R, const void* g_dev, void* lambda_dev, int32_t* iters_out);

/*
 * Replace the nodal contrast m (host, [N] complex).  The correction dV and the
 * H0 table do not depend on m; the preconditioner keeps the grid contrast it
 * was built with (it stays a valid preconditioner, only its quality changes).
 */
ls_status ls_op_set_contrast(ls_op* op, const double* m);

/* Replace the nodal contrast from a device buffer: m_dev [N] complex, or [N] double
   (the real part, imaginary part zero) when real_only; same semantics as ls_op_set_contrast. */
ls_status ls_op_set_contrast_dev(ls_op* op, const void* m_dev, int32_t real_only);

/* Far-field misfit on device buffers of `total` complex entries (e.g. R x n_ff):
   resid_dev = uinf_dev - target_dev and *J = 1/2 sum |resid|^2 (reduced in a fixed order). */
ls_status ls_misfit_dev(ls_op* op, int32_t total, const void* uinf_dev, const void* target_dev, void* resid_dev,
                        double* J);

/* b_dev [R][N] = exp(i k d . y_j), d = (cos a, sin a) for the R angles (host). */
ls_status ls_incident_dev(ls_op* op, int32_t R, const double* dir_angles, void* b_dev);

/*
 * Gradient of J = 1/2 sum_r sum_a |u_inf^(r)(theta_a) - t_a^(r)|^2 with respect to
 * the real part of each nodal contrast:
 *   grad_j = Re sum_r u_j^(r) [g_j^(r) - k^2 (V^T lambda^(r))_j],
 *   g^(r) = A^T conj(res^(r)),  L^T lambda^(r) = m * g^(r),
 *   A_aj = -k^2 e^{i pi/4} / sqrt(8 pi k) w_j e^{-i k xhat_a . y_j}.
 *   u_dev [R][N] forward solutions; resid_dev [R][n_ff] = u_inf - targets;
 *   ff_angles [n_ff] (host); grad_dev [N] double (overwritten); iters_out [R]
 *   adjoint GMRES iterations (may be NULL).  Only u and lambda are stored.
 */
ls_status ls_misfit_gradient_dev(ls_op* op, int32_t R, const void* u_dev, int32_t n_ff, const double* ff_angles,
                                 const void* resid_dev, double* grad_dev, int32_t* iters_out);

/*
 * Batched versions for many incident directions: the R transposed systems advance
 * in lock step with one batched pair-sum launch per iteration (the FP32 batched
 * kernel of ls_solve_batch_dev on unit weights, P^T batched likewise).
 *   ls_solve_transpose_batch_dev   L^T lambda_r = g_r, g_dev, lambda_dev [R][N]
 *   ls_misfit_gradient_batch_dev   as ls_misfit_gradient_dev with the batched adjoint solve
 */
ls_status ls_solve_transpose_batch_dev(ls_op* op, int32_t R, const void* g_dev, void* lambda_dev, int32_t* iters_out);

/*
 * Kernel of the batched pair sum (ls_pairsum_batch_dev, ls_solve_batch_dev,
 * ls_solve_multi_dev and the batched transposed solves):
 *   kind 0  CUDA cores: FP32 H0 table, Kahan-compensated FP32 sums per (target, RHS)
 *           (pair sum within ~1e-7 of the FP64 one)
 *   kind 1  tensor cores (default): the sum over sources as a GEMM on tcgen05
 *           kind::tf32 with 3-term TF32 splits of H and of the densities, FP32
 *           accumulation in tensor memory restarted every `fold` stages of 16
 *           sources, run totals Kahan-folded, chunks summed in FP64.  The tensor
 *           memory accumulation truncates, so the pair sum carries ~3e-7 x fold
 *           relative error; batched solves on kind 1 are therefore followed by up
 *           to `refine` steps of iterative refinement (refine = 0: none) whose
 *           residuals use the operator ls_op_set_batch_refine selects: the batched
 *           double-float one (default on double-float and mixed operators; the
 *           refinement stops at ||P r|| <= tol ||P b||) or the kind 0 one (stops at
 *           max(tol, 2e-8), or when a correction no longer halves the residual while
 *           ||P r|| <= 1e-6 ||P b||: the kind 0 operator's rounding level).
 *           LS_ENOCONV if the refinement does not stop within `refine` steps.  On
 *           kind 1 the block-LU sweeps of the preconditioner run in FP32 (FP32
 *           copies of the factors, made on first use); P only weights the residual
 *           norm, so the refined solution keeps the refinement operator's accuracy.
 *           Kind 0 keeps the FP64 sweeps.
 *   kind 2  CUDA cores in double-float (FP64-accurate): H from the operator's
 *           double-float table, densities and sums in double-float pairs; needs an
 *           operator built with LS_PREC_FP64_DF or LS_PREC_MIXED (LS_EINVAL
 *           otherwise; switching the operator away from them resets kind 2 to 0);
 *           no refinement; single-operator solves only (ls_solve_multi_dev takes 0
 *           or 1).  The same kernel forms the refinement residuals of kinds 0 and 1
 *           under ls_op_set_batch_refine(op, 1) on such operators.
 * Defaults: kind 1, fold 4, refine 4.
 * Errors: LS_EINVAL for kind outside {0, 1, 2}, fold < 1 or refine < 0.  A stalled
 * tensor-core pipeline (every wait in the kernel is bounded) makes the next call
 * that synchronises return LS_ETIMEOUT.
 */
ls_status ls_op_set_batch_kernel(ls_op* op, int32_t kind, int32_t fold, int32_t refine);

/*
 * Operator of the batched solves' iterative refinement (ls_solve_batch_dev,
 * ls_solve_multi_dev on the tensor cores, ls_solve_transpose_batch_dev).  Default: 1 on
 * operators in the double-float or mixed form, 0 otherwise, following ls_op_set_pairsum
 * until this call fixes it.
 *   accurate = 0            the kind 0 batched FP32 operator (one launch for all R systems;
 *                           solutions ~1e-6 from the FP64 ones: the per-entry FP32 rounding
 *                           of H0 limits them)
 *   accurate = 1            an FP64-accurate operator: on an operator built with
 *                           LS_PREC_FP64_DF or LS_PREC_MIXED the batched double-float pair
 *                           sum (batch kernel 2's) over all R systems, on the FP64 forms the
 *                           single-RHS pair sum one system after the other; the refined
 *                           solutions meet tol against the FP64 operator.  Also refines the
 *                           kind 0 solves.  Stops at ||P r|| <= tol ||P b|| (no 2e-8 floor).
 * Errors: LS_EINVAL (accurate not 0 or 1, a purely Cartesian operator).
 */
ls_status ls_op_set_batch_refine(ls_op* op, int32_t accurate);

/*
 * Failure-detection test hook of the tensor-core pair sum (no counterpart in the
 * paper).  With stall_ms > 0 the MMA issuer of every following tensor-core launch
 * on this operator first waits stall_ms on a barrier that nothing completes; the
 * wait is bounded like every other wait of the pipeline, so it runs out, the CTA
 * raises its abort flag, the other roles leave their (abort-aware, bounded) waits,
 * issued bulk copies are drained, tensor memory is freed, and the call returns
 * LS_ETIMEOUT.  The error word is cleared when reported, so after
 * ls_op_set_stall_test(op, 0) the next call succeeds on the same context.
 * Errors: LS_EINVAL for stall_ms outside [0, 1000].
 */
ls_status ls_op_set_stall_test(ls_op* op, double stall_ms);

/*
 * Self-check of the tensor-core MMA path (no counterpart in the paper): one
 * 128 x N x 32 product of exactly representable values through the shared-memory
 * layouts, descriptors and tcgen05.mma / tcgen05.ld sequence of the batched pair
 * sum, compared with the host product.  *max_abs_err = 0 when the path is right.
 * N a multiple of 16 in [16, 256].  Synchronises the device.
 */
ls_status ls_tc_gemm_check(int32_t N, double* max_abs_err);
ls_status ls_misfit_gradient_batch_dev(ls_op* op, int32_t R, const void* u_dev, int32_t n_ff, const double* ff_angles,
                                       const void* resid_dev, double* grad_dev, int32_t* iters_out);

/*
 * Export of the correction dV as CSR (rows = N_Q targets, columns = nodes).
 * Call with null arrays to get the size in *nnz, then with rowptr [N_Q + 1],
 * cols [nnz], vals [nnz][2] (complex) to copy it out.
 */
ls_status ls_op_correction(const ls_op* op, int64_t* nnz, int64_t* rowptr, int32_t* cols, double* vals);

/*
 * Host-only build of the correction dV for a mesh (no device work): the same
 * setup ls_operator_create runs (extended precision, OpenMP).  Two-call size
 * query as ls_op_correction: null arrays return the size in *nnz (only the
 * patches are planned, no values computed).  The values are recomputed on every
 * call that asks for them.
 */
ls_status ls_correction_host(const ls_mesh* mesh, double k, double kappa, int64_t* nnz,
                             int64_t* rowptr, int32_t* cols, double* vals);

/*
 * Host-only build of the Cartesian preconditioner's sparsifying stencils and of
 * the banded C = A L^(C) (Section 4: Eq. sparsifying_min on the neighbourhoods of
 * Eq. cart_neighbors_LS, Eq. LC_def), the same setup ls_operator_create runs,
 * for checking on machines without a GPU.
 *   box [4] = (x0, x1, y0, y1), nx x ny grid nodes including the box edges
 *   m_grid [nx*ny][2]   contrast at the grid nodes (complex, index a + nx b)
 *   stencils [9][9][2]  out: stencil of row class c = ca + 3 cb (ca = 0 / 1 / 2 for
 *                       the first / an inner / the last column; cb likewise for
 *                       rows) at offset (da+1) + 3 (db+1); zero outside the grid
 *   cband [ny][9][nx][2] out (or null): C((a, b), (a+da, b+db)) at
 *                       [b][(db+1) 3 + (da+1)][a]
 * Stencils are unit vectors fixed up to a complex phase per class (C rows carry
 * the same phase).  Errors: LS_EINVAL (null arguments, k <= 0, a grid smaller
 * than 4 x 4, unequal steps, quadrature nodes outside the box).
 */
ls_status ls_grid_host(const ls_mesh* mesh, double k, const double* box, int32_t nx, int32_t ny, const double* m_grid,
                       double* stencils, double* cband);

/*
 * Device build of the correction dV for a mesh (the setup ls_operator_create runs when
 * params->setup_on_device): per (target, subdomain patch) block the Green's-identity
 * boundary moments and the plain-quadrature patch moments in double-double arithmetic
 * on the GPU, combined with the host's long-double coefficient matrices.  Same CSR
 * layout and two-call size query as ls_correction_host (the size query does no device
 * work); values recomputed on every call that asks for them.  *host_blocks (may be
 * NULL) receives the number of blocks rebuilt on the host
 * (those whose patch reaches k r > 32, beyond the device series).
 * Errors: LS_EINVAL (null arguments, k <= 0), LS_ECUDA, LS_ESINGULAR.
 */
ls_status ls_correction_dev(const ls_mesh* mesh, double k, double kappa, void* stream, int64_t* nnz,
                            int64_t* rowptr, int32_t* cols, double* vals, int64_t* host_blocks);

/*
 * Host-only build of the transfer T_Q^C from the quadrature nodes to the grid (no device
 * work), as a CSR over the nx * ny grid rows (x fastest), two-call size query as
 * ls_correction_host:
 *   approach 2  Approach II, D^{-1} (T_C^Q)^T (Eq. T_H^C_def, Eq. D_def), T_C^Q bilinear
 *   approach 1  Approach I, E_C (M^tri)^{-1} E_Q^T W (Eq. T_HC_proj_def): a grid node inside
 *               element t (Newton inverse of t's curved map in the closed reference triangle,
 *               lowest element index on shared edges) takes w_q sum phi_i(z) (M^t)^{-1}_{ii'}
 *               phi_i'(y_q) over t's 15 nodes, phi the P1 basis of t's vertices and M^t the
 *               straight-triangle mass matrix (Eq. mass_closed_form); other rows are empty.
 * *n_interior (may be NULL): grid nodes inside the mesh (approach 1) or with a nonzero
 * T_C^Q column (approach 2).  Errors: LS_EINVAL (null arguments, bad grid, approach).
 */
ls_status ls_transfer_host(const ls_mesh* mesh, const double* box, int32_t nx, int32_t ny, int32_t approach,
                           int64_t* nnz, int64_t* rowptr, int32_t* cols, double* vals, int32_t* n_interior);

/* Diagnostic: h_dev[i] = H0^(1)(z_dev[i]) (complex) by the device routine of the pair sum. */
ls_status ls_hankel0_dev(int64_t n, const double* z_dev, void* h_dev, void* stream);

/* Switch the pair-sum kernel of an operator (LS_PREC_* as ls_params.prec); rebuilds the H0 table. */
ls_status ls_op_set_pairsum(ls_op* op, int32_t mode);

/*
 * Symmetry of the single-RHS table pair sums (LS_PREC_FP64_DF, LS_PREC_FP32 and both
 * operators of LS_PREC_MIXED).  on = 1 (default): H0(k |y_i - y_j|) is evaluated once per unordered pair
 * and feeds both y_i (with s_j) and y_j (with s_i), half the Hankel evaluations; the
 * result is deterministic (no atomics) and equal to the on = 0 sum up to the order of
 * the floating-point additions.  on = 0: every ordered pair is evaluated.  Errors:
 * LS_EINVAL (on not 0 or 1).
 */
ls_status ls_op_set_pair_symmetry(ls_op* op, int32_t on);

/*
 * Instrumentation.  ls_op_set_timing(op, on) resets the counters and, when on,
 * brackets every pair-sum launch with CUDA events on the operator's stream.
 * ls_op_stats returns the summed pair-sum kernel time (ms, event-measured),
 * the number of pair-sum launches and the number of kernels this operator
 * launched since the last reset (any pointer may be NULL).
 */
ls_status ls_op_set_timing(ls_op* op, int32_t on);
/* Wall time (s) of the setup phases: [0] correction dV (host), [1] grid transfers, stencil and C
   (host), [2] block LU of C and its transposes (device), [3] H0 table. */
ls_status ls_op_setup_times(const ls_op* op, double* t4);
/* Pair-sum autotuner result: coefficients per cell of the H0 table in use and the timed
   pair-sum launch (ms, scaled from a bounded sample of sources) of the 12-, 10-, 9- and
   (double-float form only) 8-coefficient candidates, cand_ms [4] (0 = not tried); *fp32_tail:
   in the double-float form, the top coefficients of each Horner chain summed in plain FP32
   (their terms stay below 2^-50 of |H0| on every cell; 0 otherwise).  Pointers may be NULL. */
ls_status ls_op_tuning(const ls_op* op, int32_t* table_ncoef, double* cand_ms, int32_t* fp32_tail);
ls_status ls_op_stats(ls_op* op, double* pairsum_ms, int64_t* pairsum_launches, int64_t* launches);
/* The same restricted to the timed pair-sum launches of one arithmetic: kind = LS_PREC_* of the
   kernel that ran (the mixed form's inner launches count as LS_PREC_FP32, its residuals as
   LS_PREC_FP64_DF), 10 = the CUDA-core batched kernel, 11 = the tensor-core batched kernel. */
ls_status ls_op_stats_kind(ls_op* op, int32_t kind, double* pairsum_ms, int64_t* pairsum_launches);

/* Diagnostic: measured FP64 FMA throughput of the device in GFLOP/s (2 flops per FMA). */
ls_status ls_probe_fp64(double* gflops, void* stream);

/*
 * Allocation-free pair sum, for callers that cannot allocate device memory:
 * plug-ins whose device memory is owned by a host application's allocator or a
 * fixed pool, real-time loops that must stay out of the allocator (its latency
 * is unbounded).  No counterpart in the paper; it computes the
 * same sum as ls_pairsum_dev, y_j = (i/4) sum_{n != j} H0^(1)(k |x_j - x_n|) w_n f_n,
 * with the direct FP64 H0 routine and without an operator:
 *   n          number of nodes, 2 <= n <= 1048576 (larger n: LS_EINVAL)
 *   xy_dev     [n][2] double node coordinates, w_dev [n] double weights
 *   f_dev      [n] complex density, y_dev [n] complex output (may not alias f)
 *   k          wavenumber > 0;  stream: cudaStream_t (NULL = default)
 * Its scratch (chunked partial sums) lives in a file-scope __device__ array of
 * 16 MiB that every GPU loading the library keeps until the process exits; no
 * cudaMalloc/cudaFree or allocating library routine is called.  The first call
 * on a device looks up the array's address with cudaGetSymbolAddress (make it
 * before any stream capture).  All calls share the array: calls that overlap on
 * the GPU (other streams, other host threads) race; serialise them.  Every
 * partial is overwritten before it is read, so no clearing is needed.  Like the
 * other device-buffer calls it returns after synchronising the stream.
 * Errors: LS_EINVAL (null pointer, n out of range, k <= 0), LS_ECUDA.
 */
ls_status ls_pairsum_noalloc(int32_t n, const double* xy_dev, const double* w_dev, const void* f_dev,
                             double k, void* y_dev, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* ls_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LSGPU_H */
