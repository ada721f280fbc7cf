/*
 * birkhoff.h -- C ABI of the GB300 Birkhoff trajectory-optimisation hot path.
 *
 * Method: arXiv 2509.01855, "A Million-Point Fast Trajectory Optimization Solver".
 * The library computes, on one GPU, the matrix-free Birkhoff products B v and B^T v on a
 * Chebyshev-Gauss-Lobatto (CGL) grid, the KKT operator of a Newton step built from them, the
 * Birkhoff preconditioner, a right-preconditioned Krylov solve and the Newton driver, which
 * also handles bounds on the controls and one-sided bounds on terminal conditions (the simplest
 * inequalities of the paper's general problem (P)) by logarithmic barriers.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Grid: N is a power of two, 4 <= N <= 2^24, or any other N with 4 <= N <= 2^22 (BK_F64) or
 *    2^23 (BK_F32); the L = N + 1 CGL nodes are
 *    tau_j = -cos(j pi / N), ascending (Eq. CGLpts), mapped to t_j = t0 + s (tau_j + 1),
 *    s = (tf - t0) / 2.
 *  - Vectors are device pointers owned by the caller, one length-L block per component,
 *    blocks `pitch` elements apart (pitch >= L; the library's own default pitch is L rounded up
 *    to a multiple of 32). Elements L..pitch-1 of every block are ignored on input; outputs
 *    written by the library set them to zero. Pointers must be 16-byte aligned.
 *  - dtype: BK_F64 = IEEE binary64 arithmetic and storage, BK_F32 = binary32.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Every call
 *    is asynchronous on that stream unless stated otherwise; nothing synchronises the device
 *    except where a call says so.
 *  - Errors: every call returns a bk_status; BK_OK = 0 on success. On error nothing is written
 *    to outputs that the caller can rely on, and bk_last_error() returns a thread-local
 *    message. Calls never exit the process. A CUDA error from a launch is returned as
 *    BK_ERR_CUDA.
 *  - Ownership: plans and problems are created and freed by the library (they own their
 *    device tables and scratch); all vectors and workspaces are the caller's.
 */
#ifndef BIRKHOFF_GB300_H
#define BIRKHOFF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bk_plan bk_plan;
typedef struct bk_problem bk_problem;

typedef enum { BK_F64 = 0, BK_F32 = 1 } bk_dtype;

typedef enum {
  BK_OK = 0,
  BK_ERR_ARG = 1,            /* invalid argument (size, pointer, alignment, enum)          */
  BK_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed                */
  BK_ERR_OOM = 3,            /* device allocation failed                                    */
  BK_ERR_NOT_CONVERGED = 4,  /* iteration cap reached before the tolerance                  */
  BK_ERR_TIMEOUT = 5,        /* a bounded device wait gave up                               */
  BK_ERR_INFEASIBLE = 6,     /* the line search could not reduce the residual               */
  BK_ERR_UNSUPPORTED = 7     /* valid request the library does not implement               */
} bk_status;

/* Thread-local text of the last error (never NULL). */
const char* bk_last_error(void);

/* Library version string. */
const char* bk_version(void);

/* Number of kernels this library has launched in this process (all threads, all devices). A
 * diagnostic for benchmarks: the difference across a region counts the library's launches. */
uint64_t bk_launch_count(void);

/* ------------------------------------------------------------------------------------------
 * Plan: grid tables (nodes, Clenshaw-Curtis weights, DCT twiddles) and transform scratch.
 * ------------------------------------------------------------------------------------------ */

/* Create a plan for Birkhoff products on the CGL grid of size N over [t0, tf].
 *   N          power of two, 4 <= N <= 2^24, or any other N in [4, 2^22] (BK_F64) / [4, 2^23]
 *              (BK_F32). A power of two takes the FFT chain (bk_plan_set_dense switches a plan
 *              with N <= 1024 to the dense product: BK_F32 on the tensor cores, BK_F64 on the
 *              CUDA cores); any other N <= 1024 takes the dense product in both precisions (B^a
 *              formed once in FP64 from its definition: Chebyshev coefficients of the Lagrange
 *              basis times the closed-form integrals of T_k, Eq. intChebPoly=); any other
 *              N > 1024 computes each DCT-I's length-N DFT by Bluestein's identity as a circular
 *              convolution of length M (a power of two, M >= 2N - 1) on the four-step FFT, with
 *              the chirp exp(-i pi j^2 / N) and the convolution kernel's spectrum as plan tables
 *              (about 4-8x the work of the nearest power of two)
 *   n_comp     components per batch item (>= 1)
 *   max_batch  largest `batch` later passed to birkhoff_apply / birkhoff_apply_T (>= 1); the
 *              plan's scratch is sized for max_batch * n_comp vectors
 *   dtype      arithmetic and storage type
 *   t0, tf     time interval, tf != t0 (s = (tf - t0) / 2 scales B)
 *   pitch      distance in elements between component blocks; 0 = default (L rounded up to
 *              32); otherwise pitch >= N + 1 and pitch * sizeof(dtype) a multiple of 16
 *   stream     stream for the table-building kernels; the call synchronises it before return
 * The grid tables are computed on the device (nodes and weights in FP64, copied to FP32 for a
 * BK_F32 plan). Section "Fast Computation of Birkhoff Matrix-Vector Products". */
bk_status bk_plan_create(bk_plan** plan, int64_t N, int n_comp, int max_batch, bk_dtype dtype,
                         double t0, double tf, int64_t pitch, void* stream);

/* Free a plan (NULL is allowed). The caller must make sure no work using it is in flight. */
void bk_plan_destroy(bk_plan* plan);

/* Grid facts of a plan: N, L, pitch, dtype. Any output pointer may be NULL. */
bk_status bk_plan_info(const bk_plan* plan, int64_t* N, int64_t* L, int64_t* pitch,
                       int* dtype);

/* Copy the L node times t_j (FP64) and the L Clenshaw-Curtis weights w_j (FP64, tau-domain,
 * sum 2; last row of B^a per the remark after Eq. Ba=10) to HOST arrays; either may be NULL.
 * Synchronous. */
bk_status bk_plan_grid(const bk_plan* plan, double* t_host, double* w_host);

/* out = B v for `batch * n_comp` vectors, B = s * B^a (Eq. manyDefs; FastBV).
 *   v, out  device arrays [batch][n_comp][pitch] of the plan's dtype; v == out is allowed
 *   batch   1 <= batch <= max_batch
 * Row 0 of the result is 0 and (B 1)_j = t_j - t0. Computed as a DCT-I to Chebyshev
 * coefficients (Fastv2a, Appendix B), the coefficient-integration stencil with the aliasing
 * fold (Eqs. c_k=bydef, chatk=) and a DCT-I back to nodal values (Fasta2v); the constant
 * coefficient c_0 is obtained by making the value at tau = -1 vanish, which is what its
 * closed form in Eq. c_k=bydef does. */
bk_status birkhoff_apply(const bk_plan* plan, const void* v, void* out, int batch, void* stream);

/* B v (trans = 0) or B^T v (trans = 1) for `count` plans of one dtype whose N may all differ,
 * e.g. the requests of a serving batch: entry i computes out[i] = B_i v[i] for batch[i]
 * vectors of plans[i], exactly as birkhoff_apply(_T)(plans[i], v[i], out[i], batch[i]) would
 * (bitwise the same values). Plans on the single-CTA path run in one launch, plans on the
 * unsplit four-step path in one launch per pass (five), each per 16 plans; dense, Bluestein,
 * split and double-float plans run their own launches within the call.
 *   plans, v, out, batch   host arrays of `count` entries (1 <= count <= 4096); v[i], out[i]
 *                          device arrays as for birkhoff_apply; v[i] == out[i] is allowed, but
 *                          different entries' vectors must not overlap
 * A four-step plan may appear only once per call (it owns the scratch its passes use); all
 * plans must have the same dtype. BK_ERR_ARG otherwise, before any work is queued. */
bk_status birkhoff_apply_batch(const bk_plan* const* plans, const void* const* v, void* const* out,
                               const int* batch, int count, int trans, void* stream);

/* out = B v for callers that cannot allocate device memory. The paper has no counterpart: this
 * entry point exists for programs that must not call cudaMalloc once they are running, such as
 * real-time or flight control loops whose device memory budget is fixed at start-up, or host
 * applications whose own allocator owns the whole GPU. Such callers cannot create a bk_plan,
 * because plan creation allocates its tables and scratch.
 *   v, out     device arrays of nvec FP64 vectors, `pitch` elements apart (caller-owned; the
 *              library allocates nothing); the two ranges (nvec * pitch doubles each) must
 *              not overlap (BK_ERR_ARG)
 *   N          power of two, 8192 <= N <= 65536;  nvec: 1..8;  pitch >= N + 1, even
 *   t0, tf     time interval (B = s B^a, s = (tf - t0) / 2)
 * The twiddle tables and the transform scratch live in one 16 MiB array that the library
 * reserves statically on every GPU that loads it, for the life of the process. Sizes beyond the
 * limits above are rejected with BK_ERR_ARG before any work is queued. The first call on a
 * device does a one-time set-up (looks up the array's device address and sets the kernels'
 * shared-memory limits), so make that first call before any stream capture. All calls on a
 * device share the array, which keeps the last call's contents; every call rewrites all of it
 * before reading it, so nothing needs clearing, but calls whose work overlaps on the GPU (other
 * streams, or other host threads) race on it and must be serialised by the caller. */
bk_status birkhoff_apply_noalloc(const double* v, double* out, int64_t N, int nvec, int64_t pitch,
                                 double t0, double tf, void* stream);

/* out = B^T v, the exact transpose of birkhoff_apply (the paper has no transpose product; the
 * KKT operator needs one). Same arguments and layout as birkhoff_apply. */
bk_status birkhoff_apply_T(const bk_plan* plan, const void* v, void* out, int batch,
                           void* stream);

/* out = B^b v, the b-form Birkhoff product (Eqs. xN=Birka+b, birk-conditions, manyDefs): the
 * b-form basis B^b_j vanishes at the final point tau^b = 1 instead of tau^a = -1, so
 * B^b = B^a - 1 w^T (w the Clenshaw-Curtis weights), and B^b v = B v - (B v)_N 1: the a-form
 * chain, then the last node's value subtracted (x = x^b 1 + B^b V discretises the dynamics
 * backwards from the final state). Same arguments, layout and errors as birkhoff_apply;
 * v == out is allowed. Row N of the result is 0 and (B^b 1)_j = t_j - tf. */
bk_status birkhoff_apply_b(const bk_plan* plan, const void* v, void* out, int batch, void* stream);

/* out = (B^b)^T v = B^T v - s (1 . v) w, the exact transpose of birkhoff_apply_b. */
bk_status birkhoff_apply_b_T(const bk_plan* plan, const void* v, void* out, int batch, void* stream);

/* Switch a plan with N <= 1024 between the FFT chain (on = 0) and the dense product (on = 1)
 * for birkhoff_apply, birkhoff_apply_T and every operator built on the plan. The dense path
 * multiplies by B^a itself (the matrix of Eq. manyDefs, formed once in FP64 from its
 * definition). BK_F32: B^a split into two TF32 parts, three tcgen05 TF32 products per block
 * accumulated in FP32; BK_F64: FP64 FMAs on the CUDA cores (tcgen05 has no FP64 kind). The
 * paper's Fig. 5 compares FastBV with the dense product on a CPU. The first switch on builds the
 * tables (two N+1 x N+1 matrices of 8-byte entries, ~17-19 MB at N = 1024) on `stream` and
 * synchronises it; the plan owns them. Errors: BK_ERR_UNSUPPORTED for N > 1024, or on = 0 for
 * an N that is not a power of two; BK_ERR_OOM; BK_ERR_CUDA. Not thread safe against applies of
 * the same plan in flight. */
bk_status bk_plan_set_dense(bk_plan* plan, int on, void* stream);

/* How a plan computes its products. *path: 0 one CTA per vector (small N), 1 four-step FFT,
 * 2 four-step with the split DCT-I, 3 dense product, 4 Bluestein convolution (N not a power of
 * two above 1024). For paths 1 and 2: the FFT
 * factors N1 x N2 of the (even-half) transform and the complex elements per CTA, as chosen by
 * the tile autotuner at plan creation (or by the occupancy heuristic when tuning is off:
 * environment BK_AUTOTUNE=0). Outputs may be NULL. */
bk_status bk_plan_shape(const bk_plan* plan, int* path, int* N1, int* N2, int* elems);

/* *on = 1 while the plan's products take the dense path, else 0. Plans of an N that is not a
 * power of two are always dense; power-of-two plans start on the FFT chain, or, when the
 * environment variable BK_DENSE=1 is set at plan creation, on the dense path (N <= 1024 and
 * n_comp * max_batch <= 16). */
bk_status bk_plan_dense_state(const bk_plan* plan, int* on);

/* Arithmetic of the FP64 transforms for plans (and problems) created after the call:
 *   mode 1: four-step FP64 plans (powers of two, N >= 256) compute their DCTs in double-float
 *           arithmetic, each value the unevaluated sum of two binary32 numbers (48 significand
 *           bits; Knuth's TwoSum, Dekker's FastTwoSum and an FMA product), on the FP32 pipe,
 *           which GB300 runs 64 times as fast as its FP64 pipe. Vectors stay binary64 in
 *           memory. Products agree with binary64 ones to ~1e-14 relative (2-norm).
 *   mode 0: IEEE binary64 arithmetic throughout.
 *   mode -1 (the default): double-float for N >= 2^18, where it measured faster (1.8x at
 *           2^20), binary64 below (the environment variable BK_F64_DF=0 selects mode 0).
 * Single-CTA plans (N <= 128) and dense products always use binary64. Host only; BK_ERR_ARG for
 * any other mode. This is the library's choice of arithmetic; the paper's method is exact FP64. */
bk_status bk_set_f64_transform(int mode);

/* *mode = 1 when the plan's transforms use double-float arithmetic, else 0. */
bk_status bk_plan_f64_mode(const bk_plan* plan, int* mode);

/* Test mode of the dense tensor-core product (BK_F32 plans on the dense path): while on = 1,
 * every product first makes one bounded wait on a barrier that nothing signals (1024 polls),
 * takes the kernel's timeout path (drains its copies in flight, frees its tensor memory, writes
 * the error word) and leaves its output invalid. For tests of the failure path: the error word
 * reaches bk_plan_dense_check, and krylov_solve / newton_solve on a dense problem return
 * BK_ERR_TIMEOUT. Plans created while the environment variable BK_DENSE_TEST_TIMEOUT=1 is set
 * (problems' plans included) start in this mode. The paper has no counterpart. */
bk_status bk_plan_dense_test_timeout(bk_plan* plan, int on);

/* Read (and clear) the dense kernel's error word: *err = 0 when every dense product so far
 * completed; otherwise a wait inside the kernel ran out (1: operand copy or MMA completion,
 * 2: accumulator read) and that product's output is not valid. Synchronous (device sync).
 * krylov_solve and newton_solve read the same word of their problem's plans before returning
 * and fail with BK_ERR_TIMEOUT when it is set. */
bk_status bk_plan_dense_check(const bk_plan* plan, int* err);

/* ------------------------------------------------------------------------------------------
 * Problems: dynamics x' = f(x, u) of Eq. probPbold, discretised by Eq. Prob-PNa.
 * ------------------------------------------------------------------------------------------ */

typedef enum {
  BK_DBL_INT = 0,   /* x = (p, v), x' = (v, u); x(t0) = (0,0); x(tf) = (1,0); F = u^2/2        */
  BK_ORBIT = 1,     /* x = (r, theta, v_r, v_theta), u = (u_r, u_theta) thrust acceleration:
                       r' = v_r, theta' = v_theta/r, v_r' = v_theta^2/r - 1/r^2 + u_r,
                       v_theta' = -v_r v_theta/r + u_theta (dynamics of Eq. ot);
                       x(t0) = (1,0,0,1); r(tf) = r_f, v_r(tf) = 0, v_theta(tf) = r_f^-1/2;
                       F = |u|^2/2.  params = {a_nominal, r_f}                              */
  BK_BILINEAR = 2,  /* scalar x' = u x, no cost, no terminal condition; linearised at (X, U)
                       its state Jacobian is diag(U): the Newton system [I - B diag(d)] dX =
                       x^a b of Eq. Newton-ivp with d = U. params = {x^a} (default 1)          */
  BK_ORBIT_MT = 3   /* minimum-time orbit transfer of Eq. ot: the BK_ORBIT state and dynamics
                       with the fixed-magnitude thrust a (sin u, cos u), u the steering angle
                       (n_u = 1); cost J = t_f - t_0 with t_f free: the time scale
                       s = (t_f - t_0)/2 is an unknown kept in the KKT vector's tail slot after
                       nu (index (2 n_x + n_u) pitch + n_e), and the tf given at creation only
                       sets the problem's initial s. params = {a, r_f}, a > 0 (the paper does
                       not give a; its target is r_f = 6). Start from bk_min_time_seed.        */
} bk_kind;

/* Operators addressed by kkt_apply / precond_apply / krylov_solve. */
typedef enum {
  BK_OP_STATE = 0,  /* state block G_x = I - s (B (x) I) J_x (FastAX; Eq. Achibetadef);
                       vectors have n_x component blocks                                   */
  BK_OP_KKT = 1     /* full KKT matrix of the Newton-Lagrange step; vectors are KKT vectors  */
} bk_op;

/* Create a problem of `kind` on the CGL grid of size N over [t0, tf], working dtype `dtype`.
 * The problem owns FP64 plans and linearisation data and, for BK_F32, FP32 copies used by the
 * Krylov iterations. Synchronises `stream`. */
bk_status bk_problem_create(bk_problem** prob, int kind, const double* params, int nparams,
                            int64_t N, bk_dtype dtype, double t0, double tf, void* stream);
void bk_problem_destroy(bk_problem* prob);

/* Change a problem's parameters and time interval in place (same kind, N and dtype) without
 * allocating: BK_ORBIT params = {a_nominal, r_f}, BK_BILINEAR params = {x^a}. The previous
 * linearisation is discarded. For request loops that reuse one problem per grid size. Host only;
 * must not overlap work queued on the problem. */
bk_status bk_problem_set_params(bk_problem* prob, const double* params, int nparams, double t0,
                                double tf);

/* Control bounds lo[q] <= u_q(t) <= hi[q] (the simplest path constraints h(x, u, t) <= 0 of
 * problem (P), Eq. probPbold; the paper states them but solves only the equality-constrained
 * Eq. Prob-PNa). They enter as a logarithmic barrier on the quadrature,
 *   J_mu = J - mu s sum_i w_i sum_q [log(u_qi - lo_q) + log(hi_q - u_qi)],
 * whose gradient joins the control rows of the residual and whose Hessian diagonal joins the
 * control block of the KKT matrix and of the preconditioner (still diagonal, so its block
 * elimination is unchanged). newton_solve then runs barrier stages (bk_problem_set_barrier).
 *   lo, hi  host arrays of n entries; -inf / +inf for a missing bound; lo[q] < hi[q]
 *   n       the problem's control count, or 0 to remove the bounds (lo, hi may be NULL then)
 * bk_kkt_residual, kkt_apply and precond_apply include the barrier terms at mu_final. Host only;
 * must not overlap work queued on the problem. BK_ERR_ARG for bad sizes or bounds;
 * BK_ERR_UNSUPPORTED for BK_BILINEAR (no cost) and BK_ORBIT_MT (free final time). */
bk_status bk_problem_set_control_bounds(bk_problem* prob, const double* lo, const double* hi,
                                        int n);

/* Endpoint bounds x_{idx_r}(t_f) >= lo[r] or <= hi[r] in place of terminal condition r (problem
 * (P)'s e^L <= e(x(t_0), x(t_f)) <= e^U, Eq. probPbold, for terminal conditions of the form
 * e_r = x_{idx_r}(t_f) - target_r, one bound per row; the paper states them but gives no
 * method). A bounded row takes the barrier psi_r(x) = -mu log(x - lo_r) (or -mu log(hi_r - x)),
 * a point term without quadrature weight, with nu_r as its multiplier: the gradient row of
 * x_{idx_r}(t_f) keeps + nu_r, and row r of the terminal block becomes the complementarity
 * condition (x - lo_r) nu_r + mu = 0 (or (hi_r - x) nu_r - mu = 0), whose Newton row
 * a dx + c dnu the preconditioner's terminal Schur complement absorbs as it is
 * (diag(a) E Q - diag(c)). Rows are the kind's terminal conditions in order (BK_DBL_INT: p, v;
 * BK_ORBIT: r, v_r, v_theta).
 *   lo, hi  host arrays of n entries; a row with lo = -inf and hi = +inf keeps its equality, a
 *           row with one finite bound (the other the matching infinity) is bounded; two finite
 *           bounds return BK_ERR_UNSUPPORTED (with one multiplier per row the two-sided barrier
 *           row stalled in the FP64 reference computation on the orbit transfer when its start
 *           lay at the bound away from the optimum)
 *   n       the problem's n_e, or 0 to restore every equality (lo, hi may be NULL then)
 * The barrier schedule is bk_problem_set_barrier's (both forms treat these rows alike);
 * newton_solve starts nu_r on the central path of mu0 and keeps its sign (negative for a lower
 * bound, positive for an upper one) by the fraction-to-boundary rule. The rows' Newton
 * coefficients are taken at each linearisation (bk_linearize reads x(t_f) and nu from z_lin,
 * synchronously, and returns BK_ERR_ARG if x(t_f) is not inside its bound). Host only; must not
 * overlap work queued on the problem; the problem must be linearised again before kkt_apply or
 * precond_apply. BK_ERR_ARG for bad sizes or bounds; BK_ERR_UNSUPPORTED for BK_BILINEAR and
 * BK_ORBIT_MT. */
bk_status bk_problem_set_terminal_bounds(bk_problem* prob, const double* lo, const double* hi,
                                         int n);

/* Form in which newton_solve treats the barrier problem of a bounded problem (Nocedal and
 * Wright, Numerical Optimization, Sections 19.2 and 19.6). */
typedef enum {
  BK_BARRIER_PRIMAL = 0,       /* Newton on the barrier problem's own KKT conditions           */
  BK_BARRIER_PRIMAL_DUAL = 1   /* bound multipliers z_l, z_h as unknowns with the complementarity
                                  conditions (u - lo) z_l = (hi - u) z_h = mu s w, eliminated in
                                  every step (the KKT system keeps its form with
                                  z_l / (u - lo) + z_h / (hi - u) on the control diagonal); inner
                                  GMRES in the merit's norm                                   */
} bk_barrier_form;

/* Barrier schedule of a bounded problem: newton_solve runs Newton stages with
 * mu = mu0, mu0 / 10, ... down to mu_final (each to a merit <= max(tol, 10 mu), the last to
 * tol), in the given form. Defaults 0.1, 1e-6, BK_BARRIER_PRIMAL. mu scales with the cost: the
 * barrier's gradient mu s w / (distance to the bound) should start comparable to the cost's
 * gradient (the orbit transfer, with thrusts near 1e-2, takes mu0 = 1e-4). The barrier solution
 * lies O(mu_final) from the bounded optimum, and the barrier Hessian of an active bound grows
 * like 1 / mu_final, which limits how far the last stage converges. On the orbit transfer
 * with bounded thrust (mu 1e-4 .. 1e-9) the primal form took 34-40 Newton steps and the
 * primal-dual form 33 at every N from 2^10 to 2^20, the primal form the faster at 2^20 (fewer
 * GMRES iterations); on the double integrator with |u| <= 5 (mu 0.1 .. 1e-6) the primal-dual
 * form takes 18 Newton steps against 46. mu0 = mu_final: one stage. Host only; BK_ERR_ARG unless
 * 0 < mu_final <= mu0 <= 1e6 and form is one of bk_barrier_form. */
bk_status bk_problem_set_barrier(bk_problem* prob, double mu0, double mu_final, int form);

/* Device bytes the problem holds (its plans, linearisation data and scratch); workspaces are
 * extra (bk_krylov_workspace_bytes, bk_newton_workspace_bytes). For memory-based admission. */
size_t bk_problem_device_bytes(const bk_problem* prob);

/* Precision of the preconditioner of FP64 problems created after the call (the operator, the
 * Krylov vectors and the Newton residual stay FP64):
 *   mode 1: the preconditioner's node factors, scan levels, terminal Schur columns and sweeps in
 *           FP32 (GB300 runs FP32 at 64x its FP64 rate). precond_apply then rounds its input to
 *           FP32 and widens its output. Flexible GMRES builds the iterate from the preconditioned
 *           vectors it actually computed, so the solution keeps FP64 accuracy; only the Krylov
 *           iteration counts can change.
 *   mode 0 (and -1, the default): FP64 preconditioner (environment BK_F64_PC32=1: FP32). On
 *           the orbit solve at N = 2^20 the FP32 preconditioner needed 19 instead of 11 GMRES
 *           iterations down to the tight final inner tolerances and was 13% slower overall.
 * Host only; BK_ERR_ARG for any other mode. The paper's preconditioner is this one in FP64. */
bk_status bk_set_f64_precond(int mode);

/* *dtype = BK_F64 or BK_F32: the precision of the problem's preconditioner. */
bk_status bk_problem_precond_dtype(const bk_problem* prob, int* dtype);

/* Sizes of a problem (any pointer may be NULL):
 *   n_x, n_u, n_e  state, control and terminal-condition counts
 *   pitch          component block pitch in elements
 *   kkt_len        elements of a KKT vector: (2 n_x + n_u) * pitch + 32, laid out as
 *                  [X_0..X_{n_x-1} | U_0..U_{n_u-1} | lambda_0..lambda_{n_x-1} | nu (n_e, padded
 *                  to 32)]; each block pitch elements
 *   state_len      elements of a state vector: n_x * pitch                                   */
bk_status bk_problem_info(const bk_problem* prob, int* n_x, int* n_u, int* n_e, int64_t* pitch,
                          int64_t* kkt_len, int64_t* state_len);

/* Linearise the problem at z_lin (a KKT vector in FP64, device): stores per-node Jacobians,
 * mu = B^T lambda for the Lagrangian Hessian, and the preconditioner's per-node factors and
 * terminal Schur complement. kkt_apply / precond_apply / krylov_solve use the last
 * linearisation. Section "Construction of a Low-Memory Fast Million-Point Linear Solver". */
bk_status bk_linearize(bk_problem* prob, const double* z_lin, void* stream);

/* out = Op * in at the current linearisation, in the problem's working dtype.
 *   BK_OP_STATE: out = chi - s (B (x) I)(J_x chi)            (FastAX)
 *   BK_OP_KKT:   out = [H dz + G^T dy ; G dz] with G the Jacobian of (c, e) and H the
 *                Hessian of the Lagrangian (Newton-Lagrange step).
 * in and out must not alias. */
bk_status kkt_apply(bk_problem* prob, int op, const void* in, void* out, void* stream);

/* out = P^{-1} in (transpose = 0) or P^{-T} in (transpose = 1) at the current linearisation.
 *   BK_OP_STATE: P = I - s (B-tilde (x) I) J_x, B-tilde the lower-triangular Birkhoff-like
 *                matrix; computed by the forward sweep that FastPinvY intends (the printed
 *                recurrence does not invert P; the sweep used follows from the rows of P) and
 *                its backward transpose.
 *   BK_OP_KKT:   out = K-tilde^{-1} in, K-tilde the KKT matrix with B -> B-tilde in the
 *                constraint Jacobian and the Hessian reduced to its control-cost part
 *                (transpose is ignored: K-tilde is symmetric).
 * in and out must not alias. Section "Development of a Special Birkhoff-Centric
 * Preconditioner". */
bk_status precond_apply(bk_problem* prob, int op, const void* in, void* out, int transpose,
                        void* stream);

typedef struct {
  double rtol;        /* stop when ||b - A x||_2 <= rtol * ||b||_2 (default 1e-10)           */
  int restart;        /* GMRES restart length m (default 30, at most 100)                   */
  int max_iter;       /* total iteration cap (default 300)                                  */
  int use_precond;    /* 1 = right preconditioning by P^{-1} / K-tilde^{-1} (default 1)      */
} bk_krylov_opts;

typedef struct {
  int iterations;     /* Krylov iterations performed                                       */
  int restarts;       /* restart cycles                                                     */
  double rel_resid;   /* final ||b - A x|| / ||b|| (recomputed explicitly at exit)          */
  int converged;      /* 1 if rel_resid <= rtol                                             */
} bk_krylov_info;

/* Workspace bytes krylov_solve needs for operator `op` with restart m. */
size_t bk_krylov_workspace_bytes(const bk_problem* prob, int op, int restart);

/* Solve Op x = rhs by right-preconditioned GMRES(m) (Algorithm 2 / FastLinSol: GMRES on
 * A P^{-1} Upsilon = beta, then x = P^{-1} Upsilon), x0 = 0, in the working dtype.
 *   rhs, sol   device vectors of the operator's length (working dtype)
 *   opts       NULL = defaults
 *   info       host struct, valid on return (the call synchronises `stream`)
 *   workspace  device buffer of bk_krylov_workspace_bytes(prob, op, m) bytes, 256-aligned
 * Returns BK_ERR_NOT_CONVERGED (with sol holding the last iterate) if max_iter is reached. */
bk_status krylov_solve(bk_problem* prob, int op, const void* rhs, void* sol,
                       const bk_krylov_opts* opts, bk_krylov_info* info, void* workspace,
                       void* stream);

/* How GMRES runs its Arnoldi steps (krylov_solve and the inner solves of newton_solve). The
 * Hessenberg matrix, the Givens rotations and the stopping test always live on the device. With
 * graphs, a restart cycle is one CUDA graph launch: a conditional WHILE node whose body is one
 * Arnoldi step, repeated until the device says stop, then one bounded host wait; without them
 * the host launches each step and reads the stop word after it. Both forms give bitwise the same
 * iterates.
 *   mode 0 (or -1, the default): never;  mode 1: for every problem of fixed final time.

 * A problem captures a graph on its first solve for a given workspace and vector layout and keeps
 * up to four; the captured kernels read the time scale from the problem's device copy, so
 * bk_problem_set_params (which must not overlap a solve of the problem) keeps them valid.
 * Process-wide; host only. BK_ERR_ARG for any other mode. */
bk_status bk_set_krylov_graphs(int mode);

/* Bound on the host's wait for a graph cycle (seconds; <= 0 restores the default, 60 s). When a
 * cycle has not finished within it, the solve returns BK_ERR_TIMEOUT while the cycle may still be
 * running on the stream: synchronise the stream before reusing its vectors or the workspace.
 * Process-wide; host only. BK_ERR_ARG above 1e6 s or for NaN. */
bk_status bk_set_krylov_wait_limit(double seconds);

typedef struct {
  double tol;         /* stop when the weighted KKT residual norm <= tol (default 1e-10)     */
  int max_iter;       /* Newton iteration cap (default 30)                                  */
  double krylov_rtol; /* inner relative tolerance; 0 (default) = forcing term
                         0.1 (||F_k|| / ||F_0||)^2 clamped to [1e-12 (FP64) or 1e-4 (FP32),
                         1e-2], i.e. loose early Newton steps and tight final ones           */
  int restart;        /* GMRES restart (default 30)                                         */
  int max_krylov;     /* inner iteration cap per solve (default 300 in FP64, 10 in FP32)    */
  double ir_rtol;     /* FP32 mode: linear refinement sweeps stop when the FP64 residual of
                         the Newton system is <= ir_rtol * ||F|| (default 1e-10)             */
  int max_refine;     /* FP32 mode: FP32 solves per Newton step (default 1: inexact Newton,
                         the FP64 Newton residual refines the step; > 1 adds linear
                         refinement sweeps with an FP64 KKT residual)                        */
  int precond_reuse;  /* preconditioner reuse after a full step that cut ||F||_W >= 10x:
                         0 (default) rebuild at every step; 1 keep the terminal Schur data
                         of the last rebuild; 2 keep all preconditioner data (node factors,
                         sweep levels, Schur data). The KKT operator always uses the new
                         linearisation point; flexible GMRES accepts any preconditioner.   */
  int weighted_inner; /* 1: GMRES minimises the Newton system's residual in the merit's norm
                         ||.||_W (the system scaled by D = diag(w^-1/2 on gradient rows, w^1/2
                         on constraint rows, 1 on the tail), preconditioner applied to D^-1 v),
                         so that every inexact step with relative residual < 1 descends
                         ||F||_W; 0 (default): the 2-norm, except for problems with endpoint
                         bounds or in the primal-dual barrier form, which always take the
                         merit's norm. BK_ORBIT_MT then also takes the forcing term instead
                         of its default 1e-12                                                */
} bk_newton_opts;

typedef struct {
  int iterations;          /* Newton steps taken                                            */
  int krylov_iterations;   /* total inner Krylov iterations                                 */
  int kkt_solves;          /* inner Krylov solves (one per refinement sweep in FP32 mode)   */
  int backtracks;          /* line-search step reductions                                   */
  double residual;         /* final weighted KKT residual norm                              */
  double residual0;        /* initial weighted KKT residual norm                            */
  int converged;
  int precond_builds;      /* full preconditioner rebuilds (node factors and Schur data)     */
} bk_newton_info;

/* sizeof of the option and info structs as this library was compiled (which: 0 bk_krylov_opts,
 * 1 bk_krylov_info, 2 bk_newton_opts, 3 bk_newton_info; 0 for any other value), so that a
 * binding can check its own layout of them. Host only. */
size_t bk_abi_struct_size(int which);

/* Workspace bytes newton_solve needs. */
size_t bk_newton_workspace_bytes(const bk_problem* prob, int restart);

/* Newton-Lagrange solve of the discretised problem (Eq. Prob-PNa with V = f(X, U) eliminated):
 * F(z, y) = [grad J + G^T y ; c ; e] = 0 with c = X - x0 - s (B (x) I) f(X, U), e the terminal
 * conditions and J = s sum_i w_i F(x_i, u_i). Each step solves the KKT system by
 * preconditioned GMRES (BK_F32: FP32 GMRES, refined by the FP64 Newton residual), then a
 * backtracking line search (alpha = 1, then the minimiser of a quadratic model clamped to [alpha/10, alpha/2]; Armijo 1e-4) on the weighted norm
 *   ||F||_W^2 = sum_i w_i |c_i|^2 + sum_i |g_i|^2 / w_i + |e|^2  (g: gradient rows).
 *   z_inout    device FP64 KKT vector: initial guess in, solution out (X, U, lambda, nu)
 *   info       host struct, valid on return (synchronous)
 * BK_ORBIT_MT (free final time): J = t_f - t_0 = 2 s, s is read from and written to z_inout's
 * tail slot (it must start > 0; trials with s <= 0 are rejected), the residual carries the time
 * gradient, and the inner tolerance defaults to 1e-12 instead of the forcing term. Start it from
 * bk_min_time_seed.
 * Control and endpoint bounds (bk_problem_set_control_bounds, bk_problem_set_terminal_bounds):
 * the bounded values in z_inout are first moved 1e-3 of the bound gap inside the bounds, then
 * each barrier stage runs the steps above, with every
 * step length starting at the fraction-to-boundary bound min(1, 0.995 max{alpha : lo < u +
 * alpha du < hi}) so that the iterates stay strictly inside, and halved on backtracking (the
 * quadratic model is dominated by the barrier's curvature); info counts the steps of all
 * stages, residual0 is the first stage's and residual the last stage's; max_iter (default 100
 * with bounds) caps the total.
 * Returns BK_ERR_NOT_CONVERGED / BK_ERR_INFEASIBLE with z_inout holding the last iterate. */
bk_status newton_solve(bk_problem* prob, double* z_inout, const bk_newton_opts* opts,
                       bk_newton_info* info, void* workspace, void* stream);

/* KKT residual F at z (FP64 device KKT vector) into F_out (same layout); if wnorm is not NULL
 * the weighted norm ||F||_W is returned in it (host; synchronous in that case).
 * BK_ORBIT_MT: F_out's tail slot after e holds the time gradient g_s = 2 - lambda . (B^a (x) I) f,
 * and ||F||_W adds |g_s|^2; the problem's time scale is read from z (synchronous). bk_linearize
 * reads it from z_lin the same way. */
bk_status bk_kkt_residual(bk_problem* prob, const double* z, double* F_out, double* wnorm,
                          void* stream);

/* Initial point of a minimum-time solve (BK_ORBIT_MT) from a solved minimum-energy transfer
 * (BK_ORBIT, same N, a, r_f and t0; any tf):
 *   z_me   device FP64 KKT vector of `me` (its solution)
 *   z_mt   device FP64 KKT vector of `mt`, written: X, lambda and nu of z_me, the steering angle
 *          u = atan2(u_r, u_theta) of the thrust vector, s = me's time scale; then lambda and nu
 *          scaled by 2 / (lambda . (B^a (x) I) f), which zeroes the time gradient.
 * Synchronous. BK_ERR_ARG if the problems do not match or lambda . (B^a f) <= 0. The paper does
 * not say how its solve is started; this is the library's reading. */
bk_status bk_min_time_seed(bk_problem* mt, const bk_problem* me, const double* z_me, double* z_mt,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BIRKHOFF_GB300_H */
