// Newton-Lagrange driver of the discretised problem (Eq. Prob-PNa).
//
// The paper reports SQP iteration counts (Table tab:m) but does not describe its outer loop.
// This driver takes Newton's method on the KKT conditions F(z, y) = [grad J + G^T y ; c ; e] = 0
// with the exact Lagrangian Hessian, each step solved by the Birkhoff-preconditioned GMRES, and
// a backtracking line search (alpha = 1, then quadratic-model steps; Armijo constant 1e-4) on the quadrature-
// weighted norm ||F||_W^2 = sum w c^2 + sum g^2 / w + |e|^2, which does not grow with N.
// The residual and the line search are FP64. BK_F32 problems run the GMRES iterations and their
// operator applies in FP32; the FP64 Newton residual then refines their step (inexact Newton),
// and max_refine > 1 adds linear iterative-refinement sweeps with an FP64 KKT residual.
//
// Products per step. The residual's multiplier term mu = s B^aT lambda is linear in lambda, so
// along a step mu(z + alpha d) = mu + alpha mu_d with mu_d = s B^aT d_lambda: only the initial
// residual applies B^T to lambda. FP64 solves get mu_d from the Krylov iteration itself (each
// KKT apply already forms B^T of its lambda block; GMRES combines them with the solution's
// coefficients); FP32 solves form it with one FP64 product per step. Each line-search trial then
// costs one forward product. Backtracking takes the minimiser of the quadratic model of
// ||F||_W^2 along d (slope -2 ||F||_W^2 at alpha = 0, the Newton value), safeguarded to
// [alpha / 10, alpha / 2], instead of halving.
//
// Control bounds lo <= u <= hi (bk_problem_set_control_bounds): a logarithmic barrier on the
// quadrature, -mu s sum_i w_i sum_q [log(u_qi - lo_q) + log(hi_q - u_qi)], joins J (Nocedal and
// Wright, Numerical Optimization, 2nd ed., Sections 19.2 and 19.6), in one of two forms:
//  - primal (default): Newton on the barrier problem's KKT conditions; the barrier's gradient joins
//    the control rows and its Hessian mu s w (1/(u - lo)^2 + 1/(hi - u)^2) the control diagonal;
//  - primal-dual: the bound multipliers z_l, z_h are unknowns with the complementarity conditions
//    (u - lo) z_l = (hi - u) z_h = mu s w. Each Newton step eliminates them node by node: the KKT
//    system keeps its form with Sigma = z_l / (u - lo) + z_h / (hi - u) on the control diagonal
//    and a corrected right-hand side, and dz follows from du.
// Either way the KKT system keeps a diagonal control block, so the same preconditioner applies.
// The solve runs stages mu = mu_0, mu_0 / 10, ... down to mu_final, each to a merit (||F||_W, with
// the complementarity residuals in the primal-dual form) <= max(tol, 10 mu) and the last to tol,
// from controls first moved 1e-3 of the bound gap inside (and multipliers on the first stage's
// central path); each step length starts at the fraction-to-boundary bound (0.995 of the largest
// step keeping u inside its bounds and z positive, at most 1) and is halved on backtracking; the
// forcing term restarts with each stage.
//
// Free final time (BK_ORBIT_MT): s = (t_f - t_0)/2 sits in z's tail slot. The problem's s follows
// z (read back once per step, with the step's ds), trials with s <= 0 are rejected, and mu is
// recomputed for every trial (s B^aT lambda is bilinear in s and lambda, so the update above
// does not apply).
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <utility>

#include "bk_krylov.cuh"

namespace bk {

template <typename Tin, typename Tout>
__global__ void k_cast(const Tin* __restrict__ a, Tout* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (Tout)a[i];
}

// y = a x + b y (FP64)
__global__ void k_axpby64(const double* __restrict__ x, double a, double* __restrict__ y, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = a * x[i] + (b == 0.0 ? 0.0 : b * y[i]);
}

// y += (double) x (x float)
__global__ void k_acc32(const float* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += (double)x[i];
}

// z_t = z + alpha d
__global__ void k_step(const double* __restrict__ z, const double* __restrict__ d, double alpha,
                       double* __restrict__ zt, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    zt[i] = z[i] + alpha * d[i];
}

// sum of squares partials (FP64)
__global__ void k_sumsq(const double* __restrict__ x, int64_t n, double* __restrict__ partial) {
  __shared__ double red[32];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += x[i] * x[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

constexpr double kTau = 0.995;   // fraction-to-boundary

// Controls (and endpoint-bounded x(t_f)) moved at least margin * (hi - lo) inside two-sided
// bounds (margin for one-sided ones); an endpoint row's multiplier nu_r put on the central path
// of ts.mu, nu_r = psi_r'(x) (-mu / (x - elo) or mu / (ehi - x)).
__global__ void k_interior(double* __restrict__ z, int64_t P, int64_t L, int nx, BarSpec b, TermSpec ts,
                           int64_t nu_off, double margin) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    if (k == L - 1) {
#pragma unroll
      for (int r = 0; r < NEM; ++r) {
        if (r >= ts.n_e || !ts.eb[r]) continue;
        const bool lo = isfinite(ts.elo[r]);
        double x = z[ts.idx[r] * P + k];
        x = lo ? fmax(x, ts.elo[r] + margin) : fmin(x, ts.ehi[r] - margin);
        z[ts.idx[r] * P + k] = x;
        z[nu_off + r] = lo ? -ts.mu / (x - ts.elo[r]) : ts.mu / (ts.ehi[r] - x);
      }
    }
#pragma unroll
    for (int q = 0; q < NUM; ++q) {
      const bool lo = b.has_lo[q], hi = b.has_hi[q];
      if (!lo && !hi) continue;
      const double gap = lo && hi ? b.hi[q] - b.lo[q] : 1.0;
      double u = z[(nx + q) * P + k];
      if (lo) u = fmax(u, b.lo[q] + margin * gap);
      if (hi) u = fmin(u, b.hi[q] - margin * gap);
      z[(nx + q) * P + k] = u;
    }
  }
}

// Multipliers on the central path of the current mu: z_l = mu s w / (u - lo), z_h = mu s w / (hi - u)
// (zero for an absent bound and in the padding).
__global__ void k_pd_init(const double* __restrict__ z, const double* __restrict__ w, double s, int64_t P, int64_t L,
                          int nx, int nu, BarSpec b, double* __restrict__ zb) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < NUM; ++q) {
      if (q >= nu) break;
      const double u = k < L ? z[(nx + q) * P + k] : 0.0;
      const double c = k < L ? b.mu * s * w[k] : 0.0;
      zb[q * P + k] = k < L && b.has_lo[q] ? c / (u - b.lo[q]) : 0.0;
      zb[(nu + q) * P + k] = k < L && b.has_hi[q] ? c / (b.hi[q] - u) : 0.0;
    }
  }
}

// Right-hand side of the eliminated primal-dual step: control rows += -C_l / (u - lo) + C_h / (hi - u),
// C_l = (u - lo) z_l - mu s w, C_h = (hi - u) z_h - mu s w.
__global__ void k_pd_rhs(const double* __restrict__ z, const double* __restrict__ zb, const double* __restrict__ w,
                         double s, int64_t P, int64_t L, int nx, int nu, BarSpec b, double* __restrict__ rhs) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    const double c = b.mu * s * w[k];
#pragma unroll
    for (int q = 0; q < NUM; ++q) {
      if (q >= nu) break;
      const double u = z[(nx + q) * P + k];
      double r = 0.0;
      if (b.has_lo[q]) {
        const double dl = u - b.lo[q];
        r -= (dl * zb[q * P + k] - c) / dl;
      }
      if (b.has_hi[q]) {
        const double dh = b.hi[q] - u;
        r += (dh * zb[(nu + q) * P + k] - c) / dh;
      }
      rhs[(nx + q) * P + k] += r;
    }
  }
}

// Multiplier steps from the control step du: dz_l = (-C_l - z_l du) / (u - lo),
// dz_h = (-C_h + z_h du) / (hi - u) (zero for an absent bound and in the padding).
__global__ void k_pd_dz(const double* __restrict__ z, const double* __restrict__ d, const double* __restrict__ zb,
                        const double* __restrict__ w, double s, int64_t P, int64_t L, int nx, int nu, BarSpec b,
                        double* __restrict__ dzb) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int q = 0; q < NUM; ++q) {
      if (q >= nu) break;
      double dl_ = 0.0, dh_ = 0.0;
      if (k < L) {
        const double c = b.mu * s * w[k];
        const double u = z[(nx + q) * P + k], du = d[(nx + q) * P + k];
        if (b.has_lo[q]) {
          const double dl = u - b.lo[q], zl = zb[q * P + k];
          dl_ = (-(dl * zl - c) - zl * du) / dl;
        }
        if (b.has_hi[q]) {
          const double dh = b.hi[q] - u, zh = zb[(nu + q) * P + k];
          dh_ = (-(dh * zh - c) + zh * du) / dh;
        }
      }
      dzb[q * P + k] = dl_;
      dzb[(nu + q) * P + k] = dh_;
    }
  }
}

// Per block: the largest alpha (at most 1 / kTau) keeping lo < u + alpha du < hi and the
// multipliers z + alpha dz > 0 at its nodes.
__global__ void k_max_step(const double* __restrict__ z, const double* __restrict__ d, const double* __restrict__ zb,
                           const double* __restrict__ dzb, int64_t P, int64_t L, int nx, int nu, BarSpec b,
                           TermSpec ts, int64_t nu_off, double* __restrict__ partial) {
  __shared__ double red[32];
  double a = 1.0 / kTau;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    if (k == L - 1) {   // endpoint-bounded x(t_f) and the sign of its multiplier
#pragma unroll
      for (int r = 0; r < NEM; ++r) {
        if (r >= ts.n_e || !ts.eb[r]) continue;
        const double x = z[ts.idx[r] * P + k], dx = d[ts.idx[r] * P + k];
        const double nu = z[nu_off + r], dnu = d[nu_off + r];
        if (isfinite(ts.elo[r])) {   // lower bound: x > elo, nu < 0
          if (dx < 0.0) a = fmin(a, (ts.elo[r] - x) / dx);
          if (dnu > 0.0) a = fmin(a, -nu / dnu);
        } else {                     // upper bound: x < ehi, nu > 0
          if (dx > 0.0) a = fmin(a, (ts.ehi[r] - x) / dx);
          if (dnu < 0.0) a = fmin(a, -nu / dnu);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < NUM; ++q) {
      if (q >= nu) break;
      if (!b.has_lo[q] && !b.has_hi[q]) continue;
      const double u = z[(nx + q) * P + k], du = d[(nx + q) * P + k];
      if (b.has_lo[q] && du < 0.0) a = fmin(a, (b.lo[q] - u) / du);
      if (b.has_hi[q] && du > 0.0) a = fmin(a, (b.hi[q] - u) / du);
      if (!zb) continue;   // primal form: no multipliers
      const double dzl = dzb[q * P + k], dzh = dzb[(nu + q) * P + k];
      if (b.has_lo[q] && dzl < 0.0) a = fmin(a, -zb[q * P + k] / dzl);
      if (b.has_hi[q] && dzh < 0.0) a = fmin(a, -zb[(nu + q) * P + k] / dzh);
    }
  }
  for (int o = 16; o > 0; o >>= 1) a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 1.0 / kTau;
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
  }
}

__global__ void k_min_block(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 1.0 / kTau;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fmin(a, partial[i]);
  for (int o = 16; o > 0; o >>= 1) a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 1.0 / kTau;
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if (threadIdx.x == 0) out[0] = t;
  }
}

static inline int g1(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

__global__ void k_sum_block(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += partial[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) out[0] = t;
  }
}

// ||x||_2 (FP64, fixed reduction order), synchronous.
static bk_status norm2(Problem* pr, const double* x, int64_t n, double* out, cudaStream_t st) {
  const int nb = 592;
  k_sumsq<<<nb, 256, 0, st>>>(x, n, pr->red);
  BK_CHECK_LAUNCH();
  k_sum_block<<<1, 256, 0, st>>>(pr->red, nb, pr->red + 1024);
  BK_CHECK_LAUNCH();
  BK_TRY_CUDA(cudaMemcpyAsync(pr->red_host, pr->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  *out = sqrt(pr->red_host[0]);
  return BK_OK;
}

// Fraction-to-boundary step bound min(1, kTau * max alpha) along (d, dz), synchronous.
static bk_status max_step(Problem* pr, const double* z, const double* d, const double* zb, const double* dzb,
                          double* out, cudaStream_t st) {
  const int nb = (int)((pr->L + 255) / 256 < 592 ? (pr->L + 255) / 256 : 592);
  k_max_step<<<nb, 256, 0, st>>>(z, d, zb, dzb, pr->P, pr->L, pr->n_x, pr->n_u, bar_spec(pr), term_spec(pr),
                                 (int64_t)(2 * pr->n_x + pr->n_u) * pr->P, pr->red);
  BK_CHECK_LAUNCH();
  k_min_block<<<1, 256, 0, st>>>(pr->red, nb, pr->red + 1024);
  BK_CHECK_LAUNCH();
  BK_TRY_CUDA(cudaMemcpyAsync(pr->red_host, pr->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  *out = fmin(1.0, kTau * pr->red_host[0]);
  return BK_OK;
}

// Leaves the problem's barrier parameter at mu_final and its kernels in the primal form when a
// solve returns (its residual and operator then describe the last stage's barrier problem).
struct BarrierReset {
  Problem* pr;
  ~BarrierReset() {
    if (pr->has_bounds) pr->bar_mu = pr->bar_mu_final;
    pr->bar_z = nullptr;
  }
};

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

size_t newton_workspace(const Problem* pr, int restart) {
  const int64_t n = pr->kkt_len();
  const int64_t nxP = (int64_t)pr->n_x * pr->P;
  size_t b = 0;
  b += 4 * align256(sizeof(double) * n);   // d, zt, rhs, r
  b += 3 * align256(sizeof(double) * nxP); // mu, mu_t, mu_d
  if (pr->dtype == BK_F64) b += align256(sizeof(double) * nxP * restart);  // Krylov B^T records
  if (pr->dtype == BK_F32) b += 2 * align256(sizeof(float) * n);
  b += align256(gmres_workspace_bytes(n, restart, pr->dtype));
  return b + 1024;
}

// Floor of the FP32 inner tolerance (BK_F32_FORCING_FLOOR overrides it, for tuning).
static double f32_forcing_floor() {
  static const double f = [] {
    const char* e = getenv("BK_F32_FORCING_FLOOR");
    const double v = e ? atof(e) : 0.0;
    return v >= 1e-8 && v <= 1e-2 ? v : 1e-4;
  }();
  return f;
}

static bk_status newton_impl(Problem* pr, double* z, const bk_newton_opts& o, bk_newton_info* info, void* ws,
                             cudaStream_t st) {
  const int64_t n = pr->kkt_len();
  char* p = (char*)ws;
  auto carve = [&](size_t bytes) { char* r = p; p += align256(bytes); return (void*)r; };
  double* d = (double*)carve(sizeof(double) * n);
  double* zt = (double*)carve(sizeof(double) * n);
  double* rhs = (double*)carve(sizeof(double) * n);
  double* r = (double*)carve(sizeof(double) * n);
  float* r32 = nullptr;
  float* d32 = nullptr;
  if (pr->dtype == BK_F32) {
    r32 = (float*)carve(sizeof(float) * n);
    d32 = (float*)carve(sizeof(float) * n);
  }
  void* gws = carve(gmres_workspace_bytes(n, o.restart, pr->dtype));
  const int64_t nxP = (int64_t)pr->n_x * pr->P;
  double* Mu = (double*)carve(sizeof(double) * nxP);
  double* Mut = (double*)carve(sizeof(double) * nxP);
  double* Mud = (double*)carve(sizeof(double) * nxP);
  double* Trec = pr->dtype == BK_F64 ? (double*)carve(sizeof(double) * nxP * o.restart) : nullptr;
  const double* dlam = d + (int64_t)(pr->n_x + pr->n_u) * pr->P;
  double* F = pr->F;
  const int g = g1(n);
  bk_krylov_opts ko;
  ko.restart = o.restart;
  ko.max_iter = o.max_krylov;
  ko.use_precond = 1;
  double phi = 0.0;
  const bool ft = pr->free_time;
  double* hs = pr->red_host + 200;  // pinned: s or ds read back for a free final time
  if (ft) {
    BK_TRY_CUDA(cudaMemcpyAsync(hs, z + pr->s_idx(), sizeof(double), cudaMemcpyDeviceToHost, st));
    BK_TRY_CUDA(cudaStreamSynchronize(st));
    if (!(hs[0] > 0.0) || !isfinite(hs[0])) {
      set_error("free final time: the time scale in z must be positive (got %g)", hs[0]);
      return BK_ERR_ARG;
    }
    pr->s = hs[0];
  }
  const bool bar = pr->has_bounds;
  const bool pd = pr->has_ubounds && pr->bar_form == BK_BARRIER_PRIMAL_DUAL;
  BarrierReset reset{pr};
  double mu = bar ? pr->bar_mu0 : 0.0;
  // bound multipliers (primal-dual form): current, trial and step, 2 n_u P each
  const int64_t nzb = 2 * (int64_t)pr->n_u * pr->P;
  double* zb = pd ? pr->bar_buf : nullptr;
  double* zbt = pd ? pr->bar_buf + nzb : nullptr;
  double* dzb = pd ? pr->bar_buf + 2 * nzb : nullptr;
  if (bar) {
    pr->bar_mu = mu;
    pr->bar_z = nullptr;
    k_interior<<<g1(pr->L), 256, 0, st>>>(z, pr->P, pr->L, pr->n_x, bar_spec(pr), term_spec(pr),
                                          (int64_t)(2 * pr->n_x + pr->n_u) * pr->P, 1e-3);
    BK_CHECK_LAUNCH();
  }
  if (pd) {
    k_pd_init<<<g1(pr->P), 256, 0, st>>>(z, pr->d64.plan->w64, pr->s, pr->P, pr->L, pr->n_x, pr->n_u, bar_spec(pr), zb);
    BK_CHECK_LAUNCH();
    pr->bar_z = zb;
  }
  BK_TRY(problem_residual(pr, z, F, &phi, st, Mu, false));
  info->residual0 = phi;
  info->residual = phi;
  int it = 0;
  bool fast = false;  // the last step was a full step that cut ||F||_W at least 10x
  bool last = !bar || mu <= pr->bar_mu_final * (1.0 + 1e-12);
  double tol = last ? o.tol : fmax(o.tol, 10.0 * mu);
  double phi_stage = phi;   // ||F||_W at the start of the (barrier) stage, for the forcing term
  for (;;) {
    if (phi <= tol) {
      if (last) break;
      // next barrier stage: its residual at the current point
      mu = fmax(0.1 * mu, pr->bar_mu_final);
      pr->bar_mu = mu;
      last = mu <= pr->bar_mu_final * (1.0 + 1e-12);
      tol = last ? o.tol : fmax(o.tol, 10.0 * mu);
      BK_TRY(problem_residual(pr, z, F, &phi, st, Mu, false));
      phi_stage = phi;
      fast = false;
      continue;
    }
    if (it >= o.max_iter) break;
    // Inner tolerance: fixed if the caller set one, else a forcing term that tightens with the
    // outer residual, rtol_k = 0.1 (phi_k / phi_0)^2 clamped to [floor, 1e-2] (Eisenstat and
    // Walker's choice 2 with gamma = 0.1, alpha = 2; phi_0 the merit at the start of the solve,
    // or of the barrier stage under bounds): loose early steps, tight final ones, quadratic outer
    // convergence kept. Floor 1e-12 in FP64, 1e-4 in FP32.
    if (o.krylov_rtol > 0) {
      ko.rtol = o.krylov_rtol;
    } else if (ft && !o.weighted_inner) {
      // Free final time: tight inner solves. GMRES measures its residual in the 2-norm while the
      // merit divides the gradient rows by w (w_0 ~ 1/N^2); on the minimum-time orbit the loose
      // early steps of the forcing term stopped being descent directions of ||F||_W from
      // N = 2^12 (measured), while steps solved to 1e-12 gave the same Newton count for every N.
      ko.rtol = 1e-12;
    } else {
      const double r = phi / phi_stage;
      const double lo = pr->dtype == BK_F64 ? 1e-12 : f32_forcing_floor();
      ko.rtol = fmin(1e-2, fmax(lo, 0.1 * r * r));
    }
    const int keep = (fast && o.precond_reuse > 0) ? (o.precond_reuse >= 2 ? LIN_KEEP_PRECOND : LIN_KEEP_SCHUR)
                                                  : LIN_FULL;
    if (keep == LIN_FULL) ++info->precond_builds;
    BK_TRY(problem_linearize(pr, z, st, Mu, keep));
    k_axpby64<<<g, 256, 0, st>>>(F, -1.0, rhs, 0.0, n);
    BK_CHECK_LAUNCH();
    // Primal-dual form: GMRES in the merit's norm, to a residual of (forcing term) x the merit.
    // The eliminated right-hand side carries C / (distance to the bound), which near an active
    // bound is far larger than the merit's C / sqrt(w): a tolerance relative to it alone gave
    // steps that were no descent directions (line-search failures on the bounded orbit transfer
    // at N = 2^20 on the GPU, and from N = 64 in a CPU model of this loop).
    // Endpoint bounds: GMRES in the merit's norm too. The barrier rows sit at the last node, whose
    // gradient row the merit divides by w_N ~ 1/N^2; with 2-norm inner solves the bounded orbit
    // transfer (r(t_f) >= 1.55) stopped on line-search failures from N = 2^10 on GB300, in the
    // merit's norm it took 20 Newton steps at N = 2^6, 2^10 and 2^14.
    const bool weighted = o.weighted_inner != 0 || pd || pr->has_ebounds;
    if (pd) {
      k_pd_rhs<<<g1(pr->L), 256, 0, st>>>(z, zb, pr->d64.plan->w64, pr->s, pr->P, pr->L, pr->n_x, pr->n_u,
                                          bar_spec(pr), rhs);
      BK_CHECK_LAUNCH();
      if (o.krylov_rtol <= 0) {
        double bw = 0.0;
        BK_TRY(problem_wnorm(pr, rhs, &bw, st));
        if (bw > phi) ko.rtol *= phi / bw;
      }
    }
    bk_krylov_info ki;
    if (pr->dtype == BK_F64) {
      const KrylovMu aux = {Trec, nxP, Mud, nxP};
      BK_TRY(gmres(pr, pr->d64, BK_OP_KKT, rhs, d, ko, &ki, gws, st, ft ? nullptr : &aux, weighted));
      info->krylov_iterations += ki.iterations;
      info->kkt_solves += 1;
    } else {
      // FP32 GMRES inside FP64 iterative refinement
      double rn0 = 0.0;
      BK_TRY(norm2(pr, rhs, n, &rn0, st));
      BK_TRY_CUDA(cudaMemsetAsync(d, 0, sizeof(double) * n, st));
      k_axpby64<<<g, 256, 0, st>>>(rhs, 1.0, r, 0.0, n);
      BK_CHECK_LAUNCH();
      for (int sweep = 0; sweep < o.max_refine; ++sweep) {
        k_cast<double, float><<<g, 256, 0, st>>>(r, r32, n);
        BK_CHECK_LAUNCH();
        BK_TRY(gmres(pr, pr->d32, BK_OP_KKT, r32, d32, ko, &ki, gws, st, nullptr, weighted));
        info->krylov_iterations += ki.iterations;
        info->kkt_solves += 1;
        k_acc32<<<g, 256, 0, st>>>(d32, d, n);
        BK_CHECK_LAUNCH();
        if (sweep + 1 == o.max_refine) break;  // last sweep: the Newton residual checks d
        // r = rhs - K d (FP64)
        BK_TRY(op_apply(pr, pr->d64, BK_OP_KKT, d, r, st));
        k_axpby64<<<g, 256, 0, st>>>(rhs, 1.0, r, -1.0, n);
        BK_CHECK_LAUNCH();
        double rn = 0.0;
        BK_TRY(norm2(pr, r, n, &rn, st));
        if (rn <= o.ir_rtol * rn0) break;
      }
      if (!ft) BK_TRY(plan_apply_n(pr->d64.plan, dlam, Mud, pr->n_x, true, pr->s, st));
    }
    const double s0 = pr->s;
    double ds = 0.0;
    if (ft) {
      BK_TRY_CUDA(cudaMemcpyAsync(hs, d + pr->s_idx(), sizeof(double), cudaMemcpyDeviceToHost, st));
      BK_TRY_CUDA(cudaStreamSynchronize(st));
      ds = hs[0];
    }
    // backtracking line search on ||F||_W, from the fraction-to-boundary bound under control bounds
    double alpha = 1.0, phit = 0.0;
    if (pd) {
      k_pd_dz<<<g1(pr->P), 256, 0, st>>>(z, d, zb, pr->d64.plan->w64, pr->s, pr->P, pr->L, pr->n_x, pr->n_u,
                                         bar_spec(pr), dzb);
      BK_CHECK_LAUNCH();
    }
    if (bar) BK_TRY(max_step(pr, z, d, zb, dzb, &alpha, st));
    int bt = 0;
    const double phi2 = phi * phi;
    for (;;) {
      k_step<<<g, 256, 0, st>>>(z, d, alpha, zt, n);
      BK_CHECK_LAUNCH();
      if (pd) {
        k_step<<<g1(nzb), 256, 0, st>>>(zb, dzb, alpha, zbt, nzb);
        BK_CHECK_LAUNCH();
        pr->bar_z = zbt;
      }
      if (ft) {
        pr->s = s0 + alpha * ds;
        if (!(pr->s > 0.0)) {
          phit = INFINITY;  // a non-positive final time: shrink the step
        } else {
          BK_TRY(problem_residual(pr, zt, F, &phit, st, Mut, false));
        }
      } else {
        k_step<<<g1(nxP), 256, 0, st>>>(Mu, Mud, alpha, Mut, nxP);
        BK_CHECK_LAUNCH();
        BK_TRY(problem_residual(pr, zt, F, &phit, st, Mut, true));
      }
      if (phit <= (1.0 - 1e-4 * alpha) * phi || bt >= 30) break;
      double an = phi2 * alpha * alpha / (phit * phit - phi2 + 2.0 * phi2 * alpha);
      if (!(an >= 0.1 * alpha)) an = 0.1 * alpha;  // also catches a non-finite trial residual
      // under control bounds plain halving: the barrier's curvature dominates the model, whose
      // minimiser then sits near alpha / 10 (double integrator with |u| <= 5: > 100 steps with
      // the model, 46 with halving)
      if (an > 0.5 * alpha || bar) an = 0.5 * alpha;
      alpha = an;
      ++bt;
    }
    info->backtracks += bt;
    if (pd) pr->bar_z = zb;
    if (!(phit <= (1.0 - 1e-4 * alpha) * phi)) {
      pr->s = s0;
      info->iterations = it;
      info->residual = phi;
      set_error("line search failed after %d halvings at ||F||_W = %.3e", bt, phi);
      return BK_ERR_INFEASIBLE;
    }
    BK_TRY_CUDA(cudaMemcpyAsync(z, zt, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    std::swap(Mu, Mut);
    if (pd) {
      std::swap(zb, zbt);
      pr->bar_z = zb;
    }
    fast = bt == 0 && phit <= 0.1 * phi;
    phi = phit;
    ++it;
  }
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  info->iterations = it;
  info->residual = phi;
  info->converged = last && phi <= o.tol ? 1 : 0;
  // residual products on a dense plan that ran out of a bounded wait invalidate the solve
  BK_TRY(dense_status(pr->d64.plan, st));
  return BK_OK;
}

}  // namespace bk

extern "C" {

size_t bk_abi_struct_size(int which) {
  switch (which) {
    case 0: return sizeof(bk_krylov_opts);
    case 1: return sizeof(bk_krylov_info);
    case 2: return sizeof(bk_newton_opts);
    case 3: return sizeof(bk_newton_info);
    default: return 0;
  }
}

size_t bk_newton_workspace_bytes(const bk_problem* prob, int restart) {
  const bk::Problem* p = reinterpret_cast<const bk::Problem*>(prob);
  if (!p) return 0;
  if (restart <= 0) restart = 30;
  return bk::newton_workspace(p, restart);
}

bk_status newton_solve(bk_problem* prob, double* z_inout, const bk_newton_opts* opts, bk_newton_info* info,
                       void* workspace, void* stream) {
  BK_ARG(prob != nullptr && z_inout != nullptr && info != nullptr, "NULL argument");
  BK_ARG(workspace != nullptr && ((uintptr_t)workspace & 255) == 0, "workspace must be 256-byte aligned");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  BK_ARG(p->has_cost, "newton_solve needs a problem kind with a cost (BK_DBL_INT, BK_ORBIT)");
  bk_newton_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  if (o.tol <= 0) o.tol = 1e-10;
  if (o.max_iter <= 0) o.max_iter = p->has_bounds ? 100 : 30;   // control bounds: several barrier stages
  // FP64: up to 300 inner iterations. FP32: inexact Newton, one FP32 GMRES solve (at most 10
  // iterations) per step, refined by the FP64 Newton residual.
  const bool f64 = p->dtype == BK_F64;
  if (o.krylov_rtol < 0) o.krylov_rtol = 0;  // 0 = adaptive forcing term (see newton_impl)
  if (o.restart <= 0) o.restart = 30;
  if (o.max_krylov <= 0) o.max_krylov = f64 ? 300 : 10;
  if (o.ir_rtol <= 0) o.ir_rtol = 1e-10;
  if (o.max_refine <= 0) o.max_refine = f64 ? 10 : 1;
  memset(info, 0, sizeof(*info));
  BK_TRY(bk::newton_impl(p, z_inout, o, info, workspace, (cudaStream_t)stream));
  if (!info->converged) {
    bk::set_error("Newton stopped after %d iterations at ||F||_W = %.3e", info->iterations, info->residual);
    return BK_ERR_NOT_CONVERGED;
  }
  return BK_OK;
}

}  // extern "C"
