// Problem object, dynamics device functions and sweep/operator declarations (internal).
//
// Discretisation (Eq. Prob-PNa with V = f(X, U) eliminated and x^a fixed):
//   c(X, U) = X - x0 (x) 1 - s (B^a (x) I) f(X, U),  e(X) = X[term, N] - target,
//   J = s sum_i w_i F(x_i, u_i)  (control bounds lo <= u <= hi add the barrier
//   - mu s sum_i w_i sum_q [log(u_qi - lo_q) + log(hi_q - u_qi)]).
// KKT vectors (component-major, pitch P per block): [X | U | lambda | nu (padded to 32)]; a free
// final time (BK_ORBIT_MT) keeps s = (t_f - t_0)/2 in the tail slot after nu.
#pragma once

#include <math.h>
#include <string.h>

#include "bk_common.cuh"
#include "bk_plan.cuh"

namespace bk {

constexpr int NXM = 4;   // largest state dimension of the compiled problem kinds
constexpr int NUM = 2;   // largest control dimension
constexpr int NEM = 4;   // largest terminal-condition count
// Nodes per sweep segment (one lane each) for the working precision: shorter segments in FP64,
// where the sweep is bound by dependent FP64 latency and more lanes help (measured: 8 vs 16
// nodes, KKT preconditioner at 2^20 0.75 vs 0.84 ms), 16 in FP32 (one 32-byte staging chunk).
template <typename T> struct Seg { static constexpr int v = sizeof(T) == 8 ? 8 : 16; };
inline int seg_nodes(int dtype) { return dtype == BK_F64 ? Seg<double>::v : Seg<float>::v; }
// Scan levels of the preconditioner sweep: level 0 items are segments, level l + 1 items are
// blocks of 32 level-l items, up to the first level with at most 32 items (N <= 2^24: 4 levels).
constexpr int MAXLEV = 5;
// Matrix slots stored per level item (working type, 32-interleaved): the item's map A, the spans
// M_k = product of the 2^k items ending at this one (k = 1..4, within its block of 32), and the
// products of the items before (Pre) and after (Suf) it in its block.
enum { SL_A = 0, SL_M1 = 1, SL_PRE = 5, SL_SUF = 6, NSLOT = 7 };

// ---------------------------------------------------------------------------------------------
// Dynamics of the compiled problem kinds (FP64 or FP32 arithmetic).
// ---------------------------------------------------------------------------------------------
template <int KIND> struct Dyn;

// Structural nonzeros of J_x (n_x x n_x), J_u (n_x x n_u) and the Lagrangian Hessian
// H ((n_x + n_u)^2) of a kind: the node-local kernels skip the products with structural zeros
// (the indices are compile-time constants after unrolling, so the skipped terms and their loads
// vanish). Kinds without a pattern take the dense one.
struct DenseNZ {
  __host__ __device__ static constexpr bool jx_nz(int, int) { return true; }
  __host__ __device__ static constexpr bool ju_nz(int, int) { return true; }
  __host__ __device__ static constexpr bool h_nz(int, int) { return true; }
};

__device__ inline void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }
__device__ inline void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }

// Minimum-energy double integrator: x = (p, v), x' = (v, u), F = u^2 / 2.
template <> struct Dyn<BK_DBL_INT> {
  static constexpr int nx = 2, nu = 1;
  // J_x = [[0, 1], [0, 0]], J_u = [0; 1], H = 0 (f is linear)
  __host__ __device__ static constexpr bool jx_nz(int r, int c) { return r == 0 && c == 1; }
  __host__ __device__ static constexpr bool ju_nz(int r, int q) { return r == 1 && q == 0; }
  __host__ __device__ static constexpr bool h_nz(int, int) { return false; }
  // control block of the KKT preconditioner at a node: s w_k times the running cost's curvature
  static constexpr bool huu_needs_mu = false;
  template <typename T> __device__ static T pre_huu(const T* mu, T swk, T) { return swk; }
  template <typename T> __device__ static void f(const T* x, const T* u, T* fx, T) {
    fx[0] = x[1];
    fx[1] = u[0];
  }
  template <typename T> __device__ static void jac(const T* x, const T* u, T* Jx, T* Ju, T) {
    Jx[0] = 0; Jx[1] = 1; Jx[2] = 0; Jx[3] = 0;
    Ju[0] = 0; Ju[1] = 1;
  }
  // H[(nx+nu)^2] = sum_m mu_m Hess f_m (zero: f is linear)
  template <typename T> __device__ static void hess(const T* x, const T* u, const T* mu, T* H, T) {
    for (int i = 0; i < 9; ++i) H[i] = 0;
  }
};

// Planar orbit in polar coordinates with thrust-vector control (dynamics of Eq. ot):
// x = (r, theta, v_r, v_theta), u = (u_r, u_theta).
template <> struct Dyn<BK_ORBIT> {
  static constexpr int nx = 4, nu = 2;
  // the entries jac and hess set below (theta enters no right-hand side; u enters linearly)
  __host__ __device__ static constexpr bool jx_nz(int r, int c) {
    return (r == 0 && c == 2) || (r == 1 && (c == 0 || c == 3)) || (r == 2 && (c == 0 || c == 3)) ||
           (r == 3 && (c == 0 || c == 2 || c == 3));
  }
  __host__ __device__ static constexpr bool ju_nz(int r, int q) { return (r == 2 && q == 0) || (r == 3 && q == 1); }
  __host__ __device__ static constexpr bool h_nz(int a, int b) {
    return (a == 0 && (b == 0 || b == 2 || b == 3)) || (b == 0 && (a == 2 || a == 3)) || (a == 2 && b == 3) ||
           (a == 3 && (b == 2 || b == 3));
  }
  // control block of the KKT preconditioner at a node: s w_k times the running cost's curvature
  static constexpr bool huu_needs_mu = false;
  template <typename T> __device__ static T pre_huu(const T* mu, T swk, T) { return swk; }
  template <typename T> __device__ static void f(const T* x, const T* u, T* fx, T) {
    const T r = x[0], vr = x[2], vt = x[3];
    const T ir = T(1) / r;
    fx[0] = vr;
    fx[1] = vt * ir;
    fx[2] = vt * vt * ir - ir * ir + u[0];
    fx[3] = -vr * vt * ir + u[1];
  }
  template <typename T> __device__ static void jac(const T* x, const T* u, T* Jx, T* Ju, T) {
    const T r = x[0], vr = x[2], vt = x[3];
    const T ir = T(1) / r, ir2 = ir * ir;
    for (int i = 0; i < 16; ++i) Jx[i] = 0;
    Jx[0 * 4 + 2] = 1;
    Jx[1 * 4 + 0] = -vt * ir2;
    Jx[1 * 4 + 3] = ir;
    Jx[2 * 4 + 0] = -vt * vt * ir2 + T(2) * ir2 * ir;
    Jx[2 * 4 + 3] = T(2) * vt * ir;
    Jx[3 * 4 + 0] = vr * vt * ir2;
    Jx[3 * 4 + 2] = -vt * ir;
    Jx[3 * 4 + 3] = -vr * ir;
    for (int i = 0; i < 8; ++i) Ju[i] = 0;
    Ju[2 * 2 + 0] = 1;
    Ju[3 * 2 + 1] = 1;
  }
  template <typename T> __device__ static void hess(const T* x, const T* u, const T* mu, T* H, T) {
    const T r = x[0], vr = x[2], vt = x[3];
    const T ir = T(1) / r, ir2 = ir * ir, ir3 = ir2 * ir;
    const T mth = mu[1], mvr = mu[2], mvt = mu[3];
    for (int i = 0; i < 36; ++i) H[i] = 0;
    const int R = 0, VR = 2, VT = 3;
    T hrr = mth * T(2) * vt * ir3 + mvr * (T(2) * vt * vt * ir3 - T(6) * ir2 * ir2) +
            mvt * (-T(2) * vr * vt * ir3);
    T hrvt = mth * (-ir2) + mvr * (-T(2) * vt * ir2) + mvt * (vr * ir2);
    T hrvr = mvt * (vt * ir2);
    T hvtvt = mvr * (T(2) * ir);
    T hvrvt = mvt * (-ir);
    H[R * 6 + R] = hrr;
    H[R * 6 + VT] = hrvt; H[VT * 6 + R] = hrvt;
    H[R * 6 + VR] = hrvr; H[VR * 6 + R] = hrvr;
    H[VT * 6 + VT] = hvtvt;
    H[VR * 6 + VT] = hvrvt; H[VT * 6 + VR] = hvrvt;
  }
};

// Scalar bilinear x' = u x (no cost): linearised at (X, U) the state Jacobian is diag(U).
template <> struct Dyn<BK_BILINEAR> : DenseNZ {
  static constexpr int nx = 1, nu = 1;
  // control block of the KKT preconditioner at a node: s w_k times the running cost's curvature
  static constexpr bool huu_needs_mu = false;
  template <typename T> __device__ static T pre_huu(const T* mu, T swk, T) { return swk; }
  template <typename T> __device__ static void f(const T* x, const T* u, T* fx, T) { fx[0] = u[0] * x[0]; }
  template <typename T> __device__ static void jac(const T* x, const T* u, T* Jx, T* Ju, T) {
    Jx[0] = u[0];
    Ju[0] = x[0];
  }
  template <typename T> __device__ static void hess(const T* x, const T* u, const T* mu, T* H, T) {
    H[0] = 0; H[1] = mu[0]; H[2] = mu[0]; H[3] = 0;
  }
};

// Minimum-time orbit transfer of Eq. ot: the same state, fixed-magnitude thrust a (sin u, cos u)
// steered by the angle u (pa = a), cost T = t_f - t_0 with the final time free.
template <> struct Dyn<BK_ORBIT_MT> : DenseNZ {
  // the state Jacobian of BK_ORBIT (theta enters no right-hand side); J_u and H dense
  __host__ __device__ static constexpr bool jx_nz(int r, int c) { return Dyn<BK_ORBIT>::jx_nz(r, c); }
  static constexpr int nx = 4, nu = 1;
  template <typename T> __device__ static void f(const T* x, const T* u, T* fx, T a) {
    const T r = x[0], vr = x[2], vt = x[3];
    const T ir = T(1) / r;
    T su, cu;
    sincos_t(u[0], &su, &cu);
    fx[0] = vr;
    fx[1] = vt * ir;
    fx[2] = vt * vt * ir - ir * ir + a * su;
    fx[3] = -vr * vt * ir + a * cu;
  }
  template <typename T> __device__ static void jac(const T* x, const T* u, T* Jx, T* Ju, T a) {
    Dyn<BK_ORBIT>::jac<T>(x, u, Jx, Ju, a);   // the state Jacobian is the same
    T su, cu;
    sincos_t(u[0], &su, &cu);
    for (int i = 0; i < 4; ++i) Ju[i] = 0;
    Ju[2] = a * cu;
    Ju[3] = -a * su;
  }
  // state block as BK_ORBIT; the angle adds d2/du2 (mu . f) = -a (mu_vr sin u + mu_vt cos u)
  template <typename T> __device__ static void hess(const T* x, const T* u, const T* mu, T* H, T a) {
    T H6[36];
    Dyn<BK_ORBIT>::hess<T>(x, u, mu, H6, a);
    for (int i = 0; i < 5; ++i)
      for (int j = 0; j < 5; ++j) H[i * 5 + j] = (i < 4 && j < 4) ? H6[i * 6 + j] : T(0);
    T su, cu;
    sincos_t(u[0], &su, &cu);
    H[24] = -a * (mu[2] * su + mu[3] * cu);
  }
  // the angle's Lagrangian curvature a (mu_vr sin u + mu_vt cos u) is bounded by a |mu_v|; the
  // preconditioner takes that bound plus 1e-3 s w_k (positive where mu_v vanishes)
  static constexpr bool huu_needs_mu = true;
  template <typename T> __device__ static T pre_huu(const T* mu, T swk, T a) {
    return a * sqrt(mu[2] * mu[2] + mu[3] * mu[3]) + T(1e-3) * swk;
  }
};

// Columns of J_x that are zero in every compiled kind with n_x = NX (bit c: column c). A zero
// column of h J stays exactly zero in the node deviation D = (I - h J)^{-1} h J (its right-hand
// side column is zero) and in every deviation of a product of (I + 2 D) maps, so the sweeps and
// the level products skip those entries and their loads without changing any result. Orbit kinds
// (n_x = 4): theta enters no right-hand side (column 1); double integrator (n_x = 2): the
// position enters none (column 0).
template <int NX> struct ZeroCols { static constexpr int mask = NX == 4 ? 0x2 : (NX == 2 ? 0x1 : 0); };
template <int NX> __host__ __device__ constexpr bool zcol(int c) { return ((ZeroCols<NX>::mask >> c) & 1) != 0; }

template <int KIND> constexpr bool zero_cols_hold() {
  constexpr int NX = Dyn<KIND>::nx;
  for (int c = 0; c < NX; ++c)
    for (int r = 0; r < NX; ++r)
      if (zcol<NX>(c) && Dyn<KIND>::jx_nz(r, c)) return false;
  return true;
}
static_assert(zero_cols_hold<BK_DBL_INT>() && zero_cols_hold<BK_ORBIT>() && zero_cols_hold<BK_BILINEAR>() &&
                  zero_cols_hold<BK_ORBIT_MT>(),
              "a kind's state Jacobian has an entry in a column ZeroCols skips");

// ---------------------------------------------------------------------------------------------
// Problem
// ---------------------------------------------------------------------------------------------
// Terminal conditions as a kernel argument (static indices only): e_r = x_{idx_r}(t_f) - val_r,
// or, for a row with an endpoint bound (eb_r; one of elo_r, ehi_r finite), the barrier row of
// psi_r(x) = -mu log(x - elo_r) (or -mu log(ehi_r - x)) with nu_r as its multiplier, in
// complementarity form F_r = c(x) nu_r - mu m(x): c = x - elo, m = -1 (lower) or c = ehi - x,
// m = 1 (upper); its Newton row at the linearisation is ea_r dx + ec_r dnu_r.
struct TermSpec {
  int n_e;
  int idx[NEM];
  double val[NEM];
  int eb[NEM];
  double elo[NEM], ehi[NEM];
  double mu;
  double ea[NEM], ec[NEM];
};

// c(x), c'(x), m(x) of an endpoint row (m' = 0 for one-sided rows).
__host__ __device__ inline void end_cm(const TermSpec& ts, int r, double x, double* c, double* dc, double* m) {
  if (isfinite(ts.elo[r])) {
    *c = x - ts.elo[r];
    *dc = 1.0;
    *m = -1.0;
  } else {
    *c = ts.ehi[r] - x;
    *dc = -1.0;
    *m = 1.0;
  }
}

// Control bounds and barrier parameter as a kernel argument (static indices only).
struct BarSpec {
  double mu;          // 0: no barrier terms
  double lo[NUM], hi[NUM];
  int has_lo[NUM], has_hi[NUM];
  const double* z;    // primal-dual form: bound multipliers, z_l of control q at q P + k and z_h at
                      // (n_u + q) P + k (FP64); null: primal form (multipliers on the central path)
};

// Barrier gradient g_q and Hessian diagonal h_q of -mu swk sum_q [log(u_q - lo_q) + log(hi_q - u_q)]
// at one node (swk = s w_k); zero without bounds.
template <typename T, int NU>
__device__ __forceinline__ void bar_terms(const BarSpec& b, const T* u, T swk, T* g, T* h) {
  const T c = T(b.mu) * swk;
#pragma unroll
  for (int q = 0; q < NU; ++q) {
    T gq = T(0), hq = T(0);
    if (b.mu > 0.0) {
      if (b.has_lo[q]) {
        const T d = u[q] - T(b.lo[q]);
        const T id = T(1) / d;
        gq -= id;
        hq += id * id;
      }
      if (b.has_hi[q]) {
        const T d = T(b.hi[q]) - u[q];
        const T id = T(1) / d;
        gq += id;
        hq += id * id;
      }
    }
    g[q] = c * gq;
    h[q] = c * hq;
  }
}

// Per-precision operator state: a plan and the linearisation data in that precision.
struct OpData {
  int dtype = BK_F64;
  Plan* plan = nullptr;        // n_comp = n_x, max_batch = 1
  void* xu = nullptr;          // linearisation point X, U ((n_x + n_u) * P)
  void* mu = nullptr;          // mu = s (B^a)^T lambda (n_x * P)
  void* w = nullptr;           // Clenshaw-Curtis weights (L), working type
  void* Dn = nullptr;          // per-node D_k = h_k J_k K_k, K_k = (I - h_k J_k)^{-1} = I + D_k and
                               // N_k = 2 h_k J_k K_k = 2 D_k; interleaved (n_x^2 per node)
  void* lvm[MAXLEV] = {};      // per level: NSLOT matrix slots (n_x^2 per item each), working type
  void* lvo[MAXLEV] = {};      // per level >= 1: item offsets from zero (n_x per item), per sweep
  void* lve[MAXLEV] = {};      // per level: inclusive in-block scan values (n_x per item), per sweep
  // KKT preconditioner (terminal Schur data)
  void* Zc = nullptr;          // n_e state vectors   Z = P^{-T} E^T
  void* HWc = nullptr;         // n_e control vectors H~^{-1} W, W = Pu^T Z
  void* Qc = nullptr;          // n_e state vectors   Q = P^{-1} Pu H~^{-1} W
  void* Sinv = nullptr;        // n_e x n_e inverse of S = E Q (working type, device)
  // free final time: the KKT matrix's s column a, q = K-tilde^{-1} a and 1 / (a . q)
  void* brd = nullptr;         // kkt_len, working type
  void* brq = nullptr;         // kkt_len, working type
  double* bgam = nullptr;      // device scalar 1 / (a . q), then per apply the s component
  // temporaries (each n_x * P or (n_x + n_u) * P, working type)
  void* t1 = nullptr;
  void* t2 = nullptr;
  void* t3 = nullptr;
  // control bounds: the barrier's diagonal of the control block at the linearisation (n_u * P),
  // allocated when bounds are first set
  void* hbar = nullptr;
};

struct Problem {
  int kind = 0, n_x = 0, n_u = 0, n_e = 0;
  int dtype = BK_F64;          // working precision of kkt/krylov (and of the operator)
  int pdtype = BK_F64;         // precision of the preconditioner's data and sweeps (BK_F32 for an
                               // FP64 problem created with the FP32 preconditioner)
  void* pcin = nullptr;        // FP32 copies of a preconditioner input / output (kkt_len each),
  void* pcout = nullptr;       // when pdtype differs from dtype
  int64_t N = 0, L = 0, P = 0;
  double t0 = 0, tf = 0, s = 0;
  double params[4] = {0, 0, 0, 0};
  double x0[NXM] = {0, 0, 0, 0};
  int term_idx[NEM] = {0, 0, 0, 0};
  double term_val[NEM] = {0, 0, 0, 0};
  bool has_cost = true;
  bool free_time = false;      // BK_ORBIT_MT: s = (t_f - t_0)/2 is an unknown, kept at s_idx()
  int nseg = 0;                // sweep segments (level-0 items)
  int nlev = 0;                // scan levels; level nlev - 1 has at most 32 items
  int lvn[MAXLEV] = {};        // items per level
  bool linearized = false;
  OpData d64;                  // FP64 operators (always)
  OpData d32;                  // FP32 operators (BK_F32 problems)
  double* F = nullptr;         // KKT residual scratch (FP64, kkt_len)
  double* red = nullptr;       // reduction scratch (FP64)
  double* red_host = nullptr;  // pinned host mirror of reduction results
  size_t bytes = 0;            // device bytes this problem (and its plans) allocated
  double* sred = nullptr;      // reduction scratch of the free-time terms (FP64, 2048)
  void* gcache = nullptr;      // captured GMRES cycle graphs (bk_krylov.cu), keyed by their pointers
  // control bounds lo_q <= u_q <= hi_q (+-inf: none) by a logarithmic barrier on the quadrature
  // (problem (P)'s path constraints in their simplest form) and endpoint bounds on terminal rows
  // (its e^L <= e <= e^U); bar_mu is the barrier parameter the kernels use (mu_final outside
  // newton_solve's stages), mu0 / mu_final its schedule
  bool has_bounds = false;     // either kind below
  bool has_ubounds = false;
  double ulo[NUM] = {0, 0}, uhi[NUM] = {0, 0};
  bool has_ebounds = false;
  int term_bnd[NEM] = {0, 0, 0, 0};
  double term_lo[NEM] = {0, 0, 0, 0}, term_hi[NEM] = {0, 0, 0, 0};
  double term_ea[NEM] = {1, 1, 1, 1}, term_ec[NEM] = {0, 0, 0, 0};   // Newton rows at the linearisation
  double bar_mu = 0.0, bar_mu0 = 0.1, bar_mu_final = 1e-6;
  int bar_form = BK_BARRIER_PRIMAL;  // newton_solve's form of the barrier problem
  double* bar_buf = nullptr;   // newton_solve's bound multipliers: z, trial z, dz (2 n_u P each)
  const double* bar_z = nullptr;  // multipliers the kernels use (null: primal form)
  double* s_dev = nullptr;     // device copy of s (fixed final time): the GMRES-step kernels read s
                               // from here, so captured graphs stay valid when the parameters change
  int64_t kkt_len() const { return (2 * n_x + n_u) * P + 32; }
  // tail slot of s in a KKT vector (after nu) for a free final time
  int64_t s_idx() const { return (2 * n_x + n_u) * P + n_e; }
  // curvature of the running cost in u: |u|^2/2 for the cost-carrying kinds; BK_ORBIT_MT's
  // cost is the final time
  double cost_uu() const { return has_cost && !free_time ? 1.0 : 0.0; }
  // the kind's parameter inside the dynamics (the thrust a of BK_ORBIT_MT)
  double dyn_param() const { return kind == BK_ORBIT_MT ? params[0] : 0.0; }
  int64_t state_len() const { return n_x * P; }
  OpData& work() { return dtype == BK_F64 ? d64 : d32; }
  OpData& pre() { return pdtype == BK_F64 ? d64 : d32; }
};

// Control bounds and the current barrier parameter of a problem (mu = 0: no barrier terms).
inline BarSpec bar_spec(const Problem* pr) {
  BarSpec b;
  memset(&b, 0, sizeof(b));
  b.mu = pr->has_ubounds ? pr->bar_mu : 0.0;
  b.z = pr->has_ubounds ? pr->bar_z : nullptr;
  for (int q = 0; q < NUM; ++q) {
    b.lo[q] = pr->ulo[q];
    b.hi[q] = pr->uhi[q];
    b.has_lo[q] = pr->has_ubounds && q < pr->n_u && isfinite(pr->ulo[q]) ? 1 : 0;
    b.has_hi[q] = pr->has_ubounds && q < pr->n_u && isfinite(pr->uhi[q]) ? 1 : 0;
  }
  return b;
}

// Terminal conditions of a problem, with its endpoint bounds and their Newton rows.
inline TermSpec term_spec(const Problem* pr) {
  TermSpec t;
  memset(&t, 0, sizeof(t));
  t.n_e = pr->n_e;
  t.mu = pr->has_ebounds ? pr->bar_mu : 0.0;
  for (int r = 0; r < pr->n_e; ++r) {
    t.idx[r] = pr->term_idx[r];
    t.val[r] = pr->term_val[r];
    t.eb[r] = pr->has_ebounds && pr->term_bnd[r] ? 1 : 0;
    t.elo[r] = pr->term_lo[r];
    t.ehi[r] = pr->term_hi[r];
    t.ea[r] = t.eb[r] ? pr->term_ea[r] : 1.0;
    t.ec[r] = t.eb[r] ? pr->term_ec[r] : 0.0;
  }
  return t;
}

// mu (nullable): s B^aT lambda at z_lin, already known to the caller (FP64, n_x * P); when
// null it is computed with one transposed product. `keep` keeps part of the preconditioner of
// the previous linearisation: LIN_FULL rebuilds everything, LIN_KEEP_SCHUR keeps the terminal
// Schur data, LIN_KEEP_PRECOND keeps all of it (the operator data is always updated).
enum { LIN_FULL = 0, LIN_KEEP_SCHUR = 1, LIN_KEEP_PRECOND = 2 };
bk_status problem_linearize(Problem* pr, const double* z_lin, cudaStream_t st, const double* mu = nullptr,
                            int keep = LIN_FULL);
// Operator applies on one precision's data (T = double or float). For BK_OP_KKT, mu_out
// (nullable, n_x * P of T) receives s B^aT in_lambda, the operator's transposed product.
bk_status op_apply(Problem* pr, OpData& d, int op, const void* in, void* out, cudaStream_t st,
                   void* mu_out = nullptr);
bk_status op_precond(Problem* pr, OpData& d, int op, const void* in, void* out, int transpose,
                     cudaStream_t st);
// KKT residual at z (FP64) into F; weighted norm partial sums reduced on the host if wnorm.
// Mu (n_x * P, FP64) holds s B^aT lambda: given by the caller when mu_given, else computed into
// it (null: into the problem's scratch).
bk_status problem_residual(Problem* pr, const double* z, double* F, double* wnorm, cudaStream_t st,
                           double* Mu = nullptr, bool mu_given = false);
// Weighted norm of a residual vector (FP64), synchronous.
bk_status problem_wnorm(Problem* pr, const double* F, double* wnorm, cudaStream_t st);
// Drop the problem's captured GMRES cycle graphs (at destruction, and when a parameter that the
// graphs bake in changes).
void gmres_graphs_free(Problem* pr);

}  // namespace bk
