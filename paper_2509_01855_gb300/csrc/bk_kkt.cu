// Problems, linearisation, the KKT / state operators, the Birkhoff preconditioner sweeps and the
// KKT residual.
//
// Paper: "Construction of a Low-Memory Fast Million-Point Linear Solver" (Eqs. X-V=nonlin ..
// Achibetadef, FastAX), "Development of a Special Birkhoff-Centric Preconditioner" (B-tilde,
// FastBccV, P = I - B-tilde d_X f, FastPinvY), Eq. Prob-PNa (the discretised problem).
//
// Preconditioner sweep. Row k of P xi = Y with P = I - s (B-tilde (x) I) J_x reads
//   (I - h_k J_k) xi_k = Y_k + sigma_k,   sigma_k = s sum_{j<k} w_j J_j xi_j,   h_k = s w_k / 2,
// so xi_k = K_k (Y_k + sigma_k) with K_k = (I - h_k J_k)^{-1}, and sigma_{k+1} = sigma_k +
// N_k (Y_k + sigma_k), N_k = 2 h_k J_k K_k. (The sweep printed as FastPinvY subtracts the running
// sum and accumulates the input instead of the solution, which does not invert P; the recurrence
// above is what the rows of P give.) The transpose P^T y = r runs backwards:
//   y_j = K_j^T r_j + N_j^T rho_j,  rho_{j-1} = rho_j + y_j,  (B-tilde^T y)_j = w_j (y_j/2 + rho_j).
// Both are affine recurrences sigma_{k+1} = (I + N_k) sigma_k + f_k; they run as a chunked scan:
// segments of SEG nodes (one thread each, sequential; SEG = Seg<T>::v), then levels of blocks of 32 scanned by
// warps. The matrix parts of every level's maps depend only on the linearisation and are formed
// in bk_linearize; the backward maps are their transposes.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <vector>

#include "bk_problem.cuh"

namespace bk {

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
template <int SEG>
__device__ __forceinline__ int64_t il_index(int64_t k, int c, int NC) {
  // interleaved per-node storage: node k = seg * SEG + i, seg = W * 32 + lane
  const int64_t seg = k / SEG;
  const int i = (int)(k - seg * SEG);
  const int64_t W = seg >> 5;
  const int lane = (int)(seg & 31);
  return (((W * SEG + i) * NC + c) << 5) + lane;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  T a = T(0);
  if (threadIdx.x < 32) {
    a = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  }
  return a;  // valid in thread 0
}

static inline int nblk(int64_t n, int t = 256) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + t - 1) / t, 65535)); }
// Grid of the free-final-time reductions (grid-stride; partials fit the 2048-entry scratch).
constexpr int FT_NB = 608;

// ---------------------------------------------------------------------------------------------
// Linearisation kernels (FP64 arithmetic, results stored in T)
// ---------------------------------------------------------------------------------------------
// Node deviation in the compute type Tc (FP64 for FP64 problems; FP32 for FP32 problems, whose
// preconditioner works to FP32 accuracy anyway; the level products stay FP64):
// D = h J K = (I - h J)^{-1} h J, since K = (I - h J)^{-1} commutes with h J. One LU
// factorisation of I - h J with partial pivoting and the n_x columns of h J as right-hand
// sides: about 120 operations per node at n_x = 4, where inverting I - h J by Gauss-Jordan and
// multiplying by h J took about 240 (the kernel is bound by the FP64 pipe). Solving for D
// directly keeps its relative accuracy when h J is small (forming K - I would cancel).
template <typename Tc, int KIND, int NX>
__device__ void node_deviation(const Tc* x, const Tc* u, Tc h, Tc* D, Tc pa) {
  Tc Jx[NXM * NXM], Ju[NXM * NUM];
  Dyn<KIND>::template jac<Tc>(x, u, Jx, Ju, pa);
  Tc A[NX * NX], B[NX * NX], ip[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      B[r * NX + c] = h * Jx[r * NX + c];
      A[r * NX + c] = (r == c ? Tc(1) : Tc(0)) - B[r * NX + c];
    }
#pragma unroll
  for (int c = 0; c < NX; ++c) {
    int piv = c;
    Tc best = fabs((Tc)A[c * NX + c]);
#pragma unroll
    for (int r = c + 1; r < NX; ++r)
      if (fabs((Tc)A[r * NX + c]) > best) { best = fabs((Tc)A[r * NX + c]); piv = r; }
    // row swap by selects over the candidate rows: every index stays a compile-time constant,
    // so A and B live in registers (indexing by the run-time pivot put them in local memory)
#pragma unroll
    for (int r = c + 1; r < NX; ++r) {
      const bool sw = r == piv;
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        if (q >= c) {
          const Tc a = A[c * NX + q], b = A[r * NX + q];
          A[c * NX + q] = sw ? b : a;
          A[r * NX + q] = sw ? a : b;
        }
        const Tc ba = B[c * NX + q], bb = B[r * NX + q];
        B[c * NX + q] = sw ? bb : ba;
        B[r * NX + q] = sw ? ba : bb;
      }
    }
    ip[c] = Tc(1) / A[c * NX + c];
#pragma unroll
    for (int r = c + 1; r < NX; ++r) {
      const Tc f = A[r * NX + c] * ip[c];
#pragma unroll
      for (int q = c + 1; q < NX; ++q) A[r * NX + q] -= f * A[c * NX + q];
#pragma unroll
      for (int q = 0; q < NX; ++q) B[r * NX + q] -= f * B[c * NX + q];
    }
  }
  // back substitution, the n_x right-hand sides together
#pragma unroll
  for (int c = NX - 1; c >= 0; --c)
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      Tc a = B[c * NX + q];
#pragma unroll
      for (int k = c + 1; k < NX; ++k) a -= A[c * NX + k] * D[k * NX + q];
      D[c * NX + q] = a * ip[c];
    }
}

// Per node the sweeps need K = (I - h J)^{-1} and N = 2 h J K. Since K (I - h J) = I, h J K = K - I,
// so both follow from the deviation D = h J K: K = I + D, N = 2 D. Only D is stored (solved for
// directly by node_deviation), which halves the sweeps' node factor traffic and, with
// K v = v + D v and N v = 2 D v, their FP64 products.
template <typename T, int KIND, int NX, int NU>
__global__ void k_lin_nodes(const double* __restrict__ z, int64_t P, int64_t L, const double* __restrict__ w,
                            double s, T* __restrict__ Dn, T* __restrict__ xu, double pa) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    T x[NXM], u[NUM];
#pragma unroll
    for (int m = 0; m < NX; ++m) x[m] = (T)z[m * P + k];
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = (T)z[(NX + q) * P + k];
    T D[NX * NX];
    node_deviation<T, KIND, NX>(x, u, (T)(0.5 * s * w[k]), D, (T)pa);
#pragma unroll
    for (int c = 0; c < NX * NX; ++c) Dn[il_index<Seg<T>::v>(k, c, NX * NX)] = D[c];
#pragma unroll
    for (int m = 0; m < NX + NU; ++m) xu[m * P + k] = (T)z[m * P + k];
  }
}

// Level data of the sweep's affine maps. Level 0 items are segments of SEG nodes, whose map is
// the product of (I + N_k) over the segment (latest node on the left); a level-(l+1) item is a
// block of 32 level-l items and its map the product of theirs. The backward sweep uses the
// transposed maps in reverse order. Every map M is near the identity (N_k = O(s w_k)), so the
// level data stores its deviation D = M - I and composes (I + D1)(I + D2) = I + (D1 + D2 +
// D1 D2): storing M itself would round away the small part, which in FP32 left the sweeps 100x
// less accurate than a sequential FP32 recurrence at N = 2^17. Level data is in the working
// precision (FP64 levels cost FP32 problems FP64-pipe time in every sweep) and 32-interleaved (element c of item i at il32(i, c, NC)), so that a warp reading 32
// consecutive items is coalesced; slot q of a level starts at q * npad * n_x^2, npad = the
// level's item count rounded up to 32.
__device__ __forceinline__ int64_t il32(int64_t i, int c, int NC) { return (((i >> 5) * NC + c) << 5) + (i & 31); }

// Deviation of a product: (I + A)(I + B) = I + C with C = A + B + A B (n_x x n_x, row-major),
// each entry one FMA chain started from A + B (n_x^2 (n_x + 1) operations).
// Columns in ZeroCols<NX> are zero in A and B, hence in C, and are skipped.
template <int NX, typename Tm = double>
__device__ __forceinline__ void dev_mul(const Tm* A, const Tm* B, Tm* C) {
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int c = 0; c < NX; ++c) {
      if (zcol<NX>(c)) {
        C[r * NX + c] = Tm(0);
        continue;
      }
      Tm a = A[r * NX + c] + B[r * NX + c];
#pragma unroll
      for (int q = 0; q < NX; ++q)
        if (!zcol<NX>(q)) a = fma(A[r * NX + q], B[q * NX + c], a);
      C[r * NX + c] = a;
    }
}

// Level-0 maps: prod over the segment's nodes of (I + N_k) = (I + 2 D_k) as a deviation, one
// thread per segment: A <- (I + 2 D)(I + A) - I = A + 2 (D + D A), from A = 2 D of its first node.
template <typename T, int NX>
__global__ void k_lin_seg(const T* __restrict__ Dn, int64_t L, int nseg, T* __restrict__ A0) {
  const int seg = blockIdx.x * blockDim.x + threadIdx.x;
  if (seg >= nseg) return;
  constexpr int SEG = Seg<T>::v;
  T A[NX * NX], D[NX * NX], R[NX * NX];
  const int64_t k0 = (int64_t)seg * SEG;
#pragma unroll
  for (int c = 0; c < NX * NX; ++c) A[c] = zcol<NX>(c % NX) ? T(0) : T(2) * Dn[il_index<Seg<T>::v>(k0, c, NX * NX)];
  for (int i = 1; i < SEG; ++i) {
    const int64_t k = k0 + i;
    if (k >= L) break;
#pragma unroll
    for (int c = 0; c < NX * NX; ++c) D[c] = zcol<NX>(c % NX) ? T(0) : Dn[il_index<Seg<T>::v>(k, c, NX * NX)];
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int c = 0; c < NX; ++c) {
        if (zcol<NX>(c)) {
          R[r * NX + c] = T(0);
          continue;
        }
        T a = D[r * NX + c];
#pragma unroll
        for (int q = 0; q < NX; ++q)
          if (!zcol<NX>(q)) a = fma(D[r * NX + q], A[q * NX + c], a);
        R[r * NX + c] = fma(T(2), a, A[r * NX + c]);
      }
#pragma unroll
    for (int c = 0; c < NX * NX; ++c) A[c] = R[c];
  }
#pragma unroll
  for (int c = 0; c < NX * NX; ++c) A0[il32(seg, c, NX * NX)] = A[c];
}

// Slots of one level (deviations from I), one warp per block of 32 items (items at or beyond n
// are identity maps, deviation 0):
// spans M_k(j) = M_{k-1}(j) M_{k-1}(j - 2^{k-1}) by doubling (defined for j >= 2^k - 1), Pre(i)
// and Suf(i) as products of the spans that tile [0, i) and (i, 31], and the block's product
// M_4(31) M_4(15), which is the map of the parent item at the next level.
template <typename T, int NX>
__global__ void __launch_bounds__(32) k_lin_level(T* __restrict__ m, int n, T* __restrict__ parent) {
  constexpr int NC = NX * NX;
  __shared__ T S[5][32][NC + 1];
  const int lane = threadIdx.x;
  const int64_t i = (int64_t)blockIdx.x * 32 + lane;
  const int64_t slot = (int64_t)gridDim.x * 32 * NC;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const T a = i < n ? m[il32(i, c, NC)] : T(0);
    S[0][lane][c] = a;
    if (i >= n) m[il32(i, c, NC)] = T(0);
  }
  __syncwarp();
  for (int k = 1; k < 5; ++k) {
    const int h = 1 << (k - 1);
    T R[NC];
    if (lane >= 2 * h - 1) {
      dev_mul<NX, T>(S[k - 1][lane], S[k - 1][lane - h], R);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) R[c] = T(0);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) S[k][lane][c] = R[c];
    __syncwarp();
  }
#pragma unroll
  for (int k = 1; k < 5; ++k)
#pragma unroll
    for (int c = 0; c < NC; ++c) m[k * slot + il32(i, c, NC)] = S[k][lane][c];
  T R[NC], Q[NC];
  // Pre(i) = A_{i-1} ... A_0
#pragma unroll
  for (int c = 0; c < NC; ++c) R[c] = T(0);
  int pos = 0;
  for (int k = 4; k >= 0; --k) {
    if ((lane >> k) & 1) {
      dev_mul<NX, T>(S[k][pos + (1 << k) - 1], R, Q);
#pragma unroll
      for (int c = 0; c < NC; ++c) R[c] = Q[c];
      pos += 1 << k;
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) m[SL_PRE * slot + il32(i, c, NC)] = R[c];
  // Suf(i) = A_31 ... A_{i+1}
#pragma unroll
  for (int c = 0; c < NC; ++c) R[c] = T(0);
  int end = 31;
  const int len = 31 - lane;
  for (int k = 4; k >= 0; --k) {
    if ((len >> k) & 1) {
      dev_mul<NX, T>(R, S[k][end], Q);
#pragma unroll
      for (int c = 0; c < NC; ++c) R[c] = Q[c];
      end -= 1 << k;
    }
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) m[SL_SUF * slot + il32(i, c, NC)] = R[c];
  if (parent) {
    for (int c = lane; c < NC; c += 32) {
      const int r = c / NX, cc = c % NX;
      T a = 0;
#pragma unroll
      for (int q = 0; q < NX; ++q) a += S[4][31][r * NX + q] * S[4][15][q * NX + cc];
      parent[il32(blockIdx.x, c, NC)] = (S[4][31][c] + S[4][15][c]) + a;
    }
  }
}

template <typename Tin, typename Tout>
__global__ void k_convert(const Tin* __restrict__ a, Tout* __restrict__ b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (Tout)a[i];
}

// ---------------------------------------------------------------------------------------------
// Sweep kernels. Forward (DIR = 0): sigma_{k+1} = (I + N_k) sigma_k + N_k y'_k + 2 h_k g_k with
// y'_k = Y_k + h_k g_k, output xi_k = K_k (y'_k + sigma_k). Backward (DIR = 1): rho_{j-1} =
// (I + N_j^T) rho_j + K_j^T r_j, output y_j = K_j^T r_j + N_j^T rho_j, optional b_j =
// w_j (y_j / 2 + rho_j).
//
// A sweep scans the affine maps sigma -> A sigma + b level by level. The up kernels form each
// item's offset b (its map applied to a zero state) and the inclusive scan e of the offsets
// within its block of 32: a Kogge-Stone scan over the lanes of a warp with the span matrices,
// so that every FP64 instruction runs on all 32 lanes (a warp instruction occupies the FP64
// pipe for its full width whatever its active mask). The down kernel composes, for its segment,
// the incoming state from the top level down, S <- Pre(i) S + e(i-1) (backward:
// S <- Suf(i)^T S + e(i+1)), and reruns the segment's nodes from it.
// ---------------------------------------------------------------------------------------------
template <typename T> struct Levels {
  const T* m[MAXLEV];  // matrix slots per level
  T* o[MAXLEV];        // item offsets from zero, levels >= 1
  T* e[MAXLEV];        // inclusive in-block scan values
  int n[MAXLEV];       // items per level
  int nlev;
  const double* sdev;  // the time scale on the device (null: the kernel argument s)
};

// One node of a sweep with the node's deviation D (K = I + D, N = 2 D):
//   DIR 0: v = y + h g + st,  out = K v = v + D v,  st <- st + 2 h g + N v = st + 2 h g + 2 D v
//   DIR 1: y = K^T yin + N^T st = yin + D^T (yin + 2 st),  out = y and y / 2 + st,  st <- st + y
template <typename T, int NX, int DIR>
__device__ __forceinline__ void node_step(const T* __restrict__ Dn, int64_t k, const T* yin, const T* gin, T h,
                                          T* st, T* out, bool want_out) {
  T Dm[NX * NX];   // entries in a zero column (ZeroCols) are neither loaded nor used
#pragma unroll
  for (int c = 0; c < NX * NX; ++c) Dm[c] = zcol<NX>(c % NX) ? T(0) : Dn[il_index<Seg<T>::v>(k, c, NX * NX)];
  if (DIR == 0) {
    T v[NX], dv[NX];
#pragma unroll
    for (int m = 0; m < NX; ++m) v[m] = yin[m] + h * gin[m] + st[m];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      T a = T(0);
#pragma unroll
      for (int c = 0; c < NX; ++c)
        if (!zcol<NX>(c)) a += Dm[r * NX + c] * v[c];
      dv[r] = a;
    }
    if (want_out) {
#pragma unroll
      for (int r = 0; r < NX; ++r) out[r] = v[r] + dv[r];
    }
#pragma unroll
    for (int r = 0; r < NX; ++r) st[r] = (st[r] + T(2) * h * gin[r]) + T(2) * dv[r];
  } else {
    T q[NX], y[NX];
#pragma unroll
    for (int c = 0; c < NX; ++c) q[c] = yin[c] + T(2) * st[c];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      T a = T(0);
#pragma unroll
      for (int c = 0; c < NX; ++c)
        if (!zcol<NX>(r)) a += Dm[c * NX + r] * q[c];
      y[r] = yin[r] + a;
    }
    if (want_out) {
#pragma unroll
      for (int r = 0; r < NX; ++r) { out[r] = y[r]; out[NX + r] = y[r] * T(0.5) + st[r]; }
    }
#pragma unroll
    for (int r = 0; r < NX; ++r) st[r] += y[r];
  }
}

// Inclusive scan of the offsets e within block blk (lane i holds item 32 blk + i), level slot
// size `slot`. DIR 0: e_i += M_k(i) e_{i-2^k}; DIR 1 (reverse order, transposed maps):
// e_i += M_k(i + 2^k - 1)^T e_{i+2^k}.
template <typename T, int NX, int DIR>
__device__ __forceinline__ void warp_scan(const T* __restrict__ m, int64_t slot, int64_t blk, T* e) {
  constexpr int NC = NX * NX;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const int d = 1 << k;
    T pe[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r)
      pe[r] = DIR == 0 ? shfl_up(e[r], d) : shfl_down(e[r], d);
    const bool act = DIR == 0 ? lane >= d : lane + d < 32;
    if (act) {
      const int64_t item = blk * 32 + (DIR == 0 ? lane : lane + d - 1);
      const T* M = m + k * slot;
      T Mv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) Mv[c] = zcol<NX>(c % NX) ? T(0) : M[il32(item, c, NC)];
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        T a = T(0);   // (I + D) pe = pe + D pe
#pragma unroll
        for (int c = 0; c < NX; ++c)
          if (!zcol<NX>(DIR == 0 ? c : r)) a += (DIR == 0 ? Mv[r * NX + c] : Mv[c * NX + r]) * pe[c];
        e[r] = e[r] + (pe[r] + a);
      }
    }
  }
}

// Per-node vectors of a warp's 32 segments move through shared memory in chunks of CH nodes
// (one 32-byte sector per segment and component), so that every global access is sector-
// coalesced: lane l of staging instruction q handles element q*32 + l of the [segment][node]
// chunk. Reading them lane-by-segment directly (a 16-node stride) wasted most of each sector.
template <typename T> struct SweepChunk {
  static constexpr int CH = 32 / (int)sizeof(T);   // nodes per chunk
  static constexpr int TS = CH + 1;                // padded row (bank spread)
  static_assert(Seg<T>::v % CH == 0, "segment length must be a multiple of the staging chunk");
};

template <typename T>
__device__ __forceinline__ void stage_in(const T* __restrict__ src, int64_t P, int nc, int64_t L, int64_t seg0,
                                         int i0, T* __restrict__ tile) {
  constexpr int CH = SweepChunk<T>::CH, TS = SweepChunk<T>::TS, SEG = Seg<T>::v;
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < nc; ++c) {
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int e = q * 32 + lane;
      const int sl = e / CH, nd = e - (e / CH) * CH;
      const int64_t k = (seg0 + sl) * SEG + i0 + nd;
      tile[(c * 32 + sl) * TS + nd] = k < L ? src[c * P + k] : T(0);
    }
  }
}

template <typename T>
__device__ __forceinline__ void stage_out(const T* __restrict__ tile, int nc, int64_t P, int64_t L, int64_t seg0,
                                          int i0, T* __restrict__ dst) {
  constexpr int CH = SweepChunk<T>::CH, TS = SweepChunk<T>::TS, SEG = Seg<T>::v;
  const int lane = threadIdx.x & 31;
  for (int c = 0; c < nc; ++c) {
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int e = q * 32 + lane;
      const int sl = e / CH, nd = e - (e / CH) * CH;
      const int64_t k = (seg0 + sl) * SEG + i0 + nd;
      if (k < L) dst[c * P + k] = tile[(c * 32 + sl) * TS + nd];
    }
  }
}

// Shared tiles of one warp: A (n_x components), B (n_x components), W (1 component).
template <typename T, int NX> struct SweepTiles {
  static constexpr int ROWS = 32 * SweepChunk<T>::TS;
  T a[NX * ROWS], b[NX * ROWS], w[ROWS];
};

// Nonzero test on the bit pattern (integer pipe; +0 and -0 count as zero): the sweeps use it to
// skip work whose inputs are all zero without spending FP64 instructions on the test.
__device__ __forceinline__ bool nonzero(double x) { return (__double_as_longlong(x) << 1) != 0; }
__device__ __forceinline__ bool nonzero(float x) { return (__float_as_int(x) << 1) != 0; }

// Up, level 0 (one warp per block of 32 segments, 4 warps per CTA): each lane runs its segment
// from a zero state (the segment's offset), then the warp scans the block. A chunk whose inputs
// and states are zero on every lane leaves the states zero and is skipped, and a block whose
// offsets are all zero has zero scan values: the terminal Schur columns' right-hand sides are
// unit vectors at the last node, so their up passes do almost no FP64 work.
template <typename T, int NX, int DIR>
__device__ __forceinline__ void sw_up0_warp(int g, SweepTiles<T, NX>& tl, const T* __restrict__ Dn,
                                            const T* __restrict__ Y,
                                            const T* __restrict__ G, int64_t P, int64_t L, const T* __restrict__ w,
                                            T s, const Levels<T>& lv) {
  constexpr int CH = SweepChunk<T>::CH, TS = SweepChunk<T>::TS, SEG = Seg<T>::v;
  const int nblk = (lv.n[0] + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t seg0 = (int64_t)g * 32;
  const int64_t seg = seg0 + lane;
  if (lv.sdev) s = T(*lv.sdev);
  T st[NX];
#pragma unroll
  for (int m = 0; m < NX; ++m) st[m] = T(0);
  for (int c = 0; c < SEG / CH; ++c) {
    const int i0 = (DIR == 0 ? c : SEG / CH - 1 - c) * CH;
    __syncwarp();
    stage_in<T>(Y, P, NX, L, seg0, i0, tl.a);
    if (G) stage_in<T>(G, P, NX, L, seg0, i0, tl.b);
    stage_in<T>(w, P, 1, L, seg0, i0, tl.w);
    __syncwarp();
    bool act = false;
#pragma unroll
    for (int m = 0; m < NX; ++m) {
      act |= nonzero(st[m]);
#pragma unroll
      for (int jj = 0; jj < CH; ++jj) {
        act |= nonzero(tl.a[(m * 32 + lane) * TS + jj]);
        if (G) act |= nonzero(tl.b[(m * 32 + lane) * TS + jj]);
      }
    }
    if (!__any_sync(0xffffffffu, act)) continue;
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) {
      const int nd = DIR == 0 ? jj : CH - 1 - jj;
      const int64_t k = seg * SEG + i0 + nd;
      if (seg < lv.n[0] && k < L) {
        T yin[NX], gin[NX], dummy[2 * NX];
#pragma unroll
        for (int m = 0; m < NX; ++m) {
          yin[m] = tl.a[(m * 32 + lane) * TS + nd];
          gin[m] = G ? tl.b[(m * 32 + lane) * TS + nd] : T(0);
        }
        node_step<T, NX, DIR>(Dn, k, yin, gin, T(0.5) * s * tl.w[lane * TS + nd], st, dummy, false);
      }
    }
  }
  T e[NX];
  bool any = false;
#pragma unroll
  for (int m = 0; m < NX; ++m) {
    e[m] = st[m];
    any |= nonzero(st[m]);
  }
  if (__any_sync(0xffffffffu, any)) warp_scan<T, NX, DIR>(lv.m[0], (int64_t)nblk * 32 * NX * NX, g, e);
#pragma unroll
  for (int m = 0; m < NX; ++m) lv.e[0][il32(seg, m, NX)] = e[m];
  if (lv.nlev > 1 && lane == (DIR == 0 ? 31 : 0)) {
#pragma unroll
    for (int m = 0; m < NX; ++m) lv.o[1][il32(g, m, NX)] = e[m];
  }
}

// Up, level l >= 1 (one warp per block of 32 items): scan of the items' offsets.
template <typename T, int NX, int DIR>
__device__ __forceinline__ void sw_upL_warp(int b, const Levels<T>& lv, int l) {
  const int n = lv.n[l];
  const int nblk = (n + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)b * 32 + lane;
  const T* o = lv.o[l];
  T e[NX];
  bool any = false;
#pragma unroll
  for (int m = 0; m < NX; ++m) {
    e[m] = i < n ? o[il32(i, m, NX)] : T(0);
    any |= nonzero(e[m]);
  }
  if (__any_sync(0xffffffffu, any)) warp_scan<T, NX, DIR>(lv.m[l], (int64_t)nblk * 32 * NX * NX, b, e);
  T* el = lv.e[l];
#pragma unroll
  for (int m = 0; m < NX; ++m) el[il32(i, m, NX)] = e[m];
  if (l + 1 < lv.nlev && lane == (DIR == 0 ? 31 : 0)) {
    T* op = lv.o[l + 1];
#pragma unroll
    for (int m = 0; m < NX; ++m) op[il32(b, m, NX)] = e[m];
  }
}

// Down (one warp per block of 32 segments): incoming state of the lane's segment, composed from
// the top level down, then the segment's nodes with outputs (staged like the inputs).
template <typename T, int NX, int DIR>
__device__ __forceinline__ void sw_down0_warp(int g, SweepTiles<T, NX>& tl, const T* __restrict__ Dn,
                                              const T* __restrict__ Y,
                                              const T* __restrict__ G, int64_t P, int64_t L,
                                              const T* __restrict__ w, T s, const Levels<T>& lv,
                                              T* __restrict__ out, T* __restrict__ bout) {
  constexpr int NC = NX * NX;
  constexpr int CH = SweepChunk<T>::CH, TS = SweepChunk<T>::TS, SEG = Seg<T>::v;
  const int nblk0 = (lv.n[0] + 31) >> 5;
  const int lane = threadIdx.x & 31;
  if (lv.sdev) s = T(*lv.sdev);
  const int64_t seg0 = (int64_t)g * 32;
  const int64_t seg = seg0 + lane;
  const bool live = seg < lv.n[0];
  T S[NX];
#pragma unroll
  for (int m = 0; m < NX; ++m) S[m] = T(0);
  for (int l = lv.nlev - 1; l >= 0 && live; --l) {
    const int64_t i = seg >> (5 * l);
    const int q = (int)(i & 31);
    if (DIR == 0 ? q == 0 : q == 31) continue;  // first item of its block in sweep order
    const int64_t slot = (int64_t)((lv.n[l] + 31) >> 5) * 32 * NC;
    const T* Mt = lv.m[l] + (DIR == 0 ? SL_PRE : SL_SUF) * slot;
    const T* el = lv.e[l];
    const int64_t ia = DIR == 0 ? i - 1 : i + 1;
    T Mv[NC], ns[NX];
#pragma unroll
    for (int c = 0; c < NC; ++c) Mv[c] = zcol<NX>(c % NX) ? T(0) : Mt[il32(i, c, NC)];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      T a = T(0);   // (I + D) S = S + D S
#pragma unroll
      for (int c = 0; c < NX; ++c)
        if (!zcol<NX>(DIR == 0 ? c : r)) a += (DIR == 0 ? Mv[r * NX + c] : Mv[c * NX + r]) * S[c];
      ns[r] = el[il32(ia, r, NX)] + (S[r] + a);
    }
#pragma unroll
    for (int r = 0; r < NX; ++r) S[r] = ns[r];
  }
  T st[NX];
#pragma unroll
  for (int m = 0; m < NX; ++m) st[m] = S[m];
  const bool wantb = DIR == 1 && bout != nullptr;
  for (int c = 0; c < SEG / CH; ++c) {
    const int i0 = (DIR == 0 ? c : SEG / CH - 1 - c) * CH;
    __syncwarp();
    stage_in<T>(Y, P, NX, L, seg0, i0, tl.a);
    if (DIR == 0 && G) stage_in<T>(G, P, NX, L, seg0, i0, tl.b);
    stage_in<T>(w, P, 1, L, seg0, i0, tl.w);
    __syncwarp();
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) {
      const int nd = DIR == 0 ? jj : CH - 1 - jj;
      const int64_t k = seg * SEG + i0 + nd;
      if (live && k < L) {
        T yin[NX], gin[NX], o[2 * NX];
#pragma unroll
        for (int m = 0; m < NX; ++m) {
          yin[m] = tl.a[(m * 32 + lane) * TS + nd];
          gin[m] = (DIR == 0 && G) ? tl.b[(m * 32 + lane) * TS + nd] : T(0);
        }
        const T wk = tl.w[lane * TS + nd];
        node_step<T, NX, DIR>(Dn, k, yin, gin, T(0.5) * s * wk, st, o, true);
        // outputs replace the inputs just read (same lane, same node)
#pragma unroll
        for (int m = 0; m < NX; ++m) tl.a[(m * 32 + lane) * TS + nd] = o[m];
        if (wantb) {
#pragma unroll
          for (int m = 0; m < NX; ++m) tl.b[(m * 32 + lane) * TS + nd] = wk * o[NX + m];
        }
      }
    }
    __syncwarp();
    stage_out<T>(tl.a, NX, P, L, seg0, i0, out);
    if (wantb) stage_out<T>(tl.b, NX, P, L, seg0, i0, bout);
  }
  // the warp of the last block also zeroes the outputs' padding (elements L..P-1)
  if (g == nblk0 - 1) {
    for (int c = 0; c < NX; ++c)
      for (int64_t k = L + lane; k < P; k += 32) {
        out[c * P + k] = T(0);
        if (wantb) bout[c * P + k] = T(0);
      }
  }
}

// The sweep kernels: one warp per block of 32 items, W warps per CTA (4; 1 for grids whose
// level 0 has fewer blocks than four per SM, so that their warps spread over the SMs: each
// warp's segments are sequential chains whose FP64 arithmetic would otherwise share one SM's
// FP64 pipe).
template <typename T, int NX, int DIR, int W>
__global__ void __launch_bounds__(32 * W) k_sw_up0(const T* __restrict__ Dn, const T* __restrict__ Y, const T* __restrict__ G, int64_t P,
                                                   int64_t L, const T* __restrict__ w, T s, Levels<T> lv) {
  __shared__ SweepTiles<T, NX> tiles[W];
  const int g = blockIdx.x * W + (threadIdx.x >> 5);
  if (g >= ((lv.n[0] + 31) >> 5)) return;  // whole warps
  sw_up0_warp<T, NX, DIR>(g, tiles[threadIdx.x >> 5], Dn, Y, G, P, L, w, s, lv);
}

template <typename T, int NX, int DIR, int W>
__global__ void __launch_bounds__(32 * W) k_sw_upL(Levels<T> lv, int l) {
  const int b = blockIdx.x * W + (threadIdx.x >> 5);
  if (b >= ((lv.n[l] + 31) >> 5)) return;
  sw_upL_warp<T, NX, DIR>(b, lv, l);
}

template <typename T, int NX, int DIR, int W>
__global__ void __launch_bounds__(32 * W) k_sw_down0(const T* __restrict__ Dn, const T* __restrict__ Y, const T* __restrict__ G, int64_t P,
                                                     int64_t L, const T* __restrict__ w, T s, Levels<T> lv,
                                                     T* __restrict__ out, T* __restrict__ bout) {
  __shared__ SweepTiles<T, NX> tiles[W];
  const int g = blockIdx.x * W + (threadIdx.x >> 5);
  if (g >= ((lv.n[0] + 31) >> 5)) return;  // whole warps
  sw_down0_warp<T, NX, DIR>(g, tiles[threadIdx.x >> 5], Dn, Y, G, P, L, w, s, lv, out, bout);
}

// The whole sweep in one CTA for small grids (at most two scan levels and SW1_MAXW blocks of 32
// segments): one warp per block; the level-0 up pass, the level-1 scan by warp 0 and the down
// pass are separated by barriers instead of launches (1 launch instead of nlev + 1; the serving
// mix's small problems run many sweeps per Newton step).
constexpr int SW1_MAXW = 16;
template <typename T, int NX, int DIR>
__global__ void __launch_bounds__(32 * SW1_MAXW) k_sw_one(const T* __restrict__ Dn, const T* __restrict__ Y, const T* __restrict__ G,
                                                          int64_t P, int64_t L, const T* __restrict__ w, T s,
                                                          Levels<T> lv, T* __restrict__ out, T* __restrict__ bout) {
  extern __shared__ __align__(16) unsigned char sw1_smem[];
  SweepTiles<T, NX>* tiles = reinterpret_cast<SweepTiles<T, NX>*>(sw1_smem);
  const int warp = threadIdx.x >> 5;
  const int nblk0 = (lv.n[0] + 31) >> 5;
  if (warp < nblk0) sw_up0_warp<T, NX, DIR>(warp, tiles[warp], Dn, Y, G, P, L, w, s, lv);
  __syncthreads();
  if (lv.nlev > 1 && warp == 0) sw_upL_warp<T, NX, DIR>(0, lv, 1);
  __syncthreads();
  if (warp < nblk0) sw_down0_warp<T, NX, DIR>(warp, tiles[warp], Dn, Y, G, P, L, w, s, lv, out, bout);
}

// The sweep kernels keep up to four 4-warp CTAs per SM; give shared memory the whole L1 array.
template <typename T, int NX>
static bk_status sweep_attrs() {
  BK_TRY_CUDA(cudaFuncSetAttribute(k_sw_up0<T, NX, 0, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  BK_TRY_CUDA(cudaFuncSetAttribute(k_sw_up0<T, NX, 1, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  BK_TRY_CUDA(cudaFuncSetAttribute(k_sw_down0<T, NX, 0, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  BK_TRY_CUDA(cudaFuncSetAttribute(k_sw_down0<T, NX, 1, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  const int sm1 = (int)(SW1_MAXW * sizeof(SweepTiles<T, NX>));
  BK_TRY_CUDA(cudaFuncSetAttribute(k_sw_one<T, NX, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1));
  BK_TRY_CUDA(cudaFuncSetAttribute(k_sw_one<T, NX, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm1));
  return BK_OK;
}

template <typename T>
static bk_status sweep_attrs_nx(int nx) {
  if (nx == 1) return sweep_attrs<T, 1>();
  if (nx == 2) return sweep_attrs<T, 2>();
  return sweep_attrs<T, 4>();
}

// The time scale the GMRES-step kernels read: the device copy for a fixed final time, none
// (the kernel argument) for a free one, whose s changes inside a Newton step.
static const double* sdev_of(const Problem* pr) { return pr->free_time ? nullptr : pr->s_dev; }

template <typename T>
static Levels<T> levels_of(const Problem* pr, const OpData& d) {
  Levels<T> lv;
  memset(&lv, 0, sizeof(lv));
  lv.nlev = pr->nlev;
  for (int l = 0; l < pr->nlev; ++l) {
    lv.m[l] = (const T*)d.lvm[l];
    lv.o[l] = (T*)d.lvo[l];
    lv.e[l] = (T*)d.lve[l];
    lv.n[l] = pr->lvn[l];
  }
  lv.sdev = sdev_of(pr);
  return lv;
}

// Sweep launch form: 0 automatic, 1 one CTA (small grids only), 2 one warp per CTA, 3 four
// warps per CTA (BK_SWEEP_FORM overrides the automatic choice, for timing).
static int sweep_form() {
  static const int f = [] {
    const char* e = getenv("BK_SWEEP_FORM");
    const int v = e ? atoi(e) : 0;
    return v >= 1 && v <= 3 ? v : 0;
  }();
  return f;
}

template <typename T, int NX, int DIR, int W>
static bk_status run_sweep_multi(Problem* pr, OpData& d, const T* Y, const T* G, T* out, T* bout, const T* w, T s,
                                 const Levels<T>& lv, cudaStream_t st) {
  const int g0 = (((pr->lvn[0] + 31) >> 5) + W - 1) / W;
  k_sw_up0<T, NX, DIR, W><<<g0, 32 * W, 0, st>>>((const T*)d.Dn, Y, G, pr->P, pr->L, w, s, lv);
  BK_CHECK_LAUNCH();
  for (int l = 1; l < pr->nlev; ++l) {
    const int gl = (((pr->lvn[l] + 31) >> 5) + W - 1) / W;
    k_sw_upL<T, NX, DIR, W><<<gl, 32 * W, 0, st>>>(lv, l);
    BK_CHECK_LAUNCH();
  }
  k_sw_down0<T, NX, DIR, W><<<g0, 32 * W, 0, st>>>((const T*)d.Dn, Y, G, pr->P, pr->L, w, s, lv, out, bout);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// Full sweep: out = P^{-1} (Y, forcing G) (DIR 0) or P^{-T} Y with bout = B-tilde^T out (DIR 1).
// Grids with at most two scan levels and 16 level-0 blocks: one launch (k_sw_one). Otherwise
// nlev + 1 launches (the level-0 up pass, one scan per upper level, the down pass), one warp per
// CTA while level 0 has fewer than four blocks per SM, else four. Measured orbit solves (GB300,
// host-form GMRES, ms, one CTA / 1-warp / 4-warp CTAs): FP64 2^8 7.35 / 7.61 / 7.56, FP32 2^16
// (1-warp range) - / 7.29 / 8.18, FP64 2^16 - / 12.84 / 13.04.
template <typename T, int NX, int DIR>
static bk_status run_sweep(Problem* pr, OpData& d, const T* Y, const T* G, T* out, T* bout, cudaStream_t st) {
  // segment length and level data follow the problem's preconditioner precision
  BK_ARG(d.dtype == pr->pdtype && d.Dn != nullptr, "sweeps run in the preconditioner's precision only");
  const T* w = (const T*)d.w;
  const T s = (T)pr->s;
  const Levels<T> lv = levels_of<T>(pr, d);
  const int nblk0 = (pr->lvn[0] + 31) >> 5;
  int form = sweep_form();
  if (form == 1 && !(pr->nlev <= 2 && nblk0 <= SW1_MAXW)) form = 0;
  if (form == 0) form = nblk0 < 4 * 152 ? 2 : 3;
  if (form == 1) {
    k_sw_one<T, NX, DIR><<<1, 32 * nblk0, nblk0 * sizeof(SweepTiles<T, NX>), st>>>(
        (const T*)d.Dn, Y, G, pr->P, pr->L, w, s, lv, out, bout);
    BK_CHECK_LAUNCH();
    return BK_OK;
  }
  if (form == 2) return run_sweep_multi<T, NX, DIR, 1>(pr, d, Y, G, out, bout, w, s, lv, st);
  return run_sweep_multi<T, NX, DIR, 4>(pr, d, Y, G, out, bout, w, s, lv, st);
}

// ---------------------------------------------------------------------------------------------
// KKT / state operator kernels (per node, Jacobians and Hessian recomputed from (x, u, mu))
// ---------------------------------------------------------------------------------------------
// t = J dz per node; with a free final time (ds != null) t += (ds / s) f, so that the product
// s B^a t adds the column d c / ds = -B^a f times ds.
template <typename T, int KIND>
__global__ void k_jvp(const T* __restrict__ xu, const T* __restrict__ dX, const T* __restrict__ dU, int64_t P,
                      int64_t L, T* __restrict__ t, T pa, const T* __restrict__ ds, T inv_s) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  const T dss = ds ? ds[0] * inv_s : T(0);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    T x[NXM], u[NUM], Jx[NXM * NXM], Ju[NXM * NUM], fx[NXM];
#pragma unroll
    for (int m = 0; m < NX; ++m) x[m] = xu[m * P + k];
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = xu[(NX + q) * P + k];
    Dyn<KIND>::template jac<T>(x, u, Jx, Ju, pa);
    if (ds) Dyn<KIND>::template f<T>(x, u, fx, pa);
#pragma unroll
    for (int m = 0; m < NX; ++m) {
      T a = ds ? dss * fx[m] : T(0);
#pragma unroll
      for (int p = 0; p < NX; ++p)
        if (Dyn<KIND>::jx_nz(m, p)) a += Jx[m * NX + p] * dX[p * P + k];
      if (dU) {
#pragma unroll
        for (int q = 0; q < NU; ++q)
          if (Dyn<KIND>::ju_nz(m, q)) a += Ju[m * NU + q] * dU[q * P + k];
      }
      t[m * P + k] = a;
    }
  }
}

// out = chi - Bt (state operator), padding zeroed. With sdev, Bt holds B^a (J chi) and the time
// scale is applied here from the device; without, Bt = s B^a (J chi).
template <typename T, int NX>
__global__ void k_state_post(const T* __restrict__ chi, const T* __restrict__ Bt, int64_t P, int64_t L,
                             T* __restrict__ out, const double* __restrict__ sdev) {
  const T s = sdev ? T(*sdev) : T(1);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < NX * P; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = i % P;
    out[i] = k < L ? chi[i] - (sdev ? s * Bt[i] : Bt[i]) : T(0);
  }
}


// KKT product: out = [H dz + G^T dy ; G dz], with Bt = s B^a (J dz), Mu = s B^aT dlambda.
// Free final time (part != null): the gradient rows add ds d g / ds = -(ds / s) J^T mu, and each
// block writes its partial of mu . (J dz) + f . Mu; the s row is -(1/s) times their sum
// (k_free_finish), i.e. -(B^aT lambda) . (J dz) - (B^a f) . dlambda.
template <typename T, int KIND>
__global__ void k_kkt_post(const T* __restrict__ xu, const T* __restrict__ mu, const T* __restrict__ w, T s,
                           const T* __restrict__ in, const T* __restrict__ Bt, T* __restrict__ Mu, int64_t P,
                           int64_t L, TermSpec ts, T cost_uu, T* __restrict__ out, T pa, int64_t s_idx,
                           double* __restrict__ part, const double* __restrict__ sdev,
                           const T* __restrict__ hbar) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu, NV = NX + NU;
  __shared__ double red[32];
  // sdev: Bt and Mu arrive unscaled (B^a, B^aT products) and take the device time scale here;
  // the scaled Mu is written back (the caller's record of s B^aT dlambda)
  if (sdev) s = T(*sdev);
  const T dss = part ? in[s_idx] / s : T(0);
  double sacc = 0.0;
  const T* dX = in;
  const T* dU = in + NX * P;
  const T* dL = in + NV * P;
  const T* dNu = in + (NV + NX) * P;
  T* oX = out;
  T* oU = out + NX * P;
  T* oL = out + NV * P;
  T* oNu = out + (NV + NX) * P;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    if (k >= L) {
#pragma unroll
      for (int m = 0; m < NV + NX; ++m) out[m * P + k] = T(0);
      continue;
    }
    T x[NXM], u[NUM], m_[NXM], Jx[NXM * NXM], Ju[NXM * NUM], H[(NXM + NUM) * (NXM + NUM)], dz[NXM + NUM], mp[NXM];
#pragma unroll
    for (int m = 0; m < NX; ++m) {
      x[m] = xu[m * P + k];
      m_[m] = mu[m * P + k];
      dz[m] = dX[m * P + k];
      mp[m] = Mu[m * P + k];
      if (sdev) {
        mp[m] = s * mp[m];
        Mu[m * P + k] = mp[m];
      }
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) { u[q] = xu[(NX + q) * P + k]; dz[NX + q] = dU[q * P + k]; }
    Dyn<KIND>::template jac<T>(x, u, Jx, Ju, pa);
    Dyn<KIND>::template hess<T>(x, u, m_, H, pa);
    const T swk = s * w[k] * cost_uu;
    T hb[NUM];   // control bounds: the barrier's diagonal of the control block
#pragma unroll
    for (int q = 0; q < NU; ++q) hb[q] = hbar ? hbar[q * P + k] : T(0);
    if (part) {
      T fx[NXM];
      Dyn<KIND>::template f<T>(x, u, fx, pa);
#pragma unroll
      for (int m = 0; m < NX; ++m) {
        T jd = T(0);
#pragma unroll
        for (int p = 0; p < NX; ++p)
          if (Dyn<KIND>::jx_nz(m, p)) jd += Jx[m * NX + p] * dz[p];
#pragma unroll
        for (int q = 0; q < NU; ++q)
          if (Dyn<KIND>::ju_nz(m, q)) jd += Ju[m * NU + q] * dz[NX + q];
        sacc += (double)m_[m] * (double)jd + (double)fx[m] * (double)mp[m];
      }
    }
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      T acc = T(0);
#pragma unroll
      for (int b = 0; b < NV; ++b)
        if (Dyn<KIND>::h_nz(a, b)) acc -= H[a * NV + b] * dz[b];
      if (a >= NX) acc += (swk + hb[a - NX]) * dz[a];
      if (a < NX) {
        acc += dL[a * P + k];
#pragma unroll
        for (int m = 0; m < NX; ++m)
          if (Dyn<KIND>::jx_nz(m, a)) acc -= Jx[m * NX + a] * (mp[m] + dss * m_[m]);
      } else {
#pragma unroll
        for (int m = 0; m < NX; ++m)
          if (Dyn<KIND>::ju_nz(m, a - NX)) acc -= Ju[m * NU + (a - NX)] * (mp[m] + dss * m_[m]);
      }
      if (a < NX && k == L - 1) {
        // compile-time indices into the parameter struct (a run-time index would copy it to
        // local memory in every thread)
#pragma unroll
        for (int r = 0; r < NEM; ++r)
          if (r < ts.n_e && ts.idx[r] == a) acc += dNu[r];
      }
      if (a < NX) oX[a * P + k] = acc;
      else oU[(a - NX) * P + k] = acc;
    }
#pragma unroll
    for (int m = 0; m < NX; ++m) oL[m * P + k] = dz[m] - (sdev ? s * Bt[m * P + k] : Bt[m * P + k]);
    if (k == L - 1) {
#pragma unroll
      for (int r = 0; r < NEM; ++r)
        oNu[r] = r < ts.n_e ? T(ts.ea[r]) * dX[ts.idx[r] * P + k] + T(ts.ec[r]) * dNu[r] : T(0);
      for (int r = NEM; r < 32; ++r) oNu[r] = T(0);
    }
  }
  if (part) {
    const double tot = block_sum<double>(sacc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
  }
}

// One block: *out = scale * sum of n partials (fixed order).
template <typename T>
__global__ void k_free_finish(const double* __restrict__ part, int n, double scale, T* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  const double t = block_sum<double>(a, red);
  if (threadIdx.x == 0) out[0] = (T)(scale * t);
}

// Border of the KKT preconditioner (free final time). a = the KKT matrix's s column:
// [-(1/s) J_x^T mu ; -(1/s) J_u^T mu ; -B^a f ; 0], mu = s B^aT lambda at the linearisation.
template <typename T, int KIND>
__global__ void k_border(const T* __restrict__ xu, const T* __restrict__ mu, const T* __restrict__ Baf, T inv_s,
                         int64_t P, int64_t L, T pa, T* __restrict__ a) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu, NV = NX + NU;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < 32) a[(NV + NX) * P + k] = T(0);
    if (k >= L) {
#pragma unroll
      for (int m = 0; m < NV + NX; ++m) a[m * P + k] = T(0);
      continue;
    }
    T x[NXM], u[NUM], m_[NXM], Jx[NXM * NXM], Ju[NXM * NUM];
#pragma unroll
    for (int m = 0; m < NX; ++m) { x[m] = xu[m * P + k]; m_[m] = mu[m * P + k]; }
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = xu[(NX + q) * P + k];
    Dyn<KIND>::template jac<T>(x, u, Jx, Ju, pa);
#pragma unroll
    for (int p = 0; p < NX; ++p) {
      T g = T(0);
#pragma unroll
      for (int m = 0; m < NX; ++m)
        if (Dyn<KIND>::jx_nz(m, p)) g -= Jx[m * NX + p] * m_[m];
      a[p * P + k] = g * inv_s;
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      T g = T(0);
#pragma unroll
      for (int m = 0; m < NX; ++m)
        if (Dyn<KIND>::ju_nz(m, q)) g -= Ju[m * NU + q] * m_[m];
      a[(NX + q) * P + k] = g * inv_s;
    }
#pragma unroll
    for (int m = 0; m < NX; ++m) a[(NV + m) * P + k] = -Baf[m * P + k];
  }
}

// f at the linearisation point, working type (padding left unwritten: products ignore it).
template <typename T, int KIND>
__global__ void k_fT(const T* __restrict__ xu, int64_t P, int64_t L, T pa, T* __restrict__ f) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    T x[NXM], u[NUM], fx[NXM];
#pragma unroll
    for (int m = 0; m < NX; ++m) x[m] = xu[m * P + k];
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = xu[(NX + q) * P + k];
    Dyn<KIND>::template f<T>(x, u, fx, pa);
#pragma unroll
    for (int m = 0; m < NX; ++m) f[m * P + k] = fx[m];
  }
}

// Partials of x . y over n elements (FP64 accumulation), one per block.
template <typename T>
__global__ void k_dot_part(const T* __restrict__ x, const T* __restrict__ y, int64_t n, double* __restrict__ part) {
  __shared__ double red[32];
  double a = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a += (double)x[i] * (double)y[i];
  const double t = block_sum<double>(a, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// gam[0] = 1 / sum(part) (the border's a . q), one block.
__global__ void k_border_gamma(const double* __restrict__ part, int n, double* __restrict__ gam) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  const double t = block_sum<double>(a, red);
  if (threadIdx.x == 0) gam[0] = 1.0 / t;
}

// Bordered solve, step 2 (one block): ds = (a . t - r_s) / (a . q) into gam[1].
template <typename T>
__global__ void k_border_ds(const double* __restrict__ part, int n, const T* __restrict__ rs, double* __restrict__ gam) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += part[i];
  const double t = block_sum<double>(a, red);
  if (threadIdx.x == 0) gam[1] = (t - (double)rs[0]) * gam[0];
}

// Bordered solve, step 3: y = t - ds q, y_s = ds.
template <typename T>
__global__ void k_border_fix(const T* __restrict__ q, const double* __restrict__ gam, int64_t n, int64_t s_idx,
                             T* __restrict__ y) {
  const T ds = (T)gam[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = i == s_idx ? ds : y[i] - ds * q[i];
}

// ---------------------------------------------------------------------------------------------
// KKT preconditioner elementwise kernels
// ---------------------------------------------------------------------------------------------
// yu_q = (r_u,q + s sum_m Ju[m][q] b_m) / (s w_k cost_uu);  g_m = sum_q Ju[m][q] yu_q
template <typename T, int KIND>
__global__ void k_pre_u(const T* __restrict__ xu, const T* __restrict__ w, T s, T cost_uu, const T* __restrict__ ru,
                        const T* __restrict__ b, int64_t P, int64_t L, T* __restrict__ yu, T* __restrict__ g,
                        T gsign, const T* __restrict__ mu, T pa, const double* __restrict__ sdev,
                        const T* __restrict__ hbar) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  if (sdev) s = T(*sdev);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    if (k >= L) {
#pragma unroll
      for (int q = 0; q < NU; ++q) yu[q * P + k] = T(0);
#pragma unroll
      for (int m = 0; m < NX; ++m) g[m * P + k] = T(0);
      continue;
    }
    T x[NXM], u[NUM], Jx[NXM * NXM], Ju[NXM * NUM], y[NUM];
#pragma unroll
    for (int m = 0; m < NX; ++m) x[m] = xu[m * P + k];
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = xu[(NX + q) * P + k];
    Dyn<KIND>::template jac<T>(x, u, Jx, Ju, pa);
    T mk[NXM];
#pragma unroll
    for (int m = 0; m < NX; ++m) mk[m] = Dyn<KIND>::huu_needs_mu ? mu[m * P + k] : T(0);
    const T huu = Dyn<KIND>::template pre_huu<T>(mk, s * w[k] * cost_uu, pa);
    // control bounds: the barrier's diagonal joins the (diagonal) control block, one inverse per
    // control (for two controls from one division: 1/h0 = h1 r, 1/h1 = h0 r, r = 1/(h0 h1))
    T inv[NUM];
    if (hbar) {
      T hq[NUM];
#pragma unroll
      for (int q = 0; q < NU; ++q) hq[q] = huu + hbar[q * P + k];
      if constexpr (NU == 2) {
        const T r = T(1) / (hq[0] * hq[1]);
        inv[0] = hq[1] * r;
        inv[1] = hq[0] * r;
      } else {
#pragma unroll
        for (int q = 0; q < NU; ++q) inv[q] = T(1) / hq[q];
      }
    } else {
      const T i0 = T(1) / huu;
#pragma unroll
      for (int q = 0; q < NU; ++q) inv[q] = i0;
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      T a = ru ? ru[q * P + k] : T(0);
#pragma unroll
      for (int m = 0; m < NX; ++m)
        if (Dyn<KIND>::ju_nz(m, q)) a += s * Ju[m * NU + q] * b[m * P + k];
      y[q] = a * inv[q];
      yu[q * P + k] = y[q];
    }
#pragma unroll
    for (int m = 0; m < NX; ++m) {
      T a = T(0);
#pragma unroll
      for (int q = 0; q < NU; ++q)
        if (Dyn<KIND>::ju_nz(m, q)) a += Ju[m * NU + q] * y[q];
      g[m * P + k] = gsign * a;
    }
  }
}

// y_nu = S^{-1} (q[term, N] - r_nu)   (one thread)
template <typename T>
__global__ void k_pre_nu(const T* __restrict__ q, const T* __restrict__ rnu, const T* __restrict__ Sinv, int64_t P,
                         int64_t L, TermSpec ts, T* __restrict__ ynu) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  T rhs[NEM];
  for (int r = 0; r < ts.n_e; ++r) rhs[r] = T(ts.ea[r]) * q[ts.idx[r] * P + (L - 1)] - rnu[r];
  for (int r = 0; r < 32; ++r) {
    T a = T(0);
    if (r < ts.n_e)
      for (int c = 0; c < ts.n_e; ++c) a += Sinv[r * ts.n_e + c] * rhs[c];
    ynu[r] = a;
  }
}

// y_u += HW y_nu; y_x -= Q y_nu; y_lambda -= Z y_nu
template <typename T, int NX, int NU>
__global__ void k_pre_fix(const T* __restrict__ Zc, const T* __restrict__ HWc, const T* __restrict__ Qc,
                          const T* __restrict__ ynu, int n_e, int64_t P, int64_t L, T* __restrict__ yx,
                          T* __restrict__ yu, T* __restrict__ yl) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    // the node's outputs stay in registers over the n_e columns (one read and one write each)
    T ax[NX], al[NX], au[NU];
#pragma unroll
    for (int m = 0; m < NX; ++m) { ax[m] = yx[m * P + k]; al[m] = yl[m * P + k]; }
#pragma unroll
    for (int q = 0; q < NU; ++q) au[q] = yu[q * P + k];
    for (int r = 0; r < n_e; ++r) {
      const T c = ynu[r];
#pragma unroll
      for (int m = 0; m < NX; ++m) {
        ax[m] -= c * Qc[((int64_t)r * NX + m) * P + k];
        al[m] -= c * Zc[((int64_t)r * NX + m) * P + k];
      }
#pragma unroll
      for (int q = 0; q < NU; ++q) au[q] += c * HWc[((int64_t)r * NU + q) * P + k];
    }
#pragma unroll
    for (int m = 0; m < NX; ++m) { yx[m * P + k] = ax[m]; yl[m * P + k] = al[m]; }
#pragma unroll
    for (int q = 0; q < NU; ++q) yu[q * P + k] = au[q];
  }
}

template <typename T>
__global__ void k_unit(T* v, int64_t n, int64_t idx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = i == idx ? T(1) : T(0);
}

// ---------------------------------------------------------------------------------------------
// Residual kernels (FP64)
// ---------------------------------------------------------------------------------------------
template <int KIND>
__global__ void k_feval(const double* __restrict__ z, int64_t P, int64_t L, double* __restrict__ fout, double pa) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    if (k >= L) {
#pragma unroll
      for (int m = 0; m < NX; ++m) fout[m * P + k] = 0.0;
      continue;
    }
    double x[NXM], u[NUM], f[NXM];
#pragma unroll
    for (int m = 0; m < NX; ++m) x[m] = z[m * P + k];
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = z[(NX + q) * P + k];
    Dyn<KIND>::template f<double>(x, u, f, pa);
#pragma unroll
    for (int m = 0; m < NX; ++m) fout[m * P + k] = f[m];
  }
}

struct X0Spec {
  double x0[NXM];
};

// F = [grad_X L ; grad_U L ; c ; e] and per-block partial sums of the weighted norm.
template <int KIND>
__global__ void k_resid_post(const double* __restrict__ z, const double* __restrict__ w, double s,
                             const double* __restrict__ Bf, const double* __restrict__ Mu, int64_t P, int64_t L,
                             TermSpec ts, X0Spec x0, double cost_uu, double* __restrict__ F,
                             double* __restrict__ partial, double pa, double* __restrict__ partial2, BarSpec bs) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu, NV = NX + NU;
  __shared__ double red[32];
  const double* X = z;
  const double* U = z + NX * P;
  const double* lam = z + NV * P;
  const double* nu = z + (NV + NX) * P;
  double acc = 0.0, acc2 = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    if (k >= L) {
#pragma unroll
      for (int m = 0; m < NV + NX; ++m) F[m * P + k] = 0.0;
      continue;
    }
    double x[NXM], u[NUM], Jx[NXM * NXM], Ju[NXM * NUM], mp[NXM];
#pragma unroll
    for (int m = 0; m < NX; ++m) { x[m] = X[m * P + k]; mp[m] = Mu[m * P + k]; }
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = U[q * P + k];
    Dyn<KIND>::template jac<double>(x, u, Jx, Ju, pa);
    const double wk = w[k];
    const double iw = 1.0 / wk;
#pragma unroll
    for (int p = 0; p < NX; ++p) {
      double g = lam[p * P + k];
#pragma unroll
      for (int m = 0; m < NX; ++m)
        if (Dyn<KIND>::jx_nz(m, p)) g -= Jx[m * NX + p] * mp[m];
      if (k == L - 1) {
#pragma unroll
        for (int r = 0; r < NEM; ++r)
          if (r < ts.n_e && ts.idx[r] == p) g += nu[r];
      }
      F[p * P + k] = g;
      acc += g * g * iw;
    }
    // control bounds: the primal barrier gradient, or (primal-dual form) -z_l + z_h with the
    // complementarity residuals C = (distance to the bound) z - mu s w in the norm (weight 1 / w)
    double gb[NUM], hb[NUM];
    if (bs.z) {
#pragma unroll
      for (int q = 0; q < NU; ++q) {
        gb[q] = 0.0;
        if (bs.mu > 0.0 && bs.has_lo[q]) {
          const double zl = bs.z[q * P + k];
          const double c = (u[q] - bs.lo[q]) * zl - bs.mu * s * wk;
          gb[q] -= zl;
          acc += c * c * iw;
        }
        if (bs.mu > 0.0 && bs.has_hi[q]) {
          const double zh = bs.z[(NU + q) * P + k];
          const double c = (bs.hi[q] - u[q]) * zh - bs.mu * s * wk;
          gb[q] += zh;
          acc += c * c * iw;
        }
      }
    } else {
      bar_terms<double, NU>(bs, u, s * wk, gb, hb);
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) {
      double g = s * wk * cost_uu * u[q] + gb[q];
#pragma unroll
      for (int m = 0; m < NX; ++m)
        if (Dyn<KIND>::ju_nz(m, q)) g -= Ju[m * NU + q] * mp[m];
      F[(NX + q) * P + k] = g;
      acc += g * g * iw;
    }
#pragma unroll
    for (int m = 0; m < NX; ++m) {
      const double c = x[m] - x0.x0[m] - Bf[m * P + k];
      F[(NV + m) * P + k] = c;
      acc += wk * c * c;
      if (partial2) acc2 += lam[m * P + k] * Bf[m * P + k];
    }
    if (k == L - 1) {
#pragma unroll
      for (int r = 0; r < NEM; ++r) {
        double xr = 0.0;   // x[ts.idx[r]] by selects: x stays in registers
#pragma unroll
        for (int m = 0; m < NX; ++m) xr = ts.idx[r] == m ? x[m] : xr;
        double e = r < ts.n_e ? xr - ts.val[r] : 0.0;
        if (r < ts.n_e && ts.eb[r]) {   // endpoint bound: c(x) nu_r - mu m(x)
          double c, dc, m;
          end_cm(ts, r, xr, &c, &dc, &m);
          e = c * nu[r] - ts.mu * m;
        }
        F[(NV + NX) * P + r] = e;
        acc += e * e;
      }
      for (int r = NEM; r < 32; ++r) F[(NV + NX) * P + r] = 0.0;
    }
  }
  double tot = block_sum<double>(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
  if (partial2) {
    tot = block_sum<double>(acc2, red);
    if (threadIdx.x == 0) partial2[blockIdx.x] = tot;
  }
}

// Free final time (one block): g_s = 2 - (1/s) sum lambda . Bf (Bf = s B^a f) into F_s, and the
// squared weighted norm sum(partial) + g_s^2 into out.
__global__ void k_resid_free(const double* __restrict__ partial, const double* __restrict__ partial2, int n,
                             double inv_s, double* __restrict__ Fs, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) { a += partial[i]; b += partial2[i]; }
  const double ta = block_sum<double>(a, red);
  const double tb = block_sum<double>(b, red);
  if (threadIdx.x == 0) {
    const double gs = 2.0 - inv_s * tb;
    Fs[0] = gs;
    out[0] = ta + gs * gs;
  }
}

// Weighted norm partials of an arbitrary FP64 residual vector.
template <int NX, int NU>
__global__ void k_wnorm(const double* __restrict__ F, const double* __restrict__ w, int64_t P, int64_t L, int n_e,
                        double* __restrict__ partial) {
  constexpr int NV = NX + NU;
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
    const double wk = w[k], iw = 1.0 / wk;
#pragma unroll
    for (int m = 0; m < NV; ++m) { const double g = F[m * P + k]; acc += g * g * iw; }
#pragma unroll
    for (int m = 0; m < NX; ++m) { const double c = F[(NV + m) * P + k]; acc += wk * c * c; }
    if (k == L - 1)
      for (int r = 0; r < n_e; ++r) { const double e = F[(NV + NX) * P + r]; acc += e * e; }
  }
  double tot = block_sum<double>(acc, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void k_sum_partials(const double* __restrict__ partial, int n, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a += partial[i];
  double t = block_sum<double>(a, red);
  if (threadIdx.x == 0) out[0] = t;
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------

template <int KIND> struct KindNX { static constexpr int nx = Dyn<KIND>::nx, nu = Dyn<KIND>::nu; };

#define BK_DISPATCH_KIND(kind, FN, ...)                                   \
  switch (kind) {                                                         \
    case BK_DBL_INT: return FN<BK_DBL_INT>(__VA_ARGS__);                  \
    case BK_ORBIT: return FN<BK_ORBIT>(__VA_ARGS__);                      \
    case BK_BILINEAR: return FN<BK_BILINEAR>(__VA_ARGS__);                \
    case BK_ORBIT_MT: return FN<BK_ORBIT_MT>(__VA_ARGS__);                \
    default: set_error("unknown problem kind"); return BK_ERR_ARG;        \
  }

static bk_status alloc_opdata(Problem* pr, OpData& d, int dtype) {
  d.dtype = dtype;
  BK_TRY(dtype == BK_F64 ? sweep_attrs_nx<double>(pr->n_x) : sweep_attrs_nx<float>(pr->n_x));
  const size_t es = dtype_size(dtype);
  const int64_t P = pr->P;
  const int nx = pr->n_x, nu = pr->n_u, ne = pr->n_e;
  BK_TRY(plan_create(&d.plan, pr->N, nx, 1, dtype, pr->t0, pr->tf, P, 0));
  pr->bytes += d.plan->bytes;  // the plan counted its own allocations
  BK_TRY(dmalloc(&d.xu, es * (nx + nu) * P));
  BK_TRY(dmalloc(&d.mu, es * nx * P));
  d.w = dtype == BK_F64 ? (void*)d.plan->w64 : d.plan->wT;
  // preconditioner data only in the working precision (an FP32 problem's FP64 side serves the
  // residual and the refinement products)
  const bool pre = dtype == pr->pdtype;
  const int64_t il = (int64_t)round_up(pr->nseg, 32) * seg_nodes(pr->pdtype) * nx * nx;
  if (pre) {
    BK_TRY(dmalloc(&d.Dn, es * il));   // the node deviations D (K = I + D, N = 2 D)
  }
  for (int l = 0; pre && l < pr->nlev; ++l) {
    const size_t npad = (size_t)round_up(pr->lvn[l], 32);
    BK_TRY(dmalloc(&d.lvm[l], es * NSLOT * npad * nx * nx));
    BK_TRY(dmalloc(&d.lve[l], es * npad * nx));
    if (l > 0) BK_TRY(dmalloc(&d.lvo[l], es * npad * nx));
  }
  if (pre && pr->free_time) {
    BK_TRY(dmalloc(&d.brd, es * pr->kkt_len()));
    BK_TRY(dmalloc(&d.brq, es * pr->kkt_len()));
    BK_TRY(dmalloc((void**)&d.bgam, sizeof(double) * 2));
  }
  if (pre && ne > 0) {
    BK_TRY(dmalloc(&d.Zc, es * ne * nx * P));
    BK_TRY(dmalloc(&d.HWc, es * ne * nu * P));
    BK_TRY(dmalloc(&d.Qc, es * ne * nx * P));
    BK_TRY(dmalloc(&d.Sinv, es * NEM * NEM));
  }
  BK_TRY(dmalloc(&d.t1, es * (nx + nu) * P));
  BK_TRY(dmalloc(&d.t2, es * (nx + nu) * P));
  BK_TRY(dmalloc(&d.t3, es * (nx + nu) * P));
  return BK_OK;
}

static void free_opdata(OpData& d) {
  if (d.plan) plan_destroy(d.plan);
  void* ps[] = {d.xu, d.mu, d.Dn, d.Zc, d.HWc, d.Qc, d.Sinv, d.t1, d.t2, d.t3, d.brd, d.brq, d.bgam, d.hbar};
  for (void* p : ps) dfree(p);
  for (int l = 0; l < MAXLEV; ++l) {
    dfree(d.lvm[l]);
    dfree(d.lvo[l]);
    dfree(d.lve[l]);
  }
  d = OpData();
}

// --- linearisation ---------------------------------------------------------------------------
// Control bounds: the barrier's diagonal of the control block at z_lin. Primal-dual form (b.z):
// Sigma = z_l / (u - l) + z_h / (h - u), the multipliers' elimination; primal form: the barrier
// Hessian mu s w (1 / (u - l)^2 + 1 / (h - u)^2).
template <typename T, int NU>
__global__ void k_lin_bar(const double* __restrict__ z, const double* __restrict__ w, double s, int64_t P, int64_t L,
                          int nx, BarSpec b, T* __restrict__ hbar) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
    if (k >= L) {
#pragma unroll
      for (int q = 0; q < NU; ++q) hbar[q * P + k] = T(0);
      continue;
    }
    double u[NUM], g[NUM], h[NUM];
#pragma unroll
    for (int q = 0; q < NU; ++q) u[q] = z[(nx + q) * P + k];
    if (b.z) {
#pragma unroll
      for (int q = 0; q < NU; ++q) {
        h[q] = 0.0;
        if (b.has_lo[q]) h[q] += b.z[q * P + k] / (u[q] - b.lo[q]);
        if (b.has_hi[q]) h[q] += b.z[(NU + q) * P + k] / (b.hi[q] - u[q]);
      }
    } else {
      bar_terms<double, NU>(b, u, s * w[k], g, h);
    }
#pragma unroll
    for (int q = 0; q < NU; ++q) hbar[q * P + k] = (T)h[q];
  }
}

// The barrier diagonal of one precision's data, null when the problem has no active bounds.
template <typename T>
static const T* bar_hbar(const Problem* pr, const OpData& d) {
  return pr->has_ubounds && pr->bar_mu > 0.0 ? (const T*)d.hbar : nullptr;
}

// Segment maps and scan levels from the node factors N_k (level data of the sweeps).
template <typename T, int NX>
static bk_status lin_levels(Problem* pr, OpData& d, cudaStream_t st) {
  k_lin_seg<T, NX><<<(pr->nseg + 127) / 128, 128, 0, st>>>((const T*)d.Dn, pr->L, pr->nseg, (T*)d.lvm[0]);
  BK_CHECK_LAUNCH();
  for (int l = 0; l < pr->nlev; ++l) {
    k_lin_level<T, NX><<<(pr->lvn[l] + 31) / 32, 32, 0, st>>>((T*)d.lvm[l], pr->lvn[l],
                                                              l + 1 < pr->nlev ? (T*)d.lvm[l + 1] : nullptr);
    BK_CHECK_LAUNCH();
  }
  return BK_OK;
}

template <typename T, int KIND>
static bk_status lin_factors(Problem* pr, OpData& d, const double* z, cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  k_lin_nodes<T, KIND, NX, NU><<<nblk(pr->L), 256, 0, st>>>(z, pr->P, pr->L, pr->d64.plan->w64, pr->s, (T*)d.Dn, (T*)d.xu,
                                                             pr->dyn_param());
  BK_CHECK_LAUNCH();
  return lin_levels<T, NX>(pr, d, st);
}

template <typename T>
__global__ void k_negate(T* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] = -v[i];
}

// Terminal Schur data of the KKT preconditioner (see precond_kkt): the launches, ending with the
// n_e x n_e entries of S copied into pinned host memory (lin_schur_finish inverts S).
template <typename T, int KIND>
static bk_status lin_schur_launch(Problem* pr, OpData& d, cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  const int ne = pr->n_e;
  if (ne == 0 || !pr->has_cost) return BK_OK;
  const int64_t P = pr->P, L = pr->L;
  const T s = (T)pr->s;
  T* Zc = (T*)d.Zc;
  T* HWc = (T*)d.HWc;
  T* Qc = (T*)d.Qc;
  T* unit = (T*)d.t1;   // n_x * P
  T* bz = (T*)d.t2;     // n_x * P : B-tilde^T Z_r
  T* g = (T*)d.t3;      // n_x * P : forcing
  for (int r = 0; r < ne; ++r) {
    k_unit<T><<<nblk(NX * P), 256, 0, st>>>(unit, NX * P, (int64_t)pr->term_idx[r] * P + (L - 1));
    BK_CHECK_LAUNCH();
    T* Z = Zc + (int64_t)r * NX * P;
    BK_TRY((run_sweep<T, NX, 1>(pr, d, unit, nullptr, Z, bz, st)));
    // W = Pu^T Z = -s Ju^T (B-tilde^T Z). k_pre_u with r_u = 0 and b = B-tilde^T Z gives
    // yu = s Ju^T b / (s w) = -H~^{-1} W and g = Ju yu = -Ju H~^{-1} W.
    T* HW = HWc + (int64_t)r * NU * P;
    k_pre_u<T, KIND><<<nblk(P), 256, 0, st>>>((const T*)d.xu, (const T*)d.w, s, (T)1, nullptr, bz, P, L, HW, g, T(1),
                                              (const T*)d.mu, (T)pr->dyn_param(), nullptr, bar_hbar<T>(pr, d));
    BK_CHECK_LAUNCH();
    // Q = P^{-1} Pu HW: forward sweep with Y = 0 and forcing -Ju HW = Ju (-HW) = g
    k_unit<T><<<nblk(NX * P), 256, 0, st>>>(unit, NX * P, -1);
    BK_CHECK_LAUNCH();
    T* Q = Qc + (int64_t)r * NX * P;
    BK_TRY((run_sweep<T, NX, 0>(pr, d, unit, g, Q, nullptr, st)));
  }
  // HWc holds -H~^{-1} W: negate it
  k_negate<T><<<nblk((int64_t)ne * NU * P), 256, 0, st>>>(HWc, (int64_t)ne * NU * P);
  BK_CHECK_LAUNCH();
  // S = E Q: S[r][c] = Q_c[term_idx[r]][N], into pinned host memory
  T* hq = reinterpret_cast<T*>(pr->red_host + 256);
  for (int c = 0; c < ne; ++c)
    for (int r = 0; r < ne; ++r)
      BK_TRY_CUDA(cudaMemcpyAsync(&hq[r * ne + c], Qc + ((int64_t)c * NX + pr->term_idx[r]) * P + (L - 1), sizeof(T),
                                  cudaMemcpyDeviceToHost, st));
  return BK_OK;
}

template <typename T>
static bk_status lin_schur_finish(Problem* pr, OpData& d, cudaStream_t st) {
  const int ne = pr->n_e;
  std::vector<double> S(ne * ne);
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  const T* hq = reinterpret_cast<const T*>(pr->red_host + 256);
  for (int i = 0; i < ne * ne; ++i) S[i] = (double)hq[i];
  // endpoint bounds: rows ea_r (E x)_r + ec_r nu_r = r_r give (diag(ea) E Q - diag(ec)) nu =
  // diag(ea) E x0 - r (k_pre_nu scales its E x0 by ea)
  for (int r = 0; r < ne; ++r) {
    if (!(pr->has_ebounds && pr->term_bnd[r])) continue;
    for (int c = 0; c < ne; ++c) S[r * ne + c] *= pr->term_ea[r];
    S[r * ne + r] -= pr->term_ec[r];
  }
  // invert S (n_e <= 4) by Gauss-Jordan with partial pivoting in FP64
  std::vector<double> A(S), Inv(ne * ne, 0.0);
  for (int i = 0; i < ne; ++i) Inv[i * ne + i] = 1.0;
  for (int c = 0; c < ne; ++c) {
    int piv = c;
    for (int r = c + 1; r < ne; ++r)
      if (fabs(A[r * ne + c]) > fabs(A[piv * ne + c])) piv = r;
    if (A[piv * ne + c] == 0.0) { set_error("terminal Schur complement is singular"); return BK_ERR_INFEASIBLE; }
    for (int q = 0; q < ne; ++q) { std::swap(A[c * ne + q], A[piv * ne + q]); std::swap(Inv[c * ne + q], Inv[piv * ne + q]); }
    const double ip = 1.0 / A[c * ne + c];
    for (int q = 0; q < ne; ++q) { A[c * ne + q] *= ip; Inv[c * ne + q] *= ip; }
    for (int r = 0; r < ne; ++r) {
      if (r == c) continue;
      const double f = A[r * ne + c];
      for (int q = 0; q < ne; ++q) { A[r * ne + q] -= f * A[c * ne + q]; Inv[r * ne + q] -= f * Inv[c * ne + q]; }
    }
  }
  std::vector<T> hs(NEM * NEM, T(0));
  for (int i = 0; i < ne * ne; ++i) hs[i] = (T)Inv[i];
  BK_TRY_CUDA(cudaMemcpyAsync(d.Sinv, hs.data(), sizeof(T) * ne * ne, cudaMemcpyHostToDevice, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  return BK_OK;
}

template <typename T, int KIND>
static bk_status lin_border(Problem* pr, OpData& d, cudaStream_t st);

// x_{idx_r}(t_f) and nu_r of a KKT vector (one thread)
__global__ void k_term_vals(const double* __restrict__ z, int64_t P, int64_t L, int64_t nu_off, TermSpec ts,
                            double* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int r = 0; r < ts.n_e; ++r) {
    out[r] = z[ts.idx[r] * P + (L - 1)];
    out[NEM + r] = z[nu_off + r];
  }
}

// Endpoint bounds: the Newton rows ea_r dx + ec_r dnu_r of the barrier rows at z_lin,
// ea = c'(x) nu, ec = c(x) (synchronous).
static bk_status lin_end_rows(Problem* pr, const double* z, cudaStream_t st) {
  const TermSpec ts = term_spec(pr);
  double* dv = pr->red + 1800;
  double* hv = pr->red_host + 320;
  k_term_vals<<<1, 32, 0, st>>>(z, pr->P, pr->L, (int64_t)(2 * pr->n_x + pr->n_u) * pr->P, ts, dv);
  BK_CHECK_LAUNCH();
  BK_TRY_CUDA(cudaMemcpyAsync(hv, dv, sizeof(double) * 2 * NEM, cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  for (int r = 0; r < pr->n_e; ++r) {
    pr->term_ea[r] = 1.0;
    pr->term_ec[r] = 0.0;
    if (!ts.eb[r]) continue;
    double c, dc, m;
    end_cm(ts, r, hv[r], &c, &dc, &m);
    if (!(c > 0.0) || !isfinite(c)) {
      set_error("terminal row %d: x(t_f) = %g is not inside its bound", r, hv[r]);
      return BK_ERR_ARG;
    }
    pr->term_ea[r] = dc * hv[NEM + r];
    pr->term_ec[r] = c;
  }
  return BK_OK;
}

// mu (nullable): s B^aT lambda at this z, known to the caller (e.g. from the residual that
// accepted the step); it is copied instead of recomputed.
// A BK_F32 problem builds its preconditioner data in FP32 only; the FP64 side keeps the
// linearisation point and mu, which the FP64 KKT product needs.
template <int KIND>
static bk_status linearize_kind(Problem* pr, const double* z, const double* mu, int keep, cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  const int64_t P = pr->P;
  if (!pr->linearized || pr->free_time) keep = LIN_FULL;
  if (pr->has_ebounds) {   // the terminal Schur complement carries the barrier rows' diagonal
    keep = LIN_FULL;
    BK_TRY(lin_end_rows(pr, z, st));
  }
  if (mu)
    BK_TRY_CUDA(cudaMemcpyAsync(pr->d64.mu, mu, sizeof(double) * NX * P, cudaMemcpyDeviceToDevice, st));
  else
    BK_TRY(plan_apply_n(pr->d64.plan, z + (NX + NU) * P, pr->d64.mu, NX, true, pr->s, st));
  if (pr->pdtype == BK_F64 && keep != LIN_KEEP_PRECOND)
    BK_TRY((lin_factors<double, KIND>(pr, pr->d64, z, st)));
  else
    BK_TRY_CUDA(cudaMemcpyAsync(pr->d64.xu, z, sizeof(double) * (NX + NU) * P, cudaMemcpyDeviceToDevice, st));
  if (pr->d32.plan) {
    k_convert<double, float><<<nblk(NX * P), 256, 0, st>>>((const double*)pr->d64.mu, (float*)pr->d32.mu, NX * P);
    BK_CHECK_LAUNCH();
    if (keep != LIN_KEEP_PRECOND) {
      BK_TRY((lin_factors<float, KIND>(pr, pr->d32, z, st)));
    } else {
      k_convert<double, float><<<nblk((NX + NU) * P), 256, 0, st>>>(z, (float*)pr->d32.xu, (NX + NU) * P);
      BK_CHECK_LAUNCH();
    }
  }
  if (pr->has_ubounds && pr->bar_mu > 0.0) {
    const BarSpec b = bar_spec(pr);
    k_lin_bar<double, NU><<<nblk(P), 256, 0, st>>>(z, pr->d64.plan->w64, pr->s, P, pr->L, NX, b, (double*)pr->d64.hbar);
    BK_CHECK_LAUNCH();
    if (pr->d32.plan) {
      k_lin_bar<float, NU><<<nblk(P), 256, 0, st>>>(z, pr->d64.plan->w64, pr->s, P, pr->L, NX, b, (float*)pr->d32.hbar);
      BK_CHECK_LAUNCH();
    }
  }
  pr->linearized = true;
  if (keep != LIN_FULL) return BK_OK;
  if (pr->n_e > 0 && pr->has_cost) {
    OpData& d = pr->pre();
    BK_TRY((d.dtype == BK_F64 ? lin_schur_launch<double, KIND>(pr, d, st) : lin_schur_launch<float, KIND>(pr, d, st)));
    BK_TRY(d.dtype == BK_F64 ? lin_schur_finish<double>(pr, d, st) : lin_schur_finish<float>(pr, d, st));
  }
  if (pr->free_time) {
    OpData& d = pr->pre();
    BK_TRY((d.dtype == BK_F64 ? lin_border<double, KIND>(pr, d, st) : lin_border<float, KIND>(pr, d, st)));
  }
  return BK_OK;
}

bk_status problem_linearize(Problem* pr, const double* z, cudaStream_t st, const double* mu, int keep) {
  BK_ARG(pr != nullptr && z != nullptr, "NULL problem or z_lin");
  BK_DISPATCH_KIND(pr->kind, linearize_kind, pr, z, mu, keep, st);
}

// --- operator applies --------------------------------------------------------------------------
template <typename T, int KIND>
static bk_status apply_typed(Problem* pr, OpData& d, int op, const T* in, T* out, T* mu_out, cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  const int64_t P = pr->P, L = pr->L;
  T* t1 = (T*)d.t1;
  T* t2 = (T*)d.t2;
  T* t3 = (T*)d.t3;
  if (op == BK_OP_STATE) {
    // the product ignores t1's padding (elements L..P-1), so it is never written
    k_jvp<T, KIND><<<nblk(L), 256, 0, st>>>((const T*)d.xu, in, nullptr, P, L, t1, (T)pr->dyn_param(), nullptr, T(0));
    BK_CHECK_LAUNCH();
    const double* sd = sdev_of(pr);
    BK_TRY(plan_apply_n(d.plan, t1, t2, NX, false, sd ? 1.0 : pr->s, st));
    k_state_post<T, NX><<<nblk(NX * P), 256, 0, st>>>(in, t2, P, L, out, sd);
    BK_CHECK_LAUNCH();
    return BK_OK;
  }
  const bool ft = pr->free_time;
  const T pa = (T)pr->dyn_param();
  k_jvp<T, KIND><<<nblk(L), 256, 0, st>>>((const T*)d.xu, in, in + NX * P, P, L, t1, pa,
                                          ft ? in + pr->s_idx() : nullptr, (T)(1.0 / pr->s));
  BK_CHECK_LAUNCH();
  // fixed final time: both products unscaled, k_kkt_post applies s from the device (so that a
  // captured GMRES step does not hold s); free final time: s (which changes within a step) by value
  const double* sd = sdev_of(pr);
  BK_TRY(plan_apply_n(d.plan, t1, t2, NX, false, sd ? 1.0 : pr->s, st));
  T* Mu = mu_out ? mu_out : t3;
  BK_TRY(plan_apply_n(d.plan, in + (NX + NU) * P, Mu, NX, true, sd ? 1.0 : pr->s, st));
  k_kkt_post<T, KIND><<<ft ? FT_NB : nblk(P), 256, 0, st>>>((const T*)d.xu, (const T*)d.mu, (const T*)d.w, (T)pr->s, in,
                                                            t2, Mu, P, L, term_spec(pr), (T)pr->cost_uu(), out, pa,
                                                            pr->s_idx(), ft ? pr->sred : nullptr, sd, bar_hbar<T>(pr, d));
  BK_CHECK_LAUNCH();
  if (ft) {
    k_free_finish<T><<<1, 256, 0, st>>>(pr->sred, FT_NB, -1.0 / pr->s, out + pr->s_idx());
    BK_CHECK_LAUNCH();
  }
  return BK_OK;
}

template <int KIND>
static bk_status apply_kind(Problem* pr, OpData& d, int op, const void* in, void* out, void* mu_out, cudaStream_t st) {
  if (d.dtype == BK_F64) return apply_typed<double, KIND>(pr, d, op, (const double*)in, (double*)out, (double*)mu_out, st);
  return apply_typed<float, KIND>(pr, d, op, (const float*)in, (float*)out, (float*)mu_out, st);
}

static bk_status op_apply_direct(Problem* pr, OpData& d, int op, const void* in, void* out, cudaStream_t st,
                                 void* mu_out) {
  BK_DISPATCH_KIND(pr->kind, apply_kind, pr, d, op, in, out, mu_out, st);
}

bk_status op_apply(Problem* pr, OpData& d, int op, const void* in, void* out, cudaStream_t st, void* mu_out) {
  BK_ARG(pr->linearized, "problem is not linearised (call bk_linearize first)");
  BK_ARG(op == BK_OP_STATE || op == BK_OP_KKT, "unknown operator %d", op);
  return op_apply_direct(pr, d, op, in, out, st, mu_out);
}

// --- preconditioner ---------------------------------------------------------------------------
// K-tilde^{-1} r: t_lambda = P^{-T} r_x (with b = B-tilde^T t_lambda); yu = H~^{-1}(r_u - Pu^T
// t_lambda); q = P^{-1}(r_lambda - Pu yu); y_nu = S^{-1}(E q - r_nu); y_u = yu + H~^{-1} W y_nu;
// y_x = q - Q y_nu; y_lambda = t_lambda - Z y_nu.  (Pu = -s (B-tilde (x) I) J_u, H~ = s w I.)
template <typename T, int KIND>
static bk_status precond_typed(Problem* pr, OpData& d, int op, const T* in, T* out, int transpose, cudaStream_t st,
                               bool border = true) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu, NV = NX + NU;
  const int64_t P = pr->P, L = pr->L;
  if (op == BK_OP_STATE) {
    if (!transpose) return run_sweep<T, NX, 0>(pr, d, in, nullptr, out, nullptr, st);
    return run_sweep<T, NX, 1>(pr, d, in, nullptr, out, nullptr, st);
  }
  BK_ARG(pr->has_cost, "the KKT preconditioner needs a control cost (problem kind has none)");
  const T* rx = in;
  const T* ru = in + NX * P;
  const T* rl = in + NV * P;
  const T* rnu = in + (NV + NX) * P;
  T* yx = out;
  T* yu = out + NX * P;
  T* yl = out + NV * P;
  T* ynu = out + (NV + NX) * P;
  T* b = (T*)d.t1;
  T* g = (T*)d.t2;
  BK_TRY((run_sweep<T, NX, 1>(pr, d, rx, nullptr, yl, b, st)));
  k_pre_u<T, KIND><<<nblk(P), 256, 0, st>>>((const T*)d.xu, (const T*)d.w, (T)pr->s, (T)1, ru, b, P, L, yu, g, T(1),
                                            (const T*)d.mu, (T)pr->dyn_param(), sdev_of(pr), bar_hbar<T>(pr, d));
  BK_CHECK_LAUNCH();
  BK_TRY((run_sweep<T, NX, 0>(pr, d, rl, g, yx, nullptr, st)));
  if (pr->n_e > 0) {
    k_pre_nu<T><<<1, 32, 0, st>>>(yx, rnu, (const T*)d.Sinv, P, L, term_spec(pr), ynu);
    BK_CHECK_LAUNCH();
    k_pre_fix<T, NX, NU><<<nblk(L), 256, 0, st>>>((const T*)d.Zc, (const T*)d.HWc, (const T*)d.Qc, ynu, pr->n_e, P, L, yx, yu, yl);
    BK_CHECK_LAUNCH();
  } else {
    BK_TRY_CUDA(cudaMemsetAsync(ynu, 0, sizeof(T) * 32, st));
  }
  if (pr->free_time && border) {
    // bordered by the s row and column a (zero diagonal): with t = K-tilde^{-1} r (above) and
    // q = K-tilde^{-1} a, ds = (a . t - r_s) / (a . q), y = t - ds q, y_s = ds
    const int64_t n = pr->kkt_len();
    k_dot_part<T><<<FT_NB, 256, 0, st>>>((const T*)d.brd, out, n, pr->sred);
    BK_CHECK_LAUNCH();
    k_border_ds<T><<<1, 256, 0, st>>>(pr->sred, FT_NB, in + pr->s_idx(), d.bgam);
    BK_CHECK_LAUNCH();
    k_border_fix<T><<<nblk(n), 256, 0, st>>>((const T*)d.brq, d.bgam, n, pr->s_idx(), out);
    BK_CHECK_LAUNCH();
  }
  return BK_OK;
}

// Free final time: the border a of the KKT preconditioner (the KKT matrix's s column at the
// linearisation), q = K-tilde^{-1} a and 1 / (a . q).
template <typename T, int KIND>
static bk_status lin_border(Problem* pr, OpData& d, cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx;
  const int64_t P = pr->P, L = pr->L;
  T* f = (T*)d.t1;
  T* Baf = (T*)d.t2;
  k_fT<T, KIND><<<nblk(L), 256, 0, st>>>((const T*)d.xu, P, L, (T)pr->dyn_param(), f);
  BK_CHECK_LAUNCH();
  BK_TRY(plan_apply_n(d.plan, f, Baf, NX, false, 1.0, st));
  k_border<T, KIND><<<nblk(P), 256, 0, st>>>((const T*)d.xu, (const T*)d.mu, Baf, (T)(1.0 / pr->s), P, L,
                                             (T)pr->dyn_param(), (T*)d.brd);
  BK_CHECK_LAUNCH();
  BK_TRY((precond_typed<T, KIND>(pr, d, BK_OP_KKT, (const T*)d.brd, (T*)d.brq, 0, st, false)));
  k_dot_part<T><<<FT_NB, 256, 0, st>>>((const T*)d.brd, (const T*)d.brq, pr->kkt_len(), pr->sred);
  BK_CHECK_LAUNCH();
  k_border_gamma<<<1, 256, 0, st>>>(pr->sred, FT_NB, d.bgam);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

template <int KIND>
static bk_status precond_kind(Problem* pr, OpData& d, int op, const void* in, void* out, int transpose, cudaStream_t st) {
  if (d.dtype == BK_F64) return precond_typed<double, KIND>(pr, d, op, (const double*)in, (double*)out, transpose, st);
  return precond_typed<float, KIND>(pr, d, op, (const float*)in, (float*)out, transpose, st);
}

static bk_status op_precond_direct(Problem* pr, OpData& d, int op, const void* in, void* out, int transpose,
                                   cudaStream_t st) {
  BK_DISPATCH_KIND(pr->kind, precond_kind, pr, d, op, in, out, transpose, st);
}

bk_status op_precond(Problem* pr, OpData& d, int op, const void* in, void* out, int transpose, cudaStream_t st) {
  BK_ARG(pr->linearized, "problem is not linearised (call bk_linearize first)");
  BK_ARG(op == BK_OP_STATE || op == BK_OP_KKT, "unknown operator %d", op);
  if (d.dtype == pr->pdtype) return op_precond_direct(pr, d, op, in, out, transpose, st);
  // FP64 vectors, FP32 preconditioner: round the input, apply in FP32, widen the result
  BK_ARG(d.dtype == BK_F64 && pr->pdtype == BK_F32 && pr->pcin, "preconditioner precision mismatch");
  const int64_t n = op == BK_OP_KKT ? pr->kkt_len() : pr->state_len();
  k_convert<double, float><<<nblk(n), 256, 0, st>>>((const double*)in, (float*)pr->pcin, n);
  BK_CHECK_LAUNCH();
  BK_TRY(op_precond_direct(pr, pr->d32, op, pr->pcin, pr->pcout, transpose, st));
  k_convert<float, double><<<nblk(n), 256, 0, st>>>((const float*)pr->pcout, (double*)out, n);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// --- residual -------------------------------------------------------------------------------
template <int KIND>
static bk_status residual_launch(Problem* pr, const double* z, double* F, bool want_norm, double* Mu, bool mu_given,
                                 cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  const int64_t P = pr->P, L = pr->L;
  OpData& d = pr->d64;
  double* f = (double*)d.t1;
  double* Bf = (double*)d.t2;
  if (!Mu) Mu = (double*)d.t3;
  k_feval<KIND><<<nblk(P), 256, 0, st>>>(z, P, L, f, pr->dyn_param());
  BK_CHECK_LAUNCH();
  BK_TRY(plan_apply_n(d.plan, f, Bf, NX, false, pr->s, st));
  if (!mu_given) BK_TRY(plan_apply_n(d.plan, z + (NX + NU) * P, Mu, NX, true, pr->s, st));
  X0Spec x0;
  for (int m = 0; m < NXM; ++m) x0.x0[m] = pr->x0[m];
  const int nb = 592;
  k_resid_post<KIND><<<nb, 256, 0, st>>>(z, pr->d64.plan->w64, pr->s, Bf, Mu, P, L, term_spec(pr), x0,
                                         pr->cost_uu(), F, pr->red, pr->dyn_param(),
                                         pr->free_time ? pr->sred : nullptr, bar_spec(pr));
  BK_CHECK_LAUNCH();
  if (pr->free_time) {
    // the time gradient g_s goes into F whether or not the norm is wanted
    k_resid_free<<<1, 256, 0, st>>>(pr->red, pr->sred, nb, 1.0 / pr->s, F + pr->s_idx(), pr->red + 1024);
    BK_CHECK_LAUNCH();
    if (want_norm)
      BK_TRY_CUDA(cudaMemcpyAsync(pr->red_host, pr->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, st));
  } else if (want_norm) {
    k_sum_partials<<<1, 256, 0, st>>>(pr->red, nb, pr->red + 1024);
    BK_CHECK_LAUNCH();
    BK_TRY_CUDA(cudaMemcpyAsync(pr->red_host, pr->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, st));
  }
  return BK_OK;
}

template <int KIND>
static bk_status residual_kind(Problem* pr, const double* z, double* F, bool want_norm, double* Mu, bool mu_given,
                               cudaStream_t st) {
  return residual_launch<KIND>(pr, z, F, want_norm, Mu, mu_given, st);
}

static bk_status residual_dispatch(Problem* pr, const double* z, double* F, bool want, double* Mu, bool mu_given,
                                   cudaStream_t st) {
  BK_DISPATCH_KIND(pr->kind, residual_kind, pr, z, F, want, Mu, mu_given, st);
}

bk_status problem_residual(Problem* pr, const double* z, double* F, double* wnorm, cudaStream_t st, double* Mu,
                           bool mu_given) {
  const bool want = wnorm != nullptr;
  BK_TRY(residual_dispatch(pr, z, F, want, Mu, mu_given, st));
  if (wnorm) {
    BK_TRY_CUDA(cudaStreamSynchronize(st));
    *wnorm = sqrt(pr->red_host[0]);
  }
  return BK_OK;
}

template <int KIND>
static bk_status wnorm_kind(Problem* pr, const double* F, double* wnorm, cudaStream_t st) {
  constexpr int NX = Dyn<KIND>::nx, NU = Dyn<KIND>::nu;
  const int nb = 592;
  // the tail holds e and, for a free final time, g_s right after it
  k_wnorm<NX, NU><<<nb, 256, 0, st>>>(F, pr->d64.plan->w64, pr->P, pr->L, pr->n_e + (pr->free_time ? 1 : 0), pr->red);
  BK_CHECK_LAUNCH();
  k_sum_partials<<<1, 256, 0, st>>>(pr->red, nb, pr->red + 1024);
  BK_CHECK_LAUNCH();
  BK_TRY_CUDA(cudaMemcpyAsync(pr->red_host, pr->red + 1024, sizeof(double), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  *wnorm = sqrt(pr->red_host[0]);
  return BK_OK;
}

bk_status problem_wnorm(Problem* pr, const double* F, double* wnorm, cudaStream_t st) {
  BK_DISPATCH_KIND(pr->kind, wnorm_kind, pr, F, wnorm, st);
}

// --- creation ---------------------------------------------------------------------------------
static void problem_free(Problem* pr) {
  if (!pr) return;
  gmres_graphs_free(pr);
  free_opdata(pr->d64);
  free_opdata(pr->d32);
  dfree(pr->F);
  dfree(pr->red);
  dfree(pr->sred);
  dfree(pr->s_dev);
  dfree(pr->pcin);
  dfree(pr->pcout);
  dfree(pr->bar_buf);
  if (pr->red_host) cudaFreeHost(pr->red_host);
  delete pr;
}

// Problem constants (x0, terminal targets, s) from kind, params and [t0, tf]; no allocation.
static bk_status problem_set_params(Problem* pr, const double* params, int nparams, double t0, double tf) {
  BK_ARG(tf > t0 && isfinite(t0) && isfinite(tf), "tf must be > t0 and finite");
  BK_ARG(nparams >= 0 && nparams <= 4 && (nparams == 0 || params), "bad params");
  // captured GMRES graphs read s from the device copy (fixed final time) and no other
  // parameter; a free final time keeps no graphs
  if (pr->kind == BK_ORBIT || pr->kind == BK_ORBIT_MT) {
    BK_ARG(nparams >= 2, "the orbit kinds need params {a, r_f}");
    BK_ARG(params[1] > 0 && isfinite(params[1]), "r_f must be > 0");
    BK_ARG(pr->kind == BK_ORBIT || (params[0] > 0 && isfinite(params[0])), "BK_ORBIT_MT needs a thrust a > 0");
    pr->term_val[0] = params[1];
    pr->term_val[1] = 0.0;
    pr->term_val[2] = 1.0 / sqrt(params[1]);
  } else if (pr->kind == BK_BILINEAR) {
    pr->x0[0] = nparams >= 1 ? params[0] : 1.0;
  }
  for (int i = 0; i < 4; ++i) pr->params[i] = i < nparams ? params[i] : 0.0;
  pr->t0 = t0;
  pr->tf = tf;
  pr->s = 0.5 * (tf - t0);
  pr->linearized = false;
  if (pr->s_dev) BK_TRY_CUDA(cudaMemcpy(pr->s_dev, &pr->s, sizeof(double), cudaMemcpyHostToDevice));
  return BK_OK;
}

// FP64 problems keep an FP64 preconditioner unless asked for an FP32 one: bk_set_f64_precond(1)
// for problems created afterwards, or the environment variable BK_F64_PC32=1 (read at creation).
// The FP32 sweeps are 2-3x faster, but on the orbit solve at N = 2^20 (forcing-term inner
// tolerances down to 1e-12) flexible GMRES needed 19 instead of 11 iterations, and the solve took
// 56.9 instead of 50.5 ms, so FP64 stays the default.
static std::atomic<int> g_f64_pc32{-1};
static bool f64_precond32(int64_t N) {
  (void)N;
  const int m = g_f64_pc32.load();
  if (m >= 0) return m == 1;
  const char* e = getenv("BK_F64_PC32");
  return e && e[0] == '1';
}

static bk_status problem_create(Problem** out, int kind, const double* params, int nparams, int64_t N, int dtype,
                                double t0, double tf, cudaStream_t st) {
  *out = nullptr;
  BK_ARG(kind == BK_DBL_INT || kind == BK_ORBIT || kind == BK_BILINEAR || kind == BK_ORBIT_MT,
         "unknown problem kind %d", kind);
  BK_ARG(dtype == BK_F64 || dtype == BK_F32, "dtype must be BK_F64 or BK_F32");
  // the problem's FP64 plan bounds N (FP32 problems keep one too)
  BK_ARG(plan_n_supported(N, BK_F64), "N must be a power of two in [4, 2^24] or any N in [4, 2^22], got %lld",
         (long long)N);
  BK_ARG(tf > t0, "tf must be > t0");
  BK_ARG(nparams >= 0 && nparams <= 4 && (nparams == 0 || params), "bad params");
  Problem* pr = new Problem();
  pr->kind = kind;
  pr->dtype = dtype;
  pr->N = N;
  pr->L = N + 1;
  pr->P = round_up(N + 1, 32);
  pr->t0 = t0;
  pr->tf = tf;
  pr->s = 0.5 * (tf - t0);
  for (int i = 0; i < nparams; ++i) pr->params[i] = params[i];
  if (kind == BK_DBL_INT) {
    pr->n_x = 2; pr->n_u = 1; pr->n_e = 2;
    pr->x0[0] = 0; pr->x0[1] = 0;
    pr->term_idx[0] = 0; pr->term_val[0] = 1.0;
    pr->term_idx[1] = 1; pr->term_val[1] = 0.0;
    pr->has_cost = true;
  } else if (kind == BK_ORBIT || kind == BK_ORBIT_MT) {
    if (nparams < 2) { delete pr; set_error("the orbit kinds need params {a, r_f}"); return BK_ERR_ARG; }
    const double rf = params[1];
    if (!(rf > 0)) { delete pr; set_error("r_f must be > 0"); return BK_ERR_ARG; }
    if (kind == BK_ORBIT_MT && !(params[0] > 0 && isfinite(params[0]))) {
      delete pr;
      set_error("BK_ORBIT_MT needs a thrust a > 0");
      return BK_ERR_ARG;
    }
    pr->n_x = 4; pr->n_u = kind == BK_ORBIT ? 2 : 1; pr->n_e = 3;
    pr->free_time = kind == BK_ORBIT_MT;
    pr->x0[0] = 1; pr->x0[1] = 0; pr->x0[2] = 0; pr->x0[3] = 1;
    pr->term_idx[0] = 0; pr->term_val[0] = rf;
    pr->term_idx[1] = 2; pr->term_val[1] = 0.0;
    pr->term_idx[2] = 3; pr->term_val[2] = 1.0 / sqrt(rf);
    pr->has_cost = true;
  } else {
    pr->n_x = 1; pr->n_u = 1; pr->n_e = 0;
    pr->x0[0] = nparams >= 1 ? params[0] : 1.0;
    pr->has_cost = false;
  }
  // the preconditioner of an FP64 problem runs in FP32 when asked (bk_set_f64_precond): flexible
  // GMRES keeps FP64 vectors, operator and Arnoldi, so the solution keeps FP64 accuracy
  pr->pdtype = (dtype == BK_F64 && f64_precond32(N)) ? BK_F32 : dtype;
  const int seg = seg_nodes(pr->pdtype);  // sweeps run in the preconditioner's precision
  pr->nseg = (int)((pr->L + seg - 1) / seg);
  pr->nlev = 1;
  pr->lvn[0] = pr->nseg;
  while (pr->lvn[pr->nlev - 1] > 32 && pr->nlev < MAXLEV) {
    pr->lvn[pr->nlev] = (pr->lvn[pr->nlev - 1] + 31) / 32;
    ++pr->nlev;
  }
  AllocCounter counter(&pr->bytes);
  bk_status s = alloc_opdata(pr, pr->d64, BK_F64);
  if (s == BK_OK && (dtype == BK_F32 || pr->pdtype == BK_F32)) s = alloc_opdata(pr, pr->d32, BK_F32);
  if (s == BK_OK && pr->pdtype != dtype) s = dmalloc(&pr->pcin, sizeof(float) * pr->kkt_len());
  if (s == BK_OK && pr->pdtype != dtype) s = dmalloc(&pr->pcout, sizeof(float) * pr->kkt_len());
  if (s == BK_OK) s = dmalloc((void**)&pr->F, sizeof(double) * pr->kkt_len());
  if (s == BK_OK) s = dmalloc((void**)&pr->red, sizeof(double) * 2048);
  if (s == BK_OK) s = dmalloc((void**)&pr->s_dev, 256);
  if (s == BK_OK && cudaMemcpy(pr->s_dev, &pr->s, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("time scale copy failed");
    s = BK_ERR_CUDA;
  }
  if (s == BK_OK && pr->free_time) s = dmalloc((void**)&pr->sred, sizeof(double) * 2048);
  if (s == BK_OK && cudaMallocHost((void**)&pr->red_host, sizeof(double) * 512) != cudaSuccess) {
    set_error("cudaMallocHost failed");
    s = BK_ERR_OOM;
  }
  if (s == BK_OK && cudaStreamSynchronize(st) != cudaSuccess) { set_error("sync failed"); s = BK_ERR_CUDA; }
  if (s != BK_OK) { problem_free(pr); return s; }
  *out = pr;
  return BK_OK;
}

// Free final time: the problem's s from z's tail slot (synchronous); other kinds: nothing.
static bk_status sync_time_scale(Problem* pr, const double* z, cudaStream_t st) {
  if (!pr->free_time) return BK_OK;
  double* hs = pr->red_host + 200;
  BK_TRY_CUDA(cudaMemcpyAsync(hs, z + pr->s_idx(), sizeof(double), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  BK_ARG(hs[0] > 0.0 && isfinite(hs[0]), "free final time: the time scale in z must be positive (got %g)", hs[0]);
  pr->s = hs[0];
  return BK_OK;
}

// Minimum-time seed from a minimum-energy KKT vector (layouts of BK_ORBIT and BK_ORBIT_MT, same
// pitch): X and lambda copied, u = atan2(u_r, u_theta) (the thrust direction as the angle of
// a (sin u, cos u)), nu copied, s from the minimum-energy problem.
__global__ void k_seed_mt(const double* __restrict__ zme, int64_t P, int64_t L, double s, double* __restrict__ zmt) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      zmt[m * P + k] = zme[m * P + k];
      zmt[(5 + m) * P + k] = zme[(6 + m) * P + k];
    }
    zmt[4 * P + k] = k < L ? atan2(zme[4 * P + k], zme[5 * P + k]) : 0.0;
    if (k < 32) zmt[9 * P + k] = k < 3 ? zme[10 * P + k] : (k == 3 ? s : 0.0);
  }
}

__global__ void k_scale64(double* __restrict__ v, int64_t n, double a) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] *= a;
}

// Seed, then scale lambda and nu by kappa = 2 / (lambda . (B^a (x) I) f), which zeroes the time
// gradient g_s = 2 - lambda . (B^a (x) I) f of the seed (the minimum-energy solution's thrust is
// already along B^aT lambda, so only the multipliers' scale differs).
static bk_status min_time_seed(Problem* mt, const Problem* me, const double* z_me, double* z_mt, cudaStream_t st) {
  BK_ARG(mt->kind == BK_ORBIT_MT && me->kind == BK_ORBIT, "seed needs a BK_ORBIT_MT and a BK_ORBIT problem");
  BK_ARG(mt->N == me->N && mt->P == me->P, "the two problems must have the same N");
  BK_ARG(mt->t0 == me->t0, "the two problems must start at the same t0");
  const int64_t P = mt->P;
  k_seed_mt<<<nblk(P), 256, 0, st>>>(z_me, P, mt->L, me->s, z_mt);
  BK_CHECK_LAUNCH();
  mt->s = me->s;
  double wn = 0.0;
  BK_TRY(problem_residual(mt, z_mt, mt->F, &wn, st));
  double* hs = mt->red_host + 200;
  BK_TRY_CUDA(cudaMemcpyAsync(hs, mt->F + mt->s_idx(), sizeof(double), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  const double S = 2.0 - hs[0];
  if (!(S > 0.0) || !isfinite(S)) {
    set_error("minimum-energy multipliers give a non-positive time gradient (%g)", S);
    return BK_ERR_ARG;
  }
  k_scale64<<<nblk(4 * P + 3), 256, 0, st>>>(z_mt + 5 * P, 4 * P + 3, 2.0 / S);
  BK_CHECK_LAUNCH();
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  return BK_OK;
}

}  // namespace bk

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

bk_status bk_problem_create(bk_problem** prob, int kind, const double* params, int nparams, int64_t N,
                            bk_dtype dtype, double t0, double tf, void* stream) {
  BK_ARG(prob != nullptr, "problem output pointer is NULL");
  bk::Problem* p = nullptr;
  bk_status s = bk::problem_create(&p, kind, params, nparams, N, (int)dtype, t0, tf, (cudaStream_t)stream);
  *prob = reinterpret_cast<bk_problem*>(p);
  return s;
}

void bk_problem_destroy(bk_problem* prob) { bk::problem_free(reinterpret_cast<bk::Problem*>(prob)); }

bk_status bk_problem_info(const bk_problem* prob, int* n_x, int* n_u, int* n_e, int64_t* pitch, int64_t* kkt_len,
                          int64_t* state_len) {
  BK_ARG(prob != nullptr, "problem is NULL");
  const bk::Problem* p = reinterpret_cast<const bk::Problem*>(prob);
  if (n_x) *n_x = p->n_x;
  if (n_u) *n_u = p->n_u;
  if (n_e) *n_e = p->n_e;
  if (pitch) *pitch = p->P;
  if (kkt_len) *kkt_len = p->kkt_len();
  if (state_len) *state_len = p->state_len();
  return BK_OK;
}

bk_status bk_problem_set_params(bk_problem* prob, const double* params, int nparams, double t0, double tf) {
  BK_ARG(prob != nullptr, "problem is NULL");
  return bk::problem_set_params(reinterpret_cast<bk::Problem*>(prob), params, nparams, t0, tf);
}

bk_status bk_problem_set_control_bounds(bk_problem* prob, const double* lo, const double* hi, int n) {
  BK_ARG(prob != nullptr, "problem is NULL");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  if (n == 0) {
    p->has_ubounds = false;
    p->has_bounds = p->has_ebounds;
    return BK_OK;
  }
  BK_ARG(lo != nullptr && hi != nullptr, "bounds are NULL");
  BK_ARG(n == p->n_u, "n must be 0 or the problem's control count %d (got %d)", p->n_u, n);
  if (!p->has_cost || p->free_time) {
    bk::set_error("control bounds need a fixed-final-time problem with a cost (BK_DBL_INT, BK_ORBIT)");
    return BK_ERR_UNSUPPORTED;
  }
  for (int q = 0; q < n; ++q) {
    BK_ARG(!isnan(lo[q]) && !isnan(hi[q]) && lo[q] < hi[q] && lo[q] != INFINITY && hi[q] != -INFINITY,
           "control %d: need lo < hi (got %g, %g)", q, lo[q], hi[q]);
  }
  if (!p->bar_buf) {
    // the barrier diagonals of both precisions and newton_solve's multiplier vectors
    bk::AllocCounter counter(&p->bytes);
    const size_t m = (size_t)p->n_u * p->P;
    bk_status st = bk::dmalloc((void**)&p->bar_buf, sizeof(double) * 6 * m);
    if (st == BK_OK) st = bk::dmalloc(&p->d64.hbar, sizeof(double) * m);
    if (st == BK_OK && p->d32.plan) st = bk::dmalloc(&p->d32.hbar, sizeof(float) * m);
    if (st != BK_OK) {
      bk::dfree(p->bar_buf);
      bk::dfree(p->d64.hbar);
      bk::dfree(p->d32.hbar);
      p->bar_buf = nullptr;
      p->d64.hbar = p->d32.hbar = nullptr;
      return st;
    }
  }
  for (int q = 0; q < bk::NUM; ++q) {
    p->ulo[q] = q < n ? lo[q] : -INFINITY;
    p->uhi[q] = q < n ? hi[q] : INFINITY;
  }
  p->has_ubounds = true;
  p->has_bounds = true;
  p->bar_mu = p->bar_mu_final;
  return BK_OK;
}

bk_status bk_problem_set_terminal_bounds(bk_problem* prob, const double* lo, const double* hi, int n) {
  BK_ARG(prob != nullptr, "problem is NULL");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  if (n == 0) {
    p->has_ebounds = false;
    p->has_bounds = p->has_ubounds;
    return BK_OK;
  }
  BK_ARG(lo != nullptr && hi != nullptr, "bounds are NULL");
  BK_ARG(n == p->n_e, "n must be 0 or the problem's terminal-condition count %d (got %d)", p->n_e, n);
  if (!p->has_cost || p->free_time) {
    bk::set_error("endpoint bounds need a fixed-final-time problem with a cost (BK_DBL_INT, BK_ORBIT)");
    return BK_ERR_UNSUPPORTED;
  }
  int any = 0;
  for (int r = 0; r < n; ++r) {
    BK_ARG(!isnan(lo[r]) && !isnan(hi[r]), "terminal row %d: NaN bound", r);
    const bool eq = lo[r] == -INFINITY && hi[r] == INFINITY;
    BK_ARG(eq || (isfinite(lo[r]) && hi[r] == INFINITY) || (lo[r] == -INFINITY && isfinite(hi[r])) ||
               (isfinite(lo[r]) && isfinite(hi[r])),
           "terminal row %d: bounds must be finite or the matching infinity (got %g, %g)", r, lo[r], hi[r]);
    if (isfinite(lo[r]) && isfinite(hi[r])) {
      bk::set_error("terminal row %d: two-sided endpoint bounds are not supported (one bound per row)", r);
      return BK_ERR_UNSUPPORTED;
    }
    any += eq ? 0 : 1;
  }
  for (int r = 0; r < bk::NEM; ++r) {
    const bool b = r < n && !(lo[r] == -INFINITY && hi[r] == INFINITY);
    p->term_bnd[r] = b ? 1 : 0;
    p->term_lo[r] = b ? lo[r] : 0.0;
    p->term_hi[r] = b ? hi[r] : 0.0;
  }
  p->has_ebounds = any > 0;
  p->has_bounds = p->has_ubounds || p->has_ebounds;
  p->bar_mu = p->bar_mu_final;
  p->linearized = false;
  return BK_OK;
}

bk_status bk_problem_set_barrier(bk_problem* prob, double mu0, double mu_final, int form) {
  BK_ARG(prob != nullptr, "problem is NULL");
  BK_ARG(isfinite(mu0) && isfinite(mu_final) && mu_final > 0.0 && mu0 >= mu_final && mu0 <= 1e6,
         "need 0 < mu_final <= mu0 <= 1e6 (got %g, %g)", mu0, mu_final);
  BK_ARG(form == BK_BARRIER_PRIMAL || form == BK_BARRIER_PRIMAL_DUAL, "unknown barrier form %d", form);
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  p->bar_mu0 = mu0;
  p->bar_mu_final = mu_final;
  p->bar_form = form;
  p->bar_mu = mu_final;
  return BK_OK;
}

size_t bk_problem_device_bytes(const bk_problem* prob) {
  return prob ? reinterpret_cast<const bk::Problem*>(prob)->bytes : 0;
}

bk_status bk_set_f64_precond(int mode) {
  BK_ARG(mode == 0 || mode == 1 || mode == -1, "mode must be 0 (FP64), 1 (FP32) or -1 (default)");
  bk::g_f64_pc32.store(mode);
  return BK_OK;
}

bk_status bk_problem_precond_dtype(const bk_problem* prob, int* dtype) {
  BK_ARG(prob != nullptr && dtype != nullptr, "NULL argument");
  *dtype = reinterpret_cast<const bk::Problem*>(prob)->pdtype;
  return BK_OK;
}

bk_status bk_linearize(bk_problem* prob, const double* z_lin, void* stream) {
  BK_ARG(prob != nullptr, "problem is NULL");
  BK_ARG(((uintptr_t)z_lin & 15) == 0, "z_lin must be 16-byte aligned");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  BK_TRY(bk::sync_time_scale(p, z_lin, (cudaStream_t)stream));
  return bk::problem_linearize(p, z_lin, (cudaStream_t)stream);
}

bk_status kkt_apply(bk_problem* prob, int op, const void* in, void* out, void* stream) {
  BK_ARG(prob != nullptr && in != nullptr && out != nullptr, "NULL argument");
  BK_ARG(in != out, "in and out must not alias");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  return bk::op_apply(p, p->work(), op, in, out, (cudaStream_t)stream);
}

bk_status precond_apply(bk_problem* prob, int op, const void* in, void* out, int transpose, void* stream) {
  BK_ARG(prob != nullptr && in != nullptr && out != nullptr, "NULL argument");
  BK_ARG(in != out, "in and out must not alias");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  return bk::op_precond(p, p->work(), op, in, out, transpose, (cudaStream_t)stream);
}

bk_status bk_kkt_residual(bk_problem* prob, const double* z, double* F_out, double* wnorm, void* stream) {
  BK_ARG(prob != nullptr && z != nullptr && F_out != nullptr, "NULL argument");
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  BK_TRY(bk::sync_time_scale(p, z, (cudaStream_t)stream));
  return bk::problem_residual(p, z, F_out, wnorm, (cudaStream_t)stream);
}

bk_status bk_min_time_seed(bk_problem* mt, const bk_problem* me, const double* z_me, double* z_mt, void* stream) {
  BK_ARG(mt != nullptr && me != nullptr && z_me != nullptr && z_mt != nullptr, "NULL argument");
  BK_ARG(z_me != z_mt, "z_me and z_mt must not alias");
  return bk::min_time_seed(reinterpret_cast<bk::Problem*>(mt), reinterpret_cast<const bk::Problem*>(me), z_me, z_mt,
                           (cudaStream_t)stream);
}

}  // extern "C"
