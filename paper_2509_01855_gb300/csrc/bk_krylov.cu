// Right-preconditioned restarted GMRES (Algorithm 2 / FastLinSol of the paper: GMRES on
// A P^{-1} Upsilon = beta, then chi = P^{-1} Upsilon). The flexible form is used: the
// preconditioned vectors z_j = P^{-1} v_j are kept and the iterate is x = x0 + Z y, so the
// Arnoldi relation holds for the z_j actually computed. A preconditioner applied in finite
// precision is linear only to its rounding level; forming P^{-1}(V y) afterwards (the textbook
// right-preconditioned update) would put that level under the attainable residual (measured:
// ~1e-4 in FP32 at N = 2^20).
//
// Arnoldi orthogonalisation: classical Gram-Schmidt with the Daniel-Gragg-Kaufman-Stewart test.
// One pass forms h = V^T w and |w|^2, the next w <- w - V h with |w|^2 of the result; a second
// pass runs only when the norm fell below 1/sqrt 2 of its value (cancellation). In FP64 the dot
// and update passes are bound by FP64 FMA throughput (one FMA per 8-byte operand), so each
// skipped pass counts. Dot products are FP64 sums with a fixed block count and reduction order,
// so results do not depend on scheduling. FP32 vectors are multiplied and summed in FP32 over
// runs of 16 elements per thread, each run then added to the thread's FP64 total: on GB300 FP64
// (and every float-to-double conversion) runs at 1/64 of the FP32 rate, and converting each
// operand made the FP32 passes slower than the FP64 ones.
//
// The (m+1) x m Hessenberg matrix, its Givens rotations, the DGKS test and the convergence test
// live on the device (GmState, one thread), so an Arnoldi step needs nothing from the host. A
// restart cycle can run as one CUDA graph: a conditional WHILE node whose body is one
// Arnoldi step (input pick, preconditioner, operator, Gram-Schmidt, Givens), repeated until the
// device clears the condition (converged, breakdown or the cycle's column budget), so a cycle is
// one graph launch and one bounded host wait instead of ~30 launches and one stream sync per
// step (bk_set_krylov_graphs; off by default, see graphs_wanted). Otherwise the host launches each
// step and reads the stop word after it. Both forms run the same kernels on the same values in the
// same order, so their iterates are bitwise identical.
#include <math.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <mutex>
#include <thread>
#include <vector>

#include "bk_krylov.cuh"

namespace bk {

static constexpr int DOT_BLOCKS = 608;   // 4 blocks per SM on 152 SMs, fixed for determinism
static constexpr int MAXM = 100;

// FP32 elements per thread summed in FP32 before each FP64 accumulation.
constexpr int RUN32 = 16;

// 16-byte vector of T (float4 / double2) and its element count: the dot and update passes move
// their operands 16 bytes per load when every vector is 16-byte aligned (the basis is; a caller's
// right-hand side or solution may not be, and then takes the element loop).
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 t; static constexpr int n = 4; };
template <> struct Vec16<double> { typedef double2 t; static constexpr int n = 2; };
__device__ __forceinline__ float vdot(float4 a, float4 b, float c) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, c))));
}
__device__ __forceinline__ double vdot(double2 a, double2 b, double c) { return fma(a.y, b.y, fma(a.x, b.x, c)); }

template <typename T, int CNT>
__device__ __forceinline__ void dot_group_vec(const T* __restrict__ V, int64_t ld, const T* __restrict__ w, int64_t lo,
                                              int64_t hi, double* acc) {
  typedef typename Vec16<T>::t VT;
  constexpr int VW = Vec16<T>::n;
  const int64_t c0 = lo / VW, c1 = hi / VW;   // lo is a multiple of VW
  const VT* wv = reinterpret_cast<const VT*>(w);
  if constexpr (sizeof(T) == 8) {
#pragma unroll 2
    for (int64_t c = c0 + threadIdx.x; c < c1; c += blockDim.x) {
      const VT wk = wv[c];
#pragma unroll
      for (int q = 0; q < CNT; ++q) acc[q] = vdot(reinterpret_cast<const VT*>(V + (int64_t)q * ld)[c], wk, acc[q]);
    }
  } else {
    int64_t c = c0 + threadIdx.x;
    while (c < c1) {
      float a[CNT];
#pragma unroll
      for (int q = 0; q < CNT; ++q) a[q] = 0.f;
#pragma unroll 2
      for (int it = 0; it < RUN32 / VW && c < c1; ++it, c += blockDim.x) {
        const VT wk = wv[c];
#pragma unroll
        for (int q = 0; q < CNT; ++q) a[q] = vdot(reinterpret_cast<const VT*>(V + (int64_t)q * ld)[c], wk, a[q]);
      }
#pragma unroll
      for (int q = 0; q < CNT; ++q) acc[q] += (double)a[q];
    }
  }
  // the slice's last elements (fewer than VW) one by one
  for (int64_t k = c1 * VW + threadIdx.x; k < hi; k += blockDim.x) {
#pragma unroll
    for (int q = 0; q < CNT; ++q) acc[q] += (double)V[(int64_t)q * ld + k] * (double)w[k];
  }
}

template <typename T, int CNT>
__device__ __forceinline__ void dot_group(const T* __restrict__ V, int64_t ld, const T* __restrict__ w, int64_t lo,
                                          int64_t hi, double* acc) {
  if constexpr (sizeof(T) == 8) {
#pragma unroll 2
    for (int64_t k = lo + threadIdx.x; k < hi; k += blockDim.x) {
      const double wk = w[k];
#pragma unroll
      for (int q = 0; q < CNT; ++q) acc[q] += V[(int64_t)q * ld + k] * wk;
    }
  } else {
    int64_t k = lo + threadIdx.x;
    while (k < hi) {
      float a[CNT];
#pragma unroll
      for (int q = 0; q < CNT; ++q) a[q] = 0.f;
#pragma unroll 4
      for (int it = 0; it < RUN32 && k < hi; ++it, k += blockDim.x) {
        const float wk = w[k];
#pragma unroll
        for (int q = 0; q < CNT; ++q) a[q] = fmaf(V[(int64_t)q * ld + k], wk, a[q]);
      }
#pragma unroll
      for (int q = 0; q < CNT; ++q) acc[q] += (double)a[q];
    }
  }
}

// out = sum_b partial[b * nv + i] over nb blocks, by one block in a fixed order (thread t takes
// b = t, t + blockDim, ..., then warp and block tree sums). All threads of the block call it.
__device__ void block_sum_column(const double* __restrict__ partial, int nb, int nv, int i, double* __restrict__ out) {
  __shared__ double red[32];
  double a = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a += __ldcg(partial + (int64_t)b * nv + i);
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) *out = t;
  }
  __syncthreads();
}

// After every block wrote its partials: true in the last block to arrive at *cnt, which then
// resets the counter for the next launch (the partials are visible to it after the fences).
__device__ bool last_block(unsigned* cnt) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    last = atomicAdd(cnt, 1u) == gridDim.x - 1;
    if (last) *cnt = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// out[i] = V_i . w (i < nv), FP64 sums: each block writes partial[b * nv + i] for its slice and
// the last block to finish adds the partials of every column in block order (one launch, the
// result independent of scheduling).
template <typename T>
__device__ __forceinline__ void multidot_body(const T* __restrict__ V, int64_t ld, int nv, const T* __restrict__ w,
                                              int64_t n, double* __restrict__ partial, double* __restrict__ out,
                                              unsigned* __restrict__ cnt) {
  __shared__ double red[8][8];
  // slices of a multiple of 4 elements, so that 16-byte loads start on a slice boundary
  const int64_t chunk = ((n + gridDim.x - 1) / gridDim.x + 3) & ~int64_t(3);
  const int64_t lo = blockIdx.x * chunk < n ? blockIdx.x * chunk : n;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  const bool vec = ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w) |
                     (uintptr_t)(ld * (int64_t)sizeof(T))) & 15) == 0;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    const int ng = nv - i0 < 8 ? nv - i0 : 8;
    const T* Vg = V + (int64_t)i0 * ld;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    if (vec) {
      switch (ng) {
        case 1: dot_group_vec<T, 1>(Vg, ld, w, lo, hi, acc); break;
        case 2: dot_group_vec<T, 2>(Vg, ld, w, lo, hi, acc); break;
        case 3: dot_group_vec<T, 3>(Vg, ld, w, lo, hi, acc); break;
        case 4: dot_group_vec<T, 4>(Vg, ld, w, lo, hi, acc); break;
        case 5: dot_group_vec<T, 5>(Vg, ld, w, lo, hi, acc); break;
        case 6: dot_group_vec<T, 6>(Vg, ld, w, lo, hi, acc); break;
        case 7: dot_group_vec<T, 7>(Vg, ld, w, lo, hi, acc); break;
        default: dot_group_vec<T, 8>(Vg, ld, w, lo, hi, acc); break;
      }
    } else {
      switch (ng) {
        case 1: dot_group<T, 1>(Vg, ld, w, lo, hi, acc); break;
        case 2: dot_group<T, 2>(Vg, ld, w, lo, hi, acc); break;
        case 3: dot_group<T, 3>(Vg, ld, w, lo, hi, acc); break;
        case 4: dot_group<T, 4>(Vg, ld, w, lo, hi, acc); break;
        case 5: dot_group<T, 5>(Vg, ld, w, lo, hi, acc); break;
        case 6: dot_group<T, 6>(Vg, ld, w, lo, hi, acc); break;
        case 7: dot_group<T, 7>(Vg, ld, w, lo, hi, acc); break;
        default: dot_group<T, 8>(Vg, ld, w, lo, hi, acc); break;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double a = acc[q];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = a;
    }
    __syncthreads();
    if (threadIdx.x < ng) {
      double a = 0.0;
      for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp) a += red[wp][threadIdx.x];
      partial[(int64_t)blockIdx.x * nv + i0 + threadIdx.x] = a;
    }
    __syncthreads();
  }
  if (last_block(cnt)) {
    if (nv == 1) {
      block_sum_column(partial, gridDim.x, nv, 0, out);
    } else {
      // one warp per column (fixed lane striding and shuffle tree: the order does not depend on
      // scheduling); the columns' sums run side by side instead of one after another
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int i = warp; i < nv; i += nw) {
        double a = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(partial + (int64_t)b * nv + i);
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) out[i] = a;
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_multidot(const T* __restrict__ V, int64_t ld, int nv, const T* __restrict__ w,
                                                  int64_t n, double* __restrict__ partial, double* __restrict__ out,
                                                  unsigned* __restrict__ cnt) {
  multidot_body<T>(V, ld, nv, w, n, partial, out, cnt);
}

// w <- alpha * w + cscale * sum_i c[i] V_i   (c on the device, FP64). With `partial`, each block
// also writes the sum of squares of its slice of the new w and the last block to finish writes
// their sum, |w|^2, to *sq_out (block order, as k_multidot).
template <typename T>
__device__ __forceinline__ void multiaxpy_body(const T* __restrict__ V, int64_t ld, int nv,
                                               const double* __restrict__ c, double cscale, T* __restrict__ w,
                                               double alpha, int64_t n, double* __restrict__ partial,
                                               double* __restrict__ sq_out, unsigned* __restrict__ cnt) {
  __shared__ double cs[MAXM + 1];
  __shared__ float cs32[MAXM + 1];
  __shared__ double red[8];
  for (int i = threadIdx.x; i < nv; i += blockDim.x) {
    cs[i] = cscale * c[i];
    cs32[i] = (float)(cscale * c[i]);
  }
  __syncthreads();
  double sq = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool vec = ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w) |
                     (uintptr_t)(ld * (int64_t)sizeof(T))) & 15) == 0;
  if (vec) {
    // 16-byte loads and stores; each element's update is the same chain as below (the same
    // values), only the per-thread order of the squares' sum differs
    typedef typename Vec16<T>::t VT;
    constexpr int VW = Vec16<T>::n;
    const int64_t nc = n / VW;
    VT* wv = reinterpret_cast<VT*>(w);
    if constexpr (sizeof(T) == 8) {
      for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc; c += stride) {
        const VT wk = wv[c];
        double ax = alpha == 0.0 ? 0.0 : alpha * wk.x, ay = alpha == 0.0 ? 0.0 : alpha * wk.y;
        for (int i = 0; i < nv; ++i) {
          const VT v = reinterpret_cast<const VT*>(V + (int64_t)i * ld)[c];
          ax += cs[i] * v.x;
          ay += cs[i] * v.y;
        }
        VT o;
        o.x = ax;
        o.y = ay;
        wv[c] = o;
        sq += ax * ax;
        sq += ay * ay;
      }
    } else {
      const float al = (float)alpha;
      int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
      while (c < nc) {
        float s32 = 0.f;
        for (int it = 0; it < RUN32 / VW && c < nc; ++it, c += stride) {
          const VT wk = wv[c];
          float a0 = alpha == 0.0 ? 0.f : al * wk.x, a1 = alpha == 0.0 ? 0.f : al * wk.y;
          float a2 = alpha == 0.0 ? 0.f : al * wk.z, a3 = alpha == 0.0 ? 0.f : al * wk.w;
          for (int i = 0; i < nv; ++i) {
            const VT v = reinterpret_cast<const VT*>(V + (int64_t)i * ld)[c];
            a0 = fmaf(cs32[i], v.x, a0);
            a1 = fmaf(cs32[i], v.y, a1);
            a2 = fmaf(cs32[i], v.z, a2);
            a3 = fmaf(cs32[i], v.w, a3);
          }
          VT o;
          o.x = a0;
          o.y = a1;
          o.z = a2;
          o.w = a3;
          wv[c] = o;
          s32 = fmaf(a0, a0, s32);
          s32 = fmaf(a1, a1, s32);
          s32 = fmaf(a2, a2, s32);
          s32 = fmaf(a3, a3, s32);
        }
        sq += (double)s32;
      }
    }
    // the last n mod VW elements one by one
    for (int64_t k = nc * VW + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
      T a = alpha == 0.0 ? T(0) : T(alpha) * w[k];
      for (int i = 0; i < nv; ++i) a += (sizeof(T) == 8 ? T(cs[i]) : T(cs32[i])) * V[(int64_t)i * ld + k];
      w[k] = a;
      sq += (double)a * (double)a;
    }
  } else if constexpr (sizeof(T) == 8) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
      double a = alpha == 0.0 ? 0.0 : alpha * w[k];
      int i = 0;
      for (; i + 4 <= nv; i += 4) {
        const double v0 = V[(int64_t)i * ld + k], v1 = V[(int64_t)(i + 1) * ld + k];
        const double v2 = V[(int64_t)(i + 2) * ld + k], v3 = V[(int64_t)(i + 3) * ld + k];
        a += cs[i] * v0;
        a += cs[i + 1] * v1;
        a += cs[i + 2] * v2;
        a += cs[i + 3] * v3;
      }
      for (; i < nv; ++i) a += cs[i] * V[(int64_t)i * ld + k];
      w[k] = a;
      sq += a * a;
    }
  } else {
    const float al = (float)alpha;
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    while (k < n) {
      float s32 = 0.f;
      for (int it = 0; it < RUN32 && k < n; ++it, k += stride) {
        float a = alpha == 0.0 ? 0.f : al * (float)w[k];
        int i = 0;
        for (; i + 4 <= nv; i += 4) {
          const float v0 = V[(int64_t)i * ld + k], v1 = V[(int64_t)(i + 1) * ld + k];
          const float v2 = V[(int64_t)(i + 2) * ld + k], v3 = V[(int64_t)(i + 3) * ld + k];
          a = fmaf(cs32[i], v0, a);
          a = fmaf(cs32[i + 1], v1, a);
          a = fmaf(cs32[i + 2], v2, a);
          a = fmaf(cs32[i + 3], v3, a);
        }
        for (; i < nv; ++i) a = fmaf(cs32[i], (float)V[(int64_t)i * ld + k], a);
        w[k] = (T)a;
        s32 = fmaf(a, a, s32);
      }
      sq += (double)s32;
    }
  }
  if (partial) {
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int wp = 0; wp < (int)(blockDim.x >> 5); ++wp) t += red[wp];
      partial[blockIdx.x] = t;
    }
    if (last_block(cnt)) block_sum_column(partial, gridDim.x, 1, 0, sq_out);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_multiaxpy(const T* __restrict__ V, int64_t ld, int nv,
                                                   const double* __restrict__ c, double cscale, T* __restrict__ w,
                                                   double alpha, int64_t n, double* __restrict__ partial,
                                                   double* __restrict__ sq_out = nullptr,
                                                   unsigned* __restrict__ cnt = nullptr) {
  multiaxpy_body<T>(V, ld, nv, c, cscale, w, alpha, n, partial, sq_out, cnt);
}

// --- device-resident Arnoldi state -----------------------------------------------------------
// One per GMRES workspace. j counts the columns of the current cycle; the host sets the cycle up
// (k_gm_init) and reads the first fields back at its end.
struct GmState {
  int j;          // columns finished in this cycle
  int jmax;       // columns allowed in this cycle (restart length, iteration cap)
  int m;          // restart length (row stride of H)
  int need2;      // DGKS: second Gram-Schmidt pass wanted for the current column
  int stop;       // the cycle is over (converged, breakdown, or jmax reached)
  int pad;
  double target;  // absolute residual target
  double resid;   // |g_{j}|, the Arnoldi residual estimate after the last column
  double hn;      // |w| after orthogonalisation, the new basis vector's scale
  double gv[MAXM + 1], cs[MAXM], sn[MAXM], y[MAXM];
  double H[(MAXM + 1) * MAXM];
};

__global__ void k_gm_init(GmState* s, double beta, double target, int jmax, int m) {
  const int t = threadIdx.x;
  if (t == 0) {
    s->j = 0;
    s->jmax = jmax;
    s->m = m;
    s->need2 = 0;
    s->stop = 0;
    s->target = target;
    s->resid = beta;
    s->hn = 0.0;
  }
  for (int i = t; i <= MAXM; i += blockDim.x) s->gv[i] = i == 0 ? beta : 0.0;
}

// V_i . w for i < j + add, w = V_{j + woff} (j from the state); skipped when *gate == 0.
template <typename T>
__global__ void __launch_bounds__(256) k_multidot_s(const T* __restrict__ V, int64_t ld, int add, int woff,
                                                    const GmState* __restrict__ s, const int* __restrict__ gate,
                                                    int64_t n, double* __restrict__ partial, double* __restrict__ out,
                                                    unsigned* __restrict__ cnt) {
  if (gate && *gate == 0) return;
  const int j = s->j;
  multidot_body<T>(V, ld, j + add, V + (int64_t)(j + woff) * ld, n, partial, out, cnt);
}

// w <- alpha w + cscale sum_{i < j + add} c_i V_i with w = V_{j + woff} (woff >= 0) or the
// fixed vector x (woff < 0); skipped when *gate == 0.
template <typename T>
__global__ void __launch_bounds__(256) k_multiaxpy_s(const T* __restrict__ V, int64_t ld, int add, int woff,
                                                     T* __restrict__ x, const GmState* __restrict__ s,
                                                     const int* __restrict__ gate, const double* __restrict__ c,
                                                     double cscale, double alpha, int64_t n,
                                                     double* __restrict__ partial, double* __restrict__ sq_out,
                                                     unsigned* __restrict__ cnt) {
  if (gate && *gate == 0) return;
  const int j = s->j;
  T* w = woff >= 0 ? const_cast<T*>(V) + (int64_t)(j + woff) * ld : x;
  multiaxpy_body<T>(V, ld, j + add, c, cscale, w, alpha, n, partial, sq_out, cnt);
}

// After the first Gram-Schmidt pass: column j of H from h = V^T w, and the DGKS test (|w|^2
// after the pass below half of |w|^2 before it).
__global__ void k_gm_a(GmState* s, const double* __restrict__ h1, const double* __restrict__ w2) {
  const int j = s->j, m = s->m;
  for (int i = threadIdx.x; i <= j; i += blockDim.x) s->H[i * m + j] = h1[i];
  if (threadIdx.x == 0) s->need2 = w2[0] < 0.5 * h1[j + 1] ? 1 : 0;
}

// Column j finished: the second pass's corrections, |w|, the Givens rotations of the column,
// the residual estimate and the stop test; j advances. In a graph, the WHILE condition follows.
__global__ void k_gm_b(GmState* s, const double* __restrict__ h2, const double* __restrict__ w2,
                       cudaGraphConditionalHandle cond, int in_graph) {
  if (threadIdx.x != 0) return;
  const int j = s->j, m = s->m;
  double* H = s->H;
  if (s->need2)
    for (int i = 0; i <= j; ++i) H[i * m + j] += h2[i];
  const double hnext = sqrt(w2[0]);
  s->hn = hnext;
  H[(j + 1) * m + j] = hnext;
  for (int i = 0; i < j; ++i) {
    const double a = H[i * m + j], c = H[(i + 1) * m + j];
    H[i * m + j] = s->cs[i] * a + s->sn[i] * c;
    H[(i + 1) * m + j] = -s->sn[i] * a + s->cs[i] * c;
  }
  const double a = H[j * m + j], c = H[(j + 1) * m + j];
  const double den = hypot(a, c);
  const double cj = den == 0.0 ? 1.0 : a / den;
  const double sj = den == 0.0 ? 0.0 : c / den;
  s->cs[j] = cj;
  s->sn[j] = sj;
  H[j * m + j] = den;
  H[(j + 1) * m + j] = 0.0;
  const double g = s->gv[j];
  s->gv[j + 1] = -sj * g;
  s->gv[j] = cj * g;
  const double resid = fabs(s->gv[j + 1]);
  s->resid = resid;
  s->j = j + 1;
  const int stop = (resid <= s->target || hnext == 0.0 || j + 1 >= s->jmax) ? 1 : 0;
  s->stop = stop;
  if (in_graph) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}

// V_j <- V_j / hn (j after k_gm_b, i.e. the new basis vector), unless hn == 0.
template <typename T>
__global__ void k_scale_inv_s(T* __restrict__ V, int64_t ld, const GmState* __restrict__ s, int64_t n) {
  const double hn = s->hn;
  if (!(hn > 0.0)) return;
  T* v = V + (int64_t)s->j * ld;
  const T inv = (T)(1.0 / hn);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    v[k] = v[k] * inv;
}

// y = H(0:j, 0:j)^{-1} g (back substitution, one thread).
__global__ void k_gm_solve(GmState* s) {
  if (threadIdx.x != 0) return;
  const int j = s->j, m = s->m;
  for (int i = j - 1; i >= 0; --i) {
    double a = s->gv[i];
    for (int q = i + 1; q < j; ++q) a -= s->H[i * m + q] * s->y[q];
    s->y[i] = a / s->H[i * m + i];
  }
}

// Graph form, input of a step: dst = V_j.
template <typename T>
__global__ void k_gm_pick(const T* __restrict__ V, int64_t ld, const GmState* __restrict__ s, T* __restrict__ dst,
                          int64_t n) {
  const T* v = V + (int64_t)s->j * ld;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = v[k];
}

// Graph form, outputs of a step: V_{j+1} = w, Z_j = z (Z non-null), T_j = a (T non-null).
template <typename T>
__global__ void k_gm_place(T* __restrict__ V, T* __restrict__ Z, int64_t ld, const GmState* __restrict__ s,
                           const T* __restrict__ w, const T* __restrict__ z, int64_t n, double* __restrict__ Tr,
                           int64_t tld, const double* __restrict__ a, int64_t an) {
  const int j = s->j;
  T* vd = V + (int64_t)(j + 1) * ld;
  T* zd = Z ? Z + (int64_t)j * ld : nullptr;
  double* td = Tr ? Tr + (int64_t)j * tld : nullptr;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride) {
    vd[k] = w[k];
    if (zd) zd[k] = z[k];
  }
  if (td)
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < an; k += stride) td[k] = a[k];
}

// y <- a * x + b * y  (a, b host scalars)
template <typename T>
__global__ void k_axpby(const T* __restrict__ x, double a, T* __restrict__ y, double b, int64_t n) {
  const T aa = (T)a, bb = (T)b;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = b == 0.0 ? aa * x[k] : aa * x[k] + bb * y[k];
}

// y <- x * (1 / c[0])  (scale by a device scalar)
template <typename T>
__global__ void k_scale_inv(const T* __restrict__ x, const double* __restrict__ c, T* __restrict__ y, int64_t n) {
  const T inv = (T)(1.0 / c[0]);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    y[k] = x[k] * inv;
}

template <typename T>
static bk_status dots(const T* V, int64_t ld, int nv, const T* w, int64_t n, double* partial, double* out,
                      unsigned* cnt, cudaStream_t st) {
  k_multidot<T><<<DOT_BLOCKS, 256, 0, st>>>(V, ld, nv, w, n, partial, out, cnt);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

static inline int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

size_t gmres_workspace_bytes(int64_t n, int m, int dtype) {
  const size_t es = dtype_size(dtype);
  const int64_t ld = round_up(n, 64);
  size_t b = es * (size_t)ld * (m + 1);      // basis V
  b += es * (size_t)ld * m;                  // preconditioned basis Z
  b += es * (size_t)ld * 3;                  // z scratch, r / correction, graph-step z
  b += sizeof(double) * (size_t)ld;          // graph-step transposed-product record
  b += sizeof(double) * (size_t)DOT_BLOCKS * (MAXM + 2);  // dot partials
  b += sizeof(double) * 4 * (MAXM + 2);      // device scalars
  b += sizeof(GmState);                      // device-resident Arnoldi state
  return b + 2048;
}

// out = D in (inv = 0) or D^-1 in (inv = 1) for a KKT vector: the first nz blocks (gradient rows)
// scale by w^-1/2, the next nl blocks (constraint rows) by w^1/2, the tail and padding by 1.
template <typename T>
__global__ void k_wscale(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ w, int64_t P,
                         int64_t L, int nz, int nl, int64_t n, int inv) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t blk = i / P, k = i - blk * P;
    T f = T(1);
    if (k < L && blk < nz + nl) {
      const T r = sqrt(w[k]);
      const bool grad = blk < nz;
      f = (grad != (inv != 0)) ? T(1) / r : r;
    }
    out[i] = f * in[i];
  }
}

// --- one Arnoldi step -------------------------------------------------------------------------
template <typename T>
struct GmCtx {
  Problem* pr;
  OpData* d;
  int op;
  bool weighted, precond;
  const KrylovMu* aux;
  T *V, *Zb, *z, *r, *zc;
  double* ac;
  int64_t n, ld;
  double *partial, *h1, *h2;
  unsigned* cnt;
  GmState* gs;
  int g;
};

// Column j of the Arnoldi process. Host form (graph = false): the operator reads V_j and writes
// Z_j, V_{j+1} in place (jh = j, known to the host). Graph form: the step's vectors go through
// fixed buffers (V_j picked into z or r, outputs placed into V_{j+1}, Z_j and T_j by the device's
// j), so that one captured body serves every column. Everything after the operator reads j from
// the device state in both forms.
template <typename T>
static bk_status arnoldi_step(const GmCtx<T>& c, int jh, bool graph, cudaGraphConditionalHandle cond,
                              cudaStream_t st) {
  Problem* pr = c.pr;
  OpData& d = *c.d;
  const int64_t n = c.n, ld = c.ld;
  const int wz = pr->n_x + pr->n_u, wl = pr->n_x;
  T* wout = graph ? c.r : c.V + (int64_t)(jh + 1) * ld;
  void* aout = nullptr;
  if (c.aux) aout = graph ? (void*)c.ac : (void*)(c.aux->T + (int64_t)jh * c.aux->ld);
  const T* vin = c.V + (int64_t)jh * ld;
  if (graph) {
    T* dst = c.weighted ? c.r : c.z;
    k_gm_pick<T><<<c.g, 256, 0, st>>>(c.V, ld, c.gs, dst, n);
    BK_CHECK_LAUNCH();
    vin = dst;
  }
  if (c.precond) {
    T* zout = graph ? c.zc : c.Zb + (int64_t)jh * ld;
    if (c.weighted) {
      k_wscale<T><<<c.g, 256, 0, st>>>(vin, c.z, (const T*)d.w, pr->P, pr->L, wz, wl, n, 1);
      BK_CHECK_LAUNCH();
      BK_TRY(op_precond(pr, d, c.op, c.z, zout, 0, st));
    } else {
      BK_TRY(op_precond(pr, d, c.op, vin, zout, 0, st));
    }
    BK_TRY(op_apply(pr, d, c.op, zout, wout, st, aout));
  } else {
    BK_TRY(op_apply(pr, d, c.op, vin, wout, st, aout));
  }
  if (c.weighted) {
    k_wscale<T><<<c.g, 256, 0, st>>>(wout, wout, (const T*)d.w, pr->P, pr->L, wz, wl, n, 0);
    BK_CHECK_LAUNCH();
  }
  if (graph) {
    k_gm_place<T><<<c.g, 256, 0, st>>>(c.V, c.precond ? c.Zb : nullptr, ld, c.gs, c.r, c.zc, n,
                                       c.aux ? c.aux->T : nullptr, c.aux ? c.aux->ld : 0, c.ac,
                                       c.aux ? c.aux->n : 0);
    BK_CHECK_LAUNCH();
  }
  // Gram-Schmidt (DGKS): h1 = [V_0..V_j]^T w and |w|^2 (w = V_{j+1}), w <- w - V h1 with the new
  // |w|^2; the second pass runs (its kernels do work) only when k_gm_a asked for it.
  double* w2 = c.h2 + (MAXM + 1);
  k_multidot_s<T><<<DOT_BLOCKS, 256, 0, st>>>(c.V, ld, 2, 1, c.gs, nullptr, n, c.partial, c.h1, c.cnt);
  BK_CHECK_LAUNCH();
  k_multiaxpy_s<T><<<DOT_BLOCKS, 256, 0, st>>>(c.V, ld, 1, 1, nullptr, c.gs, nullptr, c.h1, -1.0, 1.0, n, c.partial,
                                               w2, c.cnt + 1);
  BK_CHECK_LAUNCH();
  k_gm_a<<<1, 128, 0, st>>>(c.gs, c.h1, w2);
  BK_CHECK_LAUNCH();
  k_multidot_s<T><<<DOT_BLOCKS, 256, 0, st>>>(c.V, ld, 1, 1, c.gs, &c.gs->need2, n, c.partial, c.h2, c.cnt);
  BK_CHECK_LAUNCH();
  k_multiaxpy_s<T><<<DOT_BLOCKS, 256, 0, st>>>(c.V, ld, 1, 1, nullptr, c.gs, &c.gs->need2, c.h2, -1.0, 1.0, n,
                                               c.partial, w2, c.cnt + 1);
  BK_CHECK_LAUNCH();
  k_gm_b<<<1, 32, 0, st>>>(c.gs, c.h2, w2, cond, graph ? 1 : 0);
  BK_CHECK_LAUNCH();
  k_scale_inv_s<T><<<c.g, 256, 0, st>>>(c.V, ld, c.gs, n);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// --- graph cycles ------------------------------------------------------------------------------
// A captured cycle bakes in every pointer and host scalar its kernels take, so the key holds
// them all: workspace, operator data, aux record, flags and lengths. The time scale s is not
// among them: for a fixed final time the step's kernels read it from the problem's device copy,
// which bk_problem_set_params updates (a free final time, whose s changes inside a Newton step,
// never runs graphs).
struct GmGraph {
  const void* ws;
  const void* d;
  const void* auxT;
  const void* auxTd;
  int64_t auxld, auxn;
  int op, weighted, precond, m;
  int64_t n;
  double s;
  long long nbody;   // kernels in the WHILE body (one Arnoldi step)
  cudaGraph_t g;
  cudaGraphExec_t x;
  bool failed;
};

struct GmCache {
  cudaStream_t cap = nullptr;   // capture only; nothing is ever launched on it
  cudaEvent_t done = nullptr;   // recorded after a cycle's summary copy
  std::vector<GmGraph> v;
};

void gmres_graphs_free(Problem* pr) {
  GmCache* gc = reinterpret_cast<GmCache*>(pr->gcache);
  if (!gc) return;
  for (GmGraph& e : gc->v) {
    if (e.x) cudaGraphExecDestroy(e.x);
    if (e.g) cudaGraphDestroy(e.g);
  }
  if (gc->done) cudaEventDestroy(gc->done);
  if (gc->cap) cudaStreamDestroy(gc->cap);
  delete gc;
  pr->gcache = nullptr;
}

static std::mutex g_capture_mutex;
static std::atomic<int> g_graph_mode{-1};
static std::atomic<long long> g_wait_ns{-1};
static constexpr double WAIT_DEFAULT_S = 60.0;

// Off by default. Measured on GB300 (orbit solves, N = 2^8..2^16): graph cycles make a solve
// 5-13% faster, but in the serving mix (16 host threads, one problem per slot) they lowered the
// closed-loop rate from ~570 to ~510 solves/s.
static bool graphs_wanted(const Problem* pr) {
  if (pr->free_time) return false;   // s changes every Newton step
  if (pr->has_bounds) return false;  // the barrier parameter changes between stages
  return g_graph_mode.load() == 1;
}

// The cycle graph for this call's pointers: captured on first use (a WHILE node whose body is one
// Arnoldi step), null when capture or instantiation failed (the host form runs instead).
template <typename T>
static GmGraph* graph_get(const GmCtx<T>& c, const void* ws, int m) {
  Problem* pr = c.pr;
  GmCache* gc = reinterpret_cast<GmCache*>(pr->gcache);
  if (!gc) {
    gc = new GmCache();
    if (cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&gc->done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      if (gc->cap) cudaStreamDestroy(gc->cap);
      delete gc;
      return nullptr;
    }
    pr->gcache = gc;
  }
  GmGraph key;
  memset(&key, 0, sizeof(key));
  key.ws = ws;
  key.d = c.d;
  key.auxT = c.aux ? c.aux->T : nullptr;
  key.auxTd = c.aux ? c.aux->Td : nullptr;
  key.auxld = c.aux ? c.aux->ld : 0;
  key.auxn = c.aux ? c.aux->n : 0;
  key.op = c.op;
  key.weighted = c.weighted;
  key.precond = c.precond;
  key.m = m;
  key.n = c.n;
  key.s = 0.0;
  for (GmGraph& e : gc->v)
    if (e.ws == key.ws && e.d == key.d && e.auxT == key.auxT && e.auxTd == key.auxTd && e.auxld == key.auxld &&
        e.auxn == key.auxn && e.op == key.op && e.weighted == key.weighted && e.precond == key.precond &&
        e.m == key.m && e.n == key.n && e.s == key.s)
      return e.failed ? nullptr : &e;
  // captures and instantiations of all problems run one at a time (they are rare: one per
  // problem, workspace and parameter set)
  std::lock_guard<std::mutex> lock(g_capture_mutex);
  if (gc->v.size() >= 4) {   // bounded cache: drop the oldest (an in-flight launch finishes first)
    if (gc->v.front().x) cudaGraphExecDestroy(gc->v.front().x);
    if (gc->v.front().g) cudaGraphDestroy(gc->v.front().g);
    gc->v.erase(gc->v.begin());
  }
  GmGraph e = key;
  bool ok = cudaGraphCreate(&e.g, 0) == cudaSuccess;
  cudaGraphConditionalHandle h = 0;
  cudaGraph_t body = nullptr;
  if (ok) ok = cudaGraphConditionalHandleCreate(&h, e.g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    ok = cudaGraphAddNode(&node, e.g, nullptr, nullptr, 0, &cp) == cudaSuccess;
    if (ok) body = cp.conditional.phGraph_out[0];
  }
  if (ok) ok = cudaStreamBeginCaptureToGraph(gc->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) ==
               cudaSuccess;
  if (ok) {
    const unsigned long long c0 = thread_launches();
    const bk_status sst = arnoldi_step<T>(c, 0, true, h, gc->cap);
    cudaGraph_t out = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(gc->cap, &out);
    e.nbody = (long long)(thread_launches() - c0);
    note_launches(-e.nbody);   // captured, not run
    ok = sst == BK_OK && ce == cudaSuccess;
  }
  if (ok) ok = cudaGraphInstantiate(&e.x, e.g, 0) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (e.x) cudaGraphExecDestroy(e.x);
    if (e.g) cudaGraphDestroy(e.g);
    e.x = nullptr;
    e.g = nullptr;
    e.failed = true;
  }
  gc->v.push_back(e);
  return ok ? &gc->v.back() : nullptr;
}

// Bounded host wait for an event (the end of a graph cycle): BK_ERR_TIMEOUT after the limit,
// with the work possibly still running on the stream.
static bk_status wait_bounded(cudaEvent_t ev) {
  const long long lim = g_wait_ns.load();
  const double limit_s = lim > 0 ? lim * 1e-9 : WAIT_DEFAULT_S;
  const auto t0 = std::chrono::steady_clock::now();
  for (long spins = 0;; ++spins) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return BK_OK;
    if (e != cudaErrorNotReady) {
      set_error("CUDA error while waiting for a GMRES cycle: %s", cudaGetErrorString(e));
      return BK_ERR_CUDA;
    }
    const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (el > limit_s) {
      set_error("a GMRES cycle did not finish within the wait limit of %.3g s (its work may still be running "
                "on the stream: synchronise it before reusing the vectors)", limit_s);
      return BK_ERR_TIMEOUT;
    }
    if (spins > 64) std::this_thread::yield();
  }
}

// Host mirror of the head of GmState (copied back at the end of a step or cycle).
struct GmHead {
  int j, jmax, m, need2, stop, pad;
  double target, resid, hn;
};

template <typename T>
static bk_status gmres_impl(Problem* pr, OpData& d, int op, const T* b, T* x, const bk_krylov_opts& o,
                            bk_krylov_info* info, void* ws, cudaStream_t st, double* hostbuf, const KrylovMu* aux,
                            bool weighted) {
  const int64_t n = op == BK_OP_KKT ? pr->kkt_len() : pr->state_len();
  const int m = o.restart;
  const int64_t ld = round_up(n, 64);
  char* p = (char*)ws;
  auto carve = [&](size_t bytes) { char* r = p; p += (bytes + 255) / 256 * 256; return (void*)r; };
  T* V = (T*)carve(sizeof(T) * ld * (m + 1));
  T* Zb = (T*)carve(sizeof(T) * ld * m);
  T* z = (T*)carve(sizeof(T) * ld);
  T* r = (T*)carve(sizeof(T) * ld);
  T* zc = (T*)carve(sizeof(T) * ld);
  double* ac = (double*)carve(sizeof(double) * ld);
  double* partial = (double*)carve(sizeof(double) * DOT_BLOCKS * (MAXM + 2));
  double* dvec = (double*)carve(sizeof(double) * 4 * (MAXM + 2));
  GmState* gs = (GmState*)carve(sizeof(GmState));
  double* h1 = dvec;
  double* h2 = dvec + (MAXM + 2);
  // arrival counters of the one-launch reductions (k_multidot, k_multiaxpy); each launch's
  // last block resets its counter, so one clear per solve suffices
  unsigned* cnt = reinterpret_cast<unsigned*>(dvec + 3 * (MAXM + 2));
  BK_TRY_CUDA(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned), st));
  const int g = grid_for(n);
  weighted = weighted && op == BK_OP_KKT && o.use_precond;
  const int wz = pr->n_x + pr->n_u, wl = pr->n_x;
  auto wscale = [&](const T* in, T* out, int inv) -> bk_status {
    k_wscale<T><<<g, 256, 0, st>>>(in, out, (const T*)d.w, pr->P, pr->L, wz, wl, n, inv);
    BK_CHECK_LAUNCH();
    return BK_OK;
  };
  // the right-hand side the iteration sees: D b (weighted) or b
  const T* bw = b;
  if (weighted) {
    BK_TRY(wscale(b, r, 0));
    bw = r;
  }

  // ||b||
  BK_TRY(dots<T>(bw, ld, 1, bw, n, partial, h1, cnt, st));
  BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, h1, sizeof(double), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  const double bnorm = sqrt(hostbuf[0]);
  BK_TRY_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * n, st));
  if (aux) BK_TRY_CUDA(cudaMemsetAsync(aux->Td, 0, sizeof(double) * aux->n, st));
  info->iterations = 0;
  info->restarts = 0;
  info->rel_resid = 0.0;
  info->converged = 0;
  if (bnorm == 0.0) { info->converged = 1; return BK_OK; }
  const double target = o.rtol * bnorm;
  const GmCtx<T> ctx = {pr, &d, op, weighted, o.use_precond != 0, aux, V, Zb, z, r, zc, ac, n, ld, partial, h1, h2,
                        cnt, gs, g};
  GmGraph* gg = graphs_wanted(pr) ? graph_get<T>(ctx, ws, m) : nullptr;
  GmCache* gc = reinterpret_cast<GmCache*>(pr->gcache);
  GmHead hd;
  int total = 0;
  double resid = bnorm;
  bool first = true;
  while (true) {
    // r = b - A x (x = 0 on the first cycle)
    if (first) {
      if (!weighted) {  // weighted: r already holds D b
        k_axpby<T><<<g, 256, 0, st>>>(b, 1.0, r, 0.0, n);
        BK_CHECK_LAUNCH();
      }
    } else {
      BK_TRY(op_apply(pr, d, op, x, r, st));
      k_axpby<T><<<g, 256, 0, st>>>(b, 1.0, r, -1.0, n);
      BK_CHECK_LAUNCH();
      if (weighted) BK_TRY(wscale(r, r, 0));
    }
    double beta = bnorm;  // r = b on the first cycle
    if (!first) {
      BK_TRY(dots<T>(r, ld, 1, r, n, partial, h1, cnt, st));
      BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, h1, sizeof(double), cudaMemcpyDeviceToHost, st));
      BK_TRY_CUDA(cudaStreamSynchronize(st));
      beta = sqrt(hostbuf[0]);
    }
    first = false;
    resid = beta;
    if (beta <= target || total >= o.max_iter) break;
    k_axpby<T><<<g, 256, 0, st>>>(r, 1.0 / beta, V, 0.0, n);
    BK_CHECK_LAUNCH();
    const int jmax = std::min(m, o.max_iter - total);
    k_gm_init<<<1, 128, 0, st>>>(gs, beta, target, jmax, m);
    BK_CHECK_LAUNCH();
    if (gg) {
      BK_TRY_CUDA(cudaGraphLaunch(gg->x, st));
    } else {
      for (int jh = 0;; ++jh) {
        BK_TRY(arnoldi_step<T>(ctx, jh, false, 0, st));
        BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, gs, sizeof(GmHead), cudaMemcpyDeviceToHost, st));
        BK_TRY_CUDA(cudaStreamSynchronize(st));
        memcpy(&hd, hostbuf, sizeof(GmHead));
        if (hd.stop) break;
      }
    }
    // x += Z y (flexible form; Z = V without preconditioning), y = H^{-1} g on the device
    k_gm_solve<<<1, 32, 0, st>>>(gs);
    BK_CHECK_LAUNCH();
    k_multiaxpy_s<T><<<g, 256, 0, st>>>(o.use_precond ? Zb : V, ld, 0, -1, x, gs, nullptr, gs->y, 1.0, 1.0, n,
                                        nullptr, nullptr, nullptr);
    BK_CHECK_LAUNCH();
    if (aux) {
      k_multiaxpy_s<double><<<grid_for(aux->n), 256, 0, st>>>(aux->T, aux->ld, 0, -1, aux->Td, gs, nullptr, gs->y,
                                                              1.0, 1.0, aux->n, nullptr, nullptr, nullptr);
      BK_CHECK_LAUNCH();
    }
    if (gg) {
      BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, gs, sizeof(GmHead), cudaMemcpyDeviceToHost, st));
      BK_TRY_CUDA(cudaEventRecord(gc->done, st));
      BK_TRY(wait_bounded(gc->done));
      memcpy(&hd, hostbuf, sizeof(GmHead));
      note_launches(gg->nbody * hd.j);   // the body ran once per column
    }
    total += hd.j;
    resid = hd.resid;
    ++info->restarts;
    // A converged cycle returns on its Arnoldi residual estimate |g_{j+1}|: in the flexible form
    // it is the residual of the iterate built from the z_j actually computed, and recomputing
    // b - A x would cost one more operator apply per solve. The true residual is formed on
    // restarts and at the iteration cap.
    if (resid <= target) break;
    if (total >= o.max_iter) {
      // final explicit residual
      BK_TRY(op_apply(pr, d, op, x, r, st));
      k_axpby<T><<<g, 256, 0, st>>>(b, 1.0, r, -1.0, n);
      BK_CHECK_LAUNCH();
      if (weighted) BK_TRY(wscale(r, r, 0));
      BK_TRY(dots<T>(r, ld, 1, r, n, partial, h1, cnt, st));
      BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, h1, sizeof(double), cudaMemcpyDeviceToHost, st));
      BK_TRY_CUDA(cudaStreamSynchronize(st));
      resid = sqrt(hostbuf[0]);
      break;
    }
  }
  info->iterations = total;
  info->rel_resid = resid / bnorm;
  info->converged = resid <= target ? 1 : 0;
  return BK_OK;
}

bk_status gmres(Problem* pr, OpData& d, int op, const void* b, void* x, const bk_krylov_opts& o, bk_krylov_info* info,
                void* ws, cudaStream_t st, const KrylovMu* aux, bool weighted) {
  BK_ARG(o.restart >= 1 && o.restart <= MAXM, "restart must be in [1, %d]", MAXM);
  BK_ARG(o.max_iter >= 1, "max_iter must be >= 1");
  BK_ARG(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be 256-byte aligned");
  BK_ARG(aux == nullptr || (d.dtype == BK_F64 && op == BK_OP_KKT), "transposed-product record needs the FP64 KKT operator");
  if (d.dtype == BK_F64)
    BK_TRY(gmres_impl<double>(pr, d, op, (const double*)b, (double*)x, o, info, ws, st, pr->red_host, aux, weighted));
  else
    BK_TRY(gmres_impl<float>(pr, d, op, (const float*)b, (float*)x, o, info, ws, st, pr->red_host, nullptr, weighted));
  // a dense product that ran out of a bounded wait leaves invalid values behind: fail the solve
  return dense_status(d.plan, st);
}

bk_krylov_opts krylov_defaults() {
  bk_krylov_opts o;
  o.rtol = 1e-10;
  o.restart = 30;
  o.max_iter = 300;
  o.use_precond = 1;
  return o;
}

}  // namespace bk

extern "C" {

bk_status bk_set_krylov_graphs(int mode) {
  BK_ARG(mode == -1 || mode == 0 || mode == 1, "mode must be -1 (default), 0 (never) or 1 (always)");
  bk::g_graph_mode.store(mode);
  return BK_OK;
}

bk_status bk_set_krylov_wait_limit(double seconds) {
  BK_ARG(!(seconds > 1e6) && seconds == seconds, "limit must be at most 1e6 s");
  bk::g_wait_ns.store(seconds > 0 ? (long long)(seconds * 1e9) : -1);
  return BK_OK;
}

size_t bk_krylov_workspace_bytes(const bk_problem* prob, int op, int restart) {
  const bk::Problem* p = reinterpret_cast<const bk::Problem*>(prob);
  if (!p) return 0;
  if (restart <= 0) restart = 30;
  const int64_t n = op == BK_OP_KKT ? p->kkt_len() : p->state_len();
  return bk::gmres_workspace_bytes(n, restart, p->dtype);
}

bk_status krylov_solve(bk_problem* prob, int op, const void* rhs, void* sol, const bk_krylov_opts* opts,
                       bk_krylov_info* info, void* workspace, void* stream) {
  BK_ARG(prob != nullptr && rhs != nullptr && sol != nullptr && info != nullptr, "NULL argument");
  BK_ARG(op == BK_OP_STATE || op == BK_OP_KKT, "unknown operator %d", op);
  bk::Problem* p = reinterpret_cast<bk::Problem*>(prob);
  bk_krylov_opts o = opts ? *opts : bk::krylov_defaults();
  if (o.rtol <= 0) o.rtol = 1e-10;
  if (o.restart <= 0) o.restart = 30;
  if (o.max_iter <= 0) o.max_iter = 300;
  memset(info, 0, sizeof(*info));
  BK_TRY(bk::gmres(p, p->work(), op, rhs, sol, o, info, workspace, (cudaStream_t)stream));
  if (!info->converged) {
    bk::set_error("GMRES stopped after %d iterations at relative residual %.3e", info->iterations, info->rel_resid);
    return BK_ERR_NOT_CONVERGED;
  }
  return BK_OK;
}

}  // extern "C"
