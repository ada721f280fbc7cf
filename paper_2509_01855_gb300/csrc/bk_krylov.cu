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
// operand made the FP32 passes slower than the FP64 ones. The (m+1) x m Hessenberg matrix and its Givens rotations
// live on the host (FP64); the iteration reads back j+3 numbers per step.
#include <math.h>
#include <string.h>

#include <vector>

#include "bk_krylov.cuh"

namespace bk {

static constexpr int DOT_BLOCKS = 608;   // 4 blocks per SM on 152 SMs, fixed for determinism
static constexpr int MAXM = 100;

// FP32 elements per thread summed in FP32 before each FP64 accumulation.
constexpr int RUN32 = 16;

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
__global__ void __launch_bounds__(256) k_multidot(const T* __restrict__ V, int64_t ld, int nv, const T* __restrict__ w,
                                                  int64_t n, double* __restrict__ partial, double* __restrict__ out,
                                                  unsigned* __restrict__ cnt) {
  __shared__ double red[8][8];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t lo = blockIdx.x * chunk;
  const int64_t hi = lo + chunk < n ? lo + chunk : n;
  for (int i0 = 0; i0 < nv; i0 += 8) {
    const int ng = nv - i0 < 8 ? nv - i0 : 8;
    const T* Vg = V + (int64_t)i0 * ld;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
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
  if (last_block(cnt))
    for (int i = 0; i < nv; ++i) block_sum_column(partial, gridDim.x, nv, i, out + i);
}

// w <- alpha * w + cscale * sum_i c[i] V_i   (c on the device, FP64). With `partial`, each block
// also writes the sum of squares of its slice of the new w and the last block to finish writes
// their sum, |w|^2, to *sq_out (block order, as k_multidot).
template <typename T>
__global__ void __launch_bounds__(256) k_multiaxpy(const T* __restrict__ V, int64_t ld, int nv,
                                                   const double* __restrict__ c, double cscale, T* __restrict__ w,
                                                   double alpha, int64_t n, double* __restrict__ partial,
                                                   double* __restrict__ sq_out = nullptr,
                                                   unsigned* __restrict__ cnt = nullptr) {
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
  if constexpr (sizeof(T) == 8) {
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
  b += es * (size_t)ld * 2;                  // z scratch and r / correction
  b += sizeof(double) * (size_t)DOT_BLOCKS * (MAXM + 2);  // dot partials
  b += sizeof(double) * 4 * (MAXM + 2);      // device scalars
  return b + 1024;
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
  double* partial = (double*)carve(sizeof(double) * DOT_BLOCKS * (MAXM + 2));
  double* dvec = (double*)carve(sizeof(double) * 4 * (MAXM + 2));
  double* h1 = dvec;
  double* h2 = dvec + (MAXM + 2);
  double* yv = dvec + 2 * (MAXM + 2);
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
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
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
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int j = 0;
    for (; j < m && total < o.max_iter; ++j) {
      T* vj = V + (int64_t)j * ld;
      T* w = V + (int64_t)(j + 1) * ld;
      if (o.use_precond) {
        T* zj = Zb + (int64_t)j * ld;
        if (weighted) {
          BK_TRY(wscale(vj, z, 1));
          BK_TRY(op_precond(pr, d, op, z, zj, 0, st));
        } else {
          BK_TRY(op_precond(pr, d, op, vj, zj, 0, st));
        }
        BK_TRY(op_apply(pr, d, op, zj, w, st, aux ? (void*)(aux->T + (int64_t)j * aux->ld) : nullptr));
        if (weighted) BK_TRY(wscale(w, w, 0));
      } else {
        BK_TRY(op_apply(pr, d, op, vj, w, st, aux ? (void*)(aux->T + (int64_t)j * aux->ld) : nullptr));
      }
      // Gram-Schmidt (DGKS): h1 = [V_0..V_j]^T w and |w|^2 (w = V_{j+1} follows V_j), then
      // w <- w - V h1 with the new |w|^2; a second pass only on cancellation.
      BK_TRY(dots<T>(V, ld, j + 2, w, n, partial, h1, cnt, st));
      k_multiaxpy<T><<<DOT_BLOCKS, 256, 0, st>>>(V, ld, j + 1, h1, -1.0, w, 1.0, n, partial, h2 + (MAXM + 1), cnt + 1);
      BK_CHECK_LAUNCH();
      BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, h1, sizeof(double) * (j + 2), cudaMemcpyDeviceToHost, st));
      BK_TRY_CUDA(cudaMemcpyAsync(hostbuf + (MAXM + 2), h2 + (MAXM + 1), sizeof(double), cudaMemcpyDeviceToHost, st));
      BK_TRY_CUDA(cudaStreamSynchronize(st));
      double w2 = hostbuf[MAXM + 2];
      for (int i = 0; i <= j; ++i) H[i * m + j] = hostbuf[i];
      if (w2 < 0.5 * hostbuf[j + 1]) {
        BK_TRY(dots<T>(V, ld, j + 1, w, n, partial, h2, cnt, st));
        k_multiaxpy<T><<<DOT_BLOCKS, 256, 0, st>>>(V, ld, j + 1, h2, -1.0, w, 1.0, n, partial, h2 + (MAXM + 1), cnt + 1);
        BK_CHECK_LAUNCH();
        BK_TRY_CUDA(cudaMemcpyAsync(hostbuf, h2, sizeof(double) * (MAXM + 2), cudaMemcpyDeviceToHost, st));
        BK_TRY_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i <= j; ++i) H[i * m + j] += hostbuf[i];
        w2 = hostbuf[MAXM + 1];
      }
      const double hnext = sqrt(w2);
      H[(j + 1) * m + j] = hnext;
      ++total;
      // normalise v_{j+1}
      if (hnext > 0.0) {
        hostbuf[0] = hnext;
        BK_TRY_CUDA(cudaMemcpyAsync(h1, hostbuf, sizeof(double), cudaMemcpyHostToDevice, st));
        k_scale_inv<T><<<g, 256, 0, st>>>(w, h1, w, n);
        BK_CHECK_LAUNCH();
      }
      // Givens
      for (int i = 0; i < j; ++i) {
        const double a = H[i * m + j], c = H[(i + 1) * m + j];
        H[i * m + j] = cs[i] * a + sn[i] * c;
        H[(i + 1) * m + j] = -sn[i] * a + cs[i] * c;
      }
      const double a = H[j * m + j], c = H[(j + 1) * m + j];
      const double den = hypot(a, c);
      cs[j] = den == 0.0 ? 1.0 : a / den;
      sn[j] = den == 0.0 ? 0.0 : c / den;
      H[j * m + j] = den;
      H[(j + 1) * m + j] = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      resid = fabs(gv[j + 1]);
      if (resid <= target || hnext == 0.0) { ++j; break; }
    }
    // y = H(0:j,0:j)^{-1} g
    for (int i = j - 1; i >= 0; --i) {
      double a = gv[i];
      for (int q = i + 1; q < j; ++q) a -= H[i * m + q] * y[q];
      y[i] = a / H[i * m + i];
    }
    BK_TRY_CUDA(cudaMemcpyAsync(yv, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
    // x += Z y (flexible form; Z = V without preconditioning)
    k_multiaxpy<T><<<g, 256, 0, st>>>(o.use_precond ? Zb : V, ld, j, yv, 1.0, x, 1.0, n, nullptr);
    BK_CHECK_LAUNCH();
    if (aux) {
      k_multiaxpy<double><<<grid_for(aux->n), 256, 0, st>>>(aux->T, aux->ld, j, yv, 1.0, aux->Td, 1.0, aux->n, nullptr);
      BK_CHECK_LAUNCH();
    }
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
