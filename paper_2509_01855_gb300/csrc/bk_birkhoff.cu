// Birkhoff products B v and B^T v on the CGL grid (FastBV and its transpose).
//
// Paper: "Fast Computation of Birkhoff Matrix-Vector Products" (Eqs. vi=sumT .. chatk=,
// algorithms Fasta2v / FastBV) and Appendix B (Fastv2a).
//
// Formulation used by the kernels. Let R be the unnormalised type-I DCT of length N+1,
//   R(x)_k = x_0 + (-1)^k x_N + 2 sum_{m=1}^{N-1} x_m cos(pi k m / N),
// which is twice the paper's DCT-I (Eq. vm=DCT-1). Write Y = R(v). The Chebyshev coefficients
// of Fastv2a are a_k = (-1)^k h_k Y_k / N (h = 1/2 at k = 0, N), and the sign (-1)^k that the
// reversal steps of Fastv2a / Fasta2v introduce cancels inside the integration stencil of
// Eq. c_k=bydef, so with chat'_k = (-1)^k chat_k:
//   chat'_1     = (Y_2 - Y_0) / (2N)
//   chat'_k     = (Y_{k+1} - Y_{k-1}) / (2kN),                 2 <= k <= N-2
//   chat'_{N-1} = (Y_N/2 - Y_{N-2}) / (2(N-1)N) - (Y_N/2) / (2(N+1)N)   (aliasing fold, Eq. chatk=)
//   chat'_N     = -Y_{N-1} / (2N^2)
// and the nodal values are y'_i = sum_k chat'_k cos(pi k i / N) = R(g)_i with g_0 = 0,
// g_k = chat'_k / 2 (0 < k < N), g_N = chat'_N. The constant coefficient c_0 is not formed:
// row 0 of B^a is zero (B^a_j(tau^a) = 0, Eq. birk-conditions), and c_0 multiplies T_0 = 1,
// so B^a v = y' - y'_0. With the time scale s = (tf - t0)/2:  B v = s (y' - y'_0 1).
// Transpose: B = s (I - 1 e_0^T) R G R / N with R = C W (C symmetric, W = diag(1,2,..,2,1)),
// so B^T u = (s/N) W R W^{-1} G^T W R W^{-1} (I - e_0 1^T) u, and R W^{-1} (I - e_0 1^T) u =
// R(W^{-1} u) - (sum u) 1 because column 0 of R is all ones and sum_m (W^{-1}u)_ext = sum u.
//
// The DCT-I is computed by a complex FFT of length N of z_j = x_ext[2j] + i x_ext[2j+1]
// (x_ext the even 2N-periodic extension of x) and the standard real-FFT split:
//   Y_k = P + Q,  Y_{N-k} = P - Q,  P = Re(Z_k + Z_{N-k}) / 2,
//   Q = [cos(pi k/N) Im(Z_k + Z_{N-k}) - sin(pi k/N) Re(Z_k - Z_{N-k})] / 2.
// N <= NSMALL: one CTA per vector does the whole chain in shared memory (one HBM read and one
// write). Larger N: four-step FFT (N = N1 N2) in two passes per DCT, the integration stencil
// fused into the load of the second DCT, and the node-0 value gathered from per-CTA partials.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "bk_common.cuh"
#include "bk_fft.cuh"
#include "bk_plan.cuh"

namespace bk {

// The kernels compute in T and keep their internal real vectors (the stage buffers between the
// two DCTs) in T; the caller's vectors are User<T> (binary64 for double-float arithmetic, whose
// products convert the input once in k_to_arith and the output in the last epilogue).
template <typename T> using St = T;
template <typename T> using Us = typename User<T>::t;
// Conversion of a stored element S to the arithmetic type T and back (identity when S == T).
template <typename T, typename S> struct Cv;
template <typename T> struct Cv<T, T> {
  static __device__ __forceinline__ T in(T x) { return x; }
  static __device__ __forceinline__ T out(T x) { return x; }
};
template <> struct Cv<dfl, double> {
  static __device__ __forceinline__ dfl in(double x) { return d2df(x); }
  static __device__ __forceinline__ double out(dfl x) { return df2d(x); }
};
// Pass-B output type: the caller's type for the final epilogues, T for the stage buffer.
template <typename T, int E> struct OutS {
  typedef typename std::conditional<(E == 2 || E == 3), Us<T>, T>::type t;
};
template <typename T, typename S> __device__ __forceinline__ T rdv(const S* __restrict__ p, int64_t i) {
  return Cv<T, S>::in(p[i]);
}

#ifndef BK_TRANSFORM_KERNEL_UNIT  // one definition of the library's globals, in the main unit
// (bk_birkhoff_f64.cu and bk_birkhoff_f32.cu include this file for the transform kernels only)
static thread_local std::string g_last_error = "no error";
static std::atomic<unsigned long long> g_launches{0};
// When set (by the creating thread), dmalloc adds every allocation's size to it: plans and
// problems report their device footprint this way.
static thread_local size_t* g_alloc_acc = nullptr;

AllocCounter::AllocCounter(size_t* acc) : prev(g_alloc_acc) { g_alloc_acc = acc; }
AllocCounter::~AllocCounter() { g_alloc_acc = prev; }

static thread_local unsigned long long t_launches = 0;
void note_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
unsigned long long thread_launches() { return t_launches; }
void note_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

bk_status dmalloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return BK_OK;
  if (g_alloc_acc) *g_alloc_acc += bytes;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? BK_ERR_OOM : BK_ERR_CUDA;
  }
  return BK_OK;
}

void dfree(void* p) {
  if (p) cudaFree(p);
}

#endif  // BK_TRANSFORM_KERNEL_UNIT

// ---------------------------------------------------------------------------------------------
// Table construction (device, FP64 sincospi; FP32 tables are rounded copies)
// ---------------------------------------------------------------------------------------------
template <typename T>
__global__ void k_tw_table(typename V2<T>::t* tw, int64_t n, double denom_half_turns) {
  // tw[i] = (cos(2 pi i / n), -sin(2 pi i / n)) computed as sincospi(2 i / n)
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi((double)(2 * i) / denom_half_turns, &s, &c);
    tw[i] = mk2<T>((T)c, (T)(-s));
  }
}

// tw[i] = omega_n^{i * stride}, i < count (sincospi of 2 i stride / n)
template <typename T>
__global__ void k_tw_table_strided(typename V2<T>::t* tw, int64_t count, int64_t stride, double n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi((double)(2 * i * stride) / n, &s, &c);
    tw[i] = mk2<T>((T)c, (T)(-s));
  }
}

template <typename T>
__global__ void k_post_table(typename V2<T>::t* tp, int64_t N) {
  // tp[k] = (cos(pi k / N), sin(pi k / N)), k = 0..N/2
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= N / 2;
       k += (int64_t)gridDim.x * blockDim.x) {
    double s, c;
    sincospi((double)k / (double)N, &s, &c);
    tp[k] = mk2<T>((T)c, (T)s);
  }
}

// Stage twiddle table of a length-2^log2n FFT (see bk_fft.cuh): entry off + (r-1) Ns + k of the
// block of the stage with Ns = 2^l is omega_{16 Ns}^{r k}, from sincospi(2 r k / (16 Ns)).
template <typename T>
__global__ void k_stage_tw(typename V2<T>::t* stw, int log2n, int len) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < len; idx += gridDim.x * blockDim.x) {
    int l = (log2n & 3) ? (log2n & 3) : 4, off = 0;
    while (idx >= off + (15 << l)) { off += 15 << l; l += 4; }
    const int e = idx - off;
    const int r = (e >> l) + 1, k = e & ((1 << l) - 1);
    double sn, cs;
    sincospi((double)(2 * r * k) / (double)(16 << l), &sn, &cs);
    stw[idx] = mk2<T>((T)cs, (T)(-sn));
  }
}

// rk[k] = 1 / (4k), k >= 1 (rk[0] = 0), rounded once from FP64.
template <typename T>
__global__ void k_rk_table(T* rk, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    rk[k] = k == 0 ? T(0) : (T)(1.0 / (4.0 * (double)k));
}

// Bluestein chirp w_j = exp(-i pi j^2 / N) = (cos, -sin)(pi r / N), r = j^2 mod 2N in integers.
template <typename T>
__global__ void k_chirp(typename V2<T>::t* w, int64_t N) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = (j * j) % (2 * N);
    double sn, cs;
    sincospi((double)r / (double)N, &sn, &cs);
    w[j] = mk2<T>((T)cs, (T)(-sn));
  }
}

// The convolution kernel b of Bluestein's identity, scaled by 1/M, as M complex values (real
// pairs): b_m = conj(w_m) for m < N, b_{M-m} = conj(w_m) for 0 < m < N, zero between.
template <typename T>
__global__ void k_bs_kernel(T* b, int64_t N, int64_t M) {
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = m < N ? m : (m > M - N ? M - m : -1);
    double sn = 0.0, cs = 0.0;
    if (j >= 0) sincospi((double)((j * j) % (2 * N)) / (double)N, &sn, &cs);
    b[2 * m] = (T)(cs / (double)M);
    b[2 * m + 1] = (T)(sn / (double)M);
  }
}

#ifndef BK_TRANSFORM_KERNEL_UNIT
__global__ void k_grid_tables(double* t_nodes, int64_t N, double t0, double s) {
  // tau_j = -cos(j pi / N) = sin(pi (2j - N) / (2N)) (Eq. CGLpts), t_j = t0 + s (tau_j + 1)
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j <= N;
       j += (int64_t)gridDim.x * blockDim.x) {
    double tau = sinpi((double)(2 * j - N) / (double)(2 * N));
    if (j == 0) tau = -1.0;
    if (j == N) tau = 1.0;
    t_nodes[j] = t0 + s * (tau + 1.0);
  }
}
#endif  // BK_TRANSFORM_KERNEL_UNIT

// ---------------------------------------------------------------------------------------------
// Element accessors of the transform inputs
// ---------------------------------------------------------------------------------------------
// Kinds of the first-DCT input x:
//   IN_PLAIN : x_m = v_m                  (forward product)
//   IN_WINV  : x_m = v_m / W_m            (transpose product; W = 1 at the ends, 2 inside)
// Kinds of the second-DCT input (from Y = output of the first DCT):
//   ST_FWD   : x_m = g_m = G(Y)_m                          (forward stencil, includes 1/N)
//   ST_TRN   : x_m = W_m^{-1} G^T(W (Y - Y_0))_m          (transposed stencil)
enum { IN_PLAIN = 0, IN_WINV = 1, ST_FWD = 2, ST_TRN = 3 };

// rk[k] = 1 / (4k) for 1 <= k <= N + 1 (plan table): the stencils multiply instead of divide.
template <typename T, typename S>
__device__ __forceinline__ T stencil_fwd(const S* __restrict__ Y, int m, int N, T invN, const T* __restrict__ rk) {
  // g_m = chat'_m / 2 for 0 < m < N, g_N = chat'_N, g_0 = 0 (see the file comment). invN is 1/N,
  // or 1 where Y was stored already divided by N.
  if (m == 0) return T(0);
  if (m == N) return -rdv<T>(Y, N - 1) * (invN * T(2) * rk[N]);
  if (m == 1) return (rdv<T>(Y, 2) - rdv<T>(Y, 0)) * (invN * T(0.25));
  if (m == N - 1) {
    const T yN = rdv<T>(Y, N);
    return (T(0.5) * yN - rdv<T>(Y, N - 2)) * (invN * rk[N - 1]) - yN * (invN * T(0.5) * rk[N + 1]);
  }
  return (rdv<T>(Y, m + 1) - rdv<T>(Y, m - 1)) * (invN * rk[m]);
}

template <typename T, typename S>
__device__ __forceinline__ T stencil_trn(const S* __restrict__ Qs, int m, int N, T Y0, const T* __restrict__ rk,
                                         T cN) {
  auto Q = [&](int i) { return rdv<T>(Qs, i); };
  // r = W (Y - Y0); t = G^T r; return t_m / W_m. G^T rows:
  //   t_0 = -r_1/4, t_1 = -r_2/8, t_j = r_{j-1}/(4(j-1)) - r_{j+1}/(4(j+1)) (2<=j<=N-2),
  //   t_{N-1} = r_{N-2}/(4(N-2)) - r_N/(2N), t_N = r_{N-1}/(4(N^2-1)).
  // r_k = 2 (Y_k - Y0) for 0 < k < N, r_0 = Y_0 - Y0 = 0, r_N = Y_N - Y0.
  // cN = 1 / (4 (N^2 - 1))
  if (m == 0) return -(T(2) * (Q(1) - Y0)) * T(0.25);
  if (m == N) return (T(2) * (Q(N - 1) - Y0)) * cN;
  T t;
  if (m == 1) {
    t = -(T(2) * (Q(2) - Y0)) * T(0.125);
  } else if (m == N - 1) {
    t = (T(2) * (Q(N - 2) - Y0)) * rk[N - 2] - (Q(N) - Y0) * (T(2) * rk[N]);
  } else {
    t = (Q(m - 1) - Y0) * rk[m - 1] - (Q(m + 1) - Y0) * rk[m + 1];
    return t;
  }
  return T(0.5) * t;
}

// Value x_m of the transform input of kind K. `src` is the vector (first DCT) or the stage
// buffer Y (second DCT). Y0 is used by ST_TRN only.
// Stencil constants passed to the transform kernels.
template <typename T> struct StencilTab {
  const T* rk;  // rk[k] = 1/(4k), k = 1..N+1
  T cN;         // 1/(4(N^2 - 1))
};

template <typename T, int K, typename S>
__device__ __forceinline__ T load_x(const S* __restrict__ src, int m, int N, T invN, T Y0, StencilTab<T> tb) {
  if (K == IN_PLAIN) return rdv<T>(src, m);
  if (K == IN_WINV) return (m == 0 || m == N) ? rdv<T>(src, m) : T(0.5) * rdv<T>(src, m);
  if (K == ST_FWD) return stencil_fwd<T>(src, m, N, invN, tb.rk);
  return stencil_trn<T>(src, m, N, Y0, tb.rk, tb.cN);
}

// z_j = x_ext[2j] + i x_ext[2j+1]
template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t load_z(const S* __restrict__ src, int j, int N, T invN,
                                                    T Y0, StencilTab<T> tb) {
  const int m1 = 2 * j, m2 = 2 * j + 1;
  const int i1 = m1 <= N ? m1 : 2 * N - m1;
  const int i2 = m2 <= N ? m2 : 2 * N - m2;
  return mk2<T>(load_x<T, K>(src, i1, N, invN, Y0, tb), load_x<T, K>(src, i2, N, invN, Y0, tb));
}

// Split DCT-I (four-step plans): the DCT-I of length N+1 of x is, at even indices, the DCT-I of
// length M+1 (M = N/2) of the pair sums a_i = x_i + x_{N-i} (a_M = 2 x_M) and, at odd indices
// 2m+1, the DCT-III of length M, sum_{i<M} u_i cos(pi i (2m+1) / (2M)), of the pair differences
// u_0 = x_0 - x_N, u_i = 2 (x_i - x_{N-i}). Pass-A load modes:
//   PM_FULL : the unsplit length-N FFT input (load_z)
//   PM_PAIR : z_j of the length-M DCT-I of the pair sums (n = M)
//   PM_DCT3 : conj Z_k (k < n = M/2) of the DCT-III by a length-M/2 inverse FFT (Makhoul):
//             H_0 = u_0, H_k = e^{i theta k} (u_k - i u_{M-k}) / 2 (theta = pi / (2M) = pi / N,
//             u_M = 0), Z_k = (H_k + conj H_{M/2-k}) + i e^{2 pi i k / M} (H_k - conj H_{M/2-k});
//             the inverse FFT runs as conj(FFT(conj Z)).
// Two-level split (largest plans): the even half's DCT-I of length M+1 of a is split once more,
// so R(x)_{4m} is the DCT-I of length Q+1 (Q = N/4) of aa_i = a_i + a_{M-i}, R(x)_{4m+2} the
// DCT-III of length Q of u'_0 = a_0 - a_M, u'_i = 2 (a_i - a_{M-i}), and R(x)_{2m+1} the
// DCT-III of x's pair differences as above: FFTs of N/4 + N/8 + N/4 points instead of
// N/2 + N/4. The pair sums a are formed on the fly from x in the loads:
//   PM_PAIR2 : z_j of the length-Q DCT-I of aa (n = Q)
//   PM_DCT3A : conj Z_k (k < n = Q/2) of the DCT-III of u' (as PM_DCT3, on a)
//   PM_CPLX  : a plain complex vector (pairs of reals) of length n (Bluestein's convolution)
enum { PM_FULL = 0, PM_PAIR = 1, PM_DCT3 = 2, PM_PAIR2 = 3, PM_DCT3A = 4, PM_CPLX = 5 };

template <typename T, int K, typename S>
__device__ __forceinline__ T pair_sum(const S* __restrict__ src, int i, int Ns) {
  // a_i = x_i + x_{Ns-i}; IN_WINV halves interior samples (i = 0 pairs the two end samples)
  const T a = rdv<T>(src, i) + rdv<T>(src, Ns - i);
  return (K == IN_WINV && i != 0) ? T(0.5) * a : a;
}

template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t load_z_pair(const S* __restrict__ src, int j, int n, StencilTab<T> tb) {
  const int Ns = 2 * n;
  const int m1 = 2 * j, m2 = 2 * j + 1;
  const int i1 = m1 <= n ? m1 : 2 * n - m1;
  const int i2 = m2 <= n ? m2 : 2 * n - m2;
  return mk2<T>(pair_sum<T, K>(src, i1, Ns), pair_sum<T, K>(src, i2, Ns));
}

// H_k of the DCT-III input (see above), with the factors folded: for k >= 1 every sample is an
// interior one, so H_k = c e^{i theta k} ((x_k - x_{N-k}) - i (x_{M-k} - x_{M+k})) with c = 1
// (IN_PLAIN) or 1/2 (IN_WINV halves interior samples); H_0 = u_0 = W-scaled x_0 - x_N.
template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t dct3_H(const S* __restrict__ src, int i, int M,
                                                   const typename V2<T>::t* __restrict__ tpost) {
  const int N = 2 * M;
  if (i == 0) return mk2<T>(rdv<T>(src, 0) - rdv<T>(src, N), T(0));
  const T a = rdv<T>(src, i) - rdv<T>(src, N - i), b = rdv<T>(src, M - i) - rdv<T>(src, M + i);
  typename V2<T>::t cs = tpost[i];  // (cos, sin)(pi i / N)
  if (K == IN_WINV) { cs.x *= T(0.5); cs.y *= T(0.5); }
  return mk2<T>(a * cs.x + b * cs.y, a * cs.y - b * cs.x);
}

template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t load_z_dct3(const S* __restrict__ src, int k, int n,
                                                        const typename V2<T>::t* __restrict__ tpost,
                                                        const typename V2<T>::t* __restrict__ eo, StencilTab<T> tb) {
  typedef typename V2<T>::t C;
  const int M = 2 * n;
  const C Hk = dct3_H<T, K>(src, k, M, tpost);
  const C Hm = dct3_H<T, K>(src, n - k, M, tpost);  // H_{M/2 - k}; conj taken below
  const C E = mk2<T>(Hk.x + Hm.x, Hk.y - Hm.y);
  const C D = mk2<T>(Hk.x - Hm.x, Hk.y + Hm.y);
  const C w = eo[k];  // omega_M^k; e^{2 pi i k / M} = conj w
  const C O = mk2<T>(D.x * w.x + D.y * w.y, D.y * w.x - D.x * w.y);
  return mk2<T>(E.x - O.y, -(E.y + O.x));
}

// z_j of the length-Q DCT-I of aa (n = Q, x of length 4Q + 1): aa_i = a_i + a_{2Q-i}.
template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t load_z_pair2(const S* __restrict__ src, int j, int n) {
  const int Nf = 4 * n, M = 2 * n;
  const int m1 = 2 * j, m2 = 2 * j + 1;
  const int i1 = m1 <= n ? m1 : 2 * n - m1;
  const int i2 = m2 <= n ? m2 : 2 * n - m2;
  return mk2<T>(pair_sum<T, K>(src, i1, Nf) + pair_sum<T, K>(src, M - i1, Nf),
                pair_sum<T, K>(src, i2, Nf) + pair_sum<T, K>(src, M - i2, Nf));
}

// H_k of the DCT-III of length Q of u' (pair differences of a, x of length 4Q + 1): as dct3_H on
// a with theta = pi / (2Q), (cos, sin)(pi i / (2Q)) = tpost[2i]; a carries the W^{-1} scaling of
// IN_WINV already, so the factor c is 1.
template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t dct3_H_pairs(const S* __restrict__ src, int i, int Q,
                                                         const typename V2<T>::t* __restrict__ tpost) {
  const int M = 2 * Q, Nf = 4 * Q;
  if (i == 0) return mk2<T>(pair_sum<T, K>(src, 0, Nf) - pair_sum<T, K>(src, M, Nf), T(0));
  const T a = pair_sum<T, K>(src, i, Nf) - pair_sum<T, K>(src, M - i, Nf);
  const T b = pair_sum<T, K>(src, Q - i, Nf) - pair_sum<T, K>(src, Q + i, Nf);
  const typename V2<T>::t cs = tpost[2 * i];
  return mk2<T>(a * cs.x + b * cs.y, a * cs.y - b * cs.x);
}

template <typename T, int K, typename S>
__device__ __forceinline__ typename V2<T>::t load_z_dct3a(const S* __restrict__ src, int k, int n,
                                                         const typename V2<T>::t* __restrict__ tpost,
                                                         const typename V2<T>::t* __restrict__ eo) {
  typedef typename V2<T>::t C;
  const int Q = 2 * n;
  const C Hk = dct3_H_pairs<T, K>(src, k, Q, tpost);
  const C Hm = dct3_H_pairs<T, K>(src, n - k, Q, tpost);
  const C E = mk2<T>(Hk.x + Hm.x, Hk.y - Hm.y);
  const C D = mk2<T>(Hk.x - Hm.x, Hk.y + Hm.y);
  const C w = eo[2 * k];  // the table is built for the DCT-III of length 2Q
  const C O = mk2<T>(D.x * w.x + D.y * w.y, D.y * w.x - D.x * w.y);
  return mk2<T>(E.x - O.y, -(E.y + O.x));
}

// Real-FFT split: from Z_k, Z_{N-k} and (cos, sin)(pi kk / N), kk = min(k, N - k).
template <typename T>
__device__ __forceinline__ void split_pair(typename V2<T>::t zk, typename V2<T>::t zc,
                                           typename V2<T>::t cs, T& yk, T& ynk) {
  const T P = T(0.5) * (zk.x + zc.x);
  const T Q = T(0.5) * (cs.x * (zk.y + zc.y) - cs.y * (zk.x - zc.x));
  yk = P + Q;
  ynk = P - Q;
}

// ---------------------------------------------------------------------------------------------
// Single-CTA fused kernel: the whole chain for one vector in shared memory.
// ---------------------------------------------------------------------------------------------
template <typename T>
__device__ void dct1_block(const T* __restrict__ X, int kind, T* __restrict__ Y,
                           typename V2<T>::t* buf, int N, int log2N,
                           const typename V2<T>::t* __restrict__ tw, const typename V2<T>::t* __restrict__ stw,
                           const typename V2<T>::t* __restrict__ tpost, T invN, T Y0, StencilTab<T> tb) {
  typedef typename V2<T>::t C;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    C z;
    switch (kind) {
      case IN_PLAIN: z = load_z<T, IN_PLAIN>(X, j, N, invN, Y0, tb); break;
      case IN_WINV: z = load_z<T, IN_WINV>(X, j, N, invN, Y0, tb); break;
      case ST_FWD: z = load_z<T, ST_FWD>(X, j, N, invN, Y0, tb); break;
      default: z = load_z<T, ST_TRN>(X, j, N, invN, Y0, tb); break;
    }
    buf[padi(j)] = z;
  }
  __syncthreads();
  if (N >= 16) {
    fft16_any<T>(buf, N, log2N, 1, pad_stride(N), stw);
  } else {
    // N = 4 or 8: direct DFT (tw holds omega_N^i, n_tab = N)
    C zk = mk2<T>(T(0), T(0));
    const int k = threadIdx.x;
    if (k < N) {
      for (int j = 0; j < N; ++j) zk = cadd(zk, cmul(buf[padi(j)], tw[(j * k) & (N - 1)]));
    }
    __syncthreads();
    if (k < N) buf[padi(k)] = zk;
    __syncthreads();
  }
  for (int k = threadIdx.x; k <= N / 2; k += blockDim.x) {
    const C zk = buf[padi(k)];
    const C zc = buf[padi((N - k) & (N - 1))];
    T yk, ynk;
    split_pair<T>(zk, zc, tpost[k], yk, ynk);
    Y[k] = yk;
    if (k != N / 2) Y[N - k] = ynk;
  }
  __syncthreads();
}

// Thread cap of the transform kernels: each thread stages 16 complex values, so FP64 kernels
// are limited to 256 threads (up to 255 registers each) and FP32 ones to 512.
template <typename T> struct MaxThr { static constexpr int v = sizeof(T) == 8 ? 256 : 512; };
// Resident CTAs per SM the pass kernels are compiled for (register cap 64K / (threads x this)).
// Double-float: 3 (80 registers instead of 128, spills unchanged at ~50 bytes, 24 instead of 16
// warps per SM for the 128-thread tiles; the latency-bound passes gained: 4-component products
// 2^20 0.553 -> 0.519 ms, 2^22 2.48 -> 2.11 ms; 4 CTAs (64 registers) lost: 0.576, 2.33 ms).
// binary32 at 3 would cap the 512-thread tiles at 42 registers and spill ~400 bytes.
template <typename T> struct MinB { static constexpr int v = std::is_same<T, dfl>::value ? 3 : 2; };
// Element loads each thread keeps in flight in the pass kernels' load phases.
// FP32: 8 (latency-bound passes; 16 spilled under the 64-register cap of two 512-thread CTAs
// per SM), FP64: 4 (FP64-pipe-bound, register-heavy).
template <typename T> struct InFlight { static constexpr int v = sizeof(T) == 8 ? 4 : 8; };

// Whole chain for vector vec in one CTA (every value independent of the CTA's thread count, so
// a batched launch with more threads gives the same results).
template <typename T, bool TRANS>
__device__ __forceinline__ void small_body(int vec, const Us<T>* __restrict__ in, Us<T>* __restrict__ out, int N,
                                           int log2N, int64_t pitch, T s, const typename V2<T>::t* __restrict__ tw,
                                           const typename V2<T>::t* __restrict__ stw,
                                           const typename V2<T>::t* __restrict__ tpost, StencilTab<T> tb) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = N + 1;
  const int Lp = (L + 3) & ~3;
  T* X = reinterpret_cast<T*>(smem);
  T* Y = X + Lp;
  C* buf = reinterpret_cast<C*>(Y + Lp);
  const int64_t base = (int64_t)vec * pitch;
  const Us<T>* src = in + base;
  Us<T>* dst = out + base;
  typedef Cv<T, Us<T>> CV;
  const T invN = T(1.0 / (double)N);
  for (int m = threadIdx.x; m < L; m += blockDim.x) X[m] = CV::in(src[m]);
  __syncthreads();
  if (!TRANS) {
    dct1_block<T>(X, IN_PLAIN, Y, buf, N, log2N, tw, stw, tpost, invN, T(0), tb);
    dct1_block<T>(Y, ST_FWD, X, buf, N, log2N, tw, stw, tpost, invN, T(0), tb);
    const T y0 = X[0];
    for (int m = threadIdx.x; m < L; m += blockDim.x) dst[m] = CV::out(s * (X[m] - y0));
  } else {
    dct1_block<T>(X, IN_WINV, Y, buf, N, log2N, tw, stw, tpost, invN, T(0), tb);
    const T y0 = Y[0];
    dct1_block<T>(Y, ST_TRN, X, buf, N, log2N, tw, stw, tpost, invN, y0, tb);
    const T sN = s * invN;
    for (int m = threadIdx.x; m < L; m += blockDim.x)
      dst[m] = CV::out((m == 0 || m == N) ? sN * X[m] : T(2) * sN * X[m]);
  }
  for (int m = L + threadIdx.x; m < pitch; m += blockDim.x) dst[m] = Us<T>(0);
}

template <typename T, bool TRANS>
__global__ void __launch_bounds__(MaxThr<T>::v)
    k_birkhoff_small(const Us<T>* __restrict__ in, Us<T>* __restrict__ out, int N, int log2N, int64_t pitch,
                     T s, const typename V2<T>::t* __restrict__ tw, const typename V2<T>::t* __restrict__ stw,
                     const typename V2<T>::t* __restrict__ tpost, StencilTab<T> tb) {
  small_body<T, TRANS>(blockIdx.x, in, out, N, log2N, pitch, s, tw, stw, tpost, tb);
}

// ---------------------------------------------------------------------------------------------
// Four-step passes for large N (N = N1 * N2, j = N2 j1 + j2, k = k1 + N1 k2).
// Pass A: per CTA, NB columns j2; FFT over j1 (length N1), twiddle omega_N^{j2 k1}; writes
//         A[k1][j2]. Also writes the CTA's partial sum of Re z + Im z (the DC value of the DCT).
// Pass B: per CTA, P row pairs {p, N1 - p} (p = 0 pairs rows 0 and N1/2); FFT over j2 (length
//         N2), real-FFT split, epilogue.
// ---------------------------------------------------------------------------------------------
template <typename T, int K, int MODE>
__device__ __forceinline__ void passA_body(
            int bid, int nbid, const St<T>* __restrict__ src, int64_t src_stride, typename V2<T>::t* __restrict__ Aout,
            T* __restrict__ partial, int N, int N1, int log2N1, int N2, int NB, int bs,
            const typename V2<T>::t* __restrict__ stw,
            const typename V2<T>::t* __restrict__ twN, T invN, StencilTab<T> tb,
            const typename V2<T>::t* __restrict__ twLo,
            const typename V2<T>::t* __restrict__ twHi, int tw_h,
            const typename V2<T>::t* __restrict__ tpost, const typename V2<T>::t* __restrict__ eo,
            int vec_in = -1, int nthr_in = 0) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem[];
  C* buf = reinterpret_cast<C*>(smem);
  // FP32: sub-FFT twiddles in shared memory after the tile (FP64 reads the global table)
  C* tws = buf + (size_t)NB * bs;
  const bool smem_tw = sizeof(T) == 4;
  if (smem_tw) load_tw_smem<T>(tws, stw, stage_tw_len(log2N1));
  __shared__ T red[32];
  // vector and working thread count: blockIdx.y and blockDim.x, or given by a batched launch
  // (whose CTAs may have more threads than this plan's; the extra ones only meet the barriers,
  // so that the DC partial sums keep this plan's order)
  const int vec = vec_in >= 0 ? vec_in : (int)blockIdx.y;
  const int nt = nthr_in > 0 ? nthr_in : (int)blockDim.x;
  const St<T>* x = src + (int64_t)vec * src_stride;
  const int c0 = bid * NB;
  const int log2NB = __ffs(NB) - 1, log2N2 = __ffs(N2) - 1;  // NB, N2 are powers of two
  // The stage buffer read by the second DCT already holds Y / N (forward) or Y - Y0
  // (transpose), so its stencils run with scale 1 and Y0 = 0 (constants the compiler folds).
  const T Y0 = T(0);
  const T sc = K == ST_FWD ? T(1) : invN;
  // DC partials: consumed after IN_WINV (the transposed stage) and ST_FWD (the forward output);
  // in split plans the DC value is the even half's (the DCT-III has none)
  constexpr bool DC = (K == IN_WINV || K == ST_FWD) && MODE != PM_DCT3 && MODE != PM_DCT3A;
  T dc = T(0);
  const int total = NB * N1;
  // independent element loads in flight per thread before the shared-memory stores
  constexpr int LD = InFlight<T>::v;
  for (int idx0 = (int)threadIdx.x < nt ? (int)threadIdx.x : total; idx0 < total; idx0 += LD * nt) {
    C z[LD];
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < total) {
        const int b = idx & (NB - 1);
        const int j = ((idx >> log2NB) << log2N2) + c0 + b;
        if (MODE == PM_FULL) z[u] = load_z<T, K>(x, j, N, sc, Y0, tb);
        else if (MODE == PM_CPLX) z[u] = mk2<T>(x[2 * (int64_t)j], x[2 * (int64_t)j + 1]);
        else if (MODE == PM_PAIR) z[u] = load_z_pair<T, K>(x, j, N, tb);
        else if (MODE == PM_PAIR2) z[u] = load_z_pair2<T, K>(x, j, N);
        else if (MODE == PM_DCT3A) z[u] = load_z_dct3a<T, K>(x, j, N, tpost, eo);
        else z[u] = load_z_dct3<T, K>(x, j, N, tpost, eo, tb);
      }
    }
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int idx = idx0 + u * nt;
      if (idx < total) {
        if (DC) dc += z[u].x + z[u].y;
        buf[(idx & (NB - 1)) * bs + padi(idx >> log2NB)] = z[u];
      }
    }
  }
  if (DC) {
    // block reduction of dc (deterministic order)
    for (int o = 16; o > 0; o >>= 1) dc += shfl_xor(dc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dc;
  }
  __syncthreads();
  if (DC && threadIdx.x < 32) {
    T a = (int)threadIdx.x < (nt >> 5) ? red[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) a += shfl_xor(a, o);
    if (threadIdx.x == 0) partial[(int64_t)vec * nbid + bid] = a;
  }
  fft16_any<T>(buf, N1, log2N1, NB, bs, smem_tw ? tws : stw);
  C* A = Aout + (int64_t)vec * N;
  // inter-pass twiddles omega_N^{j2 k1}, 4 independent table loads in flight per thread.
  // FP64: one table of omega_N^m (the FP64 pipe, not memory, bounds these kernels).
  // FP32: omega_N^m = omega_N^{(m >> h) 2^h} omega_N^{m mod 2^h} from two tables of ~sqrt N.
  for (int idx0 = threadIdx.x; idx0 < total; idx0 += 4 * blockDim.x) {
    C w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = idx0 + u * blockDim.x;
      if (idx < total) {
        const int m = (c0 + (idx & (NB - 1))) * (idx >> log2NB);  // < N
        w[u] = sizeof(T) == 8 ? ldg(&twN[m]) : cmul(ldg(&twHi[m >> tw_h]), ldg(&twLo[m & ((1 << tw_h) - 1)]));
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = idx0 + u * blockDim.x;
      if (idx < total) {
        const int b = idx & (NB - 1);
        const int k1 = idx >> log2NB;
        A[(int64_t)k1 * N2 + c0 + b] = cmul(buf[b * bs + padi(k1)], w[u]);
      }
    }
  }
}

#define BK_PASSA_PARAMS(S)                                                                           \
  const St<T>* __restrict__ src##S, int64_t src_stride##S, typename V2<T>::t* __restrict__ Aout##S,          \
      T* __restrict__ partial##S, int N##S, int N1##S, int log2N1##S, int N2##S, int NB##S, int bs##S,      \
      const typename V2<T>::t* __restrict__ stw##S, const typename V2<T>::t* __restrict__ twN##S,           \
      const typename V2<T>::t* __restrict__ twLo##S, const typename V2<T>::t* __restrict__ twHi##S, int tw_h##S
#define BK_PASSA_ARGS(S)                                                                             \
  src##S, src_stride##S, Aout##S, partial##S, N##S, N1##S, log2N1##S, N2##S, NB##S, bs##S, stw##S, twN##S
#define BK_PASSA_TAIL(S) twLo##S, twHi##S, tw_h##S

// Pass A of one transform (unsplit, or one half of a split DCT-I).
template <typename T, int K, int MODE = PM_FULL>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v)
    k_passA(BK_PASSA_PARAMS(), T invN, StencilTab<T> tb, const typename V2<T>::t* __restrict__ tpost = nullptr,
            const typename V2<T>::t* __restrict__ eo = nullptr) {
  passA_body<T, K, MODE>(blockIdx.x, gridDim.x, BK_PASSA_ARGS(), invN, tb, BK_PASSA_TAIL(), tpost, eo);
}

// Pass A of both halves of a split DCT-I in one launch: CTAs [0, gE) run the even half (pair
// sums), the rest the odd half (DCT-III); one launch fills the GPU better than two smaller ones.
template <typename T, int K>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v)
    k_passA_split(int gE, BK_PASSA_PARAMS(E), BK_PASSA_PARAMS(O), T invN, StencilTab<T> tb,
                  const typename V2<T>::t* __restrict__ tpost, const typename V2<T>::t* __restrict__ eo) {
  if ((int)blockIdx.x < gE)
    passA_body<T, K, PM_PAIR>(blockIdx.x, gE, BK_PASSA_ARGS(E), invN, tb, BK_PASSA_TAIL(E), tpost, eo);
  else
    passA_body<T, K, PM_DCT3>(blockIdx.x - gE, gridDim.x - gE, BK_PASSA_ARGS(O), invN, tb, BK_PASSA_TAIL(O), tpost, eo);
}

// Pass A of the three parts of a two-level split DCT-I in one launch: CTAs [0, g1) the DCT-I of
// aa, [g1, g1 + g2) the DCT-III of a's pair differences, the rest the DCT-III of x's.
template <typename T, int K>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v)
    k_passA_split3(int g1, int g2, BK_PASSA_PARAMS(E), BK_PASSA_PARAMS(D), BK_PASSA_PARAMS(O), T invN,
                   StencilTab<T> tb, const typename V2<T>::t* __restrict__ tpost,
                   const typename V2<T>::t* __restrict__ eo) {
  const int b = blockIdx.x;
  if (b < g1)
    passA_body<T, K, PM_PAIR2>(b, g1, BK_PASSA_ARGS(E), invN, tb, BK_PASSA_TAIL(E), tpost, eo);
  else if (b < g1 + g2)
    passA_body<T, K, PM_DCT3A>(b - g1, g2, BK_PASSA_ARGS(D), invN, tb, BK_PASSA_TAIL(D), tpost, eo);
  else
    passA_body<T, K, PM_DCT3>(b - g1 - g2, gridDim.x - g1 - g2, BK_PASSA_ARGS(O), invN, tb, BK_PASSA_TAIL(O), tpost,
                              eo);
}

// Second-DCT input as its own elementwise pass (planned applies): x_m of kind K (ST_FWD with
// scale sc, or ST_TRN) for every m <= N, written to G, with per-CTA partial sums of W_m x_m
// (the DC value R(x)_0 of the DCT, W = 1 at the ends, 2 inside) when `partial` is given. Fusing
// the stencil into the pass-A loads instead exposes its neighbour loads: those passes ran
// 25-40% longer than plain-load ones.
// (bid, nbid, vec: block, blocks per vector and vector, from the launch or a batched launch;
// 256 threads.)
template <typename T, int K>
__device__ __forceinline__ void stencil_body(int bid, int nbid, int vec, const St<T>* __restrict__ stage, int64_t Ls,
                                             St<T>* __restrict__ G, int N, T sc, StencilTab<T> tb,
                                             T* __restrict__ partial) {
  __shared__ T red[8];
  const St<T>* Y = stage + (int64_t)vec * Ls;
  St<T>* g = G + (int64_t)vec * Ls;
  typedef Cv<T, St<T>> CV;
  T acc = T(0);
  // interior nodes 2..N-2 by the plain three-point formulas (the boundary cases, if-converted
  // into the same loop, tripled its FP64 instructions); the four boundary nodes by one thread
  const T* __restrict__ rk = tb.rk;
  for (int m = 2 + bid * blockDim.x + threadIdx.x; m <= N - 2; m += nbid * blockDim.x) {
    const T ym = CV::in(Y[m - 1]), yp = CV::in(Y[m + 1]);
    const T x = K == ST_FWD ? (yp - ym) * (sc * rk[m]) : ym * rk[m - 1] - yp * rk[m + 1];
    g[m] = CV::out(x);
    acc += T(2) * x;
  }
  if (bid == 0 && threadIdx.x == 0) {
    const int mb[4] = {0, 1, N - 1, N};
    for (int i = 0; i < 4; ++i) {
      const T x = load_x<T, K>(Y, mb[i], N, sc, T(0), tb);
      g[mb[i]] = CV::out(x);
      acc += (mb[i] == 0 || mb[i] == N) ? x : T(2) * x;
    }
  }
  if (partial) {
    for (int o = 16; o > 0; o >>= 1) acc += shfl_xor(acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      T a = T(0);
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += red[w];
      partial[(int64_t)vec * nbid + bid] = a;
    }
  }
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_stencil(const St<T>* __restrict__ stage, int64_t Ls, St<T>* __restrict__ G, int N,
                                                 T sc, StencilTab<T> tb, T* __restrict__ partial) {
  stencil_body<T, K>(blockIdx.x, gridDim.x, blockIdx.y, stage, Ls, G, N, sc, tb, partial);
}

// Caller's vectors (pitch apart) converted to the arithmetic type T, Ls apart (double-float
// products: one conversion per element instead of one per load in the transform passes).
template <typename T>
__global__ void __launch_bounds__(256) k_to_arith(const Us<T>* __restrict__ v, int64_t pitch, T* __restrict__ x,
                                                  int64_t Ls) {
  const Us<T>* src = v + (int64_t)blockIdx.y * pitch;
  T* dst = x + (int64_t)blockIdx.y * Ls;
  for (int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; m < Ls; m += (int64_t)gridDim.x * blockDim.x)
    dst[m] = Cv<T, Us<T>>::in(src[m]);
}

// Epilogue kinds of pass B:
//   EP_STORE     : stage[k] = Y_k / N                      (after the first DCT, forward)
//   EP_STORE_TRN : stage[k] = Y_k - Y0, Y0 from partials   (after the first DCT, transpose)
//   EP_FWD_OUT   : out[k] = s (Y_k - Y0), Y0 from partials (after the second DCT, forward)
//   EP_TRN_OUT   : out[k] = (s/N) W_k Y_k                   (after the second DCT, transpose)
//   EP_CPLX      : dst[k] = Z_k                          (PB_CPLX: a plain complex FFT)
//   EP_CPLX_MC   : dst[k] = conj(Z_k tab[k])             (PB_CPLX: spectral product, conjugated)
enum { EP_STORE = 0, EP_STORE_TRN = 1, EP_FWD_OUT = 2, EP_TRN_OUT = 3, EP_CPLX = 4, EP_CPLX_MC = 5 };

template <typename T, int E, typename S>
__device__ __forceinline__ void ep_write(S* __restrict__ dst, int k, T yk, int N, T s, T Y0, T invN) {
  typedef Cv<T, S> CV;
  if (E == EP_STORE) dst[k] = CV::out(yk * invN);
  else if (E == EP_STORE_TRN) dst[k] = CV::out(yk - Y0);
  else if (E == EP_FWD_OUT) dst[k] = CV::out(s * (yk - Y0));
  else dst[k] = CV::out((k == 0 || k == N) ? s * invN * yk : T(2) * s * invN * yk);
}

// ---------------------------------------------------------------------------------------------
// N that is not a power of two (N > 1024): Bluestein's identity j k = (j^2 + k^2 - (k - j)^2)/2
// turns the length-N complex DFT Z = DFT_N(z) of the DCT-I into a circular convolution of
// length M (a power of two, M >= 2N - 1), run by the four-step FFT passes above in their plain
// complex modes:
//   a_j = z_j w_j (j < N, 0 up to M),  w_j = e^{-i pi j^2 / N} (j^2 reduced mod 2N in integers),
//   c = IFFT_M(FFT_M(a) . Bh),  Bh = FFT_M(b) / M,  b_m = conj(w_m) = b_{M-m} (|m| < N, else 0),
//   Z_k = w_k c_k.
// The inverse FFT runs as conj(FFT(conj .)): the first FFT's pass B stores conj(A . Bh), the
// second FFT is a forward one, and the post kernel takes conj of its output. Then the real-FFT
// split gives the DCT-I outputs Y_k (k = 0..N) as for powers of two, with Y_0 = Re Z_0 + Im Z_0.
// ---------------------------------------------------------------------------------------------
// a = z w zero-padded to M (one complex per element), z_j from the input kind K (IN_PLAIN / IN_WINV).
template <typename T, int K>
__global__ void __launch_bounds__(256) k_bs_pre(const St<T>* __restrict__ src, int64_t sstride, int N, int64_t M,
                                                const typename V2<T>::t* __restrict__ w, T* __restrict__ a) {
  typedef typename V2<T>::t C;
  const St<T>* x = src + (int64_t)blockIdx.y * sstride;
  T* dst = a + (int64_t)blockIdx.y * 2 * M;
  StencilTab<T> tb;
  tb.rk = nullptr;
  tb.cN = T(0);
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    C r = mk2<T>(T(0), T(0));
    if (j < N) r = cmul(load_z<T, K>(x, (int)j, N, T(1), T(0), tb), w[j]);
    dst[2 * j] = r.x;
    dst[2 * j + 1] = r.y;
  }
}

// DCT-I outputs from the second FFT's output y (M complex per vector): Z_k = w_k conj(y_k), the
// real-FFT split of (Z_k, Z_{N-k}) for k <= N/2, and the epilogue E (Y0 = Y_0 = Re Z_0 + Im Z_0).
template <typename T, int E>
__global__ void __launch_bounds__(256) k_bs_post(const T* __restrict__ y, int64_t M, int N,
                                                 const typename V2<T>::t* __restrict__ w,
                                                 const typename V2<T>::t* __restrict__ tpost,
                                                 typename OutS<T, E>::t* __restrict__ dst, int64_t dstride,
                                                 int64_t zero_to, T s, T invN) {
  typedef typename V2<T>::t C;
  const T* yv = y + (int64_t)blockIdx.y * 2 * M;
  typename OutS<T, E>::t* out = dst + (int64_t)blockIdx.y * dstride;
  auto Z = [&](int k) {  // w_k conj(y_k)
    const C yk = mk2<T>(yv[2 * (int64_t)k], -yv[2 * (int64_t)k + 1]);
    return cmul(w[k], yk);
  };
  const C z0 = Z(0);
  const T Y0 = z0.x + z0.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= N / 2; k += gridDim.x * blockDim.x) {
    const int kc = k == 0 ? 0 : N - k;
    T yk, ynk;
    split_pair<T>(Z(k), Z(kc), tpost[k], yk, ynk);
    ep_write<T, E>(out, k, yk, N, s, Y0, invN);
    if (N - k != k) ep_write<T, E>(out, N - k, ynk, N, s, Y0, invN);
  }
  if ((E == EP_FWD_OUT || E == EP_TRN_OUT) && blockIdx.x == 0) {
    for (int64_t m = N + 1 + threadIdx.x; m < zero_to; m += blockDim.x) out[m] = typename OutS<T, E>::t(0);
  }
}

// Pass-B modes: PB_PAIRS, row pairs {p, N1 - p} and the real-FFT split of a DCT-I (outputs at
// ostride k of a transform of parent size Npar; (cos, sin)(pi k / n) read as tpost[tps k]);
// PB_ROWS, plain rows of the DCT-III's inverse FFT (outputs unpacked to the odd indices of the
// sub-transform, ostride (2m+1) of the whole one).
// PB_CPLX, plain rows of a complex FFT written in natural order k = k1 + N1 k2 as complex pairs
// (epilogues EP_CPLX, EP_CPLX_MC; `tpost` then holds the spectral table).
enum { PB_PAIRS = 0, PB_ROWS = 1, PB_CPLX = 2 };

template <typename T, int E, int MODE>
__device__ __forceinline__ void passB_body(
            int bid, const typename V2<T>::t* __restrict__ Ain, typename OutS<T, E>::t* __restrict__ dst, int64_t dst_stride,
            int64_t pitch_zero_to, const T* __restrict__ partial, int n_partial, int N, int N1,
            int N2, int log2N2, int P, const typename V2<T>::t* __restrict__ stw,
            const typename V2<T>::t* __restrict__ tpost, T s, T invN, int ostride, int tps, int Npar,
            int vec_in = -1, int nthr_in = 0) {
  typedef typename V2<T>::t C;
  extern __shared__ __align__(16) unsigned char smem[];
  const int bs = pad_stride(N2);
  C* buf = reinterpret_cast<C*>(smem);
  C* tws = buf + (size_t)2 * P * bs;
  const bool smem_tw = sizeof(T) == 4;
  if (smem_tw) load_tw_smem<T>(tws, stw, stage_tw_len(log2N2));
  __shared__ T red[32];
  // as in passA_body: a batched launch gives the vector and this plan's thread count
  const int vec = vec_in >= 0 ? vec_in : (int)blockIdx.y;
  const int nt = nthr_in > 0 ? nthr_in : (int)blockDim.x;
  const C* A = Ain + (int64_t)vec * N;
  typename OutS<T, E>::t* out = dst + (int64_t)vec * dst_stride;
  const int p0 = bid * P;
  T Y0 = T(0);
  if (E == EP_STORE_TRN || E == EP_FWD_OUT) {
    T acc = T(0);
    const T* pp = partial + (int64_t)vec * n_partial;
    for (int i = (int)threadIdx.x < nt ? (int)threadIdx.x : n_partial; i < n_partial; i += nt) acc += pp[i];
    for (int o = 16; o > 0; o >>= 1) acc += shfl_xor(acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
      T a = (int)threadIdx.x < (nt >> 5) ? red[threadIdx.x] : T(0);
      for (int o = 16; o > 0; o >>= 1) a += shfl_xor(a, o);
      if (threadIdx.x == 0) red[0] = a;
    }
    __syncthreads();
    Y0 = red[0];
  }
  // load 2P rows: PB_PAIRS local row q = 2 i (+1) for pair p0 + i; PB_ROWS rows 2 p0 + q
  const int total = 2 * P * N2;
  constexpr int LD = InFlight<T>::v;
  for (int idx0 = threadIdx.x; idx0 < total; idx0 += LD * blockDim.x) {
    C z[LD];
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int idx = idx0 + u * blockDim.x;
      if (idx < total) {
        const int q = idx >> log2N2;
        int row;
        if (MODE == PB_ROWS || MODE == PB_CPLX) {
          row = 2 * p0 + q;
        } else {
          const int p = p0 + (q >> 1);
          row = (q & 1) == 0 ? p : (p == 0 ? N1 / 2 : N1 - p);
        }
        z[u] = A[((int64_t)row << log2N2) + (idx & (N2 - 1))];
      }
    }
#pragma unroll
    for (int u = 0; u < LD; ++u) {
      const int idx = idx0 + u * blockDim.x;
      if (idx < total) {
        const int q = idx >> log2N2;
        buf[q * bs + padi(idx & (N2 - 1))] = z[u];
      }
    }
  }
  __syncthreads();
  fft16_any<T>(buf, N2, log2N2, 2 * P, bs, smem_tw ? tws : stw);
  if constexpr (MODE == PB_CPLX) {
    // lanes take consecutive rows, so each store run covers 2P consecutive outputs
    const int log2R = __ffs(2 * P) - 1;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int q = idx & (2 * P - 1);
      const int k2 = idx >> log2R;
      C R = buf[q * bs + padi(k2)];
      const int64_t k = (int64_t)(2 * p0 + q) + (int64_t)N1 * k2;
      if (E == EP_CPLX_MC) {
        const C t = cmul(R, tpost[k]);
        R.x = t.x;
        R.y = -t.y;
      }
      out[2 * k] = R.x;
      out[2 * k + 1] = R.y;
    }
    return;
  }
  if (MODE == PB_ROWS) {
    // output p = k1 + N1 k2 of the inverse FFT is z_p = conj(result): r_{2p} = Re, r_{2p+1} = -Im;
    // X_{2j} = r_j, X_{2j+1} = r_{M-1-j} (j < M/2 = N), and Y_{2m+1} = X_m
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int q = idx >> log2N2;
      const int k2 = idx & (N2 - 1);
      const C R = buf[q * bs + padi(k2)];
      const int64_t pz = (int64_t)(2 * p0 + q) + (int64_t)N1 * k2;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int64_t r = 2 * pz + t;
        const int64_t m = r < N ? 2 * r : 2 * (2 * (int64_t)N - 1 - r) + 1;
        ep_write<T, E>(out, (int)(ostride * (2 * m + 1)), t == 0 ? R.x : -R.y, Npar, s, Y0, invN);
      }
    }
    return;
  }
  const int half = N / 2;
  // Row pair i of the CTA and column k2 give outputs k = p0 + i + N1 k2 and N - k: lanes take
  // consecutive i (P-long runs of consecutive outputs) and load 4 split twiddles at a time.
  const int log2P = __ffs(P) - 1;  // P is a power of two
  for (int idx0 = threadIdx.x; idx0 < P * N2; idx0 += 4 * blockDim.x) {
    C cs[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = idx0 + u * blockDim.x;
      const int k = p0 + (idx & (P - 1)) + N1 * (idx >> log2P);
      if (idx < P * N2 && p0 + (idx & (P - 1)) != 0) cs[u] = tpost[(k <= half ? k : N - k) * tps];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = idx0 + u * blockDim.x;
      if (idx >= P * N2) continue;
      const int i = idx & (P - 1);
      const int k2 = idx >> log2P;
      const int p = p0 + i;
      const C* ra = buf + (2 * i) * bs;
      const C* rb = buf + (2 * i + 1) * bs;
      if (p == 0) {
        // row 0 pairs internally (k2 <-> N2 - k2); row N1/2 pairs k2 <-> N2 - 1 - k2
        if (k2 <= N2 / 2) {
          const int k = N1 * k2;
          T yk, ynk;
          split_pair<T>(ra[padi(k2)], ra[padi((N2 - k2) & (N2 - 1))], tpost[k * tps], yk, ynk);
          ep_write<T, E>(out, k * ostride, yk, Npar, s, Y0, invN);
          if (k != half) ep_write<T, E>(out, (N - k) * ostride, ynk, Npar, s, Y0, invN);
        }
        if (k2 < N2 / 2) {
          const int k = N1 / 2 + N1 * k2;
          T yk, ynk;
          split_pair<T>(rb[padi(k2)], rb[padi(N2 - 1 - k2)], tpost[k * tps], yk, ynk);
          ep_write<T, E>(out, k * ostride, yk, Npar, s, Y0, invN);
          ep_write<T, E>(out, (N - k) * ostride, ynk, Npar, s, Y0, invN);
        }
      } else {
        const int k = p + N1 * k2;
        const C zk = ra[padi(k2)];
        const C zc = rb[padi(N2 - 1 - k2)];
        T yk, ynk;
        if (k <= half) {
          split_pair<T>(zk, zc, cs[u], yk, ynk);
        } else {
          split_pair<T>(zc, zk, cs[u], ynk, yk);
        }
        ep_write<T, E>(out, k * ostride, yk, Npar, s, Y0, invN);
        ep_write<T, E>(out, (N - k) * ostride, ynk, Npar, s, Y0, invN);
      }
    }
  }
  // zero the padding of the output vectors (final epilogues only)
  if ((E == EP_FWD_OUT || E == EP_TRN_OUT) && bid == 0) {
    for (int64_t m = Npar + 1 + threadIdx.x; m < pitch_zero_to; m += blockDim.x) out[m] = typename OutS<T, E>::t(0);
  }
}

#define BK_PASSB_PARAMS(S)                                                                           \
  const typename V2<T>::t* __restrict__ Ain##S, int N##S, int N1##S, int N2##S, int log2N2##S, int P##S, \
      const typename V2<T>::t* __restrict__ stw##S

template <typename T, int E, int MODE = PB_PAIRS>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v)
    k_passB(const typename V2<T>::t* __restrict__ Ain, typename OutS<T, E>::t* __restrict__ dst, int64_t dst_stride,
            int64_t pitch_zero_to, const T* __restrict__ partial, int n_partial, int N, int N1,
            int N2, int log2N2, int P, const typename V2<T>::t* __restrict__ stw,
            const typename V2<T>::t* __restrict__ tpost, T s, T invN, int ostride, int tps, int Npar) {
  passB_body<T, E, MODE>(blockIdx.x, Ain, dst, dst_stride, pitch_zero_to, partial, n_partial, N, N1, N2, log2N2, P, stw,
                         tpost, s, invN, ostride, tps, Npar);
}

// Pass B of both halves of a split DCT-I in one launch: CTAs [0, gE) the even half's row pairs
// and real split (outputs at even indices), the rest the odd half's rows (odd indices).
template <typename T, int E>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v)
    k_passB_split(int gE, BK_PASSB_PARAMS(E), BK_PASSB_PARAMS(O), typename OutS<T, E>::t* __restrict__ dst, int64_t dst_stride,
                  int64_t pitch_zero_to, const T* __restrict__ partial, int n_partial,
                  const typename V2<T>::t* __restrict__ tpost, T s, T invN, int Npar) {
  if ((int)blockIdx.x < gE)
    passB_body<T, E, PB_PAIRS>(blockIdx.x, AinE, dst, dst_stride, pitch_zero_to, partial, n_partial, NE, N1E, N2E,
                               log2N2E, PE, stwE, tpost, s, invN, 2, 2, Npar);
  else
    passB_body<T, E, PB_ROWS>(blockIdx.x - gE, AinO, dst, dst_stride, 0, partial, n_partial, NO, N1O, N2O, log2N2O,
                              PO, stwO, tpost, s, invN, 1, 1, Npar);
}

// Pass B of a two-level split: the DCT-I of aa (outputs 4k), the DCT-III of a's pair
// differences (outputs 4m + 2) and the DCT-III of x's (outputs 2m + 1).
template <typename T, int E>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v)
    k_passB_split3(int h1, int h2, BK_PASSB_PARAMS(E), BK_PASSB_PARAMS(D), BK_PASSB_PARAMS(O), typename OutS<T, E>::t* __restrict__ dst,
                   int64_t dst_stride, int64_t pitch_zero_to, const T* __restrict__ partial, int n_partial,
                   const typename V2<T>::t* __restrict__ tpost, T s, T invN, int Npar) {
  const int b = blockIdx.x;
  if (b < h1)
    passB_body<T, E, PB_PAIRS>(b, AinE, dst, dst_stride, pitch_zero_to, partial, n_partial, NE, N1E, N2E, log2N2E, PE,
                               stwE, tpost, s, invN, 4, 4, Npar);
  else if (b < h1 + h2)
    passB_body<T, E, PB_ROWS>(b - h1, AinD, dst, dst_stride, 0, partial, n_partial, ND, N1D, N2D, log2N2D, PD, stwD,
                              tpost, s, invN, 2, 2, Npar);
  else
    passB_body<T, E, PB_ROWS>(b - h1 - h2, AinO, dst, dst_stride, 0, partial, n_partial, NO, N1O, N2O, log2N2O, PO,
                              stwO, tpost, s, invN, 1, 1, Npar);
}

// ---------------------------------------------------------------------------------------------
// Batched launches over plans of different N (birkhoff_apply_batch): one launch per pass covers
// up to BATCH_MAX plans. A job is one plan's part of a launch (its vectors, CTAs per vector and
// shapes); CTA b of the launch belongs to the job q with start[q] <= b < start[q + 1] and runs
// that job's body with that plan's own thread count, so every value it writes is the one the
// plan's own launch writes. The descriptors travel as __grid_constant__ kernel parameters.
// ---------------------------------------------------------------------------------------------
constexpr int BATCH_MAX = 16;

template <typename T> struct SmallJob {
  const T* in;
  T* out;
  int64_t pitch;
  const typename V2<T>::t* tw;
  const typename V2<T>::t* stw;
  const typename V2<T>::t* tpost;
  StencilTab<T> tb;
  T s;
  int N, log2N, nblk;
};

template <typename T> struct PassAJob {
  const T* src;
  int64_t sstride;
  typename V2<T>::t* A;
  T* partial;
  const typename V2<T>::t* stw;
  const typename V2<T>::t* twN;
  const typename V2<T>::t* twLo;
  const typename V2<T>::t* twHi;
  StencilTab<T> tb;
  T invN;
  int N, N1, log2N1, N2, NB, bs, tw_h, nthr, nblk;
};

template <typename T> struct PassBJob {
  const typename V2<T>::t* A;
  T* dst;
  int64_t dstride, zero_to;
  const T* partial;
  const typename V2<T>::t* stw;
  const typename V2<T>::t* tpost;
  T s, invN;
  int npartial, N, N1, N2, log2N2, P, nthr, nblk;
};

template <typename T> struct StencilJob {
  const T* stage;
  T* G;
  T* partial;
  int64_t Ls;
  StencilTab<T> tb;
  int N, nblk;
};

template <typename J> struct Batch {
  int njob;
  int start[BATCH_MAX + 1];   // first CTA of each job; start[njob] = the launch's CTAs
  J j[BATCH_MAX];
};

template <typename J>
__device__ __forceinline__ int batch_job(const Batch<J>& b, int cta) {
  int q = 0;
  while (q + 1 < b.njob && cta >= b.start[q + 1]) ++q;
  return q;
}

template <typename T, bool TRANS>
__global__ void __launch_bounds__(MaxThr<T>::v) k_small_batch(const __grid_constant__ Batch<SmallJob<T>> b) {
  const int q = batch_job(b, blockIdx.x);
  const SmallJob<T>& J = b.j[q];
  small_body<T, TRANS>((int)blockIdx.x - b.start[q], J.in, J.out, J.N, J.log2N, J.pitch, J.s, J.tw, J.stw, J.tpost,
                       J.tb);
}

template <typename T, int K>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v) k_passA_batch(const __grid_constant__ Batch<PassAJob<T>> b) {
  const int q = batch_job(b, blockIdx.x);
  const PassAJob<T>& J = b.j[q];
  const int local = (int)blockIdx.x - b.start[q];
  const int vec = local / J.nblk;
  passA_body<T, K, PM_FULL>(local - vec * J.nblk, J.nblk, J.src, J.sstride, J.A, J.partial, J.N, J.N1, J.log2N1, J.N2,
                            J.NB, J.bs, J.stw, J.twN, J.invN, J.tb, J.twLo, J.twHi, J.tw_h, nullptr, nullptr, vec,
                            J.nthr);
}

template <typename T, int E>
__global__ void __launch_bounds__(MaxThr<T>::v, MinB<T>::v) k_passB_batch(const __grid_constant__ Batch<PassBJob<T>> b) {
  const int q = batch_job(b, blockIdx.x);
  const PassBJob<T>& J = b.j[q];
  const int local = (int)blockIdx.x - b.start[q];
  const int vec = local / J.nblk;
  passB_body<T, E, PB_PAIRS>(local - vec * J.nblk, J.A, J.dst, J.dstride, J.zero_to, J.partial, J.npartial, J.N, J.N1,
                             J.N2, J.log2N2, J.P, J.stw, J.tpost, J.s, J.invN, 1, 1, J.N, vec, J.nthr);
}

template <typename T, int K>
__global__ void __launch_bounds__(256) k_stencil_batch(const __grid_constant__ Batch<StencilJob<T>> b) {
  const int q = batch_job(b, blockIdx.x);
  const StencilJob<T>& J = b.j[q];
  const int local = (int)blockIdx.x - b.start[q];
  const int vec = local / J.nblk;
  stencil_body<T, K>(local - vec * J.nblk, J.nblk, vec, J.stage, J.Ls, J.G, J.N, T(1), J.tb, J.partial);
}

// ---------------------------------------------------------------------------------------------
// Plan creation / destruction and the apply entry points
// ---------------------------------------------------------------------------------------------
// Stage tables and the inter-pass twiddle table of one four-step layout.
template <typename T>
static bk_status build_fs_tables(FourStep& f, cudaStream_t st) {
  typedef typename V2<T>::t C;
  for (int w = 0; w < 2; ++w) {
    const int n = w == 0 ? f.N1 : f.N2;
    void** dst = w == 0 ? &f.stw1 : &f.stw2;
    const int len = stage_tw_len(ilog2(n));
    if (len == 0) continue;
    BK_TRY(dmalloc(dst, sizeof(C) * len));
    k_stage_tw<T><<<(len + 255) / 256, 256, 0, st>>>((C*)*dst, ilog2(n), len);
    BK_CHECK_LAUNCH();
  }
  const int64_t n = f.n;
  if (sizeof(T) == 8) {
    BK_TRY(dmalloc(&f.twN, sizeof(C) * n));
    k_tw_table<T><<<(int)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>((C*)f.twN, n, (double)n);
    BK_CHECK_LAUNCH();
  } else {
    const int log2n = ilog2(n);
    f.tw_h = (log2n + 1) / 2;
    const int64_t nlo = int64_t(1) << f.tw_h, nhi = n >> f.tw_h;
    BK_TRY(dmalloc(&f.twLo, sizeof(C) * nlo));
    BK_TRY(dmalloc(&f.twHi, sizeof(C) * nhi));
    k_tw_table<T><<<(int)((nlo + 255) / 256), 256, 0, st>>>((C*)f.twLo, nlo, (double)n);
    BK_CHECK_LAUNCH();
    k_tw_table_strided<T><<<(int)((nhi + 255) / 256), 256, 0, st>>>((C*)f.twHi, nhi, nlo, (double)n);
    BK_CHECK_LAUNCH();
  }
  return BK_OK;
}

static void free_fs(FourStep& f) {
  dfree(f.stw1);
  dfree(f.stw2);
  dfree(f.twN);
  dfree(f.twLo);
  dfree(f.twHi);
  f = FourStep();
}

template <typename T>
static bk_status build_tables(Plan* p, cudaStream_t st) {
  typedef typename V2<T>::t C;
  const int64_t N = p->N;
  // FFT twiddles: single-CTA plans keep omega_N^i (direct DFT for N < 16) and the stage table of
  // N; four-step plans the stage tables of N1 and N2.
  auto stage_table = [&](void** dst, int64_t n) -> bk_status {
    const int len = stage_tw_len(ilog2(n));
    if (len == 0) return BK_OK;
    BK_TRY(dmalloc(dst, sizeof(C) * len));
    k_stage_tw<T><<<(len + 255) / 256, 256, 0, st>>>((C*)*dst, ilog2(n), len);
    BK_CHECK_LAUNCH();
    return BK_OK;
  };
  if (p->blue) {
    BK_TRY(build_fs_tables<T>(p->fsM, st));
    BK_TRY(dmalloc(&p->chirp, sizeof(C) * N));
    k_chirp<T><<<(int)std::min<int64_t>((N + 255) / 256, 4096), 256, 0, st>>>((C*)p->chirp, N);
    BK_CHECK_LAUNCH();
    BK_TRY(dmalloc(&p->bh, sizeof(C) * p->M));   // filled by blue_spectrum once the kernels are set up
  } else if (p->small) {
    BK_TRY(dmalloc(&p->tw, sizeof(C) * N));
    k_tw_table<T><<<(int)std::min<int64_t>((N + 255) / 256, 4096), 256, 0, st>>>((C*)p->tw, N, (double)N);
    BK_CHECK_LAUNCH();
    if (N >= 16) BK_TRY(stage_table(&p->stwS, N));
  } else {
    BK_TRY(build_fs_tables<T>(p->fs, st));
    if (p->split) {
      BK_TRY(build_fs_tables<T>(p->fso, st));
      if (p->split == 2) BK_TRY(build_fs_tables<T>(p->fse, st));
      const int64_t M = N / 2;
      BK_TRY(dmalloc(&p->eo, sizeof(C) * (M / 2)));
      // exp(+2 pi i k / M) = conj(omega_M^k)
      k_tw_table<T><<<(int)std::min<int64_t>((M / 2 + 255) / 256, 4096), 256, 0, st>>>((C*)p->eo, M / 2, (double)M);
      BK_CHECK_LAUNCH();
    }
  }
  BK_TRY(dmalloc(&p->rk, sizeof(T) * (N + 2)));
  k_rk_table<T><<<(int)std::min<int64_t>((N + 2 + 255) / 256, 4096), 256, 0, st>>>((T*)p->rk, N + 2);
  BK_CHECK_LAUNCH();
  BK_TRY(dmalloc(&p->tpost, sizeof(C) * (N / 2 + 1)));
  k_post_table<T><<<(int)std::min<int64_t>((N / 2 + 256) / 256, 4096), 256, 0, st>>>((C*)p->tpost, N);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

#ifndef BK_TRANSFORM_KERNEL_UNIT
__global__ void k_unit_last(double* e, int64_t L, int64_t pitch) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pitch; i += (int64_t)gridDim.x * blockDim.x)
    e[i] = (i == L - 1) ? 1.0 : 0.0;
}
__global__ void k_d2f(const double* a, float* b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// Clenshaw-Curtis weights as the last row of B^a: w = (B^a)^T e_N, computed in FP64 with the
// transpose product itself (O(N log N)). A BK_F32 plan uses a temporary FP64 plan.
static bk_status compute_weights(Plan* p, cudaStream_t st) {
  const int64_t L = p->L;
  Plan* q = p;
  Plan* tmp = nullptr;
  if (p->dtype != BK_F64) {
    BK_TRY(plan_create(&tmp, p->N, 1, 1, BK_F64, 0.0, 2.0, 0, st));
    q = tmp;
  }
  double* e = nullptr;
  bk_status r = dmalloc((void**)&e, sizeof(double) * q->pitch);
  if (r == BK_OK) r = dmalloc((void**)&p->w64, sizeof(double) * q->pitch);
  if (r == BK_OK) {
    k_unit_last<<<(int)((q->pitch + 255) / 256), 256, 0, st>>>(e, L, q->pitch);
    note_launch();
    r = cudaGetLastError() == cudaSuccess ? plan_apply_n(q, e, p->w64, 1, true, 1.0, st) : BK_ERR_CUDA;
  }
  if (r == BK_OK && p->dtype == BK_F32) {
    r = dmalloc(&p->wT, sizeof(float) * L);
    if (r == BK_OK) {
      k_d2f<<<(int)((L + 255) / 256), 256, 0, st>>>(p->w64, (float*)p->wT, L);
      note_launch();
    }
  }
  if (r == BK_OK && cudaStreamSynchronize(st) != cudaSuccess) { set_error("weights: sync failed"); r = BK_ERR_CUDA; }
  dfree(e);
  if (tmp) plan_destroy(tmp);
  return r;
}
#endif  // BK_TRANSFORM_KERNEL_UNIT

// Largest N run by the single-CTA kernel (one CTA per vector): 128 in FP64, whose single CTA
// runs on one SM's FP64 pipe (4 components, cold L2, B / four-step ms: 2^8 0.062 / 0.056,
// 2^10 0.089 / 0.068, 2^11 0.097 / 0.074), 4096 in FP32 (2^12 0.034 / 0.038, 2^13 0.044 /
// 0.042). BK_SMALL_MAX_LOG2 overrides it for tuning (at least 2^4; at most the shared-memory
// limit of 4096 in FP64, 8192 in FP32). The four-step kernels need N >= 256.
static int small_default(int dtype) { return dtype == BK_F64 ? 128 : 4096; }
static int small_limit(int dtype) {
  const int cap = dtype == BK_F64 ? 4096 : 8192;
  const char* e = getenv("BK_SMALL_MAX_LOG2");
  if (e) {
    const long v = atol(e);
    if (v >= 4 && v <= 13) return std::min(cap, 1 << (int)v);
  }
  return small_default(dtype);
}

template <typename T>
static size_t smem_small(int64_t N) {
  const int64_t L = N + 1;
  const int64_t Lp = (L + 3) & ~3;
  return sizeof(T) * 2 * Lp + sizeof(typename V2<T>::t) * (size_t)pad_stride((int)N);
}

static int round_threads(int64_t t) {
  t = (t + 31) / 32 * 32;
  return (int)std::min<int64_t>(1024, std::max<int64_t>(32, t));
}

static constexpr size_t FOURSTEP_SMEM_BUDGET = 192 * 1024;

// Complex elements one four-step CTA transforms (its tile: NB columns of N1 in pass A, 2P rows
// of N2 in pass B; 16 per thread). BK_FOURSTEP_ELEMS overrides the default (tuning).
static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;
  }
  return n;
}

// Complex elements per four-step CTA (16 per thread): enough CTAs for two per SM over the plan's
// vectors, at least one column of N1 and one row pair of 2 N2, at most the thread cap. Small
// transforms thus run many one-warp CTAs instead of a few full ones (at 2^14 x 4 components the
// full-size tiles gave 16 CTAs per pass). BK_FOURSTEP_ELEMS fixes it (tuning).
static int fourstep_elems(int dtype, int64_t n, int nvec, int N1, int N2, int Eforce = 0) {
  const int cap = dtype == BK_F64 ? 4096 : 8192;  // 16 per thread at the thread cap
  if (Eforce > 0) return std::min(cap, std::max(Eforce, std::max(N1, 2 * N2)));
  const char* e = getenv("BK_FOURSTEP_ELEMS");
  if (e) {
    long v = atol(e);
    if (v >= 16 && v <= cap && is_pow2(v)) return std::max<int>((int)v, std::max(N1, 2 * N2));
  }
  int64_t target = n * (int64_t)std::max(1, nvec) / (2 * sm_count());
  int64_t E = 1;
  while (E * 2 <= target) E *= 2;
  E = std::max<int64_t>(E, std::max(N1, 2 * N2));
  return (int)std::min<int64_t>(E, cap);
}

// Smallest log2 N planned with the two-level split: 2^18 in FP64, 2^24 in FP32
// (BK_SPLIT2_MIN_LOG2 overrides both; 30 disables). Measured products (4 components, two-level
// vs one-level ms): FP64 2^17 0.181 vs 0.178, 2^18 0.272 vs 0.313, 2^20 0.978 vs 1.084, 2^22
// 3.88 vs 4.38, 2^24 17.6 vs 19.3; FP32 2^23 1.557 vs 1.556, 2^24 4.02 vs 4.17.
static int split2_min_log2(int dtype) {
  const char* e = getenv("BK_SPLIT2_MIN_LOG2");
  if (e) {
    const long v = atol(e);
    if (v >= 13 && v <= 30) return (int)v;
  }
  return dtype == BK_F64 ? 18 : 24;
}

// Smallest log2 N planned with the split DCT-I: 2^17 in FP64, 2^23 in FP32 (BK_SPLIT_MIN_LOG2
// overrides both for tuning; 30 disables the split). Below them the half-size launches fill the
// GPU poorly. Measured products (tuned tiles, 4 components, split vs unsplit ms): FP64 2^16
// 0.158 vs 0.124, 2^17 0.179 vs 0.189, 2^18 0.316 vs 0.351, 2^19 0.570 vs 0.638, 2^20 1.09
// vs 1.27; FP32 2^20 0.21 vs 0.166, 2^21 0.349 vs 0.322, 2^22 0.715 vs 0.713, 2^23 1.55 vs
// 1.88. At 2^24 both precisions need the split (the unsplit length-2^24 FFT exceeds the
// four-step shapes).
static int split_min_log2(int dtype) {
  const char* e = getenv("BK_SPLIT_MIN_LOG2");
  if (e) {
    const long v = atol(e);
    if (v >= 13 && v <= 30) return (int)v;
  }
  return dtype == BK_F64 ? 17 : 23;
}

// Shapes of one four-step layout (tables untouched, so a built plan can be re-shaped); Eforce
// > 0 fixes the elements per CTA (the autotuner's candidates), 0 takes fourstep_elems.
static bk_status configure_fourstep(FourStep& f, int64_t n, int dtype, int nvec, int Eforce = 0) {
  const int log2n = ilog2(n);
  f.n = n;
  // balanced factors, with the rows short enough for one row pair per CTA (2 N2 / 16 threads)
  // and the columns for one column per CTA (N1 / 16 threads) under the thread cap
  const int maxthr = dtype == BK_F64 ? 256 : 512;
  int l2 = log2n - log2n / 2;
  while (l2 > 0 && (2 << l2) / 16 > maxthr) --l2;
  f.N2 = 1 << l2;
  f.N1 = 1 << (log2n - l2);
  if (f.N1 / 16 > maxthr) {
    set_error("four-step configuration failed for n=%lld (transform too long for this precision)", (long long)n);
    return BK_ERR_UNSUPPORTED;
  }
  const size_t csz = 2 * dtype_size(dtype);
  const int E = fourstep_elems(dtype, n, nvec, f.N1, f.N2, Eforce);
  // pass A: NB columns of N1; pass B: P row pairs (2P rows) of N2
  int NB = std::max(1, E / f.N1);
  if (NB > f.N2) NB = f.N2;
  int P = std::max(1, E / (2 * f.N2));
  if (P > f.N1 / 2) P = f.N1 / 2;
  f.NB = NB;
  f.P = P;
  // Pass-A batch stride: when a warp's FFT stays inside one batch (N1 / 16 >= 32 threads), the
  // column-major tile accesses of the load and store phases (lane -> column idx mod NB, row
  // idx / NB) hit distinct banks if the stride is = W / NB modulo the W complex elements of a
  // 128-byte wavefront.
  const int W = (int)(128 / csz);
  const int padA = (f.N1 / 16 >= 32 && NB < W) ? W / NB : 1;
  f.bsA = f.N1 + f.N1 / 16 + padA;
  f.smemA = csz * ((size_t)NB * f.bsA + (dtype == BK_F32 ? f.N1 : 0));
  f.smemB = csz * ((size_t)2 * P * pad_stride(f.N2) + (dtype == BK_F32 ? f.N2 : 0));
  f.thrA = round_threads((int64_t)NB * f.N1 / 16);
  f.thrB = round_threads((int64_t)2 * P * f.N2 / 16);
  if ((int64_t)NB * f.N1 / 16 > maxthr || (int64_t)2 * P * f.N2 / 16 > maxthr || f.smemA > FOURSTEP_SMEM_BUDGET ||
      f.smemB > FOURSTEP_SMEM_BUDGET) {
    set_error("four-step configuration failed for n=%lld", (long long)n);
    return BK_ERR_UNSUPPORTED;
  }
  f.nPartA = f.N2 / f.NB;
  return BK_OK;
}

// The dynamic shared-memory cap is a per-function setting shared by every plan, so it is set to
// the largest size any plan of the type can request (never to one plan's own size, which would
// lower the cap under plans created earlier).
// Kernel attributes: the dynamic shared-memory cap (largest size any plan of the type requests)
// and a carveout that gives shared memory the whole unified L1/shared array, so that several
// transform CTAs stay resident per SM.
template <typename K>
static bk_status smem_attr(K* fn, int cap) {
  BK_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, cap));
  BK_TRY_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  return BK_OK;
}

template <typename T>
bk_status set_smem_attrs(const Plan* p) {
  if (p->small) {
    const int cap = (int)smem_small<T>(p->dtype == BK_F64 ? 4096 : 8192);
    BK_TRY(smem_attr(k_birkhoff_small<T, false>, cap));
    BK_TRY(smem_attr(k_birkhoff_small<T, true>, cap));
    if constexpr (!std::is_same<T, dfl>::value) {
      BK_TRY(smem_attr(k_small_batch<T, false>, cap));
      BK_TRY(smem_attr(k_small_batch<T, true>, cap));
    }
  } else {
    const int cap = (int)FOURSTEP_SMEM_BUDGET;
    if constexpr (!std::is_same<T, dfl>::value) {
      BK_TRY(smem_attr(k_passA_batch<T, IN_PLAIN>, cap));
      BK_TRY(smem_attr(k_passA_batch<T, IN_WINV>, cap));
      BK_TRY(smem_attr(k_passB_batch<T, EP_STORE>, cap));
      BK_TRY(smem_attr(k_passB_batch<T, EP_STORE_TRN>, cap));
      BK_TRY(smem_attr(k_passB_batch<T, EP_FWD_OUT>, cap));
      BK_TRY(smem_attr(k_passB_batch<T, EP_TRN_OUT>, cap));
    }
    BK_TRY(smem_attr(k_passA<T, IN_PLAIN>, cap));
    BK_TRY(smem_attr(k_passA<T, IN_WINV>, cap));
    if constexpr (std::is_same<T, double>::value) {
      BK_TRY(smem_attr(k_passA<T, ST_FWD>, cap));
      BK_TRY(smem_attr(k_passA<T, ST_TRN>, cap));
    }
    BK_TRY(smem_attr(k_passB<T, EP_STORE>, cap));
    BK_TRY(smem_attr(k_passB<T, EP_STORE_TRN>, cap));
    BK_TRY(smem_attr(k_passB<T, EP_FWD_OUT>, cap));
    BK_TRY(smem_attr(k_passB<T, EP_TRN_OUT>, cap));
    BK_TRY(smem_attr(k_passA_split<T, IN_PLAIN>, cap));
    BK_TRY(smem_attr(k_passA_split<T, IN_WINV>, cap));
    BK_TRY(smem_attr(k_passB_split<T, EP_STORE>, cap));
    BK_TRY(smem_attr(k_passB_split<T, EP_STORE_TRN>, cap));
    BK_TRY(smem_attr(k_passB_split<T, EP_FWD_OUT>, cap));
    BK_TRY(smem_attr(k_passB_split<T, EP_TRN_OUT>, cap));
    BK_TRY(smem_attr(k_passA_split3<T, IN_PLAIN>, cap));
    BK_TRY(smem_attr(k_passA_split3<T, IN_WINV>, cap));
    BK_TRY(smem_attr(k_passB_split3<T, EP_STORE>, cap));
    BK_TRY(smem_attr(k_passB_split3<T, EP_STORE_TRN>, cap));
    BK_TRY(smem_attr(k_passB_split3<T, EP_FWD_OUT>, cap));
    BK_TRY(smem_attr(k_passB_split3<T, EP_TRN_OUT>, cap));
    if constexpr (!std::is_same<T, dfl>::value) {
      BK_TRY(smem_attr(k_passA<T, IN_PLAIN, PM_CPLX>, cap));
      BK_TRY(smem_attr(k_passB<T, EP_CPLX, PB_CPLX>, cap));
      BK_TRY(smem_attr(k_passB<T, EP_CPLX_MC, PB_CPLX>, cap));
    }
  }
  return BK_OK;
}
// Largest N that is not a power of two (Bluestein, above the dense range): the length-M FFT
// (M >= 2N - 1) must fit the four-step shapes of the precision.
static int64_t blue_max(int dtype) { return dtype == BK_F64 ? (int64_t(1) << 22) : (int64_t(1) << 23); }

#ifndef BK_TRANSFORM_KERNEL_UNIT
// The instances of set_smem_attrs and apply_impl (and with them every transform kernel) are
// compiled in bk_birkhoff_f64.cu and bk_birkhoff_f32.cu, in parallel with this unit.
extern template bk_status set_smem_attrs<double>(const Plan* p);
extern template bk_status set_smem_attrs<float>(const Plan* p);
extern template bk_status set_smem_attrs<dfl>(const Plan* p);
template <typename T> bk_status blue_spectrum(Plan* p, cudaStream_t st);
extern template bk_status blue_spectrum<double>(Plan* p, cudaStream_t st);
extern template bk_status blue_spectrum<float>(Plan* p, cudaStream_t st);
#endif

// Power-of-two plans take the FFT chain unless BK_DENSE=1 (read at plan creation; then every
// plan with N <= 1024 and at most 16 vectors per product starts on the dense product). The dense
// product is faster per call (4 vectors, cold L2, FFT / dense ms: FP32 2^10 0.027 / 0.019, FP64
// 2^8 0.056 / 0.023, 2^10 0.068 / 0.036), but small-N solves are bound by their launches and do
// not change, and in concurrent serving, where slots of other sizes are created and evicted,
// building its tables (an O(N^3) FP64 formation of B^a per plan) cut throughput from 191 to
// 152 solves/s on one GPU. BK_DENSE=0 is the default; N that is not a power of two is always
// dense.
// FP64 plans of N >= 2^18 compute their transforms in double-float arithmetic (bk_df.cuh) unless
// switched off: bk_set_f64_transform(0) for plans created afterwards, or the environment variable
// BK_F64_DF=0 (read at plan creation); bk_set_f64_transform(1) extends it to every four-step FP64
// plan (N >= 256). Measured products (4 components, cold L2, FP64 / double-float ms): 2^14 0.095 /
// 0.109, 2^16 0.123 / 0.132, 2^18 0.272 / 0.228, 2^20 0.978 / 0.553, 2^22 3.87 / 2.50, 2^24 17.6 /
// 12.3: below 2^18 the passes are latency-bound and the double-float instructions lengthen them.
#ifndef BK_TRANSFORM_KERNEL_UNIT
static std::atomic<int> g_f64_df{-1};
static bool f64_df_default(int64_t N) {
  const int m = g_f64_df.load();
  if (m >= 0) return m == 1;
  const char* e = getenv("BK_F64_DF");
  if (e && e[0] == '0') return false;
  return N >= (int64_t(1) << 18);
}
#endif

static bool dense_default(int dtype, int64_t N, int nvec) {
  (void)dtype;
  if (!dense_supported(N)) return false;
  const char* e = getenv("BK_DENSE");
  return e && e[0] == '1' && nvec <= 16;
}

// Four-step shapes of a plan for E complex elements per CTA (0: the occupancy heuristic).
static bk_status fourstep_shapes(Plan* p, int E) {
  const int nvec = p->n_comp * p->max_batch;
  if (p->split == 2) {
    BK_TRY(configure_fourstep(p->fs, p->N / 4, p->dtype, nvec, E));
    BK_TRY(configure_fourstep(p->fse, p->N / 8, p->dtype, nvec, E));
    BK_TRY(configure_fourstep(p->fso, p->N / 4, p->dtype, nvec, E));
    return BK_OK;
  }
  if (p->split) {
    BK_TRY(configure_fourstep(p->fs, p->N / 2, p->dtype, nvec, E));
    BK_TRY(configure_fourstep(p->fso, p->N / 4, p->dtype, nvec, E));
    return BK_OK;
  }
  return configure_fourstep(p->fs, p->N, p->dtype, nvec, E);
}

// Tile autotuner of the four-step transforms. The elements per CTA E (powers of two from one
// column and one row pair up to the thread cap) set the CTA count, shared memory per CTA and how
// many CTAs share an SM; the best E depends on N, the vector count and the GPU. For each
// candidate the plan is re-shaped and timed (CUDA events, one B and one B^T after a warm-up
// pair, on zero vectors: the kernels have no data-dependent paths); the fastest stays. Results
// are cached per (N, dtype, vectors, SM count, device) for the process, so plans of one size
// share one shape (and bitwise the same results). BK_AUTOTUNE=0 keeps the heuristic shape;
// BK_FOURSTEP_ELEMS, a fixed shape, also skips tuning.
static bool autotune_enabled() {
  const char* e = getenv("BK_AUTOTUNE");
  if (e && e[0] == '0') return false;
  return getenv("BK_FOURSTEP_ELEMS") == nullptr;
}

static std::mutex g_tune_mu;
static std::map<std::tuple<int64_t, int, int, int, int, int>, int> g_tune;

static bk_status autotune_tiles(Plan* p, cudaStream_t st) {
  const int nvec = p->n_comp * p->max_batch;
  int dev = 0;
  BK_TRY_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(p->N, p->dtype, (int)p->df, nvec, sm_count(), dev);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      p->tileE = it->second;
      return fourstep_shapes(p, it->second);
    }
  }
  const int cap = p->dtype == BK_F64 ? 4096 : 8192;
  const int emin = std::max(p->fs.N1, 2 * p->fs.N2);
  const size_t vbytes = dtype_size(p->dtype) * (size_t)p->pitch * nvec;
  void* vin = nullptr;
  void* vout = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  bk_status r = dmalloc(&vin, vbytes);
  if (r == BK_OK) r = dmalloc(&vout, vbytes);
  if (r == BK_OK && (cudaMemsetAsync(vin, 0, vbytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                     cudaEventCreate(&e1) != cudaSuccess)) {
    set_error("autotune: set-up failed");
    r = BK_ERR_CUDA;
  }
  int best = 0;
  float best_ms = 0.f;
  for (int E = emin; r == BK_OK && E <= cap; E *= 2) {
    if (fourstep_shapes(p, E) != BK_OK) continue;  // shape outside the thread/shared-memory caps
    r = plan_apply_n(p, vin, vout, nvec, false, p->s, st);
    if (r == BK_OK) r = plan_apply_n(p, vin, vout, nvec, true, p->s, st);
    if (r == BK_OK && cudaEventRecord(e0, st) != cudaSuccess) r = BK_ERR_CUDA;
    if (r == BK_OK) r = plan_apply_n(p, vin, vout, nvec, false, p->s, st);
    if (r == BK_OK) r = plan_apply_n(p, vin, vout, nvec, true, p->s, st);
    float ms = 0.f;
    if (r == BK_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                       cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)) {
      set_error("autotune: timing failed");
      r = BK_ERR_CUDA;
    }
    if (r == BK_OK && (best == 0 || ms < best_ms)) {
      best = E;
      best_ms = ms;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  dfree(vin);
  dfree(vout);
  if (r != BK_OK) return r;
  if (best == 0) return fourstep_shapes(p, 0);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = best;
  }
  p->tileE = best;
  return fourstep_shapes(p, best);
}

#ifndef BK_TRANSFORM_KERNEL_UNIT
bool plan_n_supported(int64_t N, int dtype) {
  return N >= 4 && (is_pow2(N) ? N <= (int64_t(1) << 24) : (dense_supported(N) || N <= blue_max(dtype)));
}

bk_status plan_create(Plan** out, int64_t N, int n_comp, int max_batch, int dtype, double t0,
                      double tf, int64_t pitch, cudaStream_t st) {
  *out = nullptr;
  BK_ARG(plan_n_supported(N, dtype),
         "N must be a power of two in [4, 2^24] or any N in [4, %lld] (this precision), got %lld",
         (long long)blue_max(dtype), (long long)N);
  BK_ARG(n_comp >= 1 && n_comp <= 64, "n_comp must be in [1, 64], got %d", n_comp);
  BK_ARG(max_batch >= 1, "max_batch must be >= 1, got %d", max_batch);
  BK_ARG(dtype == BK_F64 || dtype == BK_F32, "dtype must be BK_F64 or BK_F32");
  BK_ARG(tf != t0 && isfinite(t0) && isfinite(tf), "tf must differ from t0 and both be finite");
  const int64_t L = N + 1;
  if (pitch == 0) pitch = round_up(L, 32);
  BK_ARG(pitch >= L, "pitch %lld < N + 1", (long long)pitch);
  BK_ARG((pitch * (int64_t)dtype_size(dtype)) % 16 == 0, "pitch * sizeof(dtype) must be a multiple of 16");
  Plan* p = new Plan();
  p->N = N;
  p->L = L;
  p->n_comp = n_comp;
  p->max_batch = max_batch;
  p->dtype = dtype;
  p->t0 = t0;
  p->tf = tf;
  p->s = 0.5 * (tf - t0);
  p->pitch = pitch;
  // N not a power of two: the FFT chain does not apply; every product is the dense one
  p->generic = !is_pow2(N) && dense_supported(N);
  p->blue = !is_pow2(N) && !dense_supported(N);
  {
    const char* e = getenv("BK_DENSE_TEST_TIMEOUT");  // test mode of the dense kernel, as bk_plan_dense_test_timeout
    p->dtest = (e && e[0] == '1') ? 1 : 0;
  }
  p->small = !p->generic && !p->blue && N <= small_limit(dtype);
  bk_status st_ = BK_OK;
  AllocCounter counter(&p->bytes);
  do {
    if ((st_ = dmalloc(&p->bsc, sizeof(double) * (size_t)n_comp * max_batch)) != BK_OK) break;
    if (p->generic) {
      if ((st_ = dmalloc((void**)&p->t_nodes, sizeof(double) * (size_t)L)) != BK_OK) break;
      k_grid_tables<<<(int)((L + 255) / 256), 256, 0, st>>>(p->t_nodes, N, t0, p->s);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) { st_ = BK_ERR_CUDA; set_error("grid table launch failed"); break; }
      if ((st_ = dense_build(p, st)) != BK_OK) break;  // also the weights (last row of B^a)
      p->dense = true;
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { set_error("plan tables: %s", cudaGetErrorString(e)); st_ = BK_ERR_CUDA; }
      break;
    }
    if (p->small) {
      p->smemS = dtype == BK_F64 ? smem_small<double>(N) : smem_small<float>(N);
      p->thrS = round_threads(N / 16);
      if (p->thrS > (dtype == BK_F64 ? 256 : 512)) p->thrS = dtype == BK_F64 ? 256 : 512;
    } else if (p->blue) {
      p->M = 1;
      while (p->M < 2 * N - 1) p->M *= 2;
      const int64_t nvec = (int64_t)n_comp * max_batch;
      if ((st_ = configure_fourstep(p->fsM, p->M, dtype, (int)nvec)) != BK_OK) break;
      const size_t csz = 2 * dtype_size(dtype);
      if ((st_ = dmalloc(&p->scrA, csz * (size_t)p->M * 2 * nvec)) != BK_OK) break;   // two M-vectors
      if ((st_ = dmalloc(&p->scrY, dtype_size(dtype) * (size_t)(N + 1) * nvec)) != BK_OK) break;
      if ((st_ = dmalloc(&p->scrG, dtype_size(dtype) * (size_t)(N + 1) * nvec)) != BK_OK) break;
    } else {
      // split DCT-I from 2^split_min_log2() on: fs the length-N/2 FFT, fso the length-N/4 one
      p->split = ilog2(N) >= split2_min_log2(dtype) ? 2 : (ilog2(N) >= split_min_log2(dtype) ? 1 : 0);
      if ((st_ = fourstep_shapes(p, 0)) != BK_OK) break;
      const int64_t nvec = (int64_t)n_comp * max_batch;
      const size_t csz = 2 * dtype_size(dtype);
      if ((st_ = dmalloc(&p->scrA, csz * (size_t)N * nvec)) != BK_OK) break;
      if ((st_ = dmalloc(&p->scrY, dtype_size(dtype) * (size_t)(N + 1) * nvec)) != BK_OK) break;
      if ((st_ = dmalloc(&p->scrG, dtype_size(dtype) * (size_t)(N + 1) * nvec)) != BK_OK) break;
      // partial sums for the narrowest pass-A tile any shape may take (most CTAs per vector)
      const int nbMin = std::max(1, std::max(p->fs.N1, 2 * p->fs.N2) / p->fs.N1);
      const size_t nPartMax = (size_t)std::max(p->fs.nPartA, p->fs.N2 / std::min(nbMin, p->fs.N2));
      if ((st_ = dmalloc(&p->part1, dtype_size(dtype) * nPartMax * nvec)) != BK_OK) break;
      if ((st_ = dmalloc(&p->part2, dtype_size(dtype) * nPartMax * nvec)) != BK_OK) break;
    }
    p->df = dtype == BK_F64 && !p->small && !p->blue && f64_df_default(N);
    st_ = dtype == BK_F64 ? (p->df ? build_tables<dfl>(p, st) : build_tables<double>(p, st)) : build_tables<float>(p, st);
    if (st_ != BK_OK) break;
    if ((st_ = dmalloc((void**)&p->t_nodes, sizeof(double) * (size_t)L)) != BK_OK) break;
    k_grid_tables<<<(int)((L + 255) / 256), 256, 0, st>>>(p->t_nodes, N, t0, p->s);
    note_launch();
    if (cudaGetLastError() != cudaSuccess) { st_ = BK_ERR_CUDA; set_error("grid table launch failed"); break; }
    st_ = dtype == BK_F64 ? (p->df ? set_smem_attrs<dfl>(p) : set_smem_attrs<double>(p)) : set_smem_attrs<float>(p);
    if (st_ != BK_OK) break;
    if (p->blue && (st_ = dtype == BK_F64 ? blue_spectrum<double>(p, st) : blue_spectrum<float>(p, st)) != BK_OK) break;
    if ((st_ = compute_weights(p, st)) != BK_OK) break;
    if (!p->small && !p->blue && autotune_enabled()) {
      if ((st_ = autotune_tiles(p, st)) != BK_OK) break;
    }
    if (dense_default(dtype, N, n_comp * max_batch)) {
      if ((st_ = dense_build(p, st)) != BK_OK) break;
      p->dense = true;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { set_error("plan tables: %s", cudaGetErrorString(e)); st_ = BK_ERR_CUDA; break; }
  } while (0);
  if (st_ != BK_OK) {
    plan_destroy(p);
    return st_;
  }
  *out = p;
  return BK_OK;
}

void plan_destroy(Plan* p) {
  if (!p) return;
  dfree(p->w64);
  dfree(p->wT);
  dfree(p->tw);
  dfree(p->stwS);
  free_fs(p->fs);
  free_fs(p->fso);
  free_fs(p->fse);
  free_fs(p->fsM);
  dfree(p->chirp);
  dfree(p->bh);
  dfree(p->bsc);
  dfree(p->eo);
  dfree(p->tpost);
  dfree(p->rk);
  dfree(p->scrA);
  dfree(p->scrY);
  dfree(p->scrG);
  dfree(p->part1);
  dfree(p->part2);
  dfree(p->t_nodes);
  dfree(p->dA[0]);
  dfree(p->dA[1]);
  dfree(p->derr);
  dfree(p->dpart);
  dfree(p->dcnt);
  delete p;
}
#endif  // BK_TRANSFORM_KERNEL_UNIT

// One split DCT-I of the vectors at src (input kind K) into dst with epilogue E: pass A of the
// even half (pair sums, length-N/2 FFT on fs) and of the odd half (pair differences, length-N/4
// inverse FFT on fso), then both pass-B launches writing even and odd output indices. partA
// receives the even half's DC partial sums (IN_WINV); partB holds the partials the epilogue
// reads for Y0.
template <typename T, int K, int E>
static bk_status split_dct(const Plan* p, const St<T>* src, int64_t sstride, typename OutS<T, E>::t* dst, int64_t dstride, int64_t zero_to,
                           int nvec, void* scrA, T* partA, const T* partB, int npartB, T s, T invN, StencilTab<T> tb,
                           cudaStream_t st) {
  typedef typename V2<T>::t C;
  const int N = (int)p->N, M = N / 2;
  const FourStep& e = p->fs;
  const FourStep& o = p->fso;
  C* Ae = (C*)scrA;
  C* Ao = Ae + (int64_t)nvec * M;
  const C* tp = (const C*)p->tpost;
  const int gE = e.N2 / e.NB, gO = o.N2 / o.NB;
  k_passA_split<T, K><<<dim3(gE + gO, nvec), std::max(e.thrA, o.thrA), std::max(e.smemA, o.smemA), st>>>(
      gE, src, sstride, Ae, partA, M, e.N1, ilog2(e.N1), e.N2, e.NB, e.bsA, (const C*)e.stw1, (const C*)e.twN,
      (const C*)e.twLo, (const C*)e.twHi, e.tw_h,
      src, sstride, Ao, nullptr, M / 2, o.N1, ilog2(o.N1), o.N2, o.NB, o.bsA, (const C*)o.stw1, (const C*)o.twN,
      (const C*)o.twLo, (const C*)o.twHi, o.tw_h, invN, tb, tp, (const C*)p->eo);
  BK_CHECK_LAUNCH();
  const int hE = e.N1 / 2 / e.P, hO = o.N1 / 2 / o.P;
  k_passB_split<T, E><<<dim3(hE + hO, nvec), std::max(e.thrB, o.thrB), std::max(e.smemB, o.smemB), st>>>(
      hE, Ae, M, e.N1, e.N2, ilog2(e.N2), e.P, (const C*)e.stw2, Ao, M / 2, o.N1, o.N2, ilog2(o.N2), o.P,
      (const C*)o.stw2, dst, dstride, zero_to, partB, npartB, tp, s, invN, N);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// One two-level split DCT-I (see PM_PAIR2): pass A of its three parts in one launch, then pass B
// of the three in one launch writing outputs 4k, 4m + 2 and 2m + 1.
template <typename T, int K, int E>
static bk_status split_dct3(const Plan* p, const St<T>* src, int64_t sstride, typename OutS<T, E>::t* dst, int64_t dstride, int64_t zero_to,
                            int nvec, void* scrA, T* partA, const T* partB, int npartB, T s, T invN, StencilTab<T> tb,
                            cudaStream_t st) {
  typedef typename V2<T>::t C;
  const int N = (int)p->N, Q = N / 4;
  const FourStep& e = p->fs;   // length Q: DCT-I of aa
  const FourStep& d = p->fse;  // length Q/2: DCT-III of a's pair differences
  const FourStep& o = p->fso;  // length Q: DCT-III of x's pair differences
  C* Ae = (C*)scrA;
  C* Ad = Ae + (int64_t)nvec * Q;
  C* Ao = Ad + (int64_t)nvec * (Q / 2);
  const C* tp = (const C*)p->tpost;
  const int g1 = e.N2 / e.NB, g2 = d.N2 / d.NB, g3 = o.N2 / o.NB;
  const int thrA = std::max(e.thrA, std::max(d.thrA, o.thrA));
  const size_t smA = std::max(e.smemA, std::max(d.smemA, o.smemA));
  k_passA_split3<T, K><<<dim3(g1 + g2 + g3, nvec), thrA, smA, st>>>(
      g1, g2, src, sstride, Ae, partA, Q, e.N1, ilog2(e.N1), e.N2, e.NB, e.bsA, (const C*)e.stw1, (const C*)e.twN,
      (const C*)e.twLo, (const C*)e.twHi, e.tw_h,
      src, sstride, Ad, nullptr, Q / 2, d.N1, ilog2(d.N1), d.N2, d.NB, d.bsA, (const C*)d.stw1, (const C*)d.twN,
      (const C*)d.twLo, (const C*)d.twHi, d.tw_h,
      src, sstride, Ao, nullptr, Q, o.N1, ilog2(o.N1), o.N2, o.NB, o.bsA, (const C*)o.stw1, (const C*)o.twN,
      (const C*)o.twLo, (const C*)o.twHi, o.tw_h, invN, tb, tp, (const C*)p->eo);
  BK_CHECK_LAUNCH();
  const int h1 = e.N1 / 2 / e.P, h2 = d.N1 / 2 / d.P, h3 = o.N1 / 2 / o.P;
  const int thrB = std::max(e.thrB, std::max(d.thrB, o.thrB));
  const size_t smB = std::max(e.smemB, std::max(d.smemB, o.smemB));
  k_passB_split3<T, E><<<dim3(h1 + h2 + h3, nvec), thrB, smB, st>>>(
      h1, h2, Ae, Q, e.N1, e.N2, ilog2(e.N2), e.P, (const C*)e.stw2, Ad, Q / 2, d.N1, d.N2, ilog2(d.N2), d.P,
      (const C*)d.stw2, Ao, Q, o.N1, o.N2, ilog2(o.N2), o.P, (const C*)o.stw2, dst, dstride, zero_to, partB, npartB, tp,
      s, invN, N);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

template <typename T, int K, int E>
static bk_status split_any(const Plan* p, const St<T>* src, int64_t sstride, typename OutS<T, E>::t* dst, int64_t dstride, int64_t zero_to,
                           int nvec, void* scrA, T* partA, const T* partB, int npartB, T s, T invN, StencilTab<T> tb,
                           cudaStream_t st) {
  if (p->split == 2)
    return split_dct3<T, K, E>(p, src, sstride, dst, dstride, zero_to, nvec, scrA, partA, partB, npartB, s, invN, tb, st);
  return split_dct<T, K, E>(p, src, sstride, dst, dstride, zero_to, nvec, scrA, partA, partB, npartB, s, invN, tb, st);
}

// One length-M complex FFT on the plan's Bluestein layout: src (M complex per vector, as real
// pairs) -> dst (same), through the four-step scratch A; E = EP_CPLX_MC multiplies by the
// spectral table and conjugates in the store.
template <typename T, int E>
static bk_status blue_fft(const Plan* p, const T* src, T* dst, typename V2<T>::t* A, int nvec, cudaStream_t st) {
  typedef typename V2<T>::t C;
  const FourStep& f = p->fsM;
  const int M = (int)p->M;
  StencilTab<T> tb;
  tb.rk = nullptr;
  tb.cN = T(0);
  k_passA<T, IN_PLAIN, PM_CPLX><<<dim3(f.N2 / f.NB, nvec), f.thrA, f.smemA, st>>>(
      src, 2 * (int64_t)M, A, nullptr, M, f.N1, ilog2(f.N1), f.N2, f.NB, f.bsA, (const C*)f.stw1, (const C*)f.twN,
      (const C*)f.twLo, (const C*)f.twHi, f.tw_h, T(1), tb);
  BK_CHECK_LAUNCH();
  k_passB<T, E, PB_CPLX><<<dim3(f.N1 / 2 / f.P, nvec), f.thrB, f.smemB, st>>>(
      A, dst, 2 * (int64_t)M, 0, nullptr, 0, M, f.N1, f.N2, ilog2(f.N2), f.P, (const C*)f.stw2, (const C*)p->bh, T(1),
      T(1), 1, 1, M);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// One DCT-I of length N + 1 for N not a power of two: chirp, FFT_M, spectral product, FFT_M,
// chirp and real split (k_bs_pre, blue_fft x 2, k_bs_post).
template <typename T, int K, int E>
static bk_status blue_dct(const Plan* p, const T* src, int64_t sstride, typename OutS<T, E>::t* dst, int64_t dstride,
                          int64_t zero_to, int nvec, T s, T invN, cudaStream_t st) {
  typedef typename V2<T>::t C;
  const int64_t M = p->M;
  const int N = (int)p->N;
  T* Ma = (T*)p->scrA;
  C* Mb = (C*)(Ma + 2 * M * (int64_t)p->n_comp * p->max_batch);
  const int gp = (int)std::min<int64_t>(1024, (M + 255) / 256);
  k_bs_pre<T, K><<<dim3(gp, nvec), 256, 0, st>>>(src, sstride, N, M, (const C*)p->chirp, Ma);
  BK_CHECK_LAUNCH();
  BK_TRY((blue_fft<T, EP_CPLX_MC>(p, Ma, Ma, Mb, nvec, st)));
  BK_TRY((blue_fft<T, EP_CPLX>(p, Ma, Ma, Mb, nvec, st)));
  const int gq = (int)std::min<int64_t>(1024, (N / 2 + 256) / 256);
  k_bs_post<T, E><<<dim3(gq, nvec), 256, 0, st>>>(Ma, M, N, (const C*)p->chirp, (const C*)p->tpost, dst, dstride,
                                                  zero_to, s, invN);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// The spectral table of a Bluestein plan: bh = FFT_M(b) / M (b from k_bs_kernel, already
// scaled), through the plan's own FFT passes (scratch: the plan's two M-vectors).
template <typename T>
bk_status blue_spectrum(Plan* p, cudaStream_t st) {
  typedef typename V2<T>::t C;
  const int64_t M = p->M;
  T* Ma = (T*)p->scrA;
  C* Mb = (C*)(Ma + 2 * M * (int64_t)p->n_comp * p->max_batch);
  k_bs_kernel<T><<<(int)std::min<int64_t>((M + 255) / 256, 4096), 256, 0, st>>>(Ma, p->N, M);
  BK_CHECK_LAUNCH();
  BK_TRY((blue_fft<T, EP_CPLX>(p, Ma, (T*)p->bh, Mb, 1, st)));
  return BK_OK;
}

template <typename T>
bk_status apply_impl(const Plan* p, const Us<T>* vu, Us<T>* out, int nvec, bool trans, double s_scale,
                            cudaStream_t st, void* scrA, void* scrY, void* part1, void* part2, void* scrG) {
  typedef typename V2<T>::t C;
  const int N = (int)p->N;
  // the first DCT's input: the caller's vectors, or (double-float) their conversion into the
  // stencil buffer, which the first DCT consumes before the stencil overwrites it
  const St<T>* v = nullptr;
  int64_t vstride = p->pitch;
  if constexpr (std::is_same<T, Us<T>>::value) {
    v = vu;
  } else {
    if (!scrG) {
      set_error("internal: double-float products need the stencil buffer");
      return BK_ERR_ARG;
    }
    k_to_arith<T><<<dim3(std::max(1, std::min(1024, (N + 256) / 256)), nvec), 256, 0, st>>>(vu, p->pitch, (T*)scrG,
                                                                                              N + 1);
    BK_CHECK_LAUNCH();
    v = (const T*)scrG;
    vstride = N + 1;
  }
  const T s = (T)s_scale;
  const T invN = T(1.0 / (double)N);
  StencilTab<T> tb;
  tb.rk = (const T*)p->rk;
  tb.cN = (T)(1.0 / (4.0 * ((double)N * (double)N - 1.0)));
  if (p->small) {
    if (!trans)
      k_birkhoff_small<T, false><<<nvec, p->thrS, p->smemS, st>>>(vu, out, N, ilog2(N), p->pitch, s, (const C*)p->tw, (const C*)p->stwS, (const C*)p->tpost, tb);
    else
      k_birkhoff_small<T, true><<<nvec, p->thrS, p->smemS, st>>>(vu, out, N, ilog2(N), p->pitch, s, (const C*)p->tw, (const C*)p->stwS, (const C*)p->tpost, tb);
    BK_CHECK_LAUNCH();
    return BK_OK;
  }
  if constexpr (!std::is_same<T, dfl>::value) {
    if (p->blue) {
      const int64_t Ls = N + 1;
      T* Ystage = (T*)scrY;
      T* Gst = (T*)scrG;
      const dim3 gS((unsigned)std::min<int64_t>(1024, (N + 255) / 256), nvec);
      if (!trans) {
        BK_TRY((blue_dct<T, IN_PLAIN, EP_STORE>(p, v, vstride, Ystage, Ls, 0, nvec, s, invN, st)));
        k_stencil<T, ST_FWD><<<gS, 256, 0, st>>>(Ystage, Ls, Gst, N, T(1), tb, nullptr);
        BK_CHECK_LAUNCH();
        BK_TRY((blue_dct<T, IN_PLAIN, EP_FWD_OUT>(p, Gst, Ls, out, p->pitch, p->pitch, nvec, s, invN, st)));
      } else {
        BK_TRY((blue_dct<T, IN_WINV, EP_STORE_TRN>(p, v, vstride, Ystage, Ls, 0, nvec, s, invN, st)));
        k_stencil<T, ST_TRN><<<gS, 256, 0, st>>>(Ystage, Ls, Gst, N, T(1), tb, nullptr);
        BK_CHECK_LAUNCH();
        BK_TRY((blue_dct<T, IN_PLAIN, EP_TRN_OUT>(p, Gst, Ls, out, p->pitch, p->pitch, nvec, s, invN, st)));
      }
      return BK_OK;
    }
  }
  if (p->split && scrG) {
    const int64_t Ls = N + 1;
    St<T>* Ystage = (St<T>*)scrY;
    St<T>* Gst = (St<T>*)scrG;
    T* pa1 = (T*)part1;
    T* pa2 = (T*)part2;
    const int nPA = p->fs.nPartA;
    const dim3 gS(nPA, nvec);
    if (!trans) {
      BK_TRY((split_any<T, IN_PLAIN, EP_STORE>(p, v, vstride, Ystage, Ls, 0, nvec, scrA, nullptr, nullptr, 0, s, invN, tb, st)));
      k_stencil<T, ST_FWD><<<gS, 256, 0, st>>>(Ystage, Ls, Gst, N, T(1), tb, pa2);
      BK_CHECK_LAUNCH();
      BK_TRY((split_any<T, IN_PLAIN, EP_FWD_OUT>(p, Gst, Ls, out, p->pitch, p->pitch, nvec, scrA, nullptr, pa2, nPA, s, invN, tb, st)));
    } else {
      BK_TRY((split_any<T, IN_WINV, EP_STORE_TRN>(p, v, vstride, Ystage, Ls, 0, nvec, scrA, pa1, pa1, nPA, s, invN, tb, st)));
      k_stencil<T, ST_TRN><<<gS, 256, 0, st>>>(Ystage, Ls, Gst, N, T(1), tb, nullptr);
      BK_CHECK_LAUNCH();
      BK_TRY((split_any<T, IN_PLAIN, EP_TRN_OUT>(p, Gst, Ls, out, p->pitch, p->pitch, nvec, scrA, nullptr, nullptr, 0, s, invN, tb, st)));
    }
    return BK_OK;
  }
  const FourStep& f = p->fs;
  const int N1 = f.N1, N2 = f.N2, NB = f.NB, P = f.P;
  const int log2N1 = ilog2(N1), log2N2 = ilog2(N2);
  C* A = (C*)scrA;
  St<T>* Ystage = (St<T>*)scrY;
  T* pa1 = (T*)part1;
  T* pa2 = (T*)part2;
  const int nPA = f.nPartA;
  dim3 gA(N2 / NB, nvec), gB(N1 / 2 / P, nvec);
  const C* stw1 = (const C*)f.stw1;
  const C* stw2 = (const C*)f.stw2;
  const int bsA = f.bsA;
  const C* twN = (const C*)f.twN;
  const C* tp = (const C*)p->tpost;
  const int64_t Ls = N + 1;
  St<T>* Gst = (St<T>*)scrG;  // separate stencil pass when given (see k_stencil)
  const dim3 gS(nPA, nvec);
  if (!trans) {
    k_passA<T, IN_PLAIN><<<gA, f.thrA, f.smemA, st>>>(v, vstride, A, pa1, N, N1, log2N1, N2, NB, bsA, stw1, twN, (const C*)f.twLo, (const C*)f.twHi, f.tw_h, invN, tb);
    BK_CHECK_LAUNCH();
    k_passB<T, EP_STORE><<<gB, f.thrB, f.smemB, st>>>(A, Ystage, Ls, 0, nullptr, 0, N, N1, N2, log2N2, P, stw2, tp, s, invN, 1, 1, N);
    BK_CHECK_LAUNCH();
    if (Gst) {
      k_stencil<T, ST_FWD><<<gS, 256, 0, st>>>(Ystage, Ls, Gst, N, T(1), tb, pa2);
      BK_CHECK_LAUNCH();
      k_passA<T, IN_PLAIN><<<gA, f.thrA, f.smemA, st>>>(Gst, Ls, A, pa2, N, N1, log2N1, N2, NB, bsA, stw1, twN, (const C*)f.twLo, (const C*)f.twHi, f.tw_h, invN, tb);
    } else if constexpr (std::is_same<T, double>::value) {
      // fused stencil loads: only the allocation-free FP64 entry point has no stencil buffer
      k_passA<T, ST_FWD><<<gA, f.thrA, f.smemA, st>>>(Ystage, Ls, A, pa2, N, N1, log2N1, N2, NB, bsA, stw1, twN, (const C*)f.twLo, (const C*)f.twHi, f.tw_h, invN, tb);
    } else {
      set_error("internal: FP32 products need the stencil buffer");
      return BK_ERR_ARG;
    }
    BK_CHECK_LAUNCH();
    k_passB<T, EP_FWD_OUT><<<gB, f.thrB, f.smemB, st>>>(A, out, p->pitch, p->pitch, pa2, nPA, N, N1, N2, log2N2, P, stw2, tp, s, invN, 1, 1, N);
    BK_CHECK_LAUNCH();
  } else {
    k_passA<T, IN_WINV><<<gA, f.thrA, f.smemA, st>>>(v, vstride, A, pa1, N, N1, log2N1, N2, NB, bsA, stw1, twN, (const C*)f.twLo, (const C*)f.twHi, f.tw_h, invN, tb);
    BK_CHECK_LAUNCH();
    k_passB<T, EP_STORE_TRN><<<gB, f.thrB, f.smemB, st>>>(A, Ystage, Ls, 0, pa1, nPA, N, N1, N2, log2N2, P, stw2, tp, s, invN, 1, 1, N);
    BK_CHECK_LAUNCH();
    // the stage buffer already holds Y - Y0, so the transposed stencil runs with Y0 = 0
    if (Gst) {
      k_stencil<T, ST_TRN><<<gS, 256, 0, st>>>(Ystage, Ls, Gst, N, T(1), tb, nullptr);
      BK_CHECK_LAUNCH();
      k_passA<T, IN_PLAIN><<<gA, f.thrA, f.smemA, st>>>(Gst, Ls, A, pa2, N, N1, log2N1, N2, NB, bsA, stw1, twN, (const C*)f.twLo, (const C*)f.twHi, f.tw_h, invN, tb);
    } else if constexpr (std::is_same<T, double>::value) {
      k_passA<T, ST_TRN><<<gA, f.thrA, f.smemA, st>>>(Ystage, Ls, A, pa2, N, N1, log2N1, N2, NB, bsA, stw1, twN, (const C*)f.twLo, (const C*)f.twHi, f.tw_h, invN, tb);
    } else {
      set_error("internal: FP32 products need the stencil buffer");
      return BK_ERR_ARG;
    }
    BK_CHECK_LAUNCH();
    k_passB<T, EP_TRN_OUT><<<gB, f.thrB, f.smemB, st>>>(A, out, p->pitch, p->pitch, nullptr, 0, N, N1, N2, log2N2, P, stw2, tp, s, invN, 1, 1, N);
    BK_CHECK_LAUNCH();
  }
  return BK_OK;
}

// Batched products of plans of one precision T (binary32 or binary64 arithmetic): the small
// plans' chains in one launch, the unsplit four-step plans' five passes in one launch each, per
// chunk of BATCH_MAX plans. Each plan uses its own tables and scratch, so a plan appears at most
// once among the four-step ones (the caller checks). vec[i] / out[i]: nv[i] vectors pitch apart.
template <typename T>
static bk_status launch_small_batch(const Plan* const* ps, const void* const* vin, void* const* vout, const int* nv,
                                    int n, bool trans, cudaStream_t st) {
  typedef typename V2<T>::t C;
  for (int c0 = 0; c0 < n; c0 += BATCH_MAX) {
    Batch<SmallJob<T>> b;
    memset(&b, 0, sizeof(b));
    b.njob = std::min(BATCH_MAX, n - c0);
    int thr = 32;
    size_t smem = 0;
    int cta = 0;
    for (int q = 0; q < b.njob; ++q) {
      const Plan* p = ps[c0 + q];
      SmallJob<T>& J = b.j[q];
      J.in = (const T*)vin[c0 + q];
      J.out = (T*)vout[c0 + q];
      J.pitch = p->pitch;
      J.tw = (const C*)p->tw;
      J.stw = (const C*)p->stwS;
      J.tpost = (const C*)p->tpost;
      J.tb.rk = (const T*)p->rk;
      J.tb.cN = (T)(1.0 / (4.0 * ((double)p->N * (double)p->N - 1.0)));
      J.s = (T)p->s;
      J.N = (int)p->N;
      J.log2N = ilog2(p->N);
      J.nblk = 1;
      b.start[q] = cta;
      cta += nv[c0 + q];
      thr = std::max(thr, p->thrS);
      smem = std::max(smem, p->smemS);
    }
    b.start[b.njob] = cta;
    if (!trans)
      k_small_batch<T, false><<<cta, thr, smem, st>>>(b);
    else
      k_small_batch<T, true><<<cta, thr, smem, st>>>(b);
    BK_CHECK_LAUNCH();
  }
  return BK_OK;
}

template <typename T>
static bk_status launch_fourstep_batch(const Plan* const* ps, const void* const* vin, void* const* vout, const int* nv,
                                       int n, bool trans, cudaStream_t st) {
  typedef typename V2<T>::t C;
  for (int c0 = 0; c0 < n; c0 += BATCH_MAX) {
    const int nj = std::min(BATCH_MAX, n - c0);
    Batch<PassAJob<T>> a1, a2;
    Batch<PassBJob<T>> b1, b2;
    Batch<StencilJob<T>> sj;
    memset(&a1, 0, sizeof(a1));
    memset(&b1, 0, sizeof(b1));
    memset(&sj, 0, sizeof(sj));
    a1.njob = b1.njob = sj.njob = nj;
    int thrA = 32, thrB = 32;
    size_t smA = 0, smB = 0;
    int ca = 0, cb = 0, cs = 0;
    for (int q = 0; q < nj; ++q) {
      const Plan* p = ps[c0 + q];
      const FourStep& f = p->fs;
      const int N = (int)p->N;
      const int64_t Ls = N + 1;
      const int nvec = nv[c0 + q];
      StencilTab<T> tb;
      tb.rk = (const T*)p->rk;
      tb.cN = (T)(1.0 / (4.0 * ((double)N * (double)N - 1.0)));
      const T invN = T(1.0 / (double)N);
      PassAJob<T>& A = a1.j[q];
      A.src = (const T*)vin[c0 + q];
      A.sstride = p->pitch;
      A.A = (C*)p->scrA;
      A.partial = (T*)p->part1;
      A.stw = (const C*)f.stw1;
      A.twN = (const C*)f.twN;
      A.twLo = (const C*)f.twLo;
      A.twHi = (const C*)f.twHi;
      A.tb = tb;
      A.invN = invN;
      A.N = N;
      A.N1 = f.N1;
      A.log2N1 = ilog2(f.N1);
      A.N2 = f.N2;
      A.NB = f.NB;
      A.bs = f.bsA;
      A.tw_h = f.tw_h;
      A.nthr = f.thrA;
      A.nblk = f.N2 / f.NB;
      a1.start[q] = ca;
      ca += A.nblk * nvec;
      PassBJob<T>& B = b1.j[q];
      B.A = (const C*)p->scrA;
      B.dst = (T*)p->scrY;
      B.dstride = Ls;
      B.zero_to = 0;
      B.partial = trans ? (const T*)p->part1 : nullptr;
      B.npartial = trans ? f.nPartA : 0;
      B.stw = (const C*)f.stw2;
      B.tpost = (const C*)p->tpost;
      B.s = (T)p->s;
      B.invN = invN;
      B.N = N;
      B.N1 = f.N1;
      B.N2 = f.N2;
      B.log2N2 = ilog2(f.N2);
      B.P = f.P;
      B.nthr = f.thrB;
      B.nblk = f.N1 / 2 / f.P;
      b1.start[q] = cb;
      cb += B.nblk * nvec;
      StencilJob<T>& S = sj.j[q];
      S.stage = (const T*)p->scrY;
      S.G = (T*)p->scrG;
      S.partial = trans ? nullptr : (T*)p->part2;
      S.Ls = Ls;
      S.tb = tb;
      S.N = N;
      S.nblk = f.nPartA;
      sj.start[q] = cs;
      cs += S.nblk * nvec;
      thrA = std::max(thrA, f.thrA);
      thrB = std::max(thrB, f.thrB);
      smA = std::max(smA, f.smemA);
      smB = std::max(smB, f.smemB);
    }
    a1.start[nj] = ca;
    b1.start[nj] = cb;
    sj.start[nj] = cs;
    // second DCT: pass A reads the stencil buffer, pass B writes the caller's vectors
    a2 = a1;
    b2 = b1;
    for (int q = 0; q < nj; ++q) {
      const Plan* p = ps[c0 + q];
      a2.j[q].src = (const T*)p->scrG;
      a2.j[q].sstride = p->N + 1;
      a2.j[q].partial = (T*)p->part2;
      b2.j[q].dst = (T*)vout[c0 + q];
      b2.j[q].dstride = p->pitch;
      b2.j[q].zero_to = p->pitch;
      b2.j[q].partial = trans ? nullptr : (const T*)p->part2;
      b2.j[q].npartial = trans ? 0 : p->fs.nPartA;
    }
    if (!trans) {
      k_passA_batch<T, IN_PLAIN><<<ca, thrA, smA, st>>>(a1);
      BK_CHECK_LAUNCH();
      k_passB_batch<T, EP_STORE><<<cb, thrB, smB, st>>>(b1);
      BK_CHECK_LAUNCH();
      k_stencil_batch<T, ST_FWD><<<cs, 256, 0, st>>>(sj);
      BK_CHECK_LAUNCH();
      k_passA_batch<T, IN_PLAIN><<<ca, thrA, smA, st>>>(a2);
      BK_CHECK_LAUNCH();
      k_passB_batch<T, EP_FWD_OUT><<<cb, thrB, smB, st>>>(b2);
      BK_CHECK_LAUNCH();
    } else {
      k_passA_batch<T, IN_WINV><<<ca, thrA, smA, st>>>(a1);
      BK_CHECK_LAUNCH();
      k_passB_batch<T, EP_STORE_TRN><<<cb, thrB, smB, st>>>(b1);
      BK_CHECK_LAUNCH();
      k_stencil_batch<T, ST_TRN><<<cs, 256, 0, st>>>(sj);
      BK_CHECK_LAUNCH();
      k_passA_batch<T, IN_PLAIN><<<ca, thrA, smA, st>>>(a2);
      BK_CHECK_LAUNCH();
      k_passB_batch<T, EP_TRN_OUT><<<cb, thrB, smB, st>>>(b2);
      BK_CHECK_LAUNCH();
    }
  }
  return BK_OK;
}

template <typename T>
bk_status apply_batch_impl(const Plan* const* small_p, const void* const* small_v, void* const* small_o,
                           const int* small_n, int nsmall, const Plan* const* fs_p, const void* const* fs_v,
                           void* const* fs_o, const int* fs_n, int nfs, bool trans, cudaStream_t st) {
  if (nsmall > 0) BK_TRY(launch_small_batch<T>(small_p, small_v, small_o, small_n, nsmall, trans, st));
  if (nfs > 0) BK_TRY(launch_fourstep_batch<T>(fs_p, fs_v, fs_o, fs_n, nfs, trans, st));
  return BK_OK;
}

#ifndef BK_TRANSFORM_KERNEL_UNIT
extern template bk_status apply_impl<double>(const Plan* p, const double* v, double* out, int nvec, bool trans,
                                             double s_scale, cudaStream_t st, void* scrA, void* scrY, void* part1,
                                             void* part2, void* scrG);
extern template bk_status apply_impl<float>(const Plan* p, const float* v, float* out, int nvec, bool trans,
                                            double s_scale, cudaStream_t st, void* scrA, void* scrY, void* part1,
                                            void* part2, void* scrG);
extern template bk_status apply_batch_impl<double>(const Plan* const*, const void* const*, void* const*,
                                                   const int*, int, const Plan* const*, const void* const*,
                                                   void* const*, const int*, int, bool, cudaStream_t);
extern template bk_status apply_batch_impl<float>(const Plan* const*, const void* const*, void* const*, const int*,
                                                  int, const Plan* const*, const void* const*, void* const*,
                                                  const int*, int, bool, cudaStream_t);
extern template bk_status apply_impl<dfl>(const Plan* p, const double* v, double* out, int nvec, bool trans,
                                          double s_scale, cudaStream_t st, void* scrA, void* scrY, void* part1,
                                          void* part2, void* scrG);

bk_status plan_apply_n(const Plan* p, const void* v, void* out, int nvec, bool trans, double s,
                       cudaStream_t st) {
  if (p->dense) return dense_apply(p, v, out, nvec, trans, s, st);
  if (p->dtype == BK_F64 && p->df)
    return apply_impl<dfl>(p, (const double*)v, (double*)out, nvec, trans, s, st, p->scrA, p->scrY, p->part1, p->part2, p->scrG);
  if (p->dtype == BK_F64)
    return apply_impl<double>(p, (const double*)v, (double*)out, nvec, trans, s, st, p->scrA, p->scrY, p->part1, p->part2, p->scrG);
  return apply_impl<float>(p, (const float*)v, (float*)out, nvec, trans, s, st, p->scrA, p->scrY, p->part1, p->part2, p->scrG);
}

// b-form helpers: c[vec] = out[vec][N] (forward) or s sum_i u[vec][i] (transpose, one block per
// vector, fixed order), then out[vec][i] -= c[vec] (forward) or c[vec] w_i (transpose), i <= N.
template <typename T>
__global__ void k_bform_last(const T* __restrict__ out, int64_t pitch, int64_t N, T* __restrict__ c) {
  if (threadIdx.x == 0) c[blockIdx.x] = out[(int64_t)blockIdx.x * pitch + N];
}
template <typename T>
__global__ void __launch_bounds__(256) k_bform_sum(const T* __restrict__ u, int64_t pitch, int64_t L, double s,
                                                   T* __restrict__ c) {
  __shared__ double red[8];
  const T* x = u + (int64_t)blockIdx.x * pitch;
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < L; i += blockDim.x) a += (double)x[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    c[blockIdx.x] = (T)(s * t);
  }
}
template <typename T>
__global__ void k_bform_sub(T* __restrict__ out, int64_t pitch, int64_t L, const T* __restrict__ c,
                            const T* __restrict__ w) {
  const T cv = c[blockIdx.y];
  T* o = out + (int64_t)blockIdx.y * pitch;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < L; i += (int64_t)gridDim.x * blockDim.x)
    o[i] -= w ? cv * w[i] : cv;
}

template <typename T>
static bk_status apply_b_impl(const Plan* p, const void* v, void* out, int nvec, bool trans, cudaStream_t st) {
  T* c = (T*)p->bsc;
  const dim3 g((unsigned)std::min<int64_t>(1024, (p->L + 255) / 256), nvec);
  const T* w = p->dtype == BK_F64 ? (const T*)p->w64 : (const T*)p->wT;
  if (trans) {
    // the sum first: v may alias out
    k_bform_sum<T><<<nvec, 256, 0, st>>>((const T*)v, p->pitch, p->L, p->s, c);
    BK_CHECK_LAUNCH();
    BK_TRY(plan_apply_n(p, v, out, nvec, true, p->s, st));
    k_bform_sub<T><<<g, 256, 0, st>>>((T*)out, p->pitch, p->L, c, w);
  } else {
    BK_TRY(plan_apply_n(p, v, out, nvec, false, p->s, st));
    k_bform_last<T><<<nvec, 32, 0, st>>>((const T*)out, p->pitch, p->N, c);
    BK_CHECK_LAUNCH();
    k_bform_sub<T><<<g, 256, 0, st>>>((T*)out, p->pitch, p->L, c, nullptr);
  }
  BK_CHECK_LAUNCH();
  return BK_OK;
}

bk_status plan_apply_b(const Plan* p, const void* v, void* out, int batch, bool trans, cudaStream_t st) {
  BK_ARG(p != nullptr, "plan is NULL");
  BK_ARG(v != nullptr && out != nullptr, "NULL vector");
  BK_ARG(batch >= 1 && batch <= p->max_batch, "batch %d outside [1, max_batch=%d]", batch, p->max_batch);
  BK_ARG(((uintptr_t)v & 15) == 0 && ((uintptr_t)out & 15) == 0, "vectors must be 16-byte aligned");
  const int nvec = batch * p->n_comp;
  return p->dtype == BK_F64 ? apply_b_impl<double>(p, v, out, nvec, trans, st)
                            : apply_b_impl<float>(p, v, out, nvec, trans, st);
}

bk_status plan_apply(const Plan* p, const void* v, void* out, int batch, bool trans, cudaStream_t st) {
  BK_ARG(p != nullptr, "plan is NULL");
  BK_ARG(v != nullptr && out != nullptr, "NULL vector");
  BK_ARG(batch >= 1 && batch <= p->max_batch, "batch %d outside [1, max_batch=%d]", batch, p->max_batch);
  BK_ARG(((uintptr_t)v & 15) == 0 && ((uintptr_t)out & 15) == 0, "vectors must be 16-byte aligned");
  return plan_apply_n(p, v, out, batch * p->n_comp, trans, p->s, st);
}

// Products of several plans of one precision, N free per plan: small plans in one launch, unsplit
// four-step plans in one launch per pass (per BATCH_MAX plans), every other plan (dense,
// Bluestein, split, double-float) by its own launches.
bk_status plan_apply_batch(const Plan* const* ps, const void* const* v, void* const* out, const int* batch, int count,
                           bool trans, cudaStream_t st) {
  BK_ARG(ps != nullptr && v != nullptr && out != nullptr && batch != nullptr, "NULL argument");
  BK_ARG(count >= 1 && count <= 4096, "count %d outside [1, 4096]", count);
  BK_ARG(ps[0] != nullptr, "plan 0 is NULL");
  const int dtype = ps[0]->dtype;
  std::vector<const Plan*> sp, fp, op;
  std::vector<const void*> sv, fv, ov;
  std::vector<void*> so, fo, oo;
  std::vector<int> sn, fn, on;
  for (int i = 0; i < count; ++i) {
    const Plan* p = ps[i];
    BK_ARG(p != nullptr, "plan %d is NULL", i);
    BK_ARG(p->dtype == dtype, "plan %d: every plan of a batch has the same dtype", i);
    BK_ARG(v[i] != nullptr && out[i] != nullptr, "entry %d: NULL vector", i);
    BK_ARG(batch[i] >= 1 && batch[i] <= p->max_batch, "entry %d: batch %d outside [1, max_batch=%d]", i, batch[i],
           p->max_batch);
    BK_ARG(((uintptr_t)v[i] & 15) == 0 && ((uintptr_t)out[i] & 15) == 0, "entry %d: vectors must be 16-byte aligned",
           i);
    const int nv = batch[i] * p->n_comp;
    if (p->dense || p->blue || p->split || p->df) {
      op.push_back(p); ov.push_back(v[i]); oo.push_back(out[i]); on.push_back(nv);
    } else if (p->small) {
      sp.push_back(p); sv.push_back(v[i]); so.push_back(out[i]); sn.push_back(nv);
    } else {
      for (const Plan* q : fp) BK_ARG(q != p, "entry %d: a four-step plan may appear once per batch (its scratch)", i);
      fp.push_back(p); fv.push_back(v[i]); fo.push_back(out[i]); fn.push_back(nv);
    }
  }
  if (dtype == BK_F64)
    BK_TRY(apply_batch_impl<double>(sp.data(), sv.data(), so.data(), sn.data(), (int)sp.size(), fp.data(), fv.data(),
                                    fo.data(), fn.data(), (int)fp.size(), trans, st));
  else
    BK_TRY(apply_batch_impl<float>(sp.data(), sv.data(), so.data(), sn.data(), (int)sp.size(), fp.data(), fv.data(),
                                   fo.data(), fn.data(), (int)fp.size(), trans, st));
  for (size_t k = 0; k < op.size(); ++k) BK_TRY(plan_apply_n(op[k], ov[k], oo[k], on[k], trans, op[k]->s, st));
  return BK_OK;
}

#endif  // BK_TRANSFORM_KERNEL_UNIT
}  // namespace bk

#ifndef BK_TRANSFORM_KERNEL_UNIT

namespace bk {

// ---------------------------------------------------------------------------------------------
// Allocation-free variant of the four-step forward product.
//
// For callers that must not allocate device memory once they run: real-time or flight control
// loops with a memory budget fixed at start-up, and host programs whose own allocator owns the
// device. They cannot create a bk_plan (plan creation allocates tables and scratch). This
// variant keeps its twiddle tables and transform scratch in one file-scope device array of
// NOALLOC_BYTES, reserved on every GPU that loads the library until the process exits.
// ---------------------------------------------------------------------------------------------
static constexpr size_t NOALLOC_BYTES = size_t(16) << 20;   // 16 MiB
static constexpr int NOALLOC_MAX_DEV = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device (host code cannot use the symbol itself).
static void* g_noalloc_ptr[NOALLOC_MAX_DEV] = {nullptr};
static std::mutex g_noalloc_mu;

static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Bytes of the scratch layout for N (FP64) and nvec vectors, and the sub-buffer offsets.
static size_t noalloc_layout(const Plan& p, int nvec, size_t off[9]) {
  const int64_t N = p.N;
  size_t o = 0;
  off[0] = o; o += align256(sizeof(double2) * stage_tw_len(ilog2(p.fs.N1)));          // stw1
  off[1] = o; o += align256(sizeof(double2) * (N / 2 + 1));                           // tpost
  off[2] = o; o += align256(sizeof(double2) * N);                                     // twN
  off[3] = o; o += align256(sizeof(double2) * (size_t)N * nvec);                      // scrA
  off[4] = o; o += align256(sizeof(double) * (size_t)(N + 1) * nvec);                 // scrY
  off[5] = o; o += align256(sizeof(double) * (size_t)p.fs.nPartA * nvec);             // part1
  off[6] = o; o += align256(sizeof(double) * (size_t)p.fs.nPartA * nvec);             // part2
  off[7] = o; o += align256(sizeof(double) * (size_t)(N + 2));                        // rk
  off[8] = o; o += align256(sizeof(double2) * stage_tw_len(ilog2(p.fs.N2)));          // stw2
  return o;
}

// Per-device set-up: device address of the scratch array and the shared-memory attributes of
// the pass kernels. Runs on the first call on each device.
static bk_status noalloc_setup(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* ptr = nullptr;
    BK_TRY_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    const int smem = (int)FOURSTEP_SMEM_BUDGET;
    BK_TRY_CUDA(cudaFuncSetAttribute(k_passA<double, IN_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BK_TRY_CUDA(cudaFuncSetAttribute(k_passA<double, ST_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BK_TRY_CUDA(cudaFuncSetAttribute(k_passB<double, EP_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    BK_TRY_CUDA(cudaFuncSetAttribute(k_passB<double, EP_FWD_OUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return BK_OK;
}

bk_status noalloc_apply(const double* v, double* out, int64_t N, int nvec, int64_t pitch, double t0, double tf,
                        cudaStream_t st) {
  BK_ARG(v != nullptr && out != nullptr, "NULL vector");
  BK_ARG(is_pow2(N) && N >= 8192 && N <= 65536, "N must be a power of two in [8192, 65536], got %lld", (long long)N);
  BK_ARG(nvec >= 1 && nvec <= 8, "nvec must be in [1, 8], got %d", nvec);
  BK_ARG(pitch >= N + 1 && pitch % 2 == 0, "pitch must be >= N + 1 and even");
  BK_ARG(tf != t0 && isfinite(t0) && isfinite(tf), "tf must differ from t0 and both be finite");
  BK_ARG(((uintptr_t)v & 15) == 0 && ((uintptr_t)out & 15) == 0, "vectors must be 16-byte aligned");
  {
    // the product reads v after it has started writing out: the two ranges must not overlap
    const uintptr_t vb = (uintptr_t)v, ob = (uintptr_t)out, span = sizeof(double) * (uintptr_t)pitch * nvec;
    BK_ARG(vb + span <= ob || ob + span <= vb, "v and out overlap");
  }
  int dev = 0;
  BK_TRY_CUDA(cudaGetDevice(&dev));
  BK_ARG(dev >= 0 && dev < NOALLOC_MAX_DEV, "device index %d not supported", dev);
  Plan p;  // configuration only; owns nothing
  p.N = N;
  p.L = N + 1;
  p.pitch = pitch;
  p.n_comp = nvec;
  p.max_batch = 1;
  p.dtype = BK_F64;
  p.t0 = t0;
  p.tf = tf;
  p.s = 0.5 * (tf - t0);
  p.small = false;
  BK_TRY(configure_fourstep(p.fs, N, BK_F64, nvec));
  size_t off[9];
  const size_t need = noalloc_layout(p, nvec, off);
  BK_ARG(need <= NOALLOC_BYTES, "N=%lld with %d vectors needs %zu bytes of scratch, more than the %zu reserved",
         (long long)N, nvec, need, NOALLOC_BYTES);
  void* base = nullptr;
  BK_TRY(noalloc_setup(dev, &base));
  unsigned char* b = (unsigned char*)base;
  p.fs.stw1 = b + off[0];
  p.fs.stw2 = b + off[8];
  p.tpost = b + off[1];
  p.fs.twN = b + off[2];
  p.rk = b + off[7];
  // every table is rewritten by each call: nothing in the array has to start at zero
  k_rk_table<double><<<(int)std::min<int64_t>((N + 2 + 255) / 256, 4096), 256, 0, st>>>((double*)p.rk, N + 2);
  BK_CHECK_LAUNCH();
  const int len1 = stage_tw_len(ilog2(p.fs.N1)), len2 = stage_tw_len(ilog2(p.fs.N2));
  k_stage_tw<double><<<(len1 + 255) / 256, 256, 0, st>>>((double2*)p.fs.stw1, ilog2(p.fs.N1), len1);
  BK_CHECK_LAUNCH();
  k_stage_tw<double><<<(len2 + 255) / 256, 256, 0, st>>>((double2*)p.fs.stw2, ilog2(p.fs.N2), len2);
  BK_CHECK_LAUNCH();
  k_post_table<double><<<(int)std::min<int64_t>((N / 2 + 256) / 256, 4096), 256, 0, st>>>((double2*)p.tpost, N);
  BK_CHECK_LAUNCH();
  k_tw_table<double><<<(int)std::min<int64_t>((N + 255) / 256, 8192), 256, 0, st>>>((double2*)p.fs.twN, N, (double)N);
  BK_CHECK_LAUNCH();
  return apply_impl<double>(&p, v, out, nvec, false, p.s, st, b + off[3], b + off[4], b + off[5], b + off[6], nullptr);
}

}  // namespace bk

// ---------------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------------
extern "C" {

const char* bk_last_error(void) { return bk::g_last_error.c_str(); }
const char* bk_version(void) { return "birkhoff-gb300 0.1 (sm_103a)"; }
uint64_t bk_launch_count(void) { return bk::g_launches.load(); }

bk_status bk_plan_create(bk_plan** plan, int64_t N, int n_comp, int max_batch, bk_dtype dtype,
                         double t0, double tf, int64_t pitch, void* stream) {
  BK_ARG(plan != nullptr, "plan output pointer is NULL");
  bk::Plan* p = nullptr;
  bk_status s = bk::plan_create(&p, N, n_comp, max_batch, (int)dtype, t0, tf, pitch, (cudaStream_t)stream);
  *plan = reinterpret_cast<bk_plan*>(p);
  return s;
}

void bk_plan_destroy(bk_plan* plan) { bk::plan_destroy(reinterpret_cast<bk::Plan*>(plan)); }

bk_status bk_plan_info(const bk_plan* plan, int64_t* N, int64_t* L, int64_t* pitch, int* dtype) {
  BK_ARG(plan != nullptr, "plan is NULL");
  const bk::Plan* p = reinterpret_cast<const bk::Plan*>(plan);
  if (N) *N = p->N;
  if (L) *L = p->L;
  if (pitch) *pitch = p->pitch;
  if (dtype) *dtype = p->dtype;
  return BK_OK;
}

bk_status bk_plan_grid(const bk_plan* plan, double* t_host, double* w_host) {
  BK_ARG(plan != nullptr, "plan is NULL");
  const bk::Plan* p = reinterpret_cast<const bk::Plan*>(plan);
  if (t_host) BK_TRY_CUDA(cudaMemcpy(t_host, p->t_nodes, sizeof(double) * p->L, cudaMemcpyDeviceToHost));
  if (w_host) BK_TRY_CUDA(cudaMemcpy(w_host, p->w64, sizeof(double) * p->L, cudaMemcpyDeviceToHost));
  return BK_OK;
}

bk_status birkhoff_apply(const bk_plan* plan, const void* v, void* out, int batch, void* stream) {
  return bk::plan_apply(reinterpret_cast<const bk::Plan*>(plan), v, out, batch, false, (cudaStream_t)stream);
}

bk_status birkhoff_apply_noalloc(const double* v, double* out, int64_t N, int nvec, int64_t pitch, double t0,
                                 double tf, void* stream) {
  return bk::noalloc_apply(v, out, N, nvec, pitch, t0, tf, (cudaStream_t)stream);
}

bk_status birkhoff_apply_b(const bk_plan* plan, const void* v, void* out, int batch, void* stream) {
  return bk::plan_apply_b(reinterpret_cast<const bk::Plan*>(plan), v, out, batch, false, (cudaStream_t)stream);
}

bk_status birkhoff_apply_b_T(const bk_plan* plan, const void* v, void* out, int batch, void* stream) {
  return bk::plan_apply_b(reinterpret_cast<const bk::Plan*>(plan), v, out, batch, true, (cudaStream_t)stream);
}

bk_status birkhoff_apply_batch(const bk_plan* const* plans, const void* const* v, void* const* out, const int* batch,
                               int count, int trans, void* stream) {
  return bk::plan_apply_batch(reinterpret_cast<const bk::Plan* const*>(plans), v, out, batch, count, trans != 0,
                              (cudaStream_t)stream);
}

bk_status birkhoff_apply_T(const bk_plan* plan, const void* v, void* out, int batch, void* stream) {
  return bk::plan_apply(reinterpret_cast<const bk::Plan*>(plan), v, out, batch, true, (cudaStream_t)stream);
}

bk_status bk_plan_set_dense(bk_plan* plan, int on, void* stream) {
  BK_ARG(plan != nullptr, "plan is NULL");
  bk::Plan* p = reinterpret_cast<bk::Plan*>(plan);
  if (!on) {
    if (p->generic) {
      bk::set_error("N = %lld is not a power of two: the plan has no FFT path", (long long)p->N);
      return BK_ERR_UNSUPPORTED;
    }
    p->dense = false;
    return BK_OK;
  }
  if (!bk::dense_supported(p->N)) {
    bk::set_error("dense products need N <= 1024 (N = %lld)", (long long)p->N);
    return BK_ERR_UNSUPPORTED;
  }
  if (!p->dA[0]) {
    bk::AllocCounter counter(&p->bytes);
    BK_TRY(bk::dense_build(p, (cudaStream_t)stream));
  }
  p->dense = true;
  return BK_OK;
}

bk_status bk_plan_shape(const bk_plan* plan, int* path, int* N1, int* N2, int* elems) {
  BK_ARG(plan != nullptr, "plan is NULL");
  const bk::Plan* p = reinterpret_cast<const bk::Plan*>(plan);
  const int pth = p->dense ? 3 : (p->blue ? 4 : (p->small ? 0 : (p->split ? 2 : 1)));
  if (path) *path = pth;
  if (N1) *N1 = (pth == 1 || pth == 2) ? p->fs.N1 : 0;
  if (N2) *N2 = (pth == 1 || pth == 2) ? p->fs.N2 : 0;
  if (elems) *elems = (pth == 1 || pth == 2) ? p->fs.NB * p->fs.N1 : 0;
  return BK_OK;
}

bk_status bk_set_f64_transform(int mode) {
  BK_ARG(mode == 0 || mode == 1 || mode == -1, "mode must be 0 (FP64), 1 (double-float) or -1 (default)");
  bk::g_f64_df.store(mode);
  return BK_OK;
}

bk_status bk_plan_f64_mode(const bk_plan* plan, int* mode) {
  BK_ARG(plan != nullptr && mode != nullptr, "NULL argument");
  const bk::Plan* p = reinterpret_cast<const bk::Plan*>(plan);
  *mode = p->df ? 1 : 0;
  return BK_OK;
}

bk_status bk_plan_dense_state(const bk_plan* plan, int* on) {
  BK_ARG(plan != nullptr && on != nullptr, "NULL argument");
  *on = reinterpret_cast<const bk::Plan*>(plan)->dense ? 1 : 0;
  return BK_OK;
}

bk_status bk_plan_dense_test_timeout(bk_plan* plan, int on) {
  BK_ARG(plan != nullptr, "plan is NULL");
  reinterpret_cast<bk::Plan*>(plan)->dtest = on ? 1 : 0;
  return BK_OK;
}

bk_status bk_plan_dense_check(const bk_plan* plan, int* err) {
  BK_ARG(plan != nullptr && err != nullptr, "NULL argument");
  const bk::Plan* p = reinterpret_cast<const bk::Plan*>(plan);
  *err = 0;
  if (!p->derr) return BK_OK;
  BK_TRY_CUDA(cudaDeviceSynchronize());
  BK_TRY_CUDA(cudaMemcpy(err, p->derr, sizeof(int), cudaMemcpyDeviceToHost));
  BK_TRY_CUDA(cudaMemset(p->derr, 0, sizeof(int)));
  return BK_OK;
}

}  // extern "C"

#endif  // BK_TRANSFORM_KERNEL_UNIT
