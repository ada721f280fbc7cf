// Shared-memory batched complex FFT (Stockham autosort, radix 8/4/2) used by the DCT-I
// transforms of the Birkhoff products. Forward transform, omega_n = exp(-2 pi i / n).
//
// Twiddles come from a table tw[i] = (cos(2 pi i / n_tab), -sin(2 pi i / n_tab)), i < n_tab,
// n_tab = 2^tw_log2 >= n, built on the device with sincospi at plan creation.
#pragma once

#include "bk_common.cuh"

namespace bk {

// Radix-R DFT of v[0..R-1] in registers (forward).
template <typename C, typename T, int R> struct Radix;

template <typename C, typename T> struct Radix<C, T, 2> {
  static __device__ __forceinline__ void run(C* v) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <typename C, typename T> struct Radix<C, T, 4> {
  static __device__ __forceinline__ void run(C* v) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = cmul_mi(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  }
};

template <typename C, typename T> struct Radix<C, T, 8> {
  static __device__ __forceinline__ void run(C* v) {
    // even / odd radix-4 halves, then combine with omega_8^k
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    Radix<C, T, 4>::run(e);
    Radix<C, T, 4>::run(o);
    const T h = T(0.70710678118654752440084436210484903928483593768847);
    // omega_8^1 = (1 - i) h, omega_8^2 = -i, omega_8^3 = -(1 + i) h
    C o1, o2, o3;
    o1.x = h * (o[1].x + o[1].y);
    o1.y = h * (o[1].y - o[1].x);
    o2 = cmul_mi(o[2]);
    o3.x = h * (o[3].y - o[3].x);
    o3.y = -h * (o[3].x + o[3].y);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);
    v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);
    v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);
    v[7] = csub(e[3], o3);
  }
};

// One Stockham stage with radix R over `nbatch` transforms of length n (batch stride bs).
// Ns = product of the radices of the previous stages (1 for the first stage).
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const typename V2<T>::t* __restrict__ src,
                                               typename V2<T>::t* __restrict__ dst, int n,
                                               int log2n, int nbatch, int bs, int Ns, int log2Ns,
                                               const typename V2<T>::t* __restrict__ tw,
                                               int tw_log2) {
  typedef typename V2<T>::t C;
  const int nbf = n / R;  // butterflies per transform
  const int log2nbf = log2n - (R == 8 ? 3 : (R == 4 ? 2 : 1));
  const int total = nbatch << log2nbf;
  const int log2R = (R == 8 ? 3 : (R == 4 ? 2 : 1));
  const int tw_shift = tw_log2 - (log2Ns + log2R);
  for (int j = threadIdx.x; j < total; j += blockDim.x) {
    const int b = j >> log2nbf;
    const int jj = j & (nbf - 1);
    const int k = jj & (Ns - 1);
    const C* s = src + (size_t)b * bs;
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = s[jj + r * nbf];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], __ldg(&tw[(r * k) << tw_shift]));
    }
    Radix<C, T, R>::run(v);
    C* d = dst + (size_t)b * bs;
    const int idxD = ((jj >> log2Ns) << (log2Ns + log2R)) + k;
#pragma unroll
    for (int r = 0; r < R; ++r) d[idxD + r * Ns] = v[r];
  }
}

// Batched forward FFT of length n = 2^log2n over shared buffers a (input) and b (scratch).
// Returns the buffer holding the result. All threads of the block must call it; the input must
// be complete (a __syncthreads() before the call); the result is complete on return.
template <typename T>
__device__ typename V2<T>::t* fft_smem(typename V2<T>::t* a, typename V2<T>::t* b, int n,
                                       int log2n, int nbatch, int bs,
                                       const typename V2<T>::t* __restrict__ tw, int tw_log2) {
  typedef typename V2<T>::t C;
  C* src = a;
  C* dst = b;
  int Ns = 1, log2Ns = 0;
  const int rem = log2n % 3;
  if (rem == 1) {
    stockham_stage<T, 2>(src, dst, n, log2n, nbatch, bs, Ns, log2Ns, tw, tw_log2);
    __syncthreads();
    Ns <<= 1; log2Ns += 1;
    C* t = src; src = dst; dst = t;
  } else if (rem == 2) {
    stockham_stage<T, 4>(src, dst, n, log2n, nbatch, bs, Ns, log2Ns, tw, tw_log2);
    __syncthreads();
    Ns <<= 2; log2Ns += 2;
    C* t = src; src = dst; dst = t;
  }
  while (log2Ns < log2n) {
    stockham_stage<T, 8>(src, dst, n, log2n, nbatch, bs, Ns, log2Ns, tw, tw_log2);
    __syncthreads();
    Ns <<= 3; log2Ns += 3;
    C* t = src; src = dst; dst = t;
  }
  return src;
}

}  // namespace bk
