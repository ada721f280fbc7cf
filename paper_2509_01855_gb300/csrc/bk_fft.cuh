// Shared-memory batched complex FFT used by the DCT-I transforms of the Birkhoff products.
// Forward transform, omega_n = exp(-2 pi i / n).
//
// In-place Stockham autosort with radix 16 (one mixed radix 2/4/8 stage first when log2 n is
// not a multiple of 4). Every thread stages exactly 16 values per stage in registers (one
// radix-16 butterfly, or 16/R butterflies of radix R), so one buffer suffices: read, barrier,
// compute, write, barrier. Shared addresses are padded, a -> a + a/16, which makes the Stockham
// writes conflict-free for 8- and 16-byte complex values; batches sit bs >= n + n/16 + 1 apart.
//
// Twiddles come from a per-size stage table built on the device with sincospi at plan creation:
// for each radix-16 stage with Ns > 1 (in stage order) a block stw[off + (r - 1) Ns + k] =
// omega_{16 Ns}^{r k}, r = 1..15, k < Ns. Lanes hold consecutive k, so a warp reads consecutive
// entries: no shared-memory bank conflicts, coalesced global loads. (Indexing one table of
// omega_n^i by r k instead gave stride-r lane patterns, up to 16-way conflicts.) The table may
// be the global one or a copy in shared memory (load_tw_smem).
#pragma once

#include <type_traits>

#include "bk_common.cuh"

namespace bk {

__device__ __forceinline__ int padi(int a) { return a + (a >> 4); }
__host__ __device__ inline int pad_stride(int n) { return n + (n >> 4) + 1; }

// Entries of the stage twiddle table of a length-2^log2n FFT (radix-16 stages with Ns > 1).
__host__ __device__ inline int stage_tw_len(int log2n) {
  int len = 0;
  for (int l = (log2n & 3) ? (log2n & 3) : 4; l < log2n; l += 4) len += 15 << l;
  return len;
}

// Radix-R DFT of v[0..R-1] in registers (forward, natural order in and out).
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

// Radix 16 as 4 x 4: r = r1 + 4 r2, s = s1 + 4 s2,
//   X[s1 + 4 s2] = sum_r1 omega_4^{r1 s2} omega_16^{r1 s1} sum_r2 v[r1 + 4 r2] omega_4^{r2 s1}.
template <typename C, typename T> struct Radix<C, T, 16> {
  static __device__ __forceinline__ void run(C* v) {
    // cos(pi/8) = sqrt(2 + sqrt 2)/2, sin(pi/8) = sqrt(2 - sqrt 2)/2, sqrt(1/2)
    const T c1 = T(0.92387953251128675612818318939678828682241662586364);
    const T s1 = T(0.38268343236508977172845998403039886676134456248563);
    const T h = T(0.70710678118654752440084436210484903928483593768847);
    C y[4][4];
#pragma unroll
    for (int r1 = 0; r1 < 4; ++r1) {
      C t[4] = {v[r1], v[r1 + 4], v[r1 + 8], v[r1 + 12]};
      Radix<C, T, 4>::run(t);
#pragma unroll
      for (int q = 0; q < 4; ++q) y[r1][q] = t[q];
    }
    // internal twiddles omega_16^{r1 s1}, r1, s1 in 1..3 (exponents 1,2,3,2,4,6,3,6,9)
    C a;
    a = y[1][1]; y[1][1].x = c1 * a.x + s1 * a.y; y[1][1].y = c1 * a.y - s1 * a.x;       // w^1
    a = y[1][2]; y[1][2].x = h * (a.x + a.y); y[1][2].y = h * (a.y - a.x);                // w^2
    a = y[1][3]; y[1][3].x = s1 * a.x + c1 * a.y; y[1][3].y = s1 * a.y - c1 * a.x;       // w^3
    a = y[2][1]; y[2][1].x = h * (a.x + a.y); y[2][1].y = h * (a.y - a.x);                // w^2
    y[2][2] = cmul_mi(y[2][2]);                                                           // w^4
    a = y[2][3]; y[2][3].x = h * (a.y - a.x); y[2][3].y = -h * (a.x + a.y);               // w^6
    a = y[3][1]; y[3][1].x = s1 * a.x + c1 * a.y; y[3][1].y = s1 * a.y - c1 * a.x;       // w^3
    a = y[3][2]; y[3][2].x = h * (a.y - a.x); y[3][2].y = -h * (a.x + a.y);               // w^6
    a = y[3][3]; y[3][3].x = -c1 * a.x - s1 * a.y; y[3][3].y = s1 * a.x - c1 * a.y;      // w^9
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      C t[4] = {y[0][q], y[1][q], y[2][q], y[3][q]};
      Radix<C, T, 4>::run(t);
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2) v[q + 4 * s2] = t[s2];
    }
  }
};

// One in-place stage of radix R (16/R butterflies per thread) of a length-2^LOG2N FFT whose
// previous radices multiply to Ns = 2^LOG2NS. Threads t < nbatch * n/16 work; all threads must
// reach the barriers.
//
// Addressing. padi(a + c) = padi(a) + padi(c) whenever (a mod 16) + (c mod 16) < 16, so with
// n and Ns known at compile time every shared address of a stage is one per-thread base plus an
// immediate offset:
//   reads  tt + q n/16 + r n/R : all offsets multiples of 16 once n >= 256 (smaller n: generic);
//   writes idxD + r Ns, idxD = (j / Ns) 16 Ns + (j mod Ns): idxD mod 16 = j mod Ns < Ns when
//          Ns < 16 and r Ns mod 16 <= 16 - Ns, or both offsets multiples of 16 (Ns >= 16); in
//          the first stage (Ns = 1) idxD = R j is a multiple of R and r < R;
//   twiddles stw[(r - 1) Ns + k] from stw + k.
template <typename T, int LOG2N, int R, int LOG2NS>
__device__ __forceinline__ void stage_ct(typename V2<T>::t* __restrict__ buf, int nbatch, int bs,
                                         const typename V2<T>::t* __restrict__ stw) {
  typedef typename V2<T>::t C;
  constexpr int log2R = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
  constexpr int PER = 16 / R;
  constexpr int LOG2NB16 = LOG2N - 4;
  constexpr int nb16 = 1 << LOG2NB16;
  constexpr int nR = (1 << LOG2N) >> log2R;
  constexpr int Ns = 1 << LOG2NS;
  constexpr bool lin_rd = (nR % 16 == 0) && (PER == 1 || nb16 % 16 == 0);
  static_assert(PER == 1 || LOG2NS == 0, "mixed radix only as the first stage");
  const int t = threadIdx.x;
  const bool active = t < (nbatch << LOG2NB16);
  const int tt = t & (nb16 - 1);
  C* base = buf + (size_t)(t >> LOG2NB16) * bs;
  C v[16];
  if (active) {
    const C* src = base + padi(tt);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = q * nb16 + r * nR;
        v[q * R + r] = lin_rd ? src[c + (c >> 4)] : base[padi(tt + c)];
      }
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = tt + q * nb16;
      const int k = j & (Ns - 1);
      C* u = v + q * R;
      if (Ns > 1) {
        const C* tw = stw + k;
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw[(r - 1) * Ns]);
      }
      Radix<C, T, R>::run(u);
      C* dst = base + padi(((j >> LOG2NS) << (LOG2NS + log2R)) + k);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int c = r * Ns;
        dst[c + (c >> 4)] = u[r];
      }
    }
  }
  __syncthreads();
}

// Radix-16 stages from Ns = 2^LOG2NS on; OFF is the stage table offset of the first of them.
template <typename T, int LOG2N, int LOG2NS, int OFF>
__device__ __forceinline__ void fft_ct_r16(typename V2<T>::t* buf, int nbatch, int bs,
                                           const typename V2<T>::t* __restrict__ stw) {
  if constexpr (LOG2NS < LOG2N) {
    stage_ct<T, LOG2N, 16, LOG2NS>(buf, nbatch, bs, stw + OFF);
    fft_ct_r16<T, LOG2N, LOG2NS + 4, OFF + (LOG2NS > 0 ? (15 << LOG2NS) : 0)>(buf, nbatch, bs, stw);
  }
}

// Length-2^LOG2N FFT: one mixed radix-2/4/8 stage when LOG2N is not a multiple of 4, then
// radix-16 stages.
template <typename T, int LOG2N>
__device__ __forceinline__ void fft_ct(typename V2<T>::t* buf, int nbatch, int bs,
                                       const typename V2<T>::t* __restrict__ stw) {
  constexpr int rem = LOG2N & 3;
  if constexpr (rem != 0) stage_ct<T, LOG2N, (1 << rem), 0>(buf, nbatch, bs, stw);
  fft_ct_r16<T, LOG2N, rem, 0>(buf, nbatch, bs, stw);
}

template <typename T, int LO, int HI>
__device__ __forceinline__ void fft_ct_dispatch(typename V2<T>::t* buf, int log2n, int nbatch, int bs,
                                                const typename V2<T>::t* __restrict__ stw) {
  if constexpr (LO <= HI) {
    if (log2n == LO) fft_ct<T, LO>(buf, nbatch, bs, stw);
    else fft_ct_dispatch<T, LO + 1, HI>(buf, log2n, nbatch, bs, stw);
  }
}

// Batched in-place forward FFT of length n = 2^log2n (16 <= n <= 8192) over `nbatch` padded
// transforms bs apart in shared memory (element i of batch b at buf[b * bs + padi(i)]), stw the
// stage table of length n. The block needs at least nbatch * n / 16 threads. Input complete
// before the call (barrier); result complete on return, in natural order, in place. Each length
// is its own compile-time instance (log2n is uniform over the block).
template <typename T>
__device__ __forceinline__ void fft16(typename V2<T>::t* buf, int n, int log2n, int nbatch, int bs,
                                      const typename V2<T>::t* __restrict__ stw) {
  fft_ct_dispatch<T, 4, 13>(buf, log2n, nbatch, bs, stw);
}

// Copy a stage table (len entries) into shared memory.
template <typename T>
__device__ __forceinline__ void load_tw_smem(typename V2<T>::t* dst, const typename V2<T>::t* __restrict__ stw,
                                             int len) {
  for (int i = threadIdx.x; i < len; i += blockDim.x) dst[i] = ldg(&stw[i]);
}

}  // namespace bk

namespace bk {

// The same FFT with the length and the stage known only at run time: one radix-16 stage body
// (and one mixed-radix first stage) per kernel instead of one unrolled instance per length and
// stage. Used by the double-float kernels, whose butterflies are an order of magnitude longer
// than binary32 or binary64 ones, so that compile time and code size stay bounded; the address
// arithmetic is generic (padi per element), which costs little next to double-float arithmetic.
template <typename T, int R>
__device__ __forceinline__ void stage_rt(typename V2<T>::t* __restrict__ buf, int nbatch, int bs,
                                         const typename V2<T>::t* __restrict__ stw, int log2n, int log2ns) {
  typedef typename V2<T>::t C;
  constexpr int log2R = R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1));
  constexpr int PER = 16 / R;
  const int log2nb16 = log2n - 4;
  const int nb16 = 1 << log2nb16;
  const int nR = (1 << log2n) >> log2R;
  const int Ns = 1 << log2ns;
  const int t = threadIdx.x;
  const bool active = t < (nbatch << log2nb16);
  const int tt = t & (nb16 - 1);
  C* base = buf + (size_t)(t >> log2nb16) * bs;
  C v[16];
  if (active) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[q * R + r] = base[padi(tt + q * nb16 + r * nR)];
    }
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = tt + q * nb16;
      const int k = j & (Ns - 1);
      C* u = v + q * R;
      if (Ns > 1) {
        const C* tw = stw + k;
#pragma unroll
        for (int r = 1; r < R; ++r) u[r] = cmul(u[r], tw[(r - 1) * Ns]);
      }
      Radix<C, T, R>::run(u);
      const int d0 = ((j >> log2ns) << (log2ns + log2R)) + k;
#pragma unroll
      for (int r = 0; r < R; ++r) base[padi(d0 + r * Ns)] = u[r];
    }
  }
  __syncthreads();
}

// Run-time-length form of fft16 (same contract: 16 <= n <= 8192, nbatch * n / 16 threads).
template <typename T>
__device__ __forceinline__ void fft16_rt(typename V2<T>::t* buf, int n, int log2n, int nbatch, int bs,
                                         const typename V2<T>::t* __restrict__ stw) {
  const int rem = log2n & 3;
  if (rem == 1) stage_rt<T, 2>(buf, nbatch, bs, stw, log2n, 0);
  else if (rem == 2) stage_rt<T, 4>(buf, nbatch, bs, stw, log2n, 0);
  else if (rem == 3) stage_rt<T, 8>(buf, nbatch, bs, stw, log2n, 0);
  int off = 0;
  for (int l = rem; l < log2n; l += 4) {
    stage_rt<T, 16>(buf, nbatch, bs, stw + off, log2n, l);
    if (l > 0) off += 15 << l;
  }
}

// fft16 for binary32 / binary64, fft16_rt for double-float.
template <typename T>
__device__ __forceinline__ void fft16_any(typename V2<T>::t* buf, int n, int log2n, int nbatch, int bs,
                                          const typename V2<T>::t* __restrict__ stw) {
  if constexpr (std::is_same<T, dfl>::value) fft16_rt<T>(buf, n, log2n, nbatch, bs, stw);
  else fft16<T>(buf, n, log2n, nbatch, bs, stw);
}

}  // namespace bk
