// Common definitions of the Birkhoff GB300 library: status plumbing, vector types, launch
// helpers. Internal header; the public ABI is include/birkhoff.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/birkhoff.h"
#include "bk_df.cuh"

namespace bk {

// Record a printf-style message as the thread-local last error.
void set_error(const char* fmt, ...);

#define BK_TRY_CUDA(expr)                                                             \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      (void)cudaGetLastError();                                                       \
      bk::set_error("%s:%d %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
      return BK_ERR_CUDA;                                                             \
    }                                                                                 \
  } while (0)

#define BK_TRY(expr)                       \
  do {                                     \
    bk_status s_ = (expr);                 \
    if (s_ != BK_OK) return s_;            \
  } while (0)

// Every kernel launch of the library is followed by BK_CHECK_LAUNCH(), which also counts it
// (bk_launch_count()). Kernels captured into a graph are counted when the graph runs instead:
// the capture takes its own launches back (note_launches(-k), k from thread_launches(), the
// calling thread's count) and each execution adds the kernels it ran.
void note_launch();
unsigned long long thread_launches();
void note_launches(long long n);
#define BK_CHECK_LAUNCH()          \
  do {                             \
    bk::note_launch();             \
    BK_TRY_CUDA(cudaGetLastError()); \
  } while (0)

#define BK_ARG(cond, ...)                  \
  do {                                     \
    if (!(cond)) {                         \
      bk::set_error(__VA_ARGS__);          \
      return BK_ERR_ARG;                   \
    }                                      \
  } while (0)

// Two-component vector of the working type (complex numbers, twiddles).
template <typename T> struct V2;
template <> struct V2<double> { typedef double2 t; };
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<dfl> { typedef dfl2 t; };

template <typename T> __host__ __device__ __forceinline__ typename V2<T>::t mk2(T x, T y) {
  typename V2<T>::t r; r.x = x; r.y = y; return r;
}

// Complex product a * b.
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// a * (-i)
template <typename C> __device__ __forceinline__ C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline int ilog2(int64_t x) { int r = 0; while ((int64_t(1) << r) < x) ++r; return r; }
inline bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

inline size_t dtype_size(int dt) { return dt == BK_F64 ? 8 : 4; }

// Allocation wrapper that reports OOM as a status.
bk_status dmalloc(void** p, size_t bytes);
void dfree(void* p);

// While alive, every dmalloc on this thread adds its size to *acc (nested counters stack).
struct AllocCounter {
  explicit AllocCounter(size_t* acc);
  ~AllocCounter();
  size_t* prev;
};

}  // namespace bk
