// Plan object of the Birkhoff products (internal).
#pragma once

#include "bk_common.cuh"

namespace bk {

// One four-step complex FFT layout of length n = N1 * N2 (pass A: columns of length N1, pass B:
// rows of length N2) and its tables in the working type.
struct FourStep {
  int64_t n = 0;
  int N1 = 0, N2 = 0;
  int NB = 0, P = 0;          // pass A columns per CTA, pass B rows (or row pairs) per CTA
  int bsA = 0;                // pass-A batch stride in shared memory (complex elements)
  size_t smemA = 0, smemB = 0;
  int thrA = 256, thrB = 256; // threads of the pass kernels (16 complex values each)
  int nPartA = 0;             // pass-A CTAs per vector (partials per vector)
  void* stw1 = nullptr;       // stage twiddle table of the length-N1 FFT
  void* stw2 = nullptr;       // stage twiddle table of the length-N2 FFT
  void* twN = nullptr;        // omega_n^m, m < n (FP64)
  void* twLo = nullptr;       // omega_n^m, m < 2^tw_h (FP32)
  void* twHi = nullptr;       // omega_n^{m 2^tw_h}, m < n / 2^tw_h (FP32)
  int tw_h = 0;
};

struct Plan {
  int64_t N = 0, L = 0, pitch = 0;
  int n_comp = 1, max_batch = 1, dtype = BK_F64;
  double t0 = 0, tf = 0, s = 0;
  bool small = true;          // whole chain in one CTA per vector
  bool generic = false;       // N not a power of two: dense products only
  bool df = false;            // FP64 plan whose transforms compute in double-float arithmetic
  // N not a power of two above the dense range: each DCT-I's length-N DFT by Bluestein's
  // convolution of length M (a power of two >= 2N - 1) on the four-step layout fsM
  bool blue = false;
  int64_t M = 0;
  FourStep fsM;
  void* chirp = nullptr;      // w_j = exp(-i pi j^2 / N), j < N (working type)
  void* bh = nullptr;         // FFT_M(b) / M of the conjugate chirp b (working type)
  void* bsc = nullptr;        // one scalar per vector (b-form products), working type
  int tileE = 0;              // four-step elements per CTA chosen by the autotuner (0: heuristic)
  size_t smemS = 0;           // dynamic shared memory of the single-CTA kernel
  int thrS = 256;             // threads of the single-CTA kernel
  void* tw = nullptr;         // omega_N^i, i < N (single-CTA plans; the N < 16 direct DFT)
  void* stwS = nullptr;       // stage twiddle table of the length-N FFT (single-CTA plans)
  // Four-step plans. Unsplit: fs is the length-N FFT of the DCT-I. Split (split = 1): each DCT-I
  // of length N+1 is the DCT-I of length N/2+1 of its pair sums (even outputs; fs, length N/2)
  // and the DCT-III of length N/2 of its pair differences (odd outputs; fso, length N/4).
  // Two-level split (split = 2): the even half split once more, fs the length-N/4 FFT of the
  // DCT-I of length N/4+1, fse the length-N/8 FFT of the DCT-III of length N/4, fso as above.
  FourStep fs, fso, fse;
  int split = 0;
  void* eo = nullptr;         // split: exp(2 pi i k / (N/2)), k < N/4 (DCT-III pre-processing)
  void* tpost = nullptr;      // (cos, sin)(pi k / N), k = 0..N/2 (working type)
  void* rk = nullptr;         // 1 / (4k), k = 0..N+1 (working type; rk[0] = 0)
  void* scrA = nullptr;       // four-step complex scratch, N per vector
  void* scrY = nullptr;       // stage buffer between the two DCTs, N + 1 per vector
  void* scrG = nullptr;       // second-DCT input (stencil output), N + 1 per vector
  void* part1 = nullptr;      // pass-A partial sums, first DCT
  void* part2 = nullptr;      // pass-A partial sums, second DCT
  double* t_nodes = nullptr;  // node times t_j (FP64, device)
  double* w64 = nullptr;      // Clenshaw-Curtis weights (FP64, device, tau-domain)
  void* wT = nullptr;         // Clenshaw-Curtis weights in the working type (device)
  size_t bytes = 0;           // device bytes this plan allocated
  // Dense path (N <= 1024): B^a and (B^a)^T, FP32 plans pre-tiled as TF32 hi/lo parts for the
  // tensor cores, FP64 plans column-major FP64 (dA[0], dA[1]); used while `dense` is set.
  bool dense = false;
  void* dA[2] = {nullptr, nullptr};
  int dMp = 0;                // FP64 layout: rows padded to a multiple of 128
  int* derr = nullptr;        // device error word of the dense kernel (0 = no timeout)
  int dtest = 0;              // test mode: every dense FP32 product times out on purpose
  int dMt = 0, dnK = 0;       // 128-row output tiles, 32-wide K chunks
  void* dpart = nullptr;      // split-K partial sums (FP32)
  unsigned* dcnt = nullptr;   // split-K arrival counters, one per output tile (self-resetting)
};

// Grid sizes a plan of this precision supports: powers of two 4..2^24, any other N 4..2^22
// (BK_F64) or 4..2^23 (BK_F32).
bool plan_n_supported(int64_t N, int dtype);
bk_status plan_create(Plan** out, int64_t N, int n_comp, int max_batch, int dtype, double t0,
                      double tf, int64_t pitch, cudaStream_t st);
void plan_destroy(Plan* p);
bk_status plan_apply(const Plan* p, const void* v, void* out, int batch, bool trans,
                     cudaStream_t st);
// b-form product B^b v = B v - (B v)_N 1 (trans: B^bT u = B^T u - s (1 . u) w).
bk_status plan_apply_b(const Plan* p, const void* v, void* out, int batch, bool trans, cudaStream_t st);
// Apply to `nvec` vectors with an explicit scale (s = 1 gives B^a itself).
bk_status plan_apply_n(const Plan* p, const void* v, void* out, int nvec, bool trans, double s,
                       cudaStream_t st);

// Dense tensor-core path (bk_dense.cu).
bool dense_supported(int64_t N);
bk_status dense_build(Plan* p, cudaStream_t st);
bk_status dense_apply(const Plan* p, const void* v, void* out, int nvec, bool trans, double s, cudaStream_t st);
bk_status dense_status(const Plan* p, cudaStream_t st);

}  // namespace bk
