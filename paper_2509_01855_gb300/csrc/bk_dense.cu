// Dense small-N Birkhoff products on the 5th-generation tensor cores (tcgen05).
//
// For small N the FFT chain of a product is latency-bound (one CTA per vector runs two DCTs and
// the stencil one after the other), while the dense product out = s B^a V is a small GEMM:
// M = N + 1 output nodes, K = N + 1 input nodes, one column per vector. This path keeps B^a
// (and its transpose, for B^T) as a pre-tiled FP32 matrix split into two TF32 parts,
// A = A_hi + A_lo (each rounded to TF32), and multiplies on the tensor cores with kind::tf32:
//   D = A_hi V_hi + A_hi V_lo + A_lo V_hi        (3xTF32; the A_lo V_lo term is below FP32),
// accumulating in FP32 in tensor memory. B^a itself (Eq. xN=Birka+b: the a-form integration
// matrix) is formed once per plan in FP64 from its definition (below), so its entries are
// FP64-exact before the split. FP64 plans multiply by the FP64 matrix on the CUDA cores.
//
// Kernel shape (CTAs of 4 warps; a tile is 128 output rows x 16 vectors, its K range split
// over up to 8 CTAs so that small products still spread over the GPU; each product is one
// latency chain of copies, MMAs and the split-K sum):
//   - thread 0 streams the CTA's part of the A panel through up to four shared-memory stages
//     with bulk copies (cp.async.bulk, completion on an mbarrier) and issues the MMAs
//     (M = 128, N = 16, K = 8);
//   - all threads stage the CTA's K range of the 16 vectors once, split into TF32 hi and lo;
//   - tcgen05.commit arrives on an mbarrier when a stage's MMAs are done (the stage is then
//     refilled) and when the last MMA is done (the epilogue then reads the accumulator);
//   - each warp reads its 32 accumulator lanes with tcgen05.ld; split tiles add their partials
//     in a fixed order in the last CTA to finish (no CTA waits for another).
// Every wait is bounded; on a timeout the kernel records an error code, waits (bounded) for its
// copies in flight, frees its tensor memory and returns.
//
// Shared-memory operand layout (no swizzle, K-major): core matrices of 8 rows x 16 bytes (8 x 4
// TF32 values, rows 16 bytes apart). For one MMA k-step (8 values of K) the two core matrices
// along K sit 128 bytes apart (leading byte offset) and successive 8-row groups 256 bytes apart
// (stride byte offset); k-steps follow each other. Both strides stay inside the k-step's block
// whichever way the two offsets are read, so a misread layout gives wrong values, never an
// out-of-range shared access.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "bk_plan.cuh"

namespace bk {

constexpr int DT_M = 128;                              // output rows per CTA (MMA M)
constexpr int DT_N = 16;                               // vectors per CTA (MMA N)
constexpr int DT_KC = 32;                              // K values per pipeline chunk (4 k-steps)
constexpr int DT_SMAX = 4;                             // A chunk buffers at most
constexpr int DT_PART = DT_M * DT_KC * 4;              // one TF32 part of a chunk: 16 KB
constexpr int DT_CHUNK = 2 * DT_PART;                  // hi + lo: 32 KB
constexpr int DT_TMEM_COLS = 32;                       // accumulator columns allocated (>= DT_N)
constexpr unsigned DT_SPIN = 1u << 20;                 // mbarrier polls before a timeout
constexpr unsigned DT_TEST_SPIN = 1024;                // polls of the test wait (a barrier nothing signals)
constexpr int DENSE_MAX_N = 1024;                      // V (2 parts x 16 x K) fits in shared memory

// Byte offset of A element (m, k), m < 128, k < 32, inside one part of a chunk.
__host__ __device__ inline int dt_a_off(int m, int k) {
  return (k >> 3) * 4096 + (m >> 3) * 256 + ((k >> 2) & 1) * 128 + (m & 7) * 16 + (k & 3) * 4;
}
// Byte offset of V element (vector n < 16, node k) inside one part of the staged vectors.
__host__ __device__ inline int dt_v_off(int n, int k) {
  return (k >> 3) * 512 + (n >> 3) * 256 + ((k >> 2) & 1) * 128 + (n & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Round to TF32 (10 explicit mantissa bits), to nearest, ties away from zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor: start address, leading and stride byte offsets (all >> 4),
// descriptor version 1 (bits 46-48 = 0b001), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t dt_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
  d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t dt_idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(DT_N >> 3) << 17) | ((uint32_t)(DT_M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the phase with the given parity; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned limit = DT_SPIN) {
  for (unsigned i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// out[n][m] = s (A V)[m][n] for m < L, n < nvec, with A = A_hi + A_lo pre-tiled in `At`
// (chunk (mt, c) of 128 rows x 32 columns at ((mt nK + c) * 32 KB), hi part then lo part).
// V and out: nvec vectors `pitch` apart; out's padding [L, pitch) is zeroed.
// Split K: CTA z of the KS CTAs of a tile (blockIdx.z) takes chunks [z nK / KS, (z+1) nK / KS)
// through S shared-memory stages. With KS > 1 each CTA writes its 128 x 16 partial to `part` and
// counts itself in cnt[tile]; the last CTA to arrive sums the KS partials in the order z = 0, 1,
// ... (the result does not depend on arrival order), writes the output and resets the counter.
// No CTA waits for another.
__global__ void __launch_bounds__(128, 1)
    k_dense_tc(const unsigned char* __restrict__ At, const float* __restrict__ V, float* __restrict__ out, int nvec,
               int L, int64_t pitch, int nK, int KS, int S, float s, float* __restrict__ part,
               unsigned* __restrict__ cnt, int* __restrict__ err, int test_timeout) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[DT_SMAX];
  __shared__ __align__(8) uint64_t bar_empty[DT_SMAX];
  __shared__ __align__(8) uint64_t bar_done;
  __shared__ __align__(8) uint64_t bar_never;   // test mode: nothing ever arrives on it
  __shared__ uint32_t tmem_slot;
  __shared__ int fail;
  __shared__ int last;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mt = blockIdx.x, n0 = blockIdx.y * DT_N, z = blockIdx.z;
  const int tile = blockIdx.y * gridDim.x + mt;
  const int cb = (int)((int64_t)z * nK / KS), nloc = (int)((int64_t)(z + 1) * nK / KS) - cb;
  const int Kloc = nloc * DT_KC;
  unsigned char* sA = smem;                  // S chunks
  unsigned char* sV = smem + S * DT_CHUNK;   // hi part, then lo part (this CTA's K range)
  const int vpart = Kloc * DT_N * 4;
  const uint32_t aA = smem_u32(sA), aV = smem_u32(sV);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(DT_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(smem_u32(&bar_full[i]), 1);
      mbar_init(smem_u32(&bar_empty[i]), 1);
    }
    mbar_init(smem_u32(&bar_done), 1);
    mbar_init(smem_u32(&bar_never), 1);
    fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem_d = tmem_slot;

  // first chunks in flight while the vectors are staged
  const unsigned char* Ablk = At + ((size_t)mt * nK + cb) * DT_CHUNK;
  if (tid == 0) {
    for (int c = 0; c < S && c < nloc; ++c) {
      mbar_expect_tx(smem_u32(&bar_full[c]), DT_CHUNK);
      bulk_g2s(aA + c * DT_CHUNK, Ablk + (size_t)c * DT_CHUNK, DT_CHUNK, smem_u32(&bar_full[c]));
    }
  }
  // vectors n0..n0+15, nodes of this CTA's K range (zero beyond L and nvec), split into TF32 hi
  // and lo
  const int k0 = cb * DT_KC;
  for (int i = tid; i < DT_N * Kloc; i += blockDim.x) {
    const int n = i / Kloc, k = i - n * Kloc;
    float v = 0.f;
    if (n0 + n < nvec && k0 + k < L) v = V[(int64_t)(n0 + n) * pitch + k0 + k];
    const float hi = tf32_rna(v);
    const float lo = tf32_rna(v - hi);
    const int off = dt_v_off(n, k);
    *reinterpret_cast<float*>(sV + off) = hi;
    *reinterpret_cast<float*>(sV + vpart + off) = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staged vectors -> tensor core reads
  __syncthreads();

  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    constexpr uint32_t idesc = dt_idesc();
    int issued = nloc < S ? nloc : S;  // chunks whose copies were started
    int c = 0;
    // test mode: a bounded wait that must run out (its barrier never completes a phase), taken
    // through the same failure path as a real timeout
    bool ok = !(test_timeout && !mbar_wait(smem_u32(&bar_never), 0, DT_TEST_SPIN));
    for (; ok && c < nloc; ++c) {
      const int st = c % S;
      const uint32_t ph = (uint32_t)(c / S) & 1u;
      if (!mbar_wait(smem_u32(&bar_full[st]), ph)) { ok = false; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int ks = 0; ks < DT_KC / 8; ++ks) {
        const uint32_t ahi = aA + st * DT_CHUNK + ks * 4096, alo = ahi + DT_PART;
        const int kg = c * (DT_KC / 8) + ks;
        const uint32_t vhi = aV + kg * 512, vlo = vhi + vpart;
        const uint64_t dAh = dt_desc(ahi, 128, 256), dAl = dt_desc(alo, 128, 256);
        const uint64_t dVh = dt_desc(vhi, 128, 256), dVl = dt_desc(vlo, 128, 256);
        tc_mma(tmem_d, dAh, dVh, idesc, (c | ks) != 0 ? 1u : 0u);
        tc_mma(tmem_d, dAh, dVl, idesc, 1u);
        tc_mma(tmem_d, dAl, dVh, idesc, 1u);
      }
      tc_commit(smem_u32(&bar_empty[st]));
      if (c + S < nloc) {
        // refill this stage once its MMAs have read it
        if (!mbar_wait(smem_u32(&bar_empty[st]), ph)) { ok = false; ++c; break; }
        mbar_expect_tx(smem_u32(&bar_full[st]), DT_CHUNK);
        bulk_g2s(aA + st * DT_CHUNK, Ablk + (size_t)(c + S) * DT_CHUNK, DT_CHUNK, smem_u32(&bar_full[st]));
        ++issued;
      }
    }
    tc_commit(smem_u32(&bar_done));
    if (!ok) {
      fail = 1;
      // copies started but not consumed: wait for them (bounded) before the CTA may exit
      for (int q = c; q < issued; ++q) (void)mbar_wait(smem_u32(&bar_full[q % S]), (uint32_t)(q / S) & 1u);
    }
  }
  // every lane waits (bounded); the warp then agrees, since tcgen05.ld is warp-collective
  const bool mine = mbar_wait(smem_u32(&bar_done), 0);
  __syncwarp();
  const bool done = __all_sync(0xffffffffu, mine) && !fail;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t r[16];
#pragma unroll
  for (int n = 0; n < DT_N; ++n) r[n] = 0u;
  if (done) {
    const uint32_t taddr = tmem_d + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  } else if (lane == 0 && fail == 0) {
    fail = 2;
  }
  const int row = warp * 32 + lane;
  const int m = mt * DT_M + row;
  if (KS == 1) {
    if (m < L) {
#pragma unroll
      for (int n = 0; n < DT_N; ++n)
        if (n0 + n < nvec) out[(int64_t)(n0 + n) * pitch + m] = s * __uint_as_float(r[n]);
    }
  } else {
    float4* mine4 = reinterpret_cast<float4*>(part + (((size_t)tile * KS + z) * DT_M + row) * DT_N);
#pragma unroll
    for (int q = 0; q < DT_N / 4; ++q)
      mine4[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]), __uint_as_float(r[4 * q + 2]),
                             __uint_as_float(r[4 * q + 3]));
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&cnt[tile], 1u) == (unsigned)(KS - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      float acc[DT_N];
#pragma unroll
      for (int n = 0; n < DT_N; ++n) acc[n] = 0.f;
      for (int q = 0; q < KS; ++q) {
        const float4* src = reinterpret_cast<const float4*>(part + (((size_t)tile * KS + q) * DT_M + row) * DT_N);
#pragma unroll
        for (int u = 0; u < DT_N / 4; ++u) {
          const float4 x = __ldcg(src + u);
          acc[4 * u] += x.x; acc[4 * u + 1] += x.y; acc[4 * u + 2] += x.z; acc[4 * u + 3] += x.w;
        }
      }
      if (m < L) {
#pragma unroll
        for (int n = 0; n < DT_N; ++n)
          if (n0 + n < nvec) out[(int64_t)(n0 + n) * pitch + m] = s * acc[n];
      }
      if (tid == 0) cnt[tile] = 0u;  // ready for the next product
    }
  }
  if (mt == 0 && z == 0) {
    for (int n = 0; n < DT_N && n0 + n < nvec; ++n)
      for (int64_t mm = L + tid; mm < pitch; mm += blockDim.x) out[(int64_t)(n0 + n) * pitch + mm] = 0.f;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_d), "r"(DT_TMEM_COLS) : "memory");
  if (tid == 0 && fail) atomicExch(err, fail);
}

// Pre-tiled A = B^a (trans = 0) or (B^a)^T (trans = 1) from B^a (FP64, row-major L x L), zero
// outside L x L.
__global__ void k_dense_tile(const double* __restrict__ B, int L, int Mt, int nK, int trans,
                             unsigned char* __restrict__ dst) {
  const int Kpad = nK * DT_KC;
  const int64_t total = (int64_t)Mt * DT_M * Kpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / Kpad), k = (int)(i - (int64_t)m * Kpad);
    double a = 0.0;
    if (m < L && k < L) a = trans ? B[(int64_t)k * L + m] : B[(int64_t)m * L + k];
    const float hi = tf32_rna((float)a);
    const float lo = tf32_rna((float)(a - (double)hi));
    unsigned char* blk = dst + ((size_t)(m / DT_M) * nK + k / DT_KC) * DT_CHUNK;
    const int off = dt_a_off(m % DT_M, k % DT_KC);
    *reinterpret_cast<float*>(blk + off) = hi;
    *reinterpret_cast<float*>(blk + DT_PART + off) = lo;
  }
}

// ---------------------------------------------------------------------------------------------
// B^a in FP64 for any N (not only powers of two), from its definition: row i of B^a integrates
// the Lagrange basis of the CGL nodes over [-1, tau_i] (Eq. xN=Birka+b with Eq. birk-conditions).
// Each basis polynomial is a Chebyshev series, l_j = sum_k Psi[k][j] T_k with the discrete
// Chebyshev coefficients Psi[k][j] = 2 / (N c_k c_j) T_k(tau_j) (c_0 = c_N = 2, else 1), and
// each T_k integrates in closed form (Eq. intChebPoly=): Phi[i][k] = int_{-1}^{tau_i} T_k, so
// B^a = Phi Psi. With tau_j = -cos(j pi / N), T_m(tau_i) = (-1)^m cos(pi m i / N), read from a
// table of cos(pi q / N), q < 2N, at q = m i mod 2N. Row 0 is exactly zero.
// ---------------------------------------------------------------------------------------------
__global__ void k_cospi_table(double* __restrict__ c, int N) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < 2 * N; q += gridDim.x * blockDim.x) c[q] = cospi((double)q / N);
}

__device__ __forceinline__ double cheb_at_node(const double* __restrict__ c, int N, int m, int i) {
  const double v = c[(int)(((int64_t)m * i) % (2 * N))];
  return (m & 1) ? -v : v;
}

__global__ void k_form_phi(double* __restrict__ Phi, int N, const double* __restrict__ c) {
  const int L = N + 1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)L * L;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / L), k = (int)(idx - (int64_t)i * L);
    double tau = sinpi((double)(2 * i - N) / (double)(2 * N));
    if (i == 0) tau = -1.0;
    if (i == N) tau = 1.0;
    double v;
    if (k == 0) {
      v = tau + 1.0;
    } else if (k == 1) {
      v = 0.5 * (tau * tau - 1.0);
    } else {
      // T_{k+1} / (2(k+1)) - T_{k-1} / (2(k-1)), minus its value at -1: (-1)^{k+1} / (k^2 - 1) added
      v = cheb_at_node(c, N, k + 1, i) / (2.0 * (k + 1)) - cheb_at_node(c, N, k - 1, i) / (2.0 * (k - 1)) +
          ((k & 1) ? 1.0 : -1.0) / ((double)k * k - 1.0);
    }
    Phi[idx] = i == 0 ? 0.0 : v;
  }
}

__global__ void k_form_psi(double* __restrict__ Psi, int N, const double* __restrict__ c) {
  const int L = N + 1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)L * L;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / L), j = (int)(idx - (int64_t)k * L);
    const double ck = (k == 0 || k == N) ? 2.0 : 1.0, cj = (j == 0 || j == N) ? 2.0 : 1.0;
    Psi[idx] = 2.0 / ((double)N * ck * cj) * cheb_at_node(c, N, k, j);
  }
}

// C = A B, all row-major n x n FP64 (plan set-up only): 32 x 32 output tiles, 2 x 2 per thread.
__global__ void __launch_bounds__(256) k_gemm64(const double* __restrict__ A, const double* __restrict__ B,
                                                double* __restrict__ C, int n) {
  __shared__ double As[32][33], Bs[32][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
      const int rr = q >> 5, cc = q & 31;
      As[rr][cc] = (r0 + rr < n && k0 + cc < n) ? A[(int64_t)(r0 + rr) * n + k0 + cc] : 0.0;
      Bs[rr][cc] = (k0 + rr < n && c0 + cc < n) ? B[(int64_t)(k0 + rr) * n + c0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double a0 = As[ty][kk], a1 = As[ty + 16][kk];
      const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
      acc[0][0] = fma(a0, b0, acc[0][0]);
      acc[0][1] = fma(a0, b1, acc[0][1]);
      acc[1][0] = fma(a1, b0, acc[1][0]);
      acc[1][1] = fma(a1, b1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int r = r0 + ty + 16 * a, cc = c0 + tx + 16 * b;
      if (r < n && cc < n) C[(int64_t)r * n + cc] = acc[a][b];
    }
}

// Column-major FP64 copy of A = B^a (trans = 0) or (B^a)^T (trans = 1): Acm[k Mp + m], zero for
// m >= L.
__global__ void k_dense_cm64(const double* __restrict__ B, int L, int Mp, int trans, double* __restrict__ Acm) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)L * Mp;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(idx / Mp), m = (int)(idx - (int64_t)k * Mp);
    Acm[idx] = m < L ? (trans ? B[(int64_t)k * L + m] : B[(int64_t)m * L + k]) : 0.0;
  }
}

// Clenshaw-Curtis weights: the last row of B^a (the remark after Eq. Ba=10).
__global__ void k_last_row(const double* __restrict__ B, int L, double* __restrict__ w64, float* __restrict__ w32) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < L; j += gridDim.x * blockDim.x) {
    const double v = B[(int64_t)(L - 1) * L + j];
    w64[j] = v;
    if (w32) w32[j] = (float)v;
  }
}

// ---------------------------------------------------------------------------------------------
// FP64 dense product on the CUDA cores (GB300 has no FP64 tensor-core kind in tcgen05): one
// thread per output row, NC vectors per CTA, the K range split over KS CTAs per tile with the
// same last-arriver reduction in fixed order as the FP32 kernel. Per 8-byte matrix element NC
// FP64 FMAs: the FP64 pipe bounds it (L^2 nvec FMAs; N = 1024, 4 vectors: ~7 us at 1.25 TFLOP/s).
// ---------------------------------------------------------------------------------------------
template <int NC>
__global__ void __launch_bounds__(128)
    k_dense_f64(const double* __restrict__ Acm, int Mp, const double* __restrict__ V, double* __restrict__ out,
                int nvec, int L, int64_t pitch, int KS, double s, double* __restrict__ part,
                unsigned* __restrict__ cnt) {
  constexpr int KC = 64;
  __shared__ double Vs[NC][KC];
  __shared__ int last;
  const int tid = threadIdx.x;
  const int m = blockIdx.x * 128 + tid;  // < Mp (rows >= L are zero)
  const int n0 = blockIdx.y * NC, z = blockIdx.z;
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  const int kb = (int)((int64_t)z * L / KS), ke = (int)((int64_t)(z + 1) * L / KS);
  double acc[NC];
#pragma unroll
  for (int n = 0; n < NC; ++n) acc[n] = 0.0;
  for (int k0 = kb; k0 < ke; k0 += KC) {
    const int kc = min(KC, ke - k0);
    __syncthreads();
    for (int i = tid; i < NC * KC; i += blockDim.x) {
      const int n = i / KC, kk = i - n * KC;
      Vs[n][kk] = (kk < kc && n0 + n < nvec) ? V[(int64_t)(n0 + n) * pitch + k0 + kk] : 0.0;
    }
    __syncthreads();
    const double* a = Acm + (int64_t)k0 * Mp + m;
#pragma unroll 8
    for (int kk = 0; kk < kc; ++kk) {
      const double av = a[(int64_t)kk * Mp];
#pragma unroll
      for (int n = 0; n < NC; ++n) acc[n] = fma(av, Vs[n][kk], acc[n]);
    }
  }
  if (KS == 1) {
    if (m < L) {
#pragma unroll
      for (int n = 0; n < NC; ++n)
        if (n0 + n < nvec) out[(int64_t)(n0 + n) * pitch + m] = s * acc[n];
    }
  } else {
    double* mine = part + (((size_t)tile * KS + z) * 128 + tid) * NC;
#pragma unroll
    for (int n = 0; n < NC; ++n) mine[n] = acc[n];
    __threadfence();
    __syncthreads();
    if (tid == 0) last = atomicAdd(&cnt[tile], 1u) == (unsigned)(KS - 1);
    __syncthreads();
    if (last) {
      __threadfence();
      double sum[NC];
#pragma unroll
      for (int n = 0; n < NC; ++n) sum[n] = 0.0;
      for (int q = 0; q < KS; ++q) {
        const double* src = part + (((size_t)tile * KS + q) * 128 + tid) * NC;
#pragma unroll
        for (int n = 0; n < NC; ++n) sum[n] += __ldcg(src + n);
      }
      if (m < L) {
#pragma unroll
        for (int n = 0; n < NC; ++n)
          if (n0 + n < nvec) out[(int64_t)(n0 + n) * pitch + m] = s * sum[n];
      }
      if (tid == 0) cnt[tile] = 0u;
    }
  }
  if (blockIdx.x == 0 && z == 0) {
    for (int n = 0; n < NC && n0 + n < nvec; ++n)
      for (int64_t mm = L + tid; mm < pitch; mm += blockDim.x) out[(int64_t)(n0 + n) * pitch + mm] = 0.0;
  }
}

constexpr size_t DT_SMEM_BUDGET = 200 * 1024;       // dynamic shared memory of one CTA at most
constexpr int DT_KS_MAX = 16;                          // K splits per tile at most (FP64 kernel)
constexpr int DT_KS_MAX_TC = 8;                        // K splits per tile at most (tensor-core kernel)

// SM count of the current device, looked up once per device (products may run inside a stream
// capture, where device queries are best avoided).
static int dense_sms() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n > 0) return n;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 148;
  cache[dev].store(n, std::memory_order_relaxed);
  return n;
}

// Launch shape of one dense product of nvec vectors: K splits KS (about two CTAs per SM over all
// tiles, at most 8 and at most one per chunk; BK_DENSE_KSPLIT overrides; at N = 1024, 16 splits
// measured 15.9 us against 14.4 us for 8), pipeline stages S
// (up to 4, within the shared-memory budget next to the staged vectors).
struct DenseShape {
  int KS, S;
  size_t smem;
};
static DenseShape dense_shape(const Plan* p, int nvec) {
  const int ny = (nvec + DT_N - 1) / DT_N;
  const int tiles = p->dMt * ny;
  int KS = std::max(1, std::min(std::min(DT_KS_MAX_TC, p->dnK), 2 * dense_sms() / std::max(1, tiles)));
  if (const char* e = getenv("BK_DENSE_KSPLIT")) {
    const long v = atol(e);
    if (v >= 1) KS = (int)std::min<long>(std::min<long>(v, DT_KS_MAX_TC), p->dnK);
  }
  const int nloc = (p->dnK + KS - 1) / KS;
  const size_t vbytes = (size_t)2 * nloc * DT_KC * DT_N * 4;
  int S = std::min(DT_SMAX, nloc);
  while (S > 1 && S * (size_t)DT_CHUNK + vbytes > DT_SMEM_BUDGET) --S;
  return {KS, S, S * (size_t)DT_CHUNK + vbytes};
}

bool dense_supported(int64_t N) { return N >= 4 && N <= DENSE_MAX_N; }

static int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

bk_status dense_build(Plan* p, cudaStream_t st) {
  BK_ARG(dense_supported(p->N), "dense products: N <= %d only", DENSE_MAX_N);
  const int N = (int)p->N, L = (int)p->L;
  const bool f32 = p->dtype == BK_F32;
  const int nvec = p->n_comp * p->max_batch;
  BK_TRY(dmalloc((void**)&p->derr, sizeof(int)));
  BK_TRY_CUDA(cudaMemsetAsync(p->derr, 0, sizeof(int), st));
  if (f32) {
    p->dMt = (L + DT_M - 1) / DT_M;
    p->dnK = (L + DT_KC - 1) / DT_KC;
    const size_t bytes = (size_t)p->dMt * p->dnK * DT_CHUNK;
    for (int t = 0; t < 2; ++t) BK_TRY(dmalloc(&p->dA[t], bytes));
    const int ny = (nvec + DT_N - 1) / DT_N;
    BK_TRY(dmalloc(&p->dpart, sizeof(float) * (size_t)p->dMt * ny * DT_KS_MAX * DT_M * DT_N));
    BK_TRY(dmalloc((void**)&p->dcnt, sizeof(unsigned) * (size_t)p->dMt * ny));
    BK_TRY_CUDA(cudaMemsetAsync(p->dcnt, 0, sizeof(unsigned) * (size_t)p->dMt * ny, st));
  } else {
    p->dMp = (int)round_up(L, 128);
    for (int t = 0; t < 2; ++t) BK_TRY(dmalloc(&p->dA[t], sizeof(double) * (size_t)L * p->dMp));
    // partials: 128 rows x (vectors rounded up to the 4- or 16-vector tile) x K splits;
    // counters: one per tile, most tiles with 4 vectors per CTA
    const int mt = p->dMp / 128;
    const int tiles = mt * ((nvec + 3) / 4);
    BK_TRY(dmalloc(&p->dpart, sizeof(double) * (size_t)mt * round_up(nvec, 16) * DT_KS_MAX * 128));
    BK_TRY(dmalloc((void**)&p->dcnt, sizeof(unsigned) * (size_t)tiles));
    BK_TRY_CUDA(cudaMemsetAsync(p->dcnt, 0, sizeof(unsigned) * (size_t)tiles, st));
  }
  // B^a = Phi Psi in FP64
  double *c = nullptr, *Phi = nullptr, *Psi = nullptr, *B = nullptr;
  const size_t mat = sizeof(double) * (size_t)L * L;
  bk_status r = dmalloc((void**)&c, sizeof(double) * 2 * (size_t)N);
  if (r == BK_OK) r = dmalloc((void**)&Phi, mat);
  if (r == BK_OK) r = dmalloc((void**)&Psi, mat);
  if (r == BK_OK) r = dmalloc((void**)&B, mat);
  if (r == BK_OK) {
    k_cospi_table<<<grid_for(2 * N), 256, 0, st>>>(c, N);
    k_form_phi<<<grid_for((int64_t)L * L), 256, 0, st>>>(Phi, N, c);
    k_form_psi<<<grid_for((int64_t)L * L), 256, 0, st>>>(Psi, N, c);
    k_gemm64<<<dim3((L + 31) / 32, (L + 31) / 32), 256, 0, st>>>(Phi, Psi, B, L);
    for (int q = 0; q < 4; ++q) note_launch();
    if (cudaGetLastError() != cudaSuccess) { r = BK_ERR_CUDA; set_error("dense matrix launch failed"); }
  }
  // weights (last row) when the plan has none yet (plans off the FFT path)
  if (r == BK_OK && !p->w64) {
    r = dmalloc((void**)&p->w64, sizeof(double) * p->pitch);
    if (r == BK_OK && f32) r = dmalloc(&p->wT, sizeof(float) * p->pitch);
    if (r == BK_OK && cudaMemsetAsync(p->w64, 0, sizeof(double) * p->pitch, st) != cudaSuccess) r = BK_ERR_CUDA;
    if (r == BK_OK && f32 && cudaMemsetAsync(p->wT, 0, sizeof(float) * p->pitch, st) != cudaSuccess) r = BK_ERR_CUDA;
    if (r == BK_OK) {
      k_last_row<<<grid_for(L), 256, 0, st>>>(B, L, p->w64, f32 ? (float*)p->wT : nullptr);
      note_launch();
      if (cudaGetLastError() != cudaSuccess) { r = BK_ERR_CUDA; set_error("weights launch failed"); }
    }
  }
  for (int t = 0; t < 2 && r == BK_OK; ++t) {
    if (f32) {
      const int64_t total = (int64_t)p->dMt * DT_M * p->dnK * DT_KC;
      k_dense_tile<<<grid_for(total), 256, 0, st>>>(B, L, p->dMt, p->dnK, t, (unsigned char*)p->dA[t]);
    } else {
      k_dense_cm64<<<grid_for((int64_t)L * p->dMp), 256, 0, st>>>(B, L, p->dMp, t, (double*)p->dA[t]);
    }
    note_launch();
    if (cudaGetLastError() != cudaSuccess) { r = BK_ERR_CUDA; set_error("dense layout launch failed"); }
  }
  if (r == BK_OK && cudaStreamSynchronize(st) != cudaSuccess) { set_error("dense tables: sync failed"); r = BK_ERR_CUDA; }
  dfree(c);
  dfree(Phi);
  dfree(Psi);
  dfree(B);
  if (r != BK_OK) return r;
  if (f32) BK_TRY_CUDA(cudaFuncSetAttribute(k_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DT_SMEM_BUDGET));
  return BK_OK;
}

static bk_status dense_apply64(const Plan* p, const double* v, double* out, int nvec, bool trans, double s,
                               cudaStream_t st) {
  const int NC = nvec <= 4 ? 4 : 16;
  const int mt = p->dMp / 128, ny = (nvec + NC - 1) / NC;
  int KS = std::max(1, std::min(std::min(DT_KS_MAX, (int)((p->L + 31) / 32)), 2 * dense_sms() / std::max(1, mt * ny)));
  if (const char* e = getenv("BK_DENSE_KSPLIT")) {
    const long q = atol(e);
    if (q >= 1) KS = (int)std::min<long>(std::min<long>(q, DT_KS_MAX), (p->L + 31) / 32);
  }
  const dim3 grid(mt, ny, KS);
  const double* A = (const double*)p->dA[trans ? 1 : 0];
  if (NC == 4)
    k_dense_f64<4><<<grid, 128, 0, st>>>(A, p->dMp, v, out, nvec, (int)p->L, p->pitch, KS, s, (double*)p->dpart, p->dcnt);
  else
    k_dense_f64<16><<<grid, 128, 0, st>>>(A, p->dMp, v, out, nvec, (int)p->L, p->pitch, KS, s, (double*)p->dpart, p->dcnt);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

// BK_ERR_TIMEOUT (and the word cleared) when a dense product of the plan ran out of a bounded
// wait since the last check; synchronises the stream. BK_OK for plans off the dense path.
bk_status dense_status(const Plan* p, cudaStream_t st) {
  if (!p || !p->dense || !p->derr) return BK_OK;
  int e = 0;
  BK_TRY_CUDA(cudaMemcpyAsync(&e, p->derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  BK_TRY_CUDA(cudaStreamSynchronize(st));
  if (e == 0) return BK_OK;
  BK_TRY_CUDA(cudaMemsetAsync(p->derr, 0, sizeof(int), st));
  set_error("a dense tensor-core product ran out of a bounded wait (error word %d); its output is invalid", e);
  return BK_ERR_TIMEOUT;
}

bk_status dense_apply(const Plan* p, const void* v, void* out, int nvec, bool trans, double s, cudaStream_t st) {
  if (p->dtype == BK_F64) return dense_apply64(p, (const double*)v, (double*)out, nvec, trans, s, st);
  const DenseShape sh = dense_shape(p, nvec);
  const dim3 grid(p->dMt, (nvec + DT_N - 1) / DT_N, sh.KS);
  k_dense_tc<<<grid, 128, sh.smem, st>>>((const unsigned char*)p->dA[trans ? 1 : 0], (const float*)v, (float*)out, nvec,
                                         (int)p->L, p->pitch, p->dnK, sh.KS, sh.S, (float)s, (float*)p->dpart, p->dcnt,
                                         p->derr, p->dtest);
  BK_CHECK_LAUNCH();
  return BK_OK;
}

}  // namespace bk
