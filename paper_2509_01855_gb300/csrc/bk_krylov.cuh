// GMRES interface (internal).
#pragma once

#include "bk_problem.cuh"

namespace bk {

// Optional record of the KKT operator's transposed products (BK_OP_KKT, FP64 operators only):
// T (restart vectors, ld apart) receives s B^aT of the lambda block of each vector the operator
// is applied to in the Arnoldi loop, and Td (n values) accumulates sum_j y_j T_j alongside the
// iterate, i.e. s B^aT of the lambda block of the returned solution, at no extra product.
struct KrylovMu {
  double* T;
  int64_t ld;
  double* Td;
  int64_t n;
};

size_t gmres_workspace_bytes(int64_t n, int m, int dtype);
// weighted (BK_OP_KKT only): minimise the residual in the KKT merit norm ||.||_W, i.e. run on
// D A x = D b with D = diag(w^-1/2 on the gradient rows, w^1/2 on the constraint rows, 1 on the
// tail), preconditioned by M^-1 D^-1; the returned x and the reported residual are A's and W's.
bk_status gmres(Problem* pr, OpData& d, int op, const void* b, void* x, const bk_krylov_opts& o,
                bk_krylov_info* info, void* ws, cudaStream_t st, const KrylovMu* aux = nullptr,
                bool weighted = false);
bk_krylov_opts krylov_defaults();

}  // namespace bk
