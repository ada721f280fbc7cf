// GMRES interface (internal).
#pragma once

#include "bk_problem.cuh"

namespace bk {

size_t gmres_workspace_bytes(int64_t n, int m, int dtype);
bk_status gmres(Problem* pr, OpData& d, int op, const void* b, void* x, const bk_krylov_opts& o,
                bk_krylov_info* info, void* ws, cudaStream_t st);
bk_krylov_opts krylov_defaults();

}  // namespace bk
