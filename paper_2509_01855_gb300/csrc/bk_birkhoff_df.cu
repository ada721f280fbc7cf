// Double-float instances of the Birkhoff transform templates (the transform kernels of FP64
// plans that compute in double-float arithmetic, bk_df.cuh), compiled in their own translation
// unit so that the library builds in parallel. The definitions are those of bk_birkhoff.cu,
// included with its main-unit-only parts (globals, plans, entry points) left out.
#define BK_TRANSFORM_KERNEL_UNIT
#include "bk_birkhoff.cu"

namespace bk {

template bk_status set_smem_attrs<dfl>(const Plan* p);
template bk_status apply_impl<dfl>(const Plan* p, const double* v, double* out, int nvec, bool trans, double s_scale,
                                   cudaStream_t st, void* scrA, void* scrY, void* part1, void* part2, void* scrG);

}  // namespace bk
