// FP32 instances of the Birkhoff transform templates (every FP32 transform kernel), compiled in
// their own translation unit so that the library builds in parallel. The definitions are those
// of bk_birkhoff.cu, included with its main-unit-only parts (globals, plans, entry points) left
// out.
#define BK_TRANSFORM_KERNEL_UNIT
#include "bk_birkhoff.cu"

namespace bk {

template bk_status set_smem_attrs<float>(const Plan* p);
template bk_status blue_spectrum<float>(Plan* p, cudaStream_t st);
template bk_status apply_batch_impl<float>(const Plan* const*, const void* const*, void* const*, const int*, int,
                                        const Plan* const*, const void* const*, void* const*, const int*, int, bool,
                                        cudaStream_t);
template bk_status apply_impl<float>(const Plan* p, const float* v, float* out, int nvec, bool trans, double s_scale,
                                     cudaStream_t st, void* scrA, void* scrY, void* part1, void* part2, void* scrG);

}  // namespace bk
