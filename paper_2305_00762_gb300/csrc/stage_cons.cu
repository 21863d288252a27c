// MEG7-cons instantiations of the fused stage kernel (conservative-variable
// reconstruction), FP64 and FP32 arithmetic, seventh order, plain detector.
#include "stage_kernel.cuh"

namespace gbr {

cudaError_t launch_stage_cons_f64(const StageParams& p, cudaStream_t s)
{
    if (p.ph.mu > 0.0) return launch_stage_t<double, 16, 16, 256, true, false, 7, true>(p, s);
    return launch_stage_t<double, 16, 16, 256, false, false, 7, true>(p, s);
}

cudaError_t launch_stage_cons_f32(const StageParams& p, cudaStream_t s)
{
    if (p.ph.mu > 0.0) return launch_stage_t<float, 28, 16, 256, true, false, 7, true>(p, s);
    return launch_stage_t<float, 28, 16, 256, false, false, 7, true>(p, s);
}

}  // namespace gbr
