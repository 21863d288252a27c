// FP64 instantiation of the fused stage kernel (the plain method).
#include "stage_kernel.cuh"

namespace gbr {

cudaError_t launch_stage_f64(const StageParams& p, cudaStream_t s)
{
    if (p.ph.cons) return launch_stage_cons_f64(p, s);
    if (p.ph.order == 4) {
        if (p.ph.mu > 0.0) return launch_stage_t<double, 16, 16, 256, true, false, 4>(p, s);
        return launch_stage_t<double, 16, 16, 256, false, false, 4>(p, s);
    }
    if (p.ph.mu > 0.0) return launch_stage_t<double, 16, 16, 256, true>(p, s);
    return launch_stage_t<double, 16, 16, 256, false>(p, s);
}

}  // namespace gbr
