// FP32 instantiation of the fused stage kernel: stencil, reconstruction and
// flux arithmetic in float; state, stage combination and positivity in FP64.
#include "stage_kernel.cuh"

namespace gbr {

cudaError_t launch_stage_f32(const StageParams& p, cudaStream_t s)
{
    if (p.ph.cons) return launch_stage_cons_f32(p, s);
    if (p.ph.order == 4) {  // the learned sensor is trained for the seventh-order scheme only
        if (p.ph.mu > 0.0) return launch_stage_t<float, 28, 16, 256, true, false, 4>(p, s);
        return launch_stage_t<float, 28, 16, 256, false, false, 4>(p, s);
    }
    if (p.sensor && p.dec) {  // decisions from the separate decision pass
        if (p.ph.mu > 0.0) return launch_stage_t<float, 28, 16, 256, true, 1>(p, s);
        return launch_stage_t<float, 28, 16, 256, false, 1>(p, s);
    }
    if (p.sensor) {  // the network fused into the stage
        if (p.ph.mu > 0.0) return launch_stage_t<float, 28, 16, 256, true, 2>(p, s);
        return launch_stage_t<float, 28, 16, 256, false, 2>(p, s);
    }
    if (p.ph.mu > 0.0) return launch_stage_t<float, 28, 16, 256, true>(p, s);
    return launch_stage_t<float, 28, 16, 256, false>(p, s);
}

}  // namespace gbr
