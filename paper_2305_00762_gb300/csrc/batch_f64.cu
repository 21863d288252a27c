// FP64 instantiations of the persistent batch stage kernel (candidate tile
// shapes picked by the batch autotuner).
#include "batch_stage.cuh"

namespace gbr {

static const TileShape kShapesF64[] = {{32, 8}, {16, 16}, {64, 4}};

int batch_tile_shapes_f64(const TileShape** shapes)
{
    *shapes = kShapesF64;
    return 3;
}

cudaError_t launch_batch_stage_f64(int shape, const BatchCase* cases, int ncases, int total_tiles, int stage,
                                   cudaStream_t s)
{
    switch (shape) {
    case 0: return launch_batch_t<double, 32, 8, 256>(cases, ncases, total_tiles, stage, s);
    case 1: return launch_batch_t<double, 16, 16, 256>(cases, ncases, total_tiles, stage, s);
    default: return launch_batch_t<double, 64, 4, 256>(cases, ncases, total_tiles, stage, s);
    }
}

}  // namespace gbr
