// FP64 instantiations of the batch stage kernel (candidate tile shapes and
// launch forms picked by the batch autotuner).
#include "batch_stage.cuh"

namespace gbr {

static const TileShape kShapesF64[] = {{32, 8}, {16, 16}, {64, 4}};

int batch_tile_shapes_f64(const TileShape** shapes)
{
    *shapes = kShapesF64;
    return 3;
}

cudaError_t launch_batch_stage_f64(int shape, const BatchCase* cases, int ncases, int total_tiles, int stage,
                                   cudaStream_t s, bool per_tile)
{
    switch (shape) {
    case 0: return launch_batch_t<double, 32, 8, 256>(cases, ncases, total_tiles, stage, s, nullptr, per_tile);
    case 1: return launch_batch_t<double, 16, 16, 256>(cases, ncases, total_tiles, stage, s, nullptr, per_tile);
    default: return launch_batch_t<double, 64, 4, 256>(cases, ncases, total_tiles, stage, s, nullptr, per_tile);
    }
}

}  // namespace gbr
