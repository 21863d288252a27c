// FP32-arithmetic instantiations of the batch stage kernel (candidate tile
// shapes and launch forms picked by the batch autotuner).
#include "batch_stage.cuh"

namespace gbr {

static const TileShape kShapesF32[] = {{28, 16}, {32, 16}, {32, 8}};

int batch_tile_shapes_f32(const TileShape** shapes)
{
    *shapes = kShapesF32;
    return 3;
}

cudaError_t launch_batch_stage_f32(int shape, const BatchCase* cases, int ncases, int total_tiles, int stage,
                                   cudaStream_t s, const SensorDev* sensor, bool per_tile)
{
    if (sensor) {
        switch (shape) {
        case 0: return launch_batch_t<float, 28, 16, 256, true>(cases, ncases, total_tiles, stage, s, sensor, per_tile);
        case 1: return launch_batch_t<float, 32, 16, 256, true>(cases, ncases, total_tiles, stage, s, sensor, per_tile);
        default: return launch_batch_t<float, 32, 8, 256, true>(cases, ncases, total_tiles, stage, s, sensor, per_tile);
        }
    }
    switch (shape) {
    case 0: return launch_batch_t<float, 28, 16, 256>(cases, ncases, total_tiles, stage, s, nullptr, per_tile);
    case 1: return launch_batch_t<float, 32, 16, 256>(cases, ncases, total_tiles, stage, s, nullptr, per_tile);
    default: return launch_batch_t<float, 32, 8, 256>(cases, ncases, total_tiles, stage, s, nullptr, per_tile);
    }
}

}  // namespace gbr
