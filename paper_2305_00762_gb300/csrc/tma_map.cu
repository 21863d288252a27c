// Tensor maps of the padded FP64 state for the stage kernels' tile staging.
//
// A state is 4 planes of (ny + 12) rows of `pitch` doubles (plane stride
// g.plane doubles). Its map is 3-D: x over the nx + 12 padded columns, y over
// the ny + 12 padded rows, z over the 4 fields; the box is the tile + halo of
// the kernel instance times the 4 fields. Cells outside the padded extent
// read as zero. The encoder is the driver's cuTensorMapEncodeTiled, reached
// through the runtime's entry-point query (the library links the runtime
// statically and not the driver library).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <mutex>

#include "gbr_internal.h"

namespace gbr {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

struct MapKey {
    const double* q;
    int nx, ny, pitch, box_w, box_h;
    long long plane;
    bool operator==(const MapKey& o) const
    {
        return q == o.q && nx == o.nx && ny == o.ny && pitch == o.pitch && box_w == o.box_w && box_h == o.box_h &&
               plane == o.plane;
    }
};

// A few recent encodings per host thread (a context's three state buffers
// times the two precisions' tile shapes).
constexpr int kCache = 8;
thread_local MapKey t_keys[kCache];
thread_local CUtensorMap t_maps[kCache];
thread_local int t_used = 0, t_next = 0;

}  // namespace

cudaError_t encode_state_map(const Grid& g, const double* q, int box_w, int box_h, CUtensorMap* out)
{
    const MapKey key{q, g.nx, g.ny, g.pitch, box_w, box_h, g.plane};
    for (int k = 0; k < t_used; ++k)
        if (t_keys[k] == key) {
            *out = t_maps[k];
            return cudaSuccess;
        }
    PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)(g.nx + 2 * kGhost), (cuuint64_t)(g.ny + 2 * kGhost), 4};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * sizeof(double), (cuuint64_t)g.plane * sizeof(double)};
    const cuuint32_t box[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 4};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap m;
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double*>(q), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    t_keys[t_next] = key;
    t_maps[t_next] = m;
    t_next = (t_next + 1) % kCache;
    if (t_used < kCache) ++t_used;
    *out = m;
    return cudaSuccess;
}

}  // namespace gbr
