// slice.cu -- points of an axis-aligned 2D slice, the visualisation query of Sec. 6 (Fig. 6:
// a 2D slice reconstructed from the functional tensor), written straight into a device
// buffer for evaluation.
#include "fst_internal.cuh"

namespace fst {

__global__ void slice_points_kernel(int axis, float value, float lo0, float hi0, float lo1, float hi1, int res0,
                                    int res1, float* xyz) {
    const int64_t n = (int64_t)res0 * res1;
    const int a0 = axis == 0 ? 1 : 0, a1 = axis == 2 ? 1 : 2;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / res1), j = (int)(e - (int64_t)i * res1);
        const float t0 = res0 > 1 ? (float)i / (float)(res0 - 1) : 0.5f;
        const float t1 = res1 > 1 ? (float)j / (float)(res1 - 1) : 0.5f;
        xyz[(int64_t)axis * n + e] = value;
        xyz[(int64_t)a0 * n + e] = lo0 + t0 * (hi0 - lo0);
        xyz[(int64_t)a1 * n + e] = lo1 + t1 * (hi1 - lo1);
    }
}

}  // namespace fst

using namespace fst;

extern "C" fst_status fst_slice_points(int32_t axis, double value, const double lo[3], const double hi[3],
                                       int32_t res0, int32_t res1, float* xyz, fst_stream stream) {
    FST_REQUIRE(axis >= 0 && axis < 3, "axis must be 0, 1 or 2");
    FST_REQUIRE(lo && hi, "lo or hi is NULL");
    FST_REQUIRE(res0 >= 1 && res1 >= 1, "resolutions must be >= 1");
    FST_REQUIRE(xyz != nullptr, "xyz is NULL");
    int dev = 0;
    FST_CUDA(cudaGetDevice(&dev));
    FST_REQUIRE(pointer_device(xyz) == dev, "xyz must be device memory of device %d", dev);
    const int a0 = axis == 0 ? 1 : 0, a1 = axis == 2 ? 1 : 2;
    const int64_t n = (int64_t)res0 * res1;
    int grid = (int)((n + 255) / 256);
    if (grid > 8 * sm_count()) grid = 8 * sm_count();
    slice_points_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(axis, (float)value, (float)lo[a0], (float)hi[a0],
                                                                (float)lo[a1], (float)hi[a1], res0, res1, xyz);
    FST_CHECK_LAUNCH();
    return FST_OK;
}
