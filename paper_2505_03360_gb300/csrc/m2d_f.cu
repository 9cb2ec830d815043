// 2D Maxwell-molecule operator (m2d_impl.cuh), FP32 compute: N = 16, 32, 64.
#include "m2d_impl.cuh"

namespace coll {
int m2d_launch_f32(int N, bool io_f64, const M2Args& a, int grid, void* stream) {
  return M2Dispatch<float, 16, 32, 64>::launch(N, io_f64, a, grid, static_cast<cudaStream_t>(stream));
}
int m2d_occupancy_f32(int N, bool io_f64, int* ctas) {
  return M2Dispatch<float, 16, 32, 64>::occupancy(N, io_f64, ctas);
}
}  // namespace coll
