// 2D Maxwell-molecule operator (m2d_impl.cuh), FP64 compute: N = 16, 32.
#include "m2d_impl.cuh"

namespace coll {
int m2d_launch_f64(int N, bool io_f64, const M2Args& a, int grid, void* stream) {
  return M2Dispatch<double, 16, 32>::launch(N, io_f64, a, grid, static_cast<cudaStream_t>(stream));
}
int m2d_occupancy_f64(int N, bool io_f64, int* ctas) { return M2Dispatch<double, 16, 32>::occupancy(N, io_f64, ctas); }
}  // namespace coll
