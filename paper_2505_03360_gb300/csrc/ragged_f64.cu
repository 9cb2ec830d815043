// Ragged persistent collision kernel, double compute, double io, N in {16, 24, 32}.
#include "collision_impl.cuh"

namespace coll {
using Ragged_f64 = RaggedLaunch<double, double, 16, 24, 32>;
int ragged_launch_f64(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st) {
  return Ragged_f64::launch(t, ws, ws_per_cta, grid, st);
}
int ragged_occupancy_f64(int* ctas) { return Ragged_f64::occupancy(ctas); }
size_t ragged_smem_f64() { return Ragged_f64::smem(); }
size_t ragged_ws_f64() { return Ragged_f64::ws(); }
}  // namespace coll
