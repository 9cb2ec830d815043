// Ragged persistent collision kernel, df compute, double io, N in {16, 24, 32}.
#include "collision_impl.cuh"

namespace coll {
using Ragged_x = RaggedLaunch<df, double, 16, 24, 32>;
int ragged_launch_x(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st) {
  return Ragged_x::launch(t, ws, ws_per_cta, grid, st);
}
int ragged_occupancy_x(int* ctas) { return Ragged_x::occupancy(ctas); }
size_t ragged_smem_x() { return Ragged_x::smem(); }
size_t ragged_ws_x() { return Ragged_x::ws(); }
}  // namespace coll
