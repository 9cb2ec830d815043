// Ragged persistent collision kernel, float compute, float io, N in {16, 24, 32, 48, 64}.
#include "collision_impl.cuh"

namespace coll {
using Ragged_f32 = RaggedLaunch<float, float, 16, 24, 32, 48, 64>;
int ragged_launch_f32(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st) {
  return Ragged_f32::launch(t, ws, ws_per_cta, grid, st);
}
int ragged_occupancy_f32(int* ctas) { return Ragged_f32::occupancy(ctas); }
size_t ragged_smem_f32() { return Ragged_f32::smem(); }
size_t ragged_ws_f32() { return Ragged_f32::ws(); }
}  // namespace coll
