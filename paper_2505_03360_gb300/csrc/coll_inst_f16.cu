// Instantiation of the fused collision kernel for N = 16, float compute.
#include "collision_impl.cuh"

namespace coll {
template int launch_one<16, float, double>(const CollArgs&, int, cudaStream_t);
template int launch_one<16, float, float>(const CollArgs&, int, cudaStream_t);
template int occupancy_one<16, float, double>(int*);
template int occupancy_one<16, float, float>(int*);
}  // namespace coll
