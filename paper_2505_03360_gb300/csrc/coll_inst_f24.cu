// Instantiation of the fused collision kernel for N = 24, float compute.
#include "collision_impl.cuh"

namespace coll {
template int launch_one<24, float, double>(const CollArgs&, int, cudaStream_t);
template int launch_one<24, float, float>(const CollArgs&, int, cudaStream_t);
template int occupancy_one<24, float, double>(int*);
template int occupancy_one<24, float, float>(int*);
}  // namespace coll
