// Instantiation of the fused collision kernel for N = 24, float compute.
#include "collision_impl.cuh"

namespace coll {
template int launch_one<24, float, double, 0>(const CollArgs&, int, cudaStream_t);
template int launch_one<24, float, double, 1>(const CollArgs&, int, cudaStream_t);
template int launch_one<24, float, float, 0>(const CollArgs&, int, cudaStream_t);
template int launch_one<24, float, float, 1>(const CollArgs&, int, cudaStream_t);
template int occupancy_one<24, float, double, 0>(int*);
template int occupancy_one<24, float, double, 1>(int*);
template int occupancy_one<24, float, float, 0>(int*);
template int occupancy_one<24, float, float, 1>(int*);
}  // namespace coll
