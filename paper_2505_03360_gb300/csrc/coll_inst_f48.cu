// Instantiation of the fused collision kernel for N = 48, float compute.
#include "collision_impl.cuh"

namespace coll {
template int launch_one<48, float, double>(const CollArgs&, int, cudaStream_t);
template int launch_one<48, float, float>(const CollArgs&, int, cudaStream_t);
template int occupancy_one<48, float, double>(int*);
template int occupancy_one<48, float, float>(int*);
}  // namespace coll
