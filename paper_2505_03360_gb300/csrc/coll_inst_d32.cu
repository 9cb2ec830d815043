// Instantiation of the fused collision kernel for N = 32, double compute.
#include "collision_impl.cuh"

namespace coll {
template int launch_one<32, double, double>(const CollArgs&, int, cudaStream_t);
template int launch_one<32, double, float>(const CollArgs&, int, cudaStream_t);
template int occupancy_one<32, double, double>(int*);
template int occupancy_one<32, double, float>(int*);
}  // namespace coll
