// Instantiation of the fused collision kernel for N = 32, float-pair compute.
#include "collision_impl.cuh"

namespace coll {
template int launch_one<32, df, double>(const CollArgs&, int, cudaStream_t);
template int launch_one<32, df, float>(const CollArgs&, int, cudaStream_t);
template int occupancy_one<32, df, double>(int*);
template int occupancy_one<32, df, float>(int*);
}  // namespace coll
