// coll_advance: explicit Euler step of the space-homogeneous equation
// d f / dt = Q(f, f) (eq. 2.1 of arxiv 2505.03360 without transport, eps = 1):
// f <- f + dt Q, elementwise, in the storage type.  Used by the serving loop
// between repeated evaluations of a request's cells.
#include <cuda_runtime.h>

#include "coll_internal.h"

namespace {

template <typename T>
__global__ void advance_kernel(T* __restrict__ f, const T* __restrict__ Q, long long n, T dt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) f[i] += dt * Q[i];
}

}  // namespace

extern "C" coll_status coll_advance(void* f, const void* Q, int64_t n, double dt, int32_t io_dtype,
                                    coll_stream stream) {
  if (n < 0 || (io_dtype != 0 && io_dtype != 1)) return COLL_EINVAL;
  if (n == 0) return COLL_OK;
  if (!f || !Q || f == Q) return COLL_EINVAL;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long blocks = (n + 255) / 256;
  const long long cap = (long long)sms * 8;
  if (blocks > cap) blocks = cap;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  coll::count_launches(1);
  if (io_dtype == 0)
    advance_kernel<double><<<int(blocks), 256, 0, st>>>(static_cast<double*>(f), static_cast<const double*>(Q), n, dt);
  else
    advance_kernel<float><<<int(blocks), 256, 0, st>>>(static_cast<float*>(f), static_cast<const float*>(Q), n,
                                                       float(dt));
  return cudaGetLastError() == cudaSuccess ? COLL_OK : COLL_ECUDA;
}
