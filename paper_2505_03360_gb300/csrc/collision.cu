// Dispatch of the fused collision kernel over (N, compute type, io type).
// The kernels themselves are instantiated in coll_inst_*.cu (one translation
// unit per (N, compute type) so that they compile in parallel).
#include <cuda_runtime.h>

#include "coll_internal.h"
#include "collision_layout.cuh"

namespace coll {

template <int N, typename T, typename Tio, int V> int launch_one(const CollArgs& a, int grid, cudaStream_t st);
template <int N, typename T, typename Tio, int V> int occupancy_one(int* ctas);

template <int N, typename T, int V> LayoutInfo make_info_v() {
  using Ly = Lay<N, T, V>;
  LayoutInfo i;
  i.N = N;
  i.S0 = Ly::S0;
  i.w_smem = Cfg<N, T, V>::W;
  i.fh_smem = Cfg<N, T, V>::FH;
  i.g_smem = Cfg<N, T, V>::G;
  i.threads = kThreads;
  i.cluster = Cfg<N, T, V>::CLUSTER;
  i.w_bytes = Ly::round16(Ly::W_BYTES);
  i.fh_bytes = Ly::round16(Ly::FH_BYTES);
  i.g_bytes = Ly::round16(Ly::G_BYTES);
  i.smem = Ly::SMEM;
  i.ws = Ly::WS;
  return i;
}

template <int N, typename T> LayoutInfo make_info(int variant) {
  return variant ? make_info_v<N, T, 1>() : make_info_v<N, T, 0>();
}

bool layout_info(int N, int ctype, int variant, LayoutInfo* out) {
  if (ctype == kCMixSliced) return sliced_layout(N, out);                    // one shape for every variant
  if (is_mixed(ctype)) return mixed_layout(N, mixed_parts(ctype), out);
  if (ctype == kCDF) {
    switch (N) {
      case 16: *out = make_info<16, df>(variant); return true;
      case 24: *out = make_info<24, df>(variant); return true;
      case 32: *out = make_info<32, df>(variant); return true;
      default: return false;
    }
  }
  if (ctype == kCF64) {
    switch (N) {
      case 16: *out = make_info<16, double>(variant); return true;
      case 24: *out = make_info<24, double>(variant); return true;
      case 32: *out = make_info<32, double>(variant); return true;
      default: return false;
    }
  }
  switch (N) {
    case 16: *out = make_info<16, float>(variant); return true;
    case 24: *out = make_info<24, float>(variant); return true;
    case 32: *out = make_info<32, float>(variant); return true;
    case 48: *out = make_info<48, float>(variant); return true;
    case 64: *out = make_info<64, float>(variant); return true;
    default: return false;
  }
}

#define COLL_DISPATCH(FN, ...)                                                              \
  if (ctype == kCDF) {                                                                      \
    if (io_f64) {                                                                           \
      switch (N) {                                                                          \
        case 16: return variant ? FN<16, df, double, 1>(__VA_ARGS__) : FN<16, df, double, 0>(__VA_ARGS__);                                    \
        case 24: return variant ? FN<24, df, double, 1>(__VA_ARGS__) : FN<24, df, double, 0>(__VA_ARGS__);                                    \
        case 32: return variant ? FN<32, df, double, 1>(__VA_ARGS__) : FN<32, df, double, 0>(__VA_ARGS__);                                    \
      }                                                                                     \
    } else {                                                                                \
      switch (N) {                                                                          \
        case 16: return variant ? FN<16, df, float, 1>(__VA_ARGS__) : FN<16, df, float, 0>(__VA_ARGS__);                                     \
        case 24: return variant ? FN<24, df, float, 1>(__VA_ARGS__) : FN<24, df, float, 0>(__VA_ARGS__);                                     \
        case 32: return variant ? FN<32, df, float, 1>(__VA_ARGS__) : FN<32, df, float, 0>(__VA_ARGS__);                                     \
      }                                                                                     \
    }                                                                                       \
  } else if (ctype == kCF64) {                                                              \
    if (io_f64) {                                                                           \
      switch (N) {                                                                          \
        case 16: return variant ? FN<16, double, double, 1>(__VA_ARGS__) : FN<16, double, double, 0>(__VA_ARGS__);                                \
        case 24: return variant ? FN<24, double, double, 1>(__VA_ARGS__) : FN<24, double, double, 0>(__VA_ARGS__);                                \
        case 32: return variant ? FN<32, double, double, 1>(__VA_ARGS__) : FN<32, double, double, 0>(__VA_ARGS__);                                \
      }                                                                                     \
    } else {                                                                                \
      switch (N) {                                                                          \
        case 16: return variant ? FN<16, double, float, 1>(__VA_ARGS__) : FN<16, double, float, 0>(__VA_ARGS__);                                 \
        case 24: return variant ? FN<24, double, float, 1>(__VA_ARGS__) : FN<24, double, float, 0>(__VA_ARGS__);                                 \
        case 32: return variant ? FN<32, double, float, 1>(__VA_ARGS__) : FN<32, double, float, 0>(__VA_ARGS__);                                 \
      }                                                                                     \
    }                                                                                       \
  } else {                                                                                  \
    if (io_f64) {                                                                           \
      switch (N) {                                                                          \
        case 16: return variant ? FN<16, float, double, 1>(__VA_ARGS__) : FN<16, float, double, 0>(__VA_ARGS__);                                 \
        case 24: return variant ? FN<24, float, double, 1>(__VA_ARGS__) : FN<24, float, double, 0>(__VA_ARGS__);                                 \
        case 32: return variant ? FN<32, float, double, 1>(__VA_ARGS__) : FN<32, float, double, 0>(__VA_ARGS__);                                 \
        case 48: return variant ? FN<48, float, double, 1>(__VA_ARGS__) : FN<48, float, double, 0>(__VA_ARGS__);                                 \
        case 64: return variant ? FN<64, float, double, 1>(__VA_ARGS__) : FN<64, float, double, 0>(__VA_ARGS__);                                 \
      }                                                                                     \
    } else {                                                                                \
      switch (N) {                                                                          \
        case 16: return variant ? FN<16, float, float, 1>(__VA_ARGS__) : FN<16, float, float, 0>(__VA_ARGS__);                                  \
        case 24: return variant ? FN<24, float, float, 1>(__VA_ARGS__) : FN<24, float, float, 0>(__VA_ARGS__);                                  \
        case 32: return variant ? FN<32, float, float, 1>(__VA_ARGS__) : FN<32, float, float, 0>(__VA_ARGS__);                                  \
        case 48: return variant ? FN<48, float, float, 1>(__VA_ARGS__) : FN<48, float, float, 0>(__VA_ARGS__);                                  \
        case 64: return variant ? FN<64, float, float, 1>(__VA_ARGS__) : FN<64, float, float, 0>(__VA_ARGS__);                                  \
      }                                                                                     \
    }                                                                                       \
  }                                                                                         \
  return int(cudaErrorInvalidValue);

int ragged_launch_f32(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st);
int ragged_launch_f64(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st);
int ragged_launch_x(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st);
int ragged_occupancy_f32(int* ctas);
int ragged_occupancy_f64(int* ctas);
int ragged_occupancy_x(int* ctas);
size_t ragged_smem_f32();
size_t ragged_smem_f64();
size_t ragged_smem_x();
size_t ragged_ws_f32();
size_t ragged_ws_f64();
size_t ragged_ws_x();

int launch_ragged(int ctype, const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, void* stream) {
  count_launches(1);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (ctype) {
    case kCF32: return ragged_launch_f32(t, ws, ws_per_cta, grid, st);
    case kCF64: return ragged_launch_f64(t, ws, ws_per_cta, grid, st);
    case kCDF: return ragged_launch_x(t, ws, ws_per_cta, grid, st);
    case kCMixSliced:                 // slots after the 256-byte head, as for the SIMT kernel
      return t.n_items > 0 ? launch_sliced_ragged(t.items[0].N, t.io_f64 != 0, t, static_cast<char*>(ws) + 256,
                                                  ws_per_cta, grid, stream)
                           : int(cudaErrorInvalidValue);
  }
  return int(cudaErrorInvalidValue);
}

int ragged_layout(int ctype, size_t* smem_bytes, size_t* ws_per_cta) {
  switch (ctype) {
    case kCF32: *smem_bytes = ragged_smem_f32(); *ws_per_cta = ragged_ws_f32(); return 0;
    case kCF64: *smem_bytes = ragged_smem_f64(); *ws_per_cta = ragged_ws_f64(); return 0;
    case kCDF: *smem_bytes = ragged_smem_x(); *ws_per_cta = ragged_ws_x(); return 0;
  }
  return int(cudaErrorInvalidValue);
}

template <int N, typename T> size_t body_smem(int variant) {
  return variant ? Lay<N, T, RaggedBody<N, T, 1>::v>::SMEM : Lay<N, T, RaggedBody<N, T, 0>::v>::SMEM;
}

size_t ragged_body_smem(int N, int ctype, int variant) {
  if (ctype == kCF32) {
    switch (N) {
      case 16: return body_smem<16, float>(variant);
      case 24: return body_smem<24, float>(variant);
      case 32: return body_smem<32, float>(variant);
      case 48: return body_smem<48, float>(variant);
      case 64: return body_smem<64, float>(variant);
    }
    return 0;
  }
  if (ctype == kCF64 || ctype == kCDF) {
    switch (N) {
      case 16: return ctype == kCF64 ? body_smem<16, double>(variant) : body_smem<16, df>(variant);
      case 24: return ctype == kCF64 ? body_smem<24, double>(variant) : body_smem<24, df>(variant);
      case 32: return ctype == kCF64 ? body_smem<32, double>(variant) : body_smem<32, df>(variant);
    }
  }
  return 0;
}

int ragged_max_ctas_per_sm(int ctype, int* ctas) {
  switch (ctype) {
    case kCF32: return ragged_occupancy_f32(ctas);
    case kCF64: return ragged_occupancy_f64(ctas);
    case kCDF: return ragged_occupancy_x(ctas);
  }
  return int(cudaErrorInvalidValue);
}

int launch_collision(int N, int ctype, bool io_f64, int variant, const CollArgs& a, int grid, void* stream) {
  count_launches(1);
  if (ctype == kCMixSliced) return launch_sliced(N, io_f64, a, grid, stream);
  if (is_mixed(ctype)) return launch_mixed(N, io_f64, mixed_parts(ctype), a, grid, stream);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  COLL_DISPATCH(launch_one, a, grid, st)
}

int collision_max_ctas_per_sm(int N, int ctype, bool io_f64, int variant, int* ctas) {
  if (ctype == kCMixSliced) return sliced_max_ctas_per_sm(N, io_f64, ctas);
  if (is_mixed(ctype)) return mixed_max_ctas_per_sm(N, io_f64, mixed_parts(ctype), ctas);
  COLL_DISPATCH(occupancy_one, ctas)
}

}  // namespace coll
