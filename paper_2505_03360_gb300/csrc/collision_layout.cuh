// Compile-time layouts of the fused collision kernel (see collision_impl.cuh).
#pragma once

#include <cstddef>

namespace coll {

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };

// ----------------------------------------------------------------- layouts
template <int N, typename T> struct Cfg;
//                 S0  W_smem Fh_smem G_smem
template <> struct Cfg<16, double> { static constexpr int S0 = 1; static constexpr bool W = true, FH = true, G = true; };
template <> struct Cfg<24, double> { static constexpr int S0 = 2; static constexpr bool W = true, FH = false, G = false; };
template <> struct Cfg<32, double> { static constexpr int S0 = 4; static constexpr bool W = true, FH = false, G = false; };
template <> struct Cfg<16, float> { static constexpr int S0 = 1; static constexpr bool W = true, FH = true, G = true; };
template <> struct Cfg<24, float> { static constexpr int S0 = 1; static constexpr bool W = true, FH = true, G = true; };
template <> struct Cfg<32, float> { static constexpr int S0 = 2; static constexpr bool W = true, FH = false, G = false; };
template <> struct Cfg<48, float> { static constexpr int S0 = 4; static constexpr bool W = true, FH = false, G = false; };
template <> struct Cfg<64, float> { static constexpr int S0 = 1; static constexpr bool W = false, FH = false, G = false; };

constexpr int kThreads = 256;

template <int N, typename T> struct Lay {
  using Cf = Cfg<N, T>;
  static constexpr int H = N / 2;
  static constexpr int FH_ROW = H + 1;
  static constexpr int W_ROW = N + 1;
  static constexpr int S0 = Cf::S0;
  static constexpr int NS = N / S0;
  static constexpr size_t W_BYTES = size_t(NS) * N * W_ROW * 2 * sizeof(T);
  static constexpr size_t FH_BYTES = size_t(N) * N * FH_ROW * 2 * sizeof(T);
  static constexpr size_t G_BYTES = size_t(N) * N * N * sizeof(T);
  static constexpr size_t round16(size_t b) { return (b + 15) / 16 * 16; }
  static constexpr size_t SMEM = (Cf::W ? round16(W_BYTES) : 0) + (Cf::FH ? round16(FH_BYTES) : 0) +
                                 (Cf::G ? round16(G_BYTES) : 0);
  static constexpr size_t WS = (Cf::W ? 0 : round16(W_BYTES)) + (Cf::FH ? 0 : round16(FH_BYTES)) +
                               (Cf::G ? 0 : round16(G_BYTES));
};

}  // namespace coll
