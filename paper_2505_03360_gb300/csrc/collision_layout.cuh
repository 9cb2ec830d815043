// Compile-time layouts of the fused collision kernel (see collision_impl.cuh).
#pragma once

#include <cstddef>

#include "dfloat.cuh"

namespace coll {

template <typename T> struct C2;
template <> struct C2<double> { using type = double2; };
template <> struct C2<float> { using type = float2; };
template <> struct C2<df> { using type = cdf; };

// ----------------------------------------------------------------- layouts
// Per (N, compute type, variant V): S0 v0-slabs; which arrays live in shared
// memory (W = one slab of the per-term spectrum, Fh = forward half spectrum,
// G = one slab of the gain accumulator); whether Fh rows are padded.  Two
// variants per (N, type) give the autotuner two slab shapes to choose from.
// P1F (full first pass): the axis-0 inverse of each term runs once over full
// pencils into a global buffer of the whole term, and the slabs are copied
// from it (terms outer, slabs inner, the gain accumulator of each slab saved
// to and restored from global memory); otherwise (terms inner, slabs outer)
// every slab re-forms its planes from the spectrum by decimation in frequency.
template <int N, typename T, int V = 0> struct Cfg;
#define COLL_CFG(N_, T_, V_, S0_, W_, FH_, G_, PAD_)                                      \
  template <> struct Cfg<N_, T_, V_> {                                                     \
    static constexpr int S0 = S0_;                                                         \
    static constexpr bool W = W_, FH = FH_, G = G_, FH_PAD = PAD_;                         \
    static constexpr bool P1F = false;                                                     \
    static constexpr int CLUSTER = 0;                                                      \
  };
#define COLL_CFG_P1F(N_, T_, V_, S0_, FH_, PAD_)                                           \
  template <> struct Cfg<N_, T_, V_> {                                                     \
    static constexpr int S0 = S0_;                                                         \
    static constexpr bool W = true, FH = FH_, G = true, FH_PAD = PAD_;                     \
    static constexpr bool P1F = true;                                                      \
    static constexpr int CLUSTER = 0;                                                      \
  };
// Cluster form (full first pass shared by a thread-block cluster): C_ CTAs
// evaluate one cell together; the forward spectrum Fh and two term buffers
// (double-buffered over the terms) live in the cluster's global workspace, every
// pass's pencils are split over the CTAs, and CTA r owns S0_ / C_ of the slabs
// with their gain accumulators in its shared memory for all terms.
#define COLL_CFG_CLUSTER(N_, T_, V_, S0_, C_)                                              \
  template <> struct Cfg<N_, T_, V_> {                                                     \
    static constexpr int S0 = S0_;                                                         \
    static constexpr bool W = true, FH = false, G = true, FH_PAD = true;                   \
    static constexpr bool P1F = true;                                                      \
    static constexpr int CLUSTER = C_;                                                     \
  };
//        N   T      V  S0  W     Fh     G      Fh padded
COLL_CFG(16, double, 0,  1, true, true,  true,  true)
COLL_CFG_P1F(24, double, 0, 2, false, true)
COLL_CFG_P1F(32, double, 0, 4, false, true)
COLL_CFG(16, df,     0,  1, true, true,  true,  true)
COLL_CFG(24, df,     0,  2, true, false, true,  true)
COLL_CFG(32, df,     0,  4, true, false, true,  true)
COLL_CFG(16, float,  0,  1, true, true,  true,  true)
COLL_CFG(24, float,  0,  1, true, true,  true,  false)
COLL_CFG_P1F(32, float,  0, 4, true, false)
COLL_CFG_P1F(48, float, 0, 8, false, true)
COLL_CFG_P1F(64, float, 0, 16, false, true)
COLL_CFG(16, double, 1,  2, true, true,  true,  true)
COLL_CFG(24, double, 1,  4, true, true,  true,  true)
COLL_CFG(32, double, 1,  8, true, false, true,  true)
COLL_CFG(16, df,     1,  2, true, true,  true,  true)
COLL_CFG(24, df,     1,  4, true, true,  true,  true)
COLL_CFG(32, df,     1,  8, true, false, true,  true)
COLL_CFG(16, float,  1,  2, true, true,  true,  true)
COLL_CFG(24, float,  1,  1, true, false, true,  true)
COLL_CFG(32, float,  1,  2, true, false, true,  true)
COLL_CFG_CLUSTER(48, float, 1, 12, 4)
COLL_CFG(64, float,  1,  8, false, false, true, true)
// bodies of the ragged kernel only (RaggedBody below), not plan variants
COLL_CFG_P1F(32, float, 2, 4, false, true)
#undef COLL_CFG
#undef COLL_CFG_P1F
#undef COLL_CFG_CLUSTER

constexpr int kThreads = 256;

// The body the ragged kernel (one CTA per cell, one launch for every group) runs
// for variant V of (N, T): V itself, or a variant with the same arithmetic (equal
// results bit for bit) that fits that launch better.  The cluster form needs a
// cluster launch of its own (its cells take the one-CTA full first pass); FP32
// N = 24 and 32 variants 0 keep Fh in shared memory too (228 and 227 KB), and
// the ragged launch requests the shared memory of its largest body, so either
// would leave every other body of the launch the smallest L1 (the N = 48 body,
// which reads its spectrum and tables through L1, runs 20 % slower): their cells
// take the same schedule with Fh in global memory (N = 24 variant 1, 173 KB;
// N = 32 configuration 2, 101 KB).
template <int N, typename T, int V> struct RaggedBody { static constexpr int v = Cfg<N, T, V>::CLUSTER > 0 ? 0 : V; };
template <> struct RaggedBody<24, float, 0> { static constexpr int v = 1; };
template <> struct RaggedBody<32, float, 0> { static constexpr int v = 2; };

template <int N, typename T, int V = 0> struct Lay {
  using Cf = Cfg<N, T, V>;
  static constexpr int H = N / 2;
  static constexpr int FH_ROW = Cf::FH_PAD ? H + 1 : H;
  static constexpr int W_ROW = N + 1;
  static constexpr int G_ROW = N + 1;                                       // padded gain rows
  static constexpr int S0 = Cf::S0;
  static constexpr int NS = N / S0;
  static constexpr size_t W_BYTES = size_t(NS) * N * W_ROW * 2 * sizeof(T);
  static constexpr size_t FH_BYTES = size_t(N) * N * FH_ROW * 2 * sizeof(T);
  static constexpr size_t G_BYTES = size_t(NS) * N * G_ROW * sizeof(T);    // one slab
  static constexpr size_t round16(size_t b) { return (b + 15) / 16 * 16; }
  static constexpr int SLABS_PER_CTA = Cf::CLUSTER > 0 ? S0 / Cf::CLUSTER : 1;  // gain slabs in shared memory
  static constexpr size_t SMEM = (Cf::W ? round16(W_BYTES) : 0) + (Cf::FH ? round16(FH_BYTES) : 0) +
                                 (Cf::G ? SLABS_PER_CTA * round16(G_BYTES) : 0);
  // P1F: the whole term's spectrum after the axis-0 pass and the whole gain accumulator
  static constexpr size_t WG_BYTES = Cf::P1F ? size_t(N) * N * N * 2 * sizeof(T) : 0;
  static constexpr size_t GG_BYTES = Cf::P1F && Cf::CLUSTER == 0 ? size_t(N) * N * G_ROW * sizeof(T) : 0;
  // cluster form: Fh and two term buffers per cluster, counted as C equal shares per CTA
  static constexpr size_t WS_CLUSTER = round16(FH_BYTES) + 2 * round16(WG_BYTES);
  static constexpr size_t WS = Cf::CLUSTER > 0
                                   ? (WS_CLUSTER + Cf::CLUSTER - 1) / Cf::CLUSTER
                                   : (Cf::W ? 0 : round16(W_BYTES)) + (Cf::FH ? 0 : round16(FH_BYTES)) +
                                         (Cf::G ? 0 : round16(G_BYTES)) + round16(WG_BYTES) + round16(GG_BYTES);
  static_assert(SMEM <= 232448, "shared-memory layout exceeds 227 KB");
  static_assert(N % S0 == 0, "S0 must divide N");
  static_assert(Cf::CLUSTER == 0 || (Cf::P1F && Cf::W && Cf::G && !Cf::FH && S0 % Cf::CLUSTER == 0),
                "the cluster form: full first pass, Fh global, whole slabs per CTA");
};

}  // namespace coll
