// Internal declarations shared by the host API (api.cu, plan.cpp) and the
// CUDA kernels.  Not part of the public ABI (see include/coll.h).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/coll.h"

namespace coll {

// ---------------------------------------------------------------------------
// Compile-time layout of the fused collision kernel for (N, precision).
//
// Per cell the kernel holds three arrays:
//   Fh  forward half spectrum, [k0][k1][k2 < N/2] complex, rows padded to N/2+1
//   W   one v0-slab of the per-term spectrum after the axis-0 inverse pass,
//       [v0 / S0][k1][k2 < N] complex, rows padded to N+1 (bank-conflict free
//       row reads in the last pass); slab s holds the planes v0 = s mod S0
//   G   gain accumulator, N^3 reals
// Each array lives in shared memory when it fits (227 KB per CTA) and
// otherwise in the CTA's slice of the global workspace (L2 resident for the
// sizes used).  S0 splits the axis-0 inverse transform by decimation in
// frequency so that a slab of W fits on chip.
// ---------------------------------------------------------------------------
struct LayoutInfo {
  int N, S0;
  bool w_smem, fh_smem, g_smem;
  int threads;
  int cluster = 0;          // CTAs per cell (thread-block cluster), 0: one CTA per cell
  size_t w_bytes, fh_bytes, g_bytes;
  size_t smem = 0;          // dynamic shared memory per CTA
  size_t ws = 0;            // global workspace per CTA (the cluster form: a share of the cluster's)
  size_t smem_bytes() const { return smem; }
  size_t ws_bytes_per_cta() const { return (ws + 255) / 256 * 256; }
};

// compute types of the collision kernel
enum CType : int { kCF64 = 0, kCF32 = 1, kCDF = 2, kCMixF16 = 3, kCMixBF16 = 4, kCMixSliced = 5 };
// tensor-core compute types (N = 16 and 32, no ragged launches)
inline bool is_mixed(int ctype) { return ctype == kCMixF16 || ctype == kCMixBF16 || ctype == kCMixSliced; }
inline int mixed_parts(int ctype) { return ctype == kCMixBF16 ? 3 : 2; }

#ifdef __CUDACC__
#define COLL_HD __host__ __device__
#else
#define COLL_HD
#endif
// Device image of a mixed-precision plan (mixed.cu): per-term tables, the
// per-term bound max|A + iB|, then the tensor-core DFT matrices.
COLL_HD inline size_t mixed_tab_bytes(int N, int n_terms) { return size_t(n_terms) * N * (N / 2) * N * 8; }
COLL_HD inline size_t mixed_tmax_offset(int N, int n_terms) { return mixed_tab_bytes(N, n_terms); }
COLL_HD inline size_t mixed_img_offset(int N, int n_terms) {
  return (mixed_tab_bytes(N, n_terms) + size_t(n_terms) * 4 + 1023) / 1024 * 1024;
}

// Device image of a sliced plan (sliced.cu): per-term tables as float pairs
// (A_h, A_l, B_h, B_l), the per-term bound max|A + iB|, then the f16 matrices.
COLL_HD inline size_t sliced_tab_bytes(int N, int n_terms) { return size_t(n_terms) * N * (N / 2) * N * 16; }
COLL_HD inline size_t sliced_tmax_offset(int N, int n_terms) { return sliced_tab_bytes(N, n_terms); }
COLL_HD inline size_t sliced_img_offset(int N, int n_terms) {
  return (sliced_tab_bytes(N, n_terms) + size_t(n_terms) * 4 + 1023) / 1024 * 1024;
}

// Returns false if (N, ctype) has no kernel instantiation.
bool layout_info(int N, int ctype, int variant, LayoutInfo* out);

struct CollArgs {
  const void* f;
  void* Q;
  long long n_cells;
  const void* tab;          // [n_terms][N][N][N/2] pairs (A, B) of the compute type
  int n_terms;
  void* ws;
  size_t ws_per_cta;
  int* status;              // sticky device status bits
};

// status bits written by kernels
enum : int { kStatusNonFinite = 1, kStatusTimeout = 2 };

// Launchers (collision.cu); return cudaError_t as int.
constexpr int kVariants = 2;   // slab-shape variants per (N, compute type), chosen by the autotuner
int launch_collision(int N, int ctype, bool io_f64, int variant, const CollArgs& a, int grid, void* stream);
int collision_max_ctas_per_sm(int N, int ctype, bool io_f64, int variant, int* ctas);

// Ragged launch: one persistent kernel over groups of cells with mixed N
// (ragged_*.cu).  Groups are passed by value in the kernel parameters.
constexpr int kMaxRaggedGroups = 256;
struct RaggedItem {            // one group of cells evaluated with one plan
  const void* f;
  void* Q;
  const void* tab;
  long long n_cells;
  long long first_unit;        // prefix sum of n_cells in schedule order
  int* status;
  int N;
  int n_terms;
  int variant;                 // the plan's slab shape (coll_plan_autotune / coll_plan_set_variant)
};
struct RaggedTable {
  RaggedItem items[kMaxRaggedGroups];
  int n_items;
  long long total_units;
  size_t smem_bytes;           // dynamic shared memory of the largest body the launch runs
  int io_f64;                  // 1: double f and Q (the fixed-point-slice groups may use either)
};
// ctype: kCF32 (float io) or kCF64 / kCDF (double io)
int launch_ragged(int ctype, const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, void* stream);
int ragged_layout(int ctype, size_t* smem_bytes, size_t* ws_per_cta);
// shared memory of the body a ragged launch runs for a group of (N, compute type, variant)
size_t ragged_body_smem(int N, int ctype, int variant);
int ragged_max_ctas_per_sm(int ctype, int* ctas);

// Mixed-precision (tensor-core DFT-GEMM) collision kernel (mixed.cu)
bool mixed_layout(int N, int parts, LayoutInfo* out);
int launch_mixed(int N, bool io_f64, int parts, const CollArgs& a, int grid, void* stream);
int mixed_max_ctas_per_sm(int N, bool io_f64, int parts, int* ctas);
int mixed_set_drop_commit(int on);      // failure injection (coll_debug.h)

// Fixed-point-slice tensor-core collision kernel (sliced.cu)
bool sliced_layout(int N, LayoutInfo* out);
int launch_sliced(int N, bool io_f64, const CollArgs& a, int grid, void* stream);
// one launch over the cells of several fixed-point-slice plans of one N (a ragged table)
int launch_sliced_ragged(int N, bool io_f64, const RaggedTable& t, void* ws, size_t ws_per_cta, int grid,
                         void* stream);
int sliced_max_ctas_per_sm(int N, bool io_f64, int* ctas);

// Moments kernel (moments.cu)
int launch_moments(const void* f, int io_f64, int N, double L, long long n_cells, double eta0,
                   double delta0, coll_moments* mom, uint8_t* mask, void* stream);
// Galerkin mode (galerkin.cu): spectral resampling N^3 <-> (3N/2)^3 per cell,
// through two complex scratch buffers of galerkin_scratch_elems(N) elements per cell
size_t galerkin_scratch_elems(int N);
int launch_galerkin_resample(bool to_pad, int N, bool compute_f64, bool io_f64, const void* in, void* out,
                             void* sa, void* sb, long long n_cells, void* stream);
// Collision invariants of Q per cell (moments.cu)
int launch_conservation(const void* Q, int io_f64, int N, double L, long long n_cells, double* out, void* stream);

// Regime update on the 2D grid (regime.cu)
int launch_regime(const double* fields, const double* l1, const uint8_t* r_in, int nx, int ny,
                  const coll_regime_params& p, uint8_t* r_out, double* ind, void* stream);

// Penalised IMEX stages (imex.cu)
int launch_imex(int stage, const void* f, const void* Y, const void* Q1, const void* Q2, const void* tr,
                const coll_moments* mom0, const coll_moments* mom1, bool io_f64, int N, double L, long long n_cells,
                double dt, double eps, void* out, void* stream);

// ES-BGK relaxation step (esbgk.cu)
int launch_esbgk(const void* f, const coll_moments* mom, bool io_f64, int N, double L, long long n_cells, double dt,
                 double eps, double beta, double mu0, void* out, void* stream);

// 2D Maxwell-molecule operator (m2d_impl.cuh; m2d_d.cu, m2d_f.cu, m2d_x.cu)
struct M2Args {
  const void* f;
  void* Q;
  long long n_cells;
  const void* tab;          // [n_terms][N][N/2] pairs (A, B) of the compute type
  int n_terms;
  int* status;
};
int m2d_launch_f64(int N, bool io_f64, const M2Args& a, int grid, void* stream);
int m2d_occupancy_f64(int N, bool io_f64, int* ctas);
int m2d_launch_f32(int N, bool io_f64, const M2Args& a, int grid, void* stream);
int m2d_occupancy_f32(int N, bool io_f64, int* ctas);
int m2d_launch_df(int N, bool io_f64, const M2Args& a, int grid, void* stream);
int m2d_occupancy_df(int N, bool io_f64, int* ctas);
// host tables: [n_terms][N][N/2][2] doubles, A gain terms then the loss term
coll_status build_m2d_tables(const coll_m2d_plan_desc& d, int* n_terms, std::vector<double>* tab);

// Host-side plan building (plan.cpp)
struct HostTables {
  int n_terms;
  std::vector<double> tab;    // [n_terms][N][N][N/2][2]
};
// mode_cut > 0: the tables of a grid of d.N points that carry only the modes
// with every |k_d| < mode_cut / 2 (the Galerkin mode's padded grid)
coll_status build_tables(const coll_plan_desc& d, HostTables* out, int mode_cut = 0);
coll_status build_mixed_image(const HostTables& ht, int N, int parts, std::vector<unsigned char>* out);
coll_status build_sliced_image(const HostTables& ht, int N, std::vector<unsigned char>* out);

void count_launches(long long n);

}  // namespace coll

struct coll_plan_s {
  coll_plan_desc d;
  int device;
  int n_terms;
  int ctype;         // compute type of the transforms (coll::CType)
  bool io_f64;       // f / Q element type
  void* tab_dev;     // device tables in the compute type
  size_t tab_bytes;
  int* status_dev;   // sticky status word
  coll::LayoutInfo lay[coll::kVariants];   // per slab-shape variant
  int ctas_per_sm[coll::kVariants];
  int variant;                             // chosen by coll_plan_autotune (default 0)
  int num_sms;
  int Nk;            // grid of the collision kernel: N, or 3N/2 in the Galerkin mode
  bool galerkin;     // dealias = 1: products on the 3N/2 grid, result projected back
};

struct coll_m2d_plan_s {
  coll_m2d_plan_desc d;
  int device;
  int n_terms;
  int ctype;         // coll::kCF64, kCF32 or kCDF
  bool io_f64;
  void* tab_dev;
  size_t tab_bytes;
  int* status_dev;
  int ctas_per_sm;
  int num_sms;
};
