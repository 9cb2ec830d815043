// Fixed-point-slice tensor-core collision path (COLL_MIXED_SLICED).
//
// Same index-space algorithm and pass structure as mixed.cu (arxiv 2505.03360,
// sec. 4.4.1: F = DFT3(f), z_t = IDFT3((A_t + i B_t) F), Q = sum_t Re z_t Im z_t,
// the last term being the loss term), every 1D transform a DFT-GEMM on the
// tcgen05 tensor cores, but with an operand encoding whose leading products
// the tensor core's FP32 accumulator sums exactly, so that each transform
// keeps about 38 significant bits instead of FP32's 24.
//
// Encoding.  Every real component x of a pass input is written, with
// q = 2^(E-9) and 2^E above the maximum modulus of the pass input, as
//     x = q (s0 + 2^-9 s1 + 2^-18 (s2 + sT)),
// s0, s1, s2 integers (|s0| <= 512, |s1|, |s2| <= 256) and sT in [-1/2, 1/2]
// rounded to f16; all four parts are f16 values (integers up to 2048 are exact
// in f16).  The DFT matrix entries D (|D| <= 1) are split the same way with
// q = 2^-9:  D = 2^-9 (d0 + 2^-9 d1 + 2^-18 (d2 + dT)).  Grouping the products
// by level, x D / (q 2^-9) = L0 + 2^-9 L1 + 2^-18 L2 with
//     L0 = s0 d0                                        (exact)
//     L1 = s0 d1 + s1 d0                                (exact)
//     L2 = s0 d2 + s1 d1 + s2 d0 + s0 dT + sT d0 + 2^-9 (s1 d2 + s2 d1)
// f16 x f16 products are exact in FP32, and every partial sum of L0 and of L1
// is an integer below 2^24 in modulus (|s0| sum_k |d0| <= 512 (512 N sqrt 2 + N)
// and the like), so the FP32 accumulators of L0 and of 2^-9 L1 (taken against
// the matrices 2^-9 d1 and 2^-9 d0: multiples of 2^-9 below 2^15) are exact;
// only L2 rounds, at about 2^-42 of L0's scale.  The products left out are
// below 2^-45 of it.  Each level has its own tensor-memory accumulator (L2 two:
// L2 and L2'); the epilogue combines them into a normalised float pair (hi +
// lo, about 48 bits) in units of the level-0 accumulator, and the next pass
// rescales by a power of two.  The matrices are laid out side by side along
// the MMA's N dimension so that each part of the A tile is read once per K
// step: s0 [d0 | 2^-9 d1 | d2 | dT] -> (L0, L1, L2, L2'), s1 [2^-9 d0 | d1 |
// 2^-9 d2] -> (L1, L2, L2'), s2 [d0 | 2^-9 d1] -> (L2, L2'), sT [d0] -> L2'.
//
// Intermediates: the forward spectrum F, the pass buffer and the gain
// accumulator G are float pairs in the CTA's workspace (L2 resident), and the
// term tables (A_t, B_t) are float pairs, so that nothing between the
// transforms rounds to FP32.  The scale E of a pass is the maximum of its
// input, taken by the previous pass's epilogue (the z_t input uses the bound
// max|F| max|A_t + i B_t|, which both reach at k = 0).
//
// Layouts and row orders are those of mixed.cu.  A row of the A tile holds the
// four parts one after another (K index 2N part + 2k + ri); the matrix image
// holds NOUT rows per matrix in the order d0, 2^-9 d1, d2, dT, 2^-9 d0, d1,
// 2^-9 d2 (each row the 2N K values of one output component, 128-byte
// swizzled, zero padded to 64 K values).
// One cluster of two CTAs (two SMs) per cell, persistent over cells: the CTAs
// split the tiles of every pass, meet at a cluster barrier between passes and
// exchange the pass maxima through distributed shared memory, so the cell's
// float-pair workspace (1 MB at N = 32) is shared by two SMs and the
// workspaces of all resident cells stay in L2.  Two tile groups per CTA
// (shared memory at N = 32: 64 KB per A tile + 56 KB of matrices), each of
// two warpgroups that stage one 128-row tile together (half of its rows each)
// and drain its four accumulators of 2N tensor-memory columns together (half
// of the columns each): 16 warps per SM hide the L2 latency of the staging
// loads and the FP32 chains of slicing and combining.  Every mbarrier wait is
// bounded as in mixed.cu.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "coll_internal.h"
#include "dfloat.cuh"
#include "tcgen05.cuh"

namespace coll {

namespace {

constexpr int kSlMaxWG = 4;
constexpr int kSlParts = 4;      // s0, s1, s2, sT
constexpr int kSlMats = 7;       // d0, d1, d2, dT, 2^-9 d1, 2^-9 d2, 2^-9 d0
constexpr int kSlPairs = 10;

// A part and matrix of every product, in issue order: L0 = s0 d0;
// 2^-9 L1 = s0 (2^-9 d1) + s1 (2^-9 d0) (multiples of 2^-9 below 2^15: still
// exact); L2 = s0 d2 + s1 d1 + s2 d0 + s0 dT + sT d0 + s1 (2^-9 d2) + s2 (2^-9 d1)
__host__ __device__ constexpr int sl_pair_a(int i) {
  constexpr int v[kSlPairs] = {0, 0, 1, 0, 1, 2, 0, 3, 1, 2};
  return v[i];
}
__host__ __device__ constexpr int sl_pair_b(int i) {
  constexpr int v[kSlPairs] = {0, 4, 6, 2, 1, 0, 3, 0, 5, 4};
  return v[i];
}
__host__ __device__ constexpr int sl_pair_acc(int i) { return i == 0 ? 0 : (i < 3 ? 1 : 2); }
// Row of matrix s in the image (NOUT rows per matrix), grouped so that one MMA
// of N = 4 NOUT applies [d0 | 2^-9 d1 | d2 | dT] to s0 (accumulators L0, L1,
// L2, L2'), one of N = 3 NOUT applies [2^-9 d0 | d1 | 2^-9 d2] to s1 (L1, L2,
// L2'), and prefixes of the first group serve s2 ([d0 | 2^-9 d1]: L2, L2')
// and sT ([d0]: L2').
__host__ __device__ constexpr int sl_mat_row(int s, int nout) {
  constexpr int v[kSlMats] = {0, 5, 2, 3, 1, 6, 4};
  return v[s] * nout;
}
// the first product of each accumulator overwrites it
__host__ __device__ constexpr bool sl_pair_first(int i) { return i == 0 || i == 1 || i == 3; }

template <int N> struct SlCfg {
  static constexpr int H = N / 2;
  static constexpr int WG = 2;                             // tile groups per CTA (shared memory bound at N = 32)
  static constexpr int TGT = 256;                          // threads per tile group: two warpgroups
  static constexpr int THREADS = TGT * WG;
  static constexpr int KP = 2 * N;                         // f16 values per part per row
  static constexpr int KS = KP / 16;                       // 16-wide K steps per part
  static constexpr int KROW = kSlParts * KP;               // values per A row
  static constexpr int KB = KROW / 64;                     // 128-byte K blocks per A row
  static constexpr int PART_B = 2 * KP;                    // bytes per part in an A row
  static constexpr int NOUT = 2 * N;                       // matrix rows (v, re/im)
  static constexpr int B_BYTES = kSlMats * NOUT * 128;      // seven matrices of NOUT rows x 64 K values
  static constexpr int A_TILE = KB * 128 * 128;
  static constexpr int TCOLS_USED = WG * 4 * NOUT;           // accumulators L0, L1, L2, L2' per tile group
  static constexpr int TCOLS = 512;
  static constexpr int SMEM_USED = B_BYTES + WG * A_TILE + 1024;
  // at least half an SM's shared memory, so that no two CTAs (each holding all
  // 512 tensor-memory columns) ever share an SM: a second allocation would wait
  // for the first CTA, which may itself wait at a cluster barrier
  static constexpr int SMEM_MIN = 120 * 1024;
  static constexpr int SMEM = SMEM_USED > SMEM_MIN ? SMEM_USED : SMEM_MIN;
  static constexpr size_t F_BYTES = size_t(N) * N * H * 16;        // half spectrum, complex float pairs
  static constexpr size_t BUF_BYTES = size_t(N) * N * N * 16;      // N^2 rows of N complex float pairs
  static constexpr size_t G_BYTES = size_t(N) * N * N * 8;         // gain accumulator, float pairs
  static_assert(KROW % 64 == 0, "K blocks");
  static_assert(TCOLS_USED <= TCOLS, "tensor memory");
  static_assert(B_BYTES % 1024 == 0 && A_TILE % 1024 == 0, "1024-byte aligned tiles");
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(WG <= kSlMaxWG, "warpgroups");
};

// Parts of t = sc (th + tl) (sc a power of two, |t| < 2^9, |tl| <= ulp(th)):
// s0, s1, s2 integers and the tail sT, with t = s0 + 2^-9 s1 + 2^-18 (s2 + sT).
// th has 24 significant bits, so removing s0 and then 2^-9 s1 leaves an exact
// residual b (a bit field of th, |b| <= 256 after the scaling by 2^18); tl
// enters at the third level with one rounding (about 2^-43 of the pass
// maximum); |s2| <= 257.
__device__ __forceinline__ void slice4(float th, float tl, float sc, float (&s)[4]) {
  constexpr float M = 0x1.8p23f;                         // rounds |x| <= 2^22 to an integer
  const float s0 = __fsub_rn(__fmaf_rn(th, sc, M), M);
  const float a = __fmul_rn(__fmaf_rn(th, sc, -s0), 512.0f);
  const float s1 = __fsub_rn(__fadd_rn(a, M), M);
  const float b = __fmul_rn(__fsub_rn(a, s1), 512.0f);
  const float c = __fmaf_rn(tl, __fmul_rn(sc, 262144.0f), b);
  const float s2 = __fsub_rn(__fadd_rn(c, M), M);
  s[0] = s0;
  s[1] = s1;
  s[2] = s2;
  s[3] = __fsub_rn(c, s2);
}

// a b + c d for float pairs: exact products of the heads, first-order cross
// terms, one two-sum; the result is left unnormalised (tail below 2^-21 of the head)
__device__ __forceinline__ df fma2(df a, df b, df c, df d) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float q = __fmul_rn(c.h, d.h);
  float g = __fmaf_rn(c.h, d.h, -q);
  g = __fmaf_rn(c.h, d.l, g);
  g = __fmaf_rn(c.l, d.h, g);
  const df t = two_sum(p, q);
  return df{t.h, __fadd_rn(t.l, __fadd_rn(e, g))};
}

// value of one output component, L0 + 2^-9 L1 + 2^-18 L2, in units of the
// level-0 accumulator: an exact two-sum of the exact levels, the third level
// added to the tail, then renormalised.  The renormalisation keeps the tail
// below an ulp of the head; without it the tail of a small output would carry
// the previous pass's scale, and the next slicing's third part would grow
// from pass to pass past f16's exact integers.
__device__ __forceinline__ df combine(uint32_t u0, uint32_t u1, uint32_t u2, uint32_t u3) {
  const df s = two_sum(__uint_as_float(u0), __uint_as_float(u1));
  const float l2 = __fadd_rn(__uint_as_float(u2), __uint_as_float(u3));   // the two third-level accumulators
  return quick_two_sum(s.h, __fmaf_rn(l2, 0x1p-18f, s.l));
}

// Scales of a pass from the maximum modulus m of its input (in the unit of the
// stored input, whose true size is `unit`): the input is multiplied by
// in = 2^(9-E) before slicing (2^E > m), and one level-0 unit of the output is
// worth unit 2^(E-18)
__device__ __forceinline__ void pass_scales(float m, float unit, float* in, float* out_unit) {
  const int E = exp_of(__fmul_ru(m, 1.000001f));
  *in = ldexpf(1.0f, 9 - E);
  *out_unit = __fmul_rn(unit, ldexpf(1.0f, E - 18));
}

enum SlPass : int { kSF2 = 0, kSF1, kSF0, kSX, kSY, kSZ };

// barriers of one tile group (two warpgroups, 256 threads; named barrier tg + 1)
__device__ __forceinline__ void tg_sync(int tg) { asm volatile("bar.sync %0, 256;" ::"r"(tg + 1) : "memory"); }
// true iff p holds on all 256 threads of the tile group
__device__ __forceinline__ bool tg_all(int tg, bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n bar.red.and.pred q, %1, 256, q;\n selp.u32 %0, 1, 0, q;\n}"
      : "=r"(r)
      : "r"(tg + 1), "r"(static_cast<uint32_t>(p))
      : "memory");
  return r != 0;
}

struct SlShared {
  uint64_t bar[kSlMaxWG];
  uint64_t tbar[kSlMaxWG];   // teardown: one fresh commit per warpgroup after an expired wait
  uint32_t tbase;
  uint32_t abort;       // set in both CTAs of the cluster by a warpgroup whose wait expired
  float mx[3];          // [0], [1]: maximum modulus of the current / next pass input; [2]: max (|Re F| + |Im F|)
};
constexpr int kSlotF = 2;

template <int N, typename Tio>
struct SlCell {
  using C = SlCfg<N>;
  static constexpr int H = C::H;
  static constexpr int kWG = C::WG;

  // parts of the complex value (re, im) (scaled float pairs) into slot k of A-tile row `row`
  static __device__ __forceinline__ void put(unsigned char* atile, int row, int k, float rh, float rl, float ih,
                                             float il, float sc) {
    float a[4], b[4];
    slice4(rh, rl, sc, a);
    slice4(ih, il, sc, b);
#pragma unroll
    for (int p = 0; p < kSlParts; ++p) {
      const __half2 h = __floats2half2_rn(a[p], b[p]);
      *reinterpret_cast<uint32_t*>(atile + a_off(row, p * C::PART_B + 4 * k)) = *reinterpret_cast<const uint32_t*>(&h);
    }
  }

  // Row of a 128-row tile staged by thread lt in sweep `it`, with LPR lanes per
  // row: the rows of one warp instruction differ by 4, so that their stores fall
  // on different 16-byte chunks of the 128-byte swizzle (no bank conflicts for
  // LPR >= 16).
  template <int LPR>
  static __device__ __forceinline__ int stage_row(int it, int lt) {
    return it * (128 / LPR) + (lt >> 5) + 4 * ((lt & 31) / LPR);
  }

  // Inputs of a tile are loaded into registers one chunk at a time: the first
  // chunk of the next tile while the current tile's MMAs and epilogue run, each
  // further chunk while the previous one is split into the A tile.  Passes F2
  // (rows (v0, v1) of f, real values at slots v2) and F1, F0, Y, Z (rows of the
  // pass buffer) take one slot per lane, N sweeps in chunks of 8; pass X takes
  // H lanes per row, H sweeps in chunks of 2 (four loads per sweep).
  static constexpr int BQ = 2;
  static constexpr int XQ = 1;
  struct PreF { Tio v[BQ]; };
  struct PreBuf { float4 v[BQ]; };
  struct PreX { float4 F[XQ], T[XQ], G[XQ], U[XQ]; };
  static constexpr int chunks(int pass) { return pass == kSX ? H / XQ : N / BQ; }

  static __device__ __forceinline__ void load(PreF& p, const Tio* __restrict__ f, const float4*, const float4*,
                                              int ti, int lt, int c) {
#pragma unroll
    for (int i = 0; i < BQ; ++i)
      p.v[i] = f[size_t(ti * 128 + stage_row<N>(c * BQ + i, lt)) * N + (lt & (N - 1))];
  }
  static __device__ __forceinline__ void put_chunk(const PreF& p, int lt, int c, unsigned char* atile, float sc) {
#pragma unroll
    for (int i = 0; i < BQ; ++i) {
      df v;
      if constexpr (sizeof(Tio) == 8) v = df_from_double(double(p.v[i]));
      else v = df{float(p.v[i]), 0.0f};
      put(atile, stage_row<N>(c * BQ + i, lt), lt & (N - 1), v.h, v.l, 0.0f, 0.0f, sc);
    }
  }

  static __device__ __forceinline__ void load(PreBuf& p, const Tio* __restrict__, const float4* buf, const float4*,
                                              int ti, int lt, int c) {
#pragma unroll
    for (int i = 0; i < BQ; ++i)
      p.v[i] = __ldcg(buf + size_t(ti * 128 + stage_row<N>(c * BQ + i, lt)) * N + (lt & (N - 1)));
  }
  static __device__ __forceinline__ void put_chunk(const PreBuf& p, int lt, int c, unsigned char* atile, float sc) {
#pragma unroll
    for (int i = 0; i < BQ; ++i) {
      const float4 v = p.v[i];
      put(atile, stage_row<N>(c * BQ + i, lt), lt & (N - 1), v.x, v.y, v.z, v.w, sc);
    }
  }

  // pass X: row (k0, k1), slot k2: (A + iB) F for k2 < N/2 from row (k0, k1) of F
  // and of the term table, for k2 > N/2 from the partner row (-k0, -k1) at
  // N - k2 (conjugated F; the multipliers are even); slot N/2 is zero
  static __device__ __forceinline__ void load(PreX& p, const Tio* __restrict__, const float4* Fs,
                                              const float4* __restrict__ tab_t, int ti, int lt, int c) {
    const int k2 = lt & (H - 1);
#pragma unroll
    for (int i = 0; i < XQ; ++i) {
      const int rr = ti * 128 + stage_row<H>(c * XQ + i, lt);
      const int k0 = rr / N, k1 = rr % N;
      const int rp = ((N - k0) % N) * N + (N - k1) % N;
      p.F[i] = __ldcg(Fs + size_t(rr) * H + k2);
      p.T[i] = __ldg(tab_t + size_t(rr) * H + k2);
      p.G[i] = __ldcg(Fs + size_t(rp) * H + k2);
      p.U[i] = __ldg(tab_t + size_t(rp) * H + k2);
    }
  }
  static __device__ __forceinline__ void put_chunk(const PreX& p, int lt, int c, unsigned char* atile, float sc) {
    const int k2 = lt & (H - 1);
#pragma unroll
    for (int i = 0; i < XQ; ++i) {
      const int row = stage_row<H>(c * XQ + i, lt);
      const float4 F = p.F[i], T = p.T[i], G = p.G[i], U = p.U[i];
      {
        const df A{T.x, T.y}, B{T.z, T.w}, Fr{F.x, F.y}, Fi{F.z, F.w};
        const df zr = fma2(A, Fr, df{-B.h, -B.l}, Fi), zi = fma2(A, Fi, B, Fr);
        put(atile, row, k2, zr.h, zr.l, zi.h, zi.l, sc);
      }
      if (k2 > 0) {
        const df A{U.x, U.y}, B{U.z, U.w}, Gr{G.x, G.y}, Gi{G.z, G.w};
        const df zr = fma2(A, Gr, B, Gi), zi = fma2(B, Gr, df{-A.h, -A.l}, Gi);
        put(atile, row, N - k2, zr.h, zr.l, zi.h, zi.l, sc);
      } else {
#pragma unroll
        for (int pp = 0; pp < kSlParts; ++pp)
          *reinterpret_cast<uint32_t*>(atile + a_off(row, pp * C::PART_B + 4 * H)) = 0u;
      }
    }
  }

  // Half h of the A tile (chunks h, h + 2, ...; the tile group's other
  // warpgroup stages the rest) from its first chunk `a` (already loaded); the
  // next chunk of the half loads while the current one is split (a rolled
  // loop over chunk pairs keeps the code small); `a` is consumed
  template <int NC, class P>
  static __device__ __forceinline__ void stage(P& a, const Tio* __restrict__ f, const float4* src,
                                               const float4* __restrict__ tab_t, int ti, int lt, int h,
                                               unsigned char* atile, float sc) {
    constexpr int NH = NC / 2;
    static_assert(NC % 2 == 0 && NH % 2 == 0, "chunk pairs per half");
    P b;
#pragma unroll 1
    for (int i = 0; i < NH; i += 2) {
      load(b, f, src, tab_t, ti, lt, 2 * (i + 1) + h);
      put_chunk(a, lt, 2 * i + h, atile, sc);
      if (i + 2 < NH) load(a, f, src, tab_t, ti, lt, 2 * (i + 2) + h);
      put_chunk(b, lt, 2 * (i + 1) + h, atile, sc);
    }
  }

  // One pass over this tile group's tiles.  Returns false (uniformly over the
  // tile group) if an MMA wait expired; the expired phase stays pending.
  // `kind` selects the A-tile source (0: f, pass F2; 1: F and the term table,
  // pass X; 2: the pass buffer, passes F1, F0, Y, Z, told apart at run time).
  // tg: tile group; lt2: thread of the tile group (0 .. 255), whose warpgroup
  // half h = lt2 / 128 stages half of each tile and drains half of its output
  // columns.
  template <int kind>
  static __device__ __forceinline__ bool run(int pass, int wg, int lt2, unsigned char* atile, uint32_t abase,
                                             uint32_t bbase, uint32_t tacc, uint32_t& phase, bool& pending,
                                             SlShared& sh, const Tio* __restrict__ f, Tio* __restrict__ Q,
                                             float4* Fs, float4* buf, float2* G, const float4* __restrict__ tab_t,
                                             float sc_in, float sc_out, int next_slot, bool first_term,
                                             bool last_term, bool& bad) {
    const int rows = (pass == kSF1 || pass == kSF0) ? H * N : N * N;
    constexpr int nout = kind == 0 ? N : C::NOUT;
    const int crank = int(cluster_ctarank());          // the two CTAs of the cluster split the tiles
    // F0 writes F and Z accumulates G in true units (times sc_out); the other
    // passes store their outputs in level-0 units of the pass
    const bool to_true = kind == 2 && (pass == kSF0 || pass == kSZ);
    const int h = lt2 >> 7, lt = lt2 & 127;
    const int q = lt >> 5;                               // TMEM lane quarter of this warp
    // output columns drained by this half, in chunks of CW columns (CW / 2
    // complex outputs)
    constexpr int CW = 8, EW = CW / 2;
    constexpr int CPH = nout / 2;
    const int c_begin = h * CPH, c_end = (h + 1) * CPH < nout ? (h + 1) * CPH : nout;
    float lmax = 0.0f;
    using Pre = typename std::conditional<kind == 0, PreF,
                                          typename std::conditional<kind == 1, PreX, PreBuf>::type>::type;
    constexpr int NC = kind == 1 ? H / XQ : N / BQ;
    // the X pass reads F (Fs) and the term table; the other passes read f or the pass buffer
    const float4* src = kind == 1 ? Fs : buf;
    Pre pre;
    const int ti0 = crank * kWG + wg;
    if (ti0 < rows / 128) load(pre, f, src, tab_t, ti0, lt, h);
    for (int ti = ti0; ti < rows / 128; ti += 2 * kWG) {
      const int r = ti * 128 + lt;
      // ---- A tile
      stage<NC>(pre, f, src, tab_t, ti, lt, h, atile, sc_in);
      fence_async_smem();
      tg_sync(wg);
      // ---- MMAs: ten products into four accumulators (L0, L1 and two for L2)
      if (lt2 == 0) {
        fence_after();
        // descriptors of the tile bases; each K step adds a compile-time offset
        // to the 14-bit start-address field (addresses stay below 2^18 bytes,
        // so the field never carries)
        const uint64_t ad = sw128_desc(abase), bd = sw128_desc(bbase);
        if constexpr (kind == 0) {
          // real input, N outputs: the ten products one by one into L0, L1, L2
          const uint32_t id = idesc_f16(128, nout, 0);
#pragma unroll
          for (int pi = 0; pi < kSlPairs; ++pi) {
            const int pa = sl_pair_a(pi), pb = sl_pair_b(pi), pc = sl_pair_acc(pi);
            const bool first = sl_pair_first(pi);
#pragma unroll
            for (int j = 0; j < C::KS; ++j) {
              const int ka = pa * C::KS + j;
              mma_f16(tacc + pc * C::NOUT, ad + uint64_t(((ka >> 2) * 16384 + (ka & 3) * 32) >> 4),
                      bd + uint64_t((sl_mat_row(pb, C::NOUT) * 128 + j * 32) >> 4), id,
                      (first && j == 0) ? 0u : 1u);
            }
          }
        } else {
          // one MMA per part and K step over its matrices side by side along N
#pragma unroll
          for (int pa = 0; pa < kSlParts; ++pa) {
            const int brow = pa == 1 ? 4 * C::NOUT : 0;
            const int ncol = (pa == 0 ? 4 : pa == 1 ? 3 : pa == 2 ? 2 : 1) * C::NOUT;
            const int dcol = (pa == 0 ? 0 : pa == 1 ? 1 : pa == 2 ? 2 : 3) * C::NOUT;
            const uint32_t id = idesc_f16(128, ncol, 0);
#pragma unroll
            for (int j = 0; j < C::KS; ++j) {
              const int ka = pa * C::KS + j;
              mma_f16(tacc + dcol, ad + uint64_t(((ka >> 2) * 16384 + (ka & 3) * 32) >> 4),
                      bd + uint64_t((brow * 128 + j * 32) >> 4), id, (pa == 0 && j == 0) ? 0u : 1u);
            }
          }
        }
        mma_commit(&sh.bar[wg]);
      }
      // the next tile's first chunk is in flight during the MMAs and the epilogue
      if (ti + 2 * kWG < rows / 128) load(pre, f, src, tab_t, ti + 2 * kWG, lt, h);
      if (!tg_all(wg, wait_parity(&sh.bar[wg], phase))) {
        if (lt2 == 0) {
          st_cluster_u32(cluster_addr(su32(&sh.abort), 0), 1u);
          st_cluster_u32(cluster_addr(su32(&sh.abort), 1), 1u);
        }
        pending = true;
        return false;
      }
      phase ^= 1u;
      fence_after();
      // ---- epilogue: thread = TMEM lane = pencil row r
      const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
      // pass Z: the gain accumulator of the chunk's outputs, loaded one chunk ahead
      float2 gcur[EW], gnxt[EW];
      const bool zacc = kind == 2 && pass == kSZ && !first_term;
      if (zacc) {
#pragma unroll
        for (int e = 0; e < EW; ++e) gcur[e] = __ldcg(G + size_t(c_begin / 2 + e) * N * N + r);
      }
#pragma unroll 1
      for (int c0 = c_begin; c0 < c_end; c0 += CW) {
        if (zacc && c0 + CW < c_end) {
#pragma unroll
          for (int e = 0; e < EW; ++e) gnxt[e] = __ldcg(G + size_t((c0 + CW) / 2 + e) * N * N + r);
        }
        uint32_t u0[CW], u1[CW], u2[CW], u3[CW];
        tld8_nw(tacc + lane_base + c0, u0);
        tld8_nw(tacc + C::NOUT + lane_base + c0, u1);
        tld8_nw(tacc + 2 * C::NOUT + lane_base + c0, u2);
        if constexpr (kind != 0) tld8_nw(tacc + 3 * C::NOUT + lane_base + c0, u3);
        tld8_wait(u0, u1, u2);
        if constexpr (kind != 0) tld8_tie(u3);
        else {
#pragma unroll
          for (int e = 0; e < CW; ++e) u3[e] = 0u;             // +0.0f: no second third-level accumulator
        }
        const int v0c = c0 >> 1;                         // first complex output of this chunk
#pragma unroll
        for (int e = 0; e < EW; ++e) {
          df re = combine(u0[2 * e], u1[2 * e], u2[2 * e], u3[2 * e]);
          df im = combine(u0[2 * e + 1], u1[2 * e + 1], u2[2 * e + 1], u3[2 * e + 1]);
          if (to_true) {                                // passes F0 and Z: true units
            re = df{__fmul_rn(re.h, sc_out), __fmul_rn(re.l, sc_out)};
            im = df{__fmul_rn(im.h, sc_out), __fmul_rn(im.l, sc_out)};
          }
          const int o = v0c + e;                         // output index of this pencil
          if (kind == 2 && pass == kSZ) {
            // G[(v2, v1)][v0] with r = (v2, v1), o = v0
            const df p = re * im;
            float2* gp = G + size_t(o) * N * N + r;
            df g = p;
            if (!first_term) g = df{gcur[e].x, gcur[e].y} + p;
            if (!last_term) {
              __stcg(gp, make_float2(g.h, g.l));
            } else {
              // Q[v0][v1][v2]
              Tio* qp = Q + (size_t(o) * N + (r % N)) * N + (r / N);
              Tio out;
              if constexpr (sizeof(Tio) == 8) out = Tio(df_to_double(g));
              else out = Tio(__fadd_rn(g.h, g.l));
              bad |= !::isfinite(double(out));
              *qp = out;
            }
          } else if (kind == 2 && pass == kSF0) {
            const int k2h = r / N, k1 = r % N, k0 = o;
            float4 v = make_float4(re.h, re.l, -im.h, -im.l);       // the forward transform conjugates
            if (k0 == H || k1 == H) v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            lmax = fmaxf(lmax, __fadd_ru(fabsf(v.x), fabsf(v.z)));
            Fs[(size_t(k0) * N + k1) * H + k2h] = v;
          } else {
            // next pass's row, slot = this pencil's next-K index:
            //   F2: r = (v0, v1), out k2h -> row (k2h, v0), slot v1
            //   F1: r = (k2h, v0), out k1 -> row (k2h, k1), slot v0
            //   X:  r = (k0, k1), out v2 -> row (v2, k0), slot k1
            //   Y:  r = (v2, k0), out v1 -> row (v2, v1), slot k0
            const int dstride = kind != 2 ? N : 1;
            const int drow0 = kind != 2 ? r / N : (r / N) * N;
            lmax = fmaxf(lmax, fmaxf(fabsf(re.h), fabsf(im.h)));
            __stcg(buf + size_t(drow0 + o * dstride) * N + (r % N), make_float4(re.h, re.l, im.h, im.l));
          }
        }
        if (zacc) {
#pragma unroll
          for (int e = 0; e < EW; ++e) gcur[e] = gnxt[e];
        }
      }
      fence_before();
      tg_sync(wg);
    }
    if (next_slot >= 0) {
      // warp maximum, then into the slot of both CTAs of the cluster
      const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(lmax));
      if ((lt & 31) == 0) {
        red_max_cluster(cluster_addr(su32(&sh.mx[next_slot]), 0), __uint_as_float(wm));
        red_max_cluster(cluster_addr(su32(&sh.mx[next_slot]), 1), __uint_as_float(wm));
      }
    }
    return true;
  }

  // Whole cell; returns true (uniformly) if the CTA must stop (a wait expired).
  static __device__ bool cell(const Tio* __restrict__ f, Tio* __restrict__ Q, const float4* __restrict__ tab,
                              const float* __restrict__ tmax, int n_terms, unsigned char* ws, unsigned char* atile,
                              uint32_t abase, uint32_t bbase, uint32_t tacc, uint32_t& phase, bool& pending,
                              SlShared& sh, bool& bad) {
    const int tid = threadIdx.x, wg = tid >> 8, lt = tid & 255;   // tile group, its thread
    float4* Fs = reinterpret_cast<float4*>(ws);
    float4* buf = reinterpret_cast<float4*>(ws + C::F_BYTES);
    float2* G = reinterpret_cast<float2*>(ws + C::F_BYTES + C::BUF_BYTES);
    const int crank = int(cluster_ctarank());
    // cluster barrier; zero the maximum slot that the next pass's epilogue writes; cluster barrier
    auto stop = [&](int zero_slot) -> bool {
      cluster_sync();
      const bool v = *reinterpret_cast<volatile uint32_t*>(&sh.abort) != 0u;
      if (tid == 0 && zero_slot >= 0) sh.mx[zero_slot] = 0.0f;
      cluster_sync();
      return v;
    };

    if (tid == 0) { sh.mx[0] = 0.0f; sh.mx[1] = 0.0f; sh.mx[kSlotF] = 0.0f; }
    cluster_sync();
    float m = 0.0f;
    for (int i = crank * C::THREADS + tid; i < N * N * N; i += 2 * C::THREADS)
      m = fmaxf(m, __double2float_ru(fabs(double(f[i]))));
    const uint32_t wm = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
    if ((tid & 31) == 0) {
      red_max_cluster(cluster_addr(su32(&sh.mx[0]), 0), __uint_as_float(wm));
      red_max_cluster(cluster_addr(su32(&sh.mx[0]), 1), __uint_as_float(wm));
    }
    cluster_sync();
    // si: input scale of a pass; u: true size of one unit of the stored pass input
    float si, u = 1.0f;
    pass_scales(sh.mx[0], 1.0f, &si, &u);
    run<0>(kSF2, wg, lt, atile, abase, bbase, tacc, phase, pending, sh, f, Q, Fs, buf, G, tab, si, 1.0f, 1,
           false, false, bad);
    if (stop(0)) return true;
    pass_scales(sh.mx[1], u, &si, &u);
    run<2>(kSF1, wg, lt, atile, abase, bbase, tacc, phase, pending, sh, f, Q, Fs, buf, G, tab, si, 1.0f, 0,
           false, false, bad);
    if (stop(1)) return true;
    pass_scales(sh.mx[0], u, &si, &u);
    run<2>(kSF0, wg, lt, atile, abase, bbase, tacc, phase, pending, sh, f, Q, Fs, buf, G, tab, si, u, kSlotF,
           false, false, bad);
    if (stop(-1)) return true;
    const float Fmax = sh.mx[kSlotF];
    for (int t = 0; t < n_terms; ++t) {
      const float4* tab_t = tab + size_t(t) * N * N * H;
      pass_scales(__fmul_ru(Fmax, tmax[t]), 1.0f, &si, &u);
      run<1>(kSX, wg, lt, atile, abase, bbase, tacc, phase, pending, sh, f, Q, Fs, buf, G, tab_t, si, 1.0f, 1,
             false, false, bad);
      if (stop(0)) return true;
      pass_scales(sh.mx[1], u, &si, &u);
      run<2>(kSY, wg, lt, atile, abase, bbase, tacc, phase, pending, sh, f, Q, Fs, buf, G, tab_t, si, 1.0f, 0,
             false, false, bad);
      if (stop(1)) return true;
      pass_scales(sh.mx[0], u, &si, &u);
      run<2>(kSZ, wg, lt, atile, abase, bbase, tacc, phase, pending, sh, f, Q, Fs, buf, G, tab_t, si, u, -1,
             t == 0, t == n_terms - 1, bad);
      if (stop(-1)) return true;
    }
    return false;
  }
};

// The cells a launch evaluates: one plan's batch (SlBatch), or the cells of
// several plans of the same N in table order (SlGroups, a ragged launch: each
// group has its own f, Q, term tables and status; the DFT matrices depend on N
// only, so the first group's image serves all).
template <typename Tio> struct SlCellRef {
  const Tio* f;
  Tio* Q;
  const float4* tab;
  const float* tmax;
  int n_terms;
  int* status;
};
template <int N, typename Tio> struct SlBatch {
  const CollArgs& a;
  __device__ long long count() const { return a.n_cells; }
  __device__ const unsigned char* image() const {
    return static_cast<const unsigned char*>(a.tab) + sliced_img_offset(N, a.n_terms);
  }
  __device__ SlCellRef<Tio> cell(long long c) const {
    const unsigned char* tb = static_cast<const unsigned char*>(a.tab);
    return {static_cast<const Tio*>(a.f) + size_t(c) * N * N * N, static_cast<Tio*>(a.Q) + size_t(c) * N * N * N,
            reinterpret_cast<const float4*>(tb), reinterpret_cast<const float*>(tb + sliced_tmax_offset(N, a.n_terms)),
            a.n_terms, a.status};
  }
  __device__ void report_all(int bits) const { atomicOr(a.status, bits); }
};
template <int N, typename Tio> struct SlGroups {
  const RaggedTable& t;
  __device__ long long count() const { return t.total_units; }
  __device__ const unsigned char* image() const {
    return static_cast<const unsigned char*>(t.items[0].tab) + sliced_img_offset(N, t.items[0].n_terms);
  }
  __device__ SlCellRef<Tio> cell(long long u) const {
    int g = 0;
    while (g + 1 < t.n_items && u >= t.items[g + 1].first_unit) ++g;
    const RaggedItem& it = t.items[g];
    const long long c = u - it.first_unit;
    const unsigned char* tb = static_cast<const unsigned char*>(it.tab);
    return {static_cast<const Tio*>(it.f) + size_t(c) * N * N * N, static_cast<Tio*>(it.Q) + size_t(c) * N * N * N,
            reinterpret_cast<const float4*>(tb), reinterpret_cast<const float*>(tb + sliced_tmax_offset(N, it.n_terms)),
            it.n_terms, it.status};
  }
  __device__ void report_all(int bits) const {
    for (int g = 0; g < t.n_items; ++g) atomicOr(t.items[g].status, bits);
  }
};

// Kernel body: one cell per cluster of two CTAs, persistent over the source's
// cells; each cell's non-finite flag goes to its own plan's status.
template <int N, typename Tio, typename Src>
__device__ __forceinline__ void sliced_body(const Src& src, void* wsp, size_t ws_per_cta) {
  using C = SlCfg<N>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ SlShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, wg = tid >> 8;   // wg: tile group (two warpgroups)
  const uint32_t raw = su32(smraw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smraw + (base - raw);
  const uint32_t bbase = base;
  const uint32_t abase = base + C::B_BYTES + wg * C::A_TILE;

  // matrices: copy the pre-swizzled image
  const unsigned char* img = src.image();
  for (int i = tid; i < C::B_BYTES / 16; i += C::THREADS)
    reinterpret_cast<uint4*>(sm)[i] = __ldg(reinterpret_cast<const uint4*>(img) + i);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh.tbase)),
                 "r"(C::TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int w = 0; w < C::WG; ++w) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sh.bar[w])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&sh.tbar[w])), "r"(1));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sh.abort = 0u;
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  cluster_sync();                          // the peer CTA is running before any remote shared-memory access
  const uint32_t tbase = sh.tbase;
  const uint32_t tacc = tbase + wg * 4 * C::NOUT;
  uint32_t phase = 0;
  bool pending = false;
  // a cell per cluster of two CTAs; the cluster works in the workspace slot of its first CTA
  unsigned char* ws = static_cast<unsigned char*>(wsp) + size_t(blockIdx.x & ~1u) * ws_per_cta;
  for (long long u = blockIdx.x >> 1; u < src.count(); u += gridDim.x >> 1) {
    const SlCellRef<Tio> c = src.cell(u);
    bool bad = false;
    const bool stop = SlCell<N, Tio>::cell(c.f, c.Q, c.tab, c.tmax, c.n_terms, ws, sm + C::B_BYTES + wg * C::A_TILE,
                                           abase, bbase, tacc, phase, pending, sh, bad);
    if (__syncthreads_or(bad) && tid == 0) atomicOr(c.status, kStatusNonFinite);
    if (stop) break;                       // uniform over the cluster (abort is set in both CTAs)
  }
  // A wait that expired may leave this tile group's last MMA batch in flight.
  // A fresh commit from the issuing thread to a barrier of its own arrives once
  // every MMA that thread started has completed; tensor memory is freed only
  // after that arrival (bounded wait).
  if (pending) {
    if ((tid & 255) == 0) mma_commit(&sh.tbar[wg]);
    (void)wait_parity(&sh.tbar[wg], 0);
  }
  fence_before();
  __syncthreads();
  if (sh.abort && tid == 0) src.report_all(kStatusTimeout);
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(C::TCOLS));
  }
  cluster_sync();                          // no CTA leaves while its peer may still address its shared memory
}

template <int N, typename Tio>
__global__ void __launch_bounds__(SlCfg<N>::THREADS, 1) sliced_kernel(CollArgs a) {
  sliced_body<N, Tio>(SlBatch<N, Tio>{a}, a.ws, a.ws_per_cta);
}

template <int N, typename Tio>
__global__ void __launch_bounds__(SlCfg<N>::THREADS, 1) sliced_ragged_kernel(RaggedTable t, void* ws,
                                                                             size_t ws_per_cta) {
  sliced_body<N, Tio>(SlGroups<N, Tio>{t}, ws, ws_per_cta);
}

template <int N>
void sl_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, cudaStream_t st) {
  using C = SlCfg<N>;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg->blockDim = dim3(C::THREADS);
  cfg->dynamicSmemBytes = C::SMEM;
  cfg->stream = st;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
}

// Launch in clusters of two CTAs (one cell per cluster).  `grid` is the number
// of CTAs the caller's workspace covers (ws_per_cta each); the kernel uses
// every other slot, so any grid >= 1 fits: it runs max(1, grid / 2) clusters,
// capped at the cell count and at the number of clusters that can be resident.
template <typename K, typename... Args>
int sl_launch(K k, int smem, long long cells, int grid, cudaLaunchConfig_t* cfg, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return int(e);
  long long clusters = grid / 2 < 1 ? 1 : grid / 2;
  if (clusters > cells) clusters = cells;
  cfg->gridDim = dim3(2);
  int resident = 0;
  e = cudaOccupancyMaxActiveClusters(&resident, k, cfg);
  if (e != cudaSuccess) return int(e);
  if (resident >= 1 && clusters > resident) clusters = resident;
  cfg->gridDim = dim3(unsigned(2 * clusters));
  e = cudaLaunchKernelEx(cfg, k, args...);
  if (e != cudaSuccess) return int(e);
  return int(cudaGetLastError());
}

template <int N, typename Tio>
int launch_sliced_t(const CollArgs& a, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  sl_config<N>(&cfg, attr, st);
  return sl_launch(sliced_kernel<N, Tio>, SlCfg<N>::SMEM, a.n_cells, grid, &cfg, a);
}

template <int N, typename Tio>
int launch_sliced_ragged_t(const RaggedTable& t, void* ws, size_t ws_per_cta, int grid, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  sl_config<N>(&cfg, attr, st);
  return sl_launch(sliced_ragged_kernel<N, Tio>, SlCfg<N>::SMEM, t.total_units, grid, &cfg, t, ws, ws_per_cta);
}

template <int N, typename Tio>
int occupancy_sliced_t(int* ctas) {
  using C = SlCfg<N>;
  auto k = sliced_kernel<N, Tio>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return int(e);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, C::THREADS, C::SMEM);
  const int by_tmem = 512 / C::TCOLS;
  if (*ctas > by_tmem) *ctas = by_tmem;
  return int(e);
}

uint16_t sl_half_bits(double x) {             // IEEE binary16, round to nearest even (host)
  const __half h = __double2half(x);
  uint16_t b;
  std::memcpy(&b, &h, 2);
  return b;
}

}  // namespace

bool sliced_layout(int N, LayoutInfo* out) {
  if (N != 16 && N != 32) return false;
  LayoutInfo i;
  i.N = N;
  i.S0 = 1;
  i.threads = N == 16 ? SlCfg<16>::THREADS : SlCfg<32>::THREADS;
  i.fh_smem = false;
  i.w_smem = false;
  i.g_smem = false;
  i.fh_bytes = N == 16 ? SlCfg<16>::F_BYTES : SlCfg<32>::F_BYTES;
  i.w_bytes = N == 16 ? SlCfg<16>::BUF_BYTES : SlCfg<32>::BUF_BYTES;
  i.g_bytes = N == 16 ? SlCfg<16>::G_BYTES : SlCfg<32>::G_BYTES;
  i.smem = N == 16 ? SlCfg<16>::SMEM : SlCfg<32>::SMEM;
  i.ws = i.fh_bytes + i.w_bytes + i.g_bytes;       // F, the pass buffer and G in global memory
  *out = i;
  return true;
}

int launch_sliced(int N, bool io_f64, const CollArgs& a, int grid, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (N == 16) return io_f64 ? launch_sliced_t<16, double>(a, grid, st) : launch_sliced_t<16, float>(a, grid, st);
  if (N == 32) return io_f64 ? launch_sliced_t<32, double>(a, grid, st) : launch_sliced_t<32, float>(a, grid, st);
  return int(cudaErrorInvalidValue);
}

int launch_sliced_ragged(int N, bool io_f64, const RaggedTable& t, void* ws, size_t ws_per_cta, int grid,
                         void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (N == 16)
    return io_f64 ? launch_sliced_ragged_t<16, double>(t, ws, ws_per_cta, grid, st)
                  : launch_sliced_ragged_t<16, float>(t, ws, ws_per_cta, grid, st);
  if (N == 32)
    return io_f64 ? launch_sliced_ragged_t<32, double>(t, ws, ws_per_cta, grid, st)
                  : launch_sliced_ragged_t<32, float>(t, ws, ws_per_cta, grid, st);
  return int(cudaErrorInvalidValue);
}

int sliced_max_ctas_per_sm(int N, bool io_f64, int* ctas) {
  if (N == 16) return io_f64 ? occupancy_sliced_t<16, double>(ctas) : occupancy_sliced_t<16, float>(ctas);
  if (N == 32) return io_f64 ? occupancy_sliced_t<32, double>(ctas) : occupancy_sliced_t<32, float>(ctas);
  return int(cudaErrorInvalidValue);
}

// Device image of a sliced plan: per-term tables [t][k0][k1][k2h] (A_h, A_l,
// B_h, B_l) as float pairs, the per-term bound max|A + iB| (rounded up), then
// the swizzled f16 matrices d0, d1, d2, dT, 2^-9 d1, 2^-9 d2, 2^-9 d0 of the
// inverse N-point DFT, NOUT rows each at the rows sl_mat_row gives (K zero
// padded to 64 values).
coll_status build_sliced_image(const HostTables& ht, int N, std::vector<unsigned char>* out) {
  if (N != 16 && N != 32) return COLL_EUNSUPPORTED;
  const int H = N / 2, nt = ht.n_terms;
  const int KP = 2 * N, NOUT = 2 * N;
  const size_t img_off = sliced_img_offset(N, nt);
  const size_t img_bytes = size_t(kSlMats) * NOUT * 128;
  out->assign(img_off + img_bytes, 0);
  float* tab = reinterpret_cast<float*>(out->data());
  float* tmax = reinterpret_cast<float*>(out->data() + sliced_tmax_offset(N, nt));
  for (int t = 0; t < nt; ++t) {
    double mx = 0.0;
    for (int k0 = 0; k0 < N; ++k0)
      for (int k1 = 0; k1 < N; ++k1)
        for (int k2 = 0; k2 < H; ++k2) {
          const size_t src = ((size_t(t) * N + k0) * N + k1) * H + k2;
          const double A = ht.tab[2 * src], B = ht.tab[2 * src + 1];
          const float ah = float(A), bh = float(B);
          tab[4 * src + 0] = ah;
          tab[4 * src + 1] = float(A - double(ah));
          tab[4 * src + 2] = bh;
          tab[4 * src + 3] = float(B - double(bh));
          mx = std::fmax(mx, std::sqrt(A * A + B * B));
        }
    tmax[t] = float(mx * (1.0 + 1e-6));
  }
  unsigned char* img = out->data() + img_off;
  const double two_pi = 6.283185307179586476925286766559;
  // matrix s, output row j, K index kk: row sl_mat_row(s) + j of the image
  // (128-byte swizzled K-major rows, K zero padded to 64 values)
  auto put = [&](int s, int j, int kk, uint16_t val) {
    const int row = sl_mat_row(s, NOUT) + j, chunk = kk / 8, within = kk % 8;
    const size_t off = size_t(row) * 128 + size_t((chunk ^ (row & 7)) * 16) + size_t(within) * 2;
    std::memcpy(img + off, &val, 2);
  };
  for (int j = 0; j < NOUT; ++j) {
    const int v = j >> 1, ro = j & 1;
    for (int kk = 0; kk < KP; ++kk) {
      const int k = kk >> 1, ri = kk & 1;
      const double th = two_pi * double((size_t(k) * v) % N) / double(N);
      const double c = std::cos(th), sn = std::sin(th);
      // [[cos, -sin], [sin, cos]] for y = sum e^{+i th} x
      const double d = ro == 0 ? (ri == 0 ? c : -sn) : (ri == 0 ? sn : c);
      // d = 2^-9 (d0 + 2^-9 d1 + 2^-18 (d2 + dT)), every step exact in double
      const double t0 = d * 512.0, d0 = std::nearbyint(t0);
      const double t1 = (t0 - d0) * 512.0, d1 = std::nearbyint(t1);
      const double t2 = (t1 - d1) * 512.0, d2 = std::nearbyint(t2);
      const double dT = t2 - d2;
      const double m[kSlMats] = {d0, d1, d2, dT, d1 / 512.0, d2 / 512.0, d0 / 512.0};
      for (int s = 0; s < kSlMats; ++s) put(s, j, kk, sl_half_bits(m[s]));
    }
  }
  return COLL_OK;
}

}  // namespace coll
