// Mixed-precision collision path: every transform of the fused collision
// operator (the forward R2C transform and the per-term inverse transforms,
// arxiv 2505.03360 sec. 4.4.1) as DFT-GEMMs on the tcgen05 tensor cores.
//
// Same index-space algorithm as collision_impl.cuh:
//   F   = DFT3(f)                    half spectrum k2 < N/2, Nyquist planes zero
//   z_t = IDFT3((A_t + i B_t) F)     one complex 3D inverse per term
//   Q   = sum_t Re(z_t) Im(z_t)      (the last term is the loss term)
// Each 1D transform along an axis is a GEMM over a batch of pencils:
//   Y[pencil][(v, re/im)] = sum_{(k, re/im)} X[pencil][(k, re/im)] D[(v, re/im)][(k, re/im)]
// with D the real 2x2-block form of the N-point DFT matrix e^{+2 pi i k v / N}
// (forward transforms by conjugating input and output).
//
// Precision.  Every operand is split into P parts of a 16-bit format:
//   COLL_MIXED_F16X2  (P = 2, f16):  x = x_h + x_l,
//                     X D ~ (X_h + X_l) D_h + X_h D_l                 (3 products)
//   COLL_MIXED_BF16X3 (P = 3, bf16): x = x_h + x_m + x_l,
//                     X D ~ (X_h + X_m + X_l) D_h + (X_h + X_m) D_m + X_h D_l  (6 products)
// with FP32 accumulation; about 22 (f16) or 24 (bf16) significant bits per
// operand.  f16 has 5 exponent bits, so each cell's data are scaled by powers
// of two: the input of a three-pass transform is scaled to modulus
// <= 2^14 / N^3, which bounds every intermediate (each pass grows the modulus
// by at most N) below 2^14.  The bound of z_t's input uses max|F| (computed
// per cell) times max|A_t + iB_t| (per term, from the plan).  Scales are powers
// of two, undone exactly in FP32 (bf16 has FP32's exponent range and takes the
// same scales).
//
// Layouts.  One pencil per row; a row holds the pencil's N complex inputs
// part by part: K index 2N part + 2k + ri (16-bit pairs (re, im) per element
// and part), padded to a multiple of 64.  Matrix s (s = 0 .. P-1) holds part s
// of D in the tensor core's K-major 128-byte-swizzled shared-memory layout and
// is applied to the first P - s parts of the operand:
//   B_s[(v, ro)][(part, k, ri)] = D_s(ro, ri)(v, k),   part < P - s.
// Passes per cell (row orders chosen so that, within a warp, the next pass's
// K index varies fastest, which makes every epilogue store coalesced; F1 and
// Y write back into the rows they read, so one pass buffer serves a cell):
//   F2  rows (v0, v1), K = v2 (real f)     -> buf rows (k2h, v0), slot v1
//   F1  rows (k2h, v0), K = v1             -> buf rows (k2h, k1), slot v0 (in place)
//   F0  rows (k2h, k1), K = v0             -> F[k0][k1][k2h] (FP32 complex)
//   per term t:
//   X   rows (k0, k1), K = k2: the A tile is built from rows of F and of the
//       term's (A, B) (contiguous in k2h; k2 > N/2 from the Hermitian partner
//       row (-k0, -k1))                    -> buf rows (v2, k0), slot k1
//   Y   rows (v2, k0), K = k1              -> buf rows (v2, v1), slot k0 (in place)
//   Z   rows (v2, v1), K = k0              -> G[(v2, v1)][v0] += Re * Im in
//                                             tensor memory; Q on the last term
//
// CTA organisation: one CTA per SM (persistent over cells), four warpgroups.
// Warpgroup w takes the tiles w, w + 4, ... of each pass: it stages its
// 128-row A tile in shared memory, one thread issues the MMAs into the
// warpgroup's own accumulator columns in tensor memory and commits to the
// warpgroup's mbarrier, and the warpgroup's 128 threads (thread = TMEM lane =
// pencil) run the epilogue.  Warpgroups overlap one another's copies, MMAs
// and epilogues.  The gain accumulator G of the whole cell lives in tensor
// memory (N^3 / 128 columns).  Every mbarrier wait is bounded; on expiry the
// kernel records kStatusTimeout, stops issuing work, waits (bounded) for its
// MMAs in flight, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "coll_internal.h"
#include "tcgen05.cuh"

namespace coll {

namespace {

constexpr int kMixMaxWG = 4;

// Split of an FP32 complex value into P 16-bit parts per component, packed as
// (re, im) pairs: w[p] = part p of (re, im).  Each residual is exact in FP32.
template <int P> struct Split;
template <> struct Split<2> {                 // f16 hi + lo
  static constexpr uint32_t kFmt = 0;         // kind::f16 operand format: f16
  static __device__ __forceinline__ void split(float re, float im, uint32_t (&w)[2]) {
    const __half2 h = __floats2half2_rn(re, im);
    const float2 hb = __half22float2(h);
    const __half2 l = __floats2half2_rn(__fsub_rn(re, hb.x), __fsub_rn(im, hb.y));
    w[0] = *reinterpret_cast<const uint32_t*>(&h);
    w[1] = *reinterpret_cast<const uint32_t*>(&l);
  }
};
template <> struct Split<3> {                 // bf16 hi + mid + lo
  static constexpr uint32_t kFmt = 1;         // kind::f16 operand format: bf16
  static __device__ __forceinline__ void split(float re, float im, uint32_t (&w)[3]) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    const float2 hb = __bfloat1622float2(h);
    const float r1 = __fsub_rn(re, hb.x), i1 = __fsub_rn(im, hb.y);
    const __nv_bfloat162 m = __floats2bfloat162_rn(r1, i1);
    const float2 mb = __bfloat1622float2(m);
    const __nv_bfloat162 l = __floats2bfloat162_rn(__fsub_rn(r1, mb.x), __fsub_rn(i1, mb.y));
    w[0] = *reinterpret_cast<const uint32_t*>(&h);
    w[1] = *reinterpret_cast<const uint32_t*>(&m);
    w[2] = *reinterpret_cast<const uint32_t*>(&l);
  }
};

template <int N, int P> struct MixCfg {
  static constexpr int H = N / 2;
  static constexpr int WG = P == 2 ? 4 : 3;             // warpgroups per CTA (shared memory bound)
  static constexpr int THREADS = 128 * WG;
  static constexpr int KP = 2 * N;                      // 16-bit values per part per row
  static constexpr int KROW = (P * KP + 63) / 64 * 64;  // values per row, padded
  static constexpr int KB = KROW / 64;                  // 128-byte K blocks per row
  static constexpr int NOUT = 2 * N;                    // matrix rows (v, re/im)
  static constexpr int ROWS = N * N;                    // pencils of a full pass
  static constexpr int RB = 2 * KROW;                   // bytes per row
  static constexpr int PART_B = 2 * KP;                 // bytes per part in a row
  static constexpr int A_TILE = KB * 128 * 128;         // bytes of a 128-row A tile
  static constexpr int kb_of(int s) { return ((P - s) * KP + 63) / 64; }   // K blocks of matrix s
  static constexpr int set_bytes(int s) { return kb_of(s) * NOUT * 128; }
  static constexpr int set_off(int s) { return s == 0 ? 0 : set_off(s - 1) + set_bytes(s - 1); }
  static constexpr int B_SETS = set_off(P);
  static constexpr int GCOLS = N * N * N / 128;         // tensor-memory columns of G
  static constexpr int TCOLS_USED = WG * NOUT + GCOLS;
  static constexpr int TCOLS = TCOLS_USED <= 32 ? 32 : TCOLS_USED <= 64 ? 64 : TCOLS_USED <= 128 ? 128
                             : TCOLS_USED <= 256 ? 256 : 512;
  static constexpr int SMEM_USED = B_SETS + WG * A_TILE + 1024;
  // enough shared memory that no more CTAs share an SM than its 512 tensor-memory columns hold
  static constexpr int SMEM_MIN = 233472 / (512 / TCOLS) - 4096;
  static constexpr int SMEM = SMEM_USED > SMEM_MIN ? SMEM_USED : SMEM_MIN;
  static_assert(N % 16 == 0 && ROWS % 128 == 0 && (H * N) % 128 == 0, "tile shape");
  static_assert(WG <= kMixMaxWG, "warpgroups");
  static_assert(TCOLS_USED <= 512, "tensor memory");
  static_assert(B_SETS % 1024 == 0, "A tiles 1024-byte aligned");
  static_assert(SMEM <= 232448, "shared memory");
};

enum MixPass : int { kMF2 = 0, kMF1, kMF0, kMX, kMY, kMZ };

// Failure-injection switch for the bounded-wait test (coll_debug_mixed_drop_commit):
// when set, warpgroup 0 of every CTA omits the completion signal of its first
// MMA batch, so that its wait expires.
__device__ int g_mix_drop_commit = 0;

struct MixShared {
  uint64_t bar[kMixMaxWG];
  uint64_t tbar[kMixMaxWG];   // teardown: one fresh commit per warpgroup after an expired wait
  uint32_t tbase;
  int abort;
  int drop_commit;
  int bad;
  float fmax;
  float Fmax;
};

template <int N, typename Tio, int P>
struct MixCell {
  using C = MixCfg<N, P>;
  using S = Split<P>;
  static constexpr int H = C::H;
  static constexpr int kWG = C::WG;

  // cp.async of 128 rows (tile ti of the pass buffer) into the swizzled A tile
  static __device__ __forceinline__ void load_tile(const unsigned char* buf, int ti, int lt, uint32_t abase) {
    const unsigned char* s0 = buf + size_t(ti) * 128 * C::RB;
    for (int i = lt; i < 128 * C::KB * 8; i += 128) {
      const int row = i / (C::KB * 8), j = i % (C::KB * 8);
      cp_async16(abase + (j >> 3) * 16384 + row * 128 + (((j & 7) ^ (row & 7)) << 4),
                 s0 + size_t(row) * C::RB + j * 16);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }

  // One pass over all tiles of this warpgroup.  Returns false (uniformly over
  // the warpgroup) if an MMA wait expired; the expired phase stays pending.
  template <int pass>
  static __device__ __forceinline__ bool run(int wg, int lt, unsigned char* atile, uint32_t abase, uint32_t bbase,
                             uint32_t tacc, uint32_t tG,
                             uint32_t& phase, bool& pending, MixShared& sh, const Tio* __restrict__ f, Tio* __restrict__ Q,
                             float2* Fs, unsigned char* buf,
                             const float2* __restrict__ tab_t, float in_scale, float out_scale, bool first_term,
                             bool last_term, bool& bad, float& lmax) {
    constexpr int rows = (pass == kMF1 || pass == kMF0) ? H * N : N * N;
    constexpr int nout = pass == kMF2 ? N : C::NOUT;
    const int q = lt >> 5;
    for (int ti = wg; ti < rows / 128; ti += kWG) {
      const int r = ti * 128 + lt;
      // ---- A tile
      if constexpr (pass == kMF2) {
        const Tio* fr = f + size_t(r) * N;
#pragma unroll 1
        for (int k0 = 0; k0 < N; k0 += 4) {
          uint32_t w[4][P];
#pragma unroll
          for (int e = 0; e < 4; ++e) S::split(float(double(fr[k0 + e]) * double(in_scale)), 0.0f, w[e]);
#pragma unroll
          for (int p = 0; p < P; ++p)
            *reinterpret_cast<uint4*>(atile + a_off(lt, p * C::PART_B + 4 * k0)) =
                make_uint4(w[0][p], w[1][p], w[2][p], w[3][p]);
        }
      } else if constexpr (pass == kMX) {
        // Row (k0, k1): z[k2] = (A + iB) F for k2 < N/2 from row (k0, k1) of F
        // and of the term's table, for k2 > N/2 from the partner row (-k0, -k1)
        // at N - k2 (conjugated F).  Work item (row, j) covers k2 = 2j, 2j + 1
        // and their partners; consecutive lanes take consecutive 16-byte
        // pieces of the same rows, so every load instruction is coalesced.
        constexpr int JN = H / 2;                 // 16-byte pieces per half row
        constexpr int RPS = 128 / JN;             // rows per sweep of the warpgroup
        const float4* F4 = reinterpret_cast<const float4*>(Fs);
        const float4* T4 = reinterpret_cast<const float4*>(tab_t);
        const int j = lt % JN;
#pragma unroll 2
        for (int it = 0; it < JN; ++it) {
          const int row = it * RPS + lt / JN;
          const int rr = ti * 128 + row;
          const int k0 = rr / N, k1 = rr % N;
          const int rp = ((N - k0) % N) * N + (N - k1) % N;
          const float4 F = __ldcg(F4 + size_t(rr) * JN + j), T = __ldg(T4 + size_t(rr) * JN + j);
          const float4 G = __ldcg(F4 + size_t(rp) * JN + j), U = __ldg(T4 + size_t(rp) * JN + j);
          uint32_t a0[P], a1[P], b0[P], b1[P];
          S::split(__fmul_rn(__fsub_rn(__fmul_rn(T.x, F.x), __fmul_rn(T.y, F.y)), in_scale),
                   __fmul_rn(__fadd_rn(__fmul_rn(T.x, F.y), __fmul_rn(T.y, F.x)), in_scale), a0);
          S::split(__fmul_rn(__fsub_rn(__fmul_rn(T.z, F.z), __fmul_rn(T.w, F.w)), in_scale),
                   __fmul_rn(__fadd_rn(__fmul_rn(T.z, F.w), __fmul_rn(T.w, F.z)), in_scale), a1);
          // partner: k2 = N - 2j - 1 and (j > 0) N - 2j, with conj(F)
          S::split(__fmul_rn(__fadd_rn(__fmul_rn(U.z, G.z), __fmul_rn(U.w, G.w)), in_scale),
                   __fmul_rn(__fsub_rn(__fmul_rn(U.w, G.z), __fmul_rn(U.z, G.w)), in_scale), b1);
          if (j > 0) {
            S::split(__fmul_rn(__fadd_rn(__fmul_rn(U.x, G.x), __fmul_rn(U.y, G.y)), in_scale),
                     __fmul_rn(__fsub_rn(__fmul_rn(U.y, G.x), __fmul_rn(U.x, G.y)), in_scale), b0);
          } else {
#pragma unroll
            for (int p = 0; p < P; ++p) b0[p] = 0u;
          }
          const int k2b = N - 2 * j - 1;
          // slot N - 2j for j > 0; for j == 0 the same store zeroes the Nyquist slot N/2
          const int k2a = j > 0 ? N - 2 * j : H;
#pragma unroll
          for (int p = 0; p < P; ++p) {
            *reinterpret_cast<uint2*>(atile + a_off(row, p * C::PART_B + 8 * j)) = make_uint2(a0[p], a1[p]);
            *reinterpret_cast<uint32_t*>(atile + a_off(row, p * C::PART_B + 4 * k2b)) = b1[p];
            *reinterpret_cast<uint32_t*>(atile + a_off(row, p * C::PART_B + 4 * k2a)) = b0[p];
          }
        }
      } else {
        if (ti == wg) load_tile(buf, ti, lt, abase);     // first tile; later ones were prefetched
        cp_async_wait_all();
      }
      fence_async_smem();
      wg_sync(wg);
      // ---- MMAs: matrix s (part s of D) against the first P - s parts of the operand
      if (lt == 0) {
        fence_after();
        const uint32_t id = idesc_f16(128, nout, S::kFmt);
        // descriptors of the tile bases; each K step adds a compile-time offset
        // to the 14-bit start-address field (shared addresses stay below 2^18
        // bytes, so the field never carries)
        const uint64_t ad = sw128_desc(abase), bd = sw128_desc(bbase);
        uint32_t acc = 0;
#pragma unroll
        for (int sp = 0; sp < P; ++sp) {
#pragma unroll
          for (int kk = 0; kk < (P - sp) * C::KP / 16; ++kk) {
            mma_f16(tacc, ad + uint64_t(((kk >> 2) * 16384 + (kk & 3) * 32) >> 4),
                    bd + uint64_t((C::set_off(sp) + (kk >> 2) * (C::NOUT * 128) + (kk & 3) * 32) >> 4), id, acc);
            acc = 1;
          }
        }
        if (wg == 0 && sh.drop_commit) sh.drop_commit = 0;   // injected failure: no completion signal
        else mma_commit(&sh.bar[wg]);
      }
      if (!wg_all(wg, wait_parity(&sh.bar[wg], phase))) {
        if (lt == 0) atomicExch(&sh.abort, 1);
        pending = true;
        return false;
      }
      phase ^= 1u;
      fence_after();
      // the MMAs have read the A tile: start copying this warpgroup's next tile
      // of the pass so that the copy overlaps the epilogue
      if (pass != kMF2 && pass != kMX && ti + kWG < rows / 128) load_tile(buf, ti + kWG, lt, abase);
      // ---- epilogue: thread = TMEM lane = pencil row r
      const uint32_t lane_base = static_cast<uint32_t>(32 * q) << 16;
      for (int c0 = 0; c0 < nout; c0 += 32) {
        uint32_t a[32];
        tld32(tacc + lane_base + c0, a);
        const int v0c = c0 >> 1;                         // first output index of this chunk
        const int ne = (nout >> 1) - v0c < 16 ? (nout >> 1) - v0c : 16;
        if constexpr (pass == kMZ) {
          // G[(v0, v1)][v2] for v2 = v0c .. v0c + 15
          const uint32_t gaddr = tG + lane_base + ti * N + v0c;
          uint32_t g[16];
          if (!first_term) tld16(gaddr, g);
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const float re = __uint_as_float(a[2 * e]), im = __uint_as_float(a[2 * e + 1]);
            const float p = __fmul_rn(__fmul_rn(re, im), out_scale);
            const float gv = first_term ? p : __fadd_rn(__uint_as_float(g[e]), p);
            g[e] = __float_as_uint(gv);
          }
          if (!last_term) {
            tst16(gaddr, g);
          } else {
            // r = (v2, v1), outputs v0: Q[v0][v1][v2]
            Tio* qr = Q + (size_t(v0c) * N + (r % N)) * N + (r / N);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
              const float gv = __uint_as_float(g[e]);
              bad |= !isfinite(gv);
              qr[size_t(e) * N * N] = Tio(gv);
            }
          }
        } else if constexpr (pass == kMF0) {
          const int k2h = r / N, k1 = r % N;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            const int k0 = v0c + e;
            float re = __fmul_rn(__uint_as_float(a[2 * e]), out_scale);
            float im = -__fmul_rn(__uint_as_float(a[2 * e + 1]), out_scale);
            if (k0 == H || k1 == H) { re = 0.0f; im = 0.0f; }
            lmax = fmaxf(lmax, __fadd_rn(fabsf(re), fabsf(im)));
            Fs[(size_t(k0) * N + k1) * H + k2h] = make_float2(re, im);
          }
        } else {
          // split and store into the next pass's row, slot = this pencil's next-K index:
          //   F2: r = (v0, v1), out k2h -> row (k2h, v0), slot v1
          //   F1: r = (k2h, v0), out k1 -> row (k2h, k1), slot v0
          //   X:  r = (k0, k1), out v2 -> row (v2, k0), slot k1
          //   Y:  r = (v2, k0), out v1 -> row (v2, v1), slot k0
          constexpr int dstride = (pass == kMF2 || pass == kMX) ? N : 1;
          const int drow0 = (pass == kMF2 || pass == kMX) ? r / N : (r / N) * N;
          unsigned char* base0 = buf + size_t(drow0 + v0c * dstride) * C::RB + (r % N) * 4;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            if (e >= ne) break;
            uint32_t w[P];
            S::split(__uint_as_float(a[2 * e]), __uint_as_float(a[2 * e + 1]), w);
            unsigned char* rowp = base0 + size_t(e) * dstride * C::RB;
#pragma unroll
            for (int p = 0; p < P; ++p) *reinterpret_cast<uint32_t*>(rowp + p * C::PART_B) = w[p];
          }
        }
      }
      fence_before();
      wg_sync(wg);
    }
    return true;
  }

  // Whole cell; returns true (uniformly) if the CTA must stop (a wait expired).
  static __device__ bool cell(const Tio* __restrict__ f, Tio* __restrict__ Q, const float2* __restrict__ tab,
                              const float* __restrict__ tmax, int n_terms, unsigned char* ws, unsigned char* atile,
                              uint32_t abase,
                              uint32_t bbase, uint32_t tacc, uint32_t tG, uint32_t& phase, bool& pending,
                              MixShared& sh, bool& bad) {
    const int tid = threadIdx.x, wg = tid >> 7, lt = tid & 127;
    float2* Fs = reinterpret_cast<float2*>(ws);
    unsigned char* buf = ws + size_t(N) * H * N * 8;
    constexpr int cap = 14 - 3 * (N == 16 ? 4 : 5);     // input modulus bound 2^cap = 2^14 / N^3
    auto stop = [&]() -> bool {                          // same answer on every thread
      __syncthreads();
      const bool v = *reinterpret_cast<volatile int*>(&sh.abort) != 0;
      __syncthreads();
      return v;
    };

    // max |f| for the forward scale
    float m = 0.0f;
    for (int i = tid; i < N * N * N; i += C::THREADS) m = fmaxf(m, float(fabs(double(f[i]))));
    if (tid == 0) { sh.fmax = 0.0f; sh.Fmax = 0.0f; }
    __syncthreads();
    atomic_max_nonneg(&sh.fmax, m);
    __syncthreads();
    const int ef = cap - exp_of(sh.fmax);
    float lmax = 0.0f;
    run<kMF2>(wg, lt, atile, abase, bbase, tacc, tG, phase, pending, sh, f, Q, Fs, buf, tab, ldexpf(1.0f, ef), 1.0f,
        false, false, bad, lmax);
    if (stop()) return true;
    run<kMF1>(wg, lt, atile, abase, bbase, tacc, tG, phase, pending, sh, f, Q, Fs, buf, tab, 1.0f, 1.0f, false,
        false, bad, lmax);
    if (stop()) return true;
    run<kMF0>(wg, lt, atile, abase, bbase, tacc, tG, phase, pending, sh, f, Q, Fs, buf, tab, 1.0f, ldexpf(1.0f, -ef),
        false, false, bad, lmax);
    atomic_max_nonneg(&sh.Fmax, lmax);
    if (stop()) return true;
    const float Fmax = sh.Fmax;
    for (int t = 0; t < n_terms; ++t) {
      const float bound = __fmul_ru(__fmul_ru(Fmax, tmax[t]), 1.0000005f);
      const int et = cap - exp_of(bound);
      const float2* tab_t = tab + size_t(t) * N * N * H;
      run<kMX>(wg, lt, atile, abase, bbase, tacc, tG, phase, pending, sh, f, Q, Fs, buf, tab_t, ldexpf(1.0f, et),
          1.0f, false, false, bad, lmax);
      if (stop()) return true;
      run<kMY>(wg, lt, atile, abase, bbase, tacc, tG, phase, pending, sh, f, Q, Fs, buf, tab_t, 1.0f, 1.0f, false,
          false, bad, lmax);
      if (stop()) return true;
      run<kMZ>(wg, lt, atile, abase, bbase, tacc, tG, phase, pending, sh, f, Q, Fs, buf, tab_t, 1.0f,
          ldexpf(1.0f, -2 * et), t == 0, t == n_terms - 1, bad, lmax);
      if (stop()) return true;
    }
    return false;
  }
};

template <int N, typename Tio, int P>
__global__ void __launch_bounds__(MixCfg<N, P>::THREADS, 1) mixed_kernel(CollArgs a) {
  using C = MixCfg<N, P>;
  extern __shared__ __align__(1024) unsigned char smraw[];
  __shared__ MixShared sh;
  const int tid = threadIdx.x, warp = tid >> 5, wg = tid >> 7;
  const uint32_t raw = su32(smraw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* sm = smraw + (base - raw);
  const uint32_t bbase = base;                                   // B1, B2
  const uint32_t abase = base + C::B_SETS + wg * C::A_TILE;       // this warpgroup's A tile

  // matrices: copy the pre-swizzled image
  const unsigned char* img = static_cast<const unsigned char*>(a.tab) + mixed_img_offset(N, a.n_terms);
  static_assert(C::B_SETS % 16 == 0, "matrix image copied in 16-byte pieces");
  for (int i = tid; i < C::B_SETS / 16; i += C::THREADS)
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
    sh.abort = 0;
    sh.drop_commit = g_mix_drop_commit;
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = sh.tbase;
  const uint32_t tacc = tbase + wg * C::NOUT;
  const uint32_t tG = tbase + C::WG * C::NOUT;
  uint32_t phase = 0;
  bool pending = false, bad = false;
  const auto* tab = static_cast<const float2*>(a.tab);
  const float* tmax = reinterpret_cast<const float*>(static_cast<const unsigned char*>(a.tab) +
                                                     mixed_tmax_offset(N, a.n_terms));
  unsigned char* ws = static_cast<unsigned char*>(a.ws) + size_t(blockIdx.x) * a.ws_per_cta;
  for (long long c = blockIdx.x; c < a.n_cells; c += gridDim.x) {
    const Tio* f = static_cast<const Tio*>(a.f) + size_t(c) * N * N * N;
    Tio* Q = static_cast<Tio*>(a.Q) + size_t(c) * N * N * N;
    if (MixCell<N, Tio, P>::cell(f, Q, tab, tmax, a.n_terms, ws, sm + C::B_SETS + wg * C::A_TILE, abase, bbase, tacc, tG, phase, pending, sh, bad))
      break;
  }
  // A wait that expired may leave this warpgroup's last MMA batch in flight,
  // and its own completion signal may never come.  A fresh commit from the
  // issuing thread to a barrier of its own arrives once every MMA that thread
  // started has completed; tensor memory is freed only after that arrival
  // (bounded wait).
  if (pending) {
    if ((tid & 127) == 0) mma_commit(&sh.tbar[wg]);
    (void)wait_parity(&sh.tbar[wg], 0);
  }
  fence_before();
  if (__syncthreads_or(bad) && tid == 0) atomicOr(a.status, kStatusNonFinite);
  if (sh.abort && tid == 0) atomicOr(a.status, kStatusTimeout);
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(C::TCOLS));
  }
}

template <int N, typename Tio, int P>
int launch_mixed_t(const CollArgs& a, int grid, cudaStream_t st) {
  using C = MixCfg<N, P>;
  auto k = mixed_kernel<N, Tio, P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return int(e);
  k<<<grid, C::THREADS, C::SMEM, st>>>(a);
  return int(cudaGetLastError());
}

template <int N, typename Tio, int P>
int occupancy_mixed_t(int* ctas) {
  using C = MixCfg<N, P>;
  auto k = mixed_kernel<N, Tio, P>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
  if (e != cudaSuccess) return int(e);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k, C::THREADS, C::SMEM);
  const int by_tmem = 512 / C::TCOLS;
  if (*ctas > by_tmem) *ctas = by_tmem;
  return int(e);
}

// IEEE binary16, round to nearest even (host)
uint16_t half_bits(double x) {
  const __half h = __double2half(x);
  uint16_t b;
  std::memcpy(&b, &h, 2);
  return b;
}
double half_value(uint16_t b) {
  __half h;
  std::memcpy(&h, &b, 2);
  return double(__half2float(h));
}
// bfloat16: round the FP32 value to nearest even (host)
uint16_t bf16_bits(double x) {
  const float f = float(x);
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return uint16_t(u >> 16);
}
double bf16_value(uint16_t b) {
  const uint32_t u = uint32_t(b) << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return double(f);
}

}  // namespace

int mixed_set_drop_commit(int on) {
  const int v = on ? 1 : 0;
  return int(cudaMemcpyToSymbol(g_mix_drop_commit, &v, sizeof(int)));
}

bool mixed_layout(int N, int parts, LayoutInfo* out) {
  if ((N != 16 && N != 32) || (parts != 2 && parts != 3)) return false;
  LayoutInfo i;
  i.N = N;
  i.S0 = 1;
  i.threads = parts == 2 ? MixCfg<16, 2>::THREADS : MixCfg<16, 3>::THREADS;
  i.fh_smem = false;
  i.w_smem = false;
  i.g_smem = true;
  const size_t rb = parts == 2 ? (N == 16 ? MixCfg<16, 2>::RB : MixCfg<32, 2>::RB)
                               : (N == 16 ? MixCfg<16, 3>::RB : MixCfg<32, 3>::RB);
  i.fh_bytes = size_t(N) * (N / 2) * N * 8;        // forward half spectrum (FP32 complex)
  i.w_bytes = size_t(N) * N * rb;                  // one pass buffer
  i.g_bytes = 0;                                   // the gain accumulator lives in tensor memory
  i.ws = i.fh_bytes + i.w_bytes;
  *out = i;
  return true;
}

int launch_mixed(int N, bool io_f64, int parts, const CollArgs& a, int grid, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (parts == 2) {
    if (N == 16) return io_f64 ? launch_mixed_t<16, double, 2>(a, grid, st) : launch_mixed_t<16, float, 2>(a, grid, st);
    if (N == 32) return io_f64 ? launch_mixed_t<32, double, 2>(a, grid, st) : launch_mixed_t<32, float, 2>(a, grid, st);
  } else if (parts == 3) {
    if (N == 16) return io_f64 ? launch_mixed_t<16, double, 3>(a, grid, st) : launch_mixed_t<16, float, 3>(a, grid, st);
    if (N == 32) return io_f64 ? launch_mixed_t<32, double, 3>(a, grid, st) : launch_mixed_t<32, float, 3>(a, grid, st);
  }
  return int(cudaErrorInvalidValue);
}

int mixed_max_ctas_per_sm(int N, bool io_f64, int parts, int* ctas) {
  if (parts == 2) {
    if (N == 16) return io_f64 ? occupancy_mixed_t<16, double, 2>(ctas) : occupancy_mixed_t<16, float, 2>(ctas);
    if (N == 32) return io_f64 ? occupancy_mixed_t<32, double, 2>(ctas) : occupancy_mixed_t<32, float, 2>(ctas);
  } else if (parts == 3) {
    if (N == 16) return io_f64 ? occupancy_mixed_t<16, double, 3>(ctas) : occupancy_mixed_t<16, float, 3>(ctas);
    if (N == 32) return io_f64 ? occupancy_mixed_t<32, double, 3>(ctas) : occupancy_mixed_t<32, float, 3>(ctas);
  }
  return int(cudaErrorInvalidValue);
}

// Device image of a mixed plan: per-term tables [t][k0][k1][k2h] (A, B) as
// float2, per-term max |A + iB| (rounded up), then the swizzled 16-bit
// matrices B_s (part s of the inverse N-point DFT matrix, applied to the first
// parts - s parts of the operand).
coll_status build_mixed_image(const HostTables& ht, int N, int parts, std::vector<unsigned char>* out) {
  const int H = N / 2, nt = ht.n_terms;
  const size_t img_off = mixed_img_offset(N, nt);
  const int KP = 2 * N, NOUT = 2 * N, P = parts;
  size_t set_off[4] = {0, 0, 0, 0};
  for (int sp = 0; sp < P; ++sp) set_off[sp + 1] = set_off[sp] + size_t(((P - sp) * KP + 63) / 64) * NOUT * 128;
  out->assign(img_off + set_off[P], 0);
  float2* tab = reinterpret_cast<float2*>(out->data());
  float* tmax = reinterpret_cast<float*>(out->data() + mixed_tmax_offset(N, nt));
  for (int t = 0; t < nt; ++t) {
    double mx = 0.0;
    for (int k0 = 0; k0 < N; ++k0)
      for (int k1 = 0; k1 < N; ++k1)
        for (int k2 = 0; k2 < H; ++k2) {
          const size_t src = ((size_t(t) * N + k0) * N + k1) * H + k2;
          const double A = ht.tab[2 * src], B = ht.tab[2 * src + 1];
          tab[src] = make_float2(float(A), float(B));
          mx = std::fmax(mx, std::sqrt(A * A + B * B));
        }
    tmax[t] = float(mx * (1.0 + 1e-6));
  }
  unsigned char* img = out->data() + img_off;
  const double two_pi = 6.283185307179586476925286766559;
  auto put = [&](size_t region, int j, int kk, uint16_t val) {     // swizzled K-major position
    const int kb = kk / 64, e = kk % 64, chunk = e / 8, within = e % 8;
    const size_t off = region + size_t(kb) * NOUT * 128 + size_t(j) * 128 + size_t((chunk ^ (j & 7)) * 16) +
                       size_t(within) * 2;
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
      uint16_t part[3];
      if (P == 2) {
        part[0] = half_bits(d);
        part[1] = half_bits(d - half_value(part[0]));
      } else {
        part[0] = bf16_bits(d);
        const double r1 = d - bf16_value(part[0]);
        part[1] = bf16_bits(r1);
        part[2] = bf16_bits(r1 - bf16_value(part[1]));
      }
      for (int sp = 0; sp < P; ++sp)
        for (int q = 0; q < P - sp; ++q) put(set_off[sp], j, q * KP + kk, part[sp]);
    }
  }
  return COLL_OK;
}

}  // namespace coll
