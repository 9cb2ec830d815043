/*
 * coll.h -- C ABI of the GB300 collision-operator library (libcoll.so).
 *
 * The library evaluates, for a batch of spatial cells, the truncated Carleman
 * form of the Boltzmann collision operator on a periodic 3D velocity grid
 * (arxiv 2505.03360, sec. 4.4.1, eq. for Q^R and the separated kernel
 * beta_F = sum_p alpha_p alpha'_p), and the per-cell moments / realizability
 * test that decides which cells need it (sec. 3.2, eq. for V_eps; App. A;
 * sec. 3.3, L1 criterion).
 *
 * Conventions shared by every entry point
 *   - Memory: every data pointer (f, Q, workspace, moments, mask) is a DEVICE
 *     pointer owned by the caller; the library never frees it.  A plan owns
 *     only its device tables (allocated in coll_plan_create, freed in
 *     coll_plan_destroy).  Evaluation calls never allocate.
 *   - Streams: work is enqueued asynchronously on the given cudaStream_t
 *     (0 = legacy default stream).  Argument errors are detected on the host
 *     before anything is launched and returned synchronously.
 *   - Device-side errors (bounded-wait timeouts, non-finite results) are
 *     recorded in a sticky status word of the plan, read by
 *     coll_device_status() after the caller synchronises the stream.
 *   - The library never calls abort, exit or printf.
 *   - Threads: a plan is immutable after creation and may be used from
 *     several host threads / streams concurrently, each with its own
 *     workspace.
 *   - Layout: a cell's distribution f is N^3 contiguous values in C order,
 *     f[j0][j1][j2] = f(v_{j0}, v_{j1}, v_{j2}) with v_j = -L + j * 2L/N
 *     (velocity grid of sec. 4.1, which contains v = 0).  Cells are
 *     contiguous: cell c starts at c * N^3 elements.
 */
#ifndef COLL_H
#define COLL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without pulling in the CUDA headers. */
typedef struct CUstream_st* coll_stream;

typedef struct coll_plan_s* coll_plan;   /* opaque; immutable after create */

typedef enum {
  COLL_OK = 0,
  COLL_EINVAL = 1,        /* invalid argument (null pointer, bad size, ...) */
  COLL_EUNSUPPORTED = 2,  /* valid but not implemented (e.g. N, precision)  */
  COLL_ENOMEM = 3,        /* device allocation of plan tables failed /
                             workspace smaller than coll_workspace_size()    */
  COLL_ECUDA = 4,         /* a CUDA runtime call failed                      */
  COLL_ETIMEOUT = 5,      /* a bounded device-side wait gave up              */
  COLL_ENONFINITE = 6     /* a non-finite value was produced                 */
} coll_status;

typedef enum {
  COLL_F64 = 0,           /* transforms and products in FP64                  */
  COLL_F32 = 1,           /* transforms and products in FP32                  */
  COLL_MIXED_F16X2 = 2,   /* every transform a DFT-GEMM on the tensor cores,
                             f16 hi+lo operands (3 products), FP32 accumulate;
                             N = 16, 32; not in ragged launches              */
  COLL_MIXED_BF16X3 = 3,  /* the same with bf16 hi+mid+lo operands (6
                             products); N = 16, 32; not in ragged launches   */
  COLL_F32X2 = 4,         /* transforms in float pairs (hi + lo, ~48 bits) on
                             the FP32 pipe; N = 16, 24, 32                    */
  COLL_MIXED_SLICED = 5   /* every transform a DFT-GEMM on the tensor cores
                             with fixed-point f16 operand slices (three 9-bit
                             integer parts and an f16 tail per value); the two
                             leading product levels are summed exactly by the
                             FP32 accumulator, intermediates are float pairs:
                             about 38 significant bits per transform (relative
                             L2 error ~1e-8 against FP64); N = 16, 32; in
                             ragged launches over groups of one N              */
} coll_precision;

/*
 * Plan descriptor (sec. 4.4.1 "The 3d case", with the readings listed in the
 * design notes):
 *   N        points per velocity axis; 16, 24, 32, 48 or 64 (FP64 and
 *            COLL_F32X2: 16, 24, 32; tensor-core precisions COLL_MIXED_*:
 *            16, 32)
 *   L        half-width of the periodic velocity box [-L, L)^3
 *   S        support radius; truncation R = 2S (sec. 4.4.1, Q^R);
 *            0 selects S = 2L / (3 + sqrt 2), the no-overlap bound
 *   lambda   VHS exponent gamma of B = b0 |g|^gamma (sec. 2.1); 0 <= lambda <= 1
 *   b0       kernel constant C_gamma; <= 0 selects 1/(4 pi) for lambda = 0
 *            (int b dsigma = 1, BKW normalisation) and 1 otherwise
 *   M        number of directions on the full sphere (antipodal pairs share a
 *            multiplier, so M/2 hemisphere directions are used)
 *   Mtheta   sphere_rule 0: Gauss-Legendre nodes in cos(theta) (even);
 *            Mphi = M / Mtheta uniform azimuths (even).
 *            sphere_rule 1: A1 = Mtheta polar midpoints, A2 = M/(2 A1)
 *            azimuthal midpoints over a hemisphere (the paper's grid).
 *   Mr       Gauss-Legendre nodes of the radius |x| on [0, R]
 *   sphere_rule  0 (default) or 1, see above
 *   dealias  0: N-point circular products (default).  1: Galerkin products:
 *            f is interpolated spectrally onto the 3N/2 grid, the quadratic
 *            terms are formed there (no aliasing into the modes |k_d| < N/2)
 *            and Q is projected back onto those modes; the kernel runs on the
 *            3N/2 grid, so each evaluation costs about (3/2)^3 log(3N/2)/log N
 *            times more, plus six resampling passes.  Supported: COLL_F32 at
 *            N = 16, 32; COLL_F64 and COLL_F32X2 at N = 16; otherwise
 *            COLL_EUNSUPPORTED.  Not in ragged launches, coll_plan_autotune or
 *            coll_eval_batch_static (COLL_EUNSUPPORTED).
 *   prec     compute precision of the transforms (coll_precision)
 *   io_dtype 0: f and Q are double; 1: f and Q are float
 *   rank     lambda != 1 only: 0 (default) keeps one term per direction and
 *            radial node (M/2 x Mr gain terms); 1 <= rank <= Mr keeps `rank`
 *            terms per direction, the low-rank separable approximation of the
 *            radial kernel B~(|x|, |y|) (the separated kernel of sec. 4.4.1 in
 *            its SVD form: the eigenvectors of the Gram matrix
 *            G_ii' = a_i a_i' int_0^R g_i g_i' dr, a_i = 2 W_i rho_i,
 *            g_i(r) = 2 pi r (rho_i^2 + r^2)^((lambda-1)/2), largest first);
 *            mass stays exact for every rank; rank = Mr is the full operator.
 *            The factors are the singular vectors of the radial kernel
 *            factor (long double one-sided Jacobi at plan time), each
 *            determined to rounding over its gap to the next singular value.
 *            At lambda = 0, Mr = 8 the relative L2 distance to rank 0 is about
 *            2e-4 at rank 4, 8e-5 at rank 5, 1e-6 at rank 6, 1e-9 at rank 7.
 *            Ignored for lambda = 1 (one term per direction already).
 *            COLL_EINVAL outside 0 .. Mr.
 */
typedef struct {
  int32_t N;
  double L;
  double S;
  double lambda;
  double b0;
  int32_t M;
  int32_t Mtheta;
  int32_t Mr;
  int32_t sphere_rule;
  int32_t dealias;
  int32_t prec;
  int32_t io_dtype;
  int32_t rank;
} coll_plan_desc;

/*
 * Build a plan: quadrature rules, the multiplier tables alpha_t, alpha'_t and
 * the loss multiplier Lambda = sum_t c_t alpha_t alpha'_t on the half spectrum
 * (sec. 4.4.1, eq. beta_F ~ sum_p alpha_p(l) alpha'_p(m)), uploaded once to the
 * current device.  Returns COLL_EINVAL / COLL_EUNSUPPORTED for bad or
 * unsupported descriptors, COLL_ENOMEM / COLL_ECUDA if the upload fails; *out
 * is set only on COLL_OK.
 */
coll_status coll_plan_create(const coll_plan_desc* desc, coll_plan* out);

/* Free the plan's device tables.  The caller must ensure no launch using the
 * plan is still in flight (synchronise its streams first). */
coll_status coll_plan_destroy(coll_plan plan);

/* Number of separated terms T the plan evaluates per cell, including the loss
 * term (M/2 for lambda = 1, M/2 * Mr otherwise (M/2 * rank with a rank), plus 1). */
coll_status coll_plan_terms(coll_plan plan, int32_t* n_terms);

/*
 * Device workspace (bytes) needed by coll_eval_batch for up to max_cells
 * cells on the plan's device.  The workspace holds per-CTA scratch of the
 * persistent kernel (forward spectrum, transposed slabs, gain accumulator);
 * its size depends on the grid size, not on max_cells beyond the CTA count.
 * In the Galerkin mode (dealias = 1) it also holds, per cell, f and Q on the
 * 3N/2 grid and two complex resampling buffers of N (3N/2)^2 values, so it
 * grows with max_cells (about 2.1 MB per FP32 cell at N = 32).
 */
coll_status coll_workspace_size(coll_plan plan, int64_t max_cells, size_t* bytes);

/*
 * Q[c] = Q^R(f[c], f[c]) for c = 0 .. n_cells-1 (sec. 4.4.1):
 *   fh = DFT(f) with every |k_d| = N/2 mode dropped;
 *   Q  = sum_t IDFT(c_t alpha_t fh) * IDFT(alpha'_t fh) - IDFT(fh) * IDFT(Lambda fh).
 * f, Q: device arrays of n_cells * N^3 elements of the plan's io_dtype; Q may
 * not alias f.  ws: device workspace of at least coll_workspace_size(plan,
 * n_cells) bytes, 256-byte aligned.  n_cells = 0 is a no-op returning COLL_OK.
 */
coll_status coll_eval_batch(coll_plan plan, const void* f, void* Q, int64_t n_cells,
                            void* ws, size_t ws_bytes, coll_stream stream);

/*
 * Autotuner: the fused kernel has two slab shapes per (N, precision) (how
 * many v0-slabs the axis-0 inverse pass is split into, and which arrays stay
 * in shared memory; for FP32 N = 48 the second is the cluster form, four CTAs
 * per cell).  coll_plan_autotune times each on the caller's batch (one warm-up
 * and two timed evaluations each, on `stream`; the call synchronises) and
 * stores the faster one in the plan; *chosen (may be NULL) receives it.  Q is
 * overwritten.  ws must hold coll_workspace_size(plan, n_cells) bytes, which
 * covers every shape.  Results of both shapes agree to rounding (the same
 * operations in a different order of slabs), bit for bit where the shapes
 * share the schedule (FP32 N = 24, 48).  A new plan starts in shape 0, or in
 * the cluster form where the (N, precision) has one (faster at every batch
 * size: more SMs per cell for small batches, the cluster's workspace in L2 for
 * large ones).  coll_plan_set_variant selects a shape directly (0 or 1).
 */
coll_status coll_plan_autotune(coll_plan plan, const void* f, void* Q, int64_t n_cells, void* ws,
                               size_t ws_bytes, coll_stream stream, int32_t* chosen);
coll_status coll_plan_set_variant(coll_plan plan, int32_t variant);

/*
 * coll_eval_batch_static -- coll_eval_batch without a caller-provided
 * workspace, for callers that cannot allocate device memory: code that runs
 * while a CUDA graph is being captured (cudaMalloc is not allowed there),
 * hosts whose own allocator must own every device allocation and cannot hand
 * out a raw scratch block, or latency-critical loops that must never risk an
 * allocation.  The paper has no counterpart; this is a library convenience.
 *
 * The kernel's scratch is a fixed 32 MiB device array inside libcoll.so (every
 * GPU that loads the library keeps it until the process exits).  Its device
 * address is looked up on the first call on each device, with that device
 * current; make that first call before any stream capture.  The call
 * allocates and frees nothing.  If one CTA's scratch for this plan exceeds
 * 32 MiB it returns COLL_ENOMEM; otherwise the grid is capped so that the
 * scratch fits, so it may run fewer CTAs (and be slower) than
 * coll_eval_batch.  All calls share the array: the kernel clears what it
 * accumulates before using it, but calls whose launches overlap on the GPU
 * (different streams or host threads) race on the array and must be
 * serialised by the caller.  Arguments, errors and results are otherwise
 * those of coll_eval_batch.
 */
coll_status coll_eval_batch_static(coll_plan plan, const void* f, void* Q, int64_t n_cells,
                                   coll_stream stream);

/*
 * Ragged batch: n_groups (1 .. 256) groups, each with its own plan (its own N,
 * lambda, quadrature), its own f and Q arrays and cells_per_group[g] cells,
 * evaluated in ONE persistent launch: CTAs take cells from a device counter,
 * groups ordered by decreasing work per cell (terms x N^3 log N^3) so the
 * costliest cells start first.  Every plan must live on the current device
 * and use the same compute type, with
 * the io type that goes with it (COLL_F32: float io; COLL_F64 and COLL_F32X2:
 * double io); otherwise COLL_EUNSUPPORTED.  COLL_MIXED_SLICED groups must also
 * share N and their io type (one launch of the two-CTA-cluster tensor-core
 * kernel, cells strided over the clusters); the other tensor-core types have no
 * ragged launch (COLL_EUNSUPPORTED).  Galerkin plans (dealias = 1) are not
 * accepted (COLL_EUNSUPPORTED).  Results are bitwise identical to
 * coll_eval_batch of each group alone (same per-cell code and order of
 * operations).  ws (256-byte aligned) must hold coll_ragged_workspace_size()
 * bytes for the same groups; its first 256 bytes hold the work counter, reset
 * by an async memset on the stream before the launch (both capture into a
 * CUDA graph).
 */
typedef struct {
  coll_plan plan;
  const void* f;
  void* Q;
} coll_cell_group;

coll_status coll_ragged_workspace_size(const coll_cell_group* groups, const int64_t* cells_per_group,
                                       int32_t n_groups, size_t* bytes);
coll_status coll_eval_ragged(const coll_cell_group* groups, const int64_t* cells_per_group,
                             int32_t n_groups, void* ws, size_t ws_bytes, coll_stream stream);

/*
 * Per-cell moments record (sec. 2 H3; sec. 2.2 stress tensor; sec. 3.1 Abar,
 * Bbar; App. A tau, q, Cbar; sec. 3.2 V_eps).  Symmetric 3x3 tensors are
 * packed xx, yy, zz, xy, xz, yz.  eig are the eigenvalues of V_eps in
 * ascending order; l1 = ||f - M_{rho,u,T}||_{L1}.  40 doubles.
 */
typedef struct {
  double rho, u[3], T, Theta[6], tau[6], q[3], Abar[6], Bbar[3], Cbar, V[6], eig[3], l1;
} coll_moments;

/*
 * Moments, realizability and regime bits for n_cells cells of N^3 values
 * (io_dtype 0 = double, 1 = float) on the box [-L, L)^3.
 * mask_out[c] bits:
 *   bit0  realizability matrix M of sec. 3.2 not PSD (App. A Schur form)
 *   bit1  Euler breakdown: some eigenvalue lambda of V_eps with |lambda-1| > eta0
 *   bit2  ||f - M||_L1 > delta0 (sec. 3.3)
 *   bit7  the cell holds a non-finite value (bits 0-2 set too, moments NaN)
 * Every grid sum is an exact fixed-point integer sum, so mom_out (except eig)
 * and mask_out are bitwise reproducible and independent of launch shape.
 * f, mom_out (n_cells records) and mask_out (n_cells bytes) are device
 * pointers; N is even, 2 <= N <= 64.  Two kernels on the stream: the first
 * streams f and leaves exact integer sums in mom_out (used as scratch), the
 * second turns them into the records.  n_cells = 0 is a no-op.
 */
coll_status moments_realizability(const void* f, int32_t io_dtype, int32_t N, double L,
                                  int64_t n_cells, double eta0, double delta0,
                                  coll_moments* mom_out, uint8_t* mask_out, coll_stream stream);

/*
 * Collision invariants of Q, per cell (hypothesis H1, sec. 2: the collision
 * operator preserves mass, momentum and kinetic energy, int Q dv = 0,
 * int Q v dv = 0, int Q |v|^2 dv = 0; sec. 4.4.1: the truncated fast operator
 * keeps mass exactly, momentum and energy to its accuracy).  For n_cells
 * cells of N^3 values Q (io_dtype 0 = double, 1 = float; N in 16, 24, 32, 48,
 * 64; the grid v = -L + j 2L/N of coll_eval_batch) it writes eight doubles per
 * cell to out[c][0..7]:
 *   m0 = int Q,  m1[d] = int Q v_d (d = 0, 1, 2),  m2 = int Q |v|^2,
 *   a0 = int |Q|,  a1 = int |Q| (|v_0| + |v_1| + |v_2|),  a2 = int |Q| |v|^2,
 * so |m0| / a0, max_d |m1[d]| / a1 and |m2| / a2 are relative conservation
 * errors.  Every integral is an exact fixed-point sum (Q truncated to 2^-P,
 * P = 61 - e with max |Q| < 2^e, times integer grid monomials, v = h k) rounded
 * once to double and scaled by 2^-P h^3 (times h or h^2): bitwise reproducible
 * and independent of launch shape and order.  A cell with a non-finite value
 * gives eight NaN, an all-zero cell eight zeros.
 *   Q    device, [n_cells][N][N][N], 16-byte aligned
 *   out  device, [n_cells][8] doubles, caller-owned
 * One kernel on stream; allocates nothing.  COLL_EINVAL for negative n_cells,
 * a bad io_dtype or L, null or misaligned pointers; COLL_EUNSUPPORTED for
 * other N; n_cells = 0 is a no-op.
 */
coll_status coll_conservation(const void* Q, int32_t io_dtype, int32_t N, double L, int64_t n_cells,
                              double* out, coll_stream stream);

/*
 * Regime update on the 2D spatial grid (sec. 4.5, Algorithm 1): per cell the
 * central-difference gradients and Laplacians of rho, u_x, u_y, T over the
 * one-cell stencil (sec. 4.5), the three eigenvalues of the 2D matrix
 * V_eps^1 in closed form (sec. 3.3 and 4.5) with mu = mu0 sqrt(T) and
 * kappa = kappa0 sqrt(T) (hard spheres, sec. 3.1), the indicator
 * lambda_B = eps^2 (|grad T|^2/T + |grad u|^2
 *                   + sqrt((|Delta u|^2 + |Delta rho/rho|^2)(1 + T^2))) (sec. 3.3),
 * and the new regime:
 *   r = 2: 2 if |lambda_B| > eta1, else 1
 *   r = 1: 2 if |lambda_B| > eta1; else 0 if |lambda^k - 1| <= eta0 for all
 *          three eigenvalues and l1 <= delta0; else 1
 *   r = 0: 1 if |lambda^k - 1| > eta0 for some eigenvalue, else 0
 * Delta u is the vector (Delta u_x, Delta u_y).
 *   fields  device, 4 planes of (ny + 2) x (nx + 2) doubles, row-major
 *           [q][j][i] with q = rho, u_x, u_y, T: the nx x ny cells and a
 *           one-cell halo that the caller fills (boundary conditions)
 *   l1      device, [ny][nx] doubles: ||f - M||_L1 of each cell (the l1 field
 *           of moments_realizability); read only where r_in is 1
 *   r_in    device, [ny][nx] regimes r^n in {0, 1, 2}
 *   params  host: eps (Knudsen number), mu0, kappa0, dx, dy, eta0, eta1, delta0
 *   r_out   device, [ny][nx] regimes r^{n+1}; may be r_in (each cell reads and
 *           writes only its own entry).  A cell whose stencil holds a
 *           non-finite value, with rho <= 0 or T <= 0, a regime above 2, or
 *           (layer 1) a non-finite l1 keeps r^n with bit 7 set.
 *   ind     device, [4][ny][nx] doubles lambda^a, lambda^b, lambda^c, lambda_B,
 *           or NULL
 * Every indicator is one fixed sequence of correctly rounded double
 * operations, so r_out and ind are bitwise reproducible.  nx, ny >= 0
 * (0 cells: no-op); COLL_EINVAL for null pointers, non-positive dx, dy or
 * negative thresholds.  Asynchronous on stream.
 */
typedef struct {
  double eps, mu0, kappa0, dx, dy, eta0, eta1, delta0;
} coll_regime_params;
coll_status regime_update(const double* fields, const double* l1, const uint8_t* r_in, int32_t nx, int32_t ny,
                          const coll_regime_params* params, uint8_t* r_out, double* ind, coll_stream stream);

/*
 * Penalised IMEX time stepping of the space-homogeneous Boltzmann equation
 * df/dt = Q(f)/eps (sec. 4.4): Q is split as (Q - P) + P with the BGK-like
 * P(f) = beta (M - f), beta = 2 pi rho, M the Maxwellian with the moments of
 * f; Q - P is explicit, P implicit (solved in closed form because P keeps the
 * moments).  One elementwise stage per call, for n_cells cells of N^3 values:
 *   COLL_IMEX_FIRST_ORDER (eq. 1002): out = f^{n+1} from f, Q1 = Q(f) and
 *       mom0 (moments of f); with a transport term tr = v . grad_x f (or NULL)
 *       also mom1, the moments of f - dt tr (the U^{n+1} of the scheme):
 *       out = eps/(eps + b1 dt) (f - dt tr) + dt (Q1 - b0 (M0 - f))/(eps + b1 dt)
 *             + b1 dt/(eps + b1 dt) M1
 *   COLL_IMEX_PR_Y1 .. COLL_IMEX_PR_FINAL: the stages of PR(2,2,2) (sec. 4.3
 *       tableaux, g = 1 - 1/sqrt 2), all with the Maxwellian of f (mom0):
 *       Y1 = (eps f + dt g b M) / (eps + dt g b)                  [f, mom0]
 *       Y2 = (eps f + dt Q1 - 2 g dt b (M - Y) + dt g b M) / (eps + dt g b)
 *                                                  [f, Y = Y1, Q1 = Q(Y1), mom0]
 *       f^{n+1} = f + dt/(2 eps) (Q1 + Q2)          [f, Q1 = Q(Y1), Q2 = Q(Y2)]
 *   One PR(2,2,2) step: moments_realizability(f), Y1, coll_eval_batch(Y1),
 *   Y2, coll_eval_batch(Y2), final.
 * All arrays are device pointers of io_dtype (0 double, 1 float) holding
 * n_cells cells of N^3 values (N in {16, 24, 32, 48, 64}, other even N up to
 * 64: COLL_EUNSUPPORTED); mom0 / mom1 are moments_realizability records.  Arrays a stage does not read may be NULL;
 * out may be f (each value is read, then written, by the same thread).
 * COLL_EINVAL for a missing array, eps <= 0, dt < 0 or a bad size.
 * Asynchronous on stream; one launch.
 */
typedef enum {
  COLL_IMEX_FIRST_ORDER = 0,
  COLL_IMEX_PR_Y1 = 1,
  COLL_IMEX_PR_Y2 = 2,
  COLL_IMEX_PR_FINAL = 3
} coll_imex_stage_kind;
coll_status coll_imex_stage(int32_t stage, const void* f, const void* Y, const void* Q1, const void* Q2,
                            const void* tr, const coll_moments* mom0, const coll_moments* mom1, int32_t io_dtype,
                            int32_t N, double L, int64_t n_cells, double dt, double eps, void* out,
                            coll_stream stream);

/*
 * ES-BGK relaxation step (layer 1 of the hierarchy): one first-order IMEX step
 * of the space-homogeneous equation df/dt = Q_ES(f)/eps (sec. 4.3, eq. 1000
 * and the closed form after it) with Q_ES(f) = nu (G[f] - f), the Gaussian
 * G[f] = rho / sqrt(det(2 pi Tau)) exp(-(v - u)^T Tau^{-1} (v - u) / 2) and
 * the corrected tensor Tau = (1 - beta) T I + beta Theta (sec. 2.2,
 * Pr = 1/(1 - beta); beta = -1/2 for hard spheres).  Per cell, from its
 * moments record (rho, u, T, Theta of f^n): nu = rho sqrt(T)/((1 - beta) mu0),
 *   Theta^{n+1} = (eps Theta + (1 - beta) nu dt T I)/(eps + (1 - beta) nu dt),
 *   out = eps/(eps + nu dt) f + nu dt/(eps + nu dt) G[rho, u, Tau^{n+1}].
 * f, out: device, n_cells cells of N^3 values of io_dtype (0 double, 1 float),
 * N in {16, 24, 32, 48, 64}; mom: device records of moments_realizability for
 * f.  out may be f.  COLL_EINVAL for eps <= 0, dt < 0, beta >= 1, mu0 <= 0 or
 * a missing pointer.  Asynchronous on stream; one launch.
 */
coll_status coll_esbgk_step(const void* f, const coll_moments* mom, int32_t io_dtype, int32_t N, double L,
                            int64_t n_cells, double dt, double eps, double beta, double mu0, void* out,
                            coll_stream stream);

/*
 * Two-dimensional Maxwell molecules (sec. 4.4.1, "The 2d case"): the fast
 * spectral operator on a periodic 2D velocity grid, where the Carleman
 * weight is the constant Bt = 2 b0 (collision kernel B = b0) and the
 * separated kernel is exact up to the angle rule:
 *   K(l, m) = Bt int_0^pi phi(xi_l . e_theta) phi(xi_m . e_theta^perp) dtheta
 *          ~ sum_{p=1..A} c alpha_p(xi_l) alpha'_p(xi_m),
 *   alpha_p(xi) = phi(xi . e_p), alpha'_p(xi) = phi(xi . e_p^perp),
 *   phi(s) = 2R sinc(R s), theta_p = p pi / A, c = Bt pi / A,
 * and Q = sum_p c IDFT(alpha_p fh) IDFT(alpha'_p fh) - IDFT(fh) IDFT(Lambda fh)
 * with Lambda = sum_p c alpha_p alpha'_p and every |k_d| = N/2 mode dropped.
 * A cell is N^2 contiguous values f[j0][j1] = f(v_{j0}, v_{j1}),
 * v_j = -L + j 2L/N; cells are contiguous.
 *
 * Descriptor:
 *   N        points per velocity axis: 16, 32 (COLL_F32 also 64)
 *   L        half-width of the periodic box [-L, L)^2
 *   S        support radius; truncation R = 2S; 0 selects 2L / (3 + sqrt 2)
 *   b0       kernel constant; <= 0 selects 1/(2 pi) (int b dsigma = 1, the
 *            BKW normalisation)
 *   A        number of angles theta_p, 1 .. 4096
 *   prec     COLL_F64, COLL_F32 or COLL_F32X2 (others: COLL_EUNSUPPORTED)
 *   io_dtype 0: f and Q are double; 1: float
 * coll_m2d_plan_create builds the table of (A_t, B_t) = (c alpha_p / N^2,
 * alpha'_p / N^2) and the loss pair (-Lambda / N^2, 1 / N^2) on the half
 * spectrum and uploads it to the current device (A + 1 terms); the plan owns
 * it until coll_m2d_plan_destroy (synchronise first).  coll_m2d_eval_batch
 * computes Q[c] for n_cells cells of f (device arrays of the plan's io type,
 * Q not aliasing f) in one launch on stream, with no workspace: every
 * intermediate stays in shared memory.  n_cells = 0 is a no-op.  Errors as
 * for the 3D plan; non-finite results set the plan's sticky status, read by
 * coll_m2d_device_status (synchronous) and cleared by
 * coll_m2d_device_status_clear.
 */
typedef struct coll_m2d_plan_s* coll_m2d_plan;
typedef struct {
  int32_t N;
  double L;
  double S;
  double b0;
  int32_t A;
  int32_t prec;
  int32_t io_dtype;
} coll_m2d_plan_desc;
coll_status coll_m2d_plan_create(const coll_m2d_plan_desc* desc, coll_m2d_plan* out);
coll_status coll_m2d_plan_destroy(coll_m2d_plan plan);
coll_status coll_m2d_eval_batch(coll_m2d_plan plan, const void* f, void* Q, int64_t n_cells, coll_stream stream);
coll_status coll_m2d_device_status(coll_m2d_plan plan);
coll_status coll_m2d_device_status_clear(coll_m2d_plan plan);

/*
 * f <- f + dt * Q for n elements (io_dtype 0: double, 1: float), the explicit
 * Euler step of the space-homogeneous equation df/dt = Q(f,f) (sec. 2, the
 * kinetic equation without transport).  Device pointers, f and Q distinct;
 * asynchronous on stream.
 */
coll_status coll_advance(void* f, const void* Q, int64_t n, double dt, int32_t io_dtype, coll_stream stream);

/* Sticky device status of a plan (COLL_OK, COLL_ETIMEOUT, COLL_ENONFINITE);
 * synchronous: copies the word from the device.  Reading does not clear it. */
coll_status coll_device_status(coll_plan plan);

/* Clear the sticky device status of a plan (synchronous). */
coll_status coll_device_status_clear(coll_plan plan);

/* Static, human-readable name of a status code. */
const char* coll_status_string(coll_status s);

/* Number of kernels the library launched in this process (all entry points);
 * a host-side counter for launch accounting. */
int64_t coll_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* COLL_H */
