// extern "C" entry points of libcoll.so (declared in include/coll.h).
// Argument checking on the host, plan tables uploaded once, launches
// enqueued on the caller's stream.  No entry point aborts or prints.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "coll_internal.h"
#include "../../include/coll_debug.h"

namespace coll {
static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace coll

using namespace coll;

namespace {

bool valid_N(int N, int ctype) {
  if (is_mixed(ctype)) return N == 16 || N == 32;
  if (ctype != kCF32) return N == 16 || N == 24 || N == 32;
  return N == 16 || N == 24 || N == 32 || N == 48 || N == 64;
}

bool aligned256(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 255u) == 0; }

// CTAs of one launch (the workspace holds one slice per CTA): at most one
// resident wave and one cell per CTA; a cluster form takes whole clusters of C
// CTAs (one cell per cluster), at least one
int grid_for(const coll_plan_s* p, int variant, long long n_cells) {
  const long long C = p->lay[variant].cluster > 0 ? p->lay[variant].cluster : 1;
  long long g = static_cast<long long>(p->num_sms) * p->ctas_per_sm[variant];
  if (g > n_cells * C) g = n_cells * C;
  g = g / C * C;
  if (g < C) g = C;
  return int(g);
}

// Galerkin mode: per cell the padded f and Q (Tio) and two complex scratch
// buffers of the resampling (compute type), each slice 256-byte aligned
struct GalerkinWs {
  size_t pad_bytes, scr_bytes;
};
GalerkinWs galerkin_ws(const coll_plan_s* p, long long n_cells) {
  const size_t es = p->io_f64 ? 8 : 4, cs = p->ctype == kCF32 ? 8 : 16;
  const size_t n3 = size_t(p->Nk) * p->Nk * p->Nk;
  auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
  return {r256(size_t(n_cells) * n3 * es), r256(size_t(n_cells) * galerkin_scratch_elems(p->d.N) * cs)};
}

// workspace that serves every variant (the autotuner may switch variants)
size_t ws_need(const coll_plan_s* p, long long n_cells) {
  size_t b = 0;
  for (int v = 0; v < kVariants; ++v) {
    const size_t need = size_t(grid_for(p, v, n_cells)) * p->lay[v].ws_bytes_per_cta();
    b = need > b ? need : b;
  }
  if (p->galerkin) {
    const GalerkinWs g = galerkin_ws(p, n_cells);
    b = (b + 255) / 256 * 256 + 2 * g.pad_bytes + 2 * g.scr_bytes;
  }
  return b;
}

// Work of one cell of a plan, in units of N^3 log2 N^3 (the transforms'
// count): every term costs one complex inverse 3D transform of N^3 points.
double cell_cost(const coll_plan_s* p) {
  const double n3 = double(p->d.N) * p->d.N * p->d.N;
  return double(p->n_terms) * n3 * std::log2(n3);
}

// Validate a ragged request and build its launch table: groups sorted by
// decreasing cost per cell (terms x N^3 log N^3; the costliest cells are
// scheduled first so that the cheap ones fill the tail), prefix sums of cell
// counts.
coll_status ragged_prepare(const coll_cell_group* groups, const int64_t* cells, int32_t n, RaggedTable* t,
                           int* ctype, int* grid, size_t* ws_per_cta, size_t* total_bytes) {
  if (!groups || !cells || n <= 0 || n > kMaxRaggedGroups) return COLL_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return COLL_ECUDA;
  const coll_plan_s* p0 = groups[0].plan;
  if (!p0) return COLL_EINVAL;
  *ctype = p0->ctype;
  // SIMT compute types: one persistent kernel over every N; fixed-point slices:
  // one launch of the sliced kernel over groups of one N; other tensor-core types: none
  const bool sliced = p0->ctype == kCMixSliced;
  if (is_mixed(p0->ctype) && !sliced) return COLL_EUNSUPPORTED;
  const bool want_io_f64 = sliced ? p0->io_f64 : p0->ctype != kCF32;
  int order[kMaxRaggedGroups];
  for (int i = 0; i < n; ++i) {
    const coll_plan_s* p = groups[i].plan;
    if (!p || p->device != dev || cells[i] < 0) return COLL_EINVAL;
    if (p->galerkin) return COLL_EUNSUPPORTED;          // ragged launches run N-point products only
    if (p->ctype != *ctype) return COLL_EUNSUPPORTED;
    if (p->io_f64 != want_io_f64) return COLL_EUNSUPPORTED;
    if (sliced && p->d.N != p0->d.N) return COLL_EUNSUPPORTED;   // the sliced kernel is compiled per N
    if (cells[i] > 0 && (!groups[i].f || !groups[i].Q || groups[i].f == groups[i].Q)) return COLL_EINVAL;
    order[i] = i;
  }
  for (int i = 1; i < n; ++i)                       // stable insertion sort, cost per cell descending
    for (int j = i; j > 0 && cell_cost(groups[order[j]].plan) > cell_cost(groups[order[j - 1]].plan); --j) {
      const int tmp = order[j];
      order[j] = order[j - 1];
      order[j - 1] = tmp;
    }
  long long acc = 0;
  t->n_items = n;
  for (int k = 0; k < n; ++k) {
    const coll_cell_group& g = groups[order[k]];
    RaggedItem& it = t->items[k];
    it.f = g.f;
    it.Q = g.Q;
    it.tab = g.plan->tab_dev;
    it.n_cells = cells[order[k]];
    it.first_unit = acc;
    it.status = g.plan->status_dev;
    it.N = g.plan->d.N;
    it.n_terms = g.plan->n_terms;
    it.variant = g.plan->variant;
    acc += it.n_cells;
  }
  t->total_units = acc;
  t->io_f64 = want_io_f64 ? 1 : 0;
  t->smem_bytes = 0;
  for (int k = 0; k < n; ++k)
    if (t->items[k].n_cells > 0) {
      const size_t b = ragged_body_smem(t->items[k].N, *ctype, t->items[k].variant);
      t->smem_bytes = b > t->smem_bytes ? b : t->smem_bytes;
    }
  if (sliced) {                      // clusters of two CTAs, one cell each, workspace slot per CTA pair
    *ws_per_cta = p0->lay[0].ws_bytes_per_cta();
    long long g = static_cast<long long>(p0->num_sms) * p0->ctas_per_sm[0] / 2;
    if (g > acc) g = acc;
    if (g < 1) g = 1;
    *grid = int(2 * g);
    *total_bytes = 256 + size_t(*grid) * (*ws_per_cta);
    return COLL_OK;
  }
  int per = 0;
  if (ragged_max_ctas_per_sm(*ctype, &per) != 0 || per < 1) return COLL_ECUDA;
  size_t smem = 0;
  if (ragged_layout(*ctype, &smem, ws_per_cta) != 0) return COLL_ECUDA;
  long long g = static_cast<long long>(p0->num_sms) * per;
  if (g > acc) g = acc;
  if (g < 1) g = 1;
  *grid = int(g);
  *total_bytes = 256 + size_t(g) * (*ws_per_cta);
  return COLL_OK;
}

coll_status eval_variant(coll_plan_s* p, int v, const void* f, void* Q, int64_t n_cells, void* ws, size_t ws_bytes,
                         coll_stream stream) {
  const int grid = grid_for(p, v, n_cells);
  const size_t need = size_t(grid) * p->lay[v].ws_bytes_per_cta();
  if (need > 0 && (!ws || !aligned256(ws))) return COLL_EINVAL;
  if (ws_bytes < need) return COLL_ENOMEM;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return COLL_EINVAL;
  CollArgs a;
  a.f = f;
  a.Q = Q;
  a.n_cells = n_cells;
  a.tab = p->tab_dev;
  a.n_terms = p->n_terms;
  a.ws = ws;
  a.ws_per_cta = p->lay[v].ws_bytes_per_cta();
  a.status = p->status_dev;
  if (!p->galerkin) {
    const int e = launch_collision(p->Nk, p->ctype, p->io_f64, v, a, grid, stream);
    return e == 0 ? COLL_OK : COLL_ECUDA;
  }
  // Galerkin mode: f -> f_pad, the kernel on the padded grid, Q_pad -> Q
  if (!ws || !aligned256(ws)) return COLL_EINVAL;
  if (ws_bytes < ws_need(p, n_cells)) return COLL_ENOMEM;
  unsigned char* w = static_cast<unsigned char*>(ws) + (need + 255) / 256 * 256;
  const GalerkinWs g = galerkin_ws(p, n_cells);
  void* fpad = w;
  void* qpad = w + g.pad_bytes;
  void* sa = w + 2 * g.pad_bytes;
  void* sb = w + 2 * g.pad_bytes + g.scr_bytes;
  const bool cf64 = p->ctype != kCF32;
  int e = launch_galerkin_resample(true, p->d.N, cf64, p->io_f64, f, fpad, sa, sb, n_cells, stream);
  if (e == 0) {
    a.f = fpad;
    a.Q = qpad;
    e = launch_collision(p->Nk, p->ctype, p->io_f64, v, a, grid, stream);
  }
  if (e == 0) e = launch_galerkin_resample(false, p->d.N, cf64, p->io_f64, qpad, Q, sa, sb, n_cells, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

}  // namespace

extern "C" {

const char* coll_status_string(coll_status s) {
  switch (s) {
    case COLL_OK: return "COLL_OK";
    case COLL_EINVAL: return "COLL_EINVAL: invalid argument";
    case COLL_EUNSUPPORTED: return "COLL_EUNSUPPORTED: unsupported configuration";
    case COLL_ENOMEM: return "COLL_ENOMEM: allocation failed or workspace too small";
    case COLL_ECUDA: return "COLL_ECUDA: CUDA runtime error";
    case COLL_ETIMEOUT: return "COLL_ETIMEOUT: bounded device wait expired";
    case COLL_ENONFINITE: return "COLL_ENONFINITE: non-finite value produced";
  }
  return "unknown coll_status";
}

int64_t coll_launch_count(void) { return g_launches.load(); }

coll_status coll_plan_create(const coll_plan_desc* desc, coll_plan* out) {
  if (!desc || !out) return COLL_EINVAL;
  const coll_plan_desc d = *desc;
  if (!(d.L > 0) || !std::isfinite(d.L) || d.S < 0 || !(d.lambda >= 0 && d.lambda <= 1) || d.M <= 0 ||
      d.Mtheta <= 0 || d.Mr <= 0 || d.Mr > 256 || d.rank < 0 || d.rank > d.Mr || (d.io_dtype != 0 && d.io_dtype != 1) ||
      (d.sphere_rule != 0 && d.sphere_rule != 1) || (d.dealias != 0 && d.dealias != 1))
    return COLL_EINVAL;
  if (d.prec != COLL_F64 && d.prec != COLL_F32 && d.prec != COLL_MIXED_F16X2 && d.prec != COLL_MIXED_BF16X3 &&
      d.prec != COLL_F32X2 && d.prec != COLL_MIXED_SLICED)
    return COLL_EINVAL;
  const int ctype = d.prec == COLL_F64 ? kCF64
                  : d.prec == COLL_F32 ? kCF32
                  : d.prec == COLL_MIXED_F16X2 ? kCMixF16
                  : d.prec == COLL_MIXED_BF16X3 ? kCMixBF16
                  : d.prec == COLL_MIXED_SLICED ? kCMixSliced : kCDF;
  if (!valid_N(d.N, ctype)) return COLL_EUNSUPPORTED;
  // Galerkin mode: the kernel runs on the 3N/2 grid (FP32: N = 16, 32; FP64 and
  // float pairs: N = 16); the tensor-core paths have no padded grid
  const int Nk = d.dealias ? 3 * d.N / 2 : d.N;
  if (d.dealias && (is_mixed(ctype) || !valid_N(Nk, ctype) || !(d.N == 16 || d.N == 32))) return COLL_EUNSUPPORTED;
  coll_plan_desc kd = d;
  kd.N = Nk;

  HostTables ht;
  coll_status st = build_tables(kd, &ht, d.dealias ? d.N : 0);
  if (st != COLL_OK) return st;

  coll_plan_s* p = new (std::nothrow) coll_plan_s();
  if (!p) return COLL_ENOMEM;
  p->d = d;
  p->Nk = Nk;
  p->galerkin = d.dealias != 0;
  p->ctype = ctype;
  p->io_f64 = d.io_dtype == 0;
  p->n_terms = ht.n_terms;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return COLL_ECUDA; }
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  p->variant = 0;
  for (int v = 0; v < kVariants; ++v) {
    if (!layout_info(Nk, ctype, v, &p->lay[v])) { delete p; return COLL_EUNSUPPORTED; }
    int per = 0;
    if (collision_max_ctas_per_sm(Nk, ctype, p->io_f64, v, &per) != 0 || per < 1) {
      delete p;
      return COLL_ECUDA;
    }
    p->ctas_per_sm[v] = per;
    if (p->lay[v].cluster > 0) p->variant = v;        // the cluster form where there is one
  }

  const size_t n = ht.tab.size();
  std::vector<unsigned char> mix;
  if (is_mixed(ctype)) {
    st = ctype == kCMixSliced ? build_sliced_image(ht, d.N, &mix)
                              : build_mixed_image(ht, d.N, mixed_parts(ctype), &mix);
    if (st != COLL_OK) { delete p; return st; }
    p->tab_bytes = mix.size();
  } else {
    p->tab_bytes = n * (ctype == kCF32 ? sizeof(float) : sizeof(double));
  }
  if (cudaMalloc(&p->tab_dev, p->tab_bytes) != cudaSuccess) { delete p; return COLL_ENOMEM; }
  cudaError_t e;
  if (is_mixed(ctype)) {
    e = cudaMemcpy(p->tab_dev, mix.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  } else if (ctype == kCF64) {
    e = cudaMemcpy(p->tab_dev, ht.tab.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  } else if (ctype == kCF32) {
    std::vector<float> tf(n);
    for (size_t i = 0; i < n; ++i) tf[i] = float(ht.tab[i]);
    e = cudaMemcpy(p->tab_dev, tf.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  } else {
    // float pairs: head = nearest float, tail = nearest float to the remainder
    std::vector<float> tf(2 * n);
    for (size_t i = 0; i < n; ++i) {
      const float h = float(ht.tab[i]);
      tf[2 * i] = h;
      tf[2 * i + 1] = float(ht.tab[i] - double(h));
    }
    e = cudaMemcpy(p->tab_dev, tf.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&p->status_dev), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->status_dev, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(p->tab_dev);
    delete p;
    return COLL_ECUDA;
  }
  *out = p;
  return COLL_OK;
}

coll_status coll_plan_tables_host(const coll_plan_desc* desc, double* out, size_t cap, int32_t* n_terms,
                                  size_t* n_doubles) {
  if (!desc || !n_terms || !n_doubles) return COLL_EINVAL;
  const coll_plan_desc d = *desc;
  if (!(d.L > 0) || d.M <= 0 || d.Mtheta <= 0 || d.Mr <= 0 || d.N < 4 || d.N % 2 || d.rank < 0 || d.rank > d.Mr)
    return COLL_EINVAL;
  HostTables ht;
  const coll_status st = build_tables(d, &ht);
  if (st != COLL_OK) return st;
  *n_terms = ht.n_terms;
  *n_doubles = ht.tab.size();
  if (!out) return COLL_OK;
  if (cap < ht.tab.size()) return COLL_ENOMEM;
  std::memcpy(out, ht.tab.data(), ht.tab.size() * sizeof(double));
  return COLL_OK;
}

coll_status coll_debug_mixed_drop_commit(int32_t on) {
  return mixed_set_drop_commit(on) == 0 ? COLL_OK : COLL_ECUDA;
}

coll_status coll_plan_destroy(coll_plan p) {
  if (!p) return COLL_EINVAL;
  cudaFree(p->tab_dev);
  cudaFree(p->status_dev);
  delete p;
  return COLL_OK;
}

coll_status coll_plan_terms(coll_plan p, int32_t* n_terms) {
  if (!p || !n_terms) return COLL_EINVAL;
  *n_terms = p->n_terms;
  return COLL_OK;
}

coll_status coll_workspace_size(coll_plan p, int64_t max_cells, size_t* bytes) {
  if (!p || !bytes || max_cells < 0) return COLL_EINVAL;
  *bytes = max_cells == 0 ? 0 : ws_need(p, max_cells);
  return COLL_OK;
}

coll_status coll_eval_batch(coll_plan p, const void* f, void* Q, int64_t n_cells, void* ws, size_t ws_bytes,
                            coll_stream stream) {
  if (!p || n_cells < 0) return COLL_EINVAL;
  if (n_cells == 0) return COLL_OK;
  if (!f || !Q || f == Q) return COLL_EINVAL;
  return eval_variant(p, p->variant, f, Q, n_cells, ws, ws_bytes, stream);
}

coll_status coll_plan_autotune(coll_plan p, const void* f, void* Q, int64_t n_cells, void* ws, size_t ws_bytes,
                               coll_stream stream, int32_t* chosen) {
  if (!p || n_cells <= 0 || !f || !Q || f == Q) return COLL_EINVAL;
  if (p->galerkin) return COLL_EUNSUPPORTED;
  if (ws_bytes < ws_need(p, n_cells)) return COLL_ENOMEM;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return COLL_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return COLL_ECUDA; }
  float best = -1.0f;
  int best_v = 0;
  coll_status rc = COLL_OK;
  for (int v = 0; v < kVariants && rc == COLL_OK; ++v) {
    rc = eval_variant(p, v, f, Q, n_cells, ws, ws_bytes, stream);         // warm-up
    if (rc != COLL_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && rc == COLL_OK; ++r) rc = eval_variant(p, v, f, Q, n_cells, ws, ws_bytes, stream);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) { rc = COLL_ECUDA; break; }
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.0f || ms < best) { best = ms; best_v = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != COLL_OK) return rc;
  p->variant = best_v;
  if (chosen) *chosen = best_v;
  return COLL_OK;
}

coll_status coll_plan_set_variant(coll_plan p, int32_t variant) {
  if (!p || variant < 0 || variant >= kVariants) return COLL_EINVAL;
  p->variant = variant;
  return COLL_OK;
}

coll_status moments_realizability(const void* f, int32_t io_dtype, int32_t N, double L, int64_t n_cells,
                                  double eta0, double delta0, coll_moments* mom_out, uint8_t* mask_out,
                                  coll_stream stream) {
  if (n_cells < 0 || (io_dtype != 0 && io_dtype != 1) || !(L > 0) || !std::isfinite(L)) return COLL_EINVAL;
  if (!(N >= 2 && N <= 64 && N % 2 == 0)) return COLL_EINVAL;
  if (!(eta0 >= 0) || !(delta0 >= 0)) return COLL_EINVAL;
  if (n_cells == 0) return COLL_OK;
  if (!f || !mom_out || !mask_out) return COLL_EINVAL;
  const int e = launch_moments(f, io_dtype == 0, N, L, n_cells, eta0, delta0, mom_out, mask_out, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

coll_status coll_conservation(const void* Q, int32_t io_dtype, int32_t N, double L, int64_t n_cells, double* out,
                              coll_stream stream) {
  if (n_cells < 0 || (io_dtype != 0 && io_dtype != 1) || !(L > 0) || !std::isfinite(L)) return COLL_EINVAL;
  if (N != 16 && N != 24 && N != 32 && N != 48 && N != 64) return COLL_EUNSUPPORTED;
  if (n_cells == 0) return COLL_OK;
  if (!Q || !out || (reinterpret_cast<uintptr_t>(Q) & 15u) != 0 || (reinterpret_cast<uintptr_t>(out) & 7u) != 0)
    return COLL_EINVAL;
  const int e = launch_conservation(Q, io_dtype == 0, N, L, n_cells, out, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

coll_status regime_update(const double* fields, const double* l1, const uint8_t* r_in, int32_t nx, int32_t ny,
                          const coll_regime_params* params, uint8_t* r_out, double* ind, coll_stream stream) {
  if (nx < 0 || ny < 0 || !params) return COLL_EINVAL;
  const coll_regime_params& p = *params;
  if (!(p.dx > 0) || !(p.dy > 0) || !std::isfinite(p.dx) || !std::isfinite(p.dy) || !(p.eta0 >= 0) ||
      !(p.eta1 >= 0) || !(p.delta0 >= 0) || !std::isfinite(p.eps) || !std::isfinite(p.mu0) ||
      !std::isfinite(p.kappa0))
    return COLL_EINVAL;
  if (nx == 0 || ny == 0) return COLL_OK;
  if (!fields || !l1 || !r_in || !r_out) return COLL_EINVAL;
  count_launches(1);
  const int e = launch_regime(fields, l1, r_in, nx, ny, p, r_out, ind, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

coll_status coll_imex_stage(int32_t stage, const void* f, const void* Y, const void* Q1, const void* Q2,
                            const void* tr, const coll_moments* mom0, const coll_moments* mom1, int32_t io_dtype,
                            int32_t N, double L, int64_t n_cells, double dt, double eps, void* out,
                            coll_stream stream) {
  if (stage < COLL_IMEX_FIRST_ORDER || stage > COLL_IMEX_PR_FINAL || n_cells < 0) return COLL_EINVAL;
  if ((io_dtype != 0 && io_dtype != 1) || !(N >= 2 && N <= 64 && N % 2 == 0)) return COLL_EINVAL;
  if (N != 16 && N != 24 && N != 32 && N != 48 && N != 64) return COLL_EUNSUPPORTED;
  if (!(eps > 0) || !std::isfinite(eps) || !(dt >= 0) || !std::isfinite(dt) || !(L > 0) || !std::isfinite(L))
    return COLL_EINVAL;
  if (n_cells == 0) return COLL_OK;
  if (!f || !out) return COLL_EINVAL;
  switch (stage) {
    case COLL_IMEX_FIRST_ORDER:
      if (!Q1 || !mom0 || (tr && !mom1)) return COLL_EINVAL;
      break;
    case COLL_IMEX_PR_Y1:
      if (!mom0) return COLL_EINVAL;
      break;
    case COLL_IMEX_PR_Y2:
      if (!Y || !Q1 || !mom0) return COLL_EINVAL;
      break;
    default:
      if (!Q1 || !Q2) return COLL_EINVAL;
  }
  count_launches(1);
  const int e = launch_imex(stage, f, Y, Q1, Q2, stage == COLL_IMEX_FIRST_ORDER ? tr : nullptr, mom0, mom1,
                            io_dtype == 0, N, L, n_cells, dt, eps, out, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

coll_status coll_esbgk_step(const void* f, const coll_moments* mom, int32_t io_dtype, int32_t N, double L,
                            int64_t n_cells, double dt, double eps, double beta, double mu0, void* out,
                            coll_stream stream) {
  if (n_cells < 0 || (io_dtype != 0 && io_dtype != 1)) return COLL_EINVAL;
  if (!(N >= 2 && N <= 64 && N % 2 == 0)) return COLL_EINVAL;
  if (N != 16 && N != 24 && N != 32 && N != 48 && N != 64) return COLL_EUNSUPPORTED;
  if (!(eps > 0) || !std::isfinite(eps) || !(dt >= 0) || !std::isfinite(dt) || !(beta < 1) || !std::isfinite(beta) ||
      !(mu0 > 0) || !std::isfinite(mu0) || !(L > 0) || !std::isfinite(L))
    return COLL_EINVAL;
  if (n_cells == 0) return COLL_OK;
  if (!f || !mom || !out) return COLL_EINVAL;
  count_launches(1);
  const int e = launch_esbgk(f, mom, io_dtype == 0, N, L, n_cells, dt, eps, beta, mu0, out, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

coll_status coll_device_status(coll_plan p) {
  if (!p) return COLL_EINVAL;
  int v = 0;
  if (cudaMemcpy(&v, p->status_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return COLL_ECUDA;
  if (v & kStatusTimeout) return COLL_ETIMEOUT;
  if (v & kStatusNonFinite) return COLL_ENONFINITE;
  return COLL_OK;
}

coll_status coll_device_status_clear(coll_plan p) {
  if (!p) return COLL_EINVAL;
  return cudaMemset(p->status_dev, 0, sizeof(int)) == cudaSuccess ? COLL_OK : COLL_ECUDA;
}

coll_status coll_ragged_workspace_size(const coll_cell_group* groups, const int64_t* cells_per_group,
                                       int32_t n_groups, size_t* bytes) {
  if (!bytes) return COLL_EINVAL;
  RaggedTable t;
  int ctype = 0, grid = 0;
  size_t wsper = 0, total = 0;
  const coll_status st = ragged_prepare(groups, cells_per_group, n_groups, &t, &ctype, &grid, &wsper, &total);
  if (st != COLL_OK) return st;
  *bytes = total;
  return COLL_OK;
}

coll_status coll_eval_ragged(const coll_cell_group* groups, const int64_t* cells_per_group, int32_t n_groups,
                             void* ws, size_t ws_bytes, coll_stream stream) {
  RaggedTable t;
  int ctype = 0, grid = 0;
  size_t wsper = 0, total = 0;
  const coll_status st = ragged_prepare(groups, cells_per_group, n_groups, &t, &ctype, &grid, &wsper, &total);
  if (st != COLL_OK) return st;
  if (t.total_units == 0) return COLL_OK;
  if (!ws || !aligned256(ws)) return COLL_EINVAL;
  if (ws_bytes < total) return COLL_ENOMEM;
  if (cudaMemsetAsync(ws, 0, 256, static_cast<cudaStream_t>(stream)) != cudaSuccess) return COLL_ECUDA;
  const int e = launch_ragged(ctype, t, ws, wsper, grid, stream);
  return e == 0 ? COLL_OK : COLL_ECUDA;
}

}  // extern "C"
