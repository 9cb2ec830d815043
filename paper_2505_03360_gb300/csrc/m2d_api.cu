// extern "C" entry points of the 2D Maxwell-molecule operator (include/coll.h,
// coll_m2d_*) and its host table builder (sec. 4.4.1, "The 2d case").
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "coll_internal.h"
#include "../../include/coll_debug.h"

namespace coll {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

bool m2d_valid(const coll_m2d_plan_desc& d) {
  return d.L > 0 && std::isfinite(d.L) && d.S >= 0 && std::isfinite(d.S) && std::isfinite(d.b0) && d.A >= 1 &&
         d.A <= 4096 && (d.io_dtype == 0 || d.io_dtype == 1) && d.N >= 4 && d.N % 2 == 0 && d.N <= 256;
}

int m2d_ctype(int prec) {
  return prec == COLL_F64 ? kCF64 : prec == COLL_F32 ? kCF32 : prec == COLL_F32X2 ? kCDF : -1;
}

bool m2d_has_kernel(int N, int ctype) {
  if (ctype == kCF32) return N == 16 || N == 32 || N == 64;
  return (ctype == kCF64 || ctype == kCDF) && (N == 16 || N == 32);
}

// 2R sinc(R s): the integral of exp(i rho s) over rho in [-R, R]
double phi(double s, double R) {
  const double x = R * s;
  return x == 0.0 ? 2.0 * R : 2.0 * R * std::sin(x) / x;
}

int launch(int ctype, int N, bool io_f64, const M2Args& a, int grid, void* stream) {
  switch (ctype) {
    case kCF64: return m2d_launch_f64(N, io_f64, a, grid, stream);
    case kCF32: return m2d_launch_f32(N, io_f64, a, grid, stream);
    default: return m2d_launch_df(N, io_f64, a, grid, stream);
  }
}

int occupancy(int ctype, int N, bool io_f64, int* ctas) {
  switch (ctype) {
    case kCF64: return m2d_occupancy_f64(N, io_f64, ctas);
    case kCF32: return m2d_occupancy_f32(N, io_f64, ctas);
    default: return m2d_occupancy_df(N, io_f64, ctas);
  }
}

}  // namespace

coll_status build_m2d_tables(const coll_m2d_plan_desc& d, int* n_terms, std::vector<double>* tab) {
  const int N = d.N, H = N / 2, A = d.A;
  const double S = d.S > 0 ? d.S : 2.0 * d.L / (3.0 + std::sqrt(2.0));
  const double R = 2.0 * S;
  const double b0 = d.b0 > 0 ? d.b0 : 1.0 / (2.0 * kPi);
  const double c = 2.0 * b0 * kPi / A;               // Bt pi / A, Bt = 2 b0
  const double inv = 1.0 / (double(N) * N);
  const double h = kPi / d.L;
  *n_terms = A + 1;
  tab->assign(size_t(A + 1) * N * H * 2, 0.0);
  std::vector<double> lam(size_t(N) * H, 0.0);
  for (int p = 1; p <= A; ++p) {
    const double th = kPi * p / A, ct = std::cos(th), st = std::sin(th);
    double* tp = tab->data() + size_t(p - 1) * N * H * 2;
    for (int k0 = 0; k0 < N; ++k0) {
      if (k0 == H) continue;                           // Nyquist row: dropped
      const double x0 = h * (k0 < H ? k0 : k0 - N);
      for (int k1 = 0; k1 < H; ++k1) {
        const double x1 = h * k1;
        const double a = phi(x0 * ct + x1 * st, R), b = phi(-x0 * st + x1 * ct, R);
        const size_t i = size_t(k0) * H + k1;
        tp[2 * i] = c * a * inv;
        tp[2 * i + 1] = b * inv;
        lam[i] += c * a * b;
      }
    }
  }
  double* tl = tab->data() + size_t(A) * N * H * 2;
  for (int k0 = 0; k0 < N; ++k0) {
    if (k0 == H) continue;
    for (int k1 = 0; k1 < H; ++k1) {
      const size_t i = size_t(k0) * H + k1;
      tl[2 * i] = -lam[i] * inv;
      tl[2 * i + 1] = inv;
    }
  }
  return COLL_OK;
}

}  // namespace coll

using namespace coll;

extern "C" {

coll_status coll_m2d_tables_host(const coll_m2d_plan_desc* desc, double* out, size_t cap, int32_t* n_terms,
                                 size_t* n_doubles) {
  if (!desc || !n_terms || !n_doubles || !m2d_valid(*desc)) return COLL_EINVAL;
  int nt = 0;
  std::vector<double> tab;
  const coll_status st = build_m2d_tables(*desc, &nt, &tab);
  if (st != COLL_OK) return st;
  *n_terms = nt;
  *n_doubles = tab.size();
  if (!out) return COLL_OK;
  if (cap < tab.size()) return COLL_ENOMEM;
  std::memcpy(out, tab.data(), tab.size() * sizeof(double));
  return COLL_OK;
}

coll_status coll_m2d_plan_create(const coll_m2d_plan_desc* desc, coll_m2d_plan* out) {
  if (!desc || !out || !m2d_valid(*desc)) return COLL_EINVAL;
  const coll_m2d_plan_desc d = *desc;
  const int ctype = m2d_ctype(d.prec);
  if (ctype < 0) return d.prec >= COLL_F64 && d.prec <= COLL_MIXED_SLICED ? COLL_EUNSUPPORTED : COLL_EINVAL;
  if (!m2d_has_kernel(d.N, ctype)) return COLL_EUNSUPPORTED;
  int nt = 0;
  std::vector<double> tab;
  coll_status st = build_m2d_tables(d, &nt, &tab);
  if (st != COLL_OK) return st;
  coll_m2d_plan_s* p = new (std::nothrow) coll_m2d_plan_s();
  if (!p) return COLL_ENOMEM;
  p->d = d;
  p->ctype = ctype;
  p->io_f64 = d.io_dtype == 0;
  p->n_terms = nt;
  if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return COLL_ECUDA; }
  cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
  if (occupancy(ctype, d.N, p->io_f64, &p->ctas_per_sm) != 0 || p->ctas_per_sm < 1) { delete p; return COLL_ECUDA; }
  const size_t n = tab.size();
  cudaError_t e;
  if (ctype == kCF64) {
    p->tab_bytes = n * sizeof(double);
    e = cudaMalloc(&p->tab_dev, p->tab_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(p->tab_dev, tab.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  } else if (ctype == kCF32) {
    std::vector<float> tf(n);
    for (size_t i = 0; i < n; ++i) tf[i] = float(tab[i]);
    p->tab_bytes = n * sizeof(float);
    e = cudaMalloc(&p->tab_dev, p->tab_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(p->tab_dev, tf.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  } else {
    std::vector<float> tf(2 * n);                      // float pairs (head, tail) per value
    for (size_t i = 0; i < n; ++i) {
      const float hd = float(tab[i]);
      tf[2 * i] = hd;
      tf[2 * i + 1] = float(tab[i] - double(hd));
    }
    p->tab_bytes = 2 * n * sizeof(float);
    e = cudaMalloc(&p->tab_dev, p->tab_bytes);
    if (e == cudaSuccess) e = cudaMemcpy(p->tab_dev, tf.data(), p->tab_bytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    cudaFree(p->tab_dev);
    delete p;
    return e == cudaErrorMemoryAllocation ? COLL_ENOMEM : COLL_ECUDA;
  }
  e = cudaMalloc(reinterpret_cast<void**>(&p->status_dev), sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->status_dev, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaFree(p->tab_dev);
    delete p;
    return COLL_ECUDA;
  }
  *out = p;
  return COLL_OK;
}

coll_status coll_m2d_plan_destroy(coll_m2d_plan p) {
  if (!p) return COLL_EINVAL;
  cudaFree(p->tab_dev);
  cudaFree(p->status_dev);
  delete p;
  return COLL_OK;
}

coll_status coll_m2d_eval_batch(coll_m2d_plan p, const void* f, void* Q, int64_t n_cells, coll_stream stream) {
  if (!p || n_cells < 0) return COLL_EINVAL;
  if (n_cells == 0) return COLL_OK;
  if (!f || !Q || f == Q) return COLL_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return COLL_EINVAL;
  long long grid = static_cast<long long>(p->num_sms) * p->ctas_per_sm;
  if (grid > n_cells) grid = n_cells;
  M2Args a;
  a.f = f;
  a.Q = Q;
  a.n_cells = n_cells;
  a.tab = p->tab_dev;
  a.n_terms = p->n_terms;
  a.status = p->status_dev;
  const int e = launch(p->ctype, p->d.N, p->io_f64, a, int(grid), stream);
  if (e != 0) return COLL_ECUDA;
  count_launches(1);
  return COLL_OK;
}

coll_status coll_m2d_device_status(coll_m2d_plan p) {
  if (!p) return COLL_EINVAL;
  int s = 0;
  if (cudaMemcpy(&s, p->status_dev, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return COLL_ECUDA;
  if (s & kStatusTimeout) return COLL_ETIMEOUT;
  if (s & kStatusNonFinite) return COLL_ENONFINITE;
  return COLL_OK;
}

coll_status coll_m2d_device_status_clear(coll_m2d_plan p) {
  if (!p) return COLL_EINVAL;
  return cudaMemset(p->status_dev, 0, sizeof(int)) == cudaSuccess ? COLL_OK : COLL_ECUDA;
}

}  // extern "C"
