// Host-side construction of the plan tables (arxiv 2505.03360, sec. 4.4.1).
//
// For every term t of the separated Carleman kernel the table holds, on the
// half spectrum k0, k1 in FFT order and 0 <= k2 < N/2,
//   A_t(k) = c_t alpha_t(xi_k) / (sigma_t N^3),   B_t(k) = sigma_t alpha'_t(xi_k) / N^3,
// and the last term is the loss: A = -Lambda / (sigma N^3), B = sigma / N^3, with
// sigma_t a power of two that balances the sizes of A_t and B_t, and
// Lambda = sum_t c_t alpha_t alpha'_t accumulated here in FP64.  Every mode
// with k0 = -N/2 or k1 = -N/2 is zero (k2 = N/2 is not stored).
//
// Multipliers (x = rho e, y in the disk of radius R in the plane e-perp):
//   alpha_{p,i}(xi)  = 2 W_i rho_i cos(rho_i xi . e_p)
//   alpha'_{p,i}(xi) = Psi_{rho_i}(|xi - (xi . e_p) e_p|)
//   Psi_rho(s) = 2 pi int_0^R r (rho^2 + r^2)^{(lambda-1)/2} J0(r s) dr
//   c_p = 4 b0 w_p
// lambda = 1: Psi = 2 pi R J1(R s) / s, one term per direction with
// alpha_p = sum_i alpha_{p,i}.  lambda != 1: Psi_{rho_i} is interpolated in s
// by piecewise Chebyshev series (unit panels, degree 47) whose samples come
// from composite Gauss-Legendre quadrature in r, graded near r = 0; with a
// rank r > 0 the Mr node terms of a direction are replaced by r combinations
// of them (RadialFactors, the low-rank separable form of the radial kernel).
//
// Quadrature nodes are computed here by Newton iteration on the Legendre
// recurrence in long double.
#include <cmath>
#include <thread>
#include <vector>

#include "coll_internal.h"

namespace coll {

namespace {

const long double kPiL = 3.141592653589793238462643383279502884L;

// n-point Gauss-Legendre rule on [-1, 1]
void gauss_legendre(int n, std::vector<double>* x, std::vector<double>* w) {
  x->assign(n, 0.0);
  w->assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    long double z = cosl(kPiL * (i + 0.75L) / (n + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1; }
      dp = n * (z * p1 - p0) / (z * z - 1);
      long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    long double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1);
    long double wt = 2 / ((1 - z * z) * dp * dp);
    (*x)[i] = double(-z);
    (*x)[n - 1 - i] = double(z);
    (*w)[i] = double(wt);
    (*w)[n - 1 - i] = double(wt);
  }
  if (n % 2 == 1) (*x)[n / 2] = 0.0;
}

struct Dir {
  double e[3];
  double w;
};

bool hemisphere(int M, int Mtheta, int rule, std::vector<Dir>* out) {
  out->clear();
  if (rule == 0) {
    if (Mtheta <= 0 || Mtheta % 2 || M % Mtheta) return false;
    const int Mphi = M / Mtheta;
    if (Mphi % 2) return false;
    std::vector<double> mu, wm;
    gauss_legendre(Mtheta, &mu, &wm);
    for (int j = 0; j < Mtheta; ++j) {
      if (!(mu[j] > 0)) continue;
      const long double st = sqrtl(1.0L - (long double)mu[j] * mu[j]);
      for (int q = 0; q < Mphi; ++q) {
        const long double ph = (q + 0.5L) * 2 * kPiL / Mphi;
        Dir d;
        d.e[0] = double(st * cosl(ph));
        d.e[1] = double(st * sinl(ph));
        d.e[2] = mu[j];
        d.w = double((long double)wm[j] * 2 * kPiL / Mphi);
        out->push_back(d);
      }
    }
    return true;
  }
  if (rule == 1) {
    const int A1 = Mtheta;
    if (A1 <= 0 || M % (2 * A1)) return false;
    const int A2 = M / (2 * A1);
    for (int p = 0; p < A1; ++p) {
      const long double th = (p + 0.5L) * kPiL / A1;
      for (int q = 0; q < A2; ++q) {
        const long double ph = (q + 0.5L) * kPiL / A2;
        Dir d;
        d.e[0] = double(sinl(th) * cosl(ph));
        d.e[1] = double(sinl(th) * sinl(ph));
        d.e[2] = double(cosl(th));
        d.w = double((kPiL / A1) * (kPiL / A2) * sinl(th));
        out->push_back(d);
      }
    }
    return true;
  }
  return false;
}

// composite GL nodes on [0, R]: [0, a], then doubling panels up to width 0.5,
// then panels of width <= 0.5, 16 nodes each
void radial_panels(double a0, double R, std::vector<double>* r, std::vector<double>* w) {
  std::vector<double> edges{0.0};
  double a = std::min(a0, R);
  edges.push_back(a);
  while (a < R && a < 0.5) { a = std::min(2 * a, R); edges.push_back(a); }
  while (a < R) { a = std::min(a + 0.5, R); edges.push_back(a); }
  std::vector<double> x, wx;
  gauss_legendre(16, &x, &wx);
  r->clear();
  w->clear();
  for (size_t k = 0; k + 1 < edges.size(); ++k) {
    const double lo = edges[k], hi = edges[k + 1];
    if (!(hi > lo)) continue;
    for (int j = 0; j < 16; ++j) {
      r->push_back(0.5 * (hi - lo) * x[j] + 0.5 * (hi + lo));
      w->push_back(0.5 * (hi - lo) * wx[j]);
    }
  }
}

// Psi_rho(s) for all radial nodes rho_i by piecewise Chebyshev interpolation
struct PsiCheb {
  static constexpr int kDeg = 47;
  double width = 1.0;
  int n_panels = 0, Mr = 0;
  std::vector<double> coef;   // [panel][i][kDeg+1]

  void build(const std::vector<double>& rho, double R, double lam, double s_max) {
    Mr = int(rho.size());
    n_panels = int(std::floor(s_max / width)) + 1;
    double rmin = rho[0];
    for (double v : rho) rmin = std::min(rmin, v);
    std::vector<double> r, w;
    radial_panels(rmin, R, &r, &w);
    const int n = kDeg + 1;
    std::vector<double> th(n), xs(n);
    for (int j = 0; j < n; ++j) {
      th[j] = double(kPiL * (j + 0.5L) / n);
      xs[j] = std::cos(th[j]);
    }
    // kernel weights g[node][i]
    std::vector<double> g(r.size() * Mr);
    for (size_t k = 0; k < r.size(); ++k)
      for (int i = 0; i < Mr; ++i)
        g[k * Mr + i] = 2.0 * double(kPiL) * w[k] * r[k] * std::pow(rho[i] * rho[i] + r[k] * r[k], 0.5 * (lam - 1.0));
    coef.assign(size_t(n_panels) * Mr * n, 0.0);
    std::vector<double> vals(size_t(n) * Mr);
    for (int pnl = 0; pnl < n_panels; ++pnl) {
      const double lo = pnl * width;
      for (int j = 0; j < n; ++j) {
        const double s = lo + 0.5 * width * (xs[j] + 1.0);
        for (int i = 0; i < Mr; ++i) vals[size_t(j) * Mr + i] = 0.0;
        for (size_t k = 0; k < r.size(); ++k) {
          const double J = std::cyl_bessel_j(0.0, r[k] * s);
          for (int i = 0; i < Mr; ++i) vals[size_t(j) * Mr + i] += g[k * Mr + i] * J;
        }
      }
      // c_m = (2/n) sum_j f_j cos(m theta_j), c_0 halved
      for (int i = 0; i < Mr; ++i)
        for (int m = 0; m < n; ++m) {
          long double acc = 0;
          for (int j = 0; j < n; ++j) acc += (long double)vals[size_t(j) * Mr + i] * cosl((long double)m * th[j]);
          double c = double(2.0L * acc / n);
          if (m == 0) c *= 0.5;
          coef[(size_t(pnl) * Mr + i) * n + m] = c;
        }
    }
  }

  double eval(int i, double s) const {
    int pnl = int(std::floor(s / width));
    if (pnl >= n_panels) pnl = n_panels - 1;
    const double lo = pnl * width;
    const double t = 2.0 * (s - lo) / width - 1.0;
    const double* c = &coef[(size_t(pnl) * Mr + i) * (kDeg + 1)];
    double b1 = 0, b2 = 0;
    for (int m = kDeg; m >= 1; --m) {
      const double b0 = c[m] + 2.0 * t * b1 - b2;
      b2 = b1;
      b1 = b0;
    }
    return c[0] + t * b1 - b2;
  }
};

// Low-rank separable form of the radial sum (lambda != 1, rank r): per
// direction the Mr node terms give sum_i a_i cos(rho_i t) Psi_{rho_i}(s),
// a_i = 2 W_i rho_i, Psi_rho(s) = int_0^R g_rho(r) J0(r s) dr,
// g_rho(r) = 2 pi r (rho^2 + r^2)^((lambda-1)/2).  With U the eigenvectors of
// the Gram matrix G_ii' = a_i a_i' int_0^R g_i g_i' dr (largest eigenvalues
// first, e_q) and s_q = sqrt(e_q), term q is
//   alpha_q = sum_i P[q][i] a_i cos(rho_i t),  P[q][i] = sqrt(s_q) U_iq / a_i
//   alpha'_q = sum_i Rm[q][i] Psi_{rho_i}(s),  Rm[q][i] = U_iq a_i / sqrt(s_q)
// so that sum_q alpha_q alpha'_q = c^T U_r U_r^T diag(a) Psi (exact for r = Mr).
// U and s_q are the left singular vectors and singular values of the factor
// Y_ik = a_i g_i(r_k) sqrt(w_k) (G = Y Y^T) on the composite Gauss-Legendre
// rule of PsiCheb, by one-sided Jacobi rotations in long double: the
// subspace of the r largest is accurate to rounding over s_r - s_{r+1}.
struct RadialFactors {
  int rank = 0, Mr = 0;
  std::vector<double> P, Rm;   // [rank][Mr]

  void build(const std::vector<double>& rho, const std::vector<double>& W, double R, double lam, int r_keep) {
    Mr = int(rho.size());
    rank = r_keep;
    double rmin = rho[0];
    for (double v : rho) rmin = std::min(rmin, v);
    std::vector<double> r, w;
    radial_panels(rmin, R, &r, &w);
    // Y_ik = a_i g_i(r_k) sqrt(w_k), so that Y Y^T = G; one-sided Jacobi
    // rotations of the rows of Y until they are orthogonal: Y = U diag(s) V^T
    // with U the accumulated rotations and s the final row norms (the
    // eigenvectors of G without squaring its condition number)
    const size_t nr = r.size();
    std::vector<long double> a(Mr), Y(size_t(Mr) * nr), U(size_t(Mr) * Mr, 0.0L);
    for (int i = 0; i < Mr; ++i) a[i] = 2.0L * W[i] * rho[i];
    for (int i = 0; i < Mr; ++i)
      for (size_t k = 0; k < nr; ++k)
        Y[size_t(i) * nr + k] = a[i] * 2.0L * kPiL * r[k] *
                                powl((long double)rho[i] * rho[i] + (long double)r[k] * r[k],
                                     0.5L * ((long double)lam - 1.0L)) *
                                sqrtl((long double)w[k]);
    for (int i = 0; i < Mr; ++i) U[size_t(i) * Mr + i] = 1.0L;
    for (int sweep = 0; sweep < 60; ++sweep) {
      bool rotated = false;
      for (int p = 0; p < Mr; ++p)
        for (int q = p + 1; q < Mr; ++q) {
          long double al = 0.0L, be = 0.0L, ga = 0.0L;
          for (size_t k = 0; k < nr; ++k) {
            const long double yp = Y[size_t(p) * nr + k], yq = Y[size_t(q) * nr + k];
            al += yp * yp;
            be += yq * yq;
            ga += yp * yq;
          }
          if (fabsl(ga) <= 1e-19L * sqrtl(al * be)) continue;
          rotated = true;
          const long double zeta = (be - al) / (2.0L * ga);
          const long double t = (zeta >= 0 ? 1.0L : -1.0L) / (fabsl(zeta) + sqrtl(1.0L + zeta * zeta));
          const long double c = 1.0L / sqrtl(1.0L + t * t), sn = c * t;
          for (size_t k = 0; k < nr; ++k) {
            const long double yp = Y[size_t(p) * nr + k], yq = Y[size_t(q) * nr + k];
            Y[size_t(p) * nr + k] = c * yp - sn * yq;
            Y[size_t(q) * nr + k] = sn * yp + c * yq;
          }
          for (int k = 0; k < Mr; ++k) {
            const long double up = U[size_t(k) * Mr + p], uq = U[size_t(k) * Mr + q];
            U[size_t(k) * Mr + p] = c * up - sn * uq;
            U[size_t(k) * Mr + q] = sn * up + c * uq;
          }
        }
      if (!rotated) break;
    }
    std::vector<long double> sv(Mr, 0.0L);
    for (int i = 0; i < Mr; ++i) {
      long double acc = 0.0L;
      for (size_t k = 0; k < nr; ++k) acc += Y[size_t(i) * nr + k] * Y[size_t(i) * nr + k];
      sv[i] = sqrtl(acc);
    }
    std::vector<int> order(Mr);
    for (int i = 0; i < Mr; ++i) order[i] = i;
    for (int i = 1; i < Mr; ++i)                  // singular values descending
      for (int j = i; j > 0 && sv[order[j]] > sv[order[j - 1]]; --j) std::swap(order[j], order[j - 1]);
    P.assign(size_t(rank) * Mr, 0.0);
    Rm.assign(size_t(rank) * Mr, 0.0);
    for (int q = 0; q < rank; ++q) {
      const int col = order[q];
      const long double sq = sqrtl(sv[col]);
      for (int i = 0; i < Mr; ++i) {
        const long double u = U[size_t(i) * Mr + col];
        P[size_t(q) * Mr + i] = double(sq * u / a[i]);
        Rm[size_t(q) * Mr + i] = double(u * a[i] / sq);
      }
    }
  }
};

double psi_hs(double s, double R) {
  if (s * R < 1e-8) return double(kPiL) * R * R;
  return 2.0 * double(kPiL) * R * std::cyl_bessel_j(1.0, R * s) / s;
}

}  // namespace

coll_status build_tables(const coll_plan_desc& d, HostTables* out, int mode_cut) {
  const int N = d.N, H = N / 2;
  const double S = d.S > 0 ? d.S : 2.0 * d.L / (3.0 + std::sqrt(2.0));
  const double R = 2.0 * S;
  const double lam = d.lambda;
  const double b0 = d.b0 > 0 ? d.b0 : (lam == 0.0 ? 1.0 / (4.0 * double(kPiL)) : 1.0);
  std::vector<Dir> dirs;
  if (!hemisphere(d.M, d.Mtheta, d.sphere_rule, &dirs) || dirs.empty()) return COLL_EINVAL;
  std::vector<double> xr, wr;
  gauss_legendre(d.Mr, &xr, &wr);
  std::vector<double> rho(d.Mr), W(d.Mr);
  for (int i = 0; i < d.Mr; ++i) {
    rho[i] = 0.5 * R * (xr[i] + 1.0);
    W[i] = 0.5 * R * wr[i];
  }
  const bool hs = (lam == 1.0);
  const bool lowrank = !hs && d.rank > 0;
  const int per_dir = hs ? 1 : (lowrank ? d.rank : d.Mr);
  const int n_terms = int(dirs.size()) * per_dir + 1;
  const size_t plane = size_t(N) * N * H;
  out->n_terms = n_terms;
  out->tab.assign(size_t(n_terms) * plane * 2, 0.0);
  const double n3 = double(N) * N * N;
  const double dk = double(kPiL) / d.L;
  auto kval = [N](int idx) { return idx < N / 2 ? idx : idx - N; };
  // modes kept: every |k_d| < N / 2, or < mode_cut / 2 on a padded grid
  const int kcut = mode_cut > 0 ? mode_cut / 2 : N / 2;
  auto kept = [&](int i0, int i1, int i2) {
    const int a = kval(i0), b = kval(i1);
    return (a < 0 ? -a : a) < kcut && (b < 0 ? -b : b) < kcut && i2 < kcut;
  };

  PsiCheb cheb;
  RadialFactors rf;
  if (!hs) {
    const double kmax = dk * (N / 2);
    cheb.build(rho, R, lam, std::sqrt(3.0) * kmax + 1e-9);
    if (lowrank) rf.build(rho, W, R, lam, d.rank);
  }
  std::vector<double> Lam(plane, 0.0);

  auto work = [&](int p) {
    const Dir& dr = dirs[p];
    const double cp = 4.0 * b0 * dr.w;
    for (int i0 = 0; i0 < N; ++i0) {
      for (int i1 = 0; i1 < N; ++i1) {
        for (int i2 = 0; i2 < H; ++i2) {
          const size_t idx = (size_t(i0) * N + i1) * H + i2;
          if (i0 == N / 2 || i1 == N / 2 || !kept(i0, i1, i2)) continue;
          const double x0 = dk * kval(i0), x1 = dk * kval(i1), x2 = dk * i2;
          const double proj = x0 * dr.e[0] + x1 * dr.e[1] + x2 * dr.e[2];
          const double p0 = x0 - proj * dr.e[0], p1 = x1 - proj * dr.e[1], p2 = x2 - proj * dr.e[2];
          const double s = std::sqrt(p0 * p0 + p1 * p1 + p2 * p2);
          if (hs) {
            double a = 0.0;
            for (int i = 0; i < d.Mr; ++i) a += 2.0 * W[i] * rho[i] * std::cos(rho[i] * proj);
            const double b = psi_hs(s, R);
            double* t = &out->tab[(size_t(p) * plane + idx) * 2];
            t[0] = cp * a;
            t[1] = b;
          } else if (!lowrank) {
            for (int i = 0; i < d.Mr; ++i) {
              const double a = 2.0 * W[i] * rho[i] * std::cos(rho[i] * proj);
              const double b = cheb.eval(i, s);
              double* t = &out->tab[((size_t(p) * per_dir + i) * plane + idx) * 2];
              t[0] = cp * a;
              t[1] = b;
            }
          } else {
            double av[256], bv[256];
            for (int i = 0; i < d.Mr; ++i) {
              av[i] = 2.0 * W[i] * rho[i] * std::cos(rho[i] * proj);
              bv[i] = cheb.eval(i, s);
            }
            for (int q = 0; q < d.rank; ++q) {
              double a = 0.0, b = 0.0;
              for (int i = 0; i < d.Mr; ++i) {
                a += rf.P[size_t(q) * d.Mr + i] * av[i];
                b += rf.Rm[size_t(q) * d.Mr + i] * bv[i];
              }
              double* t = &out->tab[((size_t(p) * per_dir + q) * plane + idx) * 2];
              t[0] = cp * a;
              t[1] = b;
            }
          }
        }
      }
    }
  };
  const int nd = int(dirs.size());
  unsigned hw = std::thread::hardware_concurrency();
  int nthr = int(hw ? std::min<unsigned>(hw, 16u) : 4u);
  if (size_t(nd) * plane * per_dir < (1u << 18)) nthr = 1;
  std::vector<std::thread> pool;
  for (int tix = 0; tix < nthr; ++tix)
    pool.emplace_back([&, tix]() {
      for (int p = tix; p < nd; p += nthr) work(p);
    });
  for (auto& th : pool) th.join();

  // loss multiplier, summed in term order (unscaled values)
  for (int t = 0; t + 1 < n_terms; ++t) {
    const double* tt = &out->tab[size_t(t) * plane * 2];
    for (size_t idx = 0; idx < plane; ++idx) Lam[idx] += tt[2 * idx] * tt[2 * idx + 1];
  }
  double* last = &out->tab[size_t(n_terms - 1) * plane * 2];
  for (int i0 = 0; i0 < N; ++i0)
    for (int i1 = 0; i1 < N; ++i1)
      for (int i2 = 0; i2 < H; ++i2) {
        const size_t idx = (size_t(i0) * N + i1) * H + i2;
        if (i0 == N / 2 || i1 == N / 2 || !kept(i0, i1, i2)) continue;
        last[2 * idx] = -Lam[idx];
        last[2 * idx + 1] = 1.0;
      }
  // Balance each term: the kernel packs the two real inverse transforms of a
  // term into one complex transform, whose rounding error is relative to the
  // larger of the two; scaling A by 1/sigma and B by sigma (sigma a power of
  // two, so exact) leaves the product unchanged and equalises their sizes.
  // Then apply the 1/N^3 normalisation of the forward DFT.
  for (int t = 0; t < n_terms; ++t) {
    double* tt = &out->tab[size_t(t) * plane * 2];
    double ma = 0.0, mb = 0.0;
    for (size_t idx = 0; idx < plane; ++idx) {
      ma = std::max(ma, std::fabs(tt[2 * idx]));
      mb = std::max(mb, std::fabs(tt[2 * idx + 1]));
    }
    double sigma = 1.0;
    if (ma > 0 && mb > 0) sigma = std::ldexp(1.0, int(std::lround(0.5 * std::log2(ma / mb))));
    for (size_t idx = 0; idx < plane; ++idx) {
      tt[2 * idx] = tt[2 * idx] / sigma / n3;
      tt[2 * idx + 1] = tt[2 * idx + 1] * sigma / n3;
    }
  }
  return COLL_OK;
}

}  // namespace coll
