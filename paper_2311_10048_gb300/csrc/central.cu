// Central-LMO share of E(T) in the Laplace form (arXiv 2311.10048, Sec. 3.7,
// eqs laplace_transform and local_pt): the augmented-domain builders and the
// quadrature of 1/x.
//
// With one quadrature point (s_q, w_q) the denominator 1/D of every element
// is replaced by -w_q exp(s_q D), and exp(s_q D) factorises into one factor
// exp(+e_p s_q / 2) per occupied index and exp(-e_x s_q / 2) per virtual one,
// squared.  W and V are linear in their first occupied index, so the barred
// W of a central orbital u = sum_i U_i phi_i is the W of a pseudo-orbital
// whose DF factors, amplitudes and T1 (and f_ov) rows are the combinations
// with coefficients c_i = U_i exp(e_i s_q / 2), with orbital energy 0 (its
// factor is in c), and whose exp(...) factors of the other five indices come
// from the element weight.  The pseudo-orbitals are appended after the real
// occupied orbitals of their spin; internal (summed) occupied indices run
// over the real ones only, and no triplet holds two pseudo-orbitals.
//
// Augmented orbital order of the spin carrying P pseudo-orbitals:
//   [ real occupied (o) | pseudo (P) | virtual (v) ],  n' = nbas + P.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace lno {

namespace {

inline int grid_of(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? (b < 1 ? 1 : b) : 152 * 32);
}

// coef[p][i] = U[p][i] exp(e_i s / 2)
__global__ void lmo_coef(const double* __restrict__ U, const double* __restrict__ eps, int P,
                         int o, double s, double* __restrict__ coef) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P * o;
       idx += gridDim.x * blockDim.x)
    coef[idx] = U[idx] * exp(eps[idx % o] * (0.5 * s));
}

// augmented index r -> real orbital (>= 0) or pseudo-orbital (-1 - p)
__device__ __forceinline__ int aug_orb(int r, int o, int P) {
  return r < o ? r : (r < o + P ? -1 - (r - o) : r - P);
}

// Baug[Q][r][c] of the spin with pseudo-orbitals
__global__ void aug_B(const double* __restrict__ B, int naux, int nbas, int o, int P,
                      const double* __restrict__ coef, double* __restrict__ Baug) {
  const int n2 = nbas + P;
  const int64_t total = (int64_t)naux * n2 * n2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(idx % n2);
    const int64_t t = idx / n2;
    const int r = (int)(t % n2);
    const int Q = (int)(t / n2);
    const int x = aug_orb(r, o, P), y = aug_orb(c, o, P);
    const double* BQ = B + (int64_t)Q * nbas * nbas;
    double v = 0.0;
    if (x >= 0 && y >= 0) {
      v = BQ[(int64_t)x * nbas + y];
    } else if (x < 0 && y >= 0) {
      const double* cp = coef + (int64_t)(-1 - x) * o;
      for (int i = 0; i < o; ++i) v += cp[i] * BQ[(int64_t)i * nbas + y];
    } else if (x >= 0 && y < 0) {
      const double* cp = coef + (int64_t)(-1 - y) * o;
      for (int i = 0; i < o; ++i) v += cp[i] * BQ[(int64_t)x * nbas + i];
    }
    Baug[idx] = v;
  }
}

// same-spin doubles [o+P][o+P][v][v]: a pseudo index p in either occupied
// slot is the combination of that slot's real rows; two pseudo indices: 0
__global__ void aug_t2ss(const double* __restrict__ t2, int o, int v, int P,
                         const double* __restrict__ coef, double* __restrict__ out) {
  const int n = o + P;
  const int64_t vv = (int64_t)v * v;
  const int64_t total = (int64_t)n * n * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ab = idx % vv;
    const int64_t t = idx / vv;
    const int j = (int)(t % n), i = (int)(t / n);
    double val = 0.0;
    if (i < o && j < o) {
      val = t2[((int64_t)i * o + j) * vv + ab];
    } else if (i >= o && j < o) {
      const double* cp = coef + (int64_t)(i - o) * o;
      for (int m = 0; m < o; ++m) val += cp[m] * t2[((int64_t)m * o + j) * vv + ab];
    } else if (i < o && j >= o) {
      const double* cp = coef + (int64_t)(j - o) * o;
      for (int m = 0; m < o; ++m) val += cp[m] * t2[((int64_t)i * o + m) * vv + ab];
    }
    out[idx] = val;
  }
}

// mixed doubles t2ab [na][nb][va][vb]: pseudo-orbitals on the spin-up index
// (side 0: [na+P][nb]) or on the spin-down index (side 1: [na][nb+P])
__global__ void aug_t2ab(const double* __restrict__ t2, int na, int nb, int va, int vb, int P,
                         int side, const double* __restrict__ coef, double* __restrict__ out) {
  const int n0 = side == 0 ? na + P : na, n1 = side == 0 ? nb : nb + P;
  const int64_t vv = (int64_t)va * vb;
  const int64_t total = (int64_t)n0 * n1 * vv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ab = idx % vv;
    const int64_t t = idx / vv;
    const int J = (int)(t % n1), i = (int)(t / n1);
    double val = 0.0;
    if (side == 0) {
      if (i < na) {
        val = t2[((int64_t)i * nb + J) * vv + ab];
      } else {
        const double* cp = coef + (int64_t)(i - na) * na;
        for (int m = 0; m < na; ++m) val += cp[m] * t2[((int64_t)m * nb + J) * vv + ab];
      }
    } else {
      if (J < nb) {
        val = t2[((int64_t)i * nb + J) * vv + ab];
      } else {
        const double* cp = coef + (int64_t)(J - nb) * nb;
        for (int m = 0; m < nb; ++m) val += cp[m] * t2[((int64_t)i * nb + m) * vv + ab];
      }
    }
    out[idx] = val;
  }
}

// rows [o][v] -> [o+P][v] (T1, f_ov); pseudo rows are the combinations
__global__ void aug_rows(const double* __restrict__ x, int o, int v, int P,
                         const double* __restrict__ coef, double* __restrict__ out) {
  const int64_t total = (int64_t)(o + P) * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(idx % v), r = (int)(idx / v);
    double val = 0.0;
    if (r < o) {
      val = x[(int64_t)r * v + a];
    } else {
      const double* cp = coef + (int64_t)(r - o) * o;
      for (int m = 0; m < o; ++m) val += cp[m] * x[(int64_t)m * v + a];
    }
    out[idx] = val;
  }
}

// orbital energies [nbas] -> [nbas + P]: pseudo-orbitals at 0 (their factor
// is in the coefficients)
__global__ void aug_eps(const double* __restrict__ e, int nbas, int o, int P,
                        double* __restrict__ out) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nbas + P; r += gridDim.x * blockDim.x)
    out[r] = r < o ? e[r] : (r < o + P ? 0.0 : e[r - P]);
}

}  // namespace

cudaError_t launch_lmo_augment(const AugmentArgs& A, cudaStream_t st) {
  const int s = A.spin, o = A.nocc[s], P = A.P;
  const int v = A.nbas - o;
  lmo_coef<<<grid_of((int64_t)P * o), 256, 0, st>>>(A.U, A.eps_in, P, o, A.s, A.coef);
  aug_B<<<grid_of((int64_t)A.naux * (A.nbas + P) * (A.nbas + P)), 256, 0, st>>>(
      A.B_in, A.naux, A.nbas, o, P, A.coef, A.B_out);
  aug_eps<<<grid_of(A.nbas + P), 256, 0, st>>>(A.eps_in, A.nbas, o, P, A.eps_out);
  if (v > 0) {
    aug_rows<<<grid_of((int64_t)(o + P) * v), 256, 0, st>>>(A.t1_in, o, v, P, A.coef, A.t1_out);
    if (A.fov_in)
      aug_rows<<<grid_of((int64_t)(o + P) * v), 256, 0, st>>>(A.fov_in, o, v, P, A.coef,
                                                             A.fov_out);
    aug_t2ss<<<grid_of((int64_t)(o + P) * (o + P) * v * v), 256, 0, st>>>(A.t2ss_in, o, v, P,
                                                                           A.coef, A.t2ss_out);
  }
  const int na = A.nocc[0], nb = A.nocc[1];
  const int va = A.nbas - na, vb = A.nbas - nb;
  const int64_t n01 = (int64_t)(s == 0 ? na + P : na) * (s == 0 ? nb : nb + P) * va * vb;
  if (n01 > 0)
    aug_t2ab<<<grid_of(n01), 256, 0, st>>>(A.t2ab_in, na, nb, va, vb, P, s, A.coef, A.t2ab_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Quadrature of 1/x on [xmin, xmax]: the fewest points n (<= nmax) whose
// exponential sum sum_q w_q exp(-x s_q) has a largest relative error <= tol.
// For each n: start from the trapezoid rule of 1/x = int exp(t - x e^t) dt on
// a grid of t = ln s, then Levenberg-Marquardt on the weighted squared
// relative error over a log grid of x, with the weights pulled towards the
// error (Lawson) so that the fit approaches the minimax one.  The paper gives
// only the threshold (laptol = 1e-2, Table thresholds) and "3(-4) points";
// this construction is the reading taken.
namespace {

double rel_err_max(const std::vector<double>& p, int n, const std::vector<double>& y) {
  double m = 0.0;
  for (double x : y) {
    double f = 0.0;
    for (int q = 0; q < n; ++q) f += std::exp(p[n + q] - x * std::exp(p[q]));
    m = std::max(m, std::fabs(1.0 - x * f));
  }
  return m;
}

// Solve the symmetric positive definite system A x = b (n x n, Cholesky).
bool spd_solve(std::vector<double>& A, std::vector<double>& b, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = A[i * n + j];
      for (int k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = v / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double v = b[i];
    for (int k = 0; k < i; ++k) v -= A[i * n + k] * b[k];
    b[i] = v / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = b[i];
    for (int k = i + 1; k < n; ++k) v -= A[k * n + i] * b[k];
    b[i] = v / A[i * n + i];
  }
  return true;
}

}  // namespace

int laplace_quadrature(double xmin, double xmax, double tol, int nmax, double* s, double* w,
                       int* nq) {
  if (!(xmin > 0.0) || !(xmax > xmin) || !(tol > 0.0) || nmax < 1 || nmax > 32 || !s || !w ||
      !nq)
    return LNO_OT_EINVAL;
  const double R = xmax / xmin;
  const int M = 400;
  std::vector<double> y(M);
  for (int k = 0; k < M; ++k) y[k] = std::exp(std::log(R) * k / (M - 1));   // [1, R]
  const double tt = std::min(tol, 0.1);
  for (int n = 1; n <= nmax; ++n) {
    const double lo = std::log(tt / (4.0 * R)), hi = std::log(std::log(1.0 / tt) + 1.0);
    const double h = n > 1 ? (hi - lo) / (n - 1) : (hi - lo);
    std::vector<double> p(2 * n);   // ln s_q, ln w_q on [1, R]
    for (int q = 0; q < n; ++q) {
      p[q] = n > 1 ? lo + h * q : 0.5 * (lo + hi);
      p[n + q] = p[q] + std::log(h);
    }
    std::vector<double> wt(M, 1.0);
    const int np = 2 * n;
    for (int outer = 0; outer < 30; ++outer) {
      double lambda = 1e-3;
      for (int it = 0; it < 200; ++it) {
        // residuals r_k = wt_k (1 - y_k f(y_k)) and Jacobian in ln s, ln w
        std::vector<double> JTJ(np * np, 0.0), JTr(np, 0.0);
        double cost = 0.0;
        for (int k = 0; k < M; ++k) {
          double f = 0.0;
          std::vector<double> g(np);
          for (int q = 0; q < n; ++q) {
            const double sq = std::exp(p[q]);
            const double e = std::exp(p[n + q] - y[k] * sq);
            f += e;
            g[q] = wt[k] * y[k] * e * y[k] * sq;   // d r / d ln s_q
            g[n + q] = -wt[k] * y[k] * e;          // d r / d ln w_q
          }
          const double r = wt[k] * (1.0 - y[k] * f);
          cost += r * r;
          for (int a = 0; a < np; ++a) {
            JTr[a] += g[a] * r;
            for (int b = 0; b <= a; ++b) JTJ[a * np + b] += g[a] * g[b];
          }
        }
        for (int a = 0; a < np; ++a)
          for (int b = a + 1; b < np; ++b) JTJ[a * np + b] = JTJ[b * np + a];
        bool step_ok = false, converged = false;
        for (int tries = 0; tries < 12 && !step_ok; ++tries) {
          std::vector<double> A(JTJ), d(np);
          for (int a = 0; a < np; ++a) {
            A[a * np + a] = A[a * np + a] * (1.0 + lambda) + 1e-30;
            d[a] = -JTr[a];
          }
          if (!spd_solve(A, d, np)) {
            lambda *= 10.0;
            continue;
          }
          std::vector<double> pn(p);
          for (int a = 0; a < np; ++a) pn[a] = std::min(30.0, std::max(-60.0, p[a] + d[a]));
          double c2 = 0.0;
          for (int k = 0; k < M; ++k) {
            double f = 0.0;
            for (int q = 0; q < n; ++q) f += std::exp(pn[n + q] - y[k] * std::exp(pn[q]));
            const double r = wt[k] * (1.0 - y[k] * f);
            c2 += r * r;
          }
          if (c2 < cost) {
            converged = cost - c2 < 1e-14 * cost;
            p = pn;
            lambda = std::max(lambda * 0.3, 1e-12);
            step_ok = true;
          } else {
            lambda *= 10.0;
          }
        }
        if (!step_ok || converged) break;
      }
      // Lawson step: weights follow the error
      double rmax = 0.0;
      std::vector<double> ra(M);
      for (int k = 0; k < M; ++k) {
        double f = 0.0;
        for (int q = 0; q < n; ++q) f += std::exp(p[n + q] - y[k] * std::exp(p[q]));
        ra[k] = std::fabs(1.0 - y[k] * f);
        rmax = std::max(rmax, ra[k]);
      }
      if (!(rmax > 0.0)) break;
      double wmax = 0.0;
      for (int k = 0; k < M; ++k) {
        wt[k] = wt[k] * std::sqrt(ra[k] / rmax) + 1e-3;
        wmax = std::max(wmax, wt[k]);
      }
      for (int k = 0; k < M; ++k) wt[k] /= wmax;
    }
    // accept if the error on a finer grid is within tol
    std::vector<double> yf(4 * M);
    for (int k = 0; k < 4 * M; ++k) yf[k] = std::exp(std::log(R) * k / (4 * M - 1));
    if (rel_err_max(p, n, yf) <= tol) {
      // points driven to s xmin > 200 contribute below exp(-200): drop them
      std::vector<std::pair<double, double>> sw;
      for (int q = 0; q < n; ++q)
        if (std::exp(p[q]) <= 200.0) sw.push_back({std::exp(p[q]) / xmin, std::exp(p[n + q]) / xmin});
      std::sort(sw.begin(), sw.end());
      const int m = (int)sw.size();
      for (int q = 0; q < m; ++q) {
        s[q] = sw[q].first;
        w[q] = sw[q].second;
      }
      *nq = m;
      return LNO_OT_OK;
    }
  }
  return LNO_OT_EUNSUPPORTED;
}

}  // namespace lno
