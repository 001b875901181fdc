// Host-side 1D tables of the Q_p basis and the small dense eigenvalue step of the
// Chebyshev bound. Everything here is FP64 and runs once per level at setup.
//
//  * GLL nodes (paper Sec. 2.3, Fig. 1): end points of [0,1] plus the roots of P_p',
//    found by Newton's method from Chebyshev-Lobatto guesses.
//  * Gauss-Legendre rule with q = p+1 points (the quadrature the paper calls "Gauss
//    quadrature", Sec. 2.3), Newton on P_q, weights 2/((1-x^2) P_q'(x)^2).
//  * Lagrange tables by the barycentric formulas (Berrut & Trefethen, SIAM Review 46, 2004):
//    interpolation l_a(x) = (lam_a/(x-r_a)) / sum_m lam_m/(x-r_m), and the collocation
//    derivative D_ij = (lam_j/lam_i)/(x_i-x_j), D_ii = -sum_{j!=i} D_ij.
//  * Largest real eigenvalue of a small upper Hessenberg matrix by the Francis
//    double-shift QR iteration (Golub & Van Loan, Matrix Computations, Sec. 7.5).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace hmg {

namespace {

// P_n(x) and P_n'(x), x in [-1,1], by the three-term recurrence.
void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    const double d2 = d0 + (2.0 * k + 1.0) * p1;
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  *P = p1;
  *dP = d1;
}

void barycentric_weights(const double* x, int n, double* lam) {
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) prod *= (x[j] - x[m]);
    lam[j] = 1.0 / prod;
  }
}

}  // namespace

void lagrange_row(const double* r, int n, double x, double* out) {
  double lam[kMaxN];
  barycentric_weights(r, n, lam);
  for (int a = 0; a < n; ++a) {
    if (x == r[a]) {
      for (int b = 0; b < n; ++b) out[b] = (a == b) ? 1.0 : 0.0;
      return;
    }
  }
  double den = 0.0;
  for (int a = 0; a < n; ++a) den += lam[a] / (x - r[a]);
  for (int a = 0; a < n; ++a) out[a] = (lam[a] / (x - r[a])) / den;
}

void make_basis(int p, Basis1D* o) {
  memset(o, 0, sizeof(*o));
  const int n = p + 1;
  o->p = p;
  o->n = n;
  // GLL nodes on [-1,1]
  double t[kMaxN];
  t[0] = -1.0;
  t[p] = 1.0;
  for (int j = 1; j < p; ++j) {
    double x = -cos(M_PI * j / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, x, &P, &dP);
      const double d2P = (2.0 * x * dP - p * (p + 1.0) * P) / (1.0 - x * x);
      const double dx = dP / d2P;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    t[j] = x;
  }
  for (int j = 0; j < n; ++j) {  // symmetrize and map to [0,1]
    const double s = 0.5 * (t[j] - t[p - j]);
    o->r[j] = 0.5 * (s + 1.0);
  }
  o->r[0] = 0.0;
  o->r[p] = 1.0;
  // Gauss-Legendre with q = n points
  const int q = n;
  double gx[kMaxN], gw[kMaxN];
  for (int j = 0; j < q; ++j) {
    double x = -cos(M_PI * (j + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, x, &P, &dP);
      const double dx = P / dP;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    double P, dP;
    legendre(q, x, &P, &dP);
    gx[j] = x;
    gw[j] = 2.0 / ((1.0 - x * x) * dP * dP);
  }
  for (int j = 0; j < q; ++j) {
    const double s = 0.5 * (gx[j] - gx[q - 1 - j]);
    o->g[j] = 0.5 * (s + 1.0);
    o->w[j] = 0.25 * (gw[j] + gw[q - 1 - j]);
  }
  // B[q][a] = l_a(g_q) on the GLL nodes
  for (int i = 0; i < q; ++i) lagrange_row(o->r, n, o->g[i], &o->B[i * n]);
  // collocated derivative on the Gauss points
  double lam[kMaxN];
  barycentric_weights(o->g, q, lam);
  for (int i = 0; i < q; ++i) {
    double diag = 0.0;
    for (int j = 0; j < q; ++j) {
      if (j == i) continue;
      const double v = (lam[j] / lam[i]) / (o->g[i] - o->g[j]);
      o->D[i * q + j] = v;
      diag -= v;
    }
    o->D[i * q + i] = diag;
  }
  // Bd = D B
  for (int i = 0; i < q; ++i)
    for (int a = 0; a < n; ++a) {
      double s = 0.0;
      for (int k = 0; k < q; ++k) s += o->D[i * q + k] * o->B[k * n + a];
      o->Bd[i * n + a] = s;
    }
}

// ---------------------------------------------------------------------------------------
// Francis double-shift QR on an upper Hessenberg matrix (eigenvalues only).
// ---------------------------------------------------------------------------------------
namespace {

// Householder vector v (v[0] = 1) and beta with (I - beta v v^T) x = ||x|| e_1 direction.
void house(const double* x, int len, double* v, double* beta) {
  double sigma = 0.0;
  for (int i = 1; i < len; ++i) sigma += x[i] * x[i];
  v[0] = 1.0;
  for (int i = 1; i < len; ++i) v[i] = x[i];
  if (sigma == 0.0) {
    *beta = 0.0;
    return;
  }
  const double mu = sqrt(x[0] * x[0] + sigma);
  const double v0 = (x[0] <= 0.0) ? x[0] - mu : -sigma / (x[0] + mu);
  *beta = 2.0 * v0 * v0 / (sigma + v0 * v0);
  for (int i = 1; i < len; ++i) v[i] /= v0;
}

// One Francis double-shift step on the active block H[lo..hi][lo..hi] (size >= 3).
void francis_step(std::vector<double>& H, int m, int lo, int hi, bool exceptional) {
  auto h = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  const int n = hi - lo + 1;
  double s, t;
  if (exceptional) {  // ad-hoc shifts to break a stagnating iteration
    const double w = fabs(h(hi, hi - 1)) + fabs(h(hi - 1, hi - 2));
    s = 1.5 * w + h(hi, hi);
    t = w * w;
  } else {
    s = h(hi - 1, hi - 1) + h(hi, hi);
    t = h(hi - 1, hi - 1) * h(hi, hi) - h(hi - 1, hi) * h(hi, hi - 1);
  }
  double x = h(lo, lo) * h(lo, lo) + h(lo, lo + 1) * h(lo + 1, lo) - s * h(lo, lo) + t;
  double y = h(lo + 1, lo) * (h(lo, lo) + h(lo + 1, lo + 1) - s);
  double z = h(lo + 1, lo) * h(lo + 2, lo + 1);
  for (int k = 0; k <= n - 3; ++k) {
    double xv[3] = {x, y, z}, v[3], beta;
    house(xv, 3, v, &beta);
    const int r0 = lo + k;
    const int cq = std::max(lo, r0 - 1);
    for (int j = cq; j <= hi; ++j) {  // rows r0..r0+2 from the left
      const double d = v[0] * h(r0, j) + v[1] * h(r0 + 1, j) + v[2] * h(r0 + 2, j);
      h(r0, j) -= beta * v[0] * d;
      h(r0 + 1, j) -= beta * v[1] * d;
      h(r0 + 2, j) -= beta * v[2] * d;
    }
    const int rr = std::min(r0 + 3, hi);
    for (int i = lo; i <= rr; ++i) {  // columns r0..r0+2 from the right
      const double d = h(i, r0) * v[0] + h(i, r0 + 1) * v[1] + h(i, r0 + 2) * v[2];
      h(i, r0) -= beta * d * v[0];
      h(i, r0 + 1) -= beta * d * v[1];
      h(i, r0 + 2) -= beta * d * v[2];
    }
    x = h(r0 + 1, r0);
    y = h(r0 + 2, r0);
    if (k < n - 3) z = h(r0 + 3, r0);
  }
  double xv[2] = {x, y}, v[2], beta;
  house(xv, 2, v, &beta);
  const int r0 = hi - 1;
  for (int j = hi - 2; j <= hi; ++j) {
    const double d = v[0] * h(r0, j) + v[1] * h(r0 + 1, j);
    h(r0, j) -= beta * v[0] * d;
    h(r0 + 1, j) -= beta * v[1] * d;
  }
  for (int i = lo; i <= hi; ++i) {
    const double d = h(i, r0) * v[0] + h(i, r0 + 1) * v[1];
    h(i, r0) -= beta * d * v[0];
    h(i, r0 + 1) -= beta * d * v[1];
  }
}

}  // namespace

double hessenberg_max_real_eig(const double* Hin, int m) {
  std::vector<double> H(Hin, Hin + (size_t)m * m);
  auto h = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  const double eps = 2.220446049250313e-16;
  double best = -INFINITY;
  int hi = m - 1, iter = 0;
  while (hi >= 0) {
    if (hi == 0) {
      best = std::max(best, h(0, 0));
      hi = -1;
      break;
    }
    // deflate negligible sub-diagonal entries and find the unreduced block [lo, hi]
    int lo = 0;
    for (int i = hi; i >= 1; --i) {
      if (fabs(h(i, i - 1)) <= eps * (fabs(h(i, i)) + fabs(h(i - 1, i - 1)))) {
        h(i, i - 1) = 0.0;
        lo = i;
        break;
      }
    }
    if (lo == hi) {  // 1x1 block
      best = std::max(best, h(hi, hi));
      hi -= 1;
      iter = 0;
    } else if (lo == hi - 1) {  // 2x2 block
      const double a = h(lo, lo), b = h(lo, hi), c = h(hi, lo), d = h(hi, hi);
      const double tr = 0.5 * (a + d);
      const double disc = 0.25 * (a - d) * (a - d) + b * c;
      if (disc >= 0.0) best = std::max(best, tr + sqrt(disc));
      else best = std::max(best, tr);
      hi -= 2;
      iter = 0;
    } else {
      ++iter;
      if (iter > 60 * m) return NAN;  // no convergence
      francis_step(H, m, lo, hi, iter % 11 == 10);
    }
  }
  return best;
}

}  // namespace hmg
