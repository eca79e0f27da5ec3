// 1D rules and Lagrange tables for the sum-factorized kernels (host setup).
//
// B^{1d}_{kj} = l_j(x_k) and G^{1d}_{kj} = l_j'(x_k) are the one-dimensional
// factors of the basis evaluator B (Sec. 4.4, B_ki = B^{1d}_{k1 i1} ...
// B^{1d}_{kd id}), with l_j the Lagrange polynomials at the Gauss-Lobatto
// points (the nodal H1 basis of Sec. 3.3) and x_k the Gauss-Legendre points
// of the quadrature rule. Nodes come from Newton iteration on the Legendre
// three-term recurrence in long double; the tables use barycentric weights.
#include <cmath>

#include "fem_internal.h"

namespace {

typedef long double ld;
const ld kPi = 3.141592653589793238462643383279502884L;

// P_n(t) and P_n'(t) on [-1,1].
void legendre(int n, ld t, ld& P, ld& dP) {
  ld p0 = 1, p1 = t;
  if (n == 0) { P = 1; dP = 0; return; }
  for (int k = 1; k < n; ++k) {
    ld p2 = ((2 * k + 1) * t * p1 - k * p0) / (k + 1);
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (t * p1 - p0) / (t * t - 1);
}

}  // namespace

void fem_gauss_rule(int q, std::vector<double>& pts, std::vector<double>& wts) {
  pts.assign(q, 0.0);
  wts.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    // i-th root from below, Tricomi-style initial guess
    ld t = -cosl(kPi * (i + 0.75L) / (q + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(q, t, P, dP);
      ld dt = P / dP;
      t -= dt;
      if (fabsl(dt) < 1e-30L) break;
    }
    ld P, dP;
    legendre(q, t, P, dP);
    pts[i] = (double)((t + 1) / 2);
    wts[i] = (double)(1 / ((1 - t * t) * dP * dP));  // (2 / (...)) / 2 on [0,1]
  }
}

void fem_gll_nodes(int p, std::vector<double>& nodes) {
  nodes.assign(p + 1, 0.0);
  nodes[0] = 0.0;
  nodes[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    // roots of P_p' ; Newton on f = P_p', f' from the Legendre ODE
    ld t = -cosl(kPi * i / p);
    for (int it = 0; it < 100; ++it) {
      ld P, dP;
      legendre(p, t, P, dP);
      ld d2P = (2 * t * dP - p * (p + 1) * P) / (1 - t * t);
      ld dt = dP / d2P;
      t -= dt;
      if (fabsl(dt) < 1e-30L) break;
    }
    nodes[i] = (double)((t + 1) / 2);
  }
}

void fem_lagrange_tables(const std::vector<double>& nodes, const std::vector<double>& pts,
                         std::vector<double>& B, std::vector<double>& G) {
  const int n = (int)nodes.size(), m = (int)pts.size();
  B.assign((size_t)m * n, 0.0);
  G.assign((size_t)m * n, 0.0);
  std::vector<ld> w(n, 1);  // barycentric weights 1 / prod_{k != j} (x_j - x_k)
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) w[j] /= ((ld)nodes[j] - (ld)nodes[k]);
  for (int r = 0; r < m; ++r) {
    const ld x = pts[r];
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (fabsl(x - (ld)nodes[j]) < 1e-300L) hit = j;
    if (hit >= 0) {
      // x is a node: l_j(x) = delta; l_j'(x_i) = (w_j / w_i) / (x_i - x_j), j != i
      ld diag = 0;
      for (int j = 0; j < n; ++j) {
        B[(size_t)r * n + j] = (j == hit) ? 1.0 : 0.0;
        if (j != hit) {
          ld d = (w[j] / w[hit]) / ((ld)nodes[hit] - (ld)nodes[j]);
          G[(size_t)r * n + j] = (double)d;
          diag -= d;
        }
      }
      G[(size_t)r * n + hit] = (double)diag;
      continue;
    }
    // l_j(x) = (w_j / (x - x_j)) / sum_k (w_k / (x - x_k));
    // l_j'(x) = l_j(x) * (sum_{k != j} 1 / (x - x_k))
    ld den = 0;
    for (int k = 0; k < n; ++k) den += w[k] / (x - (ld)nodes[k]);
    ld sinv = 0;
    for (int k = 0; k < n; ++k) sinv += 1 / (x - (ld)nodes[k]);
    for (int j = 0; j < n; ++j) {
      ld lj = (w[j] / (x - (ld)nodes[j])) / den;
      B[(size_t)r * n + j] = (double)lj;
      G[(size_t)r * n + j] = (double)(lj * (sinv - 1 / (x - (ld)nodes[j])));
    }
  }
}
