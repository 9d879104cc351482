// Host-side construction of the SEM and FD discretisations.  See setup_host.h.
#include "setup_host.h"

#include <algorithm>
#include <cmath>

namespace chebmg {

namespace {

// Legendre P_{N-1}(x) and P_N(x) by Bonnet's recurrence.
void legendre_pair(int N, double x, double& pm1, double& p) {
  double a = 1.0, b = x;   // P_0, P_1
  if (N == 0) { pm1 = 0.0; p = 1.0; return; }
  for (int k = 2; k <= N; ++k) {
    double c = ((2.0 * k - 1.0) * x * b - (k - 1.0) * a) / k;
    a = b;
    b = c;
  }
  pm1 = a;
  p = b;
}

}  // namespace

void gll_rule(int N, std::vector<double>& x, std::vector<double>& w) {
  x.assign(N + 1, 0.0);
  w.assign(N + 1, 0.0);
  // Interior GLL points are the roots of q(x) = (1 - x^2) P_N'(x).  With
  // (1 - x^2) P_N' = N (P_{N-1} - x P_N) and, from Legendre's equation,
  // q'(x) = -N (N+1) P_N(x), Newton's step is x += (P_{N-1} - x P_N) / ((N+1) P_N).
  for (int j = 0; j <= N; ++j) {
    double xj = -std::cos(M_PI * j / N);
    if (j > 0 && j < N) {
      for (int it = 0; it < 100; ++it) {
        double pm1, p;
        legendre_pair(N, xj, pm1, p);
        double dx = (pm1 - xj * p) / ((N + 1.0) * p);
        xj += dx;
        if (std::fabs(dx) < 1e-16) break;
      }
    }
    x[j] = xj;
  }
  x[0] = -1.0;
  x[N] = 1.0;
  for (int j = 0; j <= N; ++j) {
    double pm1, p;
    legendre_pair(N, x[j], pm1, p);
    w[j] = 2.0 / (N * (N + 1.0) * p * p);
  }
}

void gll_derivative(int N, const std::vector<double>& x, std::vector<double>& Dm) {
  // Closed form for GLL nodes: l_j'(x_i) = P_N(x_i) / (P_N(x_j) (x_i - x_j)), i != j;
  // the diagonal vanishes except at the end points, -+ N(N+1)/4.
  const int Q = N + 1;
  Dm.assign(Q * Q, 0.0);
  std::vector<double> PN(Q);
  for (int i = 0; i < Q; ++i) {
    double pm1;
    legendre_pair(N, x[i], pm1, PN[i]);
  }
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j < Q; ++j)
      if (i != j) Dm[i * Q + j] = PN[i] / (PN[j] * (x[i] - x[j]));
  Dm[0] = -N * (N + 1.0) / 4.0;
  Dm[Q * Q - 1] = N * (N + 1.0) / 4.0;
}

void lagrange_interp(const std::vector<double>& xc, const std::vector<double>& y,
                     std::vector<double>& J) {
  // Barycentric form of the Lagrange basis.
  const int nc = (int)xc.size(), ny = (int)y.size();
  std::vector<double> lam(nc, 1.0);
  for (int b = 0; b < nc; ++b)
    for (int m = 0; m < nc; ++m)
      if (m != b) lam[b] *= 1.0 / (xc[b] - xc[m]);
  J.assign((size_t)ny * nc, 0.0);
  for (int a = 0; a < ny; ++a) {
    int hit = -1;
    for (int b = 0; b < nc; ++b)
      if (y[a] == xc[b]) hit = b;
    if (hit >= 0) {
      J[(size_t)a * nc + hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int b = 0; b < nc; ++b) den += lam[b] / (y[a] - xc[b]);
    for (int b = 0; b < nc; ++b) J[(size_t)a * nc + b] = (lam[b] / (y[a] - xc[b])) / den;
  }
}

bool build_sem_level(int nex, int ney, int nez, const double* verts, int N, SemHostLevel& L) {
  L.N = N;
  L.NQ = N + 1;
  L.NP = L.NQ * L.NQ * L.NQ;
  L.nex = nex;
  L.ney = ney;
  L.nez = nez;
  L.E = (int64_t)nex * ney * nez;
  const int64_t NX = (int64_t)nex * N + 1, NY = (int64_t)ney * N + 1, NZ = (int64_t)nez * N + 1;
  L.n = NX * NY * NZ;
  gll_rule(N, L.x, L.w);
  gll_derivative(N, L.x, L.Dm);
  const int Q = L.NQ, NP = L.NP;
  L.gid.assign((size_t)L.E * NP, 0u);
  L.G.assign((size_t)L.E * 6 * NP, 0.0);
  L.dirichlet.assign((size_t)L.n, 0);
  L.diag.assign((size_t)L.n, 0.0);

  for (int64_t gz = 0; gz < NZ; ++gz)
    for (int64_t gy = 0; gy < NY; ++gy)
      for (int64_t gx = 0; gx < NX; ++gx) {
        bool b = gx == 0 || gx == NX - 1 || gy == 0 || gy == NY - 1 || gz == 0 || gz == NZ - 1;
        L.dirichlet[(gz * NY + gy) * NX + gx] = b ? 1 : 0;
      }

  double minJ = 1e300;
  bool ok = true;
  std::vector<double> diag_local((size_t)L.E * NP, 0.0);

#pragma omp parallel for schedule(static) reduction(min : minJ)
  for (int64_t e = 0; e < L.E; ++e) {
    const int ex = (int)(e % nex), ey = (int)((e / nex) % ney), ez = (int)(e / ((int64_t)nex * ney));
    double V[2][2][2][3];
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const double* v = verts + 3 * (((int64_t)(ez + c) * (ney + 1) + (ey + b)) * (nex + 1) + (ex + a));
          for (int l = 0; l < 3; ++l) V[c][b][a][l] = v[l];
        }
    uint32_t* gid = &L.gid[(size_t)e * NP];
    double* G = &L.G[(size_t)e * 6 * NP];
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i) {
          const int p = (k * Q + j) * Q + i;
          // exact derivatives of the trilinear map at (r, s, t) = (x_i, x_j, x_k)
          const double r = L.x[i], s = L.x[j], t = L.x[k];
          const double fr[2] = {0.5 * (1 - r), 0.5 * (1 + r)}, dr[2] = {-0.5, 0.5};
          const double fs[2] = {0.5 * (1 - s), 0.5 * (1 + s)}, ds[2] = {-0.5, 0.5};
          const double ft[2] = {0.5 * (1 - t), 0.5 * (1 + t)}, dt[2] = {-0.5, 0.5};
          double Jm[3][3] = {{0}};   // Jm[l][m] = d x_l / d r_m
          for (int c = 0; c < 2; ++c)
            for (int b = 0; b < 2; ++b)
              for (int a = 0; a < 2; ++a)
                for (int l = 0; l < 3; ++l) {
                  Jm[l][0] += dr[a] * fs[b] * ft[c] * V[c][b][a][l];
                  Jm[l][1] += fr[a] * ds[b] * ft[c] * V[c][b][a][l];
                  Jm[l][2] += fr[a] * fs[b] * dt[c] * V[c][b][a][l];
                }
          // adjugate: adj[m][l] = cofactor C[l][m]; J^{-1} = adj / det
          double adj[3][3];
          adj[0][0] = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
          adj[0][1] = Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2];
          adj[0][2] = Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1];
          adj[1][0] = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
          adj[1][1] = Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0];
          adj[1][2] = Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2];
          adj[2][0] = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
          adj[2][1] = Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1];
          adj[2][2] = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
          const double det = Jm[0][0] * adj[0][0] + Jm[0][1] * adj[1][0] + Jm[0][2] * adj[2][0];
          minJ = std::min(minJ, det);
          // G_mn = w_i w_j w_k |J| (J^{-1} J^{-T})_mn = w3 / det * (adj adj^T)_mn
          const double scale = L.w[i] * L.w[j] * L.w[k] / det;
          const int mm[6] = {0, 0, 0, 1, 1, 2}, nn[6] = {0, 1, 2, 1, 2, 2};
          for (int q = 0; q < 6; ++q) {
            double acc = 0.0;
            for (int l = 0; l < 3; ++l) acc += adj[mm[q]][l] * adj[nn[q]][l];
            G[q * NP + p] = scale * acc;
          }
          const int64_t gx = (int64_t)ex * N + i, gy = (int64_t)ey * N + j, gz = (int64_t)ez * N + k;
          const int64_t g = (gz * NY + gy) * NX + gx;
          uint32_t id = (uint32_t)g;
          bool bnd = gx == 0 || gx == NX - 1 || gy == 0 || gy == NY - 1 || gz == 0 || gz == NZ - 1;
          if (bnd) id |= kGidDirichlet;
          const bool own = std::min<int64_t>(gx / N, nex - 1) == ex &&
                           std::min<int64_t>(gy / N, ney - 1) == ey &&
                           std::min<int64_t>(gz / N, nez - 1) == ez;
          if (own) id |= kGidOwner;
          gid[p] = id;
        }
    // diagonal of A_e: sum_l G_rr(l,j,k) D[l,i]^2 + ... + 2 G_rs D[i,i] D[j,j] + ...
    const double* D = L.Dm.data();
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i) {
          const int p = (k * Q + j) * Q + i;
          double acc = 0.0;
          for (int l = 0; l < Q; ++l) {
            acc += G[0 * NP + (k * Q + j) * Q + l] * D[l * Q + i] * D[l * Q + i];
            acc += G[3 * NP + (k * Q + l) * Q + i] * D[l * Q + j] * D[l * Q + j];
            acc += G[5 * NP + (l * Q + j) * Q + i] * D[l * Q + k] * D[l * Q + k];
          }
          const double di = D[i * Q + i], dj = D[j * Q + j], dk = D[k * Q + k];
          acc += 2.0 * (G[1 * NP + p] * di * dj + G[2 * NP + p] * di * dk + G[4 * NP + p] * dj * dk);
          diag_local[(size_t)e * NP + p] = acc;
        }
  }
  L.min_jacobian = minJ;
  if (!(minJ > 0.0)) ok = false;
  for (int64_t q = 0; q < L.E * NP; ++q) {
    const uint32_t id = L.gid[q];
    if (!(id & kGidDirichlet)) L.diag[id & kGidMask] += diag_local[q];
  }
  return ok;
}

void assemble_ell(const SemHostLevel& L, int& nslot, std::vector<int>& col, std::vector<double>& val) {
  const int Q = L.NQ, NP = L.NP;
  const double* D = L.Dm.data();
  struct Trip {
    uint32_t row, col;
    double v;
  };
  std::vector<Trip> trips;
  trips.reserve((size_t)L.E * NP * 27);
  std::vector<double> Ae((size_t)NP * NP);
  for (int64_t e = 0; e < L.E; ++e) {
    std::fill(Ae.begin(), Ae.end(), 0.0);
    const double* G = &L.G[(size_t)e * 6 * NP];
    // A_e[p][q] = sum_pt sum_mn Dhat_m(pt, p) G_mn(pt) Dhat_n(pt, q); Dhat_m(pt, .) is nonzero
    // only on the line through pt in direction m, with values D[pt_m][a].
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i) {
          const int pt = (k * Q + j) * Q + i;
          const int c[3] = {i, j, k};
          const double g[3][3] = {{G[0 * NP + pt], G[1 * NP + pt], G[2 * NP + pt]},
                                  {G[1 * NP + pt], G[3 * NP + pt], G[4 * NP + pt]},
                                  {G[2 * NP + pt], G[4 * NP + pt], G[5 * NP + pt]}};
          auto node = [&](int dir, int a) {
            int cc[3] = {i, j, k};
            cc[dir] = a;
            return (cc[2] * Q + cc[1]) * Q + cc[0];
          };
          for (int m = 0; m < 3; ++m)
            for (int a = 0; a < Q; ++a) {
              const double dm = D[c[m] * Q + a];
              if (dm == 0.0) continue;
              const int p = node(m, a);
              for (int n = 0; n < 3; ++n) {
                const double gm = dm * g[m][n];
                for (int b = 0; b < Q; ++b) {
                  const double dn = D[c[n] * Q + b];
                  if (dn == 0.0) continue;
                  Ae[(size_t)p * NP + node(n, b)] += gm * dn;
                }
              }
            }
        }
    const uint32_t* gid = &L.gid[(size_t)e * NP];
    for (int p = 0; p < NP; ++p) {
      if (gid[p] & kGidDirichlet) continue;
      for (int q = 0; q < NP; ++q) {
        if (gid[q] & kGidDirichlet) continue;
        trips.push_back({gid[p] & kGidMask, gid[q] & kGidMask, Ae[(size_t)p * NP + q]});
      }
    }
  }
  std::stable_sort(trips.begin(), trips.end(), [](const Trip& a, const Trip& b) {
    return a.row != b.row ? a.row < b.row : a.col < b.col;
  });
  const int64_t n = L.n;
  std::vector<int> count((size_t)n, 0);
  std::vector<int> rcol;
  std::vector<double> rval;
  std::vector<int64_t> start((size_t)n + 1, 0);
  // merge duplicates (sum in element order) into compressed rows
  for (size_t t = 0; t < trips.size();) {
    size_t u = t;
    double acc = 0.0;
    while (u < trips.size() && trips[u].row == trips[t].row && trips[u].col == trips[t].col) acc += trips[u++].v;
    rcol.push_back((int)trips[t].col);
    rval.push_back(acc);
    count[trips[t].row] += 1;
    t = u;
  }
  nslot = 1;
  for (int64_t g = 0; g < n; ++g) {
    start[g + 1] = start[g] + count[g];
    nslot = std::max(nslot, count[g]);
  }
  col.assign((size_t)nslot * n, 0);
  val.assign((size_t)nslot * n, 0.0);
  for (int64_t g = 0; g < n; ++g) {
    for (int s = 0; s < nslot; ++s) {
      const bool live = s < count[g];
      col[(size_t)s * n + g] = live ? rcol[start[g] + s] : (int)g;
      val[(size_t)s * n + g] = live ? rval[start[g] + s] : 0.0;
    }
  }
}

void fd_fine_stencil(double hx, double hy, double st[9]) {
  for (int q = 0; q < 9; ++q) st[q] = 0.0;
  st[4] = 2.0 / (hx * hx) + 2.0 / (hy * hy);
  st[3] = st[5] = -1.0 / (hx * hx);
  st[1] = st[7] = -1.0 / (hy * hy);
}

void fd_galerkin_stencil(const double fine[9], int c, double coarse[9]) {
  // Coarse basis function of node (0,0) on the fine lattice: bilinear hat of
  // half-width c.  A_c(0, (B,A)) = <phi_{(A c, B c)}, A phi_0> on an
  // unbounded lattice (the Dirichlet truncation does not change interior-
  // restricted entries for vertex-centred coarsening).
  const int R = 3 * c;
  const int W = 2 * R + 1;
  auto hat = [c](int i) { return std::max(0.0, 1.0 - std::abs(i) / (double)c); };
  std::vector<double> Aphi((size_t)W * W, 0.0);
  for (int j = -R + 1; j < R; ++j)
    for (int i = -R + 1; i < R; ++i) {
      double acc = 0.0;
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) acc += fine[(a + 1) * 3 + (b + 1)] * hat(i + b) * hat(j + a);
      Aphi[(size_t)(j + R) * W + (i + R)] = acc;
    }
  for (int A = -1; A <= 1; ++A)
    for (int B = -1; B <= 1; ++B) {
      double acc = 0.0;
      for (int j = -R + 1; j < R; ++j)
        for (int i = -R + 1; i < R; ++i)
          acc += hat(i - B * c) * hat(j - A * c) * Aphi[(size_t)(j + R) * W + (i + R)];
      coarse[(A + 1) * 3 + (B + 1)] = acc;
    }
}

bool fd_dense_inverse(const double st[9], int mx, int my, std::vector<double>& inv) {
  const int n = mx * my;
  std::vector<double> A((size_t)n * n, 0.0);
  for (int j = 0; j < my; ++j)
    for (int i = 0; i < mx; ++i)
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b) {
          const int ii = i + b, jj = j + a;
          if (ii < 0 || ii >= mx || jj < 0 || jj >= my) continue;
          A[(size_t)(j * mx + i) * n + (jj * mx + ii)] += st[(a + 1) * 3 + (b + 1)];
        }
  // Cholesky A = L L^T (lower triangle of A overwritten)
  for (int k = 0; k < n; ++k) {
    double d = A[(size_t)k * n + k];
    for (int m = 0; m < k; ++m) d -= A[(size_t)k * n + m] * A[(size_t)k * n + m];
    if (!(d > 0.0)) return false;
    d = std::sqrt(d);
    A[(size_t)k * n + k] = d;
    for (int i = k + 1; i < n; ++i) {
      double s = A[(size_t)i * n + k];
      for (int m = 0; m < k; ++m) s -= A[(size_t)i * n + m] * A[(size_t)k * n + m];
      A[(size_t)i * n + k] = s / d;
    }
  }
  inv.assign((size_t)n * n, 0.0);
  std::vector<double> y(n);
  for (int col = 0; col < n; ++col) {
    for (int i = 0; i < n; ++i) {   // L y = e_col
      double s = (i == col) ? 1.0 : 0.0;
      for (int m = 0; m < i; ++m) s -= A[(size_t)i * n + m] * y[m];
      y[i] = s / A[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {   // L^T x = y
      double s = y[i];
      for (int m = i + 1; m < n; ++m) s -= A[(size_t)m * n + i] * inv[(size_t)m * n + col];
      inv[(size_t)i * n + col] = s / A[(size_t)i * n + i];
    }
  }
  return true;
}

}  // namespace chebmg

namespace chebmg {

// gamma(lambda_min) = sup_{0 < lambda <= 1} lambda p^2 / (1 - p^2) (Eq. 2.14) of the 1st-kind
// polynomial p(lambda) = T_k((theta - lambda) / delta) / T_k(theta / delta), theta = (1 + lmin) / 2,
// delta = (1 - lmin) / 2 (lambda_max = 1): dense Chebyshev-spaced sampling, then a golden-section
// refinement around the largest sample.
static double cheb1_gamma(int k, double lmin) {
  const double theta = 0.5 * (1.0 + lmin), delta = 0.5 * (1.0 - lmin);
  auto Tk = [k](double x) {
    if (std::fabs(x) <= 1.0) return std::cos(k * std::acos(x));
    const double s = x > 0 ? 1.0 : ((k & 1) ? -1.0 : 1.0);
    return s * std::cosh(k * std::acosh(std::fabs(x)));
  };
  const double den = Tk(theta / delta);
  auto f = [&](double lam) {
    const double p = Tk((theta - lam) / delta) / den;
    const double q = 1.0 - p * p;
    return q > 0.0 ? lam * p * p / q : 1e300;
  };
  const int npts = 20000;
  double best = -1.0, bl = 0.0;
  for (int i = 1; i <= npts; ++i) {
    const double lam = 0.5 * (1.0 - std::cos(M_PI * i / npts));
    const double v = f(lam);
    if (v > best) {
      best = v;
      bl = lam;
    }
  }
  double a = std::max(1e-12, bl - 4e-4), b = std::min(1.0, bl + 4e-4);
  const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a), f1 = f(x1), f2 = f(x2);
  for (int it = 0; it < 100; ++it) {
    if (f1 > f2) {
      b = x2;
      x2 = x1;
      f2 = f1;
      x1 = b - gr * (b - a);
      f1 = f(x1);
    } else {
      a = x1;
      x1 = x2;
      f1 = f2;
      x2 = a + gr * (b - a);
      f2 = f(x2);
    }
  }
  return std::max(best, std::max(f1, f2));
}

double cheb1_optimal_lmin_ratio(int k) {
  // maximise gamma^{-1} over lambda_min / lambda_max: log-spaced scan, then golden section
  double bestl = 0.1, bestg = 1e300;
  const int nscan = 240;
  const double lo = 1e-4, hi = 0.9;
  for (int i = 0; i <= nscan; ++i) {
    const double l = lo * std::pow(hi / lo, (double)i / nscan);
    const double g = cheb1_gamma(k, l);
    if (g < bestg) {
      bestg = g;
      bestl = l;
    }
  }
  const double step = std::pow(hi / lo, 1.0 / nscan);
  double a = std::log(bestl / step), b = std::log(bestl * step);
  const double gr = 0.5 * (std::sqrt(5.0) - 1.0);
  double x1 = b - gr * (b - a), x2 = a + gr * (b - a);
  double g1 = cheb1_gamma(k, std::exp(x1)), g2 = cheb1_gamma(k, std::exp(x2));
  for (int it = 0; it < 60; ++it) {
    if (g1 < g2) {
      b = x2;
      x2 = x1;
      g2 = g1;
      x1 = b - gr * (b - a);
      g1 = cheb1_gamma(k, std::exp(x1));
    } else {
      a = x1;
      x1 = x2;
      g1 = g2;
      x2 = a + gr * (b - a);
      g2 = cheb1_gamma(k, std::exp(x2));
    }
  }
  return std::exp(0.5 * (a + b));
}

}  // namespace chebmg

// ---------------------------------------------------------------------------
// General hexahedral meshes
// ---------------------------------------------------------------------------
#include <array>
#include <unordered_map>

namespace chebmg {

namespace {

// G (six entries) and det at one point from the Jacobian Jm[l][m] = d x_l / d r_m and the
// quadrature weight w3 = w_i w_j w_k: G_mn = w3 / det (adj adj^T)_mn, adj = det J^{-1}.
double point_factors(const double Jm[3][3], double w3, double* G, int64_t stride) {
  double adj[3][3];
  adj[0][0] = Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1];
  adj[0][1] = Jm[0][2] * Jm[2][1] - Jm[0][1] * Jm[2][2];
  adj[0][2] = Jm[0][1] * Jm[1][2] - Jm[0][2] * Jm[1][1];
  adj[1][0] = Jm[1][2] * Jm[2][0] - Jm[1][0] * Jm[2][2];
  adj[1][1] = Jm[0][0] * Jm[2][2] - Jm[0][2] * Jm[2][0];
  adj[1][2] = Jm[0][2] * Jm[1][0] - Jm[0][0] * Jm[1][2];
  adj[2][0] = Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0];
  adj[2][1] = Jm[0][1] * Jm[2][0] - Jm[0][0] * Jm[2][1];
  adj[2][2] = Jm[0][0] * Jm[1][1] - Jm[0][1] * Jm[1][0];
  const double det = Jm[0][0] * adj[0][0] + Jm[0][1] * adj[1][0] + Jm[0][2] * adj[2][0];
  const double scale = w3 / det;
  const int mm[6] = {0, 0, 0, 1, 1, 2}, nn[6] = {0, 1, 2, 1, 2, 2};
  for (int q = 0; q < 6; ++q) {
    double acc = 0.0;
    for (int l = 0; l < 3; ++l) acc += adj[mm[q]][l] * adj[nn[q]][l];
    G[q * stride] = scale * acc;
  }
  return det;
}

using Key = std::array<int64_t, 7>;
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t h = 0x9E3779B97F4A7C15ull;
    for (int64_t v : k) {
      uint64_t z = (uint64_t)v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      h ^= z ^ (z >> 31);
    }
    return (size_t)h;
  }
};

}  // namespace

bool build_sem_level_mesh(const SemMeshInput& in, int Nt, SemHostLevel& L, std::string& err) {
  const int Nf = in.N, Qf = Nf + 1, NPf = Qf * Qf * Qf;
  L.N = Nt;
  L.NQ = Nt + 1;
  L.NP = L.NQ * L.NQ * L.NQ;
  L.nex = L.ney = L.nez = 0;
  L.E = in.E;
  const int Q = L.NQ, NP = L.NP;
  gll_rule(Nt, L.x, L.w);
  gll_derivative(Nt, L.x, L.Dm);
  std::vector<double> xf, wf;
  gll_rule(Nf, xf, wf);
  // coordinates at this order: the caller's, or their Lagrange interpolation (isoparametric)
  std::vector<double> X((size_t)in.E * NP * 3);
  if (Nt == Nf) {
    std::copy(in.coords, in.coords + X.size(), X.begin());
  } else {
    std::vector<double> J;
    lagrange_interp(xf, L.x, J);   // J[a * Qf + b] = l^f_b(x^t_a)
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < in.E; ++e) {
      const double* Xf = in.coords + (size_t)e * NPf * 3;
      std::vector<double> t1((size_t)Qf * Qf * Q * 3), t2((size_t)Qf * Q * Q * 3);
      for (int k = 0; k < Qf; ++k)
        for (int j = 0; j < Qf; ++j)
          for (int i = 0; i < Q; ++i)
            for (int l = 0; l < 3; ++l) {
              double acc = 0.0;
              for (int b = 0; b < Qf; ++b) acc += J[i * Qf + b] * Xf[((k * Qf + j) * Qf + b) * 3 + l];
              t1[((k * Qf + j) * Q + i) * 3 + l] = acc;
            }
      for (int k = 0; k < Qf; ++k)
        for (int j = 0; j < Q; ++j)
          for (int i = 0; i < Q; ++i)
            for (int l = 0; l < 3; ++l) {
              double acc = 0.0;
              for (int b = 0; b < Qf; ++b) acc += J[j * Qf + b] * t1[((k * Qf + b) * Q + i) * 3 + l];
              t2[((k * Q + j) * Q + i) * 3 + l] = acc;
            }
      double* Xt = &X[(size_t)e * NP * 3];
      for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j)
          for (int i = 0; i < Q; ++i)
            for (int l = 0; l < 3; ++l) {
              double acc = 0.0;
              for (int b = 0; b < Qf; ++b) acc += J[k * Qf + b] * t2[((b * Q + j) * Q + i) * 3 + l];
              Xt[((k * Q + j) * Q + i) * 3 + l] = acc;
            }
    }
  }
  // numbering and Dirichlet flags
  std::vector<int64_t> ids((size_t)in.E * NP);
  std::vector<uint8_t> dir;
  if (Nt == Nf) {
    std::copy(in.gid, in.gid + ids.size(), ids.begin());
    L.n = in.n;
    dir.assign(in.dirichlet, in.dirichlet + in.n);
  } else {
    // a coarse node lies on a vertex, an edge, a face or the interior of its element; shared
    // entities are identified by the fine global ids of their corners, and the node's place on
    // an edge or face is expressed in a frame fixed by those ids, so every element that shares
    // the entity computes the same key
    std::unordered_map<Key, int64_t, KeyHash> map;
    map.reserve((size_t)in.E * NP);
    dir.clear();
    auto fine = [&](int64_t e, int a, int b, int c) { return in.gid[(size_t)e * NPf + (c * Qf + b) * Qf + a]; };
    auto fend = [&](int t) { return t == 0 ? 0 : Nf; };
    for (int64_t e = 0; e < in.E; ++e)
      for (int k = 0; k < Q; ++k)
        for (int j = 0; j < Q; ++j)
          for (int i = 0; i < Q; ++i) {
            const int idx[3] = {i, j, k};
            const bool end[3] = {i == 0 || i == Nt, j == 0 || j == Nt, k == 0 || k == Nt};
            const int nend = end[0] + end[1] + end[2];
            Key key{};
            bool is_dir = false;
            if (nend == 3) {
              const int64_t g = fine(e, fend(i), fend(j), fend(k));
              key = {0, g, 0, 0, 0, 0, 0};
              is_dir = in.dirichlet[g] != 0;
            } else if (nend == 2) {
              const int d = !end[0] ? 0 : (!end[1] ? 1 : 2);
              int c0[3] = {fend(i), fend(j), fend(k)}, c1[3] = {fend(i), fend(j), fend(k)};
              c0[d] = 0;
              c1[d] = Nf;
              const int64_t g0 = fine(e, c0[0], c0[1], c0[2]), g1 = fine(e, c1[0], c1[1], c1[2]);
              const int pos = g0 < g1 ? idx[d] : Nt - idx[d];
              key = {1, std::min(g0, g1), std::max(g0, g1), pos, 0, 0, 0};
              is_dir = true;
              for (int q = 0; q < Qf && is_dir; ++q) {
                int c[3] = {c0[0], c0[1], c0[2]};
                c[d] = q;
                is_dir = in.dirichlet[fine(e, c[0], c[1], c[2])] != 0;
              }
            } else if (nend == 1) {
              const int f = end[0] ? 0 : (end[1] ? 1 : 2);
              const int d1 = f == 0 ? 1 : 0, d2 = f == 2 ? 1 : 2;
              int64_t C[2][2];
              for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v) {
                  int c[3];
                  c[f] = fend(idx[f]);
                  c[d1] = u ? Nf : 0;
                  c[d2] = v ? Nf : 0;
                  C[u][v] = fine(e, c[0], c[1], c[2]);
                }
              int u0 = 0, v0 = 0;
              for (int u = 0; u < 2; ++u)
                for (int v = 0; v < 2; ++v)
                  if (C[u][v] < C[u0][v0]) {
                    u0 = u;
                    v0 = v;
                  }
              const int a1 = u0 == 0 ? idx[d1] : Nt - idx[d1];
              const int a2 = v0 == 0 ? idx[d2] : Nt - idx[d2];
              const bool first = C[1 - u0][v0] < C[u0][1 - v0];
              std::array<int64_t, 4> s = {C[0][0], C[0][1], C[1][0], C[1][1]};
              std::sort(s.begin(), s.end());
              key = {2, s[0], s[1], s[2], s[3], first ? a1 : a2, first ? a2 : a1};
              is_dir = true;
              for (int q1 = 0; q1 < Qf && is_dir; ++q1)
                for (int q2 = 0; q2 < Qf && is_dir; ++q2) {
                  int c[3];
                  c[f] = fend(idx[f]);
                  c[d1] = q1;
                  c[d2] = q2;
                  is_dir = in.dirichlet[fine(e, c[0], c[1], c[2])] != 0;
                }
            } else {
              key = {3, e, i, j, k, 0, 0};
            }
            auto it = map.find(key);
            int64_t g;
            if (it == map.end()) {
              g = (int64_t)map.size();
              map.emplace(key, g);
              dir.push_back(is_dir ? 1 : 0);
            } else {
              g = it->second;
              if (is_dir) dir[g] = 1;
            }
            ids[(size_t)e * NP + (k * Q + j) * Q + i] = g;
          }
    L.n = (int64_t)map.size();
  }
  if (L.n >= (int64_t)kGidMask) {
    err = "mesh too large for 30-bit global ids";
    return false;
  }
  L.dirichlet = dir;
  L.gid.assign((size_t)in.E * NP, 0u);
  {
    std::vector<uint8_t> seen((size_t)L.n, 0);
    for (size_t q = 0; q < ids.size(); ++q) {
      const int64_t g = ids[q];
      uint32_t id = (uint32_t)g;
      if (dir[g]) id |= kGidDirichlet;
      if (!seen[g]) {
        seen[g] = 1;
        id |= kGidOwner;
      }
      L.gid[q] = id;
    }
    for (int64_t g = 0; g < L.n; ++g)
      if (!seen[g]) {
        err = "a global id is used by no element";
        return false;
      }
  }
  // geometric factors from the coordinates (derivatives by the GLL differentiation matrix) and
  // the element diagonals
  L.G.assign((size_t)in.E * 6 * NP, 0.0);
  L.diag.assign((size_t)L.n, 0.0);
  std::vector<double> diag_local((size_t)in.E * NP, 0.0);
  double minJ = 1e300;
  const double* D = L.Dm.data();
#pragma omp parallel for schedule(static) reduction(min : minJ)
  for (int64_t e = 0; e < in.E; ++e) {
    const double* Xe = &X[(size_t)e * NP * 3];
    double* G = &L.G[(size_t)e * 6 * NP];
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i) {
          const int p = (k * Q + j) * Q + i;
          double Jm[3][3] = {{0}};
          for (int q = 0; q < Q; ++q)
            for (int l = 0; l < 3; ++l) {
              Jm[l][0] += D[i * Q + q] * Xe[((k * Q + j) * Q + q) * 3 + l];
              Jm[l][1] += D[j * Q + q] * Xe[((k * Q + q) * Q + i) * 3 + l];
              Jm[l][2] += D[k * Q + q] * Xe[((q * Q + j) * Q + i) * 3 + l];
            }
          const double det = point_factors(Jm, L.w[i] * L.w[j] * L.w[k], G + p, NP);
          minJ = std::min(minJ, det);
        }
    for (int k = 0; k < Q; ++k)
      for (int j = 0; j < Q; ++j)
        for (int i = 0; i < Q; ++i) {
          const int p = (k * Q + j) * Q + i;
          double acc = 0.0;
          for (int l = 0; l < Q; ++l) {
            acc += G[0 * NP + (k * Q + j) * Q + l] * D[l * Q + i] * D[l * Q + i];
            acc += G[3 * NP + (k * Q + l) * Q + i] * D[l * Q + j] * D[l * Q + j];
            acc += G[5 * NP + (l * Q + j) * Q + i] * D[l * Q + k] * D[l * Q + k];
          }
          const double di = D[i * Q + i], dj = D[j * Q + j], dk = D[k * Q + k];
          acc += 2.0 * (G[1 * NP + p] * di * dj + G[2 * NP + p] * di * dk + G[4 * NP + p] * dj * dk);
          diag_local[(size_t)e * NP + p] = acc;
        }
  }
  L.min_jacobian = minJ;
  if (!(minJ > 0.0)) {
    err = "mesh has a non-positive Jacobian";
    return false;
  }
  for (size_t q = 0; q < diag_local.size(); ++q) {
    const uint32_t id = L.gid[q];
    if (!(id & kGidDirichlet)) L.diag[id & kGidMask] += diag_local[q];
  }
  return true;
}

}  // namespace chebmg
