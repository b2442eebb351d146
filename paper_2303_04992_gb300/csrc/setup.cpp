// Host setup of the KFBI matvec (Alg. 1 step 1; tables for Secs. 4.3-4.4).
//
// Everything here runs once per geometry.  It produces, for the device:
//   * the control points (Gamma x grid lines of each u^(c) grid, Sec. 3) with
//     the primary/secondary split (primary: the line is the most normal of the
//     three directions at the point, |n_a| >= max_b |n_b| - 1e-12);
//   * surface-fit weights: a weighted least-squares quadratic in tangent-plane
//     coordinates over the primary points of X_c' whose segment midpoints lie
//     within 3h (integer test on half-spacing keys), weights exp(-|z-y|^2/h^2);
//   * the linear jump map at each point: fitted tangential derivatives of the
//     density and f at the point -> [grad u^(c)], [Hess u^(c)], [p], [d_a p]
//     from the first-order relations A tau_a = d_a phi, tr A = 0,
//     [sigma n] = 0 and the 21 second-order relations (tangential second
//     derivatives of [u] = phi on the curved surface, grad [div u] = 0,
//     the momentum jump IUS-1 and the tangential derivative of IUS-4);
//   * Navier (Lame): c = 1/(lambda + mu) enters grad [div u + c p] = 0 and the
//     elastic traction -kappa p I + mu (grad u + grad u^T), kappa = lambda c;
//     first order A n = -(lambda/(lambda + 2 mu)) D n - ..., q = -(lambda + mu) tr A;
//   * the right-hand-side correction matrix (Sec. 4.3 items 1-4, one rule
//     C_P += a_PQ chi_Q J(Q) for every stencil neighbour Q across Gamma);
//   * the ten-node quadratic interpolation rows of the trace (Sec. 4.4).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <tuple>

#include "internal.h"

namespace kfbim {
namespace {  // file-local helpers

// ---------------------------------------------------------------- level sets
struct Level {
  const kfbim_geometry& g;
  // F, gradient (3), Hessian (9, row-major); G and H nullable.
  void eval(const double* x, double* F, double* G, double* H) const {
    if (g.kind == KFBIM_CALLBACK) {
      *F = g.F(x, g.user);
      if (G || H) {
        double gg[3], hh[9];
        g.derivs(x, gg, hh, g.user);
        if (G) std::memcpy(G, gg, sizeof(gg));
        if (H) std::memcpy(H, hh, sizeof(hh));
      }
      return;
    }
    const double d0 = x[0] - g.center[0], d1 = x[1] - g.center[1], d2 = x[2] - g.center[2];
    if (g.kind == KFBIM_SPHERE) {
      const double r = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      *F = r - g.params[0];
      if (G || H) {
        const double e[3] = {d0 / r, d1 / r, d2 / r};
        if (G) for (int i = 0; i < 3; ++i) G[i] = e[i];
        if (H)
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) H[3 * i + j] = ((i == j) - e[i] * e[j]) / r;
      }
      return;
    }
    if (g.kind == KFBIM_ELLIPSOID) {
      const double* Q = g.rot;  // row-major; xi = Q^T d
      double xi[3], w[3];
      for (int a = 0; a < 3; ++a) xi[a] = Q[0 * 3 + a] * d0 + Q[1 * 3 + a] * d1 + Q[2 * 3 + a] * d2;
      double f = -1.0;
      for (int a = 0; a < 3; ++a) {
        const double s = g.params[a];
        f += (xi[a] / s) * (xi[a] / s);
        w[a] = 2.0 / (s * s);
      }
      *F = f;
      if (G)
        for (int i = 0; i < 3; ++i) {
          double acc = 0;
          for (int a = 0; a < 3; ++a) acc += Q[i * 3 + a] * w[a] * xi[a];
          G[i] = acc;
        }
      if (H)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int a = 0; a < 3; ++a) acc += Q[i * 3 + a] * w[a] * Q[j * 3 + a];
            H[3 * i + j] = acc;
          }
      return;
    }
    if (g.kind == KFBIM_TORUS) {
      // F = (c - s)^2 + z^2 - a^2, s = distance from the z axis (Example 5.3);
      // with e = (x, y) / s: grad F = (-2 (c - s) e, 2 z),
      // Hess F on the (x, y) block = 2 e e^T - 2 (c - s) / s (I - e e^T), zz = 2.
      const double a = g.params[0], c = g.params[1];
      const double s = std::sqrt(d0 * d0 + d1 * d1);
      *F = (c - s) * (c - s) + d2 * d2 - a * a;
      const double e[2] = {d0 / s, d1 / s};
      if (G) {
        G[0] = -2.0 * (c - s) * e[0];
        G[1] = -2.0 * (c - s) * e[1];
        G[2] = 2.0 * d2;
      }
      if (H) {
        for (int i = 0; i < 9; ++i) H[i] = 0.0;
        for (int i = 0; i < 2; ++i)
          for (int j = 0; j < 2; ++j)
            H[3 * i + j] = 2.0 * e[i] * e[j] - 2.0 * (c - s) / s * ((i == j) - e[i] * e[j]);
        H[8] = 2.0;
      }
      return;
    }
    // STAR: F = rho - R(theta, phi), chain rule through spherical coordinates.
    const double r0 = g.params[0], eps = g.params[1], m = g.params[2], n = g.params[3];
    const double s = std::sqrt(d0 * d0 + d1 * d1);
    const double rho = std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    const double th = std::atan2(s, d2), ph = std::atan2(d1, d0);
    const double sm = std::sin(m * th), cm = std::cos(m * th);
    const double sn = std::sin(n * ph), cn = std::cos(n * ph);
    *F = rho - (r0 + eps * sm * cn);
    if (!G && !H) return;
    const double st = std::sin(th), ct = std::cos(th), sp = std::sin(ph), cp = std::cos(ph);
    const double Rt = eps * m * cm * cn, Rp = -eps * n * sm * sn;
    const double er[3] = {st * cp, st * sp, ct};
    const double et[3] = {ct * cp, ct * sp, -st};
    const double ep[3] = {-sp, cp, 0.0};
    double gt[3], gp[3];
    for (int i = 0; i < 3; ++i) {
      gt[i] = et[i] / rho;
      gp[i] = ep[i] / (rho * st);
    }
    if (G)
      for (int i = 0; i < 3; ++i) G[i] = er[i] - Rt * gt[i] - Rp * gp[i];
    if (H) {
      const double Rtt = -eps * m * m * sm * cn, Rtp = -eps * m * n * cm * sn,
                   Rpp = -eps * n * n * sm * cn;
      double w[3];
      for (int i = 0; i < 3; ++i) w[i] = st * er[i] + ct * et[i];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const double hr = ((i == j) - er[i] * er[j]) / rho;
          const double hth = (-er[i] * et[j] - et[i] * er[j] + (ct / st) * ep[i] * ep[j]) / (rho * rho);
          const double hph = -(w[i] * ep[j] + ep[i] * w[j]) / (rho * rho * st * st);
          H[3 * i + j] = hr - Rt * hth - Rp * hph - Rtt * gt[i] * gt[j] -
                         Rtp * (gt[i] * gp[j] + gp[i] * gt[j]) - Rpp * gp[i] * gp[j];
        }
    }
  }
  double value(const double* x) const {
    double F;
    eval(x, &F, nullptr, nullptr);
    return F;
  }
};

// ------------------------------------------------- small dense linear algebra
// In-place LU with partial pivoting of an n x n row-major matrix.
bool lu_factor(double* A, int n, int* piv) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = std::fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[i * n + k]) > best) { best = std::fabs(A[i * n + k]); p = i; }
    if (!(best > 0.0)) return false;
    piv[k] = p;
    if (p != k)
      for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[p * n + j]);
    const double inv = 1.0 / A[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double l = A[i * n + k] * inv;
      A[i * n + k] = l;
      for (int j = k + 1; j < n; ++j) A[i * n + j] -= l * A[k * n + j];
    }
  }
  return true;
}

void lu_solve(const double* LU, int n, const int* piv, double* b) {
  // all row interchanges first (they were applied to whole rows of L too)
  for (int k = 0; k < n; ++k)
    if (piv[k] != k) std::swap(b[k], b[piv[k]]);
  for (int k = 0; k < n; ++k)
    for (int i = k + 1; i < n; ++i) b[i] -= LU[i * n + k] * b[k];
  for (int k = n - 1; k >= 0; --k) {
    double acc = b[k];
    for (int j = k + 1; j < n; ++j) acc -= LU[k * n + j] * b[j];
    b[k] = acc / LU[k * n + k];
  }
}

// Order of the six independent Hessian entries: 11, 22, 33, 23, 13, 12.
int hidx(int k, int l) {
  if (k > l) std::swap(k, l);
  if (k == l) return k;
  if (k == 1 && l == 2) return 3;
  if (k == 0 && l == 2) return 4;
  return 5;
}

struct Frame {
  double n[3], t[2][3], K[2][2];
};

Frame make_frame(const Level& lev, const double* x) {
  double F, G[3], H[9];
  lev.eval(x, &F, G, H);
  const double gn = std::sqrt(G[0] * G[0] + G[1] * G[1] + G[2] * G[2]);
  Frame f;
  for (int i = 0; i < 3; ++i) f.n[i] = G[i] / gn;
  int m = 0;  // least aligned axis, first on ties
  for (int i = 1; i < 3; ++i)
    if (std::fabs(f.n[i]) < std::fabs(f.n[m])) m = i;
  double e[3] = {0, 0, 0};
  e[m] = 1.0;
  const double dot = f.n[m];
  double t1[3], nt = 0;
  for (int i = 0; i < 3; ++i) { t1[i] = e[i] - dot * f.n[i]; nt += t1[i] * t1[i]; }
  nt = std::sqrt(nt);
  for (int i = 0; i < 3; ++i) f.t[0][i] = t1[i] / nt;
  f.t[1][0] = f.n[1] * f.t[0][2] - f.n[2] * f.t[0][1];
  f.t[1][1] = f.n[2] * f.t[0][0] - f.n[0] * f.t[0][2];
  f.t[1][2] = f.n[0] * f.t[0][1] - f.n[1] * f.t[0][0];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double acc = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) acc += f.t[a][i] * H[3 * i + j] * f.t[b][j];
      f.K[a][b] = acc / gn;
    }
  return f;
}

// First-order jumps A (3x3, A[c][j] = [d_j u^(c)]) and q = [p] from the
// tangential derivatives dphi[c][a] of the density components (lam < 0: Stokes).
void first_order(const Frame& f, const double dphi[3][2], double mu, double lam, double A[3][3],
                 double* q) {
  double D = 0;
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 3; ++c) D += f.t[a][c] * dphi[c][a];
  double nd[2] = {0, 0};
  for (int a = 0; a < 2; ++a)
    for (int c = 0; c < 3; ++c) nd[a] += f.n[c] * dphi[c][a];
  const double Ann = lam < 0 ? -D : -D * lam / (lam + 2.0 * mu);
  double An[3];
  for (int c = 0; c < 3; ++c) An[c] = Ann * f.n[c] - nd[0] * f.t[0][c] - nd[1] * f.t[1][c];
  for (int c = 0; c < 3; ++c)
    for (int j = 0; j < 3; ++j)
      A[c][j] = dphi[c][0] * f.t[0][j] + dphi[c][1] * f.t[1][j] + An[c] * f.n[j];
  *q = lam < 0 ? -2.0 * mu * D : -(lam + mu) * (Ann + D);
}

// The 21 x 21 second-order system on x = (H^(1), H^(2), H^(3), s).
void second_order_matrix(const Frame& f, double mu, double lam, double* L) {
  std::memset(L, 0, sizeof(double) * 21 * 21);
  const double cpen = lam < 0 ? 0.0 : 1.0 / (lam + mu);
  const double kap = lam < 0 ? 1.0 : lam / (lam + mu);
  int row = 0;
  const int ab[3][2] = {{0, 0}, {0, 1}, {1, 1}};
  for (int c = 0; c < 3; ++c)
    for (int q = 0; q < 3; ++q, ++row)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l)
          L[row * 21 + 6 * c + hidx(k, l)] += f.t[ab[q][0]][k] * f.t[ab[q][1]][l];
  for (int j = 0; j < 3; ++j, ++row) {
    for (int c = 0; c < 3; ++c) L[row * 21 + 6 * c + hidx(c, j)] += 1.0;
    L[row * 21 + 18 + j] += cpen;
  }
  for (int c = 0; c < 3; ++c, ++row) {
    for (int k = 0; k < 3; ++k) L[row * 21 + 6 * c + hidx(k, k)] += -mu;
    L[row * 21 + 18 + c] += 1.0;
  }
  for (int a = 0; a < 2; ++a)
    for (int i = 0; i < 3; ++i, ++row)
      for (int j = 0; j < 3; ++j) {
        L[row * 21 + 18 + j] += -kap * f.t[a][j] * f.n[i];
        for (int k = 0; k < 3; ++k) {
          L[row * 21 + 6 * i + hidx(k, j)] += mu * f.t[a][j] * f.n[k];
          L[row * 21 + 6 * k + hidx(i, j)] += mu * f.t[a][j] * f.n[k];
        }
      }
}

void second_order_rhs(const Frame& f, const double A[3][3], double q, const double d2[3][3],
                      const double* fy, double mu, double lam, double* rhs) {
  const double kap = lam < 0 ? 1.0 : lam / (lam + mu);
  double An[3];
  for (int c = 0; c < 3; ++c) An[c] = A[c][0] * f.n[0] + A[c][1] * f.n[1] + A[c][2] * f.n[2];
  int row = 0;
  const int ab[3][2] = {{0, 0}, {0, 1}, {1, 1}};
  for (int c = 0; c < 3; ++c)
    for (int m = 0; m < 3; ++m) rhs[row++] = d2[c][m] + f.K[ab[m][0]][ab[m][1]] * An[c];
  for (int j = 0; j < 3; ++j) rhs[row++] = 0.0;
  for (int c = 0; c < 3; ++c) rhs[row++] = fy[c];
  double sig[3][3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) sig[i][k] = (i == k ? -kap * q : 0.0) + mu * (A[i][k] + A[k][i]);
  for (int a = 0; a < 2; ++a) {
    double dn[3];
    for (int k = 0; k < 3; ++k) dn[k] = f.K[a][0] * f.t[0][k] + f.K[a][1] * f.t[1][k];
    for (int i = 0; i < 3; ++i) {
      double v = 0;
      for (int k = 0; k < 3; ++k) v += sig[i][k] * dn[k];
      rhs[row++] = -v;
    }
  }
}

inline int64_t flat(int N, int i, int j, int k) { return ((int64_t)k * N + j) * N + i; }

}  // namespace

int build_tables(const kfbim_geometry& geom, const kfbim_grid& grid, double mu, double lam,
                 HostTables& t, std::string& err) {
  const int N = grid.N;
  t.N = N;
  t.lo = grid.lo;
  t.h = (grid.hi - grid.lo) / N;
  t.mu = mu;
  const double h = t.h, lo = grid.lo;
  const int64_t N3 = (int64_t)N * N * N;
  Level lev{geom};

  // ---- sides of all grid nodes (Omega = {F <= 0})
  auto node_x = [&](int c, int i, int j, int k, double* x) {
    const int id[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) x[a] = lo + (id[a] + ((c == a + 1) ? 0.0 : 0.5)) * h;
  };
  for (int c = 0; c < 4; ++c) {
    t.side[c].assign(N3, 0);
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          double x[3];
          node_x(c, i, j, k, x);
          t.side[c][flat(N, i, j, k)] = lev.value(x) <= 0.0 ? 1 : 0;
        }
  }
  // ---- geometry checks: clearance of 3 nodes from the wall on every grid
  for (int c = 0; c < 4; ++c)
    for (int k = 0; k < N; ++k)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i < N; ++i) {
          const bool band = i < 3 || j < 3 || k < 3 || i >= N - 3 || j >= N - 3 || k >= N - 3;
          if (band && t.side[c][flat(N, i, j, k)]) {
            err = "interface closer than 3h to the box wall";
            return KFBIM_E_GEOMETRY;
          }
        }
  // A combined u^(a)/cell line may change side twice within one face segment
  // (a grazing segment: both faces on one side, the cell centre between them
  // on the other); its two roots become control points below.

  // ---- control points: component c, line axis a, outer/inner line index, position
  for (int c = 1; c <= 3; ++c) {
    for (int a = 0; a < 3; ++a) {
      const int o0 = (a == 0) ? 1 : 0;       // lower other axis
      const int o1 = (a == 2) ? 1 : 2;       // higher other axis
      auto lo_idx = [&](int b) { return (b == c - 1) ? 1 : 0; };
      for (int u = lo_idx(o1); u < N; ++u)
        for (int v = lo_idx(o0); v < N; ++v)
          for (int s = lo_idx(a); s + 1 < N; ++s) {
            int id0[3], id1[3];
            id0[a] = s;
            id0[o0] = v;
            id0[o1] = u;
            std::memcpy(id1, id0, sizeof(id0));
            id1[a] = s + 1;
            const int s0 = t.side[c][flat(N, id0[0], id0[1], id0[2])];
            const int s1 = t.side[c][flat(N, id1[0], id1[1], id1[2])];
            const bool graze = s0 == s1 && c == a + 1 && t.side[0][flat(N, id0[0], id0[1], id0[2])] != s0;
            if (s0 == s1 && !graze) continue;
            double x0[3];
            node_x(c, id0[0], id0[1], id0[2], x0);
            // root of F on [t0, t1] of the segment by 64 bisection steps; side0 at t0
            auto add_root = [&](double lo_t, double hi_t, int side0, int8_t gflag) {
              for (int it = 0; it < 64; ++it) {
                const double mid = 0.5 * (lo_t + hi_t);
                double x[3] = {x0[0], x0[1], x0[2]};
                x[a] = x0[a] + mid * h;
                const int sm = lev.value(x) <= 0.0 ? 1 : 0;
                if (sm == side0) lo_t = mid; else hi_t = mid;
              }
              t.comp.push_back(c);
              t.axis.push_back(a);
              for (int b = 0; b < 3; ++b) t.idx.push_back(id0[b]);
              t.theta.push_back(lo_t);
              t.graze.push_back(gflag);
              double x[3] = {x0[0], x0[1], x0[2]};
              x[a] += lo_t * h;
              for (int b = 0; b < 3; ++b) t.xyz.push_back(x[b]);
            };
            if (!graze) {
              add_root(0.0, 1.0, s0, 0);
            } else {  // once below and once above the cell centre
              add_root(0.0, 0.5, s0, 1);
              add_root(0.5, 1.0, 1 - s0, 2);
            }
          }
    }
  }
  const int64_t n = (int64_t)t.comp.size();
  t.n_all = n;
  if (n == 0) {
    err = "interface does not cross the grid";
    return KFBIM_E_GEOMETRY;
  }
  std::vector<Frame> fr(n);
  t.normal.assign(3 * n, 0.0);
  t.primary.assign(n, 0);
  t.pid.assign(n, -1);
  for (int64_t y = 0; y < n; ++y) {
    fr[y] = make_frame(lev, &t.xyz[3 * y]);
    bool finite = true;
    for (int i = 0; i < 3; ++i) finite = finite && std::isfinite(fr[y].n[i]);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) finite = finite && std::isfinite(fr[y].K[a][b]);
    if (!finite) {
      err = "level-set gradient vanishes or is not finite at a control point";
      return KFBIM_E_GEOMETRY;
    }
    const double* nn = fr[y].n;
    for (int i = 0; i < 3; ++i) t.normal[3 * y + i] = nn[i];
    const double mx = std::max(std::fabs(nn[0]), std::max(std::fabs(nn[1]), std::fabs(nn[2])));
    // the roots of a grazing segment (line nearly tangent to Gamma) are secondary
    if (t.graze[y] == 0 && std::fabs(nn[t.axis[y]]) >= mx - 1e-12) {
      t.primary[y] = 1;
      t.pid[y] = (int32_t)t.n_prim++;
    }
  }

  // ---- neighbour search on integer half-spacing keys (segment midpoints)
  std::vector<int32_t> key(3 * n);
  for (int64_t y = 0; y < n; ++y)
    for (int b = 0; b < 3; ++b)
      key[3 * y + b] = 2 * t.idx[3 * y + b] + ((b == t.comp[y] - 1) ? 0 : 1) + (b == t.axis[y] ? 1 : 0);
  const int B = (2 * N + 2) / 8 + 1;  // buckets of 8 half-spacings
  std::vector<std::vector<int32_t>> bucket((size_t)3 * B * B * B);
  auto bid = [&](int c, int bx, int by, int bz) { return (((size_t)c * B + bz) * B + by) * B + bx; };
  for (int64_t y = 0; y < n; ++y)
    if (t.primary[y])
      bucket[bid(t.comp[y] - 1, key[3 * y] / 8, key[3 * y + 1] / 8, key[3 * y + 2] / 8)].push_back((int32_t)y);
  const int R2 = 36;

  t.fit_ptr.assign(3 * n + 1, 0);
  std::vector<int32_t> nb;
  std::vector<double> V, W;
  for (int64_t y = 0; y < n; ++y) {
    const Frame& f = fr[y];
    const int kx = key[3 * y], ky = key[3 * y + 1], kz = key[3 * y + 2];
    for (int cc = 0; cc < 3; ++cc) {
      nb.clear();
      for (int bz = kz / 8 - 1; bz <= kz / 8 + 1; ++bz)
        for (int by = ky / 8 - 1; by <= ky / 8 + 1; ++by)
          for (int bx = kx / 8 - 1; bx <= kx / 8 + 1; ++bx) {
            if (bx < 0 || by < 0 || bz < 0 || bx >= B || by >= B || bz >= B) continue;
            for (int32_t z : bucket[bid(cc, bx, by, bz)]) {
              const int dx = key[3 * z] - kx, dy = key[3 * z + 1] - ky, dz = key[3 * z + 2] - kz;
              if (dx * dx + dy * dy + dz * dz <= R2) nb.push_back(z);
            }
          }
      std::sort(nb.begin(), nb.end());
      const int m = (int)nb.size();
      if (m < 12) {
        err = "too few neighbours for the surface fit (interface under-resolved)";
        return KFBIM_E_GEOMETRY;
      }
      // weighted normal equations on the basis 1, s, t, s^2, st, t^2 (s, t in units of h)
      double A[36] = {0};
      V.assign(6 * m, 0.0);
      W.assign(m, 0.0);
      for (int e = 0; e < m; ++e) {
        const int32_t z = nb[e];
        double d[3];
        for (int b = 0; b < 3; ++b) d[b] = (t.xyz[3 * z + b] - t.xyz[3 * y + b]) / h;
        const double s = d[0] * f.t[0][0] + d[1] * f.t[0][1] + d[2] * f.t[0][2];
        const double tt = d[0] * f.t[1][0] + d[1] * f.t[1][1] + d[2] * f.t[1][2];
        const double w = std::exp(-(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]));
        const double row[6] = {1.0, s, tt, s * s, s * tt, tt * tt};
        for (int i = 0; i < 6; ++i) V[6 * e + i] = row[i];
        W[e] = w;
        for (int i = 0; i < 6; ++i)
          for (int j = 0; j < 6; ++j) A[6 * i + j] += w * row[i] * row[j];
      }
      int piv[6];
      if (!lu_factor(A, 6, piv)) {
        err = "singular surface fit";
        return KFBIM_E_GEOMETRY;
      }
      for (int e = 0; e < m; ++e) {
        double r[6];
        for (int i = 0; i < 6; ++i) r[i] = W[e] * V[6 * e + i];
        lu_solve(A, 6, piv, r);   // column e of (V^T W V)^{-1} V^T W
        t.fit_col.push_back(t.pid[nb[e]]);
        t.fit_w.push_back(r[0]);
        t.fit_w.push_back(r[1] / h);
        t.fit_w.push_back(r[2] / h);
        t.fit_w.push_back(2.0 * r[3] / (h * h));
        t.fit_w.push_back(r[4] / (h * h));
        t.fit_w.push_back(2.0 * r[5] / (h * h));
      }
      t.fit_ptr[3 * y + cc + 1] = (int64_t)t.fit_col.size();
    }
  }

  // ---- jump map per point (linear in the 15 surface derivatives and f)
  t.jmap.assign((size_t)n * kMapOut * kMapIn, 0.0);
  for (int64_t y = 0; y < n; ++y) {
    const Frame& f = fr[y];
    double L[21 * 21];
    int piv[21];
    second_order_matrix(f, mu, lam, L);
    if (!lu_factor(L, 21, piv)) {
      err = "singular jump system";
      return KFBIM_E_GEOMETRY;
    }
    const int c = t.comp[y] - 1, a = t.axis[y];
    for (int j = 0; j < kMapIn; ++j) {
      double in[kMapIn] = {0};
      in[j] = 1.0;
      double dphi[3][2], d2[3][3], fy[3];
      for (int cc = 0; cc < 3; ++cc) {
        dphi[cc][0] = in[5 * cc + 0];
        dphi[cc][1] = in[5 * cc + 1];
        for (int q = 0; q < 3; ++q) d2[cc][q] = in[5 * cc + 2 + q];
        fy[cc] = in[15 + cc];
      }
      double A[3][3], q;
      first_order(f, dphi, mu, lam, A, &q);
      double x[21];
      second_order_rhs(f, A, q, d2, fy, mu, lam, x);
      lu_solve(L, 21, piv, x);
      double out[kMapOut];
      for (int k = 0; k < 3; ++k) out[k] = A[c][k];
      for (int k = 0; k < 6; ++k) out[3 + k] = x[6 * c + k];
      out[9] = q;
      out[10] = x[18 + a];
      for (int r = 0; r < kMapOut; ++r) t.jmap[((size_t)y * kMapOut + r) * kMapIn + j] = out[r];
    }
  }

  // ---- corrections (Sec. 4.3): entries (target, slot*n + point, coefficient)
  std::vector<std::tuple<int64_t, int64_t, double>> ent;
  auto chi = [](int side) { return side ? 1.0 : -1.0; };
  for (int64_t y = 0; y < n; ++y) {
    const int c = t.comp[y], a = t.axis[y];
    int P0[3], P1[3];
    for (int b = 0; b < 3; ++b) P0[b] = P1[b] = t.idx[3 * y + b];
    P1[a] += 1;
    const double th = t.theta[y];
    const int s0 = t.side[c][flat(N, P0[0], P0[1], P0[2])];
    const int s1 = t.side[c][flat(N, P1[0], P1[1], P1[2])];
    const int64_t base = (int64_t)(c - 1) * N3;
    const int64_t tP0 = base + flat(N, P0[0], P0[1], P0[2]);
    const int64_t tP1 = base + flat(N, P1[0], P1[1], P1[2]);
    auto add_u = [&](int64_t target, double coef, double xi) {
      ent.emplace_back(target, 0 * n + y, coef);
      ent.emplace_back(target, (int64_t)(1 + a) * n + y, coef * xi);
      ent.emplace_back(target, (int64_t)(4 + a) * n + y, coef * 0.5 * xi * xi);
    };
    auto add_p = [&](int64_t target, double coef, double xi) {
      ent.emplace_back(target, (int64_t)10 * n + y, coef);
      ent.emplace_back(target, (int64_t)11 * n + y, coef * xi);
    };
    const double lap = -mu / (h * h);
    if (t.graze[y] == 0) {  // the faces of a grazing segment are on one side
      add_u(tP0, lap * chi(s1), (1.0 - th) * h);  // row P0, neighbour P1 across
      add_u(tP1, lap * chi(s0), -th * h);         // row P1, neighbour P0 across
    }
    if (c == a + 1) {
      const int sC = t.side[0][flat(N, P0[0], P0[1], P0[2])];
      const int64_t tC = 3 * N3 + flat(N, P0[0], P0[1], P0[2]);
      const double xiC = 0.5 * h - th * h;
      // a grazing segment has one root below and one above C
      const bool below = t.graze[y] ? t.graze[y] == 1 : sC == s1;
      if (below) {  // crossing between P0 and the cell centre C
        add_u(tC, (-1.0 / h) * chi(s0), -th * h);
        add_p(tP0, (1.0 / h) * chi(sC), xiC);
      } else {         // crossing between C and P1
        add_u(tC, (1.0 / h) * chi(s1), (1.0 - th) * h);
        add_p(tP1, (-1.0 / h) * chi(sC), xiC);
      }
    }
  }
  std::sort(ent.begin(), ent.end(), [](const auto& l, const auto& r) {
    return std::get<0>(l) != std::get<0>(r) ? std::get<0>(l) < std::get<0>(r)
                                            : std::get<1>(l) < std::get<1>(r);
  });
  for (size_t e = 0; e < ent.size(); ++e) {
    if (e == 0 || std::get<0>(ent[e]) != std::get<0>(ent[e - 1])) {
      t.corr_row.push_back(std::get<0>(ent[e]));
      t.corr_ptr.push_back((int64_t)t.corr_src.size());
    }
    if (!t.corr_src.empty() && e > 0 && std::get<0>(ent[e]) == std::get<0>(ent[e - 1]) &&
        std::get<1>(ent[e]) == t.corr_src.back()) {
      t.corr_coef.back() += std::get<2>(ent[e]);
      continue;
    }
    t.corr_src.push_back(std::get<1>(ent[e]));
    t.corr_coef.push_back(std::get<2>(ent[e]));
  }
  t.corr_ptr.push_back((int64_t)t.corr_src.size());

  // ---- trace interpolation at the primary points (Sec. 4.4)
  for (int64_t y = 0; y < n; ++y) {
    if (!t.primary[y]) continue;
    const int c = t.comp[y], a = t.axis[y];
    int base[3], sg[3] = {1, 1, 1};
    for (int b = 0; b < 3; ++b) base[b] = t.idx[3 * y + b];
    if (t.theta[y] >= 0.5) { base[a] += 1; sg[a] = -1; }
    int nodes[kStencil][3];
    int e = 0;
    for (int b = 0; b < 3; ++b) nodes[e][b] = base[b];
    ++e;
    for (int ax = 0; ax < 3; ++ax)
      for (int sgn = 1; sgn >= -1; sgn -= 2, ++e)
        for (int b = 0; b < 3; ++b) nodes[e][b] = base[b] + (b == ax ? sgn : 0);
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int pr = 0; pr < 3; ++pr, ++e)
      for (int b = 0; b < 3; ++b)
        nodes[e][b] = base[b] + (b == pairs[pr][0] ? sg[b] : 0) + (b == pairs[pr][1] ? sg[b] : 0);
    double Vs[kStencil * kStencil], rows[kStencil][kStencil];
    for (int i = 0; i < kStencil; ++i) {
      for (int b = 0; b < 3; ++b) {
        const int lim_lo = (b == c - 1) ? 1 : 0;
        if (nodes[i][b] < lim_lo || nodes[i][b] >= N) {
          err = "interpolation stencil leaves the grid";
          return KFBIM_E_GEOMETRY;
        }
      }
      double z[3];
      node_x(c, nodes[i][0], nodes[i][1], nodes[i][2], z);
      double d[3];
      for (int b = 0; b < 3; ++b) d[b] = z[b] - t.xyz[3 * y + b];
      const double phys[kStencil] = {1.0, d[0], d[1], d[2], 0.5 * d[0] * d[0], 0.5 * d[1] * d[1],
                                     0.5 * d[2] * d[2], d[1] * d[2], d[0] * d[2], d[0] * d[1]};
      for (int k = 0; k < kStencil; ++k) rows[i][k] = phys[k];
      for (int b = 0; b < 3; ++b) d[b] /= h;
      const double sc[kStencil] = {1.0, d[0], d[1], d[2], 0.5 * d[0] * d[0], 0.5 * d[1] * d[1],
                                   0.5 * d[2] * d[2], d[1] * d[2], d[0] * d[2], d[0] * d[1]};
      // transpose: solve V^T w = e_0 for the first row of V^{-1}
      for (int k = 0; k < kStencil; ++k) Vs[k * kStencil + i] = sc[k];
    }
    int piv[kStencil];
    if (!lu_factor(Vs, kStencil, piv)) {
      err = "singular interpolation stencil";
      return KFBIM_E_GEOMETRY;
    }
    double w[kStencil] = {1, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    lu_solve(Vs, kStencil, piv, w);
    double cj[kStencil] = {0};
    t.tr_comp.push_back(c);
    for (int i = 0; i < kStencil; ++i) {
      t.tr_node.push_back((int32_t)flat(N, nodes[i][0], nodes[i][1], nodes[i][2]));
      t.tr_w.push_back(w[i]);
      if (!t.side[c][flat(N, nodes[i][0], nodes[i][1], nodes[i][2])])
        for (int k = 0; k < kStencil; ++k) cj[k] += w[i] * rows[i][k];
    }
    for (int k = 0; k < kStencil; ++k) t.tr_cj.push_back(cj[k]);
  }
  return KFBIM_OK;
}

}  // namespace kfbim
