// Donor search on a 3D curvilinear mesh (Sec. 2.2: donor-receiver pairing, weights from the
// Lagrange shape functions): for each point, computational coordinates (s, r, t) with
// X(s, r, t) = p, X the mesh map interpolated by the 4 x 4 x 4 Lagrange basis on the stencil
// starting at floor(.) - 1 clamped into the mesh, by Newton's method from a nearby node (points
// outside the mesh's padded bounding box are refused without a search, points the iteration
// places outside the mesh without a second search); the
// weights are that basis at the solution. Hole cut (reading, as for the Cartesian 3D hole cut
// with the overlapping mesh's index units): a point inside the mesh more than a margin of index
// units from each of its faces is a hole. Host only: no device calls.
#include <algorithm>
#include <cmath>
#include <string>

#include "sbp_system.h"

namespace {

// Cubic Lagrange basis on the nodes 0..3 at u, and its derivative.
void cubic_basis(double u, double l[4], double dl[4]) {
  const double a = u, b = u - 1.0, c = u - 2.0, d = u - 3.0;
  l[0] = b * c * d / -6.0;
  l[1] = a * c * d / 2.0;
  l[2] = a * b * d / -2.0;
  l[3] = a * b * c / 6.0;
  dl[0] = (c * d + b * d + b * c) / -6.0;
  dl[1] = (c * d + a * d + a * c) / 2.0;
  dl[2] = (b * d + a * d + a * b) / -2.0;
  dl[3] = (b * c + a * c + a * b) / 6.0;
}

int first_node(double s, int n) { return std::max(0, std::min(n - 4, (int)std::floor(s) - 1)); }

struct Grid3 {
  int n[3];
  const double *X[3];
  size_t at(int i, int j, int k) const { return ((size_t)k * n[1] + j) * n[0] + i; }
  double dist2(size_t p, const double *q) const {
    const double dx = X[0][p] - q[0], dy = X[1][p] - q[1], dz = X[2][p] - q[2];
    return dx * dx + dy * dy + dz * dz;
  }
};

// A node near q: the nearest among every stride-th node of each line (and the last), then,
// halving the stride, the nearest within the previous stride of the node found, down to stride 1.
// (With stride 1 from the start, the nearest of all nodes.)
void near_node(const Grid3 &g, const double *q, int stride, int c[3]) {
  double best = INFINITY;
  auto scan = [&](int lo0, int hi0, int lo1, int hi1, int lo2, int hi2, int st) {
    int found[3] = {c[0], c[1], c[2]};
    for (int k = lo2; k <= hi2; k = (k == hi2) ? hi2 + 1 : std::min(k + st, hi2))
      for (int j = lo1; j <= hi1; j = (j == hi1) ? hi1 + 1 : std::min(j + st, hi1))
        for (int i = lo0; i <= hi0; i = (i == hi0) ? hi0 + 1 : std::min(i + st, hi0)) {
          const double d = g.dist2(g.at(i, j, k), q);
          if (d < best) {
            best = d;
            found[0] = i;
            found[1] = j;
            found[2] = k;
          }
        }
    c[0] = found[0];
    c[1] = found[1];
    c[2] = found[2];
  };
  c[0] = c[1] = c[2] = 0;
  scan(0, g.n[0] - 1, 0, g.n[1] - 1, 0, g.n[2] - 1, stride);
  while (stride > 1) {
    const int next = std::max(1, stride / 2);
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::max(0, c[a] - stride);
      hi[a] = std::min(g.n[a] - 1, c[a] + stride);
    }
    scan(lo[0], hi[0], lo[1], hi[1], lo[2], hi[2], next);
    stride = next;
  }
}

// Axis-aligned box of all nodes, padded by the longest edge between neighbouring nodes: the
// Lagrange-interpolated mesh map does not reach beyond it on meshes whose cells are not folded,
// so a point outside it is outside the mesh and needs no search.
struct Box {
  double lo[3], hi[3];
  bool contains(const double *q) const {
    for (int a = 0; a < 3; ++a)
      if (!(q[a] >= lo[a] && q[a] <= hi[a])) return false;
    return true;
  }
};

Box padded_box(const Grid3 &g) {
  Box b;
  for (int a = 0; a < 3; ++a) {
    b.lo[a] = INFINITY;
    b.hi[a] = -INFINITY;
  }
  double edge2 = 0.0;
  for (int k = 0; k < g.n[2]; ++k)
    for (int j = 0; j < g.n[1]; ++j)
      for (int i = 0; i < g.n[0]; ++i) {
        const size_t p = g.at(i, j, k);
        for (int a = 0; a < 3; ++a) {
          b.lo[a] = std::min(b.lo[a], g.X[a][p]);
          b.hi[a] = std::max(b.hi[a], g.X[a][p]);
        }
        const int nb[3][3] = {{i + 1, j, k}, {i, j + 1, k}, {i, j, k + 1}};
        for (int d = 0; d < 3; ++d) {
          if (nb[d][d] >= g.n[d]) continue;
          const size_t r = g.at(nb[d][0], nb[d][1], nb[d][2]);
          const double q[3] = {g.X[0][r], g.X[1][r], g.X[2][r]};
          edge2 = std::max(edge2, g.dist2(p, q));
        }
      }
  const double pad = std::sqrt(edge2);
  for (int a = 0; a < 3; ++a) {
    b.lo[a] -= pad;
    b.hi[a] += pad;
  }
  return b;
}

// The verdict on an iteration that did not converge at s: 0 (outside the mesh) when the iterate
// has left the index range by more than one cell, else -1 (retry from another start).
int failed_at(const Grid3 &g, const double s[3]) {
  for (int a = 0; a < 3; ++a)
    if (!(s[a] >= -1.0 && s[a] <= g.n[a])) return 0;
  return -1;
}

// Newton's method on the interpolated map from s: 1 when three consecutive steps stay below
// 1e-10 (the rounding floor follows two steps after the first small one) inside the mesh, 0
// when they do so outside it, or when the iteration fails (a singular Jacobian, divergence, no
// convergence in 100 steps) with the iterate more than a cell outside (the point is outside
// the mesh), -1 when it fails inside.
int newton(const Grid3 &g, const double *q, double s[3]) {
  int small = 0;
  for (int it = 0; it < 100 && small < 3; ++it) {
    int b[3];
    double l[3][4], dl[3][4];
    for (int a = 0; a < 3; ++a) {
      b[a] = first_node(s[a], g.n[a]);
      cubic_basis(s[a] - b[a], l[a], dl[a]);
    }
    double F[3] = {0, 0, 0}, Jm[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int c = 0; c < 4; ++c)
      for (int e = 0; e < 4; ++e)
        for (int d = 0; d < 4; ++d) {
          const size_t p = g.at(b[0] + d, b[1] + e, b[2] + c);
          const double w = l[0][d] * l[1][e] * l[2][c];
          const double wd[3] = {dl[0][d] * l[1][e] * l[2][c], l[0][d] * dl[1][e] * l[2][c],
                                l[0][d] * l[1][e] * dl[2][c]};
          for (int x = 0; x < 3; ++x) {
            const double v = g.X[x][p];
            F[x] += w * v;
            for (int a = 0; a < 3; ++a) Jm[x][a] += wd[a] * v;
          }
        }
    for (int x = 0; x < 3; ++x) F[x] -= q[x];
    // Cramer's rule for Jm step = F
    const double det = Jm[0][0] * (Jm[1][1] * Jm[2][2] - Jm[1][2] * Jm[2][1]) -
                       Jm[0][1] * (Jm[1][0] * Jm[2][2] - Jm[1][2] * Jm[2][0]) +
                       Jm[0][2] * (Jm[1][0] * Jm[2][1] - Jm[1][1] * Jm[2][0]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return failed_at(g, s);
    double step[3];
    for (int a = 0; a < 3; ++a) {
      double M[3][3];
      for (int r = 0; r < 3; ++r)
        for (int cc = 0; cc < 3; ++cc) M[r][cc] = (cc == a) ? F[r] : Jm[r][cc];
      step[a] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                 M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) /
                det;
    }
    bool tiny = true;
    for (int a = 0; a < 3; ++a) {
      s[a] -= step[a];
      if (!(std::fabs(s[a]) < 1e7)) return 0;  // diverged (or not finite): far outside the mesh
      tiny = tiny && std::fabs(step[a]) < 1e-10;
    }
    small = tiny ? small + 1 : 0;
  }
  if (small < 3) return failed_at(g, s);
  for (int a = 0; a < 3; ++a)
    if (s[a] < -1e-9 || s[a] > g.n[a] - 1 + 1e-9) return 0;
  return 1;
}

// Computational coordinates of q by Newton's method from a nearby node; false for points
// outside the padded box without any search, and for points the iteration places outside the
// mesh. Only when the iteration fails inside the mesh is it retried, from the nearest of all
// nodes.
bool locate(const Grid3 &g, const Box &box, int stride, const double *q, double s[3]) {
  if (!box.contains(q)) return false;
  int c[3];
  near_node(g, q, stride, c);
  for (int a = 0; a < 3; ++a) s[a] = c[a];
  const int r = newton(g, q, s);
  if (r >= 0) return r == 1;
  if (stride == 1) return false;
  near_node(g, q, 1, c);
  for (int a = 0; a < 3; ++a) s[a] = c[a];
  return newton(g, q, s) == 1;
}

}  // namespace

extern "C" sbp_status sbp3c_donor_search(const int *n, const double *x, const double *y, const double *z,
                                         const signed char *iblank, int npts, const double *pts, int *base,
                                         double *w, double *xi, int *first_failed) {
  if (first_failed) *first_failed = -1;
  if (!n || !x || !y || !z || npts < 0 || (npts > 0 && (!pts || !base || !w)))
    return sbp::fail(SBP_ERR_ARG, "null argument");
  for (int a = 0; a < 3; ++a)
    if (n[a] < 8 || n[a] > 65535) return sbp::fail(SBP_ERR_SHAPE, "each direction needs 8..65535 points");
  const Grid3 g{{n[0], n[1], n[2]}, {x, y, z}};
  const int stride = std::max(1, std::min({n[0], n[1], n[2]}) / 8);
  const Box box = padded_box(g);
  for (int t = 0; t < npts; ++t) {
    const double *q = pts + 3 * (size_t)t;
    double s[3];
    bool ok = locate(g, box, stride, q, s);
    int b[3] = {0, 0, 0};
    for (int a = 0; ok && a < 3; ++a) b[a] = first_node(s[a], n[a]);
    for (int cc = 0; ok && iblank && cc < 4; ++cc)
      for (int e = 0; ok && e < 4; ++e)
        for (int d = 0; ok && d < 4; ++d)
          if (!iblank[g.at(b[0] + d, b[1] + e, b[2] + cc)]) ok = false;
    if (!ok) {
      if (first_failed) *first_failed = t;
      return sbp::fail(SBP_ERR_DONOR, "no valid donor stencil for point " + std::to_string(t) + " at (" +
                                          std::to_string(q[0]) + ", " + std::to_string(q[1]) + ", " +
                                          std::to_string(q[2]) + ")");
    }
    for (int a = 0; a < 3; ++a) {
      double l[4], dl[4];
      cubic_basis(s[a] - b[a], l, dl);
      base[3 * (size_t)t + a] = b[a];
      for (int d = 0; d < 4; ++d) w[12 * (size_t)t + 4 * a + d] = l[d];
      if (xi) xi[3 * (size_t)t + a] = s[a];
    }
  }
  return SBP_OK;
}

extern "C" sbp_status sbp3c_hole_cut(const int *n, const double *x, const double *y, const double *z, int npts,
                                     const double *pts, double margin, signed char *iblank) {
  if (!n || !x || !y || !z || npts < 0 || (npts > 0 && (!pts || !iblank)) || !(margin >= 0.0))
    return sbp::fail(SBP_ERR_ARG, "bad argument");
  for (int a = 0; a < 3; ++a)
    if (n[a] < 8 || n[a] > 65535) return sbp::fail(SBP_ERR_SHAPE, "each direction needs 8..65535 points");
  const Grid3 g{{n[0], n[1], n[2]}, {x, y, z}};
  const int stride = std::max(1, std::min({n[0], n[1], n[2]}) / 8);
  const Box box = padded_box(g);
  for (int t = 0; t < npts; ++t) {
    const double *q = pts + 3 * (size_t)t;
    double s[3];
    bool ok = locate(g, box, stride, q, s);
    for (int a = 0; ok && a < 3; ++a) ok = s[a] > margin && s[a] < n[a] - 1 - margin;
    if (ok) iblank[t] = 0;
  }
  return SBP_OK;
}
