// Host-side setup of an overset system: hole cutting, SBP segment classes, SAT lists, donor
// search with Lagrange weights (Sec. 2.2) and the Adams-Bashforth / MRAB weight plan
// (Sec. 3.1-3.3). Runs once per system on the CPU; the per-step work runs on the GPU.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

#include "sbp_internal.h"

namespace sbp {

namespace {
int round_up(int v, int a) { return (v + a - 1) / a * a; }
}  // namespace

sbp_status setup_mesh_basic(const sbp_mesh_desc &d, MeshHost &m, std::string &err) {
  m.ni = d.n[0];
  m.nj = d.n[1];
  if (m.ni < 8 || m.nj < 8) {
    err = "mesh needs at least 8 points per direction";
    return SBP_ERR_SHAPE;
  }
  if (m.ni > 65535 || m.nj > 65535) {  // point tables pack (i, j) into 16 bits each
    err = "mesh has more than 65535 points in a direction";
    return SBP_ERR_SHAPE;
  }
  m.pitch = round_up(m.ni, 32);
  for (int k = 0; k < 2; ++k) {
    m.per[k] = d.periodic[k] ? 1 : 0;
    if (m.per[k] != (d.bc[2 * k] == SBP_BC_PERIODIC) || m.per[k] != (d.bc[2 * k + 1] == SBP_BC_PERIODIC)) {
      err = "periodic flag and face conditions disagree";
      return SBP_ERR_ARG;
    }
  }
  for (int f = 0; f < 4; ++f) {
    if (d.bc[f] < SBP_BC_PERIODIC || d.bc[f] > SBP_BC_WALL) {
      err = "unknown face condition";
      return SBP_ERR_ARG;
    }
    m.bc[f] = d.bc[f];
  }
  m.cartesian = d.cartesian ? 1 : 0;
  for (int k = 0; k < 2; ++k) {
    m.lo[k] = d.lo[k];
    m.h[k] = d.h[k];
  }
  for (int k = 0; k < 4; ++k) m.shift[k] = d.shift[k];
  size_t n = (size_t)m.ni * m.nj;
  m.x.resize(n);
  m.y.resize(n);
  if (d.x && d.y) {
    std::memcpy(m.x.data(), d.x, n * sizeof(double));
    std::memcpy(m.y.data(), d.y, n * sizeof(double));
  } else if (m.cartesian) {
    for (int j = 0; j < m.nj; ++j)
      for (int i = 0; i < m.ni; ++i) {
        m.x[(size_t)j * m.ni + i] = m.lo[0] + i * m.h[0];
        m.y[(size_t)j * m.ni + i] = m.lo[1] + j * m.h[1];
      }
  } else {
    err = "curvilinear mesh without coordinates";
    return SBP_ERR_ARG;
  }
  if (m.cartesian && !(m.h[0] > 0 && m.h[1] > 0)) {
    err = "Cartesian mesh needs positive spacing";
    return SBP_ERR_SHAPE;
  }
  m.active.assign(n, 1);
  return SBP_OK;
}

// ---------------------------------------------------------------------------------------------
// Hole cut: a background point is a hole when the fine mesh's closed outer boundary winds
// around it and the point is more than `margin` from that boundary.
namespace {
void outer_boundary(const MeshHost &f, std::vector<double> &bx, std::vector<double> &by) {
  bx.clear();
  by.clear();
  auto push = [&](int i, int j) {
    bx.push_back(f.x[(size_t)j * f.ni + i]);
    by.push_back(f.y[(size_t)j * f.ni + i]);
  };
  if (f.per[0]) {  // ring mesh: the last j line closes on itself
    for (int i = 0; i < f.ni; ++i) push(i, f.nj - 1);
    return;
  }
  for (int i = 0; i < f.ni; ++i) push(i, 0);
  for (int j = 1; j < f.nj; ++j) push(f.ni - 1, j);
  for (int i = f.ni - 2; i >= 0; --i) push(i, f.nj - 1);
  for (int j = f.nj - 2; j >= 1; --j) push(0, j);
}

// Winding number of a closed polygon around (px, py).
int winding(const std::vector<double> &bx, const std::vector<double> &by, double px, double py) {
  int wn = 0;
  size_t n = bx.size();
  for (size_t e = 0; e < n; ++e) {
    double ax = bx[e], ay = by[e], cx = bx[(e + 1) % n], cy = by[(e + 1) % n];
    double cross = (cx - ax) * (py - ay) - (px - ax) * (cy - ay);
    if (ay <= py) {
      if (cy > py && cross > 0) ++wn;
    } else {
      if (cy <= py && cross < 0) --wn;
    }
  }
  return wn;
}

double seg_dist2(double ax, double ay, double cx, double cy, double px, double py) {
  double ex = cx - ax, ey = cy - ay;
  double l2 = ex * ex + ey * ey;
  double t = l2 > 0 ? ((px - ax) * ex + (py - ay) * ey) / l2 : 0.0;
  t = std::min(1.0, std::max(0.0, t));
  double dx = px - ax - t * ex, dy = py - ay - t * ey;
  return dx * dx + dy * dy;
}
}  // namespace

sbp_status setup_holes(MeshHost &bg, const MeshHost &fine, double margin, std::string &err) {
  (void)err;
  std::vector<double> bx, by;
  outer_boundary(fine, bx, by);
  double xmin = *std::min_element(bx.begin(), bx.end()), xmax = *std::max_element(bx.begin(), bx.end());
  double ymin = *std::min_element(by.begin(), by.end()), ymax = *std::max_element(by.begin(), by.end());
  size_t nb = bx.size();
  for (size_t p = 0; p < bg.x.size(); ++p) {
    double px = bg.x[p], py = bg.y[p];
    if (px < xmin || px > xmax || py < ymin || py > ymax) continue;  // cannot be enclosed
    if (winding(bx, by, px, py) == 0) continue;
    double d2 = INFINITY;
    for (size_t e = 0; e < nb; ++e)
      d2 = std::min(d2, seg_dist2(bx[e], by[e], bx[(e + 1) % nb], by[(e + 1) % nb], px, py));
    if (std::sqrt(d2) > margin) bg.active[p] = 0;
  }
  return SBP_OK;
}

// ---------------------------------------------------------------------------------------------
// SBP segments: every maximal run of active points on a line carries the boundary closures at
// both ends; runs shorter than 8 points become holes (repeated to a fixed point).
// Runs of active points on one line; returns (start, length) pairs, start in [0, n).
std::vector<std::pair<int, int>> active_runs(const std::vector<int8_t> &a, size_t off, size_t st, int n, bool per) {
  std::vector<std::pair<int, int>> out;
  int first_hole = -1;
  for (int k = 0; k < n; ++k)
    if (!a[off + st * k]) { first_hole = k; break; }
  if (first_hole < 0) {
    out.push_back({0, n});
    return out;
  }
  if (per) {
    // walk once around the ring starting just after a hole
    int k = 0;
    while (k < n) {
      int s = (first_hole + 1 + k) % n;
      if (!a[off + st * s]) { ++k; continue; }
      int len = 0;
      while (k + len < n && a[off + st * ((first_hole + 1 + k + len) % n)]) ++len;
      out.push_back({s, len});
      k += len;
    }
  } else {
    int k = 0;
    while (k < n) {
      if (!a[off + st * k]) { ++k; continue; }
      int len = 0;
      while (k + len < n && a[off + st * (k + len)]) ++len;
      out.push_back({k, len});
      k += len;
    }
  }
  return out;
}

namespace {
auto runs = active_runs;
}  // namespace

sbp_status setup_classes(MeshHost &m, std::string &err) {
  const int ni = m.ni, nj = m.nj;
  size_t np = (size_t)ni * nj;
  for (int pass = 0;; ++pass) {
    if (pass > 64) {
      err = "hole growing did not converge";
      return SBP_ERR_SHAPE;
    }
    bool grew = false;
    for (int dir = 0; dir < 2; ++dir) {
      int nl = dir == 0 ? nj : ni, n = dir == 0 ? ni : nj;
      size_t st = dir == 0 ? 1 : (size_t)ni;
      for (int l = 0; l < nl; ++l) {
        size_t off = dir == 0 ? (size_t)l * ni : (size_t)l;
        bool per = m.per[dir] != 0;
        auto rs = runs(m.active, off, st, n, per);
        bool whole = rs.size() == 1 && rs[0].second == n;
        if (whole && per) continue;
        for (auto &r : rs)
          if (r.second < 8) {
            for (int t = 0; t < r.second; ++t) m.active[off + st * ((r.first + t) % n)] = 0;
            grew = true;
          }
      }
    }
    if (!grew) break;
  }
  m.cls.assign(np, 0);
  for (int dir = 0; dir < 2; ++dir) {
    int nl = dir == 0 ? nj : ni, n = dir == 0 ? ni : nj;
    size_t st = dir == 0 ? 1 : (size_t)ni;
    for (int l = 0; l < nl; ++l) {
      size_t off = dir == 0 ? (size_t)l * ni : (size_t)l;
      bool per = m.per[dir] != 0;
      std::vector<uint8_t> c(n, cls_code(kHole, 0));
      auto rs = runs(m.active, off, st, n, per);
      bool whole = rs.size() == 1 && rs[0].second == n;
      for (auto &r : rs) {
        for (int t = 0; t < r.second; ++t) {
          int k = (r.first + t) % n;
          uint8_t code;
          if (whole && per) code = cls_code(kInterior, 0);
          else if (t < 4) code = cls_code(kLeft, t);
          else if (r.second - 1 - t < 4) code = cls_code(kRight, r.second - 1 - t);
          else code = cls_code(kInterior, 0);
          c[k] = code;
        }
      }
      for (int k = 0; k < n; ++k) {
        size_t p = off + st * k;
        if (dir == 0) m.cls[p] = (uint8_t)((m.cls[p] & 0xF0) | c[k]);
        else m.cls[p] = (uint8_t)((m.cls[p] & 0x0F) | (c[k] << 4));
      }
    }
  }
  for (size_t p = 0; p < np; ++p)
    if (!m.active[p]) m.cls[p] = 0xFF;
  return SBP_OK;
}

// ---------------------------------------------------------------------------------------------
// SAT points: physical and interface faces of the mesh, plus segment ends next to holes (one
// interface term per direction and side). Receivers are the points with an interface term.
sbp_status setup_sat(MeshHost &m, double omega_corner, std::string &err) {
  const int ni = m.ni, nj = m.nj;
  std::map<int, std::vector<int>> terms;  // point -> term codes (dir | side<<1 | kind<<2)
  auto add = [&](int p, int dir, int side_hi, int kind) { terms[p].push_back(dir | (side_hi << 1) | (kind << 2)); };
  for (int f = 0; f < 4; ++f) {
    int bc = m.bc[f];
    if (bc == SBP_BC_PERIODIC) continue;
    int kind = bc == SBP_BC_INTERFACE ? kTermInterface : bc == SBP_BC_FARFIELD ? kTermFarfield : kTermWall;
    int dir = f / 2, hi = f % 2;
    int len = dir == 0 ? nj : ni;
    for (int t = 0; t < len; ++t) {
      int i = dir == 0 ? (hi ? ni - 1 : 0) : t;
      int j = dir == 0 ? t : (hi ? nj - 1 : 0);
      int p = j * ni + i;
      if (m.active[p]) add(p, dir, hi, kind);
    }
  }
  for (int j = 0; j < nj; ++j)
    for (int i = 0; i < ni; ++i) {
      int p = j * ni + i;
      if (!m.active[p]) continue;
      for (int dir = 0; dir < 2; ++dir) {
        int n = dir == 0 ? ni : nj, k = dir == 0 ? i : j;
        for (int hi = 0; hi < 2; ++hi) {
          int nb = hi ? k + 1 : k - 1;
          if (m.per[dir]) nb = (nb + n) % n;
          else if (nb < 0 || nb >= n) continue;
          int q = dir == 0 ? j * ni + nb : nb * ni + i;
          if (!m.active[q]) add(p, dir, hi, kTermInterface);
        }
      }
    }
  m.sat_pt.clear();
  m.sat_code.clear();
  m.sat_recv.clear();
  m.sat_scale.clear();
  m.recv_pt.clear();
  for (auto &kv : terms) {
    if (kv.second.size() > 4) {
      err = "more than four SAT terms at one point";
      return SBP_ERR_SHAPE;
    }
    int n_int = 0;
    uint32_t code = (uint32_t)kv.second.size();
    for (size_t t = 0; t < kv.second.size(); ++t) {
      code |= (uint32_t)kv.second[t] << (3 + 4 * t);
      if ((kv.second[t] >> 2) == kTermInterface) ++n_int;
    }
    m.sat_pt.push_back(kv.first);
    m.sat_code.push_back(code);
    m.sat_scale.push_back(n_int > 1 ? omega_corner : 1.0);
    if (n_int > 0) {
      m.sat_recv.push_back((int)m.recv_pt.size());
      m.recv_pt.push_back(kv.first);
    } else {
      m.sat_recv.push_back(-1);
    }
  }
  return SBP_OK;
}

// ---------------------------------------------------------------------------------------------
// Donor search: Newton iteration on the mesh map interpolated by the 4x4 Lagrange basis.
namespace {
// Cubic Lagrange basis on nodes 0..3 and its derivative at s.
void basis4(double s, double l[4], double dl[4]) {
  const double d0 = s, d1 = s - 1.0, d2 = s - 2.0, d3 = s - 3.0;
  l[0] = -d1 * d2 * d3 / 6.0;
  l[1] = d0 * d2 * d3 / 2.0;
  l[2] = -d0 * d1 * d3 / 2.0;
  l[3] = d0 * d1 * d2 / 6.0;
  dl[0] = -(d2 * d3 + d1 * d3 + d1 * d2) / 6.0;
  dl[1] = (d2 * d3 + d0 * d3 + d0 * d2) / 2.0;
  dl[2] = -(d1 * d3 + d0 * d3 + d0 * d1) / 2.0;
  dl[3] = (d1 * d2 + d0 * d2 + d0 * d1) / 6.0;
}

int start_of(double s, int n, bool per) {
  int i0 = (int)std::floor(s) - 1;
  if (!per) i0 = std::max(0, std::min(n - 4, i0));
  return i0;
}

struct MapEval {
  double X, Y, Xs, Xr, Ys, Yr;
};

MapEval eval_map(const MeshHost &d, double s, double r) {
  int i0 = start_of(s, d.ni, d.per[0]), j0 = start_of(r, d.nj, d.per[1]);
  double li[4], dli[4], lj[4], dlj[4];
  basis4(s - i0, li, dli);
  basis4(r - j0, lj, dlj);
  MapEval e{0, 0, 0, 0, 0, 0};
  for (int b = 0; b < 4; ++b) {
    int jj = j0 + b, wj = 0;
    if (jj < 0) { jj += d.nj; wj = -1; }
    if (jj >= d.nj) { jj -= d.nj; wj = 1; }
    for (int a = 0; a < 4; ++a) {
      int ii = i0 + a, wi = 0;
      if (ii < 0) { ii += d.ni; wi = -1; }
      if (ii >= d.ni) { ii -= d.ni; wi = 1; }
      size_t p = (size_t)jj * d.ni + ii;
      double xv = d.x[p] + wi * d.shift[0] + wj * d.shift[2];
      double yv = d.y[p] + wi * d.shift[1] + wj * d.shift[3];
      e.X += li[a] * lj[b] * xv;
      e.Y += li[a] * lj[b] * yv;
      e.Xs += dli[a] * lj[b] * xv;
      e.Ys += dli[a] * lj[b] * yv;
      e.Xr += li[a] * dlj[b] * xv;
      e.Yr += li[a] * dlj[b] * yv;
    }
  }
  return e;
}
}  // namespace

sbp_status setup_donors(MeshHost &rm, const MeshHost &d, std::string &err) {
  size_t nr = rm.recv_pt.size();
  rm.donor_base.assign(2 * nr, 0);
  rm.donor_w.assign(8 * nr, 0.0);
  for (size_t r = 0; r < nr; ++r) {
    double px = rm.x[rm.recv_pt[r]], py = rm.y[rm.recv_pt[r]];
    double s, t;
    if (d.cartesian) {
      s = (px - d.lo[0]) / d.h[0];
      t = (py - d.lo[1]) / d.h[1];
    } else {
      double best = INFINITY;
      size_t bp = 0;
      for (size_t p = 0; p < d.x.size(); ++p) {
        double dd = (d.x[p] - px) * (d.x[p] - px) + (d.y[p] - py) * (d.y[p] - py);
        if (dd < best) { best = dd; bp = p; }
      }
      s = (double)(bp % d.ni);
      t = (double)(bp / d.ni);
    }
    int small = 0, it = 0;
    for (; it < 100 && small < 3; ++it) {
      MapEval e = eval_map(d, s, t);
      double det = e.Xs * e.Yr - e.Xr * e.Ys;
      if (!(std::fabs(det) > 0)) break;
      double fx = e.X - px, fy = e.Y - py;
      double ds = (e.Yr * fx - e.Xr * fy) / det, dt = (e.Xs * fy - e.Ys * fx) / det;
      s -= ds;
      t -= dt;
      small = (std::fabs(ds) < 1e-10 && std::fabs(dt) < 1e-10) ? small + 1 : 0;
    }
    bool ok = small >= 3;
    if (ok && !d.per[0] && (s < -1e-9 || s > d.ni - 1 + 1e-9)) ok = false;
    if (ok && !d.per[1] && (t < -1e-9 || t > d.nj - 1 + 1e-9)) ok = false;
    if (ok && d.per[0]) s = std::fmod(std::fmod(s, (double)d.ni) + d.ni, (double)d.ni);
    if (ok && d.per[1]) t = std::fmod(std::fmod(t, (double)d.nj) + d.nj, (double)d.nj);
    int i0 = start_of(s, d.ni, d.per[0]), j0 = start_of(t, d.nj, d.per[1]);
    for (int b = 0; ok && b < 4; ++b)
      for (int a = 0; ok && a < 4; ++a) {
        int ii = ((i0 + a) % d.ni + d.ni) % d.ni, jj = ((j0 + b) % d.nj + d.nj) % d.nj;
        if (!d.active[(size_t)jj * d.ni + ii]) ok = false;
      }
    if (!ok) {
      err = "no valid donor stencil for receiver " + std::to_string(r) + " at (" + std::to_string(px) + ", " +
            std::to_string(py) + ")";
      return SBP_ERR_DONOR;
    }
    double li[4], dli[4], lj[4], dlj[4];
    basis4(s - i0, li, dli);
    basis4(t - j0, lj, dlj);
    rm.donor_base[2 * r] = i0;
    rm.donor_base[2 * r + 1] = j0;
    for (int a = 0; a < 4; ++a) {
      rm.donor_w[8 * r + a] = li[a];
      rm.donor_w[8 * r + 4 + a] = lj[a];
    }
  }
  // distinct donor points, so that per-point work (extrapolation, viscous fluxes) is done once
  std::vector<uint32_t> all;
  all.reserve(16 * nr);
  auto packed = [&](size_t r, int a, int b) {
    int ii = ((rm.donor_base[2 * r] + a) % d.ni + d.ni) % d.ni;
    int jj = ((rm.donor_base[2 * r + 1] + b) % d.nj + d.nj) % d.nj;
    return (uint32_t)ii | ((uint32_t)jj << 16);
  };
  for (size_t r = 0; r < nr; ++r)
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) all.push_back(packed(r, a, b));
  auto key = [](uint32_t v) { return ((uint64_t)(v >> 16) << 16) | (v & 0xFFFFu); };
  std::sort(all.begin(), all.end(), [&](uint32_t x, uint32_t y) { return key(x) < key(y); });
  all.erase(std::unique(all.begin(), all.end()), all.end());
  rm.donor_pts = all;
  rm.donor_idx.assign(16 * nr, 0);
  for (size_t r = 0; r < nr; ++r)
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        uint32_t v = packed(r, a, b);
        auto it = std::lower_bound(all.begin(), all.end(), v, [&](uint32_t x, uint32_t y) { return key(x) < key(y); });
        rm.donor_idx[16 * r + b * 4 + a] = (int)(it - all.begin());
      }
  return SBP_OK;
}

// ---------------------------------------------------------------------------------------------
// Adams-Bashforth weights (Sec. 3.1 eq. (vandermonde); Sec. 3.2 eq. (ext_ab)): the moment
// conditions sum_k alpha_k t_k^i = (b^(i+1) - a^(i+1))/(i+1), i < order; with more nodes than
// the order, the minimum-2-norm solution alpha = V (V^T V)^-1 rhs.
namespace {
bool gauss_solve(std::vector<double> A, std::vector<double> b, int n, std::vector<double> &x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (A[piv * n + c] == 0.0) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  x.assign(n, 0.0);
  for (int r = n - 1; r >= 0; --r) {
    double s = b[r];
    for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * x[k];
    x[r] = s / A[r * n + r];
  }
  return true;
}
}  // namespace

sbp_status solve_ab_weights(const std::vector<double> &t, double a, double b, int order, std::vector<double> &alpha) {
  int m = (int)t.size(), n = order;
  if (n < 1 || m < n) return SBP_ERR_ARG;
  std::vector<double> mom(n);
  for (int i = 0; i < n; ++i) mom[i] = (std::pow(b, i + 1) - std::pow(a, i + 1)) / (i + 1);
  // V[k][i] = t_k^i
  std::vector<double> V((size_t)m * n);
  for (int k = 0; k < m; ++k)
    for (int i = 0; i < n; ++i) V[(size_t)k * n + i] = std::pow(t[k], i);
  if (m == n) {
    // square: V^T alpha = mom
    std::vector<double> VT((size_t)n * n);
    for (int i = 0; i < n; ++i)
      for (int k = 0; k < n; ++k) VT[(size_t)i * n + k] = V[(size_t)k * n + i];
    if (!gauss_solve(VT, mom, n, alpha)) return SBP_ERR_ARG;
    return SBP_OK;
  }
  std::vector<double> G((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < n; ++l)
      for (int k = 0; k < m; ++k) G[(size_t)i * n + l] += V[(size_t)k * n + i] * V[(size_t)k * n + l];
  std::vector<double> y;
  if (!gauss_solve(G, mom, n, y)) return SBP_ERR_ARG;
  alpha.assign(m, 0.0);
  for (int k = 0; k < m; ++k)
    for (int i = 0; i < n; ++i) alpha[k] += V[(size_t)k * n + i] * y[i];
  return SBP_OK;
}

sbp_status build_plan(int order, int m, int sr, CoeffPlan &plan, std::string &err) {
  if (order < 1 || m < order || m > kMaxHist || sr < 1) {
    err = "unsupported order / history length / step ratio";
    return SBP_ERR_ARG;
  }
  plan.order = order;
  plan.m = m;
  plan.sr = sr;
  std::vector<double> nodes(m);
  for (int k = 0; k < m; ++k) nodes[k] = (double)(k - (m - 1));
  if (solve_ab_weights(nodes, 0.0, 1.0, order, plan.ab) != SBP_OK) {
    err = "singular moment system";
    return SBP_ERR_ARG;
  }
  plan.ext.assign(sr, std::vector<double>(m, 0.0));
  for (int j = 1; j < sr; ++j)
    if (solve_ab_weights(nodes, 0.0, (double)j / sr, order, plan.ext[j]) != SBP_OK) {
      err = "singular moment system";
      return SBP_ERR_ARG;
    }
  if (solve_ab_weights(nodes, 0.0, (double)sr, order, plan.fext) != SBP_OK) {
    err = "singular moment system";
    return SBP_ERR_ARG;
  }
  std::vector<double> later(m);
  for (int k = 0; k < m; ++k) later[k] = nodes[k] + 1.0;
  plan.rext.assign(sr, std::vector<double>(m, 0.0));
  for (int j = 1; j < sr; ++j)
    if (solve_ab_weights(later, 0.0, (double)j / sr, order, plan.rext[j]) != SBP_OK) {
      err = "singular moment system";
      return SBP_ERR_ARG;
    }
  return SBP_OK;
}

}  // namespace sbp
