// Host setup of 3D Cartesian overset meshes (Sec. 2.2 with the 2D readings applied per
// direction): hole cut by the fine box, SBP segment classes along i, j and k, SAT term lists
// (faces and segment ends next to holes), and 4 x 4 x 4 Lagrange donor cells.
#include <algorithm>
#include <cmath>
#include <map>
#include <string>
#include <vector>

#include "sbp_internal.h"

namespace sbp {

namespace {
int round_up32(int v) { return (v + 31) / 32 * 32; }
}  // namespace

sbp_status setup3_mesh(const sbp3_mesh_desc &d, Mesh3Host &m, std::string &err) {
  for (int a = 0; a < 3; ++a) {
    if (d.n[a] < 8 || d.n[a] > 65535) {
      err = "each mesh direction needs 8..65535 points";
      return SBP_ERR_SHAPE;
    }
    if (!(d.h[a] > 0.0)) {
      err = "spacings must be positive";
      return SBP_ERR_SHAPE;
    }
    bool lo_per = d.bc[2 * a] == SBP_BC_PERIODIC, hi_per = d.bc[2 * a + 1] == SBP_BC_PERIODIC;
    if ((d.periodic[a] != 0) != lo_per || lo_per != hi_per) {
      err = "a periodic direction needs SBP_BC_PERIODIC on both of its faces";
      return SBP_ERR_ARG;
    }
    for (int s = 0; s < 2; ++s) {
      int b = d.bc[2 * a + s];
      if (b != SBP_BC_PERIODIC && b != SBP_BC_INTERFACE && b != SBP_BC_FARFIELD) {
        err = "3D faces are periodic, interface or far field";
        return SBP_ERR_ARG;
      }
    }
    m.n[a] = d.n[a];
    m.per[a] = d.periodic[a] != 0;
    m.lo[a] = d.lo[a];
    m.h[a] = d.h[a];
  }
  for (int f = 0; f < 6; ++f) m.bc[f] = d.bc[f];
  m.pitch = round_up32(m.n[0]);
  m.active.assign(m.points(), 1);
  return SBP_OK;
}

sbp_status setup3_holes(Mesh3Host &bg, const Mesh3Host &fine, double margin, std::string &err) {
  (void)err;
  std::vector<uint8_t> in[3];
  for (int a = 0; a < 3; ++a) {
    in[a].assign(bg.n[a], 1);
    if (fine.per[a]) continue;
    double lo = fine.lo[a], hi = fine.lo[a] + (fine.n[a] - 1) * fine.h[a];
    for (int t = 0; t < bg.n[a]; ++t) {
      double x = bg.lo[a] + bg.h[a] * t;
      in[a][t] = (x > lo + margin) && (x < hi - margin);
    }
  }
  for (int k = 0; k < bg.n[2]; ++k)
    for (int j = 0; j < bg.n[1]; ++j)
      for (int i = 0; i < bg.n[0]; ++i)
        if (in[0][i] && in[1][j] && in[2][k]) bg.active[((size_t)k * bg.n[1] + j) * bg.n[0] + i] = 0;
  return SBP_OK;
}

sbp_status setup3_classes(Mesh3Host &m, std::string &err) {
  const int ni = m.n[0], nj = m.n[1], nk = m.n[2];
  const size_t st[3] = {1, (size_t)ni, (size_t)ni * nj};
  // lines along direction a: their start offsets
  auto line_offsets = [&](int a) {
    std::vector<size_t> offs;
    int o1 = a == 0 ? 1 : 0, o2 = a == 2 ? 1 : 2;
    for (int v = 0; v < m.n[o2]; ++v)
      for (int u = 0; u < m.n[o1]; ++u) offs.push_back(u * st[o1] + v * st[o2]);
    return offs;
  };
  std::vector<size_t> offs[3] = {line_offsets(0), line_offsets(1), line_offsets(2)};
  for (int pass = 0;; ++pass) {
    if (pass > 64) {
      err = "hole growing did not converge";
      return SBP_ERR_SHAPE;
    }
    bool grew = false;
    for (int a = 0; a < 3; ++a)
      for (size_t off : offs[a]) {
        auto rs = active_runs(m.active, off, st[a], m.n[a], m.per[a] != 0);
        bool whole = rs.size() == 1 && rs[0].second == m.n[a];
        if (whole && m.per[a]) continue;
        for (auto &r : rs)
          if (r.second < 8) {
            for (int t = 0; t < r.second; ++t) m.active[off + st[a] * ((r.first + t) % m.n[a])] = 0;
            grew = true;
          }
      }
    if (!grew) break;
  }
  m.cls.assign(m.points(), 0);
  for (int a = 0; a < 3; ++a)
    for (size_t off : offs[a]) {
      const int n = m.n[a];
      std::vector<uint16_t> c(n, cls_code(kHole, 0));
      auto rs = active_runs(m.active, off, st[a], n, m.per[a] != 0);
      bool whole = rs.size() == 1 && rs[0].second == n;
      for (auto &r : rs)
        for (int t = 0; t < r.second; ++t) {
          int k = (r.first + t) % n;
          uint16_t code;
          if (whole && m.per[a]) code = cls_code(kInterior, 0);
          else if (t < 4) code = cls_code(kLeft, t);
          else if (r.second - 1 - t < 4) code = cls_code(kRight, r.second - 1 - t);
          else code = cls_code(kInterior, 0);
          c[k] = code;
        }
      for (int k = 0; k < n; ++k) {
        size_t p = off + st[a] * k;
        m.cls[p] = (uint16_t)((m.cls[p] & ~(0xF << (4 * a))) | (c[k] << (4 * a)));
      }
    }
  for (size_t p = 0; p < m.points(); ++p)
    if (!m.active[p]) m.cls[p] = 0xFFF;
  return SBP_OK;
}

sbp_status setup3_sat(Mesh3Host &m, double omega_corner, std::string &err) {
  const int ni = m.n[0], nj = m.n[1], nk = m.n[2];
  std::map<int64_t, std::vector<int>> terms;  // point -> dir | side << 2 | kind << 3
  auto add = [&](int64_t p, int dir, int hi, int kind) { terms[p].push_back(dir | (hi << 2) | (kind << 3)); };
  for (int k = 0; k < nk; ++k)
    for (int j = 0; j < nj; ++j)
      for (int i = 0; i < ni; ++i) {
        int64_t p = ((int64_t)k * nj + j) * ni + i;
        if (!m.active[p]) continue;
        const int idx[3] = {i, j, k};
        for (int a = 0; a < 3; ++a)
          for (int hi = 0; hi < 2; ++hi) {
            int bc = m.bc[2 * a + hi];
            if (bc != SBP_BC_PERIODIC && idx[a] == (hi ? m.n[a] - 1 : 0))
              add(p, a, hi, bc == SBP_BC_FARFIELD ? 1 : 0);
          }
        for (int a = 0; a < 3; ++a)
          for (int hi = 0; hi < 2; ++hi) {
            int nb[3] = {i, j, k};
            nb[a] += hi ? 1 : -1;
            if (m.per[a]) nb[a] = (nb[a] + m.n[a]) % m.n[a];
            else if (nb[a] < 0 || nb[a] >= m.n[a]) continue;
            int64_t q = ((int64_t)nb[2] * nj + nb[1]) * ni + nb[0];
            if (!m.active[q]) add(p, a, hi, 0);
          }
      }
  m.sat_pt.clear();
  m.sat_code.clear();
  m.sat_recv.clear();
  m.sat_scale.clear();
  m.recv_pt.clear();
  for (auto &kv : terms) {
    if (kv.second.size() > 3) {
      err = "more than three SAT terms at one point";
      return SBP_ERR_SHAPE;
    }
    int n_int = 0;
    uint32_t code = (uint32_t)kv.second.size();
    for (size_t t = 0; t < kv.second.size(); ++t) {
      code |= (uint32_t)kv.second[t] << (2 + 4 * t);
      if (((kv.second[t] >> 3) & 1) == 0) ++n_int;
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

sbp_status setup3_donors(Mesh3Host &rm, const Mesh3Host &d, std::string &err) {
  const size_t nr = rm.recv_pt.size();
  rm.donor_base.assign(3 * nr, 0);
  rm.donor_w.assign(12 * nr, 0.0);
  const int ni = rm.n[0], nj = rm.n[1];
  std::vector<int64_t> all;
  all.reserve(64 * nr);
  for (size_t r = 0; r < nr; ++r) {
    int64_t p = rm.recv_pt[r];
    const int idx[3] = {(int)(p % ni), (int)((p / ni) % nj), (int)(p / ((int64_t)ni * nj))};
    int base[3];
    for (int a = 0; a < 3; ++a) {
      double x = rm.lo[a] + rm.h[a] * idx[a];
      double xi = (x - d.lo[a]) / d.h[a];
      int n = d.n[a];
      if (d.per[a]) xi = xi - std::floor(xi / n) * n;
      int b = (int)std::floor(xi) - 1;
      if (!d.per[a]) {
        if (xi < 0.0 || xi > n - 1) {
          err = "receiver " + std::to_string(r) + " outside the donor mesh";
          return SBP_ERR_DONOR;
        }
        b = std::max(0, std::min(n - 4, b));
      }
      double t = xi - b;
      for (int e = 0; e < 4; ++e) {
        double w = 1.0;
        for (int f = 0; f < 4; ++f)
          if (f != e) w *= (t - f) / (double)(e - f);
        rm.donor_w[12 * r + 4 * a + e] = w;
      }
      base[a] = b;
      rm.donor_base[3 * r + a] = b;
    }
    for (int c = 0; c < 4; ++c)
      for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
          int ii = ((base[0] + a) % d.n[0] + d.n[0]) % d.n[0];
          int jj = ((base[1] + b) % d.n[1] + d.n[1]) % d.n[1];
          int kk = ((base[2] + c) % d.n[2] + d.n[2]) % d.n[2];
          int64_t q = ((int64_t)kk * d.n[1] + jj) * d.n[0] + ii;
          if (!d.active[q]) {
            err = "donor cell of receiver " + std::to_string(r) + " touches a hole";
            return SBP_ERR_DONOR;
          }
          all.push_back(q);
        }
  }
  std::vector<int64_t> uniq(all);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  rm.donor_pts = uniq;
  rm.donor_idx.assign(all.size(), 0);
  for (size_t t = 0; t < all.size(); ++t)
    rm.donor_idx[t] = (int)(std::lower_bound(uniq.begin(), uniq.end(), all[t]) - uniq.begin());
  return SBP_OK;
}

}  // namespace sbp
