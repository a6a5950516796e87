// 3D curvilinear overset pairs: a background mesh (far field on its six faces) and an overset
// mesh (interface on its six faces), both curvilinear, stepped by the 2D systems' MRAB schedule
// with its Runge-Kutta bootstrap (Sec. 3.1-3.3).
//  * setup (host): hole cut of the background by the overset mesh's inverse map (sbp3c_hole_cut;
//    margin in the overset mesh's index units), SBP segment classes with hole growth and the
//    SAT term lists (the 3D Cartesian systems' setup3_classes / setup3_sat), donor stencils of
//    every receiver by the curvilinear donor search (sbp3c_donor_search), the coefficient plan;
//  * right-hand side of mesh k: donor values on the other mesh (k3c_donor: state, extrapolated
//    in time for the fast mesh's micro steps, and viscous fluxes at the distinct donor points),
//    their Lagrange gather at the receivers (k3c_gather), the curvilinear flux divergence per
//    active segment with the far-field SAT (k3c_prim / k3c_flux / k3c_update / k3c_far), and
//    the interface SAT at the receivers (k3c_isat);
//  * MRAB step: the right-hand side into the history ring and the Adams-Bashforth combine
//    (k3c_ab) per (micro) step, slow mesh first at the start of each macro step (its right-hand
//    side at t_n), then the fast mesh's micro steps against the slow extrapolant.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "sbp3_device.h"
#include "sbp3c_device.h"
#include "sbp_system.h"

using namespace sbp;

namespace {

// Host tables of one mesh of a pair.
struct PairHost {
  int n[3] = {0, 0, 0};
  std::vector<double> x, y, z;
  Mesh3Host m3;                       // active mask, classes, SAT lists, receivers
  // interface terms grouped by receiver point (Curv3Sat layout)
  std::vector<long long> ipt;
  std::vector<int> ioff, iterm;
  std::vector<double> iscale;
  std::vector<int> donor_base;        // 3 per receiver, on the other mesh
  std::vector<double> donor_w;        // 12 per receiver
  std::vector<long long> donor_pts;   // distinct donor points (linear index on the other mesh)
  std::vector<int> donor_idx;         // 64 per receiver: (c * 4 + b) * 4 + a -> index in donor_pts
  // Navier-Stokes: distinct points of the donor points' derivative stencils on the other mesh,
  // and 13 indices into them per donor point (the point, then 4 taps along i, j, k)
  std::vector<long long> tap_pts;
  std::vector<int> tap_idx;
  size_t points() const { return (size_t)n[0] * n[1] * n[2]; }
};

struct PairDev {
  void *met = nullptr, *prim = nullptr, *flux = nullptr;
  uint16_t *cls = nullptr;
  long long *ipt = nullptr;
  int *ioff = nullptr, *iterm = nullptr;
  double *iscale = nullptr;
  long long *dpts = nullptr;
  int *didx = nullptr;
  long long *tpts = nullptr;  // Navier-Stokes tap points of the donor values (PairHost::tap_pts)
  int *tidx = nullptr;
  void *tv = nullptr;         // their extrapolated primitives, 4 per set and tap point
  int ntap = 0;
  void *dwt = nullptr;
  void *dv = nullptr;
  void *qhat = nullptr, *fvhat = nullptr;
  int ndv = 0, nrecv = 0, npt = 0;
  void *q[2] = {nullptr, nullptr};
  void *hist = nullptr;
  int cur = 0, head = -1;
  void release() {
    cudaFree(met);
    cudaFree(prim);
    cudaFree(flux);
    cudaFree(cls);
    cudaFree(ipt);
    cudaFree(ioff);
    cudaFree(iterm);
    cudaFree(iscale);
    cudaFree(dpts);
    cudaFree(didx);
    cudaFree(tpts);
    cudaFree(tidx);
    cudaFree(tv);
    cudaFree(dwt);
    cudaFree(dv);
    cudaFree(qhat);
    cudaFree(fvhat);
  }
};

// The host setup of a pair (no device calls).
sbp_status pair_setup(const sbp3c_mesh_desc *meshes, int n_meshes, const sbp_params *params, sbp_params &pout,
                      PairHost mh[2], CoeffPlan &plan) {
  if (!meshes || !params) return fail(SBP_ERR_ARG, "null argument");
  if (n_meshes != 2) return fail(SBP_ERR_ARG, "a pair has two meshes (background, overset)");
  const sbp_params &p = *params;
  if (p.physics != SBP_EULER && p.physics != SBP_NS) return fail(SBP_ERR_ARG, "physics");
  if (p.dtype != SBP_F64 && p.dtype != SBP_F32) return fail(SBP_ERR_DTYPE, "dtype");
  if (p.fast_mesh != 0 && p.fast_mesh != 1) return fail(SBP_ERR_ARG, "fast_mesh");
  if (!(p.gamma > 1.0) || p.mu < 0.0 || !(p.pr > 0.0)) return fail(SBP_ERR_ARG, "gas constants");
  if (p.step_ratio < 1 || p.step_ratio > kMaxSets)
    return fail(SBP_ERR_ARG, "step_ratio must be in 1.." + std::to_string(kMaxSets));
  if (p.scheme != SBP_MRAB_FASTEST_FIRST) return fail(SBP_ERR_ARG, "curvilinear pairs are fastest-first");
  if (p.sponge_cells < 0 || p.sponge_cells > 16 || !(p.sponge_strength >= 0.0))
    return fail(SBP_ERR_ARG, "sponge_cells must be in 0..16 and sponge_strength >= 0");
  if (!(p.sigma_interface >= 0.0) || !(p.sigma_physical >= 0.0)) return fail(SBP_ERR_ARG, "penalties");
  pout = p;
  if (!(pout.hole_cells > 0.0)) pout.hole_cells = 4.0;
  for (int k = 0; k < 2; ++k) {
    const sbp3c_mesh_desc &d = meshes[k];
    if (!d.x || !d.y || !d.z) return fail(SBP_ERR_ARG, "mesh coordinates missing");
    long long N = 1;
    for (int a = 0; a < 3; ++a) {
      if (d.n[a] < 8 || d.n[a] > 65535) return fail(SBP_ERR_SHAPE, "each direction needs 8..65535 points");
      N *= d.n[a];
    }
    if (N > 2147483647LL / 17) return fail(SBP_ERR_SHAPE, "mesh too large");
    PairHost &m = mh[k];
    std::memcpy(m.n, d.n, sizeof(m.n));
    m.x.assign(d.x, d.x + N);
    m.y.assign(d.y, d.y + N);
    m.z.assign(d.z, d.z + N);
    Mesh3Host &h = m.m3;
    for (int a = 0; a < 3; ++a) {
      h.n[a] = d.n[a];
      h.per[a] = 0;
      h.lo[a] = 0.0;
      h.h[a] = 1.0;
    }
    for (int f = 0; f < 6; ++f) h.bc[f] = k == 0 ? SBP_BC_FARFIELD : SBP_BC_INTERFACE;
    h.pitch = d.n[0];
    h.active.assign((size_t)N, 1);
  }
  // hole cut of the background by the overset mesh
  {
    const PairHost &o = mh[1];
    PairHost &b = mh[0];
    const size_t N0 = b.points();
    std::vector<double> pts(3 * N0);
    for (size_t t = 0; t < N0; ++t) {
      pts[3 * t] = b.x[t];
      pts[3 * t + 1] = b.y[t];
      pts[3 * t + 2] = b.z[t];
    }
    std::vector<signed char> ib(N0, 1);
    sbp_status st = sbp3c_hole_cut(o.n, o.x.data(), o.y.data(), o.z.data(), (int)N0, pts.data(), pout.hole_cells,
                                   ib.data());
    if (st != SBP_OK) return st;
    for (size_t t = 0; t < N0; ++t) b.m3.active[t] = ib[t];
  }
  std::string err;
  sbp_status st;
  for (int k = 0; k < 2; ++k) {
    if ((st = setup3_classes(mh[k].m3, err)) != SBP_OK) return fail(st, err);
    if ((st = setup3_sat(mh[k].m3, p.omega_corner, err)) != SBP_OK) return fail(st, err);
  }
  // interface terms grouped by point (far-field terms are the far-field kernel's)
  for (int k = 0; k < 2; ++k) {
    PairHost &m = mh[k];
    const Mesh3Host &h = m.m3;
    m.ipt.clear();
    m.ioff.clear();
    m.iterm.clear();
    m.iscale.clear();
    for (size_t s = 0; s < h.sat_pt.size(); ++s) {
      const uint32_t code = h.sat_code[s];
      const int cnt = (int)(code & 3u);
      bool first = true;
      for (int e = 0; e < cnt; ++e) {
        const unsigned bits = (code >> (2 + 4 * e)) & 15u;
        if ((bits >> 3) & 1u) continue;  // far field
        if (first) {
          m.ipt.push_back((long long)h.sat_pt[s]);
          m.ioff.push_back((int)m.iscale.size());
          first = false;
        }
        m.iterm.insert(m.iterm.end(), {(int)(bits & 3u), ((bits >> 2) & 1u) ? -1 : 1, h.sat_recv[s]});
        m.iscale.push_back(h.sat_scale[s]);
      }
    }
    m.ioff.push_back((int)m.iscale.size());
  }
  // donor stencils of every receiver on the other mesh
  for (int k = 0; k < 2; ++k) {
    PairHost &m = mh[k];
    const PairHost &o = mh[1 - k];
    const size_t nr = m.m3.recv_pt.size();
    std::vector<double> pts(3 * nr);
    for (size_t r = 0; r < nr; ++r) {
      const size_t t = (size_t)m.m3.recv_pt[r];
      pts[3 * r] = m.x[t];
      pts[3 * r + 1] = m.y[t];
      pts[3 * r + 2] = m.z[t];
    }
    std::vector<signed char> ib(o.m3.active.begin(), o.m3.active.end());
    m.donor_base.assign(3 * nr, 0);
    m.donor_w.assign(12 * nr, 0.0);
    int failed = -1;
    if (nr > 0) {
      st = sbp3c_donor_search(o.n, o.x.data(), o.y.data(), o.z.data(), ib.data(), (int)nr, pts.data(),
                              m.donor_base.data(), m.donor_w.data(), nullptr, &failed);
      if (st != SBP_OK)
        return fail(st, "receiver " + std::to_string(failed) + " of mesh " + std::to_string(k) + ": " +
                            sbp_last_error_message());
    }
    std::vector<long long> all;
    all.reserve(64 * nr);
    for (size_t r = 0; r < nr; ++r)
      for (int c = 0; c < 4; ++c)
        for (int b = 0; b < 4; ++b)
          for (int a = 0; a < 4; ++a)
            all.push_back(((long long)(m.donor_base[3 * r + 2] + c) * o.n[1] + (m.donor_base[3 * r + 1] + b)) * o.n[0] +
                          (m.donor_base[3 * r] + a));
    m.donor_pts = all;
    std::sort(m.donor_pts.begin(), m.donor_pts.end());
    m.donor_pts.erase(std::unique(m.donor_pts.begin(), m.donor_pts.end()), m.donor_pts.end());
    m.donor_idx.assign(all.size(), 0);
    for (size_t t = 0; t < all.size(); ++t)
      m.donor_idx[t] = (int)(std::lower_bound(m.donor_pts.begin(), m.donor_pts.end(), all[t]) - m.donor_pts.begin());
    if (p.physics == SBP_NS) {
      // the taps of each donor point's derivative rows (the class codes and offsets the
      // kernels decode), so that every tap's extrapolated primitives are formed once per set
      static const int off[6][4] = SBP_ROW_OFFSETS;
      const long long st[3] = {1, (long long)o.n[0], (long long)o.n[0] * o.n[1]};
      std::vector<long long> taps(13 * m.donor_pts.size());
      for (size_t q = 0; q < m.donor_pts.size(); ++q) {
        const long long pnt = m.donor_pts[q];
        taps[13 * q] = pnt;
        for (int d = 0; d < 3; ++d) {
          const unsigned code = ((unsigned)o.m3.cls[(size_t)pnt] >> (4 * d)) & 15u, kind = code >> 2;
          const int row = kind == kInterior ? 4 : kind == kHole ? 5 : (int)(code & 3u);
          const int sgn = kind == kRight ? -1 : 1;
          for (int e = 0; e < 4; ++e) taps[13 * q + 1 + 4 * d + e] = pnt + (long long)sgn * off[row][e] * st[d];
        }
      }
      m.tap_pts = taps;
      std::sort(m.tap_pts.begin(), m.tap_pts.end());
      m.tap_pts.erase(std::unique(m.tap_pts.begin(), m.tap_pts.end()), m.tap_pts.end());
      const long long npo = (long long)o.points();
      if (!m.tap_pts.empty() && (m.tap_pts.front() < 0 || m.tap_pts.back() >= npo))
        return fail(SBP_ERR_DONOR, "a donor point's derivative stencil leaves mesh " + std::to_string(1 - k));
      m.tap_idx.assign(taps.size(), 0);
      for (size_t t = 0; t < taps.size(); ++t)
        m.tap_idx[t] = (int)(std::lower_bound(m.tap_pts.begin(), m.tap_pts.end(), taps[t]) - m.tap_pts.begin());
    }
  }
  if ((st = build_plan(p.order, p.hist_len, p.step_ratio, plan, err)) != SBP_OK) return fail(st, err);
  return SBP_OK;
}

}  // namespace

struct sbp3c_system_s {
  sbp_params p{};
  double qinf[5] = {1, 0, 0, 0, 0};
  PairHost mh[2];
  PairDev md[2];
  CoeffPlan plan;
  size_t esz = 8;
  int *d_err = nullptr;
  unsigned long long *d_dt = nullptr;
  double H = 0.0, t = 0.0;
  bool initialised = false;

  ~sbp3c_system_s() {
    for (auto &d : md) d.release();
    cudaFree(d_err);
    cudaFree(d_dt);
  }

  bool viscous() const { return p.physics == SBP_NS; }
  int fast() const { return p.fast_mesh; }
  int slow() const { return 1 - p.fast_mesh; }
  size_t field(int k) const { return mh[k].points(); }
  size_t state_elems(int k) const { return 5 * field(k); }
  void *hist_slot(int k, int slot) const { return (char *)md[k].hist + (size_t)slot * state_elems(k) * esz; }

  Curv3Launch curv(int k, const void *q, void *out) const {
    Curv3Launch a{};
    a.ni = mh[k].n[0];
    a.nj = mh[k].n[1];
    a.nk = mh[k].n[2];
    a.field = field(k);
    a.cls = md[k].cls;
    a.visc = viscous();
    a.gam = p.gamma;
    a.mu = a.visc ? p.mu : 0.0;
    a.lam = -2.0 / 3.0 * a.mu;
    a.kap = a.mu / (p.pr * (p.gamma - 1.0));
    a.q = q;
    a.out = out;
    a.met = md[k].met;
    a.prim = md[k].prim;
    a.flux = md[k].flux;
    a.far = k == 0;
    a.sig = p.sigma_physical;
    std::memcpy(a.qinf, qinf, sizeof(a.qinf));
    return a;
  }

  // Donor values for mesh recv's receivers from the other mesh's state q: sets set0 ..
  // set0 + nsets - 1, each extrapolated in time by the other mesh's history when asked.
  cudaError_t donors(int recv, const void *q, int set0, int nsets, bool extrapolate, cudaStream_t s) const {
    const int don = 1 - recv, m = plan.m;
    Curv3Donor a{};
    a.m = curv(don, q, nullptr);
    for (int k = 0; k < m && md[don].hist; ++k) a.hist[k] = hist_slot(don, (md[don].head + 1 + k) % m);
    for (int j = 0; j < nsets; ++j) {
      const int set = set0 + j;
      a.nb[j] = (extrapolate && set > 0) ? m : 0;
      for (int k = 0; k < m; ++k) a.beta[j][k] = extrapolate ? plan.ext[set][k] * H : 0.0;
    }
    a.nsets = nsets;
    a.npts = md[recv].ndv;
    a.pts = md[recv].dpts;
    a.dv = (char *)md[recv].dv + (size_t)set0 * kDvPitch * md[recv].ndv * esz;
    if (md[recv].tpts) {
      a.tpts = md[recv].tpts;
      a.tidx = md[recv].tidx;
      a.ntap = md[recv].ntap;
      a.tv = md[recv].tv;  // sets of this launch from the workspace's start
    }
    return launch3c_donor(a, p.dtype, s);
  }

  cudaError_t gather(int k, int set, void *qhat, void *fvhat, cudaStream_t s) const {
    Curv3Gather g{};
    g.dv = (const char *)md[k].dv + (size_t)set * kDvPitch * md[k].ndv * esz;
    g.didx = md[k].didx;
    g.dwt = md[k].dwt;
    g.nrecv = md[k].nrecv;
    g.ndv = md[k].ndv;
    g.err = d_err;
    g.nval = (viscous() && fvhat) ? 17 : 5;  // no viscous fluxes without a place for them
    g.qhat = qhat;
    g.fvhat = viscous() ? fvhat : nullptr;
    return launch3c_gather(g, p.dtype, s);
  }

  // out = dq/dt of mesh k at q_self with the receiver values of donor set `set`.
  cudaError_t rhs(int k, const void *q_self, int set, void *out, cudaStream_t s) const {
    cudaError_t e = gather(k, set, md[k].qhat, md[k].fvhat, s);
    if (e != cudaSuccess) return e;
    const Curv3Launch a = curv(k, q_self, out);
    e = launch3c_rhs(a, p.dtype, s);
    if (e != cudaSuccess) return e;
    Curv3Sat sat{};
    sat.npt = md[k].npt;
    sat.nrecv = md[k].nrecv;
    sat.pt = md[k].ipt;
    sat.off = md[k].ioff;
    sat.term = md[k].iterm;
    sat.scale = md[k].iscale;
    sat.qhat = md[k].qhat;
    sat.fvhat = md[k].fvhat;
    sat.sig = p.sigma_interface;
    e = launch3c_isat(a, sat, p.dtype, s);
    if (e != cudaSuccess || k != 0 || p.sponge_cells <= 0) return e;
    // the background's sponge layer (all six faces far field), after its SAT terms
    Curv3Sponge sp{};
    sp.depth = p.sponge_cells;
    for (int d = 0; d < p.sponge_cells; ++d) {
      const double r = (double)(p.sponge_cells - d) / p.sponge_cells;
      sp.tab[d] = p.sponge_strength * r * r;
    }
    return launch3c_sponge(a, sp, p.dtype, s);
  }

  cudaError_t rhs_plain(int k, const void *q_self, const void *q_other, void *out, cudaStream_t s) const {
    cudaError_t e = donors(k, q_other, 0, 1, false, s);
    return e != cudaSuccess ? e : rhs(k, q_self, 0, out, s);
  }

  // One Adams-Bashforth (micro) step of mesh k with step dt: its right-hand side into the next
  // history slot, then q_next = q + sum over the history of the weights times dt.
  cudaError_t fused(int k, int set, double dt, cudaStream_t s) {
    const int m = plan.m;
    PairDev &d = md[k];
    const int slot = (d.head + 1) % m;
    cudaError_t e = rhs(k, d.q[d.cur], set, hist_slot(k, slot), s);
    if (e != cudaSuccess) return e;
    Curv3Ab a{};
    a.field = field(k);
    a.cls = d.cls;
    a.q = d.q[d.cur];
    a.rhs = hist_slot(k, slot);
    a.nold = m - 1;
    for (int j = 0; j < m - 1; ++j) {
      a.hold[j] = hist_slot(k, (slot + 1 + j) % m);
      a.alpha[j] = plan.ab[j] * dt;
    }
    a.alpha[m - 1] = plan.ab[m - 1] * dt;
    a.qn = d.q[1 - d.cur];
    a.err = d_err;
    return launch3c_ab(a, p.dtype, s);
  }

  // One macro step (fastest-first, Sec. 3.3), the 3D Cartesian systems' order of launches.
  cudaError_t issue_step(cudaStream_t s) {
    const int F = fast(), Sl = slow(), sr = plan.sr;
    const double h = H / sr;
    cudaError_t e = cudaSuccess;
    auto run = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    run(donors(Sl, md[F].q[md[F].cur], 0, 1, false, s));
    run(fused(Sl, 0, H, s));
    md[Sl].head = (md[Sl].head + 1) % plan.m;
    run(donors(F, md[Sl].q[md[Sl].cur], 0, sr, true, s));
    for (int j = 0; j < sr; ++j) {
      run(fused(F, j, h, s));
      md[F].head = (md[F].head + 1) % plan.m;
      md[F].cur ^= 1;
    }
    md[Sl].cur ^= 1;
    t += H;
    return e;
  }

  // Heun's third-order Runge-Kutta method at the micro step for (m - 1) SR micro steps, each
  // stage with the overset coupling, recording the right-hand sides the MRAB history needs.
  cudaError_t bootstrap(double Hm, cudaStream_t s) {
    const int m = plan.m, sr = plan.sr, F = fast(), Sl = slow();
    const double h = Hm / sr;
    void *ystage[2] = {nullptr, nullptr}, *k1tmp[2] = {nullptr, nullptr}, *k23[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2; ++k) {
      const size_t b = state_elems(k) * esz;
      if (e == cudaSuccess) e = cudaMalloc(&ystage[k], b);
      if (e == cudaSuccess) e = cudaMalloc(&k1tmp[k], b);
      if (e == cudaSuccess) e = cudaMalloc(&k23[k], b);
      if (e == cudaSuccess) e = cudaMemsetAsync(ystage[k], 0, b, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(k1tmp[k], 0, b, s);
      if (e == cudaSuccess) e = cudaMemsetAsync(k23[k], 0, b, s);
      md[k].head = -1;
    }
    const int nsteps = (m - 1) * sr;
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
      void *y[2] = {md[0].q[md[0].cur], md[1].q[md[1].cur]};
      void *k1[2] = {k1tmp[0], k1tmp[1]};
      if (step >= nsteps - (m - 1)) {
        md[F].head = (md[F].head + 1) % m;
        k1[F] = hist_slot(F, md[F].head);
      }
      if (step % sr == 0) {
        md[Sl].head = (md[Sl].head + 1) % m;
        k1[Sl] = hist_slot(Sl, md[Sl].head);
      }
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = rhs_plain(k, y[k], y[1 - k], k1[k], s);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = launch_axpy(y[k], k1[k], h / 3.0, nullptr, 0.0, ystage[k], state_elems(k), p.dtype, s);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = rhs_plain(k, ystage[k], ystage[1 - k], k23[k], s);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = launch_axpy(y[k], k23[k], 2.0 * h / 3.0, nullptr, 0.0, ystage[k], state_elems(k), p.dtype, s);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = rhs_plain(k, ystage[k], ystage[1 - k], k23[k], s);
      for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = launch_axpy(y[k], k1[k], h / 4.0, k23[k], 3.0 * h / 4.0, y[k], state_elems(k), p.dtype, s);
    }
    const cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    for (int k = 0; k < 2; ++k) {
      cudaFree(ystage[k]);
      cudaFree(k1tmp[k]);
      cudaFree(k23[k]);
    }
    return e;
  }
};

struct sbp3c_host_tables_s {
  sbp_params p;
  PairHost mh[2];
  CoeffPlan plan;
};

extern "C" {

sbp_status sbp3c_host_tables_create(const sbp3c_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                                    sbp3c_host_tables_t *out) {
  if (!out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  std::unique_ptr<sbp3c_host_tables_s> T(new sbp3c_host_tables_s());
  sbp_status st = pair_setup(meshes, n_meshes, params, T->p, T->mh, T->plan);
  if (st != SBP_OK) return st;
  *out = T.release();
  return SBP_OK;
}

sbp_status sbp3c_host_tables_destroy(sbp3c_host_tables_t T) {
  delete T;
  return SBP_OK;
}

static void copy_tables(const PairHost &m, signed char *iblank, long long *receivers, int *donor_base,
                        double *donor_w) {
  if (iblank)
    for (size_t t = 0; t < m.points(); ++t) iblank[t] = m.m3.active[t];
  const size_t nr = m.m3.recv_pt.size();
  if (receivers)
    for (size_t r = 0; r < nr; ++r) receivers[r] = (long long)m.m3.recv_pt[r];
  if (donor_base && nr) std::memcpy(donor_base, m.donor_base.data(), 3 * nr * sizeof(int));
  if (donor_w && nr) std::memcpy(donor_w, m.donor_w.data(), 12 * nr * sizeof(double));
}

sbp_status sbp3c_host_tables_get(sbp3c_host_tables_t T, int k, signed char *iblank, long long *receivers,
                                 int *donor_base, double *donor_w, int *n_receivers) {
  if (!T || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  copy_tables(T->mh[k], iblank, receivers, donor_base, donor_w);
  if (n_receivers) *n_receivers = (int)T->mh[k].m3.recv_pt.size();
  return SBP_OK;
}

sbp_status sbp3c_system_create(const sbp3c_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                               sbp3c_system_t *out) {
  if (!meshes || !params || !out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  std::unique_ptr<sbp3c_system_s> S(new sbp3c_system_s());
  sbp_status st = pair_setup(meshes, n_meshes, params, S->p, S->mh, S->plan);
  if (st != SBP_OK) return st;
  const sbp_params &p = S->p;
  S->esz = p.dtype == SBP_F64 ? 8 : 4;
  S->qinf[0] = p.qinf[0];
  S->qinf[1] = p.qinf[1];
  S->qinf[2] = p.qinf[2];
  S->qinf[3] = 0.0;
  S->qinf[4] = p.qinf[3];
  CUDA_TRY(cudaMalloc((void **)&S->d_err, sizeof(int)));
  CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
  CUDA_TRY(cudaMalloc((void **)&S->d_dt, 2 * sizeof(unsigned long long)));
  for (int k = 0; k < 2; ++k) {
    const PairHost &m = S->mh[k];
    PairDev &d = S->md[k];
    const size_t N = m.points(), esz = S->esz;
    // metric terms on the device (FP64 arithmetic, stored in the element type)
    double *dxyz = nullptr, *ddx = nullptr;
    cudaError_t e = cudaMalloc((void **)&dxyz, 3 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void **)&ddx, 9 * N * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(dxyz, m.x.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dxyz + N, m.y.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dxyz + 2 * N, m.z.data(), N * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&d.met, 10 * N * esz);
    if (e == cudaSuccess) e = launch3c_metrics(m.n[0], m.n[1], m.n[2], dxyz, ddx, d.met, p.dtype, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(dxyz);
    cudaFree(ddx);
    CUDA_TRY(e);
    CUDA_TRY(upload(d.cls, m.m3.cls.data(), N * sizeof(uint16_t)));
    if (S->viscous()) {
      CUDA_TRY(cudaMalloc(&d.prim, 4 * N * esz));
      CUDA_TRY(cudaMemset(d.prim, 0, 4 * N * esz));
    }
    CUDA_TRY(cudaMalloc(&d.flux, 15 * N * esz));
    CUDA_TRY(cudaMemset(d.flux, 0, 15 * N * esz));
    d.npt = (int)m.ipt.size();
    d.nrecv = (int)m.m3.recv_pt.size();
    CUDA_TRY(upload(d.ipt, m.ipt.data(), m.ipt.size() * sizeof(long long)));
    CUDA_TRY(upload(d.ioff, m.ioff.data(), m.ioff.size() * sizeof(int)));
    CUDA_TRY(upload(d.iterm, m.iterm.data(), m.iterm.size() * sizeof(int)));
    CUDA_TRY(upload(d.iscale, m.iscale.data(), m.iscale.size() * sizeof(double)));
    d.ndv = (int)m.donor_pts.size();
    CUDA_TRY(upload(d.dpts, m.donor_pts.data(), m.donor_pts.size() * sizeof(long long)));
    CUDA_TRY(upload(d.didx, m.donor_idx.data(), m.donor_idx.size() * sizeof(int)));
    if (p.dtype == SBP_F64) {
      CUDA_TRY(upload(d.dwt, m.donor_w.data(), m.donor_w.size() * sizeof(double)));
    } else {
      std::vector<float> wf(m.donor_w.begin(), m.donor_w.end());
      CUDA_TRY(upload(d.dwt, wf.data(), wf.size() * sizeof(float)));
    }
    const size_t sets = k == p.fast_mesh ? (size_t)p.step_ratio : 1;
    if (!m.tap_pts.empty()) {
      d.ntap = (int)m.tap_pts.size();
      CUDA_TRY(upload(d.tpts, m.tap_pts.data(), m.tap_pts.size() * sizeof(long long)));
      CUDA_TRY(upload(d.tidx, m.tap_idx.data(), m.tap_idx.size() * sizeof(int)));
      CUDA_TRY(cudaMalloc(&d.tv, sets * 4 * (size_t)d.ntap * esz));
    }
    CUDA_TRY(cudaMalloc(&d.dv, (sets * kDvPitch * d.ndv + 1) * esz));
    CUDA_TRY(cudaMemset(d.dv, 0, (sets * kDvPitch * d.ndv + 1) * esz));
    CUDA_TRY(cudaMalloc(&d.qhat, (5 * (size_t)d.nrecv + 1) * esz));
    CUDA_TRY(cudaMemset(d.qhat, 0, (5 * (size_t)d.nrecv + 1) * esz));
    CUDA_TRY(cudaMalloc(&d.fvhat, (12 * (size_t)d.nrecv + 1) * esz));
    CUDA_TRY(cudaMemset(d.fvhat, 0, (12 * (size_t)d.nrecv + 1) * esz));
  }
  CUDA_TRY(cudaDeviceSynchronize());
  *out = S.release();
  return SBP_OK;
}

sbp_status sbp3c_system_destroy(sbp3c_system_t S) {
  delete S;
  return SBP_OK;
}

sbp_status sbp3c_system_info(sbp3c_system_t S, int k, sbp3_mesh_info *info) {
  if (!S || !info || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const PairHost &m = S->mh[k];
  info->ni = m.n[0];
  info->nj = m.n[1];
  info->nk = m.n[2];
  info->pitch = m.n[0];
  info->field_elems = S->field(k);
  info->state_bytes = S->state_elems(k) * S->esz;
  info->nvar = 5;
  info->n_holes = (int)std::count(m.m3.active.begin(), m.m3.active.end(), 0);
  info->n_receivers = (int)m.m3.recv_pt.size();
  info->n_sat_points = (int)m.m3.sat_pt.size();
  info->elem_size = (int)S->esz;
  return SBP_OK;
}

sbp_status sbp3c_system_set_freestream(sbp3c_system_t S, const double *qinf) {
  if (!S || !qinf) return fail(SBP_ERR_ARG, "bad argument");
  const double ke = 0.5 * (qinf[1] * qinf[1] + qinf[2] * qinf[2] + qinf[3] * qinf[3]) / qinf[0];
  if (!(qinf[0] > 0.0) || !((S->p.gamma - 1.0) * (qinf[4] - ke) > 0.0))
    return fail(SBP_ERR_ARG, "free stream: positive density and pressure required");
  std::memcpy(S->qinf, qinf, sizeof(S->qinf));
  return SBP_OK;
}

sbp_status sbp3c_system_tables(sbp3c_system_t S, int k, signed char *iblank, long long *receivers, int *donor_base,
                               double *donor_w) {
  if (!S || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  copy_tables(S->mh[k], iblank, receivers, donor_base, donor_w);
  return SBP_OK;
}

sbp_status sbp3c_system_interp(sbp3c_system_t S, int recv, const void *q_donor, void *qhat, void *fvhat,
                               void *stream) {
  if (!S || recv < 0 || recv > 1 || !q_donor || !qhat) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(S->donors(recv, q_donor, 0, 1, false, s));
  CUDA_TRY(S->gather(recv, 0, qhat, fvhat, s));
  return SBP_OK;
}

sbp_status sbp3c_system_rhs_eval(sbp3c_system_t S, int k, const void *q_self, const void *q_other, void *rhs,
                                 void *stream) {
  if (!S || k < 0 || k > 1 || !q_self || !q_other || !rhs) return fail(SBP_ERR_ARG, "bad argument");
  CUDA_TRY(S->rhs_plain(k, q_self, q_other, rhs, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp3c_system_timestep(sbp3c_system_t S, const void *q0, const void *q1, double *dt_mesh, double *H,
                                 void *stream) {
  if (!S || !q0 || !q1) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const void *qs[2] = {q0, q1};
  for (int k = 0; k < 2; ++k) CUDA_TRY(launch3c_dt(S->curv(k, qs[k], nullptr), S->p.pr, S->d_dt + k, s, S->p.dtype));
  unsigned long long bits[2];
  CUDA_TRY(cudaMemcpyAsync(bits, S->d_dt, sizeof(bits), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  double dt[2];
  for (int k = 0; k < 2; ++k) std::memcpy(&dt[k], &bits[k], sizeof(double));
  if (dt_mesh) {
    dt_mesh[0] = dt[0];
    dt_mesh[1] = dt[1];
  }
  if (H) *H = std::min(S->p.cfl * dt[S->slow()], S->p.step_ratio * S->p.cfl * dt[S->fast()]);
  return SBP_OK;
}

sbp_status sbp3c_system_bind(sbp3c_system_t S, int k, void *qa, void *qb, void *hist) {
  if (!S || k < 0 || k > 1 || !qa || !qb || !hist) return fail(SBP_ERR_ARG, "bad argument");
  S->md[k].q[0] = qa;
  S->md[k].q[1] = qb;
  S->md[k].hist = hist;
  S->md[k].cur = 0;
  S->md[k].head = -1;
  S->initialised = false;
  return SBP_OK;
}

sbp_status sbp3c_system_current_state(sbp3c_system_t S, int k, void **q) {
  if (!S || k < 0 || k > 1 || !q) return fail(SBP_ERR_ARG, "bad argument");
  *q = S->md[k].q[S->md[k].cur];
  return SBP_OK;
}

sbp_status sbp3c_system_mrab_init(sbp3c_system_t S, double H, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  for (int k = 0; k < 2; ++k)
    if (!S->md[k].hist) return fail(SBP_ERR_STATE, "buffers not bound");
  if (!(H > 0.0)) {
    sbp_status st = sbp3c_system_timestep(S, S->md[0].q[S->md[0].cur], S->md[1].q[S->md[1].cur], nullptr, &H, stream);
    if (st != SBP_OK) return st;
  }
  S->H = H;
  cudaError_t e = S->bootstrap(H, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(SBP_ERR_CUDA, std::string("bootstrap: ") + cudaGetErrorString(e));
  S->t = 0.0;
  S->initialised = true;
  return SBP_OK;
}

sbp_status sbp3c_system_mrab_step(sbp3c_system_t S, int n, void *stream) {
  if (!S || n < 0) return fail(SBP_ERR_ARG, "bad argument");
  if (!S->initialised) return fail(SBP_ERR_STATE, "sbp3c_system_mrab_init has not run");
  for (int i = 0; i < n; ++i) CUDA_TRY(S->issue_step((cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp3c_system_mrab_time(sbp3c_system_t S, double *H, double *t) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  if (H) *H = S->H;
  if (t) *t = S->t;
  return SBP_OK;
}

sbp_status sbp3c_system_check(sbp3c_system_t S, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, S->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
  if (e) return fail((sbp_status)e, "device error word set");
  return SBP_OK;
}

}  // extern "C"
