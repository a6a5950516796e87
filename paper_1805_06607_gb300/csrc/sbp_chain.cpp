// Chains of nested overset meshes, each stepped at its own rate (sbp_chain_*): Sec. 3.3's
// multi-rate Adams-Bashforth scheme for more than two rates, read as the two-rate recursion nested
// level by level, on Sec. 2.2's overset coupling at every level.
//
// Mesh r (r >= 1) lies inside mesh r - 1 and cuts a hole into it (the two-mesh hole rule with
// mesh r - 1's spacing). Mesh r's receivers are its interface faces, fed by mesh r - 1, and the
// segment ends next to the hole that mesh r + 1 cuts, fed by mesh r + 1; the distinct donor
// points of the two groups are kept in one list (mesh r - 1's first), so that the right-hand-side
// kernels gather every receiver's values from one donor-value array filled by one donor-value
// launch per group. Each mesh's tables and kernels are those of the two-mesh systems.
//
// A macro step of mesh 0 (step H; mesh r steps h_r = h_{r-1} / ratios[r-1]) runs, for mesh r at
// the start tau of each of its steps: the donor values (mesh r - 1's state at the start of its
// current step extrapolated to tau by the polynomial through its history; mesh r + 1's state at
// tau), the right-hand side at tau fused with the Adams-Bashforth update over [tau, tau + h_r],
// then mesh r + 1's ratios[r] steps over the same interval; mesh r's new state becomes current
// after them (the finer meshes extrapolate from its state at tau meanwhile).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <memory>
#include <string>
#include <vector>

#include "sbp_system.h"

namespace {

constexpr int kMaxChain = 8;

bool on_interface_face(const MeshHost &m, int p) {
  const int i = p % m.ni, j = p / m.ni;
  return (i == 0 && m.bc[0] == SBP_BC_INTERFACE) || (i == m.ni - 1 && m.bc[1] == SBP_BC_INTERFACE) ||
         (j == 0 && m.bc[2] == SBP_BC_INTERFACE) || (j == m.nj - 1 && m.bc[3] == SBP_BC_INTERFACE);
}

bool next_to_hole(const MeshHost &m, int p) {
  const int i = p % m.ni, j = p / m.ni;
  for (int dir = 0; dir < 2; ++dir)
    for (int s = -1; s <= 1; s += 2) {
      const int n = dir == 0 ? m.ni : m.nj;
      int c = (dir == 0 ? i : j) + s;
      if (m.per[dir]) c = (c + n) % n;
      else if (c < 0 || c >= n) continue;
      const int q = dir == 0 ? j * m.ni + c : c * m.ni + i;
      if (!m.active[q]) return true;
    }
  return false;
}

}  // namespace

struct sbp_chain_s {
  sbp_params p{};
  int R = 0, m = 0;
  std::vector<int> ratios, ticks;  // ticks[r]: steps of the innermost mesh per step of mesh r
  std::vector<double> h;           // h[0] = H, h[r] = h[r - 1] / ratios[r - 1]
  // mesh r's host setup and device tables live in mesh[r]->mh[0], md[0]
  std::vector<std::unique_ptr<sbp_system_s>> mesh;
  std::vector<std::vector<int>> recv_src;  // per mesh and receiver: its donor mesh
  std::vector<int> ndv_lo;                 // distinct donor points on mesh r - 1 (first in the list)
  std::vector<double> ab;                  // Adams-Bashforth weights over one step, oldest first
  // ext[r][j]: weights of mesh r - 1's extrapolation over j / ratios[r - 1] of its step
  std::vector<std::vector<std::vector<double>>> ext;
  std::vector<int> start;  // tick at which each mesh's current step began
  int *d_err = nullptr;
  unsigned long long *d_dt = nullptr;
  double H = 0.0, t = 0.0;
  bool initialised = false;
  size_t esz = 8;

  ~sbp_chain_s() {
    cudaFree(d_err);
    cudaFree(d_dt);
  }
  bool viscous() const { return p.physics == SBP_NS; }
  sbp_system_s &M(int r) { return *mesh[r]; }
  MeshDev &D(int r) { return mesh[r]->md[0]; }
  size_t state_elems(int r) const { return mesh[r]->state_elems(0); }
  void *slot(int r, int s) { return (char *)D(r).hist + (size_t)s * state_elems(r) * esz; }
};

namespace {

using sbp::fail;

// Host setup of the chain: meshes, hole cuts, classes, SAT lists, receivers by donor mesh, donor
// stencils, Adams-Bashforth and extrapolation weights.
sbp_status chain_host_setup(sbp_chain_s &C, const sbp_mesh_desc *meshes, int R, const int *ratios,
                            const sbp_params &p) {
  std::string err;
  sbp_status st;
  C.R = R;
  C.p = p;
  C.p.fast_mesh = 1;  // each mesh's tables sit in slot 0 of a system: no fast-mesh extras
  C.p.step_ratio = 1;
  if (C.p.hole_cells <= 0) C.p.hole_cells = 4;
  C.m = p.hist_len;
  C.esz = p.dtype == SBP_F64 ? 8 : 4;
  C.ratios.assign(ratios, ratios + R - 1);
  C.ticks.assign(R, 1);
  for (int r = R - 2; r >= 0; --r) C.ticks[r] = C.ticks[r + 1] * C.ratios[r];
  for (int r = 0; r < R; ++r) {
    C.mesh.emplace_back(new sbp_system_s());
    C.mesh[r]->p = C.p;
    C.mesh[r]->esz = C.esz;
    if ((st = setup_mesh_basic(meshes[r], C.M(r).mh[0], err)) != SBP_OK) return fail(st, "mesh " + std::to_string(r) + ": " + err);
  }
  for (int r = 1; r < R; ++r) {
    MeshHost &outer = C.M(r - 1).mh[0];
    if (!outer.cartesian) return fail(SBP_ERR_ARG, "every mesh but the innermost must be Cartesian");
    const double margin = C.p.hole_cells * std::max(outer.h[0], outer.h[1]);
    if ((st = setup_holes(outer, C.M(r).mh[0], margin, err)) != SBP_OK) return fail(st, err);
  }
  for (int r = 0; r < R; ++r) {
    MeshHost &mh = C.M(r).mh[0];
    if ((st = setup_classes(mh, err)) != SBP_OK) return fail(st, err);
    if ((st = setup_sat(mh, p.omega_corner, err)) != SBP_OK) return fail(st, err);
  }
  C.recv_src.assign(R, {});
  C.ndv_lo.assign(R, 0);
  for (int r = 0; r < R; ++r) {
    MeshHost &mh = C.M(r).mh[0];
    const size_t nr = mh.recv_pt.size();
    std::vector<int> group[2];  // receivers fed by mesh r - 1, by mesh r + 1
    for (size_t q = 0; q < nr; ++q) {
      const int pt = mh.recv_pt[q];
      const bool face = on_interface_face(mh, pt), hole = next_to_hole(mh, pt);
      if (face && hole) return fail(SBP_ERR_SHAPE, "mesh " + std::to_string(r) + ": a receiver next to both its outer face and a hole");
      const int src = face ? r - 1 : r + 1;
      if (src < 0 || src >= R)
        return fail(SBP_ERR_SHAPE, "mesh " + std::to_string(r) + ": an interface face of the outermost mesh or a hole without an overset mesh");
      C.recv_src[r].push_back(src);
      group[face ? 0 : 1].push_back((int)q);
    }
    mh.donor_base.assign(2 * nr, 0);
    mh.donor_w.assign(8 * nr, 0.0);
    mh.donor_idx.assign(16 * nr, 0);
    mh.donor_pts.clear();
    for (int g = 0; g < 2; ++g) {
      if (group[g].empty()) continue;
      MeshHost tmp = mh;
      tmp.recv_pt.clear();
      for (int q : group[g]) tmp.recv_pt.push_back(mh.recv_pt[q]);
      if ((st = setup_donors(tmp, C.M(g == 0 ? r - 1 : r + 1).mh[0], err)) != SBP_OK)
        return fail(st, "mesh " + std::to_string(r) + ": " + err);
      const int off = (int)mh.donor_pts.size();
      for (size_t e = 0; e < group[g].size(); ++e) {
        const int q = group[g][e];
        for (int c = 0; c < 2; ++c) mh.donor_base[2 * q + c] = tmp.donor_base[2 * e + c];
        for (int c = 0; c < 8; ++c) mh.donor_w[8 * q + c] = tmp.donor_w[8 * e + c];
        for (int c = 0; c < 16; ++c) mh.donor_idx[16 * q + c] = tmp.donor_idx[16 * e + c] + off;
      }
      mh.donor_pts.insert(mh.donor_pts.end(), tmp.donor_pts.begin(), tmp.donor_pts.end());
      if (g == 0) C.ndv_lo[r] = (int)tmp.donor_pts.size();
    }
  }
  // Adams-Bashforth weights over one step, and each mesh's extrapolation of its coarser
  // neighbour to the starts of its own steps within that neighbour's step (Sec. 3.1, 3.3)
  std::vector<double> nodes;
  for (int k = 0; k < C.m; ++k) nodes.push_back((double)(k - (C.m - 1)));
  if ((st = solve_ab_weights(nodes, 0.0, 1.0, p.order, C.ab)) != SBP_OK) return fail(st, "Adams-Bashforth weights");
  C.ext.assign(R, {});
  for (int r = 1; r < R; ++r)
    for (int j = 0; j < C.ratios[r - 1]; ++j) {
      std::vector<double> w;
      if ((st = solve_ab_weights(nodes, 0.0, (double)j / C.ratios[r - 1], p.order, w)) != SBP_OK)
        return fail(st, "extrapolation weights");
      C.ext[r].push_back(w);
    }
  return SBP_OK;
}

}  // namespace

namespace {

// Donor values of mesh r's receivers: the mesh r - 1 group from q_lo plus nb_lo terms of mesh
// r - 1's history ring (oldest first) weighted by beta_lo (FP64 accumulation), the mesh r + 1
// group from q_hi.
cudaError_t chain_donors(sbp_chain_s &C, int r, const void *q_lo, const double *beta_lo, int nb_lo, const void *q_hi,
                         cudaStream_t s) {
  MeshDev &d = C.D(r);
  const int nlo = C.ndv_lo[r], nhi = d.ndv - nlo;
  cudaError_t e = cudaSuccess;
  if (nlo > 0) {
    DonorLaunch a{};
    a.d = C.M(r - 1).dev_mesh(0);
    a.g = C.M(r).gas();
    a.q = q_lo;
    a.nsets = 1;
    a.npts = nlo;
    a.pts = d.dpts;
    a.dv = d.dv;
    a.stride = d.ndv;
    a.nb[0] = nb_lo;
    MeshDev &dl = C.D(r - 1);
    for (int k = 0; k < nb_lo; ++k) {
      a.hist[k] = C.slot(r - 1, (dl.head + 1 + k) % C.m);
      a.beta[0][k] = beta_lo[k];
    }
    e = launch_donor_vals(a, C.p.dtype, C.viscous(), s);
  }
  if (e == cudaSuccess && nhi > 0) {
    DonorLaunch a{};
    a.d = C.M(r + 1).dev_mesh(0);
    a.g = C.M(r).gas();
    a.q = q_hi;
    a.nsets = 1;
    a.npts = nhi;
    a.pts = d.dpts + nlo;
    a.dv = (char *)d.dv + (size_t)nlo * C.esz;
    a.stride = d.ndv;
    e = launch_donor_vals(a, C.p.dtype, C.viscous(), s);
  }
  return e;
}

// Right-hand-side launch of mesh r at state q with its receivers gathered from the donor values.
RhsLaunch chain_rhs_args(sbp_chain_s &C, int r, const void *q) {
  MeshDev &d = C.D(r);
  RhsLaunch a = C.M(r).rhs_args(0, q);
  a.dv = d.dv;
  a.didx = d.didx;
  a.ndv = d.ndv;
  a.err = C.d_err;
  return a;
}

// dq/dt of mesh r into out at the states y[] of all meshes (neighbours' states as they are).
cudaError_t chain_eval_plain(sbp_chain_s &C, int r, void *const *y, void *out, cudaStream_t s) {
  cudaError_t e = chain_donors(C, r, r > 0 ? y[r - 1] : nullptr, nullptr, 0, r + 1 < C.R ? y[r + 1] : nullptr, s);
  if (e != cudaSuccess) return e;
  RhsLaunch a = chain_rhs_args(C, r, y[r]);
  a.mode = 0;
  a.out = out;
  return launch_rhs(a, C.p.dtype, C.viscous(), s);
}

// Mesh r's step from tick tau: donor values, right-hand side at tau fused with the update over
// [tau, tau + h_r], then the finer meshes' steps over the same interval, then the new state
// becomes current.
cudaError_t chain_step(sbp_chain_s &C, int r, int tau, cudaStream_t s) {
  const int m = C.m;
  MeshDev &d = C.D(r);
  double beta[kMaxHist];
  int nb = 0;
  if (r > 0) {
    const int j = (tau - C.start[r - 1]) / C.ticks[r];
    if (j > 0) {
      nb = m;
      for (int k = 0; k < m; ++k) beta[k] = C.ext[r][j][k] * C.h[r - 1];
    }
  }
  cudaError_t e = chain_donors(C, r, r > 0 ? C.D(r - 1).q[C.D(r - 1).cur] : nullptr, beta, nb,
                               r + 1 < C.R ? C.D(r + 1).q[C.D(r + 1).cur] : nullptr, s);
  if (e != cudaSuccess) return e;
  const int slot = (d.head + 1) % m;
  RhsLaunch a = chain_rhs_args(C, r, d.q[d.cur]);
  a.mode = 1;
  a.out = C.slot(r, slot);
  a.qnext = d.q[1 - d.cur];
  a.nold = m - 1;
  for (int k = 0; k < m - 1; ++k) {
    a.hold[k] = C.slot(r, (slot + 1 + k) % m);
    a.alpha[k] = C.ab[k] * C.h[r];
  }
  a.alpha[m - 1] = C.ab[m - 1] * C.h[r];
  if ((e = launch_rhs(a, C.p.dtype, C.viscous(), s)) != cudaSuccess) return e;
  d.head = slot;
  C.start[r] = tau;
  if (r + 1 < C.R)
    for (int j = 0; j < C.ratios[r] && e == cudaSuccess; ++j) e = chain_step(C, r + 1, tau + j * C.ticks[r + 1], s);
  d.cur ^= 1;
  return e;
}

// Heun's RK3 at the innermost step h = H / ticks[0] for (m - 1) ticks[0] steps on all meshes,
// recording mesh r's right-hand side every ticks[r] steps over its last m - 1 steps into its ring.
cudaError_t chain_bootstrap(sbp_chain_s &C, double H, cudaStream_t s) {
  const int R = C.R, m = C.m;
  const double h = H / C.ticks[0];
  std::vector<void *> ystage(R, nullptr), k1tmp(R, nullptr), k23(R, nullptr);
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < R && e == cudaSuccess; ++r) {
    const size_t b = C.state_elems(r) * C.esz;
    e = cudaMalloc(&ystage[r], b);
    if (e == cudaSuccess) e = cudaMalloc(&k1tmp[r], b);
    if (e == cudaSuccess) e = cudaMalloc(&k23[r], b);
    // zeroed: the right-hand sides leave the padding columns unwritten, and the stage updates
    // run over the whole pitched arrays
    if (e == cudaSuccess) e = cudaMemsetAsync(ystage[r], 0, b, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(k1tmp[r], 0, b, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(k23[r], 0, b, s);
    C.D(r).head = -1;
    C.D(r).count = 0;
  }
  const int nsteps = (m - 1) * C.ticks[0];
  std::vector<void *> y(R), k1(R);
  for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
    for (int r = 0; r < R; ++r) {
      MeshDev &d = C.D(r);
      y[r] = d.q[d.cur];
      k1[r] = k1tmp[r];
      if (step % C.ticks[r] == 0 && step >= nsteps - (m - 1) * C.ticks[r]) {
        d.head = (d.head + 1) % m;
        d.count++;
        k1[r] = C.slot(r, d.head);
      }
    }
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = chain_eval_plain(C, r, y.data(), k1[r], s);
    for (int r = 0; r < R && e == cudaSuccess; ++r)
      e = launch_axpy(y[r], k1[r], h / 3.0, nullptr, 0.0, ystage[r], C.state_elems(r), C.p.dtype, s);
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = chain_eval_plain(C, r, ystage.data(), k23[r], s);
    for (int r = 0; r < R && e == cudaSuccess; ++r)
      e = launch_axpy(y[r], k23[r], 2.0 * h / 3.0, nullptr, 0.0, ystage[r], C.state_elems(r), C.p.dtype, s);
    for (int r = 0; r < R && e == cudaSuccess; ++r) e = chain_eval_plain(C, r, ystage.data(), k23[r], s);
    for (int r = 0; r < R && e == cudaSuccess; ++r)
      e = launch_axpy(y[r], k1[r], h / 4.0, k23[r], 3.0 * h / 4.0, y[r], C.state_elems(r), C.p.dtype, s);
  }
  cudaError_t es = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = es;
  for (int r = 0; r < R; ++r) {
    cudaFree(ystage[r]);
    cudaFree(k1tmp[r]);
    cudaFree(k23[r]);
  }
  return e;
}

}  // namespace

extern "C" {

sbp_status sbp_chain_create(const sbp_mesh_desc *meshes, int n_meshes, const int *ratios, const sbp_params *params,
                            sbp_chain_t *out) {
  if (!meshes || !params || !out || (n_meshes > 1 && !ratios)) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  if (n_meshes < 2 || n_meshes > kMaxChain) return fail(SBP_ERR_ARG, "a chain has 2..8 meshes");
  const sbp_params &p = *params;
  if (p.physics != SBP_EULER && p.physics != SBP_NS) return fail(SBP_ERR_ARG, "physics");
  if (p.dtype != SBP_F64 && p.dtype != SBP_F32) return fail(SBP_ERR_DTYPE, "dtype");
  if (!(p.gamma > 1.0) || p.mu < 0.0 || !(p.pr > 0.0)) return fail(SBP_ERR_ARG, "gas constants");
  if (p.order < 1 || p.hist_len < p.order || p.hist_len > kMaxHist) return fail(SBP_ERR_ARG, "order / hist_len");
  if (p.sponge_cells != 0) return fail(SBP_ERR_ARG, "chains take no sponge layer");
  long ticks = 1;
  for (int r = 0; r + 1 < n_meshes; ++r) {
    if (ratios[r] < 1 || ratios[r] > kMaxSets) return fail(SBP_ERR_ARG, "step ratios must be in 1..16");
    ticks *= ratios[r];
    if (ticks > (1 << 20)) return fail(SBP_ERR_ARG, "product of the step ratios above 2^20");
  }
  auto *C = new sbp_chain_s();
  std::unique_ptr<sbp_chain_s> guard(C);
  sbp_status st = chain_host_setup(*C, meshes, n_meshes, ratios, p);
  if (st != SBP_OK) return st;
  CUDA_TRY(cudaMalloc((void **)&C->d_err, sizeof(int)));
  CUDA_TRY(cudaMemset(C->d_err, 0, sizeof(int)));
  CUDA_TRY(cudaMalloc((void **)&C->d_dt, n_meshes * sizeof(unsigned long long)));
  for (int r = 0; r < n_meshes; ++r) {
    sbp_system_s &S = C->M(r);
    CUDA_TRY(cudaMalloc((void **)&S.d_err, sizeof(int)));
    CUDA_TRY(cudaMemset(S.d_err, 0, sizeof(int)));
    if ((st = sbp::upload_mesh_tables(&S, 0)) != SBP_OK) return st;
  }
  CUDA_TRY(cudaDeviceSynchronize());
  C->start.assign(n_meshes, 0);
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp_chain_destroy(sbp_chain_t C) {
  delete C;
  return SBP_OK;
}

sbp_status sbp_chain_mesh_info(sbp_chain_t C, int r, sbp_mesh_info *info) {
  if (!C || r < 0 || r >= C->R || !info) return fail(SBP_ERR_ARG, "bad argument");
  sbp_status st = sbp_mesh_info_get(C->mesh[r].get(), 0, info);
  if (st == SBP_OK) info->hist_bytes = info->state_bytes * C->m;
  return st;
}

sbp_status sbp_chain_tables(sbp_chain_t C, int r, signed char *iblank, int *receivers, int *donor_mesh,
                            int *donor_base, double *donor_w) {
  if (!C || r < 0 || r >= C->R) return fail(SBP_ERR_ARG, "bad argument");
  sbp_status st = sbp_get_tables(C->mesh[r].get(), 0, iblank, nullptr, receivers, donor_base, donor_w);
  if (st == SBP_OK && donor_mesh)
    std::copy(C->recv_src[r].begin(), C->recv_src[r].end(), donor_mesh);
  return st;
}

sbp_status sbp_chain_rhs_eval(sbp_chain_t C, int r, const void *const *q_all, void *rhs, void *stream) {
  if (!C || r < 0 || r >= C->R || !q_all || !rhs) return fail(SBP_ERR_ARG, "bad argument");
  for (int k = 0; k < C->R; ++k)
    if (!q_all[k]) return fail(SBP_ERR_ARG, "a state per mesh is required");
  std::vector<void *> y(C->R);
  for (int k = 0; k < C->R; ++k) y[k] = const_cast<void *>(q_all[k]);  // read only
  CUDA_TRY(chain_eval_plain(*C, r, y.data(), rhs, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp_chain_timestep(sbp_chain_t C, const void *const *q_all, double *dt_mesh, double *H, void *stream) {
  if (!C || !q_all) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  for (int r = 0; r < C->R; ++r) {
    if (!q_all[r]) return fail(SBP_ERR_ARG, "a state per mesh is required");
    CUDA_TRY(launch_dt(C->M(r).dev_mesh(0), C->M(r).gas(), q_all[r], C->p.dtype, C->d_dt + r, s));
  }
  std::vector<unsigned long long> bits(C->R);
  CUDA_TRY(cudaMemcpyAsync(bits.data(), C->d_dt, C->R * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  double Hmin = INFINITY;
  for (int r = 0; r < C->R; ++r) {
    double dt;
    std::memcpy(&dt, &bits[r], sizeof(double));
    if (dt_mesh) dt_mesh[r] = dt;
    Hmin = std::min(Hmin, C->p.cfl * dt * (double)(C->ticks[0] / C->ticks[r]));
  }
  if (H) *H = Hmin;
  return SBP_OK;
}

sbp_status sbp_chain_bind(sbp_chain_t C, int r, void *q_a, void *q_b, void *hist) {
  if (!C || r < 0 || r >= C->R || !q_a || !q_b || !hist) return fail(SBP_ERR_ARG, "bad argument");
  MeshDev &d = C->D(r);
  d.q[0] = q_a;
  d.q[1] = q_b;
  d.hist = hist;
  d.cur = 0;
  d.head = -1;
  d.count = 0;
  C->initialised = false;
  return SBP_OK;
}

sbp_status sbp_chain_current_state(sbp_chain_t C, int r, void **q) {
  if (!C || r < 0 || r >= C->R || !q) return fail(SBP_ERR_ARG, "bad argument");
  *q = C->D(r).q[C->D(r).cur];
  return SBP_OK;
}

sbp_status sbp_chain_mrab_init(sbp_chain_t C, double H, void *stream) {
  if (!C) return fail(SBP_ERR_ARG, "null chain");
  for (int r = 0; r < C->R; ++r)
    if (!C->D(r).hist) return fail(SBP_ERR_STATE, "buffers not bound");
  if (!(H > 0.0)) {
    std::vector<const void *> q(C->R);
    for (int r = 0; r < C->R; ++r) q[r] = C->D(r).q[C->D(r).cur];
    sbp_status st = sbp_chain_timestep(C, q.data(), nullptr, &H, stream);
    if (st != SBP_OK) return st;
  }
  C->h.assign(C->R, H);
  for (int r = 1; r < C->R; ++r) C->h[r] = C->h[r - 1] / C->ratios[r - 1];
  cudaError_t e = chain_bootstrap(*C, H, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(SBP_ERR_CUDA, std::string("bootstrap: ") + cudaGetErrorString(e));
  C->H = H;
  C->t = 0.0;
  std::fill(C->start.begin(), C->start.end(), 0);
  C->initialised = true;
  return SBP_OK;
}

sbp_status sbp_chain_mrab_step(sbp_chain_t C, int n, void *stream) {
  if (!C || n < 0) return fail(SBP_ERR_ARG, "bad argument");
  if (!C->initialised) return fail(SBP_ERR_STATE, "sbp_chain_mrab_init first");
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    CUDA_TRY(chain_step(*C, 0, 0, s));
    C->t += C->H;
  }
  return SBP_OK;
}

sbp_status sbp_chain_mrab_time(sbp_chain_t C, double *H, double *t) {
  if (!C) return fail(SBP_ERR_ARG, "null chain");
  if (H) *H = C->H;
  if (t) *t = C->t;
  return SBP_OK;
}

sbp_status sbp_chain_check(sbp_chain_t C, void *stream) {
  if (!C) return fail(SBP_ERR_ARG, "null chain");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, C->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(C->d_err, 0, sizeof(int)));
  if (e) return fail((sbp_status)e, "device error word set");
  return SBP_OK;
}

}  // extern "C"
