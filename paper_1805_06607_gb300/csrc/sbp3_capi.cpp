// C ABI of the 3D Cartesian overset systems: setup (sbp3_setup.cpp), right-hand side and
// interpolation calls, the time step, and the MRAB integrator with its Runge-Kutta bootstrap
// (Sec. 3.1-3.3), the 2D systems' schedule on 5-variable states. Kernels: sbp3_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "sbp3_device.h"
#include "sbp_system.h"

using namespace sbp;

namespace {

struct Mesh3Dev {
  uint16_t *cls = nullptr;
  void *prim = nullptr, *flux = nullptr, *sat = nullptr;
  int64_t *sat_pt = nullptr;
  uint32_t *sat_code = nullptr;
  int *sat_recv = nullptr;
  double *sat_scale = nullptr;
  int *row_sat = nullptr;
  int64_t *dpts = nullptr;
  int *didx = nullptr;
  void *dwt = nullptr;
  void *dv = nullptr;
  int ndv = 0, dv_sets = 0;
  void *q[2] = {nullptr, nullptr};
  void *hist = nullptr;
  int cur = 0, head = -1;
};

template <typename P>
cudaError_t up3(P *&dst, const void *src, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)&dst, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  if (bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  return e;
}

}  // namespace

struct sbp3_system_s {
  sbp_params p{};
  double qinf[5] = {1, 0, 0, 0, 0};
  Mesh3Host mh[2];
  Mesh3Dev md[2];
  CoeffPlan plan;
  size_t esz = 8;
  int *d_err = nullptr;
  unsigned long long *d_dt = nullptr;
  double H = 0.0, t = 0.0;
  bool initialised = false;
  int kchunk[2] = {0, 0};  // k planes per CTA of the marching right-hand side (0: per-point kernels)

  ~sbp3_system_s() {
    for (auto &d : md) {
      cudaFree(d.cls);
      cudaFree(d.prim);
      cudaFree(d.flux);
      cudaFree(d.sat);
      cudaFree(d.sat_pt);
      cudaFree(d.sat_code);
      cudaFree(d.sat_recv);
      cudaFree(d.sat_scale);
      cudaFree(d.row_sat);
      cudaFree(d.dpts);
      cudaFree(d.didx);
      cudaFree(d.dwt);
      cudaFree(d.dv);
    }
    cudaFree(d_err);
    cudaFree(d_dt);
  }

  bool viscous() const { return p.physics == SBP_NS; }
  int fast() const { return p.fast_mesh; }
  int slow() const { return 1 - p.fast_mesh; }
  size_t field(int k) const { return (size_t)mh[k].pitch * mh[k].n[1] * mh[k].n[2]; }
  size_t state_elems(int k) const { return kNvar3 * field(k); }
  void *hist_slot(int k, int slot) const { return (char *)md[k].hist + (size_t)slot * state_elems(k) * esz; }

  Dev3Mesh dev_mesh(int k) const {
    Dev3Mesh d{};
    const Mesh3Host &m = mh[k];
    d.ni = m.n[0];
    d.nj = m.n[1];
    d.nk = m.n[2];
    d.pitch = m.pitch;
    for (int a = 0; a < 3; ++a) d.per[a] = m.per[a];
    d.field = field(k);
    d.cls = md[k].cls;
    return d;
  }

  template <typename T>
  K3<T> kconst(int k) const {
    K3<T> c{};
    const double g = p.gamma, mu = viscous() ? p.mu : 0.0;
    c.gam = (T)g;
    c.mu = (T)mu;
    c.lam = (T)(-2.0 / 3.0 * mu);
    c.kap = (T)(mu / (p.pr * (g - 1.0)));
    c.sig_int = (T)p.sigma_interface;
    c.sig_phys = (T)p.sigma_physical;
    for (int v = 0; v < 5; ++v) c.qinf[v] = (T)qinf[v];
    for (int a = 0; a < 3; ++a) c.ih[a] = (T)(1.0 / mh[k].h[a]);
    c.sponge_d = 0;
    c.sponge_faces = 0;
    for (int f = 0; f < 6; ++f)
      if (mh[k].bc[f] == SBP_BC_FARFIELD) c.sponge_faces |= 1 << f;
    if (p.sponge_cells > 0 && c.sponge_faces) c.sponge_d = p.sponge_cells;
    for (int d = 0; d < 16; ++d) {
      const double r = d < p.sponge_cells ? (double)(p.sponge_cells - d) / p.sponge_cells : 0.0;
      c.sponge_tab[d] = (T)(p.sponge_strength * r * r);
    }
    return c;
  }

  Donor3Launch donor_args(int recv, const void *q, int set0, int nsets, bool extrapolate) const {
    Donor3Launch a{};
    const int don = 1 - recv, m = plan.m;
    a.d = dev_mesh(don);
    a.cf = kconst<float>(don);
    a.cd = kconst<double>(don);
    a.visc = viscous();
    a.q = q;
    a.nsets = nsets;
    a.npts = md[recv].ndv;
    a.pts = md[recv].dpts;
    a.dv = (char *)md[recv].dv + (size_t)set0 * kRv3 * md[recv].ndv * esz;
    for (int k = 0; k < m && md[don].hist; ++k) a.hist[k] = hist_slot(don, (md[don].head + 1 + k) % m);
    for (int j = 0; j < nsets; ++j) {
      int set = set0 + j;
      a.nb[j] = (extrapolate && set > 0) ? m : 0;
      for (int k = 0; k < m; ++k) a.beta[j][k] = extrapolate ? plan.ext[set][k] * H : 0.0;
    }
    return a;
  }

  Rhs3Launch rhs_args(int k, const void *q, int set) const {
    Rhs3Launch a{};
    const Mesh3Dev &d = md[k];
    a.m = dev_mesh(k);
    a.cf = kconst<float>(k);
    a.cd = kconst<double>(k);
    a.visc = viscous();
    a.q = q;
    a.prim = d.prim;
    a.flux = d.flux;
    a.sat = d.sat;
    a.nsat = (int)mh[k].sat_pt.size();
    a.sat_pt = d.sat_pt;
    a.sat_code = d.sat_code;
    a.sat_recv = d.sat_recv;
    a.sat_scale = d.sat_scale;
    a.row_sat = d.row_sat;
    a.dv = (char *)d.dv + (size_t)set * kRv3 * d.ndv * esz;
    a.didx = d.didx;
    a.dwt = d.dwt;
    a.ndv = d.ndv;
    a.nrecv = (int)mh[k].recv_pt.size();
    a.kchunk = kchunk[k];
    a.err = d_err;
    return a;
  }

  cudaError_t rhs_plain(int k, const void *q_self, const void *q_other, void *out, cudaStream_t s) {
    cudaError_t e = launch3_donor(donor_args(k, q_other, 0, 1, false), p.dtype, s);
    if (e != cudaSuccess) return e;
    Rhs3Launch a = rhs_args(k, q_self, 0);
    a.mode = 0;
    a.out = out;
    return launch3_rhs(a, p.dtype, s);
  }

  cudaError_t fused(int k, int set, double dt, cudaStream_t s) {
    const int m = plan.m;
    const Mesh3Dev &d = md[k];
    int slot = (d.head + 1) % m;
    Rhs3Launch a = rhs_args(k, d.q[d.cur], set);
    a.mode = 1;
    a.out = hist_slot(k, slot);
    a.qnext = d.q[1 - d.cur];
    a.nold = m - 1;
    for (int j = 0; j < m - 1; ++j) {
      a.hold[j] = hist_slot(k, (slot + 1 + j) % m);
      a.alpha[j] = plan.ab[j] * dt;
    }
    a.alpha[m - 1] = plan.ab[m - 1] * dt;
    return launch3_rhs(a, p.dtype, s);
  }

  // One macro step of Sec. 3.3 (the 2D systems' eager schedule).
  cudaError_t issue_step(cudaStream_t s) {
    const int F = fast(), Sl = slow(), sr = plan.sr;
    const double h = H / sr;
    cudaError_t e = cudaSuccess;
    auto run = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    run(launch3_donor(donor_args(Sl, md[F].q[md[F].cur], 0, 1, false), p.dtype, s));
    run(fused(Sl, 0, H, s));
    md[Sl].head = (md[Sl].head + 1) % plan.m;
    run(launch3_donor(donor_args(F, md[Sl].q[md[Sl].cur], 0, sr, true), p.dtype, s));
    for (int j = 0; j < sr; ++j) {
      run(fused(F, j, h, s));
      md[F].head = (md[F].head + 1) % plan.m;
      md[F].cur ^= 1;
    }
    md[Sl].cur ^= 1;
    t += H;
    return e;
  }

  cudaError_t bootstrap(double Hm, cudaStream_t s) {
    const int m = plan.m, sr = plan.sr, F = fast(), Sl = slow();
    const double h = Hm / sr;
    void *ystage[2] = {nullptr, nullptr}, *k1tmp[2] = {nullptr, nullptr}, *k23[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2; ++k) {
      size_t b = state_elems(k) * esz;
      if (e == cudaSuccess) e = cudaMalloc(&ystage[k], b);
      if (e == cudaSuccess) e = cudaMalloc(&k1tmp[k], b);
      if (e == cudaSuccess) e = cudaMalloc(&k23[k], b);
      // zeroed: the right-hand sides leave the padding columns unwritten, and the stage updates
      // run over the whole pitched arrays
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
    cudaError_t es = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = es;
    for (int k = 0; k < 2; ++k) {
      cudaFree(ystage[k]);
      cudaFree(k1tmp[k]);
      cudaFree(k23[k]);
    }
    return e;
  }
};

extern "C" {

// Host part of 3D system creation (no device calls): argument checks, per-mesh setup, hole
// cut, SBP segment classes, SAT lists, donor search and Lagrange weights, the coefficient plan.
static sbp_status host3_setup(const sbp3_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                              sbp_params &pout, Mesh3Host mh[2], CoeffPlan &plan) {
  if (!meshes || !params) return fail(SBP_ERR_ARG, "null argument");
  if (n_meshes != 2) return fail(SBP_ERR_ARG, "exactly two meshes (background, fine box) are supported");
  const sbp_params &p = *params;
  if (p.physics != SBP_EULER && p.physics != SBP_NS) return fail(SBP_ERR_ARG, "physics");
  if (p.dtype != SBP_F64 && p.dtype != SBP_F32) return fail(SBP_ERR_DTYPE, "dtype");
  if (p.fast_mesh != 0 && p.fast_mesh != 1) return fail(SBP_ERR_ARG, "fast_mesh");
  if (!(p.gamma > 1.0) || p.mu < 0.0 || !(p.pr > 0.0)) return fail(SBP_ERR_ARG, "gas constants");
  if (p.step_ratio < 1 || p.step_ratio > kMaxSets)
    return fail(SBP_ERR_ARG, "step_ratio must be in 1.." + std::to_string(kMaxSets));
  if (p.scheme != SBP_MRAB_FASTEST_FIRST) return fail(SBP_ERR_ARG, "3D systems are fastest-first");
  if (p.sponge_cells < 0 || p.sponge_cells > 16 || !(p.sponge_strength >= 0.0))
    return fail(SBP_ERR_ARG, "sponge_cells must be in 0..16 and sponge_strength >= 0");
  pout = p;
  if (pout.hole_cells <= 0) pout.hole_cells = 4;
  std::string err;
  sbp_status st;
  for (int k = 0; k < 2; ++k)
    if ((st = setup3_mesh(meshes[k], mh[k], err)) != SBP_OK) return fail(st, err);
  double margin = pout.hole_cells * std::max({mh[0].h[0], mh[0].h[1], mh[0].h[2]});
  if ((st = setup3_holes(mh[0], mh[1], margin, err)) != SBP_OK) return fail(st, err);
  for (int k = 0; k < 2; ++k) {
    if ((st = setup3_classes(mh[k], err)) != SBP_OK) return fail(st, err);
    if ((st = setup3_sat(mh[k], p.omega_corner, err)) != SBP_OK) return fail(st, err);
  }
  for (int k = 0; k < 2; ++k)
    if ((st = setup3_donors(mh[k], mh[1 - k], err)) != SBP_OK) return fail(st, err);
  if ((st = build_plan(p.order, p.hist_len, p.step_ratio, plan, err)) != SBP_OK) return fail(st, err);
  return SBP_OK;
}

}  // extern "C"

struct sbp3_host_tables_s {
  sbp_params p;
  Mesh3Host mh[2];
  CoeffPlan plan;
};

extern "C" {

sbp_status sbp3_host_tables_create(const sbp3_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                                   sbp3_host_tables_t *out) {
  if (!out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  auto *T = new sbp3_host_tables_s();
  std::unique_ptr<sbp3_host_tables_s> guard(T);
  sbp_status st = host3_setup(meshes, n_meshes, params, T->p, T->mh, T->plan);
  if (st != SBP_OK) return st;
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp3_host_tables_destroy(sbp3_host_tables_t T) {
  delete T;
  return SBP_OK;
}

sbp_status sbp3_host_tables_get(sbp3_host_tables_t T, int k, signed char *iblank, long long *receivers,
                                int *donor_base, double *donor_w, int *n_receivers) {
  if (!T || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const Mesh3Host &m = T->mh[k];
  if (iblank)
    for (size_t q = 0; q < m.points(); ++q) iblank[q] = m.active[q];
  const size_t nr = m.recv_pt.size();
  if (receivers)
    for (size_t r = 0; r < nr; ++r) receivers[r] = (long long)m.recv_pt[r];
  if (donor_base) std::memcpy(donor_base, m.donor_base.data(), 3 * nr * sizeof(int));
  if (donor_w) std::memcpy(donor_w, m.donor_w.data(), 12 * nr * sizeof(double));
  if (n_receivers) *n_receivers = (int)nr;
  return SBP_OK;
}

sbp_status sbp3_system_create(const sbp3_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                              sbp3_system_t *out) {
  if (!meshes || !params || !out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  auto *S = new sbp3_system_s();
  std::unique_ptr<sbp3_system_s> guard(S);
  sbp_status st = host3_setup(meshes, n_meshes, params, S->p, S->mh, S->plan);
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
    Mesh3Host &m = S->mh[k];
    Mesh3Dev &d = S->md[k];
    const int ni = m.n[0], nj = m.n[1], nk = m.n[2];
    const size_t fld = S->field(k);
    std::vector<uint16_t> cls(fld, 0xFFF);
    for (int kk = 0; kk < nk; ++kk)
      for (int j = 0; j < nj; ++j)
        std::memcpy(&cls[((size_t)kk * nj + j) * m.pitch], &m.cls[((size_t)kk * nj + j) * ni], ni * sizeof(uint16_t));
    CUDA_TRY(up3(d.cls, cls.data(), fld * sizeof(uint16_t)));
    if (S->viscous()) {
      CUDA_TRY(cudaMalloc(&d.prim, 4 * fld * S->esz));
      CUDA_TRY(cudaMemset(d.prim, 0, 4 * fld * S->esz));
    }
    CUDA_TRY(cudaMalloc(&d.flux, 15 * fld * S->esz));
    CUDA_TRY(cudaMemset(d.flux, 0, 15 * fld * S->esz));
    const size_t ns = m.sat_pt.size(), nr = m.recv_pt.size();
    CUDA_TRY(cudaMalloc(&d.sat, (5 * ns + 1) * S->esz));
    CUDA_TRY(cudaMemset(d.sat, 0, (5 * ns + 1) * S->esz));
    CUDA_TRY(up3(d.sat_pt, m.sat_pt.data(), ns * sizeof(int64_t)));
    CUDA_TRY(up3(d.sat_code, m.sat_code.data(), ns * sizeof(uint32_t)));
    CUDA_TRY(up3(d.sat_recv, m.sat_recv.data(), ns * sizeof(int)));
    CUDA_TRY(up3(d.sat_scale, m.sat_scale.data(), ns * sizeof(double)));
    std::vector<int> rows((size_t)nj * nk + 1, 0);
    for (int64_t pt : m.sat_pt) rows[(size_t)(pt / ni) + 1]++;
    for (size_t r = 0; r + 1 < rows.size(); ++r) rows[r + 1] += rows[r];
    CUDA_TRY(up3(d.row_sat, rows.data(), rows.size() * sizeof(int)));
    d.ndv = (int)m.donor_pts.size();
    d.dv_sets = k == p.fast_mesh ? p.step_ratio : 1;
    CUDA_TRY(up3(d.dpts, m.donor_pts.data(), m.donor_pts.size() * sizeof(int64_t)));
    CUDA_TRY(up3(d.didx, m.donor_idx.data(), m.donor_idx.size() * sizeof(int)));
    if (p.dtype == SBP_F64) {
      CUDA_TRY(up3(d.dwt, m.donor_w.data(), 12 * nr * sizeof(double)));
    } else {
      std::vector<float> wf(m.donor_w.begin(), m.donor_w.end());
      CUDA_TRY(up3(d.dwt, wf.data(), wf.size() * sizeof(float)));
    }
    CUDA_TRY(cudaMalloc(&d.dv, ((size_t)d.dv_sets * kRv3 * d.ndv + 1) * S->esz));
    CUDA_TRY(cudaMemset(d.dv, 0, ((size_t)d.dv_sets * kRv3 * d.ndv + 1) * S->esz));
  }
  CUDA_TRY(cudaDeviceSynchronize());
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp3_system_destroy(sbp3_system_t S) {
  delete S;
  return SBP_OK;
}

sbp_status sbp3_mesh_info_get(sbp3_system_t S, int k, sbp3_mesh_info *info) {
  if (!S || !info || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const Mesh3Host &m = S->mh[k];
  info->ni = m.n[0];
  info->nj = m.n[1];
  info->nk = m.n[2];
  info->pitch = m.pitch;
  info->field_elems = S->field(k);
  info->state_bytes = S->state_elems(k) * S->esz;
  info->nvar = kNvar3;
  info->n_holes = (int)std::count(m.active.begin(), m.active.end(), 0);
  info->n_receivers = (int)m.recv_pt.size();
  info->n_sat_points = (int)m.sat_pt.size();
  info->elem_size = (int)S->esz;
  return SBP_OK;
}

sbp_status sbp3_set_freestream(sbp3_system_t S, const double *qinf) {
  if (!S || !qinf) return fail(SBP_ERR_ARG, "bad argument");
  for (int v = 0; v < 5; ++v) S->qinf[v] = qinf[v];
  return SBP_OK;
}

sbp_status sbp3_get_tables(sbp3_system_t S, int k, signed char *iblank, long long *receivers, int *donor_base,
                           double *donor_w) {
  if (!S || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const Mesh3Host &m = S->mh[k];
  if (iblank)
    for (size_t p = 0; p < m.points(); ++p) iblank[p] = m.active[p];
  const size_t nr = m.recv_pt.size();
  if (receivers)
    for (size_t r = 0; r < nr; ++r) receivers[r] = (long long)m.recv_pt[r];
  if (donor_base) std::memcpy(donor_base, m.donor_base.data(), 3 * nr * sizeof(int));
  if (donor_w) std::memcpy(donor_w, m.donor_w.data(), 12 * nr * sizeof(double));
  return SBP_OK;
}

sbp_status sbp3_overset_interp(sbp3_system_t S, int recv, const void *q_donor, void *qhat, void *fvhat, void *stream) {
  if (!S || recv < 0 || recv > 1 || !q_donor || !qhat) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(launch3_donor(S->donor_args(recv, q_donor, 0, 1, false), S->p.dtype, s));
  Gather3Launch g{};
  g.dv = S->md[recv].dv;
  g.didx = S->md[recv].didx;
  g.dwt = S->md[recv].dwt;
  g.ndv = S->md[recv].ndv;
  g.nrecv = (int)S->mh[recv].recv_pt.size();
  g.nval = S->viscous() ? kRv3 : 5;
  g.qhat = qhat;
  g.fvhat = S->viscous() ? fvhat : nullptr;
  g.err = S->d_err;
  CUDA_TRY(launch3_gather(g, S->p.dtype, s));
  return SBP_OK;
}

sbp_status sbp3_rhs_eval(sbp3_system_t S, int k, const void *q_self, const void *q_other, void *rhs, void *stream) {
  if (!S || k < 0 || k > 1 || !q_self || !q_other || !rhs) return fail(SBP_ERR_ARG, "bad argument");
  CUDA_TRY(S->rhs_plain(k, q_self, q_other, rhs, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp3_timestep(sbp3_system_t S, const void *q0, const void *q1, double *dt_mesh, double *H, void *stream) {
  if (!S || !q0 || !q1) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const void *qs[2] = {q0, q1};
  const double mu = S->viscous() ? S->p.mu : 0.0;
  for (int k = 0; k < 2; ++k)
    CUDA_TRY(launch3_dt(S->dev_mesh(k), S->kconst<double>(k), mu, S->p.pr, qs[k], S->p.dtype, S->d_dt + k, s));
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

sbp_status sbp3_bind(sbp3_system_t S, int k, void *qa, void *qb, void *hist) {
  if (!S || k < 0 || k > 1 || !qa || !qb || !hist) return fail(SBP_ERR_ARG, "bad argument");
  S->md[k].q[0] = qa;
  S->md[k].q[1] = qb;
  S->md[k].hist = hist;
  S->md[k].cur = 0;
  S->md[k].head = -1;
  S->initialised = false;
  return SBP_OK;
}

sbp_status sbp3_current_state(sbp3_system_t S, int k, void **q) {
  if (!S || k < 0 || k > 1 || !q) return fail(SBP_ERR_ARG, "bad argument");
  *q = S->md[k].q[S->md[k].cur];
  return SBP_OK;
}

sbp_status sbp3_mrab_init(sbp3_system_t S, double H, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  for (int k = 0; k < 2; ++k)
    if (!S->md[k].hist) return fail(SBP_ERR_STATE, "buffers not bound");
  if (!(H > 0.0)) {
    sbp_status st = sbp3_timestep(S, S->md[0].q[S->md[0].cur], S->md[1].q[S->md[1].cur], nullptr, &H, stream);
    if (st != SBP_OK) return st;
  }
  cudaError_t e = S->bootstrap(H, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(SBP_ERR_CUDA, std::string("bootstrap: ") + cudaGetErrorString(e));
  S->H = H;
  S->t = 0.0;
  S->initialised = true;
  return SBP_OK;
}

sbp_status sbp3_mrab_step(sbp3_system_t S, int n, void *stream) {
  if (!S || n < 0) return fail(SBP_ERR_ARG, "bad argument");
  if (!S->initialised) return fail(SBP_ERR_STATE, "sbp3_mrab_init has not run");
  for (int i = 0; i < n; ++i) CUDA_TRY(S->issue_step((cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp3_set_rhs_kernel(sbp3_system_t S, int mesh, int kchunk) {
  if (!S || mesh < 0 || mesh > 1 || kchunk < 0 || kchunk > 4096) return fail(SBP_ERR_ARG, "bad argument");
  S->kchunk[mesh] = kchunk;
  return SBP_OK;
}

sbp_status sbp3_check(sbp3_system_t S, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, S->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
  if (e) return fail((sbp_status)e, "device error word set");
  return SBP_OK;
}

}  // extern "C"
