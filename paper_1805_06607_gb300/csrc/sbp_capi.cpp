// C ABI of the library: system creation (host setup + device tables), right-hand side and
// interpolation calls, the time-step reduction, and the MRAB integrator with its Runge-Kutta
// bootstrap. Device work is issued on the caller's stream; the GPU kernels live in
// sbp_kernels.cu.
#include "sbp_system.h"


extern "C" {

const char *sbp_status_string(sbp_status s) {
  switch (s) {
    case SBP_OK: return "ok";
    case SBP_ERR_ARG: return "invalid argument";
    case SBP_ERR_SHAPE: return "invalid shape";
    case SBP_ERR_DTYPE: return "unsupported element type";
    case SBP_ERR_CUDA: return "CUDA error";
    case SBP_ERR_NONFINITE: return "non-finite state";
    case SBP_ERR_DONOR: return "no donor";
    case SBP_ERR_TIMEOUT: return "device wait timed out";
    case SBP_ERR_BOUNDS: return "index out of bounds";
    case SBP_ERR_STATE: return "call out of order";
  }
  return "unknown status";
}

const char *sbp_last_error_message(void) { return g_msg.c_str(); }

// Host part of system creation (no device calls): argument checks, per-mesh setup, hole cut,
// SBP segment classes, SAT lists, donor search and Lagrange weights, the coefficient plan.
static sbp_status host_setup(const sbp_mesh_desc *meshes, int n_meshes, const sbp_params *params, sbp_params &pout,
                             MeshHost mh[2], CoeffPlan &plan) {
  if (!meshes || !params) return fail(SBP_ERR_ARG, "null argument");
  if (n_meshes != 2) return fail(SBP_ERR_ARG, "exactly two meshes (background, fine) are supported");
  const sbp_params &p = *params;
  if (p.physics != SBP_EULER && p.physics != SBP_NS) return fail(SBP_ERR_ARG, "physics");
  if (p.dtype != SBP_F64 && p.dtype != SBP_F32) return fail(SBP_ERR_DTYPE, "dtype");
  if (p.fast_mesh != 0 && p.fast_mesh != 1) return fail(SBP_ERR_ARG, "fast_mesh");
  if (!(p.gamma > 1.0) || p.mu < 0.0 || !(p.pr > 0.0)) return fail(SBP_ERR_ARG, "gas constants");
  if (p.step_ratio < 1 || p.step_ratio > kMaxSets)
    return fail(SBP_ERR_ARG, "step_ratio must be in 1.." + std::to_string(kMaxSets));
  if (p.scheme < SBP_MRAB_FASTEST_FIRST || p.scheme > SBP_MRAB_SLOWEST_FIRST_REEXTRAPOLATE)
    return fail(SBP_ERR_ARG, "scheme");
  if (p.sponge_cells < 0 || p.sponge_cells > 16 || !(p.sponge_strength >= 0.0))
    return fail(SBP_ERR_ARG, "sponge_cells must be in 0..16 and sponge_strength >= 0");
  pout = p;
  if (pout.hole_cells <= 0) pout.hole_cells = 4;
  std::string err;
  sbp_status st;
  for (int k = 0; k < 2; ++k)
    if ((st = setup_mesh_basic(meshes[k], mh[k], err)) != SBP_OK) return fail(st, err);
  if (!mh[0].cartesian) return fail(SBP_ERR_ARG, "the background (mesh 0) must be Cartesian");
  double margin = pout.hole_cells * std::max(mh[0].h[0], mh[0].h[1]);
  if ((st = setup_holes(mh[0], mh[1], margin, err)) != SBP_OK) return fail(st, err);
  for (int k = 0; k < 2; ++k) {
    if ((st = setup_classes(mh[k], err)) != SBP_OK) return fail(st, err);
    if ((st = setup_sat(mh[k], p.omega_corner, err)) != SBP_OK) return fail(st, err);
  }
  for (int k = 0; k < 2; ++k)
    if ((st = setup_donors(mh[k], mh[1 - k], err)) != SBP_OK) return fail(st, err);
  if ((st = build_plan(p.order, p.hist_len, p.step_ratio, plan, err)) != SBP_OK) return fail(st, err);
  return SBP_OK;
}

}  // extern "C"

struct sbp_host_tables_s {
  sbp_params p;
  MeshHost mh[2];
  CoeffPlan plan;
};

extern "C" {

sbp_status sbp_host_tables_create(const sbp_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                                  sbp_host_tables_t *out) {
  if (!out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  auto *T = new sbp_host_tables_s();
  std::unique_ptr<sbp_host_tables_s> guard(T);
  sbp_status st = host_setup(meshes, n_meshes, params, T->p, T->mh, T->plan);
  if (st != SBP_OK) return st;
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp_host_tables_destroy(sbp_host_tables_t T) {
  delete T;
  return SBP_OK;
}

sbp_status sbp_host_tables_get(sbp_host_tables_t T, int k, signed char *iblank, int *receivers, int *donor_base,
                               double *donor_w, int *n_receivers) {
  if (!T || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const MeshHost &m = T->mh[k];
  const size_t n = (size_t)m.ni * m.nj, nr = m.recv_pt.size();
  if (iblank)
    for (size_t q = 0; q < n; ++q) iblank[q] = m.active[q];
  if (receivers) std::memcpy(receivers, m.recv_pt.data(), nr * sizeof(int));
  if (donor_base) std::memcpy(donor_base, m.donor_base.data(), 2 * nr * sizeof(int));
  if (donor_w) std::memcpy(donor_w, m.donor_w.data(), 8 * nr * sizeof(double));
  if (n_receivers) *n_receivers = (int)nr;
  return SBP_OK;
}

sbp_status sbp_host_tables_plan(sbp_host_tables_t T, double *ab, double *ext, int *m, int *sr) {
  if (!T) return fail(SBP_ERR_ARG, "null argument");
  const CoeffPlan &c = T->plan;
  if (m) *m = c.m;
  if (sr) *sr = c.sr;
  if (ab) std::memcpy(ab, c.ab.data(), c.m * sizeof(double));
  if (ext)
    for (int j = 0; j < c.sr; ++j) std::memcpy(ext + (size_t)j * c.m, c.ext[j].data(), c.m * sizeof(double));
  return SBP_OK;
}

}  // extern "C"

// Device tables of mesh k of a system (class map, metrics, SAT lists by tile, donor tables and
// workspaces) from its host setup; used by system creation and by the chains of nested meshes.
sbp_status sbp::upload_mesh_tables(sbp_system_s *S, int k) {
  const sbp_params &p = S->p;
  MeshHost &m = S->mh[k];
  MeshDev &d = S->md[k];
  size_t field = (size_t)m.pitch * m.nj;
  std::vector<uint8_t> cls(field, 0xFF);
  for (int j = 0; j < m.nj; ++j)
    std::memcpy(&cls[(size_t)j * m.pitch], &m.cls[(size_t)j * m.ni], m.ni);
  CUDA_TRY(upload(d.cls, cls.data(), field));
  if (!m.cartesian) {
    CUDA_TRY(cudaMalloc(&d.met, 5 * field * S->esz));
    CUDA_TRY(cudaMemset(d.met, 0, 5 * field * S->esz));
    double *dx = nullptr, *dy = nullptr;
    CUDA_TRY(upload(dx, m.x.data(), m.x.size() * sizeof(double)));
    CUDA_TRY(upload(dy, m.y.data(), m.y.size() * sizeof(double)));
    DevMesh dm = S->dev_mesh(k);
    cudaError_t e = launch_metrics(dm, dx, dy, m.shift, d.met, p.dtype, 0);
    cudaError_t e2 = cudaDeviceSynchronize();
    cudaFree(dx);
    cudaFree(dy);
    CUDA_TRY(e);
    CUDA_TRY(e2);
  }
  // SAT points grouped by 32 x 8 tile, tiles in column-major order so that the tiles of a
  // taller CTA (16 or 32 rows) are contiguous
  const int ntx = (m.ni + kTileX - 1) / kTileX, nty8 = (m.nj + 7) / 8;
  size_t ns = m.sat_pt.size();
  std::vector<int> order(ns);
  for (size_t s = 0; s < ns; ++s) order[s] = (int)s;
  auto tile_of = [&](int pt) { return ((pt % m.ni) / kTileX) * nty8 + (pt / m.ni) / 8; };
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return tile_of(m.sat_pt[a]) < tile_of(m.sat_pt[b]); });
  std::vector<int> toff((size_t)ntx * nty8 + 1, 0);
  std::vector<uint32_t> ij(ns), code(ns);
  std::vector<int> recv(ns);
  std::vector<double> scale(ns);
  for (size_t s = 0; s < ns; ++s) {
    int o = order[s], pt = m.sat_pt[o];
    toff[tile_of(pt) + 1]++;
    ij[s] = (uint32_t)(pt % m.ni) | ((uint32_t)(pt / m.ni) << 16);
    code[s] = m.sat_code[o];
    recv[s] = m.sat_recv[o];
    scale[s] = m.sat_scale[o];
  }
  for (size_t t = 0; t + 1 < toff.size(); ++t) toff[t + 1] += toff[t];
  CUDA_TRY(upload(d.tile_sat, toff.data(), toff.size() * sizeof(int)));
  // workspaces start zeroed: entries no kernel writes (padding columns, holes) never carry stale
  // device memory into a result
  CUDA_TRY(cudaMalloc(&d.flux, 8 * field * S->esz));
  CUDA_TRY(cudaMemset(d.flux, 0, 8 * field * S->esz));
  d.rows_per_cta = d.e_rows = 16;
  if (p.physics == SBP_NS && k == p.fast_mesh) {
    CUDA_TRY(cudaMalloc(&d.prim, 3 * field * S->esz));
    CUDA_TRY(cudaMemset(d.prim, 0, 3 * field * S->esz));
  }
  CUDA_TRY(upload(d.sat_ij, ij.data(), ns * sizeof(uint32_t)));
  CUDA_TRY(upload(d.sat_code, code.data(), ns * sizeof(uint32_t)));
  CUDA_TRY(upload(d.sat_recv, recv.data(), ns * sizeof(int)));
  CUDA_TRY(upload(d.sat_scale, scale.data(), ns * sizeof(double)));
  size_t nr = m.recv_pt.size();
  CUDA_TRY(upload(d.base, m.donor_base.data(), 2 * nr * sizeof(int)));
  CUDA_TRY(upload(d.w, m.donor_w.data(), 8 * nr * sizeof(double)));
  if (p.dtype == SBP_F64) {
    CUDA_TRY(upload(d.wt, m.donor_w.data(), 8 * nr * sizeof(double)));
  } else {
    std::vector<float> wf(m.donor_w.begin(), m.donor_w.end());
    CUDA_TRY(upload(d.wt, wf.data(), wf.size() * sizeof(float)));
  }
  CUDA_TRY(cudaMalloc(&d.sat, (4 * ns + 1) * S->esz));
  CUDA_TRY(cudaMemset(d.sat, 0, (4 * ns + 1) * S->esz));
  CUDA_TRY(cudaMalloc(&d.qhat, (4 * nr + 1) * S->esz));
  CUDA_TRY(cudaMemset(d.qhat, 0, (4 * nr + 1) * S->esz));
  CUDA_TRY(cudaMalloc(&d.fvhat, (6 * nr + 1) * S->esz));
  CUDA_TRY(cudaMemset(d.fvhat, 0, (6 * nr + 1) * S->esz));
  d.ndv = (int)m.donor_pts.size();
  d.dv_sets = k == p.fast_mesh ? p.step_ratio : 1;
  CUDA_TRY(upload(d.dpts, m.donor_pts.data(), m.donor_pts.size() * sizeof(uint32_t)));
  CUDA_TRY(upload(d.didx, m.donor_idx.data(), m.donor_idx.size() * sizeof(int)));
  CUDA_TRY(cudaMalloc(&d.dv, ((size_t)d.dv_sets * 10 * d.ndv + 1) * S->esz));
  CUDA_TRY(cudaMemset(d.dv, 0, ((size_t)d.dv_sets * 10 * d.ndv + 1) * S->esz));
  return SBP_OK;
}

extern "C" {

sbp_status sbp_system_create(const sbp_mesh_desc *meshes, int n_meshes, const sbp_params *params,
                             sbp_system_t *out) {
  if (!meshes || !params || !out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  auto *S = new sbp_system_s();
  std::unique_ptr<sbp_system_s> guard(S);
  sbp_status st = host_setup(meshes, n_meshes, params, S->p, S->mh, S->plan);
  if (st != SBP_OK) return st;
  const sbp_params &p = S->p;
  S->esz = p.dtype == SBP_F64 ? 8 : 4;

  // device tables
  CUDA_TRY(cudaMalloc((void **)&S->d_err, sizeof(int)));
  CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
  CUDA_TRY(cudaMalloc((void **)&S->d_dt, 2 * sizeof(unsigned long long)));
  for (int k = 0; k < 2; ++k) {
    sbp_status st2 = upload_mesh_tables(S, k);
    if (st2 != SBP_OK) return st2;
  }
  CUDA_TRY(cudaDeviceSynchronize());
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp_system_destroy(sbp_system_t sys) {
  delete sys;
  return SBP_OK;
}

sbp_status sbp_mesh_info_get(sbp_system_t S, int k, sbp_mesh_info *info) {
  if (!S || !info || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const MeshHost &m = S->mh[k];
  info->ni = m.ni;
  info->nj = m.nj;
  info->pitch = m.pitch;
  info->field_elems = (size_t)m.pitch * m.nj;
  info->state_bytes = S->state_elems(k) * S->esz;
  info->hist_bytes = info->state_bytes * S->p.hist_len;
  info->nvar = kNvar;
  info->n_holes = (int)std::count(m.active.begin(), m.active.end(), 0);
  info->n_receivers = (int)m.recv_pt.size();
  info->n_sat_points = (int)m.sat_pt.size();
  info->elem_size = (int)S->esz;
  info->rows_per_cta = S->md[k].strip ? S->md[k].chunk : S->md[k].rows_per_cta;
  info->rows_update = S->md[k].strip ? 0 : (S->md[k].rows_upd ? S->md[k].rows_upd : S->md[k].rows_per_cta);
  info->strip_width = S->md[k].strip ? S->md[k].strip : kTileX;
  info->single_pass = S->md[k].strip ? 1 : 0;
  const MeshDev &d = S->md[k];
  info->eval_rows_per_cta = d.e_strip ? d.e_chunk : d.e_rows;
  info->eval_rows_update = d.e_strip ? 0 : (d.e_rows_upd ? d.e_rows_upd : d.e_rows);
  info->eval_strip_width = d.e_strip ? d.e_strip : kTileX;
  info->eval_single_pass = d.e_strip ? 1 : 0;
  return SBP_OK;
}

sbp_status sbp_get_tables(sbp_system_t S, int k, signed char *iblank, double *metrics, int *receivers,
                          int *donor_base, double *donor_w) {
  if (!S || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  const MeshHost &m = S->mh[k];
  size_t n = (size_t)m.ni * m.nj, field = (size_t)m.pitch * m.nj;
  if (iblank)
    for (size_t p = 0; p < n; ++p) iblank[p] = m.active[p];
  if (metrics) {
    if (m.cartesian) {
      double c[5] = {m.h[1], 0.0, 0.0, m.h[0], 1.0 / (m.h[0] * m.h[1])};
      for (int q = 0; q < 5; ++q)
        for (size_t p = 0; p < n; ++p) metrics[q * n + p] = m.active[p] ? c[q] : (q == 0 || q == 3 || q == 4 ? 1.0 : 0.0);
    } else {
      std::vector<char> buf(5 * field * S->esz);
      CUDA_TRY(cudaMemcpy(buf.data(), S->md[k].met, buf.size(), cudaMemcpyDeviceToHost));
      for (int q = 0; q < 5; ++q)
        for (int j = 0; j < m.nj; ++j)
          for (int i = 0; i < m.ni; ++i) {
            size_t src = q * field + (size_t)j * m.pitch + i;
            metrics[q * n + (size_t)j * m.ni + i] =
                S->esz == 8 ? ((double *)buf.data())[src] : (double)((float *)buf.data())[src];
          }
    }
  }
  size_t nr = m.recv_pt.size();
  if (receivers) std::memcpy(receivers, m.recv_pt.data(), nr * sizeof(int));
  if (donor_base) std::memcpy(donor_base, m.donor_base.data(), 2 * nr * sizeof(int));
  if (donor_w) std::memcpy(donor_w, m.donor_w.data(), 8 * nr * sizeof(double));
  return SBP_OK;
}

sbp_status sbp_overset_interp(sbp_system_t S, int recv, const void *q_donor, void *qhat, void *fvhat, void *stream) {
  if (!S || recv < 0 || recv > 1 || !q_donor || !qhat) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  InterpLaunch a{};
  a.d = S->dev_mesh(1 - recv);
  a.g = S->gas();
  a.q = q_donor;
  a.nrecv = (int)S->mh[recv].recv_pt.size();
  a.base = S->md[recv].base;
  a.w = S->md[recv].w;
  a.qhat = qhat;
  a.fvhat = S->viscous() ? fvhat : nullptr;
  CUDA_TRY(launch_interp(a, S->p.dtype, S->viscous(), s));
  return SBP_OK;
}

sbp_status sbp_rhs_eval(sbp_system_t S, int k, const void *q_self, const void *q_other, void *rhs, void *stream) {
  if (!S || k < 0 || k > 1 || !q_self || !q_other || !rhs) return fail(SBP_ERR_ARG, "bad argument");
  CUDA_TRY(S->rhs_plain(k, q_self, q_other, rhs, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp_rhs_eval_noalloc(sbp_system_t S, int k, const void *q_self, const void *q_other, void *rhs,
                                void *stream) {
  if (!S || k < 0 || k > 1 || !q_self || !q_other || !rhs) return fail(SBP_ERR_ARG, "bad argument");
  int nrecv = (int)S->mh[k].recv_pt.size();
  if (nrecv > SBP_NOALLOC_MAX_RECEIVERS)
    return fail(SBP_ERR_SHAPE, "mesh has " + std::to_string(nrecv) + " receivers; sbp_rhs_eval_noalloc supports " +
                                   std::to_string(SBP_NOALLOC_MAX_RECEIVERS));
  InterpLaunch ia{};
  ia.d = S->dev_mesh(1 - k);
  ia.g = S->gas();
  ia.q = q_other;
  ia.nrecv = nrecv;
  ia.base = S->md[k].base;
  ia.w = S->md[k].w;
  RhsLaunch ra = S->rhs_args(k, q_self, true);
  ra.mode = 0;
  ra.out = rhs;
  CUDA_TRY(rhs_eval_static_scratch(ia, ra, S->p.dtype, S->viscous(), S->esz, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp_timestep(sbp_system_t S, const void *q0, const void *q1, double *dt_mesh, double *H, void *stream) {
  if (!S || !q0 || !q1) return fail(SBP_ERR_ARG, "bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  const void *qs[2] = {q0, q1};
  for (int k = 0; k < 2; ++k) CUDA_TRY(launch_dt(S->dev_mesh(k), S->gas(), qs[k], S->p.dtype, S->d_dt + k, s));
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

sbp_status sbp_bind(sbp_system_t S, int k, void *qa, void *qb, void *hist) {
  if (!S || k < 0 || k > 1 || !qa || !qb || !hist) return fail(SBP_ERR_ARG, "bad argument");
  MeshDev &d = S->md[k];
  d.q[0] = qa;
  d.q[1] = qb;
  d.hist = hist;
  d.cur = 0;
  d.head = -1;
  d.count = 0;
  S->initialised = false;
  S->clear_graphs();
  return SBP_OK;
}

sbp_status sbp_current_state(sbp_system_t S, int k, void **q) {
  if (!S || k < 0 || k > 1 || !q) return fail(SBP_ERR_ARG, "bad argument");
  *q = S->md[k].q[S->md[k].cur];
  return SBP_OK;
}

sbp_status sbp_integrator_state(sbp_system_t S, int k, void *q, void *hist, int set, void *stream) {
  if (!S || k < 0 || k > 1 || !q || !hist || (set != 0 && set != 1)) return fail(SBP_ERR_ARG, "bad argument");
  if (!S->initialised) return fail(SBP_ERR_STATE, "sbp_mrab_init has not run");
  if (S->p.scheme != SBP_MRAB_FASTEST_FIRST) return fail(SBP_ERR_STATE, "fastest-first systems only");
  cudaStream_t s = (cudaStream_t)stream;
  const MeshDev &d = S->md[k];
  const size_t b = S->state_elems(k) * S->esz;
  const int m = S->plan.m;
  void *cur = d.q[d.cur];
  CUDA_TRY(set ? cudaMemcpyAsync(cur, q, b, cudaMemcpyDeviceToDevice, s)
               : cudaMemcpyAsync(q, cur, b, cudaMemcpyDeviceToDevice, s));
  // the m - 1 entries the next macro step reads, oldest first: slots head + 2 + j (mod m)
  for (int j = 0; j < m - 1; ++j) {
    void *slot = S->hist_slot(k, (d.head + 2 + j) % m);
    void *user = (char *)hist + (size_t)j * b;
    CUDA_TRY(set ? cudaMemcpyAsync(slot, user, b, cudaMemcpyDeviceToDevice, s)
                 : cudaMemcpyAsync(user, slot, b, cudaMemcpyDeviceToDevice, s));
  }
  return SBP_OK;
}

// Checkpoint blob: a fixed header, then per mesh the current state and the m history ring
// slots in slot order (each state_elems * esz bytes).
namespace {
struct CkptHeader {
  char magic[8];
  int32_t version, dtype, physics, scheme, m, sr;
  int64_t state_elems[2];
  int32_t cur[2], head[2], count[2], var_left;
  double H, t;
  double tnode[2][kMaxHist];
};
constexpr char kCkptMagic[8] = {'S', 'B', 'P', 'C', 'K', 'P', 'T', '1'};

size_t ckpt_bytes(const sbp_system_s *S) {
  size_t b = sizeof(CkptHeader);
  for (int k = 0; k < 2; ++k) b += (size_t)(1 + S->plan.m) * S->state_elems(k) * S->esz;
  return b;
}
}  // namespace

sbp_status sbp_checkpoint_save(sbp_system_t S, void *blob, size_t *size, void *stream) {
  if (!S || !size) return fail(SBP_ERR_ARG, "bad argument");
  if (!S->initialised) return fail(SBP_ERR_STATE, "sbp_mrab_init has not run");
  const size_t need = ckpt_bytes(S);
  if (!blob) {
    *size = need;
    return SBP_OK;
  }
  if (*size < need) return fail(SBP_ERR_ARG, "checkpoint buffer too small");
  cudaStream_t s = (cudaStream_t)stream;
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, sizeof(h.magic));
  h.version = 1;
  h.dtype = S->p.dtype;
  h.physics = S->p.physics;
  h.scheme = S->p.scheme;
  h.m = S->plan.m;
  h.sr = S->plan.sr;
  for (int k = 0; k < 2; ++k) {
    h.state_elems[k] = (int64_t)S->state_elems(k);
    h.cur[k] = S->md[k].cur;
    h.head[k] = S->md[k].head;
    h.count[k] = S->md[k].count;
  }
  h.var_left = S->var_left;
  h.H = S->H;
  h.t = S->t;
  std::memcpy(h.tnode, S->tnode, sizeof(h.tnode));
  char *out = static_cast<char *>(blob);
  std::memcpy(out, &h, sizeof(h));
  size_t off = sizeof(h);
  for (int k = 0; k < 2; ++k) {
    const size_t b = S->state_elems(k) * S->esz;
    CUDA_TRY(cudaMemcpyAsync(out + off, S->md[k].q[S->md[k].cur], b, cudaMemcpyDeviceToHost, s));
    off += b;
    CUDA_TRY(cudaMemcpyAsync(out + off, S->md[k].hist, (size_t)S->plan.m * b, cudaMemcpyDeviceToHost, s));
    off += (size_t)S->plan.m * b;
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  *size = need;
  return SBP_OK;
}

sbp_status sbp_checkpoint_load(sbp_system_t S, const void *blob, size_t size, void *stream) {
  if (!S || !blob) return fail(SBP_ERR_ARG, "bad argument");
  for (int k = 0; k < 2; ++k)
    if (!S->md[k].hist) return fail(SBP_ERR_STATE, "buffers not bound");
  if (size < sizeof(CkptHeader)) return fail(SBP_ERR_ARG, "checkpoint too short");
  CkptHeader h;
  std::memcpy(&h, blob, sizeof(h));
  if (std::memcmp(h.magic, kCkptMagic, sizeof(h.magic)) != 0 || h.version != 1)
    return fail(SBP_ERR_ARG, "not a checkpoint of this library");
  if (h.dtype != S->p.dtype || h.physics != S->p.physics || h.scheme != S->p.scheme || h.m != S->plan.m ||
      h.sr != S->plan.sr)
    return fail(SBP_ERR_ARG, "checkpoint of a system with another dtype, physics, scheme, history or ratio");
  for (int k = 0; k < 2; ++k) {
    if (h.state_elems[k] != (int64_t)S->state_elems(k)) return fail(SBP_ERR_SHAPE, "checkpoint of other meshes");
    if (h.cur[k] < 0 || h.cur[k] > 1 || h.head[k] < 0 || h.head[k] >= h.m || h.count[k] < 0)
      return fail(SBP_ERR_ARG, "corrupt checkpoint header");
  }
  if (!(h.H > 0.0) || !std::isfinite(h.H) || !std::isfinite(h.t) || h.var_left < 0 || h.var_left > h.m)
    return fail(SBP_ERR_ARG, "corrupt checkpoint header");
  if (size < ckpt_bytes(S)) return fail(SBP_ERR_ARG, "checkpoint too short");
  cudaStream_t s = (cudaStream_t)stream;
  const char *in = static_cast<const char *>(blob);
  size_t off = sizeof(h);
  for (int k = 0; k < 2; ++k) {
    const size_t b = S->state_elems(k) * S->esz;
    CUDA_TRY(cudaMemcpyAsync(S->md[k].q[h.cur[k]], in + off, b, cudaMemcpyHostToDevice, s));
    off += b;
    CUDA_TRY(cudaMemcpyAsync(S->md[k].hist, in + off, (size_t)h.m * b, cudaMemcpyHostToDevice, s));
    off += (size_t)h.m * b;
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int k = 0; k < 2; ++k) {
    S->md[k].cur = h.cur[k];
    S->md[k].head = h.head[k];
    S->md[k].count = h.count[k];
  }
  S->var_left = h.var_left;
  S->H = h.H;
  S->t = h.t;
  std::memcpy(S->tnode, h.tnode, sizeof(S->tnode));
  S->initialised = true;
  S->clear_graphs();
  return SBP_OK;
}

sbp_status sbp_mrab_init(sbp_system_t S, double H, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  for (int k = 0; k < 2; ++k)
    if (!S->md[k].hist) return fail(SBP_ERR_STATE, "buffers not bound");
  cudaStream_t s = (cudaStream_t)stream;
  if (!(H > 0.0)) {
    sbp_status st = sbp_timestep(S, S->md[0].q[S->md[0].cur], S->md[1].q[S->md[1].cur], nullptr, &H, stream);
    if (st != SBP_OK) return st;
  }
  cudaError_t e = S->bootstrap(H, s, nullptr);
  if (e != cudaSuccess) return fail(SBP_ERR_CUDA, std::string("bootstrap: ") + cudaGetErrorString(e));
  S->H = H;
  S->t = 0.0;
  S->var_left = 0;
  S->initialised = true;
  S->clear_graphs();
  if (S->autotune_on) CUDA_TRY(S->autotune(s));
  // slowest-first macro steps start with the slow history ending at the current time
  if (S->p.scheme != SBP_MRAB_FASTEST_FIRST) CUDA_TRY(S->slow_rhs_push(s));
  return SBP_OK;
}

sbp_status sbp_autotune(sbp_system_t S, int enable, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  S->autotune_on = enable != 0;
  if (S->autotune_on && S->initialised) {
    CUDA_TRY(S->autotune((cudaStream_t)stream));
    S->clear_graphs();
  }
  return SBP_OK;
}

sbp_status sbp_set_rhs_shape(sbp_system_t S, int k, int strip, int rows) {
  if (!S || k < 0 || k > 1) return fail(SBP_ERR_ARG, "bad argument");
  MeshDev &d = S->md[k];
  if (strip == 0) {
    const int rf = rows & 0xFF, ru = rows >> 8;
    if (rf != 4 && rf != 8 && rf != 16 && rf != 32)
      return fail(SBP_ERR_ARG, "split kernels take 4, 8, 16 or 32 rows per CTA");
    if (ru != 0 && ru != 4 && ru != 8 && ru != 16 && ru != 32)
      return fail(SBP_ERR_ARG, "the derivative kernel takes 4, 8, 16 or 32 rows per CTA");
    d.strip = d.e_strip = 0;
    d.rows_per_cta = d.e_rows = rf;
    d.rows_upd = d.e_rows_upd = ru;
  } else {
    if (strip != kMarchW && strip != kColW128 && strip != kColW256)
      return fail(SBP_ERR_ARG, "single-pass strips are " + std::to_string(kMarchW) + " (marching kernel), " +
                                   std::to_string(kColW128) + " or " + std::to_string(kColW256) +
                                   " (column-marching kernel) columns wide");
    if (strip != kMarchW && S->mh[k].ni < strip + 12)
      return fail(SBP_ERR_ARG, "the column-marching kernel needs a mesh at least as wide as its CTA");
    const int chunk = rows & (kStageTma - 1), staging = rows >> 16;
    if (chunk < 1 || staging < 0 || staging > 1) return fail(SBP_ERR_ARG, "chunk rows out of range");
    if (staging && strip != kMarchW) return fail(SBP_ERR_ARG, "TMA staging is the marching kernel's");
    d.strip = d.e_strip = strip;
    d.chunk = d.e_chunk = rows;
  }
  S->clear_graphs();
  return SBP_OK;
}

sbp_status sbp_mrab_step(sbp_system_t S, int n, void *stream) {
  if (!S || n < 0) return fail(SBP_ERR_ARG, "bad argument");
  if (!S->initialised) return fail(SBP_ERR_STATE, "sbp_mrab_init has not run");
  cudaStream_t s = (cudaStream_t)stream;
  for (int step = 0; step < n; ++step) {
    if (S->var_left > 0) {
      sbp_system_s::StepCoef c;
      if (!S->step_coef(c)) return fail(SBP_ERR_ARG, "singular moment system for the history's node times");
      CUDA_TRY(S->issue_step(s, nullptr, nullptr, &c));
      S->var_left--;
    } else if (S->use_graph && !S->prof) {
      CUDA_TRY(S->launch_step_graph(s));
    } else {
      CUDA_TRY(S->issue_step(s, nullptr));
    }
    S->advance();
  }
  return SBP_OK;
}

sbp_status sbp_mrab_set_step(sbp_system_t S, double H) {
  if (!S || !(H > 0.0) || !std::isfinite(H)) return fail(SBP_ERR_ARG, "bad argument");
  if (!S->initialised) return fail(SBP_ERR_STATE, "sbp_mrab_init has not run");
  if (S->p.scheme != SBP_MRAB_FASTEST_FIRST) return fail(SBP_ERR_STATE, "fastest-first systems only");
  if (H != S->H) {
    S->H = H;
    S->var_left = S->plan.m - 1;  // until the histories hold m values spaced by the new step
    S->clear_graphs();
  }
  return SBP_OK;
}

sbp_status sbp_rk4_step(sbp_system_t S, int n, double h, void *stream) {
  if (!S || n < 0 || !(h > 0.0) || !std::isfinite(h)) return fail(SBP_ERR_ARG, "bad argument");
  for (int k = 0; k < 2; ++k)
    if (!S->md[k].hist) return fail(SBP_ERR_STATE, "buffers not bound");
  CUDA_TRY(S->rk4(n, h, (cudaStream_t)stream));
  S->initialised = false;
  S->t += n * h;
  return SBP_OK;
}

sbp_status sbp_mrab_time(sbp_system_t S, double *H, double *t) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  if (H) *H = S->H;
  if (t) *t = S->t;
  return SBP_OK;
}

sbp_status sbp_use_graphs(sbp_system_t S, int enable) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  S->use_graph = enable != 0;
  return SBP_OK;
}

sbp_status sbp_graph_launches(sbp_system_t S, int *kernels) {
  if (!S || !kernels) return fail(SBP_ERR_ARG, "null argument");
  *kernels = S->last_graph_kernels;
  return SBP_OK;
}

sbp_status sbp_profile_enable(sbp_system_t S, int enable) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  S->prof = enable != 0;
  return SBP_OK;
}

sbp_status sbp_profile_read(sbp_system_t S, double *ms, int *launches, int reset) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  CUDA_TRY(S->drain());
  for (int k = 0; k < SBP_PHASE_COUNT; ++k) {
    if (ms) ms[k] = S->prof_ms[k];
    if (launches) launches[k] = S->prof_n[k];
    if (reset) {
      S->prof_ms[k] = 0.0;
      S->prof_n[k] = 0;
    }
  }
  return SBP_OK;
}

sbp_status sbp_f32_to_f64(const void *x, void *y, size_t n, void *stream) {
  if (n && (!x || !y)) return fail(SBP_ERR_ARG, "null buffer");
  CUDA_TRY(launch_widen(static_cast<const float *>(x), static_cast<double *>(y), n, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp_check(sbp_system_t S, void *stream) {
  if (!S) return fail(SBP_ERR_ARG, "null system");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaStreamSynchronize(s));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, S->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
  if (e) return fail((sbp_status)e, "device error word set");
  return SBP_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Batches: many independent overset systems advanced together, one cooperative persistent
// launch per micro step (donor values, fluxes and updates of all members, with grid barriers
// in between). The member systems keep their own tables and buffers; the batch holds, for each
// ring/buffer phase of the members, device arrays of launch descriptors and tile work lists.
namespace {
int gcd_i(int a, int b) { return b ? gcd_i(b, a % b) : a; }

struct MemberBook {
  int cur[2], head[2], count[2];
  double t;
};

MemberBook save_book(const sbp_system_s *S) {
  MemberBook b{};
  for (int k = 0; k < 2; ++k) {
    b.cur[k] = S->md[k].cur;
    b.head[k] = S->md[k].head;
    b.count[k] = S->md[k].count;
  }
  b.t = S->t;
  return b;
}

void load_book(sbp_system_s *S, const MemberBook &b) {
  for (int k = 0; k < 2; ++k) {
    S->md[k].cur = b.cur[k];
    S->md[k].head = b.head[k];
    S->md[k].count = b.count[k];
  }
  S->t = b.t;
}
}  // namespace

struct sbp_batch_s {
  std::vector<sbp_system_t> mem;
  int dtype = SBP_F64;
  bool visc = false, curvf = false;
  int ty = 16, grid = 0, srmax = 1, period = 1, variant = 0;
  std::vector<std::vector<BatchSubstep>> subs;  // [period][srmax]
  std::vector<void *> allocs;
  unsigned *bar = nullptr;
  int *err = nullptr;
  cudaStream_t cap = nullptr;
  std::map<int, cudaGraphExec_t> graphs;

  void free_plan() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    for (void *p : allocs) cudaFree(p);
    allocs.clear();
    subs.clear();
  }
  ~sbp_batch_s() {
    free_plan();
    cudaFree(bar);
    cudaFree(err);
    if (cap) cudaStreamDestroy(cap);
  }

  template <typename V>
  cudaError_t up(const std::vector<V> &v, const V *&dst) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(v.size() * sizeof(V), 16));
    if (e != cudaSuccess) return e;
    allocs.push_back(p);
    if (!v.empty()) e = cudaMemcpy(p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice);
    dst = static_cast<const V *>(p);
    return e;
  }

  // Launch descriptors and work lists for `period` consecutive macro steps from the members'
  // current ring/buffer phase (which they return to after `period` steps).
  cudaError_t build_plan() {
    free_plan();
    std::vector<MemberBook> start;
    for (auto *S : mem) start.push_back(save_book(S));
    subs.assign(period, std::vector<BatchSubstep>(srmax));
    for (int v = 0; v < period; ++v) {
      std::vector<std::vector<DonorLaunch>> dl(srmax);
      std::vector<std::vector<RhsLaunch>> rl(srmax);
      std::vector<std::vector<int4>> items(srmax);
      std::vector<std::vector<int>> sat_off(srmax, std::vector<int>(1, 0)), rl_curv(srmax);
      auto add_rhs = [&](int j, sbp_system_s *S, int k, RhsLaunch a) {
        a.rows_per_cta = ty;
        a.err = err;  // failures inside the batch launch are reported by sbp_batch_check
        int r = (int)rl[j].size();
        rl[j].push_back(a);
        sat_off[j].push_back(sat_off[j].back() + a.nsat);
        const int curv = S->mh[k].cartesian ? 0 : 1;
        rl_curv[j].push_back(curv);
        // ty >= 32: single-pass strips of kMarchW columns and ty rows; else 32 x ty tiles
        const int tw = ty >= 32 ? kMarchW : kTileX;
        int ntx = (S->mh[k].ni + tw - 1) / tw, nty = (S->mh[k].nj + ty - 1) / ty;
        for (int by = 0; by < nty; ++by)
          for (int bx = 0; bx < ntx; ++bx) items[j].push_back(make_int4(r, bx, by, curv));
      };
      for (auto *S : mem) {
        MemberBook b0 = save_book(S);
        const int F = S->fast(), Sl = S->slow(), sr = S->plan.sr, m = S->plan.m;
        const double H = S->H, h = H / sr;
        dl[0].push_back(S->donor_args(Sl, S->md[F].q[S->md[F].cur], 0, 1, false, H));
        dl[0].push_back(S->donor_args(F, S->md[Sl].q[S->md[Sl].cur], 0, 1, false, H));
        add_rhs(0, S, Sl, S->fused_args(Sl, 0, H));
        S->md[Sl].head = (S->md[Sl].head + 1) % m;
        for (int j = 0; j < sr; ++j) {
          if (j > 0) dl[j].push_back(S->donor_args(F, S->md[Sl].q[S->md[Sl].cur], j, 1, true, H));
          add_rhs(j, S, F, S->fused_args(F, j, h));
          S->md[F].head = (S->md[F].head + 1) % m;
          S->md[F].cur ^= 1;
        }
        load_book(S, b0);
        S->advance();
      }
      for (int j = 0; j < srmax; ++j) {
        BatchSubstep &b = subs[v][j];
        std::vector<int> off(1, 0);
        for (auto &a : dl[j]) off.push_back(off.back() + a.nsets * a.npts);
        cudaError_t e;
        const DonorLaunch *ddl;
        const RhsLaunch *drl;
        if ((e = up(dl[j], ddl)) != cudaSuccess) return e;
        if ((e = up(off, b.dl_off)) != cudaSuccess) return e;
        if ((e = up(rl[j], drl)) != cudaSuccess) return e;
        if ((e = up(items[j], b.items)) != cudaSuccess) return e;
        if ((e = up(sat_off[j], b.sat_off)) != cudaSuccess) return e;
        if ((e = up(rl_curv[j], b.rl_curv)) != cudaSuccess) return e;
        b.dl = ddl;
        b.rl = drl;
        b.n_rl = (int)rl[j].size();
        b.n_dl = (int)dl[j].size();
        b.n_items = (int)items[j].size();
        b.chunk = ty;
        b.bar_count = bar;
        b.bar_gen = bar + 1;
        b.err = err;
      }
    }
    for (size_t i = 0; i < mem.size(); ++i) load_book(mem[i], start[i]);
    variant = 0;
    return batch_grid_size(dtype, visc, curvf, ty, &grid);
  }

  cudaError_t launch_variant(cudaStream_t s) {
    auto it = graphs.find(variant);
    if (it == graphs.end()) {
      cudaError_t e;
      if (!cap && (e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
      if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
      cudaError_t ei = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), cap);
      for (int j = 0; j < srmax && ei == cudaSuccess; ++j)
        ei = launch_batch_substep(subs[variant][j], grid, dtype, visc, curvf, ty, cap);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cap, &g);
      if (ei != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ei;
      }
      if (e != cudaSuccess) return e;
      cudaGraphExec_t ex = nullptr;
      e = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
      it = graphs.emplace(variant, ex).first;
    }
    return cudaGraphLaunch(it->second, s);
  }

  cudaError_t step(cudaStream_t s) {
    cudaError_t e = launch_variant(s);
    if (e != cudaSuccess) return e;
    for (auto *S : mem) S->advance();
    variant = (variant + 1) % period;
    return cudaSuccess;
  }
};

extern "C" {

sbp_status sbp_batch_create(const sbp_system_t *systems, int n, int autotune, void *stream, sbp_batch_t *out) {
  if (!systems || n < 1 || !out) return fail(SBP_ERR_ARG, "bad argument");
  *out = nullptr;
  auto *B = new sbp_batch_s();
  std::unique_ptr<sbp_batch_s> guard(B);
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n; ++i) {
    sbp_system_s *S = systems[i];
    if (!S) return fail(SBP_ERR_ARG, "null member");
    if (!S->initialised) return fail(SBP_ERR_STATE, "member " + std::to_string(i) + " has not run sbp_mrab_init");
    if (S->p.scheme != SBP_MRAB_FASTEST_FIRST) return fail(SBP_ERR_ARG, "batches need fastest-first members");
    for (int j = 0; j < i; ++j)
      if (systems[j] == S) return fail(SBP_ERR_ARG, "a system appears twice in the batch");
    bool cf = !S->mh[S->fast()].cartesian;
    if (i == 0) {
      B->dtype = S->p.dtype;
      B->visc = S->viscous();
      B->curvf = cf;
    } else if (S->p.dtype != B->dtype || S->viscous() != B->visc || cf != B->curvf) {
      return fail(SBP_ERR_ARG, "batch members must share element type, physics and fine-mesh kind");
    }
    if (!S->mh[S->slow()].cartesian) return fail(SBP_ERR_ARG, "batch members need a Cartesian slow mesh");
    B->srmax = std::max(B->srmax, S->plan.sr);
    B->mem.push_back(S);
  }
  // common period of the members' ring/buffer phases
  int period = 1;
  for (auto *S : B->mem) {
    MemberBook b0 = save_book(S);
    uint64_t k0 = S->phase_key();
    int pb = 0;
    do {
      S->advance();
      ++pb;
    } while (S->phase_key() != k0 && pb < 64);
    load_book(S, b0);
    if (pb >= 64) return fail(SBP_ERR_STATE, "ring phase period above 64");
    period = period / gcd_i(period, pb) * pb;
    if (period > 64) return fail(SBP_ERR_STATE, "common ring phase period above 64");
  }
  B->period = period;
  CUDA_TRY(cudaMalloc((void **)&B->bar, 2 * sizeof(unsigned)));
  CUDA_TRY(cudaMemset(B->bar, 0, 2 * sizeof(unsigned)));
  CUDA_TRY(cudaMalloc((void **)&B->err, sizeof(int)));
  CUDA_TRY(cudaMemset(B->err, 0, sizeof(int)));
  if (autotune) {
    // time two macro steps per tile height on a snapshot of every member, then restore
    std::vector<void *> snap;
    std::vector<std::pair<void *, size_t>> bufs;
    for (auto *S : B->mem)
      for (int k = 0; k < 2; ++k) {
        size_t sb = S->state_elems(k) * S->esz;
        bufs.push_back({S->md[k].q[0], sb});
        bufs.push_back({S->md[k].q[1], sb});
        bufs.push_back({S->md[k].hist, sb * S->plan.m});
      }
    size_t total = 0;
    for (auto &b : bufs) total += b.second;
    void *store = nullptr;
    CUDA_TRY(cudaMalloc(&store, total));
    auto copy = [&](bool save) {
      size_t off = 0;
      for (auto &b : bufs) {
        cudaError_t e = save ? cudaMemcpyAsync((char *)store + off, b.first, b.second, cudaMemcpyDeviceToDevice, s)
                             : cudaMemcpyAsync(b.first, (char *)store + off, b.second, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
        off += b.second;
      }
      return cudaSuccess;
    };
    std::vector<MemberBook> books;
    for (auto *S : B->mem) books.push_back(save_book(S));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_ty = 16;
    cudaError_t e = copy(true);
    std::vector<int> shapes = {8, 16};
    if (!B->visc) shapes.insert(shapes.end(), {32, 64});  // single-pass strips (Euler)
    for (int ty : shapes) {
      if (e != cudaSuccess) break;
      B->ty = ty;
      if ((e = B->build_plan()) != cudaSuccess) break;
      if ((e = B->step(s)) != cudaSuccess) break;  // capture + warm-up
      cudaEventRecord(e0, s);
      for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = B->step(s);
      cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_ty = ty;
      }
      if (e == cudaSuccess) e = copy(false);
      for (size_t i = 0; i < B->mem.size(); ++i) load_book(B->mem[i], books[i]);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(store);
    CUDA_TRY(e);
    int flag = 0;
    CUDA_TRY(cudaMemcpy(&flag, B->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail((sbp_status)flag, "batch autotune step failed");
    B->ty = best_ty;
  }
  CUDA_TRY(B->build_plan());
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp_batch_destroy(sbp_batch_t B) {
  delete B;
  return SBP_OK;
}

sbp_status sbp_batch_step(sbp_batch_t B, int n, void *stream) {
  if (!B || n < 0) return fail(SBP_ERR_ARG, "bad argument");
  for (int i = 0; i < n; ++i) CUDA_TRY(B->step((cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp_batch_info(sbp_batch_t B, int *members, int *rows_per_cta, int *grid, int *period) {
  if (!B) return fail(SBP_ERR_ARG, "null batch");
  if (members) *members = (int)B->mem.size();
  if (rows_per_cta) *rows_per_cta = B->ty;
  if (grid) *grid = B->grid;
  if (period) *period = B->period;
  return SBP_OK;
}

sbp_status sbp_batch_set_shape(sbp_batch_t B, int rows) {
  if (!B) return fail(SBP_ERR_ARG, "null batch");
  if (!(rows == 8 || rows == 16 || ((rows == 32 || rows == 64 || rows == 128) && !B->visc)))
    return fail(SBP_ERR_ARG, "rows must be 8 or 16 (tile pairs) or, for Euler batches, 32, 64 or 128 (strips)");
  B->ty = rows;
  CUDA_TRY(B->build_plan());
  return SBP_OK;
}

sbp_status sbp_batch_check(sbp_batch_t B, void *stream) {
  if (!B) return fail(SBP_ERR_ARG, "null batch");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int flag = 0;
  CUDA_TRY(cudaMemcpy(&flag, B->err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(B->err, 0, sizeof(int)));
  if (flag) return fail((sbp_status)flag, "batch device error word set");
  return SBP_OK;
}

}  // extern "C"
