// C ABI of the discrete adjoint (FP64): vector-Jacobian and Jacobian-vector products of the
// right-hand side and of the interface interpolation, and the gradient of a probe-pressure
// objective through the whole MRAB run (Runge-Kutta bootstrap of Sec. 3.1 and the macro steps
// of Sec. 3.3) by reverse sweeps over binomially checkpointed forward steps. The device work is
// in sbp_adjoint.cu; every reduction is a fixed-order gather, so results are deterministic.
#include <cstdio>

#include "sbp_system.h"

namespace {

using sbp::fail;

cudaError_t adj_alloc(sbp_system_s *S, double **p, size_t n) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(n, 1) * sizeof(double));
  if (e != cudaSuccess) return e;
  S->adj_allocs.push_back(ptr);
  *p = static_cast<double *>(ptr);
  return cudaMemset(ptr, 0, std::max<size_t>(n, 1) * sizeof(double));
}

// Workspace and the inverse donor lists (per distinct donor point of mesh k's receivers, the
// entries receiver * 16 + stencil slot that read it, in receiver order).
cudaError_t ensure_ws(sbp_system_s *S) {
  if (S->aws_ready) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    const MeshHost &m = S->mh[k];
    size_t f = (size_t)m.pitch * m.nj, nr = m.recv_pt.size(), ns = m.sat_pt.size();
    auto &w = S->aws[k];
    if (e == cudaSuccess) e = adj_alloc(S, &w.mu, 8 * f);
    if (e == cudaSuccess) e = adj_alloc(S, &w.ld, 6 * f);
    if (e == cudaSuccess) e = adj_alloc(S, &w.lp, 3 * f);
    if (e == cudaSuccess) e = adj_alloc(S, &w.rv, 10 * nr);
    if (e == cudaSuccess) e = adj_alloc(S, &w.lrv, 10 * nr);
    if (e == cudaSuccess) e = adj_alloc(S, &w.lqinf, 4 * ns);
    if (e == cudaSuccess) e = adj_alloc(S, &w.satlin, 24 * ns);
    if (e == cudaSuccess) e = adj_alloc(S, &w.ldv, 10 * m.donor_pts.size());
    const int nd = (int)m.donor_pts.size();
    std::vector<int> off(nd + 1, 0), ent(m.donor_idx.size());
    for (int d : m.donor_idx) off[d + 1]++;
    for (int d = 0; d < nd; ++d) off[d + 1] += off[d];
    std::vector<int> fill(off.begin(), off.end() - 1);
    for (size_t t = 0; t < m.donor_idx.size(); ++t) ent[fill[m.donor_idx[t]]++] = (int)t;
    if (e == cudaSuccess) e = upload(S->md[k].inv_off, off.data(), off.size() * sizeof(int));
    if (e == cudaSuccess) e = upload(S->md[k].inv_re, ent.data(), ent.size() * sizeof(int));
  }
  if (e == cudaSuccess) e = adj_alloc(S, &S->d_qinf_acc, 4);
  if (e == cudaSuccess) S->aws_ready = true;
  return e;
}

KConst<double> kconst(const sbp_system_s *S, int k) {
  KConst<double> c{};
  S->fill_consts(k, c);
  return c;
}

// Receiver values of mesh k (state, then viscous fluxes; 10 x n_receivers) from the donor
// state q_donor of the other mesh, into the workspace.
cudaError_t recv_values(sbp_system_s *S, int k, const double *q_donor, cudaStream_t s) {
  InterpLaunch a{};
  const int nr = (int)S->mh[k].recv_pt.size();
  a.d = S->dev_mesh(1 - k);
  a.g = S->gas();
  a.q = q_donor;
  a.nrecv = nr;
  a.base = S->md[k].base;
  a.w = S->md[k].w;
  a.qhat = S->aws[k].rv;
  a.fvhat = S->viscous() ? S->aws[k].rv + 4 * (size_t)nr : nullptr;
  return launch_interp(a, SBP_F64, S->viscous(), s);
}

// Adjoint of the receiver values lrv (workspace of mesh k) through the interpolation from the
// donor state q_donor: lq_donor += I^T lrv, viscous fluxes included.
cudaError_t interp_vjp(sbp_system_s *S, int k, const double *q_donor, double *lq_donor, cudaStream_t s) {
  AdjDonorLaunch d{};
  d.d = S->dev_mesh(1 - k);
  d.k = kconst(S, 1 - k);
  d.viscous = S->viscous();
  d.shat = q_donor;
  d.npts = S->md[k].ndv;
  d.pts = S->md[k].dpts;
  d.inv_off = S->md[k].inv_off;
  d.inv_re = S->md[k].inv_re;
  d.w = S->md[k].w;
  d.lrv = S->aws[k].lrv;
  d.nrecv = (int)S->mh[k].recv_pt.size();
  d.ldv = S->aws[k].ldv;
  d.lshat = lq_donor;
  d.ld = S->aws[1 - k].ld;
  d.lp = S->aws[1 - k].lp;
  return launch_donor_adjoint(d, s);
}

// lq_self += (dR_k/dq_self)^T lam, lq_other += (dR_k/dq_other)^T lam (through the receivers),
// far-field adjoint accumulated into S->d_qinf_acc.
cudaError_t rhs_vjp(sbp_system_s *S, int k, const double *q_self, const double *q_other, const double *lam,
                    double *lq_self, double *lq_other, cudaStream_t s) {
  cudaError_t e = recv_values(S, k, q_other, s);
  if (e != cudaSuccess) return e;
  const MeshHost &m = S->mh[k];
  const MeshDev &md = S->md[k];
  auto &w = S->aws[k];
  AdjLaunch a{};
  a.m = S->dev_mesh(k);
  a.k = kconst(S, k);
  a.viscous = S->viscous();
  a.q = q_self;
  a.lam = lam;
  a.lq = lq_self;
  a.mu = w.mu;
  a.ld = w.ld;
  a.lp = w.lp;
  a.nsat = (int)m.sat_pt.size();
  a.sat_ij = md.sat_ij;
  a.sat_code = md.sat_code;
  a.sat_recv = md.sat_recv;
  a.sat_scale = md.sat_scale;
  a.rv = w.rv;
  a.nrecv = (int)m.recv_pt.size();
  a.lrv = w.lrv;
  a.lqinf = w.lqinf;
  a.satlin = w.satlin;
  if ((e = launch_rhs_adjoint(a, s)) != cudaSuccess) return e;
  if ((e = launch_sum4(w.lqinf, a.nsat, S->d_qinf_acc, s)) != cudaSuccess) return e;
  if (a.nrecv > 0 && lq_other) e = interp_vjp(S, k, q_other, lq_other, s);
  return e;
}

cudaError_t lincomb(double *out, const double *base, std::initializer_list<std::pair<double, const double *>> terms,
                    size_t n, cudaStream_t s) {
  LinComb lc{};
  int nx = 0;
  for (auto &t : terms) {
    lc.c[nx] = t.first;
    lc.x[nx] = t.second;
    ++nx;
  }
  return launch_lincomb(out, base, lc, nx, n, s);
}

// Binomial coefficient C(c + r, c), saturated.
double beta_cr(int c, int r) {
  double b = 1.0;
  for (int t = 1; t <= c; ++t) b = b * (r + t) / t;
  return b;
}

struct ProbeSpec {
  int n = 0;
  std::vector<int> base;
  std::vector<double> w;
};

// 4 x 4 Lagrange stencils of the probes on the Cartesian background (the stencil of
// Sec. 2.2's interpolation): base (i0, j0) with the probe inside cell (i0 + 1, j0 + 1) where
// possible, weights of the cubic through the 4 nodes along each direction.
sbp_status probe_stencils(const sbp_system_s *S, int n, const double *xy, ProbeSpec &ps) {
  const MeshHost &m = S->mh[0];
  ps.n = n;
  ps.base.assign(2 * n, 0);
  ps.w.assign(8 * n, 0.0);
  for (int p = 0; p < n; ++p) {
    int nn[2] = {m.ni, m.nj};
    for (int d = 0; d < 2; ++d) {
      double x = (xy[2 * p + d] - m.lo[d]) / m.h[d];
      if (!std::isfinite(x)) return fail(SBP_ERR_ARG, "probe coordinate not finite");
      int i0 = (int)std::floor(x) - 1;
      if (!m.per[d]) {
        if (x < 0.0 || x > nn[d] - 1) return fail(SBP_ERR_ARG, "probe " + std::to_string(p) + " outside the background");
        i0 = std::max(0, std::min(nn[d] - 4, i0));
      }
      double t = x - i0;
      for (int a = 0; a < 4; ++a) {
        double l = 1.0;
        for (int b = 0; b < 4; ++b)
          if (b != a) l *= (t - b) / (double)(a - b);
        ps.w[8 * p + 4 * d + a] = l;
      }
      ps.base[2 * p + d] = i0;
    }
    for (int b = 0; b < 4; ++b)
      for (int a = 0; a < 4; ++a) {
        int ii = ps.base[2 * p] + a, jj = ps.base[2 * p + 1] + b;
        if (m.per[0]) ii = (ii % m.ni + m.ni) % m.ni;
        if (m.per[1]) jj = (jj % m.nj + m.nj) % m.nj;
        if (!m.active[(size_t)jj * m.ni + ii])
          return fail(SBP_ERR_ARG, "probe " + std::to_string(p) + " stencil touches a hole");
      }
  }
  return SBP_OK;
}

// The reverse sweep of the probe objective over one system (see sbp_adjoint_probe).
struct ProbeAdjoint {
  sbp_system_s *S;
  cudaStream_t s;
  int N = 0, C = 0, np = 0;
  double H = 0.0;
  int m = 0, sr = 0, F = 0, Sl = 0;
  size_t n[2] = {0, 0};  // elements of one state
  std::vector<void *> allocs;
  // working forward buffers
  double *q[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}}, *hist[2] = {nullptr, nullptr};
  // checkpoints: state + rings of both meshes, and ring heads
  struct Slot {
    double *q[2], *hist[2];
    int head[2];
    int pos = -1;
  };
  std::vector<Slot> slots;
  int pos = 0;       // macro step index of the state in the working buffers
  int next_new = 0;  // first macro step whose probe pressures are not yet recorded
  long fwd = 0;      // macro steps run
  double *ystore[2] = {nullptr, nullptr};
  std::vector<double *> frec;
  // adjoint buffers
  double *lam_sp = nullptr, *lam_sin = nullptr, *lam_f = nullptr, *lamR = nullptr, *lshat = nullptr, *shat = nullptr;
  std::vector<double *> lSring, lFring, lSfull;
  int *d_base = nullptr;
  double *d_w = nullptr, *d_p = nullptr;

  ~ProbeAdjoint() {
    cudaStreamSynchronize(s);
    for (void *p : allocs) cudaFree(p);
  }

  cudaError_t alloc(double **p, size_t elems) {
    void *ptr = nullptr;
    cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(elems, 1) * sizeof(double));
    if (e != cudaSuccess) return e;
    allocs.push_back(ptr);
    *p = static_cast<double *>(ptr);
    return cudaMemsetAsync(ptr, 0, std::max<size_t>(elems, 1) * sizeof(double), s);
  }

  cudaError_t store(Slot &sl) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaMemcpyAsync(sl.q[k], S->md[k].q[S->md[k].cur], n[k] * 8, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(sl.hist[k], hist[k], m * n[k] * 8, cudaMemcpyDeviceToDevice, s);
      sl.head[k] = S->md[k].head;
    }
    sl.pos = pos;
    return e;
  }
  cudaError_t restore(const Slot &sl) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      S->md[k].cur = 0;
      S->md[k].head = sl.head[k];
      e = cudaMemcpyAsync(q[k][0], sl.q[k], n[k] * 8, cudaMemcpyDeviceToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hist[k], sl.hist[k], m * n[k] * 8, cudaMemcpyDeviceToDevice, s);
    }
    pos = sl.pos;
    return e;
  }

  // One macro step from the working state; with rec, the fast states of its micro steps are
  // kept in frec. Probe pressures of steps run for the first time are recorded.
  cudaError_t step(bool rec) {
    void *const *fr = rec ? reinterpret_cast<void *const *>(frec.data()) : nullptr;
    cudaError_t e = S->issue_step(s, nullptr, fr);
    if (e != cudaSuccess) return e;
    S->advance();
    ++fwd;
    if (pos == next_new) {
      e = launch_probe(S->dev_mesh(0), (const double *)S->md[0].q[S->md[0].cur], np, d_base, d_w,
                       d_p + (size_t)pos * np, nullptr, 0.0, S->p.gamma, s);
      ++next_new;
    }
    ++pos;
    return e;
  }

  // Reverse of macro step i; the working buffers hold the state after it (just recorded).
  cudaError_t reverse_step() {
    cudaError_t e = cudaSuccess;
    auto run = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    const CoeffPlan &P = S->plan;
    const double h = H / sr;
    const MeshDev &ds = S->md[Sl];
    const double *s_i = (const double *)ds.q[1 - ds.cur];
    std::vector<const double *> Sfull(m);
    for (int k = 0; k < m; ++k) Sfull[k] = (const double *)S->hist_slot(Sl, (ds.head + 1 + k) % m);
    // probe seed at the state after the step (mesh 0)
    double *seed = Sl == 0 ? lam_sp : lam_f;
    run(launch_probe(S->dev_mesh(0), (const double *)S->md[0].q[S->md[0].cur], np, d_base, d_w, nullptr, seed, H,
                     S->p.gamma, s));
    run(cudaMemsetAsync(lam_sin, 0, n[Sl] * 8, s));
    for (int k = 0; k < m; ++k) run(cudaMemsetAsync(lSfull[k], 0, n[Sl] * 8, s));
    // fast micro steps, last first
    for (int j = sr - 1; j >= 0; --j) {
      run(lincomb(lamR, nullptr, {{h * P.ab[m - 1], lam_f}, {1.0, lFring[m - 2]}}, n[F], s));
      double *tmp = lFring[m - 2];
      for (int k = m - 2; k >= 1; --k) lFring[k] = lFring[k - 1];
      lFring[0] = tmp;
      for (int k = 1; k <= m - 2; ++k) run(lincomb(lFring[k], lFring[k], {{h * P.ab[k], lam_f}}, n[F], s));
      run(lincomb(lFring[0], nullptr, {{h * P.ab[0], lam_f}}, n[F], s));
      const double *sh = s_i;
      if (j > 0) {
        LinComb lc{};
        for (int k = 0; k < m; ++k) {
          lc.c[k] = H * P.ext[j][k];
          lc.x[k] = Sfull[k];
        }
        run(launch_lincomb(shat, s_i, lc, m, n[Sl], s));
        sh = shat;
      }
      run(cudaMemsetAsync(lshat, 0, n[Sl] * 8, s));
      run(rhs_vjp(S, F, frec[j], sh, lamR, lam_f, lshat, s));
      run(lincomb(lam_sin, lam_sin, {{1.0, lshat}}, n[Sl], s));
      if (j > 0)
        for (int k = 0; k < m; ++k) run(lincomb(lSfull[k], lSfull[k], {{H * P.ext[j][k], lshat}}, n[Sl], s));
    }
    // slow step
    run(lincomb(lamR, nullptr, {{H * P.ab[m - 1], lam_sp}, {1.0, lSring[m - 2]}, {1.0, lSfull[m - 1]}}, n[Sl], s));
    double *tmp = lSring[m - 2];
    for (int k = m - 2; k >= 1; --k) lSring[k] = lSring[k - 1];
    lSring[0] = tmp;
    for (int k = 1; k <= m - 2; ++k)
      run(lincomb(lSring[k], lSring[k], {{H * P.ab[k], lam_sp}, {1.0, lSfull[k]}}, n[Sl], s));
    run(lincomb(lSring[0], nullptr, {{H * P.ab[0], lam_sp}, {1.0, lSfull[0]}}, n[Sl], s));
    run(rhs_vjp(S, Sl, s_i, frec[0], lamR, lam_sin, lam_f, s));
    run(lincomb(lam_sin, lam_sin, {{1.0, lam_sp}}, n[Sl], s));
    std::swap(lam_sp, lam_sin);
    return e;
  }

  // Reverse of steps [n0, n1) with c free checkpoint slots above slot `top` (which holds n0).
  cudaError_t reverse_range(int n0, int n1, int c, int top) {
    cudaError_t e = cudaSuccess;
    const int l = n1 - n0;
    if (l <= 0) return e;
    if (l == 1) {
      if (pos != n0 && (e = restore(slots[top])) != cudaSuccess) return e;
      if ((e = step(true)) != cudaSuccess) return e;
      return reverse_step();
    }
    if (c == 0) {
      for (int i = n1 - 1; i >= n0; --i) {
        if (pos != n0 && (e = restore(slots[top])) != cudaSuccess) return e;
        while (pos < i)
          if ((e = step(false)) != cudaSuccess) return e;
        if ((e = step(true)) != cudaSuccess) return e;
        if ((e = reverse_step()) != cudaSuccess) return e;
      }
      return e;
    }
    // least repetition number r with C(c + r, c) >= l, then a split that keeps both parts
    // within it: right part l - k <= C(c - 1 + r, c - 1)
    int r = 0;
    while (beta_cr(c, r) < l) ++r;
    int k = std::max(1, l - (int)std::min<double>(beta_cr(c - 1, r), (double)l));
    k = std::min(k, l - 1);
    if (pos != n0 && (e = restore(slots[top])) != cudaSuccess) return e;
    while (pos < n0 + k)
      if ((e = step(false)) != cudaSuccess) return e;
    if ((e = store(slots[top + 1])) != cudaSuccess) return e;
    if ((e = reverse_range(n0 + k, n1, c - 1, top + 1)) != cudaSuccess) return e;
    return reverse_range(n0, n0 + k, c, top);
  }

  // Reverse of the Runge-Kutta bootstrap: lam[k] holds the adjoint of its final states on
  // entry and of its initial states on return.
  cudaError_t reverse_bootstrap(double *lam[2]) {
    cudaError_t e = cudaSuccess;
    auto run = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    const double h = H / sr;
    const int nsteps = (m - 1) * sr;
    double *Y2[2], *Y3[2], *K[2], *B[2], *Cc[2], *LK[2];
    for (int k = 0; k < 2; ++k) {
      run(alloc(&Y2[k], n[k]));
      run(alloc(&Y3[k], n[k]));
      run(alloc(&K[k], n[k]));
      run(alloc(&B[k], n[k]));
      run(alloc(&Cc[k], n[k]));
      run(alloc(&LK[k], n[k]));
    }
    auto joint_vjp = [&](double *const y[2], double *const lk[2], double *out[2]) {
      for (int k = 0; k < 2; ++k) run(rhs_vjp(S, k, y[k], y[1 - k], lk[k], out[k], out[1 - k], s));
    };
    for (int st = nsteps - 1; st >= 0 && e == cudaSuccess; --st) {
      double *y[2] = {ystore[0] + (size_t)st * n[0], ystore[1] + (size_t)st * n[1]};
      // stage states
      for (int k = 0; k < 2; ++k) run(S->rhs_plain(k, y[k], y[1 - k], K[k], s));
      for (int k = 0; k < 2; ++k) run(lincomb(Y2[k], y[k], {{h / 3.0, K[k]}}, n[k], s));
      for (int k = 0; k < 2; ++k) run(S->rhs_plain(k, Y2[k], Y2[1 - k], K[k], s));
      for (int k = 0; k < 2; ++k) run(lincomb(Y3[k], y[k], {{2.0 * h / 3.0, K[k]}}, n[k], s));
      // reverse of the stages
      for (int k = 0; k < 2; ++k) {
        run(lincomb(LK[k], nullptr, {{0.75 * h, lam[k]}}, n[k], s));
        run(cudaMemsetAsync(B[k], 0, n[k] * 8, s));
        run(cudaMemsetAsync(Cc[k], 0, n[k] * 8, s));
      }
      joint_vjp(Y3, LK, B);
      for (int k = 0; k < 2; ++k) run(lincomb(LK[k], nullptr, {{2.0 * h / 3.0, B[k]}}, n[k], s));
      joint_vjp(Y2, LK, Cc);
      for (int k = 0; k < 2; ++k) {
        const double *rec = nullptr;
        if (k == Sl && st % sr == 0) rec = lSring[st / sr];
        if (k == F && st >= nsteps - (m - 1)) rec = lFring[st - (nsteps - (m - 1))];
        if (rec) run(lincomb(LK[k], nullptr, {{0.25 * h, lam[k]}, {h / 3.0, Cc[k]}, {1.0, rec}}, n[k], s));
        else run(lincomb(LK[k], nullptr, {{0.25 * h, lam[k]}, {h / 3.0, Cc[k]}}, n[k], s));
        run(lincomb(lam[k], lam[k], {{1.0, B[k]}, {1.0, Cc[k]}}, n[k], s));
      }
      joint_vjp(y, LK, lam);
    }
    return e;
  }
};

}  // namespace

extern "C" {

sbp_status sbp_set_freestream(sbp_system_t S, const double *qinf) {
  if (!S || !qinf) return fail(SBP_ERR_ARG, "bad argument");
  for (int v = 0; v < 4; ++v)
    if (!std::isfinite(qinf[v])) return fail(SBP_ERR_ARG, "qinf not finite");
  for (int v = 0; v < 4; ++v) S->p.qinf[v] = qinf[v];
  S->clear_graphs();
  return SBP_OK;
}

sbp_status sbp_rhs_eval_vjp(sbp_system_t S, int k, const void *q_self, const void *q_other, const void *lam,
                            void *lq_self, void *lq_other, double *lqinf, void *stream) {
  if (!S || k < 0 || k > 1 || !q_self || !q_other || !lam || !lq_self || !lq_other)
    return fail(SBP_ERR_ARG, "bad argument");
  if (S->p.dtype != SBP_F64) return fail(SBP_ERR_DTYPE, "the adjoint needs an SBP_F64 system");
  if (S->p.sponge_cells > 0) return fail(SBP_ERR_ARG, "the adjoint does not cover the sponge layer");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(ensure_ws(S));
  CUDA_TRY(cudaMemsetAsync(lq_self, 0, S->state_elems(k) * 8, s));
  CUDA_TRY(cudaMemsetAsync(lq_other, 0, S->state_elems(1 - k) * 8, s));
  CUDA_TRY(cudaMemsetAsync(S->d_qinf_acc, 0, 4 * sizeof(double), s));
  CUDA_TRY(rhs_vjp(S, k, (const double *)q_self, (const double *)q_other, (const double *)lam, (double *)lq_self,
                   (double *)lq_other, s));
  if (lqinf) {
    CUDA_TRY(cudaMemcpyAsync(lqinf, S->d_qinf_acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  return SBP_OK;
}

sbp_status sbp_rhs_eval_jvp(sbp_system_t S, int k, const void *q_self, const void *q_other, const void *dq_self,
                            const void *dq_other, const double *dqinf, void *drhs, void *stream) {
  if (!S || k < 0 || k > 1 || !q_self || !q_other || !dq_self || !dq_other || !drhs)
    return fail(SBP_ERR_ARG, "bad argument");
  if (S->p.dtype != SBP_F64) return fail(SBP_ERR_DTYPE, "the tangent needs an SBP_F64 system");
  if (S->p.sponge_cells > 0) return fail(SBP_ERR_ARG, "the tangent does not cover the sponge layer");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(ensure_ws(S));
  CUDA_TRY(recv_values(S, k, (const double *)q_other, s));
  const MeshHost &m = S->mh[k];
  const MeshDev &md = S->md[k];
  TlDonorLaunch dn{};
  dn.d = S->dev_mesh(1 - k);
  dn.k = kconst(S, 1 - k);
  dn.viscous = S->viscous();
  dn.q = (const double *)q_other;
  dn.qd = (const double *)dq_other;
  dn.pd = S->aws[1 - k].lp;
  dn.nrecv = (int)m.recv_pt.size();
  dn.base = md.base;
  dn.w = md.w;
  dn.rvd = S->aws[k].lrv;
  TlLaunch a{};
  a.m = S->dev_mesh(k);
  a.k = kconst(S, k);
  a.viscous = S->viscous();
  a.q = (const double *)q_self;
  a.qd = (const double *)dq_self;
  a.pd = S->aws[k].lp;
  a.fd = S->aws[k].mu;
  a.out = (double *)drhs;
  a.nsat = (int)m.sat_pt.size();
  a.sat_ij = md.sat_ij;
  a.sat_code = md.sat_code;
  a.sat_recv = md.sat_recv;
  a.sat_scale = md.sat_scale;
  a.rv = S->aws[k].rv;
  a.rvd = S->aws[k].lrv;
  a.nrecv = dn.nrecv;
  for (int v = 0; v < 4; ++v) a.qinfd[v] = dqinf ? dqinf[v] : 0.0;
  CUDA_TRY(launch_rhs_tangent(a, dn, s));
  return SBP_OK;
}

sbp_status sbp_overset_interp_vjp(sbp_system_t S, int recv, const void *q_donor, const void *lqhat,
                                  const void *lfvhat, void *lq_donor, void *stream) {
  if (!S || recv < 0 || recv > 1 || !q_donor || !lqhat || !lq_donor) return fail(SBP_ERR_ARG, "bad argument");
  if (S->p.dtype != SBP_F64) return fail(SBP_ERR_DTYPE, "the adjoint needs an SBP_F64 system");
  if (S->p.sponge_cells > 0) return fail(SBP_ERR_ARG, "the adjoint does not cover the sponge layer");
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(ensure_ws(S));
  const size_t nr = S->mh[recv].recv_pt.size();
  double *lrv = S->aws[recv].lrv;
  CUDA_TRY(cudaMemsetAsync(lrv, 0, std::max<size_t>(10 * nr, 1) * sizeof(double), s));
  if (nr) {
    CUDA_TRY(cudaMemcpyAsync(lrv, lqhat, 4 * nr * sizeof(double), cudaMemcpyDeviceToDevice, s));
    if (lfvhat && S->viscous())
      CUDA_TRY(cudaMemcpyAsync(lrv + 4 * nr, lfvhat, 6 * nr * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  CUDA_TRY(cudaMemsetAsync(lq_donor, 0, S->state_elems(1 - recv) * 8, s));
  CUDA_TRY(interp_vjp(S, recv, (const double *)q_donor, (double *)lq_donor, s));
  return SBP_OK;
}

sbp_status sbp_adjoint_probe(sbp_system_t S, const sbp_adjoint_desc *desc, const void *q0_mesh0,
                             const void *q0_mesh1, double *J, double *probe_p, void *dJ_dq0_mesh0,
                             void *dJ_dq0_mesh1, double *dJ_dqinf, long *forward_steps, void *stream) {
  if (!S || !desc || !q0_mesh0 || !q0_mesh1) return fail(SBP_ERR_ARG, "bad argument");
  if (S->p.dtype != SBP_F64) return fail(SBP_ERR_DTYPE, "the adjoint needs an SBP_F64 system");
  if (S->p.sponge_cells > 0) return fail(SBP_ERR_ARG, "the adjoint does not cover the sponge layer");
  if (S->p.scheme != SBP_MRAB_FASTEST_FIRST) return fail(SBP_ERR_ARG, "the adjoint needs a fastest-first system");
  if (desc->n_steps < 0 || desc->n_snapshots < 0 || desc->n_probes < 1 || !desc->probe_xy || !(desc->H > 0.0))
    return fail(SBP_ERR_ARG, "descriptor: n_steps >= 0, n_snapshots >= 0, n_probes >= 1, probe_xy, H > 0");
  if (S->plan.m < 2) return fail(SBP_ERR_ARG, "the adjoint needs hist_len >= 2");
  const bool want_grad = dJ_dq0_mesh0 || dJ_dq0_mesh1 || dJ_dqinf;
  if (want_grad && !(dJ_dq0_mesh0 && dJ_dq0_mesh1))
    return fail(SBP_ERR_ARG, "give both initial-state gradient buffers or neither");
  ProbeSpec ps;
  sbp_status st = probe_stencils(S, desc->n_probes, desc->probe_xy, ps);
  if (st != SBP_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(ensure_ws(S));

  // the system's own buffers and bookkeeping are put back on every return
  struct Saved {
    sbp_system_s *S;
    MeshDev md[2];
    double H, t;
    bool init, prof;
    ~Saved() {
      for (int k = 0; k < 2; ++k) S->md[k] = md[k];
      S->H = H;
      S->t = t;
      S->initialised = init;
      S->prof = prof;
    }
  } saved{S, {S->md[0], S->md[1]}, S->H, S->t, S->initialised, S->prof};
  S->prof = false;

  ProbeAdjoint A;
  A.S = S;
  A.s = s;
  A.N = desc->n_steps;
  A.C = std::min(desc->n_snapshots, std::max(A.N - 1, 0));
  A.np = ps.n;
  A.H = desc->H;
  A.m = S->plan.m;
  A.sr = S->plan.sr;
  A.F = S->fast();
  A.Sl = S->slow();
  for (int k = 0; k < 2; ++k) A.n[k] = S->state_elems(k);
  const int m = A.m, sr = A.sr, nboot = (m - 1) * sr;
  for (int k = 0; k < 2; ++k) {
    CUDA_TRY(A.alloc(&A.q[k][0], A.n[k]));
    CUDA_TRY(A.alloc(&A.q[k][1], A.n[k]));
    CUDA_TRY(A.alloc(&A.hist[k], m * A.n[k]));
    S->md[k].q[0] = A.q[k][0];
    S->md[k].q[1] = A.q[k][1];
    S->md[k].hist = A.hist[k];
    S->md[k].cur = 0;
  }
  CUDA_TRY(cudaMemcpyAsync(A.q[0][0], q0_mesh0, A.n[0] * 8, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(A.q[1][0], q0_mesh1, A.n[1] * 8, cudaMemcpyDeviceToDevice, s));
  S->H = A.H;
  S->t = 0.0;
  S->var_left = 0;
  CUDA_TRY(upload(A.d_base, ps.base.data(), ps.base.size() * sizeof(int)));
  A.allocs.push_back(A.d_base);
  CUDA_TRY(upload(A.d_w, ps.w.data(), ps.w.size() * sizeof(double)));
  A.allocs.push_back(A.d_w);
  CUDA_TRY(A.alloc(&A.d_p, (size_t)std::max(A.N, 1) * A.np));
  if (want_grad)
    for (int k = 0; k < 2; ++k) CUDA_TRY(A.alloc(&A.ystore[k], (size_t)nboot * A.n[k]));
  CUDA_TRY(S->bootstrap(A.H, s, want_grad ? reinterpret_cast<void *const *>(A.ystore) : nullptr));
  S->initialised = true;

  if (!want_grad) {
    for (int i = 0; i < A.N; ++i) CUDA_TRY(A.step(false));
  } else {
    A.slots.resize(A.C + 1);
    for (auto &sl : A.slots)
      for (int k = 0; k < 2; ++k) {
        CUDA_TRY(A.alloc(&sl.q[k], A.n[k]));
        CUDA_TRY(A.alloc(&sl.hist[k], m * A.n[k]));
      }
    A.frec.resize(sr);
    for (auto &f : A.frec) CUDA_TRY(A.alloc(&f, A.n[A.F]));
    size_t nmax = std::max(A.n[0], A.n[1]);
    CUDA_TRY(A.alloc(&A.lam_sp, A.n[A.Sl]));
    CUDA_TRY(A.alloc(&A.lam_sin, A.n[A.Sl]));
    CUDA_TRY(A.alloc(&A.lam_f, A.n[A.F]));
    CUDA_TRY(A.alloc(&A.lamR, nmax));
    CUDA_TRY(A.alloc(&A.lshat, A.n[A.Sl]));
    CUDA_TRY(A.alloc(&A.shat, A.n[A.Sl]));
    A.lSring.resize(m - 1);
    A.lFring.resize(m - 1);
    A.lSfull.resize(m);
    for (auto &b : A.lSring) CUDA_TRY(A.alloc(&b, A.n[A.Sl]));
    for (auto &b : A.lFring) CUDA_TRY(A.alloc(&b, A.n[A.F]));
    for (auto &b : A.lSfull) CUDA_TRY(A.alloc(&b, A.n[A.Sl]));
    CUDA_TRY(cudaMemsetAsync(S->d_qinf_acc, 0, 4 * sizeof(double), s));
    A.pos = 0;
    CUDA_TRY(A.store(A.slots[0]));
    CUDA_TRY(A.reverse_range(0, A.N, A.C, 0));
    double *lam[2];
    lam[A.Sl] = A.lam_sp;
    lam[A.F] = A.lam_f;
    CUDA_TRY(A.reverse_bootstrap(lam));
    CUDA_TRY(cudaMemcpyAsync(dJ_dq0_mesh0, lam[0], A.n[0] * 8, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(dJ_dq0_mesh1, lam[1], A.n[1] * 8, cudaMemcpyDeviceToDevice, s));
    if (dJ_dqinf) CUDA_TRY(cudaMemcpyAsync(dJ_dqinf, S->d_qinf_acc, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  std::vector<double> pv((size_t)A.N * A.np);
  if (!pv.empty())
    CUDA_TRY(cudaMemcpyAsync(pv.data(), A.d_p, pv.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  int flag = 0;
  CUDA_TRY(cudaMemcpy(&flag, S->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    CUDA_TRY(cudaMemset(S->d_err, 0, sizeof(int)));
    return fail((sbp_status)flag, "device error word set during the adjoint run");
  }
  // J = H sum over macro steps of sum over probes of p^2, summed in step order
  double Jv = 0.0;
  for (int i = 0; i < A.N; ++i) {
    double si = 0.0;
    for (int p = 0; p < A.np; ++p) si += pv[(size_t)i * A.np + p] * pv[(size_t)i * A.np + p];
    Jv += A.H * si;
  }
  if (J) *J = Jv;
  if (probe_p) std::copy(pv.begin(), pv.end(), probe_p);
  if (forward_steps) *forward_steps = A.fwd;
  return SBP_OK;
}

}  // extern "C"
