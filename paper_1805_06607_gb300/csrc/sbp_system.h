// The system object behind sbp_system_t: host setup products, device tables, integrator
// bookkeeping, CUDA graphs and phase timers. Shared by the C ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "sbp_device.h"
#include "sbp_internal.h"
#include "sbp_tune.h"

using namespace sbp;

namespace sbp {
inline thread_local std::string g_msg;

inline sbp_status fail(sbp_status s, const std::string &msg) {
  g_msg = msg;
  return s;
}

#define CUDA_TRY(expr)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (expr);                                                             \
    if (e_ != cudaSuccess) return fail(SBP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Weights of the SBP 4-2 derivative rows in the device table's order and tap order (closure
// rows 0-3 of the diagonal-norm operator, the interior row, a hole row), for the Cartesian
// meshes' scaled copies.
inline constexpr double kSbpRows[6][4] = {{-24.0 / 17.0, 59.0 / 34.0, -4.0 / 17.0, -3.0 / 34.0},
                                          {-0.5, 0.5, 0.0, 0.0},
                                          {4.0 / 43.0, -59.0 / 86.0, 59.0 / 86.0, -4.0 / 43.0},
                                          {3.0 / 98.0, -59.0 / 98.0, 32.0 / 49.0, -4.0 / 49.0},
                                          {1.0 / 12.0, -2.0 / 3.0, 2.0 / 3.0, -1.0 / 12.0},
                                          {0.0, 0.0, 0.0, 0.0}};

struct MeshDev {
  uint8_t *cls = nullptr;
  void *met = nullptr;
  int *tile_sat = nullptr;
  void *flux = nullptr;
  uint32_t *sat_ij = nullptr, *sat_code = nullptr;
  int *sat_recv = nullptr;
  double *sat_scale = nullptr;
  int *base = nullptr;
  double *w = nullptr;
  void *wt = nullptr;   // donor weights in the compute type
  void *sat = nullptr;  // per SAT point: 4 penalty terms
  void *qhat = nullptr, *fvhat = nullptr;
  // distinct donor points of this mesh's receivers, per-receiver indices into them, and the
  // per-step donor values (10 planes per extrapolation set)
  uint32_t *dpts = nullptr;
  int *didx = nullptr;
  void *dv = nullptr;
  int ndv = 0, dv_sets = 0;
  // inverse donor lists for the adjoint (built on first use): per distinct donor point, the
  // (receiver * 16 + stencil slot) entries that read it
  int *inv_off = nullptr, *inv_re = nullptr;
  int rows_per_cta = 16;
  int rows_upd = 0;           // rows per CTA of the update kernel (0: rows_per_cta)
  int strip = 0, chunk = 64;  // strip > 0: the single-pass marching kernel (see RhsLaunch)
  // the same choice for right-hand sides without the update (rhs_eval, Runge-Kutta stages)
  int e_strip = 0, e_chunk = 64, e_rows = 16, e_rows_upd = 0;
  void *prim = nullptr;       // Navier-Stokes fast mesh: primitives handed from micro step to micro step
  // bound integrator buffers
  void *q[2] = {nullptr, nullptr};
  void *hist = nullptr;
  int cur = 0, head = -1, count = 0;
};

template <typename P>
inline cudaError_t upload(P *&dst, const void *src, size_t bytes) {
  cudaError_t e = cudaMalloc((void **)&dst, bytes ? bytes : 16);
  if (e != cudaSuccess) return e;
  if (bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
  return e;
}
}  // namespace sbp

struct sbp_system_s {
  sbp_params p{};
  MeshHost mh[2];
  MeshDev md[2];
  CoeffPlan plan;
  size_t esz = 8;
  int *d_err = nullptr;
  unsigned long long *d_dt = nullptr;
  double H = 0.0, t = 0.0;
  bool initialised = false;
  // Node times of the history entries per mesh and ring slot (time since the end of the
  // bootstrap), and the number of coming macro steps whose histories are not uniform in the
  // current H (after sbp_mrab_set_step): those take weights solved on the node times.
  double tnode[2][kMaxHist] = {};
  int var_left = 0;
  // phase timers
  bool prof = false;
  struct Pending {
    int phase;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[SBP_PHASE_COUNT] = {0, 0, 0, 0};
  int prof_n[SBP_PHASE_COUNT] = {0, 0, 0, 0};
  // CUDA graphs of one macro step, one per ring/buffer phase (the kernel arguments differ by
  // phase), captured on internal streams with the slow RHS and the first fast micro step on
  // parallel branches.
  bool use_graph = true;
  // cap, side: the fast chain (high priority); side2: the slow right-hand side's tiles away from
  // the fast receivers' donors (low priority), beside the fast micro steps
  cudaStream_t cap = nullptr, side = nullptr, side2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_a = nullptr, ev_b = nullptr;
  std::map<uint64_t, cudaGraphExec_t> graphs;
  std::map<uint64_t, int> graph_kernels;  // kernel nodes of each phase's graph
  int last_graph_kernels = 0;             // of the graph launched last
  // FP64 workspace of the adjoint and tangent calls, per mesh (allocated on first use):
  // mu 8 planes, ld 6 planes, lp 3 planes, receiver values rv and their adjoint lrv (10 per
  // receiver), far-field adjoint per SAT point (4), donor-point adjoint ldv (10 per point)
  struct AdjWs {
    double *mu = nullptr, *ld = nullptr, *lp = nullptr, *rv = nullptr, *lrv = nullptr, *lqinf = nullptr,
           *ldv = nullptr, *satlin = nullptr;
  } aws[2];
  double *d_qinf_acc = nullptr;  // 4 doubles: accumulated far-field adjoint
  bool aws_ready = false;
  std::vector<void *> adj_allocs;

  // Classical fourth-order Runge-Kutta, the single-rate baseline integrator (Sec. 4.4, 6.1):
  // per mesh a stage state and the four stage derivatives (allocated on first use), and the
  // CUDA graph of one step for the step size and state buffers it was captured with.
  void *rk_buf[2] = {nullptr, nullptr};
  cudaGraphExec_t rk_graph = nullptr;
  double rk_graph_h = 0.0;
  int rk_graph_cur = -1;

  void clear_graphs() {
    for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    graph_kernels.clear();
    if (rk_graph) cudaGraphExecDestroy(rk_graph);
    rk_graph = nullptr;
  }

  cudaEvent_t take_event() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // Launch `fn` on stream s, bracketed by an event pair when the timers are on.
  template <typename Fn>
  cudaError_t timed(int phase, cudaStream_t s, Fn &&fn) {
    if (!prof) return fn();
    Pending p{phase, take_event(), take_event()};
    cudaEventRecord(p.a, s);
    cudaError_t e = fn();
    cudaEventRecord(p.b, s);
    pending.push_back(p);
    return e;
  }
  cudaError_t drain() {
    for (auto &p : pending) {
      cudaError_t e = cudaEventSynchronize(p.b);
      if (e != cudaSuccess) return e;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, p.a, p.b);
      prof_ms[p.phase] += ms;
      prof_n[p.phase] += 1;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
    return cudaSuccess;
  }

  ~sbp_system_s() {
    for (auto &d : md) {
      cudaFree(d.cls);
      cudaFree(d.met);
      cudaFree(d.tile_sat);
      cudaFree(d.flux);
      cudaFree(d.sat_ij);
      cudaFree(d.sat_code);
      cudaFree(d.sat_recv);
      cudaFree(d.sat_scale);
      cudaFree(d.base);
      cudaFree(d.w);
      cudaFree(d.wt);
      cudaFree(d.sat);
      cudaFree(d.qhat);
      cudaFree(d.fvhat);
      cudaFree(d.dpts);
      cudaFree(d.didx);
      cudaFree(d.dv);
      cudaFree(d.inv_off);
      cudaFree(d.inv_re);
      cudaFree(d.prim);
    }
    cudaFree(d_err);
    cudaFree(d_dt);
    for (void *b : rk_buf) cudaFree(b);
    for (void *ptr : adj_allocs) cudaFree(ptr);
    drain();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    clear_graphs();
    if (cap) cudaStreamDestroy(cap);
    if (side) cudaStreamDestroy(side);
    if (side2) cudaStreamDestroy(side2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
  }

  bool viscous() const { return p.physics == SBP_NS; }
  int fast() const { return p.fast_mesh; }
  int slow() const { return 1 - p.fast_mesh; }
  size_t state_elems(int k) const { return (size_t)kNvar * mh[k].pitch * mh[k].nj; }

  DevMesh dev_mesh(int k) const {
    DevMesh d{};
    const MeshHost &m = mh[k];
    d.ni = m.ni;
    d.nj = m.nj;
    d.pitch = m.pitch;
    d.per_i = m.per[0];
    d.per_j = m.per[1];
    d.cart = m.cartesian;
    d.field = (size_t)m.pitch * m.nj;
    d.cls = md[k].cls;
    d.met = md[k].met;
    if (m.cartesian) {
      d.mc[0] = m.h[1];
      d.mc[1] = 0.0;
      d.mc[2] = 0.0;
      d.mc[3] = m.h[0];
      d.mc[4] = 1.0 / (m.h[0] * m.h[1]);
    }
    return d;
  }

  Gas gas() const {
    Gas g{};
    g.gamma = p.gamma;
    g.mu = viscous() ? p.mu : 0.0;
    g.pr = p.pr;
    g.twall = p.twall;
    g.sig_int = p.sigma_interface;
    g.sig_phys = p.sigma_physical;
    for (int v = 0; v < 4; ++v) g.qinf[v] = p.qinf[v];
    return g;
  }

  // Interpolate the donor state (optionally extrapolated) to recv's receivers, into recv's
  // workspace.
  cudaError_t interp(int recv, const void *q_donor, const void *const *hist, const double *beta, int nbeta,
                     cudaStream_t s) {
    InterpLaunch a{};
    a.d = dev_mesh(1 - recv);
    a.g = gas();
    a.q = q_donor;
    a.nbeta = nbeta;
    for (int k = 0; k < nbeta; ++k) {
      a.hist[k] = hist[k];
      a.beta[k] = beta[k];
    }
    a.nrecv = (int)mh[recv].recv_pt.size();
    a.base = md[recv].base;
    a.w = md[recv].w;
    a.qhat = md[recv].qhat;
    a.fvhat = viscous() ? md[recv].fvhat : nullptr;
    return launch_interp(a, p.dtype, viscous(), s);
  }

  // Launch descriptor of mesh k's right-hand side at state q, with the kernel shape chosen for
  // the fused right-hand side + update (eval = false) or for the right-hand side alone (true).
  RhsLaunch rhs_args(int k, const void *q, bool eval = false) const {
    RhsLaunch a{};
    a.m = dev_mesh(k);
    a.g = gas();
    a.q = q;
    a.tile_sat = md[k].tile_sat;
    a.rows_per_cta = eval ? md[k].e_rows : md[k].rows_per_cta;
    a.rows_upd = eval ? md[k].e_rows_upd : md[k].rows_upd;
    a.strip = eval ? md[k].e_strip : md[k].strip;
    a.chunk = eval ? md[k].e_chunk : md[k].chunk;
    a.flux = md[k].flux;
    a.sat_ij = md[k].sat_ij;
    a.sat_code = md[k].sat_code;
    a.sat_recv = md[k].sat_recv;
    a.sat_scale = md[k].sat_scale;
    a.qhat = md[k].qhat;
    a.fvhat = md[k].fvhat;
    a.nrecv = (int)mh[k].recv_pt.size();
    a.err = d_err;
    a.sat = md[k].sat;
    a.nsat = (int)mh[k].sat_pt.size();
    a.dwt = md[k].wt;
    fill_consts(k, a.cf);
    fill_consts(k, a.cd);
    return a;
  }

  template <typename T>
  void fill_consts(int k, KConst<T> &c) const {
    const double g = p.gamma, mu = viscous() ? p.mu : 0.0;
    c.gam = (T)g;
    c.g1 = (T)(g - 1.0);
    c.mu = (T)mu;
    c.kap = (T)(mu / (p.pr * (g - 1.0)));
    c.mu43 = (T)(4.0 / 3.0 * mu);
    c.mu23 = (T)(2.0 / 3.0 * mu);
    c.sig_int = (T)p.sigma_interface;
    c.sig_phys = (T)p.sigma_physical;
    c.tw = (T)(p.twall / (g * (g - 1.0)));
    for (int v = 0; v < 4; ++v) c.qinf[v] = (T)p.qinf[v];
    const MeshHost &m = mh[k];
    c.sponge_d = 0;
    c.sponge_faces = 0;
    for (int f = 0; f < 4; ++f)
      if (m.bc[f] == SBP_BC_FARFIELD) c.sponge_faces |= 1 << f;
    if (p.sponge_cells > 0 && c.sponge_faces) c.sponge_d = p.sponge_cells;
    for (int d = 0; d < 16; ++d) {
      const double r = d < p.sponge_cells ? (double)(p.sponge_cells - d) / p.sponge_cells : 0.0;
      c.sponge_tab[d] = (T)(p.sponge_strength * r * r);
    }
    if (m.cartesian) {
      c.mc[0] = (T)m.h[1];
      c.mc[1] = (T)0;
      c.mc[2] = (T)0;
      c.mc[3] = (T)m.h[0];
      c.mc[4] = (T)(1.0 / (m.h[0] * m.h[1]));
      c.jx = (T)(1.0 / m.h[0]);
      c.jy = (T)(1.0 / m.h[1]);
      for (int r = 0; r < 6; ++r)
        for (int e = 0; e < 4; ++e) {
          c.wx[r][e] = (T)(kSbpRows[r][e] / m.h[0]);
          c.wy[r][e] = (T)(kSbpRows[r][e] / m.h[1]);
        }
    } else {
      for (int q = 0; q < 5; ++q) c.mc[q] = (T)0;
      c.jx = c.jy = (T)0;
      for (int r = 0; r < 6; ++r)
        for (int e = 0; e < 4; ++e) c.wx[r][e] = c.wy[r][e] = (T)0;
    }
  }

  cudaError_t rhs_plain(int k, const void *q_self, const void *q_other, void *out, cudaStream_t s) {
    cudaError_t e = interp(k, q_other, nullptr, nullptr, 0, s);
    if (e != cudaSuccess) return e;
    RhsLaunch a = rhs_args(k, q_self, true);
    a.mode = 0;
    a.out = out;
    return launch_rhs(a, p.dtype, viscous(), s);
  }

  void *hist_slot(int k, int slot) const { return (char *)md[k].hist + (size_t)slot * state_elems(k) * esz; }

  // Donor values of mesh `recv`'s receivers from the other mesh's state at `q`, for the
  // extrapolation sets [set0, set0 + nsets) of the plan (set j: slow extrapolant over [0, j/SR]).
  DonorLaunch donor_args(int recv, const void *q, int set0, int nsets, bool extrapolate, double Hh) const {
    DonorLaunch a{};
    const int don = 1 - recv, m = plan.m;
    a.d = dev_mesh(don);
    a.g = gas();
    a.q = q;
    a.nsets = nsets;
    a.npts = md[recv].ndv;
    a.pts = md[recv].dpts;
    a.dv = (char *)md[recv].dv + (size_t)set0 * 10 * md[recv].ndv * esz;
    for (int k = 0; k < m; ++k) a.hist[k] = hist_slot(don, (md[don].head + 1 + k) % m);
    for (int j = 0; j < nsets; ++j) {
      int set = set0 + j;
      a.nb[j] = (extrapolate && set > 0) ? m : 0;
      for (int k = 0; k < m; ++k) a.beta[j][k] = extrapolate ? plan.ext[set][k] * Hh : 0.0;
    }
    return a;
  }

  // Adams-Bashforth weights of one fastest-first macro step solved on the history's node times
  // (macro steps that change H, Sec. 3.3 Step 1), already multiplied by their steps: the slow
  // update, the slow extrapolation sets, and the update of each fast micro step. The nodes of
  // each weight set are shifted to the start of the interval it integrates and scaled by its
  // step, so that a uniform history gives the plan's weights.
  struct StepCoef {
    double as[kMaxHist];
    double ext[kMaxSets][kMaxHist];
    double af[kMaxSets][kMaxHist];
  };
  bool step_coef(StepCoef &c) const {
    const int F = fast(), Sl = slow(), m = plan.m, sr = plan.sr, n = plan.order;
    const double h = H / sr;
    std::vector<double> rel(m), w;
    const int hs = (md[Sl].head + 1) % m;  // the slot a_s(t) is pushed into
    for (int k = 0; k < m; ++k) {
      const int slot = (hs + 1 + k) % m;
      rel[k] = ((slot == hs ? t : tnode[Sl][slot]) - t) / H;
    }
    if (solve_ab_weights(rel, 0.0, 1.0, n, w) != SBP_OK) return false;
    for (int k = 0; k < m; ++k) c.as[k] = w[k] * H;
    for (int j = 1; j < sr; ++j) {
      if (solve_ab_weights(rel, 0.0, (double)j / sr, n, w) != SBP_OK) return false;
      for (int k = 0; k < m; ++k) c.ext[j][k] = w[k] * H;
    }
    double ring[kMaxHist];
    for (int k = 0; k < m; ++k) ring[k] = tnode[F][k];
    int hf = md[F].head;
    for (int j = 0; j < sr; ++j) {
      const double tj = t + j * h;
      hf = (hf + 1) % m;
      ring[hf] = tj;
      for (int k = 0; k < m; ++k) rel[k] = (ring[(hf + 1 + k) % m] - tj) / h;
      if (solve_ab_weights(rel, 0.0, 1.0, n, w) != SBP_OK) return false;
      for (int k = 0; k < m; ++k) c.af[j][k] = w[k] * h;
    }
    return true;
  }

  cudaError_t donor_vals(int recv, const void *q, int set0, int nsets, bool extrapolate, double Hh,
                         cudaStream_t s) {
    return launch_donor_vals(donor_args(recv, q, set0, nsets, extrapolate, Hh), p.dtype, viscous(), s);
  }

  // Fused right-hand side + Adams-Bashforth update of mesh k with step dt, receivers gathered
  // from donor-value set `set`. Pushes the new right-hand side into the ring slot after head.
  cudaError_t fused(int k, int set, double dt, cudaStream_t s, const double *alpha = nullptr) {
    return launch_rhs(fused_args(k, set, dt, alpha), p.dtype, viscous(), s);
  }

  // alpha: the m weights (oldest first, multiplied by the step) instead of the plan's
  RhsLaunch fused_args(int k, int set, double dt, const double *alpha = nullptr) const {
    const int m = plan.m;
    const MeshDev &d = md[k];
    int slot = (d.head + 1) % m;
    RhsLaunch a = rhs_args(k, d.q[d.cur]);
    a.dv = (char *)d.dv + (size_t)set * 10 * d.ndv * esz;
    a.didx = d.didx;
    a.ndv = d.ndv;
    a.mode = 1;
    a.out = hist_slot(k, slot);
    a.qnext = d.q[1 - d.cur];
    a.nold = m - 1;
    for (int j = 0; j < m - 1; ++j) {
      a.hold[j] = hist_slot(k, (slot + 1 + j) % m);
      a.alpha[j] = alpha ? alpha[j] : plan.ab[j] * dt;
    }
    a.alpha[m - 1] = alpha ? alpha[m - 1] : plan.ab[m - 1] * dt;
    // fast micro steps hand the primitives of the state they produce to the next micro step
    // (the split kernels' flux kernel then loads them instead of computing its halo's)
    if (k == fast() && d.prim && d.strip == 0) {
      if (set > 0) a.prim_in = d.prim;
      if (set < plan.sr - 1) a.prim_out = d.prim;
    }
    return a;
  }

  cudaError_t ensure_capture_streams() {
    cudaError_t e = cudaSuccess;
    if (!cap) {
      int least = 0, greatest = 0;
      if ((e = cudaDeviceGetStreamPriorityRange(&least, &greatest)) != cudaSuccess) return e;
      if ((e = cudaStreamCreateWithPriority(&cap, cudaStreamNonBlocking, greatest)) != cudaSuccess) return e;
      if ((e = cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, greatest)) != cudaSuccess) return e;
      if ((e = cudaStreamCreateWithPriority(&side2, cudaStreamNonBlocking, least)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&ev_a, cudaEventDisableTiming)) != cudaSuccess) return e;
      if ((e = cudaEventCreateWithFlags(&ev_b, cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    return e;
  }

  // ---- slowest-first variants (sbp_params.scheme) ----------------------------------------------
  // The slow right-hand side at the slow mesh's state q with receivers from the donor values in
  // set 0 of its workspace, into the slow ring slot after head (mode 0; head unchanged).
  cudaError_t slow_rhs_at(const void *q, cudaStream_t s) {
    const int Sl = slow();
    const MeshDev &d = md[Sl];
    RhsLaunch a = rhs_args(Sl, q, true);
    a.dv = d.dv;
    a.didx = d.didx;
    a.ndv = d.ndv;
    a.mode = 0;
    a.out = hist_slot(Sl, (d.head + 1) % plan.m);
    return launch_rhs(a, p.dtype, viscous(), s);
  }

  // a_s at the current states (receivers from the fast mesh's current state), pushed into the
  // slow ring: the slowest-first variants' first macro step needs the slow history to end at
  // the current time.
  cudaError_t slow_rhs_push(cudaStream_t s) {
    const int Sl = slow(), F = fast();
    cudaError_t e = donor_vals(Sl, md[F].q[md[F].cur], 0, 1, false, H, s);
    if (e == cudaSuccess) e = slow_rhs_at(md[Sl].q[md[Sl].cur], s);
    if (e == cudaSuccess) {
      md[Sl].head = (md[Sl].head + 1) % plan.m;
      md[Sl].count++;
      tnode[Sl][md[Sl].head] = t;
    }
    return e;
  }

  // s(t + H) = s(t) + sum_k alpha_k H a_s,k over the m slow history values (oldest first).
  cudaError_t slow_combine(const void *q_in, void *q_out, cudaStream_t s) {
    const int Sl = slow(), m = plan.m;
    ABCombine c{};
    c.nh = m;
    for (int k = 0; k < m; ++k) {
      c.hist[k] = hist_slot(Sl, (md[Sl].head + 1 + k) % m);
      c.alpha[k] = plan.ab[k] * H;
    }
    return launch_ab_combine(q_in, c, q_out, state_elems(Sl), p.dtype, s);
  }

  // One macro step of the slowest-first variants for the state at entry f(t), s(t), the fast
  // ring ending at a_f(t - h), the slow ring ending at a_s(t):
  //  fast chain: receivers' donor values (set 0 = s(t); without re-extrapolation every set from
  //    the slow extrapolant of the ring ending at a_s(t)), micro step 0 (pushes a_f(t)), and,
  //    once f^ is taken, micro steps 1..SR-1;
  //  slow chain: s(t + H) by the slow extrapolant; after micro step 0, f^(t + H) = f(t) + the
  //    fast extrapolant over the macro step at the slow receivers' donors; a_s(t + H) =
  //    RHS(s(t + H), f^) pushed into the slow ring; with re-extrapolation, then the fast
  //    receivers' sets 1..SR-1 from the slow ring ending at a_s(t + H).
  // With `sd`, the fast chain runs on sd: without re-extrapolation the slow right-hand side
  // and micro steps 1..SR-1 run side by side.
  cudaError_t issue_step_sf(cudaStream_t s, cudaStream_t sd) {
    const int F = fast(), Sl = slow(), sr = plan.sr, m = plan.m;
    const bool rex = p.scheme == SBP_MRAB_SLOWEST_FIRST_REEXTRAPOLATE;
    const double h = H / sr;
    MeshDev saved_s = md[Sl], saved_f = md[F];
    cudaError_t e = cudaSuccess;
    auto run = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    cudaStream_t fs = sd ? sd : s;
    void *s_t = md[Sl].q[md[Sl].cur], *s_new = md[Sl].q[1 - md[Sl].cur];
    void *f_t = md[F].q[md[F].cur];
    if (sd) {
      run(cudaEventRecord(ev_fork, s));
      run(cudaStreamWaitEvent(sd, ev_fork, 0));
    }
    run(timed(SBP_PHASE_INTERP_FAST, fs, [&] { return donor_vals(F, s_t, 0, rex ? 1 : sr, !rex, H, fs); }));
    run(timed(SBP_PHASE_RHS_FAST, fs, [&] { return fused(F, 0, h, fs); }));
    md[F].head = (md[F].head + 1) % m;
    md[F].cur ^= 1;
    if (sd) run(cudaEventRecord(ev_a, sd));
    run(timed(SBP_PHASE_RHS_SLOW, s, [&] { return slow_combine(s_t, s_new, s); }));
    if (sd) run(cudaStreamWaitEvent(s, ev_a, 0));
    run(timed(SBP_PHASE_INTERP_SLOW, s, [&] {
      DonorLaunch a = donor_args(Sl, f_t, 0, 1, false, h);
      a.nb[0] = m;
      for (int k = 0; k < m; ++k) a.beta[0][k] = plan.fext[k] * h;
      return launch_donor_vals(a, p.dtype, viscous(), s);
    }));
    if (sd && !rex) run(cudaEventRecord(ev_b, s));
    run(timed(SBP_PHASE_RHS_SLOW, s, [&] { return slow_rhs_at(s_new, s); }));
    md[Sl].head = (md[Sl].head + 1) % m;
    md[Sl].cur ^= 1;
    if (rex && sr > 1)
      run(timed(SBP_PHASE_INTERP_FAST, s, [&] {
        DonorLaunch a = donor_args(F, s_t, 1, sr - 1, false, H);
        for (int j = 0; j < sr - 1; ++j) {
          a.nb[j] = m;
          for (int k = 0; k < m; ++k) a.beta[j][k] = plan.rext[1 + j][k] * H;
        }
        return launch_donor_vals(a, p.dtype, viscous(), s);
      }));
    if (sd) {
      if (rex) run(cudaEventRecord(ev_b, s));
      run(cudaStreamWaitEvent(sd, ev_b, 0));
    }
    for (int j = 1; j < sr; ++j) {
      run(timed(SBP_PHASE_RHS_FAST, fs, [&] { return fused(F, j, h, fs); }));
      md[F].head = (md[F].head + 1) % m;
      md[F].cur ^= 1;
    }
    if (sd) {
      run(cudaEventRecord(ev_join, sd));
      run(cudaStreamWaitEvent(s, ev_join, 0));
    }
    md[Sl] = saved_s;
    md[F] = saved_f;
    return e;
  }

  // The slow mesh's tiles that the fast receivers' donor values depend on: the update tiles
  // (rows ty_u) holding the distinct donor points and their derivative taps (3 points either
  // way), and the flux tiles (rows ty_f) holding the update tiles' 3-point halos. False (no
  // split) when the split kernels are not the slow mesh's design, the region reaches across a
  // periodic edge, or it covers more than a quarter of the update tiles.
  bool slow_core_boxes(TileBox &fb, TileBox &ub) const {
    const int F = fast(), Sl = slow();
    const MeshDev &d = md[Sl];
    const MeshHost &m = mh[Sl];
    const std::vector<uint32_t> &pts = mh[F].donor_pts;
    if (d.strip != 0 || pts.empty()) return false;
    const int ty_f = d.rows_per_cta, ty_u = d.rows_upd ? d.rows_upd : d.rows_per_cta;
    int i0 = m.ni, i1 = -1, j0 = m.nj, j1 = -1;
    for (uint32_t ij : pts) {
      const int i = (int)(ij & 0xFFFFu), j = (int)(ij >> 16);
      i0 = std::min(i0, i);
      i1 = std::max(i1, i);
      j0 = std::min(j0, j);
      j1 = std::max(j1, j);
    }
    // a point range widened by w on each side: clamped at the ends, refused across a periodic edge
    auto widen = [](int &a, int &b, int w, int n, int per) {
      a -= w;
      b += w;
      if (a < 0 || b > n - 1) {
        if (per) return false;
        a = std::max(a, 0);
        b = std::min(b, n - 1);
      }
      return true;
    };
    if (!widen(i0, i1, 3, m.ni, m.per[0]) || !widen(j0, j1, 3, m.nj, m.per[1])) return false;
    const int nx = (m.ni + kTileX - 1) / kTileX, nyu = (m.nj + ty_u - 1) / ty_u;
    ub = {1, i0 / kTileX, i1 / kTileX + 1, j0 / ty_u, j1 / ty_u + 1};
    if (4L * (ub.x1 - ub.x0) * (ub.y1 - ub.y0) > (long)nx * nyu) return false;
    int fi0 = ub.x0 * kTileX, fi1 = std::min(ub.x1 * kTileX, m.ni) - 1;
    int fj0 = ub.y0 * ty_u, fj1 = std::min(ub.y1 * ty_u, m.nj) - 1;
    if (!widen(fi0, fi1, 3, m.ni, m.per[0]) || !widen(fj0, fj1, 3, m.nj, m.per[1])) return false;
    fb = {1, fi0 / kTileX, fi1 / kTileX + 1, fj0 / ty_f, fj1 / ty_f + 1};
    return true;
  }

  // Enqueue one macro step (Sec. 3.3) for the current ring heads and state buffers, without
  // changing them. With `side` set, the slow right-hand side and the first fast micro step
  // (which needs only s(t) and f(t)) run on two streams joined before the second micro step.
  // With side2 as well (graph capture), the slow right-hand side is split: the tiles that the
  // fast receivers' extrapolated donor values read (slow_core_boxes) stay on the critical path,
  // and the rest of the mesh runs on side2 beside the fast micro steps (the same kernels and
  // arithmetic on fewer tiles: the same bits), joined at the end of the macro step.
  // frec (eager mode only): the fast state before micro step j is copied to frec[j].
  cudaError_t issue_step(cudaStream_t s, cudaStream_t sd, void *const *frec = nullptr, const StepCoef *cf = nullptr) {
    if (p.scheme != SBP_MRAB_FASTEST_FIRST) return issue_step_sf(s, sd);
    const int F = fast(), Sl = slow(), sr = plan.sr;
    const double h = H / sr;
    MeshDev saved_s = md[Sl], saved_f = md[F];
    cudaError_t e = cudaSuccess;
    auto run = [&](cudaError_t x) {
      if (e == cudaSuccess) e = x;
    };
    if (sd) {
      run(cudaEventRecord(ev_fork, s));
      run(cudaStreamWaitEvent(sd, ev_fork, 0));
      // side: fast receivers from s(t), first micro step
      run(donor_vals(F, md[Sl].q[md[Sl].cur], 0, 1, false, H, sd));
      run(fused(F, 0, h, sd));
    }
    // slow: receivers from f(t), fused RHS + update into the other buffer
    run(timed(SBP_PHASE_INTERP_SLOW, s, [&] { return donor_vals(Sl, md[F].q[md[F].cur], 0, 1, false, H, s); }));
    TileBox fb{}, ub{};
    const bool split = sd && side2 && sd != side2 && sr > 1 && slow_core_boxes(fb, ub);
    if (split) {
      RhsLaunch a = fused_args(Sl, 0, H, cf ? cf->as : nullptr);
      a.fbox = fb;
      a.ubox = ub;
      run(launch_rhs(a, p.dtype, viscous(), s));
      run(cudaEventRecord(ev_a, s));
      run(cudaStreamWaitEvent(side2, ev_a, 0));
      a.fbox.mode = 2;
      a.ubox.mode = 2;
      run(launch_rhs(a, p.dtype, viscous(), side2));
      run(cudaEventRecord(ev_b, side2));
    } else {
      run(timed(SBP_PHASE_RHS_SLOW, s, [&] { return fused(Sl, 0, H, s, cf ? cf->as : nullptr); }));
    }
    md[Sl].head = (md[Sl].head + 1) % plan.m;
    // fast receivers for the micro steps that need the slow extrapolant (a_s(t) is now in the ring)
    int first = sd ? 1 : 0;
    if (sr > first)
      run(timed(SBP_PHASE_INTERP_FAST, s, [&] {
        DonorLaunch a = donor_args(F, md[Sl].q[md[Sl].cur], first, sr - first, true, H);
        if (cf)
          for (int j = 0; j < sr - first; ++j)
            for (int k = 0; k < plan.m; ++k) a.beta[j][k] = cf->ext[first + j][k];
        return launch_donor_vals(a, p.dtype, viscous(), s);
      }));
    if (sd) {
      md[F].head = (md[F].head + 1) % plan.m;
      md[F].cur ^= 1;
      run(cudaEventRecord(ev_join, sd));
      run(cudaStreamWaitEvent(s, ev_join, 0));
    }
    for (int j = first; j < sr; ++j) {
      if (frec)
        run(cudaMemcpyAsync(frec[j], md[F].q[md[F].cur], state_elems(F) * esz, cudaMemcpyDeviceToDevice, s));
      run(timed(SBP_PHASE_RHS_FAST, s, [&] { return fused(F, j, h, s, cf ? cf->af[j] : nullptr); }));
      md[F].head = (md[F].head + 1) % plan.m;
      md[F].cur ^= 1;
    }
    if (split) run(cudaStreamWaitEvent(s, ev_b, 0));
    md[Sl] = saved_s;
    md[F] = saved_f;
    return e;
  }

  // Host bookkeeping after one macro step.
  void advance() {
    md[slow()].head = (md[slow()].head + 1) % plan.m;
    md[slow()].cur ^= 1;
    // a_s(t); the slowest-first orderings push a_s(t + H)
    tnode[slow()][md[slow()].head] = p.scheme == SBP_MRAB_FASTEST_FIRST ? t : t + H;
    for (int j = 0; j < plan.sr; ++j) {
      md[fast()].head = (md[fast()].head + 1) % plan.m;
      md[fast()].cur ^= 1;
      tnode[fast()][md[fast()].head] = t + j * (H / plan.sr);
    }
    t += H;
  }

  // Autotuner of the right-hand side's kernel and block shape: for each mesh and each use, time
  // every candidate on the bound state and keep the fastest. The uses are the fused right-hand
  // side + MRAB update of the macro step (a fast mesh's micro step 1, which takes the primitives
  // handed over by micro step 0) and the right-hand side alone (rhs_eval, Runge-Kutta stages),
  // both with their outputs in the state buffer the next step overwrites (each point's stores
  // come from its own thread; the bound history is only read). Candidates: the split kernels at
  // 4, 8, 16 and 32 rows per CTA, the marching kernel (strips of kMarchW columns) at chunks of
  // 8, 16, 32, 64 and 128 rows, staged by cp.async or (chunks of 16 to 128) by TMA tensor
  // copies, and the column-marching kernel (CTAs of 128 or 256 threads, on
  // meshes at least that wide) at chunks of 32 to 256 rows; each timed as the faster of two runs
  // of three launches. A fast mesh's fused step follows the rules of sbp_tune.h (tune_eligible,
  // tune_pick: every SM a CTA, Navier-Stokes flux tiles of at least 8 rows, the most CTAs among
  // the candidates within 3 % of the fastest). Timed alone, shapes of fewer, larger CTAs can win
  // by a few percent and then lose in the macro step, where the slow mesh's CTAs share the SMs:
  // on the cylinder's O-grid, 16-row flux tiles time within 2 % of 8-row ones alone, but the
  // FP64 macro step takes 0.357 ms with them, 0.335 ms with 8-row flux and derivative tiles and
  // 0.322 ms with 4-row derivative tiles.
  bool autotune_on = true;
  cudaError_t autotune(cudaStream_t s) {
    using Cand = TuneCand;
    static const std::vector<Cand> cand_list = tune_candidates(kMarchW, kColW128, kColW256, kStageTma);
    const Cand *cands = cand_list.data();
    const int ncand = (int)cand_list.size();
    Cand step_shape[2] = {{0, 16, 0}, {0, 16, 0}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int n_sm = 1, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      MeshDev &d = md[k];
      if (!d.hist) continue;
      e = interp(k, md[1 - k].q[md[1 - k].cur], nullptr, nullptr, 0, s);
      for (int use = 0; use < 2 && e == cudaSuccess; ++use) {  // 0: fused step, 1: rhs alone
        Cand best_c{0, 16, 0};
        const bool critical = use == 0 && k == fast() && plan.sr > 1;
        const TuneMesh tm{mh[k].ni, mh[k].nj, viscous(), kTileX, kStageTma, kMarchW};
        std::vector<std::pair<float, int>> timed;
        for (int ci : tune_eligible(cands, ncand, tm, critical, n_sm)) {
          const Cand &c = cands[ci];
          if (e != cudaSuccess) continue;
          d.strip = d.e_strip = c.strip;
          if (c.strip) d.chunk = d.e_chunk = c.rows;
          else d.rows_per_cta = d.e_rows = c.rows;
          d.rows_upd = d.e_rows_upd = c.rows_upd;
          RhsLaunch a;
          if (use == 0) {
            a = fused_args(k, (k == fast() && plan.sr > 1) ? 1 : 0, k == fast() ? H / plan.sr : H);
            a.out = a.qnext = d.q[1 - d.cur];
          } else {
            a = rhs_args(k, d.q[d.cur], true);
            a.mode = 0;
            a.out = d.q[1 - d.cur];
          }
          // timing runs: micro step 1's history ring holds a slot micro step 0 has not written
          // yet, so the values are scratch and are not checked
          a.err = nullptr;
          e = launch_rhs(a, p.dtype, viscous(), s);
          float ms = 1e30f;
          for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaEventRecord(e0, s);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r) e = launch_rhs(a, p.dtype, viscous(), s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && t < ms) ms = t;
          }
          if (e == cudaSuccess) timed.push_back({ms, ci});
        }
        const int pick = tune_pick(cands, timed, tm, critical);
        if (pick >= 0) best_c = cands[pick];
        if (use == 0) {
          step_shape[k] = best_c;
        } else {
          d.e_strip = best_c.strip;
          if (best_c.strip) d.e_chunk = best_c.rows;
          else d.e_rows = best_c.rows;
          d.e_rows_upd = best_c.rows_upd;
        }
      }
      d.strip = step_shape[k].strip;
      if (step_shape[k].strip) d.chunk = step_shape[k].rows;
      else d.rows_per_cta = step_shape[k].rows;
      d.rows_upd = step_shape[k].rows_upd;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
  }

  // Bootstrap of Sec. 3.1 on the bound buffers: Heun's third-order Runge-Kutta at the micro
  // step h = H / SR for (m - 1) SR steps on both meshes, recording the fast right-hand side of
  // the last m - 1 steps and the slow one every SR steps into the rings. With ystore set, the
  // state of mesh k before step n is copied to ystore[k] + n * state size first.
  cudaError_t bootstrap(double Hm, cudaStream_t s, void *const *ystore) {
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
      md[k].count = 0;
    }
    const int nsteps = (m - 1) * sr;
    for (int step = 0; step < nsteps && e == cudaSuccess; ++step) {
      void *y[2] = {md[0].q[md[0].cur], md[1].q[md[1].cur]};
      void *k1[2] = {k1tmp[0], k1tmp[1]};
      if (ystore)
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
          size_t b = state_elems(k) * esz;
          e = cudaMemcpyAsync((char *)ystore[k] + (size_t)step * b, y[k], b, cudaMemcpyDeviceToDevice, s);
        }
      bool rec_f = step >= nsteps - (m - 1), rec_s = step % sr == 0;
      if (rec_f) {
        MeshDev &d = md[F];
        d.head = (d.head + 1) % m;
        d.count++;
        k1[F] = hist_slot(F, d.head);
        tnode[F][d.head] = (double)(step - nsteps) * h;
      }
      if (rec_s) {
        MeshDev &d = md[Sl];
        d.head = (d.head + 1) % m;
        d.count++;
        k1[Sl] = hist_slot(Sl, d.head);
        tnode[Sl][d.head] = (double)((step - nsteps) / sr) * Hm;
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

  // One classical Runge-Kutta step of size h on both meshes, in place on the current state
  // buffers: k_i = f(y_i) with y_1 = y, y_2 = y + h/2 k_1, y_3 = y + h/2 k_2, y_4 = y + h k_3,
  // each stage with the overset coupling to the other mesh's stage state, then
  // y + h/6 k_1 + h/3 k_2 + h/3 k_3 + h/6 k_4 (two FP64-accumulated passes).
  cudaError_t issue_rk4(double h, cudaStream_t s) {
    void *y[2], *ys[2], *kk[2][4];
    for (int k = 0; k < 2; ++k) {
      const size_t b = state_elems(k) * esz;
      y[k] = md[k].q[md[k].cur];
      ys[k] = rk_buf[k];
      for (int i = 0; i < 4; ++i) kk[k][i] = (char *)rk_buf[k] + (size_t)(1 + i) * b;
    }
    cudaError_t e = cudaSuccess;
    auto stage = [&](void *const *in, int i) {
      for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = rhs_plain(k, in[k], in[1 - k], kk[k][i], s);
    };
    const double c[3] = {0.5 * h, 0.5 * h, h};
    stage(y, 0);
    for (int i = 0; i < 3; ++i) {
      for (int k = 0; k < 2 && e == cudaSuccess; ++k)
        e = launch_axpy(y[k], kk[k][i], c[i], nullptr, 0.0, ys[k], state_elems(k), p.dtype, s);
      stage(ys, i + 1);
    }
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = launch_axpy(y[k], kk[k][0], h / 6.0, kk[k][1], h / 3.0, ys[k], state_elems(k), p.dtype, s);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = launch_axpy(ys[k], kk[k][2], h / 3.0, kk[k][3], h / 6.0, y[k], state_elems(k), p.dtype, s);
    return e;
  }

  cudaError_t rk4(int n, double h, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      if (rk_buf[k]) continue;
      const size_t b = 5 * state_elems(k) * esz;
      e = cudaMalloc(&rk_buf[k], b);
      if (e == cudaSuccess) e = cudaMemsetAsync(rk_buf[k], 0, b, s);
    }
    if (e != cudaSuccess) return e;
    const int key = md[0].cur | (md[1].cur << 1);
    if (use_graph && !prof) {
      if (!rk_graph || rk_graph_h != h || rk_graph_cur != key) {
        if (rk_graph) cudaGraphExecDestroy(rk_graph);
        rk_graph = nullptr;
        if ((e = ensure_capture_streams()) != cudaSuccess) return e;
        if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
        cudaError_t ei = issue_rk4(h, cap);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        if (ei != cudaSuccess) {
          if (g) cudaGraphDestroy(g);
          return ei;
        }
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&rk_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return e;
        rk_graph_h = h;
        rk_graph_cur = key;
      }
      for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaGraphLaunch(rk_graph, s);
    } else {
      for (int i = 0; i < n && e == cudaSuccess; ++i) e = issue_rk4(h, s);
    }
    return e;
  }

  uint64_t phase_key() const {
    const MeshDev &a = md[slow()], &b = md[fast()];
    return (uint64_t)a.cur | ((uint64_t)a.head << 1) | ((uint64_t)b.cur << 8) | ((uint64_t)b.head << 9);
  }

  cudaError_t launch_step_graph(cudaStream_t s) {
    uint64_t key = phase_key();
    auto it = graphs.find(key);
    if (it == graphs.end()) {
      cudaError_t e;
      if ((e = ensure_capture_streams()) != cudaSuccess) return e;
      if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
      cudaError_t ei = issue_step(cap, side);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cap, &g);
      if (ei != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return ei;
      }
      if (e != cudaSuccess) return e;
      // count the kernel nodes (the macro step's launches of this library)
      size_t nn = 0;
      int nk = 0;
      e = cudaGraphGetNodes(g, nullptr, &nn);
      if (e == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        e = cudaGraphGetNodes(g, nodes.data(), &nn);
        for (size_t i = 0; i < nn && e == cudaSuccess; ++i) {
          cudaGraphNodeType t;
          e = cudaGraphNodeGetType(nodes[i], &t);
          if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
        }
      }
      if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return e;
      }
      graph_kernels[key] = nk;
      cudaGraphExec_t ex = nullptr;
      // kernel nodes keep the priorities of the streams they were captured on
      e = cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
      it = graphs.emplace(key, ex).first;
    }
    last_graph_kernels = graph_kernels[key];
    return cudaGraphLaunch(it->second, s);
  }
};

namespace sbp {
// Device tables of mesh k of S from its host setup (sbp_capi.cpp).
sbp_status upload_mesh_tables(sbp_system_s *S, int k);
}  // namespace sbp
