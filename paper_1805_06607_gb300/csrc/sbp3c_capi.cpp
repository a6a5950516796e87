// C ABI of the 3D curvilinear operator: a mesh object holding the device metric terms, and the
// flux divergence of a state (App. C.1's equations in curvilinear coordinates, Sec. 2.1's SBP
// 4-2 derivative with closures on every line; optionally the far-field SAT of Sec. 5.1 on every
// face), the interface SAT at given receivers and the overset gather. Kernels: sbp3c_kernels.cu;
// host donor search and hole cut: sbp3c_setup.cpp.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "sbp3c_device.h"
#include "sbp_system.h"

using namespace sbp;

struct sbp3c_mesh_s {
  int n[3] = {0, 0, 0};
  sbp_params p{};
  size_t field = 0, esz = 8;
  void *met = nullptr, *prim = nullptr, *flux = nullptr;
  int *d_err = nullptr;  // device error word (SBP_ERR_BOUNDS from the gather)
  int far = 0;
  double sig = 0.0, qinf[5] = {0, 0, 0, 0, 0};
  // interface SAT terms grouped by receiver point (device)
  int i_npt = 0, i_nrecv = 0;
  double i_sig = 0.0;
  long long *i_pt = nullptr;
  int *i_off = nullptr, *i_term = nullptr;
  double *i_scale = nullptr;
  void free_interface() {
    cudaFree(i_pt);
    cudaFree(i_off);
    cudaFree(i_term);
    cudaFree(i_scale);
    i_pt = nullptr;
    i_off = i_term = nullptr;
    i_scale = nullptr;
    i_npt = i_nrecv = 0;
  }
  ~sbp3c_mesh_s() {
    cudaFree(d_err);
    cudaFree(met);
    cudaFree(prim);
    cudaFree(flux);
    free_interface();
  }
};

extern "C" {

sbp_status sbp3c_mesh_create(const int *n, const double *x, const double *y, const double *z,
                             const sbp_params *params, sbp3c_mesh_t *out) {
  if (!n || !x || !y || !z || !params || !out) return fail(SBP_ERR_ARG, "null argument");
  *out = nullptr;
  const sbp_params &p = *params;
  if (p.physics != SBP_EULER && p.physics != SBP_NS) return fail(SBP_ERR_ARG, "physics");
  if (p.dtype != SBP_F64 && p.dtype != SBP_F32) return fail(SBP_ERR_DTYPE, "dtype");
  if (!(p.gamma > 1.0) || p.mu < 0.0 || !(p.pr > 0.0)) return fail(SBP_ERR_ARG, "gas constants");
  for (int a = 0; a < 3; ++a)
    if (n[a] < 8 || n[a] > 65535) return fail(SBP_ERR_SHAPE, "each direction needs 8..65535 points");
  const long long N = (long long)n[0] * n[1] * n[2];
  if (N > 2147483647LL / 16) return fail(SBP_ERR_SHAPE, "mesh too large");
  auto *M = new sbp3c_mesh_s();
  std::unique_ptr<sbp3c_mesh_s> guard(M);
  std::memcpy(M->n, n, sizeof(M->n));
  M->p = p;
  M->field = (size_t)N;
  M->esz = p.dtype == SBP_F64 ? 8 : 4;
  double *dxyz = nullptr, *ddx = nullptr;
  cudaError_t e = cudaMalloc((void **)&dxyz, 3 * M->field * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void **)&ddx, 9 * M->field * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(dxyz, x, M->field * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dxyz + M->field, y, M->field * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dxyz + 2 * M->field, z, M->field * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&M->met, 10 * M->field * M->esz);
  if (e == cudaSuccess) e = launch3c_metrics(n[0], n[1], n[2], dxyz, ddx, M->met, p.dtype, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(dxyz);
  cudaFree(ddx);
  CUDA_TRY(e);
  if (p.physics == SBP_NS) CUDA_TRY(cudaMalloc(&M->prim, 4 * M->field * M->esz));
  CUDA_TRY(cudaMalloc(&M->flux, 15 * M->field * M->esz));
  CUDA_TRY(cudaMalloc((void **)&M->d_err, sizeof(int)));
  CUDA_TRY(cudaMemset(M->d_err, 0, sizeof(int)));
  *out = guard.release();
  return SBP_OK;
}

sbp_status sbp3c_mesh_check(sbp3c_mesh_t M, void *stream) {
  if (!M) return fail(SBP_ERR_ARG, "null mesh");
  CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  int e = 0;
  CUDA_TRY(cudaMemcpy(&e, M->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(M->d_err, 0, sizeof(int)));
  if (e) return fail((sbp_status)e, "device error word set");
  return SBP_OK;
}

sbp_status sbp3c_mesh_destroy(sbp3c_mesh_t M) {
  delete M;
  return SBP_OK;
}

sbp_status sbp3c_get_metrics(sbp3c_mesh_t M, double *metrics) {
  if (!M || !metrics) return fail(SBP_ERR_ARG, "bad argument");
  const size_t n = 10 * M->field;
  if (M->esz == 8) {
    CUDA_TRY(cudaMemcpy(metrics, M->met, n * sizeof(double), cudaMemcpyDeviceToHost));
  } else {
    std::unique_ptr<float[]> buf(new float[n]);
    CUDA_TRY(cudaMemcpy(buf.get(), M->met, n * sizeof(float), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < n; ++i) metrics[i] = buf[i];
  }
  return SBP_OK;
}

sbp_status sbp3c_set_farfield(sbp3c_mesh_t M, const double *qinf, double sigma) {
  if (!M) return fail(SBP_ERR_ARG, "null mesh");
  if (!qinf) {
    M->far = 0;
    return SBP_OK;
  }
  if (!(sigma >= 0.0) || !(qinf[0] > 0.0)) return fail(SBP_ERR_ARG, "far field: sigma >= 0 and rho > 0 required");
  const double ke = 0.5 * (qinf[1] * qinf[1] + qinf[2] * qinf[2] + qinf[3] * qinf[3]) / qinf[0];
  if (!((M->p.gamma - 1.0) * (qinf[4] - ke) > 0.0)) return fail(SBP_ERR_ARG, "far field: pressure must be positive");
  M->far = 1;
  M->sig = sigma;
  std::memcpy(M->qinf, qinf, sizeof(M->qinf));
  return SBP_OK;
}

sbp_status sbp3c_interp(sbp3c_mesh_t M, const void *q, int nrecv, const int *base, const double *w, void *out,
                        void *stream) {
  if (!M || nrecv < 0 || (nrecv > 0 && (!q || !base || !w || !out))) return fail(SBP_ERR_ARG, "bad argument");
  CUDA_TRY(launch3c_interp(M->n[0], M->n[1], M->n[2], q, nrecv, base, w, out, M->d_err, M->p.dtype,
                           (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp3c_set_interface(sbp3c_mesh_t M, int nterms, const int *terms, const double *scale, int nrecv,
                               double sigma) {
  if (!M || nterms < 0 || nrecv < 0 || (nterms > 0 && !terms) || !(sigma >= 0.0))
    return fail(SBP_ERR_ARG, "bad argument");
  std::vector<std::pair<long long, int>> order;  // (point, term) sorted by point, stable
  order.reserve(nterms);
  for (int e = 0; e < nterms; ++e) {
    const int *t = terms + 6 * (size_t)e;
    if (t[0] < 0 || t[0] >= M->n[0] || t[1] < 0 || t[1] >= M->n[1] || t[2] < 0 || t[2] >= M->n[2])
      return fail(SBP_ERR_ARG, "interface term " + std::to_string(e) + ": point outside the mesh");
    if (t[3] < 0 || t[3] > 2 || (t[4] != 1 && t[4] != -1) || t[5] < 0 || t[5] >= nrecv)
      return fail(SBP_ERR_ARG, "interface term " + std::to_string(e) + ": direction, side or receiver column");
    order.emplace_back(((long long)t[2] * M->n[1] + t[1]) * M->n[0] + t[0], e);
  }
  std::stable_sort(order.begin(), order.end(),
                   [](const std::pair<long long, int> &x, const std::pair<long long, int> &y) { return x.first < y.first; });
  std::vector<long long> pt;
  std::vector<int> off, term;
  std::vector<double> sc;
  for (size_t u = 0; u < order.size(); ++u) {
    if (u == 0 || order[u].first != order[u - 1].first) {
      pt.push_back(order[u].first);
      off.push_back((int)u);
    }
    const int *t = terms + 6 * (size_t)order[u].second;
    term.insert(term.end(), {t[3], t[4], t[5]});
    sc.push_back(scale ? scale[order[u].second] : 1.0);
  }
  off.push_back((int)order.size());
  M->free_interface();
  CUDA_TRY(upload(M->i_pt, pt.data(), pt.size() * sizeof(long long)));
  CUDA_TRY(upload(M->i_off, off.data(), off.size() * sizeof(int)));
  CUDA_TRY(upload(M->i_term, term.data(), term.size() * sizeof(int)));
  CUDA_TRY(upload(M->i_scale, sc.data(), sc.size() * sizeof(double)));
  M->i_npt = (int)pt.size();
  M->i_nrecv = nrecv;
  M->i_sig = sigma;
  return SBP_OK;
}

static Curv3Launch curv_args(sbp3c_mesh_t M, const void *q, void *rhs) {
  Curv3Launch a{};
  a.ni = M->n[0];
  a.nj = M->n[1];
  a.nk = M->n[2];
  a.field = M->field;
  a.visc = M->p.physics == SBP_NS;
  a.gam = M->p.gamma;
  a.mu = a.visc ? M->p.mu : 0.0;
  a.lam = -2.0 / 3.0 * a.mu;
  a.kap = a.mu / (M->p.pr * (M->p.gamma - 1.0));
  a.q = q;
  a.out = rhs;
  a.met = M->met;
  a.prim = M->prim;
  a.flux = M->flux;
  a.far = M->far;
  a.sig = M->sig;
  std::memcpy(a.qinf, M->qinf, sizeof(a.qinf));
  return a;
}

sbp_status sbp3c_interface_sat(sbp3c_mesh_t M, const void *q, const void *qhat, const void *fvhat, void *rhs,
                               void *stream) {
  if (!M || !q || !rhs || (M->i_npt > 0 && !qhat)) return fail(SBP_ERR_ARG, "bad argument");
  if (M->p.physics == SBP_NS && M->i_npt > 0 && !fvhat)
    return fail(SBP_ERR_ARG, "Navier-Stokes interface terms need the donor viscous fluxes");
  Curv3Sat sat{};
  sat.npt = M->i_npt;
  sat.nrecv = M->i_nrecv;
  sat.pt = M->i_pt;
  sat.off = M->i_off;
  sat.term = M->i_term;
  sat.scale = M->i_scale;
  sat.qhat = qhat;
  sat.fvhat = fvhat;
  sat.sig = M->i_sig;
  CUDA_TRY(launch3c_isat(curv_args(M, q, rhs), sat, M->p.dtype, (cudaStream_t)stream));
  return SBP_OK;
}

sbp_status sbp3c_rhs_eval(sbp3c_mesh_t M, const void *q, void *rhs, void *stream) {
  if (!M || !q || !rhs) return fail(SBP_ERR_ARG, "bad argument");
  Curv3Launch a{};
  a.ni = M->n[0];
  a.nj = M->n[1];
  a.nk = M->n[2];
  a.field = M->field;
  a.visc = M->p.physics == SBP_NS;
  a.gam = M->p.gamma;
  a.mu = a.visc ? M->p.mu : 0.0;
  a.lam = -2.0 / 3.0 * a.mu;
  a.kap = a.mu / (M->p.pr * (M->p.gamma - 1.0));
  a.q = q;
  a.out = rhs;
  a.met = M->met;
  a.prim = M->prim;
  a.flux = M->flux;
  a.far = M->far;
  a.sig = M->sig;
  std::memcpy(a.qinf, M->qinf, sizeof(a.qinf));
  CUDA_TRY(launch3c_rhs(a, M->p.dtype, (cudaStream_t)stream));
  return SBP_OK;
}

}  // extern "C"
