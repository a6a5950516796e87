// Host-only rules of the right-hand-side autotuner (no CUDA): which candidate shapes a mesh's
// use times, and which timed candidate it keeps. The autotuner in sbp_system.h times the
// eligible candidates on the GPU; these functions decide around the timing, so the host test
// (tests/test_host_tune.py) checks them with given times.
#pragma once
#include <algorithm>
#include <utility>
#include <vector>

namespace sbp {

// A right-hand-side shape: strip 0 is the kernel pair (rows: flux rows per CTA, rows_upd:
// derivative rows, 0 = the same); strip > 0 a single-pass kernel of that strip width with
// chunks of rows & (stage_flag - 1) rows.
struct TuneCand {
  int strip, rows, rows_upd;
};

// CTAs of a candidate's launches on an ni x nj mesh: the smaller grid of the pair (total =
// false) or the sum of its grids (total = true); a single-pass kernel has one grid.
inline long tune_ctas(const TuneCand &c, int ni, int nj, int tile_x, int stage_flag, bool total) {
  if (c.strip == 0) {
    const long nx = (ni + tile_x - 1) / tile_x, ru = c.rows_upd ? c.rows_upd : c.rows;
    const long gf = nx * ((nj + c.rows - 1) / c.rows), gu = nx * ((nj + ru - 1) / ru);
    return total ? gf + gu : std::min(gf, gu);
  }
  const long ch = c.rows & (stage_flag - 1);
  return (long)((ni + c.strip - 1) / c.strip) * ((nj + ch - 1) / ch);
}

// The candidates the autotuner times: the kernel pair at 4, 8, 16 and 32 flux rows (with
// derivative rows 4, 8 or 16 for some), the marching kernel (strip march_w) at chunks of 8-128
// rows, cp.async- or (chunks of 16-128) TMA-staged, and the column-marching kernels (strips
// col128 and col256) at chunks of 32-256 rows.
inline std::vector<TuneCand> tune_candidates(int march_w, int col128, int col256, int stage_flag) {
  return {{0, 4, 0},         {0, 8, 0},          {0, 8, 4},
          {0, 16, 0},        {0, 16, 8},         {0, 16, 4},
          {0, 32, 0},        {0, 32, 16},        {march_w, 8, 0},
          {march_w, 16, 0},  {march_w, 32, 0},   {march_w, 64, 0},
          {march_w, 128, 0}, {march_w, 16 | stage_flag, 0},  {march_w, 32 | stage_flag, 0},
          {march_w, 64 | stage_flag, 0},         {march_w, 128 | stage_flag, 0},
          {col128, 32, 0},   {col128, 64, 0},    {col128, 128, 0},
          {col256, 64, 0},   {col256, 128, 0},   {col256, 256, 0}};
}

struct TuneMesh {
  int ni, nj;
  bool viscous;
  int tile_x, stage_flag, march_w;
};

// A candidate the mesh can run at all: pair tiles no taller than the mesh, marching chunks no
// taller than twice the mesh, column-marching CTAs no wider than the mesh.
inline bool tune_usable(const TuneCand &c, const TuneMesh &m) {
  if (c.strip == 0 && c.rows > m.nj) return false;
  if (c.strip > 0 && (c.rows & (m.stage_flag - 1)) > 2 * m.nj) return false;
  if (c.strip > m.march_w && m.ni < c.strip + 12) return false;
  return true;
}

// The candidates one use times (indices into cands). A fast mesh's fused step (critical: its
// micro steps follow one another on the critical path while the slow right-hand side runs
// beside them) takes only shapes whose launches give every SM a CTA (or the most CTAs any
// shape gives) and, for Navier-Stokes, flux tiles of at least 8 rows (a 4-row tile loads its
// two 3-row halos of primitives for every 4 rows) when a pair of 8 rows or more fits the mesh.
inline std::vector<int> tune_eligible(const TuneCand *cands, int n, const TuneMesh &m, bool critical,
                                      int n_sm) {
  bool tall_pair = false;
  for (int i = 0; i < n; ++i)
    tall_pair = tall_pair || (cands[i].strip == 0 && cands[i].rows >= 8 && tune_usable(cands[i], m));
  const bool floor8 = critical && m.viscous && tall_pair;
  auto allowed = [&](const TuneCand &c) {
    return tune_usable(c, m) && !(floor8 && c.strip == 0 && c.rows < 8);
  };
  long min_ctas = 0;
  if (critical) {
    long most = 0;
    for (int i = 0; i < n; ++i)
      if (allowed(cands[i]))
        most = std::max(most, tune_ctas(cands[i], m.ni, m.nj, m.tile_x, m.stage_flag, false));
    min_ctas = std::min((long)n_sm, most);
  }
  std::vector<int> out;
  for (int i = 0; i < n; ++i)
    if (allowed(cands[i]) && tune_ctas(cands[i], m.ni, m.nj, m.tile_x, m.stage_flag, false) >= min_ctas)
      out.push_back(i);
  return out;
}

// The kept candidate of the timed ones ((time, index into cands) pairs; -1 if none): the
// fastest (the first of equal times), and for a critical use, of the candidates within 3 % of
// the fastest, the one with the most CTAs over its launches. Timed alone, shapes of fewer,
// larger CTAs can win by a few percent and then lose in the macro step, where the slow mesh's
// CTAs share the SMs.
inline int tune_pick(const TuneCand *cands, const std::vector<std::pair<float, int>> &timed, const TuneMesh &m,
                     bool critical) {
  int best = -1;
  float best_ms = 0.f;
  for (const auto &t : timed)
    if (best < 0 || t.first < best_ms) {
      best = t.second;
      best_ms = t.first;
    }
  if (best < 0 || !critical) return best;
  long most = tune_ctas(cands[best], m.ni, m.nj, m.tile_x, m.stage_flag, true);
  for (const auto &t : timed) {
    const long c = tune_ctas(cands[t.second], m.ni, m.nj, m.tile_x, m.stage_flag, true);
    if (t.first <= 1.03f * best_ms && c > most) {
      most = c;
      best = t.second;
    }
  }
  return best;
}

}  // namespace sbp
