// Internal types shared by the host setup, the C ABI and the CUDA kernels of the library.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "sbp_mrab.h"

namespace sbp {

constexpr int kMaxHist = 6;   // longest Adams-Bashforth history supported (AB46)
constexpr int kNvar = 4;      // 2D conserved variables

// Stencil class of a point along one direction, 4 bits: kind in bits 2-3, closure row in
// bits 0-1. Interior: 5-point central row; left/right: closure row r counted from the
// segment's low/high end; hole: inactive.
enum : uint8_t { kInterior = 0, kLeft = 1, kRight = 2, kHole = 3 };
inline uint8_t cls_code(int kind, int row) { return (uint8_t)((kind << 2) | row); }

// SAT term kinds (physical and interface boundaries).
enum : int { kTermInterface = 1, kTermFarfield = 2, kTermWall = 3 };

// Tile of the fused right-hand-side kernels (points per CTA along i and j).
struct TileShape {
  int tx, ty;
};

// Host-side products of the setup of one mesh.
struct MeshHost {
  int ni = 0, nj = 0, pitch = 0;
  int per[2] = {0, 0};
  int bc[4] = {0, 0, 0, 0};
  int cartesian = 0;
  double lo[2] = {0, 0}, h[2] = {0, 0};
  double shift[4] = {0, 0, 0, 0};
  std::vector<double> x, y;          // nj*ni, i fastest
  std::vector<int8_t> active;        // nj*ni
  std::vector<uint8_t> cls;          // nj*ni: (class_j << 4) | class_i
  // SAT points: one entry per point with at least one term; terms packed 4 bits each
  // (bit 0 direction, bit 1 side (0 = low face "+", 1 = high face "-"), bits 2-3 kind),
  // count in bits 0-2 and terms from bit 3 upward.
  std::vector<int> sat_pt;           // j*ni+i
  std::vector<uint32_t> sat_code;
  std::vector<int> sat_recv;         // receiver index or -1
  std::vector<double> sat_scale;     // Omega for corner interface points, else 1
  // receivers of this mesh (sorted by point) and their donors on the other mesh
  std::vector<int> recv_pt;
  std::vector<int> donor_base;       // 2 per receiver
  std::vector<double> donor_w;       // 8 per receiver
  // the distinct donor points of all receivers (i | j << 16 on the other mesh, sorted) and,
  // per receiver, the index of each of its 16 stencil points (b * 4 + a) in that list
  std::vector<uint32_t> donor_pts;
  std::vector<int> donor_idx;
};

// Adams-Bashforth / MRAB coefficient plan (Sec. 3.1-3.3), weights oldest first, in units of
// the step (multiply by h or H).
struct CoeffPlan {
  int order = 3, m = 3, sr = 1;
  std::vector<double> ab;                 // m: one step over [0, 1] on the nodes -(m-1)..0
  std::vector<std::vector<double>> ext;   // sr entries: slow extrapolant integrated over [0, j/sr]
  // slowest-first variants: the fast extrapolant integrated over a whole macro step [0, sr]
  // (units of the micro step), and the slow polynomial through the history ending one macro
  // step later (nodes -(m-2)..1) integrated over [0, j/sr] (re-extrapolation)
  std::vector<double> fext;
  std::vector<std::vector<double>> rext;
};

// Host setup (sbp_setup.cpp).
sbp_status setup_mesh_basic(const sbp_mesh_desc &d, MeshHost &m, std::string &err);
sbp_status setup_holes(MeshHost &bg, const MeshHost &fine, double margin, std::string &err);
sbp_status setup_classes(MeshHost &m, std::string &err);
sbp_status setup_sat(MeshHost &m, double omega_corner, std::string &err);
sbp_status setup_donors(MeshHost &recv, const MeshHost &donor, std::string &err);
sbp_status solve_ab_weights(const std::vector<double> &nodes, double a, double b, int order,
                            std::vector<double> &alpha);
sbp_status build_plan(int order, int m, int sr, CoeffPlan &plan, std::string &err);
// Maximal runs of active points (a[off + st * k] != 0) on a line of n points: (start, length).
std::vector<std::pair<int, int>> active_runs(const std::vector<int8_t> &a, size_t off, size_t st, int n, bool per);

// ---------------------------------------------------------------------------------------------
// 3D Cartesian meshes (sbp3_setup.cpp). Points (i, j, k) have the linear index
// (k * nj + j) * ni + i on the host; class codes are 4 bits per direction (i, j, k) in a 16-bit
// word, 0xFFF for a hole. SAT codes: term count in bits 0-1, then per term 4 bits from bit 2:
// direction (2 bits), side (1 bit: 0 low face "+", 1 high face "-"), kind (1 bit: 0 interface,
// 1 far field).
constexpr int kNvar3 = 5;
struct Mesh3Host {
  int n[3] = {0, 0, 0}, pitch = 0;
  int per[3] = {0, 0, 0};
  int bc[6] = {0, 0, 0, 0, 0, 0};
  double lo[3] = {0, 0, 0}, h[3] = {0, 0, 0};
  std::vector<int8_t> active;
  std::vector<uint16_t> cls;
  std::vector<int64_t> sat_pt;
  std::vector<uint32_t> sat_code;
  std::vector<int> sat_recv;
  std::vector<double> sat_scale;
  std::vector<int64_t> recv_pt;
  std::vector<int> donor_base;       // 3 per receiver
  std::vector<double> donor_w;       // 12 per receiver (i, j, k)
  std::vector<int64_t> donor_pts;    // distinct donor points (linear index on the donor mesh)
  std::vector<int> donor_idx;        // 64 per receiver: (c * 4 + b) * 4 + a -> index in donor_pts
  size_t points() const { return (size_t)n[0] * n[1] * n[2]; }
};
sbp_status setup3_mesh(const sbp3_mesh_desc &d, Mesh3Host &m, std::string &err);
sbp_status setup3_holes(Mesh3Host &bg, const Mesh3Host &fine, double margin, std::string &err);
sbp_status setup3_classes(Mesh3Host &m, std::string &err);
sbp_status setup3_sat(Mesh3Host &m, double omega_corner, std::string &err);
sbp_status setup3_donors(Mesh3Host &rm, const Mesh3Host &d, std::string &err);

}  // namespace sbp
