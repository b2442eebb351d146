// Internal declarations shared by the host setup and the CUDA solver.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/kfbim.h"

namespace kfbim {

// Number of jump values kept per control point (slot order):
//   0 [u^(c)], 1..3 [d_x u^(c)], [d_y u^(c)], [d_z u^(c)],
//   4..9 [Hess u^(c)] entries 11, 22, 33, 23, 13, 12, 10 [p], 11 [d_a p].
constexpr int kSlots = 12;
// Inputs of the per-point jump map: 5 fitted surface derivatives
// (d_1, d_2, d_11, d_12, d_22) of each density component, then f (3).
constexpr int kMapIn = 18;
// Outputs of the jump map: slots 1..11 (slot 0 is the density value itself).
constexpr int kMapOut = 11;
// Weights per fit neighbour: value, d_1, d_2, d_11, d_12, d_22.
constexpr int kFitW = 6;
constexpr int kStencil = 10;

struct HostTables {
  int N = 0;
  double lo = 0, h = 0, mu = 1;
  int64_t n_all = 0, n_prim = 0;
  // control points (canonical order)
  std::vector<int32_t> comp, axis, primary, pid;   // pid: primary index or -1
  std::vector<int32_t> idx;                        // 3 per point: lower node (i,j,k)
  std::vector<double> theta, xyz;                  // xyz: 3 per point
  std::vector<double> normal;                      // 3 per point: outward unit normal
  // 0, or 1 / 2 for the root below / above the cell centre of a grazing face
  // segment (both face nodes on one side, the cell centre between them on the
  // other; combined u^(c)/cell lines only)
  std::vector<int8_t> graze;
  std::vector<uint8_t> side[4];                    // N^3 per grid (0 cells, 1..3 faces)
  // surface fits: CSR over rows y*3 + c'; columns are primary indices
  std::vector<int64_t> fit_ptr;
  std::vector<int32_t> fit_col;
  std::vector<double> fit_w;                       // kFitW per entry
  // jump map: kMapOut x kMapIn per point (row-major)
  std::vector<double> jmap;
  // corrections: CSR over target rows of the RHS vector [f1 | f2 | f3 | g]
  std::vector<int64_t> corr_row;                   // target index in [0, 4 N^3)
  std::vector<int64_t> corr_ptr;
  std::vector<int64_t> corr_src;                   // slot * n_all + point
  std::vector<double> corr_coef;
  // trace interpolation, per primary point
  std::vector<int32_t> tr_comp;
  std::vector<int32_t> tr_node;                    // kStencil flat node indices
  std::vector<double> tr_w, tr_cj;                 // kStencil each
};

// Alg. 1 step 1 and every table of the matvec.  lam < 0: Stokes; otherwise
// the Navier (Lame) jump relations with Lame lambda.  Returns a kfbim_status.
int build_tables(const kfbim_geometry& geom, const kfbim_grid& grid, double mu, double lam,
                 HostTables& t, std::string& err);

}  // namespace kfbim
