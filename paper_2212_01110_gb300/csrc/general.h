// Host side of the general form (general.cpp).
#pragma once

#include <string>
#include <vector>

#include "spock_internal.h"

namespace spock {

// The general form's per-node matrices in internal node order, FP64, in the
// device layouts of DevFactors (column-major and transposed, padded leading
// dimensions in d), and the largest squared norm of the (x, u) / x column
// blocks of L.
struct GenHost {
  GenDims d;
  std::vector<double> gc, gt, fqc, fqt, frc, frt, fnc, fnt, gnc, gnt, clo, chi;
  double normL2_xu = 0.0;
  // risk measures (internal order): b^k and S2 projectors, flat, with their
  // offsets; rows of y^k and orthant rows of K^k; rows of y per user node
  std::vector<double> rb, rpi;
  std::vector<int64_t> rboff, rpoff;
  std::vector<int32_t> rny, rkp, ny_user;
  double normL2_ys = 0.0;   // largest squared norm of the (y, s) blocks
};

// Largest z_2 block (ny + 2 m) the general kernels hold in registers.
constexpr int kMaxZ2 = 160;

// Builds GenHost from user-order inputs (see spock_problem_create_general):
// dense (Q, R, QN full matrices) or diagonal costs, constraint matrices and
// bounds, risk measures (risk == nullptr: AV@R with parameter a).  Returns
// SPOCK_OK, or an error code with a message in err.
int build_general(const Tree& t, int nx, int nu, bool dense, const double* Q, const double* R, const double* QN,
                  const double* a, const spock_risk* risk, int nc, const double* Gx, const double* Gu,
                  const double* cmin, const double* cmax, int ncN, const double* GN, const double* cNmin,
                  const double* cNmax, int threads, GenHost& o, std::string& err);

}  // namespace spock
