// Internal data structures of libspock (not part of the ABI).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/spock.h"

namespace spock {

enum : int32_t { TAG_TREE = 0x54524545, TAG_PROBLEM = 0x50524f42, TAG_BATCH = 0x42415443 };

// Maximum Anderson memory and per-node dimension handled by the kernels.
constexpr int kMaxMemory = 16;
constexpr int kMaxDim = 128;   // nx + nu
constexpr int kNumStats = 8;   // residual statistics, see kernels.cuh

struct Error {
  int code;
  std::string msg;
};

void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

// Scenario tree in the caller's numbering plus a breadth-first ("internal")
// renumbering: nodes of a stage are contiguous, children of a node are
// contiguous and in increasing user id, so the nonleaf nodes are the
// internal ids [0, n_nonleaf) and the nonroot nodes [1, n).
struct Tree {
  int32_t tag = TAG_TREE;
  int32_t n = 0, N = 0, n_nonleaf = 0, n_leaf = 0;
  std::vector<int32_t> anc_user;
  std::vector<double> prob_user;
  std::vector<int32_t> user_of, int_of;        // internal -> user, user -> internal
  std::vector<int32_t> parent, ch_begin, ch_count, stage, sib;  // internal
  std::vector<int32_t> stage_begin;            // [N + 2]
  std::vector<int32_t> stage_maxch;            // [N + 1] most children of a node at each stage
  std::vector<double> prob;                    // internal, conditional
  // chain region: every node at stages >= chain_stage (and < N) has one child
  int32_t chain_stage = 0;
};

// Offsets of every node's blocks inside the user-layout z and eta vectors
// (documented in spock.h), indexed by internal id; -1 where absent.
struct Offsets {
  int64_t n_z = 0, n_eta = 0;
  std::vector<int64_t> zx, zu, zz2, zs, ztau;   // ztau/zs of nonroot nodes (zs[0] = 0)
  std::vector<int64_t> enl, enr, elf;
};

// Device copy of the problem for one scalar type S.
template <typename S>
struct DevFactors {
  S* Gb = nullptr;   // [n-1][nx][nx+nu]  rows of [Abar^c | B^c], nonroot c
  S* Gf = nullptr;   // [n-1][nx+nu][nx]  transpose of the above
  S* NB = nullptr;   // [nl][K (nu x nx) | K + W^T (nu x nx) | Rtilde^-1 (nu x nu)]
  S* Kt = nullptr;   // [nl][nx][nu]      K^T
  S* qs = nullptr;   // [n][nx]  sqrt(Q) of the edge into the node
  S* rs = nullptr;   // [n][nu]  sqrt(R)
  S* qns = nullptr;  // [n][nx]  sqrt(Q_N) (leaves)
  S* xlo = nullptr; S* xhi = nullptr;   // [n][nx]
  S* ulo = nullptr; S* uhi = nullptr;   // [n][nu]
  S* av = nullptr;   // [n] AV@R parameter
  S* prob = nullptr; // [n] conditional probability
  S* s2inv = nullptr; // [n][2] 1 / c and 1 / (c + m_i), c = a_i^2 + 3 (closed form of proj_S2^i)
  // general form (spock_problem_create_general): per-node matrices of the
  // rows of L, each in two layouts -- column-major (element (r, c) at
  // c * ld + r: a warp's lanes run over rows, M v) and transposed (element
  // (r, c) at r * ldT + c: lanes over columns, M^T w)
  S* gc = nullptr;  S* gt = nullptr;    // Gamma^k = [Gx | Gu] (nonleaf): [n][nx+nu][ldc], [n][nc][ldxu]
  S* fqc = nullptr; S* fqt = nullptr;   // Q^k 1/2 (edge into k):  [n][nx][ldx] both
  S* frc = nullptr; S* frt = nullptr;   // R^k 1/2:                [n][nu][ldu] both
  S* fnc = nullptr; S* fnt = nullptr;   // Q_N^k 1/2 (leaves):     [n][nx][ldx] both
  S* gnc = nullptr; S* gnt = nullptr;   // Gamma_N^k (leaves):     [n][nx][ldcn], [n][ncN][ldx]
  S* clo = nullptr; S* chi = nullptr;   // [n][cst] bounds of C^k (nc rows) or C_N^k (ncN rows)
  // risk measures of the general form: per nonleaf node b^k (ny_k entries
  // at rboff[k]) and the projector on S2^k (nz2 x nz2 column-major,
  // nz2 = ny_k + 2 m_k, at rpoff[k])
  S* rb = nullptr;
  S* rpi = nullptr;
  // scratch of the Riccati passes
  S* xbar = nullptr;  // [n][nx]
  S* ubar = nullptr;  // [nl][nu]
  S* q = nullptr;     // [n][nx]
  S* d = nullptr;     // [nl][nu]
  S* x0 = nullptr;    // [nx]
  // per-node strides in elements, padded to a multiple of 16 bytes
  int32_t xs = 0, us = 0, gstride = 0, nbstride = 0, ktstride = 0;
};

struct DevIndex {
  int32_t* parent = nullptr;
  int32_t* ch_begin = nullptr;
  int32_t* ch_count = nullptr;
  int32_t* sib = nullptr;
  int64_t *zx = nullptr, *zu = nullptr, *zz2 = nullptr, *zs = nullptr, *ztau = nullptr;
  int64_t *enl = nullptr, *enr = nullptr, *elf = nullptr;
  int32_t* stage_begin = nullptr;  // [N + 2]
  struct NodeDesc* desc = nullptr; // [n] per-node record (kernels.cuh)
  // general form: rows of y^k, orthant rows of K^k, offsets of b^k and of
  // the S2 projector (nonleaf nodes)
  int32_t *rny = nullptr, *rkp = nullptr;
  int64_t *rboff = nullptr, *rpoff = nullptr;
};

// Padded leading dimensions of the general form's matrices (elements).
struct GenDims {
  int32_t nc = 0, ncN = 0;                  // constraint rows per nonleaf / leaf node
  int32_t ldc = 0, ldxu = 0, ldx = 0, ldu = 0, ldcn = 0, cst = 0;
  int32_t max_nz2 = 0;                      // largest z_2 block (ny + 2 m) of a node
};

struct Problem {
  int32_t tag = TAG_PROBLEM;
  int device = 0;
  Tree tree;
  Offsets off;
  int32_t nx = 0, nu = 0;
  bool general = false;   // general form: the L kernels are the matrix-row ones
  GenDims gd;
  double normL = 0.0;
  double factor_seconds = 0.0;
  DevIndex idx;
  int32_t* err = nullptr;  // device flag set by a kernel whose bounded wait gave up
  DevFactors<double> f64;
  DevFactors<float> f32;
  std::vector<void*> allocations;
  // device staging buffers of the host-buffer entry points
  double* io_x0 = nullptr;
  double* io_z = nullptr;
  double* io_eta = nullptr;
  double* io_grad = nullptr;   // outputs of spock_grad (host-buffer variant)
  double* adj = nullptr;       // vectors of the adjoint solve (spock_adjoint_dev)
  int32_t adj_restart = 0;     // its GMRES restart length, fixed at the first call
  double* adj_pinned = nullptr;  // pinned host copy of a GMRES step's coefficients
  // solver workspace, allocated on first use per precision
  struct Workspace* ws64 = nullptr;
  struct Workspace* ws32 = nullptr;
  // clones (spock_problem_clone) share this problem's data, factors and
  // index arrays; a base freed while clones exist is deleted with its last clone
  struct Problem* base = nullptr;
  int32_t n_clones = 0;
  bool free_pending = false;
  ~Problem();
};

// host-side helpers (tree.cpp, factor.cpp)
int build_tree(int32_t n, const int32_t* anc, const double* prob, Tree& t);
// nc / ncN: constraint rows of the nonleaf / leaf blocks of eta (box form:
// nx + nu and nx); ny_user: rows of y per node in the caller's numbering
// (nullptr: AV@R's 2 m + 1).
void build_offsets(const Tree& t, int nx, int nu, int nc, int ncN, const std::vector<int32_t>* ny_user,
                   Offsets& o);

// Offline factorisation of the projection on S1 (Algorithm 1), FP64.
// Inputs in internal numbering: A [n][nx][nx], B [n][nx][nu].
// Outputs (internal numbering):
//   Gb  [n-1][nx][nx+nu]  [Abar^c | B^c]     (c = 1..n-1)
//   NB  [nl][K | K + W^T | Rtilde^-1]
// Returns false if some Rtilde is numerically singular (cannot happen for
// finite data since Rtilde >= I).
bool riccati_factor(const Tree& t, int nx, int nu, const std::vector<double>& A,
                    const std::vector<double>& B, std::vector<double>& Gb,
                    std::vector<double>& NB, int threads);

}  // namespace spock
