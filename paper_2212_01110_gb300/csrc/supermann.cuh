// Device-resident state of Algorithm 3 (SPOCK) and the launchers of its
// scalar and vector kernels (supermann.cu).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "spock_internal.h"

namespace spock {

enum SmAction : int32_t {
  A_NONE = 0, A_DONE = 1, A_MAXIT = 2, A_K0 = 3, A_LS = 4,
  A_K1 = 5, A_K2 = 6, A_CAP = 7, A_RETRY = 8, A_NUMERICAL = 9, A_STALL = 10
};

struct SmState {
  // settings
  double alpha, eps_abs, eps_rel, c0, c1, c2, beta, sigma, lam, rho_coef;
  int32_t max_iter, max_back, mem, record_trace;
  // iteration state
  double zeta, omega_safe, omega, xi, xi0, tol, tau, omega_t, rho, coef;
  int32_t k, nb, action, initialized;
  int32_t n_k0, n_k1, n_k2, n_cap, n_back, pad_;
  // stagnation test (FP32 mode): best xi so far and the iteration it was seen
  double best_xi;
  int32_t best_k, stall_window;
  // Anderson: Gram of the stored M^R columns (slot-indexed), right-hand side,
  // least-squares coefficients
  double G[kMaxMemory * kMaxMemory];
  double rhs[kMaxMemory];
  double gamma[kMaxMemory];
  int32_t aa_dropped;
  // device-driven rounds (rounds.cu): what the last evaluation of T was for,
  // what this round does, and whether the solve has finished
  int32_t pending, op_accept, op_aa, op_point;
  int32_t done, have_prev, aa_cnt, aa_next;
  int32_t aa_slot, n_T, rounds, pad2_;
  double stats_cur[8];
};

// Round-driver codes.
enum SmPending : int32_t { P_INIT = 0, P_K0 = 1, P_LS = 2, P_K2 = 3 };
enum SmPoint : int32_t { PT_NONE = 0, PT_DIR = 1, PT_LS = 2, PT_K2 = 3, PT_KM = 4 };

// One round = decide (from the statistics of the last T evaluation) ->
// commit/Anderson update -> Gram solve -> next evaluation point; the T
// evaluation of that point follows (skipped once done).  Every kernel reads
// its orders from the state, so the sequence can be captured in a graph.
void launch_round_decide(SmState* st, const double* stats_t, int32_t* trace, cudaStream_t s);
template <typename S>
void launch_round_commit(SmState* st, S* V, S* TV, const S* Vt, const S* TVt, S* MR, S* D,
                         int64_t n, int64_t ld, int mem, double* partials, int grid, cudaStream_t s);
void launch_round_aa_solve(SmState* st, const double* partials, int nblocks, cudaStream_t s);
template <typename S>
void launch_round_point(SmState* st, const S* V, const S* TV, S* Vt, const S* TVt, S* d, const S* D, int64_t n,
                        int64_t ld, int mem, int grid, cudaStream_t s);

void sm_init_state(SmState* st_dev, const SmState& host_init, cudaStream_t s);
void launch_sm_after_eval(SmState* st, const double* stats, int32_t* trace, cudaStream_t s);
void launch_sm_line_search(SmState* st, const double* stats, int32_t* trace, cudaStream_t s);

// Anderson update: writes column `slot` of M^R and of D = M^P - M^R from the
// current (v, Tv) and previous (vp, Tvp) iterates, then the Gram row of the
// new column and the right-hand side M^RT r, and solves for gamma (FP64).
// Column j of M^R / D starts at j * ld (ld >= n, 256-byte aligned columns).
template <typename S>
void launch_aa_update(SmState* st, const S* v, const S* Tv, const S* vp, const S* Tvp, S* MR, S* D, int64_t n,
                      int64_t ld, int slot, int cnt, int newest_first_order[kMaxMemory], double* partials, int grid,
                      cudaStream_t s);
// d = -(v - Tv) - sum_j gamma_j D_j over the cnt stored columns; vt = v + d.
template <typename S>
void launch_aa_direction(const SmState* st, const S* v, const S* Tv, const S* D, int64_t n, int64_t ld, int cnt,
                         S* d, S* vt, int grid, cudaStream_t s);
// vt = v + tau d (tau from the state).
template <typename S>
void launch_ls_point(const SmState* st, const S* v, const S* d, S* vt, int64_t n, int grid, cudaStream_t s);
// vn = v - coef (vt - Tvt)   (K2; coef = lambda rho / omega~^2 from the state)
template <typename S>
void launch_k2_point(const SmState* st, const S* v, const S* vt, const S* Tvt, S* vn, int64_t n, int grid,
                     cudaStream_t s);
// vn = v - lambda (v - Tv)   (line search capped: tau = 0)
template <typename S>
void launch_km_point(const SmState* st, const S* v, const S* Tv, S* vn, int64_t n, int grid, cudaStream_t s);

}  // namespace spock
