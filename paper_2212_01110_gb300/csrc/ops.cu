// Warp-per-node vector kernels of the CP operator T:
//   k_lstar  L* applied to eta (or to r_eta = eta - eta+), in three uses:
//            LS_PREP   zbar = z - alpha L* eta; s^0 - alpha; proj_S2 on z_2;
//                      the (x, u) part goes to the Riccati scratch (prox of
//                      f, Sec. "Proximal operator of f", Sec. "Projection on
//                      S2");
//            LS_APPLY  z_out = L* eta (operator-level ABI).
//   k_dual_fused  eta+ = prox_{alpha g*}(eta + alpha L (2 z+ - z)) with the
//            cone projections of Eq. (S3-def) and every residual statistic of
//            Sec. "The Chambolle-Pock method" / Algorithm 3 in one pass.
//   k_dual   the same update without statistics, L z, and prox_{alpha g*}(eta)
//            alone for the operator-level ABI.
// L and its adjoint are never stored: each entry of eta = L z is a sum over
// the node's own variables and its ancestor's (definition of L).
//
// Memory-level parallelism: a lane owns entries e = lane + 32 j, j < J, of
// the node's blocks (J = ceil((nx + nu + 2) / 32), a template parameter), so
// every load of a node is a predicated straight-line load into registers,
// issued before any arithmetic; the node descriptor of the next node is
// fetched (one word per lane) while the current one is processed.  Cone
// norms are warp-shuffle reductions over registers: no shared memory and no
// warp barriers inside the node loop.
#include "batch.cuh"
#include "kernels.cuh"
#include "ops_body.cuh"
#include "spock_internal.h"

namespace spock {

template <typename S, int MODE, int J>
__global__ void __launch_bounds__(128) k_lstar(KP<S> p, const S* __restrict__ eta, const S* __restrict__ z,
                                               S* __restrict__ zo) {
  lstar_body<S, MODE, J>(p, blockIdx.x, gridDim.x, eta, z, zo);
}

template <typename S, int MODE, int J>
__global__ void __launch_bounds__(128) k_dual(KP<S> p, const S* __restrict__ z, const S* __restrict__ zp,
                                              const S* __restrict__ eta, S* __restrict__ out) {
  dual_body<S, MODE, J>(p, blockIdx.x, gridDim.x, z, zp, eta, out);
}

// FP32: at most 128 registers, four resident blocks per SM (16 warps) for
// this latency-bound kernel; FP64 keeps its registers (FP64-pipe bound).
template <typename S, bool DIR, int J>
__global__ void __launch_bounds__(128, sizeof(S) == 4 ? 4 : 1)
    k_dual_fused(KP<S> p, const S* __restrict__ z, const S* __restrict__ zp,
                                                    const S* __restrict__ eta, S* __restrict__ out,
                                                    const S* __restrict__ dir, double* __restrict__ partials) {
  dual_fused_body<S, DIR, J>(p, blockIdx.x, gridDim.x, z, zp, eta, out, dir, partials);
}

__global__ void k_reduce_stats(const double* __restrict__ pd, int nd, const double* __restrict__ pp, int np,
                               double* __restrict__ out, const int32_t* __restrict__ skip) {
  reduce_stats_body(pd, nd, pp, np, out, skip);
}

// ---------------------------------------------------------------------------
// batched kernels: every block looks its instance up in the launch's block
// map and runs the single-problem body on that instance's buffers (the T
// evaluation of a round: Vt -> TVt, with the direction d for the
// line-search statistics)
// ---------------------------------------------------------------------------
template <typename S, int J>
__global__ void __launch_bounds__(128) k_prep_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const BInst<S>& b = bi[i];
  const KP<S> p = b.kp;
  lstar_body<S, LS_PREP, J>(p, blockIdx.x - m.base[i], m.cnt[i], b.Vt + p.n_z, b.Vt, b.TVt);
}

template <typename S, int J>
__global__ void __launch_bounds__(128) k_dual_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const BInst<S>& b = bi[i];
  const KP<S> p = b.kp;
  dual_fused_body<S, true, J>(p, blockIdx.x - m.base[i], m.cnt[i], b.Vt, b.TVt, b.Vt + p.n_z, b.TVt + p.n_z,
                              b.d, b.pd);
}

template <typename S>
__global__ void k_reduce_stats_b(const BInst<S>* __restrict__ bi) {
  const BInst<S>& b = bi[blockIdx.x];
  reduce_stats_body(b.pd, b.nb_node, nullptr, 0, b.stats, b.kp.skip);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
inline int warp_grid(int n, int max_blocks) {
  int b = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return b < max_blocks ? (b > 0 ? b : 1) : max_blocks;
}

// entries per lane for blocks of nx + nu + 2 entries
inline int lane_slots(int nx, int nu) { return (nx + nu + 2 + 31) / 32; }

template <typename S, int MODE>
static void lstar_j(const KP<S>& p, const S* eta, const S* z, S* zo, int grid, cudaStream_t st) {
  switch (lane_slots(p.nx, p.nu)) {
    case 1: k_lstar<S, MODE, 1><<<grid, 128, 0, st>>>(p, eta, z, zo); break;
    case 2: k_lstar<S, MODE, 2><<<grid, 128, 0, st>>>(p, eta, z, zo); break;
    case 3: k_lstar<S, MODE, 3><<<grid, 128, 0, st>>>(p, eta, z, zo); break;
    case 4: k_lstar<S, MODE, 4><<<grid, 128, 0, st>>>(p, eta, z, zo); break;
    default: k_lstar<S, MODE, kMaxJ><<<grid, 128, 0, st>>>(p, eta, z, zo); break;
  }
}

template <typename S, int MODE>
static void dual_j(const KP<S>& p, const S* z, const S* zp, const S* eta, S* out, int grid, cudaStream_t st) {
  switch (lane_slots(p.nx, p.nu)) {
    case 1: k_dual<S, MODE, 1><<<grid, 128, 0, st>>>(p, z, zp, eta, out); break;
    case 2: k_dual<S, MODE, 2><<<grid, 128, 0, st>>>(p, z, zp, eta, out); break;
    case 3: k_dual<S, MODE, 3><<<grid, 128, 0, st>>>(p, z, zp, eta, out); break;
    case 4: k_dual<S, MODE, 4><<<grid, 128, 0, st>>>(p, z, zp, eta, out); break;
    default: k_dual<S, MODE, kMaxJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out); break;
  }
}

// the general form's kernels (ops_gen.cu)
template <typename S>
void launch_lstar_gen(const KP<S>& p, int mode, const S* eta, const S* z, S* zo, int grid, cudaStream_t st);
template <typename S>
void launch_dual_gen(const KP<S>& p, int mode, bool stats, const S* z, const S* zp, const S* eta, S* out,
                     const S* dir, double* partials, int grid, cudaStream_t st);

template <typename S>
void launch_prep(const KP<S>& p, const S* z, const S* eta, S* zo, int max_blocks, cudaStream_t st) {
  if (p.gen) {
    launch_lstar_gen<S>(p, LS_PREP, eta, z, zo, warp_grid(p.n, max_blocks), st);
    return;
  }
  lstar_j<S, LS_PREP>(p, eta, z, zo, warp_grid(p.n, max_blocks), st);
}

template <typename S>
void launch_dual(const KP<S>& p, int mode, bool stats, const S* z, const S* zp, const S* eta, S* out,
                 const S* dir, double* partials, int grid, cudaStream_t st) {
  if (p.gen) {
    launch_dual_gen<S>(p, mode, stats, z, zp, eta, out, dir, partials, grid, st);
    return;
  }
  // operator-level modes (not on the solve path) use the widest lane layout
  if (mode == DM_APPLY_L) {
    k_dual<S, DM_APPLY_L, kMaxJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out);
  } else if (mode == DM_PROXG) {
    k_dual<S, DM_PROXG, kMaxJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out);
  } else if (!stats) {
    dual_j<S, DM_DUAL>(p, z, zp, eta, out, grid, st);
  } else {
    // with statistics: the fused kernel (warp per nonleaf node), which also
    // accumulates the primal statistics
    switch (lane_slots(p.nx, p.nu)) {
#define SPOCK_DF(JJ)                                                                                     \
  case JJ:                                                                                               \
    if (dir) k_dual_fused<S, true, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);         \
    else k_dual_fused<S, false, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);            \
    break;
      SPOCK_DF(1) SPOCK_DF(2) SPOCK_DF(3) SPOCK_DF(4)
      default: SPOCK_DF(kMaxJ)
#undef SPOCK_DF
    }
  }
}

// z_out = L* eta
template <typename S>
void launch_lstar(const KP<S>& p, const S* eta, S* zout, int grid, cudaStream_t st) {
  if (p.gen) {
    launch_lstar_gen<S>(p, LS_APPLY, eta, nullptr, zout, grid, st);
    return;
  }
  k_lstar<S, LS_APPLY, kMaxJ><<<grid, 128, 0, st>>>(p, eta, nullptr, zout);
}

void launch_reduce_stats(const double* pd, int nd, const double* pp, int np, double* out, cudaStream_t st,
                         const int32_t* skip) {
  k_reduce_stats<<<1, 256, 0, st>>>(pd, nd, pp, np, out, skip);
}

template <typename S>
void launch_node_ops_b(int which, const BInst<S>* bi, const BMap& m, int nblocks, int n_inst, int J,
                       cudaStream_t st) {
  if (which == 3) {
    k_reduce_stats_b<S><<<n_inst, 256, 0, st>>>(bi);
    return;
  }
#define SPOCK_NB(JJ)                                                              \
  case JJ:                                                                        \
    if (which == 0) k_prep_b<S, JJ><<<nblocks, 128, 0, st>>>(bi, m);              \
    else k_dual_b<S, JJ><<<nblocks, 128, 0, st>>>(bi, m);                         \
    break;
  switch (J) {
    SPOCK_NB(1) SPOCK_NB(2) SPOCK_NB(3) SPOCK_NB(4)
    default: SPOCK_NB(kMaxJ)
  }
#undef SPOCK_NB
}
template void launch_node_ops_b<double>(int, const BInst<double>*, const BMap&, int, int, int, cudaStream_t);
template void launch_node_ops_b<float>(int, const BInst<float>*, const BMap&, int, int, int, cudaStream_t);

template void launch_prep<double>(const KP<double>&, const double*, const double*, double*, int, cudaStream_t);
template void launch_prep<float>(const KP<float>&, const float*, const float*, float*, int, cudaStream_t);
template void launch_dual<double>(const KP<double>&, int, bool, const double*, const double*, const double*,
                                  double*, const double*, double*, int, cudaStream_t);
template void launch_dual<float>(const KP<float>&, int, bool, const float*, const float*, const float*, float*,
                                 const float*, double*, int, cudaStream_t);
template void launch_lstar<double>(const KP<double>&, const double*, double*, int, cudaStream_t);
template void launch_lstar<float>(const KP<float>&, const float*, float*, int, cudaStream_t);

}  // namespace spock
