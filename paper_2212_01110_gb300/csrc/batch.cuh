// Batched SPOCK: one launch per kernel type covers every instance of a
// batch.  Each instance keeps its own problem view, iterate buffers and
// SuperMann state; a block finds its instance, and its block index within
// that instance, in the launch's block map (built once per batch on the
// host), then runs the same body as the single-problem kernel.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "supermann.cuh"

namespace spock {

// One instance as the batched kernels see it.  kp.skip points at st->done,
// so every kernel of a finished instance returns at once.
template <typename S>
struct BInst {
  KP<S> kp;
  SmState* st;
  S* V;     // accepted iterate and T of it
  S* TV;
  S* Vt;    // evaluation point and T of it
  S* TVt;
  S* d;     // direction
  S* MR;    // Anderson columns (stride ld)
  S* D;
  double* stats;   // [8] statistics of the last evaluation
  double* pd;      // partial statistics of the dual kernel, nb_node rows
  double* paa;     // partial Gram rows of the commit kernel, nb_vec rows
  int64_t n_v, ld;
  int32_t nb_node, nb_vec;
};

// Block -> instance map of one batched launch: block b runs for instance
// inst[b] as its block b - base[inst[b]] of cnt[inst[b]]; stage[i] is the
// instance's tree stage for the stage-by-stage Riccati launches.
struct BMap {
  const int32_t* inst;
  const int32_t* base;
  const int32_t* cnt;
  const int32_t* stage;
};

// ops.cu: which = 0 prox-f preparation (L* eta, proj_S2), 1 dual update with
// the dual and primal statistics (warp per nonleaf node), 3 reduction of the
// statistics (one block per instance; m unused).  J = lane slots for blocks
// of nx + nu + 2.
template <typename S>
void launch_node_ops_b(int which, const BInst<S>* bi, const BMap& m, int nblocks, int n_inst, int J,
                       cudaStream_t st);
// riccati.cu: which = 0 backward chains, 1 backward stage, 2 forward stage,
// 3 forward chains (direct kernels, warp per chain / node); SL = lane slots
// for nx + nu.
template <typename S>
void launch_riccati_b(int which, const BInst<S>* bi, const BMap& m, int nblocks, int SL, cudaStream_t st);
// riccati_tma.cu: the same passes with the staged (bulk-copy) kernels: chain
// blocks of wpb warps, one block per node for the stages.
struct TmaBatchShape {
  uint32_t slot_bwd = 0, slot_fwd = 0;   // bytes of shared memory per chain warp
  int wpb_bwd = 1, wpb_fwd = 1;          // warps per chain block
  int nw_stage_bwd = 1, nw_stage_fwd = 1;  // warps per stage block
  uint32_t smem_stage_bwd = 0, smem_stage_fwd = 0;
};
template <typename S>
bool tma_batch_shape(const std::vector<KP<S>>& kps, int max_children, TmaBatchShape& sh);
template <typename S>
void launch_riccati_tma_b(int which, const BInst<S>* bi, const BMap& m, int nblocks, int SL, const TmaBatchShape& sh,
                          cudaStream_t st);
// cta.cu: whole solves, one 128-thread block per instance (instances with
// nx + nu <= max_nxu <= 62, Anderson memory 0, 3 or 5), at most max_rounds
// rounds each; trace (or NULL) for a single instance.
bool cta_supported(int nx, int nu, int mem);
template <typename S>
void launch_solve_cta(const BInst<S>* bi, int n_inst, int max_nxu, int mem, int64_t max_rounds, int32_t* trace,
                      cudaStream_t st);
// rounds.cu: the four kernels of a round.
template <typename S>
void launch_round_decide_b(const BInst<S>* bi, int n_inst, cudaStream_t st);
template <typename S>
void launch_round_commit_b(const BInst<S>* bi, const BMap& m, int nblocks, int mem, cudaStream_t st);
template <typename S>
void launch_round_aa_solve_b(const BInst<S>* bi, int n_inst, cudaStream_t st);
template <typename S>
void launch_round_point_b(const BInst<S>* bi, const BMap& m, int nblocks, int mem, cudaStream_t st);

}  // namespace spock
