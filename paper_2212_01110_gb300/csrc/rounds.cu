// Device-driven iteration of Algorithm 3 (SPOCK).
//
// The buffers are fixed: (V, TV) the accepted iterate and T of it, (Vp, TVp)
// the previously accepted one (for the Anderson differences), (Vt, TVt) the
// point being evaluated and T of it, d the direction, the Anderson columns.
// Each round: k_round_decide reads the statistics of the last evaluation and
// the state, takes the SuperMann decision of Algorithm 3 (same readings as
// supermann.cu) and writes this round's orders; k_round_commit copies an
// accepted (Vt, TVt) into (V, TV) -- the old pair into (Vp, TVp) -- and in the
// same pass writes the new Anderson column and its Gram row; k_round_aa_solve
// solves for gamma; k_round_point forms the next evaluation point in Vt
// (v + d with the Anderson direction, v + tau d, the K2 point, or the relaxed
// step); then T(Vt) is evaluated.  No decision is taken on the host, so a
// run of rounds can be captured in a CUDA graph and replayed.
#include <cmath>

#include "batch.cuh"
#include "kernels.cuh"
#include "supermann.cuh"

namespace spock {

__device__ void round_trace(SmState* st, int32_t* trace, int branch, int nb) {
  if (st->record_trace && trace && st->k < st->max_iter) {
    trace[2 * st->k] = branch;
    trace[2 * st->k + 1] = nb;
  }
}

// Decisions after an iterate has been accepted (its statistics in stats_cur).
__device__ void round_after_accept(SmState* st, int32_t* trace) {
  const double* sc = st->stats_cur;
  const double om2 = sc[ST_RZ2] + sc[ST_RE2] - 2.0 * st->alpha * sc[ST_RE_LRZ];
  const double omega = sqrt(fmax(om2, 0.0));
  const double xi = fmax(sc[ST_XIP], sc[ST_XID]);
  if (!st->initialized) {
    st->zeta = omega;
    st->omega_safe = omega;
    st->xi0 = xi;
    if (!(st->tol > 0.0)) st->tol = fmax(st->eps_abs, st->eps_rel * xi);
    st->best_xi = xi;
    st->best_k = 0;
    st->initialized = 1;
  }
  st->omega = omega;
  st->xi = xi;
  if (xi < 0.5 * st->best_xi) {
    st->best_xi = xi;
    st->best_k = st->k;
  }
  st->op_aa = 0;
  st->op_point = PT_NONE;
  int act;
  if (!isfinite(om2) || !isfinite(xi)) act = A_NUMERICAL;
  else if (xi <= st->tol) act = A_DONE;
  else if (st->k >= st->max_iter) act = A_MAXIT;
  else if (st->stall_window > 0 && st->k - st->best_k > st->stall_window && xi <= 30.0 * st->tol) act = A_STALL;
  else act = A_NONE;
  if (act != A_NONE) {
    st->action = act;
    st->done = 1;
    return;
  }
  if (st->have_prev && st->mem > 0) {  // Anderson update with (v, c = r) of this iterate
    st->op_aa = 1;
    st->aa_slot = st->aa_next;
    st->aa_next = (st->aa_next + 1) % st->mem;
    st->aa_cnt = min(st->aa_cnt + 1, st->mem);
  }
  st->have_prev = 1;
  st->op_point = PT_DIR;
  if (omega <= st->c0 * st->zeta) {  // K0: blind step v + d
    st->zeta = omega;
    round_trace(st, trace, 0, 0);
    st->n_k0++;
    st->k++;
    st->pending = P_K0;
    st->action = A_K0;
  } else {
    st->tau = 1.0;
    st->nb = 0;
    st->pending = P_LS;
    st->action = A_LS;
  }
}

__device__ void round_decide_body(SmState* st, const double* __restrict__ stats_t, int32_t* trace) {
  st->op_accept = 0;
  st->op_aa = 0;
  st->op_point = PT_NONE;
  if (st->done) return;
  st->rounds++;
  const int pend = st->pending;
  bool accept = false;
  if (pend == P_INIT || pend == P_K0 || pend == P_K2) {
    accept = true;
  } else {  // P_LS: line-search trial v~ = v + tau d evaluated
    const double om2 = stats_t[ST_RZ2] + stats_t[ST_RE2] - 2.0 * st->alpha * stats_t[ST_RE_LRZ];
    const double omt = sqrt(fmax(om2, 0.0));
    st->omega_t = omt;
    const double omega = st->omega;
    if (!isfinite(om2)) {
      st->action = A_NUMERICAL;
      st->done = 1;
      return;
    }
    if (omega <= st->omega_safe && omt <= st->c1 * omega) {  // K1
      st->omega_safe = omt + pow(st->c2, (double)st->k);
      round_trace(st, trace, 1, st->nb);
      st->n_k1++;
      st->k++;
      accept = true;
    } else {
      const double rdM = stats_t[ST_RD] - st->alpha * (stats_t[ST_LRZ_DE] + stats_t[ST_RE_LDZ]);
      const double rho = om2 - st->rho_coef * st->tau * rdM;
      st->rho = rho;
      if (rho >= st->sigma * omt * omega && omt > 0.0) {  // K2
        st->coef = st->lam * rho / (omt * omt);
        round_trace(st, trace, 2, st->nb);
        st->n_k2++;
        st->k++;
        st->op_point = PT_K2;
        st->pending = P_K2;
        st->action = A_K2;
      } else {
        st->nb++;
        st->n_back++;
        st->tau *= st->beta;
        if (st->nb >= st->max_back) {  // cap: tau = 0, relaxed step v - lambda r
          round_trace(st, trace, 3, st->nb);
          st->n_cap++;
          st->k++;
          st->op_point = PT_KM;
          st->pending = P_K2;
          st->action = A_CAP;
        } else {
          st->op_point = PT_LS;
          st->pending = P_LS;
          st->action = A_RETRY;
        }
      }
    }
  }
  if (accept) {
    st->op_accept = 1;
    for (int i = 0; i < 8; ++i) st->stats_cur[i] = stats_t[i];
    round_after_accept(st, trace);
  }
  if (!st->done) st->n_T++;  // the T evaluation that follows this round
}

__global__ void k_round_decide(SmState* st, const double* __restrict__ stats_t, int32_t* trace) {
  if (threadIdx.x != 0) return;
  round_decide_body(st, stats_t, trace);
}

template <typename S>
struct RPack;
template <>
struct RPack<float> {
  using T = float4;
  static constexpr int N = 4;
};
template <>
struct RPack<double> {
  using T = double2;
  static constexpr int N = 2;
};
template <typename S>
__device__ __forceinline__ S& rpk(typename RPack<S>::T& v, int e) {
  return reinterpret_cast<S*>(&v)[e];
}
template <typename S>
__device__ __forceinline__ typename RPack<S>::T rld(const S* p, int64_t q) {
  return reinterpret_cast<const typename RPack<S>::T*>(p)[q];
}
template <typename S>
__device__ __forceinline__ void rst(S* p, int64_t q, const typename RPack<S>::T& v) {
  reinterpret_cast<typename RPack<S>::T*>(p)[q] = v;
}

// Commit an accepted (Vt, TVt) and, with op_aa, write the new Anderson
// column (slot st->aa_slot) and the dot products of the stored columns with
// it and with the new residual (terms in S, FP64 accumulation per pack).
template <typename S, int MEM>
__device__ __forceinline__ void round_commit_body(SmState* st, S* __restrict__ V, S* __restrict__ TV,
                                                  S* __restrict__ Vp, S* __restrict__ TVp,
                                                  const S* __restrict__ Vt, const S* __restrict__ TVt,
                                                  S* __restrict__ MR, S* __restrict__ D, int64_t n, int64_t ld,
                                                  double* __restrict__ partials, int bid, int nblk) {
  if (!st->op_accept) return;
  const bool aa = st->op_aa != 0;
  const int slot = st->aa_slot, cnt = st->aa_cnt;
  constexpr int NP = RPack<S>::N;
  using PT = typename RPack<S>::T;
  double gr[MEM > 0 ? MEM : 1], rh[MEM > 0 ? MEM : 1];
#pragma unroll
  for (int j = 0; j < MEM; ++j) gr[j] = rh[j] = 0.0;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  const int64_t gt = (int64_t)bid * blockDim.x + threadIdx.x;
  const int64_t npack = n / NP;
  for (int64_t q = gt; q < npack; q += stride) {
    PT nv = rld(Vt, q), nt = rld(TVt, q), ov = rld(V, q), ot = rld(TV, q);
    rst(Vp, q, ov);
    rst(TVp, q, ot);
    rst(V, q, nv);
    rst(TV, q, nt);
    if (MEM > 0 && aa) {
      PT rr, dc, dd;
#pragma unroll
      for (int t = 0; t < NP; ++t) {
        rpk<S>(rr, t) = rpk<S>(nv, t) - rpk<S>(nt, t);
        rpk<S>(dc, t) = rpk<S>(rr, t) - (rpk<S>(ov, t) - rpk<S>(ot, t));
        rpk<S>(dd, t) = (rpk<S>(nv, t) - rpk<S>(ov, t)) - rpk<S>(dc, t);
      }
      rst(MR + (int64_t)slot * ld, q, dc);
      rst(D + (int64_t)slot * ld, q, dd);
#pragma unroll
      for (int j = 0; j < MEM; ++j) {
        if (j < cnt) {
          PT col = (j == slot) ? dc : rld(MR + (int64_t)j * ld, q);
          S g = 0, h = 0;
#pragma unroll
          for (int t = 0; t < NP; ++t) {
            g += rpk<S>(col, t) * rpk<S>(dc, t);
            h += rpk<S>(col, t) * rpk<S>(rr, t);
          }
          gr[j] += (double)g;
          rh[j] += (double)h;
        }
      }
    }
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) {  // tail
    const S nv = Vt[i], nt = TVt[i], ov = V[i], ot = TV[i];
    Vp[i] = ov;
    TVp[i] = ot;
    V[i] = nv;
    TV[i] = nt;
    if (MEM > 0 && aa) {
      const S r = nv - nt, dc = r - (ov - ot);
      MR[(int64_t)slot * ld + i] = dc;
      D[(int64_t)slot * ld + i] = (nv - ov) - dc;
#pragma unroll
      for (int j = 0; j < MEM; ++j) {
        if (j < cnt) {
          const S c = (j == slot) ? dc : MR[(int64_t)j * ld + i];
          gr[j] += (double)(c * dc);
          rh[j] += (double)(c * r);
        }
      }
    }
  }
  if (MEM == 0 || !aa) return;
  __shared__ double red[8][2 * kMaxMemory];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < MEM; ++j) {
    const double a = warp_sum(gr[j]), b = warp_sum(rh[j]);
    if (lane == 0) {
      red[w][j] = a;
      red[w][kMaxMemory + j] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * kMaxMemory) {
    const int j = threadIdx.x % kMaxMemory;
    double sum = 0.0;
    if (j < cnt)
      for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) sum += red[ww][threadIdx.x];
    partials[(int64_t)bid * 2 * kMaxMemory + threadIdx.x] = sum;
  }
}

template <typename S, int MEM>
__global__ void __launch_bounds__(256, 4) k_round_commit(SmState* st, S* __restrict__ V, S* __restrict__ TV,
                                                         S* __restrict__ Vp, S* __restrict__ TVp,
                                                         const S* __restrict__ Vt, const S* __restrict__ TVt,
                                                         S* __restrict__ MR, S* __restrict__ D, int64_t n,
                                                         int64_t ld, double* __restrict__ partials) {
  round_commit_body<S, MEM>(st, V, TV, Vp, TVp, Vt, TVt, MR, D, n, ld, partials, blockIdx.x, gridDim.x);
}

// Gram update and least squares for gamma (FP64), newest columns first;
// numerically singular Gram matrices drop their oldest columns from the solve.
__device__ __forceinline__ void round_aa_solve_body(SmState* st, const double* __restrict__ partials,
                                                    int nblocks) {
  if (!st->op_aa) return;
  __shared__ double part[8][2 * kMaxMemory];
  __shared__ double sums[2 * kMaxMemory];
  const int t = threadIdx.x;
  {
    const int val = t & 31, grp = t >> 5;
    double s = 0.0;
    for (int b = grp; b < nblocks; b += 8) s += partials[(int64_t)b * 2 * kMaxMemory + val];
    part[grp][val] = s;
  }
  __syncthreads();
  if (t < 2 * kMaxMemory) {
    double s = 0.0;
    for (int g = 0; g < 8; ++g) s += part[g][t];
    sums[t] = s;
  }
  __syncthreads();
  if (t != 0) return;
  const int M = kMaxMemory, slot = st->aa_slot, cnt = st->aa_cnt, mem = st->mem;
  for (int j = 0; j < cnt; ++j) {
    st->G[slot * M + j] = sums[j];
    st->G[j * M + slot] = sums[j];
    st->rhs[j] = sums[M + j];
  }
  int order[kMaxMemory];
  for (int j = 0; j < cnt; ++j) order[j] = ((slot - j) % mem + mem) % mem;
  for (int j = 0; j < M; ++j) st->gamma[j] = 0.0;
  st->aa_dropped = 0;
  for (int use = cnt; use >= 1; --use) {
    double Lm[kMaxMemory * kMaxMemory];
    double maxd = 0.0;
    for (int a = 0; a < use; ++a) maxd = fmax(maxd, st->G[order[a] * M + order[a]]);
    bool ok = maxd > 0.0;
    for (int a = 0; a < use && ok; ++a) {
      for (int b = 0; b <= a; ++b) {
        double s = st->G[order[a] * M + order[b]];
        for (int c = 0; c < b; ++c) s -= Lm[a * M + c] * Lm[b * M + c];
        if (a == b) {
          if (!(s > 1e-13 * maxd)) {
            ok = false;
            break;
          }
          Lm[a * M + a] = sqrt(s);
        } else {
          Lm[a * M + b] = s / Lm[b * M + b];
        }
      }
    }
    if (!ok) {
      st->aa_dropped++;
      continue;
    }
    double y[kMaxMemory];
    for (int a = 0; a < use; ++a) {
      double s = st->rhs[order[a]];
      for (int c = 0; c < a; ++c) s -= Lm[a * M + c] * y[c];
      y[a] = s / Lm[a * M + a];
    }
    for (int a = use - 1; a >= 0; --a) {
      double s = y[a];
      for (int c = a + 1; c < use; ++c) s -= Lm[c * M + a] * y[c];
      y[a] = s / Lm[a * M + a];
    }
    for (int a = 0; a < use; ++a) st->gamma[order[a]] = y[a];
    break;
  }
}

__global__ void __launch_bounds__(256) k_round_aa_solve(SmState* st, const double* __restrict__ partials,
                                                        int nblocks) {
  round_aa_solve_body(st, partials, nblocks);
}

// Next evaluation point in Vt (and the direction d for PT_DIR).
template <typename S, int MEM>
__device__ __forceinline__ void round_point_body(const SmState* __restrict__ st, const S* __restrict__ V,
                                                 const S* __restrict__ TV, S* __restrict__ Vt,
                                                 const S* __restrict__ TVt, S* __restrict__ d,
                                                 const S* __restrict__ D, int64_t n, int64_t ld, int bid,
                                                 int nblk) {
  const int op = st->op_point;
  if (op == PT_NONE) return;
  constexpr int NP = RPack<S>::N;
  using PT = typename RPack<S>::T;
  const int cnt = st->aa_cnt;
  S g[MEM > 0 ? MEM : 1];
#pragma unroll
  for (int j = 0; j < MEM; ++j) g[j] = (j < cnt) ? (S)st->gamma[j] : S(0);
  const S tau = (S)st->tau, coef = (S)st->coef, lam = (S)st->lam;
  const int64_t stride = (int64_t)nblk * blockDim.x;
  const int64_t gt = (int64_t)bid * blockDim.x + threadIdx.x;
  const int64_t npack = n / NP;
  for (int64_t q = gt; q < npack; q += stride) {
    PT v = rld(V, q), out;
    if (op == PT_DIR) {
      PT tv = rld(TV, q), dd;
#pragma unroll
      for (int t = 0; t < NP; ++t) rpk<S>(dd, t) = rpk<S>(tv, t) - rpk<S>(v, t);
#pragma unroll
      for (int j = 0; j < MEM; ++j) {
        if (j < cnt) {
          PT c = rld(D + (int64_t)j * ld, q);
#pragma unroll
          for (int t = 0; t < NP; ++t) rpk<S>(dd, t) -= g[j] * rpk<S>(c, t);
        }
      }
      rst(d, q, dd);
#pragma unroll
      for (int t = 0; t < NP; ++t) rpk<S>(out, t) = rpk<S>(v, t) + rpk<S>(dd, t);
    } else if (op == PT_LS) {
      PT dd = rld(d, q);
#pragma unroll
      for (int t = 0; t < NP; ++t) rpk<S>(out, t) = rpk<S>(v, t) + tau * rpk<S>(dd, t);
    } else if (op == PT_K2) {
      PT a = rld(Vt, q), b = rld(TVt, q);
#pragma unroll
      for (int t = 0; t < NP; ++t) rpk<S>(out, t) = rpk<S>(v, t) - coef * (rpk<S>(a, t) - rpk<S>(b, t));
    } else {  // PT_KM
      PT tv = rld(TV, q);
#pragma unroll
      for (int t = 0; t < NP; ++t) rpk<S>(out, t) = rpk<S>(v, t) - lam * (rpk<S>(v, t) - rpk<S>(tv, t));
    }
    rst(Vt, q, out);
  }
  for (int64_t i = npack * NP + gt; i < n; i += stride) {
    const S v = V[i];
    S o;
    if (op == PT_DIR) {
      S di = TV[i] - v;
#pragma unroll
      for (int j = 0; j < MEM; ++j)
        if (j < cnt) di -= g[j] * D[(int64_t)j * ld + i];
      d[i] = di;
      o = v + di;
    } else if (op == PT_LS) {
      o = v + tau * d[i];
    } else if (op == PT_K2) {
      o = v - coef * (Vt[i] - TVt[i]);
    } else {
      o = v - lam * (v - TV[i]);
    }
    Vt[i] = o;
  }
}

template <typename S, int MEM>
__global__ void __launch_bounds__(256) k_round_point(const SmState* __restrict__ st, const S* __restrict__ V,
                                                     const S* __restrict__ TV, S* __restrict__ Vt,
                                                     const S* __restrict__ TVt, S* __restrict__ d,
                                                     const S* __restrict__ D, int64_t n, int64_t ld) {
  round_point_body<S, MEM>(st, V, TV, Vt, TVt, d, D, n, ld, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// batched rounds
// ---------------------------------------------------------------------------
template <typename S>
__global__ void k_round_decide_b(const BInst<S>* __restrict__ bi, int n_inst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_inst) round_decide_body(bi[i].st, bi[i].stats, nullptr);
}
template <typename S, int MEM>
__global__ void __launch_bounds__(256, 4) k_round_commit_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const BInst<S>& b = bi[i];
  round_commit_body<S, MEM>(b.st, b.V, b.TV, b.Vp, b.TVp, b.Vt, b.TVt, b.MR, b.D, b.n_v, b.ld, b.paa,
                            blockIdx.x - m.base[i], m.cnt[i]);
}
template <typename S>
__global__ void __launch_bounds__(256) k_round_aa_solve_b(const BInst<S>* __restrict__ bi) {
  const BInst<S>& b = bi[blockIdx.x];
  round_aa_solve_body(b.st, b.paa, b.nb_vec);
}
template <typename S, int MEM>
__global__ void __launch_bounds__(256) k_round_point_b(const BInst<S>* __restrict__ bi, BMap m) {
  const int i = m.inst[blockIdx.x];
  const BInst<S>& b = bi[i];
  round_point_body<S, MEM>(b.st, b.V, b.TV, b.Vt, b.TVt, b.d, b.D, b.n_v, b.ld, blockIdx.x - m.base[i],
                           m.cnt[i]);
}

void launch_round_decide(SmState* st, const double* stats_t, int32_t* trace, cudaStream_t s) {
  k_round_decide<<<1, 32, 0, s>>>(st, stats_t, trace);
}
void launch_round_aa_solve(SmState* st, const double* partials, int nblocks, cudaStream_t s) {
  k_round_aa_solve<<<1, 256, 0, s>>>(st, partials, nblocks);
}

template <typename S>
void launch_round_commit(SmState* st, S* V, S* TV, S* Vp, S* TVp, const S* Vt, const S* TVt, S* MR, S* D,
                         int64_t n, int64_t ld, int mem, double* partials, int grid, cudaStream_t s) {
  switch (mem) {
#define SPOCK_RC(M) \
  case M: k_round_commit<S, M><<<grid, 256, 0, s>>>(st, V, TV, Vp, TVp, Vt, TVt, MR, D, n, ld, partials); break;
    SPOCK_RC(0) SPOCK_RC(1) SPOCK_RC(2) SPOCK_RC(3) SPOCK_RC(4) SPOCK_RC(5) SPOCK_RC(6) SPOCK_RC(7) SPOCK_RC(8)
    SPOCK_RC(9) SPOCK_RC(10) SPOCK_RC(11) SPOCK_RC(12) SPOCK_RC(13) SPOCK_RC(14) SPOCK_RC(15) SPOCK_RC(16)
#undef SPOCK_RC
    default: break;
  }
}
template <typename S>
void launch_round_point(SmState* st, const S* V, const S* TV, S* Vt, const S* TVt, S* d, const S* D, int64_t n,
                        int64_t ld, int mem, int grid, cudaStream_t s) {
  switch (mem) {
#define SPOCK_RP(M) case M: k_round_point<S, M><<<grid, 256, 0, s>>>(st, V, TV, Vt, TVt, d, D, n, ld); break;
    SPOCK_RP(0) SPOCK_RP(1) SPOCK_RP(2) SPOCK_RP(3) SPOCK_RP(4) SPOCK_RP(5) SPOCK_RP(6) SPOCK_RP(7) SPOCK_RP(8)
    SPOCK_RP(9) SPOCK_RP(10) SPOCK_RP(11) SPOCK_RP(12) SPOCK_RP(13) SPOCK_RP(14) SPOCK_RP(15) SPOCK_RP(16)
#undef SPOCK_RP
    default: break;
  }
}

template <typename S>
void launch_round_decide_b(const BInst<S>* bi, int n_inst, cudaStream_t st) {
  k_round_decide_b<S><<<(n_inst + 63) / 64, 64, 0, st>>>(bi, n_inst);
}
template <typename S>
void launch_round_aa_solve_b(const BInst<S>* bi, int n_inst, cudaStream_t st) {
  k_round_aa_solve_b<S><<<n_inst, 256, 0, st>>>(bi);
}
template <typename S>
void launch_round_commit_b(const BInst<S>* bi, const BMap& m, int nblocks, int mem, cudaStream_t st) {
  switch (mem) {
#define SPOCK_RC(M) case M: k_round_commit_b<S, M><<<nblocks, 256, 0, st>>>(bi, m); break;
    SPOCK_RC(0) SPOCK_RC(1) SPOCK_RC(2) SPOCK_RC(3) SPOCK_RC(4) SPOCK_RC(5) SPOCK_RC(6) SPOCK_RC(7) SPOCK_RC(8)
    SPOCK_RC(9) SPOCK_RC(10) SPOCK_RC(11) SPOCK_RC(12) SPOCK_RC(13) SPOCK_RC(14) SPOCK_RC(15) SPOCK_RC(16)
#undef SPOCK_RC
    default: break;
  }
}
template <typename S>
void launch_round_point_b(const BInst<S>* bi, const BMap& m, int nblocks, int mem, cudaStream_t st) {
  switch (mem) {
#define SPOCK_RP(M) case M: k_round_point_b<S, M><<<nblocks, 256, 0, st>>>(bi, m); break;
    SPOCK_RP(0) SPOCK_RP(1) SPOCK_RP(2) SPOCK_RP(3) SPOCK_RP(4) SPOCK_RP(5) SPOCK_RP(6) SPOCK_RP(7) SPOCK_RP(8)
    SPOCK_RP(9) SPOCK_RP(10) SPOCK_RP(11) SPOCK_RP(12) SPOCK_RP(13) SPOCK_RP(14) SPOCK_RP(15) SPOCK_RP(16)
#undef SPOCK_RP
    default: break;
  }
}
#define SPOCK_RB_INST(S)                                                                          \
  template void launch_round_decide_b<S>(const BInst<S>*, int, cudaStream_t);                     \
  template void launch_round_aa_solve_b<S>(const BInst<S>*, int, cudaStream_t);                   \
  template void launch_round_commit_b<S>(const BInst<S>*, const BMap&, int, int, cudaStream_t);   \
  template void launch_round_point_b<S>(const BInst<S>*, const BMap&, int, int, cudaStream_t);
SPOCK_RB_INST(double)
SPOCK_RB_INST(float)
#undef SPOCK_RB_INST

template void launch_round_commit<double>(SmState*, double*, double*, double*, double*, const double*,
                                          const double*, double*, double*, int64_t, int64_t, int, double*, int,
                                          cudaStream_t);
template void launch_round_commit<float>(SmState*, float*, float*, float*, float*, const float*, const float*,
                                         float*, float*, int64_t, int64_t, int, double*, int, cudaStream_t);
template void launch_round_point<double>(SmState*, const double*, const double*, double*, const double*, double*,
                                         const double*, int64_t, int64_t, int, int, cudaStream_t);
template void launch_round_point<float>(SmState*, const float*, const float*, float*, const float*, float*,
                                        const float*, int64_t, int64_t, int, int, cudaStream_t);

}  // namespace spock
