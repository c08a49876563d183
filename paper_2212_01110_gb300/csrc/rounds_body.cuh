// Device bodies of the round kernels (rounds.cu), shared with the
// single-block solve kernel (cta.cu): decision, commit with the Anderson
// column and Gram row, Gram solve, next evaluation point.
#pragma once

#include <cmath>
#include <cstdint>

#include "kernels.cuh"
#include "supermann.cuh"

namespace spock {

static __device__ void round_trace(SmState* st, int32_t* trace, int branch, int nb) {
  if (st->record_trace && trace && st->k < st->max_iter) {
    trace[2 * st->k] = branch;
    trace[2 * st->k + 1] = nb;
  }
}

// Decisions after an iterate has been accepted (its statistics in stats_cur).
static __device__ void round_after_accept(SmState* st, int32_t* trace) {
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

static __device__ void round_decide_body(SmState* st, const double* __restrict__ stats_t, int32_t* trace) {
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
// The Anderson differences are formed from the old (V, TV) as it is read, so
// the previous pair is not kept.
template <typename S, int MEM>
__device__ __forceinline__ void round_commit_body(SmState* st, S* __restrict__ V, S* __restrict__ TV,
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


// Gram update and least squares for gamma (FP64), newest columns first;
// numerically singular Gram matrices drop their oldest columns from the solve.
__device__ __forceinline__ void round_aa_solve_body(SmState* st, const double* __restrict__ partials,
                                                    int nblocks) {
  if (!st->op_aa) return;
  __shared__ double part[8][2 * kMaxMemory];
  __shared__ double sums[2 * kMaxMemory];
  const int t = threadIdx.x;
  const int ngrp = blockDim.x >> 5;  // 1..8 warps
  {
    const int val = t & 31, grp = t >> 5;
    double s = 0.0;
    for (int b = grp; b < nblocks; b += ngrp) s += partials[(int64_t)b * 2 * kMaxMemory + val];
    part[grp][val] = s;
  }
  __syncthreads();
  if (t < 2 * kMaxMemory) {
    double s = 0.0;
    for (int g = 0; g < ngrp; ++g) s += part[g][t];
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

}  // namespace spock
