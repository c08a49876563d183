// Device bodies of the vector kernels of T (ops.cu), shared with the
// single-block solve kernel (cta.cu): every body works for block `bid` of
// `nblk` blocks of one problem.
#pragma once

#include <cstdint>

#include "kernels.cuh"
#include "spock_internal.h"

namespace spock {

enum DualMode : int { DM_APPLY_L = 0, DM_PROXG = 1, DM_DUAL = 2 };
enum LstarMode : int { LS_APPLY = 0, LS_PREP = 2 };
constexpr int kMaxJ = (kMaxDim + 2 + 31) / 32;   // entries per lane for the largest blocks

// ---------------------------------------------------------------------------
// k_lstar
// ---------------------------------------------------------------------------
// (L* w) at the entries of node k, from the rows of L that involve them:
//   x^k, u^k  (nonleaf):  w_nl[x, u] + sum_c (Q^c or R^c)^1/2 w_nr^c[x, u]
//   x^k       (leaf):     w_lf[x] + Q_N^1/2 w_lf[soc x]
//   y^k_l:                w_nl[y_l] - b_l w_nl[s - b'y],   b = (p^children, 0, 1)
//   tau^c:                (w_nr^c[tau 1] + w_nr^c[tau 2]) / 2
//   s^c:                  w_nl^c[s - b'y] (c nonleaf) or (w_lf^c[s 1] + w_lf^c[s 2]) / 2
//   s^0:                  w_nl^0[s - b'y]
// Body shared by the single-problem and the batched kernels: block `bid` of
// `nblk` working for problem p.
// prox-f preparation of the z_2 block of a chain node k (one child): zbar =
// z - alpha L* eta on (y, tau, s), then the projection on ker [E^T, -I, -I]
// (the m = 1 case of the closed form in lstar_body), by one lane.
template <typename S>
__device__ __forceinline__ void prep_z2_chain(const KP<S>& p, int k, const S* __restrict__ eta,
                                              const S* __restrict__ z, S* __restrict__ zo) {
  const S al = p.alpha;
  const int64_t el = p.enl[k], z2 = p.zz2[k];
  const int c = p.ch_begin[k];
  const int64_t er = p.enr[c], es = __ldg(&p.desc[c].es);
  const int nxu = p.nx + p.nu;
  const S sb = eta[el + 3];
  const S tl = S(0.5) * (eta[er + nxu] + eta[er + nxu + 1]);
  const S sl = (c < p.nl) ? eta[es] : S(0.5) * (eta[es] + eta[es + 1]);
  const S a = p.av[k];
  const S y3 = z[z2 + 2] - al * (eta[el + 2] - sb);
  const S y1 = z[z2] - al * (eta[el] - p.prob[c] * sb);
  const S y2 = z[z2 + 1] - al * eta[el + 1];
  const S ta = z[z2 + 3] - al * tl;
  const S sv = z[z2 + 4] - al * sl;
  const S mw = a * y1 - y2 + y3 - ta - sv;
  const S lam = (mw - mw * p.s2inv[2 * (int64_t)k + 1]) * p.s2inv[2 * (int64_t)k];
  zo[z2] = y1 - a * lam;
  zo[z2 + 1] = y2 + lam;
  zo[z2 + 2] = y3 - lam;
  zo[z2 + 3] = ta + lam;
  zo[z2 + 4] = sv + lam;
  if (k == 0) zo[0] = (z[0] - al * sb) - al;   // prox of alpha * s^0 (a tree that is one chain)
}

template <typename S, int MODE, int J>
__device__ __forceinline__ void lstar_body(const KP<S>& p, int bid, int nblk, const S* __restrict__ eta,
                                           const S* __restrict__ z, S* __restrict__ zo) {
  if (p.skip && *p.skip) return;
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const int nx = p.nx, nu = p.nu;
  const S al = p.alpha;
  auto E = [&](int64_t i) -> S { return eta[i]; };
  auto emit = [&](int64_t zi, S lt) { zo[zi] = lt; };   // LS_APPLY
  const int kc0 = p.stage_begin[p.chain_stage];          // first node of the chain region
  uint32_t wnext = gw < p.n ? desc_word(p.desc, gw, lane) : 0u;
  for (int k = gw; k < p.n; k += nw) {
    const NodeF D = node_fields(wnext);
    if (k + nw < p.n) wnext = desc_word(p.desc, k + nw, lane);
    if (k < p.nl) {
      const int m = D.m, c0 = D.c0;
      const int nxu = nx + nu;
      const int64_t ex = D.enl + 2 * m + 2;
      // ---- (x, u): own rows and the first child's nonroot rows, in registers
      S lt[J], zv[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        lt[j] = zv[j] = S(0);
        if (e < nxu) {
          const S coef = e < nx ? p.qs[(int64_t)c0 * nx + e] : p.rs[(int64_t)c0 * nu + (e - nx)];
          lt[j] = E(ex + e) + coef * E(D.enr_c0 + e);
          if (MODE == LS_PREP) zv[j] = z[e < nx ? D.zx + e : D.zu + (e - nx)];
        }
      }
      for (int c = 1; c < m; ++c) {   // further children (branching stages only)
        const int64_t er = __ldg(&p.desc[c0 + c].enr);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < nxu) {
            const S coef = e < nx ? p.qs[(int64_t)(c0 + c) * nx + e] : p.rs[(int64_t)(c0 + c) * nu + (e - nx)];
            lt[j] += coef * E(er + e);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        if (e < nxu) {
          if (MODE == LS_PREP) {
            if (e < nx) p.xbar[(int64_t)k * p.xs + e] = zv[j] - al * lt[j];
            else p.ubar[(int64_t)k * p.us + (e - nx)] = zv[j] - al * lt[j];
          } else {
            zo[e < nx ? D.zx + e : D.zu + (e - nx)] = lt[j];
          }
        }
      }
      // ---- z_2 block (chain nodes of the prox-f preparation: one lane per
      // node after this loop)
      if (MODE == LS_PREP && k >= kc0) continue;
      const int64_t el = D.enl, z2 = D.zz2;
      const S sb = E(el + 2 * m + 1);
      // child j's tau and s rows of L* w
      auto child_rows = [&](int jc, S& tau_l, S& s_l) {
        const int c = c0 + jc;
        const int64_t er = jc == 0 ? D.enr_c0 : __ldg(&p.desc[c].enr);
        const int64_t es = jc == 0 ? D.es_c0 : __ldg(&p.desc[c].es);
        tau_l = S(0.5) * (E(er + nxu) + E(er + nxu + 1));
        s_l = (c < p.nl) ? E(es) : S(0.5) * (E(es) + E(es + 1));
      };
      if (MODE != LS_PREP) {
        for (int l = lane; l < 2 * m + 1; l += 32) {
          const S bl = l < m ? p.prob[c0 + l] : (l < 2 * m ? S(0) : S(1));
          emit(z2 + l, E(el + l) - bl * sb);
        }
        for (int jc = lane; jc < m; jc += 32) {
          S tl, sl;
          child_rows(jc, tl, sl);
          emit(z2 + 2 * m + 1 + jc, tl);
          emit(z2 + 3 * m + 1 + jc, sl);
        }
        if (k == 0 && lane == 0) emit(0, sb);
      } else {
        // zbar = z - alpha L* eta on z_2, then the projection on
        // ker [E^T, -I, -I] with (M M^T)^-1 = (I - 11^T / (c + m)) / c,
        // c = a^2 + 3 (Sherman-Morrison); M w = a y1 - y2 + y3 - tau - s per child.
        const S a = p.av[k];
        const S y3 = z[z2 + 2 * m] - al * (E(el + 2 * m) - sb);
        auto bars = [&](int jc, S& y1, S& y2, S& ta, S& sv) {
          S tl, sl;
          child_rows(jc, tl, sl);
          y1 = z[z2 + jc] - al * (E(el + jc) - p.prob[c0 + jc] * sb);
          y2 = z[z2 + m + jc] - al * E(el + m + jc);
          ta = z[z2 + 2 * m + 1 + jc] - al * tl;
          sv = z[z2 + 3 * m + 1 + jc] - al * sl;
        };
        // children 0..31 kept in registers; further ones recomputed
        S y1 = 0, y2 = 0, ta = 0, sv = 0, sumMw = 0;
        if (lane < m) {
          bars(lane, y1, y2, ta, sv);
          sumMw = a * y1 - y2 + y3 - ta - sv;
        }
        for (int jc = lane + 32; jc < m; jc += 32) {
          S b1, b2, bt, bs;
          bars(jc, b1, b2, bt, bs);
          sumMw += a * b1 - b2 + y3 - bt - bs;
        }
        sumMw = lanes_sum(sumMw, m);
        const S inv_cc = p.s2inv[2 * (int64_t)k];                // 1 / cc, precomputed
        const S shift = sumMw * p.s2inv[2 * (int64_t)k + 1];     // sumMw / (cc + m)
        S sumlam = 0;
        if (lane < m) {
          const S lam = (a * y1 - y2 + y3 - ta - sv - shift) * inv_cc;
          zo[z2 + lane] = y1 - a * lam;
          zo[z2 + m + lane] = y2 + lam;
          zo[z2 + 2 * m + 1 + lane] = ta + lam;
          zo[z2 + 3 * m + 1 + lane] = sv + lam;
          sumlam = lam;
        }
        for (int jc = lane + 32; jc < m; jc += 32) {
          S b1, b2, bt, bs;
          bars(jc, b1, b2, bt, bs);
          const S lam = (a * b1 - b2 + y3 - bt - bs - shift) * inv_cc;
          zo[z2 + jc] = b1 - a * lam;
          zo[z2 + m + jc] = b2 + lam;
          zo[z2 + 2 * m + 1 + jc] = bt + lam;
          zo[z2 + 3 * m + 1 + jc] = bs + lam;
          sumlam += lam;
        }
        sumlam = lanes_sum(sumlam, m);
        if (lane == 0) {
          zo[z2 + 2 * m] = y3 - sumlam;
          if (k == 0) zo[0] = (z[0] - al * sb) - al;   // prox of alpha * s^0
        }
      }
    } else {
      // ---- leaf: x^k
      const int64_t ef = D.elf;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        if (e < nx) {
          const S lt = E(ef + e) + p.qns[(int64_t)k * nx + e] * E(ef + nx + e);
          if (MODE == LS_PREP) p.xbar[(int64_t)k * p.xs + e] = z[D.zx + e] - al * lt;
          else emit(D.zx + e, lt);
        }
      }
    }
  }
  if (MODE == LS_PREP)
    for (int64_t base = (int64_t)kc0 + 32 * (int64_t)gw; base < p.nl; base += 32 * (int64_t)nw)
      if (base + lane < p.nl) prep_z2_chain<S>(p, (int)(base + lane), eta, z, zo);
}


// ---------------------------------------------------------------------------
// k_dual
// ---------------------------------------------------------------------------
// Per entry of eta: the value of the L row at z (Lz), at z+ (Lzp) and at the
// direction (Ld).  For DM_DUAL, w = eta + alpha (2 Lzp - Lz) and the
// residual row of L is L r_z = Lz - Lzp.

template <typename S, int MODE>
__device__ __forceinline__ S dual_w(S alpha, S e, S Lz, S Lzp) {
  if (MODE == DM_APPLY_L) return Lz;
  if (MODE == DM_PROXG) return e;
  return e + alpha * (S(2) * Lzp - Lz);
}

// Residual statistics of one eta row: r_eta = eta - eta+ against L r_z, and
// with a direction d the inner products of the line search.
template <typename S, bool ST, bool DR>
__device__ __forceinline__ void dual_stat(NodeAcc<S>& a, S inv_alpha, S e_old, S e_new, S lrz, S de, S ld) {
  if (!ST) return;
  const S re = e_old - e_new;
  a.s[ST_RE2] += re * re;
  a.s[ST_RE_LRZ] += re * lrz;
  a.s[ST_XID] = vmax(a.s[ST_XID], vabs(re * inv_alpha - lrz));
  if (DR) {
    a.s[ST_RD] += re * de;
    a.s[ST_LRZ_DE] += lrz * de;
    a.s[ST_RE_LDZ] += re * ld;
  }
}

// Translated second-order cone of S3, SOC + sh with SOC = {(v, t): ||v|| <= t}
// (t the last entry) and sh = (0, .., 1/2, -1/2).  The caller holds in y[j]
// (entry lane + 32 j of a block of `dim` entries) the point y = w / alpha - sh
// of the Moreau decomposition w - alpha proj(w / alpha) = alpha (y - P(y)),
// P the projection on SOC.  o[j] receives alpha (y - P(y)):
//   ||v|| <= t:  0;   ||v|| <= -t:  alpha y;
//   otherwise:   v-part alpha (1 - s) v, t-part alpha (t - s ||v||),
//                s = (||v|| + t) / (2 ||v||),
// with one reciprocal square root per block (the case tests use ||v||^2).
template <typename S, int J>
__device__ __forceinline__ void soc_moreau(const S (&y)[J], int dim, S al, int lane, S (&o)[J]) {
  S s2 = 0, tl = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int e = lane + 32 * j;
    if (e < dim - 1) s2 += y[j] * y[j];
    else if (e == dim - 1) tl = y[j];
  }
  s2 = warp_sum(s2);
  const S t = __shfl_sync(kFull, tl, (dim - 1) & 31);
  const bool in_cone = s2 <= t * t;
  if (in_cone && t >= S(0)) {
#pragma unroll
    for (int j = 0; j < J; ++j) o[j] = S(0);
  } else if (in_cone) {
#pragma unroll
    for (int j = 0; j < J; ++j) o[j] = al * y[j];
  } else {
    const S rs = vrsqrt(s2);
    const S c = S(0.5) * al * (S(1) - t * rs);
    const S ot = S(0.5) * al * (t - s2 * rs);
#pragma unroll
    for (int j = 0; j < J; ++j) o[j] = (lane + 32 * j == dim - 1) ? ot : c * y[j];
  }
}

// y = w / alpha - sh of the translated SOC block (entries e < dim).
template <typename S>
__device__ __forceinline__ S soc_shift(S y, int e, int dim) {
  if (e == dim - 2) return y - S(0.5);
  if (e == dim - 1) return y + S(0.5);
  return y;
}

// Without statistics: the dual update (DM_DUAL), L z (DM_APPLY_L) or
// prox_{alpha g*}(eta) (DM_PROXG); warp per node, each node's own rows, its
// nonroot block and (leaves) its leaf block.
template <typename S, int MODE, int J>
__device__ __forceinline__ void dual_body(const KP<S>& p, int bid, int nblk, const S* __restrict__ z,
                                          const S* __restrict__ zp, const S* __restrict__ eta,
                                          S* __restrict__ out) {
  if (p.skip && *p.skip) return;
  constexpr bool HZ = MODE != DM_PROXG;     // rows of L at z
  constexpr bool HZP = MODE == DM_DUAL;     // ... and at z+
  constexpr bool HE = MODE != DM_APPLY_L;   // eta is read
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const S al = p.alpha, ial = p.inv_alpha;
  const int nx = p.nx, nu = p.nu;
  uint32_t wnext = gw < p.n ? desc_word(p.desc, gw, lane) : 0u;
  for (int k = gw; k < p.n; k += nw) {
    const NodeF D = node_fields(wnext);
    if (k + nw < p.n) wnext = desc_word(p.desc, k + nw, lane);
    const bool nonleaf = k < p.nl;
    const int na = nonleaf ? nx + nu : nx;          // own (x, u) or x entries
    const int64_t ea = nonleaf ? D.enl + 2 * D.m + 2 : D.elf;   // eta row of the box on x^k
    const int nb = nx + nu + 2;                      // nonroot block
    // ---- loads: own (x, u) with its box rows, the nonroot block, s^k
    S az[J], azp[J], ae[J], alo[J], ahi[J];
    S bz[J], bzp[J], bc[J], be[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int e = lane + 32 * j;
      az[j] = azp[j] = ae[j] = alo[j] = ahi[j] = S(0);
      bz[j] = bzp[j] = bc[j] = be[j] = S(0);
      if (e < na) {
        const int64_t zi = e < nx ? D.zx + e : D.zu + (e - nx);
        if (HZ) az[j] = z[zi];
        if (HZP) azp[j] = zp[zi];
        if (HE) ae[j] = eta[ea + e];
        if (MODE != DM_APPLY_L) {
          alo[j] = e < nx ? p.xlo[(int64_t)k * nx + e] : p.ulo[(int64_t)k * nu + (e - nx)];
          ahi[j] = e < nx ? p.xhi[(int64_t)k * nx + e] : p.uhi[(int64_t)k * nu + (e - nx)];
        }
      }
      if (k > 0 && e < nb) {
        const int64_t zi = e < nx ? D.zxp + e : (e < nx + nu ? D.zup + (e - nx) : D.ztau);
        bc[j] = e < nx ? p.qs[(int64_t)k * nx + e] : (e < nx + nu ? p.rs[(int64_t)k * nu + (e - nx)] : S(0.5));
        if (HZ) bz[j] = z[zi];
        if (HZP) bzp[j] = zp[zi];
        if (HE) be[j] = eta[D.enr + e];
      }
    }
    const S sz = HZ ? z[D.zs] : S(0), szp = HZP ? zp[D.zs] : S(0);
    // ---- box rows on the node's own x (and u)
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int e = lane + 32 * j;
      if (e < na) {
        const S w = dual_w<S, MODE>(al, ae[j], az[j], azp[j]);
        out[ea + e] = (MODE == DM_APPLY_L) ? w : w - al * clampv(w * ial, alo[j], ahi[j]);
      }
    }
    // ---- nonroot block: SOC on (Q^1/2 x^anc, R^1/2 u^anc, tau/2, tau/2)
    if (k > 0) {
      S w[J];
#pragma unroll
      for (int j = 0; j < J; ++j) w[j] = dual_w<S, MODE>(al, be[j], bc[j] * bz[j], bc[j] * bzp[j]);
      if (MODE == DM_APPLY_L) {
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (lane + 32 * j < nb) out[D.enr + lane + 32 * j] = w[j];
      } else {
        S y[J], o[J];
#pragma unroll
        for (int j = 0; j < J; ++j) y[j] = lane + 32 * j < nb ? soc_shift(w[j] * ial, lane + 32 * j, nb) : S(0);
        soc_moreau<S, J>(y, nb, al, lane, o);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < nb) out[D.enr + e] = o[j];
        }
      }
    }
    if (nonleaf) {
      // ---- y rows (K* cone: y1, y2 <= 0 after the prox, y3 free) and the
      // s - b'y row, b = (p^children, 0, 1)
      const int m = D.m, c0 = D.c0;
      const int64_t el = D.enl, z2 = D.zz2;
      S bs = 0, bsp = 0;
      for (int e = lane; e < 2 * m + 1; e += 32) {
        const S Lz = HZ ? z[z2 + e] : S(0);
        const S Lzp = HZP ? zp[z2 + e] : S(0);
        const S w = dual_w<S, MODE>(al, HE ? eta[el + e] : S(0), Lz, Lzp);
        out[el + e] = (MODE == DM_APPLY_L) ? w : (e < 2 * m ? vmin(w, S(0)) : S(0));
        if (e < m) {
          const S pj = p.prob[c0 + e];
          bs += pj * Lz;
          bsp += pj * Lzp;
        }
      }
      if (MODE != DM_PROXG) {
        bs = lanes_sum(bs, m);   // lanes < m hold the children's terms
        if (HZP) bsp = lanes_sum(bsp, m);
      }
      if (lane == 0) {
        const int64_t ie = el + 2 * m + 1;
        const S y3 = HZ ? z[z2 + 2 * m] : S(0), y3p = HZP ? zp[z2 + 2 * m] : S(0);
        const S Lz = sz - (bs + y3), Lzp = HZP ? szp - (bsp + y3p) : S(0);
        const S w = dual_w<S, MODE>(al, HE ? eta[ie] : S(0), Lz, Lzp);
        out[ie] = (MODE == DM_APPLY_L) ? w : vmin(w, S(0));
      }
    } else {
      // ---- leaf SOC on (Q_N^1/2 x, s/2, s/2)
      const int dim = nx + 2;
      const int64_t es = D.elf + nx;
      S w[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        S Lz = S(0), Lzp = S(0), ev = S(0);
        if (e < dim) {
          if (e < nx) {
            const S c = p.qns[(int64_t)k * nx + e];
            Lz = c * az[j];
            Lzp = c * azp[j];
          } else {
            Lz = S(0.5) * sz;
            Lzp = S(0.5) * szp;
          }
          if (HE) ev = eta[es + e];
        }
        w[j] = dual_w<S, MODE>(al, ev, Lz, Lzp);
      }
      if (MODE == DM_APPLY_L) {
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (lane + 32 * j < dim) out[es + lane + 32 * j] = w[j];
      } else {
        S y[J], o[J];
#pragma unroll
        for (int j = 0; j < J; ++j) y[j] = lane + 32 * j < dim ? soc_shift(w[j] * ial, lane + 32 * j, dim) : S(0);
        soc_moreau<S, J>(y, dim, al, lane, o);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < dim) out[es + e] = o[j];
        }
      }
    }
  }
}


// ---------------------------------------------------------------------------
// k_dual_fused: the dual update with all residual statistics in one pass.
// One warp per NONLEAF node k owns every eta row that involves k's
// variables: k's nonleaf block, the nonroot block of each child c (rows of
// Q^c 1/2 x^k, R^c 1/2 u^k, tau^c) and the leaf block of each leaf child.
// Each z entry's rows of L then lie in one warp, which therefore has the
// whole of (L* r_eta) there and accumulates the primal statistics as well:
//   x^k, u^k:  own box rows + sum_c (Q^c or R^c)^1/2 nonroot rows of c
//   y^k:       y rows - b (s - b'y) row;   s^k (nonleaf): the s - b'y row
//   tau^c:     the two tau rows of c's nonroot block
//   x^c, s^c (leaf c): c's leaf block.
// The nonroot blocks reuse x^k, u^k already in registers.
// ---------------------------------------------------------------------------
// rz = z - z+ of one entry, lt = (L* r_eta) there, dv the direction
template <typename S, bool DR>
__device__ __forceinline__ void primal_stat(NodeAcc<S>& a, S inv_alpha, S rz, S dv, S lt) {
  a.s[ST_RZ2] += rz * rz;
  a.s[ST_XIP] = vmax(a.s[ST_XIP], vabs(rz * inv_alpha - lt));
  if (DR) a.s[ST_RD] += rz * dv;
}

// The s - b'y row and the y rows of a chain node k (one child, b = (p, 0, 1))
// with their residual statistics, by one lane (the m = 1 case of the warp
// code in dual_fused_body).
template <typename S, bool DR>
__device__ __forceinline__ void dual_y_chain(const KP<S>& p, int k, const S* __restrict__ z,
                                             const S* __restrict__ zp, const S* __restrict__ eta,
                                             S* __restrict__ out, const S* __restrict__ dz,
                                             const S* __restrict__ deta, NodeAcc<S>& nacc) {
  const S al = p.alpha, ial = p.inv_alpha;
  const int64_t el = p.enl[k], z2 = p.zz2[k], zsk = p.zs[k];
  const S pr = p.prob[p.ch_begin[k]];
  S yz[3], yzp[3], yd[3], ye[3], yde[3];
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    yz[e] = z[z2 + e];
    yzp[e] = zp[z2 + e];
    yd[e] = DR ? dz[z2 + e] : S(0);
    ye[e] = eta[el + e];
    yde[e] = DR ? deta[el + e] : S(0);
  }
  const S sk = z[zsk], skp = zp[zsk], skd = DR ? dz[zsk] : S(0);
  const S esb = eta[el + 3], desb = DR ? deta[el + 3] : S(0);
  const S Lz = sk - (pr * yz[0] + yz[2]), Lzp = skp - (pr * yzp[0] + yzp[2]);
  const S Ld = DR ? skd - (pr * yd[0] + yd[2]) : S(0);
  const S w = dual_w<S, DM_DUAL>(al, esb, Lz, Lzp);
  const S o = vmin(w, S(0));
  const S re_sb = esb - o;
  out[el + 3] = o;
  dual_stat<S, true, DR>(nacc, ial, esb, o, Lz - Lzp, desb, Ld);
  primal_stat<S, DR>(nacc, ial, sk - skp, skd, re_sb);
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const S yw = dual_w<S, DM_DUAL>(al, ye[e], yz[e], yzp[e]);
    const S yo = e < 2 ? vmin(yw, S(0)) : S(0);
    out[el + e] = yo;
    dual_stat<S, true, DR>(nacc, ial, ye[e], yo, yz[e] - yzp[e], yde[e], yd[e]);
    const S bl = e == 0 ? pr : (e == 1 ? S(0) : S(1));
    primal_stat<S, DR>(nacc, ial, yz[e] - yzp[e], yd[e], (ye[e] - yo) - bl * re_sb);
  }
}

template <typename S, bool DIR, int J>
__device__ __forceinline__ void dual_fused_body(const KP<S>& p, int bid, int nblk, const S* __restrict__ z,
                                                const S* __restrict__ zp, const S* __restrict__ eta,
                                                S* __restrict__ out, const S* __restrict__ dir,
                                                double* __restrict__ partials) {
  if (p.skip && *p.skip) return;
  constexpr bool DR = DIR;
  const int lane = threadIdx.x & 31;
  const int gw = (bid * blockDim.x + threadIdx.x) >> 5;
  const int nw = (nblk * blockDim.x) >> 5;
  const S al = p.alpha, ial = p.inv_alpha;
  const int nx = p.nx, nu = p.nu, nxu = nx + nu, nb = nxu + 2;
  const S* dz = DR ? dir : nullptr;
  const S* deta = DR ? dir + p.n_z : nullptr;
  StatAcc acc;
  acc.zero();
  NodeAcc<S> nacc;
  nacc.zero();
  const int kc0 = p.stage_begin[p.chain_stage];   // chain nodes: y rows one lane per node, below
  uint32_t wnext = gw < p.nl ? desc_word(p.desc, gw, lane) : 0u;
  for (int k = gw; k < p.nl; k += nw) {
    const NodeF D = node_fields(wnext);
    if (k + nw < p.nl) wnext = desc_word(p.desc, k + nw, lane);
    const int m = D.m, c0 = D.c0;
    const bool warp_y = k < kc0;
    const int64_t el = D.enl, ea = el + 2 * m + 2, z2 = D.zz2;
    // ---- loads issued up front with the node's own rows (one memory round
    // trip per node on chains): the first child's nonroot rows and tau, the
    // first 32 y rows and the s - b'y row
    S pbe[J], pbde[J], pbc[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int e = lane + 32 * j;
      pbe[j] = pbde[j] = pbc[j] = S(0);
      if (e < nb) {
        pbc[j] = e < nx ? p.qs[(int64_t)c0 * nx + e] : (e < nxu ? p.rs[(int64_t)c0 * nu + (e - nx)] : S(0.5));
        pbe[j] = eta[D.enr_c0 + e];
        if (DR) pbde[j] = deta[D.enr_c0 + e];
      }
    }
    const S ptz = z[z2 + 2 * m + 1], ptzp = zp[z2 + 2 * m + 1], ptdz = DR ? dz[z2 + 2 * m + 1] : S(0);
    S yz0 = 0, yzp0 = 0, yd0 = 0, ye0 = 0, yde0 = 0, pr0 = 0;
    S sk = 0, skp = 0, skd = 0, y3 = 0, y3p = 0, y3d = 0, esb = 0, desb = 0;
    const int64_t ie_sb = el + 2 * m + 1;
    if (warp_y) {
      if (lane < 2 * m + 1) {
        yz0 = z[z2 + lane];
        yzp0 = zp[z2 + lane];
        if (DR) yd0 = dz[z2 + lane];
        ye0 = eta[el + lane];
        if (DR) yde0 = deta[el + lane];
        if (lane < m) pr0 = p.prob[c0 + lane];
      }
      sk = z[D.zs];
      skp = zp[D.zs];
      if (DR) skd = dz[D.zs];
      y3 = z[z2 + 2 * m];
      y3p = zp[z2 + 2 * m];
      if (DR) y3d = dz[z2 + 2 * m];
      esb = eta[ie_sb];
      if (DR) desb = deta[ie_sb];
    }
    // ---- own (x, u) and its box rows.  Per entry the differences r_z = z - z+
    // (the residual, also L r_z of every row of L that reads it, scaled) and
    // q_z = z+ - r_z = 2 z+ - z (the point L is applied to in the dual update)
    // are formed once and reused by every row of L that reads the entry.
    S rzv[J], qzv[J], adz[J], lt[J];
    {
      S az[J], azp[J], ae[J], ade[J], alo[J], ahi[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        az[j] = azp[j] = adz[j] = lt[j] = ae[j] = ade[j] = alo[j] = ahi[j] = S(0);
        if (e < nxu) {
          const int64_t zi = e < nx ? D.zx + e : D.zu + (e - nx);
          az[j] = z[zi];
          azp[j] = zp[zi];
          if (DR) adz[j] = dz[zi];
          ae[j] = eta[ea + e];
          if (DR) ade[j] = deta[ea + e];
          alo[j] = e < nx ? p.xlo[(int64_t)k * nx + e] : p.ulo[(int64_t)k * nu + (e - nx)];
          ahi[j] = e < nx ? p.xhi[(int64_t)k * nx + e] : p.uhi[(int64_t)k * nu + (e - nx)];
        }
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        rzv[j] = az[j] - azp[j];
        qzv[j] = azp[j] - rzv[j];
        if (e < nxu) {
          const S w = ae[j] + al * qzv[j];
          const S o = w - al * clampv(w * ial, alo[j], ahi[j]);
          out[ea + e] = o;
          dual_stat<S, true, DR>(nacc, ial, ae[j], o, rzv[j], ade[j], adz[j]);
          lt[j] = ae[j] - o;
        }
      }
    }
    // ---- children
    for (int jc = 0; jc < m; ++jc) {
      const int c = c0 + jc;
      const int64_t ztau = z2 + 2 * m + 1 + jc;
      const int64_t er = jc == 0 ? D.enr_c0 : __ldg(&p.desc[c].enr);
      S tz = ptz, tzp = ptzp, tdz = ptdz;
      S be[J], bde[J], bc[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        be[j] = pbe[j];
        bde[j] = pbde[j];
        bc[j] = pbc[j];
      }
      if (jc > 0) {  // further children (branching stages only)
        tz = z[ztau];
        tzp = zp[ztau];
        if (DR) tdz = dz[ztau];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < nb) {
            bc[j] = e < nx ? p.qs[(int64_t)c * nx + e] : (e < nxu ? p.rs[(int64_t)c * nu + (e - nx)] : S(0.5));
            be[j] = eta[er + e];
            if (DR) bde[j] = deta[er + e];
          }
        }
      }
      {  // nonroot block of c: SOC on (Q^c 1/2 x^k, R^c 1/2 u^k, tau^c / 2, tau^c / 2)
        const S rt = tz - tzp, qt = tzp - rt;
        S y[J], lrz[J], ld[J], o[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          y[j] = lrz[j] = ld[j] = S(0);
          if (e < nb) {
            const S coef = bc[j];
            const bool xu = e < nxu;
            lrz[j] = coef * (xu ? rzv[j] : rt);
            if (DR) ld[j] = coef * (xu ? adz[j] : tdz);
            // w / alpha = eta / alpha + (L (2 z+ - z))_e
            y[j] = soc_shift(be[j] * ial + coef * (xu ? qzv[j] : qt), e, nb);
          }
        }
        soc_moreau<S, J>(y, nb, al, lane, o);
        S tau_part = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < nb) {
            out[er + e] = o[j];
            dual_stat<S, true, DR>(nacc, ial, be[j], o[j], lrz[j], bde[j], ld[j]);
            const S re = be[j] - o[j];
            if (e < nxu) lt[j] += bc[j] * re;
            else tau_part += re;
          }
        }
        tau_part = two_lanes_sum(tau_part, nxu & 31, (nxu + 1) & 31);   // the two tau rows
        if (lane == 0) primal_stat<S, DR>(nacc, ial, rt, tdz, S(0.5) * tau_part);
      }
      if (c >= p.nl) {  // leaf block of c: box on x^c, SOC on (Q_N^1/2 x^c, s^c / 2, s^c / 2)
        const int64_t ef = (jc == 0 ? D.es_c0 : __ldg(&p.desc[c].es)) - 2 * nx;
        const int64_t zxc = __ldg(&p.desc[c].zx);
        const int64_t zsc = z2 + 3 * m + 1 + jc;
        const S sz = z[zsc], szp = zp[zsc], sdz = DR ? dz[zsc] : S(0);
        const S rs_ = sz - szp, qs_ = szp - rs_;
        S rx[J], qx[J], xdz[J], ltx[J];
        {
          S xz[J], xzp[J], fe[J], fde[J], flo[J], fhi[J];
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const int e = lane + 32 * j;
            xz[j] = xzp[j] = xdz[j] = ltx[j] = fe[j] = fde[j] = flo[j] = fhi[j] = S(0);
            if (e < nx) {
              xz[j] = z[zxc + e];
              xzp[j] = zp[zxc + e];
              if (DR) xdz[j] = dz[zxc + e];
              fe[j] = eta[ef + e];
              if (DR) fde[j] = deta[ef + e];
              flo[j] = p.xlo[(int64_t)c * nx + e];
              fhi[j] = p.xhi[(int64_t)c * nx + e];
            }
          }
#pragma unroll
          for (int j = 0; j < J; ++j) {
            const int e = lane + 32 * j;
            rx[j] = xz[j] - xzp[j];
            qx[j] = xzp[j] - rx[j];
            if (e < nx) {
              const S w = fe[j] + al * qx[j];
              const S o = w - al * clampv(w * ial, flo[j], fhi[j]);
              out[ef + e] = o;
              dual_stat<S, true, DR>(nacc, ial, fe[j], o, rx[j], fde[j], xdz[j]);
              ltx[j] = fe[j] - o;
            }
          }
        }
        const int dim = nx + 2;
        const int64_t es = ef + nx;
        S y[J], lrz[J], ld[J], ev[J], dev[J], qn[J], o[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          y[j] = lrz[j] = ld[j] = ev[j] = dev[j] = qn[j] = S(0);
          if (e < dim) {
            const bool xr = e < nx;
            const S coef = xr ? p.qns[(int64_t)c * nx + e] : S(0.5);
            ev[j] = eta[es + e];
            lrz[j] = coef * (xr ? rx[j] : rs_);
            if (DR) {
              dev[j] = deta[es + e];
              ld[j] = coef * (xr ? xdz[j] : sdz);
            }
            y[j] = soc_shift(ev[j] * ial + coef * (xr ? qx[j] : qs_), e, dim);
            qn[j] = coef;
          }
        }
        soc_moreau<S, J>(y, dim, al, lane, o);
        S s_part = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < dim) {
            out[es + e] = o[j];
            dual_stat<S, true, DR>(nacc, ial, ev[j], o[j], lrz[j], dev[j], ld[j]);
            const S re = ev[j] - o[j];
            if (e < nx) ltx[j] += qn[j] * re;
            else s_part += re;
          }
        }
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (lane + 32 * j < nx) primal_stat<S, DR>(nacc, ial, rx[j], xdz[j], ltx[j]);
        s_part = two_lanes_sum(s_part, nx & 31, (nx + 1) & 31);   // the two s rows
        if (lane == 0) primal_stat<S, DR>(nacc, ial, rs_, sdz, S(0.5) * s_part);
      }
    }
    // ---- primal statistics at x^k, u^k
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (lane + 32 * j < nxu) primal_stat<S, DR>(nacc, ial, rzv[j], adz[j], lt[j]);
    // ---- the s - b'y row of k (b = (p^children, 0, 1)), then the y rows
    if (warp_y) {
      S bs = pr0 * yz0, bsp = pr0 * yzp0, bsd = DR ? pr0 * yd0 : S(0);
      for (int jj = lane + 32; jj < m; jj += 32) {  // nodes with more than 32 children
        const S pj = p.prob[c0 + jj];
        bs += pj * z[z2 + jj];
        bsp += pj * zp[z2 + jj];
        if (DR) bsd += pj * dz[z2 + jj];
      }
      bs = lanes_sum(bs, m);   // lanes < m hold the children's terms
      bsp = lanes_sum(bsp, m);
      if (DR) bsd = lanes_sum(bsd, m);
      const S Lz = sk - (bs + y3), Lzp = skp - (bsp + y3p), Ld = DR ? skd - (bsd + y3d) : S(0);
      const S w = dual_w<S, DM_DUAL>(al, esb, Lz, Lzp);
      const S o = vmin(w, S(0));
      const S re_sb = esb - o;
      if (lane == 0) {
        out[ie_sb] = o;
        dual_stat<S, true, DR>(nacc, ial, esb, o, Lz - Lzp, desb, Ld);
        primal_stat<S, DR>(nacc, ial, sk - skp, skd, re_sb);   // s^k (s^0 at the root)
      }
      auto yrow = [&](int e, S yz, S yzp, S yd, S ye, S yde) {
        const S yw = dual_w<S, DM_DUAL>(al, ye, yz, yzp);
        const S yo = e < 2 * m ? vmin(yw, S(0)) : S(0);
        out[el + e] = yo;
        dual_stat<S, true, DR>(nacc, ial, ye, yo, yz - yzp, yde, yd);
        const S bl = e < m ? p.prob[c0 + e] : (e < 2 * m ? S(0) : S(1));
        primal_stat<S, DR>(nacc, ial, yz - yzp, yd, (ye - yo) - bl * re_sb);
      };
      if (lane < 2 * m + 1) yrow(lane, yz0, yzp0, yd0, ye0, yde0);
      for (int e = lane + 32; e < 2 * m + 1; e += 32)
        yrow(e, z[z2 + e], zp[z2 + e], DR ? dz[z2 + e] : S(0), eta[el + e], DR ? deta[el + e] : S(0));
    }
    nacc.node_done(acc);
  }
  for (int64_t base = (int64_t)kc0 + 32 * (int64_t)gw; base < p.nl; base += 32 * (int64_t)nw) {
    if (base + lane < p.nl) dual_y_chain<S, DR>(p, (int)(base + lane), z, zp, eta, out, dz, deta, nacc);
    nacc.node_done(acc);
  }
  nacc.flush(acc);
  block_stats_store<sizeof(S) == 4>(acc, partials, bid);
}


// Sums (maxima for xi) of the per-block partial statistics of the dual and
// primal kernels; one block, fixed order (deterministic).
// (any block of 32..256 threads: warp w reduces statistics w, w + warps, ..)
static __device__ __forceinline__ void reduce_stats_body(const double* __restrict__ pd, int nd,
                                                         const double* __restrict__ pp, int np,
                                                         double* __restrict__ out,
                                                         const int32_t* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int i = threadIdx.x >> 5; i < 8; i += nwarps) {
    const bool mx = (i == ST_XIP || i == ST_XID);
    double v = 0.0;
    for (int b = lane; b < nd; b += 32) v = mx ? fmax(v, pd[(int64_t)b * 8 + i]) : v + pd[(int64_t)b * 8 + i];
    for (int b = lane; b < np; b += 32) v = mx ? fmax(v, pp[(int64_t)b * 8 + i]) : v + pp[(int64_t)b * 8 + i];
    v = mx ? warp_max(v) : warp_sum(v);
    if (lane == 0) red[i] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) out[threadIdx.x] = red[threadIdx.x];
}

}  // namespace spock
