// Warp-per-node vector kernels of the CP operator T:
//   k_prep   zbar = z - alpha L* eta; s^0 - alpha; proj_S2 on z_2; the (x, u)
//            part goes to the Riccati scratch (prox of f, Sec. "Proximal
//            operator of f", Sec. "Projection on S2").
//   k_dual   eta+ = prox_{alpha g*}(eta + alpha L (2 z+ - z)) with the cone
//            projections of Eq. (S3-def); optional residual statistics
//            (Sec. "The Chambolle-Pock method", Algorithm 3).  Also L z
//            and prox_{alpha g*}(eta) alone for the operator-level ABI.
//   k_primal L* eta, or the primal residual statistics (xi_p, ||r_z||^2).
// L and its adjoint are never stored: each entry of eta = L z is a sum over
// the node's own variables and its ancestor's (definition of L).
#include "kernels.cuh"
#include "spock_internal.h"

namespace spock {

enum DualMode : int { DM_APPLY_L = 0, DM_PROXG = 1, DM_DUAL = 2 };
enum PrimalMode : int { PM_APPLY_LT = 0, PM_STATS = 1 };

// ---------------------------------------------------------------------------
// k_prep
// ---------------------------------------------------------------------------
template <typename S>
__global__ void __launch_bounds__(128) k_prep(KP<S> p, const S* __restrict__ z,
                                              const S* __restrict__ eta, S* __restrict__ zo) {
  if (p.skip && *p.skip) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const S al = p.alpha;
  const int nx = p.nx, nu = p.nu;
  for (int k = gw; k < p.n; k += nw) {
    const NodeDesc D = p.desc[k];
    if (k < p.nl) {
      const int m = D.m, c0 = D.c0;
      const int64_t el = D.enl, ex = el + 2 * m + 2, eu = ex + nx, z2 = D.zz2;
      for (int r = lane; r < nx; r += 32) {
        S acc = eta[ex + r];
        for (int j = 0; j < m; ++j) acc += p.qs[(int64_t)(c0 + j) * nx + r] * eta[p.desc[c0 + j].enr + r];
        p.xbar[(int64_t)k * p.xs + r] = z[D.zx + r] - al * acc;
      }
      for (int r = lane; r < nu; r += 32) {
        S acc = eta[eu + r];
        for (int j = 0; j < m; ++j) acc += p.rs[(int64_t)(c0 + j) * nu + r] * eta[p.desc[c0 + j].enr + nx + r];
        p.ubar[(int64_t)k * p.us + r] = z[D.zu + r] - al * acc;
      }
      // z_2 block: zbar = z - alpha L* eta, then projection on ker [E^T, -I, -I]
      // with (M M^T)^-1 = (I - 11^T / (c + m)) / c, c = a^2 + 3 (Sherman-Morrison).
      const S sb = eta[el + 2 * m + 1];
      const S a = p.av[k];
      const S cc = a * a + S(3);
      const S y3 = z[z2 + 2 * m] - al * (eta[el + 2 * m] - sb);
      auto bars = [&](int j, S& y1, S& y2, S& ta, S& sv) {
        const int c = c0 + j;
        const NodeDesc& Dc = p.desc[c];
        const int64_t er = Dc.enr, es = Dc.es;
        y1 = z[z2 + j] - al * (eta[el + j] - p.prob[c] * sb);
        y2 = z[z2 + m + j] - al * eta[el + m + j];
        ta = z[z2 + 2 * m + 1 + j] - al * S(0.5) * (eta[er + nx + nu] + eta[er + nx + nu + 1]);
        const S ls = (c < p.nl) ? eta[es] : S(0.5) * (eta[es] + eta[es + 1]);
        sv = z[z2 + 3 * m + 1 + j] - al * ls;
      };
      S sumMw = 0;
      for (int j = lane; j < m; j += 32) {
        S y1, y2, ta, sv;
        bars(j, y1, y2, ta, sv);
        sumMw += a * y1 - y2 + y3 - ta - sv;
      }
      sumMw = warp_sum(sumMw);
      S sumlam = 0;
      for (int j = lane; j < m; j += 32) {
        S y1, y2, ta, sv;
        bars(j, y1, y2, ta, sv);
        const S Mw = a * y1 - y2 + y3 - ta - sv;
        const S lam = (Mw - sumMw / (cc + S(m))) / cc;
        zo[z2 + j] = y1 - a * lam;
        zo[z2 + m + j] = y2 + lam;
        zo[z2 + 2 * m + 1 + j] = ta + lam;
        zo[z2 + 3 * m + 1 + j] = sv + lam;
        sumlam += lam;
      }
      sumlam = warp_sum(sumlam);
      if (lane == 0) {
        zo[z2 + 2 * m] = y3 - sumlam;
        if (k == 0) zo[0] = (z[0] - al * sb) - al;   // prox of alpha * s^0
      }
    } else {
      const int64_t ef = D.elf;
      for (int r = lane; r < nx; r += 32)
        p.xbar[(int64_t)k * p.xs + r] =
            z[D.zx + r] - al * (eta[ef + r] + p.qns[(int64_t)k * nx + r] * eta[ef + nx + r]);
    }
  }
}

// ---------------------------------------------------------------------------
// k_dual
// ---------------------------------------------------------------------------
// Per entry of eta: the value of the L row at z (Lz), at z+ (Lzp) and at the
// direction (Ld).  For DM_DUAL, w = eta + alpha (2 Lzp - Lz) and the
// residual row of L is L r_z = Lz - Lzp.

template <typename S, int MODE, bool STATS, bool DIR>
__device__ __forceinline__ void dual_emit(const KP<S>& p, NodeAcc<S>& acc, const S* __restrict__ eta,
                                          S* __restrict__ out, const S* __restrict__ deta,
                                          int64_t ie, S Lz, S Lzp, S Ld, S outv) {
  out[ie] = outv;
  if (MODE == DM_DUAL && STATS) {
    const S re = eta[ie] - outv;
    const S lrz = Lz - Lzp;
    acc.s[ST_RE2] += re * re;
    acc.s[ST_RE_LRZ] += re * lrz;
    acc.s[ST_XID] = fmax(acc.s[ST_XID], fabs(re * p.inv_alpha - lrz));
    if (DIR) {
      const S de = deta[ie];
      acc.s[ST_RD] += re * de;
      acc.s[ST_LRZ_DE] += lrz * de;
      acc.s[ST_RE_LDZ] += re * Ld;
    }
  }
}

template <typename S, int MODE>
__device__ __forceinline__ S dual_w(const KP<S>& p, const S* __restrict__ eta, int64_t ie, S Lz, S Lzp) {
  if (MODE == DM_APPLY_L) return Lz;
  if (MODE == DM_PROXG) return eta[ie];
  return eta[ie] + p.alpha * (S(2) * Lzp - Lz);
}

// Translated SOC block: entries w[0..dim-1] already in the warp's buffer;
// projects w / alpha onto SOC + (0, .., 1/2, -1/2) and returns, per entry,
// w - alpha * projection.  SOC = {(v, t) : ||v|| <= t}, t the last entry.
template <typename S>
__device__ __forceinline__ void soc_prox(const S* wb, int dim, S ial, int lane, S& nv_out, S& t_out,
                                         S& scale_out) {
  S s2 = 0;
  for (int e = lane; e < dim - 1; e += 32) {
    S v = wb[e] * ial;
    if (e == dim - 2) v -= S(0.5);
    s2 += v * v;
  }
  s2 = warp_sum(s2);
  nv_out = sqrt(s2);
  t_out = wb[dim - 1] * ial + S(0.5);
  // one division per block: scale of the v part when projecting on the boundary
  scale_out = (nv_out > t_out && nv_out > -t_out) ? S(0.5) * (nv_out + t_out) / nv_out : S(0);
}

template <typename S>
__device__ __forceinline__ S soc_out(const S* wb, int dim, int e, S al, S ial, S nv, S t, S scale) {
  // projection of (v, t) = w / alpha - shift
  S v = wb[e] * ial;
  if (e == dim - 2) v -= S(0.5);
  if (e == dim - 1) v = t;
  S pr;
  if (nv <= t) {
    pr = v;
  } else if (nv <= -t) {
    pr = S(0);
  } else {
    pr = (e == dim - 1) ? S(0.5) * (nv + t) : scale * v;
  }
  if (e == dim - 2) pr += S(0.5);
  if (e == dim - 1) pr -= S(0.5);
  return wb[e] - al * pr;
}

template <typename S, int MODE, bool STATS, bool DIR>
__global__ void __launch_bounds__(128) k_dual(KP<S> p, const S* __restrict__ z, const S* __restrict__ zp,
                                              const S* __restrict__ eta, S* __restrict__ out,
                                              const S* __restrict__ dir, double* __restrict__ partials) {
  if (p.skip && *p.skip) return;
  __shared__ S wbuf[kWarpsPerBlock][kVecPad];
  __shared__ S lbuf[kWarpsPerBlock][kVecPad];   // L r_z of SOC rows (statistics)
  __shared__ S dbuf[kWarpsPerBlock][kVecPad];   // L d_z of SOC rows
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const S al = p.alpha;
  const int nx = p.nx, nu = p.nu;
  const S* dz = DIR ? dir : nullptr;
  const S* deta = DIR ? dir + p.n_z : nullptr;
  StatAcc acc;
  acc.zero();
  NodeAcc<S> nacc;
  nacc.zero();
  const S ial = p.inv_alpha;
  S* wb = wbuf[wl];
  S* lb = lbuf[wl];
  S* db = dbuf[wl];
  auto row = [&](int64_t zi, S coef, S& Lz, S& Lzp, S& Ld) {
    if (MODE == DM_PROXG) {  // no z in this mode
      Lz = Lzp = Ld = S(0);
      return;
    }
    Lz = coef * z[zi];
    Lzp = (MODE == DM_DUAL) ? coef * zp[zi] : S(0);
    Ld = DIR ? coef * dz[zi] : S(0);
  };
  for (int k = gw; k < p.n; k += nw) {
    const NodeDesc D = p.desc[k];
    // ---- nonleaf block (y, s - b'y, x, u)
    if (k < p.nl) {
      const int m = D.m, c0 = D.c0;
      const int64_t el = D.enl, z2 = D.zz2;
      for (int e = lane; e < 2 * m + 1; e += 32) {
        S Lz, Lzp, Ld;
        row(z2 + e, S(1), Lz, Lzp, Ld);
        const S w = dual_w<S, MODE>(p, eta, el + e, Lz, Lzp);
        const S o = (MODE == DM_APPLY_L) ? w : (e < 2 * m ? fmin(w, S(0)) : S(0));
        dual_emit<S, MODE, STATS, DIR>(p, nacc, eta, out, deta, el + e, Lz, Lzp, Ld, o);
      }
      {  // s^k - b^T y^k, b = (p^children, 0, 1)
        S bz = 0, bzp = 0, bd = 0;
        for (int j = lane; j < m && MODE != DM_PROXG; j += 32) {
          const S pj = p.prob[c0 + j];
          bz += pj * z[z2 + j];
          if (MODE == DM_DUAL) bzp += pj * zp[z2 + j];
          if (DIR) bd += pj * dz[z2 + j];
        }
        bz = warp_sum(bz);
        if (MODE == DM_DUAL) bzp = warp_sum(bzp);
        if (DIR) bd = warp_sum(bd);
        if (lane == 0) {
          const int64_t si = D.zs;
          const S Lz = (MODE == DM_PROXG) ? S(0) : z[si] - (bz + z[z2 + 2 * m]);
          const S Lzp = (MODE == DM_DUAL) ? zp[si] - (bzp + zp[z2 + 2 * m]) : S(0);
          const S Ld = DIR ? dz[si] - (bd + dz[z2 + 2 * m]) : S(0);
          const int64_t ie = el + 2 * m + 1;
          const S w = dual_w<S, MODE>(p, eta, ie, Lz, Lzp);
          const S o = (MODE == DM_APPLY_L) ? w : fmin(w, S(0));
          dual_emit<S, MODE, STATS, DIR>(p, nacc, eta, out, deta, ie, Lz, Lzp, Ld, o);
        }
      }
      const int64_t ex = el + 2 * m + 2;
      for (int e = lane; e < nx + nu; e += 32) {
        S Lz, Lzp, Ld, lo, hi;
        if (e < nx) {
          row(D.zx + e, S(1), Lz, Lzp, Ld);
          lo = p.xlo[(int64_t)k * nx + e];
          hi = p.xhi[(int64_t)k * nx + e];
        } else {
          row(D.zu + (e - nx), S(1), Lz, Lzp, Ld);
          lo = p.ulo[(int64_t)k * nu + (e - nx)];
          hi = p.uhi[(int64_t)k * nu + (e - nx)];
        }
        const S w = dual_w<S, MODE>(p, eta, ex + e, Lz, Lzp);
        const S o = (MODE == DM_APPLY_L) ? w : w - al * clampv(w * ial, lo, hi);
        dual_emit<S, MODE, STATS, DIR>(p, nacc, eta, out, deta, ex + e, Lz, Lzp, Ld, o);
      }
    }
    // ---- nonroot block (Q^1/2 x^anc, R^1/2 u^anc, tau/2, tau/2)
    if (k > 0) {
      const int64_t er = D.enr;
      const int dim = nx + nu + 2;
      for (int e = lane; e < dim; e += 32) {
        S Lz, Lzp, Ld;
        if (e < nx) row(D.zxp + e, p.qs[(int64_t)k * nx + e], Lz, Lzp, Ld);
        else if (e < nx + nu) row(D.zup + (e - nx), p.rs[(int64_t)k * nu + (e - nx)], Lz, Lzp, Ld);
        else row(D.ztau, S(0.5), Lz, Lzp, Ld);
        wb[e] = dual_w<S, MODE>(p, eta, er + e, Lz, Lzp);
        lb[e] = Lz - Lzp;
        db[e] = Ld;
        if (MODE == DM_APPLY_L) out[er + e] = wb[e];
      }
      __syncwarp();
      if (MODE != DM_APPLY_L) {
        S nv, t, sc;
        soc_prox(wb, dim, ial, lane, nv, t, sc);
        for (int e = lane; e < dim; e += 32) {
          const S o = soc_out(wb, dim, e, al, ial, nv, t, sc);
          // Lz - Lzp = lb[e]; pass (lb, 0) so that dual_emit sees L r_z
          dual_emit<S, MODE, STATS, DIR>(p, nacc, eta, out, deta, er + e, lb[e], S(0), db[e], o);
        }
      }
      __syncwarp();
    }
    // ---- leaf block (x, Q_N^1/2 x, s/2, s/2)
    if (k >= p.nl) {
      const int64_t ef = D.elf;
      for (int e = lane; e < nx; e += 32) {
        S Lz, Lzp, Ld;
        row(D.zx + e, S(1), Lz, Lzp, Ld);
        const S w = dual_w<S, MODE>(p, eta, ef + e, Lz, Lzp);
        const S o = (MODE == DM_APPLY_L) ? w
                                         : w - al * clampv(w * ial, p.xlo[(int64_t)k * nx + e], p.xhi[(int64_t)k * nx + e]);
        dual_emit<S, MODE, STATS, DIR>(p, nacc, eta, out, deta, ef + e, Lz, Lzp, Ld, o);
      }
      const int dim = nx + 2;
      const int64_t es = ef + nx;
      for (int e = lane; e < dim; e += 32) {
        S Lz, Lzp, Ld;
        if (e < nx) row(D.zx + e, p.qns[(int64_t)k * nx + e], Lz, Lzp, Ld);
        else row(D.zs, S(0.5), Lz, Lzp, Ld);
        wb[e] = dual_w<S, MODE>(p, eta, es + e, Lz, Lzp);
        lb[e] = Lz - Lzp;
        db[e] = Ld;
        if (MODE == DM_APPLY_L) out[es + e] = wb[e];
      }
      __syncwarp();
      if (MODE != DM_APPLY_L) {
        S nv, t, sc;
        soc_prox(wb, dim, ial, lane, nv, t, sc);
        for (int e = lane; e < dim; e += 32) {
          const S o = soc_out(wb, dim, e, al, ial, nv, t, sc);
          dual_emit<S, MODE, STATS, DIR>(p, nacc, eta, out, deta, es + e, lb[e], S(0), db[e], o);
        }
      }
      __syncwarp();
    }
    if (MODE == DM_DUAL && STATS) nacc.flush(acc);
  }
  if (MODE == DM_DUAL && STATS) block_stats_store(acc, partials);
}

// ---------------------------------------------------------------------------
// k_primal: L* applied to E = eta (PM_APPLY_LT) or to r_eta = eta - eta+
// (PM_STATS, with r_z = z - z+ and optional direction).
// ---------------------------------------------------------------------------
template <typename S, int MODE, bool DIR>
__global__ void __launch_bounds__(128) k_primal(KP<S> p, const S* __restrict__ eta, const S* __restrict__ etap,
                                                const S* __restrict__ z, const S* __restrict__ zp,
                                                S* __restrict__ zout, const S* __restrict__ dir,
                                                double* __restrict__ partials) {
  if (p.skip && *p.skip) return;
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nx = p.nx, nu = p.nu;
  StatAcc acc;
  acc.zero();
  NodeAcc<S> nacc;
  nacc.zero();
  auto E = [&](int64_t i) -> S { return MODE == PM_APPLY_LT ? eta[i] : eta[i] - etap[i]; };
  auto emit = [&](int64_t zi, S lt) {
    if (MODE == PM_APPLY_LT) {
      zout[zi] = lt;
    } else {
      const S rz = z[zi] - zp[zi];
      nacc.s[ST_RZ2] += rz * rz;
      nacc.s[ST_XIP] = fmax(nacc.s[ST_XIP], fabs(rz * p.inv_alpha - lt));
      if (DIR) nacc.s[ST_RD] += rz * dir[zi];
    }
  };
  for (int k = gw; k < p.n; k += nw) {
    const NodeDesc D = p.desc[k];
    if (k < p.nl) {
      const int m = D.m, c0 = D.c0;
      const int64_t el = D.enl, ex = el + 2 * m + 2, eu = ex + nx, z2 = D.zz2;
      for (int r = lane; r < nx; r += 32) {
        S acc2 = E(ex + r);
        for (int j = 0; j < m; ++j) acc2 += p.qs[(int64_t)(c0 + j) * nx + r] * E(p.desc[c0 + j].enr + r);
        emit(D.zx + r, acc2);
      }
      for (int r = lane; r < nu; r += 32) {
        S acc2 = E(eu + r);
        for (int j = 0; j < m; ++j) acc2 += p.rs[(int64_t)(c0 + j) * nu + r] * E(p.desc[c0 + j].enr + nx + r);
        emit(D.zu + r, acc2);
      }
      const S sb = E(el + 2 * m + 1);
      for (int l = lane; l < 2 * m + 1; l += 32) {
        const S bl = l < m ? p.prob[c0 + l] : (l < 2 * m ? S(0) : S(1));
        emit(z2 + l, E(el + l) - bl * sb);
      }
      for (int j = lane; j < m; j += 32) {
        const int c = c0 + j;
        const NodeDesc& Dc = p.desc[c];
        const int64_t er = Dc.enr, es = Dc.es;
        emit(z2 + 2 * m + 1 + j, S(0.5) * (E(er + nx + nu) + E(er + nx + nu + 1)));
        emit(z2 + 3 * m + 1 + j, (c < p.nl) ? E(es) : S(0.5) * (E(es) + E(es + 1)));
      }
      if (k == 0 && lane == 0) emit(0, sb);
    } else {
      const int64_t ef = D.elf;
      for (int r = lane; r < nx; r += 32)
        emit(D.zx + r, E(ef + r) + p.qns[(int64_t)k * nx + r] * E(ef + nx + r));
    }
    if (MODE == PM_STATS) nacc.flush(acc);
  }
  if (MODE == PM_STATS) block_stats_store(acc, partials);
}

// Sums (maxima for xi) of the per-block partial statistics of the dual and
// primal kernels; one block, fixed order (deterministic).
__global__ void k_reduce_stats(const double* __restrict__ pd, int nd, const double* __restrict__ pp, int np,
                               double* __restrict__ out, const int32_t* __restrict__ skip) {
  if (skip && *skip) return;
  __shared__ double red[8][32];
  const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;  // 8 warps, one per statistic
  const bool mx = (i == ST_XIP || i == ST_XID);
  double v = 0.0;
  for (int b = lane; b < nd; b += 32) v = mx ? fmax(v, pd[(int64_t)b * 8 + i]) : v + pd[(int64_t)b * 8 + i];
  for (int b = lane; b < np; b += 32) v = mx ? fmax(v, pp[(int64_t)b * 8 + i]) : v + pp[(int64_t)b * 8 + i];
  v = mx ? warp_max(v) : warp_sum(v);
  if (lane == 0) red[i][0] = v;
  __syncthreads();
  if (threadIdx.x < 8) out[threadIdx.x] = red[threadIdx.x][0];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
inline int warp_grid(int n, int max_blocks) {
  int b = (n + kWarpsPerBlock - 1) / kWarpsPerBlock;
  return b < max_blocks ? (b > 0 ? b : 1) : max_blocks;
}

template <typename S>
void launch_prep(const KP<S>& p, const S* z, const S* eta, S* zo, int max_blocks, cudaStream_t st) {
  k_prep<S><<<warp_grid(p.n, max_blocks), 128, 0, st>>>(p, z, eta, zo);
}

template <typename S>
void launch_dual(const KP<S>& p, int mode, bool stats, const S* z, const S* zp, const S* eta, S* out,
                 const S* dir, double* partials, int grid, cudaStream_t st) {
  if (mode == DM_APPLY_L) {
    k_dual<S, DM_APPLY_L, false, false><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);
  } else if (mode == DM_PROXG) {
    k_dual<S, DM_PROXG, false, false><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);
  } else if (!stats) {
    k_dual<S, DM_DUAL, false, false><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);
  } else if (dir) {
    k_dual<S, DM_DUAL, true, true><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);
  } else {
    k_dual<S, DM_DUAL, true, false><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);
  }
}

template <typename S>
void launch_primal(const KP<S>& p, int mode, const S* eta, const S* etap, const S* z, const S* zp, S* zout,
                   const S* dir, double* partials, int grid, cudaStream_t st) {
  if (mode == PM_APPLY_LT) {
    k_primal<S, PM_APPLY_LT, false><<<grid, 128, 0, st>>>(p, eta, etap, z, zp, zout, dir, partials);
  } else if (dir) {
    k_primal<S, PM_STATS, true><<<grid, 128, 0, st>>>(p, eta, etap, z, zp, zout, dir, partials);
  } else {
    k_primal<S, PM_STATS, false><<<grid, 128, 0, st>>>(p, eta, etap, z, zp, zout, dir, partials);
  }
}

void launch_reduce_stats(const double* pd, int nd, const double* pp, int np, double* out, cudaStream_t st,
                         const int32_t* skip) {
  k_reduce_stats<<<1, 256, 0, st>>>(pd, nd, pp, np, out, skip);
}

template void launch_prep<double>(const KP<double>&, const double*, const double*, double*, int, cudaStream_t);
template void launch_prep<float>(const KP<float>&, const float*, const float*, float*, int, cudaStream_t);
template void launch_dual<double>(const KP<double>&, int, bool, const double*, const double*, const double*,
                                  double*, const double*, double*, int, cudaStream_t);
template void launch_dual<float>(const KP<float>&, int, bool, const float*, const float*, const float*, float*,
                                 const float*, double*, int, cudaStream_t);
template void launch_primal<double>(const KP<double>&, int, const double*, const double*, const double*,
                                    const double*, double*, const double*, double*, int, cudaStream_t);
template void launch_primal<float>(const KP<float>&, int, const float*, const float*, const float*, const float*,
                                   float*, const float*, double*, int, cudaStream_t);

}  // namespace spock
