// Vector kernels of T for the general form (spock_problem_create_general):
// polyhedral constraints Gamma_x x + Gamma_u u in C, Gamma_N x in C_N (Eq.
// (constraints)) and dense Q^1/2, R^1/2, Q_N^1/2 in L (definition of L).
// The same three uses as the box-form kernels of ops.cu:
//   k_lstar_g       L* eta, or the prox-f preparation zbar = z - alpha L* eta
//                   with proj_S2 on z_2 (Sec. "Proximal operator of f");
//   k_dual_g        L z, prox_{alpha g*}(eta), or the dual update without
//                   statistics;
//   k_dual_fused_g  the dual update with every residual statistic of
//                   Sec. "The Chambolle-Pock method" / Algorithm 3.
// Each row of L that reads (x^k, u^k) is now a dot product with a row of a
// per-node matrix, done as a warp matrix-vector product: the vector lives in
// the lanes' register slots (entry e at lane e % 32, slot e / 32), each
// column's entry is broadcast with a shuffle and every lane accumulates the
// rows it owns, reading the matrix column-major (lanes over rows: coalesced).
// The adjoint rows use the transposed copy of each matrix the same way.
// Risk measures are in the conic form of Sec. "Conic representation of risk
// measures": per nonleaf node k, y^k has ny_k rows, the row s^k - b^kT y^k
// reads all of them, (K^k)* = R^kp_+ x R^(ny - kp) in S3, and the projection
// on S2^k is the node's dense projector applied by the same warp
// matrix-vector product (AV@R without a given risk measure: the closed form).
// The cone projections of the cost epigraphs and the statistics are as in
// the box form.
#include "kernels.cuh"
#include "ops_body.cuh"
#include "spock_internal.h"

namespace spock {

// y[v][j] += sum_q M(e - r0, q) x[v][c0 + q] for the entries e = lane + 32 j
// in [r0, r0 + nrows), v < NV; M (nrows x ncols) column-major with leading
// dimension ld.  All lanes of the warp call it (the shuffles).  The next
// column's entries are loaded while the current column is applied (one
// column of lookahead: two loads per lane slot in flight).
template <typename S, int J, int NV, int NA>
__device__ __forceinline__ void wmv(const S* __restrict__ M, int ld, int nrows, int r0, int ncols, int c0,
                                    const S (&x)[NA][J], S (&y)[NA][J], int lane) {
  if (ncols <= 0) return;
  bool live[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int r = lane + 32 * j - r0;
    live[j] = r >= 0 && r < nrows;
  }
  auto load = [&](int q, S (&m)[J]) {
    const S* col = M + (int64_t)q * ld - r0;
#pragma unroll
    for (int j = 0; j < J; ++j) m[j] = live[j] ? __ldg(col + lane + 32 * j) : S(0);
  };
  S cur[J], nxt[J];
  load(0, cur);
  for (int q = 0; q < ncols; ++q) {   // warp-uniform bounds
    if (q + 1 < ncols) load(q + 1, nxt);
    const int cq = c0 + q;
    S xv[NV];
#pragma unroll
    for (int js = 0; js < J; ++js) {
      if (js == (cq >> 5)) {
#pragma unroll
        for (int v = 0; v < NV; ++v) xv[v] = __shfl_sync(kFull, x[v][js], cq & 31);
      }
    }
#pragma unroll
    for (int j = 0; j < J; ++j)
#pragma unroll
      for (int v = 0; v < NV; ++v) y[v][j] = fma(cur[j], xv[v], y[v][j]);
#pragma unroll
    for (int j = 0; j < J; ++j) cur[j] = nxt[j];
  }
}

template <typename S, int J, int NA>
__device__ __forceinline__ void zero_slots(S (&y)[NA][J]) {
#pragma unroll
  for (int v = 0; v < NA; ++v)
#pragma unroll
    for (int j = 0; j < J; ++j) y[v][j] = S(0);
}

// Per-node matrix pointers of the general form.
template <typename S>
struct GenMats {
  const KP<S>& p;
  __device__ const S* gc(int k) const { return p.gc + (int64_t)k * (p.nx + p.nu) * p.ldc; }
  __device__ const S* gt(int k) const { return p.gt + (int64_t)k * p.nc * p.ldxu; }
  __device__ const S* fqc(int k) const { return p.fqc + (int64_t)k * p.nx * p.ldx; }
  __device__ const S* fqt(int k) const { return p.fqt + (int64_t)k * p.nx * p.ldx; }
  __device__ const S* frc(int k) const { return p.frc + (int64_t)k * p.nu * p.ldu; }
  __device__ const S* frt(int k) const { return p.frt + (int64_t)k * p.nu * p.ldu; }
  __device__ const S* fnc(int k) const { return p.fnc + (int64_t)k * p.nx * p.ldx; }
  __device__ const S* fnt(int k) const { return p.fnt + (int64_t)k * p.nx * p.ldx; }
  __device__ const S* gnc(int k) const { return p.gnc + (int64_t)k * p.nx * p.ldcn; }
  __device__ const S* gnt(int k) const { return p.gnt + (int64_t)k * p.ncN * p.ldx; }
  __device__ S lo(int k, int r) const { return p.clo[(int64_t)k * p.cst + r]; }
  __device__ S hi(int k, int r) const { return p.chi[(int64_t)k * p.cst + r]; }
};

// ---------------------------------------------------------------------------
// L* (LS_APPLY) and the prox-f preparation (LS_PREP), warp per node
// ---------------------------------------------------------------------------
template <typename S, int MODE, int J>
__global__ void __launch_bounds__(128) k_lstar_g(KP<S> p, const S* __restrict__ eta, const S* __restrict__ z,
                                                 S* __restrict__ zo) {
  if (p.skip && *p.skip) return;
  const GenMats<S> G{p};
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nx = p.nx, nu = p.nu, nxu = nx + nu;
  const S al = p.alpha;
  for (int k = gw; k < p.n; k += nw) {
    const NodeF D = node_fields(desc_word(p.desc, k, lane));
    S lt[1][J], w[1][J];
    zero_slots(lt);
    if (k < p.nl) {
      const int m = D.m, c0 = D.c0;
      // Gamma^T w over the nc constraint rows
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int r = lane + 32 * j;
        w[0][j] = r < p.nc ? eta[D.enl + p.rny[k] + 1 + r] : S(0);
      }
      wmv<S, J, 1>(G.gt(k), p.ldxu, nxu, 0, p.nc, 0, w, lt, lane);
      // (Q^c 1/2)^T and (R^c 1/2)^T over each child's nonroot rows
      for (int c = c0; c < c0 + m; ++c) {
        const int64_t er = __ldg(&p.desc[c].enr);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          w[0][j] = e < nxu ? eta[er + e] : S(0);
        }
        wmv<S, J, 1>(G.fqt(c), p.ldx, nx, 0, nx, 0, w, lt, lane);
        wmv<S, J, 1>(G.frt(c), p.ldu, nu, nx, nu, nx, w, lt, lane);
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        if (e < nxu) {
          const int64_t zi = e < nx ? D.zx + e : D.zu + (e - nx);
          if (MODE == LS_PREP) {
            const S v = z[zi] - al * lt[0][j];
            if (e < nx) p.xbar[(int64_t)k * p.xs + e] = v;
            else p.ubar[(int64_t)k * p.us + (e - nx)] = v;
          } else {
            zo[zi] = lt[0][j];
          }
        }
      }
      // z_2 block: the rows of the risk constraints, y^k (ny rows), tau^[k], s^[k]
      const int ny = p.rny[k];
      const S* __restrict__ bk = p.rb + p.rboff[k];
      const int64_t el = D.enl, z2 = D.zz2;
      const S sb = eta[el + ny];
      auto child_rows = [&](int jc, S& tau_l, S& s_l) {
        const int c = c0 + jc;
        const int64_t er = __ldg(&p.desc[c].enr), es = __ldg(&p.desc[c].es);
        tau_l = S(0.5) * (eta[er + nxu] + eta[er + nxu + 1]);
        s_l = (c < p.nl) ? eta[es] : S(0.5) * (eta[es] + eta[es + 1]);
      };
      if (MODE != LS_PREP) {
        for (int l = lane; l < ny; l += 32) zo[z2 + l] = eta[el + l] - bk[l] * sb;
        for (int jc = lane; jc < m; jc += 32) {
          S tl, sl;
          child_rows(jc, tl, sl);
          zo[z2 + ny + jc] = tl;
          zo[z2 + ny + m + jc] = sl;
        }
        if (k == 0 && lane == 0) zo[0] = sb;
      } else if (p.rpoff[k] < 0) {
        // AV@R: zbar on z_2, then the projection on ker [E^T, -I, -I] by the
        // closed form (M M^T)^-1 = (I - 11^T / (c + m)) / c, c = a^2 + 3
        const S a = p.av[k];
        const S y3 = z[z2 + 2 * m] - al * (eta[el + 2 * m] - sb);
        auto bars = [&](int jc, S& y1, S& y2, S& ta, S& sv) {
          S tl, sl;
          child_rows(jc, tl, sl);
          y1 = z[z2 + jc] - al * (eta[el + jc] - bk[jc] * sb);
          y2 = z[z2 + m + jc] - al * eta[el + m + jc];
          ta = z[z2 + 2 * m + 1 + jc] - al * tl;
          sv = z[z2 + 3 * m + 1 + jc] - al * sl;
        };
        S sumMw = 0;
        for (int jc = lane; jc < m; jc += 32) {
          S b1, b2, bt, bs;
          bars(jc, b1, b2, bt, bs);
          sumMw += a * b1 - b2 + y3 - bt - bs;
        }
        sumMw = warp_sum(sumMw);
        const S inv_cc = p.s2inv[2 * (int64_t)k];
        const S shift = sumMw * p.s2inv[2 * (int64_t)k + 1];
        S sumlam = 0;
        for (int jc = lane; jc < m; jc += 32) {
          S b1, b2, bt, bs;
          bars(jc, b1, b2, bt, bs);
          const S lam = (a * b1 - b2 + y3 - bt - bs - shift) * inv_cc;
          zo[z2 + jc] = b1 - a * lam;
          zo[z2 + m + jc] = b2 + lam;
          zo[z2 + 2 * m + 1 + jc] = bt + lam;
          zo[z2 + 3 * m + 1 + jc] = bs + lam;
          sumlam += lam;
        }
        sumlam = warp_sum(sumlam);
        if (lane == 0) {
          zo[z2 + 2 * m] = y3 - sumlam;
          if (k == 0) zo[0] = (z[0] - al * sb) - al;   // prox of alpha * s^0
        }
      } else {
        // zbar = z - alpha L* eta on z_2, then the projection on
        // S2^k = ker [[E^T, -I, -I], [F^T, 0, 0]] by the node's projector
        const int nz2 = ny + 2 * m;
        S zb[1][J], o[1][J];
        zero_slots(o);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          zb[0][j] = S(0);
          if (e < ny) {
            zb[0][j] = z[z2 + e] - al * (eta[el + e] - bk[e] * sb);
          } else if (e < nz2) {
            const int jc = (e - ny) % m;
            S tl, sl;
            child_rows(jc, tl, sl);
            zb[0][j] = z[z2 + e] - al * (e < ny + m ? tl : sl);
          }
        }
        wmv<S, J, 1>(p.rpi + p.rpoff[k], nz2, nz2, 0, nz2, 0, zb, o, lane);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          if (e < nz2) zo[z2 + e] = o[0][j];
        }
        if (k == 0 && lane == 0) zo[0] = (z[0] - al * sb) - al;   // prox of alpha * s^0
      }
    } else {
      // leaf: Gamma_N^T w + (Q_N^1/2)^T w
      const int64_t ef = D.elf;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int r = lane + 32 * j;
        w[0][j] = r < p.ncN ? eta[ef + r] : S(0);
      }
      wmv<S, J, 1>(G.gnt(k), p.ldx, nx, 0, p.ncN, 0, w, lt, lane);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        w[0][j] = e < nx ? eta[ef + p.ncN + e] : S(0);
      }
      wmv<S, J, 1>(G.fnt(k), p.ldx, nx, 0, nx, 0, w, lt, lane);
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        if (e < nx) {
          if (MODE == LS_PREP) p.xbar[(int64_t)k * p.xs + e] = z[D.zx + e] - al * lt[0][j];
          else zo[D.zx + e] = lt[0][j];
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// L z (DM_APPLY_L), prox_{alpha g*}(eta) (DM_PROXG), the dual update without
// statistics (DM_DUAL); warp per node: its constraint rows, its nonroot block
// and (leaves) its leaf block
// ---------------------------------------------------------------------------
template <typename S, int MODE, int J>
__global__ void __launch_bounds__(128) k_dual_g(KP<S> p, const S* __restrict__ z, const S* __restrict__ zp,
                                                const S* __restrict__ eta, S* __restrict__ out) {
  if (p.skip && *p.skip) return;
  constexpr bool HZ = MODE != DM_PROXG;
  constexpr bool HZP = MODE == DM_DUAL;
  constexpr bool HE = MODE != DM_APPLY_L;
  const GenMats<S> G{p};
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const S al = p.alpha, ial = p.inv_alpha;
  const int nx = p.nx, nu = p.nu, nxu = nx + nu;
  for (int k = gw; k < p.n; k += nw) {
    const NodeF D = node_fields(desc_word(p.desc, k, lane));
    const bool nonleaf = k < p.nl;
    const int na = nonleaf ? nxu : nx;
    // own (x, u) at z and z+ (entries e < na)
    S a[2][J], v[2][J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int e = lane + 32 * j;
      a[0][j] = a[1][j] = S(0);
      if (e < na) {
        const int64_t zi = e < nx ? D.zx + e : D.zu + (e - nx);
        if (HZ) a[0][j] = z[zi];
        if (HZP) a[1][j] = zp[zi];
      }
    }
    // ---- constraint rows: Gamma (x, u) in C (nonleaf) or Gamma_N x in C_N (leaf)
    {
      const int nr = nonleaf ? p.nc : p.ncN;
      const int64_t ea = nonleaf ? D.enl + p.rny[k] + 1 : D.elf;
      zero_slots(v);
      if (MODE != DM_PROXG) {
        if (nonleaf) wmv<S, J, HZP ? 2 : 1>(G.gc(k), p.ldc, nr, 0, nxu, 0, a, v, lane);
        else wmv<S, J, HZP ? 2 : 1>(G.gnc(k), p.ldcn, nr, 0, nx, 0, a, v, lane);
      }
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int r = lane + 32 * j;
        if (r < nr) {
          const S w = dual_w<S, MODE>(al, HE ? eta[ea + r] : S(0), v[0][j], v[1][j]);
          out[ea + r] = (MODE == DM_APPLY_L) ? w : w - al * clampv(w * ial, G.lo(k, r), G.hi(k, r));
        }
      }
    }
    // ---- nonroot block: SOC on (Q^1/2 x^anc, R^1/2 u^anc, tau/2, tau/2)
    if (k > 0) {
      const int nb = nxu + 2;
      S b[2][J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        b[0][j] = b[1][j] = S(0);
        if (e < nxu && MODE != DM_PROXG) {
          const int64_t zi = e < nx ? D.zxp + e : D.zup + (e - nx);
          if (HZ) b[0][j] = z[zi];
          if (HZP) b[1][j] = zp[zi];
        }
      }
      zero_slots(v);
      if (MODE != DM_PROXG) {
        wmv<S, J, HZP ? 2 : 1>(G.fqc(k), p.ldx, nx, 0, nx, 0, b, v, lane);
        wmv<S, J, HZP ? 2 : 1>(G.frc(k), p.ldu, nu, nx, nu, nx, b, v, lane);
      }
      const S tz = HZ ? z[D.ztau] : S(0), tzp = HZP ? zp[D.ztau] : S(0);
      S w[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        const bool tr = e == nxu || e == nxu + 1;
        const S Lz = tr ? S(0.5) * tz : v[0][j], Lzp = tr ? S(0.5) * tzp : v[1][j];
        w[j] = e < nb ? dual_w<S, MODE>(al, HE ? eta[D.enr + e] : S(0), Lz, Lzp) : S(0);
      }
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
        for (int j = 0; j < J; ++j)
          if (lane + 32 * j < nb) out[D.enr + lane + 32 * j] = o[j];
      }
    }
    if (nonleaf) {
      // ---- y rows (prox of (K^k)*: R^kp_+ x R^(ny - kp)) and the s - b'y row
      const int ny = p.rny[k], kp = p.rkp[k];
      const S* __restrict__ bk = p.rb + p.rboff[k];
      const int64_t el = D.enl, z2 = D.zz2;
      S bs = 0, bsp = 0;
      for (int e = lane; e < ny; e += 32) {
        const S Lz = HZ ? z[z2 + e] : S(0);
        const S Lzp = HZP ? zp[z2 + e] : S(0);
        const S w = dual_w<S, MODE>(al, HE ? eta[el + e] : S(0), Lz, Lzp);
        out[el + e] = (MODE == DM_APPLY_L) ? w : (e < kp ? vmin(w, S(0)) : S(0));
        bs += bk[e] * Lz;
        bsp += bk[e] * Lzp;
      }
      bs = warp_sum(bs);
      bsp = warp_sum(bsp);
      if (lane == 0) {
        const int64_t ie = el + ny;
        const S sz = HZ ? z[D.zs] : S(0), szp = HZP ? zp[D.zs] : S(0);
        const S Lz = sz - bs, Lzp = HZP ? szp - bsp : S(0);
        const S w = dual_w<S, MODE>(al, HE ? eta[ie] : S(0), Lz, Lzp);
        out[ie] = (MODE == DM_APPLY_L) ? w : vmin(w, S(0));
      }
    } else {
      // ---- leaf SOC on (Q_N^1/2 x, s/2, s/2)
      const int dim = nx + 2;
      const int64_t es = D.elf + p.ncN;
      zero_slots(v);
      if (MODE != DM_PROXG) wmv<S, J, HZP ? 2 : 1>(G.fnc(k), p.ldx, nx, 0, nx, 0, a, v, lane);
      const S sz = HZ ? z[D.zs] : S(0), szp = HZP ? zp[D.zs] : S(0);
      S w[J];
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int e = lane + 32 * j;
        const bool sr = e >= nx;
        const S Lz = sr ? S(0.5) * sz : v[0][j], Lzp = sr ? S(0.5) * szp : v[1][j];
        w[j] = e < dim ? dual_w<S, MODE>(al, HE ? eta[es + e] : S(0), Lz, Lzp) : S(0);
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
        for (int j = 0; j < J; ++j)
          if (lane + 32 * j < dim) out[es + lane + 32 * j] = o[j];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The dual update with every residual statistic; one warp per NONLEAF node k
// owns the eta rows that read k's variables (k's nonleaf block, each child's
// nonroot block, each leaf child's leaf block), so it also has (L* r_eta) at
// x^k, u^k and at its leaf children's x, s (primal statistics).
// ---------------------------------------------------------------------------
template <typename S, bool DR, int J>
__global__ void __launch_bounds__(128) k_dual_fused_g(KP<S> p, const S* __restrict__ z, const S* __restrict__ zp,
                                                      const S* __restrict__ eta, S* __restrict__ out,
                                                      const S* __restrict__ dir, double* __restrict__ partials) {
  if (p.skip && *p.skip) return;
  constexpr int NV = DR ? 3 : 2;   // the rows at q_z = 2 z+ - z, r_z = z - z+ and the direction d_z
  const GenMats<S> G{p};
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const S al = p.alpha, ial = p.inv_alpha;
  const int nx = p.nx, nu = p.nu, nxu = nx + nu, nb = nxu + 2;
  const S* dz = DR ? dir : nullptr;
  const S* deta = DR ? dir + p.n_z : nullptr;
  StatAcc acc;
  acc.zero();
  NodeAcc<S> nacc;
  nacc.zero();
  for (int k = gw; k < p.nl; k += nw) {
    const NodeF D = node_fields(desc_word(p.desc, k, lane));
    const int m = D.m, c0 = D.c0;
    const int ny = p.rny[k], kp = p.rkp[k];
    const S* __restrict__ bk = p.rb + p.rboff[k];
    const int64_t el = D.enl, ea = el + ny + 1, z2 = D.zz2;
    // own (x, u): zv[0] = q_z, zv[1] = r_z, zv[2] = d_z
    S zv[3][J], lt[1][J], v[3][J], re[1][J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int e = lane + 32 * j;
      zv[0][j] = zv[1][j] = zv[2][j] = lt[0][j] = S(0);
      if (e < nxu) {
        const int64_t zi = e < nx ? D.zx + e : D.zu + (e - nx);
        const S az = z[zi], azp = zp[zi];
        zv[1][j] = az - azp;
        zv[0][j] = azp - zv[1][j];
        if (DR) zv[2][j] = dz[zi];
      }
    }
    // ---- constraint rows of k
    zero_slots(v);
    wmv<S, J, NV>(G.gc(k), p.ldc, p.nc, 0, nxu, 0, zv, v, lane);
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int r = lane + 32 * j;
      re[0][j] = S(0);
      if (r < p.nc) {
        const S ae = eta[ea + r], ade = DR ? deta[ea + r] : S(0);
        const S w = ae + al * v[0][j];
        const S o = w - al * clampv(w * ial, G.lo(k, r), G.hi(k, r));
        out[ea + r] = o;
        dual_stat<S, true, DR>(nacc, ial, ae, o, v[1][j], ade, DR ? v[2][j] : S(0));
        re[0][j] = ae - o;
      }
    }
    wmv<S, J, 1>(G.gt(k), p.ldxu, nxu, 0, p.nc, 0, re, lt, lane);
    // ---- children
    for (int jc = 0; jc < m; ++jc) {
      const int c = c0 + jc;
      const int64_t er = __ldg(&p.desc[c].enr);
      const int64_t ztau = z2 + ny + jc;
      const S tz = z[ztau], tzp = zp[ztau], tdz = DR ? dz[ztau] : S(0);
      const S rt = tz - tzp, qt = tzp - rt;
      {  // nonroot block of c: SOC on (Q^c 1/2 x^k, R^c 1/2 u^k, tau^c / 2, tau^c / 2)
        zero_slots(v);
        wmv<S, J, NV>(G.fqc(c), p.ldx, nx, 0, nx, 0, zv, v, lane);
        wmv<S, J, NV>(G.frc(c), p.ldu, nu, nx, nu, nx, zv, v, lane);
        S y[J], o[J], be[J], bde[J], lr[J], ld[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          const bool tr = e == nxu || e == nxu + 1;
          be[j] = bde[j] = y[j] = lr[j] = ld[j] = S(0);
          if (e < nb) {
            be[j] = eta[er + e];
            if (DR) bde[j] = deta[er + e];
            const S q = tr ? S(0.5) * qt : v[0][j];
            lr[j] = tr ? S(0.5) * rt : v[1][j];
            if (DR) ld[j] = tr ? S(0.5) * tdz : v[2][j];
            y[j] = soc_shift(be[j] * ial + q, e, nb);
          }
        }
        soc_moreau<S, J>(y, nb, al, lane, o);
        S tau_part = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          re[0][j] = S(0);
          if (e < nb) {
            out[er + e] = o[j];
            dual_stat<S, true, DR>(nacc, ial, be[j], o[j], lr[j], bde[j], ld[j]);
            if (e < nxu) re[0][j] = be[j] - o[j];
            else tau_part += be[j] - o[j];
          }
        }
        wmv<S, J, 1>(G.fqt(c), p.ldx, nx, 0, nx, 0, re, lt, lane);
        wmv<S, J, 1>(G.frt(c), p.ldu, nu, nx, nu, nx, re, lt, lane);
        tau_part = warp_sum(tau_part);   // the two tau rows
        if (lane == 0) primal_stat<S, DR>(nacc, ial, rt, tdz, S(0.5) * tau_part);
      }
      if (c >= p.nl) {  // leaf block of c: Gamma_N x^c in C_N, SOC on (Q_N^1/2 x^c, s^c / 2, s^c / 2)
        const int64_t ef = __ldg(&p.desc[c].elf);
        const int64_t zxc = __ldg(&p.desc[c].zx);
        const int64_t zsc = z2 + ny + m + jc;
        const S sz = z[zsc], szp = zp[zsc], sdz = DR ? dz[zsc] : S(0);
        const S rs_ = sz - szp, qs_ = szp - rs_;
        S xv[3][J], ltx[1][J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          xv[0][j] = xv[1][j] = xv[2][j] = ltx[0][j] = S(0);
          if (e < nx) {
            const S xz = z[zxc + e], xzp = zp[zxc + e];
            xv[1][j] = xz - xzp;
            xv[0][j] = xzp - xv[1][j];
            if (DR) xv[2][j] = dz[zxc + e];
          }
        }
        zero_slots(v);
        wmv<S, J, NV>(G.gnc(c), p.ldcn, p.ncN, 0, nx, 0, xv, v, lane);
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int r = lane + 32 * j;
          re[0][j] = S(0);
          if (r < p.ncN) {
            const S fe = eta[ef + r], fde = DR ? deta[ef + r] : S(0);
            const S w = fe + al * v[0][j];
            const S o = w - al * clampv(w * ial, G.lo(c, r), G.hi(c, r));
            out[ef + r] = o;
            dual_stat<S, true, DR>(nacc, ial, fe, o, v[1][j], fde, DR ? v[2][j] : S(0));
            re[0][j] = fe - o;
          }
        }
        wmv<S, J, 1>(G.gnt(c), p.ldx, nx, 0, p.ncN, 0, re, ltx, lane);
        const int dim = nx + 2;
        const int64_t es = ef + p.ncN;
        zero_slots(v);
        wmv<S, J, NV>(G.fnc(c), p.ldx, nx, 0, nx, 0, xv, v, lane);
        S y[J], o[J], ev[J], dev[J], lr[J], ld[J];
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          const bool sr = e >= nx;
          y[j] = lr[j] = ld[j] = ev[j] = dev[j] = S(0);
          if (e < dim) {
            ev[j] = eta[es + e];
            if (DR) dev[j] = deta[es + e];
            const S q = sr ? S(0.5) * qs_ : v[0][j];
            lr[j] = sr ? S(0.5) * rs_ : v[1][j];
            if (DR) ld[j] = sr ? S(0.5) * sdz : v[2][j];
            y[j] = soc_shift(ev[j] * ial + q, e, dim);
          }
        }
        soc_moreau<S, J>(y, dim, al, lane, o);
        S s_part = 0;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int e = lane + 32 * j;
          re[0][j] = S(0);
          if (e < dim) {
            out[es + e] = o[j];
            dual_stat<S, true, DR>(nacc, ial, ev[j], o[j], lr[j], dev[j], ld[j]);
            if (e < nx) re[0][j] = ev[j] - o[j];
            else s_part += ev[j] - o[j];
          }
        }
        wmv<S, J, 1>(G.fnt(c), p.ldx, nx, 0, nx, 0, re, ltx, lane);
#pragma unroll
        for (int j = 0; j < J; ++j)
          if (lane + 32 * j < nx) primal_stat<S, DR>(nacc, ial, xv[1][j], xv[2][j], ltx[0][j]);
        s_part = warp_sum(s_part);   // the two s rows
        if (lane == 0) primal_stat<S, DR>(nacc, ial, rs_, sdz, S(0.5) * s_part);
      }
    }
    // ---- primal statistics at x^k, u^k
#pragma unroll
    for (int j = 0; j < J; ++j)
      if (lane + 32 * j < nxu) primal_stat<S, DR>(nacc, ial, zv[1][j], zv[2][j], lt[0][j]);
    // ---- the s - b'y row of k, then the y rows (prox of (K^k)*)
    {
      S bs = 0, bsp = 0, bsd = 0;
      for (int jj = lane; jj < ny; jj += 32) {
        const S bj = bk[jj];
        bs += bj * z[z2 + jj];
        bsp += bj * zp[z2 + jj];
        if (DR) bsd += bj * dz[z2 + jj];
      }
      bs = warp_sum(bs);
      bsp = warp_sum(bsp);
      if (DR) bsd = warp_sum(bsd);
      const S sk = z[D.zs], skp = zp[D.zs], skd = DR ? dz[D.zs] : S(0);
      const int64_t ie_sb = el + ny;
      const S esb = eta[ie_sb], desb = DR ? deta[ie_sb] : S(0);
      const S Lz = sk - bs, Lzp = skp - bsp, Ld = DR ? skd - bsd : S(0);
      const S w = dual_w<S, DM_DUAL>(al, esb, Lz, Lzp);
      const S o = vmin(w, S(0));
      const S re_sb = esb - o;
      if (lane == 0) {
        out[ie_sb] = o;
        dual_stat<S, true, DR>(nacc, ial, esb, o, Lz - Lzp, desb, Ld);
        primal_stat<S, DR>(nacc, ial, sk - skp, skd, re_sb);   // s^k (s^0 at the root)
      }
      for (int e = lane; e < ny; e += 32) {
        const S yz = z[z2 + e], yzp = zp[z2 + e], yd = DR ? dz[z2 + e] : S(0);
        const S ye = eta[el + e], yde = DR ? deta[el + e] : S(0);
        const S yw = dual_w<S, DM_DUAL>(al, ye, yz, yzp);
        const S yo = e < kp ? vmin(yw, S(0)) : S(0);
        out[el + e] = yo;
        dual_stat<S, true, DR>(nacc, ial, ye, yo, yz - yzp, yde, yd);
        primal_stat<S, DR>(nacc, ial, yz - yzp, yd, (ye - yo) - bk[e] * re_sb);
      }
    }
    nacc.node_done(acc);
  }
  nacc.flush(acc);
  block_stats_store<sizeof(S) == 4>(acc, partials, blockIdx.x);
}

// ---------------------------------------------------------------------------
// launchers (lane slots J in {1, 3, 5}: the smallest that holds the largest
// block -- nx + nu + 2, nc, ncN -- of the problem)
// ---------------------------------------------------------------------------
template <typename S>
static int gen_slots(const KP<S>& p) {
  const int w = max(max(max(p.nx + p.nu + 2, p.nc), p.ncN), p.max_nz2);
  const int j = (w + 31) / 32;
  return j <= 1 ? 1 : (j <= 3 ? 3 : 5);
}

template <typename S>
void launch_lstar_gen(const KP<S>& p, int mode, const S* eta, const S* z, S* zo, int grid, cudaStream_t st) {
#define SPOCK_LG(JJ)                                                                        \
  if (mode == LS_PREP) k_lstar_g<S, LS_PREP, JJ><<<grid, 128, 0, st>>>(p, eta, z, zo);     \
  else k_lstar_g<S, LS_APPLY, JJ><<<grid, 128, 0, st>>>(p, eta, z, zo);
  switch (gen_slots(p)) {
    case 1: SPOCK_LG(1) break;
    case 3: SPOCK_LG(3) break;
    default: SPOCK_LG(5) break;
  }
#undef SPOCK_LG
}

template <typename S>
void launch_dual_gen(const KP<S>& p, int mode, bool stats, const S* z, const S* zp, const S* eta, S* out,
                     const S* dir, double* partials, int grid, cudaStream_t st) {
#define SPOCK_DG(JJ)                                                                                     \
  if (mode == DM_APPLY_L) k_dual_g<S, DM_APPLY_L, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out);         \
  else if (mode == DM_PROXG) k_dual_g<S, DM_PROXG, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out);        \
  else if (!stats) k_dual_g<S, DM_DUAL, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out);                   \
  else if (dir) k_dual_fused_g<S, true, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);    \
  else k_dual_fused_g<S, false, JJ><<<grid, 128, 0, st>>>(p, z, zp, eta, out, dir, partials);
  switch (gen_slots(p)) {
    case 1: SPOCK_DG(1) break;
    case 3: SPOCK_DG(3) break;
    default: SPOCK_DG(5) break;
  }
#undef SPOCK_DG
}

template void launch_lstar_gen<double>(const KP<double>&, int, const double*, const double*, double*, int,
                                       cudaStream_t);
template void launch_lstar_gen<float>(const KP<float>&, int, const float*, const float*, float*, int, cudaStream_t);
template void launch_dual_gen<double>(const KP<double>&, int, bool, const double*, const double*, const double*,
                                      double*, const double*, double*, int, cudaStream_t);
template void launch_dual_gen<float>(const KP<float>&, int, bool, const float*, const float*, const float*, float*,
                                     const float*, double*, int, cudaStream_t);

}  // namespace spock
