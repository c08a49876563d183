// riccati_cpu -- a plain FP64 CPU implementation of the Chambolle-Pock
// operator T of Eq. (chambolle-pock-operator) for the RAOCP splitting of
// Sec. "Operator splitting", with the projection on the tree dynamics S1
// computed by Algorithm 1 (offline) and Algorithm 2 (online) exactly as the
// paper prints them, and OpenMP over the nodes of a stage where the paper
// writes "for all ... in parallel".
//
// TEST INFRASTRUCTURE ONLY (part of the oracle): used by the tests, as the
// timed CPU baseline and as a full-size checker where the Python oracle's
// sparse KKT solve is too large.  It shares no code with the CUDA library.
// Pinned against the Python oracle (KKT projection, sparse L) at 1e-12 on
// small trees (tests/test_oracle_riccati_cpu.py).
//
// Layout of z and eta: the user-order layout the Python oracle and the C
// ABI document (z = s0, x of every node, u of every nonleaf, then per
// nonleaf (y, tau of the children, s of the children); eta = per nonleaf
// (y, s - b'y, x, u), per nonroot (Q^1/2 x^anc, R^1/2 u^anc, tau/2, tau/2),
// per leaf (x, Q_N^1/2 x, s/2, s/2)).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Oracle {
  int n = 0, nx = 0, nu = 0, N = 0, threads = 1;
  std::vector<int> anc, depth, nch;
  std::vector<std::vector<int>> ch;       // children, increasing id
  std::vector<std::vector<int>> stage;    // nodes of each stage
  std::vector<int> sib;                   // position among the siblings
  std::vector<double> prob;               // conditional
  std::vector<double> A, B, Q, R, QN, a, xmin, xmax, umin, umax;
  // offsets (user order)
  int64_t n_z = 0, n_eta = 0;
  std::vector<int64_t> zx, zu, zy, ztau, zs, ey, esb, ex, eu, eqx, eru, et, elx, eqn, els;
  // Algorithm 1 outputs
  std::vector<double> P;      // [n][nx][nx]
  std::vector<double> Rc;     // [n][nu][nu] lower Cholesky factor of Rtilde (nonleaf)
  std::vector<double> K;      // [n][nu][nx] (nonleaf)
  std::vector<double> Abar;   // [n][nx][nx] (nonroot)
  // S2: lower Cholesky factor of M M^T per nonleaf, M = [E^T, -I, -I]
  std::vector<std::vector<double>> S2c;
  // scratch of Algorithm 2
  std::vector<double> q, d;
};

inline double* at(std::vector<double>& v, int node, int size) { return v.data() + (size_t)node * size; }
inline const double* at(const std::vector<double>& v, int node, int size) {
  return v.data() + (size_t)node * size;
}

// Cholesky factor (lower, row-major) of an SPD matrix; false if not SPD.
bool cholesky(const double* M, int m, double* L) {
  for (int i = 0; i < m * m; ++i) L[i] = 0.0;
  for (int j = 0; j < m; ++j) {
    double s = M[j * m + j];
    for (int k = 0; k < j; ++k) s -= L[j * m + k] * L[j * m + k];
    if (!(s > 0.0)) return false;
    const double ljj = std::sqrt(s);
    L[j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double t = M[i * m + j];
      for (int k = 0; k < j; ++k) t -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = t / ljj;
    }
  }
  return true;
}

// Solves (L L^T) x = b in place.
void chol_solve(const double* L, int m, double* x) {
  for (int i = 0; i < m; ++i) {
    double s = x[i];
    for (int k = 0; k < i; ++k) s -= L[i * m + k] * x[k];
    x[i] = s / L[i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = x[i];
    for (int k = i + 1; k < m; ++k) s -= L[k * m + i] * x[k];
    x[i] = s / L[i * m + i];
  }
}

void set_threads(const Oracle& o) {
#ifdef _OPENMP
  omp_set_num_threads(o.threads);
#else
  (void)o;
#endif
}

// ---------------------------------------------------------------------------
// Algorithm 1: P, Rtilde (Cholesky), K, Abar, stage by stage from the leaves
// ---------------------------------------------------------------------------
bool offline(Oracle& o) {
  const int nx = o.nx, nu = o.nu;
  o.P.assign((size_t)o.n * nx * nx, 0.0);
  o.Rc.assign((size_t)o.n * nu * nu, 0.0);
  o.K.assign((size_t)o.n * nu * nx, 0.0);
  o.Abar.assign((size_t)o.n * nx * nx, 0.0);
  for (int j : o.stage[o.N]) {
    double* Pj = at(o.P, j, nx * nx);
    for (int r = 0; r < nx; ++r) Pj[r * nx + r] = 1.0;
  }
  bool ok = true;
  for (int t = 0; t < o.N; ++t) {
    const std::vector<int>& nodes = o.stage[o.N - (t + 1)];
#pragma omp parallel for schedule(dynamic, 4) reduction(&& : ok)
    for (size_t idx = 0; idx < nodes.size(); ++idx) {
      const int i = nodes[idx];
      std::vector<double> Rt((size_t)nu * nu, 0.0), SA((size_t)nu * nx, 0.0), Pt((size_t)nu * nx);
      for (int r = 0; r < nu; ++r) Rt[r * nu + r] = 1.0;
      for (int c : o.ch[i]) {
        const double* Pc = at(o.P, c, nx * nx);
        const double* Bc = at(o.B, c, nx * nu);
        const double* Ac = at(o.A, c, nx * nx);
        // Ptilde = B^T P  (nu x nx)
        for (int r = 0; r < nu; ++r)
          for (int k = 0; k < nx; ++k) {
            double s = 0.0;
            for (int l = 0; l < nx; ++l) s += Bc[l * nu + r] * Pc[l * nx + k];
            Pt[r * nx + k] = s;
          }
        // Rtilde += Ptilde B ; SA += Ptilde A
        for (int r = 0; r < nu; ++r) {
          for (int k = 0; k < nu; ++k) {
            double s = 0.0;
            for (int l = 0; l < nx; ++l) s += Pt[r * nx + l] * Bc[l * nu + k];
            Rt[r * nu + k] += s;
          }
          for (int k = 0; k < nx; ++k) {
            double s = 0.0;
            for (int l = 0; l < nx; ++l) s += Pt[r * nx + l] * Ac[l * nx + k];
            SA[r * nx + k] += s;
          }
        }
      }
      double* Lr = at(o.Rc, i, nu * nu);
      if (!cholesky(Rt.data(), nu, Lr)) {
        ok = false;
        continue;
      }
      // K = -Rtilde^{-1} SA, column by column
      double* Ki = at(o.K, i, nu * nx);
      std::vector<double> col(nu);
      for (int k = 0; k < nx; ++k) {
        for (int r = 0; r < nu; ++r) col[r] = SA[r * nx + k];
        chol_solve(Lr, nu, col.data());
        for (int r = 0; r < nu; ++r) Ki[r * nx + k] = -col[r];
      }
      // Abar^c = A^c + B^c K ; P^i = I + K^T K + sum_c Abar^T P^c Abar
      double* Pi = at(o.P, i, nx * nx);
      for (int r = 0; r < nx; ++r)
        for (int k = 0; k < nx; ++k) {
          double s = r == k ? 1.0 : 0.0;
          for (int l = 0; l < nu; ++l) s += Ki[l * nx + r] * Ki[l * nx + k];
          Pi[r * nx + k] = s;
        }
      std::vector<double> PA((size_t)nx * nx);
      for (int c : o.ch[i]) {
        const double* Ac = at(o.A, c, nx * nx);
        const double* Bc = at(o.B, c, nx * nu);
        const double* Pc = at(o.P, c, nx * nx);
        double* Ab = at(o.Abar, c, nx * nx);
        for (int r = 0; r < nx; ++r)
          for (int k = 0; k < nx; ++k) {
            double s = Ac[r * nx + k];
            for (int l = 0; l < nu; ++l) s += Bc[r * nu + l] * Ki[l * nx + k];
            Ab[r * nx + k] = s;
          }
        for (int r = 0; r < nx; ++r)
          for (int k = 0; k < nx; ++k) {
            double s = 0.0;
            for (int l = 0; l < nx; ++l) s += Pc[r * nx + l] * Ab[l * nx + k];
            PA[r * nx + k] = s;
          }
        for (int r = 0; r < nx; ++r)
          for (int k = 0; k < nx; ++k) {
            double s = 0.0;
            for (int l = 0; l < nx; ++l) s += Ab[l * nx + r] * PA[l * nx + k];
            Pi[r * nx + k] += s;
          }
      }
    }
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Algorithm 2: projection of (xbar, ubar) (read from zb) on S1, into zo
// ---------------------------------------------------------------------------
void online(Oracle& o, const double* x0, const double* zb, double* zo) {
  const int nx = o.nx, nu = o.nu;
  o.q.assign((size_t)o.n * nx, 0.0);
  o.d.assign((size_t)o.n * nu, 0.0);
  for (int j : o.stage[o.N]) {
    double* qj = at(o.q, j, nx);
    for (int r = 0; r < nx; ++r) qj[r] = -zb[o.zx[j] + r];
  }
  for (int t = 0; t < o.N; ++t) {
    const std::vector<int>& nodes = o.stage[o.N - (t + 1)];
#pragma omp parallel for schedule(static)
    for (size_t idx = 0; idx < nodes.size(); ++idx) {
      const int i = nodes[idx];
      const double* xb = zb + o.zx[i];
      const double* ub = zb + o.zu[i];
      double* di = at(o.d, i, nu);
      // d = Rtilde^{-1} (ubar - sum_c B^T q^c)
      for (int r = 0; r < nu; ++r) di[r] = ub[r];
      for (int c : o.ch[i]) {
        const double* Bc = at(o.B, c, nx * nu);
        const double* qc = at(o.q, c, nx);
        for (int r = 0; r < nu; ++r) {
          double s = 0.0;
          for (int l = 0; l < nx; ++l) s += Bc[l * nu + r] * qc[l];
          di[r] -= s;
        }
      }
      chol_solve(at(o.Rc, i, nu * nu), nu, di);
      // q = K^T (d - ubar) - xbar + sum_c Abar^T (P B d + q^c)
      const double* Ki = at(o.K, i, nu * nx);
      double* qi = at(o.q, i, nx);
      for (int r = 0; r < nx; ++r) {
        double s = -xb[r];
        for (int l = 0; l < nu; ++l) s += Ki[l * nx + r] * (di[l] - ub[l]);
        qi[r] = s;
      }
      std::vector<double> Bd(nx), w(nx);
      for (int c : o.ch[i]) {
        const double* Bc = at(o.B, c, nx * nu);
        const double* Pc = at(o.P, c, nx * nx);
        const double* Ab = at(o.Abar, c, nx * nx);
        const double* qc = at(o.q, c, nx);
        for (int r = 0; r < nx; ++r) {
          double s = 0.0;
          for (int l = 0; l < nu; ++l) s += Bc[r * nu + l] * di[l];
          Bd[r] = s;
        }
        for (int r = 0; r < nx; ++r) {
          double s = qc[r];
          for (int l = 0; l < nx; ++l) s += Pc[r * nx + l] * Bd[l];
          w[r] = s;
        }
        for (int r = 0; r < nx; ++r) {
          double s = 0.0;
          for (int l = 0; l < nx; ++l) s += Ab[l * nx + r] * w[l];
          qi[r] += s;
        }
      }
    }
  }
  // forward: x^0 = x0; u^i = K x^i + d; x^c = A^c x^i + B^c u^i
  for (int r = 0; r < nx; ++r) zo[o.zx[0] + r] = x0[r];
  for (int t = 0; t < o.N; ++t) {
    const std::vector<int>& nodes = o.stage[t];
#pragma omp parallel for schedule(static)
    for (size_t idx = 0; idx < nodes.size(); ++idx) {
      const int i = nodes[idx];
      const double* xi = zo + o.zx[i];
      double* ui = zo + o.zu[i];
      const double* Ki = at(o.K, i, nu * nx);
      const double* di = at(o.d, i, nu);
      for (int r = 0; r < nu; ++r) {
        double s = di[r];
        for (int l = 0; l < nx; ++l) s += Ki[r * nx + l] * xi[l];
        ui[r] = s;
      }
      for (int c : o.ch[i]) {
        const double* Ac = at(o.A, c, nx * nx);
        const double* Bc = at(o.B, c, nx * nu);
        double* xc = zo + o.zx[c];
        for (int r = 0; r < nx; ++r) {
          double s = 0.0;
          for (int l = 0; l < nx; ++l) s += Ac[r * nx + l] * xi[l];
          for (int l = 0; l < nu; ++l) s += Bc[r * nu + l] * ui[l];
          xc[r] = s;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// L, L* (definition of L), S2 and S3 projections
// ---------------------------------------------------------------------------
void apply_L(const Oracle& o, const double* z, double* e) {
  const int nx = o.nx, nu = o.nu;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < o.n; ++i) {
    const int m = o.nch[i];
    if (m > 0) {
      for (int k = 0; k < 2 * m + 1; ++k) e[o.ey[i] + k] = z[o.zy[i] + k];
      double s = z[o.zs[i]];
      for (int k = 0; k < m; ++k) s -= o.prob[o.ch[i][k]] * z[o.zy[i] + k];   // b = (p, 0, 1)
      s -= z[o.zy[i] + 2 * m];
      e[o.esb[i]] = s;
      for (int k = 0; k < nx; ++k) e[o.ex[i] + k] = z[o.zx[i] + k];
      for (int k = 0; k < nu; ++k) e[o.eu[i] + k] = z[o.zu[i] + k];
    } else {
      for (int k = 0; k < nx; ++k) {
        e[o.elx[i] + k] = z[o.zx[i] + k];
        e[o.eqn[i] + k] = std::sqrt(o.QN[(size_t)i * nx + k]) * z[o.zx[i] + k];
      }
      e[o.els[i]] = 0.5 * z[o.zs[i]];
      e[o.els[i] + 1] = 0.5 * z[o.zs[i]];
    }
    if (i > 0) {
      const int p = o.anc[i];
      for (int k = 0; k < nx; ++k) e[o.eqx[i] + k] = std::sqrt(o.Q[(size_t)i * nx + k]) * z[o.zx[p] + k];
      for (int k = 0; k < nu; ++k) e[o.eru[i] + k] = std::sqrt(o.R[(size_t)i * nu + k]) * z[o.zu[p] + k];
      e[o.et[i]] = 0.5 * z[o.ztau[i]];
      e[o.et[i] + 1] = 0.5 * z[o.ztau[i]];
    }
  }
}

// z = L^T e: every z entry gathers the rows of L that touch it
void apply_Lt(const Oracle& o, const double* e, double* z) {
  const int nx = o.nx, nu = o.nu;
  z[0] = e[o.esb[0]];   // s^0 appears only in the root's row s^0 - b'y
#pragma omp parallel for schedule(static)
  for (int i = 0; i < o.n; ++i) {
    const int m = o.nch[i];
    double* zxi = z + o.zx[i];
    if (m > 0) {
      double* zui = z + o.zu[i];
      for (int k = 0; k < nx; ++k) zxi[k] = e[o.ex[i] + k];
      for (int k = 0; k < nu; ++k) zui[k] = e[o.eu[i] + k];
      for (int c : o.ch[i]) {
        for (int k = 0; k < nx; ++k) zxi[k] += std::sqrt(o.Q[(size_t)c * nx + k]) * e[o.eqx[c] + k];
        for (int k = 0; k < nu; ++k) zui[k] += std::sqrt(o.R[(size_t)c * nu + k]) * e[o.eru[c] + k];
      }
      const double r_sb = e[o.esb[i]];
      for (int k = 0; k < 2 * m + 1; ++k) {
        const double bk = k < m ? o.prob[o.ch[i][k]] : (k == 2 * m ? 1.0 : 0.0);
        z[o.zy[i] + k] = e[o.ey[i] + k] - bk * r_sb;
      }
      for (int k = 0; k < m; ++k) {
        const int c = o.ch[i][k];
        z[o.ztau[c]] = 0.5 * (e[o.et[c]] + e[o.et[c] + 1]);
        // s^c: the child's own row s^c - b'y (nonleaf child) or its leaf rows
        z[o.zs[c]] = o.nch[c] > 0 ? e[o.esb[c]] : 0.5 * (e[o.els[c]] + e[o.els[c] + 1]);
      }
    } else {
      for (int k = 0; k < nx; ++k)
        zxi[k] = e[o.elx[i] + k] + std::sqrt(o.QN[(size_t)i * nx + k]) * e[o.eqn[i] + k];
    }
  }
}

// projection of the z2 block of every nonleaf node on ker [E^T, -I, -I]
void proj_S2(const Oracle& o, double* z) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < o.n; ++i) {
    const int m = o.nch[i];
    if (m == 0) continue;
    const double ai = o.a[i];
    double* y = z + o.zy[i];   // (y1 [m], y2 [m], y3), then tau [m], s [m]
    std::vector<double> lam(m);
    for (int j = 0; j < m; ++j)
      lam[j] = ai * y[j] - y[m + j] + y[2 * m] - y[2 * m + 1 + j] - y[3 * m + 1 + j];
    chol_solve(o.S2c[i].data(), m, lam.data());
    double sum = 0.0;
    for (int j = 0; j < m; ++j) {
      y[j] -= ai * lam[j];
      y[m + j] += lam[j];
      y[2 * m + 1 + j] += lam[j];
      y[3 * m + 1 + j] += lam[j];
      sum += lam[j];
    }
    y[2 * m] -= sum;
  }
}

void proj_soc_shift(double* w, int dim) {
  // SOC + (0, .., 0, 1/2, -1/2) with SOC = {(v, t) : |v| <= t}, t last
  w[dim - 2] -= 0.5;
  w[dim - 1] += 0.5;
  double nv = 0.0;
  for (int k = 0; k < dim - 1; ++k) nv += w[k] * w[k];
  nv = std::sqrt(nv);
  const double t = w[dim - 1];
  if (nv <= t) {
  } else if (nv <= -t) {
    for (int k = 0; k < dim; ++k) w[k] = 0.0;
  } else {
    const double sc = 0.5 * (nv + t);
    for (int k = 0; k < dim - 1; ++k) w[k] *= sc / nv;
    w[dim - 1] = sc;
  }
  w[dim - 2] += 0.5;
  w[dim - 1] -= 0.5;
}

// e <- prox_{alpha g*}(e) = e - alpha proj_S3(e / alpha)
void prox_gconj(const Oracle& o, double alpha, double* e) {
  const int nx = o.nx, nu = o.nu;
  auto moreau_box = [&](double* v, const double* lo, const double* hi, int len) {
    for (int k = 0; k < len; ++k) {
      const double w = v[k] / alpha;
      v[k] -= alpha * std::min(std::max(w, lo[k]), hi[k]);
    }
  };
  auto moreau_plus = [&](double* v, int len) {
    for (int k = 0; k < len; ++k) v[k] -= alpha * std::max(v[k] / alpha, 0.0);
  };
#pragma omp parallel for schedule(static)
  for (int i = 0; i < o.n; ++i) {
    const int m = o.nch[i];
    std::vector<double> w(nx + nu + 2);
    if (m > 0) {
      moreau_plus(e + o.ey[i], 2 * m);   // y: R^{2m}_+ x R (last entry free: projection = itself)
      e[o.ey[i] + 2 * m] -= alpha * (e[o.ey[i] + 2 * m] / alpha);
      moreau_plus(e + o.esb[i], 1);
      moreau_box(e + o.ex[i], o.xmin.data() + (size_t)i * nx, o.xmax.data() + (size_t)i * nx, nx);
      moreau_box(e + o.eu[i], o.umin.data() + (size_t)i * nu, o.umax.data() + (size_t)i * nu, nu);
    } else {
      moreau_box(e + o.elx[i], o.xmin.data() + (size_t)i * nx, o.xmax.data() + (size_t)i * nx, nx);
      // (Q_N^1/2 x, s/2, s/2) are contiguous
      double* v = e + o.eqn[i];
      for (int k = 0; k < nx + 2; ++k) w[k] = v[k] / alpha;
      proj_soc_shift(w.data(), nx + 2);
      for (int k = 0; k < nx + 2; ++k) v[k] -= alpha * w[k];
    }
    if (i > 0) {
      double* v = e + o.eqx[i];   // (Q^1/2 x, R^1/2 u, tau/2, tau/2) contiguous
      for (int k = 0; k < nx + nu + 2; ++k) w[k] = v[k] / alpha;
      proj_soc_shift(w.data(), nx + nu + 2);
      for (int k = 0; k < nx + nu + 2; ++k) v[k] -= alpha * w[k];
    }
  }
}

void prox_f(Oracle& o, const double* x0, double alpha, const double* zb, double* zo) {
  std::memcpy(zo, zb, sizeof(double) * (size_t)o.n_z);
  zo[0] = zb[0] - alpha;
  online(o, x0, zb, zo);
  proj_S2(o, zo);
}

}  // namespace

extern "C" {

void* rc_create(int32_t n, const int32_t* anc, const double* prob, int32_t nx, int32_t nu, const double* A,
                const double* B, const double* Q, const double* R, const double* QN, const double* a,
                const double* xmin, const double* xmax, const double* umin, const double* umax, int32_t threads) {
  auto* o = new Oracle();
  o->n = n;
  o->nx = nx;
  o->nu = nu;
  o->threads = threads > 0 ? threads : 1;
  set_threads(*o);
  o->anc.assign(anc, anc + n);
  o->prob.assign(prob, prob + n);
  const size_t nn = (size_t)n;
  o->A.assign(A, A + nn * nx * nx);
  o->B.assign(B, B + nn * nx * nu);
  o->Q.assign(Q, Q + nn * nx);
  o->R.assign(R, R + nn * nu);
  o->QN.assign(QN, QN + nn * nx);
  o->a.assign(a, a + nn);
  o->xmin.assign(xmin, xmin + nn * nx);
  o->xmax.assign(xmax, xmax + nn * nx);
  o->umin.assign(umin, umin + nn * nu);
  o->umax.assign(umax, umax + nn * nu);
  o->ch.assign(n, {});
  o->nch.assign(n, 0);
  o->sib.assign(n, 0);
  o->depth.assign(n, 0);
  for (int i = 1; i < n; ++i) {   // parents precede children in these trees' numbering
    if (anc[i] < 0 || anc[i] >= i) {
      delete o;
      return nullptr;
    }
    o->sib[i] = (int)o->ch[anc[i]].size();
    o->ch[anc[i]].push_back(i);
    o->depth[i] = o->depth[anc[i]] + 1;
  }
  for (int i = 0; i < n; ++i) o->nch[i] = (int)o->ch[i].size();
  int N = 0;
  for (int i = 0; i < n; ++i) N = std::max(N, o->depth[i]);
  o->N = N;
  o->stage.assign(N + 1, {});
  for (int i = 0; i < n; ++i) o->stage[o->depth[i]].push_back(i);
  // z offsets
  o->zx.assign(n, -1); o->zu.assign(n, -1); o->zy.assign(n, -1); o->ztau.assign(n, -1); o->zs.assign(n, -1);
  int64_t pos = 1;
  for (int i = 0; i < n; ++i) { o->zx[i] = pos; pos += nx; }
  for (int i = 0; i < n; ++i) if (o->nch[i]) { o->zu[i] = pos; pos += nu; }
  for (int i = 0; i < n; ++i) {
    const int m = o->nch[i];
    if (!m) continue;
    o->zy[i] = pos;
    for (int k = 0; k < m; ++k) {
      o->ztau[o->ch[i][k]] = pos + 2 * m + 1 + k;
      o->zs[o->ch[i][k]] = pos + 3 * m + 1 + k;
    }
    pos += 4 * m + 1;
  }
  o->zs[0] = 0;
  o->n_z = pos;
  // eta offsets
  o->ey.assign(n, -1); o->esb.assign(n, -1); o->ex.assign(n, -1); o->eu.assign(n, -1);
  o->eqx.assign(n, -1); o->eru.assign(n, -1); o->et.assign(n, -1);
  o->elx.assign(n, -1); o->eqn.assign(n, -1); o->els.assign(n, -1);
  pos = 0;
  for (int i = 0; i < n; ++i) {
    const int m = o->nch[i];
    if (!m) continue;
    o->ey[i] = pos; pos += 2 * m + 1;
    o->esb[i] = pos; pos += 1;
    o->ex[i] = pos; pos += nx;
    o->eu[i] = pos; pos += nu;
  }
  for (int c = 1; c < n; ++c) {
    o->eqx[c] = pos; pos += nx;
    o->eru[c] = pos; pos += nu;
    o->et[c] = pos; pos += 2;
  }
  for (int j = 0; j < n; ++j) {
    if (o->nch[j]) continue;
    o->elx[j] = pos; pos += nx;
    o->eqn[j] = pos; pos += nx;
    o->els[j] = pos; pos += 2;
  }
  o->n_eta = pos;
  // S2: M M^T for M = [a I, -I, 1, -I, -I] (m x (4m+1)), factored per node
  o->S2c.assign(n, {});
  for (int i = 0; i < n; ++i) {
    const int m = o->nch[i];
    if (!m) continue;
    std::vector<double> MM((size_t)m * m, 1.0);   // the column of ones
    for (int j = 0; j < m; ++j) MM[j * m + j] += o->a[i] * o->a[i] + 3.0;
    o->S2c[i].assign((size_t)m * m, 0.0);
    if (!cholesky(MM.data(), m, o->S2c[i].data())) {
      delete o;
      return nullptr;
    }
  }
  if (!offline(*o)) {
    delete o;
    return nullptr;
  }
  return o;
}

void rc_sizes(void* h, int64_t* n_z, int64_t* n_eta) {
  auto* o = static_cast<Oracle*>(h);
  *n_z = o->n_z;
  *n_eta = o->n_eta;
}

void rc_set_threads(void* h, int32_t threads) {
  auto* o = static_cast<Oracle*>(h);
  o->threads = threads > 0 ? threads : 1;
}

void rc_apply_L(void* h, const double* z, double* e) {
  auto* o = static_cast<Oracle*>(h);
  set_threads(*o);
  apply_L(*o, z, e);
}

void rc_apply_Lt(void* h, const double* e, double* z) {
  auto* o = static_cast<Oracle*>(h);
  set_threads(*o);
  apply_Lt(*o, e, z);
}

// z_out = prox_{alpha f}(z): s^0 - alpha, proj_S1 (Algorithms 1-2), proj_S2
void rc_prox_f(void* h, const double* x0, double alpha, const double* z, double* zo) {
  auto* o = static_cast<Oracle*>(h);
  set_threads(*o);
  prox_f(*o, x0, alpha, z, zo);
}

// eta_out = prox_{alpha g*}(eta)
void rc_prox_gconj(void* h, double alpha, const double* e, double* eo) {
  auto* o = static_cast<Oracle*>(h);
  set_threads(*o);
  std::memcpy(eo, e, sizeof(double) * (size_t)o->n_eta);
  prox_gconj(*o, alpha, eo);
}

// (z_out, eta_out) = T(z, eta) of Eq. (chambolle-pock-operator)
void rc_T(void* h, const double* x0, double alpha, const double* z, const double* e, double* zo, double* eo) {
  auto* o = static_cast<Oracle*>(h);
  set_threads(*o);
  std::vector<double> zb((size_t)o->n_z), w((size_t)o->n_z);
  apply_Lt(*o, e, zb.data());
  for (int64_t k = 0; k < o->n_z; ++k) zb[k] = z[k] - alpha * zb[k];
  prox_f(*o, x0, alpha, zb.data(), zo);
  for (int64_t k = 0; k < o->n_z; ++k) w[k] = 2.0 * zo[k] - z[k];
  apply_L(*o, w.data(), eo);
  for (int64_t k = 0; k < o->n_eta; ++k) eo[k] = e[k] + alpha * eo[k];
  prox_gconj(*o, alpha, eo);
}

void rc_free(void* h) { delete static_cast<Oracle*>(h); }

}  // extern "C"
