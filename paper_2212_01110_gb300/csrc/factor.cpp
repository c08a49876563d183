// Offline factorisation of the projection on S1 (Algorithm 1, FP64, host).
//
// For every nonleaf node i, stage by stage from the leaves (P = I there):
//   Pt^c   = B^cT P^c                          (nu x nx), c in ch(i)
//   Rt^i   = I + sum_c Pt^c B^c                (nu x nu), Cholesky factor
//   K^i    = -(Rt^i)^-1 sum_c Pt^c A^c         (nu x nx)
//   Abar^c = A^c + B^c K^i
//   P^i    = I + K^iT K^i + sum_c Abar^cT P^c Abar^c
// and, for the online pass (Algorithm 2), W^i = sum_c Abar^cT P^c B^c
// (= sum_c Abar^cT Pt^cT), which turns the term sum_c Abar^cT P^c B^c d^i of
// the backward recursion into one product.  P is discarded after use.
// Nodes of one stage are independent and are spread over host threads.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "spock_internal.h"

namespace spock {
namespace {

// C (r x c) = A (r x k) * B (k x c), row-major, C overwritten.
void gemm(int r, int k, int c, const double* A, const double* B, double* C) {
  for (int i = 0; i < r * c; ++i) C[i] = 0.0;
  for (int i = 0; i < r; ++i)
    for (int l = 0; l < k; ++l) {
      const double a = A[i * k + l];
      const double* b = B + l * c;
      double* o = C + i * c;
      for (int j = 0; j < c; ++j) o[j] += a * b[j];
    }
}

// C (r x c) += A^T B with A (k x r), B (k x c).
void gemm_tn_acc(int r, int k, int c, const double* A, const double* B, double* C) {
  for (int l = 0; l < k; ++l)
    for (int i = 0; i < r; ++i) {
      const double a = A[l * r + i];
      const double* b = B + l * c;
      double* o = C + i * c;
      for (int j = 0; j < c; ++j) o[j] += a * b[j];
    }
}

// In-place Cholesky L L^T of an SPD n x n matrix (lower triangle kept).
bool cholesky(int n, double* M) {
  for (int j = 0; j < n; ++j) {
    double s = M[j * n + j];
    for (int k = 0; k < j; ++k) s -= M[j * n + k] * M[j * n + k];
    if (!(s > 0.0)) return false;
    const double d = std::sqrt(s);
    M[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = M[i * n + j];
      for (int k = 0; k < j; ++k) t -= M[i * n + k] * M[j * n + k];
      M[i * n + j] = t / d;
    }
  }
  return true;
}

// Solve (L L^T) X = Bm in place for nrhs columns stored row-major (n x nrhs).
void chol_solve(int n, const double* Lc, int nrhs, double* X) {
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < nrhs; ++c) {
      double s = X[i * nrhs + c];
      for (int k = 0; k < i; ++k) s -= Lc[i * n + k] * X[k * nrhs + c];
      X[i * nrhs + c] = s / Lc[i * n + i];
    }
  for (int i = n - 1; i >= 0; --i)
    for (int c = 0; c < nrhs; ++c) {
      double s = X[i * nrhs + c];
      for (int k = i + 1; k < n; ++k) s -= Lc[k * n + i] * X[k * nrhs + c];
      X[i * nrhs + c] = s / Lc[i * n + i];
    }
}

}  // namespace

bool riccati_factor(const Tree& t, int nx, int nu, const std::vector<double>& A,
                    const std::vector<double>& B, std::vector<double>& Gb,
                    std::vector<double>& NB, int threads) {
  const int32_t n = t.n, nl = t.n_nonleaf;
  const int ncol = nx + nu;
  const size_t gsz = (size_t)nx * ncol;
  const size_t nbsz = 2 * (size_t)nu * nx + (size_t)nu * nu;
  Gb.assign((size_t)(n - 1) * gsz, 0.0);
  NB.assign((size_t)nl * nbsz, 0.0);
  // P of every node of the stage below (index: internal id - stage_begin)
  std::vector<double> Pbelow, Pcur;
  {
    const int32_t N = t.N;
    const int32_t cnt = t.stage_begin[N + 1] - t.stage_begin[N];
    Pbelow.assign((size_t)cnt * nx * nx, 0.0);
    for (int32_t j = 0; j < cnt; ++j)
      for (int r = 0; r < nx; ++r) Pbelow[(size_t)j * nx * nx + r * nx + r] = 1.0;
  }
  bool ok = true;
  for (int32_t s = t.N - 1; s >= 0; --s) {
    const int32_t b0 = t.stage_begin[s], b1 = t.stage_begin[s + 1];
    const int32_t cnt = b1 - b0;
    const int32_t below0 = t.stage_begin[s + 1];
    Pcur.assign((size_t)cnt * nx * nx, 0.0);
    int nth = std::max(1, std::min(threads, (int)((cnt + 7) / 8)));
    std::vector<char> okv(nth, 1);
    auto work = [&](int tid) {
      std::vector<double> Pt(nu * nx), Rt(nu * nu), SA(nu * nx), K(nu * nx), Ab(nx * nx),
          PA(nx * nx), W(nx * nu), Rinv(nu * nu), PB(nx * nu);
      for (int32_t k = b0 + tid; k < b1; k += nth) {
        const int32_t c0 = t.ch_begin[k], m = t.ch_count[k];
        std::fill(Rt.begin(), Rt.end(), 0.0);
        std::fill(SA.begin(), SA.end(), 0.0);
        for (int r = 0; r < nu; ++r) Rt[r * nu + r] = 1.0;
        for (int j = 0; j < m; ++j) {
          const int32_t c = c0 + j;
          const double* Pc = &Pbelow[(size_t)(c - below0) * nx * nx];
          const double* Bc = &B[(size_t)c * nx * nu];
          const double* Ac = &A[(size_t)c * nx * nx];
          // Pt = B^T P  (nu x nx)
          std::fill(Pt.begin(), Pt.end(), 0.0);
          gemm_tn_acc(nu, nx, nx, Bc, Pc, Pt.data());
          // Rt += Pt B ; SA += Pt A
          for (int r = 0; r < nu; ++r)
            for (int l = 0; l < nx; ++l) {
              const double a = Pt[r * nx + l];
              for (int q = 0; q < nu; ++q) Rt[r * nu + q] += a * Bc[l * nu + q];
              for (int q = 0; q < nx; ++q) SA[r * nx + q] += a * Ac[l * nx + q];
            }
        }
        if (!cholesky(nu, Rt.data())) { okv[tid] = 0; continue; }
        // K = -Rt^-1 SA
        for (size_t e = 0; e < K.size(); ++e) K[e] = -SA[e];
        chol_solve(nu, Rt.data(), nx, K.data());
        // Rinv = Rt^-1
        std::fill(Rinv.begin(), Rinv.end(), 0.0);
        for (int r = 0; r < nu; ++r) Rinv[r * nu + r] = 1.0;
        chol_solve(nu, Rt.data(), nu, Rinv.data());
        for (int r = 0; r < nu; ++r)  // symmetrise
          for (int q = r + 1; q < nu; ++q) {
            const double v = 0.5 * (Rinv[r * nu + q] + Rinv[q * nu + r]);
            Rinv[r * nu + q] = Rinv[q * nu + r] = v;
          }
        double* Pi = &Pcur[(size_t)(k - b0) * nx * nx];
        // P = I + K^T K
        std::fill(Pi, Pi + nx * nx, 0.0);
        for (int r = 0; r < nx; ++r) Pi[r * nx + r] = 1.0;
        gemm_tn_acc(nx, nu, nx, K.data(), K.data(), Pi);
        std::fill(W.begin(), W.end(), 0.0);
        for (int j = 0; j < m; ++j) {
          const int32_t c = c0 + j;
          const double* Pc = &Pbelow[(size_t)(c - below0) * nx * nx];
          const double* Bc = &B[(size_t)c * nx * nu];
          const double* Ac = &A[(size_t)c * nx * nx];
          // Abar = A + B K
          gemm(nx, nu, nx, Bc, K.data(), Ab.data());
          for (int e = 0; e < nx * nx; ++e) Ab[e] += Ac[e];
          // PA = P Abar ; P_i += Abar^T PA
          gemm(nx, nx, nx, Pc, Ab.data(), PA.data());
          gemm_tn_acc(nx, nx, nx, Ab.data(), PA.data(), Pi);
          // W += Abar^T (P B)
          gemm(nx, nx, nu, Pc, Bc, PB.data());
          gemm_tn_acc(nx, nx, nu, Ab.data(), PB.data(), W.data());
          // store [Abar | B] rows
          double* g = &Gb[(size_t)(c - 1) * gsz];
          for (int r = 0; r < nx; ++r) {
            for (int q = 0; q < nx; ++q) g[r * ncol + q] = Ab[r * nx + q];
            for (int q = 0; q < nu; ++q) g[r * ncol + nx + q] = Bc[r * nu + q];
          }
        }
        // symmetrise P (round-off)
        for (int r = 0; r < nx; ++r)
          for (int q = r + 1; q < nx; ++q) {
            const double v = 0.5 * (Pi[r * nx + q] + Pi[q * nx + r]);
            Pi[r * nx + q] = Pi[q * nx + r] = v;
          }
        double* nb = &NB[(size_t)k * nbsz];
        for (int r = 0; r < nu; ++r)
          for (int q = 0; q < nx; ++q) {
            nb[r * nx + q] = K[r * nx + q];                       // K   (nu x nx)
            // C = K + W^T (nu x nx): the backward step forms K^T (d - ubar) + W d
            // as C^T d - K^T ubar, without the difference d - ubar
            nb[(size_t)nu * nx + r * nx + q] = K[r * nx + q] + W[q * nu + r];
          }
        for (int e = 0; e < nu * nu; ++e) nb[2 * (size_t)nu * nx + e] = Rinv[e];
      }
    };
    if (nth == 1) {
      work(0);
    } else {
      std::vector<std::thread> pool;
      for (int tid = 0; tid < nth; ++tid) pool.emplace_back(work, tid);
      for (auto& th : pool) th.join();
    }
    for (char c : okv) ok = ok && c;
    if (!ok) return false;
    Pbelow.swap(Pcur);
  }
  return ok;
}

}  // namespace spock
