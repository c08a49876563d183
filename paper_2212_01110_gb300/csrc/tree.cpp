// Scenario tree validation, breadth-first renumbering and the offsets of
// every node's blocks in z and eta (Sec. "Scenario trees", Sec. "Operator
// splitting").
#include <algorithm>
#include <cmath>
#include <string>

#include "spock_internal.h"

namespace spock {

int build_tree(int32_t n, const int32_t* anc, const double* prob, Tree& t) {
  if (n < 2) return fail(SPOCK_ERR_INVALID_ARG, "tree needs at least 2 nodes");
  if (!anc || !prob) return fail(SPOCK_ERR_INVALID_ARG, "anc/prob must not be NULL");
  if (anc[0] != -1) return fail(SPOCK_ERR_BAD_TREE, "anc[0] must be -1 (node 0 is the root)");
  for (int32_t i = 1; i < n; ++i)
    if (anc[i] < 0 || anc[i] >= n || anc[i] == i)
      return fail(SPOCK_ERR_BAD_TREE, "anc[" + std::to_string(i) + "] out of range");
  t.n = n;
  t.anc_user.assign(anc, anc + n);
  t.prob_user.assign(prob, prob + n);
  // children lists in user numbering (increasing user id)
  std::vector<std::vector<int32_t>> ch(n);
  for (int32_t i = 1; i < n; ++i) ch[anc[i]].push_back(i);
  // breadth-first traversal from the root; nodes not reached => cycle
  t.user_of.clear();
  t.user_of.reserve(n);
  t.user_of.push_back(0);
  std::vector<int32_t> depth(n, -1);
  depth[0] = 0;
  for (size_t h = 0; h < t.user_of.size(); ++h) {
    int32_t u = t.user_of[h];
    for (int32_t c : ch[u]) {
      if (depth[c] >= 0) return fail(SPOCK_ERR_BAD_TREE, "ancestor array has a cycle");
      depth[c] = depth[u] + 1;
      t.user_of.push_back(c);
    }
  }
  if ((int32_t)t.user_of.size() != n)
    return fail(SPOCK_ERR_BAD_TREE, "ancestor array has a cycle (node not reachable from the root)");
  t.int_of.assign(n, -1);
  for (int32_t k = 0; k < n; ++k) t.int_of[t.user_of[k]] = k;
  t.parent.assign(n, -1);
  t.ch_begin.assign(n, 0);
  t.ch_count.assign(n, 0);
  t.stage.assign(n, 0);
  t.sib.assign(n, 0);
  t.prob.assign(n, 1.0);
  for (int32_t k = 0; k < n; ++k) {
    int32_t u = t.user_of[k];
    t.stage[k] = depth[u];
    t.ch_count[k] = (int32_t)ch[u].size();
    if (!ch[u].empty()) t.ch_begin[k] = t.int_of[ch[u][0]];
    for (size_t j = 0; j < ch[u].size(); ++j) {
      int32_t c = t.int_of[ch[u][j]];
      if (c != t.ch_begin[k] + (int32_t)j) return fail(SPOCK_ERR_BAD_TREE, "internal: children not contiguous");
      t.parent[c] = k;
      t.sib[c] = (int32_t)j;
      t.prob[c] = prob[ch[u][j]];
    }
  }
  // all leaves at one stage N >= 1
  int32_t N = -1;
  t.n_leaf = 0;
  for (int32_t k = 0; k < n; ++k) {
    if (t.ch_count[k] == 0) {
      ++t.n_leaf;
      if (N < 0) N = t.stage[k];
      else if (N != t.stage[k]) return fail(SPOCK_ERR_BAD_TREE, "all leaves must lie at the same stage");
    }
  }
  t.N = N;
  t.n_nonleaf = n - t.n_leaf;
  // breadth-first order puts stages in order; nonleaf nodes come first
  for (int32_t k = 0; k < n; ++k)
    if ((k < t.n_nonleaf) != (t.ch_count[k] > 0))
      return fail(SPOCK_ERR_BAD_TREE, "internal: nonleaf nodes are not the first ids");
  t.stage_begin.assign(N + 2, n);
  for (int32_t k = n - 1; k >= 0; --k) t.stage_begin[t.stage[k]] = k;
  t.stage_begin[N + 1] = n;
  t.stage_maxch.assign(N + 1, 0);
  for (int32_t k = 0; k < n; ++k) t.stage_maxch[t.stage[k]] = std::max(t.stage_maxch[t.stage[k]], t.ch_count[k]);
  // probabilities
  for (int32_t k = 0; k < t.n_nonleaf; ++k) {
    double s = 0.0;
    for (int32_t j = 0; j < t.ch_count[k]; ++j) {
      double p = t.prob[t.ch_begin[k] + j];
      if (!(p > 0.0) || !std::isfinite(p))
        return fail(SPOCK_ERR_INVALID_ARG, "child probabilities must be positive and finite");
      s += p;
    }
    if (std::fabs(s - 1.0) > 1e-9) return fail(SPOCK_ERR_INVALID_ARG, "child probabilities of a node must sum to 1");
  }
  // chain region: smallest stage from which every nonleaf node has one child
  int32_t cs = N;
  for (int32_t s = N - 1; s >= 0; --s) {
    bool one = true;
    for (int32_t k = t.stage_begin[s]; k < t.stage_begin[s + 1]; ++k) one = one && t.ch_count[k] == 1;
    if (!one) break;
    cs = s;
  }
  t.chain_stage = cs;
  return SPOCK_OK;
}

void build_offsets(const Tree& t, int nx, int nu, int nc, int ncN, const std::vector<int32_t>* ny_user,
                   Offsets& o) {
  const int32_t n = t.n;
  o.zx.assign(n, -1); o.zu.assign(n, -1); o.zz2.assign(n, -1); o.zs.assign(n, -1); o.ztau.assign(n, -1);
  o.enl.assign(n, -1); o.enr.assign(n, -1); o.elf.assign(n, -1);
  // user-order enumeration
  std::vector<int32_t> m(n, 0);
  for (int32_t i = 1; i < n; ++i) m[t.anc_user[i]]++;
  int64_t pos = 1;  // z[0] = s^0
  for (int32_t u = 0; u < n; ++u) { o.zx[t.int_of[u]] = pos; pos += nx; }
  for (int32_t u = 0; u < n; ++u) if (m[u]) { o.zu[t.int_of[u]] = pos; pos += nu; }
  auto ny = [&](int32_t u) { return ny_user ? (*ny_user)[u] : 2 * m[u] + 1; };
  for (int32_t u = 0; u < n; ++u) if (m[u]) { o.zz2[t.int_of[u]] = pos; pos += ny(u) + 2 * m[u]; }
  o.n_z = pos;
  o.zs[0] = 0;
  for (int32_t k = 1; k < n; ++k) {
    int32_t p = t.parent[k];
    int32_t mp = t.ch_count[p];
    const int32_t nyp = ny(t.user_of[p]);
    o.ztau[k] = o.zz2[p] + nyp + t.sib[k];
    o.zs[k] = o.zz2[p] + nyp + mp + t.sib[k];
  }
  pos = 0;
  for (int32_t u = 0; u < n; ++u) if (m[u]) { o.enl[t.int_of[u]] = pos; pos += ny(u) + 1 + nc; }
  for (int32_t u = 1; u < n; ++u) { o.enr[t.int_of[u]] = pos; pos += nx + nu + 2; }
  for (int32_t u = 0; u < n; ++u) if (!m[u]) { o.elf[t.int_of[u]] = pos; pos += ncN + nx + 2; }
  o.n_eta = pos;
}

}  // namespace spock
