"""Projections onto the sets of the splitting: S2 (Sec. "Projection on S2")
and S3 (Eq. (S3-def)), and prox of g* (Eq. (prox:g)).  Oracle (test
infrastructure only).

Readings taken where the paper is silent or garbled:
  * SOC_d = {(v, t) in R^{d-1} x R : ||v|| <= t} with t the LAST coordinate;
    it is the orientation for which the translation (0, 1/2, -1/2) encodes
    x'Qx + u'Ru <= tau.
  * Eq. (prox:g) prints eta - proj_S3(eta / alpha); the extended Moreau
    decomposition for g = indicator of S3 gives
    prox_{alpha g*}(eta) = eta - alpha proj_S3(eta / alpha), used here.
  * (K^i)* for K^i = R^{2m}_+ x {0} is R^{2m}_+ x R; for a general conic
    risk measure K^i = R^kp_+ x {0}^(ny - kp) and (K^i)* = R^kp_+ x R^(ny - kp).

Pins (tests/test_oracle_cones.py): Moreau decomposition and orthogonality
for the SOC, a brute-force grid search for SOC dims 2-3, the optimality
condition of prox_{alpha g*} checked against sampled points of S3, the
kernel property and idempotence of proj_S2.
"""
from __future__ import annotations

import numpy as np

from .problem import Problem


def proj_soc(w):
    """Euclidean projection onto SOC = {(v, t): ||v|| <= t}."""
    w = np.asarray(w, float)
    v, t = w[:-1], w[-1]
    nv = float(np.linalg.norm(v))
    if nv <= t:
        return w.copy()
    if nv <= -t:
        return np.zeros_like(w)
    scale = 0.5 * (nv + t)
    return np.concatenate([scale * v / nv, [scale]])


def proj_translated_soc(w, shift):
    """Projection onto SOC + shift."""
    return shift + proj_soc(w - shift)


def proj_S3(w, P: Problem):
    """Projection of an eta-shaped vector onto S3, block by block."""
    t, lay = P.tree, P.lay
    out = np.array(w, dtype=float, copy=True)
    for i in t.nonleaf:
        ey = lay.e_y[i]
        kp = P.kp(i)
        out[ey[:kp]] = np.maximum(w[ey[:kp]], 0.0)           # (K^i)* = R^kp_+ x R^(ny - kp)
        out[lay.e_sb[i]] = max(w[lay.e_sb[i]], 0.0)          # R_+
        if P.general:                                        # C^i = [cmin, cmax]
            out[lay.e_c[i]] = np.clip(w[lay.e_c[i]], P.cmin[i], P.cmax[i])
        else:                                                # C^i = box on (x, u)
            out[lay.e_x[i]] = np.clip(w[lay.e_x[i]], P.xmin[i], P.xmax[i])
            out[lay.e_u[i]] = np.clip(w[lay.e_u[i]], P.umin[i], P.umax[i])
    shift_nr = np.zeros(P.nx + P.nu + 2)
    shift_nr[-2:] = (0.5, -0.5)
    for c in t.nonroot:
        idx = np.concatenate([lay.e_qx[c], lay.e_ru[c], lay.e_t[c]])
        out[idx] = proj_translated_soc(w[idx], shift_nr)
    shift_lf = np.zeros(P.nx + 2)
    shift_lf[-2:] = (0.5, -0.5)
    for j in t.leaves:
        if P.general:                                        # C_N^j
            out[lay.e_lc[j]] = np.clip(w[lay.e_lc[j]], P.cNmin[j], P.cNmax[j])
        else:
            out[lay.e_lx[j]] = np.clip(w[lay.e_lx[j]], P.xmin[j], P.xmax[j])
        idx = np.concatenate([lay.e_qn[j], lay.e_ls[j]])
        out[idx] = proj_translated_soc(w[idx], shift_lf)
    return out


def prox_gconj(eta, alpha, P: Problem):
    """prox_{alpha g*}(eta) = eta - alpha proj_S3(eta / alpha)."""
    return eta - alpha * proj_S3(eta / alpha, P)


def s2_matrix(P: Problem, i):
    """The matrix [[E^iT, -I, -I], [F^iT, 0, 0]] whose kernel is S2^i (F^i
    has no columns for AV@R), acting on (y^i, tau^[i], s^[i])."""
    m = len(P.tree.children[i])
    top = np.hstack([P.E(i).T, -np.eye(m), -np.eye(m)])
    F = P.F(i)
    if F.shape[1] == 0:
        return top
    return np.vstack([top, np.hstack([F.T, np.zeros((F.shape[1], 2 * m))])])


def z2_block(P: Problem, i):
    """Indices of (y^i, tau^[i], s^[i]) in z (contiguous)."""
    lay = P.lay
    ch = P.tree.children[i]
    return np.concatenate([lay.y[i], [lay.tau[c] for c in ch], [lay.s[c] for c in ch]]).astype(int)


def proj_S2_block(w, M):
    """Projection onto ker M through the pseudoinverse: w - M^+ M w."""
    return w - np.linalg.pinv(M) @ (M @ w)


def proj_S2(z, P: Problem):
    """Apply proj_S2^i to every z_2 block of a z-shaped vector (other entries
    are copied)."""
    out = np.array(z, dtype=float, copy=True)
    for i in P.tree.nonleaf:
        idx = z2_block(P, i)
        out[idx] = proj_S2_block(z[idx], s2_matrix(P, i))
    return out
