"""FP64 ORACLE of the partial diffusion approximation (App. A) on spherical-polar grids.

Test infrastructure only (tests, the smoke check, the bench's CPU legs); the CUDA library
never imports it.  Follows App. A as written:

* cells with dust that the Monte-Carlo step sampled with fewer than ``n_min`` packet path
  segments get their temperature from the diffusion equation div(D grad T^4) = 0,
  D = 1 / (3 rho chi_R) (the paper solves for Adot / kappa_P(Adot), which in LTE equals
  4 sigma T^4 (Eq. 3), i.e. T^4 up to a constant);
* the discrete equation per cell (i, j, k) is the one printed in App. A: for each coordinate, the
  difference of T^4 to the neighbour divided by the sum of the two cells' Rosseland optical
  depths across them along that coordinate (Delta tau^r = rho chi_R Delta r,
  Delta tau^theta = rho chi_R r Delta theta, Delta tau^phi = rho chi_R r sin(theta) Delta phi),
  weighted by r^2 at the radial walls over r_i^2 Delta r_i, by sin(theta) at the polar walls over
  sin(theta_j) r Delta theta_j, and by 1 / (r sin(theta) Delta phi_k) in phi; r, theta at cell
  centres;
* well-sampled neighbours act as boundary values (App. A: "these values act as boundary
  conditions"); the solution is the formal solution of the linear system (here a sparse
  direct solve).

Readings where App. A is silent: chi_R is the Rosseland mean of the extinction at the cell's
temperature from the previous iteration; a neighbour outside the grid or without dust adds no
term (no flux); phi is periodic; a connected region of diffusion cells with no well-sampled
neighbour keeps its Monte-Carlo temperatures; Adot of a diffusion cell is E(T) (Eq. 3).
"""
from __future__ import annotations

import numpy as np
from scipy import sparse
from scipy.sparse import csgraph
from scipy.sparse import linalg as splinalg

from . import tables as T


def _faces(shape):
    """Neighbour index arrays and face kinds of an (n3, n2, n1) grid in C order.
    Yields (axis, sign, neighbour flat index or -1 outside the grid)."""
    n3, n2, n1 = shape
    k, j, i = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    out = []
    for axis, sign in ((0, +1), (0, -1), (1, +1), (1, -1), (2, +1), (2, -1)):
        ii, jj, kk = i.copy(), j.copy(), k.copy()
        if axis == 0:
            ii = ii + sign
            inside = (ii >= 0) & (ii < n1)
        elif axis == 1:
            jj = jj + sign
            inside = (jj >= 0) & (jj < n2)
        else:
            kk = (kk + sign) % n3           # phi is periodic
            inside = np.ones_like(kk, dtype=bool)
        nb = np.where(inside, (kk * n2 + np.clip(jj, 0, n2 - 1)) * n1 + np.clip(ii, 0, n1 - 1), -1)
        out.append((axis, sign, nb.reshape(-1)))
    return out


def face_weights(walls_cm, rho, chi_r):
    """Weights W[f][c] of the App. A equation of cell c multiplied by r_i^2 Delta r_i
    sin(theta_j) Delta theta_j Delta phi_k, which makes the system symmetric (the weight of a
    face is the same seen from both cells).  rho and chi_r are flat [k][j][i] arrays."""
    rw, tw, pw = (np.asarray(w, dtype=np.float64) for w in walls_cm)
    n1, n2, n3 = len(rw) - 1, len(tw) - 1, len(pw) - 1
    rc = 0.5 * (rw[1:] + rw[:-1])
    dr = np.diff(rw)
    tc = 0.5 * (tw[1:] + tw[:-1])
    dt = np.diff(tw)
    dp = np.diff(pw)
    K, J, I = np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij")
    I, J, K = I.reshape(-1), J.reshape(-1), K.reshape(-1)
    rk = rho * chi_r                                   # extinction per length
    dtau = [rk * dr[I], rk * rc[I] * dt[J], rk * rc[I] * np.sin(tc[J]) * dp[K]]
    W = []
    for axis, sign, nb in _faces((n3, n2, n1)):
        ok = nb >= 0
        nbs = np.where(ok, nb, 0)
        den = dtau[axis] + dtau[axis][nbs]
        if axis == 0:
            r_face = rw[I + (sign > 0)]                 # r_{i+1/2} or r_{i-1/2}
            num = r_face ** 2 * np.sin(tc[J]) * dt[J] * dp[K]
        elif axis == 1:
            s_face = np.sin(tw[J + (sign > 0)])         # sin(theta_{j+-1/2})
            num = rc[I] * dr[I] * dp[K] * s_face
        else:
            num = rc[I] * dr[I] * dt[J]
        with np.errstate(divide="ignore", invalid="ignore"):
            w = np.where(ok & (den > 0), num / den, 0.0)
        W.append((nb, w))
    return W


def pda_mask(rho, visits, n_min):
    """Cells with dust sampled by fewer than n_min packet path segments."""
    return (np.asarray(rho) > 0) & (np.asarray(visits) < n_min)


def solve(walls_cm, rho, T_mc, T_prev, visits, n_min, T_nodes, chi_r_nodes):
    """Temperatures after the PDA: T_mc outside the diffusion region, the formal solution of
    the App. A system inside it.  Returns (T, mask of the cells solved)."""
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)
    T_mc = np.asarray(T_mc, dtype=np.float64).reshape(-1)
    nc = rho.size
    mask = pda_mask(rho, np.asarray(visits).reshape(-1), n_min)
    dust = rho > 0
    chi_r = T.interp_loglog(np.asarray(T_prev, dtype=np.float64).reshape(-1), T_nodes, chi_r_nodes)
    W = face_weights(walls_cm, rho, chi_r)
    # keep the regions that touch a well-sampled cell
    rows, cols = [], []
    anchored = np.zeros(nc, dtype=bool)
    for nb, w in W:
        use = mask & (nb >= 0) & (w > 0)
        nbs = np.where(use, nb, 0)
        inner = use & mask[nbs] & dust[nbs]
        rows.append(np.flatnonzero(inner))
        cols.append(nbs[inner])
        anchored |= use & dust[nbs] & ~mask[nbs]
    g = sparse.coo_matrix((np.ones(sum(len(r) for r in rows)), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(nc, nc)).tocsr()
    ncomp, label = csgraph.connected_components(g, directed=False)
    good = np.zeros(ncomp, dtype=bool)
    good[np.unique(label[anchored & mask])] = True
    mask = mask & good[label]
    idx = np.flatnonzero(mask)
    T_out = T_mc.copy()
    if idx.size == 0:
        return T_out, mask
    pos = -np.ones(nc, dtype=np.int64)
    pos[idx] = np.arange(idx.size)
    x_known = T_mc ** 4
    diag = np.zeros(idx.size)
    b = np.zeros(idx.size)
    ar, ac, av = [], [], []
    for nb, w in W:
        wc = w[idx]
        nbc = nb[idx]
        use = (nbc >= 0) & (wc > 0)
        nbs = np.where(use, nbc, 0)
        use &= dust[nbs]
        diag += np.where(use, wc, 0.0)
        inner = use & mask[nbs]
        ar.append(np.flatnonzero(inner))
        ac.append(pos[nbs[inner]])
        av.append(-wc[inner])
        bnd = use & ~mask[nbs]
        b += np.where(bnd, wc * x_known[nbs], 0.0)
    A = sparse.coo_matrix((np.concatenate([np.concatenate(av), diag]),
                           (np.concatenate([np.concatenate(ar), np.arange(idx.size)]),
                            np.concatenate([np.concatenate(ac), np.arange(idx.size)]))),
                          shape=(idx.size, idx.size)).tocsc()
    x = splinalg.spsolve(A, b)
    T_out[idx] = np.clip(x, 1e-300, None) ** 0.25
    return T_out, mask
