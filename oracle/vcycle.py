"""Reference multigrid cycle on the assembled Galerkin hierarchy — oracle, test infra.

The standard geometric-multigrid recursion of Alg. 1: on every level but the coarsest,
smooth, form the residual, restrict it with R = P^T, solve the coarse problem from a zero
guess (recursively), add the prolongated correction and smooth again; the coarsest level is
solved directly:

    for l = 1..L-1: pre-smooth; r^l = f^l - K^l u^l; f^{l+1} = R r^l; u^{l+1} = 0
    coarsest solve
    for l = L-1..1: u^l += P u^{l+1}; post-smooth

The smoother is selectable: damped block-Jacobi, u <- u + omega D^-1 (f - K u)
applied to all nodes at once (the update form of Sec. 4.6), or Chebyshev, or the 8-colour
Gauss-Seidel form of Sec. 4.6. D^l is the block diagonal of K^l (D x D node blocks). The
coarsest solve (an exact solve in place of Alg. 1's inexact coarsest smoothing) is the
solution of (K^L + rho J) u = f^L, J the per-component all-ones coupling and rho the mean
diagonal of K^L: for right-hand sides orthogonal to translations this is the zero-mean
solution of K^L u = f^L.

8-colour Gauss-Seidel (Sec. 4.6): the nodes of a level are coloured by the parity of their
coordinates, c = (x&1) + 2(y&1) + 4(z&1); nodes of one colour share no stencil entry, so
each colour is updated at once with the damped block-Jacobi step
u_c <- u_c + omega (D^{-1} (f - K u))_c on the latest u, colours 0..7 in turn, per sweep.

Injected corrections (Alg. 2): the only change to the recursion is the starting value of
each coarse unknown on the first descent, a given field e^l instead of zero, from which it
is pre-smoothed as usual; the fine level starts from the given u. With the coarsest level
solved exactly, its entry has no effect.

Cycle schedules (Sec. 5 compares V-, W- and F-cycles; it prints no pseudocode): the coarse
problem of level l is solved by one cycle of the same kind (V), by two W-cycles (the second
starting from the first's result), or by an F-cycle followed by a V-cycle; the coarsest
level is solved once.

Chebyshev: one polynomial of degree k = nu (the sweep count, so that both smoothers apply K
the same number of times) on D^{-1}K over [a, b] = [lmax/ratio, upper*lmax]:
theta = (b+a)/2, delta = (b-a)/2, sigma = theta/delta, rho_0 = 1/sigma; d = D^{-1} r/theta;
then k times: u += d; if not last: r = f - K u, rho' = 1/(2 sigma - rho),
d = rho' rho d + (2 rho'/delta) D^{-1} r, rho = rho'. After k steps the error component
along an eigenvector of D^{-1}K with eigenvalue lam is multiplied by
T_k((theta - lam)/delta) / T_k(theta/delta) (the textbook Chebyshev semi-iteration).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def block_diag_inverse(K, D: int):
    """Inverse of the D x D node blocks on the diagonal of K, as a sparse matrix."""
    n = K.shape[0] // D
    Kd = K.tocsr()
    blocks = np.zeros((n, D, D))
    for i in range(D):
        for j in range(D):
            rows = np.arange(n) * D + i
            cols = np.arange(n) * D + j
            blocks[:, i, j] = np.asarray(Kd[rows, cols]).reshape(-1)
    inv = np.linalg.inv(blocks)
    r = (np.arange(n)[:, None, None] * D + np.arange(D)[None, :, None]).repeat(D, axis=2)
    c = (np.arange(n)[:, None, None] * D + np.arange(D)[None, None, :]).repeat(D, axis=1)
    return sp.csr_matrix((inv.reshape(-1), (r.reshape(-1), c.reshape(-1))), shape=K.shape)


def coarsest_matrix(KL, D: int) -> np.ndarray:
    A = KL.toarray()
    n = A.shape[0] // D
    rho = float(np.mean(np.diag(A)))
    for c in range(D):
        idx = np.arange(n) * D + c
        A[np.ix_(idx, idx)] += rho
    return A


class VCycle:
    def __init__(self, Ks, Ps, D: int, nu_pre=2, nu_post=2, omega=0.6, smoother="jacobi",
                 cheb_lmax=None, cheb_ratio=30.0, cheb_upper=1.1, kind="V", levels=None,
                 nu_coarse=0):
        """nu_pre / nu_post sweeps on level 0; nu_coarse (> 0) sweeps before and after the
        coarse correction on every level >= 1 (0: nu_pre / nu_post there too)."""
        self.Ks, self.Ps, self.D = Ks, Ps, D
        self.nu_pre, self.nu_post, self.omega = nu_pre, nu_post, omega
        self.nu_coarse = nu_coarse
        self.smoother = smoother
        self.Dinv = [block_diag_inverse(K, D) for K in Ks[:-1]]
        self.Ainv = np.linalg.inv(coarsest_matrix(Ks[-1], D))
        self.lmax = cheb_lmax
        self.ratio, self.upper = cheb_ratio, cheb_upper
        self.kind = kind
        # per-dof colour masks for the 8-colour smoother (levels: the oracle grid.Level list)
        self.colour_masks = None
        if smoother == "gs8":
            self.colour_masks = []
            for lev in levels[:-1]:
                xyz = lev.node_xyz()
                col = (xyz[:, 0] & 1) + 2 * (xyz[:, 1] & 1) + 4 * (xyz[:, 2] & 1)
                self.colour_masks.append([np.repeat(col == c, D) for c in range(8)])

    def smooth(self, l: int, u, f, sweeps: int):
        K, Di = self.Ks[l], self.Dinv[l]
        if self.smoother == "jacobi":
            for _ in range(sweeps):
                u = u + self.omega * (Di @ (f - K @ u))
            return u
        if self.smoother == "gs8":
            for _ in range(sweeps):
                for c in range(8):
                    m = self.colour_masks[l][c]
                    step = self.omega * (Di @ (f - K @ u))
                    u = u.copy()
                    u[m] += step[m]
            return u
        lmax = self.lmax[l]
        b = self.upper * lmax
        a = lmax / self.ratio
        theta, delta = 0.5 * (b + a), 0.5 * (b - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = (Di @ (f - K @ u)) / theta
        for i in range(sweeps):
            u = u + d
            if i == sweeps - 1:
                break
            r = f - K @ u
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (Di @ r)
            rho = rho_new
        return u

    def cycle(self, f, u=None, level: int = 0, kind=None, e=None):
        """One cycle on K_level u = f from u (zero if None). e: the injected corrections of
        Alg. 2, one entry per level (None, or the starting value of that level's coarse
        unknown on the first descent instead of zero); the coarsest level is solved
        exactly, so its entry changes nothing."""
        L = len(self.Ks)
        kind = self.kind if kind is None else kind
        if level == L - 1:
            return self.Ainv @ f
        if u is None:
            u = np.zeros_like(f)
        pre, post = self.nu_pre, self.nu_post
        if level > 0 and self.nu_coarse > 0:
            pre = post = self.nu_coarse
        u = self.smooth(level, u, f, pre)
        r = f - self.Ks[level] @ u
        fc = self.Ps[level].T @ r
        start = None if e is None or e[level + 1] is None else np.array(e[level + 1], dtype=float)
        uc = self.cycle(fc, start, level + 1, kind, e)
        if level + 2 < L and kind != "V":
            uc = self.cycle(fc, uc, level + 1, "W" if kind == "W" else "V")
        u = u + self.Ps[level] @ uc
        u = self.smooth(level, u, f, post)
        return u
