"""Oracle visibility-gridding data reduction (Sec. 3.4, Eqs. 4-5).

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.

For channel l, with the whitened de-gridding matrix Theta_l G_l (the rows of
``nufft.Operator.G[l]``, 1/sigma_l folded in) and the whitened data y_l:

  H_l      = (Theta_l G_l)^H (Theta_l G_l)         K x K, Hermitian, sparse
  Lambda_l = 1 / sqrt(H_l[k, k]) on the rows k with H_l[k, k] > 0, else 0
  Gamma_l  = Lambda_l (Theta_l G_l)^H               gridding operator
  y'_l     = Gamma_l y_l                            (Eq. 4)
  Phi'_l   = Lambda_l H_l F Z                       (Eq. 5)

kept on the M'_l rows where Lambda_l is nonzero (the gridded data points).
Readings where the paper is silent:

* Blocks are aggregated after gridding: one l2 ball per channel, over all of
  the channel's visibilities (the paper's own DR experiment uses one block).
* Default bound: for unit-variance whitened noise n, E ||Gamma_l n||^2 =
  trace(Lambda_l H_l Lambda_l) = M'_l, so Eq. 2's chi-square bound is taken
  with M'_l degrees of freedom: eps'_l^2 = M'_l + 2 sqrt(M'_l).  The paper
  sets eps' from model visibilities of a calibration step instead
  (eps' = ||y' - Gamma ybar||), which a caller can pass as eps.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import nufft, prox


class Reduced:
    """Phi'_l, y'_l and Lambda_l for every channel of a problem."""

    def __init__(self, op: nufft.Operator, yw: list):
        self.op = op
        self.L = op.L
        self.K = op.geom.K1 * op.geom.K2
        self.rows, self.lam, self.Hr, self.y = [], [], [], []
        for l in range(self.L):
            G = sp.csr_matrix(op.G[l])
            Gh = sp.csr_matrix(G.conj().T)
            H = sp.csr_matrix(Gh @ G)                      # (Theta G)^H (Theta G)
            d = np.real(H.diagonal())
            rows = np.flatnonzero(d > 0.0)
            lam = 1.0 / np.sqrt(d[rows])
            self.rows.append(rows)
            self.lam.append(lam)
            self.Hr.append(sp.csr_matrix(H[rows, :]))      # the M'_l nonzero rows of H
            self.y.append(lam * (Gh @ np.asarray(yw[l]))[rows])

    def m_red(self, l: int) -> int:
        return len(self.rows[l])

    def gamma(self, v: np.ndarray, l: int) -> np.ndarray:
        """Gamma_l v for visibilities v of channel l (the gridding of Eq. 4)."""
        return self.lam[l] * (self.op.G[l].conj().T @ v)[self.rows[l]]

    def forward(self, x: np.ndarray, l: int) -> np.ndarray:
        """Phi'_l x = Lambda_l H_l F Z x on the M'_l gridded points."""
        return self.lam[l] * (self.Hr[l] @ self.op.fzx(x).ravel())

    def adjoint(self, v: np.ndarray, l: int) -> np.ndarray:
        """Re(Phi'_l^H v) = Re(Z^T F^H H_l Lambda_l v) (H_l Hermitian)."""
        grid = (self.Hr[l].conj().T @ (self.lam[l] * v)).reshape(self.op.geom.K1, self.op.geom.K2)
        return self.op.zf_adj(grid)

    def eps_default(self) -> np.ndarray:
        """eps'_l = sqrt(M'_l + 2 sqrt(M'_l)) per channel (one block each)."""
        return np.array([prox.eps_blocks(self.m_red(l), np.array([self.m_red(l)]))[0] if self.m_red(l) else 0.0
                         for l in range(self.L)])

    def norm2_eigsh(self, l: int, tol: float = 1e-12) -> float:
        """||Phi'_l||^2 as the largest eigenvalue of Re(Phi'_l^H Phi'_l) by ARPACK's
        implicitly restarted Lanczos (scipy ``eigsh``)."""
        from scipy.sparse.linalg import LinearOperator, eigsh
        ny, nx = self.op.geom.ny, self.op.geom.nx

        def mv(x):
            return np.asarray(self.adjoint(self.forward(np.asarray(x).reshape(ny, nx), l), l)).ravel()

        A = LinearOperator((ny * nx, ny * nx), matvec=mv, dtype=np.float64)
        v0 = np.random.default_rng(0).standard_normal(ny * nx)
        return float(eigsh(A, k=1, which="LA", tol=tol, v0=v0, return_eigenvectors=False)[0])

    def norm2(self, l: int, n_iter: int = 200, tol: float = 1e-10, seed: int = 0) -> float:
        """||Phi'_l||^2 by power iteration on Re(Phi'_l^H Phi'_l)."""
        rng = np.random.default_rng(seed)
        x = rng.standard_normal((self.op.geom.ny, self.op.geom.nx))
        x /= np.linalg.norm(x)
        lam = 0.0
        for _ in range(n_iter):
            y = self.adjoint(self.forward(x, l), l)
            lam_new = float(np.vdot(x, y).real)
            x = y / np.linalg.norm(y)
            if abs(lam_new - lam) <= tol * abs(lam_new):
                return lam_new
            lam = lam_new
        return lam
