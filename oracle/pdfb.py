"""Oracle Faceted HyperSARA PDFB iteration with reweighting (Eq. 3, Sec. 2.2.3).

Test infrastructure: imported only by the tests, the smoke check and the
CPU-baseline leg of the benchmark.  Parity unpinned for the iterate after k
steps (the paper prints none); see the package header.

The paper states the objective (Eq. 2-3), the priors (Sec. 2.2.2) and that
the solver is a primal-dual forward-backward method (Condat 2013, Vu 2013)
inside a log-sum reweighting loop (Candes 2009); the steps themselves are in
the companion paper.  This is the plain Condat-Vu reading with three dual
groups, taken one step at a time:

  x+    = max(0, x - tau (L0^T u0 + L1^T u1 + L2^T u2))      non-negativity
  xbar  = 2 x+ - x
  u_i   = u_i + s_i L_i xbar - s_i prox_{g_i / s_i}(u_i / s_i + L_i xbar)

with L0 = the stacked facet selections S_q (low-rankness, weighted nuclear
norm mu_bar), L1 = Psi^dagger per channel (average joint sparsity, weighted
l21 norm mu), L2 = Phi_{l,b} (l2 balls).  Steps: s1 = 1 (||Psi|| = 1),
s0 = 1 / max facet coverage (= ||L0||^2), s2 = 1 / max_l ||Phi_l||^2,
tau = 0.99 / 3.  Start: x = 0, all duals 0, all weights 1.  Reweighting:
w_r = upsilon / (upsilon + ||(Psi^dagger X)_r||), w_{q,i} = upsilon_bar /
(upsilon_bar + sigma_i(S_q X)), duals kept.  Channels l of sub-cube c are
l = c, c + C, ... (channel interleaving, Eq. 3).  With ``reduction`` the data
term is that of the gridded data (Sec. 3.4, see ``reduction.py``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import nufft, prox, wavelets
from . import reduction as reduction_mod


@dataclass
class Steps:
    tau: float
    sigma0: float
    sigma1: float
    sigma2: float


class FHS:
    """Whole-problem state: C sub-cubes of the image cube X (L, ny, nx)."""

    def __init__(self, omega, w, y, sigma, block_offsets, ny, nx, C, qy, qx, overlap,
                 mu, mu_bar, upsilon=1e-3, upsilon_bar=1e-3, w_max=0.0, n_wplanes=64,
                 pixel_size=0.0, levels=4, eps=None, steps: Steps | None = None,
                 faceted_sara: bool = False, sara_q=(1, 1), dde=None, reduction: bool = False):
        self.L = omega.shape[0]
        self.ny, self.nx, self.C = ny, nx, C
        self.geom = nufft.Geometry(ny, nx, w_max=w_max, n_wplanes=n_wplanes, pixel_size=pixel_size)
        self.op = nufft.Operator(omega, w, sigma, self.geom, dde=dde)
        self.yw = [y[l] / sigma[l] for l in range(self.L)]                 # Theta_l y_l
        self.bo = np.asarray(block_offsets, dtype=np.int64)
        # data term: Phi_l on the visibility blocks, or with the data reduction of
        # Sec. 3.4 Phi'_l on the gridded data y'_l, one block per channel
        self.data = self.op
        if reduction:
            self.red = reduction_mod.Reduced(self.op, self.yw)
            self.data = self.red
            self.yw = self.red.y
            self.bo = np.array([[0, self.red.m_red(l)] for l in range(self.L)], dtype=np.int64)
            if eps is None:
                eps = self.red.eps_default()
        B = self.bo.shape[1] - 1
        if eps is None:
            eps = np.stack([prox.eps_blocks(len(self.yw[l]), np.diff(self.bo[l])) for l in range(self.L)])
        self.eps = np.asarray(eps, dtype=np.float64).reshape(self.L, B)
        self.sara = (wavelets.FacetedSara(ny, nx, *sara_q, levels) if faceted_sara
                     else wavelets.Sara(ny, nx, levels))
        self.facets = prox.nuclear_facets(ny, nx, qy, qx, overlap)
        self.mu, self.mu_bar = float(mu), float(mu_bar)
        self.upsilon, self.upsilon_bar = float(upsilon), float(upsilon_bar)
        self.chans = [list(range(c, self.L, C)) for c in range(C)]
        if steps is None:
            nrm = max(self.data.norm2(l) for l in range(self.L))
            cov = prox.facet_coverage(ny, nx, self.facets).max()
            steps = Steps(tau=0.99 / 3.0, sigma0=1.0 / cov, sigma1=1.0, sigma2=1.0 / nrm)
        self.steps = steps
        # state
        self.X = np.zeros((self.L, ny, nx))
        self.v = [np.zeros_like(self.yw[l]) for l in range(self.L)]
        self.W = [np.zeros((len(ch), self.sara.n_coef)) for ch in self.chans]
        self.P = [[np.zeros((len(ch), y1 - y0, x1 - x0)) for (y0, y1, x0, x1) in self.facets]
                  for ch in self.chans]
        self.w21 = [np.ones(self.sara.n_coef) for _ in self.chans]
        self.wnuc = [[np.ones(len(ch)) for _ in self.facets] for ch in self.chans]
        self.A_data = np.zeros_like(self.X)
        self.A_sara = np.zeros_like(self.X)
        self.A_nuc = np.zeros_like(self.X)
        self.n_done = 0

    # -- one PDFB iteration --------------------------------------------------
    def step(self) -> float:
        st = self.steps
        X = self.X
        Xp = np.maximum(0.0, X - st.tau * (self.A_nuc + self.A_sara + self.A_data))
        Xb = 2.0 * Xp - X
        # data fidelity: l2 balls per block, then the adjoint Re(Phi_l^H v_l)
        for l in range(self.L):
            phix = self.data.forward(Xb[l], l)
            for b in range(self.bo.shape[1] - 1):
                s0, s1 = self.bo[l, b], self.bo[l, b + 1]
                self.v[l][s0:s1] = prox.l2ball_dual(self.v[l][s0:s1], phix[s0:s1],
                                                    self.yw[l][s0:s1], self.eps[l, b], st.sigma2)
            self.A_data[l] = self.data.adjoint(self.v[l], l)
        # average joint sparsity: weighted l21 over each sub-cube
        for c, ch in enumerate(self.chans):
            Aw = self.sara.analysis(Xb[ch])
            self.W[c] = prox.l21_dual(self.W[c], Aw, st.sigma1, self.mu, self.w21[c])
            self.A_sara[ch] = self.sara.synthesis(self.W[c])
        # faceted low-rankness: weighted nuclear norm per spatio-spectral facet
        self.A_nuc[:] = 0.0
        for c, ch in enumerate(self.chans):
            for q, (y0, y1, x0, x1) in enumerate(self.facets):
                self.P[c][q] = prox.nuclear_dual(self.P[c][q], Xb[ch, y0:y1, x0:x1], st.sigma0,
                                                 self.mu_bar, self.wnuc[c][q])
                self.A_nuc[ch, y0:y1, x0:x1] += self.P[c][q]
        num = np.linalg.norm(Xp - X)
        den = np.linalg.norm(Xp)
        self.X = Xp
        self.n_done += 1
        return float(num / den) if den > 0 else float("inf")

    # -- outer reweighting ---------------------------------------------------
    def reweight(self):
        for c, ch in enumerate(self.chans):
            self.w21[c] = prox.l21_weights(self.sara.analysis(self.X[ch]), self.upsilon)
            for q, (y0, y1, x0, x1) in enumerate(self.facets):
                Z = self.X[ch, y0:y1, x0:x1].reshape(len(ch), -1).T
                self.wnuc[c][q] = prox.nuclear_weights(Z, self.upsilon_bar, len(ch))

    def run(self, n_iter: int, n_reweight: int = 0) -> list:
        """n_reweight + 1 inner runs of n_iter // (n_reweight + 1) iterations
        each (the remainder in the last), reweighting between them."""
        rels = []
        per = n_iter // (n_reweight + 1)
        for r in range(n_reweight + 1):
            k = per if r < n_reweight else n_iter - per * n_reweight
            for _ in range(k):
                rels.append(self.step())
            if r < n_reweight:
                self.reweight()
        return rels

    def residual_norms(self) -> np.ndarray:
        """||Phi_{l,b} x_l - y_{l,b}|| for every block (feasibility check)."""
        out = np.zeros(self.eps.shape)
        for l in range(self.L):
            r = self.data.forward(self.X[l], l) - self.yw[l]
            for b in range(self.bo.shape[1] - 1):
                out[l, b] = np.linalg.norm(r[self.bo[l, b]:self.bo[l, b + 1]])
        return out
