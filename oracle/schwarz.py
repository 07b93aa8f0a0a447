"""One- and two-level additive Schwarz preconditioners (oracle, FP64).

Eq. 2.22: M_AS,1^{-1} = sum_i E_i (B_i)^{-1} R_i with B_i = R_i B E_i, where
R_i is the Boolean restriction to dof(Omega_i) (the L^2 adjoint of the zero
extension E_i, Sec. 2.3).  The sum is unweighted.  With one decomposition
(the coarse and fine subdomains coincide, Q_i = 1) the local problems are
posed on the same overlapping subdomains as the eigenproblems.

Eq. 2.23: M_AS,2^{-1} = E_0 B_0^{-1} R_0 + M_AS,1^{-1}, B_0 = R_0 B E_0,
in matrix form Z E^{-1} Z^T with E = Z^T B Z.

Variants selected by `levels`: "two" (Eq. 2.23), "one" (Eq. 2.22 alone),
"coarse" (the coarse term alone).  `weighting="ras_pou"` multiplies each
local solution by the partition-of-unity weights 1/mu before summing (a
variant; the paper's Eq. 2.22 is unweighted).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class SingularLocal(RuntimeError):
    pass


class SingularCoarse(RuntimeError):
    pass


# A pivot below PIVOT_TOL * max|entry| marks the matrix singular.  An exactly
# singular local matrix (k^2 a Dirichlet eigenvalue, Remark after Lemma 3.4)
# leaves a rounding-level pivot of 1e-14 .. 1e-10 relative at these sizes, so
# the threshold sits above that floor.
PIVOT_TOL = 1e-10


def _checked_lu(Mat, what, exc):
    lu, piv = sla.lu_factor(Mat, check_finite=True)
    d = np.abs(np.diag(lu))
    scale = max(np.abs(Mat).max(), 1e-300)
    if d.size and d.min() <= PIVOT_TOL * scale:
        raise exc(f"{what}: pivot {d.min():.3e} below {PIVOT_TOL:g} * {scale:.3e}")
    return lu, piv


class AdditiveSchwarz:
    def __init__(self, B, subs, mu, Z=None, levels: str = "two", weighting: str = "as"):
        self.levels = levels
        self.weighting = weighting
        self.subs = subs
        self.mu = mu
        self.n = B.shape[0]
        self.local = []
        if levels in ("two", "one"):
            Bd = B.tocsr()
            for i, sd in enumerate(subs):
                Bi = Bd[sd.dof][:, sd.dof].toarray()
                self.local.append(_checked_lu(Bi, f"local matrix of subdomain {i}", SingularLocal))
        self.Z = None
        if levels in ("two", "coarse") and Z is not None and Z.shape[1] > 0:
            from .geneo import coarse_matrix
            self.Z = Z.tocsr()
            self.E = coarse_matrix(B, self.Z)
            self.E_lu = _checked_lu(self.E, "coarse matrix", SingularCoarse)

    def apply(self, v: np.ndarray) -> np.ndarray:
        z = np.zeros(self.n)
        if self.levels in ("two", "one"):
            for sd, f in zip(self.subs, self.local):
                y = sla.lu_solve(f, v[sd.dof])
                if self.weighting == "ras_pou":
                    y = y / self.mu[sd.dof]
                z[sd.dof] += y
        if self.Z is not None:
            z += self.Z @ sla.lu_solve(self.E_lu, self.Z.T @ v)
        return z
