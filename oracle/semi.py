"""FP64 oracle of the semi-implicit (lagged-diffusivity) fixed-point scheme.
TEST INFRASTRUCTURE ONLY (see the package docstring).

The explicit iteration of App. A-A needs tau < 2/(||D Delta|| + lambda M),
and ||D Delta|| grows like 8/eps: with the paper's eps = 1e-3 no practical
tau converges.  The semi-implicit scheme takes the diffusion term implicitly
with its coefficient D frozen at the current iterate (lagged diffusivity) and
the nonlocal term explicitly:

    (I/s + L_n) u^{n+1} = u^n/s - lambda G(u^n) + Phi,
    (L_n v)_i = sum over the faces f of pixel i of D_f(u^n) (v_i - v_nb(f)),

v_nb the neighbour across the face, extended by the boundary rule (reflecting:
the ghost equals v_i, so border faces drop out; Dirichlet: the ghost is 0).
L_n v = -div(D(u^n) grad v), so a fixed point satisfies -div(D grad u) +
lambda G(u) = Phi, the equation of Sec. II.  I/s + L_n is symmetric positive
definite.  Here each step is solved exactly (scipy sparse LU); the stop rule
is the explicit solver's: rho_n = ||F(u^n)|| / ||Phi|| per channel, stop at
the first n with max_c rho_n <= tol or n == max_iter.

Parity status: pinned by tests/test_oracle_semi.py (the frozen operator
applied to u is -or_div(u); symmetry and definiteness; the constant-image
closed form; the fixed point equals the explicit scheme's; F(u) = 0 at the
paper's eps through the pinned or_F).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import F, OrParams, faces, gauss


def matrix(Dx, Dy, s: float, boundary: int = 0):
    """I/s + L for one channel, from the face coefficients of `faces`."""
    H, W = Dy.shape[0] - 1, Dx.shape[1] - 1
    N = H * W
    idx = np.arange(N).reshape(H, W)
    diag = np.full(N, 1.0 / s)
    rows, cols, vals = [], [], []
    # interior x-faces (i+1/2, j), i = 0..W-2: couple (j, i) and (j, i+1)
    d = Dx[:, 1:W].ravel()
    a, b = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    rows += [a, b]
    cols += [b, a]
    vals += [-d, -d]
    np.add.at(diag, a, d)
    np.add.at(diag, b, d)
    # interior y-faces (i, j+1/2), j = 0..H-2
    d = Dy[1:H, :].ravel()
    a, b = idx[:-1, :].ravel(), idx[1:, :].ravel()
    rows += [a, b]
    cols += [b, a]
    vals += [-d, -d]
    np.add.at(diag, a, d)
    np.add.at(diag, b, d)
    if boundary == 1:  # the ghost neighbour is 0: the face adds to the diagonal
        np.add.at(diag, idx[:, 0], Dx[:, 0])
        np.add.at(diag, idx[:, W - 1], Dx[:, W])
        np.add.at(diag, idx[0, :], Dy[0, :])
        np.add.at(diag, idx[H - 1, :], Dy[H, :])
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def step(u, Phi, lam, p: OrParams, s: float):
    """One semi-implicit step from u (3xHxW), solved exactly."""
    u = np.asarray(u, np.float64)
    _, H, W = u.shape
    out = np.empty_like(u)
    no_edge = (p.variant & 2) != 0
    for c in range(3):
        Dx, Dy = faces(u[c], p.eps, p.boundary, no_edge)
        A = matrix(Dx, Dy, s, p.boundary)
        rhs = u[c] / s - lam * gauss(u[c], p.sigma, p.radius, p.boundary) + Phi[c]
        out[c] = spla.spsolve(A.tocsc(), rhs.ravel()).reshape(H, W)
    return out


def solve(u0, Phi, lam, p: OrParams, s: float, max_iter: int, tol: float):
    """Semi-implicit iteration from u0.  Returns (u^n, n, rho[n+1, 3])."""
    u = np.array(u0, np.float64)
    Phi = np.asarray(Phi, np.float64)
    lam = np.asarray(lam, np.float64)
    phin = np.sqrt((Phi.reshape(3, -1) ** 2).sum(axis=1))
    rho = []
    n = 0
    while True:
        f = np.sqrt((F(u, Phi, lam, p).reshape(3, -1) ** 2).sum(axis=1))
        r = np.where(phin > 0, f / np.where(phin > 0, phin, 1.0), f)
        rho.append(r)
        if (np.all(np.isfinite(r)) and r.max() <= tol) or n == max_iter:
            break
        u = step(u, Phi, lam, p, s)
        n += 1
    return u, n, np.array(rho)
