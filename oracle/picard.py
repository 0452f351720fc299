"""Plain FP64 oracle of the paper's time step with K Picard iterations and the
Jacobian of the nonlinear term in direction eta_j (Alg. 1, Sec. II.A).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

In the finite-difference setting with M = I, iteration k of time step m solves
for every amplitude j (all amplitudes read the previous iterate eta^(k-1)):

    [ I           -G_h                          ] [zeta]   [ 0                                         ]
    [ kap Bx G_h  (1/dt + kap dB) I + kap D_j   ] [eta ] = [ eta^{m-1}/dt - kap (N_j - D_j eta_j)(eta^(k-1)) ]

with D_j = dN_j / d eta_j (the Wirtinger derivative in direction eta_j only, the
paper's dF_j = d^2 f / d eta_j d conj(eta_j) without its dB part, which sits in
the linear operator) evaluated at eta^(k-1); the paper's J^j and h^j with the
sign that makes the system a linearisation of the backward Euler step.  D_j is
real (a mixed second derivative of the real bulk density).  ``jacobian=False``
drops D (plain Picard); K = 1 without the Jacobian is ``oracle.step``.  A
converged iteration solves the fully implicit backward Euler step
(eta - eta^{m-1})/dt = -kap [(dB + Bx G_h^2) eta + N(eta)].

The variable-coefficient Schur complement S_j + kap D_j is solved by a sparse
direct solve (scipy.sparse.linalg.spsolve) of the periodic stencil matrices.
Parity status: pinned by ``tests/test_oracle_picard.py``.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .apfc import Lattice, Params, _mode_value, apply_G, zeta_of


def jacobian_diag_hex(eta, p: Params) -> np.ndarray:
    """D_j = dN_j/d eta_j = 3v A^2 for the triangular closed form."""
    A2 = 2.0 * np.sum(np.abs(eta) ** 2, axis=0)
    return np.stack([3.0 * p.v * A2 for _ in range(eta.shape[0])]).astype(complex)


def jacobian_diag_table(eta, p: Params, table) -> np.ndarray:
    """D_j from the resonance table: the derivative of every monomial of N_j by
    each of its unconjugated eta_j factors."""
    coef = {3: -p.t / 3.0, 4: 0.25 * p.v}
    J = eta.shape[0]
    out = np.zeros_like(eta, dtype=complex)
    for pw in (3, 4):
        for mono, mult in table[pw].items():
            for j in range(J):
                cnt = mono.count((j, -1))
                if cnt == 0:
                    continue
                rest = list(mono)
                rest.remove((j, -1))
                c = coef[pw] * mult * cnt
                for f, (cf, sf) in enumerate(rest):
                    if cf != j or sf < 0:
                        continue
                    d = np.full(eta.shape[1:], c, dtype=complex)
                    for g_, (cg, sg) in enumerate(rest):
                        if g_ != f:
                            d = d * _mode_value(eta, cg, sg)
                    out[j] = out[j] + d
    return out


def jacobian_diag(eta, p: Params, lat: Lattice) -> np.ndarray:
    if lat.kind == "hex":
        return jacobian_diag_hex(eta, p)
    return jacobian_diag_table(eta, p, lat.table)


def _diff_matrices(shape, h):
    """Sparse periodic L_h and D_d (d = 0 is x, the last array axis)."""
    dim = len(h)
    sizes = [shape[-1 - d] for d in range(dim)]  # n_x, n_y[, n_z]

    def one_d(n, kind):
        e = np.ones(n)
        if kind == "lap":
            m = sp.diags([e[:-1], -2 * e, e[:-1]], [-1, 0, 1], shape=(n, n), format="lil")
            m[0, n - 1] = 1.0
            m[n - 1, 0] = 1.0
        else:
            m = sp.diags([-e[:-1], e[:-1]], [-1, 1], shape=(n, n), format="lil") * 0.5
            m[0, n - 1] = -0.5
            m[n - 1, 0] = 0.5
        return m.tocsr()

    def embed(mat, d):
        # flattened index = x + n_x (y + n_y z): the x factor is the rightmost Kronecker factor
        out = None
        for a in range(dim - 1, -1, -1):
            f = mat if a == d else sp.identity(sizes[a], format="csr")
            out = f if out is None else sp.kron(out, f, format="csr")
        return out

    lap = sum(embed(one_d(sizes[d], "lap"), d) / (h[d] * h[d]) for d in range(dim))
    dd = [embed(one_d(sizes[d], "d"), d) / h[d] for d in range(dim)]
    return lap, dd


def g_matrix(kj, shape, h):
    lap, dd = _diff_matrices(shape, h)
    return lap + 2j * sum(kj[d] * dd[d] for d in range(len(h)))


def step_picard(eta, dt: float, p: Params, lat: Lattice, h, K: int, jacobian: bool = True):
    """One time step with K Picard iterations; returns (eta^m, zeta^m)."""
    eta_prev = np.array(eta, dtype=complex)
    it = eta_prev.copy()
    shape = eta.shape[1:]
    n = int(np.prod(shape))
    Gs = [g_matrix(lat.k[j], shape, h) for j in range(lat.J)]
    for _ in range(K):
        N = lat.nonlinear(it, p)
        D = jacobian_diag(it, p, lat).real if jacobian else np.zeros(it.shape)
        new = np.empty_like(it)
        for j in range(lat.J):
            kap = float(np.dot(lat.k[j], lat.k[j]))
            b = eta_prev[j] / dt - kap * (N[j] - D[j] * it[j])
            diag = (1.0 / dt + kap * p.dB) + kap * D[j].ravel()
            S = sp.diags(diag) + kap * p.Bx * (Gs[j] @ Gs[j])
            new[j] = spla.spsolve(S.tocsc(), b.ravel()).reshape(shape)
        it = new
    return it, zeta_of(it, lat, h)


def backward_euler_residual(eta, eta_prev, dt: float, p: Params, lat: Lattice, h) -> np.ndarray:
    """(eta - eta_prev)/dt + kap [(dB + Bx G_h^2) eta + N(eta)] per amplitude."""
    N = lat.nonlinear(eta, p)
    out = np.empty_like(eta, dtype=complex)
    for j in range(lat.J):
        kap = float(np.dot(lat.k[j], lat.k[j]))
        gg = apply_G(apply_G(eta[j], lat.k[j], h), lat.k[j], h)
        out[j] = (eta[j] - eta_prev[j]) / dt + kap * (p.dB * eta[j] + p.Bx * gg + N[j])
    return out
