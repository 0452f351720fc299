"""Plain FP64 adjoint of the oracle's semi-implicit step and of a rollout loss.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Gradient convention: for a real loss L of complex fields, the gradient with
respect to eta is the complex field dL/dRe(eta) + i dL/dIm(eta) (twice the
Wirtinger derivative dL/d conj(eta)), so that dL = Re sum conj(grad) d(eta).
This is the convention of PyTorch's complex autograd.

The step (Alg. 1 with one nonlinear iterate, nonlinear term explicit) is, per
amplitude j,

    eta_j^{n+1} = S_j^{-1} w_j,   w_j = eta_j^n / dt - kap_j N_j(eta^n),
    S_j = (1/dt + kap_j dB) I + kap_j Bx G_h^2   (Hermitian: G_h is Hermitian).

Its adjoint, for lam = grad of L with respect to eta^{n+1}:

    g_j = S_j^{-H} lam_j = S_j^{-1} lam_j,
    grad wrt eta^n_k = g_k / dt - sum_j kap_j [ g_j conj(dN_j/d eta_k) + conj(g_j) dN_j/d conj(eta_k) ],
    dL/d dB (through S) = -sum_j kap_j Re sum_points conj(g_j) eta_j^{n+1}.

N_j is not complex-analytic (it contains conjugates), hence both Wirtinger
derivatives.  Parity status: pinned by ``tests/test_oracle_adjoint.py``
(central finite differences of the oracle's own forward map, the closed-form
triangular derivatives against the table, and a Fourier closed form of the
gradient in the linear case t = v = 0).
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np

from .apfc import Lattice, Params, _mode_value, energy, energy_gradient, run, solve_schur


def nonlinear_vjp_table(eta: np.ndarray, w: np.ndarray, p: Params, table) -> np.ndarray:
    """sum_j [ w_j conj(dN_j/d eta_k) + conj(w_j) dN_j/d conj(eta_k) ] for every k.

    N_j = d f_bulk / d conj(eta_j) - dB eta_j is the sum, over the resonant
    cubic and quartic monomials containing the mode (j, -1), of coefficient x
    multiplicity x count x the product of the other modes; each factor of that
    product is eta_c (mode (c, +1)) or conj(eta_c) (mode (c, -1)).
    """
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
                    d = np.full(eta.shape[1:], c, dtype=complex)
                    for g_, (cg, sg) in enumerate(rest):
                        if g_ != f:
                            d = d * _mode_value(eta, cg, sg)
                    if sf > 0:  # factor eta_cf: d is dN_j / d eta_cf
                        out[cf] = out[cf] + w[j] * np.conj(d)
                    else:  # factor conj(eta_cf): d is dN_j / d conj(eta_cf)
                        out[cf] = out[cf] + np.conj(w[j]) * d
    return out


def nonlinear_vjp_hex(eta: np.ndarray, w: np.ndarray, p: Params) -> np.ndarray:
    """The same product for the closed-form triangular N_j.

    N_j = 3v (A^2 - |eta_j|^2) eta_j - 2t conj(eta_k eta_l), A^2 = 2 sum |eta_m|^2:
      dN_j/d eta_j = 3v A^2,           dN_j/d conj(eta_j) = 3v eta_j^2,
      dN_j/d eta_m = 6v eta_j conj(eta_m),
      dN_j/d conj(eta_m) = 6v eta_j eta_m - 2t conj(eta_o)   (m != j, o the third index).
    """
    A2 = 2.0 * np.sum(np.abs(eta) ** 2, axis=0)
    out = np.zeros_like(eta, dtype=complex)
    for j in range(3):
        a_jj = 3.0 * p.v * A2
        b_jj = 3.0 * p.v * eta[j] ** 2
        out[j] = out[j] + w[j] * np.conj(a_jj) + np.conj(w[j]) * b_jj
        for m in range(3):
            if m == j:
                continue
            o = 3 - j - m
            a_jm = 6.0 * p.v * eta[j] * np.conj(eta[m])
            b_jm = 6.0 * p.v * eta[j] * eta[m] - 2.0 * p.t * np.conj(eta[o])
            out[m] = out[m] + w[j] * np.conj(a_jm) + np.conj(w[j]) * b_jm
    return out


def nonlinear_vjp(eta: np.ndarray, w: np.ndarray, p: Params, lat: Lattice) -> np.ndarray:
    if lat.kind == "hex":
        return nonlinear_vjp_hex(eta, w, p)
    return nonlinear_vjp_table(eta, w, p, lat.table)


def kappas(lat: Lattice) -> np.ndarray:
    return np.array([float(np.dot(lat.k[j], lat.k[j])) for j in range(lat.J)])


def step_adjoint(eta_n, eta_np1, lam_np1, dt: float, p: Params, lat: Lattice, h):
    """Adjoint of ``step``: returns (grad wrt eta^n, dL/d dB through this step)."""
    kap = kappas(lat)
    g = np.stack([solve_schur(lam_np1[j], lat.k[j], dt, p, h) for j in range(lat.J)])
    w = kap.reshape((-1,) + (1,) * (g.ndim - 1)) * g
    lam_n = g / dt - nonlinear_vjp(eta_n, w, p, lat)
    d_dB = -float(sum(kap[j] * np.sum(np.conj(g[j]) * eta_np1[j]).real for j in range(lat.J)))
    return lam_n, d_dB


def rollout_loss(eta0, dB: float, target, dt: float, nsteps: int, p: Params, lat: Lattice, h, w_energy=1.0):
    """L = 1/2 h^d sum |eta^K - target|^2 + w_energy F(eta^K), K = nsteps, with dB as given."""
    q = replace(p, dB=float(dB))
    eta = run(eta0, dt, nsteps, q, lat, h)[-1] if nsteps > 0 else np.array(eta0, dtype=complex)
    vol = float(np.prod(h))
    return 0.5 * vol * float(np.sum(np.abs(eta - target) ** 2)) + w_energy * energy(eta, q, lat, h)


def final_gradient(eta, target, dB: float, p: Params, lat: Lattice, h, w_energy=1.0):
    """(grad of L wrt eta^K, partial dL/d dB at fixed eta^K)."""
    q = replace(p, dB=float(dB))
    vol = float(np.prod(h))
    lam = vol * (eta - target) + w_energy * 2.0 * vol * energy_gradient(eta, q, lat, h)
    # F is affine in dB: its partial derivative is F(dB = 1) - F(dB = 0)
    dF = energy(eta, replace(p, dB=1.0), lat, h) - energy(eta, replace(p, dB=0.0), lat, h)
    return lam, w_energy * dF


def rollout_gradient(eta0, dB: float, target, dt: float, nsteps: int, p: Params, lat: Lattice, h, w_energy=1.0):
    """(grad of rollout_loss wrt eta0, dL/d dB) by the adjoint recursion over stored states."""
    q = replace(p, dB=float(dB))
    states = [np.array(eta0, dtype=complex)] + run(eta0, dt, nsteps, q, lat, h)
    lam, d_dB = final_gradient(states[-1], target, dB, p, lat, h, w_energy)
    for n in range(nsteps - 1, -1, -1):
        lam, d = step_adjoint(states[n], states[n + 1], lam, dt, q, lat, h)
        d_dB += d
    return lam, d_dB
