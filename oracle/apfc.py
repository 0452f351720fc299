"""Plain FP64 oracle of the APFC semi-implicit amplitude step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the CUDA product path
shares no code, table or constant generator with this module.

Paper: Praetorius, Salvalaglio, Voigt, "An efficient numerical framework for
the amplitude expansion of the phase-field crystal model" (arXiv:1902.09761).

Model (Sec. II, Eqs. energyamplitude, amplitudetime, gs).  Expanding the
paper's gradient flow with kappa_j = a0|k_j|^2 and the paper's bulk
polynomial gives, per amplitude j,

    d eta_j/dt = -|k_j|^2 [ (dB + Bx G_j^2) eta_j + N_j(eta) ],
    N_j (triangular lattice) = 3v (A^2 - |eta_j|^2) eta_j - 2t prod_{k!=j} conj(eta_k),
    A^2 = 2 sum_k |eta_k|^2,

with Bx = a0, dB = 2 a1, v = 4 a2 / 3, t = a3 (``params_from_paper``).

Discretisation: a uniform periodic grid (node i sits at r = i h) with
second-order central differences replaces the paper's P1 finite elements:

    G_h = L_h + 2i sum_d k_d D_d,   L_h the (2d+1)-point Laplacian,
    D_d u = (u(r + h_d e_d) - u(r - h_d e_d)) / (2 h_d).

Time step (Alg. 1 with one nonlinear iterate and the nonlinear term explicit;
split block form of Eq. linear_system2 with M = I):

    [ I          -G_h          ] [zeta]   [ 0                                ]
    [ kap Bx G_h  (1/dt + kap dB) ] [eta ] = [ eta^n/dt - kap N(eta^n)         ]

whose Schur complement S = (1/dt + kap dB) I + kap Bx G_h^2 is Hermitian
positive definite, so the step has a unique result that any converged Krylov
solve must reproduce.  The oracle computes it exactly by diagonalising S with
the FFT (``step``).

Array conventions: amplitudes are complex128 arrays of shape (J, ny, nx) in 2D
or (J, nz, ny, nx) in 3D; x is the fastest axis.  Spacings ``h`` and lattice
vectors are given in (x, y[, z]) order.

Parity status: every function below is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_pins.py`` (closed forms, the paper's printed spectrum
numbers, dense direct solves, brute-force cell averages, invariances).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------
# Parameters and lattices (Sec. II)
# ----------------------------------------------------------------------------


@dataclass(frozen=True)
class Params:
    """Standard APFC energy parameters (dB, Bx, t, v)."""

    dB: float
    Bx: float
    t: float
    v: float


def params_from_paper(a0: float, a1: float, a2: float, a3: float) -> Params:
    """Map the paper's (a0, a1, a2, a3) of Sec. II to (dB, Bx, t, v).

    Multiplying the paper's flow by kappa_j = a0|k_j|^2 gives the prefactors
    a0 G^2, 2 a1, 4 a2 (A_paper - |eta_j|^2) and -2 a3, which are Bx G^2, dB,
    3v (A^2 - |eta_j|^2) and -2t in the standard notation.
    """
    return Params(dB=2.0 * a1, Bx=a0, t=a3, v=4.0 * a2 / 3.0)


def hex_k() -> np.ndarray:
    """Reciprocal vectors of the triangular lattice (Sec. II, J = 3)."""
    s3 = np.sqrt(3.0)
    return np.array([[-s3 / 2, -0.5], [0.0, 1.0], [s3 / 2, -0.5]])


def bcc_k() -> np.ndarray:
    """bcc reciprocal vectors: the six <110>/sqrt(2) directions (J = 6, |k| = 1)."""
    r = 1.0 / np.sqrt(2.0)
    return r * np.array(
        [[1, 1, 0], [1, -1, 0], [1, 0, 1], [1, 0, -1], [0, 1, 1], [0, 1, -1]], dtype=float
    )


def kappa(k: np.ndarray) -> np.ndarray:
    """Mobility factor |k_j|^2 of each amplitude (Eq. amplitudetime, divided by a0)."""
    return np.sum(np.asarray(k, dtype=float) ** 2, axis=1)


def uniform_solid_hex(p: Params) -> float:
    """Real amplitude phi of the relaxed triangular solid.

    Setting eta_j = phi in (dB + Bx G^2) eta_j + N_j = 0 (G annihilates
    constants) gives dB + 15 v phi^2 - 2 t phi = 0; the larger root is the solid.
    """
    return (p.t + np.sqrt(p.t * p.t - 15.0 * p.v * p.dB)) / (15.0 * p.v)


def uniform_solid_bcc(p: Params) -> float:
    """Real amplitude phi of the relaxed bcc solid (J = 6, <110>/sqrt2 vectors).

    With the resonance rule of ``resonance_table`` the uniform bulk density is
    6 dB phi^2 - 16 t phi^3 + 135 v phi^4; its stationary point solves
    dB - 4 t phi + 45 v phi^2 = 0; the larger root is the solid.
    """
    return (2.0 * p.t + np.sqrt(4.0 * p.t * p.t - 45.0 * p.v * p.dB)) / (45.0 * p.v)


# ----------------------------------------------------------------------------
# Finite-difference operators on the periodic grid
# ----------------------------------------------------------------------------


def _neighbour(u: np.ndarray, d: int, s: int) -> np.ndarray:
    """u evaluated at r + s h_d e_d (periodic); spatial dim d = 0 is the last axis."""
    return np.roll(u, -s, axis=u.ndim - 1 - d)


def laplacian(u: np.ndarray, h) -> np.ndarray:
    """(2d+1)-point Laplacian L_h over the last len(h) axes."""
    out = np.zeros_like(u)
    for d in range(len(h)):
        out = out + (_neighbour(u, d, 1) - 2.0 * u + _neighbour(u, d, -1)) / (h[d] * h[d])
    return out


def central_diff(u: np.ndarray, h, d: int) -> np.ndarray:
    """Central first difference D_d along spatial dim d."""
    return (_neighbour(u, d, 1) - _neighbour(u, d, -1)) / (2.0 * h[d])


def apply_G(u: np.ndarray, kj, h) -> np.ndarray:
    """G_h u = L_h u + 2i k_j . D_h u, the discrete form of Delta + 2i k_j . grad (Sec. II)."""
    out = laplacian(u, h)
    for d in range(len(h)):
        out = out + 2j * kj[d] * central_diff(u, h, d)
    return out


def _q_axes(shape, h):
    """Angular grid frequencies q_d, reshaped to broadcast over the spatial shape."""
    dim = len(h)
    qs = []
    for d in range(dim):
        n = shape[-1 - d]
        q = 2.0 * np.pi * np.fft.fftfreq(n, d=h[d])
        view = [1] * dim
        view[dim - 1 - d] = n
        qs.append(q.reshape(view))
    return qs


def symbol_K(shape, h) -> np.ndarray:
    """Fourier symbol of the stiffness K = -L_h: sum_d (4/h_d^2) sin^2(q_d h_d / 2)."""
    out = np.zeros(shape)
    for d, q in enumerate(_q_axes(shape, h)):
        out = out + 4.0 / (h[d] * h[d]) * np.sin(q * h[d] / 2.0) ** 2
    return out


def symbol_G(kj, shape, h) -> np.ndarray:
    """Fourier symbol of G_h (real: G_h is Hermitian).

    g(q) = -sum_d (4/h_d^2) sin^2(q_d h_d/2) - (2/h_d) k_d sin(q_d h_d).
    """
    out = -symbol_K(shape, h)
    for d, q in enumerate(_q_axes(shape, h)):
        out = out - 2.0 * kj[d] * np.sin(q * h[d]) / h[d]
    return out


def _fft(u, dim):
    return np.fft.fftn(u, axes=tuple(range(u.ndim - dim, u.ndim)))


def _ifft(u, dim):
    return np.fft.ifftn(u, axes=tuple(range(u.ndim - dim, u.ndim)))


# ----------------------------------------------------------------------------
# Bulk polynomial: resonance tables (Sec. II, density Eq. and f^s)
# ----------------------------------------------------------------------------


def resonance_table(k, tol: float = 1e-9):
    """Resonant monomials of the cell-averaged density powers <n^p>, p = 2, 3, 4.

    n = sum_j (eta_j e^{i k_j.r} + c.c.) (Eq. density with n0 = 0) is a sum of
    2J signed modes m = (j, s): amplitude eta_j for s = +1 and conj(eta_j) for
    s = -1, wavevector s k_j.  The cell average of n^p keeps the ordered
    p-tuples of modes whose wavevectors sum to zero.  Returns
    {p: {monomial: multiplicity}} with a monomial a sorted tuple of modes.
    """
    k = np.asarray(k, dtype=float)
    modes = [(j, s) for j in range(len(k)) for s in (1, -1)]
    table = {}
    for p in (2, 3, 4):
        terms: dict = {}
        for tup in itertools.product(modes, repeat=p):
            vec = np.zeros(k.shape[1])
            for j, s in tup:
                vec = vec + s * k[j]
            if np.all(np.abs(vec) < tol):
                key = tuple(sorted(tup))
                terms[key] = terms.get(key, 0) + 1
        table[p] = terms
    return table


def _mode_value(eta, j, s):
    return eta[j] if s == 1 else np.conj(eta[j])


def density_power_average(eta: np.ndarray, table, p: int) -> np.ndarray:
    """<n^p> at every grid point from the resonance table (real up to rounding)."""
    out = np.zeros(eta.shape[1:], dtype=complex)
    for mono, mult in table[p].items():
        term = np.full(eta.shape[1:], float(mult), dtype=complex)
        for j, s in mono:
            term = term * _mode_value(eta, j, s)
        out = out + term
    return out


def bulk_density_table(eta: np.ndarray, p: Params, table) -> np.ndarray:
    """Bulk density dB/2 <n^2> - t/3 <n^3> + v/4 <n^4> (real part)."""
    f = (
        0.5 * p.dB * density_power_average(eta, table, 2)
        - p.t / 3.0 * density_power_average(eta, table, 3)
        + 0.25 * p.v * density_power_average(eta, table, 4)
    )
    return f.real


def bulk_derivative_table(eta: np.ndarray, p: Params, table) -> np.ndarray:
    """Wirtinger derivative d f_bulk / d conj(eta_j) for every j, from the table."""
    coef = {2: 0.5 * p.dB, 3: -p.t / 3.0, 4: 0.25 * p.v}
    J = eta.shape[0]
    out = np.zeros_like(eta, dtype=complex)
    for pw, terms in table.items():
        for mono, mult in terms.items():
            for j in range(J):
                cnt = mono.count((j, -1))
                if cnt == 0:
                    continue
                rest = list(mono)
                rest.remove((j, -1))
                term = np.full(eta.shape[1:], coef[pw] * mult * cnt, dtype=complex)
                for jj, s in rest:
                    term = term * _mode_value(eta, jj, s)
                out[j] = out[j] + term
    return out


def nonlinear_table(eta: np.ndarray, p: Params, table) -> np.ndarray:
    """N_j = d f_bulk / d conj(eta_j) - dB eta_j for any lattice (cubic + quartic part)."""
    return bulk_derivative_table(eta, p, table) - p.dB * eta


def nonlinear_hex(eta: np.ndarray, p: Params) -> np.ndarray:
    """Closed-form N_j of the triangular lattice (Sec. II, f^s and g^s with J = 3).

    N_j = 3v (A^2 - |eta_j|^2) eta_j - 2t conj(eta_k) conj(eta_l), {j,k,l} = {1,2,3}.
    """
    A2 = 2.0 * np.sum(np.abs(eta) ** 2, axis=0)
    out = np.empty_like(eta, dtype=complex)
    for j in range(3):
        k, l = [i for i in range(3) if i != j]
        out[j] = 3.0 * p.v * (A2 - np.abs(eta[j]) ** 2) * eta[j] - 2.0 * p.t * np.conj(eta[k] * eta[l])
    return out


def bulk_density_hex(eta: np.ndarray, p: Params) -> np.ndarray:
    """Closed-form triangular bulk density (Sec. II f^s, standard parameters).

    dB/2 A^2 + 3v/4 A^4 - 3v/2 sum|eta_j|^4 - 2t (eta1 eta2 eta3 + c.c.).
    """
    A2 = 2.0 * np.sum(np.abs(eta) ** 2, axis=0)
    cubic = eta[0] * eta[1] * eta[2]
    return (
        0.5 * p.dB * A2
        + 0.75 * p.v * A2 * A2
        - 1.5 * p.v * np.sum(np.abs(eta) ** 4, axis=0)
        - 2.0 * p.t * 2.0 * cubic.real
    )


class Lattice:
    """Reciprocal vectors plus the nonlinear term that goes with them."""

    def __init__(self, k, kind: str):
        self.k = np.asarray(k, dtype=float)
        self.kind = kind
        self.J, self.dim = self.k.shape
        self.table = resonance_table(self.k)

    def nonlinear(self, eta, p: Params):
        if self.kind == "hex":
            return nonlinear_hex(eta, p)
        return nonlinear_table(eta, p, self.table)

    def bulk_density(self, eta, p: Params):
        if self.kind == "hex":
            return bulk_density_hex(eta, p)
        return bulk_density_table(eta, p, self.table)


def hex_lattice() -> Lattice:
    return Lattice(hex_k(), "hex")


def bcc_lattice() -> Lattice:
    return Lattice(bcc_k(), "bcc")


# ----------------------------------------------------------------------------
# The semi-implicit step (Alg. 1 with K = 1, explicit nonlinear term)
# ----------------------------------------------------------------------------


def rhs(eta: np.ndarray, dt: float, p: Params, lat: Lattice) -> np.ndarray:
    """Second block of the right-hand side: eta^n/dt - |k_j|^2 N_j(eta^n)."""
    kap = kappa(lat.k).reshape((-1,) + (1,) * lat.dim)
    return eta / dt - kap * lat.nonlinear(eta, p)


def schur_symbol(kj, dt: float, p: Params, shape, h) -> np.ndarray:
    """Symbol of S_j = (1/dt + kap dB) I + kap Bx G_h^2 (Schur complement, Eq. linear_system2)."""
    kap = float(np.dot(kj, kj))
    g = symbol_G(kj, shape, h)
    return 1.0 / dt + kap * p.dB + kap * p.Bx * g * g


def solve_schur(b: np.ndarray, kj, dt: float, p: Params, h) -> np.ndarray:
    """Exact S_j^{-1} b for one amplitude by FFT diagonalisation."""
    dim = len(h)
    s = schur_symbol(kj, dt, p, b.shape, h)
    return _ifft(_fft(b, dim) / s, dim)


def zeta_of(eta: np.ndarray, lat: Lattice, h) -> np.ndarray:
    """Auxiliary field zeta_j = G_h eta_j (Sec. II.A)."""
    return np.stack([apply_G(eta[j], lat.k[j], h) for j in range(lat.J)])


def step(eta: np.ndarray, dt: float, p: Params, lat: Lattice, h):
    """One semi-implicit step; returns (eta^{n+1}, zeta^{n+1}).

    All amplitudes use the same eta^n in the nonlinear term (the j-loop of
    Alg. 1 reads the previous iterate), then each block system is solved
    exactly through its Schur complement and zeta = G_h eta.
    """
    b = rhs(eta, dt, p, lat)
    new = np.stack([solve_schur(b[j], lat.k[j], dt, p, h) for j in range(lat.J)])
    return new, zeta_of(new, lat, h)


def run(eta0: np.ndarray, dt: float, nsteps: int, p: Params, lat: Lattice, h):
    """nsteps oracle steps; returns the list of eta after each step."""
    out = []
    eta = np.array(eta0, dtype=complex)
    for _ in range(nsteps):
        eta, _ = step(eta, dt, p, lat, h)
        out.append(eta)
    return out


# ----------------------------------------------------------------------------
# Block operator and the Schur-complement preconditioner (Sec. II.B)
# ----------------------------------------------------------------------------


def apply_A(zeta, eta, kj, dt: float, p: Params, h):
    """(y1, y2) = A_j (zeta, eta) with A_j = [[I, -G_h], [kap Bx G_h, (1/dt + kap dB) I]]."""
    kap = float(np.dot(kj, kj))
    y1 = zeta - apply_G(eta, kj, h)
    y2 = kap * p.Bx * apply_G(zeta, kj, h) + (1.0 / dt + kap * p.dB) * eta
    return y1, y2


def precond_coeffs(kj, dt: float, p: Params, tau_mode: str = "fold"):
    """Coefficients (kt, sD, mu) of the preconditioner for one amplitude.

    The (2,1) block of A_j is kap Bx G_h, so the paper's kappa becomes
    kt = kap Bx.  ``tau_mode='fold'`` folds the constant shift kap dB of the
    (2,2) block into the time step: 1/tau = 1/dt + kap dB; ``'plain'`` uses
    tau = dt.  The diffusion operator is D = sD I + mu K with sD = 1/sqrt(tau),
    mu = sqrt(kt), K = -L_h.
    """
    kap = float(np.dot(kj, kj))
    kt = kap * p.Bx
    inv_tau = 1.0 / dt + (kap * p.dB if tau_mode == "fold" else 0.0)
    return kt, np.sqrt(inv_tau), np.sqrt(kt)


def apply_D(u, sD: float, mu: float, h):
    """D u = sD u + mu (-L_h u)."""
    return sD * u - mu * laplacian(u, h)


def apply_P(x1, x2, kj, dt: float, p: Params, h, tau_mode: str = "fold"):
    """P x with P the factorised preconditioner of Eq. preconditioner, M = I.

    P = [[I, 0], [kt G_h, D]] [[I, -K], [0, D]].
    """
    kt, sD, mu = precond_coeffs(kj, dt, p, tau_mode)
    u1 = x1 + laplacian(x2, h)  # x1 - K x2
    u2 = apply_D(x2, sD, mu, h)
    return u1, kt * apply_G(u1, kj, h) + apply_D(u2, sD, mu, h)


def solve_D_exact(f, sD: float, mu: float, h):
    """Exact D^{-1} f by FFT."""
    dim = len(h)
    lam = sD + mu * symbol_K(f.shape, h)
    return _ifft(_fft(f, dim) / lam, dim)


def chebyshev_bounds(sD: float, mu: float, h):
    """Spectral interval of D: [sD, sD + mu sum_d 4/h_d^2]."""
    return sD, sD + mu * sum(4.0 / (hd * hd) for hd in h)


def solve_D_chebyshev(f, sD: float, mu: float, h, m: int):
    """Approximate D^{-1} f by Chebyshev acceleration with m applications of D.

    Chebyshev iteration for a Hermitian positive definite operator with
    spectrum in [lmin, lmax] (Saad, Iterative Methods for Sparse Linear
    Systems, Sec. 12.3), started from zero:
        theta = (lmax+lmin)/2, delta = (lmax-lmin)/2, sigma = theta/delta,
        x = 0, r = f, d = r/theta, rho = 1/sigma,
        repeat m times: x += d; r -= D d; rho' = 1/(2 sigma - rho);
                        d = rho' rho d + (2 rho'/delta) r; rho = rho',
        then x += d.
    The result's residual polynomial is T_{m+1}((theta-l)/delta)/T_{m+1}(sigma).
    """
    lmin, lmax = chebyshev_bounds(sD, mu, h)
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(f)
    r = f.copy()
    d = r / theta
    for _ in range(m):
        x = x + d
        r = r - apply_D(d, sD, mu, h)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return x + d


def apply_Pinv(b1, b2, kj, dt: float, p: Params, h, m: int | None = None, tau_mode: str = "fold"):
    """chi = P^{-1} b in the four steps of Sec. II.B with M = I.

    1. beta1' = beta1 (the mass solve is the identity);
    2. D beta2' = beta2 - kt G_h beta1';
    3. D chi2 = beta2';
    4. chi1 = beta1' + (beta2' - sD chi2) / mu.
    Step 4 takes the sign that makes this the exact inverse of the displayed
    factorisation (whose (1,2) block is -K); the printed step has the opposite
    sign.  D^{-1} is exact (FFT) for m=None, else Chebyshev with m applications.
    """
    kt, sD, mu = precond_coeffs(kj, dt, p, tau_mode)
    if m is None:
        dsolve = lambda f: solve_D_exact(f, sD, mu, h)  # noqa: E731
    else:
        dsolve = lambda f: solve_D_chebyshev(f, sD, mu, h, m)  # noqa: E731
    b1p = b1
    b2p = dsolve(b2 - kt * apply_G(b1p, kj, h))
    chi2 = dsolve(b2p)
    chi1 = b1p + (b2p - sD * chi2) / mu
    return chi1, chi2


def symbol_AP_inv_eigs(g, kK, a: float, kt: float, inv_tau: float):
    """Eigenvalues of the 2x2 symbol A(q) P(q)^{-1} per frequency.

    A(q) = [[1, -g], [kt g, a]], P(q) = [[1, 0], [kt g, dq]] [[1, -kK], [0, dq]],
    dq = sqrt(inv_tau) + sqrt(kt) kK.  g, kK: symbols of G and K (arrays).
    """
    g = np.asarray(g, dtype=float)
    kK = np.asarray(kK, dtype=float)
    dq = np.sqrt(inv_tau) + np.sqrt(kt) * kK
    A = np.zeros(g.shape + (2, 2))
    A[..., 0, 0] = 1.0
    A[..., 0, 1] = -g
    A[..., 1, 0] = kt * g
    A[..., 1, 1] = a
    L = np.zeros_like(A)
    L[..., 0, 0] = 1.0
    L[..., 1, 0] = kt * g
    L[..., 1, 1] = dq
    U = np.zeros_like(A)
    U[..., 0, 0] = 1.0
    U[..., 0, 1] = -kK
    U[..., 1, 1] = dq
    P = L @ U
    return np.linalg.eigvals(A @ np.linalg.inv(P))


# ----------------------------------------------------------------------------
# Energy functional (Eq. energyamplitude)
# ----------------------------------------------------------------------------


def energy(eta: np.ndarray, p: Params, lat: Lattice, h) -> float:
    """Discrete free energy F_h = h^d sum_points [f_bulk + Bx sum_j |G_h eta_j|^2].

    The gradient term carries Bx (not Bx/2) so that dF/d conj(eta_j) equals the
    variational derivative driving the flow, (dB + Bx G_h^2) eta_j + N_j, with
    G_h Hermitian.
    """
    vol = float(np.prod(h))
    grad = sum(np.abs(apply_G(eta[j], lat.k[j], h)) ** 2 for j in range(lat.J))
    return vol * float(np.sum(lat.bulk_density(eta, p) + p.Bx * grad))


def energy_gradient(eta: np.ndarray, p: Params, lat: Lattice, h) -> np.ndarray:
    """dF_h/d conj(eta_j) per point divided by h^d: (dB + Bx G_h^2) eta_j + N_j."""
    N = lat.nonlinear(eta, p)
    out = np.empty_like(eta, dtype=complex)
    for j in range(lat.J):
        g1 = apply_G(eta[j], lat.k[j], h)
        out[j] = p.dB * eta[j] + p.Bx * apply_G(g1, lat.k[j], h) + N[j]
    return out


# ----------------------------------------------------------------------------
# Dense assembly for tiny grids
# ----------------------------------------------------------------------------


def dense_operator(apply, shape) -> np.ndarray:
    """Dense matrix of a linear map on complex grid functions of ``shape``."""
    n = int(np.prod(shape))
    M = np.zeros((n, n), dtype=complex)
    for i in range(n):
        e = np.zeros(n, dtype=complex)
        e[i] = 1.0
        M[:, i] = apply(e.reshape(shape)).ravel()
    return M


def dense_block_matrix(kj, dt: float, p: Params, shape, h) -> np.ndarray:
    """Assembled 2n x 2n block matrix A_j of Eq. linear_system2 (M = I)."""
    n = int(np.prod(shape))
    G = dense_operator(lambda u: apply_G(u, kj, h), shape)
    kap = float(np.dot(kj, kj))
    I = np.eye(n)
    return np.block([[I, -G], [kap * p.Bx * G, (1.0 / dt + kap * p.dB) * I]])
