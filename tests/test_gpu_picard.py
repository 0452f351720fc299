"""The paper's time step with K Picard iterations and the Jacobian in direction
eta_j (Alg. 1) on the GPU against the oracle (``oracle/picard.py``: sparse direct
solves of the variable-coefficient Schur complement).  Solves stop at relative
residual 1e-13, so each iterate matches the oracle to ~1e-12 and a few steps of
K iterations to 1e-10 relative."""
import numpy as np
import pytest

import oracle as O
from oracle import picard as PC
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, H3, P, ensure_built, lattice, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _state(kind, shape, h, seed):
    L, _ = lattice(kind)
    if kind == "hex":
        return inputs.single_grain(L.k, O.uniform_solid_hex(P), shape, h, 0.3 * min(shape) * h[0], 6.0,
                                   seed=seed, noise=1e-2)
    phi = O.uniform_solid_bcc(P)
    return inputs.single_grain(L.k, phi, shape, h, 0.3 * min(shape) * h[0], 8.0, seed=seed, noise=1e-2, matrix=phi)


def _run(kind, shape, h, K, jac, prec, fused=1, nsteps=2, dt=1.0):
    L, code = lattice(kind)
    eta0 = _state(kind, shape, h, 3)
    o = A.apfc_default_opts(precision=prec, tol=1e-13, picard_iters=K, jacobian=jac, fused=fused)
    with A.Context(L.k, code, (P.dB, P.Bx, P.t, P.v), shape, h, o) as c:
        c.set_amplitudes(eta0)
        ref = eta0
        for _ in range(nsteps):
            c.step(dt)
            ref, _ = PC.step_picard(ref, dt, P, L, h, K, jacobian=bool(jac))
            got = c.get_amplitudes()
            assert rel_l2(got, ref) <= 1e-10, rel_l2(got, ref)
        st = c.stats()
    return got, ref, st


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
@pytest.mark.parametrize("kind,shape,h", [("hex", (40, 48), H2), ("hex", (33, 50), (1.2, 0.8)),
                                          ("bcc", (6, 8, 10), H3)])
def test_picard_with_jacobian_matches_oracle(kind, shape, h, prec):
    _run(kind, shape, h, 3, 1, prec)


@pytest.mark.parametrize("fused", [1, 0])
def test_plain_picard_matches_oracle(fused):
    _run("hex", (40, 48), H2, 2, 0, A.APFC_FP32_REFINED, fused=fused)


def test_converged_picard_solves_backward_euler():
    shape, h, dt = (36, 40), H2, 1.0
    L, code = lattice("hex")
    eta0 = _state("hex", shape, h, 5)
    o = A.apfc_default_opts(tol=1e-13, picard_iters=16, jacobian=1)
    with A.Context(L.k, code, (P.dB, P.Bx, P.t, P.v), shape, h, o) as c:
        c.set_amplitudes(eta0)
        c.step(dt)
        e = c.get_amplitudes()
    res = PC.backward_euler_residual(e, eta0, dt, P, L, h)
    assert np.max(np.abs(res)) / (np.max(np.abs(eta0)) / dt) <= 1e-10


def test_adjoint_rejects_the_picard_step():
    shape = (16, 16)
    L, code = lattice("hex")
    o = A.apfc_default_opts(picard_iters=2)
    with A.Context(L.k, code, (P.dB, P.Bx, P.t, P.v), shape, H2, o) as c:
        eta = _state("hex", shape, H2, 1)
        c.set_amplitudes(eta)
        with pytest.raises(A.ApfcError):
            c.adjoint_step(1.0, eta, eta, eta)
