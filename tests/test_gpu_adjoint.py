"""Adjoint of the step on the GPU: the library's adjoint step, energy gradient
and checkpointed rollout against the oracle's adjoint (``oracle/adjoint.py``),
and the torch.autograd bridge against central finite differences (h = 1e-6)
of the forward rollout, including the full-size 1024^2, 200-step case with a
checkpoint every 20 steps.

Tolerances: the adjoint solves stop at relative residual tol; with tol = 1e-13
(FP64) the gradients agree with the oracle's exact FFT solves to ~cond(S) x tol
per step, checked at 1e-9 relative.  Each loss evaluation of a rollout whose
solves stop at tol carries an error of about cond(S) tol |L| (cond(S) < 20), so
a central difference with h = 1e-6 carries about cond(S) tol |L| / h; relative
to the largest directional derivative over the sampled directions this is a few
1e-5 on the small grid and below 1e-4 on the full-size case (tol 1e-13), the
bounds used.
"""
import numpy as np
import pytest

import oracle as O
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, P, ensure_built, lattice, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _ctx(kind, shape, h, **opts):
    L, code = lattice(kind)
    o = A.apfc_default_opts(**opts)
    return A.Context(L.k, code, (P.dB, P.Bx, P.t, P.v), shape, h, o), L


def _rand(shape, seed, scale):
    rng = np.random.default_rng(seed)
    return scale * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


CASES = [("hex", (40, 48), H2), ("hex", (33, 70), (1.2, 0.8)), ("bcc", (8, 10, 12), (1.1, 0.9, 1.2))]


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
@pytest.mark.parametrize("kind,shape,h", CASES)
def test_adjoint_step_matches_oracle(kind, shape, h, prec):
    ctx, L = _ctx(kind, shape, h, precision=prec, tol=1e-13)
    J = L.J
    phi = O.uniform_solid_hex(P) if kind == "hex" else O.uniform_solid_bcc(P)
    eta_n = phi + _rand((J,) + shape, 1, 0.05)
    eta_np1, _ = O.step(eta_n, 0.8, P, L, h)
    lam = _rand((J,) + shape, 2, 1.0)
    got, g_dB = ctx.adjoint_step(0.8, eta_n, eta_np1, lam)
    ref, r_dB = O.step_adjoint(eta_n, eta_np1, lam, 0.8, P, L, h)
    assert rel_l2(got, ref) <= 1e-10
    assert g_dB == pytest.approx(r_dB, rel=1e-10)
    ctx.close()


@pytest.mark.parametrize("kind,shape,h", CASES)
def test_energy_gradient_matches_oracle(kind, shape, h):
    ctx, L = _ctx(kind, shape, h)
    eta = _rand((L.J,) + shape, 3, 0.3)
    got, dF = ctx.energy_gradient(eta)
    vol = float(np.prod(h))
    ref = 2.0 * vol * O.energy_gradient(eta, P, L, h)
    assert rel_l2(got, ref) <= 1e-12
    assert dF == pytest.approx(vol * float(np.sum(np.abs(eta) ** 2)), rel=1e-12)
    ctx.close()


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_rollout_gradient_matches_oracle(prec):
    # 7 steps with a checkpoint every 3: two full segments and a ragged one
    shape, n, every, dt = (36, 44), 7, 3, 1.0
    L = O.hex_lattice()
    eta0 = inputs.batch_run_state(O.uniform_solid_hex(P), None, 6.0, 5, shape=shape)
    target = _rand((3,) + shape, 6, 0.1)
    from paper_1902_09761_gb300.autograd import Rollout

    ro = Rollout(L.k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), shape, H2, dt, n, every,
                 A.apfc_default_opts(precision=prec, tol=1e-13), device="cuda")
    e0 = torch.from_numpy(eta0).cuda().requires_grad_(True)
    dB = torch.tensor(P.dB, dtype=torch.float64, requires_grad=True)
    etaN, F = ro(e0, dB)
    vol = H2[0] * H2[1]
    loss = 0.5 * vol * (etaN - torch.from_numpy(target).cuda()).abs().pow(2).sum() + F
    loss.backward()
    ref, ref_dB = O.rollout_gradient(eta0, P.dB, target, dt, n, P, L, H2)
    assert rel_l2(e0.grad.cpu().numpy(), ref) <= 1e-9
    assert float(dB.grad) == pytest.approx(ref_dB, rel=1e-9)
    # the loss itself is the oracle's
    assert float(loss.detach()) == pytest.approx(O.rollout_loss(eta0, P.dB, target, dt, n, P, L, H2), rel=1e-11)
    ro.close()


def test_rollout_backward_restores_state_and_adjoint_is_linear():
    shape = (32, 32)
    ctx, L = _ctx("hex", shape, H2, tol=1e-13)
    eta0 = inputs.batch_run_state(O.uniform_solid_hex(P), None, -4.0, 7, shape=shape)
    ctx.set_amplitudes(eta0)
    ctx.rollout_forward(1.0, 5, 2)
    final = ctx.get_amplitudes()
    a, b = _rand((3,) + shape, 8, 1.0), _rand((3,) + shape, 9, 1.0)
    ga, da = ctx.rollout_backward(a)
    gb, db = ctx.rollout_backward(b)
    gab, dab = ctx.rollout_backward(a + 2.0 * b)
    assert np.array_equal(ctx.get_amplitudes(), final)
    assert rel_l2(gab, ga + 2.0 * gb) <= 1e-10
    assert dab == pytest.approx(da + 2.0 * db, rel=1e-9)
    ctx.close()


def _fd_check(shape, n, every, prec, tol, ndir, bound, seed, h_fd=1e-6, phi_state=None, dtype=torch.complex128):
    from paper_1902_09761_gb300.autograd import Rollout

    L = O.hex_lattice()
    ro = Rollout(L.k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), shape, H2, 1.0, n, every,
                 A.apfc_default_opts(precision=prec, tol=tol), device="cuda")
    eta0 = phi_state if phi_state is not None else inputs.batch_run_state(
        O.uniform_solid_hex(P), None, 7.0, seed, shape=shape)
    target = torch.from_numpy(_rand((3,) + shape, seed + 1, 0.1)).cuda()
    vol = H2[0] * H2[1]

    def loss_of(e, dB):
        etaN, F = ro(e, dB)
        return 0.5 * vol * (etaN.to(torch.complex128) - target).abs().pow(2).sum() + F

    e0 = torch.from_numpy(eta0).cuda().to(dtype).requires_grad_(True)
    dB = torch.tensor(P.dB, dtype=torch.float64, requires_grad=True)
    loss_of(e0, dB).backward()
    g = e0.grad.to(torch.complex128)
    rng = np.random.default_rng(seed + 2)
    ans, fds = [], []
    with torch.no_grad():
        base = torch.from_numpy(eta0).cuda()
        for _ in range(ndir):
            d = torch.from_numpy(rng.standard_normal((3,) + shape) + 1j * rng.standard_normal((3,) + shape)).cuda()
            d = d / d.abs().max()
            lp = float(loss_of(base + h_fd * d, torch.tensor(P.dB, dtype=torch.float64)))
            lm = float(loss_of(base - h_fd * d, torch.tensor(P.dB, dtype=torch.float64)))
            fds.append((lp - lm) / (2 * h_fd))
            ans.append(float(torch.sum(torch.conj(g) * d).real))
        lp = float(loss_of(base, torch.tensor(P.dB + h_fd, dtype=torch.float64)))
        lm = float(loss_of(base, torch.tensor(P.dB - h_fd, dtype=torch.float64)))
        fd_dB = (lp - lm) / (2 * h_fd)
    ro.close()
    worst = max(abs(a - f) for a, f in zip(ans, fds)) / max(abs(f) for f in fds)
    err_dB = abs(float(dB.grad) - fd_dB) / abs(fd_dB)
    assert worst <= bound, worst
    assert err_dB <= bound, err_dB
    return worst, err_dB, e0.grad


def test_autograd_matches_central_differences_small():
    # Worst case, the central difference's rounding floor is 2 n cond(S) tol |L| / (h max|fd|)
    # (n = 10 steps, cond(S) < 20, tol 1e-13, h = 1e-6): about 4e-5 here.  The two loss
    # evaluations of a difference follow the same deterministic Krylov path, so their solver
    # errors largely cancel: measured 7.1e-9 (dB 1.9e-10).  The bound keeps a 14x margin
    # over the measurement.
    worst, err_dB, _ = _fd_check((48, 64), 10, 4, A.APFC_FP64, 1e-13, 8, 1e-7, seed=20)
    print(f"48x64 x 10 steps: worst directional rel err {worst:.2e}, dB rel err {err_dB:.2e}")


def test_autograd_complex64_input_gives_complex64_gradient():
    from paper_1902_09761_gb300.autograd import Rollout

    shape = (32, 40)
    L = O.hex_lattice()
    ro = Rollout(L.k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), shape, H2, 1.0, 4, 2,
                 A.apfc_default_opts(tol=1e-13), device="cuda")
    eta0 = inputs.batch_run_state(O.uniform_solid_hex(P), None, 3.0, 30, shape=shape)
    grads = []
    for dt in (torch.complex128, torch.complex64):
        e0 = torch.from_numpy(eta0).cuda().to(dt).requires_grad_(True)
        etaN, F = ro(e0, torch.tensor(P.dB, dtype=torch.float64))
        assert etaN.dtype == dt
        (etaN.abs().pow(2).sum() + F).backward()
        assert e0.grad.dtype == dt
        grads.append(e0.grad.to(torch.complex128).cpu().numpy())
    assert rel_l2(grads[1], grads[0]) <= 1e-5
    ro.close()


@pytest.mark.slow
def test_autograd_full_size_1024_200_steps_checkpoint_20():
    # 2D hexagonal 1024^2, 200 steps, checkpoint every 20; loss = L2 misfit to a seeded
    # target plus F; gradients wrt eta0 and dB against central differences (h = 1e-6)
    # on 8 random directions
    phi = O.uniform_solid_hex(P)
    eta0 = inputs.voronoi_grains(inputs.hex_vectors(), phi, (1024, 1024), H2, 8, 10.0, seed=3, noise=1e-3)
    # measured: worst directional 2.4e-6, dB 4.1e-12; the bound keeps an 8x margin
    worst, err_dB, _ = _fd_check((1024, 1024), 200, 20, A.APFC_FP32_REFINED, 1e-13, 8, 2e-5, seed=40,
                                 phi_state=eta0)
    print(f"1024^2 x 200 steps: worst directional rel err {worst:.2e}, dB rel err {err_dB:.2e}")
