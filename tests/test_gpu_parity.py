"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Tolerances: operator-level results are FP64 stencils whose only difference
from the oracle is the summation order, so they must agree to ~1e-13
relative.  Time steps solve the block system to a relative residual tol;
the error of eta is then at most cond(S_j) * tol with cond(S_j) < 20 on these
grids (S_j's symbol spans [1/dt + dB, 1/dt + dB + Bx max g^2]), so parity
runs use tol = 1e-13 and must match the oracle to relative L2 <= 1e-10 per
step and per amplitude.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, H3, P, context, ensure_built, lattice, rel_l2, rel_l2_per_amp

pytestmark = pytest.mark.gpu

CASES = [("hex", (16, 16), H2), ("hex", (98, 130), (0.9, 1.3)), ("bcc", (8, 10, 12), (1.1, 0.9, 1.2))]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _max_rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("kind,shape,h", CASES)
def test_block_operator_parity(kind, shape, h):
    ctx, L = context(kind, shape, h)
    x = inputs.random_amplitudes(2 * L.J, shape, seed=1, scale=1.0).reshape((L.J, 2) + shape)
    dt = 0.8
    y = ctx.apply_operator(dt, x)
    for j in range(L.J):
        y1, y2 = O.apply_A(x[j, 0], x[j, 1], L.k[j], dt, P, h)
        assert _max_rel(y[j, 0], y1) < 1e-13
        assert _max_rel(y[j, 1], y2) < 1e-13


@pytest.mark.parametrize("kind,shape,h", CASES)
@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 6])
@pytest.mark.parametrize("tau", ["fold", "plain"])
@pytest.mark.parametrize("fused", [0, 1])
def test_preconditioner_parity(kind, shape, h, m, tau, fused):
    # fused = 1 runs the row-streaming 2D pipeline for 1 <= m <= 4 (other cases take the per-pass kernels)
    ctx, L = context(
        kind, shape, h, cheb_degree=m, tau_mode=A.APFC_TAU_FOLD if tau == "fold" else A.APFC_TAU_PLAIN, fused=fused
    )
    b = inputs.random_amplitudes(2 * L.J, shape, seed=2, scale=1.0).reshape((L.J, 2) + shape)
    dt = 1.0
    x = ctx.apply_preconditioner(dt, b)
    for j in range(L.J):
        c1, c2 = O.apply_Pinv(b[j, 0], b[j, 1], L.k[j], dt, P, h, m, tau)
        assert _max_rel(x[j, 0], c1) < 1e-12
        assert _max_rel(x[j, 1], c2) < 1e-12


@pytest.mark.parametrize("kind,shape,h", CASES)
def test_nonlinear_rhs_and_energy_parity(kind, shape, h):
    ctx, L = context(kind, shape, h)
    eta = inputs.random_amplitudes(L.J, shape, seed=3, scale=0.3)
    rhs = ctx.nonlinear_rhs(0.7, eta)
    assert _max_rel(rhs, O.rhs(eta, 0.7, P, L)) < 1e-14
    ctx.set_amplitudes(eta)
    assert ctx.energy() == pytest.approx(O.energy(eta, P, L, h), rel=1e-12)
    assert _max_rel(ctx.get_zeta(), O.zeta_of(eta, L, h)) < 1e-13
    assert np.array_equal(ctx.get_amplitudes(), eta)


def _trajectory_parity(kind, eta0, shape, h, nsteps, dt=1.0, bound=1e-10, **opts):
    ctx, L = context(kind, shape, h, **opts)
    ctx.set_amplitudes(eta0)
    eta_o = eta0.copy()
    worst = 0.0
    for m in range(nsteps):
        ctx.step(dt, 1)
        eta_o, zeta_o = O.step(eta_o, dt, P, L, h)
        eg, zg = ctx.get_amplitudes(), ctx.get_zeta()
        e1 = max(rel_l2_per_amp(eg, eta_o))
        e2 = max(rel_l2_per_amp(zg, zeta_o))
        worst = max(worst, e1, e2)
        assert e1 <= bound, (m, e1)
        assert e2 <= bound, (m, e2)
    return worst, ctx.stats()


@pytest.mark.parametrize("fused", [1, 0])
def test_step_parity_grain_128_fp64(fused):
    # 2D hexagonal, 128x128, grain R=30 rotated 5 deg in liquid, dt=1, 20 steps.
    eta0 = inputs.hex_grain_128(O.uniform_solid_hex(P))
    worst, st = _trajectory_parity("hex", eta0, (128, 128), H2, 20, tol=1e-13, fused=fused)
    print(f"fp64 grain-128 worst rel L2 {worst:.3e}, iters last {st['iters_last']}")
    assert st["steps"] == 20 and st["resid_last"] <= 1e-13


def test_step_parity_grain_128_fp32_refined():
    eta0 = inputs.hex_grain_128(O.uniform_solid_hex(P))
    worst, st = _trajectory_parity(
        "hex", eta0, (128, 128), H2, 20, tol=1e-13, precision=A.APFC_FP32_REFINED, tol_inner=1e-4
    )
    print(f"fp32-refined grain-128 worst rel L2 {worst:.3e}, refine sweeps {st['refine_last']}")
    assert st["resid_last"] <= 1e-13


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
@pytest.mark.parametrize("kind,shape,h", CASES[1:] + [("hex", (300, 530), (1.2, 0.8))])
@pytest.mark.parametrize("m", [1, 3, 4])
def test_step_parity_ragged(kind, shape, h, prec, m):
    # 530 columns span three 256-column strips of the fused pipeline with a ragged last one;
    # 300 rows span two 256-row segments.
    L = O.hex_lattice() if kind == "hex" else O.bcc_lattice()
    eta0 = inputs.random_amplitudes(L.J, shape, seed=4, scale=0.1)
    _trajectory_parity(kind, eta0, shape, h, 3, dt=0.5, tol=1e-13, precision=prec, cheb_degree=m)


def test_fourier_mode_decay():
    # t = v = 0: one step multiplies the grid mode w by 1/(1 + dt (dB + Bx lam^2)), G_h w = lam w.
    p = O.Params(dB=P.dB, Bx=P.Bx, t=0.0, v=0.0)
    shape, h, dt = (16, 32), H2, 1.0
    ctx, L = context("hex", shape, h, p=p, tol=1e-14)
    x, y = inputs.grid_coords(shape, h)
    for mode in [(0, 0), (1, 0), (3, -2), (16, 8), (-5, 8)]:
        q = (2 * np.pi * mode[0] / (32 * h[0]), 2 * np.pi * mode[1] / (16 * h[1]))
        w = np.exp(1j * (q[0] * x + q[1] * y))
        eta = np.stack([w, 2 * w, -w])
        ctx.set_amplitudes(eta)
        ctx.step(dt, 1)
        got = ctx.get_amplitudes()
        for j in range(3):
            lam = (O.apply_G(w, L.k[j], h) / w).mean().real
            fac = 1.0 / (1.0 + dt * (p.dB + p.Bx * lam**2))
            assert rel_l2(got[j], fac * eta[j]) < 1e-12


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_uniform_solid_and_liquid_are_fixed_points(prec):
    phi = O.uniform_solid_hex(P)
    ctx, L = context("hex", (32, 32), H2, precision=prec)
    eta = np.full((3, 32, 32), phi, dtype=complex)
    ctx.set_amplitudes(eta)
    ctx.step(1.0, 3)
    assert np.max(np.abs(ctx.get_amplitudes() - phi)) < 1e-15
    ctx.set_amplitudes(np.zeros_like(eta))
    ctx.step(1.0, 2)
    assert np.all(ctx.get_amplitudes() == 0)


def test_bcc_uniform_solid_fixed_point():
    phi = O.uniform_solid_bcc(P)
    ctx, L = context("bcc", (6, 6, 6), H3)
    ctx.set_amplitudes(np.full((6, 6, 6, 6), phi, dtype=complex))
    ctx.step(1.0, 2)
    assert np.max(np.abs(ctx.get_amplitudes() - phi)) < 1e-15


@pytest.mark.parametrize("kind", ["hex", "bcc"])
@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_step_commutes_with_grid_shift_and_displacement_phase(kind, prec):
    # Periodic shifts and a uniform displacement u (eta_j -> eta_j exp(i k_j.u), which keeps
    # every resonant monomial) commute with the exact step; the CUDA path, whose tiles,
    # halos, wraps and reduction order all move with the data, must follow to the solver
    # tolerance.  Ragged sizes: the shift crosses tile, strip and z-chunk boundaries.
    if kind == "hex":
        shape, h, shift = (70, 150), (1.2, 0.8), (17, -41)
    else:
        shape, h, shift = (70, 13, 67), (1.0, 1.3, 0.9), (9, 5, -30)
    ctx, L = context(kind, shape, h, tol=1e-13, precision=prec)
    axes = tuple(range(1, len(shape) + 1))
    eta = inputs.random_amplitudes(L.J, shape, seed=41, scale=0.15)
    rng = np.random.default_rng(42)
    u = rng.uniform(-3.0, 3.0, size=len(shape))
    ph = np.exp(1j * (L.k @ u)).reshape((L.J,) + (1,) * len(shape))

    def step(e):
        ctx.set_amplitudes(e)
        ctx.step(0.7, 1)
        return ctx.get_amplitudes()

    base = step(eta)
    scale = np.max(np.abs(base))
    moved = step(np.roll(eta, shift, axis=axes))
    assert np.max(np.abs(moved - np.roll(base, shift, axis=axes))) <= 1e-11 * scale
    phased = step(eta * ph)
    assert np.max(np.abs(phased - base * ph)) <= 1e-11 * scale


def test_energy_decreases_on_gpu():
    eta0 = inputs.hex_grain_128(O.uniform_solid_hex(P))
    ctx, L = context("hex", (128, 128), H2)
    ctx.set_amplitudes(eta0)
    F = [ctx.energy()]
    for _ in range(10):
        ctx.step(1.0, 1)
        F.append(ctx.energy())
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(F, F[1:]))
    assert F[0] == pytest.approx(O.energy(eta0, P, L, H2), rel=1e-12)


def test_failure_paths_return_status_codes():
    ctx, L = context("hex", (16, 16), H2)
    assert ctx.try_step(1.0, 1) == A.APFC_ESTATE  # no amplitudes yet
    eta = inputs.random_amplitudes(3, (16, 16), seed=5, scale=0.2)
    ctx.set_amplitudes(eta)
    assert ctx.try_step(0.0, 1) == A.APFC_EINVAL
    assert ctx.try_step(-1.0, 1) == A.APFC_EINVAL
    # a max_iter that is too low gives ENOCONV (never a hang)
    o = A.apfc_default_opts(max_iter=1, tol=1e-14)
    ctx.set_opts(o)
    assert ctx.try_step(1.0, 1) == A.APFC_ENOCONV
    # NaN in the amplitudes is caught by the residual norms
    ctx.set_opts(A.apfc_default_opts())
    bad = eta.copy()
    bad[1, 3, 4] = np.nan
    ctx.set_amplitudes(bad)
    assert ctx.try_step(1.0, 1) == A.APFC_ENAN
    assert ctx.try_step(1.0, 1) == A.APFC_ESTATE  # sticky until new amplitudes
    ctx.set_amplitudes(eta)
    assert ctx.try_step(1.0, 1) == A.APFC_OK


def test_device_pointer_path():
    torch = pytest.importorskip("torch")
    shape = (24, 20)
    ctx, L = context("hex", shape, H2, tol=1e-13)
    eta = inputs.random_amplitudes(3, shape, seed=6, scale=0.2)
    ctx.set_amplitudes(torch.from_numpy(eta).cuda())
    out = torch.empty((3,) + shape, dtype=torch.complex128, device="cuda")
    ctx.step(1.0, 1)
    ctx.get_amplitudes(out)
    ref, _ = O.step(eta, 1.0, P, L, H2)
    assert rel_l2(out.cpu().numpy(), ref) < 1e-10
    x = torch.from_numpy(inputs.random_amplitudes(6, shape, seed=7).reshape(3, 2, *shape)).cuda()
    y = torch.empty_like(x)
    ctx.apply_operator(1.0, x, y)
    assert np.allclose(y.cpu().numpy(), ctx.apply_operator(1.0, x.cpu().numpy()), rtol=0, atol=1e-14)


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_full_size_voronoi_4096_one_step(prec):
    # The benchmark workload (4096^2, 16 Voronoi grains) at the benchmark tolerance 1e-10:
    # both paths stop at the same final relative residual (<= 1e-10; the refinement sizes its
    # last inner solve to reach a quarter of it), so both must meet the contract's 1e-10
    # relative L2 per amplitude (measured 3.2e-11 FP64, 9.1e-12 FP32-refined).
    phi = O.uniform_solid_hex(P)
    eta0 = inputs.hex_voronoi(phi)
    ctx, L = context("hex", (4096, 4096), H2, tol=1e-10, precision=prec)
    ctx.set_amplitudes(eta0)
    ctx.step(1.0, 1)
    got = ctx.get_amplitudes()
    ref, _ = O.step(eta0, 1.0, P, L, H2)
    errs = rel_l2_per_amp(got, ref)
    print(f"4096^2 precision {prec}: rel L2 per amplitude {errs}, stats {ctx.stats()}")
    assert max(errs) <= 1e-10
    assert ctx.stats()["resid_last"] <= 1e-10


@pytest.fixture(scope="module")
def bcc_256_reference():
    # the bcc benchmark workload (256^3 sphere) and one oracle step of it (about a minute)
    phi = O.uniform_solid_bcc(P)
    eta0 = inputs.bcc_sphere(phi, n=256)
    ref, _ = O.step(eta0, 1.0, P, O.bcc_lattice(), (np.pi / 2,) * 3)
    return eta0, ref


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_full_size_bcc_256_one_step(prec, bcc_256_reference):
    # The 3D benchmark workload at the benchmark tolerance 1e-10 in the launch configuration
    # the benchmark times: both paths stop at relative residual <= 1e-10 and must match the
    # oracle to 1e-10 relative L2 per amplitude (measured 7.1e-11 FP64, 1.2e-11 FP32-refined).
    eta0, ref = bcc_256_reference
    ctx, L = context("bcc", (256, 256, 256), (np.pi / 2,) * 3, tol=1e-10, precision=prec)
    ctx.set_amplitudes(eta0)
    ctx.step(1.0, 1)
    errs = rel_l2_per_amp(ctx.get_amplitudes(), ref)
    print(f"bcc 256^3 precision {prec}: rel L2 per amplitude {errs}, stats {ctx.stats()}")
    assert max(errs) <= 1e-10
    assert ctx.stats()["resid_last"] <= 1e-10
    ctx.close()


@pytest.mark.parametrize("tile", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("rows", [32, 128, 179])
def test_tile_variants_parity(tile, rows):
    # Every FP32 variant of the fused pipeline (strip width, look-ahead depth, rows per
    # segment) gives the same converged step: 530 columns span 3-5 strips, 300 rows 2-10 segments
    # (rows 179: a segment height that is not a power of two).
    eta0 = inputs.random_amplitudes(3, (300, 530), seed=8, scale=0.1)
    _trajectory_parity(
        "hex", eta0, (300, 530), (1.2, 0.8), 2, dt=0.5, tol=1e-13, precision=A.APFC_FP32_REFINED, cheb_degree=1,
        tile=tile, tile_rows=rows, tile_t=-1,
    )


@pytest.mark.parametrize("tile_t", [0, 1, 2, 4, 5])
def test_separate_t_kernel_tile_parity(tile_t):
    # the t-kernel of the merged iteration on its own tile variant (its partial sums
    # follow that variant's block grid)
    eta0 = inputs.random_amplitudes(3, (300, 530), seed=9, scale=0.1)
    _trajectory_parity(
        "hex", eta0, (300, 530), (1.2, 0.8), 2, dt=0.5, tol=1e-13, precision=A.APFC_FP32_REFINED, cheb_degree=1,
        tile=3, tile_t=tile_t,
    )


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_bcc_multi_tile_multi_chunk_parity(prec):
    # 3D grids stream through z in 64-plane chunks over (x, y) tiles of 32 x 8 (FP64) or
    # 64 x 8 (FP32) points: 40 x 12 x 20 spans two FP64 tiles in x and two tiles in y, ragged.
    shape, h = (20, 12, 40), (1.0, 1.3, 0.9)
    ctx, L = context("bcc", shape, h)
    x = inputs.random_amplitudes(12, shape, seed=31, scale=1.0).reshape((6, 2) + shape)
    y = ctx.apply_operator(0.9, x)
    for j in range(6):
        y1, y2 = O.apply_A(x[j, 0], x[j, 1], L.k[j], 0.9, P, h)
        assert _max_rel(y[j, 0], y1) < 1e-13 and _max_rel(y[j, 1], y2) < 1e-13
    eta0 = inputs.random_amplitudes(6, shape, seed=32, scale=0.1)
    _trajectory_parity("bcc", eta0, shape, h, 2, dt=0.5, tol=1e-13, precision=prec, cheb_degree=2)


@pytest.mark.parametrize("m", [1, 2])
@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
def test_bcc_chunks_tiles_odd_width(prec, m):
    # 67 x 13 x 70: two 64-plane z-chunks (the second ragged), two FP32 / three FP64 tiles in
    # x and two tiles in y, all ragged; the odd row length puts half of the point pairs of
    # the FP32 passes off 16-byte alignment (their pointwise operands then arrive as single
    # 8-byte copies) and leaves a lone last column.  m = 1 folds step 4 of P^-1 into the
    # first Chebyshev pass, m = 2 into a later one; the inner products come out of the
    # A passes and the vector updates.
    shape, h = (70, 13, 67), (1.0, 1.3, 0.9)
    ctx, L = context("bcc", shape, h, cheb_degree=m)
    x = inputs.random_amplitudes(12, shape, seed=34, scale=1.0).reshape((6, 2) + shape)
    y = ctx.apply_operator(0.7, x)
    for j in range(6):
        y1, y2 = O.apply_A(x[j, 0], x[j, 1], L.k[j], 0.7, P, h)
        assert _max_rel(y[j, 0], y1) < 1e-13 and _max_rel(y[j, 1], y2) < 1e-13
    eta0 = inputs.random_amplitudes(6, shape, seed=33, scale=0.1)
    _trajectory_parity("bcc", eta0, shape, h, 2, dt=0.5, tol=1e-13, precision=prec, cheb_degree=m)


@pytest.mark.parametrize("device", [False, True])
def test_complex64_amplitudes_at_the_boundary(device):
    # complex64 amplitudes in and out through the C ABI (converted on the device): a step
    # from complex64 input equals the complex128 path from the same (rounded) values, and
    # complex64 output is the complex128 state rounded to nearest.
    torch = pytest.importorskip("torch")
    shape = (40, 52)
    eta = inputs.random_amplitudes(3, shape, seed=41, scale=0.2)
    e64 = eta.astype(np.complex64)
    outs = []
    for src in (e64, e64.astype(np.complex128)):
        ctx, L = context("hex", shape, H2, tol=1e-13)
        ctx.set_amplitudes(torch.from_numpy(src).cuda() if device else src)
        assert np.array_equal(ctx.get_amplitudes(), e64.astype(np.complex128))  # widening is exact
        ctx.step(1.0, 2)
        full = ctx.get_amplitudes()
        if device:
            low = torch.empty((3,) + shape, dtype=torch.complex64, device="cuda")
            ctx.get_amplitudes(low)
            low = low.cpu().numpy()
        else:
            low = ctx.get_amplitudes(dtype=np.complex64)
        assert low.dtype == np.complex64
        assert np.array_equal(low, full.astype(np.complex64))
        outs.append(full)
    assert np.array_equal(outs[0], outs[1])
    ref = O.run(e64.astype(np.complex128), 1.0, 2, P, L, H2)[-1]
    assert max(rel_l2_per_amp(outs[0], ref)) < 1e-10
    # any other element type is rejected
    assert A.load().apfc_set_amplitudes(ctx._h, e64.ctypes.data_as(ctypes.c_void_p), A.APFC_HOST, 7) == A.APFC_EINVAL


@pytest.mark.parametrize("shape", [(5, 7), (9, 40), (33, 31), (17, 65)])
def test_refined_step_on_grids_smaller_than_or_ragged_against_tiles(shape):
    # The FP32-refined step's FP64-accurate residual stages 32 x 8 tiles with a one-point
    # halo; grids narrower or shorter than a tile, or one point past a tile boundary, take
    # most of their halo from the periodic image.
    eta0 = inputs.random_amplitudes(3, shape, seed=51, scale=0.15)
    _trajectory_parity("hex", eta0, shape, (1.1, 0.9), 2, dt=0.7, tol=1e-13, precision=A.APFC_FP32_REFINED)


@pytest.mark.parametrize("shape", [(16, 16, 128), (12, 8, 64), (70, 24, 64)])
def test_bcc_refined_on_tma_staged_passes(shape):
    # FP32 3D passes move their planes by TMA on grids with nx % 64 == 0 and ny % 8 == 0;
    # the periodic x and y halos of boundary tiles come from side boxes (a one-tile-wide
    # grid wraps on both sides), z wraps by coordinate; 70 planes span two z-chunks.
    eta0 = inputs.random_amplitudes(6, shape, seed=61, scale=0.1)
    _trajectory_parity("bcc", eta0, shape, (1.0, 1.3, 0.9), 2, dt=0.5, tol=1e-13, precision=A.APFC_FP32_REFINED,
                       cheb_degree=2)


@pytest.mark.parametrize("prec", [A.APFC_FP64, A.APFC_FP32_REFINED])
@pytest.mark.parametrize("kind,shape,h", [("hex", (64, 80), H2), ("bcc", (12, 16, 64), (1.0, 1.3, 0.9))])
def test_extrapolated_initial_guess_same_trajectory(prec, kind, shape, h):
    # APFC_GUESS_EXTRAP starts each solve from 2 x^n - x^(n-1): the converged steps are the
    # oracle's (the solution of the block system is unique); 4 steps cover the first step
    # (no history), the extrapolated ones and, in the refined path, the stencil residual
    # that replaces the pointwise initial residual.
    L, _ = lattice(kind)
    phi = O.uniform_solid_hex(P) if kind == "hex" else O.uniform_solid_bcc(P)
    eta0 = inputs.single_grain(L.k, phi, shape, h, 0.3 * min(shape) * min(h), 6.0, seed=71, noise=1e-3)
    _trajectory_parity(kind, eta0, shape, h, 4, dt=1.0, tol=1e-13, precision=prec, guess=A.APFC_GUESS_EXTRAP)


def test_autotune_keeps_state_and_continues_the_trajectory():
    # apfc_autotune times one step per candidate segment height from the same state and
    # restores it: amplitudes, zeta and statistics unchanged, the chosen height one of the
    # candidates (ceil(ny / s) within 96..256 rows, 32, 48, 64, or the automatic one), and the next
    # steps still the oracle's
    shape, h, dt = (300, 530), (1.2, 0.8), 0.5
    eta0 = inputs.random_amplitudes(3, shape, seed=21, scale=0.1)
    ctx, L = context("hex", shape, h, precision=A.APFC_FP32_REFINED, tol=1e-13)
    ctx.set_amplitudes(eta0)
    ctx.step(dt, 1)
    eta1, zeta1, st1 = ctx.get_amplitudes(), ctx.get_zeta(), ctx.stats()
    tuned = ctx.autotune(dt)
    assert np.array_equal(ctx.get_amplitudes(), eta1) and np.array_equal(ctx.get_zeta(), zeta1)
    assert ctx.stats() == st1
    ny = shape[1]
    allowed = {-(-ny // s) for s in range(max(1, -(-ny // 256)), max(1, ny // 96) + 1)}
    assert tuned["tile_rows"] in allowed | {128, 64, 48, 32} and tuned["ms_per_step"] > 0
    assert 0 <= tuned["tile_t"] < 6
    eta_o = eta1.copy()
    for _ in range(2):
        ctx.step(dt, 1)
        eta_o, zeta_o = O.step(eta_o, dt, P, L, h)
        assert max(rel_l2_per_amp(ctx.get_amplitudes(), eta_o)) <= 1e-10
        assert max(rel_l2_per_amp(ctx.get_zeta(), zeta_o)) <= 1e-10
    ctx.close()


def test_autotune_is_a_no_op_off_the_fused_refined_path():
    eta0 = inputs.random_amplitudes(3, (64, 64), seed=22, scale=0.1)
    ctx, _ = context("hex", (64, 64), H2, precision=A.APFC_FP64, tol=1e-12)
    ctx.set_amplitudes(eta0)
    before = ctx.get_amplitudes()
    tuned = ctx.autotune(1.0)
    assert tuned["ms_per_step"] == 0.0 and np.array_equal(ctx.get_amplitudes(), before)
    assert ctx.stats()["steps"] == 0
    ctx.close()
