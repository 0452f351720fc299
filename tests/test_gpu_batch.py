"""Batched independent runs on the GPU: every run of a batch against the same
run done alone on its own context (same options), and one run against the
FP64 oracle.

A batched run executes the same kernels on the same data with the same
reduction trees as the run alone (the run table only changes which block of
a launch handles which tile), so the amplitudes must agree bit for bit; a
run that converges before the others is left unchanged (it adds P^{-1} 0).
"""
import numpy as np
import pytest

import oracle as O
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, P, ensure_built, rel_l2

pytestmark = pytest.mark.gpu

# uneven sizes: several fused strips and row segments, ragged last ones, a run
# narrower than one strip, and non-square grids
SHAPES = [(128, 128), (64, 64), (96, 160), (200, 136), (256, 256), (300, 530), (40, 48)]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _states(shapes, seed=3):
    phi = O.uniform_solid_hex(P)
    rng = np.random.default_rng(seed)
    out = []
    for r, shp in enumerate(shapes):
        th = float(rng.uniform(-10, 10))
        out.append(inputs.batch_run_state(phi, None, th, 1000 + r, shape=shp))
    return out


def _opts(**kw):
    # explicit segment height: a batch uses one height for all runs (tile_rows 0 is 128
    # rows there), a run alone would pick its own
    base = dict(precision=A.APFC_FP32_REFINED, tol=1e-12, tile_rows=128)
    base.update(kw)
    return A.apfc_default_opts(**base)


def _alone(eta0, shape, steps, dt, opts):
    L = O.hex_lattice()
    with A.Context(L.k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), shape, H2, opts) as c:
        c.set_amplitudes(eta0)
        out = []
        for _ in range(steps):
            c.step(dt)
            out.append((c.get_amplitudes(), c.stats()))
        return out


def _batch(states, shapes, opts, graph=True):
    L = O.hex_lattice()
    b = A.Batch(L.k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), shapes, H2, opts, graph=graph)
    for r, e in enumerate(states):
        b.set_amplitudes(r, e)
    return b


@pytest.mark.parametrize("graph", [True, False])
def test_each_batched_run_equals_the_run_alone(graph):
    states = _states(SHAPES)
    opts = _opts()
    steps, dt = 3, 1.0
    with _batch(states, SHAPES, opts, graph) as b:
        got = []
        for _ in range(steps):
            b.step(dt)
            got.append([(b.get_amplitudes(r), b.stats(r)) for r in range(len(SHAPES))])
        replays = b.graph_replays()
    for r, shp in enumerate(SHAPES):
        ref = _alone(states[r], shp, steps, dt, opts)
        for s in range(steps):
            eta_b, st_b = got[s][r]
            eta_a, st_a = ref[s]
            diff = float(np.max(np.abs(eta_b - eta_a)))
            assert diff == 0.0, f"run {r} {shp} step {s}: max |diff| {diff:.3e}"
            assert st_b["iters_last"] == st_a["iters_last"], (r, s, st_b, st_a)
            assert st_b["refine_last"] == st_a["refine_last"], (r, s, st_b, st_a)
            assert st_b["resid_last"] == pytest.approx(st_a["resid_last"], rel=1e-12, abs=1e-300)
    if graph:
        assert replays > 0
    else:
        assert replays == 0


@pytest.mark.parametrize("m,tile,rows,tile_t", [(1, 0, 64, -1), (1, 2, 256, 4), (1, 5, 128, 0), (3, 0, 128, -1)])
def test_batched_runs_equal_alone_across_tiles_and_degrees(m, tile, rows, tile_t):
    shapes = SHAPES[:4] + [(300, 530)]
    states = _states(shapes, seed=9)
    opts = _opts(cheb_degree=m, tile=tile, tile_rows=rows, check_every=3, tile_t=tile_t)
    with _batch(states, shapes, opts) as b:
        b.step(1.0, 2)
        got = [b.get_amplitudes(r) for r in range(len(shapes))]
    for r, shp in enumerate(shapes):
        ref = _alone(states[r], shp, 2, 1.0, opts)[-1][0]
        assert float(np.max(np.abs(got[r] - ref))) == 0.0, (r, shp)


def test_batched_run_matches_fp64_oracle():
    shapes = [(48, 40), (32, 64), (40, 40)]
    states = _states(shapes, seed=11)
    opts = _opts(tol=1e-13)
    steps, dt = 3, 1.0
    with _batch(states, shapes, opts) as b:
        b.step(dt, steps)
        got = [b.get_amplitudes(r) for r in range(len(shapes))]
        for r in range(len(shapes)):
            assert b.stats(r)["resid_last"] <= 1e-13
    L = O.hex_lattice()
    for r, shp in enumerate(shapes):
        ref = O.run(states[r], dt, steps, P, L, H2)[-1]
        err = max(rel_l2(got[r][j], ref[j]) for j in range(3))
        assert err <= 1e-10, (r, err)


def test_autotune_keeps_state_and_parity():
    shapes = [(128, 128), (256, 256), (64, 64)]
    states = _states(shapes, seed=13)
    opts = _opts()
    with _batch(states, shapes, opts) as b:
        before = [b.get_amplitudes(r) for r in range(len(shapes))]
        best = b.autotune(1.0)
        assert 0 <= best["tile"] < 6 and best["tile_rows"] in (32, 48, 64, 96, 128, 192, 256)
        assert best["ms_per_iter"] > 0
        o = b.opts
        assert o.tile == best["tile"] and o.tile_rows == best["tile_rows"] and 0 <= o.tile_t < 6
        for r in range(len(shapes)):
            assert np.array_equal(b.get_amplitudes(r), before[r])
        b.step(1.0, 2)
        got = [b.get_amplitudes(r) for r in range(len(shapes))]
    for r, shp in enumerate(shapes):
        ref = _alone(states[r], shp, 2, 1.0, o)[-1][0]
        assert float(np.max(np.abs(got[r] - ref))) == 0.0, r


def test_batch_measurement_counts_every_run():
    shapes = [(64, 64), (128, 96)]
    states = _states(shapes, seed=17)
    with _batch(states, shapes, _opts()) as b:
        b.profile_start("fused_apinv_f32")
        b.step(1.0)
        rec = b.profile_read("fused_apinv_f32")
        b.profile_stop()
        st = [b.stats(r) for r in range(len(shapes))]
    assert rec["launches"] > 0 and rec["ms"] > 0
    # one merged v-kernel launch per iteration moves 20 FP32 complex fields per amplitude
    # of every run still iterating; at least the first launch covers all runs
    assert rec["bytes"] >= 20 * 8 * 3 * sum(a * c for a, c in shapes)
    assert all(s["iters_last"] > 0 for s in st)


def test_batch_status_paths():
    L = O.hex_lattice()
    shapes = [(32, 32), (48, 40)]
    b = A.Batch(L.k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), shapes, H2, _opts())
    with b:
        assert b.try_step(1.0) == A.APFC_ESTATE  # amplitudes unset
        with pytest.raises(A.ApfcError):
            b.set_amplitudes(2, np.zeros((3, 32, 32), np.complex128))
        states = _states(shapes)
        for r, e in enumerate(states):
            b.set_amplitudes(r, e)
        b.step(1.0)
        bad = states[1].copy()
        bad[0, 3, 4] = np.nan
        b.set_amplitudes(1, bad)
        assert b.try_step(1.0) == A.APFC_ENAN
        assert "run 1" in b.last_error()
        assert b.try_step(1.0) == A.APFC_ESTATE  # sticky


def test_full_size_batch_64_runs_autotuned():
    # The batched benchmark workload in its launch configuration: 64 runs with N drawn from
    # {128, 256, 512, 1024}, tiles picked by the autotuner, Krylov blocks in CUDA graphs.
    # One run of each size matches the same run alone (same options) bit for bit, and the
    # smallest of them matches the FP64 oracle to the contract's 1e-10 relative L2 per
    # amplitude (the runs stop at relative residual <= 1e-10).
    phi = O.uniform_solid_hex(P)
    spec = inputs.batch_spec(64, (128, 256, 512, 1024), seed=7)
    states = [inputs.batch_run_state(phi, n, th, sd) for n, th, sd in spec]
    shapes = [(n, n) for n, _, _ in spec]
    opts = _opts(tol=1e-10)
    steps, dt = 2, 1.0
    with _batch(states, shapes, opts) as b:
        b.autotune(dt)
        o = b.opts
        for r, e in enumerate(states):
            b.set_amplitudes(r, e)
        b.step(dt, steps)
        picks = sorted({n: r for r, (n, _, _) in reversed(list(enumerate(spec)))}.items())
        got = {r: b.get_amplitudes(r) for _, r in picks}
        for _, r in picks:
            assert b.stats(r)["resid_last"] <= 1e-10
        b_resid = b.stats(picks[0][1])["resid_last"]
    assert [n for n, _ in picks] == [128, 256, 512, 1024]
    for n, r in picks:
        ref = _alone(states[r], shapes[r], steps, dt, o)[-1][0]
        assert float(np.max(np.abs(got[r] - ref))) == 0.0, (r, n)
    r = picks[0][1]
    ref = O.run(states[r], dt, steps, P, O.hex_lattice(), H2)[-1]
    errs = [rel_l2(got[r][j], ref[j]) for j in range(3)]
    print(f"batch 64 runs: smallest run ({picks[0][0]}^2) rel L2 per amplitude vs oracle {errs}, "
          f"resid {b_resid}")
    assert max(errs) <= 1e-10
