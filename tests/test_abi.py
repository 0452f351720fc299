"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point that include/apfc.h declares, and its host-only functions
behave as documented."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)


@pytest.fixture(scope="module")
def lib():
    srcs = [os.path.join(B.CSRC, s) for s in os.listdir(B.CSRC)] + [os.path.join(ROOT, "include", "apfc.h")]
    if not os.path.exists(B.LIB) or os.path.getmtime(B.LIB) < max(os.path.getmtime(s) for s in srcs):
        B.build()
    return A.load()


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "apfc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(apfc_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_entry_points()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(A.EXPORTS), "binding and header disagree"


def test_default_opts(lib):
    o = A.apfc_default_opts()
    assert o.precision == A.APFC_FP64 and o.krylov == A.APFC_BICGSTAB
    assert o.tol == 1e-10 and o.max_iter == 500 and o.cheb_degree == 1 and o.tile == 3
    assert o.picard_iters == 1 and o.jacobian == 0 and o.tile_t == 1
    assert o.tau_mode == A.APFC_TAU_FOLD and 0 < o.tol_inner < 1 and o.check_every >= 1


def test_uniform_amplitude_matches_closed_forms(lib):
    prm = A.make_params(P.dB, P.Bx, P.t, P.v)
    hexL = A.make_lattice(O.hex_k(), A.APFC_LATTICE_HEX2D)
    bccL = A.make_lattice(O.bcc_k(), A.APFC_LATTICE_BCC3D)
    assert A.apfc_uniform_amplitude(hexL, prm) == pytest.approx(O.uniform_solid_hex(P), rel=1e-15)
    assert A.apfc_uniform_amplitude(bccL, prm) == pytest.approx(O.uniform_solid_bcc(P), rel=1e-15)
    with pytest.raises(A.ApfcError):
        A.apfc_uniform_amplitude(A.make_lattice(O.hex_k(), A.APFC_LATTICE_CUSTOM), prm)
    with pytest.raises(A.ApfcError):  # no real root
        A.apfc_uniform_amplitude(hexL, A.make_params(1.0, 1.0, 0.1, 1.0))


@pytest.mark.parametrize(
    "case",
    [
        "J0",
        "J9",
        "dim4",
        "hex_bad_sum",
        "grid_small",
        "h_zero",
        "nz_2d",
        "Bx_zero",
        "cheb_big",
        "tol_zero",
        "prec",
        "picard0",
        "picard101",
        "jac2",
        "tile_t5",
        "tile_t_neg2",
        "guess2",
    ],
)
def test_init_rejects_invalid_arguments_before_touching_cuda(lib, case):
    k = O.hex_k()
    kind = A.APFC_LATTICE_HEX2D
    shape, h = (8, 8), (1.0, 1.0)
    prm = A.make_params(P.dB, P.Bx, P.t, P.v)
    opts = A.apfc_default_opts()
    L = A.make_lattice(k, kind)
    G = A.make_grid(shape, h)
    if case == "J0":
        L.J = 0
    elif case == "J9":
        L.J = 9
    elif case == "dim4":
        L.dim = 4
    elif case == "hex_bad_sum":
        L.k[0][0] += 0.1
    elif case == "grid_small":
        G.n[0] = 2
    elif case == "h_zero":
        G.h[1] = 0.0
    elif case == "nz_2d":
        G.n[2] = 4
    elif case == "Bx_zero":
        prm.Bx = 0.0
    elif case == "cheb_big":
        opts.cheb_degree = 17
    elif case == "tol_zero":
        opts.tol = 0.0
    elif case == "prec":
        opts.precision = 7
    elif case == "picard0":
        opts.picard_iters = 0
    elif case == "picard101":
        opts.picard_iters = 101
    elif case == "jac2":
        opts.jacobian = 2
    elif case == "tile_t5":
        opts.tile_t = 6
    elif case == "tile_t_neg2":
        opts.tile_t = -2
    elif case == "guess2":
        opts.guess = 2
    import ctypes as C

    h_ = C.c_void_p()
    st = lib.apfc_init(C.byref(h_), C.byref(L), C.byref(prm), C.byref(G), C.byref(opts), None)
    assert st == A.APFC_EINVAL
    assert not h_.value
    # without a context the failed init explains itself (per thread)
    msg = lib.apfc_last_error(None).decode()
    assert msg and msg != "null context", msg


def test_init_failure_message_names_the_cause(lib):
    k = O.hex_k()
    with pytest.raises(A.ApfcError) as e:
        A.Context(k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), (2, 8), (1.0, 1.0))
    assert e.value.status == A.APFC_EINVAL
    assert "grid sizes" in str(e.value)
    import torch

    if not torch.cuda.is_available():
        # a host without a usable GPU: ECUDA with the reason, never a CPU fallback
        with pytest.raises(A.ApfcError) as e:
            A.Context(k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), (8, 8), (1.0, 1.0))
        assert e.value.status == A.APFC_ECUDA and "no CUDA device" in str(e.value)


def test_binding_fails_loudly_without_library(tmp_path):
    saved = A._lib
    try:
        A._lib = None
        with pytest.raises(RuntimeError, match="not built"):
            A.load(str(tmp_path / "missing.so"))
    finally:
        A._lib = saved


@pytest.mark.parametrize("case", ["nruns0", "nx2", "bcc", "fp64", "unfused", "flags", "hx0", "cheb5", "picard", "jac", "guess"])
def test_batch_init_rejects_invalid_arguments_before_touching_cuda(lib, case):
    import ctypes as C

    k, kind = O.hex_k(), A.APFC_LATTICE_HEX2D
    prm = A.make_params(P.dB, P.Bx, P.t, P.v)
    opts = A.apfc_default_opts(precision=A.APFC_FP32_REFINED)
    nx, ny, R, hx, flags = [64, 128], [64, 96], 2, 1.0, 0
    if case == "nruns0":
        R = 0
    elif case == "nx2":
        nx[1] = 2
    elif case == "bcc":
        k, kind = O.bcc_k(), A.APFC_LATTICE_BCC3D
    elif case == "fp64":
        opts.precision = A.APFC_FP64
    elif case == "unfused":
        opts.fused = 0
    elif case == "flags":
        flags = 6
    elif case == "hx0":
        hx = 0.0
    elif case == "cheb5":
        opts.cheb_degree = 5
    elif case == "picard":
        opts.picard_iters = 2
    elif case == "jac":
        opts.jacobian = 1
    elif case == "guess":
        opts.guess = A.APFC_GUESS_EXTRAP
    L = A.make_lattice(k, kind)
    h_ = C.c_void_p()
    st = lib.apfc_batch_init(
        C.byref(h_), C.byref(L), C.byref(prm), R, (C.c_int * 2)(*nx), (C.c_int * 2)(*ny), hx, 1.0, C.byref(opts),
        flags, None,
    )
    assert st == A.APFC_EINVAL
    assert not h_.value


def test_batch_spec_draws_sizes_and_rotations():
    from paper_1902_09761_gb300 import inputs

    spec = inputs.batch_spec(64, seed=7)
    assert len(spec) == 64
    assert {n for n, _, _ in spec} <= {128, 256, 512, 1024} and len({n for n, _, _ in spec}) == 4
    assert all(-10 <= th <= 10 for _, th, _ in spec)
    assert spec == inputs.batch_spec(64, seed=7)


def test_batch_init_failure_message_names_the_cause(lib):
    k = O.hex_k()
    with pytest.raises(A.ApfcError) as e:
        A.Batch(k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), [(8, 8), (2, 8)], (1.0, 1.0))
    assert e.value.status == A.APFC_EINVAL and "run 1" in str(e.value)
    import torch

    if not torch.cuda.is_available():
        with pytest.raises(A.ApfcError) as e:
            A.Batch(k, A.APFC_LATTICE_HEX2D, (P.dB, P.Bx, P.t, P.v), [(8, 8)], (1.0, 1.0))
        assert e.value.status == A.APFC_ECUDA and "no CUDA device" in str(e.value)
