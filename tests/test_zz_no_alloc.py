"""The preconditioner entry point that allocates nothing.

apfc_apply_preconditioner_static() serves callers that may not allocate device
memory where they apply the preconditioner (an allocator owned by a framework,
a latency-critical path, a plugin handed buffers and a stream only).  It keeps
its intermediates in a fixed device array instead of context workspace, so it
must give the same result as the context entry point apfc_apply_preconditioner
and as the oracle's P^{-1}, call after call, even though the array keeps the
previous call's contents; and repeated calls must not change the device's free
memory.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, P, context, ensure_built

pytestmark = pytest.mark.gpu

CASES = [
    ("hex", (96, 80), H2, 3, A.APFC_TAU_FOLD, 1.0),
    ("hex", (61, 47), (0.9, 1.3), 5, A.APFC_TAU_PLAIN, 0.7),
    ("hex", (33, 40), H2, 0, A.APFC_TAU_FOLD, 1.0),
    ("bcc", (10, 12, 14), (1.1, 0.9, 1.2), 2, A.APFC_TAU_FOLD, 1.0),
    ("bcc", (9, 8, 11), (np.pi / 2,) * 3, 1, A.APFC_TAU_PLAIN, 0.8),
]
TAU = {A.APFC_TAU_FOLD: "fold", A.APFC_TAU_PLAIN: "plain"}


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def _static_args(L, kind, shape, h):
    lat = A.make_lattice(L.k, A.APFC_LATTICE_HEX2D if kind == "hex" else A.APFC_LATTICE_BCC3D)
    return lat, A.make_params(P.dB, P.Bx, P.t, P.v), A.make_grid(shape, h)


@pytest.mark.parametrize("kind,shape,h,m,tau,dt", CASES)
def test_static_preconditioner_matches_context_entry_point_and_oracle(kind, shape, h, m, tau, dt):
    torch = pytest.importorskip("torch")
    ctx, L = context(kind, shape, h, cheb_degree=m, tau_mode=tau)
    lat, prm, grid = _static_args(L, kind, shape, h)
    stream = torch.cuda.current_stream()
    for call in range(2):  # two calls in a row: the shared array keeps the previous contents
        b = inputs.random_amplitudes(2 * L.J, shape, seed=20 + call, scale=1.0).reshape((L.J, 2) + shape)
        ref = ctx.apply_preconditioner(dt, b)
        b_dev = torch.from_numpy(b).cuda()
        x_dev = torch.full_like(b_dev, complex(np.nan, np.nan))
        st = A.apfc_apply_preconditioner_static(
            lat, prm, grid, m, tau, dt, b_dev.data_ptr(), x_dev.data_ptr(), stream.cuda_stream
        )
        assert st == A.APFC_OK, A.STATUS_NAMES.get(st, st)
        stream.synchronize()
        got = x_dev.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(got, ref) < 1e-12
        for j in range(L.J):
            c1, c2 = O.apply_Pinv(b[j, 0], b[j, 1], L.k[j], dt, P, h, m, TAU[tau])
            assert _rel(got[j, 0], c1) < 1e-12
            assert _rel(got[j, 1], c2) < 1e-12


def test_static_preconditioner_leaves_free_device_memory_unchanged():
    torch = pytest.importorskip("torch")
    kind, shape, h, m, tau, dt = CASES[0]
    L = O.hex_lattice()
    lat, prm, grid = _static_args(L, kind, shape, h)
    b = torch.from_numpy(inputs.random_amplitudes(2 * L.J, shape, seed=5, scale=1.0)).cuda()
    x = torch.empty_like(b)
    stream = torch.cuda.current_stream()

    def call():
        st = A.apfc_apply_preconditioner_static(lat, prm, grid, m, tau, dt, b.data_ptr(), x.data_ptr(),
                                                stream.cuda_stream)
        assert st == A.APFC_OK
        stream.synchronize()

    call()  # the first call on a device may load the module that holds the array
    free0, _ = torch.cuda.mem_get_info()
    first = x.cpu()
    for _ in range(3):
        call()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(x.cpu(), first)


def test_static_preconditioner_rejects_oversized_aliased_and_bad_arguments():
    torch = pytest.importorskip("torch")
    L = A.make_lattice(inputs.hex_vectors(), A.APFC_LATTICE_HEX2D)
    prm = A.make_params(P.dB, P.Bx, P.t, P.v)
    n = 512  # 3 * 512^2 > APFC_STATIC_MAX_DOF
    assert 3 * n * n > A.APFC_STATIC_MAX_DOF
    big = A.make_grid((n, n), H2)
    b = torch.zeros((3, 2, 8), dtype=torch.complex128, device="cuda")  # never touched
    x = torch.zeros_like(b)
    st = A.apfc_apply_preconditioner_static(L, prm, big, 3, A.APFC_TAU_FOLD, 1.0, b.data_ptr(), x.data_ptr(), None)
    assert st == A.APFC_ETOOBIG
    assert A.STATUS_NAMES[st] == "ETOOBIG"
    # bad arguments are EINVAL and launch nothing
    small = A.make_grid((16, 16), H2)
    buf = torch.zeros((3, 2, 16, 16), dtype=torch.complex128, device="cuda")
    out = torch.zeros_like(buf)
    st = A.apfc_apply_preconditioner_static(L, prm, small, 3, A.APFC_TAU_FOLD, -1.0, buf.data_ptr(),
                                            out.data_ptr(), None)
    assert st == A.APFC_EINVAL
    # in place, or output overlapping the input by one element: EINVAL
    st = A.apfc_apply_preconditioner_static(L, prm, small, 3, A.APFC_TAU_FOLD, 1.0, buf.data_ptr(),
                                            buf.data_ptr(), None)
    assert st == A.APFC_EINVAL
    flat = torch.zeros(2 * buf.numel(), dtype=torch.complex128, device="cuda")
    st = A.apfc_apply_preconditioner_static(L, prm, small, 3, A.APFC_TAU_FOLD, 1.0, flat.data_ptr(),
                                            flat[buf.numel() - 1:].data_ptr(), None)
    assert st == A.APFC_EINVAL
    # 1/dt + |k|^2 dB <= 0 (the check the context makes): EINVAL
    neg = A.make_params(-2.0, P.Bx, P.t, P.v)
    st = A.apfc_apply_preconditioner_static(L, neg, small, 3, A.APFC_TAU_FOLD, 1.0, buf.data_ptr(),
                                            out.data_ptr(), None)
    assert st == A.APFC_EINVAL
    assert torch.count_nonzero(out).item() == 0
