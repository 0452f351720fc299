"""The preconditioner entry point that allocates nothing.

apfc_apply_preconditioner_static() serves callers that may not allocate device
memory where they apply the preconditioner (an allocator owned by a framework,
a latency-critical path, a plugin handed buffers and a stream only).  It keeps
its intermediates in a fixed device array instead of context workspace, so it
must give the same result as the context entry point apfc_apply_preconditioner,
call after call, even though the array keeps the previous call's contents.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, P, context, ensure_built

pytestmark = pytest.mark.gpu

CASES = [
    ("hex", (96, 80), H2, 3, A.APFC_TAU_FOLD, 1.0),
    ("hex", (61, 47), (0.9, 1.3), 5, A.APFC_TAU_PLAIN, 0.7),
    ("bcc", (10, 12, 14), (1.1, 0.9, 1.2), 2, A.APFC_TAU_FOLD, 1.0),
]


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("kind,shape,h,m,tau,dt", CASES)
def test_static_preconditioner_matches_context_entry_point(kind, shape, h, m, tau, dt):
    torch = pytest.importorskip("torch")
    ctx, L = context(kind, shape, h, cheb_degree=m, tau_mode=tau)
    lat = A.make_lattice(L.k, A.APFC_LATTICE_HEX2D if kind == "hex" else A.APFC_LATTICE_BCC3D)
    prm = A.make_params(P.dB, P.Bx, P.t, P.v)
    grid = A.make_grid(shape, h)
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


def test_static_preconditioner_rejects_oversized_problems():
    torch = pytest.importorskip("torch")
    L = A.make_lattice(inputs.hex_vectors(), A.APFC_LATTICE_HEX2D)
    prm = A.make_params(P.dB, P.Bx, P.t, P.v)
    n = 512  # 3 * 512^2 > APFC_STATIC_MAX_DOF
    assert 3 * n * n > A.APFC_STATIC_MAX_DOF
    grid = A.make_grid((n, n), H2)
    b = torch.zeros((3, 2, 8), dtype=torch.complex128, device="cuda")  # never touched
    st = A.apfc_apply_preconditioner_static(L, prm, grid, 3, A.APFC_TAU_FOLD, 1.0, b.data_ptr(), b.data_ptr(), None)
    assert st == A.APFC_ETOOBIG
    assert A.STATUS_NAMES[st] == "ETOOBIG"
    # bad arguments are still EINVAL
    st = A.apfc_apply_preconditioner_static(L, prm, grid, 3, A.APFC_TAU_FOLD, -1.0, b.data_ptr(), b.data_ptr(), None)
    assert st == A.APFC_EINVAL
    assert isinstance(C.c_void_p(b.data_ptr()).value, int)
