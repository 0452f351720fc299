"""Rotation diagnostic and adaptivity map on the GPU against the oracle
(``oracle/diagnostics.py``): omega, A and the map of Eq. hhh element by element
on grains, polycrystals and a 3D bcc sphere.

The kernel takes each phase difference arg(a conj(b)) with FP32 atan2 of the FP64
product scaled to unit size: an absolute error of a few 1e-8 rad per difference,
divided by 2h and summed with weights |M^{-1} k_j| <= 1, so omega agrees to 1e-6
absolute and h_amp (a smooth function of omega) to 1e-5 relative.  A and grad A
are FP64 on both sides, so the branches of Eq. hhh are the oracle's."""
import numpy as np
import pytest

import oracle as O
from oracle import diagnostics as D
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import inputs

from gpu_common import H2, H3, P, ensure_built, lattice

pytestmark = pytest.mark.gpu

ADAPT = dict(n=10.0, h_int=1.0, h_max=40.0, eps=0.02, A_min=0.05)


@pytest.fixture(scope="module", autouse=True)
def lib():
    return ensure_built()


def _check(kind, eta, shape, h, device=None):
    L, code = lattice(kind)
    with A.Context(L.k, code, (P.dB, P.Bx, P.t, P.v), shape, h) as c:
        c.set_amplitudes(eta)
        om, am, hm = c.rotation_field(ADAPT, device=device)
    if device is not None:
        om, am, hm = om.cpu().numpy(), am.cpu().numpy(), hm.cpu().numpy()
    ref_om = D.rotation_field(eta, L.k, h)
    ref_A = D.amplitude_A(eta)
    ref_h = D.adaptivity_map(eta, L.k, h, **ADAPT)
    assert np.max(np.abs(om - ref_om)) <= 1e-6
    assert np.max(np.abs(am - ref_A)) <= 1e-13 * max(1.0, np.max(ref_A))
    # branch decisions: equal except where |grad A| or A sits on a threshold to rounding
    gA = D.grad_norm(ref_A, h)
    edge = (np.abs(gA - ADAPT["eps"]) <= 1e-12) | (np.abs(ref_A - ADAPT["A_min"]) <= 1e-12)
    both_inf = np.isinf(hm) & np.isinf(ref_h)
    close = both_inf | (np.abs(hm - ref_h) <= 1e-5 * np.maximum(1.0, np.abs(ref_h)))
    assert np.all(close | edge)
    return om, hm


@pytest.mark.parametrize("device", [None, "cuda"])
def test_rotation_and_map_single_grain(device):
    shape = (96, 112)
    eta = inputs.single_grain(O.hex_k(), O.uniform_solid_hex(P), shape, H2, 40.0, 7.0, seed=1, noise=1e-3)
    om, hm = _check("hex", eta, shape, H2, device)
    assert np.min(hm) == ADAPT["h_int"] and np.max(hm) == ADAPT["h_max"]


def test_rotation_and_map_polycrystal_ragged():
    shape = (130, 170)
    eta = inputs.voronoi_grains(O.hex_k(), O.uniform_solid_hex(P), shape, (1.3, 1.4), 6, 12.0, seed=2, noise=1e-3)
    _check("hex", eta, shape, (1.3, 1.4))


def test_rotation_and_map_bcc_sphere():
    shape = (20, 24, 28)
    phi = O.uniform_solid_bcc(P)
    eta = inputs.single_grain(O.bcc_k(), phi, shape, H3, 12.0, 8.0, seed=3, noise=1e-3, matrix=phi)
    om, _ = _check("bcc", eta, shape, H3)
    assert om.shape == (3,) + shape
