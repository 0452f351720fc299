"""Shared helpers of the GPU parity tests (CUDA library vs FP64 oracle)."""
import os

import numpy as np

import oracle as O
from paper_1902_09761_gb300 import apfc as A
from paper_1902_09761_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P = O.params_from_paper(0.98, 0.01, 0.25, 0.5)
H2 = (np.pi / 2, np.pi / 2)
H3 = (np.pi / 2,) * 3


def ensure_built():
    srcs = [os.path.join(B.CSRC, s) for s in os.listdir(B.CSRC)] + [os.path.join(ROOT, "include", "apfc.h")]
    if not os.path.exists(B.LIB) or os.path.getmtime(B.LIB) < max(os.path.getmtime(s) for s in srcs):
        B.build()
    return A.load()


def lattice(kind):
    if kind == "hex":
        return O.hex_lattice(), A.APFC_LATTICE_HEX2D
    return O.bcc_lattice(), A.APFC_LATTICE_BCC3D


def context(kind, shape, h, p=P, **opts):
    L, code = lattice(kind)
    o = A.apfc_default_opts(**opts)
    return A.Context(L.k, code, (p.dB, p.Bx, p.t, p.v), shape, h, o), L


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def rel_l2_per_amp(a, b):
    return [rel_l2(a[j], b[j]) for j in range(a.shape[0])]
