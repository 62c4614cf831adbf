"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol that
include/hps.h declares; its host-only functions agree with the oracle's point bookkeeping."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.grid import Grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hps.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("hps_", "ark_"))))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_02526_gb300 import build, _lib
    build.build()
    return _lib.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("hps_build", "hps_solve", "ark_step", "hps_free", "hps_bytes", "hps_strerror"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2306_02526_gb300 import _lib
    names = declared_functions()
    assert set(names) <= set(_lib.SIGNATURES), "binding misses a declared function"
    for n in names:
        assert hasattr(lib, n), n


@pytest.mark.parametrize("n1,n2,p", [(1, 1, 4), (4, 2, 7), (2, 8, 9), (16, 16, 16)])
def test_host_bookkeeping_matches_oracle(lib, n1, n2, p):
    from paper_2306_02526_gb300 import hps
    t = hps.Tree(n1, n2, -0.5, 2.0, 0.25, 1.5)
    g = Grid(n1, n2, p, -0.5, 2.0, 0.25, 1.5)
    N, Ni, Nb = hps.hps_sizes(t, p)
    assert (N, Ni) == (g.N, g.N_int)
    x, y = hps.hps_coords(t, p)
    X, Y = g.coords()
    assert np.abs(x - X).max() < 1e-14 and np.abs(y - Y).max() < 1e-14
    assert np.array_equal(hps.hps_boundary_index(t, p), g.boundary_indices())
    assert Nb == g.boundary_indices().size


def test_argument_checks(lib):
    from paper_2306_02526_gb300 import hps, _lib
    with pytest.raises(_lib.HPSError):
        hps.hps_sizes(hps.Tree(3, 2), 8)          # not a power of two
    with pytest.raises(_lib.HPSError):
        hps.hps_sizes(hps.Tree(2, 2), 3)          # p too small
    with pytest.raises(_lib.HPSError):
        hps.hps_sizes(hps.Tree(2, 2, 1.0, 0.0), 8)  # empty domain
    assert hps.hps_bytes(hps.Tree(3, 2), 8) == 0
    assert lib.hps_strerror(-3).decode().startswith("zero or non-finite pivot")


def test_bytes_grow_with_per_node_operators(lib):
    from paper_2306_02526_gb300 import hps
    t = hps.Tree(64, 64)
    shared = hps.hps_bytes(t, 16)
    nodal = hps.hps_bytes(t, 16, nodal=True)
    assert 0 < shared < nodal
    # per-node operator bytes of 64x64 leaves, p = 16: sum over leaves of q^2 + q b and over
    # merges of n3^2 + 2 n3 nb (root: n3^2 + n3 nb), FP64, rows padded to even length
    assert 2.1e9 < nodal < 2.6e9
