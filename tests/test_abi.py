"""CPU checks of the boundary: the C-ABI library builds, loads and exports every symbol
declared in include/kite_gb.h; host-only entry points behave.  No compute calls."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(kite_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def built():
    from paper_1910_05194_gb300 import _build
    return _build.build()


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    names = declared_symbols()
    assert "kite_moments_1d" in names and "kite_reconstruct_dos" in names
    for n in sorted(names):
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"
    import paper_1910_05194_gb300 as kite
    assert set(kite.EXPORTED) == names


def test_status_strings_and_host_bounds(built):
    import paper_1910_05194_gb300 as kite
    L = kite.lib()
    for s in (0, -1, -2, -3, -4, -5, -6, 99):
        assert L.kite_status_string(s)
    lo, hi = kite.bounds(kite.make_system(kite.HONEYCOMB, 8, 8, t=-2.7, W=1.0))
    assert hi == -lo and abs(hi - (3 * 2.7 + 0.5) * 1.01) < 1e-15
    import oracle
    assert (lo, hi) == oracle.bounds_auto(oracle.make_system(Lx=8, Ly=8, t=-2.7, W=1.0))
    lo, hi = kite.bounds(kite.make_system(kite.SQUARE, 8, 8, t=-1.0, W=3.0))
    assert hi == (4.0 + 1.5) * 1.01
    with pytest.raises(kite.KiteError):
        kite.bounds(kite.make_system(kite.HONEYCOMB, 0, 8))
    # Gaussian disorder: the transform's largest draw, 8.58 standard deviations
    g = dict(Lx=8, Ly=8, t=-2.7, W=0.4, delta=0.2)
    lo, hi = kite.bounds(kite.make_system(kite.HONEYCOMB, disorder=kite.DISORDER_GAUSSIAN, **g))
    assert (lo, hi) == oracle.bounds_auto(oracle.make_system(disorder=oracle.GAUSSIAN, **g))
    assert abs(hi - (3 * 2.7 + 8.58 * 0.4 + 0.1) * 1.01) < 1e-14
    with pytest.raises(kite.KiteError):
        kite.bounds(kite.make_system(kite.HONEYCOMB, 8, 8, disorder=2))


def test_context_creation_fails_cleanly_without_gpu(built):
    import paper_1910_05194_gb300 as kite
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    with pytest.raises(kite.KiteError) as e:
        kite.Context(0)
    assert e.value.status in (kite.ERR_ARG, kite.ERR_CUDA)
