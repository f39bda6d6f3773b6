"""Host-side checks of the C ABI library (no GPU needed): it builds for
sm_103a, loads, and exports every function include/sldqmc.h declares."""
import pytest

from paper_1612_03804_gb300 import build as B
from paper_1612_03804_gb300 import sldqmc


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sldqmc.load()


def test_exports_every_declared_symbol(lib):
    names = sldqmc.declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing


def test_strerror_and_null_args(lib):
    assert lib.sldqmc_strerror(0) == b"ok"
    assert lib.sldqmc_strerror(-4).startswith(b"numerical")
    # argument validation happens before any device work
    assert lib.sldqmc_create(None, None, None) == -1
    assert lib.sldqmc_weight(None, None, 1, None, None) == -1
    assert lib.sldqmc_sync(None) == -1


def test_create_rejects_bad_params(lib):
    import ctypes
    h = ctypes.c_void_p()
    bad = [
        sldqmc.Params(4, 4, 1.0, 0.0, 1.0, 2.0, 0.3, 10, 1.0, 2.774, 0, 1),   # beta not a multiple of dtau
        sldqmc.Params(0, 4, 1.0, 0.0, 1.0, 2.0, 0.1, 10, 1.0, 2.774, 0, 1),   # empty lattice
        sldqmc.Params(4, 4, 1.0, 0.0, 1.0, 2.0, 0.1, 0, 1.0, 2.774, 0, 1),    # n_wrap 0
        sldqmc.Params(4, 4, 1.0, 0.0, 1.0, 2.0, 0.1, 10, 1.0, 2.774, 7, 1),   # unknown precision
        sldqmc.Params(4, 4, 1.0, 0.0, 1.0, 2.0, 0.1, 10, 1.0, 2.774, 0, 0),   # empty batch
        sldqmc.Params(4, 4, 1.0, 0.0, 1.0, 20.0, 0.5, 40, 1.0, 2.774, 0, 1),  # block too ill-conditioned
    ]
    for p in bad:
        assert lib.sldqmc_create(ctypes.byref(p), None, ctypes.byref(h)) in (-1, -6)
