"""CPU checks of the C ABI library: it loads and exports every declared symbol.

No compute calls: this runs without a GPU.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vegas_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2010_09341_gb300 import build as B
    from paper_2010_09341_gb300 import _native as nat
    try:
        B.build()
    except RuntimeError as exc:  # no nvcc
        pytest.skip(str(exc))
    return nat.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared("vegas.h")
    assert "vegas_create" in names and "vegas_iterate" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2010_09341_gb300 import _native as nat
    assert sorted(nat.declared_symbols()) == _declared("vegas.h")


def test_workspace_bytes_validates_config(lib):
    import ctypes
    from paper_2010_09341_gb300 import _native as nat

    def ws(**kw):
        base = dict(n_dim=4, n_bins=50, n_events=1000, events_limit=0, alpha=1.5, seed=0,
                    integral_id=0, precision=0, smooth=1)
        base.update(kw)
        c = nat.VegasConfig(**base)
        return lib.vegas_workspace_bytes(ctypes.byref(c))

    assert ws() > 0
    assert ws() % 256 == 0
    assert ws(n_dim=0) == 0
    assert ws(n_dim=33) == 0
    assert ws(n_bins=1) == 0
    assert ws(n_bins=1025) == 0
    assert ws(n_events=1) == 0
    assert ws(alpha=-1.0) == 0
    assert ws(precision=7) == 0
    assert ws(n_dim=32, n_bins=1024) > ws(n_dim=4, n_bins=50)


def test_strerror(lib):
    assert lib.vegas_strerror(0) == b"ok"
    assert b"invalid" in lib.vegas_strerror(1)


def test_step_many_rejects_bad_arguments_before_any_launch(lib):
    """vegas_step_many validates on the host: a NULL array, a count out of
    [1, VEGAS_MAX_STEP_MANY] and NULL contexts return VEGAS_EINVAL (no device
    call is reached, so this runs without a GPU)."""
    import ctypes
    from paper_2010_09341_gb300 import _native as nat
    P = ctypes.c_void_p
    assert lib.vegas_step_many(None, 1) == nat.VEGAS_EINVAL
    two = (P * 2)(None, None)
    assert lib.vegas_step_many(two, 2) == nat.VEGAS_EINVAL
    nine = (P * 9)()
    assert lib.vegas_step_many(nine, 9) == nat.VEGAS_EINVAL
    assert lib.vegas_step_many(two, 0) == nat.VEGAS_EINVAL
    assert lib.vegas_step_many(two, -1) == nat.VEGAS_EINVAL
