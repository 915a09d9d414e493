"""The package's smoke entry point (one small FP64 run on cuda:0 checked
against the oracle every iteration) stays green."""
import pytest

pytestmark = pytest.mark.gpu


def test_graft_entry_smoke():
    import __graft_entry__ as g

    g.smoke()
