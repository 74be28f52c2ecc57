"""The round-trip the build entry point runs on a GPU machine: __graft_entry__.smoke()."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import __graft_entry__ as g
    g.smoke()
