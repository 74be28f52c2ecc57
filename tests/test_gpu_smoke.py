"""__graft_entry__.smoke(): one small fused step sequence on cuda:0, checked against the oracle."""
import pytest

pytestmark = pytest.mark.gpu


def test_smoke_entry_point():
    import __graft_entry__ as g
    g.smoke()
