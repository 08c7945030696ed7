"""The entry point's smoke() on the GPU: a whole robust adjustment of a small
block in both precisions, each ending within 1e-3 px of the oracle's RMS."""

import pytest

pytestmark = pytest.mark.gpu


def test_smoke():
    import __graft_entry__

    __graft_entry__.smoke()
