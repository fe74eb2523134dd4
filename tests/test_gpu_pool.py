"""The caching allocator: handles created and destroyed in a loop reuse cached device and
pinned blocks, give bitwise the same matrices, and fl_pool_trim releases the cache."""
import pytest

torch = pytest.importorskip("torch")

from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_handles_reuse_cached_blocks():
    V, T = synth.disc(8)
    m = F.Mesh(V, T)
    A0 = m.assemble(0.75, "mixed").clone()
    b0 = m.load_vector(0.75).clone()
    m.solve(A0, b0, tol=1e-10)
    m.close()
    st0 = F.fl_pool_stats()
    assert st0["cached_device_bytes"] > 0 and st0["cached_host_bytes"] > 0
    for _ in range(3):
        m = F.Mesh(V, T)
        A = m.assemble(0.75, "mixed")
        u, info = m.solve(A, m.load_vector(0.75), tol=1e-10)
        assert torch.equal(A, A0)
        assert info.status == F.FL_OK
        m.close()
    st1 = F.fl_pool_stats()
    assert st1["hits"] > st0["hits"]
    assert st1["misses"] == st0["misses"]  # same sizes: every request served from the cache
    released = F.fl_pool_trim()
    assert released >= st1["cached_device_bytes"] > 0
    st2 = F.fl_pool_stats()
    assert st2["cached_device_bytes"] == 0 and st2["cached_host_bytes"] == 0
    # the library works after a trim
    m = F.Mesh(V, T)
    assert torch.equal(m.assemble(0.75, "mixed"), A0)
    assert torch.equal(m.load_vector(0.75), b0)
    m.close()
