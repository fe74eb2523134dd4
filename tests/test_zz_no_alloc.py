"""The allocation-free float32 matvec (fl_matvec_f32_static) is for callers that
cannot allocate device memory: code under a caller-owned memory budget or inside
another allocator's arena, real-time loops that must stay out of the driver's
allocator, and hosts that only receive device pointers.  Its product must equal
the float64 product of the float32-rounded operands within the float32
summation bound, and agree with the allocating fl_matvec(FL_F32), on consecutive
calls that share its fixed device array; and the calls must allocate nothing.
Collected last on purpose; it also passes alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def _cases():
    """(float64 matrix on the device, row pitch of its float32 copy)."""
    V, T = synth.disc(8)
    m = F.Mesh(V, T)
    A = m.assemble(0.6, "fp64")  # odd n = 49: unaligned rows, the scalar loop only
    m.close()
    g = torch.Generator(device="cpu").manual_seed(11)
    Ar = torch.randn(1024, 1024, generator=g, dtype=torch.float64).cuda()  # 16-byte rows, no tail
    Ap = torch.randn(1000, 1000, generator=g, dtype=torch.float64).cuda()  # 16-byte rows + a tail, lda > n
    return [(A, A.shape[0]), (Ar, 1024), (Ap, 1004)], g


def _host_bound(A32, x):
    """float64 product of the float32-rounded operands and the bound of float32 lane sums."""
    a = A32.double().cpu().numpy()
    xr = x.float().double().cpu().numpy()
    n = a.shape[0]
    ref = a @ xr
    # every lane sums at most ceil(n / 32) products by fmaf; the float64 total adds ~2^-52
    bound = (np.ceil(n / 32) + 2) * U32 * (np.abs(a) @ np.abs(xr))
    return ref, bound


def test_static_matvec_matches_host_product_and_fl_matvec_twice():
    cases, g = _cases()
    for A64, lda in cases:
        n = A64.shape[0]
        buf = torch.zeros((n, lda), dtype=torch.float32, device="cuda")
        A32 = buf[:, :n]
        F.fl_convert(A64, F.FL_F32, A32)
        for call in range(2):  # two calls in a row reuse the same device array
            x = torch.randn(n, generator=g, dtype=torch.float64).cuda()
            y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            assert F.fl_matvec_f32_static(A32, x, y) == F.FL_OK
            y_ref = torch.empty(n, 1, dtype=torch.float64, device="cuda")
            F.fl_matvec(F.FL_F32, A32, x[:, None].contiguous(), y_ref)
            torch.cuda.synchronize()
            yh = y.cpu().numpy()
            ref, bound = _host_bound(A32, x)
            assert np.all(np.abs(yh - ref) <= bound), f"n {n} lda {lda} call {call}"
            # the allocating entry point: same arithmetic, within twice the bound
            assert np.all(np.abs(yh - y_ref[:, 0].cpu().numpy()) <= 2 * bound), f"n {n} lda {lda} call {call}"


def test_static_matvec_allocates_nothing():
    cases, g = _cases()
    A64, lda = cases[1]
    n = A64.shape[0]
    A32 = torch.empty((n, n), dtype=torch.float32, device="cuda")
    F.fl_convert(A64, F.FL_F32, A32)
    x = torch.randn(n, generator=g, dtype=torch.float64).cuda()
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    assert F.fl_matvec_f32_static(A32, x, y) == F.FL_OK  # first call: symbol lookup, kernels loaded
    torch.cuda.synchronize()
    pool0 = F.fl_pool_stats()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert F.fl_matvec_f32_static(A32, x, y) == F.FL_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert F.fl_pool_stats() == pool0
    assert free1 == free0


def test_static_matvec_rejects_oversize():
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    xd = torch.zeros(4, dtype=torch.float64, device="cuda")
    code = F.lib().fl_matvec_f32_static(F._ptr(dummy), F.FL_STATIC_MAX_N + 1, F.FL_STATIC_MAX_N + 1, F._ptr(xd),
                                        F._ptr(xd), F._stream())
    assert code == F.FL_EINVAL
