"""The allocation-free float32 matvec (fl_matvec_f32_static), for callers that
cannot allocate device memory, must give the product of the allocating
fl_matvec(FL_F32) on consecutive calls that share its fixed device array.
Collected last on purpose; it also passes alone in a fresh process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1708_03912_gb300 import fraclap as F  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def test_static_matvec_matches_allocating_matvec_twice():
    # a real stiffness matrix (odd n: unaligned rows) and a random one with aligned rows
    V, T = synth.disc(8)
    m = F.Mesh(V, T)
    A = m.assemble(0.6, "fp64")
    m.close()
    g = torch.Generator(device="cpu").manual_seed(11)
    Ar = torch.randn(1024, 1024, generator=g, dtype=torch.float64).cuda()
    for A64 in (A, Ar):
        n = A64.shape[0]
        A32 = torch.empty((n, n), dtype=torch.float32, device="cuda")
        F.fl_convert(A64, F.FL_F32, A32)
        for call in range(2):  # two calls in a row reuse the same device array
            x = torch.randn(n, 1, generator=g, dtype=torch.float64).cuda()
            y_ref = torch.empty(n, 1, dtype=torch.float64, device="cuda")
            F.fl_matvec(F.FL_F32, A32, x, y_ref)
            y = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
            assert F.fl_matvec_f32_static(A32, x[:, 0].contiguous(), y) == F.FL_OK
            torch.cuda.synchronize()
            yr = y_ref[:, 0].cpu().numpy()
            scale = float(np.abs(A32.double().cpu().numpy()).sum(axis=1).max() * x.abs().max().item())
            assert np.allclose(y.cpu().numpy(), yr, rtol=1e-5, atol=1e-5 * scale), f"call {call}"


def test_static_matvec_rejects_oversize():
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    xd = torch.zeros(4, dtype=torch.float64, device="cuda")
    code = F.lib().fl_matvec_f32_static(F._ptr(dummy), F.FL_STATIC_MAX_N + 1, F.FL_STATIC_MAX_N + 1, F._ptr(xd),
                                        F._ptr(xd), F._stream())
    assert code == F.FL_EINVAL
