"""The allocation-free residual entry point (lbms_residual_sums_noalloc).

Some callers cannot allocate device memory (a CUDA graph under capture, a
host framework that owns all device memory, a loop that must not call
cudaMalloc because it synchronises the device).  For them the library offers
one entry point whose scratch lives in a fixed device array.  This test calls
it through the C ABI on caller-owned FP64 fields and checks, on two calls in
a row, that it reproduces the residual of the existing lbms_residual entry
point and that it refreshes the caller's snapshot.  It sits in its own file,
collected last, and passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import cases

pytestmark = pytest.mark.gpu


def test_noalloc_residual_matches_lbms_residual():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms as L
    lib = L.load()
    case = cases.porous((16, 24, 30), radius=2, porosity=0.5, seed=31, current_A_cm2=1.0)
    fluid = ~case.solid.reshape(-1)
    s = L.Solver.from_case(case, precision="fp64")
    s.set_bc(case.x_in, case.current_A_cm2)
    s.step(40)
    s.residual(1)                     # the solver's snapshot is now X_0

    def fluid_field():
        X = s.fields().reshape(3, -1)[:, fluid]
        return torch.tensor(np.ascontiguousarray(X), dtype=torch.float64, device="cuda")

    snap = fluid_field()
    n = snap.shape[1]
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    K = 25
    for call in range(2):
        s.step(K)
        X = fluid_field()
        expected = s.residual(K)      # existing entry point: X_{call+1} against X_call
        before = snap.clone()
        st = lib.lbms_residual_sums_noalloc(X.data_ptr(), snap.data_ptr(), n, 1, out.data_ptr(),
                                            C.c_void_p(stream))
        assert st == L.LBMS_OK
        torch.cuda.synchronize()
        sums = out.cpu().numpy()
        res = max(np.sqrt(sums[i]) / (K * np.sqrt(sums[3 + i])) for i in range(3) if sums[3 + i] > 0)
        assert res == pytest.approx(expected, rel=1e-12)
        ref = X.cpu().numpy()
        assert np.allclose(sums[6:9], ref.sum(axis=1), rtol=1e-12)
        assert np.allclose(sums[0:3], ((ref - before.cpu().numpy()) ** 2).sum(axis=1), rtol=1e-10)
        assert sums[9] == 0.0
        assert torch.equal(snap, X)   # update = 1 refreshed the caller's snapshot
    s.close()


def test_noalloc_rejects_bad_sizes():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms as L
    lib = L.load()
    buf = torch.zeros(30, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    assert lib.lbms_residual_sums_noalloc(p, p, 0, 0, p, None) == L.LBMS_EINVAL
    assert lib.lbms_residual_sums_noalloc(p, p, 2 ** 31, 0, p, None) == L.LBMS_EINVAL
    assert lib.lbms_residual_sums_noalloc(None, p, 5, 0, p, None) == L.LBMS_EINVAL
