"""The allocation-free inner product (csm_dot_noalloc), for callers that cannot allocate
device memory, against the workspace version csm_dot.  Kept in its own file that pytest
collects last; it passes alone in a fresh process and after the other tests."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_dot_on_two_calls_in_a_row():
    from paper_2511_12235_gb300 import _capi as capi
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev).cuda_stream
    rng = np.random.default_rng(11)
    cases = [(torch.float32, capi.CSM_F32, 5, 100_003), (torch.float64, capi.CSM_F64, 64, 4_099),
             (torch.float32, capi.CSM_F32, 1, 1)]
    for tdt, cdt, B, n in cases:
        a = torch.from_numpy(rng.normal(size=(B, n))).to(dev, tdt)
        c = torch.from_numpy(rng.normal(size=(B, n))).to(dev, tdt)
        ref = torch.zeros(B, dtype=torch.float64, device=dev)
        ws = torch.empty(capi.csm_dot_workspace_bytes(B), dtype=torch.uint8, device=dev)
        capi.csm_dot(a.data_ptr(), c.data_ptr(), n, B, cdt, ref.data_ptr(), ws.data_ptr(), ws.numel(), stream)
        for _ in range(2):   # the shared array keeps the previous call's partial sums
            out = torch.full((B,), float("nan"), dtype=torch.float64, device=dev)
            capi.csm_dot_noalloc(a.data_ptr(), c.data_ptr(), n, B, cdt, out.data_ptr(), stream)
            torch.cuda.synchronize()
            assert torch.allclose(out, ref, rtol=1e-12, atol=0.0), (out, ref)
        exact = (a.double() * c.double()).sum(dim=1)
        assert torch.allclose(ref, exact, rtol=1e-10, atol=1e-10)


def test_dot_noalloc_refuses_batches_beyond_its_array():
    from paper_2511_12235_gb300 import _capi as capi
    dev = torch.device("cuda", 0)
    B = capi.CSM_DOT_NOALLOC_MAX_BATCH + 1
    a = torch.ones(B, 8, device=dev)
    out = torch.zeros(B, dtype=torch.float64, device=dev)
    st = capi.lib.csm_dot_noalloc(a.data_ptr(), a.data_ptr(), 8, B, capi.CSM_F32, out.data_ptr(),
                                  torch.cuda.current_stream(dev).cuda_stream)
    assert st == capi.CSM_EINVAL
