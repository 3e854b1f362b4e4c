"""The allocation-free tensor-core product against the allocating entry point.

sim_tc_gemm_noalloc serves callers that cannot allocate device memory (a
serving process with all of HBM divided into fixed slots, or a loop where
cudaMalloc would synchronise the device); it keeps its scratch in one fixed
device array inside the library.  It must give the same result as
sim_debug_tc_gemm, within the tolerance of the other tensor-core tests, on
consecutive calls that reuse that scratch.  This file is collected last.
"""
import numpy as np
import pytest

import paper_2303_00689_gb300 as kx

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2303_00689_gb300 import build
    build.build()


def test_no_alloc_matches_allocating_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(2024)
    for n, terms, sym in ((256, 10, False), (100, 6, True)):
        A = rng.normal(size=(n, n))
        B = A if sym else rng.normal(size=(n, n))
        ref = kx.sim_debug_tc_gemm(A, B, terms=terms, sym=sym)
        dA = torch.from_numpy(A).to(dev)
        dB = torch.from_numpy(B).to(dev)
        dC = torch.full((n, n), np.nan, dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream().cuda_stream
        rc = kx.sim_tc_gemm_noalloc(n, dA.data_ptr(), dB.data_ptr(), terms, sym, dC.data_ptr(), stream)
        assert rc == kx.SIM_OK
        C = dC.cpu().numpy()
        scale = np.abs(A) @ np.abs(B).T
        assert np.max(np.abs(C - ref) / scale) < 2.0 ** -40
        if sym:
            assert np.array_equal(C, C.T)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    x = torch.zeros((257, 257), dtype=torch.float64, device=dev)
    assert kx.sim_tc_gemm_noalloc(257, x.data_ptr(), x.data_ptr(), 1, 0, x.data_ptr()) == kx.SIM_EINVAL
