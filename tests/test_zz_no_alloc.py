"""spirec_toeplitz_noalloc: the Toeplitz apply for callers that cannot
allocate device memory (a fixed memory budget, no footprint growth after
start-up).  Its scratch is a file-scope device array, so it needs no plan and
no cudaMalloc.  Checked through the C ABI against spirec_toeplitz_dev (the
plan-based entry point) on two calls in a row, with different inputs, so a
call that left stale state in the shared array would show.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_0908_3252_gb300 import synth
from tests.helpers import c64, empty_c64, from_dev, rel, to_dev, workload_c1, workload_ragged

pytestmark = pytest.mark.gpu

TOL = 1e-5  # the FP32 tolerance of the other parity tests


@pytest.fixture(scope="module")
def sp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0908_3252_gb300 import build, spirec
    build.build()
    spirec.load()
    return spirec


@pytest.mark.parametrize("wname,M", [("c1", 0), ("ragged", 75)])
def test_noalloc_matches_plan_toeplitz(sp, wname, M):
    import torch
    w = workload_c1() if wname == "c1" else workload_ragged()
    N = w["N"]
    stream = torch.cuda.current_stream().cuda_stream
    with sp.Plan(N, w["kx"].shape[0], M, 0, stream, w["kx"], w["ky"]) as p:
        Mp = p.M
        spec = torch.zeros((Mp, Mp), dtype=torch.float32, device="cuda:0")
        sp.spirec_kernel_spectrum_dev(p.h, spec)
        g = synth.rng(31)
        for call in range(2):
            x = to_dev(c64(synth.complex_normal((N, N), g)))
            want = empty_c64((N, N))
            sp.spirec_toeplitz_dev(p.h, x, want)
            got = empty_c64((N, N))
            sp.spirec_toeplitz_noalloc(x, spec, got, N, Mp, stream)
            assert rel(from_dev(got), from_dev(want)) < TOL, f"call {call}"


def test_noalloc_rejects_sizes_beyond_its_array(sp):
    import torch
    N, M = 600, 1200
    x = torch.zeros((8,), dtype=torch.complex64, device="cuda:0")
    spec = torch.zeros((8,), dtype=torch.float32, device="cuda:0")
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_toeplitz_noalloc(x, spec, x, N, M)
    assert e.value.code == sp.SPIREC_EINVAL
    assert "512" in str(e.value)
    with pytest.raises(sp.SpirecError) as e:
        sp.spirec_toeplitz_noalloc(x, spec, x, 32, 40)  # M < 2N - 1
    assert e.value.code == sp.SPIREC_EINVAL
