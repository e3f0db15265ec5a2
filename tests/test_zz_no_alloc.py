"""The no-allocation merge-path product, spmv_csr_merge_noalloc.

Some callers cannot let a library allocate device memory during a call:
code running inside a host application that owns every device allocation
through its own fixed pool, latency-bound loops where an allocation may
synchronise or grow a pool at an unpredictable moment, and work recorded into
a CUDA graph whose owner does not accept memory-allocation nodes.  For them
the library keeps the merge-path scratch in a fixed device array.  These
tests call that entry point through the C ABI twice in a row, with inputs of
different sizes so the second call runs over leftovers of the first, and
check each result against the allocating entry point spmv_csr_merge within
the FP64 tolerance the other parity tests use.  This file is collected last.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02530_gb300 import workloads as W
from tests.gpu_util import assert_fp64_close, dev, torch_cuda

pytestmark = pytest.mark.gpu


def _device_csr(torch, n, rp, ci, va, x):
    return (dev(rp.astype(np.int32)), dev(ci), dev(va), dev(x),
            torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))


def test_no_alloc_matches_allocating_entry_point_on_two_calls():
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    s = torch.cuda.Stream()
    inputs = [W.powerlaw(300_000, seed=13),          # skewed rows, many tiles
              W.stencil_27pt(0, seed=14, dims=(9, 17, 23))]   # fewer tiles
    for n, rp, ci, va in inputs:
        x = W.uniform_x(n, seed=15)
        scale = oracle.csr_absdot(n, rp, ci, va, x)
        rp_d, ci_d, va_d, x_d, y_ref = _device_csr(torch, n, rp, ci, va, x)
        y_new = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        nnz = int(rp[-1])
        spmv.spmv_csr_merge(n, nnz, rp_d, ci_d, va_d, x_d, y_ref, s)
        spmv.spmv_csr_merge_noalloc(n, nnz, rp_d, ci_d, va_d, x_d, y_new, s)
        s.synchronize()
        assert_fp64_close(y_new.cpu().numpy(), y_ref.cpu().numpy(), scale, "no-alloc n=%d" % n)
    assert spmv.spmv_csr_error() == 0


def test_no_alloc_rejects_inputs_beyond_its_scratch():
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_csr_merge_noalloc(100_000_000, 100_000_000, 0, 0, 0, 0, 0, None)
    assert e.value.code == spmv.EBOUNDS
