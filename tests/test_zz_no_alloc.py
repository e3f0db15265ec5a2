"""The no-allocation merge-path product, spmv_csr_merge_noalloc.

Some callers cannot let a library allocate device memory during a call:
code running inside a host application that owns every device allocation
through its own fixed pool, latency-bound loops where an allocation may
synchronise or grow a pool at an unpredictable moment, and work recorded into
a CUDA graph whose owner does not accept memory-allocation nodes.  For them
the library keeps the merge-path scratch in a fixed device array.  These
tests call that entry point through the C ABI twice in a row, with inputs of
different sizes so the second call runs over leftovers of the first, and
check each result against the allocating entry point spmv_csr_merge: equal
bit for bit (the same tiling and kernels), hence within the FP64 tolerance
the other parity tests use.  They also check that the calls take no memory:
neither from the device's stream-ordered pool (where cudaMallocAsync takes
it), nor from PyTorch's allocator, nor from the device's free memory.  This
file is collected last.
"""
import ctypes
import glob

import numpy as np
import pytest

import oracle
from paper_2203_02530_gb300 import workloads as W
from tests.gpu_util import assert_fp64_close, dev, synced, torch_cuda

pytestmark = pytest.mark.gpu

_USED_MEM_HIGH = 8   # cudaMemPoolAttrUsedMemHigh


def _device_csr(torch, n, rp, ci, va, x):
    return (dev(rp.astype(np.int32)), dev(ci), dev(va), dev(x),
            synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")))


def _cudart():
    names = ["libcudart.so.13", "libcudart.so"] + sorted(glob.glob("/usr/local/cuda/lib64/libcudart.so*"))
    for name in names:
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


class _PoolWatch:
    """High-water mark of the memory in use in the current device's default
    memory pool, the pool cudaMallocAsync draws from; reset() clears it."""

    def __init__(self, torch):
        self.rt = _cudart()
        self.pool = ctypes.c_void_p()
        if self.rt is not None:
            rc = self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool),
                                                     ctypes.c_int(torch.cuda.current_device()))
            if rc != 0:
                self.rt = None

    def reset(self):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0

    def high(self):
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


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
        y_new = synced(torch.full((n,), float("nan"), dtype=torch.float64, device="cuda"))
        nnz = int(rp[-1])
        spmv.spmv_csr_merge(n, nnz, rp_d, ci_d, va_d, x_d, y_ref, s)
        spmv.spmv_csr_merge_noalloc(n, nnz, rp_d, ci_d, va_d, x_d, y_new, s)
        s.synchronize()
        got, want = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert_fp64_close(got, want, scale, "no-alloc n=%d" % n)
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), "no-alloc n=%d: not bit-identical" % n
    assert spmv.spmv_csr_error() == 0


def test_no_alloc_calls_take_no_memory():
    """Two calls after the set-up call take nothing from the device's default
    memory pool, from PyTorch's allocator or from the free device memory,
    while one call of the allocating entry point does show up in the pool
    (so the check can see an allocation)."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    s = torch.cuda.Stream()
    n, rp, ci, va = W.powerlaw(200_000, seed=16)
    x = W.uniform_x(n, seed=17)
    rp_d, ci_d, va_d, x_d, y_a = _device_csr(torch, n, rp, ci, va, x)
    y_b = torch.empty_like(y_a)
    nnz = int(rp[-1])
    spmv.spmv_csr_merge_noalloc(n, nnz, rp_d, ci_d, va_d, x_d, y_a, s)   # set-up call
    s.synchronize()
    watch = _PoolWatch(torch)
    if watch.rt is None:
        pytest.skip("the CUDA runtime library cannot be loaded to read the pool")
    torch.cuda.synchronize()
    stats0 = torch.cuda.memory_stats()
    free0 = torch.cuda.mem_get_info()[0]
    watch.reset()
    spmv.spmv_csr_merge_noalloc(n, nnz, rp_d, ci_d, va_d, x_d, y_a, s)
    spmv.spmv_csr_merge_noalloc(n, nnz, rp_d, ci_d, va_d, x_d, y_b, s)
    s.synchronize()
    assert watch.high() == 0, "the no-allocation calls drew on the stream-ordered pool"
    stats1 = torch.cuda.memory_stats()
    for key in ("allocation.all.allocated", "segment.all.allocated"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    assert torch.cuda.mem_get_info()[0] >= free0
    assert torch.equal(y_a, y_b)
    watch.reset()
    spmv.spmv_csr_merge(n, nnz, rp_d, ci_d, va_d, x_d, y_b, s)
    s.synchronize()
    assert watch.high() > 0, "the pool watch does not see cudaMallocAsync"
    assert torch.equal(y_a, y_b)
    assert spmv.spmv_csr_error() == 0


def test_no_alloc_rejects_inputs_beyond_its_scratch():
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    with pytest.raises(spmv.SpmvError) as e:
        spmv.spmv_csr_merge_noalloc(100_000_000, 100_000_000, 0, 0, 0, 0, 0, None)
    assert e.value.code == spmv.EBOUNDS
