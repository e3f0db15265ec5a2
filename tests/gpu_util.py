"""Helpers for the GPU parity tests: device tensors, the FP64 tolerance and
oracle references."""
import numpy as np

import oracle


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a):
    torch = torch_cuda()
    return torch.as_tensor(np.ascontiguousarray(a)).cuda()


def synced(t):
    """`t` once the current stream's work on it is done: tensors made by
    PyTorch kernels come from its current stream, while the library runs on
    streams that do not wait for it."""
    torch_cuda().cuda.synchronize()
    return t


def refill(t, value=float("nan")):
    """Fill a device tensor and wait for the fill (see synced)."""
    t.fill_(value)
    return synced(t)


def assert_fp64_close(got, want, scale, what=""):
    """|got - want| <= 1e-12 * sum_j |a_ij x_j| per element (plus 1e-300).

    Two FP64 evaluations of a dot product of length k in different orders
    differ by at most 2 * gamma_k * sum |a_ij x_j| with gamma_k = k u / (1 - k u),
    u = 2^-53; for rows up to 4096 entries this is below 9.1e-13, so the
    bound 1e-12 holds for every correct kernel (one more rounding for the
    local + remote split stays inside it)."""
    got = np.asarray(got)
    want = np.asarray(want)
    err = np.abs(got - want)
    lim = 1e-12 * np.asarray(scale) + 1e-300
    bad = np.nonzero(~(err <= lim))[0]
    if bad.size:
        i = bad[0]
        raise AssertionError("%s: %d elements out of tolerance; first at %d: got %r want %r "
                             "(|diff| %.3e > %.3e)" % (what, bad.size, i, got[i], want[i], err[i], lim[i]))


def reference(n, rp, ci, va, x):
    """Oracle product and its error scale."""
    return oracle.csr_spmv(n, rp, ci, va, x), oracle.csr_absdot(n, rp, ci, va, x)
