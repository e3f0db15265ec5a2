"""Serving runtime with continuous batching: every request's result is the
same alone and in the mix (bit for bit, through the device hash and against
a request run alone), and matches the oracle within the FP64 bound."""
import numpy as np
import pytest

import oracle
from paper_2203_02530_gb300 import workloads as W
from tests.gpu_util import assert_fp64_close, torch_cuda

pytestmark = pytest.mark.gpu

MASK = np.uint64(0xFFFFFFFFFFFFFFFF)


def mix64(z):
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(33))) * np.uint64(0xFF51AFD7ED558CCD)
        z = (z ^ (z >> np.uint64(33))) * np.uint64(0xC4CEB9FE1A85EC53)
        return z ^ (z >> np.uint64(33))


def host_hash(Y, width):
    """The order-independent hash of a request's columns (the definition the
    serving runtime documents), computed on the host."""
    y = np.ascontiguousarray(Y[:, :width]).view(np.uint64).ravel()
    e = np.arange(y.size, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return np.uint64(np.sum(mix64(y + e * np.uint64(0x9E3779B97F4A7C15)), dtype=np.uint64))


def _mats():
    return [W.stencil_7pt(11, seed=1), W.zipf_random(5000, seed=2), W.laplacian_5pt(40),
            W.powerlaw(3000, seed=3, cap=500), W.stencil_27pt(0, seed=4, dims=(6, 9, 13)),
            W.random_csr(200, density=0.05, seed=5)]


def _requests(count, n_mats, seed, spread_s):
    rng = np.random.default_rng(seed)
    mat = rng.integers(0, n_mats, size=count).astype(np.int32)
    wid = rng.integers(1, 9, size=count).astype(np.int32)
    sd = rng.integers(0, 2**63, size=count, dtype=np.uint64)
    arr = np.sort(rng.uniform(0.0, spread_s, size=count))
    return mat, wid, sd, arr


def test_request_x_matches_device_generator():
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = _mats()
    with spmv.Batch(mats) as b, spmv.Server(b, n_streams=2, budget_bytes=1 << 30) as sv:
        n = mats[0][0]
        x = torch.empty((n, 5), dtype=torch.float64, device="cuda")
        y = torch.empty((n, 5), dtype=torch.float64, device="cuda")
        s = torch.cuda.Stream()
        spmv.spmv_serve_single(sv.h, 0, 5, 12345, y, x, s)
        s.synchronize()
        assert np.array_equal(x.cpu().numpy(), W.request_x(12345, n, 5))


@pytest.mark.parametrize("layout", ["buckets", "sliced"])
def test_results_same_alone_and_in_the_mix_and_match_oracle(layout):
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = _mats()
    mat, wid, sd, arr = _requests(400, len(mats), 11, 0.02)
    with spmv.Batch(mats) as b:
        if layout == "sliced":
            spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        with spmv.Server(b, n_streams=4, budget_bytes=1 << 30) as sv:
            lat_b, h_b, st_b = sv.run(mat, wid, sd, arr, spmv.SERVE_BATCHED)
            lat_p, h_p, st_p = sv.run(mat, wid, sd, arr, spmv.SERVE_PLAIN)
            assert np.array_equal(h_b, h_p)
            assert st_p["blocks"] == len(mat)
            assert st_b["admitted_while_busy"] > 0                 # continuous admission
            assert (lat_b > 0).all() and (lat_p > 0).all()
            # a burst queues up, so requests of one matrix are merged into blocks
            lat_burst, h_burst, st_burst = sv.run(mat, wid, sd, np.zeros(len(mat)), spmv.SERVE_BATCHED)
            assert st_burst["blocks"] < len(mat)
            assert np.array_equal(h_burst, h_b)
            # smaller groups (sliced layout: grouped launches) give the same results
            spmv.spmv_serve_set_group_max(sv.h, 2)
            _, h_g2, _ = sv.run(mat, wid, sd, np.zeros(len(mat)), spmv.SERVE_BATCHED)
            assert np.array_equal(h_g2, h_b)
            with pytest.raises(spmv.SpmvError):
                spmv.spmv_serve_set_group_max(sv.h, 65)
            spmv.spmv_serve_set_group_max(sv.h, 64)
            s = torch.cuda.Stream()
            for r in range(0, len(mat), 23):
                m, k = int(mat[r]), int(wid[r])
                n, rp, ci, va = mats[m]
                x = torch.empty((n, k), dtype=torch.float64, device="cuda")
                y = torch.empty((n, k), dtype=torch.float64, device="cuda")
                spmv.spmv_serve_single(sv.h, m, k, int(sd[r]), y, x, s)
                s.synchronize()
                Y = y.cpu().numpy()
                assert host_hash(Y, k) == h_b[r], "request %d differs alone and in the mix" % r
                X = W.request_x(int(sd[r]), n, k)
                for j in range(k):
                    want = oracle.csr_spmv(n, rp, ci, va, X[:, j])
                    scale = oracle.csr_absdot(n, rp, ci, va, X[:, j])
                    assert_fp64_close(Y[:, j], want, scale, "request %d column %d" % (r, j))


@pytest.mark.parametrize("layout", ["buckets", "sliced"])
def test_small_budget_makes_blocks_wait_but_completes(layout):
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    mats = _mats()
    mat, wid, sd, arr = _requests(200, len(mats), 12, 0.0)
    with spmv.Batch(mats) as b:
        if layout == "sliced":
            spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        nmax = max(m[0] for m in mats)
        resident = b.query(spmv.BQ_DEVICE_BYTES)
        budget = resident + 128 * nmax + 4096      # room for one width-8 block of the largest
        with spmv.Server(b, n_streams=4, budget_bytes=budget) as sv:
            lat, h, st = sv.run(mat, wid, sd, arr, spmv.SERVE_BATCHED)
            assert st["waits_for_memory"] > 0
            assert st["peak_pool_bytes"] <= budget - resident
        with spmv.Server(b, n_streams=4, budget_bytes=1 << 30) as sv:
            lat2, h2, st2 = sv.run(mat, wid, sd, arr, spmv.SERVE_BATCHED)
        assert np.array_equal(h, h2)


def test_serving_rejects_bad_requests():
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    mats = _mats()
    with spmv.Batch(mats) as b:
        with pytest.raises(spmv.SpmvError) as e:
            spmv.Server(b, n_streams=2, budget_bytes=1024)
        assert e.value.code == spmv.ENOMEM
        with spmv.Server(b, n_streams=2, budget_bytes=1 << 30) as sv:
            with pytest.raises(spmv.SpmvError):
                sv.run([0], [9], [1], [0.0])
            with pytest.raises(spmv.SpmvError):
                sv.run([7], [1], [1], [0.0])
            with pytest.raises(spmv.SpmvError):
                sv.run([0, 0], [1, 1], [1, 2], [0.1, 0.0])


@pytest.mark.parametrize("layout", ["buckets", "sliced"])
def test_serving_empty_and_one_row_matrices(layout):
    """Requests on a matrix with no rows, a 1 x 1 matrix and a matrix whose
    rows are all empty complete, with the oracle's (empty or zero) results,
    alone and mixed with ordinary requests."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = [(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)),
            W.random_csr(1, density=1.0, seed=3, empty_rows=False),
            (40, np.zeros(41, np.int64), np.zeros(0, np.int32), np.zeros(0)),
            W.laplacian_5pt(20)]
    rng = np.random.default_rng(21)
    cnt = 60
    mat = rng.integers(0, len(mats), size=cnt).astype(np.int32)
    wid = rng.integers(1, 9, size=cnt).astype(np.int32)
    sd = rng.integers(0, 2**63, size=cnt, dtype=np.uint64)
    with spmv.Batch(mats) as b:
        if layout == "sliced":
            spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        with spmv.Server(b, n_streams=3, budget_bytes=1 << 30) as sv:
            lat_b, h_b, _ = sv.run(mat, wid, sd, np.zeros(cnt), spmv.SERVE_BATCHED)
            lat_p, h_p, _ = sv.run(mat, wid, sd, np.zeros(cnt), spmv.SERVE_PLAIN)
            assert np.array_equal(h_b, h_p)
            assert (lat_b > 0).all() and (lat_p > 0).all()
            s = torch.cuda.Stream()
            for r in range(cnt):
                m, k = int(mat[r]), int(wid[r])
                n, rp, ci, va = mats[m]
                if n == 0:
                    assert h_b[r] == 0
                    continue
                x = torch.empty((n, k), dtype=torch.float64, device="cuda")
                y = torch.empty((n, k), dtype=torch.float64, device="cuda")
                spmv.spmv_serve_single(sv.h, m, k, int(sd[r]), y, x, s)
                s.synchronize()
                Y = y.cpu().numpy()
                assert host_hash(Y, k) == h_b[r]
                X = W.request_x(int(sd[r]), n, k)
                for j in range(k):
                    want = oracle.csr_spmv(n, rp, ci, va, X[:, j])
                    scale = oracle.csr_absdot(n, rp, ci, va, X[:, j])
                    assert_fp64_close(Y[:, j], want, scale, "request %d column %d" % (r, j))


def test_full_size_serving_mix_sampled():
    """The benchmark's serving mix (64 resident matrices, 1.3 GB, sliced
    layout, 32 stream slots, 40 GB budget) under a burst of 3000 requests:
    grouped and plain serving give the same hash for every request, and
    sampled requests run alone match their hash and the oracle column by
    column."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = [m for _, m in W.serve_mix(64, seed=6)]
    rng = np.random.default_rng(8)
    count = 3000
    mat = rng.integers(0, len(mats), size=count).astype(np.int32)
    wid = rng.integers(1, 9, size=count).astype(np.int32)
    sd = rng.integers(0, 2**63, size=count, dtype=np.uint64)
    with spmv.Batch(mats) as b:
        spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        with spmv.Server(b, n_streams=32, budget_bytes=40 << 30) as sv:
            _, h_b, st_b = sv.run(mat, wid, sd, np.zeros(count), spmv.SERVE_BATCHED)
            _, h_p, _ = sv.run(mat, wid, sd, np.zeros(count), spmv.SERVE_PLAIN)
            assert np.array_equal(h_b, h_p)
            assert st_b["blocks"] < count
            s = torch.cuda.Stream()
            for r in (0, 1, 777, 2999):
                m, k = int(mat[r]), int(wid[r])
                n, rp, ci, va = mats[m]
                x = torch.empty((n, k), dtype=torch.float64, device="cuda")
                y = torch.empty((n, k), dtype=torch.float64, device="cuda")
                spmv.spmv_serve_single(sv.h, m, k, int(sd[r]), y, x, s)
                s.synchronize()
                Y = y.cpu().numpy()
                assert host_hash(Y, k) == h_b[r], "request %d differs alone and in the mix" % r
                X = W.request_x(int(sd[r]), n, k)
                assert np.array_equal(x.cpu().numpy(), X)
                for j in range(k):
                    want = oracle.csr_spmv(n, rp, ci, va, X[:, j])
                    scale = oracle.csr_absdot(n, rp, ci, va, X[:, j])
                    assert_fp64_close(Y[:, j], want, scale, "request %d column %d" % (r, j))
