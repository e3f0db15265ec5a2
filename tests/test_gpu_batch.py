"""Batched products (many independent CSR matrices in one persistent
launch) against the oracle and against one launch per matrix."""
import numpy as np
import pytest

import oracle
from paper_2203_02530_gb300 import workloads as W
from tests.gpu_util import assert_fp64_close, dev, refill, synced, torch_cuda

pytestmark = pytest.mark.gpu


def _mix():
    mats = [W.laplacian_5pt(17), W.stencil_7pt(9, seed=1), W.powerlaw(5000, seed=2, cap=2000),
            W.random_csr(1, density=1.0, seed=3, empty_rows=False),
            (0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0)),
            W.random_csr(300, density=0.05, seed=4, duplicates=True, shuffle_cols=True),
            (50, np.zeros(51, np.int64), np.zeros(0, np.int32), np.zeros(0)),
            W.stencil_27pt(0, seed=5, dims=(5, 7, 11)), W.zipf_random(3000, seed=6)]
    return mats


def _oracle(mats, x, offs):
    want, scale = np.zeros(offs[-1]), np.zeros(offs[-1])
    for m, (n, rp, ci, va) in enumerate(mats):
        xs = x[offs[m]:offs[m] + n]
        want[offs[m]:offs[m] + n] = oracle.csr_spmv(n, rp, ci, va, xs)
        scale[offs[m]:offs[m] + n] = oracle.csr_absdot(n, rp, ci, va, xs)
    return want, scale


@pytest.mark.parametrize("lanes", [0, 1, 2, 4, 8, 16, 32, 64, "mixed"])
def test_batch_matches_oracle_and_separate_launches(lanes):
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = _mix()
    with spmv.Batch(mats) as b:
        offs = b.offsets()
        assert offs[-1] == sum(m[0] for m in mats)
        if lanes == "mixed":
            for m in range(b.count):
                spmv.spmv_batch_set_lanes(b.h, m, [0, 1, 2, 4, 8, 16, 32, 64][m % 8])
        else:
            spmv.spmv_batch_set_lanes(b.h, -1, lanes)
        x = W.uniform_x(offs[-1], seed=9)
        want, scale = _oracle(mats, x, offs)
        s = torch.cuda.Stream()
        x_d = dev(x)
        y1 = synced(torch.full((offs[-1],), float("nan"), dtype=torch.float64, device="cuda"))
        y2 = synced(torch.full((offs[-1],), float("nan"), dtype=torch.float64, device="cuda"))
        spmv.spmv_batch_run(b.h, x_d, y1, s)
        spmv.spmv_batch_run_separate(b.h, -1, x_d, y2, s)
        s.synchronize()
        a1, a2 = y1.cpu().numpy(), y2.cpu().numpy()
        assert np.array_equal(a1, a2), "batched and separate launches differ"
        assert_fp64_close(a1, want, scale, "batch lanes=%s" % lanes)
        spmv.spmv_batch_run(b.h, x_d, y1, s)   # ticket reset between launches
        s.synchronize()
        assert np.array_equal(y1.cpu().numpy(), a1)


def test_batch_rejects_bad_arguments():
    from paper_2203_02530_gb300 import spmv
    torch_cuda()
    with spmv.Batch(_mix()[:3]) as b:
        with pytest.raises(spmv.SpmvError):
            spmv.spmv_batch_set_lanes(b.h, 0, 3)
        with pytest.raises(spmv.SpmvError):
            spmv.spmv_batch_set_lanes(b.h, 7, 2)
        with pytest.raises(spmv.SpmvError):
            spmv.spmv_batch_query(b.h, spmv.BQ_N, 5)
    with pytest.raises(spmv.SpmvError):
        spmv.Batch([(2, np.array([0, 1, 2]), np.array([0, 9], np.int32), np.ones(2))])


def test_batch_autotune_keeps_results():
    from paper_2203_02530_gb300 import autotune, spmv
    torch = torch_cuda()
    mats = _mix()
    with spmv.Batch(mats) as b:
        offs = b.offsets()
        x = W.uniform_x(offs[-1], seed=10)
        want, scale = _oracle(mats, x, offs)
        s = torch.cuda.Stream()
        x_d = dev(x)
        y = torch.empty(offs[-1], dtype=torch.float64, device="cuda")
        chosen = autotune.tune_batch(b, x_d, y, s)
        assert len(chosen) == len(mats)
        assert [b.query(spmv.BQ_LANES, m) for m in range(b.count)] == chosen
        spmv.spmv_batch_run(b.h, x_d, y, s)
        s.synchronize()
        assert_fp64_close(y.cpu().numpy(), want, scale, "tuned batch")


def test_sliced_mode_round_trip_and_long_rows():
    """The sliced layout (natural order for stencils, length-sorted with
    whole-warp long rows for skewed matrices) gives the oracle's y; switching
    modes back and forth keeps every mode's result."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = [W.stencil_7pt(12, seed=1), W.zipf_random(20000, seed=2), W.laplacian_5pt(33),
            W.powerlaw(6000, seed=3, cap=3000), W.random_csr(50000, density=0.0001, seed=4)]
    with spmv.Batch(mats) as b:
        offs = b.offsets()
        x = W.uniform_x(offs[-1], seed=12)
        want, scale = _oracle(mats, x, offs)
        s = torch.cuda.Stream()
        x_d = dev(x)
        y = torch.empty(offs[-1], dtype=torch.float64, device="cuda")
        res = {}
        for lanes in (spmv.BATCH_SLICED, 1, spmv.BATCH_SLICED, 0):
            spmv.spmv_batch_set_lanes(b.h, -1, lanes)
            assert b.query(spmv.BQ_LANES, 1) == lanes
            spmv.spmv_batch_run(b.h, x_d, y, s)
            s.synchronize()
            a = y.cpu().numpy()
            assert_fp64_close(a, want, scale, "lanes %d" % lanes)
            if lanes in res:
                assert np.array_equal(a, res[lanes])
            res[lanes] = a


@pytest.mark.parametrize("chunks", [1, 3, 64])
def test_batch_run_host_matches_device_run(chunks):
    """Chunked host-buffer runs (x in, products, y out overlapped) give the
    device run's y bit for bit, in both layouts."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = _mix()
    with spmv.Batch(mats) as b:
        offs = b.offsets()
        x = W.uniform_x(offs[-1], seed=13)
        s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        x_d = dev(x)
        y_d = torch.empty(offs[-1], dtype=torch.float64, device="cuda")
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.full((offs[-1],), float("nan"), dtype=torch.float64).pin_memory()
        for lanes in (2, spmv.BATCH_SLICED):
            spmv.spmv_batch_set_lanes(b.h, -1, lanes)
            spmv.spmv_batch_run(b.h, x_d, y_d, s_c)
            s_c.synchronize()
            spmv.spmv_batch_run_host(b.h, xh, yh, chunks, s_in, s_c, s_out)
            a, h = y_d.cpu().numpy(), yh.numpy()
            assert np.array_equal(a.view(np.uint64), h.view(np.uint64)), lanes
        with pytest.raises(spmv.SpmvError):
            spmv.spmv_batch_run_host(b.h, xh, yh, chunks, s_c, s_c, s_out)
        with pytest.raises(spmv.SpmvError):
            spmv.spmv_batch_run_host(b.h, xh, yh, 0, s_in, s_c, s_out)


@pytest.mark.parametrize("chunks", [1, 5])
def test_batch_run_host_many_matches_single_runs(chunks):
    """A stream of batched products through host buffers, consecutive ones
    overlapped on two pairs of device vectors: each y_k equals the chunked
    host-buffer run of x_k bit for bit, with distinct and with shared host
    vectors, in both layouts."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = _mix()
    count = 4
    with spmv.Batch(mats) as b:
        tot = b.offsets()[-1]
        rng = np.random.default_rng(17)
        xh = torch.from_numpy(rng.uniform(-1, 1, (count, tot))).pin_memory()
        s_in, s_c, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        y1 = torch.empty(tot, dtype=torch.float64).pin_memory()
        for lanes in (2, spmv.BATCH_SLICED):
            spmv.spmv_batch_set_lanes(b.h, -1, lanes)
            want = []
            for k in range(count):
                spmv.spmv_batch_run_host(b.h, xh[k], y1, chunks, s_in, s_c, s_out)
                want.append(y1.numpy().copy())
            for _ in range(2):
                yh = torch.full((count, tot), float("nan"), dtype=torch.float64).pin_memory()
                spmv.spmv_batch_run_host_many(b.h, count, xh, tot, yh, tot, chunks, s_in, s_c, s_out)
                for k in range(count):
                    assert np.array_equal(yh[k].numpy().view(np.uint64), want[k].view(np.uint64)), (lanes, k)
            ys = torch.full((tot,), float("nan"), dtype=torch.float64).pin_memory()
            spmv.spmv_batch_run_host_many(b.h, count, xh[1], 0, ys, 0, chunks, s_in, s_c, s_out)
            assert np.array_equal(ys.numpy().view(np.uint64), want[1].view(np.uint64))
        spmv.spmv_batch_run_host_many(b.h, 0, None, 0, None, 0, chunks, s_in, s_c, s_out)
        for args in [(-1, tot, tot, chunks, s_in), (2, tot, 1, chunks, s_in), (2, tot, tot, 0, s_in),
                     (2, tot, tot, chunks, s_c)]:
            with pytest.raises(spmv.SpmvError) as e:
                spmv.spmv_batch_run_host_many(b.h, args[0], xh, args[1], yh, args[2], args[3], args[4], s_c, s_out)
            assert e.value.code == spmv.EINVAL


def test_full_size_batch_mix_256_sliced():
    """The benchmark's batch (256 matrices, n log-uniform in [1e3, 1e6],
    5-point / 7-point / Zipf rows, 4.19 GB) in the sliced layout the tuner
    picks: the persistent launch gives the oracle's y in full, bit-identical
    to one launch per matrix and to the chunked host-buffer path, twice."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = [m for _, m in W.batch_mix(256, seed=5)]
    with spmv.Batch(mats) as b:
        offs = b.offsets()
        spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        x = W.uniform_x(offs[-1], seed=6)
        want, scale = _oracle(mats, x, offs)
        del mats
        s, s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        x_d = dev(x)
        y1 = synced(torch.full((offs[-1],), float("nan"), dtype=torch.float64, device="cuda"))
        y2 = synced(torch.full((offs[-1],), float("nan"), dtype=torch.float64, device="cuda"))
        spmv.spmv_batch_run(b.h, x_d, y1, s)
        spmv.spmv_batch_run_separate(b.h, -1, x_d, y2, s)
        s.synchronize()
        a1 = y1.cpu().numpy()
        assert np.array_equal(a1, y2.cpu().numpy()), "batched and separate launches differ"
        assert_fp64_close(a1, want, scale, "batch mix 256 sliced")
        refill(y1)
        spmv.spmv_batch_run(b.h, x_d, y1, s)
        s.synchronize()
        assert np.array_equal(y1.cpu().numpy(), a1)
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.full((offs[-1],), float("nan"), dtype=torch.float64).pin_memory()
        spmv.spmv_batch_run_host(b.h, xh, yh, 16, s_in, s, s_out)
        assert np.array_equal(yh.numpy(), a1)


def test_batch_release_csr_keeps_y_and_restores():
    """spmv_batch_release_csr keeps only the rows longer than 64 of the CSR
    once every matrix is sliced: less device memory; the batched, per-matrix
    and host-buffer products and a served request give the same results bit
    for bit; a CSR layout afterwards rebuilds the full CSR (results within the
    oracle's bound); back in the sliced layout the results match again; and
    the release is refused while a matrix is not sliced."""
    from paper_2203_02530_gb300 import spmv
    torch = torch_cuda()
    mats = _mix()
    with spmv.Batch(mats) as b:
        offs = b.offsets()
        spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        spmv.spmv_batch_set_lanes(b.h, 0, 2)
        with pytest.raises(spmv.SpmvError) as e:
            spmv.spmv_batch_release_csr(b.h)
        assert e.value.code == spmv.EINVAL
        spmv.spmv_batch_set_lanes(b.h, 0, spmv.BATCH_SLICED)
        x = W.uniform_x(offs[-1], seed=19)
        want, scale = _oracle(mats, x, offs)
        s, s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        x_d = dev(x)
        y = synced(torch.full((offs[-1],), float("nan"), dtype=torch.float64, device="cuda"))
        xh = torch.from_numpy(x).pin_memory()
        yh = torch.empty(offs[-1], dtype=torch.float64).pin_memory()
        sv = spmv.Server(b, n_streams=2, budget_bytes=1 << 30)
        big = max(range(b.count), key=lambda m: mats[m][0])
        n_big = mats[big][0]
        yq = synced(torch.zeros(n_big * 3, dtype=torch.float64, device="cuda"))
        xq = synced(torch.zeros(n_big * 3, dtype=torch.float64, device="cuda"))

        def results():
            out = []
            refill(y)
            spmv.spmv_batch_run(b.h, x_d, y, s)
            s.synchronize()
            out.append(y.cpu().numpy().copy())
            refill(y)
            spmv.spmv_batch_run_separate(b.h, -1, x_d, y, s)
            s.synchronize()
            out.append(y.cpu().numpy().copy())
            yh.fill_(float("nan"))
            spmv.spmv_batch_run_host(b.h, xh, yh, 3, s_in, s, s_out)
            out.append(yh.numpy().copy())
            spmv.spmv_serve_single(sv.h, big, 3, 12345, yq, xq, s)
            s.synchronize()
            out.append(yq.cpu().numpy().copy())
            return out

        before = results()
        assert_fp64_close(before[0], want, scale, "sliced batch")
        bytes0 = b.query(spmv.BQ_DEVICE_BYTES)
        spmv.spmv_batch_release_csr(b.h)
        assert b.query(spmv.BQ_DEVICE_BYTES) < bytes0
        for a, c in zip(before, results()):
            assert np.array_equal(a.view(np.uint64), c.view(np.uint64))
        spmv.spmv_batch_set_lanes(b.h, -1, 2)      # a CSR layout: the full CSR is rebuilt
        refill(y)
        spmv.spmv_batch_run(b.h, x_d, y, s)
        s.synchronize()
        assert_fp64_close(y.cpu().numpy(), want, scale, "CSR layout after the rebuild")
        spmv.spmv_batch_set_lanes(b.h, -1, spmv.BATCH_SLICED)
        assert np.array_equal(results()[0].view(np.uint64), before[0].view(np.uint64))
        spmv.spmv_batch_release_csr(b.h)
        assert np.array_equal(results()[0].view(np.uint64), before[0].view(np.uint64))
        sv.close()
