"""Seeded synthetic inputs: CSR matrices and x vectors.

This module builds inputs only; it holds none of the SpMV arithmetic, so both
the CUDA path and the CPU oracle may draw from it.  Every generator takes a
seed (numpy ``default_rng``) and returns plain numpy arrays:
``(n, row_ptr int64[n+1], col_idx int32[nnz], vals float64[nnz])``.

Workloads (sizes as named):
  * ``laplacian_5pt(64)``: 2-D 5-point Laplacian on a 64 x 64 grid, 4 on the
    diagonal and -1 off it (n = 4096, nnz = 20224).
  * ``stencil_27pt(150, seed)``: 3-D 27-point stencil on 150^3 (n = 3 375 000,
    nnz = 448^3), values U[-1, 1] with the diagonal set to 27.
  * ``powerlaw(4_000_000, seed)``: random rows with Zipf(2) lengths (capped),
    80 % of columns within +-n/8 of the row, 20 % uniform.
  * ``band(150_000, 1_500_000, 37_500, seed)``: the paper's band matrix
    (Sec. III): nonzeros uniformly random within a band.
  * ``stencil_7pt``, ``zipf_random``: members of the batched mix.
"""
import numpy as np

__all__ = ["laplacian_5pt", "stencil_7pt", "stencil_27pt", "powerlaw",
           "zipf_random", "band", "random_csr", "uniform_x", "batch_mix",
           "csr_nbytes"]


def _stencil(dims, offsets, diag_value, offdiag, rng):
    """CSR of a stencil on a grid with row-major (last dim fastest) numbering.

    ``offsets`` are given in lexicographic order, which makes the columns of
    every row ascending.  ``offdiag``: a constant, or None for U[-1, 1].
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    nd = len(dims)
    coords = np.indices(dims, dtype=np.int32).reshape(nd, n)
    strides = [int(np.prod(dims[i + 1:])) for i in range(nd)]
    m = len(offsets)
    valid = np.ones((n, m), dtype=bool)
    colmat = np.empty((n, m), dtype=np.int32)
    rows = np.arange(n, dtype=np.int64)
    for j, off in enumerate(offsets):
        c = rows.copy()
        for d in range(nd):
            if off[d]:
                v = coords[d] + off[d]
                valid[:, j] &= (v >= 0) & (v < dims[d])
                c += off[d] * strides[d]
        colmat[:, j] = np.where(valid[:, j], c, 0).astype(np.int32)
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = colmat[valid]
    del colmat
    nnz = int(row_ptr[-1])
    if offdiag is None:
        vals = rng.uniform(-1.0, 1.0, size=nnz)
    else:
        vals = np.full(nnz, float(offdiag))
    center = offsets.index(tuple([0] * nd))
    before = valid[:, :center].sum(axis=1)
    vals[row_ptr[:-1] + before] = diag_value
    return n, row_ptr, col_idx, vals


def _offsets(nd, kind):
    import itertools
    if kind == "box":   # 3^nd box: 9-point in 2-D, 27-point in 3-D
        return [tuple(o) for o in itertools.product((-1, 0, 1), repeat=nd)]
    # star: the 2*nd+1-point stencil, in lexicographic order
    offs = [tuple([0] * nd)]
    for d in range(nd):
        for s in (-1, 1):
            o = [0] * nd
            o[d] = s
            offs.append(tuple(o))
    return sorted(offs)


def laplacian_5pt(g=64):
    """2-D 5-point Laplacian on a g x g grid: 4 on the diagonal, -1 off."""
    return _stencil((g, g), _offsets(2, "star"), 4.0, -1.0, None)


def stencil_7pt(g, seed=0, dims=None):
    """3-D 7-point stencil: U[-1,1] off-diagonal values, diagonal 7."""
    rng = np.random.default_rng(seed)
    return _stencil(dims or (g, g, g), _offsets(3, "star"), 7.0, None, rng)


def stencil_5pt(g, seed=0, dims=None):
    """2-D 5-point stencil: U[-1,1] off-diagonal values, diagonal 5."""
    rng = np.random.default_rng(seed)
    return _stencil(dims or (g, g), _offsets(2, "star"), 5.0, None, rng)


def stencil_27pt(g=150, seed=1, dims=None):
    """3-D 27-point stencil on g^3: U[-1,1] values with the diagonal 27."""
    rng = np.random.default_rng(seed)
    return _stencil(dims or (g, g, g), _offsets(3, "box"), 27.0, None, rng)


def _zipf_lengths(rng, n, alpha, cap_k, mult, cap):
    """K ~ Zipf(alpha) truncated to [1, cap_k] (by rejection); L = min(cap, mult*K)."""
    k = rng.zipf(alpha, size=n)
    bad = k > cap_k
    while bad.any():
        k[bad] = rng.zipf(alpha, size=int(bad.sum()))
        bad = k > cap_k
    return np.minimum(cap, mult * k).astype(np.int64)


def _fill_rows(rng, n, lengths, local_frac, window):
    """Distinct, ascending columns per row: a fraction within +-window of the
    row (uniform on the clipped window), the rest uniform on [0, n)."""
    lengths = np.minimum(lengths, n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    rows = np.repeat(np.arange(n, dtype=np.int64), lengths)

    def draw(r, frac=local_frac):
        """One column per entry of row array r."""
        lo = np.maximum(r - window, 0)
        hi = np.minimum(r + window, n - 1)
        loc = rng.random(r.size) < frac
        c = rng.integers(0, n, size=r.size)
        c[loc] = lo[loc] + (rng.random(int(loc.sum())) * (hi[loc] - lo[loc] + 1)).astype(np.int64)
        return c

    cols = draw(rows)
    for rnd in range(400):
        # rows stay grouped and ascending; sort columns within each row by
        # sorting the combined key row * n + column
        key = rows * n + cols
        key.sort()
        cols = key - rows * n
        del key
        dup = np.zeros(nnz, dtype=bool)
        dup[1:] = (cols[1:] == cols[:-1]) & (rows[1:] == rows[:-1])
        if not dup.any():
            break
        redo = np.nonzero(dup)[0]
        # a row longer than its window allows ends with uniform redraws
        cols[redo] = draw(rows[redo], local_frac if rnd < 20 else 0.0)
    else:
        raise RuntimeError("could not make columns distinct")
    return row_ptr, cols.astype(np.int32)


def powerlaw(n=4_000_000, seed=3, alpha=2.0, cap=4096, mult=3,
             local_frac=0.8, window=None):
    """Random power-law matrix: row lengths L = min(cap, mult*K) with
    K ~ Zipf(alpha) truncated to [1, cap]; columns 80 % within +-n/8 of the
    row (clipped), 20 % uniform; distinct and ascending; values U[-1,1]."""
    rng = np.random.default_rng(seed)
    lengths = _zipf_lengths(rng, n, alpha, cap, mult, cap)
    w = n // 8 if window is None else window
    row_ptr, col_idx = _fill_rows(rng, n, lengths, local_frac, w)
    vals = rng.uniform(-1.0, 1.0, size=int(row_ptr[-1]))
    return n, row_ptr, col_idx, vals


def zipf_random(n, seed=0, mult=2, cap=4096):
    """Zipf-row random matrix of the batched mix (mean about 10 nnz/row);
    rows hold at most min(cap, n/4) entries."""
    return powerlaw(n, seed=seed, mult=mult, cap=max(1, min(cap, n // 4)))


def band(n=150_000, nnz=1_500_000, half_width=37_500, seed=7):
    """The paper's band matrix (Sec. III): nnz positions drawn uniformly
    from the band |i - j| <= half_width, values U[-1, 1]."""
    rng = np.random.default_rng(seed)
    rows = np.arange(n, dtype=np.int64)
    lo = np.maximum(rows - half_width, 0)
    hi = np.minimum(rows + half_width, n - 1)
    width = hi - lo + 1
    cdf = np.cumsum(width, dtype=np.float64)
    cdf /= cdf[-1]
    keys = np.empty(0, dtype=np.int64)
    while keys.size < nnz:
        need = int((nnz - keys.size) * 1.05) + 16
        r = np.searchsorted(cdf, rng.random(need), side="right")
        r = np.minimum(r, n - 1)
        c = lo[r] + (rng.random(need) * width[r]).astype(np.int64)
        keys = np.unique(np.concatenate([keys, r * n + c]))
    keys = rng.permutation(keys)[:nnz]
    keys.sort()
    r = keys // n
    c = keys % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, r + 1, 1)
    np.cumsum(row_ptr, out=row_ptr)
    vals = rng.uniform(-1.0, 1.0, size=nnz)
    return n, row_ptr, c.astype(np.int32), vals


def random_csr(n, density=0.2, seed=0, integer=False, empty_rows=True,
               shuffle_cols=False, duplicates=False, max_len=None):
    """Small random CSR for brute-force tests.  ``integer`` draws values in
    {-4..4} (exact FP64 sums); ``duplicates`` repeats some columns within a
    row; ``shuffle_cols`` leaves columns unsorted."""
    rng = np.random.default_rng(seed)
    ptr = [0]
    cols = []
    for i in range(n):
        k = rng.binomial(n, density) if n else 0
        if max_len is not None:
            k = min(k, max_len)
        if empty_rows and rng.random() < 0.1:
            k = 0
        c = rng.choice(n, size=min(k, n), replace=False) if k else np.zeros(0, np.int64)
        if duplicates and c.size and rng.random() < 0.3:
            c = np.concatenate([c, rng.choice(c, size=1 + c.size // 3)])
        c = np.sort(c)
        if shuffle_cols:
            c = rng.permutation(c)
        cols.append(c)
        ptr.append(ptr[-1] + c.size)
    col_idx = (np.concatenate(cols) if cols else np.zeros(0)).astype(np.int32)
    nnz = col_idx.size
    if integer:
        vals = rng.integers(-4, 5, size=nnz).astype(np.float64)
    else:
        vals = rng.uniform(-1.0, 1.0, size=nnz)
    return n, np.asarray(ptr, dtype=np.int64), col_idx, vals


def uniform_x(n, seed=2, integer=False):
    """x ~ U[-1, 1] (or integers in {-4..4})."""
    rng = np.random.default_rng(seed)
    if integer:
        return rng.integers(-4, 5, size=n).astype(np.float64)
    return rng.uniform(-1.0, 1.0, size=n)


def batch_mix(count=256, seed=5, n_lo=1e3, n_hi=1e6):
    """The batched workload: ``count`` matrices with n log-uniform in
    [n_lo, n_hi], kinds cycling 5-point / 7-point / Zipf-row random
    (mean about 10 nnz per row).  Stencil n is rounded to g^2 / g^3."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        target = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        kind = ("5pt", "7pt", "zipf")[i % 3]
        s = int(rng.integers(0, 2**31 - 1))
        if kind == "5pt":
            g = max(2, int(round(target ** 0.5)))
            out.append(("5pt", stencil_5pt(g, seed=s)))
        elif kind == "7pt":
            g = max(2, int(round(target ** (1.0 / 3.0))))
            out.append(("7pt", stencil_7pt(g, seed=s)))
        else:
            out.append(("zipf", zipf_random(int(round(target)), seed=s)))
    return out


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed, t):
    """SplitMix64 (Steele, Lea and Flood) output for state seed + (t+1)*golden,
    elementwise over uint64 arrays t (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(t, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def request_x(seed, n, width):
    """X (n x width) of a serving request: element (i, j) = 2u - 1 with
    u = (splitmix64(seed, 8 i + j) >> 11) * 2^-53."""
    i = np.arange(n, dtype=np.uint64)[:, None]
    j = np.arange(width, dtype=np.uint64)[None, :]
    z = splitmix64(seed, i * np.uint64(8) + j)
    return (z >> np.uint64(11)).astype(np.float64) * 2.0 ** -53 * 2.0 - 1.0


def serve_mix(count=64, seed=6, n_lo=1e4, n_hi=2e6, total_bytes=1.5e9):
    """Resident matrices of the serving workload: n log-uniform in
    [n_lo, n_hi], alternating 7-point stencils and power-law rows, with every
    n scaled by one factor so the CSR bytes total about total_bytes."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=count))
    est = sum((104.0 if i % 2 == 0 else 146.0) * n for i, n in enumerate(ns))
    ns = ns * min(1.0, total_bytes / est)
    out = []
    for i, n in enumerate(ns):
        s = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            g = max(2, int(round(n ** (1.0 / 3.0))))
            out.append(("7pt", stencil_7pt(g, seed=s)))
        else:
            out.append(("powerlaw", zipf_random(max(16, int(round(n))), seed=s)))
    return out


def poisson_arrivals(rate, duration_s, seed=7):
    """Arrival times (s) of a Poisson process of `rate` per second."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=int(rate * duration_s * 1.2) + 16)
    t = np.cumsum(gaps)
    return t[t < duration_s]


def csr_nbytes(n, nnz):
    """Bytes of a CSR matrix with int32 columns, int64 row pointers."""
    return 12 * nnz + 8 * (n + 1)
