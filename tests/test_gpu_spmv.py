"""GPU SpMV (lilac_spmv through the C ABI) against the FP64 oracle.

Every kernel variant and lanes-per-row, FP64 and FP32, on matrices that span
many tiles with a ragged tail, empty rows, unsorted and duplicate columns,
rows longer than a tile (split rows), degenerate shapes, and the full-size
workloads (2D Laplacian 64x64; random SPD n=75,000; R-MAT scale 22; 3D
Laplacian 192^3) in the launch configuration the benchmark uses.
"""
import numpy as np
import pytest

import oracle
from paper_2001_07938_gb300 import inputs
from paper_2001_07938_gb300 import lilac as L
from lilac_testutil import ALL_VARIANTS, assert_spmv_close, dev, host, torch_cuda, true_rel_residual
from conftest import load_golden

pytestmark = pytest.mark.gpu


def _run(M, x_np, dtype):
    torch = torch_cuda()
    xd = dev(x_np.astype(dtype))
    yd = torch.full((M.rows,), float("nan"), dtype=xd.dtype, device="cuda")
    M.spmv(xd, yd)
    torch.cuda.synchronize()
    return host(yd)


def _check_all_variants(A, dtype, seed=0, variants=ALL_VARIANTS):
    fp32 = dtype == np.float32
    Ad = A.astype(dtype)
    x = inputs.uniform(seed + 17, max(A.ncols, 1), dtype=dtype)[: A.ncols]
    M = L.CsrMatrix.from_csr(Ad)
    results = {}
    for var, w in variants:
        M.set_variant(var, w)
        y = _run(M, x, dtype)
        assert_spmv_close(Ad, x.astype(np.float64), y, fp32, f"variant {var} width {w}")
        results[(var, w)] = y
    M.close()
    return results


def test_paper_example_bit_exact():
    g = load_golden("csr_example_5x5.txt")
    A = inputs.CSR(5, 5, np.array(g["row_ptr"], np.int32), np.array(g["col_ind"], np.int32),
                   np.array(g["val"], np.float64))
    x = np.array(g["x"], np.float64)
    M = L.CsrMatrix.from_csr(A)
    assert M.info()["ncols"] == 5  # max(col_ind) + 1, the cached invariant
    for var, w in ALL_VARIANTS:
        M.set_variant(var, w)
        assert list(_run(M, x, np.float64)) == [float(t) for t in g["y"]]
    M.close()


def test_paper_jds_example_bit_exact():
    """The handle's JDS form of the paper's CSR example is the paper's printed
    JDS example (Section 3.2), array for array."""
    g = load_golden("csr_example_5x5.txt")
    j = load_golden("jds_example_5x5.txt")
    A = inputs.CSR(5, 5, np.array(g["row_ptr"], np.int32), np.array(g["col_ind"], np.int32),
                   np.array(g["val"], np.float64))
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    perm, jd_ptr, col, val, nzcnt = M.jds()
    M.close()
    assert perm.tolist() == j["perm"]
    assert jd_ptr.tolist() == j["jd_ptr"]
    assert col.tolist() == j["col_ind"]
    assert val.tolist() == [float(t) for t in j["val"]]
    assert nzcnt.tolist() == j["nzcnt"]


def test_jds_matches_oracle_conversion_and_follows_value_updates():
    """JDS arrays equal the oracle's CSR-to-JDS conversion (bit-exact) on a
    matrix with empty rows and ties; the JDS kernel follows
    lilac_csr_update_values."""
    torch = torch_cuda()
    A = inputs.random_csr(4000, 3000, 12, 0.2, seed=11)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_JDS)
    perm, jd_ptr, col, val, nzcnt = M.jds()
    J = oracle.csr_to_jds(A.row_ptr, A.col_ind, A.vals)
    assert np.array_equal(perm, J["perm"]) and np.array_equal(jd_ptr, J["jd_ptr"])
    assert np.array_equal(col, J["col_ind"]) and np.array_equal(val, J["val"])
    assert np.array_equal(nzcnt, J["nzcnt"])
    x = inputs.uniform(5, A.ncols)
    assert_spmv_close(A, x, _run(M, x, np.float64), False, "jds")
    v2 = inputs.uniform(6, A.nnz)
    M2 = inputs.CSR(A.n, A.ncols, A.row_ptr, A.col_ind, v2)
    v2d = dev(v2)
    L.lilac_csr_update_values(M.handle, v2d.data_ptr(), L.LILAC_MEM_DEVICE)
    torch.cuda.synchronize()
    assert_spmv_close(M2, x, _run(M, x, np.float64), False, "jds after update")
    M.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape", [(3000, 2500, 40), (777, 5000, 9), (5000, 300, 3)])
def test_random_with_empty_rows_duplicates_unsorted(dtype, shape):
    n, ncols, max_len = shape
    A = inputs.random_csr(n, ncols, max_len, 0.2, seed=n)
    _check_all_variants(A, dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_laplacian2d_full_and_ragged(dtype):
    for m in (64, 97):
        _check_all_variants(inputs.laplacian2d(m), dtype, seed=m)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_split_rows_longer_than_a_tile(dtype):
    A = inputs.powerlaw_csr(6000, 9000, 60000, power=8, seed=3)
    assert np.diff(A.row_ptr).max() > 2048 * 3
    res = _check_all_variants(A, dtype)
    M = L.CsrMatrix.from_csr(A.astype(dtype))
    assert M.info()["num_long_rows"] > 0
    M.close()
    assert res


def test_one_huge_row_and_tiny_shapes():
    n1 = 100_003
    A = inputs.CSR(1, n1, np.array([0, n1], np.int32), np.arange(n1, dtype=np.int32),
                   inputs.uniform(9, n1))
    _check_all_variants(A, np.float64)
    one = inputs.CSR(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([2.5]))
    _check_all_variants(one, np.float64)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sell_row_order_sorted_and_split_rows(dtype):
    """SELL: a stencil keeps row order, irregular rows are sorted by length,
    and rows longer than the piece cap are cut into pieces that are finished
    in piece order (powerlaw rows up to ~60,000 nonzeros)."""
    cases = [(inputs.laplacian2d(97), False), (inputs.random_csr(3000, 2500, 40, 0.2, seed=5), False),
             (inputs.powerlaw_csr(6000, 9000, 60000, power=8, seed=3), True)]
    for A, split in cases:
        Ad = A.astype(dtype)
        M = L.CsrMatrix.from_csr(Ad, flags=L.LILAC_CREATE_NO_TUNE)
        M.set_variant(L.LILAC_VARIANT_SELL, 1)
        info = M.info()
        assert info["active_variant"] == L.LILAC_VARIANT_SELL, A.name
        assert (info["sell_split_rows"] > 0) == split
        assert A.nnz <= info["sell_padded_nnz"] <= 1.5 * A.nnz + 64 * (A.n // 32 + 1)
        x = inputs.uniform(21, A.ncols, dtype=dtype)
        y1 = _run(M, x, dtype)
        assert_spmv_close(Ad, x.astype(np.float64), y1, dtype == np.float32, f"sell {A.name}")
        np.testing.assert_array_equal(_run(M, x, dtype), y1)  # fixed order: reproducible
        M.close()


@pytest.mark.parametrize("variant", [5, 7])
def test_slab_and_sell_padding_ignore_nonfinite_x_and_follow_updates(variant):
    """Padding elements contribute nothing even where x holds inf / nan (a
    padding slot never reads a caller's x), and value updates reach the copy."""
    torch = torch_cuda()
    A = inputs.spd_random(20000, 30, 20.0, 2)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(variant, 4)
    assert M.info()["active_variant"] == variant
    x = inputs.uniform(4, A.n)
    assert_spmv_close(A, x, _run(M, x, np.float64), False, f"variant {variant}")
    # x[j] = inf for a column that few rows reference: the others stay finite
    counts = np.bincount(A.col_ind, minlength=A.n)
    j = int(np.argmin(np.where(counts > 0, counts, 1 << 30)))
    xi = x.copy()
    xi[j] = np.inf
    y = _run(M, xi, np.float64)
    touches = np.zeros(A.n, bool)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    touches[rows[A.col_ind == j]] = True
    ref = oracle.spmv(A.row_ptr, A.col_ind, A.vals, np.where(np.isfinite(xi), xi, 0.0))
    assert np.all(np.isfinite(y[~touches]))
    assert np.all(~np.isfinite(y[touches]))
    tol = 1e-12 * oracle.spmv_abs_bound(A.row_ptr, A.col_ind, A.vals, x)
    assert np.all(np.abs(y[~touches] - ref[~touches]) <= tol[~touches])
    # new values reach the copy
    v2 = inputs.uniform(6, A.nnz)
    L.lilac_csr_update_values(M.handle, v2.ctypes.data, L.LILAC_MEM_HOST)
    torch.cuda.synchronize()
    A2 = inputs.CSR(A.n, A.ncols, A.row_ptr, A.col_ind, v2)
    assert M.info()["active_variant"] == variant
    assert_spmv_close(A2, x, _run(M, x, np.float64), False, f"variant {variant} after update")
    M.close()


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_hub_variant_on_a_power_law_graph(dtype):
    """HUB (the hub columns' x gathered per call and held in shared memory, in
    slabs; the cold nonzeros as a sliced ELL copy that adds the slab sums) on
    an R-MAT graph whose x exceeds 1 MB: built, within the oracle's bound,
    bitwise the same on repeat, ignoring an inf in x where no nonzero reads
    it, and following value updates.  A matrix with uniform random columns
    gets no hub copy and runs STAGED."""
    fp32 = dtype == np.float32
    torch = torch_cuda()
    A = inputs.rmat_transposed(19 if fp32 else 18, 8, seed=21).astype(dtype)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_HUB, 1)
    info = M.info()
    assert info["active_variant"] == L.LILAC_VARIANT_HUB
    assert info["spmv_kernels"] in (3, 4)
    x = inputs.uniform(22, A.ncols, dtype=dtype)
    y = _run(M, x, dtype)
    assert_spmv_close(A, x.astype(np.float64), y, fp32, "hub")
    np.testing.assert_array_equal(y, _run(M, x, dtype))
    counts = np.bincount(A.col_ind, minlength=A.ncols)
    empty = np.nonzero(counts == 0)[0]
    if empty.size:
        xi = x.copy()
        xi[empty[:1000]] = np.inf
        np.testing.assert_array_equal(_run(M, xi, dtype), y)
    v2 = inputs.uniform(23, A.nnz, 0.0, 1.0, dtype=dtype)
    L.lilac_csr_update_values(M.handle, v2.ctypes.data, L.LILAC_MEM_HOST)
    torch.cuda.synchronize()
    A2 = inputs.CSR(A.n, A.ncols, A.row_ptr, A.col_ind, v2)
    assert_spmv_close(A2, x.astype(np.float64), _run(M, x, dtype), fp32, "hub after update")
    M.close()
    U = inputs.spd_random(200000, 4, 20.0, 5)
    MU = L.CsrMatrix.from_csr(U, flags=L.LILAC_CREATE_NO_TUNE)
    MU.set_variant(L.LILAC_VARIANT_HUB, 1)
    assert MU.info()["active_variant"] == L.LILAC_VARIANT_STAGED
    xu = inputs.uniform(24, U.ncols)
    assert_spmv_close(U, xu, _run(MU, xu, np.float64), False, "hub not built")
    MU.close()


def test_hub_cg_on_a_symmetrised_power_law_matrix():
    """FP64 CG on a HUB handle (the SpMV with the CG epilogue through the hub
    slabs and the cold copy): converges like the oracle, bitwise run to run."""
    import scipy.sparse as sp
    G = inputs.rmat_transposed(18, 8, seed=31)
    B = sp.csr_matrix((np.ones(G.nnz), G.col_ind, G.row_ptr), shape=(G.n, G.n))
    S = (B + B.T).tocsr()
    S.sum_duplicates()
    S.setdiag(0)
    S.eliminate_zeros()
    d = np.asarray(abs(S).sum(axis=1)).ravel() + 1.0
    S = (S + sp.diags(d)).tocsr()
    S.sort_indices()
    A = inputs.CSR(S.shape[0], S.shape[1], S.indptr.astype(np.int32), S.indices.astype(np.int32),
                   S.data.astype(np.float64))
    b = inputs.uniform(32, A.n)
    torch = torch_cuda()
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_HUB, 1)
    assert M.info()["active_variant"] == L.LILAC_VARIANT_HUB
    xs = []
    for _ in range(2):
        x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        st, info = M.cg(dev(b), x, rtol=1e-10, max_iter=3000)
        torch.cuda.synchronize()
        assert st == L.LILAC_OK
        xs.append(host(x))
    M.close()
    np.testing.assert_array_equal(xs[0], xs[1])
    _, itr, _ = oracle.cg(A.row_ptr, A.col_ind, A.vals, b, max_iter=3000, rtol=1e-10)
    # ~600 iterations: rounding in another summation order moves the count a little
    assert abs(info.iters - itr) <= max(2, itr // 50)
    assert true_rel_residual(A, b, xs[0]) <= 1e-10


def test_slab_fp32_values_and_vectors():
    """SLAB on an FP32 handle: the slab of x in shared memory holds FP32 values
    and rows accumulate in FP32; two slabs of 20,000 columns."""
    A = inputs.spd_random(40000, 30, 20.0, 3).astype(np.float32)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_SLAB, 4)
    assert M.info()["active_variant"] == L.LILAC_VARIANT_SLAB
    x = inputs.uniform(12, A.n, dtype=np.float32)
    y = _run(M, x, np.float32)
    assert_spmv_close(A, x.astype(np.float64), y, True, "slab fp32")
    np.testing.assert_array_equal(_run(M, x, np.float32), y)
    M.close()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_merge_empty_runs_and_rows_across_ctas(dtype):
    """MERGE: runs of empty rows longer than a CTA's path range, rows whose
    nonzeros span many sub-tiles and CTAs, tiny rows between them, an empty
    tail; every row closed exactly once, and the same bits on a second call."""
    rng = np.random.default_rng(1)
    lens = np.concatenate([np.zeros(50_000, np.int64), [400_000], rng.integers(0, 4, 200_000),
                           np.zeros(30_000, np.int64), [90_000], rng.integers(0, 40, 30_000),
                           np.zeros(1_000, np.int64)])
    rp = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    nnz = int(rp[-1])
    ncols = 50_000
    A = inputs.CSR(len(lens), ncols, rp, rng.integers(0, ncols, nnz).astype(np.int32),
                   rng.uniform(-1, 1, nnz)).astype(dtype)
    x = inputs.uniform(23, ncols, dtype=dtype)
    M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    M.set_variant(L.LILAC_VARIANT_MERGE, 0)
    y1 = _run(M, x, dtype)
    y2 = _run(M, x, dtype)
    M.close()
    assert_spmv_close(A, x.astype(np.float64), y1, dtype == np.float32, "merge extremes")
    assert np.array_equal(y1, y2)


def test_all_empty_rows_and_zero_rows():
    torch = torch_cuda()
    A = inputs.CSR(1000, 10, np.zeros(1001, np.int32), np.zeros(0, np.int32), np.zeros(0))
    M = L.CsrMatrix(A.row_ptr, A.col_ind, A.vals, ncols=10)
    for var, w in ALL_VARIANTS:
        M.set_variant(var, w)
        y = _run(M, np.ones(10), np.float64)
        assert np.all(y == 0.0)
    M.close()
    Z = L.CsrMatrix(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), ncols=0)
    assert Z.info()["rows"] == 0
    Z.spmv(torch.zeros(0, dtype=torch.float64, device="cuda"),
           torch.zeros(0, dtype=torch.float64, device="cuda"))
    Z.close()


def test_invalid_csr_is_rejected():
    bad_col = inputs.CSR(2, 2, np.array([0, 1, 2], np.int32), np.array([0, 5], np.int32),
                         np.ones(2))
    with pytest.raises(L.LilacError) as e:
        L.CsrMatrix(bad_col.row_ptr, bad_col.col_ind, bad_col.vals, ncols=2)
    assert e.value.status == L.LILAC_ERR_INVALID_CSR
    with pytest.raises(L.LilacError) as e:
        L.CsrMatrix(np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32), np.ones(2))
    assert e.value.status == L.LILAC_ERR_INVALID_CSR
    with pytest.raises(L.LilacError) as e:
        L.CsrMatrix(np.array([0, 1, 3], np.int32), np.array([0, 1], np.int32), np.ones(2))
    assert e.value.status == L.LILAC_ERR_INVALID_CSR
    with pytest.raises(L.LilacError) as e:
        L.CsrMatrix(np.array([0, 1], np.int32), np.array([-1], np.int32), np.ones(1))
    assert e.value.status == L.LILAC_ERR_INVALID_CSR


def test_device_input_host_vectors_update_values_and_determinism():
    torch = torch_cuda()
    A = inputs.random_csr(4000, 3000, 30, 0.1, seed=5)
    # create from device arrays
    M = L.CsrMatrix(dev(A.row_ptr), dev(A.col_ind), dev(A.vals))
    info = M.info()
    assert info["ncols"] == oracle.csr_ncols(A.col_ind)
    x = inputs.uniform(1, info["ncols"])
    y1 = _run(M, x, np.float64)
    y2 = _run(M, x, np.float64)
    np.testing.assert_array_equal(y1, y2)  # static schedule: bitwise reproducible
    # host vectors through the library's own staging buffers
    yh = np.empty(A.n)
    M.spmv(x, yh)
    np.testing.assert_array_equal(yh, y1)
    # update_values: the paper's "update" step
    v2 = inputs.uniform(2, A.nnz)
    before = M.info()["h2d_bytes"]
    L.lilac_csr_update_values(M.handle, v2.ctypes.data, L.LILAC_MEM_HOST)
    torch.cuda.synchronize()
    assert M.info()["h2d_bytes"] == before + 8 * A.nnz
    A2 = inputs.CSR(A.n, info["ncols"], A.row_ptr, A.col_ind, v2)
    assert_spmv_close(A2, x, _run(M, x, np.float64), False, "after update")
    M.close()


def test_autotuner_timed_and_heuristic_choices_are_valid():
    A = inputs.spd_random(20000, 30, 20.0, 1)
    x = inputs.uniform(3, A.n)
    for flags in (0, L.LILAC_CREATE_NO_TUNE):
        M = L.CsrMatrix.from_csr(A, flags=flags)
        info = M.info()
        assert info["variant"] in ((1, 2, 3) if flags else (1, 2, 3, 4, 5, 6, 7))
        assert_spmv_close(A, x, _run(M, x, np.float64), False, f"tuned flags={flags}")
        M.close()


def _time_calls(M, x, calls=20):
    """Fastest of three rounds of `calls` SpMVs, ms per call (CUDA events)."""
    torch = torch_cuda()
    xd = dev(x)
    yd = torch.empty(M.rows, dtype=xd.dtype, device="cuda")
    for _ in range(3):
        M.spmv(xd, yd)
    best = float("inf")
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(calls):
            M.spmv(xd, yd)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) / calls)
    return best


@pytest.mark.parametrize("kind", ["random_columns", "power_law_rows"])
def test_tuned_choice_is_within_a_factor_of_the_fastest_candidate(kind):
    """The timed autotuner (the per-matrix tuning phase; no single kernel wins
    everywhere) records its trial; the kernel it keeps is the trial's fastest
    entry or a sliced ELL entry (SELL, SLAB, HUB) within 3% of it (a tie),
    and re-timed after create on a separate untuned handle it is within 1.3x
    of the fastest candidate re-timed the same way."""
    if kind == "random_columns":
        A = inputs.spd_random(40000, 40, 20.0, 11)
    else:
        A = inputs.powerlaw_csr(60000, 60000, 3000, 6, 12)
    x = inputs.uniform(13, A.ncols)
    M = L.CsrMatrix.from_csr(A)
    table = M.tune_table()
    info = M.info()
    M.close()
    assert len(table) >= 5 and all(t["ms"] > 0 for t in table)
    best = min(table, key=lambda t: t["ms"])
    kept = [t for t in table if (t["variant"], t["width"]) == (info["variant"], info["vector_width"])]
    assert kept, (info, table)
    sliced = (L.LILAC_VARIANT_SELL, L.LILAC_VARIANT_SLAB, L.LILAC_VARIANT_HUB)
    if (best["variant"], best["width"]) != (info["variant"], info["vector_width"]):
        ties = [t for t in table if t["variant"] in sliced and t["ms"] <= 1.03 * best["ms"] * (1 + 1e-6)]
        assert ties and kept[0]["ms"] == min(t["ms"] for t in ties), (info, table)
    R = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
    assert R.tune_table() == []
    retimed = {}
    for t in table:
        R.set_variant(t["variant"], t["width"])
        retimed[(t["variant"], t["width"])] = _time_calls(R, x)
    R.close()
    chosen = retimed[(info["variant"], info["vector_width"])]
    assert chosen <= 1.3 * min(retimed.values()), (info, retimed)


def _heuristic(A):
    """The choice from row statistics alone, as the header documents it:
    short regular rows -> STAGED, one lane per row; irregular rows (coefficient
    of variation > 1, or a row longer than a 2048-nonzero tile) -> STAGED with
    min(w, 8) lanes, w the smallest power of two >= mean/2; long regular rows
    -> VECTOR with the smallest power of two >= mean/16 lanes (2 .. 32)."""
    lens = np.diff(A.row_ptr).astype(np.float64)
    mean = lens.mean()
    cv = lens.std() / mean if mean > 0 else 0.0
    if cv > 1.0 or lens.max() > 2048 or mean <= 12.0:
        if mean <= 12.0 and cv <= 1.0:
            return L.LILAC_VARIANT_STAGED, 1
        w = 1
        while w < 32 and w < mean / 2.0:
            w *= 2
        return L.LILAC_VARIANT_STAGED, min(w, 8)
    v = 2
    while v < 32 and v < mean / 16.0:
        v *= 2
    return L.LILAC_VARIANT_VECTOR, v


def test_heuristic_choice_follows_row_statistics():
    """LILAC_CREATE_NO_TUNE keeps the choice made from the row statistics."""
    cases = [inputs.laplacian2d(100), inputs.spd_random(20000, 30, 20.0, 1),
             inputs.spd_random(20000, 90, 20.0, 2), inputs.powerlaw_csr(30000, 30000, 5000, 6, 3),
             inputs.random_csr(5000, 5000, 40, 0.2, 4)]
    seen = set()
    for A in cases:
        M = L.CsrMatrix.from_csr(A, flags=L.LILAC_CREATE_NO_TUNE)
        info = M.info()
        M.close()
        want = _heuristic(A)
        assert (info["variant"], info["vector_width"]) == want, (A.name, info, want)
        seen.add(want)
    assert len(seen) >= 3  # the cases reach different branches of the rule


# --- full-size workloads ---------------------------------------------------------

def test_full_laplacian2d_64_fp64():
    A, x = inputs.workload_laplacian2d_spmv(64)
    assert A.n == 4096 and A.nnz == 20224
    M = L.CsrMatrix.from_csr(A)
    assert_spmv_close(A, x, _run(M, x, np.float64), False, "laplacian2d 64")
    M.close()


@pytest.mark.slow
def test_full_spd_75k_fp64():
    A, _ = inputs.workload_spd_cg()
    x = inputs.uniform(7, A.n)
    M = L.CsrMatrix.from_csr(A)
    assert_spmv_close(A, x, _run(M, x, np.float64), False, "spd 75k")
    for var in (L.LILAC_VARIANT_SLAB, L.LILAC_VARIANT_SELL):
        M.set_variant(var, 4)
        assert M.info()["active_variant"] == var
        assert_spmv_close(A, x, _run(M, x, np.float64), False, f"spd 75k variant {var}")
    M.close()


@pytest.mark.slow
def test_full_rmat22_fp32():
    A = inputs.workload_rmat_pagerank()
    x = inputs.uniform(8, A.n, 0.0, 1.0, dtype=np.float32)
    M = L.CsrMatrix.from_csr(A)
    assert M.info()["num_long_rows"] > 0
    assert_spmv_close(A, x.astype(np.float64), _run(M, x, np.float32), True, "rmat 22")
    M.set_variant(L.LILAC_VARIANT_SELL, 1)
    info = M.info()
    assert info["active_variant"] == L.LILAC_VARIANT_SELL and info["sell_split_rows"] > 0
    assert_spmv_close(A, x.astype(np.float64), _run(M, x, np.float32), True, "rmat 22 sell")
    M.close()


@pytest.mark.slow
def test_full_laplacian3d_192_fp32():
    A, _ = inputs.workload_poisson3d_ir()
    assert A.nnz == 7 * 192 ** 3 - 6 * 192 ** 2
    x = inputs.uniform(9, A.n, dtype=np.float32)
    M = L.CsrMatrix.from_csr(A)
    assert_spmv_close(A, x.astype(np.float64), _run(M, x, np.float32), True, "laplacian3d 192")
    M.set_variant(L.LILAC_VARIANT_SELL, 1)
    assert M.info()["active_variant"] == L.LILAC_VARIANT_SELL
    assert_spmv_close(A, x.astype(np.float64), _run(M, x, np.float32), True, "laplacian3d 192 sell")
    M.close()
