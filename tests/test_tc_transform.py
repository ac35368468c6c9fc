"""The tensor-core axis transform of the fast-diagonalisation preconditioner (tdz_tc_axis_transform:
TMA-fed tcgen05 MMAs of kind::tf32, accumulator in tensor memory) against a binary64 product of the same
operands, over tile-aligned and ragged shapes (rows, k and columns not multiples of the tile, a plane
boundary inside a row tile), both column-tile widths and both output forms (FP32, TF32 pair)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tdz():
    import torch
    assert torch.cuda.is_available()
    import paper_2608_18472_b300 as m
    return m


def _tf32(x):
    """Nearest TF32 value (ties away from zero), as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


# (planes, plane_rows, k, ncols, tile_n): tile_n 0 = the library's choice (128-column tiles unless
# tiles_m * ceil(ncols / 256) >= 296); 64 = the autotuner's narrow tiles for small planes
CASES = [
    (2, 128, 64, 128, 0),       # one k-block ring pass, two row tiles
    (2, 200, 200, 200, 0),      # ragged k (7 blocks, the stage ring wraps), ragged columns, plane edge in a tile
    (2, 200, 200, 200, 256),    # the same with 256-column tiles
    (2, 200, 200, 200, 64),     # and with 64-column tiles (4 column tiles, the last one ragged)
    (2, 728, 728, 728, 64),     # the largest dot grid's padded plane in 64-column tiles
    (2, 1024, 1024, 1024, 0),   # the 2-D fast-diagonalisation shape, 128 blocks
    (2, 32768, 256, 256, 0),    # 512 row tiles: 256-column tiles
    (2, 20000, 200, 200, 128),  # ragged rows, k and columns, forced 128-column tiles
]


@pytest.mark.parametrize("planes,plane_rows,k,ncols,tile_n", CASES)
@pytest.mark.parametrize("split", [True, False])
@pytest.mark.parametrize("blo", [False, True])
@pytest.mark.parametrize("asplit", [False, True])
def test_tc_axis_transform(tdz, planes, plane_rows, k, ncols, tile_n, split, blo, asplit):
    """asplit: A given in FP32 and split into the TF32 pair by the kernel, in shared memory."""
    import torch
    rng = np.random.default_rng(plane_rows * 7 + k + ncols)
    rows = planes * plane_rows
    A = rng.standard_normal((rows, k)).astype(np.float32)
    a_hi = _tf32(A)
    a_lo = (A - a_hi).astype(np.float32)
    Bf = (rng.standard_normal((ncols, k)) / np.sqrt(k)).astype(np.float32)
    b_hi = _tf32(Bf)
    b_lo = (Bf - b_hi).astype(np.float32) if blo else np.zeros_like(b_hi)
    dev = torch.device("cuda")
    t_hi, t_lo, t_b, t_bl = (torch.from_numpy(np.ascontiguousarray(x)).to(dev) for x in (a_hi, a_lo, b_hi, b_lo))
    if asplit:
        t_hi, t_lo = torch.from_numpy(np.ascontiguousarray(A)).to(dev), None
    stride = plane_rows * ncols
    o_hi = torch.full((planes * stride,), np.nan, dtype=torch.float32, device=dev)
    o_lo = torch.full((planes * stride,), np.nan, dtype=torch.float32, device=dev) if split else None
    tdz.tc_axis_transform(t_hi, t_lo, t_b, rows, k, ncols, plane_rows, stride, o_hi, o_lo,
                          b_lo=t_bl if blo else None, tile_n=tile_n)
    torch.cuda.synchronize()
    # the three products the kernel forms, in binary64
    a64, al64, b64, bl64 = (x.astype(np.float64) for x in (a_hi, a_lo, b_hi, b_lo))
    D = (a64 + al64) @ b64.T + a64 @ bl64.T
    want = D.reshape(planes, plane_rows, ncols).transpose(0, 2, 1).reshape(-1)
    got_hi = o_hi.cpu().numpy()
    assert np.all(np.isfinite(got_hi))
    got = got_hi.astype(np.float64)
    if split:
        got_lo = o_lo.cpu().numpy()
        assert np.array_equal(got_hi, _tf32(got_hi))        # the high term is a TF32 value
        assert np.all(np.abs(got_lo) <= np.abs(got_hi) * 2.0 ** -11 + 1e-30)
        got = got + got_lo.astype(np.float64)
    # FP32 accumulation of k products (the lo operands read as TF32): well inside k * 2^-24 * sum |a||b|
    scale = (np.abs(a64) + np.abs(al64)) @ (np.abs(b64) + np.abs(bl64)).T
    bound = k * 2.0 ** -24 * scale.reshape(planes, plane_rows, ncols).transpose(0, 2, 1).reshape(-1)
    err = np.abs(got - want)
    assert np.all(err <= bound), float(np.max(err / bound))
    rel = np.linalg.norm(got - want) / np.linalg.norm(want)
    assert rel < 1e-5, rel
    if blo:
        # with both operands split, the product is the FP32 product of A and B to FP32 accuracy
        exact = A.astype(np.float64) @ Bf.astype(np.float64).T
        exact = exact.reshape(planes, plane_rows, ncols).transpose(0, 2, 1).reshape(-1)
        assert np.linalg.norm(got - exact) / np.linalg.norm(exact) < 1e-5


def test_tc_axis_transform_rejects_bad_sizes(tdz):
    import torch
    x = torch.zeros(64 * 64, dtype=torch.float32, device="cuda")
    with pytest.raises(tdz.TDZError):
        tdz.tc_axis_transform(x, x, x, 64, 6, 64, 64, 64 * 64, x)     # k not a multiple of 4
    with pytest.raises(tdz.TDZError):
        tdz.tc_axis_transform(x[1:], x, x, 64, 64, 64, 64, 64 * 64, x)  # a_hi not 16-byte aligned
    with pytest.raises(tdz.TDZError):
        tdz.tc_axis_transform(x, x, x, 64, 64, 64, 64, 64 * 64, x, tile_n=96)  # no such tile width


def test_preconditioner_autotuner(tdz):
    """A mixed 2-D batch times its preconditioner in the six transform variants at creation and keeps
    the fastest; a binary64 batch (cuBLAS DGEMM transforms) reports nothing."""
    import workloads as wl
    p = 6
    t = wl.knots_for_nsplines(-20.0, 20.0, 90, p)
    ops = tdz.Ops([tdz.Basis(t, p, p + 1) for _ in range(2)], wl.softcore_medium(0.5))
    b = tdz.Batch([ops], [0], tdz.MIXED)
    v, ms = b.precond_tuning(0)
    assert v in range(6)
    assert len(ms) == 6 and min(ms) > 0
    assert ms[v] == min(ms)
    b64 = tdz.Batch([ops], [0], tdz.FP64)
    assert b64.precond_tuning(0) == (-1, [])


def test_operator_timing(tdz):
    """tdz_batch_time_operator times one inner-solve operator apply of a 2-D/3-D batch; 1-D batches have
    no such operator."""
    import workloads as wl
    p = 6
    t = wl.knots_for_nsplines(-20.0, 20.0, 40, p)
    for dim in (2, 3):
        ops = tdz.Ops([tdz.Basis(t, p, p + 1) for _ in range(dim)], wl.softcore_medium(0.5))
        for prec in (tdz.MIXED, tdz.FP64):
            b = tdz.Batch([ops], [0], prec)
            assert b.time_operator(0, 2) > 0
    ops1 = tdz.assemble_1d(t, p, wl.softcore_medium(0.5))
    b1 = tdz.Batch([ops1], [0], tdz.MIXED)
    with pytest.raises(tdz.TDZError):
        b1.time_operator(0, 2)


def test_autotuner_cache(tdz, tmp_path, monkeypatch):
    """With TDZ_TUNE_CACHE set, the autotuners write their results (one JSON object per line, keyed by
    what was tuned, the sizes and the GPU) and a later batch of the same shapes reads them instead of
    timing again."""
    import json
    import workloads as wl
    path = tmp_path / "tune.jsonl"
    monkeypatch.setenv("TDZ_TUNE_CACHE", str(path))
    p = 7
    t = wl.knots_for_nsplines(-20.0, 20.0, 70, p)
    ops = tdz.Ops([tdz.Basis(t, p, p + 1) for _ in range(2)], wl.softcore_medium(0.5))
    b1 = tdz.Batch([ops], [0], tdz.MIXED)
    first = (b1.tuning(0), b1.precond_tuning(0))
    lines = [json.loads(x) for x in path.read_text().splitlines()]
    keys = [x["key"] for x in lines]
    assert any(k.startswith("apply2d p=7 n=") for k in keys) and any(k.startswith("fdtc dim=2 np=") for k in keys)
    b2 = tdz.Batch([ops], [0], tdz.MIXED)
    assert (b2.tuning(0), b2.precond_tuning(0)) == first      # the cached values, not a new timing
    assert len(path.read_text().splitlines()) == len(lines)   # nothing new written
