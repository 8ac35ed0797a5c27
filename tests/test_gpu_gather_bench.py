"""The gather-ceiling measurement (pdlp_gather_bench): each method computes the same
synthetic product (TMA gathers and the hybrid against the LSU result), invalid sizes
are rejected, and the reported counts match the requested shape."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_2501_07018_gb300 as p

    return p


@pytest.mark.parametrize("method,row_len,deg", [("lsu", 24, 0.0), ("lsu", 7, 2.08),
                                                ("tma", 24, 0.0), ("tma", 8, 2.08),
                                                ("hybrid", 24, 2.08)])
def test_methods_agree(pkg, method, row_len, deg):
    r = pkg.gather_bench(method, 8, 100_000, row_len, 2_000_000, deg, reps=2)
    assert r["entries"] == (2_000_000 // (32 * row_len)) * 32 * row_len
    assert r["us"] > 0 and r["entries_per_s"] > 0
    # the same products in another order of the four-entry groups at most
    assert r["max_diff_vs_lsu"] <= 1e-12


def test_fp32_and_rejections(pkg):
    r = pkg.gather_bench("lsu", 4, 100_000, 10, 1_000_000, 0.0, reps=2)
    assert r["entries"] == (1_000_000 // 320) * 320
    for bad in (dict(method="tma", elem_bytes=4), dict(table_len=10), dict(row_len=9, method="tma"),
                dict(nnz=10), dict(degree_s=0.5), dict(degree_s=2.0), dict(degree_s=3.0, dmax=1.0)):
        args = dict(method="lsu", elem_bytes=8, table_len=100_000, row_len=8, nnz=1_000_000,
                    degree_s=0.0, reps=1)
        args.update(bad)
        with pytest.raises(pkg.PdlpError) as ei:
            pkg.gather_bench(**args)
        assert ei.value.code == -1, bad
