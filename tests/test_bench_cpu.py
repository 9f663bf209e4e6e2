"""Host-side arithmetic of bench.py (no GPU): the algorithmic flop count behind
the reported GFLOP/s."""


def test_algorithmic_gflops_counts():
    import bench

    # Algorithm 1 at m = 2n: Cholesky 8n^3/3 + W 4n^3/3 + SYMV 16n^3/3 + rank-2k
    # 16n^3/3 + back-transform 24n^3 = 116 n^3 / 3
    r = bench.algorithmic_gflops(3, 2.0)
    assert abs(r["flops_per_solve"] - 116.0 * 27 / 3) <= 1e-9
    assert abs(r["value"] - 2.0 * 116.0 * 27 / 3 / 1e9) <= 1e-18
    big = bench.algorithmic_gflops(8192, 0.343)
    assert 7.0e3 < big["value"] < 7.5e3 and big["unit"] == "GFLOP/s"
