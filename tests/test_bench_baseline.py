"""bench.py's CPU baseline object (CPU only): the oracle's all-core rate with
its core count, a single-core rate, and the extrapolated full H.x and FP64
time-to-E0 (rows per H.x times the measured time per row)."""
import pytest


def test_oracle_baseline_fields():
    import bench
    import oracle
    from edinputs import configs as C
    p = C.chain(12, 1.0, 0.3, translations=True)
    cores = oracle.num_threads()
    d = bench.oracle_baseline(p, 0.3, False, 1000, 40)
    assert d["kind"] == "oracle" and d["unit"] == bench.UNIT and d["cores"] == cores
    assert d["value"] > 0 and d["single_core"]["value"] > 0
    assert oracle.num_threads() == cores                   # thread count restored
    assert d["time_to_E0_seconds_extrapolated"] == pytest.approx(40 * d["hx_seconds_extrapolated"])
    # rows per second implied by the all-core rate and the extrapolated H.x agree
    n_terms = len(p.terms.bonds)
    assert 1000 * n_terms / d["hx_seconds_extrapolated"] / 1e9 == pytest.approx(d["value"], rel=1e-9)
    assert "time_to_E0_seconds_extrapolated" not in bench.oracle_baseline(p, 0.1, False, 1000, None)


def test_bench_measurement_functions_exist():
    """Every measurement the default bench line calls is defined (CPU-only import check)."""
    import bench
    for name in ("hx_timing", "stored_bytes", "matrix_free_bytes", "lanczos_pair", "workload_summary", "sun_summary",
                 "batching_measurement", "oracle_baseline", "replica_aggregate", "main"):
        assert callable(getattr(bench, name)), name
    # algorithmic bytes: per row and per element as documented
    assert bench.stored_bytes(10, 100, 8) == 10 * (2 + 8 + 16) + 100 * 12
    assert bench.matrix_free_bytes(10, 100, 4, 8) == 10 * (8 + 2 + 8) + 100 * 4
