"""Host-side arithmetic of bench.py on CPU: the roofline figures the
benchmark line reports (algorithmic bytes per granule-substep over the
dominant entry point's mean duration, against the measured peak)."""
import pytest


def test_algo_bytes_charge_alpha_once_per_window():
    import bench

    # the fused step is charged 90 B per granule, plus the alpha_s share of the
    # last substep spread over the window's K calls; the FP64 path twice that
    assert bench.algo_bytes("gic_step", 20) == pytest.approx(90 + 20 / 20)
    assert bench.algo_bytes("gic_step", 100, fp64=True) == pytest.approx(2 * (90 + 20 / 100))
    # entry points without an alpha_s scatter carry no share
    assert bench.algo_bytes("gic_sort", 20) == 88
    assert bench.algo_bytes("gic_substep_adj", 20) == 100


def test_roofline_picks_the_slowest_entry_point_and_divides_by_the_peak():
    import bench

    n, K, hbm = 16_000_000, 20, 6663.9
    per_call = {"gic_step": 1.5, "gic_sort": 0.2}
    r = bench.roofline_of(per_call, n, K, False, hbm, traffic=2.7e9)
    assert r["kernel"] == "gic_step" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    expect = (90 + 20 / K) * n / 1.5e-3 / 1e9  # bytes per call over the call's seconds
    assert r["achieved"] == pytest.approx(expect)
    assert r["frac"] == pytest.approx(expect / hbm)
    assert r["per_call_frac"]["gic_step"] == pytest.approx(r["frac"])
    assert r["per_call_frac"]["gic_sort"] == pytest.approx(88 * n / 0.2e-3 / 1e9 / hbm)
    assert r["traffic"] == 2.7e9 and r["peak"] == hbm


def test_window_traffic_lies_between_its_calls():
    import bench

    # the sweep's figure is a mean over one rebuilding call, 18 list-keeping
    # calls and the alpha_s call, so it lies between the cheapest and the
    # dearest of them and near the list-keeping calls that dominate it
    t = bench.NCU_TRAFFIC[("scale_sweep_16m", "gic_step")]
    assert 2.4e9 < t < 7.1e9
    assert t < 3.0e9  # 18 of the 20 calls keep the lists


def test_oracle_configs_time_each_configuration_and_never_raise(monkeypatch):
    import bench

    monkeypatch.setattr(bench, "ORACLE_CONFIGS", (("plain_fp64_8k", None), ("plain_fp64_8k", 2000),
                                                  ("no_such_workload", None)))
    r = bench.oracle_configs({}, 2)
    whole = r["plain_fp64_8k"]  # the later entry of the same name: its first 2000 granules
    assert whole["granules"] == 2000 and whole["of"] == 8000 and whole["substeps"] == 10
    assert whole["one_core"] > 0 and whole["all_cores"] > 0 and whole["cores"] == 2
    assert "first 2000 granules" in whole["sample"]
    assert "error" in r["no_such_workload"]  # a failed leg is reported, not raised
