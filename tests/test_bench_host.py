"""bench.py's roofline bookkeeping, without a GPU: the algorithmic byte
counts per launch, the achieved bandwidth and fraction, and the ncu traffic
figure, which is reported only for the kernel source it was captured from
and for the form of the ordinary step the run used."""
import bench

# a window of 10 launches: 9 ordinary steps and 1 density step, 1e6
# carrier-steps, 2e4 eventful carriers, 1.9e4 changed records, 500 placed
# secondaries; 14 ms of kernel time in a 15 ms step
DELTA = {"particle_steps": 1_000_000, "eventful": 20_000, "changed": 19_000, "spawned": 500}
KT = {"step": (9, 8.0), "step_moments": (1, 1.5), "step_events": (10, 4.5), "compact": (0, 0.0)}


def fixed_peak(monkeypatch):
    monkeypatch.setattr(bench, "measured_peak", lambda: (5000.0, "measured"))


def test_roofline_counts_the_method_bytes(monkeypatch):
    fixed_peak(monkeypatch)
    r = bench.roofline_of(DELTA, KT, ms=15.0)
    # 20 B per carrier-step, 12 B per eventful carrier, 16 B per secondary
    alg = 20 * 1_000_000 + 12 * 20_000 + 16 * 500
    assert r["algorithmic_bytes_per_launch"] == alg / 10
    gbs = alg / 10 / (14.0 / 10 * 1e-3) / 1e9
    assert abs(r["achieved"] - gbs) < 1e-9 * gbs
    assert abs(r["frac"] - gbs / 5000.0) < 1e-12
    assert r["peak"] == 5000.0 and r["bound"] == "hbm" and r["unit"] == "GB/s"
    # the strict count: 16 B per carrier-step, 8 B per changed record
    strict = 16 * 1_000_000 + 8 * 19_000 + 16 * 500
    assert r["strict"]["bytes_per_launch"] == strict / 10
    assert abs(r["strict"]["frac"] - strict / 14.0e-3 / 1e9 / 5000.0) < 1e-12
    assert abs(r["avg_launch_ms"] - 1.4) < 1e-12
    assert abs(r["kernel_share_of_step_time"] - 14.0 / 15.0) < 1e-12


def test_roofline_is_absent_without_timed_launches(monkeypatch):
    fixed_peak(monkeypatch)
    kt = {k: (0, 0.0) for k in KT}
    assert bench.roofline_of(DELTA, kt, ms=15.0) is None


def test_traffic_follows_the_form_and_the_source(monkeypatch):
    fixed_peak(monkeypatch)
    sha = bench.kernel_sha()
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"separate": 16.0, "fused": 14.0, "src_sha": sha})
    sep = bench.roofline_of(DELTA, KT, ms=15.0)
    fus = bench.roofline_of(DELTA, KT, ms=15.0, fused=True)
    assert sep["form"] == "separate" and fus["form"] == "fused"
    assert sep["traffic"] == 16.0 * 1_000_000 / 10
    assert fus["traffic"] == 14.0 * 1_000_000 / 10
    assert "k_event" in sep["kernel"] and "general step inside" in fus["kernel"]
    # captured from another source: no traffic figure
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"separate": 16.0, "fused": 14.0, "src_sha": "0" * 16})
    assert bench.roofline_of(DELTA, KT, ms=15.0)["traffic"] is None
    # no capture of this form
    monkeypatch.setattr(bench, "NCU_TRAFFIC", {"separate": 16.0, "fused": None, "src_sha": sha})
    assert bench.roofline_of(DELTA, KT, ms=15.0, fused=True)["traffic"] is None

