"""bench.py's host-side legs on the CPU: the oracle baseline's line (kind,
cores, bounded sample, single-core sample, CPU model) on a small workload of
the same kind, and the peaks file reader's fallback."""
import numpy as np

from paper_2507_15683_gb300 import synth


def test_cpu_baseline_reports_its_sample():
    import bench
    scene = synth.aerial_scene(2, 20_000, extent=(0.0, 200.0, 0.0, 200.0))
    cam = synth.camera(192, 108, 140.0)
    T_ref = synth.look_pose((100.0, 100.0, 60.0), 0.0, 0.5)
    T_q = synth.perturb_pose(T_ref, synth.rng(1), 2.0, 1.0)
    cb = bench.cpu_baseline(scene, cam, T_ref, T_q, 1.0)
    assert cb["kind"] == "oracle" and cb["unit"] == "Mpix/s" and cb["cores"] >= 1
    assert cb["value"] > 0 and np.isfinite(cb["loss"])
    assert "random pixels" in cb["sample"]
    st = cb["single_thread"]
    assert st["cores"] == 1 and st["value"] > 0 and "random pixels" in st["sample"]
    assert isinstance(cb["cpu_model"], str) and cb["cpu_model"]


def test_peaks_fall_back_without_the_measured_file(tmp_path, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "PEAKS_FILE", str(tmp_path / "missing.json"))
    pk, src = bench.peaks()
    assert src == "fallback" and pk["hbm_gbs"] == bench.FALLBACK_HBM_GBS


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_samples_report_median_under_load_and_reasons(tmp_path):
    """The nvidia-smi sampler's summary: the SM clock is the median of the
    samples taken under load, and every throttle reason seen active is named."""
    import bench
    rows = [
        "0, 1200, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active, 0",
        "0, 2070, 2070, 600.5, 0x0, Not Active, Not Active, Not Active, Not Active, 97",
        "0, 2055, 2070, 800.0, 0x4, Not Active, Not Active, Not Active, Active, 99",
        "0, 1980, 2070, 790.0, 0x8, Active, Not Active, Not Active, Not Active, 98",
    ]
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    cs = bench.ClockSampler(None)
    cs.proc, cs.path = _Done(), str(p)
    out = cs.stop()
    assert out["sm_mhz"] == 2055.0  # median of the three samples at >= 50 % utilisation
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown", "sw_power_cap"]
    assert out["samples"] == 4 and out["samples_under_load"] == 3
    assert out["power_w_max"] == 800.0
