"""Host logic of bench.py on CPU: the clock record taken during the timed region and the rule
that rejects a throttled run, the DRAM-traffic record's tie to the kernel sources, the
roofline peak's source, and the garbage-collector pause around timed regions."""
import gc
import json
import os
import shutil

import pytest

import bench


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler_with(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.fh = open(str(tmp_path / "unused.csv"), "w")
    s.proc = _FakeProc()
    return s


def test_clock_record_median_max_and_active_reasons(tmp_path):
    """nvidia-smi csv,noheader,nounits lines: index, clocks.sm, clocks.max.sm, power, the
    active mask, then hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap."""
    lines = ["0, 2070, 2070, 912.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 2055, 2070, 1390.12, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 1201.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "malformed line",
             "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    clk = _sampler_with(tmp_path, lines).stop()
    assert clk == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not bench.clocks_bad(clk)


def test_clock_record_without_samples(tmp_path):
    assert _sampler_with(tmp_path, ["garbage"]).stop()["reasons"] == ["no samples"]
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


@pytest.mark.parametrize("clk,bad", [
    ({"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": []}, False),
    ({"sm_mhz": 1900, "sm_max_mhz": 2070, "reasons": ["sw_power_cap"]}, False),
    ({"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": ["hw_slowdown"]}, True),
    ({"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": ["hw_thermal_slowdown", "sw_power_cap"]}, True),
    ({"sm_mhz": 2070, "sm_max_mhz": 2070, "reasons": ["sw_thermal_slowdown"]}, True),
    ({"sm_mhz": 1000, "sm_max_mhz": 2070, "reasons": []}, True),              # a leftover clock lock
    ({"sm_mhz": 1000, "sm_max_mhz": 2070, "reasons": ["sw_power_cap"]}, False),
    ({"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}, False),
])
def test_throttled_runs_are_rejected(clk, bad):
    assert bench.clocks_bad(clk) is bad


def _tree_with_record(tmp_path, key, nbytes):
    """A copy of the three hashed kernel sources and a traffic record stamped with their
    hash (computed here independently: sha256 over the files in order, first 16 hex)."""
    import hashlib
    root = tmp_path / "root"
    csrc = root / "paper_1308_0692_gb300" / "csrc"
    os.makedirs(csrc)
    os.makedirs(root / "profiles")
    h = hashlib.sha256()
    for name in ("step_kernel.cuh", "step_tma.cuh", "step_march.cuh"):
        shutil.copy(os.path.join(bench.ROOT, "paper_1308_0692_gb300", "csrc", name), csrc / name)
        h.update((csrc / name).read_bytes())
    rec = {key: {"dram_bytes_per_launch": nbytes, "source_sha256_16": h.hexdigest()[:16]}}
    (root / "profiles" / "traffic.json").write_text(json.dumps(rec))
    return root


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    """A record stamped with the sources' hash is reported; editing a kernel source (even a
    comment) or removing the record drops it, and the bench then reports traffic null."""
    key = "step_f32_m12_g6_pf4"
    root = _tree_with_record(tmp_path, key, 4.9e9)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic_record(key) == 4.9e9
    assert bench._traffic_record("no_such_kernel") is None
    with open(root / "paper_1308_0692_gb300" / "csrc" / "step_march.cuh", "a") as f:
        f.write("\n// edited\n")
    assert bench._traffic_record(key) is None
    os.remove(root / "profiles" / "traffic.json")
    assert bench._traffic_record(key) is None


def test_peak_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6791.0, "bf16_tflops": 1900.0}))
    assert bench._peaks() == (6791.0, "measured")


def test_gc_paused_restores_the_collector():
    assert gc.isenabled()
    with bench.gc_paused():
        assert not gc.isenabled()
    assert gc.isenabled()
    with pytest.raises(RuntimeError):
        with bench.gc_paused():
            raise RuntimeError("inside a timed region")
    assert gc.isenabled()
    gc.disable()
    try:
        with bench.gc_paused():
            pass
        assert not gc.isenabled()          # a collector that was off stays off
    finally:
        gc.enable()


def _fake_ttr():
    def run(sec, err, n):
        return {"seconds": sec, "max_err_vs_fp64": err, "checked": n, "speedup_vs_fp64": 100.0 / sec}
    full = {"fp64": {"seconds": 100.0, "steps": [1000] * 256},
            "batch_dc": run(8.0, 2e-6, 256), "warm_dc": run(5.0, 3e-6, 256)}
    sub = {"fp64": {"seconds": 22.0}, "fp64_concurrent": {"seconds": 12.0}, "fp32_dc": {"seconds": 7.0},
           "batch_dc": run(1.0, 1e-6, 32), "warm_dc": run(0.7, 1e-6, 32)}
    return {"held_out_256": full, "ablation_32": sub}


def test_time_to_residual_digest_is_short_and_complete():
    """The digest printed as the bench line's last key (the part of a long line that a
    tail-truncated log keeps): counts, seconds, speed-up and worst error of each variant."""
    d = bench.ttr_summary(_fake_ttr(), oracle_rate=1e9)
    assert d["n"] == 256 and d["checked"] == 256
    assert d["fp64_s"] == 100.0 and d["warm_dc_s"] == 5.0 and d["warm_vs_fp64"] == 20.0
    assert d["warm_dc_max_du"] == 3e-6 and d["batch_dc_max_du"] == 2e-6
    assert d["first32"]["fp32_dc_s"] == 7.0
    assert d["oracle_extrap_s"] == pytest.approx(256 * 1000 * 128 * 128 * 64 / 1e9, rel=1e-3)
    assert len(json.dumps(d)) < 700


def test_oracle_band_one_contiguous_chunk_per_thread():
    """The CPU baseline's sample: a band of middle rows of the 2048^2 workload, split into one
    contiguous run of cells per thread, all chunks together covering the band once."""
    import numpy as np
    band = bench.OracleBand(rows=3, threads=4)
    try:
        cells = np.concatenate(band.chunks)
        assert len(band.chunks) == 4 and band.ncells == 3 * 2048
        np.testing.assert_array_equal(np.diff(cells), 1)
        assert all(len(c) == 3 * 2048 // 4 for c in band.chunks)
        assert band.updates_per_step() == 3 * 2048 * 144
        band.step()
    finally:
        band.close()
