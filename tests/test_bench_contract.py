"""bench.py keeps its output contract: one JSON line with the required keys
(the reference arm here, on CPU; our arm in tests/test_gpu_bench_contract.py),
and a clock record taken from the samples of the timed region."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in out, k
    assert out["impl"] == "reference" and out["value"] > 0 and out["higher_is_better"] is True
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] >= 1
    assert "workload" in out["config"]


def test_clock_samples_are_filtered_and_parsed():
    # The clock record of the bench line: only samples inside the timed
    # region (plus one sampling period), the median SM clock, and the
    # throttle reasons reported Active in any of them; malformed lines skipped.
    import bench

    class FakeProc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c = bench.Clocks(0)
    c.p = FakeProc()
    row = lambda sm, hw="Not Active", pc="Not Active": "0, %d, 2070, 900.0, 0x0, %s, Not Active, Not Active, %s" % (
        sm, hw, pc)
    c.lines = [(0.5, row(1000, hw="Active")),          # before the timed region: ignored
               (1.0, row(2070)), (1.1, row(1995, pc="Active")), (1.2, row(2070)), (1.25, "garbage"),
               (1.3, row(2040)), (2.5, row(900, hw="Active"))]   # after it: ignored
    out = c.stop(1.0, 1.3)
    assert out == {"sm_mhz": 2055.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    c.lines = [(5.0, row(1900))]                       # nothing inside: every sample is used
    assert bench.Clocks.stop(c, 1.0, 1.3)["samples"] == 1


def test_profile_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    # roofline.traffic comes from the committed ncu summary only while the
    # evaluation kernel's source (comments and blank lines aside) is the one
    # that was profiled.
    import shutil
    import bench
    src = tmp_path / "paper_2209_13168_gb300" / "csrc"
    src.mkdir(parents=True)
    for f in ("dd_kernels.cu", "dd_internal.cuh"):
        shutil.copy(os.path.join(ROOT, "paper_2209_13168_gb300", "csrc", f), src / f)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.kernel_hash()
    (tmp_path / "profiles" / "k_eval_config2.json").write_text(
        json.dumps({"kernel_source_sha256": h, "dram_bytes_per_launch": 123.0}))
    assert bench.profile_traffic(bench.kernel_hash()) == 123.0
    k = src / "dd_kernels.cu"
    k.write_text(k.read_text() + "\n// a comment\n\n")             # comments do not count
    assert bench.kernel_hash() == h
    k.write_text(k.read_text() + "static int changed;\n")           # code does
    assert bench.kernel_hash() != h and bench.profile_traffic(bench.kernel_hash()) is None


def test_clock_sampler_names_the_visible_gpu_not_the_rank():
    # nvidia-smi numbers GPUs physically and ignores CUDA_VISIBLE_DEVICES: the
    # sampled GPU is named by the device's UUID, else by the visible-devices
    # entry the local rank maps to, and only without either by the index.
    import bench
    u = "58e7a8b3-1c2d-4e5f-8a9b-0c1d2e3f4a5b"
    assert bench.nvsmi_gpu_id(u, "3,5", 1) == "GPU-" + u
    assert bench.nvsmi_gpu_id("GPU-" + u, None, 0) == "GPU-" + u
    assert bench.nvsmi_gpu_id(None, "3,5", 1) == "5"
    assert bench.nvsmi_gpu_id(None, "GPU-abc,GPU-def", 0) == "GPU-abc"
    assert bench.nvsmi_gpu_id(None, None, 2) == "2"
    assert bench.nvsmi_gpu_id(None, "", 0) == "0"
