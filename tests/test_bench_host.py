"""Host logic of bench.py that needs no GPU: the gate that lets the bench
report a kernel's measured DRAM traffic only while the kernel's source is the
one the counters were taken from, and the FP64 peak it divides by."""
import json
import os

import bench


def _write_profile(root, name, sources, sha, traffic=12345):
    os.makedirs(os.path.join(root, "profiles"), exist_ok=True)
    with open(os.path.join(root, "profiles", name + ".json"), "w") as f:
        json.dump({"traffic_bytes_per_launch": traffic, "source_sha256": sha, "sources": sources}, f)


def test_traffic_gate_follows_the_kernel_source(tmp_path, monkeypatch):
    root = str(tmp_path)
    monkeypatch.setattr(bench, "ROOT", root)
    src = tmp_path / "k.cu"
    src.write_text("__global__ void k(float* x) {\n    x[0] = 1.0f;   // store\n}\n\n// tail\nint host_part;\n")
    sources = [{"path": "k.cu", "until": "// tail"}]
    _write_profile(root, "k_prof", sources, bench.source_sha256(sources))
    assert bench.profiled_traffic("k_prof") == 12345
    # comments, trailing blanks, empty lines and text past the marker do not count
    src.write_text("__global__ void k(float* x) {   \n\n    x[0] = 1.0f;   // the store\n}\n// tail\nint other;\n")
    assert bench.profiled_traffic("k_prof") == 12345
    # a change of code does
    src.write_text("__global__ void k(float* x) {\n    x[0] = 2.0f;\n}\n// tail\n")
    assert bench.profiled_traffic("k_prof") is None
    # a missing or malformed profile reports nothing
    assert bench.profiled_traffic("absent") is None
    with open(os.path.join(root, "profiles", "bad.json"), "w") as f:
        f.write("{")
    assert bench.profiled_traffic("bad") is None
    _write_profile(root, "nosrc", [{"path": "gone.cu"}], "0" * 64)
    assert bench.profiled_traffic("nosrc") is None


def test_profile_files_name_their_sources_and_traffic():
    # every committed traffic record lists existing source files and a byte count
    pdir = os.path.join(bench.ROOT, "profiles")
    names = [f for f in os.listdir(pdir) if f.endswith(".json")]
    assert names
    for f in names:
        prof = json.load(open(os.path.join(pdir, f)))
        assert int(prof["traffic_bytes_per_launch"]) > 0
        assert len(prof["source_sha256"]) == 64
        for s in prof["sources"]:
            assert os.path.isfile(os.path.join(bench.ROOT, s["path"])), s["path"]


def test_fp64_peak_from_unit_counts():
    # 152 SMs x 2 FP64 lanes x 2 flops x 2.07 GHz: the nominal dense FP64 rate
    assert abs(bench.fp64_peak_tflops() - 1.25856) < 1e-9
    assert abs(bench.fp64_peak_tflops(1000.0) - 0.608) < 1e-9
