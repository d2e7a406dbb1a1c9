"""Host checks of the committed profile summaries and of how bench.py reads
them: every ncu command recorded there leaves the GPU clocks alone, the
summaries are text only, and the DRAM traffic of the benchmark's roofline is
reported only while the kernel source is the one the counters were taken on."""
import hashlib
import os
import re
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")


def _ncu_commands(text):
    joined = re.sub(r"\\\n\s*", " ", text)  # join continuation lines
    return [line.strip() for line in joined.splitlines() if re.match(r"\s*ncu\s", line)]


def test_every_recorded_ncu_command_leaves_the_clocks_alone():
    names = sorted(os.listdir(PROFILES))
    assert names
    n = 0
    for name in names:
        assert name.endswith((".md", ".txt")), name  # summaries, nothing that runs
        for cmd in _ncu_commands(open(os.path.join(PROFILES, name)).read()):
            assert "--clock-control none" in cmd, (name, cmd)
            n += 1
    assert n >= 5


def test_traffic_summaries_exist_and_name_kernel_and_source():
    for fn in bench.TRAFFIC_FILES.values():
        vals = {}
        for line in open(os.path.join(PROFILES, fn)):
            if ":" in line:
                k, v = line.split(":", 1)
                vals.setdefault(k.strip(), v.strip())
        assert int(vals["traffic_bytes_per_launch"]) > 0
        assert re.fullmatch(r"[0-9a-f]{64}", vals["source_sha256"])
        assert vals["kernel"]


def test_traffic_withheld_once_the_source_differs(tmp_path, monkeypatch):
    src = tmp_path / "paper_1308_5299_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "legendre.cu").write_bytes(b"source as profiled\n")
    sha = hashlib.sha256(b"source as profiled\n").hexdigest()
    fn = bench.TRAFFIC_FILES["legendre_adjoint_f64"]
    (tmp_path / "profiles" / fn).write_text(
        "kernel: leg_adjoint_kernel<double, 0, 8, 0, 1>\ntraffic_bytes_per_launch: 1234\nsource_sha256: %s\n" % sha)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    traffic, kernel = bench.profile_traffic("legendre_adjoint_f64")
    assert traffic == 1234.0 and kernel.startswith("leg_adjoint_kernel<double")
    (src / "legendre.cu").write_bytes(b"source changed since\n")
    traffic, kernel = bench.profile_traffic("legendre_adjoint_f64")
    assert traffic is None and "withheld" in kernel
    assert bench.profile_traffic("legendre_synth_f32") == (None, None)
