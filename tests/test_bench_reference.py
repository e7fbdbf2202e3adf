"""The bench's reference arm (the CPU oracle timed on the host cores) prints one JSON line with the
contract's keys; a short sample keeps it quick (no GPU)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "coupled Gibbs site-updates/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert isinstance(d["cpu_baseline"]["cpu_model"], str) and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]
    assert "workload" in d["config"]


def test_reference_arm_under_torchrun_two_ranks():
    """Launched as the multi-GPU bench is (torchrun, two ranks), rank 0 alone times the oracle and
    prints; the other rank exits 0 without work."""
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    out = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                          "--master-addr", "127.0.0.1", "--master-port", str(port),
                          os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
                          "--warmup", "0", "--ref-seconds", "1"], cwd=ROOT, capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_cpu_model_on_an_arm_host(monkeypatch):
    """Arm kernels name no model in /proc/cpuinfo: the implementer and part codes stand in."""
    import io
    sys.path.insert(0, ROOT)
    import bench
    text = "processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n"
    monkeypatch.setattr(bench, "open", lambda *a, **k: io.StringIO(text), raising=False)
    assert bench.cpu_model() == "implementer 0x41 part 0xd4f"


def test_a_failing_auxiliary_leg_is_reported_in_the_line():
    """A leg beside the main figure that raises leaves its error in the line instead of ending the
    bench; a leg that works returns its own result."""
    sys.path.insert(0, ROOT)
    import bench

    def broken(x):
        raise RuntimeError(f"leg failed at {x}")

    assert bench.auxiliary_leg(lambda x: {"value": x}, 3) == {"value": 3}
    assert bench.auxiliary_leg(broken, 7) == {"error": "RuntimeError: leg failed at 7"}
