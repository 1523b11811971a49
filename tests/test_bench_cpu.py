"""The benchmark's JSON contract on the CPU: the reference arm (the FP64
oracle on a bounded sample of the workload) prints one line with the keys
the driver reads, on the same metric, unit and workload as the GPU arm."""
import json
import subprocess
import sys
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["config"]["workload"] == bench.WORKLOAD_TEXT
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_hop_byte_model():
    """compulsory bytes V/2 (8 L_p + 2 S_p), the effective count V/2 (8 L_p + 9 S_p)"""
    import bench
    vh = 1000
    # SU(3) sextet FP32: L_p = 36 * 8, S_p = 24 * 8
    assert bench.hop_bytes(6, False, 1, vh) == vh * (8 * 288 + 2 * 192)
    assert bench.hop_bytes(6, False, 1, vh, 8) == vh * (8 * 288 + 9 * 192)
    # adjoint links are real: L_p = 64 * 4 in FP32
    assert bench.hop_bytes(8, True, 1, vh) == vh * (8 * 256 + 2 * 256)
    # F16 spinors carry a 4-byte scale
    assert bench.hop_bytes(6, False, 2, vh) == vh * (8 * 144 + 2 * (96 + 4))


def test_link_and_spinor_bytes():
    """bytes a launch reads per link and per spinor, by link mode and precision"""
    import bench
    # rebuilt links read the N x N fundamental link: SU(3) FP32 72 B, FP64 144 B
    assert bench.link_bytes(3, 6, "SYM", 1, True) == 72
    assert bench.link_bytes(3, 8, "ADJ", 0, True) == 144
    # stored: D_R^2 complex, or D_R^2 real for the adjoint
    assert bench.link_bytes(3, 6, "SYM", 1, False) == 288
    assert bench.link_bytes(3, 8, "ADJ", 2, False) == 128
    assert bench.link_bytes(4, 6, "ASYM_REAL", 1, False) == 144
    assert bench.spinor_bytes(6, 3) == 4 * 6 * 4 + 4
    assert bench.spinor_bytes(8, 0) == 4 * 8 * 16
