"""Host-side measurement logic of bench.py (no GPU): the algorithmic byte model,
the traffic record's source-hash gate, the clock / throttle-reason parsing, the
sign-error closed form and the JSON line of the oracle (reference) arm."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_byte_model():
    # two passes, each reading its input spinor and all links once: 120 w_s + 16 r w_g / Ls
    assert bench.bytes_per_site(4, 4, 16) == 552.0
    assert bench.bytes_per_site(8, 8, 16) == 1104.0
    n5 = 16 ** 3 * 32 // 2 * 16
    assert n5 * bench.bytes_per_site(4, 4, 16) == 578813952.0


def test_traffic_record_is_gated_by_source_hash(tmp_path, monkeypatch):
    rec = {"kernel_hash": bench.kernel_hash(), "dram_bytes_per_apply_full_size": 123}
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "dbb_apply_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: rec["kernel_hash"])
    assert bench.measured_traffic() == 123
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.measured_traffic() is None


def test_clock_parsing():
    rows = [
        "0, 2070, 2070, 980.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1001.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage",
    ]
    c = bench.parse_clock_samples(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c = bench.parse_clock_samples(["0, 1400, 2070, 700, 0x8, Active, Not Active, Not Active, Not Active"])
    assert c["reasons"] == ["hw_slowdown"] and c["sm_mhz"] == 1400.0
    assert bench.parse_clock_samples([]) is None


def test_sign_error_matches_zolotarev_ripple():
    """The sign-approximation error used to match Ls in --zolo-projection equals the
    equal-ripple maximum of the Zolotarev coefficients, and for constant a_i = 2
    (Mobius b + c = 2) it is the closed form at the interval ends:
    1 - R(x) = 2 q^L / (1 + q^L), q = |1 - 2x| / (1 + 2x)."""
    import numpy as np
    from synthetic import zolotarev_sign_coefficients
    a, delta = zolotarev_sign_coefficients(8, 0.05, 6.0)
    assert abs(bench.sign_error(a) - delta) < 1e-3 * delta
    L = 16
    q = [abs(1 - 2 * x) / (1 + 2 * x) for x in (0.05, 6.0)]
    closed = max(2 * v ** L / (1 + v ** L) for v in q)
    assert abs(bench.sign_error(np.full(L, 2.0)) - closed) < 1e-6 * closed


def test_reference_arm_json_contract():
    """bench.py --impl reference (the oracle arm) prints one JSON line with the
    contract's keys on rank 0 and nothing on the other ranks."""
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "3"]
    out = subprocess.run(cmd, check=True, capture_output=True, text=True, cwd=ROOT).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["cpu_baseline"]["value"] == d["value"]
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    other = subprocess.run(cmd, check=True, capture_output=True, text=True, cwd=ROOT, env=env)
    assert other.stdout.strip() == ""
