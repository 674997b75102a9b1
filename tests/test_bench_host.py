"""Host-side parts of bench.py that need no GPU: the clock summary keeps only
the nvidia-smi samples taken inside the timed region, and the DRAM-traffic
record is keyed to the kernel's code (comments and the rest of the C header
do not void it)."""
import datetime
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _ts(t):
    return datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]


def test_clock_summary_keeps_the_timed_region():
    now = time.time()
    lines = [
        f"{_ts(now - 1.0)}, 1200, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        f"{_ts(now + 0.1)}, 2070, 2070, 900.0, 0x4, Not Active, Not Active, Not Active, Active",
        f"{_ts(now + 0.2)}, 2050, 2070, 950.0, 0x4, Not Active, Not Active, Not Active, Active",
        f"{_ts(now + 5.0)}, 900, 2070, 200.0, 0x0, Not Active, Active, Not Active, Not Active",
        "garbage line",
    ]
    inside = bench.ClockSampler.parse(lines, now, now + 1.0)
    assert inside == {"sm_mhz": 2060.0, "sm_max_mhz": 2070.0, "samples": 2,
                      "in_timed_region": True, "reasons": ["sw_power_cap"]}
    # no window: every sample, and the thermal flag of the last one shows
    everything = bench.ClockSampler.parse(lines)
    assert everything["samples"] == 4 and not everything["in_timed_region"]
    assert everything["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    assert bench.ClockSampler.parse([]) is None


def test_traffic_key_ignores_header_comments(tmp_path, monkeypatch):
    files = {}
    for rel in bench.KERNEL_SOURCES["sod32_stage_kernel"]:
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
        files[rel] = dst
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.source_sha("sod32_stage_kernel")
    hdr = files["include/rslb.h"]
    hdr.write_text(hdr.read_text() + "\n/* a comment */\n")
    assert bench.source_sha("sod32_stage_kernel") == base
    dev = files["paper_1612_01287_gb300/csrc/rslb_device.cuh"]
    dev.write_text(dev.read_text().replace("namespace rslb {", "// reworded\n// note\nnamespace rslb {", 1))
    assert bench.source_sha("sod32_stage_kernel") == base
    hdr.write_text(hdr.read_text().replace("#define RSLB_PACKED_TILE_CELLS 28",
                                           "#define RSLB_PACKED_TILE_CELLS 20"))
    assert bench.source_sha("sod32_stage_kernel") != base
    kern = files["paper_1612_01287_gb300/csrc/sod32.cu"]
    kern.write_text(kern.read_text() + "\n")
    assert bench.source_sha("sod32_stage_kernel") != base


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` runs the FP64 oracle on the host cores (no
    GPU, no library build) and prints one JSON line with the arm's keys."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["metric"] == "cell-velocity updates/s" and d["higher_is_better"] is True


def test_recorded_counters_follow_the_current_kernel_sources():
    """Every ncu record the bench reads (DRAM traffic, FP64 operation counts) was
    taken on the kernel source as it stands; a changed kernel voids its record,
    so a stale one would silently drop a roofline key from the bench line."""
    import json
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for kernel, rec in d.items():
        assert rec["source_sha"] == bench.source_sha(kernel), kernel
