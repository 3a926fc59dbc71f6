"""Host-side parts of bench.py that decide whether a bench line is accepted:
the clock record taken during the timed region (median SM clock, maximum,
throttle reasons) and the algorithmic-byte counts behind the roofline
fractions.  No GPU is used."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler_with(lines):
    s = bench.ClockSampler(0)
    fd, s.path = tempfile.mkstemp(suffix=".csv")
    with os.fdopen(fd, "w") as f:
        f.write("\n".join(lines) + "\n")
    return s


def test_clock_summary_median_maximum_and_reasons():
    # index, sm, max sm, power, active, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    s = _sampler_with([
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ])
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3
    assert not os.path.exists(s.path)


def test_clock_summary_flags_thermal_slowdown():
    s = _sampler_with(["0, 1500, 2070, 800, 0x20, Not Active, Active, Active, Not Active"])
    out = s.summary()
    assert out["reasons"] == ["hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1500.0


def test_clock_summary_without_samples():
    s = _sampler_with([])
    assert s.summary()["reasons"] == ["unsampled"]
    s2 = bench.ClockSampler(0)
    assert s2.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}


def test_algorithmic_bytes_of_the_benchmark_plate():
    """The 100x150x4.4 mm plate (393,216 hexes, 344,064 interfaces, 771,807
    nodes, 24,897 surface nodes): per hex 32 B connectivity + 1 B ply + 448 B
    of history read and written, per node 24 B; a whole step as stated in
    bench.step_alg_bytes."""
    assert bench.hex_alg_bytes(393216, 771807) == 393216 * 481 + 771807 * 24 == 207660264
    assert bench.coh_alg_bytes(344064) == 344064 * 64
    assert bench.step_alg_bytes(393216, 344064, 771807, 24897) == (
        393216 * 481 + 344064 * 64 + 771807 * 141 + 24897 * 48)


def test_algorithmic_bytes_of_a_loaded_window():
    """The 400x600x32 plate in its loaded window: per hex 32 B connectivity,
    1 B ply, the pristine flag read and written (2 B), history bytes (448 B)
    only for the elements that left the initial state; per node 24 B."""
    assert bench.hex_alg_bytes_state(7680000, 11327047, 145) == (
        7680000 * 35 + 145 * 448 + 11327047 * 24) == 540714088
    assert bench.step_alg_bytes_state(393216, 8, 344064, 0, 771807, 24897) == (
        393216 * 35 + 8 * 448 + 344064 * 34 + 771807 * 141 + 24897 * 48)


def test_issue_bound_of_a_launch():
    """566.0 M warp instructions at 2,070 MHz on 152 SMs with four
    schedulers each: 0.450 ms."""
    assert bench.issue_bound_ms(566001765, 2070.0) == pytest.approx(566001765 / (152 * 4 * 2.07e9) * 1e3)
    assert bench.issue_bound_ms(566001765, 2070.0) == pytest.approx(0.4497, abs=1e-4)


def test_algorithmic_bytes_of_one_division():
    """The AS4/8552 coupon divided once: coarse mesh read once, divided mesh
    written once (25 B per node, 33 B per hex, 32 B per interface, 4 B per
    surface node)."""
    coarse = (433680, 228528, 171396, 28912)
    nn1, ns1 = 2643965, 114955
    got = bench.mmu_alg_bytes(*coarse, nn1, ns1)
    want = (433680 * 25 + 228528 * 33 + 171396 * 32 + 28912 * 4) + (
        nn1 * 25 + 8 * 228528 * 33 + 4 * 171396 * 32 + ns1 * 4)
    assert got == want == 172812769


def test_bench_help_runs_without_a_gpu():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--help"], capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and "--workload" in r.stdout


def test_traffic_record_hash_covers_the_hex_kernel_only():
    """The stored k_hex DRAM-traffic record is keyed by a hash of the source
    k_hex is compiled from: the element sections of the item bodies count,
    the contact, interface, tail and gather sections do not."""
    with open(os.path.join(ROOT, "paper_2301_05552_gb300", "csrc", "pdn_items.cuh"), encoding="utf-8") as f:
        text = f.read()
    kept = bench.hex_sections(text)
    for name in ("element_slots", "hex_box_pairs_core", "hex_item_box_pairs", "hex_item("):
        assert name in kept
    for name in ("contact_item", "coh_item", "tail_block", "gather_item"):
        assert name in text and name not in kept
    assert len(bench.kernel_source_hash()) == 16


def test_bench_functions_use_only_defined_names():
    """Every name a function of bench.py reads is a parameter, a local, a
    module-level name or a builtin (the GPU legs cannot run here, so a name
    left behind by an edit would otherwise surface only on the GPU)."""
    import ast
    import builtins

    src = open(os.path.join(ROOT, "bench.py"), encoding="utf-8").read()
    tree = ast.parse(src)
    module = set()
    for n in tree.body:
        if isinstance(n, (ast.FunctionDef, ast.ClassDef)):
            module.add(n.name)
        elif isinstance(n, (ast.Import, ast.ImportFrom)):
            module.update((a.asname or a.name).split(".")[0] for a in n.names)
        elif isinstance(n, (ast.Assign, ast.AnnAssign)):
            for t in (n.targets if isinstance(n, ast.Assign) else [n.target]):
                module.update(m.id for m in ast.walk(t) if isinstance(m, ast.Name))
    missing = []
    for fn in [n for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)]:
        local = set()
        for n in ast.walk(fn):
            if isinstance(n, ast.arg):
                local.add(n.arg)
            elif isinstance(n, ast.Name) and isinstance(n.ctx, (ast.Store, ast.Del)):
                local.add(n.id)
            elif isinstance(n, ast.FunctionDef):
                local.add(n.name)
            elif isinstance(n, (ast.Import, ast.ImportFrom)):
                local.update((a.asname or a.name).split(".")[0] for a in n.names)
            elif isinstance(n, ast.ExceptHandler) and n.name:
                local.add(n.name)
        for n in ast.walk(fn):
            if isinstance(n, ast.Name) and isinstance(n.ctx, ast.Load):
                if n.id not in local and n.id not in module and not hasattr(builtins, n.id):
                    missing.append(f"{fn.name}:{n.lineno}:{n.id}")
    assert not missing, missing


def test_kernels_per_pass():
    """Four kernels a pass with node pairs or the mixed element kernel,
    five with a separate interface kernel, four without interfaces."""
    assert bench.kernels_per_pass({"coh_pairs": 2, "hex_variant": 0}, 100) == 4
    assert bench.kernels_per_pass({"coh_pairs": 0, "hex_variant": 0}, 100) == 5
    assert bench.kernels_per_pass({"coh_pairs": 0, "hex_variant": 5}, 100) == 4
    assert bench.kernels_per_pass({"coh_pairs": 0, "hex_variant": 0}, 0) == 4
