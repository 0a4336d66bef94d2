"""Host-side pieces of bench.py that decide what the JSON line reports (CPU only).

The algorithmic byte counts are the roofline denominators, so they are pinned
here against the pipeline written out by hand (what each pass must read and
write at least); the traffic figure is only reported for the sources it was
measured on; the CPU baseline block carries the fields the report needs.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_pass_bytes_at_256_cubed():
    """Per pass, counted by hand at 256^3 (complex 8 B, real 4 B):
    P1 reads rho (256^3 real) and writes one half spectrum Z = 257 x 256 x 256 complex;
    P2 reads Z and writes it padded to 512 rows (2Z); P3 reads 2Z and the 257^3 kernel
    octant and writes two 2Z streams; P4 reads those and writes three Z; P5 reads them and
    writes phi and three field components (4 x 256^3 real)."""
    n = 256
    Z = 257 * 256 * 256 * 8
    cells = n ** 3
    want = {
        "p1_fwd": 4 * cells + Z,
        "p2_fwd": Z + 2 * Z,
        "p3_fwd": 2 * Z + 4 * 257 ** 3 + 2 * 2 * Z,
        "p4_fwd": 2 * 2 * Z + 3 * Z,
        "p5_fwd": 3 * Z + 4 * 4 * cells,
    }
    got = bench.pass_bytes((n, n, n), True)
    assert got == want
    assert sum(got.values()) == 3098283012
    # about 184 n^3, the figure the roofline fraction is quoted against
    assert abs(sum(got.values()) / n ** 3 - 184) < 1.0


def test_pass_bytes_phi_only_is_smaller():
    full = bench.pass_bytes((64, 64, 64), True)
    phi = bench.pass_bytes((64, 64, 64), False)
    assert all(phi[k] <= full[k] for k in full) and sum(phi.values()) < sum(full.values())


def test_traffic_is_reported_only_for_the_measured_sources(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    (prof / "traffic.json").write_text(json.dumps({"vgf256": {"p3_fwd": {"dram_bytes": 123, "source_hash": "abc"}}}))
    assert bench.ncu_traffic("p3_fwd", "vgf256") == 123
    (prof / "traffic.json").write_text(json.dumps({"vgf256": {"p3_fwd": {"dram_bytes": 123, "source_hash": "old"}}}))
    assert bench.ncu_traffic("p3_fwd", "vgf256") is None
    assert bench.ncu_traffic("p4_fwd", "vgf256") is None


def test_cpu_baseline_block_fields():
    pytest.importorskip("oracle")
    b = bench.cpu_baseline_block(16, 16, full_n=16)
    for key in ("value", "unit", "cores", "kind", "sample", "cpu", "single_thread", "scaled_sample"):
        assert key in b
    assert b["kind"] == "oracle" and b["cores"] >= 1 and b["value"] > 0
    assert b["single_thread"]["cores"] == 1 and b["single_thread"]["value"] > 0
    times, cores = bench.oracle_headline(5, budget_s=0.0, n=16)
    assert len(times) == 1 and cores >= 1   # the budget stops after the first timed solve


def test_padded_fft_context_solve_matches_oracle():
    """The torch.fft context solve in bench.py is the same discrete convolution as the oracle's."""
    import numpy as np
    import torch
    oracle = pytest.importorskip("oracle")
    oracle.build()
    shape, h = (10, 12, 8), (0.07, 0.05, 0.09)
    rho = np.random.default_rng(3).standard_normal(shape)
    g = oracle.kernel_vgf(list(shape), h)
    octant = torch.from_numpy(oracle.scaled_spectrum_octant(g, h))
    phi, E = bench.padded_fft_solve(octant, torch.from_numpy(rho), h)
    p_ref, E_ref = oracle.solve_with_kernel(g, rho, h)
    assert np.max(np.abs(phi.numpy() - p_ref)) <= 1e-12 * np.max(np.abs(p_ref))
    assert np.max(np.abs(torch.stack(E).numpy() - E_ref)) <= 1e-12 * np.max(np.abs(E_ref))


def test_compulsory_bytes_at_256_cubed():
    """rho (4 n^3) + the kernel octant (4 x 257^3) + phi and three field components (16 n^3): about 24 n^3."""
    n = 256
    assert bench.compulsory_bytes((n, n, n)) == 4 * n ** 3 + 4 * 257 ** 3 + 16 * n ** 3 == 403442692
    assert bench.compulsory_bytes((n, n, n), False) == 8 * n ** 3 + 4 * 257 ** 3
    # 2D: rho, the (n+1)^2 kernel quadrant, phi and two field components
    assert bench.compulsory_bytes((4096, 4096)) == 16 * 4096 ** 2 + 4 * 4097 ** 2


def test_pipeline_flops_by_line_count():
    """At 256^3 every transform has padded length 512 (5 * 512 * 9 = 23040 flops per complex line):
    65536 real R2C lines, 65792 forward lines along y, 3 x 131584 lines along z (one forward, two
    inverse streams), 3 x 65792 inverse lines along y, 4 x 65536 real C2R lines; about 1.9e10."""
    c = 23040
    want = 65536 * c / 2 + 65792 * c + 3 * 131584 * c + 3 * 65792 * c + 4 * 65536 * c / 2
    got = bench.pipeline_flops((256, 256, 256))
    assert got == want == 18933350400
    # 2D 4096^2: lengths 8192 (5 * 8192 * 13 = 532480): 4096 R2C lines, 3 x 4097 lines in the fused pass,
    # 3 x 4096 C2R lines
    c2 = 532480
    assert bench.pipeline_flops((4096, 4096)) == 4096 * c2 / 2 + 3 * 4097 * c2 + 3 * 4096 * c2 / 2
    assert bench.pipeline_flops((64, 64, 64), False) < bench.pipeline_flops((64, 64, 64))


def test_pass_flops_split_and_alu_peak():
    """Per-pass flops sum to the pipeline count; the middle pass carries three of the 512-point
    transforms per line (9.1e9 at 256^3); the FP32 peak is SMs x 128 x 2 x clock (152 SMs at 2.07 GHz:
    80.5 TFLOP/s), with the clock taken from the samples when there are any."""
    f = bench.pass_flops((256, 256, 256))
    assert set(f) == set(bench.pass_bytes((256, 256, 256)))
    assert sum(f.values()) == bench.pipeline_flops((256, 256, 256))
    assert f["p3_fwd"] == 3 * 257 * 512 * 23040
    assert abs(bench.fp32_peak_tflops(152, 2070) - 80.54784) < 1e-9
    a = bench.alu_check("p3_fwd", f["p3_fwd"], 0.25, 152, 2070.0, "test")
    assert abs(a["tflops"] - f["p3_fwd"] / 0.25e-3 / 1e12) < 1e-9 and 0 < a["frac"] < 1
    assert abs(a["peak_tflops"] - 80.54784) < 1e-9
    assert bench.alu_clock({"sm_mhz": 1800.0, "sm_max_mhz": 2070.0})[0] == 1800.0
    assert bench.alu_clock(None)[0] == 2070.0
    f2 = bench.pass_flops((4096, 4096))
    assert set(f2) == set(bench.pass_bytes_2d((4096, 4096))) and sum(f2.values()) == bench.pipeline_flops((4096, 4096))
