"""The byte and flop models behind bench.py's roofline and HBM fractions,
rebuilt here from the arrays each kernel touches (numpy sizes), at the
256x256x4 benchmark film (padded 512x512x8)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

GRID = (256, 256, 4)


def _arrays():
    nx, ny, nz = GRID
    M = np.zeros((3, nz, ny, nx), np.float32)                     # magnetisation, SoA FP32
    S = np.zeros((nx + 1, 3, nz, ny), np.complex64)               # x half-spectrum, 3 components
    Ks = np.zeros((nx + 1, ny + 1, nz + 1, 6), np.float32)        # tensor octant (padded 512 x 512 x 8)
    Kd = np.zeros((nx + 1, nz, 6, ny + 1), np.float32)            # 2-D spectrum per z offset
    return M, S, Ks, Kd


def test_bytes_of_the_two_kernel_step():
    M, S, Ks, Kd = _arrays()
    b = bench.algorithmic_bytes(GRID)
    # K_A: S in, Sh out, the 2-D spectrum once; K_B: Sh in, S out, M in and out
    assert b["kA"] == 2 * S.nbytes + Kd.nbytes == 18972768
    assert b["kB"] == 2 * S.nbytes + 2 * M.nbytes
    assert b["step2"] == b["kA"] + b["kB"] == 37896288
    assert b["floor2"] == 2 * M.nbytes + Kd.nbytes == 12632160


def test_bytes_of_the_three_pass_model():
    M, S, Ks, Kd = _arrays()
    b = bench.algorithmic_bytes(GRID)
    assert b["pass1"] == M.nbytes + S.nbytes
    assert b["plane3"] == 2 * S.nbytes + Ks.nbytes
    assert b["pass3"] == S.nbytes + 2 * M.nbytes
    assert b["step3"] == b["pass1"] + b["plane3"] + b["pass3"] == 42627192
    assert b["demag"] == 2 * M.nbytes + 4 * S.nbytes + Ks.nbytes


def test_flop_model_and_alu_peak():
    import math
    nx, ny, nz = GRID
    fft = lambda n: 5 * n * math.log2(n)
    # x: 3 ny nz / 2 row pairs, a forward and an inverse pruned length-2nx
    # transform each (two length-nx FFTs); y: 3 nz (nx + 1) lines, forward and
    # inverse pruned length 2ny; z: 9 nz^2 real-by-complex multiply-adds per
    # (kx, ky) bin; 100 flops per cell for the field and the update
    want = (2 * (3 * ny * nz // 2) * 2 * fft(nx) + 2 * (3 * nz * (nx + 1)) * 2 * fft(ny)
            + (nx + 1) * 2 * ny * 9 * nz * nz * 4 + 100 * nx * ny * nz)
    assert bench.algorithmic_flops(GRID) == want == 291241984
    assert abs(bench.alu_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9


def test_recorded_traffic_only_for_the_captured_kernel_sources(tmp_path):
    """roofline.traffic comes from an ncu capture committed under profiles/;
    it is reported only while the step kernels' sources hash to the value
    recorded with that capture, and is null once they change."""
    import json
    f = tmp_path / "traffic.txt"
    f.write_text(json.dumps({"kA_plane_y_zsum_product": 1.5e7, "kernel_sources_sha16": bench.step_kernel_hash()}))
    assert bench.recorded_traffic("kA_plane_y_zsum_product", str(f)) == 1.5e7
    f.write_text(json.dumps({"kA_plane_y_zsum_product": 1.5e7, "kernel_sources_sha16": "0" * 16}))
    assert bench.recorded_traffic("kA_plane_y_zsum_product", str(f)) is None
    f.write_text(json.dumps({"kA_plane_y_zsum_product": 1.5e7}))
    assert bench.recorded_traffic("kA_plane_y_zsum_product", str(f)) is None


def test_batch_byte_model_uses_the_plan_lengths():
    """bench.batch_bytes: the three-pass and fused byte models summed over
    samples, with the padded lengths of the plan (restated in the tests'
    helpers independently)."""
    from tests._helpers import padded_length
    for n in list(range(1, 300)) + [512, 1000, 2048]:
        assert bench.padded_length(n) == padded_length(n), n
    grids = [(256, 256, 4), (200, 60, 3), (17, 33, 1)]
    by = bench.batch_bytes(grids)
    g3 = sum(bench.algorithmic_bytes(g)["step3"] for g in grids[:1])
    assert by["three_pass"] > g3 and by["persistent"] == by["graph"] < by["three_pass"]
    nx, ny, nz = 200, 60, 3
    X = (400 // 2 + 1) * ny * nz
    Ks = (400 // 2 + 1) * (120 // 2 + 1) * (5 // 2 + 1)          # Lz = 5 for nz = 3
    one = bench.batch_bytes([(nx, ny, nz)])
    assert one["three_pass"] == 36 * nx * ny * nz + 96 * X + 24 * Ks
    assert one["three_pass"] - one["graph"] == 12 * nx * ny * nz


def test_bench_truncation_floor_equals_the_oracle_floor():
    """The surrogate workload measures the FNO truncation floor of its
    training targets with torch on the device; it is the oracle's floor."""
    import torch
    from oracle import fno as F
    rng = np.random.default_rng(4)
    for H, W, m in ((32, 40, 6), (16, 16, 8), (64, 48, 5)):
        h = rng.standard_normal((2, 3, H, W))
        assert abs(bench.truncation_floor(torch.from_numpy(h), m) - F.truncation_floor(h, m)) < 1e-12
