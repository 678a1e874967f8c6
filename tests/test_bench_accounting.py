"""The benchmark's algorithmic accounting (CPU): which shells and rings a pass transforms, and the
flop counts built on that, against the oracle's own cutoff functions (Sec. II.C); the recorded
DRAM-traffic file's structure."""
import json
import math
import os

import numpy as np
import pytest

import bench
import oracle
from paper_2305_01537_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def active_counts(g):
    """Active theta shells and active rings, from the oracle's l_max and m_max: a pass is the
    identity exactly when every multiplier is 1, i.e. for the exponential and sharp filters with
    cutoff >= the Nyquist mode; the Gaussian filter never is."""
    shells, rings = 0, 0
    for v in range(g.nvars):
        gauss = g.kind[v] == W.GAUSS
        for i in range(g.Nr):
            if gauss or oracle.lmax(g.r[i], g.dr_min, g.L[v], g.floor) < g.Ntheta:
                shells += 1
            for j in range(g.Ntheta):
                if gauss or oracle.mmax(g.r[i], g.dr_min, g.L[v], j, g.Ntheta, g.floor) < g.Nphi / 2:
                    rings += 1
    return shells, rings


@pytest.mark.parametrize("Nr,Nth,Nph", [(6, 8, 16), (12, 16, 32), (40, 8, 24)])
def test_flop_counts_follow_the_oracle_cutoffs(Nr, Nth, Nph):
    g = W.grid_28(Nr, Nth, Nph)
    shells, rings = active_counts(g)
    fft = shells * Nth * Nph * (5 * math.log2(2 * Nth) + 1) + rings * Nph * (5 * math.log2(Nph) + 1)
    assert bench.algorithmic_flops(g) == pytest.approx(fft, rel=1e-12)
    circles, direct = shells * (Nph // 2), (Nph // 2) % 64 == 0
    tc = -(-circles // 64) * bench.tc_tile_flops(2 * Nth, not direct) + -(-rings // 64) * bench.tc_tile_flops(Nph, True)
    assert bench.tc_tensor_flops(g) == pytest.approx(tc, rel=1e-12)


def test_tc_block_shapes():
    """The GEMM shapes of the symmetry-block form: levels while a quarter of the vector is at least 16
    (two halves per GEMM, K = N = the padded quarter), then the base halves side by side."""
    assert bench.tc_blocks(256) == [(64, 64, 1), (32, 32, 1), (16, 16, 1), (16, 32, 1)]
    assert bench.tc_blocks(128) == [(32, 32, 1), (16, 16, 1), (16, 32, 1)]
    assert bench.tc_blocks(16) == [(16, 32, 1)]
    assert bench.tc_blocks(74) == [(48, 48, 2)]  # 37-point halves: two GEMMs (side by side needs 1024 columns)
    # a 128-point tile, factored: 2 x (128 rows x (32x32 + 16x16 + 16x32)) x 21 pairs x 2 flops
    assert bench.tc_tile_flops(128, True) == 2 * 128 * (32 * 32 + 16 * 16 + 16 * 32) * 21 * 2


def test_traffic_record_names_known_families():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert set(rec["families"]) <= set(bench.KERNEL_FAMILIES)
    for fam, entry in rec["families"].items():
        assert len(entry["sources_sha256_16"]) == 16
        for key, val in entry.items():
            if key != "sources_sha256_16":
                prec, wl = key.split(":")
                assert prec in bench.PRECISIONS
                assert bench.single_grid_workload(wl).name == wl  # a workload bench.py runs
                assert isinstance(val, int) and val > 0
    for fam in bench.KERNEL_FAMILIES:
        assert len(bench.kernel_sources_hash(fam)) == 16
