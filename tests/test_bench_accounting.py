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
    tc = shells * (Nph // 2) * bench.tc_slice_products(2 * Nth) + rings * bench.tc_slice_products(Nph)
    assert bench.tc_tensor_flops(g) == pytest.approx(tc, rel=1e-12)


def test_tc_slice_products_counts_the_four_gemms():
    """Length L = 8 (H = 4): cos forward 4 x 5, sin forward 3 x 3, the same two inverse; 21 slice
    pairs, 2 flops per multiply-add."""
    assert bench.tc_slice_products(8) == 21 * 2 * (4 * 5 + 3 * 3 + 4 * 5 + 3 * 3)


def test_traffic_record_names_known_families():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    assert set(rec["families"]) <= set(bench.KERNEL_FAMILIES)
    for fam, entry in rec["families"].items():
        assert len(entry["sources_sha256_16"]) == 16
        for key, val in entry.items():
            if key != "sources_sha256_16":
                prec, wl = key.split(":")
                assert prec in ("f64", "f32x2", "tc")
                assert bench.single_grid_workload(wl).name == wl  # a workload bench.py runs
                assert isinstance(val, int) and val > 0
    for fam in bench.KERNEL_FAMILIES:
        assert len(bench.kernel_sources_hash(fam)) == 16
