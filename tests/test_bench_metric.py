"""The bench's metric: useful FLOP per sample of both sweeps, 3 sum_b M_b^2 (first sweep: S
symmetric, H full) + 4 n K + 3 (N_B K)^2 (second sweep), against the per-configuration totals
of the measurement plan (first / second sweep over all samples)."""
import pytest

import bench
import synth


@pytest.mark.parametrize("name,ns,pass1,pass2", [
    ("n200", 20000, 6.0e8, 1.0e8),
    ("n2048", 200000, 1.57e11, 3.2e10),
    ("n16384", 1000000, 1.26e13, 6.2e12),
])
def test_useful_flop_matches_the_plan(name, ns, pass1, pass2):
    wl = synth.workload(name)
    assert wl.n_samples == ns
    m = [wl.block_offsets[b + 1] - wl.block_offsets[b] for b in range(wl.n_blocks)]
    p1 = sum(3 * mb * mb for mb in m) * ns
    total = bench.useful_flop_per_sample(wl) * ns
    assert p1 == pytest.approx(pass1, rel=0.02)
    assert total - p1 == pytest.approx(pass2, rel=0.04)
