"""The tile autotuner (blm_autotune) and its candidates (blm_set_tiles) on the split-precision
paths: every candidate -- per-block tiles or packed band tiles, long or short work units --
gives the same step, within the mixed-path tolerances, against the FP64 oracle; the tuner picks
one of them and the step it leaves behind starts afresh.  Blocks of 20-70 parameters (far smaller
than a 128 x 256 tile) and uneven offsets, where the band layout is the one that can win.
"""
import numpy as np
import pytest

import synth
from oracle import blm_oracle
from tests.parity import matrix_err, mixed_tolerances

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


OFFS = [0, 20, 90, 131, 180, 250, 300, 333, 400, 470, 500]


def _step(blm, torch, prec, O, G, E, choice=None, tune=False):
    n = O.shape[1]
    step = blm.Step(n, OFFS, 6, precision=getattr(blm, prec), input_type=blm.BLM_IN_F32)
    picked = None
    if tune:
        picked = blm.blm_autotune(step.h, O, G, E, None, O.shape[0], n)
    if choice is not None:
        blm.blm_set_tiles(step.h, choice)
    step.accumulate(O, G, E)
    step.block_solve()
    blocks = [step.block(b) for b in range(len(OFFS) - 1)]
    step.project(O, G, E)
    dmu = torch.empty(n, dtype=torch.float64, device="cuda:0")
    e = step.combined_solve(dmu)
    step.close()
    return blocks, e, picked


@pytest.mark.parametrize("prec", ["BLM_PREC_BF16X4", "BLM_PREC_TF32X4"])
def test_every_tile_candidate_gives_the_step(torch_cuda, prec):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    wl = synth.Workload("t", OFFS[-1], 12000, OFFS, 6, decades=4.0, chunk=12000, seed=23)
    O, G, E = synth.samples(wl, dtype=np.float32)
    ref = blm_oracle.blm_step(*(a.astype(np.float64) for a in (O, G, E)), None, OFFS, 6)
    tol_mat, tol_e = mixed_tolerances(O.shape[0])
    tO, tG, tE = (torch.from_numpy(a).to("cuda:0") for a in (O, G, E))
    for choice in range(4):
        blocks, e, _ = _step(blm, torch, prec, tO, tG, tE, choice=choice)
        em = max(matrix_err(S, Sr, H, Hr) for (S, H, _, _), Sr, Hr in
                 zip(blocks, ref["S_b"], ref["H_b"]))
        assert em < tol_mat, (choice, em)
        assert abs(e - ref["e_pred"]) < tol_e, (choice, e, ref["e_pred"])
    blocks, e, picked = _step(blm, torch, prec, tO, tG, tE, tune=True)
    assert picked in (0, 1, 2, 3)
    assert abs(e - ref["e_pred"]) < tol_e, (picked, e)
