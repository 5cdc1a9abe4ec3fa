"""The allocation-free block solve (blm_block_solve_noalloc) against the regular entry point.

Some callers cannot allocate device memory when they need a block solved (a VMC program that
reserves the whole device up front, code that must avoid cudaMalloc's implicit
synchronisation).  The allocation-free entry point runs the same solver on a caller-supplied
block problem with a static workspace inside the library; its eigenvalues and directions must
match what blm_block_solve / blm_get_block report for the same block, on two calls in a row
(the second call reuses the workspace the first one left behind).

This file is collected last on purpose; it passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

import synth
from tests.parity import eig_err, subspace_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("n,nb,k", [(200, 4, 5), (512, 2, 20)])
def test_noalloc_block_solve_matches_block_solve(torch_cuda, n, nb, k):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    dev = torch.device("cuda:0")
    wl = synth.Workload("t", n, 6000, synth.equal_blocks(n, nb), k, decades=5.0, chunk=6000, seed=21)
    O, G, E = (torch.from_numpy(a).to(dev) for a in synth.samples(wl))
    step = blm.Step(n, wl.block_offsets, k)
    step.accumulate(O, G, E)
    step.block_solve()
    for b in range(nb):
        S, H, lam_ref, B_ref = step.block(b)
        dim = S.shape[0]
        assert dim <= blm.blm_noalloc_max_dim()
        dS = torch.from_numpy(S).to(dev)
        dH = torch.from_numpy(H).to(dev)
        for call in range(2):
            lam = torch.full((k,), np.nan, dtype=torch.float64, device=dev)
            B = torch.full((k, dim - 1), np.nan, dtype=torch.float64, device=dev)
            blm.blm_block_solve_noalloc(dS, dH, dim, k, lam, B)
            lam_h, B_h = lam.cpu().numpy(), B.cpu().numpy()
            assert eig_err(lam_h, lam_ref) < 1e-9, (b, call)
            assert subspace_err(B_h, B_ref) < 1e-8, (b, call)
            np.testing.assert_allclose(np.linalg.norm(B_h, axis=1), 1.0, atol=1e-12)
    step.close()


def test_noalloc_rejects_sizes_beyond_its_workspace(torch_cuda):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    dim = blm.blm_noalloc_max_dim() + 1
    z = torch.zeros((dim, dim), dtype=torch.float64, device="cuda:0")
    out = torch.zeros((4, dim), dtype=torch.float64, device="cuda:0")
    with pytest.raises(blm.BLMError) as e:
        blm.blm_block_solve_noalloc(z, z, dim, 2, out, out)
    assert e.value.status == blm.BLM_ERR_ARG
