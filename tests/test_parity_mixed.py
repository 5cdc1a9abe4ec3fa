"""GPU parity of the split-BF16 tensor-core path against the FP64 oracle.

The inputs are FP32; the oracle receives the same FP32 values widened to FP64, so the comparison
measures only the path's arithmetic: operands split into bf16 hi + lo (four products, so every
product is exact to ~2^-16 relative and unbiased), FP32 tensor-memory accumulation restarted every
128 samples, FP64 centring and FP64 solves.

Error model.  hi + lo represents each FP32 operand v to |v - hi - lo| <= 2^-16 |v| with a
zero-mean residual (RMS ~ 6e-6 relative); each product carries two such residuals, independent
from sample to sample, so their contribution to a sum over N samples falls as 1/sqrt(N): RMS
~ 2 * 6e-6 * sqrt(3 / N) of the correlation-scaled entry, and the largest of ~10^5 - 10^6 entries
sits ~ 4.5 RMS out.  (Restarting the FP32 tensor-memory accumulator every 64, 128 or 256 samples
gives the same errors to three digits: accumulation is not the limit.)  The targets hold at the
size of the step they are stated for, N = 10^6 samples; for a test sample of N the tolerances are
the targets widened by sqrt(10^6 / N):
  S_b, H_b and the combined matrices (the latter against the oracle's second sweep run with the
  GPU's B^(b)): 1e-6 in correlation scaling (|dA_xy| / sqrt(S_xx S_yy));
  E_pred: 1e-8 Hartree;  Delta mu: 1e-4 relative;
  kept eigenvalues 1e-5 relative and retained subspaces 1e-4 (matrix error times the
  conditioning of the block problem).
The FP64 eigen-solves themselves are held to max(1e-9, 10 x the oracle's sample-order
sensitivity) against LAPACK on the GPU's own matrices.
"""
import numpy as np
import pytest

import synth
from oracle import blm_oracle
from tests.parity import check_step, self_variation

pytestmark = pytest.mark.gpu

TOL_MAT = 1e-6
TOL_EIG = 1e-5
TOL_SUB = 1e-4
TOL_E = 1e-8
TOL_DMU = 1e-4


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_mixed(torch, O, G, E, w, offsets, n_keep, chunks=None):
    import paper_1702_01481_gb300 as blm
    dev = torch.device("cuda:0")
    tO, tG, tE = (torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in (O, G, E))
    tw = torch.from_numpy(np.asarray(w, dtype=np.float32)).to(dev) if w is not None else None
    n = O.shape[1]
    step = blm.Step(n, offsets, n_keep, precision=blm.BLM_PREC_BF16X4, input_type=blm.BLM_IN_F32)
    ns = O.shape[0]
    chunks = chunks or [ns]
    bounds = np.cumsum([0] + list(chunks))
    for a, b in zip(bounds[:-1], bounds[1:]):
        step.accumulate(tO[a:b], tG[a:b], tE[a:b], tw[a:b] if tw is not None else None)
    step.block_solve()
    blocks = [step.block(b) for b in range(len(offsets) - 1)]
    for a, b in zip(bounds[:-1], bounds[1:]):
        step.project(tO[a:b], tG[a:b], tE[a:b], tw[a:b] if tw is not None else None)
    dmu = torch.empty(n, dtype=torch.float64, device=dev)
    e = step.combined_solve(dmu)
    Sc, Hc = step.combined()
    step.close()
    return dict(blocks=blocks, e_pred=e, dmu=dmu.cpu().numpy(), S_c=Sc, H_c=Hc)


def f32_inputs(wl, count=None):
    O, G, E = synth.samples(wl, count=count, dtype=np.float32)
    return O, G, E


def check(got, ref, O, G, E, w, offsets, n_keep):
    scale = max(1.0, np.sqrt(1.0e6 / O.shape[0]))
    O, G, E = (a.astype(np.float64) for a in (O, G, E))
    w = None if w is None else np.asarray(w, np.float32).astype(np.float64)
    de, dd, dl, ds = self_variation(blm_oracle, O, G, E, w, offsets, n_keep, ref)
    return check_step(blm_oracle, got, ref, O, G, E, w, offsets, n_keep, tol_mat=TOL_MAT * scale,
                      tol_e=TOL_E * scale, tol_dmu=TOL_DMU * scale, tol_eig=TOL_EIG * scale,
                      tol_sub=TOL_SUB * scale, tol_own=max(1e-9, 10 * dl, 10 * ds))


def oracle_f32(O, G, E, w, offsets, n_keep):
    return blm_oracle.blm_step(O.astype(np.float64), G.astype(np.float64), E.astype(np.float64),
                               None if w is None else np.asarray(w, np.float32).astype(np.float64),
                               offsets, n_keep)


def test_equal_blocks_of_256(torch_cuda):
    """Tile shape of the 16384-parameter workload (blocks of 256, K = 20), fewer blocks."""
    wl = synth.Workload("t", 1024, 8192, synth.equal_blocks(1024, 4), 20, decades=6.0, chunk=8192,
                        noise="student3")
    O, G, E = f32_inputs(wl)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[5000, 3192])
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_n200_workload_mixed(torch_cuda):
    wl = synth.workload("n200")
    O, G, E = f32_inputs(wl)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep)
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_uneven_blocks_weights_ragged(torch_cuda):
    wl = synth.Workload("t", 337, 3001, [0, 100, 300, 337], 6, decades=4.0, chunk=3001, seed=3,
                        offset=0.5)
    O, G, E = f32_inputs(wl)
    w = np.linspace(0.5, 1.5, O.shape[0]).astype(np.float32)
    ref = oracle_f32(O, G, E, w, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, w, wl.block_offsets, wl.n_keep, chunks=[1, 63, 2937])
    check(got, ref, O, G, E, w, wl.block_offsets, wl.n_keep)


def test_block_larger_than_tile(torch_cuda):
    """A block of 600 parameters: several row and column tiles, partial last tiles."""
    wl = synth.Workload("t", 700, 2048, [0, 600, 700], 8, decades=4.0, chunk=2048, seed=6)
    O, G, E = f32_inputs(wl)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep)
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)
