"""GPU parity of the split-precision tensor-core path against the FP64 oracle.

The inputs are FP32; the oracle receives the same FP32 values widened to FP64, so the comparison
measures only the path's arithmetic: operands split into hi + lo (bf16 + bf16, or TF32 + FP32),
products accumulated in FP32 tensor memory, FP64 centring and FP64 solves.

Error model.  hi + lo represents each operand to 2^-16 (BF16X4) or 2^-22 (TF32X3) relative with a
zero-mean residual, independent from sample to sample, so its contribution to a sum over N
samples falls as 1/sqrt(N).  The tensor core's accumulation truncates; the kernel's short,
preloaded accumulator intervals keep that bias to a few 1e-7 at these sizes and below it at the
full step's long work units.  The targets hold at the size of the step they are stated for,
N = 10^6 samples; for a test sample of N the tolerances are the targets widened by
sqrt(10^6 / N):
  S_b, H_b and the combined matrices (the latter against the oracle's second sweep run with the
  GPU's B^(b)): 1e-6 in correlation scaling (|dA_xy| / sqrt(S_xx S_yy));
  E_pred end to end: 1e-8 Hartree.
Each later stage is checked against the oracle given the same inputs (check_step_stagewise):
the FP64 block solves against LAPACK on the GPU's own matrices, the kept eigenvalues' change
against the first-order change the measured matrix differences predict, and E_pred and Delta mu
against the oracle's combined solve on the GPU's combined matrices, all to max(1e-9, 10 x the
oracle's own sample-order sensitivity).
"""
import numpy as np
import pytest

import synth
from oracle import blm_oracle
from tests.parity import check_step_stagewise, self_variation

pytestmark = pytest.mark.gpu

TOL_MAT = 1e-6
TOL_E = 1e-8


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_mixed(torch, O, G, E, w, offsets, n_keep, chunks=None, prec=None):
    import paper_1702_01481_gb300 as blm
    prec = blm.BLM_PREC_BF16X4 if prec is None else prec
    dev = torch.device("cuda:0")
    tO, tG, tE = (torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev) for a in (O, G, E))
    tw = torch.from_numpy(np.asarray(w, dtype=np.float32)).to(dev) if w is not None else None
    n = O.shape[1]
    step = blm.Step(n, offsets, n_keep, precision=prec, input_type=blm.BLM_IN_F32)
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
    return check_step_stagewise(blm_oracle, got, ref, O, G, E, w, offsets, n_keep,
                                tol_mat=TOL_MAT * scale, tol_e=TOL_E * scale,
                                tol_own=max(1e-9, 10 * dl, 10 * ds))


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


def test_combined_sums_of_256_directions(torch_cuda):
    """16 blocks of 32 with K = 16: the combined problem has 256 directions, so the second sweep's
    contraction runs with full-width tiles as in the 16384-parameter step."""
    wl = synth.Workload("t", 512, 4096, synth.equal_blocks(512, 16), 16, decades=4.0, chunk=4096,
                        seed=8)
    O, G, E = f32_inputs(wl)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[2048, 2048])
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_more_than_20_directions_per_block(torch_cuda):
    """8 blocks of 64 with K = 24: more directions per block than the register-blocked
    projection holds (20), so the second sweep takes the 2 x 8-direction projection kernel."""
    wl = synth.Workload("t", 512, 4096, synth.equal_blocks(512, 8), 24, decades=4.0, chunk=4096,
                        seed=9)
    O, G, E = f32_inputs(wl)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[1500, 2596])
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


@pytest.mark.parametrize("which", ["n200", "blocks256"])
def test_tf32_split_precision(torch_cuda, which):
    """The TF32 hi/lo split (2^-22 operand representation): same checks, with the matrix and
    energy errors reported for comparison with the BF16 split."""
    import paper_1702_01481_gb300 as blm
    if which == "n200":
        wl = synth.workload("n200")
    else:
        wl = synth.Workload("t", 1024, 8192, synth.equal_blocks(1024, 4), 20, decades=6.0,
                            chunk=8192, noise="student3")
    O, G, E = f32_inputs(wl)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, prec=blm.BLM_PREC_TF32X3)
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_uneven_blocks_full_parameter_count_tf32(torch_cuda):
    """The uneven-block workload at its full shape (16384 parameters in 48 blocks of 64 - 640,
    K = 16, TF32X3 contractions) on its first 2048 samples: block problems up to 617, a
    769-direction combined problem (Davidson), unaligned block offsets (register-staged tiles)."""
    import paper_1702_01481_gb300 as blm
    wl = synth.workload("n16384u")
    O, G, E = f32_inputs(wl, count=2048)
    ref = oracle_f32(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_mixed(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[2048],
                    prec=blm.BLM_PREC_TF32X3)
    check(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)
