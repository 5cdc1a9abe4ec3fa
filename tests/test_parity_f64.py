"""GPU parity of the FP64 path (libblm.so through its C ABI) against the FP64 oracle.

Element by element on the same seeded inputs: block matrices S_b, H_b, kept eigenvalues, the
retained subspaces B^(b), the combined matrices, the predicted energy and the update.  Cases
cover several tiles and ragged tails, uneven blocks, weights, an offset that stresses the
centring, the diagonal shift, history directions (Eq. 9-10), chunked and host-memory input,
the zero-variance limit and the out-of-order call errors.

Tolerances (FP64 path): 1e-10 throughout -- matrices in correlation scaling (block matrices
against the oracle; combined matrices against the oracle's second sweep run with the GPU's
B^(b)), eigenvalues relative to max(1, |lambda|) (also against LAPACK on the GPU's own
matrices), retained subspaces (1 - cos of the largest principal angle), E_pred in Hartree and
Delta mu relative -- except where the oracle's own result moves more than that when the sample
order is reversed or when its eigenproblems are solved through a second backward-stable route
(Cholesky and the standard eigenproblem instead of QZ): eigen quantities carry the conditioning
of S (10^6 - 10^8 here) on top of the rounding of both sides, so each is held to
max(1e-10, 10 x the larger of those two self-variations).
"""
import numpy as np
import pytest

import synth
from synth import toy as T
from oracle import blm_oracle
from tests.parity import check_step, rel_err, self_variation, solver_variation

pytestmark = pytest.mark.gpu

TOL_MAT = 1e-10
TOL_EIG = 1e-10
TOL_SUB = 1e-10
TOL_E = 1e-10
TOL_DMU = 1e-10


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def run_gpu(torch, O, G, E, w, offsets, n_keep, chunks=None, shift=0.0, old_dirs=None,
            host=False):
    import paper_1702_01481_gb300 as blm
    dev = torch.device("cuda:0")
    if host:
        tO, tG, tE = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (O, G, E))
        tw = torch.from_numpy(w).pin_memory() if w is not None else None
    else:
        tO, tG, tE = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (O, G, E))
        tw = torch.from_numpy(w).to(dev) if w is not None else None
    n = O.shape[1]
    n_old = 0 if old_dirs is None else old_dirs.shape[0]
    D = torch.from_numpy(np.ascontiguousarray(old_dirs)).to(dev) if n_old else None
    step = blm.Step(n, offsets, n_keep, n_old=n_old, old_dirs=D, shift=shift)
    ns = O.shape[0]
    chunks = chunks or [ns]
    bounds = np.cumsum([0] + list(chunks))
    for a, b in zip(bounds[:-1], bounds[1:]):
        step.accumulate(tO[a:b], tG[a:b], tE[a:b], tw[a:b] if tw is not None else None)
    step.block_solve()
    blocks = [step.block(b) for b in range(len(offsets) - 1)]
    for a, b in reversed(list(zip(bounds[:-1], bounds[1:]))):
        step.project(tO[a:b], tG[a:b], tE[a:b], tw[a:b] if tw is not None else None)
    dmu = torch.empty(n, dtype=torch.float64, device=dev)
    e = step.combined_solve(dmu)
    Sc, Hc = step.combined()
    step.close()
    return dict(blocks=blocks, e_pred=e, dmu=dmu.cpu().numpy(), S_c=Sc, H_c=Hc)


def compare(got, ref, O, G, E, w, offsets, n_keep, shift=0.0, old_dirs=None):
    """FP64 parity; eigen quantities get max(floor, 10x the oracle's own sample-order
    sensitivity) since both sides round differently through the conditioning of S."""
    kw = dict(shift=shift, old_dirs=old_dirs)
    v1 = self_variation(blm_oracle, O, G, E, w, offsets, n_keep, ref, **kw)
    v2 = solver_variation(blm_oracle, O, G, E, w, offsets, n_keep, ref, **kw)
    de, dd, dl, ds = (max(a, b) for a, b in zip(v1, v2))
    return check_step(blm_oracle, got, ref, O, G, E, w, offsets, n_keep, tol_mat=TOL_MAT,
                      tol_e=max(TOL_E, 10 * de), tol_dmu=max(TOL_DMU, 10 * dd),
                      tol_eig=max(TOL_EIG, 10 * dl), tol_sub=max(TOL_SUB, 10 * ds),
                      shift=shift, old_dirs=old_dirs)


def test_n200_workload(torch_cuda):
    wl = synth.workload("n200")
    O, G, E = synth.samples(wl)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[7001, 12999])
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_uneven_blocks_weights_offset_ragged(torch_cuda):
    wl = synth.Workload("t", 150, 5003, [0, 37, 80, 81, 150], 4, decades=5.0, chunk=5003,
                        offset=1.0, seed=7)
    O, G, E = synth.samples(wl)
    w = np.linspace(0.3, 1.7, O.shape[0])
    ref = blm_oracle.blm_step(O, G, E, w, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, w, wl.block_offsets, wl.n_keep, chunks=[1, 2047, 2955])
    compare(got, ref, O, G, E, w, wl.block_offsets, wl.n_keep)


def test_shift(torch_cuda):
    wl = synth.Workload("t", 64, 4000, [0, 20, 44, 64], 3, decades=4.0, chunk=4000, seed=2)
    O, G, E = synth.samples(wl)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep, shift=0.1)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, shift=0.1)
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep, shift=0.1)


def test_history_directions(torch_cuda):
    wl = synth.Workload("t", 72, 3000, [0, 24, 48, 72], 2, decades=3.0, chunk=3000, seed=4)
    O, G, E = synth.samples(wl)
    rng = np.random.default_rng(1)
    D = rng.normal(size=(2, 72)) * 0.1
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep, old_dirs=D)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, old_dirs=D)
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep, old_dirs=D)


def test_host_memory_input_matches_device(torch_cuda):
    wl = synth.Workload("t", 96, 3000, [0, 48, 96], 3, decades=4.0, chunk=3000, seed=5)
    O, G, E = synth.samples(wl)
    a = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep)
    b = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, host=True)
    assert abs(a["e_pred"] - b["e_pred"]) < 1e-12
    assert rel_err(b["dmu"], a["dmu"]) < 1e-10


def test_zero_variance_toy(torch_cuda):
    toy = T.make_toy()
    O, G, E, w = T.sample(toy, np.zeros(toy.n), 3000)
    got = run_gpu(torch_cuda, O, G, E, w, [0, 4, 8, 12], 4)
    assert abs(got["e_pred"] - toy.e_ground) < 1e-9
    assert np.max(np.abs(got["dmu"] - toy.a)) < 1e-8


def test_n2048_full_parameter_count(torch_cuda):
    """The 2048-parameter workload (16 blocks of 128, K = 10, overlap condition 1e8) at its full
    parameter count and launch shape, on its first 20000 samples."""
    wl = synth.workload("n2048")
    O, G, E = synth.samples(wl, count=20000)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[16384, 3616])
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_call_order_is_enforced(torch_cuda):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    step = blm.Step(16, [0, 8, 16], 2)
    O = torch.zeros(4, 16, dtype=torch.float64, device="cuda:0")
    E = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    with pytest.raises(blm.BLMError) as e:
        step.block_solve()
    assert e.value.status == blm.BLM_ERR_STATE
    with pytest.raises(blm.BLMError) as e:
        step.project(O, O, E)
    assert e.value.status == blm.BLM_ERR_STATE
    dmu = torch.empty(16, dtype=torch.float64, device="cuda:0")
    with pytest.raises(blm.BLMError) as e:
        step.combined_solve(dmu)
    assert e.value.status == blm.BLM_ERR_STATE
    step.close()


def test_singular_overlap_is_reported(torch_cuda):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    ns, n = 64, 8
    rng = np.random.default_rng(0)
    O = rng.normal(size=(ns, n))
    O[:, 3] = O[:, 2]                       # two identical derivative vectors: S singular
    G = rng.normal(size=(ns, n))
    E = rng.normal(size=ns)
    dev = torch.device("cuda:0")
    step = blm.Step(n, [0, 4, 8], 2)
    step.accumulate(*(torch.from_numpy(a).to(dev) for a in (O, G, E)))
    with pytest.raises(blm.BLMError) as e:
        step.block_solve()
    assert e.value.status == blm.BLM_ERR_NUMERIC
    step.close()


def test_empty_chunk_is_a_noop(torch_cuda):
    wl = synth.Workload("t", 40, 800, [0, 20, 40], 2, decades=3.0, chunk=800, seed=9)
    O, G, E = synth.samples(wl)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep, chunks=[0, 800, 0])
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_large_combined_problem_davidson(torch_cuda):
    """Combined dimension 1 + 360 > 320: the lowest eigenpair comes from the Davidson solver."""
    wl = synth.Workload("t", 1280, 6000, synth.equal_blocks(1280, 8), 45, decades=4.0, chunk=6000,
                        seed=11)
    O, G, E = synth.samples(wl)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep)
    assert got["S_c"].shape[0] == 361
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_blocks_of_256_windowed_qr(torch_cuda):
    """Blocks of 256 (problem dimension 257): the QR sweeps span several shared-memory windows
    and the off-window row and column operations run from the stored reflectors."""
    wl = synth.Workload("t", 768, 6000, synth.equal_blocks(768, 3), 20, decades=6.0, chunk=6000,
                        seed=12, noise="student3")
    O, G, E = synth.samples(wl)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep)
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)


def test_more_block_problems_than_sms(torch_cuda):
    """170 block problems (more than the GPU's 152 SMs): the block solves run as one persistent
    grid, the three 200-parameter blocks on teams of CTAs and the 167 blocks of 8 taken one at a
    time from the shared queue; the combined problem (dimension 681) goes to Davidson."""
    offs = [0, 200, 400, 600] + [600 + 8 * (i + 1) for i in range(167)]
    wl = synth.Workload("t", offs[-1], 3000, offs, 4, decades=4.0, chunk=3000, seed=21)
    O, G, E = synth.samples(wl)
    ref = blm_oracle.blm_step(O, G, E, None, wl.block_offsets, wl.n_keep)
    got = run_gpu(torch_cuda, O, G, E, None, wl.block_offsets, wl.n_keep)
    compare(got, ref, O, G, E, None, wl.block_offsets, wl.n_keep)
