"""A batch of independent optimisations in one captured graph (blm_batch_*) against the eager
step of each problem on the same samples.

Problems of different sizes, block partitions and precisions share the batch: the split-BF16
and split-TF32 tensor-core paths and the FP64 path, a combined problem above the dense limit
(Davidson, run inside the graph after the branches join), uneven blocks.  Within a batch each
problem runs the kernels its eager step runs, on the same sample ranges; the block eigen-solves
of all problems share one launch and the dense combined solves another, one CTA per problem, so
each result matches its eager step up to the run-to-run order of the FP64 atomic sums.  A second
launch after the sample buffers were refilled must follow the new samples.
"""
import numpy as np
import pytest

import synth
from tests.parity import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


PROBLEMS = [
    dict(n=700, offs=synth.equal_blocks(700, 5), k=10, ns=9000, prec="BLM_PREC_BF16X4"),
    dict(n=512, offs=[0, 40, 300, 512], k=10, ns=5000, prec="BLM_PREC_TF32X4"),
    dict(n=1280, offs=synth.equal_blocks(1280, 8), k=45, ns=6000, prec="BLM_PREC_F64"),
    dict(n=96, offs=[0, 30, 64, 96], k=4, ns=3000, prec="BLM_PREC_F64"),
    dict(n=2000, offs=synth.equal_blocks(2000, 32), k=10, ns=12000, prec="BLM_PREC_TF32X4"),
]
CHUNK = 4096


def _inputs(torch, i, p, seed):
    wl = synth.Workload("b%d" % i, p["n"], p["ns"], p["offs"], p["k"], decades=4.0,
                        chunk=p["ns"], seed=seed, opt=i)
    dt = np.float64 if p["prec"] == "BLM_PREC_F64" else np.float32
    return [torch.from_numpy(a).to("cuda:0") for a in synth.samples(wl, dtype=dt)]


def _eager(blm, torch, p, O, G, E):
    f32 = O.dtype == torch.float32
    step = blm.Step(p["n"], p["offs"], p["k"], precision=getattr(blm, p["prec"]),
                    input_type=blm.BLM_IN_F32 if f32 else blm.BLM_IN_F64)
    for s0 in range(0, p["ns"], CHUNK):
        step.accumulate(O[s0:s0 + CHUNK], G[s0:s0 + CHUNK], E[s0:s0 + CHUNK])
    step.block_solve()
    for s0 in range(0, p["ns"], CHUNK):
        step.project(O[s0:s0 + CHUNK], G[s0:s0 + CHUNK], E[s0:s0 + CHUNK])
    dmu = torch.empty(p["n"], dtype=torch.float64, device="cuda:0")
    e = step.combined_solve(dmu)
    step.close()
    return e, dmu.cpu().numpy()


def test_batch_graph_matches_eager_steps(torch_cuda):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    data = [_inputs(torch, i, p, 50) for i, p in enumerate(PROBLEMS)]
    ref = [_eager(blm, torch, p, *d) for p, d in zip(PROBLEMS, data)]
    probs = [blm.make_problem(p["n"], p["offs"], p["k"], precision=getattr(blm, p["prec"]),
                              input_type=blm.BLM_IN_F64 if p["prec"] == "BLM_PREC_F64"
                              else blm.BLM_IN_F32) for p in PROBLEMS]
    b = blm.blm_batch_create(probs)
    dmu = [torch.full((p["n"],), np.nan, dtype=torch.float64, device="cuda:0") for p in PROBLEMS]
    blm.blm_batch_capture(b, [d[0] for d in data], [d[1] for d in data], [d[2] for d in data],
                          None, [p["ns"] for p in PROBLEMS], [p["n"] for p in PROBLEMS], CHUNK,
                          dmu)
    for rep in range(2):
        blm.blm_batch_launch(b)
        e, st, rc = blm.blm_batch_result(b, len(PROBLEMS))
        assert rc == blm.BLM_OK and list(st) == [0] * len(PROBLEMS), (rep, st)
        for i, (e_ref, d_ref) in enumerate(ref):
            assert abs(e[i] - e_ref) < 1e-12 * max(1.0, abs(e_ref)), (rep, i, e[i], e_ref)
            assert rel_err(dmu[i].cpu().numpy(), d_ref) < 1e-9, (rep, i)
    # block matrices of a problem are readable through its handle
    h = blm.blm_batch_handle(b, 0)
    d = blm.blm_block_dim(h, 0)
    S = np.empty((d + 1, d + 1))
    blm.blm_get_block(h, 0, S, None, None, None)
    assert abs(S[0, 0] - 1.0) < 1e-12
    # refill every problem's buffers with other samples
    data2 = [_inputs(torch, i, p, 51) for i, p in enumerate(PROBLEMS)]
    ref2 = [_eager(blm, torch, p, *d) for p, d in zip(PROBLEMS, data2)]
    for d_old, d_new in zip(data, data2):
        for a, c in zip(d_old, d_new):
            a.copy_(c)
    blm.blm_batch_launch(b)
    e, st, rc = blm.blm_batch_result(b, len(PROBLEMS))
    assert rc == blm.BLM_OK
    for i, (e_ref, d_ref) in enumerate(ref2):
        assert abs(e[i] - e_ref) < 1e-12 * max(1.0, abs(e_ref)), (i, e[i], e_ref)
        assert rel_err(dmu[i].cpu().numpy(), d_ref) < 1e-9, i
    blm.blm_batch_destroy(b)


def test_batch_after_eager_steps_and_autotuning(torch_cuda):
    """The bench's order of calls on the batch's own handles: tiles autotuned per problem, one
    eager step per problem (profiled), a reset, then the captured step -- whose results must
    match the eager ones.  Blocks of about 270 parameters and passes of 8192 samples."""
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    probs_def = [dict(n=2700, offs=synth.equal_blocks(2700, 10), k=10, ns=20480),
                 dict(n=1300, offs=synth.equal_blocks(1300, 6), k=10, ns=12288)]
    data = [_inputs(torch, i, dict(p, prec="BLM_PREC_BF16X4"), 60) for i, p in enumerate(probs_def)]
    probs = [blm.make_problem(p["n"], p["offs"], p["k"], precision=blm.BLM_PREC_BF16X4,
                              input_type=blm.BLM_IN_F32, pass_samples=8192) for p in probs_def]
    b = blm.blm_batch_create(probs)
    hs = [blm.blm_batch_handle(b, i) for i in range(len(probs_def))]
    for h, (O, G, E), p in zip(hs, data, probs_def):
        blm.blm_autotune(h, O, G, E, None, 8192, p["n"])
    eager = []
    for h, (O, G, E), p in zip(hs, data, probs_def):
        blm.blm_profile(h, 1)
        blm.blm_accumulate(h, O, G, E, None, p["ns"], p["n"])
        blm.blm_block_solve(h)
        blm.blm_project(h, O, G, E, None, p["ns"], p["n"])
        d = torch.empty(p["n"], dtype=torch.float64, device="cuda:0")
        eager.append((blm.blm_combined_solve(h, d), d.cpu().numpy()))
        blm.blm_profile(h, 0)
        blm.blm_reset(h)
    dmu = [torch.empty(p["n"], dtype=torch.float64, device="cuda:0") for p in probs_def]
    blm.blm_batch_capture(b, [d[0] for d in data], [d[1] for d in data], [d[2] for d in data],
                          None, [p["ns"] for p in probs_def], [p["n"] for p in probs_def],
                          65536, dmu)
    for rep in range(2):
        blm.blm_batch_launch(b)
        e, st, rc = blm.blm_batch_result(b, len(probs_def))
        assert rc == blm.BLM_OK, (rep, list(st), blm._lib.blm_batch_last_error(b).decode())
        for i, (e_ref, d_ref) in enumerate(eager):
            assert abs(e[i] - e_ref) < 1e-12 * max(1.0, abs(e_ref)), (rep, i, e[i], e_ref)
            assert rel_err(dmu[i].cpu().numpy(), d_ref) < 1e-9, (rep, i)
    blm.blm_batch_destroy(b)
