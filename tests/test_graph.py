"""The whole step captured as a CUDA graph (blm_graph_capture / blm_graph_launch /
blm_graph_result) against the eager calls on the same handle configuration.

The graph replays the eager step's kernels in the same order, so its results match the eager
step's to the run-to-run variation of the FP64 atomic sums (1e-12 relative here).  A second
launch, after the sample buffers were refilled with other samples, must give the eager result
of those samples: the graph reads the arrays at launch time.  Cases: the split-BF16 path
(prepared operands, tensor cores), the TF32 split on uneven blocks, and the FP64 path with a
combined problem above the dense limit (the cooperative Davidson launch inside the graph, with
its dense fallback decided on the device).
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


CASES = {
    "bf16x4": dict(n=1024, offs=synth.equal_blocks(1024, 4), k=20, ns=8192, chunk=4096,
                   prec="BLM_PREC_BF16X4", f32=True),
    "tf32x4_uneven": dict(n=900, offs=[0, 64, 300, 333, 640, 900], k=16, ns=6000, chunk=4000,
                          prec="BLM_PREC_TF32X4", f32=True),
    "f64_davidson": dict(n=1280, offs=synth.equal_blocks(1280, 8), k=45, ns=6000, chunk=6000,
                         prec="BLM_PREC_F64", f32=False),
}


def _inputs(torch, c, seed):
    wl = synth.Workload("g", c["n"], c["ns"], c["offs"], c["k"], decades=4.0, chunk=c["chunk"],
                        seed=seed)
    dt = np.float32 if c["f32"] else np.float64
    O, G, E = synth.samples(wl, dtype=dt)
    dev = torch.device("cuda:0")
    return [torch.from_numpy(a).to(dev) for a in (O, G, E)]


def _eager(blm, torch, c, O, G, E):
    p = getattr(blm, c["prec"])
    step = blm.Step(c["n"], c["offs"], c["k"], precision=p,
                    input_type=blm.BLM_IN_F32 if c["f32"] else blm.BLM_IN_F64)
    for s0 in range(0, c["ns"], c["chunk"]):
        sl = slice(s0, s0 + c["chunk"])
        step.accumulate(O[sl], G[sl], E[sl])
    step.block_solve()
    for s0 in range(0, c["ns"], c["chunk"]):
        sl = slice(s0, s0 + c["chunk"])
        step.project(O[sl], G[sl], E[sl])
    dmu = torch.empty(c["n"], dtype=torch.float64, device=O.device)
    e = step.combined_solve(dmu)
    S0 = step.block(0)[0]
    step.close()
    return e, dmu.cpu().numpy(), S0


@pytest.mark.parametrize("case", list(CASES))
def test_captured_step_matches_the_eager_step(torch_cuda, case):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    c = CASES[case]
    O, G, E = _inputs(torch, c, 41)
    e_ref, dmu_ref, S0_ref = _eager(blm, torch, c, O, G, E)
    p = getattr(blm, c["prec"])
    step = blm.Step(c["n"], c["offs"], c["k"], precision=p,
                    input_type=blm.BLM_IN_F32 if c["f32"] else blm.BLM_IN_F64)
    dmu = torch.full((c["n"],), np.nan, dtype=torch.float64, device=O.device)
    blm.blm_graph_capture(step.h, O, G, E, None, c["ns"], c["chunk"], c["n"], dmu)
    for rep in range(2):
        blm.blm_graph_launch(step.h)
        e = blm.blm_graph_result(step.h)
        assert abs(e - e_ref) < 1e-12 * max(1.0, abs(e_ref)), (rep, e, e_ref)
        assert rel_err(dmu.cpu().numpy(), dmu_ref) < 1e-9, rep
        S0 = step.block(0)[0]
        assert np.max(np.abs(S0 - S0_ref)) <= 1e-12 * np.max(np.abs(S0_ref))
    # refill the same buffers with other samples: the next launch reads them
    O2, G2, E2 = _inputs(torch, c, 42)
    e2_ref, dmu2_ref, _ = _eager(blm, torch, c, O2, G2, E2)
    O.copy_(O2)
    G.copy_(G2)
    E.copy_(E2)
    blm.blm_graph_launch(step.h)
    e2 = blm.blm_graph_result(step.h)
    assert abs(e2 - e2_ref) < 1e-12 * max(1.0, abs(e2_ref))
    assert rel_err(dmu.cpu().numpy(), dmu2_ref) < 1e-9
    assert abs(e2 - e_ref) > 1e-9            # the samples did change
    step.close()


def test_capture_rejects_host_arrays(torch_cuda):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    c = CASES["bf16x4"]
    O = torch.zeros((16, c["n"]), dtype=torch.float32)
    E = torch.zeros(16, dtype=torch.float32)
    dmu = torch.zeros(c["n"], dtype=torch.float64, device="cuda:0")
    step = blm.Step(c["n"], c["offs"], c["k"], precision=blm.BLM_PREC_BF16X4,
                    input_type=blm.BLM_IN_F32)
    with pytest.raises(blm.BLMError) as e:
        blm.blm_graph_capture(step.h, O, O, E, None, 16, 16, c["n"], dmu)
    assert e.value.status == blm.BLM_ERR_ARG
    with pytest.raises(blm.BLMError) as e:
        blm.blm_graph_launch(step.h)
    assert e.value.status == blm.BLM_ERR_STATE
    step.close()
