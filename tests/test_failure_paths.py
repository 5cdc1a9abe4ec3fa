"""Failure detection on the GPU, without faulting it.

* A bounded pipeline wait that runs out: with the wait limit at 0 polls every mbarrier wait of
  the tensor-core kernels gives up at once, the kernel records the timeout, drains what it has
  in flight and returns; the next solve reports BLM_ERR_TIMEOUT.  The same handle, reset and
  given the default limit, then runs a correct step, so the context stays usable.
* Non-finite samples (a NaN and an Inf written into the host arrays before the copy to the
  device) reach the sums and are reported as BLM_ERR_NUMERIC by the block solve, on the FP64
  path and on the split-BF16 tensor-core path.
"""
import numpy as np
import pytest

import synth
from oracle import blm_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _workload():
    wl = synth.Workload("t", 512, 4096, synth.equal_blocks(512, 2), 8, decades=4.0, chunk=4096,
                        seed=31)
    return wl, synth.samples(wl, dtype=np.float32)


@pytest.mark.parametrize("prec", ["bf16x4", "tf32x4"])
def test_wait_timeout_is_reported_and_the_handle_recovers(torch_cuda, prec):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    wl, (O, G, E) = _workload()
    dev = torch.device("cuda:0")
    tO, tG, tE = (torch.from_numpy(a).to(dev) for a in (O, G, E))
    p = blm.BLM_PREC_BF16X4 if prec == "bf16x4" else blm.BLM_PREC_TF32X4
    step = blm.Step(wl.n, wl.block_offsets, wl.n_keep, precision=p, input_type=blm.BLM_IN_F32)
    blm.blm_set_wait_limit(step.h, 0)
    step.accumulate(tO, tG, tE)
    with pytest.raises(blm.BLMError) as e:
        step.block_solve()
    assert e.value.status == blm.BLM_ERR_TIMEOUT
    torch.cuda.synchronize()                  # the context is still healthy
    blm.blm_set_wait_limit(step.h, blm.BLM_WAIT_LIMIT_DEFAULT)
    step.reset()
    step.accumulate(tO, tG, tE)
    step.block_solve()
    step.project(tO, tG, tE)
    dmu = torch.empty(wl.n, dtype=torch.float64, device=dev)
    e_pred = step.combined_solve(dmu)
    step.close()
    ref = blm_oracle.blm_step(*(a.astype(np.float64) for a in (O, G, E)), None, wl.block_offsets,
                              wl.n_keep)
    assert abs(e_pred - ref["e_pred"]) < 1e-7


@pytest.mark.parametrize("prec,bad", [("f64", np.nan), ("f64", np.inf), ("bf16x4", np.nan),
                                      ("bf16x4", np.inf)])
def test_non_finite_samples_are_reported(torch_cuda, prec, bad):
    import paper_1702_01481_gb300 as blm
    torch = torch_cuda
    wl, (O, G, E) = _workload()
    if prec == "f64":
        O, G, E = (a.astype(np.float64) for a in (O, G, E))
        kw = dict(precision=blm.BLM_PREC_F64, input_type=blm.BLM_IN_F64)
    else:
        kw = dict(precision=blm.BLM_PREC_BF16X4, input_type=blm.BLM_IN_F32)
    O = O.copy()
    O[1234, 300] = bad                        # one sample of one parameter of block 1
    dev = torch.device("cuda:0")
    tO, tG, tE = (torch.from_numpy(a).to(dev) for a in (O, G, E))
    step = blm.Step(wl.n, wl.block_offsets, wl.n_keep, **kw)
    step.accumulate(tO, tG, tE)
    with pytest.raises(blm.BLMError) as e:
        step.block_solve()
    assert e.value.status == blm.BLM_ERR_NUMERIC
    assert "block" in blm.blm_last_error(step.h)
    step.close()
    torch.cuda.synchronize()
