"""The iteration driver (repeated steps, history directions, adaptive shift).

CPU: the driver's loop runs the FP64 oracle as its step; with exact sampling on the zero-variance
toy and two history directions it must reach the ground state (the oracle's own convergence
pin), and the shift rule must retry a rejected step with ten times the shift.
GPU: the same loop through the library's FP64 path must follow the oracle-driven loop.
"""
import numpy as np
import pytest

from oracle import blm_oracle
from synth import toy as T
from paper_1702_01481_gb300 import driver

OFFS = [0, 4, 8, 12]


def oracle_step(O, G, E, w, offsets, n_keep, D, shift):
    r = blm_oracle.blm_step(O, G, E, w, offsets, n_keep, old_dirs=D, shift=shift)
    return r["e_pred"], r["dmu"]


def test_driver_with_history_reaches_ground_state():
    toy = T.make_toy()
    res = driver.optimize(lambda mu: T.exact(toy, mu), np.zeros(toy.n), OFFS, 1, n_iter=15,
                          n_old=2, adaptive=False, step_fn=oracle_step)
    for rec in res.history:
        assert rec.retries == 0
    assert T.energy(toy, res.mu) - toy.e_ground < 1e-9
    # exact sampling: the sample energy of each step is the true energy, non-increasing
    es = [r.e_sample for r in res.history]
    assert all(b <= a + 1e-12 for a, b in zip(es, es[1:]))


def test_driver_without_history_is_slower():
    toy = T.make_toy()
    finals = {}
    for n_old in (0, 2):
        res = driver.optimize(lambda mu: T.exact(toy, mu), np.zeros(toy.n), OFFS, 1, n_iter=15,
                              n_old=n_old, adaptive=False, step_fn=oracle_step)
        finals[n_old] = T.energy(toy, res.mu) - toy.e_ground
    assert finals[2] < finals[0]


def test_adaptive_shift_retries_and_relaxes():
    calls = []

    def fake_step(O, G, E, w, offsets, n_keep, D, shift):
        calls.append(shift)
        good = shift >= 1e-2
        return (-1.0 if good else 5.0), np.full(O.shape[1], 0.01)

    def sampler(mu):
        O = np.zeros((4, 3))
        return O, O, np.zeros(4), None

    res = driver.optimize(sampler, np.zeros(3), [0, 3], 1, n_iter=2, adaptive=True,
                          shift=1e-6, step_fn=fake_step)
    first = res.history[0]
    assert first.retries == 4 and first.shift == pytest.approx(1e-2)
    assert calls[:5] == pytest.approx([1e-6, 1e-5, 1e-4, 1e-3, 1e-2])
    # the next step starts from half the accepted shift, is rejected once and accepted at 5e-2
    assert calls[5] == pytest.approx(5e-3)
    assert res.history[1].shift == pytest.approx(5e-2)


@pytest.mark.gpu
def test_driver_on_gpu_follows_the_oracle_loop():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    toy = T.make_toy()
    kw = dict(n_iter=15, n_old=2, adaptive=False)
    ref = driver.optimize(lambda mu: T.exact(toy, mu), np.zeros(toy.n), OFFS, 1,
                          step_fn=oracle_step, **kw)
    got = driver.optimize(lambda mu: T.exact(toy, mu), np.zeros(toy.n), OFFS, 1, **kw)
    for a, b in zip(got.history, ref.history):
        assert abs(a.e_pred - b.e_pred) < 1e-9
    np.testing.assert_allclose(got.mu, ref.mu, atol=1e-8)
    assert T.energy(toy, got.mu) - toy.e_ground < 1e-9
