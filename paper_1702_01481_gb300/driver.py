"""Iteration driver: repeated BLM steps with history directions and an adaptive shift.

Sec. II.B: each step samples at the current parameters, builds and solves the block problems,
re-projects the same samples, solves the combined problem and moves mu by Delta mu.  The
updates of the previous N_O steps are the history directions of the next one (Eq. 9: the
rows D_j of old_dirs, newest first).

The diagonal shift of Sec. II.A acts as a trust radius; the paper does not say how it is chosen.
This driver takes the usual rule of thumb: a step whose predicted energy is not below the
current sample energy by more than the noise, or whose parameter change exceeds max_step, is
rejected and retried with ten times the shift; an accepted step halves the shift (never below
min_shift).

The step itself runs in the library (libblm.so through `Step`); `step_fn` can replace it with
any callable of the same signature (the tests drive the oracle through the same loop).
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class IterationRecord:
    it: int
    shift: float
    e_sample: float           # weighted sample mean of E_L at the current parameters
    e_pred: float             # predicted energy of the accepted step
    step_norm: float          # ||Delta mu||
    retries: int              # shifts tried before acceptance


@dataclass
class Result:
    mu: np.ndarray
    history: list = field(default_factory=list)


def gpu_step(O, G, E, w, offsets, n_keep, old_dirs, shift):
    """One step through the C ABI (FP64 path): returns (e_pred, dmu)."""
    import torch
    import paper_1702_01481_gb300 as blm
    dev = torch.device("cuda", torch.cuda.current_device())
    tO, tG, tE = (torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(dev) for a in (O, G, E))
    tw = torch.from_numpy(np.asarray(w, dtype=np.float64)).to(dev) if w is not None else None
    n = O.shape[1]
    D = None
    n_old = 0
    if old_dirs is not None and len(old_dirs):
        D = torch.from_numpy(np.ascontiguousarray(old_dirs, dtype=np.float64)).to(dev)
        n_old = D.shape[0]
    step = blm.Step(n, offsets, n_keep, n_old=n_old, old_dirs=D, shift=shift)
    try:
        step.accumulate(tO, tG, tE, tw)
        step.block_solve()
        step.project(tO, tG, tE, tw)
        dmu = torch.empty(n, dtype=torch.float64, device=dev)
        e = step.combined_solve(dmu)
        return e, dmu.cpu().numpy()
    finally:
        step.close()


def optimize(sampler, mu0, offsets, n_keep, n_iter=10, n_old=0, shift=0.0, adaptive=True,
             min_shift=1e-6, max_shift=1e3, max_step=None, noise=0.0, step_fn=gpu_step):
    """Run n_iter BLM steps from mu0.

    sampler(mu) -> (O, G, E, w) host arrays at parameters mu (w may be None).
    With adaptive=True the shift follows the rule in the module docstring; noise is the
    tolerance on the energy test (0 for exact sampling).  Returns the final parameters and one
    IterationRecord per step."""
    mu = np.array(mu0, dtype=np.float64)
    hist = []
    res = Result(mu=mu)
    sh = float(shift)
    for it in range(n_iter):
        O, G, E, w = sampler(mu)
        ww = np.ones(len(E)) if w is None else np.asarray(w, dtype=np.float64)
        e_sample = float(np.sum(ww * E) / np.sum(ww))
        D = np.array(hist[:n_old]) if n_old and hist else None
        retries = 0
        while True:
            e_pred, dmu = step_fn(O, G, E, w, offsets, n_keep, D, sh)
            norm = float(np.linalg.norm(dmu))
            ok = np.isfinite(e_pred) and np.all(np.isfinite(dmu))
            if adaptive:
                ok = ok and e_pred <= e_sample + noise
                if max_step is not None:
                    ok = ok and norm <= max_step
            if ok or not adaptive or sh >= max_shift:
                break
            sh = max(10.0 * sh, min_shift)
            retries += 1
        mu = mu + dmu
        hist.insert(0, dmu)
        res.history.append(IterationRecord(it, sh, e_sample, float(e_pred), norm, retries))
        if adaptive:
            sh = max(0.5 * sh, min_shift) if sh > 0 else 0.0
    res.mu = mu
    return res
