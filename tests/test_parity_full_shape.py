"""Parity of the split-BF16 tensor-core step at the full shape of the 16384-parameter workload.

The 16384-parameter workload (64 blocks of 256, K = 20, Student-t local-energy noise), FP32
samples generated on the device by the seeded generator, in the launch configuration bench.py
times (chunks of 65536 samples; tensor-core work units of 16384 samples in the first sweep and
8192 in the second, i.e. 128 and 64 preloaded accumulator intervals per unit).

Two sample counts:
  * one chunk of 65536 samples, checked in detail: sampled blocks (first, middle, last) against
    the FP64 oracle given the same FP32 values; every block against the FP64 GPU path (FP32
    input widened on load, itself held to the oracle within 1e-10 on the sampled blocks); the
    rows and columns of two blocks' directions in the combined matrices against the oracle's
    second sweep with the same path's B^(b); the kept eigenvalues against the first-order change
    the matrix differences predict; E_pred and Delta mu of each path against the oracle's
    combined solve and Eq. 8 update on that path's own combined matrices (dimension 1281, the
    Davidson solver); tolerances from tests/parity.py, mixed_tolerances, at N = 65536;
  * the whole 10^6-sample step, held to the stated targets without any widening: S_b, H_b within
    1e-6 (correlation scaling) of the FP64 GPU path and, for a sampled block, of the FP64
    oracle; E_pred within 1e-8 Hartree of the FP64 path's.
"""
import numpy as np
import pytest

import synth
from oracle import blm_oracle
from tests.parity import eig_first_order, matrix_err, mixed_tolerances, rel_err, subspace_err

pytestmark = pytest.mark.gpu

NS = 65536
TOL_MAT, TOL_E = mixed_tolerances(NS)   # mixed path at 65536 samples
TOL_MAT_F64 = 1e-10                     # FP64 path
NS_FULL = 1000000
TARGET_MAT, TARGET_E = 1e-6, 1e-8       # mixed path, the full step


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(blm, torch, prec, wl, O, G, E, chunk=65536):
    dev = O.device
    ns = O.shape[0]
    step = blm.Step(wl.n, wl.block_offsets, wl.n_keep, precision=prec, input_type=blm.BLM_IN_F32)
    for s0 in range(0, ns, chunk):
        step.accumulate(O[s0:s0 + chunk], G[s0:s0 + chunk], E[s0:s0 + chunk])
    step.block_solve()
    blocks = [step.block(b) for b in range(wl.n_blocks)]
    for s0 in range(0, ns, chunk):
        step.project(O[s0:s0 + chunk], G[s0:s0 + chunk], E[s0:s0 + chunk])
    dmu = torch.empty(wl.n, dtype=torch.float64, device=dev)
    e = step.combined_solve(dmu)
    Sc, Hc = step.combined()
    step.close()
    return dict(blocks=blocks, e_pred=e, dmu=dmu.cpu().numpy(), S_c=Sc, H_c=Hc)


@pytest.fixture(scope="module")
def full_shape(torch_cuda):
    torch = torch_cuda
    import paper_1702_01481_gb300 as blm
    from synth import device as sdev
    dev = torch.device("cuda:0")
    wl = synth.workload("n16384")
    O = torch.empty((NS, wl.n), dtype=torch.float32, device=dev)
    G = torch.empty((NS, wl.n), dtype=torch.float32, device=dev)
    E = torch.empty((NS,), dtype=torch.float32, device=dev)
    dm = sdev.DeviceModel(wl, dev)
    for s0 in range(0, NS, 16384):
        sdev.fill(dm, s0, O[s0:s0 + 16384], G[s0:s0 + 16384], E[s0:s0 + 16384])
    torch.cuda.synchronize()
    mixed = _run(blm, torch, blm.BLM_PREC_BF16X4, wl, O, G, E)
    f64 = _run(blm, torch, blm.BLM_PREC_F64, wl, O, G, E)
    sampled = [0, 31, 63]
    cols = {}
    for b in sampled:
        lo, hi = wl.block_offsets[b], wl.block_offsets[b + 1]
        cols[b] = (O[:, lo:hi].double().cpu().numpy(), G[:, lo:hi].double().cpu().numpy())
    Eh = E.double().cpu().numpy()
    # the sample mean of O (FP64, over all samples), which Eq. 8's alpha needs
    m = np.zeros(wl.n)
    for s0 in range(0, NS, 8192):
        m += O[s0:s0 + 8192].cpu().numpy().astype(np.float64).sum(axis=0)
    m /= NS
    del O, G, E
    torch.cuda.empty_cache()
    return dict(wl=wl, mixed=mixed, f64=f64, cols=cols, E=Eh, m=m, sampled=sampled)


def test_sampled_blocks_against_oracle(full_shape):
    wl, cols, E = full_shape["wl"], full_shape["cols"], full_shape["E"]
    worst = {"mixed": 0.0, "f64": 0.0}
    for b in full_shape["sampled"]:
        Ob, Gb = cols[b]
        m = Ob.shape[1]
        S_ref, H_ref = blm_oracle.block_matrices(Ob, Gb, E, None, [0, m], 0)
        for path in ("mixed", "f64"):
            S, H, _, _ = full_shape[path]["blocks"][b]
            worst[path] = max(worst[path], matrix_err(S, S_ref, H, H_ref))
    print("full shape, sampled blocks vs oracle:", worst)
    assert worst["f64"] < TOL_MAT_F64, worst
    assert worst["mixed"] < TOL_MAT, worst


def test_all_blocks_against_fp64_path(full_shape):
    wl, mixed, f64 = full_shape["wl"], full_shape["mixed"], full_shape["f64"]
    em = 0.0
    diag_s, diag_h = [], []
    for b in range(wl.n_blocks):
        S, H, lam, B = mixed["blocks"][b]
        S64, H64, lam64, B64 = f64["blocks"][b]
        em = max(em, matrix_err(S, S64, H, H64))
        diag_s.append(np.mean((np.diag(S)[1:] - np.diag(S64)[1:]) / np.diag(S64)[1:]))
        diag_h.append(np.mean((np.diag(H)[1:] - np.diag(H64)[1:]) / np.abs(np.diag(H64)[1:])))
    print("full shape, all blocks vs FP64 path: max %.3g, mean relative diagonal bias S %.3g H %.3g"
          % (em, np.mean(diag_s), np.mean(diag_h)))
    assert em < TOL_MAT, em


def test_kept_eigenvalues_follow_matrix_differences(full_shape):
    """The kept eigenvalues move from the FP64 path's by no more than three times the first-order
    change the measured matrix differences predict."""
    wl, mixed, f64 = full_shape["wl"], full_shape["mixed"], full_shape["f64"]
    worst, sub = 0.0, 0.0
    for b in range(0, wl.n_blocks, 8):
        S, H, lam, B = mixed["blocks"][b]
        S64, H64, lam64, B64 = f64["blocks"][b]
        pred = eig_first_order(S64, H64, S, H, lam64)
        dl = np.abs(np.asarray(lam) - np.asarray(lam64))
        worst = max(worst, float(np.max(dl / (3.0 * pred + 1e-12 * np.maximum(1.0, np.abs(lam64))))))
        sub = max(sub, subspace_err(B, B64))
    print("full shape, kept eigenvalues: ratio to first-order prediction %.3g, subspace %.3g"
          % (worst, sub))
    assert worst <= 1.0, worst


def test_combined_matrices_against_oracle(full_shape):
    wl, cols, E = full_shape["wl"], full_shape["cols"], full_shape["E"]
    pick = full_shape["sampled"][:2]
    offs, K = wl.block_offsets, wl.n_keep
    Osub = np.hstack([cols[b][0] for b in pick])
    Gsub = np.hstack([cols[b][1] for b in pick])
    sub_offs = [0]
    for b in pick:
        sub_offs.append(sub_offs[-1] + offs[b + 1] - offs[b])
    # directions of block b occupy combined indices 1 + K b .. K (b + 1) (equal blocks, K <= M_b)
    idx = [0] + [1 + K * b + j for b in pick for j in range(K)]
    out = {}
    for path, tol in (("mixed", TOL_MAT), ("f64", TOL_MAT_F64)):
        res = full_shape[path]
        Bs = [res["blocks"][b][3] for b in pick]
        Sc_ref, Hc_ref = blm_oracle.combined_matrices(Osub, Gsub, E, None, sub_offs, Bs)
        Sc = res["S_c"][np.ix_(idx, idx)]
        Hc = res["H_c"][np.ix_(idx, idx)]
        out[path] = matrix_err(Sc, Sc_ref, Hc, Hc_ref)
        assert out[path] < tol, (path, out)
    print("full shape, combined sub-matrices vs oracle:", out)


def test_energy_and_update(full_shape):
    wl, mixed, f64 = full_shape["wl"], full_shape["mixed"], full_shape["f64"]
    offs = wl.block_offsets
    report = {}
    for path in ("mixed", "f64"):
        res = full_shape[path]
        Bs = [blk[3] for blk in res["blocks"]]
        # the oracle's combined solve (QZ) and Eq. 8 update on this path's own combined matrices
        e_own, dmu_own = blm_oracle.combined_update(res["S_c"], res["H_c"], offs, Bs,
                                                    full_shape["m"])
        report[path + "_e_vs_own_solve"] = abs(e_own - res["e_pred"])
        report[path + "_dmu_vs_own_solve"] = rel_err(res["dmu"], dmu_own)
        assert report[path + "_e_vs_own_solve"] < 1e-9 * max(1.0, abs(e_own)), report
        assert report[path + "_dmu_vs_own_solve"] < 1e-8, report
    de = abs(mixed["e_pred"] - f64["e_pred"])
    dd = rel_err(mixed["dmu"], f64["dmu"])
    report.update(e_pred_mixed_vs_f64=de, dmu_mixed_vs_f64=dd, e_pred=mixed["e_pred"])
    print("full shape, energy and update:", report)
    assert de < TOL_E, report


@pytest.fixture(scope="module")
def full_step(torch_cuda, full_shape):
    torch = torch_cuda
    import paper_1702_01481_gb300 as blm
    from synth import device as sdev
    dev = torch.device("cuda:0")
    wl = synth.workload("n16384")
    O = torch.empty((NS_FULL, wl.n), dtype=torch.float32, device=dev)
    G = torch.empty((NS_FULL, wl.n), dtype=torch.float32, device=dev)
    E = torch.empty((NS_FULL,), dtype=torch.float32, device=dev)
    dm = sdev.DeviceModel(wl, dev)
    for s0 in range(0, NS_FULL, 32768):
        c = min(32768, NS_FULL - s0)
        sdev.fill(dm, s0, O[s0:s0 + c], G[s0:s0 + c], E[s0:s0 + c])
    torch.cuda.synchronize()
    mixed = _run(blm, torch, blm.BLM_PREC_BF16X4, wl, O, G, E)
    f64 = _run(blm, torch, blm.BLM_PREC_F64, wl, O, G, E)
    b = 17
    lo, hi = wl.block_offsets[b], wl.block_offsets[b + 1]
    col = (O[:, lo:hi].double().cpu().numpy(), G[:, lo:hi].double().cpu().numpy(),
           E.double().cpu().numpy())
    del O, G, E
    torch.cuda.empty_cache()
    return dict(wl=wl, mixed=mixed, f64=f64, block=b, col=col)


def test_full_step_meets_the_stated_targets(full_step):
    wl, mixed, f64 = full_step["wl"], full_step["mixed"], full_step["f64"]
    em = max(matrix_err(m[0], r[0], m[1], r[1]) for m, r in zip(mixed["blocks"], f64["blocks"]))
    Ob, Gb, E = full_step["col"]
    S_ref, H_ref = blm_oracle.block_matrices(Ob, Gb, E, None, [0, Ob.shape[1]], 0)
    b = full_step["block"]
    e_oracle_mixed = matrix_err(mixed["blocks"][b][0], S_ref, mixed["blocks"][b][1], H_ref)
    e_oracle_f64 = matrix_err(f64["blocks"][b][0], S_ref, f64["blocks"][b][1], H_ref)
    de = abs(mixed["e_pred"] - f64["e_pred"])
    dd = rel_err(mixed["dmu"], f64["dmu"])
    report = dict(blocks_vs_fp64=em, block_vs_oracle=e_oracle_mixed, fp64_block_vs_oracle=e_oracle_f64,
                  e_pred_vs_fp64=de, dmu_vs_fp64=dd)
    print("full step (10^6 samples):", report)
    assert e_oracle_f64 < TOL_MAT_F64, report
    assert em < TARGET_MAT, report
    assert e_oracle_mixed < TARGET_MAT, report
    assert de < TARGET_E, report
    assert dd < 1e-2, report
