"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU needed).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign or index,
a transposed operand, a wrong alpha) fails at least one of them:
  * Eq. 3 written as explicit per-sample loops on tiny inputs (brute force);
  * the centred basis is a change of basis: same eigenvalues as the raw Eq. 3 matrices;
  * one block with every direction kept is the traditional linear method (Sec. III.B: N_B = 1
    reduces to the LM), and so is any blocking that keeps every direction;
  * zero-variance principle (Sec. I/II.A): when the ground state lies in the self-plus-tangent
    space the estimate is exact for any sample; the update then reaches it exactly;
  * for a linear ansatz sampled exactly, the predicted energy of Eq. 7 must equal the true
    energy of Psi(mu + Delta mu) built with Eq. 8 (checks alpha and the index of Eq. 8);
  * previous-update directions (Eq. 9-10) converge the iteration to the exact minimum;
  * storage figures printed in the paper (tests/golden/memory_example.txt);
  * a symmetric pencil reduces to scipy.linalg.eigh; a 2x2 pencil to the quadratic formula.
"""
import os

import numpy as np
import scipy.linalg
import pytest

from oracle import blm_oracle as B
import synth
from synth import toy as T

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _small(n=9, ns=400, seed=3, offset=0.0):
    wl = synth.Workload("t", n, ns, synth.equal_blocks(n, 3), 2, decades=3.0, chunk=ns, seed=seed,
                        offset=offset)
    return synth.samples(wl)


def test_eq3_brute_force_loops():
    rng = np.random.default_rng(0)
    ns, n = 7, 3
    O = rng.normal(size=(ns, n))
    G = rng.normal(size=(ns, n))
    E = rng.normal(size=ns)
    w = rng.uniform(0.5, 2.0, size=ns)
    S, H = B.lm_matrices_raw(O, G, E, w)
    Sb = np.zeros((n + 1, n + 1))
    Hb = np.zeros((n + 1, n + 1))
    for s in range(ns):
        ratio = [1.0] + [O[s, x] for x in range(n)]                 # <n|Psi^x>/<n|Psi>
        hratio = [E[s]] + [E[s] * O[s, y] + G[s, y] for y in range(n)]  # <n|H|Psi^y>/<n|Psi>
        for x in range(n + 1):
            for y in range(n + 1):
                Sb[x, y] += w[s] * ratio[x] * ratio[y]
                Hb[x, y] += w[s] * ratio[x] * hratio[y]
    Sb /= w.sum()
    Hb /= w.sum()
    np.testing.assert_allclose(S, Sb, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(H, Hb, rtol=1e-13, atol=1e-14)


def test_block_matrix_brute_force_loops():
    """Centred block matrices of one block by explicit loops (two-pass mean, then sums)."""
    O, G, E = _small(n=6, ns=50, offset=0.7)
    offs = [0, 2, 6]
    w = np.linspace(0.5, 1.5, 50)
    S, H = B.block_matrices(O, G, E, w, offs, 1)
    sw = sum(w)
    m = [sum(w[s] * O[s, x] for s in range(50)) / sw for x in range(6)]
    idx = [2, 3, 4, 5]
    Sb = np.zeros((5, 5))
    Hb = np.zeros((5, 5))
    for s in range(50):
        ob = [O[s, x] - m[x] for x in idx]
        xb = [E[s] * ob[k] + G[s, x] for k, x in enumerate(idx)]
        left = [1.0] + ob
        right = [E[s]] + xb
        for a in range(5):
            for c in range(5):
                Sb[a, c] += w[s] * left[a] * left[c]
                Hb[a, c] += w[s] * left[a] * right[c]
    Sb /= sw
    Hb /= sw
    np.testing.assert_allclose(S[1:, 1:], Sb[1:, 1:], rtol=1e-12, atol=1e-14)
    assert np.all(S[0, 1:] == 0) and np.all(S[1:, 0] == 0) and S[0, 0] == pytest.approx(1.0)
    assert np.max(np.abs(Sb[0, 1:])) < 1e-13       # the loops' <Obar> is zero up to rounding
    np.testing.assert_allclose(H, Hb, rtol=1e-12, atol=1e-14)


def test_overlap_properties():
    O, G, E = _small(offset=2.0)
    S, H = B.block_matrices(O, G, E, None, [0, 3, 6, 9], 1)
    assert np.allclose(S, S.T, atol=0, rtol=0)
    assert np.linalg.eigvalsh(S).min() > 0
    assert S[0, 0] == pytest.approx(1.0)
    assert H[0, 0] == pytest.approx(E.mean(), rel=1e-14)
    # H is not symmetric (Eq. 3 puts H on the ket only); its antisymmetric tangent part is
    # <Obar G^T> - <G Obar^T>, the E-terms cancelling.
    m = O.mean(0)
    Ob = O[:, 3:6] - m[3:6]
    Gb = G[:, 3:6]
    asym = (Ob.T @ Gb - Gb.T @ Ob) / O.shape[0]
    np.testing.assert_allclose(H[1:, 1:] - H[1:, 1:].T, asym, atol=1e-13)


def test_centred_basis_keeps_eigenvalues():
    O, G, E = _small(offset=1.5)
    S_raw, H_raw = B.lm_matrices_raw(O, G, E)
    S_c, H_c = B.block_matrices(O, G, E, None, [0, 9], 0)
    l_raw = np.sort_complex(np.linalg.eigvals(np.linalg.solve(S_raw, H_raw)))
    l_c = np.sort_complex(np.linalg.eigvals(np.linalg.solve(S_c, H_c)))
    np.testing.assert_allclose(l_c, l_raw, rtol=1e-8)


@pytest.mark.parametrize("shift", [0.0, 0.1])
def test_one_block_all_kept_is_lm(shift):
    O, G, E = _small(offset=0.4)
    lam, dmu = B.lm_step(O, G, E, shift=shift)
    r = B.blm_step(O, G, E, None, [0, 9], 9, shift=shift)
    assert r["e_pred"] == pytest.approx(lam, abs=1e-11)
    np.testing.assert_allclose(r["dmu"], dmu, rtol=1e-8, atol=1e-10)


def test_every_direction_kept_is_lm():
    O, G, E = _small(offset=0.4)
    lam, dmu = B.lm_step(O, G, E)
    r = B.blm_step(O, G, E, None, [0, 3, 6, 9], 3)
    assert r["e_pred"] == pytest.approx(lam, abs=1e-11)
    np.testing.assert_allclose(r["dmu"], dmu, rtol=1e-8, atol=1e-10)


def test_zero_variance_recovers_ground_state():
    toy = T.make_toy()
    O, G, E, w = T.sample(toy, np.zeros(toy.n), 3000)
    lam, dmu = B.lm_step(O, G, E, w)
    assert lam == pytest.approx(toy.e_ground, abs=1e-10)
    np.testing.assert_allclose(dmu, toy.a, atol=1e-10)
    r = B.blm_step(O, G, E, w, [0, 4, 8, 12], 4)
    assert r["e_pred"] == pytest.approx(toy.e_ground, abs=1e-10)
    np.testing.assert_allclose(r["dmu"], toy.a, atol=1e-10)
    p = T.psi(toy, r["dmu"])
    assert abs(abs(p @ toy.psi_g) / np.linalg.norm(p) - 1.0) < 1e-12


@pytest.mark.parametrize("n_keep,n_old", [(1, 0), (2, 0), (1, 1)])
def test_predicted_energy_is_energy_of_update(n_keep, n_old):
    toy = T.make_toy()
    mu = np.zeros(toy.n)
    D = None
    if n_old:
        D = 0.1 * np.ones((1, toy.n))
    O, G, E, w = T.exact(toy, mu)
    r = B.blm_step(O, G, E, w, [0, 4, 8, 12], n_keep, old_dirs=D)
    assert r["e_pred"] == pytest.approx(T.energy(toy, mu + r["dmu"]), abs=1e-10)
    assert r["e_pred"] < T.energy(toy, mu)


def test_history_directions_converge_to_minimum():
    toy = T.make_toy()
    offs = [0, 4, 8, 12]
    finals = {}
    for n_old in (0, 2):
        mu = np.zeros(toy.n)
        hist = []
        e_prev = T.energy(toy, mu)
        for it in range(15):
            O, G, E, w = T.exact(toy, mu)
            D = np.array(hist[:n_old]) if n_old and hist else None
            r = B.blm_step(O, G, E, w, offs, 1, old_dirs=D)
            mu = mu + r["dmu"]
            hist.insert(0, r["dmu"])
            e = T.energy(toy, mu)
            assert e <= e_prev + 1e-12          # exact sampling: each step is variational
            e_prev = e
        finals[n_old] = e_prev - toy.e_ground
    assert finals[2] < 1e-9
    assert finals[2] < finals[0]


def test_memory_figures_of_the_paper():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "memory_example.txt"))
            if l.strip() and not l.startswith("#")]
    for method, n, nb, no, gb in rows:
        n, nb, no, gb = int(n), int(nb), int(no), float(gb)
        digits = len(str(gb).split(".")[1])
        if method == "LM":
            got = B.lm_matrix_bytes(n) / 1e9
        else:
            got = B.blm_matrix_bytes_dominant(n, nb, no) / 1e9
        assert round(got, digits) == gb


def test_symmetric_pencil_matches_eigh():
    rng = np.random.default_rng(5)
    m = 12
    X = rng.normal(size=(40, m))
    S = X.T @ X / 40
    Hs = rng.normal(size=(m, m))
    Hs = 0.5 * (Hs + Hs.T)
    lam_k, Bk, lam_all = B.block_solve(np.block([[np.ones((1, 1)), np.zeros((1, m))],
                                                 [np.zeros((m, 1)), S]]),
                                       np.block([[np.zeros((1, 1)), np.zeros((1, m))],
                                                 [np.zeros((m, 1)), Hs]]), 3, m)
    ev, V = __import__("scipy.linalg").linalg.eigh(Hs, S)
    vals = np.sort(np.concatenate([[0.0], ev]))
    np.testing.assert_allclose(np.sort(lam_all.real), vals, atol=1e-10)
    np.testing.assert_allclose(lam_k, vals[:3], atol=1e-10)
    for j in range(3):
        if abs(vals[j]) < 1e-12:
            continue
    # B rows span the eigh eigenvectors of the three lowest (excluding the Psi direction at 0
    # if it is among them)
    want = [V[:, i] for i in range(m) if ev[i] <= vals[2] + 1e-12][:3]
    W = np.array(want).T
    Qb, _ = np.linalg.qr(Bk[[j for j in range(3) if abs(lam_k[j]) > 1e-12]].T)
    Qw, _ = np.linalg.qr(W[:, :Qb.shape[1]])
    s = np.linalg.svd(Qb.T @ Qw, compute_uv=False)
    assert s.min() > 1 - 1e-10


def test_two_by_two_closed_form():
    S = np.array([[1.0, 0.0], [0.0, 2.0]])
    H = np.array([[-1.0, 0.3], [0.2, 1.5]])
    lam_k, Bk, lam_all = B.block_solve(S, H, 1, 1)
    # det(H - l S) = (-1 - l)(1.5 - 2 l) - 0.06 = 2 l^2 + 0.5 l - 1.56 = 0
    a, b, c = 2.0, 0.5, -1.56
    roots = sorted([(-b - np.sqrt(b * b - 4 * a * c)) / (2 * a), (-b + np.sqrt(b * b - 4 * a * c)) / (2 * a)])
    np.testing.assert_allclose(sorted(lam_all.real), roots, rtol=1e-13)
    assert lam_k[0] == pytest.approx(roots[0], rel=1e-13)
    assert Bk.shape == (1, 1) and Bk[0, 0] == pytest.approx(1.0)


def test_complex_pair_gives_real_and_imaginary_parts():
    # tangent block: a rotation-like H gives eigenvalues -1 +- 0.5i for the first two
    # directions, and 3 for the third; S = I.
    S = np.eye(4)
    H = np.zeros((4, 4))
    H[0, 0] = 5.0
    H[1:3, 1:3] = [[-1.0, 0.5], [-0.5, -1.0]]
    H[3, 3] = 3.0
    lam_k, Bk, _ = B.block_solve(S, H, 2, 3)
    np.testing.assert_allclose(lam_k, [-1.0, -1.0], atol=1e-12)
    # the two retained directions span exactly the invariant plane of parameters 1 and 2
    assert np.allclose(Bk[:, 2], 0.0, atol=1e-12)
    assert abs(np.linalg.det(Bk[:, :2])) > 0.5


def test_sample_order_does_not_matter():
    O, G, E = _small(offset=0.3)
    r1 = B.blm_step(O, G, E, None, [0, 3, 6, 9], 2)
    r2 = B.blm_step(O[::-1], G[::-1], E[::-1], None, [0, 3, 6, 9], 2)
    assert r1["e_pred"] == pytest.approx(r2["e_pred"], abs=1e-12)
    np.testing.assert_allclose(r1["dmu"], r2["dmu"], rtol=1e-8, atol=1e-12)


def test_weights_scale_invariance():
    O, G, E = _small(offset=0.3)
    w = np.linspace(0.2, 2.0, O.shape[0])
    r1 = B.blm_step(O, G, E, w, [0, 3, 6, 9], 2)
    r2 = B.blm_step(O, G, E, 7.0 * w, [0, 3, 6, 9], 2)
    assert r1["e_pred"] == pytest.approx(r2["e_pred"], abs=1e-12)
    np.testing.assert_allclose(r1["dmu"], r2["dmu"], rtol=1e-9, atol=1e-12)


def test_generator_population_overlap():
    """Statistical check of the generator's closed form E[Obar Obar^T] = Q diag(sigma^2) Q^T."""
    wl = synth.Workload("t", 16, 40000, [0, 16], 2, decades=2.0, chunk=40000)
    model = synth.make_model(wl)
    O, G, E = synth.samples(wl, model)
    C = np.cov(O.T, bias=True)
    Q = np.eye(16)
    for r in range(4):                       # Q = H_0 H_1 H_2 H_3, H_r = I - 2 u_r u_r^T
        Q = Q - 2.0 * np.outer(Q @ model.u[r], model.u[r])
    want = Q @ np.diag(model.sigma ** 2) @ Q.T
    scale = np.sqrt(np.outer(np.diag(want), np.diag(want)))
    assert np.max(np.abs(C - want) / scale) < 6.0 / np.sqrt(40000) * 2


def test_generator_chunking_invariance():
    wl = synth.workload("n200")
    model = synth.make_model(wl)
    a = synth.chunk(wl, model, 0, 64)
    b = synth.chunk(wl, model, 32, 16)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x[32:48], y, rtol=1e-14, atol=1e-15)


def _projected_lm_eigs(O, G, E, w, C, shift=0.0):
    """Eigenvalues of the raw Eq. 3 problem restricted to span{Psi, columns of C}: the basis of
    any reduced problem (Eq. 5, 7, 10) is such a span, and centring does not change it."""
    S, H = B.lm_matrices_raw(O, G, E, w)
    if shift:
        H[1:, 1:] += shift * np.eye(S.shape[0] - 1)
    n = O.shape[1]
    P = np.zeros((1 + n, 1 + C.shape[1]))
    P[0, 0] = 1.0
    P[1:, 1:] = C
    lam = scipy.linalg.eigvals(P.T @ H @ P, P.T @ S @ P)
    return np.sort(lam.real)


@pytest.mark.parametrize("shift", [0.0, 0.05])
def test_block_problem_with_history_is_projected_lm(shift):
    O, G, E = _small(offset=0.5)
    offs = [0, 3, 6, 9]
    D = np.vstack([np.linspace(-1, 1, 9), np.cos(np.arange(9.0))])
    for b in range(3):
        S, H = B.block_matrices(O, G, E, None, offs, b, old_dirs=D, shift=shift)
        got = np.sort(scipy.linalg.eigvals(H, S).real)
        cols = [np.eye(9)[:, i] for i in range(offs[b], offs[b + 1])]
        for j in range(2):
            for k in range(3):
                if k != b:
                    d = np.zeros(9)
                    d[offs[k]:offs[k + 1]] = D[j, offs[k]:offs[k + 1]]
                    cols.append(d)
        want = _projected_lm_eigs(O, G, E, None, np.array(cols).T, shift)
        np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("shift", [0.0, 0.05])
def test_combined_problem_is_projected_lm(shift):
    O, G, E = _small(offset=0.5)
    offs = [0, 3, 6, 9]
    r = B.blm_step(O, G, E, None, offs, 2, shift=shift)
    got = np.sort(scipy.linalg.eigvals(r["H_c"], r["S_c"]).real)
    cols = []
    for b in range(3):
        for j in range(r["B"][b].shape[0]):
            d = np.zeros(9)
            d[offs[b]:offs[b + 1]] = r["B"][b][j]
            cols.append(d)
    want = _projected_lm_eigs(O, G, E, None, np.array(cols).T, shift)
    np.testing.assert_allclose(got, want, rtol=1e-8, atol=1e-9)
    assert r["e_pred"] == pytest.approx(want[0], abs=1e-9)
