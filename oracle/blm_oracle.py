"""FP64 CPU oracle for one step of the blocked linear method (Zhao & Neuscamman, arXiv:1702.01481).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
reference leg may import or run this module.  The product (the CUDA library and its binding)
never calls it, and it shares no code with the CUDA path.

Plain, slow, obviously correct: numpy float64 array operations (a matrix product is the only
library primitive used for the sums) and scipy.linalg.eig (LAPACK QZ) for the generalized
eigenproblems.  Every function follows the paper's equations in their order:

  Sec. II.A, Eq. 1   linear-method eigenproblem  sum_y <Psi^x|H|Psi^y> c_y = lambda sum_y <Psi^x|Psi^y> c_y
  Sec. II.A, Eq. 2   update  mu_x <- mu_x + c_x / c_0
  Sec. II.A, Eq. 3   Monte Carlo estimate: sum over samples of w * (Psi^x/Psi)* (H Psi^y / Psi)
  Sec. II.B, Eq. 4-5 one-block expansion and its eigenproblem; keep the N_K lowest directions
  Sec. II.B, Eq. 6-7 combined expansion in the retained directions and its eigenproblem
  Sec. II.B, Eq. 8   BLM update  mu_{i,b} <- mu_{i,b} + [A B^(b)]_{bi} / alpha
  Sec. II.B, Eq. 9-10 previous-update directions Theta_jk added to every other block's problem

Notation: O[s, x] = <n_s|Psi^x>/<n_s|Psi> (raw log-derivative ratios), E[s] = local energy,
G[s, x] = dE_L/dmu_x, so the Hamiltonian ratio of Eq. 3 is h_x = <n|H|Psi^x>/<n|Psi> = E O_x + G_x
(H acting on dPsi/dmu gives d(E_L Psi)/dmu).  w[s] = |Psi|^2/P (1 when P = |Psi|^2).

Readings where the paper is silent:
  * centring: the tangent vectors are taken as Psi^x - <O_x> Psi, a change of basis inside
    span{Psi, Psi^x}; eigenvalues and the tangent parts of eigenvectors are unchanged, and the
    update converts back with alpha = c_0 - sum_x c_x <O_x>.
  * averages are normalised by sum(w), so S_00 = 1.
  * H is kept non-symmetric (strong zero-variance principle).
  * the diagonal shift of Sec. II.A is shift * (Gram matrix of the basis directions in parameter
    space), i.e. shift * I on the tangent space, carried into every reduced basis.
  * "lowest" = smallest real part; a complex pair contributes the real and imaginary parts of its
    eigenvector, taken with the phase that makes the largest-magnitude component real and
    positive (only the real part when N_K ends inside the pair).
  * B^(b) rows are the beta parts of the chosen eigenvectors, each scaled to unit 2-norm with its
    largest-magnitude entry positive.
"""
import numpy as np
import scipy.linalg


# --------------------------------------------------------------------------------------------
# Sec. II.A, Eq. 3: Monte Carlo matrix estimate in the raw self-plus-tangent basis (1 + n).
# --------------------------------------------------------------------------------------------
def lm_matrices_raw(O, G, E, w=None):
    """S_xy = <O_x O_y>, H_xy = <O_x h_y> with O_0 = 1, h_0 = E, h_y = E O_y + G_y (Eq. 3).

    Rows index the bra (the left ratio), columns the ket (the Hamiltonian ratio)."""
    O = np.asarray(O, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    ns = O.shape[0]
    w = np.ones(ns) if w is None else np.asarray(w, dtype=np.float64)
    left = np.hstack([np.ones((ns, 1)), O])                     # <n|Psi^x>/<n|Psi>, x = 0..n
    right = np.hstack([E[:, None], E[:, None] * O + G])          # <n|H|Psi^y>/<n|Psi>
    sw = w.sum()
    S = (left * w[:, None]).T @ left / sw
    H = (left * w[:, None]).T @ right / sw
    return S, H


# --------------------------------------------------------------------------------------------
# Generic centred linear-method matrices for a set of tangent directions.
# --------------------------------------------------------------------------------------------
def centred_lm_matrices(V, XV, E, w, gram=None, shift=0.0):
    """Eq. 3 written in a centred basis {Psi, Vbar_1 .. Vbar_m}.

    V[s, k]  : ratio <n|Vbar_k>/<n|Psi> of tangent direction k (already centred: <V_k> = 0)
    XV[s, k] : ratio <n|H|Vbar_k>/<n|Psi>
    Returns S (1+m)^2 and H (1+m)^2 normalised by sum(w):
        S = [[1, 0], [0, <V V^T>]],  H = [[<E>, <XV>^T], [<V E>, <V XV^T>]]
    plus shift * gram on the tangent block of H (gram = Gram matrix of the directions'
    coefficient vectors in parameter space; identity for the raw derivatives)."""
    ns, m = V.shape
    w = np.ones(ns) if w is None else np.asarray(w, dtype=np.float64)
    sw = w.sum()
    left = np.hstack([np.ones((ns, 1)), V])
    right = np.hstack([E[:, None], XV])
    S = (left * w[:, None]).T @ left / sw
    H = (left * w[:, None]).T @ right / sw
    # The centred tangent directions have zero mean overlap with Psi by construction: set the
    # S_0x entries to the exact value rather than to the rounding residue of <Vbar>.
    S[0, 1:] = 0.0
    S[1:, 0] = 0.0
    if shift:
        g = np.eye(m) if gram is None else gram
        H[1:, 1:] += shift * g
    return S, H


def sample_means(O, E, w=None):
    """m_x = <O_x> and <E> over all samples (first pass of the two-pass centring)."""
    O = np.asarray(O, dtype=np.float64)
    w = np.ones(O.shape[0]) if w is None else np.asarray(w, dtype=np.float64)
    sw = w.sum()
    return (w @ O) / sw, float(w @ np.asarray(E, dtype=np.float64)) / sw


# --------------------------------------------------------------------------------------------
# Sec. II.B, Eq. 4, 5, 9, 10: the block problems.
# --------------------------------------------------------------------------------------------
def block_basis(O, G, E, m, offsets, b, old_dirs=None):
    """Tangent directions of block b's expansion (Eq. 4): its own centred derivatives
    Psibar^{i,b}, followed by Theta_jk = sum_l D_jkl Psibar^{l,k} for every other block k and
    history row j (Eq. 9).  Returns V, XV and the coefficient vectors C (n x m_b) of the
    directions in parameter space (for the shift)."""
    n = O.shape[1]
    lo, hi = offsets[b], offsets[b + 1]
    Obar = O - m[None, :]
    Xbar = E[:, None] * Obar + G
    V = [Obar[:, lo:hi]]
    XV = [Xbar[:, lo:hi]]
    C = [np.eye(n)[:, lo:hi]]
    if old_dirs is not None and len(old_dirs):
        D = np.asarray(old_dirs, dtype=np.float64)
        for j in range(D.shape[0]):
            for k in range(len(offsets) - 1):
                if k == b:
                    continue
                kl, kh = offsets[k], offsets[k + 1]
                d = np.zeros(n)
                d[kl:kh] = D[j, kl:kh]
                V.append((Obar @ d)[:, None])      # t_jk = Obar_k . D_jk
                XV.append((Xbar @ d)[:, None])     # E t_jk + G_k . D_jk
                C.append(d[:, None])
    return np.hstack(V), np.hstack(XV), np.hstack(C)


def block_matrices(O, G, E, w, offsets, b, old_dirs=None, shift=0.0):
    """S_b, H_b of block b (Eq. 5 with N_O = 0, Eq. 10 otherwise) in the centred basis."""
    O = np.asarray(O, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    m, _ = sample_means(O, E, w)
    V, XV, C = block_basis(O, G, E, m, offsets, b, old_dirs)
    return centred_lm_matrices(V, XV, E, w, gram=C.T @ C, shift=shift)


def _lowest_directions(lam, vecs, k):
    """Choose the k eigen-directions with the lowest real eigenvalue parts (Sec. II.B: the
    lowest eigenvalues mark the best update directions).  A complex pair contributes the real
    and imaginary parts of one member's eigenvector.  Returns (eigenvalues used, real vectors)."""
    finite = np.isfinite(lam)
    order = [i for i in np.argsort(lam.real, kind="stable") if finite[i]]
    out_lam, out_vec, used = [], [], set()
    tol = 1e-12
    for i in order:
        if len(out_vec) >= k:
            break
        if i in used:
            continue
        used.add(i)
        li = lam[i]
        if abs(li.imag) > tol * max(1.0, abs(li)):
            # find the conjugate partner and mark it used
            partner = [j for j in order if j not in used
                       and abs(lam[j] - np.conj(li)) <= 1e-8 * max(1.0, abs(li))]
            if partner:
                used.add(partner[0])
            # fix the eigenvector's complex phase: largest-magnitude component real and positive,
            # so that its real part (kept alone when N_K splits the pair) is well defined
            v = vecs[:, i]
            kmax = np.argmax(np.abs(v))
            v = v * (np.conj(v[kmax]) / np.abs(v[kmax]))
            out_lam.append(li.real)
            out_vec.append(v.real)
            if len(out_vec) < k:
                out_lam.append(li.real)
                out_vec.append(v.imag)
        else:
            out_lam.append(li.real)
            out_vec.append(vecs[:, i].real)
    return np.array(out_lam), np.array(out_vec)


def normalise_direction(beta):
    """Unit 2-norm, largest-magnitude entry positive."""
    nrm = np.linalg.norm(beta)
    if nrm == 0.0:
        raise FloatingPointError("zero update direction")
    beta = beta / nrm
    if beta[np.argmax(np.abs(beta))] < 0:
        beta = -beta
    return beta


def block_solve(S, H, n_keep, m_b):
    """Solve H v = lambda S v (Eq. 5 / 10) and keep the n_keep lowest directions; the rows of
    B^(b) are the beta parts (components 1 .. m_b) of those eigenvectors (Sec. II.B)."""
    lam, vecs = scipy.linalg.eig(H, S)
    lam_k, v_k = _lowest_directions(lam, vecs, n_keep)
    B = np.array([normalise_direction(v[1:1 + m_b]) for v in v_k])
    return lam_k, B, lam


# --------------------------------------------------------------------------------------------
# Sec. II.B, Eq. 6-8: the combined problem and the update.
# --------------------------------------------------------------------------------------------
def combined_matrices(O, G, E, w, offsets, Bs, shift=0.0):
    """Second sweep (Sec. II.B: re-run the same sample): the directions are
    u_bj = sum_i B^(b)_ji Psibar^{i,b} (Eq. 6); their ratios are p_bj = Obar_b . B^(b)_j and
    x_bj = E p_bj + G_b . B^(b)_j.  Returns S_c, H_c of Eq. 7 (dimension 1 + sum_b N_K)."""
    O = np.asarray(O, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    n = O.shape[1]
    m, _ = sample_means(O, E, w)
    Obar = O - m[None, :]
    P, X, C = [], [], []
    for b in range(len(offsets) - 1):
        lo, hi = offsets[b], offsets[b + 1]
        Bb = Bs[b]
        p = Obar[:, lo:hi] @ Bb.T
        r = G[:, lo:hi] @ Bb.T
        P.append(p)
        X.append(E[:, None] * p + r)
        c = np.zeros((n, Bb.shape[0]))
        c[lo:hi, :] = Bb.T
        C.append(c)
    P, X, C = np.hstack(P), np.hstack(X), np.hstack(C)
    return centred_lm_matrices(P, X, E, w, gram=C.T @ C, shift=shift)


def lowest_eigenpair(S, H):
    """Lowest-real-part eigenpair of H c = lambda S c with a real eigenvector (Eq. 7)."""
    lam, vecs = scipy.linalg.eig(H, S)
    finite = np.isfinite(lam)
    order = [i for i in np.argsort(lam.real, kind="stable") if finite[i]]
    i = order[0]
    if abs(lam[i].imag) > 1e-12 * max(1.0, abs(lam[i])):
        raise FloatingPointError("lowest eigenvalue is complex")
    return lam[i].real, vecs[:, i].real


def combined_update(S_c, H_c, offsets, Bs, m):
    """Eq. 8: Delta mu_{i,b} = sum_j A_bj B^(b)_ji / alpha.  The eigenvector (c_0, A) is in the
    centred basis; the coefficient of the raw Psi is alpha = c_0 - sum_bj A_bj (B^(b)_j . m_b)."""
    lam, c = lowest_eigenpair(S_c, H_c)
    n = len(m)
    dmu = np.zeros(n)
    alpha = c[0]
    k = 1
    for b in range(len(offsets) - 1):
        lo, hi = offsets[b], offsets[b + 1]
        Bb = Bs[b]
        A_b = c[k:k + Bb.shape[0]]
        k += Bb.shape[0]
        dmu[lo:hi] = A_b @ Bb
        alpha -= A_b @ (Bb @ m[lo:hi])
    if abs(alpha) < 1e-12 * np.linalg.norm(c):
        raise FloatingPointError("alpha ~ 0: update direction orthogonal to Psi")
    return lam, dmu / alpha


# --------------------------------------------------------------------------------------------
# One whole step, and the traditional linear method for comparison.
# --------------------------------------------------------------------------------------------
def blm_step(O, G, E, w, offsets, n_keep, old_dirs=None, shift=0.0):
    """Both sweeps and both solves of one BLM step.  Returns a dict with the block matrices,
    retained directions, combined matrices, predicted energy and parameter update."""
    O = np.asarray(O, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    E = np.asarray(E, dtype=np.float64)
    m, e_mean = sample_means(O, E, w)
    nb = len(offsets) - 1
    S_b, H_b, lam_b, B = [], [], [], []
    for b in range(nb):
        S, H = block_matrices(O, G, E, w, offsets, b, old_dirs, shift)
        m_b = offsets[b + 1] - offsets[b]
        lam_k, Bb, _ = block_solve(S, H, min(n_keep, m_b), m_b)
        S_b.append(S)
        H_b.append(H)
        lam_b.append(lam_k)
        B.append(Bb)
    S_c, H_c = combined_matrices(O, G, E, w, offsets, B, shift)
    e_pred, dmu = combined_update(S_c, H_c, offsets, B, m)
    return dict(m=m, e_mean=e_mean, S_b=S_b, H_b=H_b, lam_b=lam_b, B=B, S_c=S_c, H_c=H_c,
                e_pred=e_pred, dmu=dmu)


def lm_step(O, G, E, w=None, shift=0.0):
    """Traditional LM (Eq. 1-3) in the raw basis: lowest eigenpair, then Eq. 2."""
    S, H = lm_matrices_raw(O, G, E, w)
    if shift:
        H[1:, 1:] += shift * np.eye(S.shape[0] - 1)
    lam, c = lowest_eigenpair(S, H)
    return lam, c[1:] / c[0]


# --------------------------------------------------------------------------------------------
# Sec. II.B memory discussion: stored matrix elements.
# --------------------------------------------------------------------------------------------
def lm_matrix_bytes(n_params, word=8):
    """H and S of the traditional LM, (1 + N_V)^2 elements each (Sec. II.A)."""
    return 2 * word * (1 + n_params) ** 2


def blm_matrix_bytes_dominant(n_params, n_blocks, n_old, word=8):
    """Dominant BLM storage (Sec. II.B): the Hamiltonian keeps N_V^2/N_B green block elements and
    2 N_V N_O (N_B - 1) block-Theta elements; the overlap keeps N_V^2/N_B and, being symmetric,
    one block-Theta side N_V N_O (N_B - 1)."""
    nv, nb, no = n_params, n_blocks, n_old
    h = nv * nv / nb + 2 * nv * no * (nb - 1)
    s = nv * nv / nb + nv * no * (nb - 1)
    return word * (h + s)
