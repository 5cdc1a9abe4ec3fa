"""Seeded synthetic Monte Carlo samples with the shape of a VMC optimisation step.

For one optimisation (key = (seed, opt)) with n parameters this module draws, sample by sample,
  O_s = Q (sigma * z_s)                    log-derivative ratios <n|Psi^x>/<n|Psi>
  E_s = -1 + O_s . g + 0.01 * eps_s        local energy (eps normal, or Student-t with nu=3)
  G_s = M O_s + 0.01 * Q (sigma * eta_s)   local-energy derivatives dE_L/dmu_x
with z, eta ~ N(0, 1)^n (the derivative noise has the shape of O: a parameter that barely changes
Psi barely changes E_L), sigma_i = 10^(-(d/2) i/(n-1)) (so the population overlap Q diag(sigma^2) Q^T
has spectrum 1 -> 10^-d), Q a product of four Householder reflectors with seeded unit vectors,
g ~ N(0, 1/n)^n and M = Q diag(mu) Q^T with mu_i ~ U(1/2, 3/2).  Weights are 1.
With <E> = -1 the population tangent-space energies are mu_i - 1 in [-1/2, 1/2]: the Psi direction
lies below them, so the lowest eigenvalue of the step is real and separated, as near a VMC minimum.

Every random number is a function of (seed, opt, tag, global index) through Philox4x32-10, so a
chunk is the same whichever way the samples are split.  Nothing here computes any quantity of the
blocked linear method; the oracle and the CUDA library both receive these arrays as inputs.
"""
from dataclasses import dataclass, field
import numpy as np

from . import philox

TAG_HOUSEHOLDER = 1
TAG_G = 2
TAG_MU = 3
TAG_Z = 4
TAG_EPS = 5          # Student-t uses TAG_EPS .. TAG_EPS + 3
TAG_ETA = 9
TAG_BLOCK_SIZE = 10
TAG_BLOCK_STEP = 11
N_REFLECTORS = 4


@dataclass
class Workload:
    name: str
    n: int
    n_samples: int
    block_offsets: list
    n_keep: int
    decades: float = 6.0          # spectrum of the population overlap decays 1 -> 10^-decades
    noise: str = "normal"         # "normal" or "student3" for eps
    chunk: int = 65536
    seed: int = 0
    opt: int = 0
    offset: float = 0.0           # constant added to every O (tests the centring)
    n_old: int = 0

    @property
    def n_blocks(self):
        return len(self.block_offsets) - 1


def equal_blocks(n, nb):
    base, rem = divmod(n, nb)
    offs = [0]
    for b in range(nb):
        offs.append(offs[-1] + base + (1 if b < rem else 0))
    return offs


def uneven_blocks(n, nb, lo, hi, seed=0, opt=0):
    """Block sizes drawn iid from U{lo..hi}, then stepped one at a time (a seeded block, +-1,
    staying in [lo, hi]) until they sum to n."""
    u = philox.uniform(seed, opt, TAG_BLOCK_SIZE, np.arange(nb, dtype=np.uint64))
    sizes = (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)
    sizes = np.minimum(sizes, hi)
    k = 0
    while sizes.sum() != n:
        b = int(np.floor(philox.uniform(seed, opt, TAG_BLOCK_STEP, np.array([k], dtype=np.uint64))[0] * nb))
        b = min(b, nb - 1)
        k += 1
        if sizes.sum() < n and sizes[b] < hi:
            sizes[b] += 1
        elif sizes.sum() > n and sizes[b] > lo:
            sizes[b] -= 1
        if k > 10_000_000:
            raise RuntimeError("block-size adjustment did not converge")
    return [0] + list(np.cumsum(sizes).astype(int))


# The five workloads of the step (the first two run the FP64 path, the third the split-BF16
# path with FP64 solves, the fourth uneven blocks; the fifth, a batch, is generated per member).
def workload(name):
    if name == "n200":
        return Workload("n200", 200, 20000, equal_blocks(200, 4), 5, decades=6.0, chunk=20000)
    if name == "n2048":
        return Workload("n2048", 2048, 200000, equal_blocks(2048, 16), 10, decades=8.0, chunk=65536)
    if name == "n16384":
        return Workload("n16384", 16384, 1000000, equal_blocks(16384, 64), 20, decades=6.0,
                        noise="student3", chunk=65536)
    if name == "n16384u":
        return Workload("n16384u", 16384, 500000, uneven_blocks(16384, 48, 64, 640), 16, decades=6.0,
                        chunk=65536)
    raise KeyError(name)


TAG_BATCH_N = 20
TAG_BATCH_NS = 21
TAG_BATCH_NB = 22


def batch_workloads(count=32, seed=0, max_block=640):
    """The batch of independent optimisations: for optimisation i (opt = i + 1, its own draws),
    n ~ U{500..8000}, N_s ~ U{50000..400000} rounded to a multiple of 256, N_B ~ U{2..32} raised
    to ceil(n / max_block) so that no block exceeds max_block parameters, near-equal contiguous
    blocks, K = min(10, smallest block), normal local-energy noise."""
    idx = np.arange(count, dtype=np.uint64)
    un = philox.uniform(seed, 0, TAG_BATCH_N, idx)
    us = philox.uniform(seed, 0, TAG_BATCH_NS, idx)
    ub = philox.uniform(seed, 0, TAG_BATCH_NB, idx)
    out = []
    for i in range(count):
        n = int(500 + np.floor(un[i] * 7501))
        ns = int(np.round((50000 + np.floor(us[i] * 350001)) / 256.0) * 256)
        nb = int(2 + np.floor(ub[i] * 31))
        nb = max(nb, -(-n // max_block))
        offs = equal_blocks(n, nb)
        k = min(10, min(np.diff(offs)))
        out.append(Workload("batch%d" % i, n, ns, offs, int(k), decades=6.0, chunk=65536,
                            seed=seed, opt=i + 1))
    return out


@dataclass
class Model:
    """The fixed (sample-independent) random draws of one optimisation."""
    n: int
    u: np.ndarray        # N_REFLECTORS x n unit vectors
    sigma: np.ndarray    # n
    g: np.ndarray        # n
    mu: np.ndarray       # n


def make_model(wl: Workload) -> Model:
    n = wl.n
    idx = np.arange(N_REFLECTORS * n, dtype=np.uint64)
    u = philox.normal(wl.seed, wl.opt, TAG_HOUSEHOLDER, idx).reshape(N_REFLECTORS, n)
    u /= np.sqrt(np.sum(u * u, axis=1, keepdims=True))
    i = np.arange(n, dtype=np.float64)
    sigma = 10.0 ** (-(wl.decades / 2.0) * i / max(n - 1, 1))
    g = philox.normal(wl.seed, wl.opt, TAG_G, np.arange(n, dtype=np.uint64)) / np.sqrt(n)
    mu = philox.uniform(wl.seed, wl.opt, TAG_MU, np.arange(n, dtype=np.uint64)) + 0.5
    return Model(n, u, sigma, g, mu)


def _apply_q(model, V):
    """V <- V Q^T row-wise, i.e. each row v -> Q v with Q = H_0 H_1 H_2 H_3."""
    for r in reversed(range(N_REFLECTORS)):
        ur = model.u[r]
        V -= 2.0 * np.outer(V @ ur, ur)
    return V


def _apply_qt(model, V):
    """Each row v -> Q^T v = H_3 H_2 H_1 H_0 v."""
    for r in range(N_REFLECTORS):
        ur = model.u[r]
        V -= 2.0 * np.outer(V @ ur, ur)
    return V


def _eps(wl, s_idx):
    if wl.noise == "normal":
        return philox.normal(wl.seed, wl.opt, TAG_EPS, s_idx)
    if wl.noise == "student3":
        z0 = philox.normal(wl.seed, wl.opt, TAG_EPS, s_idx)
        chi = sum(philox.normal(wl.seed, wl.opt, TAG_EPS + k, s_idx) ** 2 for k in (1, 2, 3))
        return z0 / np.sqrt(chi / 3.0)
    raise ValueError(wl.noise)


def chunk(wl: Workload, model: Model, s0: int, count: int):
    """Samples s0 .. s0+count-1 as float64 arrays O (count x n), G (count x n), E (count)."""
    n = wl.n
    s_idx = np.arange(s0, s0 + count, dtype=np.uint64)
    flat = (s_idx[:, None] * np.uint64(n) + np.arange(n, dtype=np.uint64)[None, :]).ravel()
    z = philox.normal(wl.seed, wl.opt, TAG_Z, flat).reshape(count, n)
    O = _apply_q(model, z * model.sigma[None, :])
    eta = philox.normal(wl.seed, wl.opt, TAG_ETA, flat).reshape(count, n)
    T = _apply_qt(model, O.copy()) * model.mu[None, :] + 0.01 * model.sigma[None, :] * eta
    G = _apply_q(model, T)
    E = -1.0 + O @ model.g + 0.01 * _eps(wl, s_idx)
    if wl.offset:
        O = O + wl.offset
    return O, G, E


def samples(wl: Workload, model: Model = None, count: int = None, dtype=np.float64):
    """All samples (or the first `count`) as contiguous arrays of `dtype` (float32 inputs are the
    float64 draws rounded once)."""
    model = model or make_model(wl)
    count = wl.n_samples if count is None else count
    O = np.empty((count, wl.n), dtype=dtype)
    G = np.empty((count, wl.n), dtype=dtype)
    E = np.empty(count, dtype=dtype)
    step = max(1, min(wl.chunk, (1 << 22) // max(wl.n, 1)))
    for s in range(0, count, step):
        c = min(step, count - s)
        o, g, e = chunk(wl, model, s, c)
        O[s:s + c], G[s:s + c], E[s:s + c] = o, g, e
    return O, G, E
