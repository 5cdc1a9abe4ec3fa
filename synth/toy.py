"""A finite Hilbert space with a linear-parameter ansatz, for exact tests of the step.

Psi(mu) = phi_0 + sum_x mu_x phi_x over D configurations, with a random symmetric Hamiltonian
Hm (D x D).  The vectors are drawn so that the exact ground state psi_g = phi_0 + sum_x a_x phi_x
lies in the self-plus-tangent space at mu = 0: the linear method's eigenproblem then holds
sample by sample (the zero-variance case), and the right update is Delta mu = a exactly.

The per-sample inputs are the ratios a VMC code would hand over:
  O_x = phi_x(i) / Psi(i),  E = (Hm Psi)(i) / Psi(i),  G_x = (Hm phi_x)(i) / Psi(i) - E O_x.
Configurations are drawn uniformly (P = 1/D) and carry the weight w = |Psi(i)|^2 / P, or every
configuration is listed once ("exact" sampling, weights |Psi|^2).
"""
from dataclasses import dataclass
import numpy as np

from . import philox

TAG_TOY_H = 21
TAG_TOY_PHI = 22
TAG_TOY_A = 23
TAG_TOY_SAMPLE = 24


@dataclass
class Toy:
    D: int
    n: int
    Hm: np.ndarray      # D x D symmetric
    phi: np.ndarray     # (1 + n) x D, row 0 is phi_0
    a: np.ndarray       # n, the exact update
    e_ground: float
    psi_g: np.ndarray


def make_toy(D=48, n=12, seed=0, opt=0):
    A = philox.normal(seed, opt, TAG_TOY_H, np.arange(D * D, dtype=np.uint64)).reshape(D, D)
    Hm = 0.5 * (A + A.T) + np.diag(np.linspace(0.0, 4.0, D))
    evals, evecs = np.linalg.eigh(Hm)
    psi_g = evecs[:, 0]
    # keep Psi nonzero on every configuration: psi_g plus a small positive background is
    # not needed since phi_0 is drawn below; instead resample rows until |Psi| is bounded away
    phi = philox.normal(seed, opt, TAG_TOY_PHI, np.arange((1 + n) * D, dtype=np.uint64)).reshape(1 + n, D)
    a = 0.3 * philox.normal(seed, opt, TAG_TOY_A, np.arange(n, dtype=np.uint64))
    phi[0] = psi_g * np.sqrt(D) - a @ phi[1:]     # phi_0 + a . phi = sqrt(D) psi_g
    return Toy(D, n, Hm, phi, a, float(evals[0]), psi_g)


def psi(toy, mu):
    return toy.phi[0] + mu @ toy.phi[1:]


def ratios(toy, mu, configs):
    """O (len x n), G (len x n), E (len) at parameters mu for the listed configurations."""
    P = psi(toy, mu)
    HP = toy.Hm @ P
    Hphi = toy.phi[1:] @ toy.Hm            # rows: (Hm phi_x)^T (Hm symmetric)
    den = P[configs]
    O = (toy.phi[1:, configs] / den).T
    E = HP[configs] / den
    G = (Hphi[:, configs] / den).T - E[:, None] * O
    return O, G, E


def sample(toy, mu, n_samples, seed=0, opt=0):
    """Uniformly drawn configurations with weights |Psi|^2 / P (P = 1/D)."""
    u = philox.uniform(seed, opt, TAG_TOY_SAMPLE, np.arange(n_samples, dtype=np.uint64))
    configs = np.minimum((u * toy.D).astype(np.int64), toy.D - 1)
    O, G, E = ratios(toy, mu, configs)
    w = psi(toy, mu)[configs] ** 2 * toy.D
    return O, G, E, w


def exact(toy, mu):
    """Every configuration once with weight |Psi|^2: the infinite-sampling limit."""
    configs = np.arange(toy.D)
    O, G, E = ratios(toy, mu, configs)
    w = psi(toy, mu) ** 2
    return O, G, E, w


def energy(toy, mu):
    P = psi(toy, mu)
    return float(P @ toy.Hm @ P / (P @ P))
