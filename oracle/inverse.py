"""Iterative inversion of a hierarchical matrix from products (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Follows Appendix A of the paper:
* Newton-Schulz: X_{k+1} = (2I - X_k A) X_k (Algorithm 1, without the
  stabilisation step), globally convergent for symmetric positive definite A
  from a scaled identity X_0 = alpha I with 0 < alpha < 2 / lambda_max(A).
* Order-l hyperpower iteration (Eq. A.1): X_{k+1} = X_k sum_{i<l} R_k^i,
  R_k = I - A X_k; l = 2 is Newton-Schulz.  Its samples Y = X_{k+1} Omega are
  accumulated as in Algorithm 4: Y = R = Omega; l - 1 times R <- (I - A X_k) R,
  Y <- Y + R; finally Y <- X_k Y.
* Hierarchical iteration (Algorithm 2): every iterate is a new H^2 matrix
  constructed (Section 3.3) from the sampler of the previous one, to a
  construction threshold eps_k chosen from the current residual
  E = ||A X_k - I||_2 (the paper's dynamic threshold; reading below).
* Warm start and unrolled iterations (Appendix A, "Unrolling iterations"): the
  iteration may start from a given X_0 (a previous approximate inverse), and k
  Newton-Schulz steps may be constructed at once: X_k = X_0 prod_{j<k} (I + R_0^(2^j))
  = X_0 sum_{i<2^k} R_0^i, R_0 = I - A X_0 (R_{j+1} = R_j^2 for Newton-Schulz), i.e.
  the order-2^k hyperpower step.  Reading: the paper prints this as
  X_{k-1}(2I + AX_{k-1}) and a binomial sum up to 2^k, which is not the Newton-Schulz
  iteration; the geometric sum above is what k unrolled Newton-Schulz steps equal.

Readings (the paper leaves them open): alpha = 1 / ||A||_2 with ||A||_2 from
power iteration (the paper uses 1/||A||_inf; any alpha in (0, 2/lambda_max)
converges).  A construction error eps_k relative to ||X|| moves A X by up to
kappa_k eps_k, kappa_k = ||A||_2 ||X_k||_2 (||X_k|| from the construction's own
norm estimate, alpha for X_0), and the residual squares at every Newton-Schulz
step, so eps_k = max(eps / kappa_k, min(eps_loose, theta E^2)) (eps_loose = eps
gives the static threshold).  E from power iteration on (X A - I)(A X - I),
stopped at 1e-2 relative change.  The iteration stops at E <= eps, after
max_iter iterates, or when it stalls: the new residual is above 0.9 of the
previous one although the exact iteration would have reached less than half of
it (E_{k+1} > 0.9 E_k and E_k^l < 0.5 E_{k+1}: the construction floor).
"""
from __future__ import annotations

import numpy as np

from . import rng
from .h2 import matvec


def hyperpower_sample(apply_X, apply_A, omega: np.ndarray, order: int) -> np.ndarray:
    """Y = X_{k+1} Omega for the order-`order` hyperpower iterate of X_k (Algorithm 4)."""
    if order < 2:
        raise ValueError("order must be >= 2")
    Y = omega.copy()
    R = omega.copy()
    for _ in range(order - 1):
        R = R - apply_A(apply_X(R))
        Y = Y + R
    return apply_X(Y)


def construction_threshold(E: float, eps_floor: float, eps_loose: float, theta: float) -> float:
    return max(eps_floor, min(eps_loose, theta * E * E))


def residual_norm(apply_A, apply_X, N: int, seed: int, maxit: int = 50, rtol: float = 1e-2) -> float:
    """||A X - I||_2 by power iteration on (X A - I)(A X - I) (A, X symmetric)."""
    v = rng.gaussian(seed, rng.STREAM_ERR, 0, np.arange(N, dtype=np.uint64)[:, None],
                     np.zeros((1, 1), dtype=np.uint64))[:, 0]
    v = v / np.linalg.norm(v)
    E, prev = 0.0, 0.0
    for it in range(maxit):
        w = apply_A(apply_X(v[:, None]))[:, 0] - v
        E = float(np.linalg.norm(w))
        z = apply_X(apply_A(w[:, None]))[:, 0] - w
        nz = float(np.linalg.norm(z))
        if nz == 0.0:
            break
        v = z / nz
        if it > 0 and abs(E - prev) <= rtol * E:
            break
        prev = E
    return E


class Sampler:
    """Operator whose products are the samples of the next iterate (Algorithm 3 / 4)."""

    def __init__(self, apply_X, apply_A, order: int):
        self.apply_X, self.apply_A, self.order = apply_X, apply_A, order

    def __call__(self, omega: np.ndarray) -> np.ndarray:
        return hyperpower_sample(self.apply_X, self.apply_A, np.asarray(omega, dtype=np.float64), self.order)


class InvertResult:
    def __init__(self):
        self.errors = []          # E before each iteration, and the final one
        self.eps_k = []           # construction threshold of each iterate
        self.samples = []         # peeling products of each iterate's construction
        self.alpha = 0.0
        self.h2 = None


def hns_invert(apply_A, norm_A: float, build, N: int, order: int = 2, eps: float = 1e-6,
               eps_loose: float = 1e-6, theta: float = 0.1, max_iter: int = 50, seed: int = 9,
               x0=None, unroll: int = 0) -> InvertResult:
    """Hierarchical hyperpower inversion of the symmetric positive definite A (Algorithm 2).

    build(op, tol) -> (H2Matrix, PeelResult) constructs an iterate from its sampler.
    x0: optional (apply_X0, norm_X0) warm start; unroll = k >= 1: one construction of the k-th
    Newton-Schulz iterate of X_0 (order 2^k, one iterate)."""
    res = InvertResult()
    res.alpha = 1.0 / norm_A
    apply_X = lambda v: res.alpha * v
    norm_X = res.alpha
    if x0 is not None:
        apply_X, norm_X = x0
    if unroll > 0:
        order, max_iter = 1 << unroll, 1
    for k in range(max_iter + 1):
        E = residual_norm(apply_A, apply_X, N, seed)
        res.errors.append(E)
        if E <= eps or k == max_iter:
            break
        if k > 0:
            Ep = res.errors[-2]
            if E > 0.9 * Ep and Ep ** order < 0.5 * E:
                break
        # an unrolled step is the final construction: built to the floor the target allows
        eps_k = (eps / (norm_A * norm_X) if unroll > 0
                 else construction_threshold(E, eps / (norm_A * norm_X), eps_loose, theta))
        h, peel_res = build(Sampler(apply_X, apply_A, order), eps_k)
        res.eps_k.append(eps_k)
        res.samples.append(int(peel_res.samples - peel_res.norm_its))
        res.h2 = h
        norm_X = float(peel_res.norm_est)
        apply_X = (lambda hh: (lambda v: matvec(hh, v)))(h)
    return res
