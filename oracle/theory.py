"""Probability bounds of Section 2.1 and Section 3.

Test infrastructure only (see ``oracle/__init__.py``).

For an m x l matrix H of i.i.d. N(0,1) entries (l >= m):

* Lemma 2.1 (Eq. 3): sigma_max(H) <= sqrt(2 l) alpha with probability at least
  pi_plus = 1 - (2 alpha^2 / e^(alpha^2 - 1))^l / (4 (alpha^2 - 1) sqrt(pi l alpha^2)).
* Lemma 2.2 (Eq. 4): sigma_min(H) >= 1/(sqrt(l) beta) with probability at least
  pi_minus = 1 - (e / ((l - m + 1) beta))^(l-m+1) / sqrt(2 pi (l - m + 1)).
* Lemma 2.3 (Eq. 5): kappa(H) <= sqrt(2) l alpha beta with probability at least
  pi_0 = pi_plus + pi_minus - 1.
* Theorem 3.1: the same bound holds for kappa(P^{-1} A) when G is Gaussian.
* Observation 3.2 (Eq. 10): for m >= 2 and alpha >= 2, pi_0 is at least the
  expression with l replaced by l - m + 2 in the first term.

Values are computed in log space so that tiny failure probabilities do not
underflow.
"""
from __future__ import annotations

import math

__all__ = ["fail_plus", "fail_minus", "pi_plus", "pi_minus", "pi_zero", "pi_zero_simple",
           "kappa_bound"]


def fail_plus(l: int, alpha: float) -> float:
    """1 - pi_plus of Eq. 3."""
    a2 = alpha * alpha
    log_t = l * (math.log(2.0 * a2) - (a2 - 1.0)) - math.log(4.0 * (a2 - 1.0) * math.sqrt(math.pi * l * a2))
    return math.exp(log_t)


def fail_minus(l: int, m: int, beta: float) -> float:
    """1 - pi_minus of Eq. 4."""
    j = l - m + 1
    log_t = j * (1.0 - math.log(j * beta)) - 0.5 * math.log(2.0 * math.pi * j)
    return math.exp(log_t)


def pi_plus(l, alpha):
    return 1.0 - fail_plus(l, alpha)


def pi_minus(l, m, beta):
    return 1.0 - fail_minus(l, m, beta)


def pi_zero(l: int, m: int, alpha: float, beta: float) -> float:
    """Eq. 5."""
    return 1.0 - fail_plus(l, alpha) - fail_minus(l, m, beta)


def pi_zero_simple(l: int, m: int, alpha: float, beta: float) -> float:
    """The lower bound of Eq. 10 (Observation 3.2): l replaced by l - m + 2 in the first term."""
    return 1.0 - fail_plus(l - m + 2, alpha) - fail_minus(l, m, beta)


def kappa_bound(l: int, alpha: float, beta: float) -> float:
    """sqrt(2) l alpha beta (Lemma 2.3, Theorem 3.1)."""
    return math.sqrt(2.0) * l * alpha * beta
