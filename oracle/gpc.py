"""Total-degree Hermite gPC basis (oracle), Section 2.2.
TEST INFRASTRUCTURE ONLY: part of the CPU oracle (imported by tests/,
__graft_entry__.smoke() and bench.py's CPU legs, never by the library).

psi_k(xi) = prod_l psi_{k_l}(xi_l) over the multi-indices with |k|_1 <= p
(eq. complete), P = (p + N_p)! / (p! N_p!).  xi ~ N(0, I) selects the
Hermite family (Table tab:wiener_askey_correspondence); the univariate basis
is orthonormal under the standard normal density: psi_k = He_k / sqrt(k!),
from the three-term recurrence He_{k+1} = x He_k - k He_{k-1}.

Reading: the paper fixes no ordering of the multi-indices.  Here they are
sorted by total degree, and within one degree in decreasing lexicographic
order of (k_1, ..., k_M) (first variable slowest, highest power first).
"""
from __future__ import annotations

import math
import numpy as np


def _exact_degree(M: int, d: int):
    """All k in N_0^M with |k|_1 = d, decreasing lexicographic order."""
    if M == 1:
        yield (d,)
        return
    for first in range(d, -1, -1):
        for rest in _exact_degree(M - 1, d - first):
            yield (first,) + rest


def multi_indices(M: int, p: int) -> np.ndarray:
    out = []
    for d in range(p + 1):
        out.extend(_exact_degree(M, d))
    return np.array(out, dtype=np.int64).reshape(-1, M)


def hermite_orthonormal(kmax: int, x: np.ndarray) -> np.ndarray:
    """Values psi_0..psi_kmax at x, shape [kmax+1, *x.shape]."""
    x = np.asarray(x, dtype=np.float64)
    He = [np.ones_like(x)]
    if kmax >= 1:
        He.append(x.copy())
    for k in range(1, kmax):
        He.append(x * He[k] - k * He[k - 1])
    return np.stack([He[k] / math.sqrt(math.factorial(k)) for k in range(kmax + 1)])


def psi_matrix(xi: np.ndarray, p: int) -> np.ndarray:
    """B-matrix of eq. (least square A): rows psi_1..psi_P at each row of xi."""
    xi = np.atleast_2d(np.asarray(xi, dtype=np.float64))
    S, M = xi.shape
    idx = multi_indices(M, p)
    uni = hermite_orthonormal(p, xi)            # [p+1, S, M]
    B = np.ones((S, len(idx)))
    for j, k in enumerate(idx):
        for l in range(M):
            if k[l]:
                B[:, j] *= uni[k[l], :, l]
    return B
