"""Error bounds and counts of Sec. IV (oracle; test infrastructure only).

* noise rate ||M_E - I|| (spectral norm), as defined in Sec. IV;
* Theorem 1: |F - A(l)| < (1+8p)^N - sum_{i<=l} C(N,i) (4p)^i (1+4p)^(N-i),
  and 2 sum_{i<=l} C(N,i) 3^i contractions;
* the level-1 corollary: <= 32 sqrt(e) N^2 p^2 when p <= 1/(8N);
* a per-site bound: the dropped part of the expansion is a sum over site sets
  S with |S| > l of products of ||M-bar_s|| (s in S) and ||M'_s|| (s not in
  S), each gate superoperator U (x) U^* having norm 1 and |psi>, |v> unit
  vectors.
"""

import math

import numpy as np

from .expansion import matrix_representation, dominant_and_rest


def spectral_norm(m):
    return float(np.linalg.norm(m, 2))


def noise_rate(kraus):
    return spectral_norm(matrix_representation(kraus) - np.eye(4))


def theorem1_bound(n_noise, p, level):
    level = min(level, n_noise)
    head = sum(math.comb(n_noise, i) * (4 * p) ** i * (1 + 4 * p) ** (n_noise - i)
               for i in range(level + 1))
    return (1 + 8 * p) ** n_noise - head


def level1_corollary(n_noise, p):
    return 32.0 * math.sqrt(math.e) * n_noise ** 2 * p ** 2


def contraction_count(n_noise, level):
    level = min(level, n_noise)
    return 2 * sum(math.comb(n_noise, i) * 3 ** i for i in range(level + 1))


def per_site_bound(kraus_lists, level):
    """sum over |S| > level of prod_{s in S} ||M-bar_s|| prod_{s not in S} ||M'_s||,
    by the coefficients of prod_s (||M'_s|| + ||M-bar_s|| x)."""
    poly = [1.0]
    for k in kraus_lists:
        m_dom, m_rest = dominant_and_rest(k)
        a, b = spectral_norm(m_rest), spectral_norm(m_dom)
        nxt = [0.0] * (len(poly) + 1)
        for i, c in enumerate(poly):
            nxt[i] += c * b
            nxt[i + 1] += c * a
        poly = nxt
    return math.fsum(poly[level + 1:])
