"""Quadrature nodes and MRSDC weights (oracle; test infrastructure only).

Follows Sec. 3 of the paper:

* collocation weights q_{m,j} = int_{t_n}^{tau_m} l_j (Eq. collocation), with
  s_{m,j} = q_{m,j} - q_{m-1,j};
* the four MRSDC weight tables (the definitions following Eq. embedded_quad,
  summarised in Table 1):
      s_{m,j}      = int_{tau_{m-1}}^{tau_m}       l_j          standard -> standard
      shat_{m,q}   = int_{tau_{m-1}}^{tau_m}       l_{m,q}      embedded -> standard
      stil_{m,p,j} = int_{tau_{m,p-1}}^{tau_{m,p}} l_j          standard -> embedded
      s_{m,p,q}    = int_{tau_{m,p-1}}^{tau_{m,p}} l_{m,q}      embedded -> embedded
  where l_j are the Lagrange polynomials of the M standard nodes and l_{m,q}
  those of the P embedded nodes of interval m.

Readings where the paper is silent (each listed in the design notes):

* Node families: 'equi_noleft' (the paper's c_j = j/M), 'radau_right'
  (Radau IIA, right end included) and 'lobatto' (both ends). For Lobatto the
  first interval [t_n, tau_1] has zero length; its weights are all zero.
* Embedded nodes are equidistant inside each interval, tau_{m,p} =
  tau_{m-1} + p (tau_m - tau_{m-1}) / P, so tau_{m,P} = tau_m.
* Embedded interpolation window w: s_{m,p,q} integrates the Lagrange
  polynomials of the w consecutive embedded nodes starting at
  j0 = clamp(p - floor(w/2), 1, P - w + 1) (zero outside the window), and
  shat_{m,q} := sum_p s_{m,p,q}. With w = P this is exactly the paper's
  definition; smaller w bounds the weights for large P.

Weights are returned for a unit step [0, 1]; multiply by dt.

Parity: pinned by tests/test_oracle_weights.py (exact rational identities,
textbook Simpson / Radau IIA / Lobatto weights, polynomial exactness).
"""

from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence

import mpmath as mp
import numpy as np

mp.mp.dps = 60

NODE_KINDS = ("equi_noleft", "radau_right", "lobatto")


# ----------------------------------------------------------------------------
# polynomials with ascending coefficients, over Fraction or mpf
# ----------------------------------------------------------------------------

def _poly_mul(a: Sequence, b: Sequence) -> list:
    out = [0] * (len(a) + len(b) - 1)
    for i, ai in enumerate(a):
        for j, bj in enumerate(b):
            out[i + j] = out[i + j] + ai * bj
    return out


def _poly_integral(coef: Sequence, a, b):
    """int_a^b sum_k coef[k] s^k ds."""
    total = 0
    for k, ck in enumerate(coef):
        total = total + ck * (b ** (k + 1) - a ** (k + 1)) / (k + 1)
    return total


def lagrange_poly(nodes: Sequence, j: int) -> list:
    """Coefficients of l_j with l_j(nodes[i]) = delta_ij."""
    coef = [1]
    denom = 1
    for i, xi in enumerate(nodes):
        if i == j:
            continue
        coef = _poly_mul(coef, [-xi, 1])
        denom = denom * (nodes[j] - xi)
    return [c / denom for c in coef]


def lagrange_integral(nodes: Sequence, j: int, a, b):
    return _poly_integral(lagrange_poly(nodes, j), a, b)


# ----------------------------------------------------------------------------
# standard nodes on [0, 1]
# ----------------------------------------------------------------------------

def _legendre(n: int) -> List[Fraction]:
    """Ascending coefficients of the Legendre polynomial P_n (Bonnet recursion)."""
    p0, p1 = [Fraction(1)], [Fraction(0), Fraction(1)]
    if n == 0:
        return p0
    for k in range(1, n):
        xp1 = [Fraction(0)] + p1
        nxt = [Fraction(0)] * (k + 2)
        for i, c in enumerate(xp1):
            nxt[i] += Fraction(2 * k + 1, k + 1) * c
        for i, c in enumerate(p0):
            nxt[i] -= Fraction(k, k + 1) * c
        p0, p1 = p1, nxt
    return p1


def _real_roots(coef_asc: Sequence[Fraction]) -> list:
    desc = [mp.mpf(c.numerator) / c.denominator for c in reversed(coef_asc)]
    while desc and desc[0] == 0:
        desc = desc[1:]
    roots = mp.polyroots(desc, maxsteps=400, extraprec=400)
    return sorted(mp.re(r) for r in roots)


def standard_nodes(kind: str, M: int, exact: bool = False) -> list:
    """Nodes 0 <= c_1 < ... < c_M <= 1 of one macro step.

    exact=True returns Fractions and is only allowed when the nodes are rational.
    """
    if kind not in NODE_KINDS:
        raise ValueError(kind)
    if M < 1:
        raise ValueError("M >= 1")
    if kind == "equi_noleft":
        return [Fraction(j, M) if exact else mp.mpf(j) / M for j in range(1, M + 1)]
    if kind == "lobatto":
        if M < 2:
            raise ValueError("Lobatto needs M >= 2")
        if exact:
            if M == 2:
                return [Fraction(0), Fraction(1)]
            if M == 3:
                return [Fraction(0), Fraction(1, 2), Fraction(1)]
            raise ValueError("Lobatto nodes are irrational for M > 3")
        if M == 2:
            return [mp.mpf(0), mp.mpf(1)]
        pn = _legendre(M - 1)
        dp = [c * k for k, c in enumerate(pn)][1:]  # P'_{M-1}
        xs = _real_roots(dp)
        return [mp.mpf(0)] + [(x + 1) / 2 for x in xs] + [mp.mpf(1)]
    # Radau IIA: zeros of P_M(x) - P_{M-1}(x) on (-1, 1], mapped to (0, 1]
    if exact:
        if M == 1:
            return [Fraction(1)]
        raise ValueError("Radau nodes are irrational for M > 1")
    pm, pm1 = _legendre(M), _legendre(M - 1)
    diff = [pm[i] - (pm1[i] if i < len(pm1) else 0) for i in range(len(pm))]
    xs = _real_roots(diff)
    cs = [(x + 1) / 2 for x in xs]
    cs[-1] = mp.mpf(1)  # the root x = 1 exactly
    return cs


def collocation_matrix(nodes: Sequence) -> list:
    """q_{m,j} = int_0^{c_m} l_j (Eq. collocation), as nested lists."""
    M = len(nodes)
    return [[lagrange_integral(nodes, j, 0 * nodes[0], nodes[m]) for j in range(M)]
            for m in range(M)]


# ----------------------------------------------------------------------------
# the four MRSDC tables
# ----------------------------------------------------------------------------

def window_start(p: int, P: int, w: int) -> int:
    """First (1-based) embedded node of the interpolation window of substep p."""
    return min(max(p - w // 2, 1), P - w + 1)


def mrsdc_tables(kind: str, M: int, P: int, window: int = 0, exact: bool = False) -> dict:
    """All weights of one MRSDC scheme on the unit step, as nested lists.

    Keys: c (M+1 values, c[0] = 0), emb[m][p] (interval m = 1..M stored at
    index m-1, p = 0..P), S[m][j], Shat[m][q], Stil[m][p][j], Semb[m][p][q]
    (0-based indices), w (window actually used).
    """
    w = min(M, P) if window == 0 else int(window)
    if not 1 <= w <= P:
        raise ValueError("window must be in [1, P]")
    std = standard_nodes(kind, M, exact=exact)
    zero = Fraction(0) if exact else mp.mpf(0)
    c = [zero] + list(std)
    Lstd = [lagrange_poly(std, j) for j in range(M)]
    S = [[zero] * M for _ in range(M)]
    Shat = [[zero] * P for _ in range(M)]
    Stil = [[[zero] * M for _ in range(P)] for _ in range(M)]
    Semb = [[[zero] * P for _ in range(P)] for _ in range(M)]
    emb = []
    for m in range(1, M + 1):
        a, b = c[m - 1], c[m]
        nodes_e = [a + (b - a) * p / P for p in range(P + 1)]
        emb.append(nodes_e)
        if a == b:
            continue  # zero-length interval: every integral over it vanishes
        for j in range(M):
            S[m - 1][j] = _poly_integral(Lstd[j], a, b)
        for p in range(1, P + 1):
            lo, hi = nodes_e[p - 1], nodes_e[p]
            for j in range(M):
                Stil[m - 1][p - 1][j] = _poly_integral(Lstd[j], lo, hi)
            j0 = window_start(p, P, w)
            win = nodes_e[j0:j0 + w]
            for qq in range(w):
                Semb[m - 1][p - 1][j0 - 1 + qq] = lagrange_integral(win, qq, lo, hi)
        for q in range(P):
            acc = zero
            for p in range(P):
                acc = acc + Semb[m - 1][p][q]
            Shat[m - 1][q] = acc
    return {"c": c, "emb": emb, "S": S, "Shat": Shat, "Stil": Stil, "Semb": Semb, "w": w,
            "kind": kind, "M": M, "P": P}


def to_float(x):
    if isinstance(x, list):
        return np.array([to_float(v) for v in x], dtype=np.float64)
    return float(x)  # Fraction and mpf both round to nearest


def mrsdc_weights(kind: str, M: int, P: int, window: int = 0) -> dict:
    """The tables of `mrsdc_tables` rounded to float64 numpy arrays."""
    exact = (kind == "equi_noleft") or (kind == "lobatto" and M <= 3) or (kind == "radau_right" and M == 1)
    t = mrsdc_tables(kind, M, P, window, exact=exact)
    return {
        "c": to_float(t["c"]),
        "emb": to_float(t["emb"]),
        "S": to_float(t["S"]),
        "Shat": to_float(t["Shat"]),
        "Stil": to_float(t["Stil"]),
        "Semb": to_float(t["Semb"]),
        "w": t["w"], "kind": kind, "M": M, "P": P,
    }
