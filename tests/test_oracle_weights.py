"""Pins for oracle.weights: quadrature nodes and the MRSDC weight tables (Sec. 3).

Everything here is checked against values fixed by mathematics: textbook
Lobatto / Radau IIA nodes and weights, hand-computed Lagrange integrals, the
consistency identities stated after Eq. discrete-node-to-node-embedded, and
exactness on polynomials.
"""

from fractions import Fraction as F
import math
import os

import mpmath as mp
import numpy as np
import pytest

from oracle import weights as wt


def test_simpson_from_lobatto3():
    # Gauss-Lobatto with 3 nodes is Simpson's rule: 1/6, 2/3, 1/6 on [0, 1].
    nodes = wt.standard_nodes("lobatto", 3, exact=True)
    assert nodes == [F(0), F(1, 2), F(1)]
    q = wt.collocation_matrix(nodes)
    assert q[2] == [F(1, 6), F(2, 3), F(1, 6)]
    # the Lobatto IIIA tableau row for c = 1/2: 5/24, 1/3, -1/24
    assert q[1] == [F(5, 24), F(1, 3), F(-1, 24)]


def test_lobatto4_nodes_and_weights():
    s5 = math.sqrt(5.0)
    nodes = [float(x) for x in wt.standard_nodes("lobatto", 4)]
    np.testing.assert_allclose(nodes, [0.0, (5 - s5) / 10, (5 + s5) / 10, 1.0], atol=1e-15)
    q = wt.collocation_matrix(wt.standard_nodes("lobatto", 4))
    np.testing.assert_allclose([float(v) for v in q[3]], [1 / 12, 5 / 12, 5 / 12, 1 / 12], atol=1e-15)


def test_radau_iia_tableaux():
    # Radau IIA, s = 2: c = (1/3, 1), A = [[5/12, -1/12], [3/4, 1/4]]
    n2 = wt.standard_nodes("radau_right", 2)
    np.testing.assert_allclose([float(x) for x in n2], [1 / 3, 1.0], atol=1e-15)
    A2 = np.array([[float(v) for v in row] for row in wt.collocation_matrix(n2)])
    np.testing.assert_allclose(A2, [[5 / 12, -1 / 12], [3 / 4, 1 / 4]], atol=1e-15)
    # Radau IIA, s = 3: c = ((4 - sqrt6)/10, (4 + sqrt6)/10, 1), b = ((16 - sqrt6)/36, (16 + sqrt6)/36, 1/9)
    s6 = math.sqrt(6.0)
    n3 = wt.standard_nodes("radau_right", 3)
    np.testing.assert_allclose([float(x) for x in n3], [(4 - s6) / 10, (4 + s6) / 10, 1.0], atol=1e-15)
    b3 = [float(v) for v in wt.collocation_matrix(n3)[2]]
    np.testing.assert_allclose(b3, [(16 - s6) / 36, (16 + s6) / 36, 1 / 9], atol=1e-15)
    # s = 4 nodes (tabulated values)
    n4 = [float(x) for x in wt.standard_nodes("radau_right", 4)]
    np.testing.assert_allclose(n4, [0.088587959512704, 0.409466864440735, 0.787659461760847, 1.0],
                               atol=1e-12)


def test_equidistant_noleft_by_hand():
    # nodes 1/2, 1: l_1 = 2(1 - s), l_2 = 2s - 1
    nodes = wt.standard_nodes("equi_noleft", 2, exact=True)
    assert nodes == [F(1, 2), F(1)]
    q = wt.collocation_matrix(nodes)
    assert q == [[F(3, 4), F(-1, 4)], [F(1), F(0)]]
    t = wt.mrsdc_tables("equi_noleft", 2, 2, window=2, exact=True)
    # s_{m,j} = q_{m,j} - q_{m-1,j}
    assert t["S"] == [[F(3, 4), F(-1, 4)], [F(1, 4), F(1, 4)]]
    # substep [0, 1/4] of interval 1: int_0^{1/4} 2(1-s) = 7/16, int_0^{1/4} (2s-1) = -3/16
    assert t["Stil"][0][0] == [F(7, 16), F(-3, 16)]
    # embedded nodes of interval 1: 1/4, 1/2; l = (1/2 - s)/(1/4), (s - 1/4)/(1/4)
    # int_0^{1/4}: (1/2*1/4 - 1/32)*4 = 3/8, (1/32 - 1/16)*4 = -1/8
    assert t["Semb"][0][0] == [F(3, 8), F(-1, 8)]


@pytest.mark.parametrize("kind,M,P,w", [("equi_noleft", 3, 2, 0), ("equi_noleft", 3, 8, 8),
                                        ("equi_noleft", 5, 8, 8), ("lobatto", 3, 20, 0),
                                        ("equi_noleft", 4, 20, 4)])
def test_consistency_identities_exact(kind, M, P, w):
    # s_{m,j} = sum_p stil_{m,p,j} and shat_{m,q} = sum_p s_{m,p,q}
    t = wt.mrsdc_tables(kind, M, P, window=w, exact=True)
    for m in range(M):
        for j in range(M):
            assert t["S"][m][j] == sum(t["Stil"][m][p][j] for p in range(P))
        for q in range(P):
            assert t["Shat"][m][q] == sum(t["Semb"][m][p][q] for p in range(P))
        # embedded steps add up to the interval
        emb = t["emb"][m]
        assert emb[0] == t["c"][m] and emb[P] == t["c"][m + 1]


@pytest.mark.parametrize("kind,M,P", [("equi_noleft", 3, 2), ("equi_noleft", 3, 8), ("lobatto", 3, 5)])
def test_literal_shat_is_the_interval_integral(kind, M, P):
    # with w = P, shat_{m,q} = int_{tau_{m-1}}^{tau_m} l_{m,q} (the paper's definition)
    t = wt.mrsdc_tables(kind, M, P, window=P, exact=True)
    for m in range(M):
        a, b = t["c"][m], t["c"][m + 1]
        if a == b:
            continue
        nodes_e = t["emb"][m][1:]
        for q in range(P):
            assert t["Shat"][m][q] == wt.lagrange_integral(nodes_e, q, a, b)


@pytest.mark.parametrize("kind,M,P,w", [("radau_right", 4, 40, 0), ("lobatto", 3, 20, 0),
                                        ("equi_noleft", 5, 8, 8), ("radau_right", 3, 7, 5)])
def test_polynomial_exactness(kind, M, P, w):
    W = wt.mrsdc_weights(kind, M, P, w)
    c, emb = W["c"], W["emb"]
    ww = W["w"]
    for deg in range(M):
        f = lambda s: s ** deg
        Fint = lambda a, b: (b ** (deg + 1) - a ** (deg + 1)) / (deg + 1)
        for m in range(M):
            got = np.dot(W["S"][m], f(c[1:]))
            assert abs(got - Fint(c[m], c[m + 1])) < 1e-14
            for p in range(P):
                got = np.dot(W["Stil"][m, p], f(c[1:]))
                assert abs(got - Fint(emb[m][p], emb[m][p + 1])) < 1e-14
    for deg in range(ww):
        f = lambda s: s ** deg
        Fint = lambda a, b: (b ** (deg + 1) - a ** (deg + 1)) / (deg + 1)
        for m in range(M):
            got = np.dot(W["Shat"][m], f(emb[m][1:]))
            assert abs(got - Fint(c[m], c[m + 1])) < 1e-13
            for p in range(P):
                got = np.dot(W["Semb"][m, p], f(emb[m][1:]))
                assert abs(got - Fint(emb[m][p], emb[m][p + 1])) < 1e-14


def test_window_start_and_zero_length_interval():
    assert [wt.window_start(p, 20, 3) for p in (1, 2, 3, 10, 19, 20)] == [1, 1, 2, 9, 18, 18]
    assert [wt.window_start(p, 8, 8) for p in range(1, 9)] == [1] * 8
    W = wt.mrsdc_weights("lobatto", 3, 20)
    # Lobatto: interval 1 is [t_n, t_n]; all of its weights vanish
    assert not W["S"][0].any() and not W["Shat"][0].any()
    assert not W["Stil"][0].any() and not W["Semb"][0].any()


def test_large_P_literal_weights_amplify():
    # the literal (w = P) embedded weights grow fast with P; the window keeps them bounded
    lit = wt.mrsdc_weights("equi_noleft", 1, 20, window=20)
    win = wt.mrsdc_weights("equi_noleft", 1, 20, window=0)
    dtp = 1.0 / 20
    amp_lit = np.abs(lit["Semb"][0]).sum(axis=1).max() / dtp
    amp_win = np.abs(win["Semb"][0]).sum(axis=1).max() / dtp
    assert amp_lit > 1e4 and amp_win < 2.0 + 1e-12


def test_float_tables_round_high_precision_values():
    W = wt.mrsdc_weights("radau_right", 4, 40)
    t = wt.mrsdc_tables("radau_right", 4, 40)
    assert W["S"][2, 1] == float(t["S"][2][1])
    assert W["Semb"][3, 7, 6] == float(t["Semb"][3][7][6])
    assert isinstance(t["S"][2][1], mp.mpf)


def _golden(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    with open(path) as f:
        return [line.split() for line in f if line.strip() and not line.startswith("#")]


def test_node_layout_of_the_sec3_figure():
    # tests/golden/nodes_equi_noleft_M4_P3.txt: the M = 4, P = 3 layout of the node figure of Sec. 3
    t = wt.mrsdc_tables("equi_noleft", 4, 3, exact=True)
    rows = _golden("nodes_equi_noleft_M4_P3.txt")
    for kind, m, p, pos in rows:
        want = F(pos)
        if kind == "standard":
            assert t["c"][int(m)] == want, (m, t["c"][int(m)], want)
        else:
            assert t["emb"][int(m) - 1][int(p)] == want, (m, p)
    assert len([r for r in rows if r[0] == "embedded"]) == 4 * 3
    # t_n (0) is no standard node, and each interval's embedded set ends on its standard node
    assert F(0) not in t["c"][1:]
    assert all(t["emb"][m][3] == t["c"][m + 1] for m in range(4))

