"""Pins of the oracle's lattice tables against the paper's Tables I-II and against the
algebra those tables must satisfy (exact rationals, orthogonality, isotropy)."""
import itertools
import math
from fractions import Fraction

import numpy as np

from conftest import read_golden
from oracle import rflbm_oracle as o


def test_velocity_set_is_the_full_d3q27_cube_grouped_as_table1():
    c = o.velocities()
    assert c.shape == (27, 3)
    assert sorted(map(tuple, c)) == sorted(itertools.product((-1, 0, 1), repeat=3))
    for first, last, norm2, _ in read_golden("table1_d3q27.txt"):
        block = c[int(first):int(last) + 1]
        assert np.all((block * block).sum(axis=1) == int(norm2))


def test_weights_match_table1():
    w = o.weights()
    for first, last, _, wt in read_golden("table1_d3q27.txt"):
        assert np.allclose(w[int(first):int(last) + 1], float(Fraction(wt)), rtol=0, atol=1e-16)


def test_weight_moments_isotropy():
    """sum w = 1, odd moments vanish, sum w c_a c_b = cs2 delta, and the fourth moment
    is cs2^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc): the isotropy a D3Q27 quadrature needs."""
    c, w = o.velocities().astype(float), o.weights()
    d = np.eye(3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(w @ c, 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), o.CS2 * d, atol=1e-16)
    m3 = np.einsum("i,ia,ib,ic->abc", w, c, c, c)
    assert np.allclose(m3, 0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, o.CS2 ** 2 * iso, atol=1e-16)


def test_opposite_is_an_involution_mapping_c_to_minus_c():
    c, opp = o.velocities(), o.opposite()
    assert np.all(c[opp] == -c)
    assert np.all(opp[opp] == np.arange(27))


def test_norms_match_table2_and_eq23():
    """b_k = sum_i w_i e_ki^2 (Eq. 6) equals Table II's printed b_k and n_k! cs^(2 n_k)/mu_k
    (Eq. 23) with Table II's n_k and mu_k."""
    b = o.norms()
    rows = read_golden("table2_hermite.txt")
    assert len(rows) == 27
    for k, sym, n, mu, bk in rows:
        k, n, mu = int(k), int(n), int(mu)
        assert abs(b[k] - float(Fraction(bk))) < 1e-15, (k, b[k], bk)
        assert abs(b[k] - math.factorial(n) * o.CS2 ** n / mu) < 1e-15
        assert o.MODE_ORDER[k] == n and o.MODE_MULT[k] == mu
        assert o.MODE_SEQ[k] == ("" if sym == "1" else sym)


def test_basis_orthogonal_under_weighted_product():
    """sum_i w_i e_ki e_li = b_k delta_kl (Sec. II.A, below Eq. 5)."""
    E, w = o.basis(), o.weights()
    G = (E * w) @ E.T
    assert np.allclose(G, np.diag(o.norms()), rtol=0, atol=1e-15)


def test_inverse_transform_is_the_inverse():
    """M_ki = e_ki and M^-1_ik = w_i b_k^-1 e_ki (Sec. II.B): M^-1 M = M M^-1 = I."""
    E, w, b = o.basis(), o.weights(), o.norms()
    Minv = (w[:, None] * E.T) / b[None, :]
    assert np.allclose(Minv @ E, np.eye(27), atol=1e-13)
    assert np.allclose(E @ Minv, np.eye(27), atol=1e-13)


def test_basis_rows_are_products_of_1d_hermite_polynomials():
    """Each e_k of Table II is h_p(c_x) h_q(c_y) h_r(c_z) with h_0 = 1, h_1 = c,
    h_2 = c^2 - cs2, where (p, q, r) counts x, y, z in the Hermite symbol."""
    E, c = o.basis(), o.velocities().astype(float)
    h = [lambda v: np.ones_like(v), lambda v: v, lambda v: v * v - o.CS2]
    for k, seq in enumerate(o.MODE_SEQ):
        p, q, r = (seq.count(a) for a in "xyz")
        assert max(p, q, r) <= 2 and p + q + r == o.MODE_ORDER[k]
        assert np.allclose(E[k], h[p](c[:, 0]) * h[q](c[:, 1]) * h[r](c[:, 2]), atol=1e-15)
    exps = {tuple(seq.count(a) for a in "xyz") for seq in o.MODE_SEQ}
    assert len(exps) == 27


def test_exact_rationals_of_the_weights_with_fractions():
    """Re-derive every b_k in exact rational arithmetic (no floating point)."""
    third = Fraction(1, 3)
    wt = {0: Fraction(8, 27), 1: Fraction(2, 27), 2: Fraction(1, 54), 3: Fraction(1, 216)}
    h = [lambda v: Fraction(1), lambda v: Fraction(v), lambda v: Fraction(v * v) - third]
    rows = read_golden("table2_hermite.txt")
    for k, sym, _, _, bk in rows:
        seq = "" if sym == "1" else sym
        p, q, r = (seq.count(a) for a in "xyz")
        tot = Fraction(0)
        for cx, cy, cz in itertools.product((-1, 0, 1), repeat=3):
            e = h[p](cx) * h[q](cy) * h[r](cz)
            tot += wt[cx * cx + cy * cy + cz * cz] * e * e
        assert tot == Fraction(bk), (k, tot, bk)
