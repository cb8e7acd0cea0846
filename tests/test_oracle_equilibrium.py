"""Pins of the oracle's equilibrium (Eqs. 21, 26) and non-equilibrium recursion (Eq. 22)
against closed forms derived independently of the oracle's code."""
import itertools

import numpy as np

from oracle import rflbm_oracle as o
from paper_2507_08820_gb300 import workloads as W


def _product_form(rho, u):
    """Closed form of the full D3Q27 Hermite equilibrium, derived by hand: because the
    basis, the weights and a_0 = rho u_x^p u_y^q u_z^r all factor over the axes, Eq. 26
    is rho Psi(c_x, u_x) Psi(c_y, u_y) Psi(c_z, u_z) with the 1-D factor
    W(c) [1 + c u / cs2 + (c^2 - cs2) u^2 / (2 cs2^2)], i.e. Psi(0, u) = 2/3 - u^2 and
    Psi(+-1, u) = (1/3 +- u + u^2) / 2."""
    c = o.velocities()

    def psi(ci, ua):
        return np.where(ci[:, None] == 0, 2.0 / 3.0 - ua[None, :] ** 2,
                        (1.0 / 3.0 + ci[:, None] * ua[None, :] + ua[None, :] ** 2) / 2.0)

    return rho[None, :] * psi(c[:, 0], u[0]) * psi(c[:, 1], u[1]) * psi(c[:, 2], u[2])


def test_full_hermite_equilibrium_equals_product_form():
    rho, u = W.random_fields(5, 4, 3, seed=1, drho=0.1, du=0.2)
    assert np.allclose(o.hermite_equilibrium(rho, u), _product_form(rho, u),
                       rtol=0, atol=1e-15)


def test_second_order_truncation_equals_classic_equilibrium():
    """Sec. II.B: truncating Eq. 17 at second order gives Eq. 2 exactly."""
    rho, u = W.random_fields(4, 4, 4, seed=2, drho=0.1, du=0.2)
    assert np.allclose(o.hermite_equilibrium(rho, u, max_order=2),
                       o.second_order_equilibrium(rho, u), rtol=0, atol=1e-15)


def test_equilibrium_moments_are_the_recursive_coefficients():
    """Projecting the product-form equilibrium (Eq. 19) gives rho u_x^p u_y^q u_z^r for
    every mode, which is what Eq. 21's recursion yields; in particular rho and rho u."""
    rho, u = W.random_fields(3, 3, 3, seed=3, drho=0.1, du=0.2)
    m = o.moments(_product_form(rho, u))
    for k, seq in enumerate(o.MODE_SEQ):
        p, q, r = (seq.count(a) for a in "xyz")
        assert np.allclose(m[k], rho * u[0] ** p * u[1] ** q * u[2] ** r, atol=1e-15)
        assert np.allclose(o.a0_coefficient(seq, rho, u), m[k], atol=1e-15)
    assert np.allclose(o.density(_product_form(rho, u)), rho, atol=1e-15)


def _monomial_second_derivative(e, a, b, u):
    """d^2/(du_a du_b) of u_x^e0 u_y^e1 u_z^e2 (plain calculus)."""
    e = list(e)
    coef = 1.0
    for ax in (a, b):
        coef = coef * e[ax]
        e[ax] -= 1
    if min(e) < 0 or coef == 0:
        return np.zeros_like(u[0])
    return coef * u[0] ** e[0] * u[1] ** e[1] * u[2] ** e[2]


def test_nonequilibrium_recursion_equals_derivative_form():
    """Eq. 22 read as the sum over the n-1 pairings of the last index: its closed form is
    a_1^(n) = 1/2 sum_ab a_1^(2)_ab d^2(u_x^p u_y^q u_z^r)/(du_a du_b), the
    linearisation of a_0^(n) = rho u^p u^q u^r around the equilibrium (the recursive
    regularisation of Malaspinas 2015). Checked for every mode of order 2..6."""
    g = np.random.default_rng(4)
    u = g.uniform(-0.2, 0.2, (3, 7))
    a2 = g.normal(size=(3, 3, 7))
    a2 = 0.5 * (a2 + a2.transpose(1, 0, 2))
    pairs = {(x, y): a2["xyz".index(x), "xyz".index(y)] for x in "xyz" for y in "xyz"}
    for k, seq in enumerate(o.MODE_SEQ):
        if len(seq) < 2:
            continue
        e = tuple(seq.count(a) for a in "xyz")
        ref = sum(0.5 * a2[a, b] * _monomial_second_derivative(e, a, b, u)
                  for a in range(3) for b in range(3))
        assert np.allclose(o.a1_coefficient(seq, pairs, u), ref, atol=1e-14), seq


def test_recursion_third_order_textbook_form():
    """a_1,xxy = u_y a_1,xx + 2 u_x a_1,xy (third-order recursive regularisation)."""
    u = np.array([[0.1], [-0.05], [0.02]])
    vals = {"xx": 0.3, "yy": -0.2, "zz": 0.1, "xy": 0.05, "xz": -0.07, "yz": 0.04}
    pairs = {}
    for key, v in vals.items():
        pairs[(key[0], key[1])] = pairs[(key[1], key[0])] = np.array([v])
    got = o.a1_coefficient("xxy", pairs, u)
    assert np.allclose(got, u[1] * 0.3 + 2 * u[0] * 0.05)


def test_recursion_is_symmetric_in_index_order():
    """A Hermite coefficient is a symmetric tensor: every ordering of the same indices
    gives the same a_1^(n)."""
    g = np.random.default_rng(5)
    u = g.uniform(-0.2, 0.2, (3, 4))
    a2 = g.normal(size=(3, 3, 4))
    a2 = a2 + a2.transpose(1, 0, 2)
    pairs = {(x, y): a2["xyz".index(x), "xyz".index(y)] for x in "xyz" for y in "xyz"}
    for seq in ("xxy", "xyzz", "xxyzz", "xxyyzz"):
        vals = [o.a1_coefficient("".join(p), pairs, u) for p in set(itertools.permutations(seq))]
        for v in vals:
            assert np.allclose(v, vals[0], atol=1e-14)
