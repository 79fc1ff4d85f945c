"""Oracle pins for the homomorphic polynomial evaluation (the activations of
the paper's Criteo models are polynomials: Sec. 2.1.4, Sec. 5.4): the product
tree's structure and depth, the decrypted result against the polynomial
evaluated in the clear, the simulated output level and scale against the
evaluation's own, and the SiLU stand-in's fit."""
import numpy as np
import pytest

from oracle import ckks, poly
from paper_2506_18150_gb300 import synthetic as syn


def test_tree_structure_and_depth():
    assert poly.depth(1) == 1 and poly.depth(2) == 2 and poly.depth(3) == poly.depth(4) == 3
    assert [poly.depth(d) for d in (5, 8, 9, 16)] == [4, 4, 5, 5]
    dense = [1.0] * 17                                  # every power 2..16
    tree = poly.product_tree(dense)
    assert [k for k, _, _ in tree] == list(range(2, 17))
    for k, a, b in tree:
        assert a + b == k and a & (a - 1) == 0 and a >= b
        # both operands sit above x^k: x^k is one product below the deeper one
        assert max(poly.power_depth(a), poly.power_depth(b)) + 1 == poly.power_depth(k)
    # only the powers a non-zero coefficient needs, with their operands
    assert poly.product_tree([0, 1, 0, 0, 0, 0, 1]) == [(2, 1, 1), (4, 2, 2), (6, 4, 2)]
    assert poly.product_tree([0, 0, 0, 0, 0, 0, 0, 1]) == [(2, 1, 1), (3, 2, 1), (4, 2, 2), (7, 4, 3)]
    assert poly.product_tree([1, 2]) == []


@pytest.mark.parametrize("coeffs", [
    (0.0, 1.0),                                   # degree 1: one constant multiplication
    (0.0, 0.0, 1.0),                              # x^2
    (0.5, -1.0, 0.0, 2.0),                        # a cubic with a gap
    (0.1, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.01),    # only x^7 (powers 2, 3, 4, 7)
    "silu",
])
def test_poly_eval_decrypts_to_the_polynomial(small_params, coeffs):
    p = small_params
    if coeffs == "silu":
        coeffs = syn.silu_poly(7)
    sk, keys = ckks.keygen(p, 31, relin=True)
    rng = np.random.default_rng(5)
    x = rng.uniform(-1, 1, p.n)
    lvl = p.L
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, x, p.delta), lvl, p.delta, 77)
    y = poly.poly_eval(p, keys, ct, coeffs, p.delta)
    d = len(coeffs) - 1
    assert y.level == lvl - poly.depth(d)
    assert (y.level, y.scale) == poly.simulate(p.q, lvl, p.delta, coeffs, p.delta)
    assert abs(y.scale / p.delta - 1) < 1e-3
    want = np.polynomial.polynomial.polyval(x, np.asarray(coeffs))
    got = ckks.decrypt(p, sk, y)
    assert np.max(np.abs(got - want)) < 1e-4


def test_poly_eval_refuses_what_it_cannot_do(small_params):
    p = small_params
    _, keys = ckks.keygen(p, 32, relin=True)
    ct = ckks.encrypt(p, keys, ckks.encode_real(p, np.zeros(p.n), p.delta), 2, p.delta, 1)
    with pytest.raises(ValueError):
        poly.poly_eval(p, keys, ct, (1.0, 0.0, 0.0, 0.0, 1.0), p.delta)   # depth 3 at level 2
    with pytest.raises(ValueError):
        poly.poly_eval(p, keys, ct, (1.0,), p.delta)                       # constant


def test_silu_fit():
    """The SiLU stand-in: even apart from x/2 (so its odd terms above x^1 are
    exact zeros and its degree is 6), within 0.06 of SiLU on [-6, 6]."""
    c = syn.silu_poly(7)
    assert len(c) == 7 and c[3] == 0.0 and c[5] == 0.0 and abs(c[1] - 0.5) < 1e-12
    x = np.linspace(-6, 6, 2001)
    err = np.polynomial.polynomial.polyval(x, np.asarray(c)) - x / (1 + np.exp(-x))
    assert np.max(np.abs(err)) < 0.06
