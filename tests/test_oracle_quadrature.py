"""Pins of the quadrature rules: exactness on monomials (closed-form simplex moments)."""
import math

import numpy as np
import pytest

from oracle import quadrature as Q


def simplex_moment(exps):
    """int over the unit simplex of prod x_i^a_i, normalized by the simplex measure."""
    d = len(exps)
    num = math.prod(math.factorial(a) for a in exps)
    return num * math.factorial(d) / math.factorial(sum(exps) + d)


@pytest.mark.parametrize("rule,deg,dim", [
    (Q.tet4, 2, 3), (Q.tri3, 2, 2),
    (lambda: Q.tet_conical(2), 3, 3), (lambda: Q.tet_conical(3), 5, 3), (lambda: Q.tet_conical(4), 7, 3),
    (lambda: Q.tri_conical(2), 3, 2), (lambda: Q.tri_conical(3), 5, 2),
])
def test_rule_exact_to_degree(rule, deg, dim):
    lam, w = rule()
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.all(w > 0) and np.all(lam >= 0)
    x = lam[:, 1:]
    for exps in np.ndindex(*(deg + 1,) * dim):
        if sum(exps) > deg:
            continue
        val = (w * np.prod(x ** np.array(exps), axis=1)).sum()
        assert abs(val - simplex_moment(exps)) < 1e-13, exps
