"""Host-side set logic of the h-p sparse combination (no GPU): the set and
its coefficients against the oracle's expansion of the sparse sum."""
import os

import pytest

from oracle import hp


@pytest.fixture(scope="module")
def hps():
    from paper_1707_09598_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_1707_09598_gb300 import hp_sparse
    return hp_sparse


@pytest.mark.parametrize("d,w,Q,m", [(2, 3, 0, 1), (2, 6, 2, 1), (3, 4, 1, 1), (3, 5, 2, 1), (2, 4, 1, 0)])
def test_coefficients_match_the_oracle(hps, d, w, Q, m):
    assert hps.coefficients(d, w, Q, m) == hp.hp_coefficients_by_expansion(d, w, Q, m)


@pytest.mark.parametrize("d,w,Q", [(2, 5, 2), (3, 4, 1)])
def test_index_set_matches_the_oracle(hps, d, w, Q):
    mine = sorted(hps.index_set(d, w, Q))
    ref = sorted(tuple(b + 1 for b in a[:d]) + (a[d],) for a in hp.hp_index_set(d, w, Q))
    assert mine == ref


def test_degree_and_continuity_limits_are_refused(hps):
    with pytest.raises(ValueError):
        hps.HPCombination(2, 2, 2, 4, 1)       # r = p0: spaces not nested under degree elevation
    with pytest.raises(ValueError):
        hps.HPCombination(2, 3, 1, 4, 2)       # degree 5
