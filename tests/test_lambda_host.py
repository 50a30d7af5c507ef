"""The library's host-side fit and choice of the viscosity scaling factor
(ns_energy_efolds, ns_lambda_select: pure host functions, callable without a GPU)
against the oracle's, on the paper's table and on random series."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from tests.test_oracle_lambda import _table


@pytest.fixture(scope="module")
def api():
    from paper_1511_06959_gb300 import api, build
    import os
    if not os.path.exists(build.OUT):
        build.build()
    return api


def test_efolds_match_oracle_per_box(api):
    rng = np.random.default_rng(8)
    for N in (2, 3, 9, 40):
        B = 3
        E = np.exp(rng.normal(scale=2.0, size=(N + 1, B)))
        E[:, 2] = [7.0 * math.exp(0.25 * (N - m)) for m in range(N + 1)]
        got = api.energy_efolds(E.tolist(), N, B)
        for b in range(B):
            assert got[b] == pytest.approx(O.energy_efolds(E[:, b]), rel=1e-12, abs=1e-12)
        E[1, 0] = 0.0
        assert api.energy_efolds(E.tolist(), N, B)[0] == math.inf


def test_efolds_rejects_short_series(api):
    with pytest.raises(api.NsError) as e:
        api.energy_efolds([1.0, 2.0], 1, 1)
    assert e.value.code == api.NS_ERR_ARG


def test_selection_matches_oracle(api):
    t = _table()
    adj = t[:, 2]
    change = [O.sensitivity_change([adj[i]], [adj[i + 1]]) for i in range(len(adj) - 1)]
    ef = [0.0] * len(adj)
    for tol in (0.05, 0.1, 0.2, 0.3, 10.0):
        assert api.lambda_select(ef, change, 1.0, tol) == O.select_lambda(ef, change, 1.0, tol)
    assert t[api.lambda_select(ef, change, 1.0, 0.1), 0] == 0.005
    rng = np.random.default_rng(9)
    for _ in range(200):
        n = int(rng.integers(2, 8))
        ef = list(rng.uniform(-1, 3, size=n))
        ch = list(rng.uniform(0, 0.4, size=n - 1))
        if rng.random() < 0.2:
            ch[int(rng.integers(0, n - 1))] = math.nan
        assert api.lambda_select(ef, ch, 1.0, 0.1) == O.select_lambda(ef, ch, 1.0, 0.1)
    assert api.lambda_select([0.0], [], 1.0, 0.1) == -1
