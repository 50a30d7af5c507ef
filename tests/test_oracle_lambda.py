"""Pins of the oracle's choice of the viscosity scaling factor (the conclusion's open
question, read through the results section's table of adjoint against finite-difference
sensitivities and section "Energy analysis"): the plateau rule against the paper's own
table, the energy-growth fit against closed forms, and the candidate sweep against the
pinned store-all adjoint.  No GPU."""
import math
import os

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "lambda_sweep_table.txt")


def _table():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    return np.array([[float(v) for v in r] for r in rows])


def test_plateau_rule_picks_the_row_where_the_paper_matches_fd():
    """On the printed sensitivities, the smallest factor whose sensitivity moves by at
    most 10 % to the next factor's is the row where the paper's adjoint equals its finite
    difference value (and no other row comes closer)."""
    t = _table()
    lam, fd, adj = t[:, 0], t[:, 1], t[:, 2]
    change = [O.sensitivity_change([adj[i]], [adj[i + 1]]) for i in range(len(lam) - 1)]
    i = O.select_lambda([0.0] * len(lam), change, 1.0, 0.1)
    assert lam[i] == 0.005
    assert adj[i] == fd[i]
    err = np.abs(adj - fd) / fd
    assert np.argmin(err) == i
    # a tighter tolerance finds no plateau in the printed range; a looser one still
    # starts at the same row, since every earlier step moves the sensitivity by > 20 %
    assert O.select_lambda([0.0] * len(lam), change, 1.0, 0.05) == -1
    assert O.select_lambda([0.0] * len(lam), change, 1.0, 0.2) == i
    # an energy criterion that rejects the row moves the choice to the next plateau row
    ef = [0.0] * len(lam)
    ef[i] = 2.0
    assert lam[O.select_lambda(ef, change, 1.0, 0.2)] == 0.007


@pytest.mark.parametrize("N", [2, 3, 10, 41])
def test_efolds_of_an_exact_exponential(N):
    """E^m = C (N - m + 1)^2 exp(a (N - m)): the normalised energy is exponential in m,
    so the fit returns a M exactly; a = 0 is a stable adjoint accumulating a constant
    source (energy growing as the square of the number of sources) and gives 0."""
    M = N // 2
    for a, C in [(0.3, 5.0), (-0.7, 1e-9), (0.0, 2.0)]:
        E = [C * (N - m + 1) ** 2 * math.exp(a * (N - m)) for m in range(N + 1)]
        assert O.energy_efolds(E) == pytest.approx(a * M, rel=1e-12, abs=1e-12)


def test_efolds_window_scale_and_degenerate_cases():
    N = 12
    rng = np.random.default_rng(4)
    E = np.exp(rng.normal(size=N + 1))
    ref = O.energy_efolds(E)
    # only m = 0..N/2 enters (the start of the backward sweep, m > N/2, is the ramp-up)
    E2 = E.copy()
    E2[N // 2 + 1:] *= 1e6
    assert O.energy_efolds(E2) == ref
    # a constant factor drops out of the slope
    assert O.energy_efolds(3.0 * E) == pytest.approx(ref, abs=1e-12)
    # brute force: the slope of np.polyfit on the normalised energy
    m = np.arange(N // 2 + 1)
    slope = np.polyfit(m, np.log(E[: N // 2 + 1]) - 2.0 * np.log(N - m + 1.0), 1)[0]
    assert ref == pytest.approx(-(N // 2) * slope, rel=1e-12)
    # a pure exponential in the raw energy reads a M less the accumulation's share
    a = 0.2
    Ee = [math.exp(a * (N - k)) for k in range(N + 1)]
    share = -(N // 2) * np.polyfit(m, 2.0 * np.log(N - m + 1.0), 1)[0]
    assert O.energy_efolds(Ee) == pytest.approx(a * (N // 2) - share, rel=1e-12)
    for bad in (0.0, -1.0, math.inf, math.nan):
        E3 = E.copy()
        E3[1] = bad
        assert O.energy_efolds(E3) == math.inf
    with pytest.raises(ValueError):
        O.energy_efolds([1.0, 2.0])


def test_sensitivity_change_and_selection_edge_cases():
    assert O.sensitivity_change([1.0, 2.0], [1.0, 2.0]) == 0.0
    assert O.sensitivity_change([3.0, 4.0], [0.0, 0.0]) == math.inf
    assert O.sensitivity_change([0.0], [0.0]) == 0.0
    assert O.sensitivity_change([0.0, 0.0], [3.0, 4.0]) == 1.0
    assert O.select_lambda([0.0], [], 1.0, 0.1) == -1
    assert O.select_lambda([math.nan, 0.0, 0.0], [0.0, 0.0], 1.0, 0.1) == 1
    assert O.select_lambda([0.0, 0.0, 0.0], [math.nan, 0.0], 1.0, 0.1) == 1


def test_candidate_sweep_follows_the_store_all_adjoint():
    """Each candidate's source sensitivity is the pinned adjoint_run's, with the sigma_1
    viscosity rule; the energy at m = 0 is that of its lam^0."""
    w0 = synth.isentropic_vortex(12, 10, 1, noise=1e-3, seed=3)
    P = params_for(w0, mu=1e-3, dt=4e-3)
    s = np.zeros_like(w0)
    s[1] = 0.05 * synth.forcing_bumps(12, 10, 1, n=4)[0]
    N = 5
    lambdas = [0.0, 0.5 * P.dx[0] ** 2, 1.0 * P.dx[0] ** 2]
    chosen, efolds, change, sbars, energies = O.estimate_lambda(w0, P, N, lambdas, s, tau=0.0)
    ws, _ = O.primal_run(w0, P, N, s)
    for k, lc in enumerate(lambdas):
        nu = (lambda w, lc=lc: lc * O.sigma1_field(w, P)) if lc > 0 else None
        lam0, sbar = O.adjoint_run(ws, P, s, nu)
        np.testing.assert_allclose(sbars[k], sbar, rtol=0, atol=1e-14 * np.abs(sbar).max())
        assert energies[k][0] == pytest.approx(O.adjoint_energy(w0, lam0, P), rel=1e-13)
        assert efolds[k] == O.energy_efolds(energies[k])
    assert change[0] == O.sensitivity_change(sbars[0], sbars[1])
    assert chosen == O.select_lambda(efolds, change, 1.0, 0.1)
    # more viscosity, less adjoint energy at the end of the sweep
    assert energies[2][0] < energies[1][0] < energies[0][0]


@pytest.mark.parametrize("efold_tol,rel_tol", [(1.0, 0.1), (1.0, 0.02), (0.25, 0.1), (3.0, 0.5), (-0.5, 0.1)])
def test_rule_on_a_constructed_family_with_a_closed_form_answer(efold_tol, rel_tol):
    """A family of candidate runs built so that the right factor follows in closed form,
    independent of the paper's table: candidate i (lambda_i = i h) has the adjoint
    energy E_i^m = (N - m + 1)^2 exp(a_i (N - m)) with a growth rate a_i = a0 - k lambda_i
    that the viscosity lowers, and the source sensitivity g_i = s + b lambda_i v (the
    bias the viscosity adds) plus, while a_i > 0, an error that grows with exp(a_i N)
    (the growing, wrong adjoint).  The energy fit returns a_i M exactly, and for damped
    neighbours the change is b h |v| / |s + b lambda_{i+1} v|; the rule must pick the
    smallest i meeting both thresholds."""
    N, M = 40, 20
    h, a0, k, b = 1e-3, 0.12, 30.0, 2.0
    lam = h * np.arange(12)
    rng = np.random.default_rng(3)
    s = rng.standard_normal(50)
    v = rng.standard_normal(50)
    err = rng.standard_normal((12, 50))
    a = a0 - k * lam
    E = [[(N - m + 1) ** 2 * math.exp(a[i] * (N - m)) for m in range(N + 1)] for i in range(12)]
    g = [s + b * lam[i] * v + (1e-3 * math.exp(a[i] * N) * err[i] if a[i] > 0 else 0.0) for i in range(12)]
    ef = [O.energy_efolds(E[i]) for i in range(12)]
    np.testing.assert_allclose(ef, a * M, rtol=1e-12, atol=1e-12)
    ch = [O.sensitivity_change(g[i], g[i + 1]) for i in range(11)]
    expect = -1
    for i in range(11):
        damped = a[i] * M <= efold_tol
        if a[i + 1] <= 0 and a[i] <= 0:
            closed = b * h * np.linalg.norm(v) / np.linalg.norm(s + b * lam[i + 1] * v)
            assert ch[i] == pytest.approx(closed, rel=1e-12)
        if damped and ch[i] <= rel_tol:
            expect = i
            break
    assert O.select_lambda(ef, ch, efold_tol, rel_tol) == expect
    if efold_tol >= 0.25 and rel_tol >= 0.1:
        # with these thresholds the first damped candidate (a_i <= efold_tol / M) is chosen
        first = int(np.argmax(a * M <= efold_tol))
        assert expect == first
