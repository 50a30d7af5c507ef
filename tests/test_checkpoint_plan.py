"""Checkpoint planner of the host runtime (no GPU): every plan reverses each step once,
in order, with the right primal state at hand, within its slot count, and replays
each step no more often than its schedule allows.  Executing a plan with the oracle's
step functions gives exactly the store-all adjoint."""
import math

import numpy as np
import pytest

from oracle import ns_oracle as O
from paper_1511_06959_gb300 import synth
from tests.test_oracle_primal import params_for

ADV, STORE, LOAD, ADJ, FREE, SRC = 1, 2, 3, 4, 5, 6
HSTORE, HLOAD, HFREE = 7, 8, 9


def _api():
    from tests.test_abi import _lib_path
    _lib_path()
    from paper_1511_06959_gb300 import api
    return api


def simulate(actions, N, slots_used, host_peak=None):
    """Symbolic run: the state is its step index.  Returns (first-touch order, number of
    adjoint steps, peak live slots, advances); host_peak, a list, receives the peak of
    live host slots."""
    cur = 0
    slots = {}
    hslots = {}
    hpeak = 0
    touched = 0
    first = []
    adj = []
    peak = 0
    adv = 0
    src_done = False
    for op, a, b in actions:
        if op == ADV:
            assert cur == a and b > a
            for n in range(a, b):
                if n + 1 > touched:
                    first.append(n + 1)
                    touched = n + 1
            adv += b - a
            cur = b
        elif op == STORE:
            assert cur == a and b not in slots
            slots[b] = a
            peak = max(peak, len(slots))
            assert b < max(slots_used, 1)
        elif op == LOAD:
            cur = 0 if b == -1 else slots[b]
            assert cur == a
        elif op == FREE:
            assert slots.pop(b) == a
        elif op == HSTORE:
            assert cur == a and a > 0 and b not in hslots
            hslots[b] = a
            hpeak = max(hpeak, len(hslots))
        elif op == HLOAD:
            cur = hslots[b]
            assert cur == a
        elif op == HFREE:
            assert hslots.pop(b) == a
        elif op == SRC:
            assert a == N and cur == N and not adj
            src_done = True
        elif op == ADJ:
            assert src_done and cur == a
            assert a == (adj[-1] - 1 if adj else N - 1)
            adj.append(a)
    assert not slots and not hslots
    if host_peak is not None:
        host_peak.append(hpeak)
    return first, adj, peak, adv


CASES = [(0, 0), (1, 1), (1, 4), (1, 50), (2, 1), (2, 2), (2, 3), (2, 5), (2, 20), (3, 1), (3, 4), (3, 50)]


@pytest.mark.parametrize("N", [1, 2, 3, 7, 13, 50, 201])
@pytest.mark.parametrize("schedule,param", CASES)
def test_plan_invariants(N, schedule, param):
    api = _api()
    actions, slots_used, advances = api.plan(N, schedule, param)
    hp = []
    first, adj, peak, adv = simulate(actions, N, slots_used, hp)
    assert first == list(range(1, N + 1))
    assert adj == list(range(N - 1, -1, -1))
    assert peak == slots_used and adv == advances
    if schedule != 3:
        assert hp == [0]
    else:
        # the stride plan's steps, with the snapshots in host slots and only the replayed
        # segment's states in device slots; the last segment's states, its first included,
        # stay in device slots from the forward pass
        k = param
        assert hp == [max((N - 1) // k - 1, 0)]
        assert slots_used <= k
        ref_actions, _, ref_adv = api.plan(N, 1, k)
        assert advances == ref_adv
        assert [x for x in actions if x[0] in (ADV, ADJ, SRC)] == [x for x in ref_actions if x[0] in (ADV, ADJ, SRC)]
    if schedule == 0:
        assert advances == N and slots_used == max(N - 1, 0)
    if schedule in (1, 3):
        # every segment but the last is replayed once, from its snapshot; the last one is
        # reversed from the states the forward pass stored
        k = param
        assert advances == N + ((N - 1) // k) * (k - 1)
    if schedule == 1:
        k = param
        assert advances <= 2 * N
        assert slots_used <= (N - 1) // k + k


def _beta(s, r):
    return math.comb(s + r, s)


@pytest.mark.parametrize("N,S", [(20, 3), (100, 5), (1000, 10), (20000, 80), (50, 1), (7, 6)])
def test_revolve_repetition_bound(N, S):
    """Binomial checkpointing: with S slots every step is advanced at most r + 1 times
    (the first pass plus r replays), r the least integer with C(S + r, S) >= N; the
    total stays within (r + 1) N."""
    api = _api()
    actions, slots_used, advances = api.plan(N, 2, S)
    assert slots_used <= S
    r = 0
    while _beta(S, r) < N:
        r += 1
    counts = np.zeros(N + 1, dtype=int)
    cur = 0
    slots = {}
    for op, a, b in actions:
        if op == ADV:
            counts[a:b] += 1
            cur = b
        elif op == STORE:
            slots[b] = a
        elif op == LOAD:
            cur = a
        elif op == FREE:
            slots.pop(b)
    assert counts[:N].max() <= r + 1, (counts.max(), r)
    assert advances <= (r + 1) * N


@pytest.mark.parametrize("N,k", [(1, 1), (13, 4), (201, 50)])
def test_disk_tier_plan_is_the_host_tier_plan(N, k):
    """NS_CKPT_STRIDE_DISK runs the host tier's plan, its host slots being file slots."""
    api = _api()
    assert api.plan(N, api.NS_CKPT_STRIDE_DISK, k) == api.plan(N, api.NS_CKPT_STRIDE_HOST, k)
    with pytest.raises(api.NsError):
        api.plan(N, api.NS_CKPT_STRIDE_DISK, 0)


@pytest.mark.parametrize("N,S", [(1, 1), (13, 3), (201, 5), (1000, 10)])
def test_revolve_host_and_disk_tiers_plan_the_revolve_steps_in_host_slots(N, S):
    """NS_CKPT_REVOLVE_HOST / _DISK run the binomial plan with every checkpoint slot a host
    (file) slot: the same actions with STORE, LOAD (but the caller's w0) and FREE turned
    into their host forms, no device slot, the revolve plan's slot count as the host
    peak, and the plan's invariants under the symbolic run."""
    api = _api()
    ref, ref_slots, ref_adv = api.plan(N, api.NS_CKPT_REVOLVE, S)
    to_host = {STORE: HSTORE, FREE: HFREE}
    want = [(to_host.get(op, HLOAD if op == LOAD and b >= 0 else op), a, b) for op, a, b in ref]
    for sched in (api.NS_CKPT_REVOLVE_HOST, api.NS_CKPT_REVOLVE_DISK):
        actions, slots_used, advances = api.plan(N, sched, S)
        assert actions == want and slots_used == 0 and advances == ref_adv
        hp = []
        first, adj, peak, adv = simulate(actions, N, slots_used, hp)
        assert first == list(range(1, N + 1))
        assert adj == list(range(N - 1, -1, -1))
        assert adv == advances and hp == [ref_slots]
    with pytest.raises(api.NsError):
        api.plan(N, api.NS_CKPT_REVOLVE_HOST, 0)


def test_plan_rejects_bad_arguments():
    api = _api()
    with pytest.raises(api.NsError):
        api.plan(0, 0, 0)
    with pytest.raises(api.NsError):
        api.plan(10, 1, 0)
    with pytest.raises(api.NsError):
        api.plan(10, 9, 3)
    with pytest.raises(api.NsError):
        api.plan(10, 3, 0)


def execute_with_oracle(actions, w0, P, N, s=None):
    """Run a plan with the oracle's step functions (what the GPU executor does)."""
    slots = {}
    hslots = {}
    cur = w0
    lam = np.zeros_like(w0)
    J = 0.0
    touched = 0
    sbar = np.zeros_like(w0)
    for op, a, b in actions:
        if op == ADV:
            for n in range(a, b):
                cur, _ = O.rk4_step(cur, P, s)
                if n + 1 > touched:
                    J += O.objective(cur, P) / N
                    touched = n + 1
        elif op == STORE:
            slots[b] = cur
        elif op == LOAD:
            cur = w0 if b == -1 else slots[b]
        elif op == FREE:
            slots.pop(b)
        elif op == HSTORE:
            hslots[b] = cur.copy()
        elif op == HLOAD:
            cur = hslots[b].copy()
        elif op == HFREE:
            hslots.pop(b)
        elif op == SRC:
            lam = lam + O.objective_grad(cur, P) / N
        elif op == ADJ:
            lam, sb = O.rk4_adjoint_step(cur, lam, P, s)
            sbar += sb
            if a >= 1:
                lam = lam + O.objective_grad(cur, P) / N
    return J, lam, sbar


@pytest.mark.parametrize("schedule,param", [(0, 0), (1, 4), (2, 2), (2, 3), (3, 4), (3, 3), (3, 1), (5, 2), (6, 3)])
def test_plan_executed_with_oracle_equals_store_all(schedule, param):
    api = _api()
    w0 = synth.isentropic_vortex(8, 6, 1, noise=1e-3, seed=4)
    P = params_for(w0, mu=0.01, dt=5e-3)
    N = 11
    s = np.zeros_like(w0)
    s[1] = 0.1
    actions, _, _ = api.plan(N, schedule, param)
    J, lam, sbar = execute_with_oracle(actions, w0, P, N, s)
    ws, Jref = O.primal_run(w0, P, N, s)
    lam_ref, sbar_ref = O.adjoint_run(ws, P, s)
    assert J == pytest.approx(Jref, rel=1e-14)
    assert np.array_equal(lam, lam_ref)
    np.testing.assert_allclose(sbar, sbar_ref, rtol=1e-13, atol=1e-16)
