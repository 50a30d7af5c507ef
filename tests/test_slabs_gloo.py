"""The host logic of the x-slab decomposition on two CPU ranks (gloo): each rank holds one
padded slab of a box, fills its ghost columns from its neighbour with exchange_ghosts,
and evaluates the oracle's residual, transposed residual and objective on its slab.
The interior columns equal the whole box's values bit for bit (the residual and its
transpose reach one cell in x), and allreduce_sum of the per-slab partial sums gives
the whole box's dot products and objective plane sums to roundoff."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    from oracle import ns_oracle as O
    from paper_1511_06959_gb300 import synth
    from tests.test_oracle_primal import params_for
    w = synth.isentropic_vortex(16, 6, 3, noise=1e-3, seed=21)
    P = params_for(w, mu=1e-3, dt=3e-3)
    a = synth.perturbed_uniform(16, 6, 3, seed=22, amp=0.3) - 1.0
    return O, w, P, a


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    from paper_1511_06959_gb300 import slabs as SL
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        O, w, P, a = _case()
        cuts = [(0, 7), (7, 16)]            # uneven; the objective plane (12) is in slab 1
        a0, b0 = cuts[rank]
        mine = SL.split(w, cuts)[rank].copy()
        amine = SL.split(a, cuts)[rank].copy()
        # ghosts start as NaN: only the exchange can make the interior results finite
        mine[..., 0] = mine[..., -1] = np.nan
        amine[..., 0] = amine[..., -1] = np.nan
        tw, ta = torch.from_numpy(mine), torch.from_numpy(amine)
        SL.exchange_ghosts(tw, rank, world)
        SL.exchange_ghosts(ta, rank, world)
        import dataclasses
        Ps = dataclasses.replace(P, plane_i=P.plane_i - a0 + 1)
        R = O.residual(tw.numpy(), Ps)[..., 1:-1]
        T = O.residual_transpose(tw.numpy(), ta.numpy(), Ps)[..., 1:-1]
        ok_R = np.array_equal(R, O.residual(w, P)[..., a0:b0])
        ok_T = np.array_equal(T, O.residual_transpose(w, a, P)[..., a0:b0])
        # per-slab partial sums over interior columns, added over the ranks in FP64
        part = torch.tensor([float(np.sum(ta.numpy()[..., 1:-1] * R))], dtype=torch.float64)
        SL.allreduce_sum(part)
        whole = float(np.sum(a * O.residual(w, P)))
        # the objective: evaluated by the slab that holds the plane, zero elsewhere
        Jp = torch.tensor([O.objective(tw.numpy(), Ps) if a0 < P.plane_i <= b0 - 1 else 0.0],
                          dtype=torch.float64)
        SL.allreduce_sum(Jp)
        q.put((rank, ok_R, ok_T, abs(part.item() - whole) / abs(whole), abs(Jp.item() - O.objective(w, P))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_ghosts_and_reduce():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ok_R, ok_T, dot_err, J_err in res:
        assert ok_R and ok_T, rank
        assert dot_err < 1e-13
        assert J_err == 0.0


def test_split_and_join_are_inverse_and_ghosts_are_periodic():
    from paper_1511_06959_gb300 import slabs as SL
    w = np.arange(2 * 3 * 11, dtype=float).reshape(2, 3, 11)
    cuts = SL.cuts_even(11, 3)
    assert cuts == [(0, 3), (3, 7), (7, 11)]
    parts = SL.split(w, cuts)
    assert np.array_equal(SL.join(parts), w)
    assert np.array_equal(parts[0][..., 0], w[..., 10])       # slab 0's left ghost: the box's last column
    assert np.array_equal(parts[2][..., -1], w[..., 0])       # the last slab's right ghost: column 0
    assert np.array_equal(parts[1][..., 0], w[..., 2]) and np.array_equal(parts[1][..., -1], w[..., 7])


def test_one_rank_exchange_is_the_periodic_wrap():
    from paper_1511_06959_gb300 import slabs as SL
    w = torch.arange(24, dtype=torch.float64).reshape(2, 12)
    t = SL.split(w, [(0, 12)])[0].clone()
    t[..., 0] = t[..., -1] = -1.0
    SL.exchange_ghosts(t, 0, 1)
    assert torch.equal(t, SL.split(w, [(0, 12)])[0])
