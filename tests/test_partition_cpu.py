"""The source partition on CPU ranks (gloo, world size 2): ownership, the
plan each rank's context makes, and the one exchange of a step.

Each rank's context owns the source domains `partition.owners` gives it
(`rp_own_sources`, plan-only: no GPU); its pairs of other sources are
RP_PAIR_OTHER, and every ordered pair is evaluated by exactly one rank.  The
contributions a rank's `rp_evaluate` would write are stood in for by the
FP64 oracle over its owned sources alone (the other histories zero).  The
packed partial fields are reduce-scattered over gloo, and each rank's
targets must then equal the oracle's full sum (every source).
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2311_15429_gb300 import partition, rp, synth  # noqa: E402


def _geometry():
    doms = [synth.cubic((0.0, 0.0, 0.0), 6, 0.3), synth.Domain((3.0, -0.5, 0.2), (5, 7, 4), 0.3),
            synth.cubic((-2.4, 2.0, 1.1), 6, 0.25)]
    return doms, synth.seeded_sources(doms), 20.0, 0.05


def test_owners_balance_the_points():
    """Largest first, each to the least-loaded rank: 4096 -> 0, then 1728,
    512, 512 and 64 all to rank 1 (never above rank 0's load)."""
    sizes = [512, 4096, 512, 1728, 64]
    own = partition.owners(sizes, 2)
    assert own == [1, 0, 1, 1, 1]
    assert [sum(n for n, r in zip(sizes, own) if r == k) for k in range(2)] == [4096, 2816]
    assert partition.owners([10], 3) == [0]


def _plan(doms, c, dt, owned):
    ctx = rp.rp_create(c, dt, flags=rp.RP_FLAG_PLAN_ONLY)
    try:
        for d in doms:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        rp.rp_own_sources(ctx, owned)
        rp.rp_finalize(ctx)
        n = len(doms)
        kinds = {(t, s): rp.rp_pair_info(ctx, t, s)["kind"] for t in range(n) for s in range(n)}
        return kinds, rp.rp_query(ctx)
    finally:
        rp.rp_destroy(ctx)


def test_each_pair_evaluated_by_exactly_one_rank():
    doms, _, c, dt = _geometry()
    own = partition.owners([d.N for d in doms], 2)
    seen = {}
    for rank in range(2):
        owned = partition.owned_by(rank, own)
        kinds, q = _plan(doms, c, dt, owned)
        assert q["owned_sources"] == len(owned)
        assert q["npairs_other"] == len(doms) * (len(doms) - len(owned))
        for (t, s), k in kinds.items():
            assert (k == rp.RP_PAIR_OTHER) == (s not in owned), (rank, t, s, k)
            if k != rp.RP_PAIR_OTHER:
                assert (t, s) not in seen
                seen[(t, s)] = rank
    assert len(seen) == len(doms) ** 2


def test_own_sources_refuses_bad_ids():
    doms, _, c, dt = _geometry()
    ctx = rp.rp_create(c, dt, flags=rp.RP_FLAG_PLAN_ONLY)
    try:
        for d in doms:
            rp.rp_add_domain(ctx, d.origin, d.n, d.h)
        for bad in ([3], [0, 0], []):
            with pytest.raises(rp.RPError) as e:
                rp.rp_own_sources(ctx, bad)
            assert e.value.status == rp.RP_ERR_ARG
    finally:
        rp.rp_destroy(ctx)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2311_15429_gb300 import partition as P
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        doms, srcs, c, dt = _geometry()
        sizes = [d.N for d in doms]
        own = P.owners(sizes, world)
        owned = P.owned_by(rank, own)
        kinds, _ = _plan(doms, c, dt, owned)
        T = 20
        hists = [s.history(0, T, dt) for s in srcs]
        mine = [h if d in owned else np.zeros_like(h) for d, h in enumerate(hists)]
        args = ([d.origin for d in doms], [d.n for d in doms], [d.h for d in doms])
        # the partial field of every target from this rank's sources
        fields = []
        for t, d in enumerate(doms):
            v = oracle.eval_points(*args, mine, 0, c, dt, t, T - 1, np.arange(d.N))
            fields.append(torch.from_numpy(np.ascontiguousarray(v.T.reshape(-1))))
        chunk = P.exchange(P.pack(fields, sizes, own, world), world)
        got = P.unpack(chunk, rank, sizes, own)
        worst = 0.0
        for t, tot in got.items():
            want = oracle.eval_points(*args, hists, 0, c, dt, t, T - 1, np.arange(doms[t].N)).T.reshape(-1)
            worst = max(worst, float(np.max(np.abs(tot.numpy() - want)) / np.max(np.abs(want))))
        q.put((rank, sorted(got), worst, all(k != rp.RP_PAIR_OTHER for (t, s), k in kinds.items() if s in owned)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_scatter_equals_the_full_sum():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=300) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    doms, _, _, _ = _geometry()
    own = partition.owners([d.N for d in doms], 2)
    for rank, targets, worst, plan_ok in res:
        assert targets == partition.owned_by(rank, own)
        assert worst <= 1e-12, (rank, worst)
        assert plan_ok
