"""Overlapped pushes (RP_FLAG_OVERLAP_PUSH): step l+1's push runs on the
library's push stream while step l's evaluation runs on the context stream.
The rings hold one slot more, so the results must be those of a context
without the flag, bit for bit, over runs longer than the rings (every slot
reused several times), for FFT, direct and two-sided far pairs, through the
host-buffer calls, under a source partition and across a save and load."""
import numpy as np
import pytest
import torch

from paper_2311_15429_gb300 import rp, synth

pytestmark = pytest.mark.gpu


def _run(doms, hists, flags, steps_from, event=False, host=False, owned=None, **kw):
    dev = torch.device("cuda", 0)
    T = hists[0].shape[0]
    out = {}
    if owned is not None:
        kw["owned_sources"] = owned
    own = set(range(len(doms)) if owned is None else owned)
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, flags=flags, **kw) as lib:
        if host:
            hin = [torch.from_numpy(np.ascontiguousarray(h)).pin_memory() for h in hists]
            hout = [torch.zeros(4 * d.N).pin_memory() for d in doms]
        else:
            slices = [[torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) if d in own else None
                       for d, h in enumerate(hists)] for i in range(T)]
            pick = lambda sl, f: [None if x is None else f(x) for x in sl]
        for i in range(T):
            if host:
                rp.rp_push_all_host(lib.ctx, [x[i, 0] for x in hin], [x[i, 1:].reshape(-1) for x in hin])
            elif event:
                rp.rp_push_all_event(lib.ctx, pick(slices[i], lambda x: x[0]),
                                     pick(slices[i], lambda x: x[1:].reshape(-1)))
            else:
                lib.push_all(pick(slices[i], lambda x: x[0]), pick(slices[i], lambda x: x[1:].reshape(-1)))
            if i >= steps_from:
                if host:
                    rp.rp_evaluate_host(lib.ctx, [x[:d.N] for x, d in zip(hout, doms)],
                                        [x[d.N:] for x, d in zip(hout, doms)])
                    rp.rp_sync(lib.ctx)
                    out[i] = [x.numpy().copy() for x in hout]
                else:
                    lib.evaluate()
                    out[i] = [torch.cat([lib.phi[d], lib.A[d]]).cpu().numpy() for d in range(len(doms))]
        lib.sync()
        q = lib.query()
    return out, q


CASES = {
    "fft": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.25), synth.cubic((8.0, 0.5, -0.3), 12, 0.25)], {}, 40, 8),
    "direct": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.3), synth.cubic((9.0, 2.0, -1.0), 10, 0.25)], {}, 40, 8),
    "far2": ([synth.cubic((0.0, 0.0, 0.0), 12, 0.25), synth.cubic((8.0, 0.5, -0.3), 12, 0.25),
              synth.cubic((600.0, 50.0, -30.0), 12, 0.25)],
             dict(mode=rp.RP_MODE_LOWRANK, far_distance=100.0, far_batch=32, far_source_points=4), 200, 100),
}


@pytest.mark.parametrize("case,event,host", [("fft", True, False), ("fft", False, False), ("direct", True, False),
                                             ("far2", True, False), ("fft", False, True)])
def test_overlapped_pushes_give_the_same_bits(case, event, host):
    doms, kw, T, start = CASES[case]
    hists = [s.history(0, T, 0.05) for s in synth.seeded_sources(doms)]
    flags = rp.RP_FLAG_GROUND_STATE_CLAMP if case != "far2" else 0
    want, q0 = _run(doms, hists, flags, start, **kw)
    got, q1 = _run(doms, hists, flags | rp.RP_FLAG_OVERLAP_PUSH, start, event=event, host=host, **kw)
    assert q1["spectral_depth"] == q0["spectral_depth"] + 1 or q1["raw_depth"] == q0["raw_depth"] + 1
    for i in want:
        for d in range(len(doms)):
            np.testing.assert_array_equal(got[i][d], want[i][d], err_msg=f"{case} step {i} domain {d}")


@pytest.mark.parametrize("owned", [[2], [0, 1]])
def test_overlapped_pushes_under_a_source_partition(owned):
    """A context that owns some sources (its partial fields of every target):
    the same bits with and without the flag, two-sided far pairs included."""
    doms, kw, T, start = CASES["far2"]
    hists = [s.history(0, T, 0.05) for s in synth.seeded_sources(doms)]
    want, _ = _run(doms, hists, 0, start, owned=owned, **kw)
    got, _ = _run(doms, hists, rp.RP_FLAG_OVERLAP_PUSH, start, event=True, owned=owned, **kw)
    for i in want:
        for d in range(len(doms)):
            np.testing.assert_array_equal(got[i][d], want[i][d], err_msg=f"owned {owned} step {i} domain {d}")


def test_overlapped_context_save_and_load(tmp_path):
    """rp_save_state in the middle of overlapped steps (the push stream still
    busy) and rp_load_state into a fresh overlapped context: the steps after
    it give the bits of the uninterrupted sequential run."""
    doms, kw, T, start = CASES["fft"]
    hists = [s.history(0, T, 0.05) for s in synth.seeded_sources(doms)]
    flags = rp.RP_FLAG_GROUND_STATE_CLAMP
    want, _ = _run(doms, hists, flags, start, **kw)
    dev = torch.device("cuda", 0)
    slices = [[torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) for h in hists] for i in range(T)]
    push = lambda lib, i: rp.rp_push_all_event(lib.ctx, [x[0] for x in slices[i]],
                                                [x[1:].reshape(-1) for x in slices[i]])
    cut = T // 2 + 3
    path = str(tmp_path / "state.bin")
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, flags=flags | rp.RP_FLAG_OVERLAP_PUSH, **kw) as lib:
        for i in range(cut):
            push(lib, i)
            lib.evaluate()
        rp.rp_save_state(lib.ctx, path)
    got = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, flags=flags | rp.RP_FLAG_OVERLAP_PUSH, **kw) as lib:
        rp.rp_load_state(lib.ctx, path)
        assert lib.query()["step"] == cut - 1
        for i in range(cut, T):
            push(lib, i)
            lib.evaluate()
            got[i] = [torch.cat([lib.phi[d], lib.A[d]]).cpu().numpy() for d in range(len(doms))]
    for i in range(cut, T):
        for d in range(len(doms)):
            np.testing.assert_array_equal(got[i][d], want[i][d], err_msg=f"step {i} domain {d}")


def test_push_event_orders_a_side_stream_producer():
    """Each step's inputs written on another stream after a delay (a spin
    on that stream), with the event recorded after the writes: a push that
    did not wait for the event would read the zero buffers.  The results are
    the bits of the sequential context."""
    doms, kw, T, start = CASES["fft"]
    hists = [s.history(0, T, 0.05) for s in synth.seeded_sources(doms)]
    flags = rp.RP_FLAG_GROUND_STATE_CLAMP
    want, _ = _run(doms, hists, flags, start, **kw)
    dev = torch.device("cuda", 0)
    slices = [[torch.from_numpy(np.ascontiguousarray(h[i])).to(dev) for h in hists] for i in range(T)]
    bufs = [[torch.zeros(4 * d.N, device=dev) for d in doms] for _ in range(T)]   # one set per step
    side = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    got = {}
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, flags=flags | rp.RP_FLAG_OVERLAP_PUSH, **kw) as lib:
        for i in range(T):
            with torch.cuda.stream(side):
                torch.cuda._sleep(200000)            # the producer is late
                for d in range(len(doms)):
                    bufs[i][d].copy_(slices[i][d].reshape(-1))
                ready = torch.cuda.Event()
                ready.record(side)
            rp.rp_push_all_event(lib.ctx, [x[:d.N] for x, d in zip(bufs[i], doms)],
                                 [x[d.N:] for x, d in zip(bufs[i], doms)], ready)
            if i >= start:
                lib.evaluate()
                got[i] = [torch.cat([lib.phi[d], lib.A[d]]).cpu().numpy() for d in range(len(doms))]
        lib.sync()
    for i in want:
        for d in range(len(doms)):
            np.testing.assert_array_equal(got[i][d], want[i][d], err_msg=f"step {i} domain {d}")


def test_overlap_refusals():
    doms = CASES["fft"][0]
    with rp.RetardedPotentials(doms, synth.C_AU, 0.05, flags=rp.RP_FLAG_GROUND_STATE_CLAMP) as lib:
        z = [torch.zeros(d.N, device="cuda") for d in doms], [torch.zeros(3 * d.N, device="cuda") for d in doms]
        with pytest.raises(rp.RPError) as e:
            rp.rp_push_all_event(lib.ctx, *z)
        assert e.value.status == rp.RP_ERR_STATE
    with pytest.raises(rp.RPError) as e:
        rp.RetardedPotentials(doms, synth.C_AU, 0.05,
                              flags=rp.RP_FLAG_OVERLAP_PUSH | rp.RP_FLAG_GROUND_STATE_SPLIT)
    assert e.value.status == rp.RP_ERR_UNSUPPORTED
