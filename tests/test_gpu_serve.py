"""Serving engine (continuous batching of posterior-sampling requests).

Each request runs `steps` denoising steps z <- z + c (GPA(z) - z) with its
state kept on the device; engine iterations batch all active requests into one
ragged attention launch and one merge-update launch (CUDA graph).  Checked:
one step against the FP64 oracle, bitwise identity of a request's result alone
and in a mix, admission under the HBM budget and the slot limit (unclaimed
results moved to host memory to make room), results taken once or released,
statistics.
"""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2604_16590_gb300 import build, gattn, serving
from paper_2604_16590_gb300.inputs import ServeRequestSpec, request_state
from tests._parity import assert_close

pytestmark = pytest.mark.gpu

Y, X, D = 32, 64, 64
CORE, HALO = (1, 16, 16), (0, 4, 4)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    gattn.load_library()


def _cfg(**kw):
    base = dict(d=D, Y=Y, X=X, core=CORE, halo=HALO, steps=1, c=0.5, max_active=16, hbm_budget=8 * 10**9)
    base.update(kw)
    return gattn.serve_cfg(**base)


def test_one_step_matches_oracle():
    spec = ServeRequestSpec(0.0, 2, 2, 77)
    z0 = request_state(spec, Y, X, D)
    with gattn.Server(_cfg(steps=1)) as srv:
        rid = srv.submit(z0)
        srv.step()
        z1, lat = srv.result(rid, z0.shape)
    assert z1 is not None and lat >= 0
    T = spec.T
    geo = oracle.Geometry(1, spec.nh, D, T, Y, X, CORE, HALO)
    z = z0.double().numpy()[None]
    att = oracle.forward(geo, z, z, z)[0]
    ref = z[0] + 0.5 * (att - z[0])
    assert_close("serve/z1", z1.double().numpy()[None], ref[None], 2e-2, 3e-3)


def test_one_step_matches_oracle_d128_mixed_requests():
    """d = 128 runs the ragged one-box kernel (sm103_fwd.cu): two requests of
    different lengths and head counts in one iteration, each checked against
    the oracle."""
    specs = [ServeRequestSpec(0.0, 3, 2, 81), ServeRequestSpec(0.0, 1, 1, 82)]
    states = [request_state(sp, Y, X, 128) for sp in specs]
    with gattn.Server(_cfg(d=128, steps=1)) as srv:
        ids = [srv.submit(z) for z in states]
        while not all(srv.done(r) for r in ids):
            srv.step()
        outs = [srv.result(r, z.shape)[0] for r, z in zip(ids, states)]
    for sp, z0, z1 in zip(specs, states, outs):
        geo = oracle.Geometry(1, sp.nh, 128, sp.T, Y, X, CORE, HALO)
        z = z0.double().numpy()[None]
        att = oracle.forward(geo, z, z, z)[0]
        ref = z[0] + 0.5 * (att - z[0])
        assert_close(f"serve128/T{sp.T}", z1.double().numpy()[None], ref[None], 2e-2, 3e-3)


@pytest.mark.parametrize("d", [64, 128])
def test_one_step_with_a_temporal_halo_matches_oracle(d):
    """Tiles of two frames with a one-frame halo: up to eight tiles cover a
    token, so the merge-and-update takes its eight-cover form."""
    core, halo = (2, 16, 16), (1, 4, 4)
    spec = ServeRequestSpec(0.0, 5, 2, 91)
    z0 = request_state(spec, Y, X, d)
    with gattn.Server(_cfg(d=d, steps=1, core=core, halo=halo)) as srv:
        rid = srv.submit(z0)
        while not srv.done(rid):
            srv.step()
        z1, _ = srv.result(rid, z0.shape)
    geo = oracle.Geometry(1, spec.nh, d, spec.T, Y, X, core, halo)
    z = z0.double().numpy()[None]
    att = oracle.forward(geo, z, z, z)[0]
    ref = z[0] + 0.5 * (att - z[0])
    assert_close(f"serve_thalo/d{d}", z1.double().numpy()[None], ref[None], 2e-2, 3e-3)


@pytest.mark.parametrize("use_graph", [True, False], ids=["graph", "direct"])
def test_result_is_identical_alone_and_in_a_mix(use_graph):
    a = ServeRequestSpec(0.0, 3, 2, 101)
    others = [ServeRequestSpec(0.0, 1 + i, 8 if i % 2 else 4, 200 + i) for i in range(4)]
    za = request_state(a, Y, X, D)
    with gattn.Server(_cfg(steps=3, use_graph=use_graph)) as srv:
        rid = srv.submit(za)
        while not srv.done(rid):
            srv.step()
        alone, _ = srv.result(rid, za.shape)
    with gattn.Server(_cfg(steps=3, use_graph=use_graph)) as srv:
        ids = [srv.submit(request_state(o, Y, X, D)) for o in others[:2]]
        srv.step()  # the mix is already one step in when the request arrives
        rid = srv.submit(za)
        ids += [srv.submit(request_state(o, Y, X, D, device="cuda")) for o in others[2:]]
        while not srv.done(rid):
            srv.step()
        mixed, _ = srv.result(rid, za.shape)
        while srv.stats().active + srv.stats().waiting > 0:
            srv.step()
        st = srv.stats()
    assert torch.equal(alone, mixed)
    assert st.completed == 5


def test_admission_respects_hbm_budget_and_slots():
    cfg = _cfg(steps=2, max_active=8)
    per = gattn.gattn_serve_request_bytes(cfg, 2, 4)
    cfg.hbm_budget = 2 * per + per // 2  # room for two such requests at a time
    specs = [ServeRequestSpec(0.0, 2, 4, 300 + i) for i in range(5)]
    with gattn.Server(cfg) as srv:
        ids = [srv.submit(request_state(s, Y, X, D)) for s in specs]
        seen = 0
        while not all(srv.done(r) for r in ids):
            active, waiting = srv.step()
            seen = max(seen, active)
            assert srv.stats().hbm_in_use <= cfg.hbm_budget
        st = srv.stats()
        # a request larger than the whole budget is refused
        big = request_state(ServeRequestSpec(0.0, 64, 16, 9), Y, X, D)
        with pytest.raises(gattn.GattnError) as e:
            srv.submit(big)
        assert e.value.status == 6
    assert seen <= 2
    assert st.completed == 5 and st.hbm_peak <= cfg.hbm_budget
    assert 0 < st.p50_latency_s <= st.p99_latency_s <= st.max_latency_s


def test_request_loop_reports_latency_percentiles():
    specs = [ServeRequestSpec(0.002 * i, 1 + (i % 3), 8, 400 + i) for i in range(6)]
    with gattn.Server(_cfg(steps=4, max_active=4)) as srv:
        lat = serving.run(srv, specs, Y, X, D, device="cuda", realtime=True)
        st = srv.stats()
    assert len(lat) == 6 and all(v > 0 for v in lat.values())
    assert st.completed == 6 and st.iterations >= 4
    assert st.p50_latency_s <= st.p99_latency_s
    assert st.token_steps == sum(8 * s.T * Y * X * 4 for s in specs)


def test_five_steps_replay_through_the_oracle():
    """The serving step loop over several denoising steps (the per-step
    Hann-weighted merge is what carries context from tile to tile, Sec. III-C):
    servers running 1..5 steps on the same request give every intermediate
    BF16 state; each step is replayed by the FP64 oracle from the previous GPU
    state (BF16 bar), and the 5-step state is compared with the oracle's own
    5-step trajectory on BF16-rounded states, within 5 times the per-step bar
    (per-step errors add at most linearly: the update is a convex blend)."""
    spec = ServeRequestSpec(0.0, 1, 2, 91)
    z0 = request_state(spec, Y, X, D)
    states = [z0]
    for k in range(1, 6):
        with gattn.Server(_cfg(steps=k)) as srv:
            rid = srv.submit(z0)
            while not srv.done(rid):
                srv.step()
            zk, _ = srv.result(rid, z0.shape)
        states.append(zk)
    geo = oracle.Geometry(1, spec.nh, D, spec.T, Y, X, CORE, HALO)

    def step(z):
        att = oracle.forward(geo, z[None], z[None], z[None])[0]
        return z + 0.5 * (att - z)

    for k in range(1, 6):
        prev = states[k - 1].double().numpy()
        assert_close(f"serve/step{k}", states[k].double().numpy()[None], step(prev)[None], 2e-2, 3e-3)
    z = z0.double().numpy()
    for _ in range(5):
        z = torch.from_numpy(step(z)).to(torch.bfloat16).double().numpy()
    assert_close("serve/trajectory5", states[5].double().numpy()[None], z[None], 5 * 2e-2, 5 * 3e-3)


def test_results_are_taken_once_and_release_frees_memory():
    specs = [ServeRequestSpec(0.0, 2, 2, 600 + i) for i in range(3)]
    states = [request_state(sp, Y, X, D) for sp in specs]
    with gattn.Server(_cfg(steps=2)) as srv:
        ids = [srv.submit(z) for z in states]
        with pytest.raises(gattn.GattnError) as e:
            srv.release(ids[0])  # not finished yet
        assert e.value.status == 1
        while not all(srv.done(r) for r in ids):
            srv.step()
        per = gattn.gattn_serve_request_bytes(srv.cfg, 2, 2)
        held = srv.stats().hbm_in_use
        assert 0 < held < 3 * per  # the final states only: scratch went back to the pool
        # taken into a device tensor, then into a host tensor: the same bytes
        dev = torch.empty(states[0].shape, dtype=torch.bfloat16, device="cuda")
        a, lat = srv.result(ids[0], out=dev)
        assert lat > 0
        b, _ = srv.result(ids[1], states[1].shape)
        with pytest.raises(gattn.GattnError) as e:
            srv.result(ids[0], states[0].shape)  # already taken
        assert e.value.status == 9
        srv.release(ids[2])
        assert srv.stats().hbm_in_use == 0
        with pytest.raises(gattn.GattnError) as e:
            srv.release(12345)
        assert e.value.status == 9
    # the same requests served one at a time give the same final states
    for z0, got in ((states[0], a.cpu()), (states[1], b)):
        with gattn.Server(_cfg(steps=2)) as srv:
            rid = srv.submit(z0)
            while not srv.done(rid):
                srv.step()
            ref, _ = srv.result(rid, z0.shape)
        assert torch.equal(ref, got)


def test_asynchronous_take_overlaps_the_next_iterations():
    """gattn_serve_take_async: the copy runs on the server's copy stream while
    the engine keeps stepping; once copied() the tensor holds the same bytes
    as a synchronous take, and the result's memory has gone back to the pool."""
    specs = [ServeRequestSpec(0.0, 2, 2, 700 + i) for i in range(2)] + [ServeRequestSpec(0.0, 4, 2, 702)]
    states = [request_state(sp, Y, X, D) for sp in specs]
    with gattn.Server(_cfg(steps=2)) as srv:
        ids = [srv.submit(z) for z in states[:2]]
        while not all(srv.done(r) for r in ids):
            srv.step()
        late = srv.submit(states[2])  # still running while the first results move
        host = torch.empty(states[0].shape, dtype=torch.bfloat16, pin_memory=True)
        dev = torch.empty(states[1].shape, dtype=torch.bfloat16, device="cuda")
        with pytest.raises(ValueError):
            srv.take_async(ids[0], torch.empty(3, dtype=torch.bfloat16, pin_memory=True))  # wrong size
        srv.take_async(ids[0], host)
        srv.take_async(ids[1], dev)
        with pytest.raises(gattn.GattnError) as e:
            srv.take_async(ids[0], host)  # already taken
        assert e.value.status == 9
        with pytest.raises(gattn.GattnError) as e:
            srv.release(ids[1])  # taken: its copy may be in flight
        assert e.value.status == 9
        with pytest.raises(gattn.GattnError) as e:
            srv.take_async(late, torch.empty(states[2].shape, dtype=torch.bfloat16, pin_memory=True))  # not finished
        assert e.value.status == 1
        while not srv.done(late):
            srv.step()
        t0 = time.monotonic()
        for r in ids:
            while not srv.copied(r):
                assert time.monotonic() - t0 < 30, "asynchronous copy did not complete"
                time.sleep(0.001)
        late_state, _ = srv.result(late, states[2].shape)
        assert srv.copied(late)
        assert srv.stats().hbm_in_use == 0
        got = [host.clone(), dev.cpu()]
    for z0, g in zip(states[:2], got):
        with gattn.Server(_cfg(steps=2)) as srv:
            rid = srv.submit(z0)
            while not srv.done(rid):
                srv.step()
            ref, _ = srv.result(rid, z0.shape)
        assert torch.equal(ref, g)
    assert late_state is not None and torch.isfinite(late_state.float()).all()
