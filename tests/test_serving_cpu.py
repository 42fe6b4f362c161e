"""Scheduling logic of the continuous-batching server, on a fake engine with a virtual clock
(no GPU): every request gets exactly its steps, slots are never over-committed, admission is
first come first served per mesh, and the statistics add up."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2605_00619_gb300.serving import Request, Server, Slot, _quantile, poisson_requests


class FakeEngine:
    """Advances a virtual clock by a fixed launch overhead plus a cost per cell-step, and
    records every step each slot takes for the request it holds."""

    def __init__(self, slots, overhead=1e-3, per_node_step=1e-6, fail_rid=None):
        self.slots = [Slot(i, k, None, n, 0) for i, (k, n) in enumerate(slots)]
        self.t = 0.0
        self.overhead = overhead
        self.per = per_node_step
        self.steps_of = {}
        self.batches = []
        self.fail_rid = fail_rid

    def clock(self):
        return self.t

    def sleep(self, dt):
        self.t += dt

    def load(self, slot, q0):
        assert slot.busy is None, "slot loaded while busy"
        slot.loaded = q0

    def _advance(self, slots, nsteps):
        for s in slots:
            assert s.busy is not None
            assert nsteps <= s.remaining, "request stepped past its nsteps"
            self.steps_of[s.busy.rid] = self.steps_of.get(s.busy.rid, 0) + nsteps
        self.t += nsteps * (self.overhead + self.per * sum(s.n_nodes for s in slots))

    def step(self, slots, nsteps):
        self.batches.append((tuple(s.sid for s in slots), nsteps))
        self._advance(slots, nsteps)
        return [5 if s.busy.rid == self.fail_rid else 0 for s in slots]

    def step_alone(self, slot, nsteps):
        self.batches.append(((slot.sid,), nsteps))
        self._advance([slot], nsteps)
        return 0

    def read(self, slot):
        return np.zeros((slot.n_nodes, 5)), 0.0


def _server(eng, mode="batch", max_chunk=4):
    return Server(eng, mode=mode, max_chunk=max_chunk, clock=eng.clock, sleep=eng.sleep)


def test_every_request_gets_exactly_its_steps():
    eng = FakeEngine([("a", 100)] * 3 + [("b", 300)] * 2)
    reqs = poisson_requests(200.0, 40, ["a", "b"], [3, 5, 8, 13], seed=1)
    st = _server(eng).run(reqs)
    assert st.requests == 40 and st.failed == 0
    for r in reqs:
        assert eng.steps_of[r.rid] == r.nsteps
        assert r.done >= r.admitted >= r.arrival
    assert st.dof_updates == pytest.approx(sum(5 * (100 if r.mesh == "a" else 300) * r.nsteps for r in reqs))
    assert st.p50_s <= st.p99_s
    assert st.makespan_s >= max(r.done for r in reqs) - 1e-12


def test_batches_never_exceed_slots_and_hold_one_request_per_slot():
    eng = FakeEngine([("a", 10)] * 2 + [("b", 10)])
    reqs = [Request(i, "a" if i % 3 else "b", 4, 0.0) for i in range(9)]
    _server(eng, max_chunk=2).run(reqs)
    for sids, n in eng.batches:
        assert len(set(sids)) == len(sids) <= 3
        assert 1 <= n <= 2


def test_fifo_per_mesh():
    eng = FakeEngine([("a", 10)])
    reqs = [Request(i, "a", 2, 0.01 * i) for i in range(6)]
    _server(eng).run(reqs)
    order = sorted(reqs, key=lambda r: r.admitted)
    assert [r.rid for r in order] == list(range(6))


def test_other_meshes_pass_a_blocked_request():
    eng = FakeEngine([("a", 10), ("b", 10)])
    # two requests for "a" arrive first; the "b" request must not wait for the second "a"
    reqs = [Request(0, "a", 10, 0.0), Request(1, "a", 10, 0.0), Request(2, "b", 1, 0.0)]
    _server(eng).run(reqs)
    assert reqs[2].admitted < reqs[1].admitted
    assert reqs[2].done < reqs[0].done


def test_new_requests_join_a_running_batch():
    eng = FakeEngine([("a", 10)] * 2, overhead=1.0, per_node_step=0.0)
    reqs = [Request(0, "a", 20, 0.0), Request(1, "a", 2, 2.5)]
    _server(eng, max_chunk=1).run(reqs)
    # the late request is admitted at the first step boundary after its arrival, long before
    # the first request finishes
    assert reqs[1].admitted < 4.0
    assert reqs[1].done < reqs[0].done
    assert any(len(sids) == 2 for sids, _ in eng.batches)


def test_serial_mode_runs_one_request_at_a_time():
    eng = FakeEngine([("a", 10)] * 4)
    reqs = [Request(i, "a", 3, 0.0) for i in range(5)]
    st = _server(eng, mode="serial").run(reqs)
    assert all(len(sids) == 1 for sids, _ in eng.batches)
    assert st.mean_batch == 1.0
    spans = sorted((r.admitted, r.done) for r in reqs)
    for (a0, d0), (a1, _) in zip(spans, spans[1:]):
        assert a1 >= d0


def test_batching_beats_serial_when_launches_dominate():
    mk = lambda: FakeEngine([("a", 10)] * 8, overhead=1e-3, per_node_step=1e-7)  # noqa: E731
    reqs = lambda: [Request(i, "a", 6, 0.0) for i in range(16)]  # noqa: E731
    eb, es = mk(), mk()
    sb = _server(eb).run(reqs())
    ss = _server(es, mode="serial").run(reqs())
    assert sb.throughput > 4 * ss.throughput
    assert sb.p99_s < ss.p99_s


def test_failed_status_is_reported():
    eng = FakeEngine([("a", 10)] * 2, fail_rid=3)
    reqs = [Request(i, "a", 2, 0.0) for i in range(5)]
    st = _server(eng).run(reqs)
    assert st.failed == 1 and reqs[3].status == 5


def test_unknown_mesh_is_rejected():
    eng = FakeEngine([("a", 10)])
    with pytest.raises(ValueError):
        _server(eng).run([Request(0, "zzz", 1, 0.0)])


def test_idle_server_sleeps_until_the_next_arrival():
    eng = FakeEngine([("a", 10)], overhead=0.0, per_node_step=0.0)
    reqs = [Request(0, "a", 1, 5.0)]
    st = _server(eng).run(reqs)
    assert reqs[0].admitted == pytest.approx(5.0)
    assert st.makespan_s == pytest.approx(5.0)


def test_quantile_is_nearest_rank():
    v = sorted(np.random.default_rng(0).random(101).tolist())
    for q in (0.5, 0.9, 0.99):
        assert _quantile(v, q) == pytest.approx(np.quantile(v, q, method="inverted_cdf"))
    assert math.isnan(_quantile([], 0.5))


def test_poisson_arrivals_have_the_requested_rate():
    reqs = poisson_requests(50.0, 4000, ["a"], [1], seed=3)
    gaps = np.diff([0.0] + [r.arrival for r in reqs])
    assert np.mean(gaps) == pytest.approx(1 / 50.0, rel=0.05)
    assert all(r.nsteps == 1 and r.mesh == "a" for r in reqs)


class ElasticFakeEngine(FakeEngine):
    """FakeEngine whose slot pool grows and shrinks within a byte budget; footprints per mesh."""

    def __init__(self, sizes, footprint, budget, **kw):
        super().__init__([], **kw)
        self.sizes = dict(sizes)
        self._fp = dict(footprint)
        self.budget_bytes = budget
        self.device_bytes = 0
        self.peak_bytes = 0
        self._sid = 0
        self.added, self.removed = [], []

    def keys(self):
        return set(self.sizes)

    def footprint(self, key):
        return self._fp[key]

    def add_slot(self, key):
        if self.device_bytes + self._fp[key] > self.budget_bytes:
            return None
        s = Slot(self._sid, key, None, self.sizes[key], self._fp[key])
        self._sid += 1
        self.slots.append(s)
        self.device_bytes += s.nbytes
        self.peak_bytes = max(self.peak_bytes, self.device_bytes)
        self.added.append(key)
        return s

    def remove_slot(self, slot):
        assert slot.busy is None, "evicted a busy slot"
        self.slots.remove(slot)
        self.device_bytes -= slot.nbytes
        self.removed.append(slot.mesh)


def test_elastic_admission_by_footprint():
    """No slot exists up front; slots are made per request within the budget (a: 1 unit,
    b: 3 units, budget 4) and idle slots of other meshes are evicted to make room.  Every
    request gets exactly its steps, the budget is never exceeded and no busy slot is evicted."""
    eng = ElasticFakeEngine({"a": 100, "b": 400}, {"a": 1, "b": 3}, 4)
    reqs = poisson_requests(300.0, 30, ["a", "b"], [2, 3, 5], seed=3)
    srv = Server(eng, max_chunk=2, clock=eng.clock, sleep=eng.sleep, elastic=True)
    st = srv.run(reqs)
    assert st.requests == 30 and st.failed == 0
    for r in reqs:
        assert eng.steps_of[r.rid] == r.nsteps
    assert eng.peak_bytes <= 4
    assert srv.slots_added == len(eng.added) and srv.slots_evicted == len(eng.removed) > 0
    assert {"a", "b"} <= set(eng.added)
    for sids, _ in eng.batches:  # a batch never holds more than the budget allows
        assert len(sids) <= 4


def test_elastic_admission_rejects_what_can_never_fit():
    eng = ElasticFakeEngine({"a": 100, "c": 900}, {"a": 1, "c": 9}, 4)
    with pytest.raises(ValueError, match="exceeds the budget"):
        Server(eng, clock=eng.clock, sleep=eng.sleep, elastic=True).run([Request(0, "c", 1, 0.0)])
    with pytest.raises(ValueError, match="not in the catalogue"):
        Server(eng, clock=eng.clock, sleep=eng.sleep, elastic=True).run([Request(0, "z", 1, 0.0)])
    with pytest.raises(ValueError, match="elastic"):
        Server(eng, mode="serial", elastic=True)


class _FakeLib:
    """Stands in for the C-ABI binding under GpuEngine (host logic only): handles are
    integers, a mesh's device bytes are given per catalogue object, batches are recorded."""

    def __init__(self, nbytes):
        self.nbytes = nbytes
        self.live = {}
        self.batches = {}
        self._id = 0
        self.AFE_OK = 0

    def create_from_polymesh(self, pm, prm, stream=0):
        self._id += 1
        self.live[self._id] = pm
        return self._id

    def afe_device_bytes(self, h):
        return self.nbytes[self.live[h]]

    def afe_num_nodes(self, h):
        return 10

    def afe_get_node_coords(self, h):
        return np.zeros((10, 3))

    def afe_mesh_destroy(self, h):
        del self.live[h]

    def afe_set_state(self, h, q):
        assert h in self.live

    def afe_batch_create(self, handles, stream=0):
        for h in handles:
            assert h in self.live
        self._id += 1
        self.batches[self._id] = list(handles)
        return self._id

    def afe_batch_destroy(self, b):
        del self.batches[b]

    def afe_batch_step_async(self, b, dt, n, use_graph):
        for h in self.batches[b]:
            assert h in self.live, "batch holds a destroyed handle"

    def afe_batch_sync(self, b, n, check=True):
        return 0, [0] * n


def test_gpu_engine_host_logic_with_elastic_admission(monkeypatch):
    """GpuEngine's slot bookkeeping over a fake binding: slots made and released within the
    budget, cached batches that hold an evicted slot destroyed with it, and no handle leaked."""
    from types import SimpleNamespace

    from paper_2605_00619_gb300 import serving
    fake = _FakeLib({"mesh-a": 100, "mesh-b": 300})
    monkeypatch.setattr(serving, "_afe", fake)
    prm = SimpleNamespace(order=2)
    eng = serving.GpuEngine({"a": "mesh-a", "b": "mesh-b"}, {"a": 1}, params=prm, budget_bytes=400,
                            default_state={"a": np.zeros((10, 5)), "b": np.zeros((10, 5))})
    assert len(eng.slots) == 1 and eng.device_bytes == 100
    assert eng.footprint("b") == 300 and len(fake.live) == 1      # measured on a handle made and freed
    reqs = poisson_requests(1000.0, 24, ["a", "b"], [1, 2, 3], seed=5)
    clock = {"t": 0.0}

    def tick():
        clock["t"] += 1e-3
        return clock["t"]

    srv = serving.Server(eng, max_chunk=2, clock=tick, sleep=lambda dt: clock.__setitem__("t", clock["t"] + dt),
                         elastic=True)
    st = srv.run(reqs)
    assert st.requests == 24 and st.failed == 0
    assert eng.device_bytes <= 400 and srv.slots_evicted > 0
    assert len(fake.live) == len(eng.slots)
    for b, handles in fake.batches.items():
        assert all(h in fake.live for h in handles)
    eng.close()
    assert not fake.live and not fake.batches
