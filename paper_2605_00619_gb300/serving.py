"""Continuous batching of many independent ADER-AFE simulations on one GPU.

A request asks for ``nsteps`` CFL steps of one simulation: a mesh from a catalogue of
resident meshes and an initial state.  Meshes are set up once (topology, mass matrices and
their inverses: the costly part), as a pool of *slots* -- mesh handles whose state buffers
are reused by successive requests, sized up front to a device-memory budget.  With
``elastic`` admission the pool changes with the load instead: a request whose mesh has no
free slot gets a new one when its device footprint (dominated by the cells' M_i^-1) fits
the budget, after evicting idle slots of other meshes, least recently used first.  The server
loop admits arrived requests into free slots of their mesh, advances every occupied slot
together with one launch per stage (``afe_batch_step_async``: the kernels take a table of
meshes, so a batch of small meshes fills the GPU as one large mesh does), and retires
requests as they finish, so that new requests join a running batch at the next step
boundary instead of waiting for the whole batch to drain.

The GPU engine is a thin layer over the C ABI; every step of the computation runs in the
library's kernels.  The scheduling logic is independent of it (any object with the
engine's methods will do), which keeps it testable without a GPU.
"""
from __future__ import annotations

import math
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np

from . import afe as _afe


@dataclass
class Request:
    rid: int
    mesh: str                       # catalogue key
    nsteps: int                     # CFL steps to take
    arrival: float                  # seconds after the start of the run
    q0: object = None               # initial state [n_nodes, 5], a callable of the node
                                    # coordinates [n_nodes, 3], or None (the engine's default)
    # filled in by the server
    admitted: float = math.nan
    done: float = math.nan
    status: int = 0
    q: Optional[np.ndarray] = None  # final state (when the server keeps results)
    t: float = math.nan             # simulated time reached

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class Slot:
    sid: int
    mesh: str
    handle: object
    n_nodes: int
    nbytes: int
    busy: Optional[Request] = None
    remaining: int = 0
    order: int = 0
    xyz: Optional[np.ndarray] = None  # node coordinates (initial states given as functions)
    last_used: float = 0.0            # when the slot last stepped (eviction order)


class GpuEngine:
    """Slot pool on the current CUDA device.

    catalogue: key -> mesh (an object with the arrays of ``afe_mesh_create``: ``xyz``,
    ``cell_subtet_ptr``, ``subtet_vtx``, ``subtet_shift``, ``periodic``, ``period``), or
    key -> (mesh, afe_params) to give that mesh its own parameters (order, equations,
    limiter).  slots: key -> number of slots of that mesh.  params: ``afe_params`` of the keys
    without their own.  default_state: key -> [n_nodes, 5] state used when a request brings
    none.  budget_bytes: the pool may not exceed this much device memory (None: no limit).
    Batched steps need AFE_FP32 slots; slots of different orders run as one batch per order,
    each batch on its own stream, so the groups overlap on the GPU.
    """

    def __init__(self, catalogue, slots: Dict[str, int], params=None, default_state=None, budget_bytes=None,
                 stream: int = 0, use_graph: bool = True, max_cached_batches: int = 16):
        self.params = params
        self.stream = stream
        self.use_graph = use_graph
        self.catalogue = dict(catalogue)
        self.budget_bytes = budget_bytes
        self.slots: List[Slot] = []
        self.default_state = dict(default_state or {})
        self._batches: "OrderedDict[tuple, object]" = OrderedDict()
        self._max_cached = max_cached_batches
        self._footprint: Dict[str, int] = {}
        self._next_sid = 0
        self.device_bytes = 0
        for key, count in slots.items():
            for _ in range(count):
                if self.add_slot(key) is None:
                    break

    def _entry(self, key):
        entry = self.catalogue[key]
        return entry if isinstance(entry, tuple) else (entry, self.params)

    def keys(self):
        return set(self.catalogue)

    def footprint(self, key) -> int:
        """Device bytes of one slot of ``key`` (measured once, on a handle made for it)."""
        if key not in self._footprint:
            pm, prm = self._entry(key)
            h = _afe.create_from_polymesh(pm, prm, self.stream)
            self._footprint[key] = _afe.afe_device_bytes(h)
            _afe.afe_mesh_destroy(h)
        return self._footprint[key]

    def add_slot(self, key) -> Optional[Slot]:
        """A new slot of ``key``, or None when it would exceed the budget."""
        pm, prm = self._entry(key)
        h = _afe.create_from_polymesh(pm, prm, self.stream)
        nb = _afe.afe_device_bytes(h)
        self._footprint[key] = nb
        if self.budget_bytes is not None and self.device_bytes + nb > self.budget_bytes:
            _afe.afe_mesh_destroy(h)
            return None
        self.device_bytes += nb
        s = Slot(self._next_sid, key, h, _afe.afe_num_nodes(h), nb, order=int(prm.order),
                 xyz=_afe.afe_get_node_coords(h))
        self._next_sid += 1
        self.slots.append(s)
        return s

    def remove_slot(self, slot: Slot):
        """Release an idle slot and every cached batch that holds it."""
        for key in [k for k in self._batches if slot.sid in k]:
            _afe.afe_batch_destroy(self._batches.pop(key))
        _afe.afe_mesh_destroy(slot.handle)
        self.slots.remove(slot)
        self.device_bytes -= slot.nbytes

    # -- engine interface used by the server
    def load(self, slot: Slot, q0):
        q = self.default_state[slot.mesh] if q0 is None else q0
        if callable(q):
            q = q(slot.xyz)
        _afe.afe_set_state(slot.handle, q)

    def _batch(self, slots: Sequence[Slot]):
        key = tuple(s.sid for s in slots)
        b = self._batches.pop(key, None)
        if b is None:
            # a private stream per batch (stream NULL): groups of different orders overlap
            b = _afe.afe_batch_create([s.handle for s in slots], 0)
            while len(self._batches) >= self._max_cached:
                _, old = self._batches.popitem(last=False)
                _afe.afe_batch_destroy(old)
        self._batches[key] = b
        return b

    def step(self, slots: Sequence[Slot], nsteps: int) -> List[int]:
        groups: Dict[int, List[int]] = {}
        for i, s in enumerate(slots):
            groups.setdefault(s.order, []).append(i)
        launched = []
        for idx in groups.values():
            b = self._batch([slots[i] for i in idx])
            _afe.afe_batch_step_async(b, 0.0, nsteps, self.use_graph)
            launched.append((b, idx))
        out = [0] * len(slots)
        for b, idx in launched:
            _, ms = _afe.afe_batch_sync(b, len(idx), check=False)
            for i, st in zip(idx, ms):
                out[i] = int(st)
        return out

    def step_alone(self, slot: Slot, nsteps: int) -> int:
        _afe.afe_step_async(slot.handle, 0.0, nsteps)
        return _afe.afe_sync(slot.handle, check=False)

    def read(self, slot: Slot):
        return _afe.afe_get_state(slot.handle), _afe.afe_get_stats(slot.handle).t

    def close(self):
        for b in self._batches.values():
            _afe.afe_batch_destroy(b)
        self._batches.clear()
        for s in self.slots:
            _afe.afe_mesh_destroy(s.handle)
        self.slots = []


@dataclass
class RunStats:
    requests: int
    makespan_s: float
    dof_updates: float
    throughput: float               # DOF-updates per second over the run
    p50_s: float
    p99_s: float
    mean_s: float
    steps_launched: int             # batch steps (or single steps) issued
    mean_batch: float               # mean members per batch step
    failed: int
    latencies: List[float] = field(default_factory=list)

    def as_dict(self):
        d = dict(self.__dict__)
        d.pop("latencies")
        return d


class Server:
    """Continuous-batching loop over an engine's slots.

    mode "batch": all occupied slots advance together, ``chunk`` steps per iteration with
    chunk = min(max_chunk, fewest steps any running request still needs), so no request is
    stepped past its nsteps and a finished slot is refilled at the next iteration.
    mode "serial": one request at a time, alone (the unbatched baseline).
    Admission is first come, first served per mesh: a request waits until a slot of its mesh
    is free; requests for other meshes may pass it.  ``elastic`` (batch mode): a waiting
    request with no free slot of its mesh gets a new slot when the engine's budget allows
    it, after evicting idle slots of meshes nobody waits for (least recently used first).
    The engine then needs ``keys()``, ``footprint(key)``, ``add_slot(key)``,
    ``remove_slot(slot)``, ``device_bytes`` and ``budget_bytes``.
    """

    def __init__(self, engine, mode: str = "batch", max_chunk: int = 4, keep_results: bool = False,
                 clock: Callable[[], float] = time.perf_counter, sleep: Callable[[float], None] = time.sleep,
                 elastic: bool = False):
        if mode not in ("batch", "serial"):
            raise ValueError("mode is 'batch' or 'serial'")
        if elastic and mode != "batch":
            raise ValueError("elastic admission needs mode 'batch'")
        self.engine = engine
        self.mode = mode
        self.max_chunk = max(1, int(max_chunk))
        self.keep_results = keep_results
        self.clock = clock
        self.sleep = sleep
        self.elastic = elastic
        self.slots_added = 0
        self.slots_evicted = 0

    def run(self, requests: Sequence[Request]) -> RunStats:
        pending = deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        waiting: Dict[str, deque] = {}
        slots = self.engine.slots
        mesh_keys = {s.mesh for s in slots}
        if self.elastic:
            budget = self.engine.budget_bytes
            for r in pending:
                if r.mesh not in self.engine.keys():
                    raise ValueError(f"request {r.rid}: mesh {r.mesh!r} is not in the catalogue")
                if budget is not None and self.engine.footprint(r.mesh) > budget:
                    raise ValueError(f"request {r.rid}: one slot of mesh {r.mesh!r} exceeds the budget")
        else:
            for r in pending:
                if r.mesh not in mesh_keys:
                    raise ValueError(f"request {r.rid}: no slot holds mesh {r.mesh!r}")
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        finished: List[Request] = []
        steps_launched = 0
        members_total = 0
        dof_updates = 0.0
        n_total = len(pending)
        while len(finished) < n_total:
            # arrivals
            tnow = now()
            while pending and pending[0].arrival <= tnow:
                r = pending.popleft()
                waiting.setdefault(r.mesh, deque()).append(r)
            # admission
            free_by_mesh: Dict[str, List[Slot]] = {}
            for s in slots:
                if s.busy is None:
                    free_by_mesh.setdefault(s.mesh, []).append(s)
            if self.mode == "serial":
                running = [s for s in slots if s.busy is not None]
                if not running:
                    # the oldest waiting request of any mesh
                    cands = [(q[0].arrival, q[0].rid, k) for k, q in waiting.items() if q and free_by_mesh.get(k)]
                    if cands:
                        _, _, k = min(cands)
                        self._admit(waiting[k].popleft(), free_by_mesh[k][0], tnow)
            else:
                for k, q in waiting.items():
                    free = free_by_mesh.get(k, [])
                    while q and free:
                        self._admit(q.popleft(), free.pop(0), tnow)
                if self.elastic:
                    for k, q in waiting.items():
                        while q:
                            s = self._new_slot(k, waiting)
                            if s is None:
                                break
                            self._admit(q.popleft(), s, tnow)
            running = [s for s in slots if s.busy is not None]
            if not running:
                if pending:
                    dt = pending[0].arrival - now()
                    if dt > 0:
                        self.sleep(dt)
                    continue
                raise RuntimeError("requests left waiting with no slot able to take them")
            # advance
            if self.mode == "serial":
                s = running[0]
                chunk = s.remaining
                statuses = [self.engine.step_alone(s, chunk)]
            else:
                chunk = min(self.max_chunk, min(s.remaining for s in running))
                statuses = self.engine.step(running, chunk)
            steps_launched += chunk
            members_total += chunk * len(running)
            tdone = now()
            for s, st in zip(running, statuses):
                s.last_used = tdone
                s.remaining -= chunk
                dof_updates += 5.0 * s.n_nodes * chunk
                if st != 0 and s.busy.status == 0:
                    s.busy.status = st
                if s.remaining == 0:
                    r = s.busy
                    if self.keep_results:
                        r.q, r.t = self.engine.read(s)
                    r.done = tdone
                    finished.append(r)
                    s.busy = None
        makespan = now()
        lat = sorted(r.latency for r in finished)
        return RunStats(
            requests=n_total,
            makespan_s=makespan,
            dof_updates=dof_updates,
            throughput=dof_updates / makespan if makespan > 0 else math.nan,
            p50_s=_quantile(lat, 0.50),
            p99_s=_quantile(lat, 0.99),
            mean_s=float(np.mean(lat)) if lat else math.nan,
            steps_launched=steps_launched,
            mean_batch=members_total / steps_launched if steps_launched else 0.0,
            failed=sum(1 for r in finished if r.status != 0),
            latencies=lat,
        )

    def _new_slot(self, key, waiting) -> Optional[Slot]:
        """A new slot of ``key`` within the budget, evicting idle slots of meshes with no
        waiting request (least recently used first); None if it cannot fit now."""
        eng = self.engine
        need = eng.footprint(key)
        budget = eng.budget_bytes
        if budget is not None and eng.device_bytes + need > budget:
            idle = sorted((s for s in eng.slots if s.busy is None and s.mesh != key and not waiting.get(s.mesh)),
                          key=lambda s: (s.last_used, s.sid))
            freeable = sum(s.nbytes for s in idle)
            if eng.device_bytes - freeable + need > budget:
                return None
            for s in idle:
                if eng.device_bytes + need <= budget:
                    break
                eng.remove_slot(s)
                self.slots_evicted += 1
        s = eng.add_slot(key)
        if s is not None:
            self.slots_added += 1
        return s

    def _admit(self, r: Request, s: Slot, tnow: float):
        self.engine.load(s, r.q0)
        s.busy = r
        s.remaining = int(r.nsteps)
        r.admitted = tnow


def _quantile(sorted_vals: Sequence[float], q: float) -> float:
    """Nearest-rank quantile of sorted values."""
    if not sorted_vals:
        return math.nan
    k = max(0, min(len(sorted_vals) - 1, int(math.ceil(q * len(sorted_vals))) - 1))
    return float(sorted_vals[k])


def poisson_requests(rate_per_s: float, n: int, meshes: Sequence[str], nsteps: Sequence[int], seed: int = 0,
                     weights: Optional[Sequence[float]] = None) -> List[Request]:
    """n requests with exponential inter-arrival times (a Poisson process of the given
    rate), each for a mesh and a step count drawn uniformly (or with ``weights``)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_per_s) if rate_per_s > 0 else 0.0
        k = rng.choice(len(meshes), p=None if weights is None else np.asarray(weights) / np.sum(weights))
        out.append(Request(rid=i, mesh=meshes[k], nsteps=int(rng.choice(nsteps)), arrival=t))
    return out
