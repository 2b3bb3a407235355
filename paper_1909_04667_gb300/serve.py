"""Continuous-batching force server over device-resident trees.

A request asks for the forces on a subset of one system's particles.  The
server keeps the trees of recently used systems resident on the GPU under the
context's HBM budget and serves requests in rounds: requests that arrive while
a round is on the GPU are admitted as plan capacity and memory free up (one
round in flight by default, optionally two on their own streams), their
missing trees are built on a separate stream -- overlapping the walk in
flight -- and each round runs as one batched walk launch
(``tpm_compute_forces_batch``).  When memory runs short, resident systems
that no waiting or running request needs are evicted, least recently used
first; their |a| stays on the host for the relative criterion after a
rebuild.

The first request for a system uses the geometric criterion; later requests
use the relative criterion (paper Sec. 3.1) when every requested particle has
an |a| from an earlier evaluation, unless the server runs with a fixed
criterion.  ``serve_per_request`` is the plain baseline: one build (if
needed), one ``tpm_compute_forces`` call and one synchronisation per request,
in arrival order.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import CRIT_BH, CRIT_RELATIVE, BuildParams, Context, ForceParams, TreePMError

_EBUDGET = -2


@dataclass(eq=False)
class ServeRequest:
    """Forces on particles ``ids`` of system ``sid`` (arrival in seconds).
    Requests compare by identity."""

    rid: int
    sid: int
    ids: np.ndarray
    arrival: float = 0.0
    acc: np.ndarray = None
    pot: np.ndarray = None
    n_int: np.ndarray = None
    criterion: int = -1
    t_start: float = float("nan")  # when its walk was enqueued (the build, if any, came before)
    t_done: float = float("nan")

    @property
    def latency(self) -> float:
        return self.t_done - self.arrival


@dataclass
class _Resident:
    system: object
    aold: object          # torch float32 (n,), on the device
    aold_valid: object    # numpy bool (n,), on the host: which particles have an |a|
    inflight: int = 0
    n_valid: int = 0      # particles with an |a| (once all have one, no per-id checks)
    built: object = None  # event recorded after the build on the build stream

    def all_valid(self, ids) -> bool:
        return self.n_valid == len(self.aold_valid) or bool(self.aold_valid[ids].all())

    def mark_valid(self, ids):
        if self.n_valid < len(self.aold_valid):
            self.aold_valid[ids] = True
            self.n_valid = int(np.count_nonzero(self.aold_valid))

    def ready(self) -> bool:
        if self.built is not None and self.built.query():
            self.built = None  # built: no later round needs to wait for it
        return self.built is None


@dataclass
class _Round:
    reqs: list
    acc: object
    pot: object
    nint: object
    offsets: np.ndarray
    event: object          # results copied to the host
    done: object = None    # and the |a| bookkeeping after them
    sids: list = field(default_factory=list)
    slot: object = None


class _RingIndex:
    """Placement of saved entries in a ring of ``cap`` elements (host logic
    only; the server keeps the data in a pinned buffer): entries go one after
    another, wrapping to the start when one does not fit at the end, and the
    entries a new one overlaps are forgotten (they are older: an entry from
    two laps back can survive past the end of the last lap, so these are not
    always the oldest ones)."""

    def __init__(self, cap: int):
        self.cap = int(cap)
        self.head = 0
        self.entries = collections.OrderedDict()  # key -> (offset, n, payload), oldest first

    def place(self, key, n: int, payload=None):
        """Offset of a new entry of ``n`` elements, or None if it cannot fit."""
        n = int(n)
        if n > self.cap:
            return None
        self.entries.pop(key, None)
        off = self.head if self.head + n <= self.cap else 0
        for old in [k for k, (o, m, _) in self.entries.items() if o < off + n and off < o + m]:
            del self.entries[old]
        self.head = off + n
        self.entries[key] = (off, n, payload)
        return off

    def take(self, key):
        """(offset, n, payload) of the entry, removed, or None."""
        return self.entries.pop(key, None)

    def clear(self):
        self.entries.clear()


class _Slot:
    """What one round in flight needs: a stream, a plan (batched calls on one
    plan must not overlap), device buffers and pinned staging."""

    def __init__(self, torch, ctx, dev, max_ids, max_req, group_size, priority=0):
        self.stream = torch.cuda.Stream(dev, priority=priority)
        self.plan = ctx.create_plan(max_ids, max_req)
        if group_size:
            self.plan.group_size = group_size
        m = max_ids
        self.ids_h = torch.empty(m, dtype=torch.int32).pin_memory()
        self.acc_h = torch.empty((m, 3), dtype=torch.float32).pin_memory()
        self.pot_h = torch.empty(m, dtype=torch.float32).pin_memory()
        self.nint_h = torch.empty(m, dtype=torch.int32).pin_memory()
        with torch.cuda.stream(self.stream):
            self.ids_d = torch.empty(m, dtype=torch.int32, device=dev)
            self.acc_d = torch.empty((m, 3), dtype=torch.float32, device=dev)
            self.pot_d = torch.empty(m, dtype=torch.float32, device=dev)
            self.nint_d = torch.empty(m, dtype=torch.int32, device=dev)
        self.busy = False


class ForceServer:
    """Serves ``ServeRequest``s for systems described by ``source(sid)``, which
    returns ``(pos float64 (n,3), mass float32 (n,), BuildParams)`` (host
    arrays in pinned memory keep the uploads asynchronous; device tensors are
    taken as they are).

    Up to ``slots`` rounds are in flight at once, each on its own stream with
    its own plan and buffers (with two, a request arriving while a long round
    walks starts at once and shares the GPU with it; on the serving workload
    one slot measured better: concurrent rounds stretch the large rounds that
    set the tail); a system is in at most one round in flight, with at most
    one request (its |a| bookkeeping is ordered on that round's stream, and a
    later request on it can use the relative criterion with this round's |a|).
    A round takes the waiting requests whose trees are ready first (in arrival
    order); requests whose trees are still building wait for a later round
    rather than hold ready ones back.  A tree that a queued request needs is
    not evicted before that request has been served (trees built ahead for
    waiting requests would otherwise be evicted by the next build ahead).
    With ``keep_aold`` an evicted system's |a| (and which particles have one)
    is kept in a pinned host ring of ``aold_cache_bytes`` (entries that a
    later one overwrites as the ring wraps are forgotten) and restored when
    its tree is rebuilt: the rebuilt tree is the same tree, so the relative
    criterion stays available.
    ``keep_results`` is a bool or a
    predicate on the request: results of the others are timed back to the
    host and dropped."""

    def __init__(self, ctx: Context, source, max_round_ids: int = 1 << 21, max_round_requests: int = 512,
                 theta: float = 0.5, alpha: float = 0.0025, policy: str = "adaptive", group_size: int = None,
                 keep_results=True, slots: int = 1, prioritise_large: bool = True, keep_aold: bool = True,
                 aold_cache_bytes: int = 256 << 20):
        import torch

        self.torch = torch
        self.ctx = ctx
        self.source = source
        self.max_ids, self.max_req = int(max_round_ids), int(max_round_requests)
        self.large_round_ids = 1 << 16
        self.theta, self.alpha, self.policy = theta, alpha, policy
        self.dev = torch.device("cuda", ctx.device)
        # the first slot's stream (and the builds) run at high priority: a large
        # round there keeps its pace while small rounds share the GPU with it
        self.prioritise_large = bool(prioritise_large)
        pri = -1 if self.prioritise_large else 0
        self.build_stream = torch.cuda.Stream(self.dev, priority=pri)
        self.slots = [_Slot(torch, ctx, self.dev, self.max_ids, self.max_req, group_size, priority=pri if k == 0 else 0)
                      for k in range(slots)]
        self.plan = self.slots[0].plan
        self.resident: "collections.OrderedDict[int, _Resident]" = collections.OrderedDict()
        self.builds = 0
        self.evictions = 0
        self.keep_results = keep_results
        self._wanted = collections.Counter()  # queued requests per system: not evictable
        self._busy = set()  # systems in a round in flight
        self._t0 = time.perf_counter()  # start of the current serve() call
        # |a| of evicted systems (pinned host copies): a rebuilt tree is the
        # same tree (the build is deterministic), so its particles' |a| stay
        # valid for the relative criterion
        self.keep_aold = bool(keep_aold)
        # pinned float32 ring, allocated here: a pinned allocation of this size
        # takes tens of milliseconds and must not fall inside a request
        self._ring_index = _RingIndex(max(int(aold_cache_bytes) // 4, 1 << 20))  # payload: (valid mask, n_valid)
        self._ring = torch.empty(self._ring_index.cap, dtype=torch.float32).pin_memory() if self.keep_aold else None
        # a build was refused for memory: no other is tried (and no system drawn
        # for it) until a round completes and systems become evictable again
        self._blocked = False

    def close(self):
        for r in self.resident.values():
            r.system.release()
        self.resident.clear()
        self._ring_index.clear()
        for sl in self.slots:
            sl.plan.close()

    def _keep(self, r) -> bool:
        return self.keep_results(r) if callable(self.keep_results) else bool(self.keep_results)

    # -------------------------------------------------------------- residency
    def _evict_one(self) -> bool:
        for sid, r in self.resident.items():  # least recently used first
            if r.inflight == 0 and r.ready() and not self._wanted[sid]:
                if self.keep_aold and r.n_valid:
                    self._save_aold(sid, r)
                r.system.release()
                del self.resident[sid]
                self.evictions += 1
                return True
        return False

    def _save_aold(self, sid, r):
        """Copies the system's |a| into the pinned ring on the build stream
        (its last round's bookkeeping has completed: the system is not in
        flight).  Saved entries the copy overwrites (the oldest) are
        forgotten.  Saves and uploads all run on the build stream, in order,
        and the device copy was allocated on it, so none needs an event."""
        torch = self.torch
        n = int(r.aold.shape[0])
        off = self._ring_index.place(sid, n, (r.aold_valid, r.n_valid))
        if off is None:
            return
        with torch.cuda.stream(self.build_stream):
            self._ring[off:off + n].copy_(r.aold, non_blocking=True)

    def ensure_resident(self, sid: int) -> bool:
        """Enqueues the build of ``sid`` on the build stream if it is not
        resident; False if the budget cannot hold it while the systems in
        flight or wanted by waiting requests stay (after one such refusal,
        until a round completes)."""
        torch = self.torch
        if sid in self.resident:
            self.resident.move_to_end(sid)
            return True
        if self._blocked:
            return False
        with torch.cuda.stream(self.build_stream):  # a source may draw the particles on the device
            pos, mass, bp = self.source(sid)
        while True:
            try:
                system = self.ctx.build_tree(pos, mass, bp, stream=self.build_stream.cuda_stream)
                break
            except TreePMError as e:
                if e.status != _EBUDGET or not self._evict_one():
                    if e.status == _EBUDGET:
                        self._blocked = True
                        return False
                    raise
        n = system.n
        saved = self._ring_index.take(sid) if self.keep_aold else None
        with torch.cuda.stream(self.build_stream):
            aold = torch.empty(n, dtype=torch.float32, device=self.dev)
            if saved is not None:  # the copy to the host came earlier on this stream
                aold.copy_(self._ring[saved[0]:saved[0] + n], non_blocking=True)
            else:
                aold.zero_()
            ev = torch.cuda.Event()
            ev.record(self.build_stream)
        if saved is not None:
            res = _Resident(system, aold, saved[2][0], built=ev, n_valid=saved[2][1])
        else:
            res = _Resident(system, aold, np.zeros(n, dtype=bool), built=ev)
        self.resident[sid] = res
        self.builds += 1
        return True

    # -------------------------------------------------------------- rounds
    def _params_for(self, res: _Resident, ids) -> ForceParams:
        if self.policy == "bh":
            return ForceParams(crit=CRIT_BH, theta=self.theta)
        if self.policy == "relative" or (self.policy == "adaptive" and res.all_valid(ids)):
            return ForceParams(crit=CRIT_RELATIVE, alpha=self.alpha)
        return ForceParams(crit=CRIT_BH, theta=self.theta)

    def _launch(self, reqs, slot: _Slot) -> _Round:
        """Enqueues one round on ``slot``: the walk and the copies of its
        results come first (the round is complete when they are), the
        bookkeeping of |a| for later criteria after them, overlapping the
        walk."""
        torch = self.torch
        st = slot.stream
        slot.busy = True
        now = time.perf_counter() - self._t0
        for r in reqs:
            r.t_start = now
        for r in reqs:  # the round waits for its own systems' builds only
            self.resident.move_to_end(r.sid)  # most recently used
            b = self.resident[r.sid].built
            if b is not None:
                st.wait_event(b)
        with torch.cuda.stream(st):
            sizes = [len(r.ids) for r in reqs]
            off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
            n = int(off[-1])
            ids_np = slot.ids_h.numpy()
            for k, r in enumerate(reqs):
                ids_np[off[k]:off[k + 1]] = r.ids
            ids_d = slot.ids_d[:n]
            ids_d.copy_(slot.ids_h[:n], non_blocking=True)
            systems, params, aolds, parts = [], [], [], []
            for k, r in enumerate(reqs):
                res = self.resident[r.sid]
                res.inflight += 1
                self._busy.add(r.sid)
                part = ids_d[off[k]:off[k + 1]]
                fp = self._params_for(res, r.ids)
                r.criterion = fp.crit
                systems.append(res.system)
                params.append(fp)
                parts.append(part)
                aolds.append(torch.index_select(res.aold, 0, part))
            a_old = aolds[0] if len(aolds) == 1 else torch.cat(aolds)
            acc, pot, nint = slot.acc_d[:n], slot.pot_d[:n], slot.nint_d[:n]
            walked = False
            plan = slot.plan
            if len(reqs) == 1 and plan.group_size == 32 and plan.stack_depth == 192:
                # a round of one request (light load): the plain call runs the
                # same walk without the batch's request sort and group table;
                # its scratch comes from the budget, else the batch path runs
                try:
                    systems[0].compute_forces(active_ids=ids_d, a_old=a_old, fp=params[0], acc=acc, pot=pot,
                                              n_int=nint, stream=st.cuda_stream)
                    walked = True
                except TreePMError as e:
                    if e.status != _EBUDGET:
                        raise
            if not walked:
                plan.compute_forces_batch(systems, off, params, ids_d, acc, a_old=a_old, pot=pot, n_int=nint,
                                          stream=st.cuda_stream)
            slot.acc_h[:n].copy_(acc, non_blocking=True)
            slot.pot_h[:n].copy_(pot, non_blocking=True)
            slot.nint_h[:n].copy_(nint, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(st)
            # |a| of this evaluation becomes a_old of later ones (stream-ordered
            # before any later round on this system: a system is in one round
            # in flight at a time)
            amag = torch.linalg.vector_norm(acc, dim=1)
            for k, r in enumerate(reqs):
                res = self.resident[r.sid]
                res.aold.index_copy_(0, parts[k].long(), amag[off[k]:off[k + 1]])
                res.mark_valid(r.ids)
            done = torch.cuda.Event()
            done.record(st)
        return _Round(reqs, slot.acc_h[:n], slot.pot_h[:n], slot.nint_h[:n], off, ev, done,
                      [r.sid for r in reqs], slot)

    def _complete(self, rnd: _Round, t0: float):
        rnd.event.synchronize()
        now = time.perf_counter() - t0
        rnd.done.synchronize()  # a system the round used may be evicted after this
        acc, pot, nint = rnd.acc.numpy(), rnd.pot.numpy(), rnd.nint.numpy()
        for k, r in enumerate(rnd.reqs):
            lo, hi = rnd.offsets[k], rnd.offsets[k + 1]
            if self._keep(r):  # copies: the pinned buffers serve the next round
                r.acc, r.pot, r.n_int = acc[lo:hi].copy(), pot[lo:hi].copy(), nint[lo:hi].copy()
            r.t_done = now
            res = self.resident.get(r.sid)
            if res is not None:
                res.inflight -= 1
            self._busy.discard(r.sid)
        rnd.slot.busy = False
        self._blocked = False

    def _form_round(self, queue):
        """Requests for one round, taken out of ``queue``: those whose trees
        are ready first (arrival order), else -- none being ready -- those
        whose trees are building (the round then waits for their builds on the
        GPU), else the first waiting request whose build can start now.
        Requests of a system in flight stay queued; no build is started while
        ready requests can go (builds ahead start between rounds, one at a
        time, in ``serve``)."""
        # a system goes into one round once: a second request for it waits
        # for the next round, whose criterion can then use this round's |a|
        busy = set(self._busy)
        ready, building = [], []
        nids_r = nids_b = 0
        first_cold = None
        for r in queue:
            if len(ready) >= self.max_req or nids_r >= self.max_ids:
                break
            if r.sid in busy:
                continue
            res = self.resident.get(r.sid)
            if res is None:
                if first_cold is None:
                    first_cold = r
                continue
            if res.ready():
                if nids_r + len(r.ids) <= self.max_ids:
                    ready.append(r)
                    nids_r += len(r.ids)
                    busy.add(r.sid)
            elif len(building) < self.max_req and nids_b + len(r.ids) <= self.max_ids:
                building.append(r)
                nids_b += len(r.ids)
                busy.add(r.sid)
        batch = ready or building
        if not batch and first_cold is not None and self.ensure_resident(first_cold.sid):
            batch = [first_cold]
        if batch:
            taken = {id(r) for r in batch}
            rest = [r for r in queue if id(r) not in taken]
            queue.clear()
            queue.extend(rest)
            for r in batch:
                self._wanted[r.sid] -= 1
        return batch

    def _pick_slot(self, free, batch):
        """The high-priority slot for a large round (or a round that waits for
        a build), a low-priority one for a small round when one is free."""
        if len(free) == 1 or not self.prioritise_large:
            return free[0]
        large = sum(len(r.ids) for r in batch) >= self.large_round_ids or any(
            self.resident[r.sid].built is not None for r in batch)
        return free[0] if large else free[-1]

    def _build_ahead(self, queue) -> bool:
        """Starts the build of the first waiting request's system that is not
        resident (one per call); False if there is none or it does not fit."""
        for k, r in enumerate(queue):
            if k >= self.max_req:
                break
            if r.sid not in self.resident:
                return self.ensure_resident(r.sid)
        return False

    def serve(self, requests, realtime: bool = True):
        """Serves ``requests`` (sorted by arrival).  With ``realtime`` a request
        becomes visible at its arrival time; otherwise all are visible at once.
        Returns the requests with results and completion times."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        queue = collections.deque()
        inflight = []
        i = 0
        t0 = self._t0 = time.perf_counter()
        while i < len(reqs) or queue or inflight:
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                queue.append(reqs[i])
                self._wanted[reqs[i].sid] += 1
                i += 1
            for rnd in [x for x in inflight if x.event.query()]:
                self._complete(rnd, t0)
                inflight.remove(rnd)
            if not inflight:
                self._blocked = False  # every resident system not wanted is evictable
            free = [sl for sl in self.slots if not sl.busy]
            if queue and free:
                batch = self._form_round(queue)
                if batch:
                    inflight.append(self._launch(batch, self._pick_slot(free, batch)))
                    continue
                if not inflight:
                    r = queue[0]
                    if len(r.ids) > self.max_ids:
                        raise ValueError("request %d larger than the server's round size" % r.rid)
                    raise MemoryError("the tree of system %d does not fit in the HBM budget" % r.sid)
            if queue:
                # admit while the GPU walks: start a build a waiting request
                # needs -- one per pass, so that finished rounds are seen
                self._build_ahead(queue)
                time.sleep(0)
            elif inflight:
                time.sleep(0)
            elif i < len(reqs):
                time.sleep(max(0.0, min(1e-3, reqs[i].arrival - now)))
        return reqs


def serve_per_request(ctx: Context, source, requests, theta: float = 0.5, alpha: float = 0.0025,
                      policy: str = "adaptive", realtime: bool = True, keep_results=True, resident=None,
                      plain_fp32: bool = False):
    """Baseline: requests in arrival order, each with its own build (if the
    system is not resident), ``tpm_compute_forces`` call and synchronisation;
    LRU eviction under the same budget, for a build or for the scratch memory
    of a force call.  ``resident`` (an OrderedDict) keeps the resident systems
    across calls; without it they are released at the end.  ``plain_fp32``
    evaluates in the plain FP32 form (absolute FP32 coordinates), the
    comparison arm of the mixed-precision scheme.  ``keep_results`` is a bool
    or a predicate on the request."""
    import torch

    dev = torch.device("cuda", ctx.device)
    keep = resident is not None
    resident = resident if keep else collections.OrderedDict()
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in reqs:
        if realtime:
            wait = r.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        if r.sid in resident:
            resident.move_to_end(r.sid)
        else:
            pos, mass, bp = source(r.sid)
            while True:
                try:
                    system = ctx.build_tree(pos, mass, bp)
                    break
                except TreePMError as e:
                    if e.status != _EBUDGET or not resident:
                        raise
                    _, (old, _, _) = resident.popitem(last=False)
                    old.release()
            resident[r.sid] = (system, torch.zeros(system.n, device=dev),
                               _Resident(None, None, np.zeros(system.n, dtype=bool)))
        system, aold, valid = resident[r.sid]
        ids_d = torch.from_numpy(r.ids.astype(np.int32)).to(dev)
        part = ids_d.long()
        if policy == "bh" or (policy == "adaptive" and not valid.all_valid(r.ids)):
            fp = ForceParams(crit=CRIT_BH, theta=theta, plain_fp32=plain_fp32)
        else:
            fp = ForceParams(crit=CRIT_RELATIVE, alpha=alpha, plain_fp32=plain_fp32)
        r.criterion = fp.crit
        r.t_start = time.perf_counter() - t0
        while True:
            try:
                acc, pot, nint = system.compute_forces(active_ids=ids_d, a_old=aold[part].contiguous(), fp=fp)
                break
            except TreePMError as e:
                # the call's scratch does not fit: evict another system
                victim = next((sid for sid in resident if sid != r.sid), None)
                if e.status != _EBUDGET or victim is None:
                    raise
                resident.pop(victim)[0].release()
        aold[part] = torch.linalg.vector_norm(acc, dim=1)
        valid.mark_valid(r.ids)
        a_h, p_h, n_h = acc.cpu().numpy(), pot.cpu().numpy(), nint.cpu().numpy()
        if (keep_results(r) if callable(keep_results) else keep_results):
            r.acc, r.pot, r.n_int = a_h, p_h, n_h
        r.t_done = time.perf_counter() - t0
    if not keep:
        for system, _, _ in resident.values():
            system.release()
    return reqs
