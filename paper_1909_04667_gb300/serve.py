"""Continuous-batching force server over device-resident trees.

A request asks for the forces on a subset of one system's particles.  The
server keeps the trees of recently used systems resident on the GPU under the
context's HBM budget and serves requests in rounds: all requests that have
arrived while the previous round was on the GPU are admitted (as long as the
plan's slots last and their trees fit in memory), their missing trees are
built on a second stream -- overlapping the walk still in flight -- and the
whole round runs as one batched walk launch (``tpm_compute_forces_batch``).
When memory runs short, resident systems that no request in flight needs are
evicted, least recently used first.

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


@dataclass
class ServeRequest:
    """Forces on particles ``ids`` of system ``sid`` (arrival in seconds)."""

    rid: int
    sid: int
    ids: np.ndarray
    arrival: float = 0.0
    acc: np.ndarray = None
    pot: np.ndarray = None
    n_int: np.ndarray = None
    criterion: int = -1
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

    def all_valid(self, ids) -> bool:
        return self.n_valid == len(self.aold_valid) or bool(self.aold_valid[ids].all())

    def mark_valid(self, ids):
        if self.n_valid < len(self.aold_valid):
            self.aold_valid[ids] = True
            self.n_valid = int(np.count_nonzero(self.aold_valid))


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


class ForceServer:
    """Serves ``ServeRequest``s for systems described by ``source(sid)``, which
    returns ``(pos float64 (n,3), mass float32 (n,), BuildParams)`` as host
    arrays (pinned memory keeps the uploads asynchronous)."""

    def __init__(self, ctx: Context, source, max_round_ids: int = 1 << 21, max_round_requests: int = 512,
                 theta: float = 0.5, alpha: float = 0.0025, policy: str = "adaptive", group_size: int = None,
                 keep_results: bool = True):
        import torch

        self.torch = torch
        self.ctx = ctx
        self.source = source
        self.plan = ctx.create_plan(max_round_ids, max_round_requests)
        if group_size:
            self.plan.group_size = group_size
        self.max_ids, self.max_req = int(max_round_ids), int(max_round_requests)
        self.theta, self.alpha, self.policy = theta, alpha, policy
        self.dev = torch.device("cuda", ctx.device)
        self.walk_stream = torch.cuda.Stream(self.dev)
        self.build_stream = torch.cuda.Stream(self.dev)
        self.resident: "collections.OrderedDict[int, _Resident]" = collections.OrderedDict()
        self.builds = 0
        self.evictions = 0
        self.keep_results = keep_results  # False: time the results' return, then drop them
        # pinned staging, reused by every round (one round is in flight at a
        # time): ids in, results out -- asynchronous copies need pinned memory
        m = self.max_ids
        self.ids_h = torch.empty(m, dtype=torch.int32).pin_memory()
        self.acc_h = torch.empty((m, 3), dtype=torch.float32).pin_memory()
        self.pot_h = torch.empty(m, dtype=torch.float32).pin_memory()
        self.nint_h = torch.empty(m, dtype=torch.int32).pin_memory()
        # and their device counterparts (the walk stream orders the rounds)
        with torch.cuda.stream(self.walk_stream):
            self.ids_d = torch.empty(m, dtype=torch.int32, device=self.dev)
            self.acc_d = torch.empty((m, 3), dtype=torch.float32, device=self.dev)
            self.pot_d = torch.empty(m, dtype=torch.float32, device=self.dev)
            self.nint_d = torch.empty(m, dtype=torch.int32, device=self.dev)

    def close(self):
        for r in self.resident.values():
            r.system.release()
        self.resident.clear()
        self.plan.close()

    # -------------------------------------------------------------- residency
    def _evict_one(self) -> bool:
        for sid, r in self.resident.items():  # least recently used first
            if r.inflight == 0:
                r.system.release()
                del self.resident[sid]
                self.evictions += 1
                return True
        return False

    def ensure_resident(self, sid: int) -> bool:
        """Builds the tree of ``sid`` on the build stream if it is not resident;
        False if the budget cannot hold it while the systems in flight stay."""
        torch = self.torch
        if sid in self.resident:
            self.resident.move_to_end(sid)
            return True
        with torch.cuda.stream(self.build_stream):  # a source may draw the particles on the device
            pos, mass, bp = self.source(sid)
        while True:
            try:
                system = self.ctx.build_tree(pos, mass, bp, stream=self.build_stream.cuda_stream)
                break
            except TreePMError as e:
                if e.status != _EBUDGET or not self._evict_one():
                    if e.status == _EBUDGET:
                        return False
                    raise
        n = system.n
        with torch.cuda.stream(self.build_stream):
            aold = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.resident[sid] = _Resident(system, aold, np.zeros(n, dtype=bool))
        self.builds += 1
        return True

    # -------------------------------------------------------------- rounds
    def _params_for(self, res: _Resident, ids) -> ForceParams:
        if self.policy == "bh":
            return ForceParams(crit=CRIT_BH, theta=self.theta)
        if self.policy == "relative" or (self.policy == "adaptive" and res.all_valid(ids)):
            return ForceParams(crit=CRIT_RELATIVE, alpha=self.alpha)
        return ForceParams(crit=CRIT_BH, theta=self.theta)

    def _launch(self, reqs) -> _Round:
        """Enqueues one round: the walk and the copies of its results come
        first (the round is complete when they are), the bookkeeping of |a|
        for later criteria after them, overlapping the walk."""
        torch = self.torch
        self.walk_stream.wait_stream(self.build_stream)
        with torch.cuda.stream(self.walk_stream):
            sizes = [len(r.ids) for r in reqs]
            off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
            n = int(off[-1])
            ids_np = self.ids_h.numpy()
            for k, r in enumerate(reqs):
                ids_np[off[k]:off[k + 1]] = r.ids
            ids_d = self.ids_d[:n]
            ids_d.copy_(self.ids_h[:n], non_blocking=True)
            systems, params, aolds, parts = [], [], [], []
            for k, r in enumerate(reqs):
                res = self.resident[r.sid]
                res.inflight += 1
                part = ids_d[off[k]:off[k + 1]]
                fp = self._params_for(res, r.ids)
                r.criterion = fp.crit
                systems.append(res.system)
                params.append(fp)
                parts.append(part)
                aolds.append(torch.index_select(res.aold, 0, part))
            a_old = aolds[0] if len(aolds) == 1 else torch.cat(aolds)
            acc, pot, nint = self.acc_d[:n], self.pot_d[:n], self.nint_d[:n]
            walked = False
            if len(reqs) == 1 and self.plan.group_size == 32 and self.plan.stack_depth == 192:
                # a round of one request (light load): the plain call runs the
                # same walk without the batch's request sort and group table;
                # its scratch comes from the budget, else the batch path runs
                try:
                    systems[0].compute_forces(active_ids=ids_d, a_old=a_old, fp=params[0], acc=acc, pot=pot,
                                              n_int=nint, stream=self.walk_stream.cuda_stream)
                    walked = True
                except TreePMError as e:
                    if e.status != _EBUDGET:
                        raise
            if not walked:
                self.plan.compute_forces_batch(systems, off, params, ids_d, acc, a_old=a_old, pot=pot, n_int=nint,
                                               stream=self.walk_stream.cuda_stream)
            self.acc_h[:n].copy_(acc, non_blocking=True)
            self.pot_h[:n].copy_(pot, non_blocking=True)
            self.nint_h[:n].copy_(nint, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.walk_stream)
            # |a| of this evaluation becomes a_old of later ones (stream-ordered
            # before any later round)
            amag = torch.linalg.vector_norm(acc, dim=1)
            for k, r in enumerate(reqs):
                res = self.resident[r.sid]
                res.aold.index_copy_(0, parts[k].long(), amag[off[k]:off[k + 1]])
                res.mark_valid(r.ids)
            done = torch.cuda.Event()
            done.record(self.walk_stream)
        return _Round(reqs, self.acc_h[:n], self.pot_h[:n], self.nint_h[:n], off, ev, done, [r.sid for r in reqs])

    def _complete(self, rnd: _Round, t0: float):
        rnd.event.synchronize()
        now = time.perf_counter() - t0
        rnd.done.synchronize()  # a system the round used may be evicted after this
        acc, pot, nint = rnd.acc.numpy(), rnd.pot.numpy(), rnd.nint.numpy()
        for k, r in enumerate(rnd.reqs):
            lo, hi = rnd.offsets[k], rnd.offsets[k + 1]
            if self.keep_results:  # copies: the pinned buffers serve the next round
                r.acc, r.pot, r.n_int = acc[lo:hi].copy(), pot[lo:hi].copy(), nint[lo:hi].copy()
            r.t_done = now
            res = self.resident.get(r.sid)
            if res is not None:
                res.inflight -= 1

    def serve(self, requests, realtime: bool = True):
        """Serves ``requests`` (sorted by arrival).  With ``realtime`` a request
        becomes visible at its arrival time; otherwise all are visible at once.
        Returns the requests with results and completion times."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        queue = collections.deque()
        inflight = None
        i = 0
        t0 = time.perf_counter()
        while i < len(reqs) or queue or inflight is not None:
            now = time.perf_counter() - t0
            while i < len(reqs) and (not realtime or reqs[i].arrival <= now):
                queue.append(reqs[i])
                i += 1
            if inflight is not None and inflight.event.query():
                self._complete(inflight, t0)
                inflight = None
            if queue and inflight is None:
                batch, nids = [], 0
                while queue and len(batch) < self.max_req and nids + len(queue[0].ids) <= self.max_ids:
                    if not self.ensure_resident(queue[0].sid):
                        break  # waits for memory held by the round in flight
                    r = queue.popleft()
                    batch.append(r)
                    nids += len(r.ids)
                if not batch:
                    if len(queue[0].ids) > self.max_ids:
                        raise ValueError("request %d larger than the server's round size" % queue[0].rid)
                    raise MemoryError("the tree of system %d does not fit in the HBM budget" % queue[0].sid)
                inflight = self._launch(batch)
            elif queue and inflight is not None:
                # admit while the GPU walks: build a tree a waiting request
                # needs -- one per pass, so that the round in flight is seen
                # to finish between builds
                for r in list(queue)[:self.max_req]:
                    if r.sid not in self.resident:
                        self.ensure_resident(r.sid)
                        break
                if not inflight.event.query():
                    time.sleep(0)
            elif inflight is not None:
                time.sleep(0)
            elif i < len(reqs):
                time.sleep(max(0.0, min(1e-3, reqs[i].arrival - now)))
        return reqs


def serve_per_request(ctx: Context, source, requests, theta: float = 0.5, alpha: float = 0.0025,
                      policy: str = "adaptive", realtime: bool = True, keep_results: bool = True, resident=None):
    """Baseline: requests in arrival order, each with its own build (if the
    system is not resident), ``tpm_compute_forces`` call and synchronisation;
    LRU eviction under the same budget, for a build or for the scratch memory
    of a force call.  ``resident`` (an OrderedDict) keeps the resident systems
    across calls; without it they are released at the end."""
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
            fp = ForceParams(crit=CRIT_BH, theta=theta)
        else:
            fp = ForceParams(crit=CRIT_RELATIVE, alpha=alpha)
        r.criterion = fp.crit
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
        if keep_results:
            r.acc, r.pot, r.n_int = a_h, p_h, n_h
        r.t_done = time.perf_counter() - t0
    if not keep:
        for system, _, _ in resident.values():
            system.release()
    return reqs
