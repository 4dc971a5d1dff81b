"""Continuous-batching solve server over libmfs.

Requests (a coupled block system plus a right-hand side) arrive at any time;
a request is admitted when a slot is free and its device memory fits the HBM
budget, and new requests keep being admitted as slots and memory free up.  A
request may reuse a resident hierarchy of the same system (a clone: no
setup, only a new workspace) or bring a new matrix (a full setup).  Resident
hierarchies are evicted least-recently-used when the budget is short.

Solves run in one of two modes.  Per request (fused=False): every admitted
request is solved on its own handle and CUDA stream by its worker thread, so
the requests' kernels overlap on the GPU.  Fused (fused=True): workers only
admit and set up; one solver thread takes every request that is ready when
it is free and solves them together with the fused batch executor
(mfs_solve_batch, nthreads = 0): the live requests' V-cycles, matvecs and
Arnoldi passes run as shared multi-system launches, and requests that become
ready meanwhile join the next batch.  Either way every result is the one a
solo solve of that request gives, which the serving test checks.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

from . import mfs

BYTES_PER_DOF_ESTIMATE = 3200  # before a system's first setup (measured after it)
# device memory a setup holds beyond its final footprint (input copy, GPU
# setup products, candidate layouts), as a multiple of the final shared bytes
SETUP_TRANSIENT_FACTOR = 2


class Request:
    def __init__(self, rid, key, system, rhs, reuse):
        self.rid, self.key, self.system, self.rhs, self.reuse = rid, key, system, rhs, reuse
        self.t_arrive = time.perf_counter()
        self.t_admit = self.t_start = self.t_setup = self.t_done = None
        self.x = None
        self.info = None
        self.rc = None
        self.error = None
        self.reserved = 0
        self.setup_done_here = False
        self.event = threading.Event()

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.t_arrive


class Server:
    """hbm_budget: bytes of device memory the server may hold (resident
    hierarchies + running requests); workers: requests in flight at once."""

    def __init__(self, hbm_budget, workers=8, tol=1e-8, keep_resident=True, max_setups=4, fused=False,
                 max_inflight=None, max_batch=64, **solver_kw):
        """max_setups: setups (new matrices) in flight at once, which bounds
        their transient device memory.  fused: solve the ready requests
        together (see the module docstring); max_inflight: admitted requests
        at once (default: workers, or 8 x workers when fused); max_batch:
        requests per fused batch."""
        self.budget = int(hbm_budget)
        self.fused = fused
        self.max_inflight = max_inflight or (8 * workers if fused else workers)
        self.max_batch = max_batch
        self.ready = collections.deque()  # fused: (request, handle, base) set up and waiting for a batch
        self.batches = []                 # fused: sizes of the batches solved
        self.tol = tol
        self.kw = solver_kw
        self.keep_resident = keep_resident
        self.cv = threading.Condition()
        self.pending = collections.deque()
        self.resident = collections.OrderedDict()  # key -> [Solver, shared_bytes, own_bytes, users]
        self.footprint = {}  # key -> (shared bytes, workspace bytes) measured
        self.used = 0
        self.peak_used = 0
        self.running = 0
        self.peak_running = 0
        self.done = []
        self.stop = False
        self.next_id = 0
        self.setups_running = 0
        self.max_setups = max_setups
        self.threads = [threading.Thread(target=self._work, daemon=True) for _ in range(workers)]
        if fused:
            self.threads.append(threading.Thread(target=self._solve_loop, daemon=True))
        for t in self.threads:
            t.start()

    # ------------------------------------------------------------------ API
    def submit(self, key, system, rhs, reuse=True):
        with self.cv:
            r = Request(self.next_id, key, system, rhs, reuse)
            self.next_id += 1
            self.pending.append(r)
            self.cv.notify_all()
        return r

    def drain(self, timeout=None):
        """Wait until every submitted request has finished."""
        t0 = time.perf_counter()
        with self.cv:
            while self.pending or self.running:
                left = None if timeout is None else timeout - (time.perf_counter() - t0)
                if left is not None and left <= 0:
                    raise TimeoutError("serving drain timed out")
                self.cv.wait(left if left is not None else 1.0)

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        for t in self.threads:
            t.join()
        for entry in self.resident.values():
            entry[0].close()
        self.resident.clear()

    def stats(self):
        ran = [r for r in self.done if r.t_done is not None and r.t_start is not None]
        lat = np.array([r.latency for r in self.done if r.latency is not None])
        solve = np.array([r.t_done - r.t_start for r in ran]) if ran else np.zeros(1)
        setup = np.array([r.t_start - r.t_admit for r in ran if r.setup_done_here])
        errors = collections.Counter(r.error for r in self.done if r.error)
        t0 = min(r.t_arrive for r in self.done)
        t1 = max(r.t_done for r in self.done)
        ok = sum(1 for r in self.done if r.rc == mfs.OK)
        return {"requests": len(self.done), "converged": ok,
                "p50_latency_ms": float(np.percentile(lat, 50) * 1e3), "p99_latency_ms": float(np.percentile(lat, 99) * 1e3),
                "p50_solve_ms": float(np.percentile(solve, 50) * 1e3), "p99_solve_ms": float(np.percentile(solve, 99) * 1e3),
                "mean_setup_ms": float(setup.mean() * 1e3) if len(setup) else 0.0,
                "solves_per_s": ok / (t1 - t0), "peak_hbm_bytes": self.peak_used, "peak_in_flight": self.peak_running,
                "setups": int(sum(1 for r in self.done if r.setup_done_here)),
                "solve_mode": "fused batches" if self.fused else "one handle and stream per request",
                "fused_batches": len(self.batches),
                "mean_batch": float(np.mean(self.batches)) if self.batches else None,
                "failed": int(sum(errors.values())), "errors": dict(errors.most_common(3))}

    # ------------------------------------------------------------- internals
    def _estimate(self, r, transient=True):
        """Bytes to reserve: the workspace for a clone; for a setup also the
        hierarchy and (transient=True) the setup's transient memory."""
        shared, own = self.footprint.get(r.key, (None, None))
        if shared is None:
            n = r.system.ndofs
            shared, own = BYTES_PER_DOF_ESTIMATE * n // 2, BYTES_PER_DOF_ESTIMATE * n // 2
        if r.reuse and r.key in self.resident:
            return own
        return (1 + (SETUP_TRANSIENT_FACTOR if transient else 0)) * shared + own

    def _needs_setup(self, r):
        return not (r.reuse and r.key in self.resident)

    def _evict_for(self, need):
        """Drop idle resident hierarchies (LRU first) until `need` bytes fit."""
        for key in list(self.resident.keys()):
            if self.used + need <= self.budget:
                return
            sv, shared, own, users = self.resident[key]
            if users:
                continue
            del self.resident[key]
            self.used -= shared + own
            sv.close()

    def _take(self):
        """Admit the oldest pending request that fits (called with the lock held)."""
        if not self.pending or self.running >= self.max_inflight:
            return None
        r = self.pending[0]
        if self._needs_setup(r) and self.setups_running >= self.max_setups:
            return None
        need = self._estimate(r)
        if self.used + need > self.budget:
            self._evict_for(need)
        if self.used + need > self.budget and self.running == 0:
            # alone on the device: the transient reserve is not needed to fit,
            # and a system never set up before is tried whatever its estimate
            need = self._estimate(r, transient=False)
            self._evict_for(need)
            if r.key not in self.footprint:
                need = min(need, max(0, self.budget - self.used))
        if self.used + need > self.budget:
            if self.running == 0 and need > self.budget:
                self.pending.popleft()
                r.error = "request larger than the HBM budget"
                r.rc = mfs.ERR_OOM
                r.t_done = time.perf_counter()
                self.done.append(r)
                r.event.set()
            return None
        self.pending.popleft()
        r.reserved = need
        self.used += need
        self.peak_used = max(self.peak_used, self.used)
        self.running += 1
        self.peak_running = max(self.peak_running, self.running)
        r.t_admit = time.perf_counter()
        if r.reuse and r.key in self.resident:
            self.resident.move_to_end(r.key)
            self.resident[r.key][3] += 1
        else:
            self.setups_running += 1
        return r

    def _work(self):
        while True:
            with self.cv:
                r = None
                while not self.stop:
                    r = self._take()
                    if r is not None:
                        break
                    self.cv.wait(0.05)
                if r is None:
                    return
                base = self.resident[r.key][0] if (r.reuse and r.key in self.resident) else None
            sv = None
            try:
                if base is not None:
                    sv = base.clone()
                else:
                    try:
                        sv = mfs.Solver(r.system, **self.kw)
                    finally:
                        with self.cv:
                            self.setups_running -= 1
                            self.cv.notify_all()
                    r.setup_done_here = True
                if self.fused:
                    with self.cv:
                        self.ready.append((r, sv, base))
                        self.cv.notify_all()
                    continue
                r.t_start = time.perf_counter()
                x = np.zeros(r.system.ndofs)
                _, r.info, r.rc = sv.solve(r.rhs, x, tol=self.tol)
                r.x = x
            except mfs.MfsError as e:
                r.rc, r.error = e.code, str(e)
            r.t_done = time.perf_counter()
            self._finish(r, sv, base)

    def _solve_loop(self):
        """Fused mode: solve every ready request together, batch after batch."""
        while True:
            with self.cv:
                while not self.ready and not self.stop:
                    self.cv.wait(0.05)
                if not self.ready and self.stop:
                    return
                batch = []
                while self.ready and len(batch) < self.max_batch:
                    batch.append(self.ready.popleft())
            t0 = time.perf_counter()
            for r, _, _ in batch:
                r.t_start = t0
            xs = [np.zeros(r.system.ndofs) for r, _, _ in batch]
            try:
                _, infos, status = mfs.solve_batch([sv for _, sv, _ in batch], [r.rhs for r, _, _ in batch], xs,
                                                   tol=self.tol, nthreads=0, check=False)
                for (r, _, _), x, info, st in zip(batch, xs, infos, status):
                    r.x, r.info, r.rc = x, info, st
            except mfs.MfsError as e:
                for r, _, _ in batch:
                    r.rc, r.error = e.code, str(e)
            t1 = time.perf_counter()
            self.batches.append(len(batch))
            for r, sv, base in batch:
                r.t_done = t1
                self._finish(r, sv, base)

    def _finish(self, r, sv, base):
        """Release a finished request's reservation, keep a new hierarchy
        resident when it fits, release the handle otherwise."""
        keep = False
        with self.cv:
            self.used -= r.reserved
            if sv is not None:
                shared, own = sv.device_bytes(True), sv.device_bytes(False)
                if r.setup_done_here:
                    self.footprint[r.key] = (shared, own)
                    if self.keep_resident and r.key not in self.resident and self.used + shared + own <= self.budget:
                        self.resident[r.key] = [sv, shared, own, 0]
                        self.used += shared + own
                        keep = True
            if base is not None and r.key in self.resident:
                self.resident[r.key][3] -= 1
        # release a handle that is not kept before the request counts as
        # finished, so that drain() never returns with device work in flight
        if sv is not None and not keep:
            sv.close()
        with self.cv:
            self.running -= 1
            self.done.append(r)
            self.cv.notify_all()
        r.event.set()
