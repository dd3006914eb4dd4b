"""Request loop over the C ABI: GIBC scattering solves of different meshes,
materials and frequencies admitted into concurrent slots.

* A request is a closed mesh (V, T), a frequency, a material (eps_r, sigma), a
  plane wave (khat, epol) and observation directions; its answer is the RCS in
  those directions with the solve's iteration count and residual.
* Slots: each slot is a worker thread with its own library context on its own
  CUDA stream, so requests in different slots run on the GPU at the same time.
  A request that arrives while every slot is busy waits in the queue and is
  admitted as soon as any slot frees up (continuous admission, no batch
  boundaries).
* Resident state: the operator of a (mesh, frequency, material) key -- kernel
  spectra, near-region matrices, dense constraint factorisations, Krylov
  bases, the captured system-product graph -- stays on the device and serves
  every later request with the same key, whichever slot takes it: one cache
  for all slots, so no operator is built twice.  An operator lives in the
  context of the slot that built it; a request that uses it holds that
  context's lock (calls on one context never overlap), and a key being built
  makes the other requests for it wait instead of building it again.
* Cross-request batching: when a slot is about to solve on an operator, it
  takes every queued request of the same operator whose plane waves still
  fit in max_batch_rhs (8) together with its own, and solves all of them as
  one several-right-hand-side solve: lockstep blocks whose iterations apply
  the system product and the constraint preconditioner to all of the
  block's vectors at once (the dense factorisation is read once for them).
* Device memory: before a slot builds an operator it needs free device memory
  of at least the reserve (10% of the device by default) plus an estimate of
  the operator's size (bytes per RWG unknown: the median of the ratios
  measured on earlier builds, so one build inflated by other slots'
  concurrent allocations does not skew it); it first releases least recently
  used operators whose context is idle, then waits for other slots to
  finish; a request that cannot fit with every other slot idle and the cache
  empty fails with MemoryError.
* Latency: per request, from submit to answer (queue + build + solve + RCS);
  stats() reports p50 / p99 and the counters.

The backend is pluggable so that the admission logic can be exercised without
a GPU; LibraryBackend drives the library.
"""
import collections
import concurrent.futures
import hashlib
import threading
import time

import numpy as np


class Request:
    """One scattering solve.  khat, epol: one plane wave (3,) or several (k, 3)
    -- each is one right-hand side of the same operator; the answer's rcs is
    then (k, ndir).  params: extra sie_params fields (e.g. tol_outer)."""

    def __init__(self, V, T, freq, eps_r, sigma, khat, epol, rhat, params=None):
        self.V = np.ascontiguousarray(V, dtype=np.float64)
        self.T = np.ascontiguousarray(T, dtype=np.int32)
        self.freq, self.eps_r, self.sigma = float(freq), float(eps_r), float(sigma)
        self.single = np.ndim(khat) == 1
        self.khat = np.atleast_2d(np.asarray(khat, float))
        self.epol = np.atleast_2d(np.asarray(epol, float))
        if self.khat.shape != self.epol.shape or self.khat.shape[1] != 3:
            raise ValueError("khat and epol: (3,) or (k, 3) each, the same shape")
        self.rhat = np.atleast_2d(np.asarray(rhat, float))
        self.params = dict(params or {})
        self.ne = 3 * len(self.T) // 2

    @property
    def nrhs(self):
        return len(self.khat)

    def key(self):
        """Operators are shared by requests with the same mesh, frequency,
        material and operator parameters."""
        h = hashlib.sha1(self.V.tobytes())
        h.update(self.T.tobytes())
        h.update(repr((self.freq, self.eps_r, self.sigma, sorted(self.params.items()))).encode())
        return h.hexdigest()


class LibraryBackend:
    """A slot's binding to the library: one context on its own CUDA stream
    (created with torch, which only provides the stream and the memory query)."""

    def __init__(self, device=0):
        import torch

        from . import Context
        self.device = device
        self.stream = torch.cuda.Stream(device=device)
        self.ctx = Context(device, stream=self.stream.cuda_stream)

    def build(self, req):
        from . import Mesh, Operator, params
        mesh = Mesh(self.ctx, req.V, req.T)
        try:
            op = Operator(mesh, req.freq, req.eps_r, 1.0, req.sigma, params(**req.params))
        except Exception:
            mesh.close()
            raise
        return (mesh, op)

    def run(self, handle, req):
        return self.run_batch(handle, [req])[0]

    def run_batch(self, handle, reqs):
        """All plane waves of reqs (requests of one operator) as one
        several-right-hand-side solve: lockstep blocks of 8, so the product
        and the preconditioner of an iteration serve every request of the
        block together."""
        _, op = handle
        n = op.mesh.ne + op.mesh.nt
        k = sum(r.nrhs for r in reqs)
        B = np.zeros((k, n), np.complex128)
        i = 0
        for r in reqs:
            for kh, ep in zip(r.khat, r.epol):
                op.rhs_planewave(kh, ep, out=B[i])
                i += 1
        X, it, rr = op.solve(B if k > 1 else B[0], nrhs=k, check=False)
        X = X.reshape(k, n)
        outs, i = [], 0
        for r in reqs:
            rcs = np.stack([op.rcs(X[i + q], r.rhat) for q in range(r.nrhs)])
            its = [int(v) for v in it[i:i + r.nrhs]]
            res = [float(v) for v in rr[i:i + r.nrhs]]
            i += r.nrhs
            if r.single:
                outs.append({"rcs": rcs[0], "iters": its[0], "relres": res[0], "batch_rhs": k})
            else:
                outs.append({"rcs": rcs, "iters": its, "relres": res, "batch_rhs": k})
        return outs

    def release(self, handle):
        mesh, op = handle
        op.close()
        mesh.close()

    def memory(self):
        """(free, total) device bytes."""
        import torch
        return torch.cuda.mem_get_info(self.device)

    def close(self):
        self.ctx.close()


class Server:
    """Slots, queue, one shared operator cache and memory admission (module docstring)."""

    def __init__(self, slots=2, backend_factory=None, reserve_fraction=0.10, bytes_per_unknown=128 * 1024,
                 wait_s=0.05, max_batch_rhs=8):
        self.backend_factory = backend_factory or (lambda slot: LibraryBackend(0))
        self.reserve_fraction = reserve_fraction
        self.bytes_per_unknown = float(bytes_per_unknown)   # estimate until builds are measured
        self.wait_s = wait_s
        self.max_batch_rhs = int(max_batch_rhs)
        self._cv = threading.Condition()
        self._queue = collections.deque()
        self._busy = 0
        self._closed = False
        self._lat = []
        self._samples = []            # measured operator bytes per RWG unknown
        self.counters = collections.Counter()
        self._build_lock = threading.Lock()   # one operator set-up at a time
        self._backends = [None] * slots
        self._cache = collections.OrderedDict()   # key -> (handle, owner slot), least recently used first
        self._building = set()                    # keys being built
        self._ctx_locks = [threading.Lock() for _ in range(slots)]  # held while a slot's context is in use
        self._init_errors = []
        self._threads = [threading.Thread(target=self._loop, args=(s,), daemon=True) for s in range(slots)]
        self._ready = threading.Barrier(slots + 1)
        for t in self._threads:
            t.start()
        self._ready.wait()
        if self._init_errors:
            self.close()
            raise self._init_errors[0]

    # ---------------------------------------------------------------- public
    def submit(self, req):
        fut = concurrent.futures.Future()
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            self._queue.append((req, fut, time.perf_counter()))
            self._cv.notify_all()
        return fut

    def stats(self):
        with self._cv:
            lat = np.array(self._lat)
            out = dict(self.counters)
        out["completed"] = int(len(lat))
        if len(lat):
            out["p50_s"] = float(np.percentile(lat, 50))
            out["p99_s"] = float(np.percentile(lat, 99))
        out["bytes_per_unknown"] = self._estimate_per_unknown()
        return out

    def close(self):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()
        # every slot has stopped: release what the cache still holds, then the contexts
        for key, (h, owner) in list(self._cache.items()):
            self._backends[owner].release(h)
        self._cache.clear()
        for b in self._backends:
            if b is not None:
                b.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- slots
    def _estimate_per_unknown(self):
        with self._cv:
            return float(np.median(self._samples)) if self._samples else self.bytes_per_unknown

    def _loop(self, slot):
        try:
            self._backends[slot] = self.backend_factory(slot)  # its context lives in this thread's slot
        except BaseException as e:  # reported by the constructor
            self._init_errors.append(e)
        self._ready.wait()
        if self._backends[slot] is None:
            return
        while True:
            with self._cv:
                while not self._queue and not self._closed:
                    self._cv.wait()
                if not self._queue:
                    break
                req, fut, t0 = self._queue.popleft()
                self._busy += 1
            batch = [(req, fut, t0)]
            try:
                if fut.set_running_or_notify_cancel():
                    self._serve(slot, batch)
            except BaseException as e:
                for _, f, _ in batch:
                    if not f.done():
                        f.set_exception(e)
            finally:
                with self._cv:
                    self._busy -= 1
                    self._cv.notify_all()

    def _take_same_key(self, key, batch):
        """Cross-request batching: move queued requests of the operator `key`
        into batch while its right-hand sides fit in max_batch_rhs (called
        with self._cv held)."""
        have = sum(r.nrhs for r, _, _ in batch)
        keep = collections.deque()
        while self._queue:
            item = self._queue.popleft()
            r, f, _ = item
            if r.key() == key and have + r.nrhs <= self.max_batch_rhs:
                if f.set_running_or_notify_cancel():
                    batch.append(item)
                    have += r.nrhs
                    self.counters["batched"] += 1
            else:
                keep.append(item)
        self._queue = keep

    def _finish(self, batch, outs, slot):
        now = time.perf_counter()
        for (_, f, t0), out in zip(batch, outs):
            out["slot"] = slot
            with self._cv:
                self._lat.append(now - t0)
            f.set_result(out)

    def _run(self, backend, handle, batch):
        reqs = [r for r, _, _ in batch]
        if len(reqs) > 1 and hasattr(backend, "run_batch"):
            return backend.run_batch(handle, reqs)
        return [backend.run(handle, r) for r in reqs]

    def _count(self, name):
        with self._cv:
            self.counters[name] += 1

    def _serve(self, slot, batch):
        """Run the batch (its first request, plus queued requests of the same
        operator taken just before the solve) on the cached operator of the
        key (built here, in this slot's context, if no slot has it)."""
        req = batch[0][0]
        key = req.key()
        while True:
            with self._cv:
                while key in self._building:
                    self._cv.wait()
                entry = self._cache.get(key)
                if entry is None:
                    self._building.add(key)
            if entry is None:
                break
            handle, owner = entry
            with self._ctx_locks[owner]:
                with self._cv:
                    still = self._cache.get(key) is entry
                    if still:
                        self._cache.move_to_end(key)
                        self.counters["reused"] += 1
                        self._take_same_key(key, batch)
                if still:
                    self._finish(batch, self._run(self._backends[owner], handle, batch), slot)
                    return
            # evicted between the look-up and the lock: look again
        try:
            with self._ctx_locks[slot]:
                handle = self._build(slot, req)
                with self._cv:
                    self._cache[key] = (handle, slot)
                    self.counters["built"] += 1
                    self._take_same_key(key, batch)
                self._finish(batch, self._run(self._backends[slot], handle, batch), slot)
        finally:
            with self._cv:
                self._building.discard(key)
                self._cv.notify_all()

    def _evict_one(self, slot):
        """Release the least recently used operator whose context is idle (this
        slot's own, whose lock the caller holds, or an idle slot's).  False
        when nothing could be released."""
        with self._cv:
            order = list(self._cache.items())
        for key, entry in order:
            handle, owner = entry
            if owner != slot and not self._ctx_locks[owner].acquire(blocking=False):
                continue  # that context is serving a request
            try:
                with self._cv:
                    if self._cache.get(key) is not entry:
                        continue
                    del self._cache[key]
                self._backends[owner].release(handle)
                self._count("evicted")
                return True
            finally:
                if owner != slot:
                    self._ctx_locks[owner].release()
        return False

    def _build(self, slot, req):
        """An operator for req in this slot's context, once memory allows."""
        backend = self._backends[slot]
        need = self._estimate_per_unknown() * req.ne
        while True:
            free, total = backend.memory()
            if free - need >= self.reserve_fraction * total:
                break
            if self._evict_one(slot):
                continue
            with self._cv:
                if self._busy <= 1:  # no other request in flight will free memory
                    self.counters["rejected"] += 1
                    raise MemoryError(f"operator for {req.ne} unknowns (~{need / 2**30:.1f} GiB) does not fit "
                                      f"in the device-memory budget")
                self._cv.wait(self.wait_s)
        with self._build_lock:
            free0 = backend.memory()[0]
            handle = backend.build(req)
            used = free0 - backend.memory()[0]
        if used > 0:
            with self._cv:
                self._samples.append(used / req.ne)
        return handle
