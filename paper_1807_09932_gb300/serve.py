"""Continuous-batching server for population-evaluation requests from many concurrent EBIC runs.

Each EBIC run owns one matrix and an elite archive. It sends one request per generation (its
population) and waits for that request's counts and fitness before it breeds the next one.
The server:
  * admits runs by device-memory footprint (rank matrix + population, bitmap and archive
    buffers). A run that does not fit waits until a finished run frees its memory;
  * keeps every admitted run's rank matrix and archive resident on the device;
  * batches the requests that have arrived into one launch. It keeps up to `max_inflight`
    batches on the GPU (one stream each), so a request that arrives while others run is
    launched as soon as a slot frees. Its upload overlaps the running batch, and its kernels
    start as the running batch drains;
  * records per-request latency (completion minus arrival, host clock), p50/p99 and
    throughput in candidate-row evals/s.

The device work goes through a backend: ``GpuBackend`` (the C ABI: ebic_batch_run in a CUDA
graph; a run with a pair table gets its fitness against its resident archive inside the batch,
the others through ebic_fitness per request; a batch of a single pair-table request goes through
ebic_eval_fitness instead, which launches less) or, in tests, a fake one. ``plain_serve`` is the comparison point: the same arrivals served one request at a time
with the per-population call (ebic_eval_fitness), in arrival order.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    run_id: int
    cols: np.ndarray          # uint16 CSR columns
    offsets: np.ndarray       # uint32 CSR offsets
    t_arrival: float
    flags: int = 0
    rid: int = -1
    t_launch: float = float("nan")
    t_done: float = float("nan")
    counts: np.ndarray | None = None
    fitness: np.ndarray | None = None

    @property
    def n_cand(self):
        return len(self.offsets) - 1

    @property
    def latency(self):
        return self.t_done - self.t_arrival


@dataclasses.dataclass
class RunSpec:
    run_id: int
    X: np.ndarray             # float32 [rows, cols]
    max_cand: int
    max_len: int = 64
    exclude_missing: bool = True
    archive_cols: np.ndarray | None = None      # CSR of the initial archive (may be empty)
    archive_offsets: np.ndarray | None = None


def percentile(values, q):
    if not values:
        return float("nan")
    v = sorted(values)
    k = (len(v) - 1) * q / 100.0
    lo = int(np.floor(k))
    hi = min(lo + 1, len(v) - 1)
    return v[lo] + (v[hi] - v[lo]) * (k - lo)


class Server:
    """Batches of at most `max_batch` requests, up to `max_inflight` of them on the GPU at once.
    On the 32-run methylation-to-expression mix, 16 and 3 gave the highest saturated throughput
    of 4-32 x 2-4: smaller batches let the next batch's packing overlap the running ones."""

    def __init__(self, backend, hbm_budget, max_batch=16, max_inflight=3):
        self.be = backend
        self.budget = hbm_budget
        self.used = 0
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.open = {}                      # run_id -> footprint
        self.waiting_runs = collections.deque()
        self.queue = collections.deque()    # arrived requests, FIFO
        self.busy_runs = set()              # runs with a request in flight
        self.inflight = []                  # (token, [requests])
        self.done = []
        self._next_rid = 0
        self.batches = 0

    # ---- runs ---------------------------------------------------------------------------------
    def add_run(self, spec: RunSpec):
        need = self.be.footprint(spec)
        if need > self.budget:
            raise ValueError(f"run {spec.run_id} needs {need} bytes, more than the budget")
        if self.used + need <= self.budget and not self.waiting_runs:
            self._open(spec, need)
            return True
        self.waiting_runs.append((spec, need))
        return False

    def _open(self, spec, need):
        self.be.open_run(spec)
        self.open[spec.run_id] = need
        self.used += need

    def finish_run(self, run_id):
        if run_id in self.busy_runs:
            raise RuntimeError("run has a request in flight")
        need = self.open.pop(run_id)
        self.be.close_run(run_id)
        self.used -= need
        while self.waiting_runs and self.used + self.waiting_runs[0][1] <= self.budget:
            spec, n = self.waiting_runs.popleft()
            self._open(spec, n)

    def is_open(self, run_id):
        return run_id in self.open

    # ---- requests -----------------------------------------------------------------------------
    def submit(self, req: Request):
        req.rid = self._next_rid
        self._next_rid += 1
        self.queue.append(req)
        return req.rid

    def pump(self):
        """Collect finished batches, then launch the waiting requests if a slot is free.
        Returns the requests completed in this call."""
        finished = []
        still = []
        for token, reqs in self.inflight:
            if self.be.done(token):
                self.be.collect(token, reqs)
                t = self.be.now()
                for r in reqs:
                    r.t_done = t
                    self.busy_runs.discard(r.run_id)
                finished.extend(reqs)
            else:
                still.append((token, reqs))
        self.inflight = still
        self.done.extend(finished)
        while len(self.inflight) < self.max_inflight and self.queue:
            batch, rest = [], collections.deque()
            seen = set()
            while self.queue and len(batch) < self.max_batch:
                r = self.queue.popleft()
                if (r.run_id in self.open and r.run_id not in self.busy_runs
                        and r.run_id not in seen):
                    batch.append(r)
                    seen.add(r.run_id)
                else:
                    rest.append(r)
            rest.extend(self.queue)
            self.queue = rest
            if not batch:
                break
            t = self.be.now()
            for r in batch:
                r.t_launch = t
                self.busy_runs.add(r.run_id)
            try:
                token = self.be.launch(batch)
            except Exception:
                # the batch never ran: its runs may send again, and the caller sees the error
                for r in batch:
                    self.busy_runs.discard(r.run_id)
                raise
            self.inflight.append((token, batch))
            self.batches += 1
        return finished

    def idle(self):
        return not self.queue and not self.inflight

    # ---- statistics ---------------------------------------------------------------------------
    def stats(self, t0, t1, rows_of):
        lat = [r.latency for r in self.done]
        evals = sum(r.n_cand * rows_of[r.run_id] for r in self.done)
        return {"requests": len(self.done), "batches": self.batches,
                "p50_ms": 1000 * percentile(lat, 50), "p99_ms": 1000 * percentile(lat, 99),
                "mean_ms": 1000 * (sum(lat) / len(lat)) if lat else float("nan"),
                "evals_per_s": evals / (t1 - t0) if t1 > t0 else float("nan"),
                "wall_s": t1 - t0}


def drive(server, arrivals, rows_of, on_done=None, clock=None, spin=None):
    """Open-loop driver: submit each request when its arrival time has passed, pump until all
    are done. ``arrivals`` is a list of Requests sorted by t_arrival (relative seconds).
    Returns the server's stats over the whole run."""
    be = server.be
    clock = clock or be.now
    t0 = clock()
    for r in arrivals:
        r.t_arrival += t0
    i = 0
    while i < len(arrivals) or not server.idle():
        now = clock()
        while i < len(arrivals) and arrivals[i].t_arrival <= now:
            server.submit(arrivals[i])
            i += 1
        for r in server.pump():
            if on_done:
                on_done(r)
        if spin:
            spin(arrivals[i].t_arrival if i < len(arrivals) else None)
    return server.stats(t0, clock(), rows_of)


# ---- GPU backend ------------------------------------------------------------------------------

class GpuBackend:
    """Resident rank matrices, per-run device buffers and archives; batched graph launches."""

    def __init__(self, max_batch=16, max_inflight=3, device=0, pair_budget=0):
        """pair_budget: a run whose matrix's pair table takes at most this many bytes gets one
        when it opens (its requests then run on the pair-table passes); 0: none."""
        import torch

        from . import ebic
        self.torch = torch
        self.ebic = ebic
        self.pair_budget = int(pair_budget)
        self.dev = torch.device("cuda", device)
        self.runs = {}
        # each slot stages a whole batch: every request's lists packed into one pinned buffer and
        # sent with one copy, every request's counts and fitness brought back with one copy
        self.slots = [dict(stream=torch.cuda.Stream(self.dev), batch=ebic.ebic_batch_create(max_batch),
                           busy=False, event=torch.cuda.Event(), hin=None, din=None, hout=None,
                           dout=None) for _ in range(max_inflight)]
        # the plain arm's pinned lists and outputs, read and written in place by the fused call
        self.plain_io = dict(hin=None, hout=None)
        # a batch's request table as a numpy record array laid out like ebic_eval_request
        self._req_dtype = np.dtype(ebic.EbicEvalRequest)
        self._req_ptr = ctypes.POINTER(ebic.EbicEvalRequest)

    _ALIGN = 256  # every staged array starts on this boundary

    @classmethod
    def _layout(cls, reqs):
        """Byte offsets of each request's columns and offsets in the input staging, and of its
        counts (uint32) and fitness (uint64) in the output staging; the two sizes."""
        a = cls._ALIGN

        def up(x):
            return (x + a - 1) // a * a

        ins, outs, i_off, o_off = [], [], 0, 0
        for r in reqs:
            n = r.n_cand
            oc = i_off
            i_off = up(i_off + 2 * int(r.offsets[-1]))
            oo = i_off
            i_off = up(i_off + 4 * (n + 1))
            ins.append((oc, oo))
            cnt = o_off
            o_off = up(o_off + 4 * n)
            fit = o_off
            o_off = up(o_off + 8 * n)
            outs.append((cnt, fit))
        return ins, outs, max(i_off, a), max(o_off, a)

    def _pinned(self, nbytes):
        t = self.torch.empty(nbytes, dtype=self.torch.uint8).pin_memory()
        return t, t.numpy()

    def _staging(self, slot, in_bytes, out_bytes):
        """The slot's staging buffers, grown (never shrunk) to the sizes asked for."""
        torch = self.torch
        if slot["hin"] is None or slot["hin"][0].numel() < in_bytes:
            slot["hin"] = self._pinned(2 * in_bytes)
            slot["din"] = torch.empty(2 * in_bytes, dtype=torch.uint8, device=self.dev)
        if slot["hout"] is None or slot["hout"][0].numel() < out_bytes:
            slot["hout"] = self._pinned(2 * out_bytes)
            slot["dout"] = torch.empty(2 * out_bytes, dtype=torch.uint8, device=self.dev)

    @staticmethod
    def _pack(hin_np, reqs, ins):
        for r, (oc, oo) in zip(reqs, ins):
            c = np.ascontiguousarray(r.cols, dtype=np.uint16).view(np.uint8)
            o = np.ascontiguousarray(r.offsets, dtype=np.uint32).view(np.uint8)
            hin_np[oc:oc + c.size] = c
            hin_np[oo:oo + o.size] = o

    def close(self):
        for s in self.slots:
            s["stream"].synchronize()
            self.ebic.ebic_batch_free(s["batch"])
        self.slots = []
        for rid in list(self.runs):
            self.close_run(rid)

    @staticmethod
    def pair_bytes(spec: RunSpec):
        """Device bytes of the run matrix's pair table (C*C rows of W rounded up to 512 words,
        and one all-ones row of 128 words)."""
        R, C = spec.X.shape
        W = (R + 31) // 32
        return C * C * ((W + 511) // 512 * 512) * 4 + 512

    def footprint(self, spec: RunSpec):
        R, C = spec.X.shape
        W = (R + 31) // 32
        rank_bytes = R * C * (1 if C <= 127 else 2) * 1.02 + 4096
        pb = self.pair_bytes(spec)
        if 0 < pb <= self.pair_budget:
            rank_bytes += pb
        k = 0 if spec.archive_offsets is None else len(spec.archive_offsets) - 1
        # row bitmaps for the fitness call when the run has no pair table; the archive's lists
        # and bitmaps (the requests' lists and outputs live in the shared batch staging)
        per_run = (0 if 0 < pb <= self.pair_budget else spec.max_cand * W * 4) \
            + k * (W * 4 + 64 * 2 + 4) + 4096
        return int(rank_bytes + per_run)

    def now(self):
        return time.perf_counter()

    def open_run(self, spec: RunSpec):
        torch = self.torch
        m = self.ebic.Matrix(spec.X, exclude_missing=spec.exclude_missing)
        pairs = 0 < self.pair_bytes(spec) <= self.pair_budget
        if pairs:
            m.build_pairs(max_bytes=self.pair_budget)
        W = m.words
        P = spec.max_cand
        # the rank-code pass writes row bitmaps for the fitness call; pair-table runs need none
        run = dict(m=m, P=P, W=W, rows=spec.X.shape[0], pairs=pairs,
                   bitmaps=None if pairs else torch.empty((P, W), dtype=torch.int32,
                                                          device=self.dev))
        # resident archive: its members scored once on this matrix
        if spec.archive_offsets is not None and len(spec.archive_offsets) > 1:
            ac, ao = spec.archive_cols, spec.archive_offsets
            _, abm = self.ebic.eval_population(m, ac, ao)
            run["acols"] = torch.from_numpy(np.ascontiguousarray(ac).view(np.int16)).to(self.dev)
            run["aoffs"] = torch.from_numpy(np.ascontiguousarray(ao).view(np.int32)).to(self.dev)
            run["abm"] = torch.from_numpy(abm.view(np.int32)).to(self.dev)
            run["K"] = len(ao) - 1
        else:
            run["acols"] = torch.zeros(1, dtype=torch.int16, device=self.dev)
            run["aoffs"] = torch.zeros(1, dtype=torch.int32, device=self.dev)
            run["abm"] = torch.zeros((1, W), dtype=torch.int32, device=self.dev)
            run["K"] = 0
        # the run's fixed fields of a batch request, as addresses (0: none)
        k = run["K"]
        run["req"] = (m.handle.value, run["bitmaps"].data_ptr() if not pairs else 0,
                      run["acols"].data_ptr() if pairs and k else 0,
                      run["aoffs"].data_ptr() if pairs and k else 0,
                      run["abm"].data_ptr() if pairs and k else 0, k if pairs else 0)
        self.runs[spec.run_id] = run

    def close_run(self, run_id):
        run = self.runs.pop(run_id)
        self.torch.cuda.synchronize(self.dev)
        run["m"].close()

    def launch(self, reqs):
        slot = next(s for s in self.slots if not s["busy"])
        slot["busy"] = True
        try:
            return self._launch(slot, reqs)
        except Exception:
            # nothing of this batch is waited for: let the stream finish what was queued, then
            # give the slot back
            slot["stream"].synchronize()
            slot["busy"] = False
            raise

    def _launch(self, slot, reqs):
        ebic = self.ebic
        st = slot["stream"]
        sp = st.cuda_stream
        ins, outs, in_bytes, out_bytes = self._layout(reqs)
        self._staging(slot, in_bytes, out_bytes)
        self._pack(slot["hin"][1], reqs, ins)
        hin = slot["hin"][0].data_ptr()
        din, dout = slot["din"].data_ptr(), slot["dout"].data_ptr()
        if len(reqs) == 1 and self.runs[reqs[0].run_id]["pairs"]:
            # a batch of one: the per-population fused call (three launches) costs less than the
            # batch graph's fixed launches, with the same results; its kernels read the pinned
            # lists in place, so nothing is uploaded
            r = reqs[0]
            run = self.runs[r.run_id]
            (oc, oo), (cnt, fit) = ins[0], outs[0]
            rc = ebic.ebic_eval_fitness(run["m"].handle, hin + oc, hin + oo, r.n_cand, r.flags,
                                        run["acols"], run["aoffs"], run["abm"], run["K"],
                                        dout + cnt, None, dout + fit, None, sp)
            if rc:
                raise ebic.EbicError(rc, "ebic_eval_fitness")
        else:
            # the batch's request table, filled column by column (a pair-table run gets its
            # fitness inside the batch; the others write bitmaps for the fitness call)
            n = len(reqs)
            req = np.zeros(n, dtype=self._req_dtype)
            fixed = np.array([self.runs[r.run_id]["req"] for r in reqs], dtype=np.uint64)
            place = np.array([io + oo_ for io, oo_ in zip(ins, outs)], dtype=np.uint64)
            pairs = np.array([self.runs[r.run_id]["pairs"] for r in reqs], dtype=bool)
            req["m"] = fixed[:, 0]
            req["cols"] = din + place[:, 0]
            req["offsets"] = din + place[:, 1]
            req["n_cand"] = [r.n_cand for r in reqs]
            req["flags"] = [r.flags for r in reqs]
            req["counts"] = dout + place[:, 2]
            req["bitmaps"] = fixed[:, 1]
            req["arch_cols"] = fixed[:, 2]
            req["arch_offsets"] = fixed[:, 3]
            req["arch_bitmaps"] = fixed[:, 4]
            req["n_arch"] = fixed[:, 5]
            req["fitness"] = np.where(pairs, dout + place[:, 3], 0)
            rc = ebic.ebic_copy_async(din, hin, in_bytes, sp)  # every list in one copy
            if rc:
                raise ebic.EbicError(rc, "ebic_copy_async")
            rc = ebic.ebic_batch_run(slot["batch"], req.ctypes.data_as(self._req_ptr), n, sp)
            if rc:
                raise ebic.EbicError(rc, "ebic_batch_run")
            for r, (oc, oo), (cnt, fit) in zip(reqs, ins, outs):
                run = self.runs[r.run_id]
                if not run["pairs"]:  # the rank-code pass wrote bitmaps: the fitness call
                    rc = ebic.ebic_fitness(run["m"].handle, din + oc, din + oo, r.n_cand,
                                           dout + cnt, run["bitmaps"], run["acols"],
                                           run["aoffs"], run["abm"], run["K"], 0, dout + fit,
                                           None, sp)
                    if rc:
                        raise ebic.EbicError(rc, "ebic_fitness")
        # every request's counts and fitness back in one copy
        rc = ebic.ebic_copy_async(slot["hout"][0].data_ptr(), dout, out_bytes, sp)
        if rc:
            raise ebic.EbicError(rc, "ebic_copy_async")
        slot["event"].record(st)
        return dict(slot=slot, outs=outs)

    def done(self, token):
        return token["slot"]["event"].query()

    def collect(self, token, reqs):
        slot = token["slot"]
        slot["event"].synchronize()
        hout = slot["hout"][1]
        for r, (cnt, fit) in zip(reqs, token["outs"]):
            n = r.n_cand
            r.counts = hout[cnt:cnt + 4 * n].view(np.uint32).copy()
            r.fitness = hout[fit:fit + 8 * n].view(np.uint64).copy()
        slot["busy"] = False

    # the comparison point: one request at a time, one per-population call (ebic_eval_fitness);
    # its lists and outputs are pinned host memory that the call's kernels read and write in
    # place (a call with host outputs returns once they are written)
    def plain(self, r, stream):
        ebic = self.ebic
        run = self.runs[r.run_id]
        ins, outs, in_bytes, out_bytes = self._layout([r])
        io = self.plain_io
        if io["hin"] is None or io["hin"][0].numel() < in_bytes:
            io["hin"] = self._pinned(2 * in_bytes)
        if io["hout"] is None or io["hout"][0].numel() < out_bytes:
            io["hout"] = self._pinned(2 * out_bytes)
        self._pack(io["hin"][1], [r], ins)
        hin, hout = io["hin"][0].data_ptr(), io["hout"][0].data_ptr()
        (oc, oo), (cnt, fit) = ins[0], outs[0]
        rc = ebic.ebic_eval_fitness(run["m"].handle, hin + oc, hin + oo, r.n_cand, r.flags,
                                    run["acols"], run["aoffs"], run["abm"], run["K"],
                                    hout + cnt, None, hout + fit, None, stream.cuda_stream)
        if rc:
            raise ebic.EbicError(rc, "ebic_eval_fitness")
        h = io["hout"][1]
        r.counts = h[cnt:cnt + 4 * r.n_cand].view(np.uint32).copy()
        r.fitness = h[fit:fit + 8 * r.n_cand].view(np.uint64).copy()


def plain_serve(backend, arrivals, rows_of, stream):
    """The comparison point: FIFO, one request at a time through the per-population calls."""
    t0 = backend.now()
    for r in arrivals:
        r.t_arrival += t0
    for r in arrivals:
        while backend.now() < r.t_arrival:
            pass
        r.t_launch = backend.now()
        backend.plain(r, stream)
        r.t_done = backend.now()
    t1 = backend.now()
    lat = [r.latency for r in arrivals]
    evals = sum(r.n_cand * rows_of[r.run_id] for r in arrivals)
    return {"requests": len(arrivals), "p50_ms": 1000 * percentile(lat, 50),
            "p99_ms": 1000 * percentile(lat, 99), "mean_ms": 1000 * sum(lat) / len(lat),
            "evals_per_s": evals / (t1 - t0), "wall_s": t1 - t0}
