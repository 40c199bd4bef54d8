"""A serving backend for host-only tests: results from the oracle, time from a fake clock."""
import numpy as np

import oracle


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t


class FakeBackend:
    """Each launched batch finishes `fixed + per_eval * evals` fake seconds after its launch.
    With two slots busy at once their device time is shared (the GPU is one resource)."""

    def __init__(self, clock, fixed=1e-3, per_eval=1e-9):
        self.clock = clock
        self.fixed, self.per_eval = fixed, per_eval
        self.runs = {}
        self.launched = []
        self.gpu_free_at = 0.0

    def footprint(self, spec):
        return spec.X.shape[0] * spec.X.shape[1] + spec.max_cand * 100

    def now(self):
        return self.clock.t

    def open_run(self, spec):
        self.runs[spec.run_id] = spec

    def close_run(self, run_id):
        del self.runs[run_id]

    def launch(self, reqs):
        evals = sum(r.n_cand * self.runs[r.run_id].X.shape[0] for r in reqs)
        start = max(self.clock.t, self.gpu_free_at)
        finish = start + self.fixed + self.per_eval * evals
        self.gpu_free_at = finish
        self.launched.append([r.rid for r in reqs])
        return {"finish": finish}

    def done(self, token):
        return self.clock.t >= token["finish"]

    def collect(self, token, reqs):
        for r in reqs:
            spec = self.runs[r.run_id]
            c, b = oracle.eval_population(spec.X, r.cols, r.offsets)
            ac = spec.archive_cols if spec.archive_cols is not None else np.zeros(0, np.uint16)
            ao = spec.archive_offsets if spec.archive_offsets is not None else np.zeros(1, np.uint32)
            _, abm = oracle.eval_population(spec.X, ac, ao)
            f, _ = oracle.fitness(spec.X.shape[0], r.cols, r.offsets, c, b, ac, ao, abm,
                                  want_overlaps=False)
            r.counts, r.fitness = c, f

    def next_event(self, inflight):
        return min((t["finish"] for t, _ in inflight), default=None)
