"""An EBIC generation scorer built on the oracle, for driving ebic_run_custom in tests."""
import ctypes

import numpy as np

import oracle
from paper_1807_09932_gb300 import ebic


class OracleScorer:
    """Implements the three callbacks of ebic_evaluator with the CPU oracle."""

    def __init__(self, X, exclude_missing=True, negative=False):
        self.X = np.ascontiguousarray(X, dtype=np.float32)
        self.R, self.C = self.X.shape
        self.W = (self.R + 31) // 32
        self.exclude = exclude_missing
        self.negative = negative
        self.arch_lists = []
        self.arch_bm = np.zeros((0, self.W), np.uint32)
        self.pop_lists = []
        self.pop_bm = None
        self.pop_counts = None
        self.error = None
        self._cbs = ebic.EbicEvaluator(None, ebic.EVALUATE_FN(self._evaluate),
                                       ebic.PAIR_FN(self._pairs),
                                       ebic.SET_ARCHIVE_FN(self._set_archive))

    @property
    def evaluator(self):
        return self._cbs

    def _csr(self, lists):
        offs = np.zeros(len(lists) + 1, np.uint32)
        offs[1:] = np.cumsum([len(c) for c in lists])
        cols = np.array([c for l in lists for c in l], np.uint16)
        return cols, offs

    def _evaluate(self, user, cols_p, offs_p, n, counts_p, fit_p, ov_p):
        try:
            offs = np.ctypeslib.as_array(offs_p, (n + 1,)).copy()
            cols = np.ctypeslib.as_array(cols_p, (int(offs[-1]),)).copy()
            c, b = oracle.eval_population(self.X, cols, offs, exclude_missing=self.exclude,
                                          negative=self.negative)
            self.pop_lists = [cols[offs[i]:offs[i + 1]].tolist() for i in range(n)]
            self.pop_bm, self.pop_counts = b, c
            acols, aoffs = self._csr(self.arch_lists)
            f, ov = oracle.fitness(self.R, cols, offs, c, b, acols, aoffs, self.arch_bm)
            np.ctypeslib.as_array(counts_p, (n,))[:] = c
            np.ctypeslib.as_array(fit_p, (n,))[:] = f
            K = len(self.arch_lists)
            if K:
                np.ctypeslib.as_array(ov_p, (n * K,))[:] = ov.reshape(-1)
            return 0
        except Exception as e:  # reported to the test through self.error
            self.error = e
            return 1

    def _pairs(self, user, idx_p, t, out_p):
        try:
            idx = np.ctypeslib.as_array(idx_p, (t,)).copy()
            lists = [self.pop_lists[i] for i in idx]
            cols, offs = self._csr(lists)
            bm = np.ascontiguousarray(self.pop_bm[idx])
            _, ov = oracle.fitness(self.R, cols, offs, self.pop_counts[idx], bm, cols, offs, bm)
            np.ctypeslib.as_array(out_p, (t * t,))[:] = ov.reshape(-1)
            return 0
        except Exception as e:
            self.error = e
            return 1

    def _set_archive(self, user, src_p, k):
        try:
            src = np.ctypeslib.as_array(src_p, (k,)).copy() if k else np.zeros(0, np.int32)
            lists, rows = [], []
            for s in src:
                if s >= 0:
                    lists.append(self.pop_lists[s])
                    rows.append(self.pop_bm[s])
                else:
                    lists.append(self.arch_lists[-s - 1])
                    rows.append(self.arch_bm[-s - 1])
            self.arch_lists = lists
            self.arch_bm = np.array(rows, np.uint32).reshape(len(lists), self.W)
            return 0
        except Exception as e:
            self.error = e
            return 1
