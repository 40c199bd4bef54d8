"""The oracle against facts that do not come from itself (CPU only)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1807_09932_gb300 import synth

import pins


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_bruteforce_every_candidate(seed):
    pins.check_bruteforce(seed)


def test_bruteforce_ragged_rows():
    # row counts that are not multiples of 32 exercise the bitmap padding bits
    for R in (1, 31, 33, 64, 65):
        pins.check_bruteforce(100 + R, R=R, C=4, max_len=4)


@pytest.mark.parametrize("negative", [False, True])
def test_closed_form_match_rate(negative):
    pins.check_closed_form(11, negative=negative)


@pytest.mark.parametrize("seed", [5, 6])
def test_invariants(seed):
    pins.check_invariants(seed)


def test_planted_recovery():
    pins.check_planted_recovery(21)


@pytest.mark.parametrize("seed", [31, 32])
def test_fitness(seed):
    pins.check_fitness(seed)


@pytest.mark.parametrize("seed", [41, 42])
def test_dense_ranks(seed):
    pins.check_dense_ranks(seed)


def _golden(name):
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        return json.load(f)


def test_golden_missing_value_emptiness():
    g = _golden("missing_values_emptiness.json")
    X = np.array([[np.nan if v is None else v for v in row] for row in g["matrix"]],
                 dtype=np.float32)
    cols, offs = synth.population_from_lists(g["candidates"])
    for case in g["cases"]:
        X2 = X.copy()
        if case["marker"] is not None:
            # the file format's missing cells hold the marker value ...
            X2[np.isnan(X2)] = np.float32(case["marker"])
            if case["marker_is_missing"]:
                # ... which a loader maps back to NaN when the marker means "missing"
                X2[X2 == np.float32(case["marker"])] = np.nan
        c, b = oracle.eval_population(X2, cols, offs, exclude_missing=case["exclude_missing"],
                                      fill_value=case["fill_value"], negative=case["negative"])
        assert c.tolist() == case["counts"], case["name"]
        rows = [sorted(pins.bits_to_rows(b[i])) for i in range(len(c))]
        assert rows == case["rows"], case["name"]


def test_rejects_invalid_candidates():
    X = np.zeros((4, 3), np.float32)
    for cands in ([[0, 0]], [[3]], [[]], [list(range(3)) * 22]):
        if cands == [[]]:
            cols, offs = np.zeros(0, np.uint16), np.zeros(2, np.uint32)
        else:
            cols, offs = synth.population_from_lists(cands)
        with pytest.raises(ValueError):
            oracle.eval_population(X, cols, offs)
