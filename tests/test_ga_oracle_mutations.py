"""Plant a plausible mistake in a copy of the generation-loop oracle and check that a pin of
tests/test_ga_oracle.py catches it (on the CPU).

Each mutation edits oracle/ga.py textually, loads the edited copy as a module of the oracle
package, and runs every pin of test_ga_oracle.py against it. A mutation no pin detects would
mean the oracle could carry that mistake unnoticed, so the test fails.
"""
import importlib.util
import os
import sys

import pytest

import oracle
import test_ga_oracle as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "ga.py")

MUTATIONS = {
    "generator increment": ("GAMMA = 0x9E3779B97F4A7C15", "GAMMA = 0x9E3779B97F4A7C17"),
    "biased shuffle": ("j = i + rng.below(C - i)", "j = rng.below(C)"),
    "crossover keeps repeated columns": ("        if x not in child:\n            child.append(x)",
                                         "        if True:\n            child.append(x)"),
    "swap may pick one position": ("            if j >= i:\n                j += 1",
                                   "            if False:\n                j += 1"),
    "operators tried backwards": ("op = (first + k) % 4", "op = (first - k) % 4"),
    "tournament keeps the worse": ("if comes_before(c, best, pop, fit, counts):",
                                   "if comes_before(best, c, pop, fit, counts):"),
    "order by count first": ("return (-int(fit[i]), -int(counts[i]), -len(pop[i]), pop[i], i)",
                             "return (-int(counts[i]), -int(fit[i]), -len(pop[i]), pop[i], i)"),
    "archived sequences offered": ("if s in held or s in taken:", "if s in taken:"),
    "overlap at the limit penalises": ("if float(overlap_with_member(t, a)) <= limit:",
                                       "if float(overlap_with_member(t, a)) < limit:"),
    "equal quality replaced": ("if c.q > m.q:", "if c.q >= m.q:"),
    "earlier offers not checked": ("if shares_column(c.cols, offered[u].cols) and \\",
                                   "if False and \\"),
    "archive ordered by count first": (
        "merged.sort(key=lambda m: (-m.q, -m.count, -len(m.cols), m.cols))",
        "merged.sort(key=lambda m: (-m.count, -m.q, -len(m.cols), m.cols))"),
    "repeats not varied": ("        if tuple(child) in held:", "        if False:"),
    "repeat pass ignores tabu": ("return tuple(child) in tabu or tuple(child) in held",
                                 "return tuple(child) in held"),
    "tabu not retried": ("while t < p.tabu_retries and tuple(child) in tabu:",
                         "while False:"),
}

PINS = sorted(n for n in dir(pins) if n.startswith("test_"))


def _load(text, tmp_path, name):
    path = os.path.join(str(tmp_path), name + ".py")
    with open(path, "w") as f:
        f.write(text)
    spec = importlib.util.spec_from_file_location("oracle." + name, path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod   # dataclasses look their module up while it executes
    try:
        spec.loader.exec_module(mod)
    finally:
        del sys.modules[spec.name]
    return mod


def _run_pins(mod):
    saved = pins.ga
    pins.ga = mod
    failed = []
    try:
        for n in PINS:
            try:
                getattr(pins, n)()
            except Exception:   # an assertion, or a crash the mistake causes
                failed.append(n)
    finally:
        pins.ga = saved
    return failed


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    text = open(SRC).read()
    old, new = MUTATIONS[name]
    assert text.count(old) == 1, f"mutation anchor not found once: {name}"
    mod = _load(text.replace(old, new), tmp_path, "_ga_mutant")
    assert _run_pins(mod), f"no pin detects the mutation '{name}'"


def test_unmutated_copy_passes(tmp_path):
    mod = _load(open(SRC).read(), tmp_path, "_ga_copy")
    assert _run_pins(mod) == []
