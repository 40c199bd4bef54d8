"""Plant a plausible mistake in a copy of the oracle (on the CPU) and check that the pins catch it.

Each mutation edits the oracle's C source textually, compiles it into a temporary library and
runs every pin against it. A mutation that no pin detects would mean the oracle could carry that
mistake unnoticed, so the test fails.
"""
import os
import subprocess

import pytest

import oracle

import pins

MUTATIONS = {
    "strict relation": ("if (!(v[i] <= v[i + 1])) asc = 0;", "if (!(v[i] < v[i + 1])) asc = 0;"),
    "transposed operand": ("if (!(v[i] <= v[i + 1])) asc = 0;",
                           "if (!(v[i + 1] <= v[i])) asc = 0;"),
    "exclusion dropped": ("if (exclude_missing) return 0;", "if (0) return 0;"),
    "fill value ignored": ("x = fill_value;                /*", "x = 0.0f;                /*"),
    "negative option ignored": ("return asc || (negative && desc);", "return asc;"),
    "negative always on": ("return asc || (negative && desc);", "return asc || desc;"),
    "bit index off by one": ("bm[r >> 5] |= 1u << (r & 31);", "bm[r >> 5] |= 1u << ((r + 1) & 31);"),
    "last row skipped": ("for (int64_t r = 0; r < R; ++r) {\n            int m",
                         "for (int64_t r = 0; r + 1 < R; ++r) {\n            int m"),
    "penalty without shared columns": ("if (s && at_least_as_good && o > penalty) penalty = o;",
                                       "if (at_least_as_good && o > penalty) penalty = o;"),
    "penalty from worse members": ("if (s && at_least_as_good && o > penalty) penalty = o;",
                                   "if (s && o > penalty) penalty = o;"),
    "penalty summed": ("if (s && at_least_as_good && o > penalty) penalty = o;",
                       "if (s && at_least_as_good) penalty += o;"),
    "domination compared strictly": ("int at_least_as_good = quality(na, La) >= qc;",
                                     "int at_least_as_good = quality(na, La) > qc;"),
    "weight exponent off by one": ("uint32_t shift = (L < 33 ? L : 33) - 1;",
                                   "uint32_t shift = (L < 33 ? L : 33);"),
    "rank counts duplicates": ("rank += (uint32_t)first;", "rank += 1u;"),
    "rank uses <=": ("if (miss[i] || !(v[i] < v[j])) continue;",
                     "if (miss[i] || !(v[i] <= v[j])) continue;"),
    "overlap drops last word": ("o += popcount32(bitmaps[p * W + w] & abitmaps[(int64_t)a * W + w]);",
                                "o += (w + 1 < W) ? popcount32(bitmaps[p * W + w] & "
                                "abitmaps[(int64_t)a * W + w]) : 0u;"),
}

CHECKS = [
    lambda: pins.check_bruteforce(1),
    lambda: pins.check_bruteforce(2, R=33, C=4, max_len=4),
    lambda: pins.check_closed_form(11, R=20000),
    lambda: pins.check_closed_form(11, R=20000, negative=True),
    lambda: pins.check_invariants(5),
    lambda: pins.check_planted_recovery(21),
    lambda: pins.check_fitness(31),
    lambda: pins.check_dense_ranks(41),
]


def _compile(src_text, path):
    src = path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", src, "-o", path, "-lm"],
                   check=True, capture_output=True)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_mutation(name, tmp_path):
    with open(oracle._SRC) as f:
        text = f.read()
    old, new = MUTATIONS[name]
    assert text.count(old) == 1, f"mutation anchor not found once: {name}"
    path = os.path.join(str(tmp_path), "libmut.so")
    _compile(text.replace(old, new), path)
    saved = oracle._load()
    oracle._lib = oracle._open(path)
    caught = False
    try:
        for check in CHECKS:
            try:
                check()
            except AssertionError:
                caught = True
                break
    finally:
        oracle._lib = saved
    assert caught, f"no pin detects the mutation '{name}'"


def test_unmutated_copy_passes(tmp_path):
    """The same harness on an unchanged copy: every pin passes."""
    with open(oracle._SRC) as f:
        text = f.read()
    path = os.path.join(str(tmp_path), "libsame.so")
    _compile(text, path)
    saved = oracle._load()
    oracle._lib = oracle._open(path)
    try:
        for check in CHECKS:
            check()
    finally:
        oracle._lib = saved
