"""Text matrix loader and bicluster writer (host code, CPU tests): the hand-worked golden files,
numpy.loadtxt on plain numeric files, the plain-Python reference reader/writer on randomised
files, and the error cases."""
import json
import math
import os

import numpy as np
import pytest

from oracle import textio as ref

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def ebic():
    from paper_1807_09932_gb300 import ebic as e
    return e


def _same(a, b):
    a = np.asarray(a, dtype=np.float32)
    b = np.asarray(b, dtype=np.float32)
    return a.shape == b.shape and np.array_equal(np.isnan(a), np.isnan(b)) and \
        np.array_equal(a[~np.isnan(a)].view(np.uint32), b[~np.isnan(b)].view(np.uint32))


def test_golden_files(ebic):
    spec = json.load(open(os.path.join(GOLDEN, "text_loader_cases.json")))
    for case in spec["cases"]:
        path = os.path.join(GOLDEN, case["file"])
        want = np.array([[math.nan if v is None else v for v in row] for row in case["values"]],
                        dtype=np.float32)
        for reader in (ebic.read_matrix_text, ref.read_matrix_text):
            X, rn, cn = reader(path, delimiter=case["delimiter"], missing=case["missing"])
            assert _same(X, want), (reader, case["file"])
            assert rn == case["row_names"] and cn == case["col_names"]


@pytest.mark.parametrize("delim", [",", "\t", ";"])
def test_plain_numeric_files_match_numpy(ebic, tmp_path, delim):
    rng = np.random.default_rng(len(delim) + ord(delim))
    A = rng.standard_normal((57, 9)) * 10.0 ** rng.integers(-3, 4, (57, 9))
    path = tmp_path / "m.txt"
    np.savetxt(path, A, delimiter=delim, fmt="%.9g")
    X, rn, cn = ebic.read_matrix_text(str(path))
    assert rn is None and cn is None
    assert _same(X, np.loadtxt(path, delimiter=delim).astype(np.float32))


def _random_file(rng, path):
    R, C = int(rng.integers(1, 40)), int(rng.integers(1, 12))
    delim = [",", "\t", ";"][int(rng.integers(3))]
    header, rownames = bool(rng.integers(2)), bool(rng.integers(2))
    corner = header and rownames and bool(rng.integers(2))
    quote = bool(rng.integers(2))
    q = (lambda s: f'"{s}"') if quote else (lambda s: s)
    marker = [None, "999", "0", "NA"][int(rng.integers(4))]
    lines = []
    if header:
        names = [q(f"c{j}x") for j in range(C)]
        lines.append(delim.join(([q("id")] if corner else []) + names))
    for r in range(R):
        cells = []
        for _ in range(C):
            u = rng.random()
            if u < 0.08:
                cells.append("")
            elif u < 0.14:
                cells.append("NA")
            elif u < 0.2 and marker in ("999", "0"):
                cells.append(marker if rng.integers(2) else marker + ".0")
            else:
                v = rng.standard_normal() * 10 ** int(rng.integers(-4, 5))
                cells.append(f"{v:.{int(rng.integers(1, 10))}g}")
        if rownames:
            cells = [q(f"r{r}")] + cells
        lines.append(delim.join(cells))
        if rng.random() < 0.05:
            lines.append("")
    eol = "\r\n" if rng.integers(2) else "\n"
    path.write_text(eol.join(lines) + (eol if rng.integers(2) else ""))
    return delim if rng.integers(2) else None, marker


def test_random_files_match_reference(ebic, tmp_path):
    rng = np.random.default_rng(1807)
    checked = 0
    for i in range(300):
        path = tmp_path / f"f{i}.txt"
        delim, marker = _random_file(rng, path)
        try:
            want = ref.read_matrix_text(str(path), delimiter=delim, missing=marker)
        except ValueError:
            with pytest.raises(ebic.EbicError):
                ebic.read_matrix_text(str(path), delimiter=delim, missing=marker)
            continue
        got = ebic.read_matrix_text(str(path), delimiter=delim, missing=marker)
        assert _same(got[0], want[0]), path.read_text()[:300]
        assert got[1] == want[1] and got[2] == want[2]
        checked += 1
    assert checked > 200


def test_errors_name_the_line(ebic, tmp_path):
    p = tmp_path / "bad.csv"
    p.write_text("1,2,3\n4,5\n")
    with pytest.raises(ebic.EbicError) as ei:
        ebic.read_matrix_text(str(p))
    assert ei.value.code == ebic.EBIC_ERR_INVALID_ARG and "line 2" in str(ei.value)
    p.write_text("1,2,3\n4,x,6\n")
    with pytest.raises(ebic.EbicError) as ei:
        ebic.read_matrix_text(str(p))
    assert "line 2, column 2" in str(ei.value)
    with pytest.raises(ebic.EbicError):
        ebic.read_matrix_text(str(tmp_path / "missing.csv"))
    with pytest.raises(ebic.EbicError):
        ebic.read_matrix_text(str(p), delimiter="|")


def test_writer_matches_reference(ebic, tmp_path):
    rng = np.random.default_rng(5)
    R, C = 70, 9
    members = [list(rng.choice(C, int(rng.integers(1, 6)), replace=False)) for _ in range(6)]
    W = (R + 31) // 32
    bits = rng.random((6, W * 32)) < 0.3
    bits[:, R:] = False
    bm = np.packbits(bits.astype(np.uint8), axis=1, bitorder="little").view("<u4") \
        .astype(np.uint32)
    cols = np.array([c for m in members for c in m], dtype=np.uint16)
    offs = np.cumsum([0] + [len(m) for m in members]).astype(np.uint32)
    result = {"members": members, "cols": cols, "offsets": offs,
              "counts": np.array([int(b.sum()) for b in bits], dtype=np.uint32),
              "quality": np.zeros(6, dtype=np.uint64), "bitmaps": bm}
    # indices only
    ebic.write_biclusters(str(tmp_path / "a.txt"), result, R, title="run1")
    ref.write_biclusters(str(tmp_path / "b.txt"), "run1", members, bm)
    assert (tmp_path / "a.txt").read_text() == (tmp_path / "b.txt").read_text()
    # with the names of a loaded matrix
    names_file = tmp_path / "names.csv"
    lines = [",".join(f"col{j}" for j in range(C))]
    lines += [f"row{r}," + ",".join("1" for _ in range(C)) for r in range(R)]
    names_file.write_text("\n".join(lines) + "\n")
    with ebic.TextMatrix(str(names_file)) as t:
        ebic.write_biclusters(str(tmp_path / "c.txt"), result, R, names=t, title="run1")
        ref.write_biclusters(str(tmp_path / "d.txt"), "run1", members, bm, t.row_names,
                             t.col_names)
    assert (tmp_path / "c.txt").read_text() == (tmp_path / "d.txt").read_text()
    text = (tmp_path / "c.txt").read_text().splitlines()
    assert text[0] == "run1" and text[1] == f"{int(bits[0].sum())} {len(members[0])}"
