"""Reference reader of delimited text matrices and writer of bicluster result files.

Test infrastructure only: the tests compare the library's C++ loader and writer with these
plain-Python restatements. Nothing in the library imports this module.

What it follows (arXiv 1807.09932, Methods):
- "Different input file formats support": values separated by a comma, a tabulator or a
  semicolon; the upper-left header field is not required (R writes a header row with one field
  fewer than the data rows when the data have row names).
- "Handling missing values": a predefined value (e.g. 0 or 999) marks a missing value, which no
  longer counts; here such cells, empty cells and NA / NaN become NaN.
- "Compatibility with R and Bioconductor": results saved in a form the biclust package loads;
  here its bicluster result-file layout (a title line; per bicluster "rows cols", the row names,
  the column names).

Readings taken where the text is silent (the same ones the library documents): blank lines are
skipped; names lose surrounding spaces and quotes; the delimiter, when not given, is the one of
tab, semicolon, comma occurring most often in the first line (ties in that order; comma when none
occurs); the first line is a header when it has one field fewer than the second, when a field
other than its first is not a number, or when none of its fields is a number; the data rows have
a row-name column when the first field of the first data row is not a number.
"""
import math

import numpy as np

_NA = {"", "NA", "NaN", "nan", "NAN", "na"}


def _trim(s):
    return s.strip(" \"'").rstrip("\r").strip(" \"'")


def _number(s):
    """float of s when s is a plain decimal number (as strtod-like parsing reads it), else None."""
    t = s[1:] if s.startswith("+") else s
    if not t or t[0] in "+":
        return None
    low = t.lower()
    if low in ("inf", "-inf", "infinity", "-infinity"):
        return float(t)
    if low in ("nan", "-nan"):
        return float("nan")
    try:
        if any(c not in "0123456789.eE-+" for c in t):
            return None
        return float(t)
    except ValueError:
        return None


def _cell(s, missing):
    """(ok, value): value of a data cell, NaN for missing cells."""
    if missing is not None and missing[0] == "text" and s == missing[1]:
        return True, math.nan
    if s in _NA:
        return True, math.nan
    v = _number(s)
    if v is None:
        return False, None
    if missing is not None and missing[0] == "num" and v == missing[1]:
        return True, math.nan
    return True, v


def read_matrix_text(path, delimiter=None, missing=None):
    """(values float32 [rows][cols], row_names or None, col_names or None)."""
    with open(path, "rb") as f:
        text = f.read().decode()
    lines = [ln[:-1] if ln.endswith("\r") else ln for ln in text.split("\n")]
    lines = [ln for ln in lines if _trim(ln) != ""]
    if not lines:
        raise ValueError("the file has no data")
    if delimiter is None:
        counts = [(lines[0].count(c), c) for c in ("\t", ";", ",")]
        best = max(n for n, _ in counts)
        delimiter = next(c for n, c in counts if n == best) if best > 0 else ","
    mk = None
    if missing is not None and str(missing).strip(" \"'") != "":
        tok = str(missing).strip(" \"'")
        v = _number(tok)
        mk = ("num", v) if v is not None else ("text", tok)

    def fields(line):
        return [_trim(x) for x in line.split(delimiter)]

    f0 = fields(lines[0])
    nxt = fields(lines[1]) if len(lines) > 1 else None
    text_idx = [i for i, x in enumerate(f0) if not _cell(x, mk)[0]]
    header = (nxt is not None and len(f0) + 1 == len(nxt)) or any(i > 0 for i in text_idx) \
        or len(text_idx) == len(f0)
    first = 1 if header else 0
    if first >= len(lines):
        raise ValueError("no data rows")
    f1 = fields(lines[first])
    row_names = not _cell(f1[0], mk)[0]
    nfield = len(f1)
    cols = nfield - (1 if row_names else 0)
    if cols < 1:
        raise ValueError("no data columns")
    col_names = None
    if header:
        if len(f0) == cols:
            col_names = f0
        elif len(f0) == cols + 1 and row_names:
            col_names = f0[1:]
        else:
            raise ValueError("the header has a different number of fields from the data rows")
    rows = len(lines) - first
    X = np.zeros((rows, cols), dtype=np.float32)
    rn = [] if row_names else None
    for r in range(rows):
        fs = fields(lines[first + r])
        if len(fs) != nfield:
            raise ValueError(f"line {first + r + 1}: wrong number of fields")
        k = 0
        if row_names:
            rn.append(fs[0])
            k = 1
        for c in range(cols):
            ok, v = _cell(fs[k + c], mk)
            if not ok:
                raise ValueError(f"line {first + r + 1}, column {c + 1}: not a number")
            X[r, c] = np.float32(v)
    return X, rn, col_names


def write_biclusters(path, title, members, bitmaps, row_names=None, col_names=None):
    """members: list of column lists; bitmaps: [n][W] uint32 row bitmaps (LSB-first)."""
    out = [title]
    for b, cols in enumerate(members):
        rows = [w * 32 + i for w, word in enumerate(bitmaps[b]) for i in range(32)
                if (int(word) >> i) & 1]
        out.append(f"{len(rows)} {len(cols)}")
        out.append(" ".join(row_names[r] if row_names else str(r + 1) for r in rows))
        out.append(" ".join(col_names[c] if col_names and c < len(col_names) else str(c + 1)
                            for c in cols))
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")
