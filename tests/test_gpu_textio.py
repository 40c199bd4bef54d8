"""The paper's workflow end to end on the GPU: a planted dataset written as an R-style CSV
(quoted names, no corner field, the marker 999 for missing values), read by the library's
loader, searched by ebic_run, and the archive written in the biclust result-file layout; the
file is read back and checked against the run and against the oracle's rows of each member."""
import numpy as np
import pytest

import oracle
from paper_1807_09932_gb300 import synth

pytestmark = pytest.mark.gpu


def test_csv_to_biclust_file(tmp_path):
    import torch
    torch.cuda.init()
    from paper_1807_09932_gb300 import ebic
    ds = synth.make_dataset(21, 800, 20, kind="normal", planted=[(200, 6, False)],
                            nan_frac=0.01)
    X = ds.X
    R, C = X.shape
    path = tmp_path / "data.csv"
    lines = [",".join(f'"s{j}"' for j in range(C))]
    for r in range(R):
        cells = ["999" if np.isnan(v) else repr(float(v)) for v in X[r]]
        lines.append(f'"g{r}",' + ",".join(cells))
    path.write_text("\n".join(lines) + "\n")
    with ebic.TextMatrix(str(path), missing=999) as t:
        assert t.row_names[:2] == ["g0", "g1"] and t.col_names[-1] == f"s{C - 1}"
        assert np.array_equal(np.isnan(t.values), np.isnan(X))
        assert np.array_equal(t.values[~np.isnan(X)], X[~np.isnan(X)])
        params = ebic.ebic_params_default(population=200, generations=25, archive_size=5,
                                          max_init_len=5, max_len=10, seed=3)
        with ebic.Matrix(t.values) as m:
            m.build_pairs()
            res = ebic.ebic_run(m.handle, params)
        out = tmp_path / "biclusters.txt"
        ebic.write_biclusters(str(out), res, R, names=t, title="EBIC run")
    text = out.read_text().splitlines()
    assert text[0] == "EBIC run"
    k = 1
    for b, members in enumerate(res["members"]):
        nr, nc = map(int, text[k].split())
        rows = [int(x[1:]) for x in text[k + 1].split()]
        cols = [int(x[1:]) for x in text[k + 2].split()]
        k += 3
        assert nc == len(members) and cols == list(members)
        assert nr == int(res["counts"][b]) == len(rows)
        # the rows in the file are exactly the rows the oracle matches for this member
        mc, mo = synth.population_from_lists([members])
        cnt, bm = oracle.eval_population(X, mc, mo)
        want = [r for r in range(R) if (int(bm[0][r // 32]) >> (r % 32)) & 1]
        assert rows == want
    assert k == len(text) and len(res["members"]) > 0
