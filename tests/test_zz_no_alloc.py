"""The allocation-free entry point gives exactly the results of the regular one.

ebic_eval_population_noalloc exists for callers that cannot allocate device memory while they
evaluate. Examples: a serving loop that must never wait on the allocator or hit an out-of-memory
error mid-request; a process whose device memory another framework's caching allocator already
owns. It uses a fixed scratch area inside the library instead of per-call allocations. This file
checks it through the C ABI against ebic_eval_population on two calls in a row, bit for bit
(results are integers), on the default stream and on a side stream; that a failed device-side
list check is reported and does not leak into the next call through the shared scratch; and that
memory of another device is refused. The file is named to be collected last, and it passes on
its own in a fresh process too.
"""
import numpy as np
import pytest

from paper_1807_09932_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    view = {np.dtype(np.uint16): np.int16, np.dtype(np.uint32): np.int32}[a.dtype]
    return torch.from_numpy(np.ascontiguousarray(a).view(view)).cuda()


def _run_pair(ebic, m, cols, offs, flags):
    import torch
    n = len(offs) - 1
    dcols, doffs = _dev(cols), _dev(offs)
    ref_c = torch.zeros(n, dtype=torch.int32, device="cuda")
    ref_b = torch.zeros((n, m.words), dtype=torch.int32, device="cuda")
    rc = ebic.ebic_eval_population(m.handle, dcols, doffs, n, flags, ref_c, ref_b)
    assert rc == ebic.EBIC_OK, ebic.ebic_last_error()
    # two calls in a row: population in device memory, then in host memory (staged through the
    # library's fixed scratch); outputs poisoned beforehand so unwritten words would show
    for c_in, o_in in ((dcols, doffs), (cols, offs)):
        got_c = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        got_b = torch.full((n, m.words), -1, dtype=torch.int32, device="cuda")
        rc = ebic.ebic_eval_population_noalloc(m.handle, c_in, o_in, n, flags, got_c, got_b)
        assert rc == ebic.EBIC_OK, ebic.ebic_last_error()
        assert m.status() == ebic.EBIC_OK
        assert torch.equal(got_c, ref_c)
        assert torch.equal(got_b, ref_b)
        # counts only
        got_c.fill_(-1)
        rc = ebic.ebic_eval_population_noalloc(m.handle, c_in, o_in, n, flags, got_c, None)
        assert rc == ebic.EBIC_OK, ebic.ebic_last_error()
        assert m.status() == ebic.EBIC_OK
        assert torch.equal(got_c, ref_c)


@pytest.mark.parametrize("negative", [False, True])
def test_noalloc_matches_regular_entry_point_8bit_ranks(negative):
    from paper_1807_09932_gb300 import ebic
    ds, cols, offs = synth.config3(rows=30011)
    with ebic.Matrix(ds.X) as m:
        assert m.rank_bits == 8
        _run_pair(ebic, m, cols, offs, ebic.EBIC_NEGATIVE_TRENDS if negative else 0)


def test_noalloc_matches_regular_entry_point_16bit_ranks():
    from paper_1807_09932_gb300 import ebic
    ds = synth.make_dataset(5, 9001, 200, planted=[(900, 10, True)], nan_frac=0.01)
    cols, offs = synth.make_population(6, 700, 200, 2, 20)
    with ebic.Matrix(ds.X) as m:
        assert m.rank_bits == 16
        _run_pair(ebic, m, cols, offs, ebic.EBIC_NEGATIVE_TRENDS)


def test_noalloc_rejects_what_it_cannot_do_without_allocating():
    import torch
    from paper_1807_09932_gb300 import ebic
    X = np.random.default_rng(1).standard_normal((2000, 40)).astype(np.float32)
    with ebic.Matrix(X) as m:
        # a host population beyond the fixed 1 MiB scratch: clear error, nothing launched
        cols, offs = synth.make_population(2, 40000, 40, 16, 16)   # 1.28 MB of columns
        n = len(offs) - 1
        cnt = torch.zeros(n, dtype=torch.int32, device="cuda")
        rc = ebic.ebic_eval_population_noalloc(m.handle, cols, offs, n, 0, cnt, None)
        assert rc == ebic.EBIC_ERR_UNSUPPORTED
        assert "scratch" in ebic.ebic_last_error()
        # ... the same population in device memory needs no staging and works
        rc = ebic.ebic_eval_population_noalloc(m.handle, _dev(cols), _dev(offs), n, 0, cnt, None)
        assert rc == ebic.EBIC_OK and m.status() == ebic.EBIC_OK
        ref, _ = ebic.eval_population(m, cols, offs, want_bitmaps=False)
        assert np.array_equal(cnt.cpu().numpy().view(np.uint32), ref)
        # host outputs would need a staging buffer: rejected
        small_c, small_o = synth.make_population(3, 10, 40, 2, 5)
        host_counts = np.zeros(10, np.uint32)
        rc = ebic.ebic_eval_population_noalloc(m.handle, small_c, small_o, 10, 0, host_counts,
                                               None)
        assert rc == ebic.EBIC_ERR_INVALID_ARG


def test_noalloc_on_a_side_stream_and_after_a_failed_device_check():
    import torch
    from paper_1807_09932_gb300 import ebic
    ds, cols, offs = synth.config3(rows=20011)
    with ebic.Matrix(ds.X) as m:
        n = len(offs) - 1
        ref_c, ref_b = ebic.eval_population(m, cols, offs)
        # a device-resident list with a column past the matrix: the device check reports it
        # through the matrix status and the counts stay zero
        bad = cols.copy()
        bad[offs[3]] = m.cols + 5
        got_c = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        rc = ebic.ebic_eval_population_noalloc(m.handle, _dev(bad), _dev(offs), n, 0, got_c, None)
        assert rc == ebic.EBIC_OK, ebic.ebic_last_error()
        assert m.status() == ebic.EBIC_ERR_INVALID_ARG
        assert int(torch.count_nonzero(got_c)) == 0
        # the next valid calls, on a side stream, start from a cleared status word
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        dcols, doffs = _dev(cols), _dev(offs)
        for c_in, o_in in ((dcols, doffs), (cols, offs)):
            with torch.cuda.stream(side):
                got_c = torch.full((n,), -1, dtype=torch.int32, device="cuda")
                got_b = torch.full((n, m.words), -1, dtype=torch.int32, device="cuda")
            rc = ebic.ebic_eval_population_noalloc(m.handle, c_in, o_in, n, 0, got_c, got_b,
                                                   stream=side.cuda_stream)
            assert rc == ebic.EBIC_OK, ebic.ebic_last_error()
            assert m.status(side.cuda_stream) == ebic.EBIC_OK
            assert np.array_equal(got_c.cpu().numpy().view(np.uint32), ref_c)
            assert np.array_equal(got_b.cpu().numpy().view(np.uint32), ref_b)


def test_noalloc_refuses_memory_of_another_device():
    import torch
    from paper_1807_09932_gb300 import ebic
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    X = np.random.default_rng(3).standard_normal((3000, 30)).astype(np.float32)
    cols, offs = synth.make_population(4, 50, 30, 2, 6)
    n = len(offs) - 1
    with ebic.Matrix(X) as m:
        here = torch.zeros(n, dtype=torch.int32, device="cuda:0")
        with torch.cuda.device(1):
            there_c = torch.from_numpy(cols.view(np.int16)).to("cuda:1")
            there_o = torch.from_numpy(offs.view(np.int32)).to("cuda:1")
            there_n = torch.zeros(n, dtype=torch.int32, device="cuda:1")
        for args in ((there_c, there_o, here), (cols, offs, there_n)):
            rc = ebic.ebic_eval_population_noalloc(m.handle, args[0], args[1], n, 0, args[2],
                                                   None)
            assert rc == ebic.EBIC_ERR_INVALID_ARG
            assert "another device" in ebic.ebic_last_error()
