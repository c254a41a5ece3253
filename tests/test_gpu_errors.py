"""The C ABI's error contract on a GPU, and concurrent use from host threads.

Every error case here is caught on the host before anything is launched:
the call returns its status and nothing is enqueued.
"""
import threading

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2503_06763_gb300 import Batch, Regex, ReError
    return Batch, Regex, ReError


def status_of(excinfo):
    return excinfo.value.status


def test_parse_argument_errors(lib):
    Batch, Regex, ReError = lib
    rx = Regex(W.DNA_RE)
    n = 100_000
    t = torch.from_numpy(W.dna_text(n, seed=1)).cuda()
    kind, cb, _ = rx.layout(n, "auto")
    dt = {1: torch.uint8, 2: torch.int16, 4: torch.int32, 8: torch.int64}[cb]
    out = torch.empty(n + 1, dtype=dt, device="cuda")
    st = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    wsz = rx.workspace_size(n)
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    cap = out.numel() * out.element_size()
    with pytest.raises(ReError) as e:                                   # workspace too small
        rx.parse_raw(t.data_ptr(), n, out.data_ptr(), cap, kind, cb, st.data_ptr(), ws.data_ptr(), wsz // 2, s)
    assert status_of(e) == -8
    with pytest.raises(ReError) as e:                                   # workspace not 256-byte aligned
        rx.parse_raw(t.data_ptr(), n, out.data_ptr(), cap, kind, cb, st.data_ptr(), ws.data_ptr() + 16, wsz - 16, s)
    assert status_of(e) == -8
    with pytest.raises(ReError) as e:                                   # column buffer too small
        rx.parse(t, out=out[:n // 2], status=st, workspace=ws)
    assert status_of(e) == -8
    wide = torch.empty(n + 16, dtype=dt, device="cuda")
    with pytest.raises(ReError) as e:                                   # columns not 16-byte aligned
        rx.parse_raw(t.data_ptr(), n, wide.data_ptr() + cb, (n + 15) * cb, kind, cb, st.data_ptr(),
                     ws.data_ptr(), wsz, s)
    assert status_of(e) == -1
    big = torch.empty(n + 64, dtype=torch.uint8, device="cuda")
    big[1:n + 1].copy_(t)
    with pytest.raises(ReError) as e:                                   # text not 16-byte aligned
        rx.parse(big[1:n + 1], out=out, status=st, workspace=ws)
    assert status_of(e) == -1
    with pytest.raises(ReError) as e:                                   # chunk length not a multiple of 64
        rx.parse(t, chunk_len=100, out=out, status=st, workspace=ws)
    assert status_of(e) == -1
    with pytest.raises(ReError) as e:                                   # DENSE needs at most 64 segments
        Regex(W.LOG_RE).layout(10, "dense")
    assert status_of(e) == -8
    torch.cuda.synchronize()
    assert int(st.item()) == 12345                                      # nothing was enqueued
    cols, st2, _ = rx.parse(t)                                          # the handle still parses
    torch.cuda.synchronize()
    assert int(st2.item()) == 0


def test_batch_and_match_argument_errors(lib):
    Batch, Regex, ReError = lib
    rx = Regex(W.AB_RE)
    t = torch.from_numpy(W.ab_text(5000, seed=2)).cuda()
    b = Batch([rx, rx], [5000, 5000])
    with pytest.raises(ValueError):
        b.parse([t])                                                    # one text per planned length
    with pytest.raises(ReError) as e:
        Batch([rx], [1000], chunk_len=100)                              # chunk length not a multiple of 64
    assert status_of(e) == -1
    cols, st, kind = rx.parse(t)
    with pytest.raises(ReError) as e:
        rx.matches(cols, st, 5000, 0, kind)                             # 0 is no group
    assert status_of(e) == -1
    with pytest.raises(ReError) as e:
        rx.matches(cols, st, 5000, 99, kind)                            # no such group
    assert status_of(e) == -1
    torch.cuda.synchronize()


@pytest.mark.parametrize("shared", [False, True], ids=["own_handles", "one_handle"])
def test_concurrent_host_threads(lib, shared):
    """Several host threads parse at once, each on its own stream and
    buffers, with a handle each or one handle per RE shared by all of them;
    every result equals the single-threaded one."""
    Batch, Regex, ReError = lib
    cases = [(W.DNA_RE, W.dna_text(300_000, seed=s)) for s in range(3)] + \
            [(W.AB_RE, W.ab_text(200_000 + 77 * s, seed=s)) for s in range(3)]
    handles = {pat: Regex(pat) for pat, _ in cases}
    want = []
    for pat, host in cases:
        cols, st, _ = handles[pat].parse(torch.from_numpy(host).cuda())
        torch.cuda.synchronize()
        want.append((cols.cpu().numpy(), int(st.item())))
    errors = []
    start = threading.Barrier(len(cases))

    def worker(j):
        try:
            pat, host = cases[j]
            rx = handles[pat] if shared else Regex(pat)
            s = torch.cuda.Stream()
            t = torch.from_numpy(host).cuda()
            torch.cuda.synchronize()
            start.wait(timeout=60)
            for _ in range(10):
                cols, st, _ = rx.parse(t, stream=s)
                s.synchronize()
                if int(st.item()) != want[j][1] or not np.array_equal(cols.cpu().numpy(), want[j][0]):
                    errors.append(j)
                    return
        except Exception as ex:                                         # reported below
            errors.append((j, repr(ex)))

    threads = [threading.Thread(target=worker, args=(j,)) for j in range(len(cases))]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=300)
    assert not any(th.is_alive() for th in threads)
    assert errors == []
