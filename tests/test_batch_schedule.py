"""hef_batch_schedule on the host (no device work): the longest-first
assignment of the batched form's hypergraphs to pool streams, and its
argument checks.  The item arrays are only checked for NULL, never read, so
placeholder addresses stand in for them."""
import ctypes

import pytest

from paper_2511_06600_gb300 import _binding as B

HEF_OK = 0


@pytest.fixture(autouse=True, scope="module")
def built_library():
    from paper_2511_06600_gb300 import build
    build.build()


def items(sizes):
    arr = (B._BatchItem * len(sizes))()
    fake = ctypes.c_void_p(0x1000)  # never dereferenced by the scheduler
    for it, (n, m, P) in zip(arr, sizes):
        it.n, it.m, it.P = n, m, P
        for f in ("eptr", "pins", "w", "x0_clique", "x0_star", "R_out"):
            setattr(it, f, fake)
    return arr


def schedule(sizes, k=5, S=2, nstreams=4):
    arr = items(sizes)
    out = (ctypes.c_int32 * len(sizes))()
    rc = B.lib().hef_batch_schedule(arr, len(sizes), k, S, nstreams, out)
    return rc, list(out)


SIZES = [(5000, 5200, 18000), (200, 210, 700), (90000, 95000, 330000), (12, 8, 15),
         (40000, 41000, 150000), (5000, 5200, 18000), (700, 720, 2600)]


def test_streams_in_range_and_deterministic():
    rc, a = schedule(SIZES, nstreams=3)
    assert rc == HEF_OK
    assert all(0 <= s < 3 for s in a)
    assert schedule(SIZES, nstreams=3) == (rc, a)


def test_one_stream_and_one_stream_per_item():
    rc, a = schedule(SIZES, nstreams=1)
    assert rc == HEF_OK and a == [0] * len(SIZES)
    # with a stream per item, longest first onto the least loaded stream
    # gives every item a stream of its own, the largest the first stream
    rc, a = schedule(SIZES, nstreams=len(SIZES))
    assert rc == HEF_OK and sorted(a) == list(range(len(SIZES)))
    assert a[2] == 0


def test_larger_items_never_share_while_a_stream_is_empty():
    # two large items and many small ones on two streams: the large ones go
    # to different streams (the second large item finds the other stream
    # empty), and no stream is left without work
    sizes = [(100000, 100000, 400000), (90000, 90000, 360000)] + [(100, 100, 300)] * 6
    rc, a = schedule(sizes, nstreams=2)
    assert rc == HEF_OK
    assert a[0] != a[1] and set(a) == {0, 1}


@pytest.mark.parametrize("k,S,nstreams", [(5, 3, 4), (5, 2, 0), (5, 2, 1000), (0, 2, 4),
                                          (200, 4, 4)])
def test_bad_arguments_are_rejected(k, S, nstreams):
    rc, _ = schedule(SIZES, k=k, S=S, nstreams=nstreams)
    assert rc != HEF_OK


def test_null_array_in_an_item_is_rejected():
    arr = items(SIZES)
    arr[3].pins = None
    out = (ctypes.c_int32 * len(SIZES))()
    assert B.lib().hef_batch_schedule(arr, len(SIZES), 5, 2, 4, out) != HEF_OK
    assert B.lib().hef_batch_schedule(items(SIZES), len(SIZES), 5, 2, 4, None) != HEF_OK


def test_incidence_workspace_size_query():
    """hef_incidence_workspace_bytes (host arithmetic over the layout): 0 for
    negative sizes, 256-byte multiples, never smaller for a larger hypergraph,
    and room for at least the CSC, CSR and per-edge / per-vertex arrays."""
    f = B.lib().hef_incidence_workspace_bytes
    assert f(-1, 5, 5) == 0 and f(5, -1, 5) == 0 and f(5, 5, -1) == 0
    base = f(210000, 200000, 716793)
    assert base % 256 == 0
    for n, m, P in [(210001, 200000, 716793), (210000, 200001, 716793), (210000, 200000, 716794),
                    (420000, 400000, 1433586)]:
        assert f(n, m, P) >= base
    n, m, P = 210000, 200000, 716793
    # ceptr, perm, 3 FP64 + 3 FP32 edge arrays; vptr, 5 FP64 + 5 FP32 vertex
    # arrays; cpins, slot_edge, vedge, vslot
    floor = 4 * (2 * m) + 8 * 3 * m + 4 * 3 * m + 4 * n + 8 * 5 * n + 4 * 5 * n + 4 * 4 * P
    assert base >= floor
