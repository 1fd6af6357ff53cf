"""The serving loop's admission policy, on a virtual clock (host only).

tw_serve_simulate runs the same policy object as tw_serve_replay with a
modelled batch time cost_ms + cost_ms_per_req * size.  The checks are the
policy's defining properties, read back from the latencies: requests are
served in arrival order, no batch exceeds max_batch, no request starts
before it arrives, the server never idles while a request waits, and a
batch takes everything that has arrived when it starts (up to max_batch).
"""
import numpy as np
import pytest

from paper_2504_16344_gb300 import build, tw

COST, PER = 5.0, 0.5      # ms


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    tw.load()


def _batches(arr, lat, bid, max_batch):
    """(start, end, members) per batch, checking each batch has one end time."""
    out = []
    for k in range(bid.max() + 1):
        idx = np.flatnonzero(bid == k)
        ends = arr[idx] + lat[idx] / 1e3
        assert np.allclose(ends, ends[0], rtol=0, atol=1e-9)
        service = (COST + PER * len(idx)) / 1e3
        out.append((ends[0] - service, ends[0], idx))
    return out


def _trace(n, rate, seed):
    g = np.random.default_rng(seed)
    return np.cumsum(g.exponential(1.0 / rate, size=n))


@pytest.mark.parametrize("rate,max_batch", [(50.0, 8), (400.0, 8), (2000.0, 16), (1e5, 4)])
def test_policy_properties(rate, max_batch):
    arr = _trace(300, rate, seed=int(rate) + max_batch)
    lat, bid = tw.serve_simulate(arr, max_batch, COST, PER)
    assert np.all(np.diff(bid) >= 0)                       # FIFO
    b = _batches(arr, lat, bid, max_batch)
    prev_end = -np.inf
    for k, (start, end, idx) in enumerate(b):
        assert 1 <= len(idx) <= max_batch
        assert np.all(arr[idx] <= start + 1e-12)            # nobody starts before arriving
        # work-conserving: the batch starts when the server frees up or,
        # if it was idle, when its first request arrives
        assert start == pytest.approx(max(prev_end, arr[idx[0]]), abs=1e-9)
        # maximal: a smaller batch means the next request had not arrived
        if len(idx) < max_batch and idx[-1] + 1 < len(arr):
            assert arr[idx[-1] + 1] > start
        prev_end = end
    assert np.all(lat >= (COST + PER) - 1e-9)


def test_light_load_serves_each_request_alone():
    arr = np.arange(50) * 0.1                               # 100 ms apart, service 5.5 ms
    lat, bid = tw.serve_simulate(arr, 8, COST, PER)
    assert np.array_equal(bid, np.arange(50))
    assert np.allclose(lat, COST + PER)


def test_burst_fills_batches_in_order():
    arr = np.zeros(20)
    lat, bid = tw.serve_simulate(arr, 8, COST, PER)
    assert np.array_equal(bid, np.repeat([0, 1, 2], [8, 8, 4]))
    full = COST + 8 * PER
    assert np.allclose(lat[:8], full)
    assert np.allclose(lat[8:16], 2 * full)
    assert np.allclose(lat[16:], 2 * full + COST + 4 * PER)


def test_rejects_unsorted_arrivals():
    with pytest.raises(tw.TwError):
        tw.serve_simulate(np.array([0.0, 1.0, 0.5]), 4, COST, PER)
    with pytest.raises(tw.TwError):
        tw.serve_simulate(np.array([0.0]), 0, COST, PER)


# ---- several lanes: batches in flight at the same time ----------------------

def _intervals(arr, lat, bid):
    """(start, end, members) per batch in start order (modelled service time)."""
    out = []
    for k in range(bid.max() + 1):
        idx = np.flatnonzero(bid == k)
        ends = arr[idx] + lat[idx] / 1e3
        assert np.allclose(ends, ends[0], rtol=0, atol=1e-9)
        out.append((ends[0] - (COST + PER * len(idx)) / 1e3, ends[0], idx))
    return out


@pytest.mark.parametrize("lanes", [2, 3])
@pytest.mark.parametrize("rate,max_batch", [(200.0, 8), (2000.0, 16), (1e5, 4)])
def test_lanes_policy_properties(lanes, rate, max_batch):
    arr = _trace(400, rate, seed=int(rate) + 10 * lanes)
    lat, bid = tw.serve_simulate(arr, max_batch, COST, PER, lanes=lanes)
    assert np.all(np.diff(bid) >= 0)                       # batches start in request order
    b = _intervals(arr, lat, bid)
    starts = np.array([s for s, _, _ in b])
    ends = np.array([e for _, e, _ in b])
    assert np.all(np.diff(starts) >= -1e-12)
    for k, (start, end, idx) in enumerate(b):
        assert 1 <= len(idx) <= max_batch
        assert np.all(arr[idx] <= start + 1e-12)
        # never more than `lanes` batches in flight
        inflight = np.sum((starts <= start + 1e-12) & (ends > start + 1e-12))
        assert inflight <= lanes
        # work-conserving: a batch starts when its first request arrives or
        # when a lane frees up (some earlier batch ends then)
        freed = np.any(np.isclose(ends[:k], start, rtol=0, atol=1e-9))
        assert np.isclose(start, arr[idx[0]], rtol=0, atol=1e-9) or freed
        # a lane idles only when nothing waits: if fewer than `lanes` batches
        # were in flight just before the start, the first request had just arrived
        if not freed and k > 0:
            assert arr[idx[0]] > starts[k - 1] - 1e-12


def test_lanes_overlap_under_load():
    """At 2000 requests/s against a 9 ms batch, two lanes keep two batches in
    flight: arrivals during a batch start before it ends, and the mean
    latency is below the one-lane policy's."""
    arr = _trace(400, 2000.0, seed=77)
    lat1, _ = tw.serve_simulate(arr, 8, COST, PER, lanes=1)
    lat2, bid2 = tw.serve_simulate(arr, 8, COST, PER, lanes=2)
    b = _intervals(arr, lat2, bid2)
    overlaps = sum(1 for k in range(1, len(b)) if b[k][0] < b[k - 1][1] - 1e-12)
    assert overlaps > len(b) // 2
    assert lat2.mean() < lat1.mean()


def test_lanes_burst():
    arr = np.zeros(20)
    lat, bid = tw.serve_simulate(arr, 8, COST, PER, lanes=2)
    assert np.array_equal(bid, np.repeat([0, 1, 2], [8, 8, 4]))
    full = COST + 8 * PER
    assert np.allclose(lat[:16], full)                       # two batches side by side
    assert np.allclose(lat[16:], full + COST + 4 * PER)      # the third when a lane frees
    with pytest.raises(tw.TwError):
        tw.serve_simulate(arr, 8, COST, PER, lanes=0)
