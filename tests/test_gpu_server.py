"""The serving loop (abea_server_*): results equal to the batch and one-read
calls and to the oracle, admission under a memory budget, bounded waits."""
import os
import time

import numpy as np
import pytest

from oracle import oracle
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def mix():
    batch, arrival, is_prefix = synth.serving_requests(160, load=10.0)
    return batch, arrival, is_prefix


@pytest.fixture(scope="module")
def ctx(mix):
    batch = mix[0]
    c = binding.Context(0)
    c.set_model(batch.k, batch.model_mean, batch.model_stdv)
    yield c
    c.close()


def submit_all(srv, batch, ids):
    return {i: srv.submit(*batch.read(i)) for i in ids}


def collect(srv, tickets, wait_s=60.0):
    out = {}
    t_end = time.monotonic() + wait_s
    for i, t in tickets.items():
        while True:
            r = srv.poll(t, wait_us=100_000)
            if r is not None:
                out[i] = r
                break
            assert time.monotonic() < t_end, "request did not finish"
    return out


def test_each_result_same_alone_and_in_the_mix(ctx, mix):
    batch = mix[0]
    ids = list(range(batch.n))
    with binding.Server(ctx, batch.W, max_batch_reads=32, max_wait_us=500) as srv:
        got = collect(srv, submit_all(srv, batch, ids))
    # the same reads as one batch
    res, pairs, po = ctx.align_packed(batch)
    for i in ids:
        r, p, lat = got[i]
        assert r["status"] == res["status"][i] and np.float32(r["score"]) == res["score"][i]
        assert r["e_end"] == res["e_end"][i] and r["cells"] == res["cells"][i]
        assert np.array_equal(p, pairs[po[i]:po[i] + res["n_pairs"][i]])
        assert lat > 0
    # alone, one read per call, on a sample
    for i in ids[::20]:
        r1, p1 = ctx.align(*batch.read(i), batch.W)
        assert np.float32(r1["score"]) == np.float32(got[i][0]["score"]) and np.array_equal(p1, got[i][1])
    # and the FP32 oracle on a sample
    sample = ids[::16]
    o = oracle.abea_batch(batch.subset(sample), "f32", n_threads=THREADS)
    for t, i in enumerate(sample):
        assert got[i][0]["status"] == o["status"][t]
        assert np.float32(o["score"][t]) == np.float32(got[i][0]["score"])
        assert np.array_equal(got[i][1], o["pairs"][o["pair_off"][t]:o["pair_off"][t] + o["n_pairs"][t]])


def test_single_queue_gives_the_same_results(ctx, mix):
    """short_bases < 0: one queue for all requests; the results do not change."""
    batch = mix[0]
    ctx.set_model(batch.k, batch.model_mean, batch.model_stdv)
    ids = list(range(0, batch.n, 2))
    got = {}
    for sb in (0, -1):
        with binding.Server(ctx, batch.W, max_batch_reads=16, max_wait_us=300, short_bases=sb) as srv:
            got[sb] = collect(srv, submit_all(srv, batch, ids))
    for i in ids:
        assert np.float32(got[0][i][0]["score"]) == np.float32(got[-1][i][0]["score"])
        assert np.array_equal(got[0][i][1], got[-1][i][1])


def test_admission_under_memory_budget(mix):
    batch = mix[0]
    w = synth.WORKLOADS["batch_4096_ln5kb"]
    L = synth.read_lengths(w)
    huge = synth.make_batch(w, read_ids=[int(np.argmax(L))])     # 135,514 bands: about 6.6 MB of work
    ids = list(range(60))
    # three internal contexts of 5.5 MB each: a micro-batch holds only a few reads; the mix's
    # largest read (81,054 bands, about 4 MB) fits, the 50 kb read does not
    with binding.Context(0, mem_budget_bytes=16_500_000) as small:
        small.set_model(batch.k, batch.model_mean, batch.model_stdv)
        with binding.Server(small, batch.W, max_batch_reads=64, max_wait_us=2000) as srv:
            got = collect(srv, submit_all(srv, batch, ids + [int(np.argmax(batch.n_events()))]))
            with pytest.raises(binding.AbeaError) as ei:
                srv.submit(*huge.read(0))
            assert ei.value.code == binding.ABEA_ERR_NOMEM
    ids = sorted(got)
    with binding.Context(0) as c:
        c.set_model(batch.k, batch.model_mean, batch.model_stdv)
        res, pairs, po = c.align_packed(batch.subset(ids))
    for t, i in enumerate(ids):
        assert np.float32(got[i][0]["score"]) == res["score"][t]
        assert np.array_equal(got[i][1], pairs[po[t]:po[t] + res["n_pairs"][t]])


def test_bounded_wait_capacity_and_tickets(ctx):
    w = synth.WORKLOADS["batch_4096_ln5kb"]
    L = synth.read_lengths(w)
    long_read = synth.make_batch(w, read_ids=[int(np.argmax(L))])
    ctx.set_model(long_read.k, long_read.model_mean, long_read.model_stdv)
    with binding.Server(ctx, long_read.W, max_wait_us=50) as srv:
        t = srv.submit(*long_read.read(0))
        assert srv.poll(t, wait_us=0) is None              # a 50 kb read takes tens of ms
        # a pair buffer that is too small: the ticket stays valid
        deadline = time.monotonic() + 60
        while True:
            res = binding.Result()
            rc = srv.lib.abea_server_poll(srv.h, t, 100_000, res, None, 0, None)
            if rc != binding.ABEA_ERR_TIMEOUT:
                break
            assert time.monotonic() < deadline
        assert rc == binding.ABEA_ERR_CAPACITY and res.n_pairs > 0
        r, p, lat = srv.poll(t, wait_us=0)
        assert r["status"] == 0 and len(p) == res.n_pairs and lat > 0
        # a retired ticket and a ticket never issued are rejected
        for bad in (t, t + 12345):
            rc = srv.lib.abea_server_poll(srv.h, bad, 0, binding.Result(), None, 0, None)
            assert rc == binding.ABEA_ERR_ARG
    r1, p1 = ctx.align(*long_read.read(0), long_read.W)
    assert np.float32(r1["score"]) == np.float32(r["score"]) and np.array_equal(p1, p)


def test_queue_full(ctx, mix):
    batch = mix[0]
    ctx.set_model(batch.k, batch.model_mean, batch.model_stdv)
    with binding.Server(ctx, batch.W, max_requests=4) as srv:
        ts = [srv.submit(*batch.read(i)) for i in range(4)]
        with pytest.raises(binding.AbeaError) as ei:
            srv.submit(*batch.read(4))
        assert ei.value.code == binding.ABEA_ERR_CAPACITY
        got = collect(srv, dict(enumerate(ts)))
        assert all(g[0]["status"] == 0 for g in got.values())
        srv.submit(*batch.read(4))                          # room again
