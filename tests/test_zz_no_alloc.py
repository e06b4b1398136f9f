"""The allocation-free batch call (abea_align_batch_device_noalloc).

It serves callers that cannot call cudaMalloc (a plugin whose host
application already holds the device memory in its own pool, or a path on
which an allocation's implicit device synchronisation is not allowed).  Its
results must equal those of abea_align_batch_device on the same inputs, on
two calls in a row (the second call reuses the scratch array the first one
left behind).  The cases reach every part of its own working-set layout: the
4-word and 16-word records (W = 100, 200), the per-band move bytes (W = 128,
all 32 lanes live), the largest model (k = 7), a read long enough for block
mode, 4,000 short reads (more than the launch has warps, so that most are
walked two at a time) and a batch just under the 64 MiB working set.  This
file is collected last.
"""
import dataclasses

import numpy as np
import pytest

from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _device_inputs(batch, torch, dev):
    po = binding.pair_offsets(batch.n_events(), np.maximum(batch.n_kmers(), 1))
    d_seq = torch.from_numpy(batch.seq).to(dev)
    d_ev = torch.from_numpy(batch.events).to(dev)
    return po, d_seq, d_ev


def _noalloc(b, po, d_seq, d_ev, torch, dev, stream=None):
    out = torch.full((b.n * 24,), 0xAB, dtype=torch.uint8, device=dev)
    pairs = torch.full((int(po[-1]) * 2,), -7, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    binding.align_batch_device_noalloc(b.k, b.model_mean, b.model_stdv, b.n, b.W, d_seq, b.seq_off, d_ev,
                                       b.ev_off, b.scalings, out, pairs, po,
                                       stream=0 if stream is None else stream.cuda_stream)
    torch.cuda.synchronize(dev)
    return binding.results_from_bytes(out.cpu().numpy()), pairs.cpu().numpy().reshape(-1, 2)


def _device_call(b, po, d_seq, d_ev, torch, dev, stream):
    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        out = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
        pairs = torch.zeros(int(po[-1]) * 2, dtype=torch.int32, device=dev)
        ctx.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, out, pairs, po,
                               stream=stream.cuda_stream)
        stream.synchronize()
        return binding.results_from_bytes(out.cpu().numpy()), pairs.cpu().numpy().reshape(-1, 2)


def _same(got, got_pairs, want, want_pairs, po, tag):
    assert np.array_equal(got, want), tag               # scores bit-identical, as in the parity tests
    for i in range(len(want)):
        n = want["n_pairs"][i]
        assert np.array_equal(got_pairs[po[i]:po[i] + n], want_pairs[po[i]:po[i] + n]), (tag, i)


def _batch(case):
    if case == "w100_k6":
        return synth.make_batch("plain_64x1kb", n_reads=48)
    if case == "w200_k6":
        return synth.make_batch(dataclasses.replace(synth.WORKLOADS["plain_64x1kb"], W=200), n_reads=32)
    if case == "w128_k6":
        return synth.make_batch(dataclasses.replace(synth.WORKLOADS["plain_64x1kb"], W=128), n_reads=32)
    if case == "w100_k7":
        return synth.make_batch(dataclasses.replace(synth.WORKLOADS["plain_64x1kb"], k=7), n_reads=32)
    if case == "w100_k6_many_short":
        # more reads than the launch has warps, so that most are walked two at a time
        w = dataclasses.replace(synth.WORKLOADS["plain_64x1kb"], n_reads=4000, length=("fixed", 100))
        return synth.make_batch(w)
    if case == "w200_k7_block":
        # one read far longer than the rest: it runs in block mode (default theta = 1)
        w = dataclasses.replace(synth.WORKLOADS["batch_4096_ln5kb"], k=7, W=200)
        L = synth.read_lengths(w)
        ids = [int(np.argmax(L))] + [int(i) for i in np.argsort(L)[:23]]
        return synth.make_batch(w, read_ids=ids)
    raise ValueError(case)


@pytest.mark.parametrize("case", ["w100_k6", "w200_k6", "w128_k6", "w100_k7", "w200_k7_block", "w100_k6_many_short"])
def test_noalloc_matches_device_call_twice(case):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    b = _batch(case)
    po, d_seq, d_ev = _device_inputs(b, torch, dev)
    s = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)
    want, want_pairs = _device_call(b, po, d_seq, d_ev, torch, dev, s)
    assert np.all(want["status"] == 0)
    for call in range(2):
        got, got_pairs = _noalloc(b, po, d_seq, d_ev, torch, dev, s)
        _same(got, got_pairs, want, want_pairs, po, (case, call))


def test_noalloc_batch_just_under_the_working_set():
    """The largest prefix of the 4,096-read batch the 64 MiB working set admits (found by
    bisection on the reads; a rejected call does no work) equals the device call."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    full = synth.make_batch("batch_4096_ln5kb", n_reads=1024)

    def fits(n):
        b = full.subset(np.arange(n))
        po, d_seq, d_ev = _device_inputs(b, torch, dev)
        try:
            _noalloc(b, po, d_seq, d_ev, torch, dev)
            return True
        except binding.AbeaError as e:
            assert e.code == binding.ABEA_ERR_NOMEM
            return False

    lo, hi = 1, full.n
    assert fits(lo) and not fits(hi)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if fits(mid):
            lo = mid
        else:
            hi = mid
    b = full.subset(np.arange(lo))
    po, d_seq, d_ev = _device_inputs(b, torch, dev)
    s = torch.cuda.Stream(dev)
    want, want_pairs = _device_call(b, po, d_seq, d_ev, torch, dev, s)
    assert np.all(want["status"] == 0)
    got, got_pairs = _noalloc(b, po, d_seq, d_ev, torch, dev, s)
    _same(got, got_pairs, want, want_pairs, po, ("limit", lo))


def test_noalloc_rejects_oversized_batch():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    mm, ms = synth.make_model(6, 0)
    # 16385 reads: over the per-call read limit; rejected before any work
    n = 16385
    seq_off = np.arange(n + 1, dtype=np.int64) * 10
    ev_off = np.arange(n + 1, dtype=np.int64) * 10
    po = np.arange(n + 1, dtype=np.int64) * 20
    sc = np.ones((n, 3), np.float32)
    d = torch.zeros(16, dtype=torch.uint8, device=dev)
    with pytest.raises(binding.AbeaError) as e:
        binding.align_batch_device_noalloc(6, mm, ms, n, 100, d, seq_off, d.view(torch.float32), ev_off, sc, d,
                                           d.view(torch.int32), po)
    assert e.value.code == binding.ABEA_ERR_NOMEM
    # one read too long for the 64 MiB working set
    seq_off = np.array([0, 3_000_000], np.int64)
    ev_off = np.array([0, 5_000_000], np.int64)
    po = np.array([0, 8_000_000], np.int64)
    with pytest.raises(binding.AbeaError) as e:
        binding.align_batch_device_noalloc(6, mm, ms, 1, 100, d, seq_off, d.view(torch.float32), ev_off,
                                           np.ones((1, 3), np.float32), d, d.view(torch.int32), po)
    assert e.value.code == binding.ABEA_ERR_NOMEM
