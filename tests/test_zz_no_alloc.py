"""The allocation-free batch call (abea_align_batch_device_noalloc).

It serves callers that cannot call cudaMalloc (a plugin whose host
application already holds the device memory in its own pool, or a path on
which an allocation's implicit device synchronisation is not allowed).  Its
results must equal those of abea_align_batch_device on the same inputs, on
two calls in a row (the second call reuses the scratch array the first one
left behind).  This file is collected last.
"""
import numpy as np
import pytest

from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _device_inputs(batch, torch, dev):
    po = binding.pair_offsets(batch.n_events(), np.maximum(batch.n_kmers(), 1))
    d_seq = torch.from_numpy(batch.seq).to(dev)
    d_ev = torch.from_numpy(batch.events).to(dev)
    return po, d_seq, d_ev


def test_noalloc_matches_device_call_twice():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    b = synth.make_batch("plain_64x1kb", n_reads=48)
    po, d_seq, d_ev = _device_inputs(b, torch, dev)
    s = torch.cuda.Stream(dev)
    torch.cuda.synchronize(dev)

    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        out = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
        pairs = torch.zeros(int(po[-1]) * 2, dtype=torch.int32, device=dev)
        ctx.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, out, pairs, po,
                               stream=s.cuda_stream)
        s.synchronize()
        want = binding.results_from_bytes(out.cpu().numpy())
        want_pairs = pairs.cpu().numpy().reshape(-1, 2)
    assert np.all(want["status"] == 0)

    for call in range(2):
        out2 = torch.full((b.n * 24,), 0xAB, dtype=torch.uint8, device=dev)
        pairs2 = torch.full((int(po[-1]) * 2,), -7, dtype=torch.int32, device=dev)
        torch.cuda.synchronize(dev)
        binding.align_batch_device_noalloc(b.k, b.model_mean, b.model_stdv, b.n, b.W, d_seq, b.seq_off, d_ev,
                                           b.ev_off, b.scalings, out2, pairs2, po, stream=s.cuda_stream)
        s.synchronize()
        got = binding.results_from_bytes(out2.cpu().numpy())
        got_pairs = pairs2.cpu().numpy().reshape(-1, 2)
        assert np.array_equal(got, want), call          # scores bit-identical, as in the parity tests
        for i in range(b.n):
            n = want["n_pairs"][i]
            assert np.array_equal(got_pairs[po[i]:po[i] + n], want_pairs[po[i]:po[i] + n]), (call, i)


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
