"""GPU: calls on one context never wait for work of another context.

abea_set_model replaces the model rows of its own context only after that
context's last batch; it must not synchronise the device, so a long batch
running on another context (on another stream) keeps running while it
returns.  The long batch is a few of the longest reads of the 50,000-read
workload (about 200 kb each, one warp per read), which run for tens of
milliseconds.
"""
import time

import numpy as np
import pytest

from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def test_set_model_does_not_wait_for_another_context():
    torch = pytest.importorskip("torch")
    w = synth.WORKLOADS["large_50k_ln8kb"]
    L = synth.read_lengths(w)
    b = synth.make_batch(w, read_ids=np.argsort(-L)[:4])
    dev = torch.device("cuda", 0)
    pair_off = binding.pair_offsets(b.n_events(), np.maximum(b.n_kmers(), 1))
    d_seq = torch.from_numpy(b.seq).to(dev)
    d_ev = torch.from_numpy(b.events).to(dev)
    d_out = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
    d_pairs = torch.zeros(int(pair_off[-1]) * 2, dtype=torch.int32, device=dev)
    st = torch.cuda.Stream(dev)
    with binding.Context(0) as busy, binding.Context(0) as other:
        busy.set_model(b.k, b.model_mean, b.model_stdv)
        other.set_model(b.k, b.model_mean, b.model_stdv)
        # warm-up (kernel loading, buffer growth), then the timed batch
        busy.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_out, d_pairs, pair_off,
                                stream=st.cuda_stream)
        torch.cuda.synchronize(dev)
        ref_out = d_out.clone()
        ref_pairs = d_pairs.clone()
        d_out.zero_()
        d_pairs.zero_()
        torch.cuda.synchronize(dev)
        t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_start.record(st)
        busy.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_out, d_pairs, pair_off,
                                stream=st.cuda_stream)
        t_end.record(st)
        t0 = time.perf_counter()
        other.set_model(b.k, b.model_mean[::-1].copy(), b.model_stdv)
        dt_ms = 1e3 * (time.perf_counter() - t0)
        still_running = not t_end.query()
        t_end.synchronize()
        batch_ms = t_start.elapsed_time(t_end)
        assert batch_ms > 10.0, batch_ms                 # the batch is long enough to tell
        assert still_running, (dt_ms, batch_ms)         # set_model returned while the batch ran
        assert dt_ms < 0.5 * batch_ms, (dt_ms, batch_ms)
        assert torch.equal(d_out, ref_out) and torch.equal(d_pairs, ref_pairs)
        res = binding.results_from_bytes(d_out.cpu().numpy())
        assert np.all(res["status"] == binding.READ_OK)
