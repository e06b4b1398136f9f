"""GPU per-read scaling estimate (abea_estimate_scalings) against the FP64
oracle: statuses equal; scale and shift equal to the oracle's values rounded
to float, within one float ulp (the sums run in another order)."""
import numpy as np
import pytest

from oracle import scalings_oracle as so
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def run(batch):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    with binding.Context(0) as ctx:
        ctx.set_model(batch.k, batch.model_mean, batch.model_stdv)
        d_seq = torch.from_numpy(np.ascontiguousarray(batch.seq)).to(dev)
        d_ev = torch.from_numpy(np.ascontiguousarray(batch.events)).to(dev)
        d_out = torch.zeros(batch.n * 3, dtype=torch.float32, device=dev)
        d_st = torch.full((batch.n,), -1, dtype=torch.int32, device=dev)
        s = torch.cuda.Stream(dev)
        ctx.estimate_scalings(batch.n, d_seq, batch.seq_off, d_ev, batch.ev_off, d_out, d_st, stream=s.cuda_stream)
        s.synchronize()
        return d_out.cpu().numpy().reshape(-1, 3), d_st.cpu().numpy()


def compare(batch):
    out, st = run(batch)
    scale, shift, status = so.estimate_batch(batch)
    assert np.array_equal(st, status)
    for got, want in ((out[:, 0], scale), (out[:, 1], shift)):
        want32 = want.astype(np.float32)
        ulp = np.spacing(np.abs(want32))
        assert np.all(np.abs(got - want32) <= ulp), np.max(np.abs(got - want32) / ulp)
    assert np.all(out[:, 2] == 1.0)
    return out, st


def test_plain_reads():
    compare(synth.make_batch("plain_64x1kb"))


def test_batch_sample_and_recovery_of_true_scalings():
    w = synth.WORKLOADS["batch_4096_ln5kb"]
    b = synth.make_batch(w, read_ids=range(0, w.n_reads, 8))
    out, st = compare(b)
    assert np.all(st == binding.SCALE_OK)
    # the generator's scalings are recovered up to the event noise and the dwell weighting
    true = b.scalings
    assert np.median(np.abs(out[:, 0] / true[:, 0] - 1)) < 0.02
    assert np.median(np.abs(out[:, 1] - true[:, 1])) < 3.0


def test_degenerate_and_rejected_reads():
    mm, ms = synth.make_model(3, 9)
    ev_ok = np.array([80.0, 95.0, 101.0, 120.0, 77.0], np.float32)
    cases = [
        (ev_ok, b"ACGTTGCA"),                    # fine
        (ev_ok, b"AAAAAAAA"),                    # one rank: no level variance
        (ev_ok[:1], b"ACGTTGCA"),                # one event
        (np.full(4, 90.0, np.float32), b"ACGTTGCA"),   # constant events
        (ev_ok, b"ACGNTGCA"),                    # bad base
        (np.array([80.0, np.nan], np.float32), b"ACGTTGCA"),
        (ev_ok[:0], b"ACGTTGCA"),                # no event
        (ev_ok, b"AC"),                          # shorter than k
    ]
    b = synth.custom_batch([c[0] for c in cases], [c[1] for c in cases], [(1.0, 0.0, 1.0)] * len(cases), mm, ms, 3,
                           100)
    out, st = compare(b)
    assert list(st) == [binding.SCALE_OK, binding.SCALE_DEGENERATE, binding.SCALE_DEGENERATE,
                        binding.SCALE_DEGENERATE] + [binding.SCALE_BAD_INPUT] * 4
