"""GPU event detection (abea_detect_events) against the oracle: event counts,
starts and lengths identical, means and standard deviations bit-identical
(the same FP32 operations on the same exact integer sums)."""
import numpy as np
import pytest

from oracle import event_oracle as eo
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def run(raws, calib, window, tau2, caps=None):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    raw = np.concatenate(raws).astype(np.int16) if raws else np.zeros(0, np.int16)
    raw_off = np.zeros(len(raws) + 1, np.int64)
    np.cumsum([len(r) for r in raws], out=raw_off[1:])
    if caps is None:
        caps = [len(r) // window + 2 for r in raws]
    ev_off = np.zeros(len(raws) + 1, np.int64)
    np.cumsum(caps, out=ev_off[1:])
    with binding.Context(0) as ctx:
        d_raw = torch.from_numpy(raw if len(raw) else np.zeros(1, np.int16)).to(dev)
        d_ev = torch.zeros(max(int(ev_off[-1]), 1) * 16, dtype=torch.uint8, device=dev)
        d_n = torch.full((len(raws),), -1, dtype=torch.int32, device=dev)
        s = torch.cuda.Stream(dev)
        ctx.detect_events(len(raws), d_raw, raw_off, calib, window, tau2, d_ev, ev_off, d_n, stream=s.cuda_stream)
        s.synchronize()
        evs = np.frombuffer(d_ev.cpu().numpy().tobytes(), binding.EVENT_DTYPE)
        return evs, ev_off, d_n.cpu().numpy()


def compare(raws, calib, window, tau2, caps=None):
    evs, ev_off, counts = run(raws, calib, window, tau2, caps)
    for i, x in enumerate(raws):
        m, s, a, L = eo.detect(x, window, tau2, calib[i])
        assert counts[i] == len(m), (i, counts[i], len(m))
        k = min(len(m), int(ev_off[i + 1] - ev_off[i]))
        g = evs[ev_off[i]:ev_off[i] + k]
        assert np.array_equal(g["start"], a[:k]) and np.array_equal(g["length"], L[:k])
        assert np.array_equal(g["mean"], m[:k]) and np.array_equal(g["stdv"], s[:k])
    return evs, counts


def test_synthetic_reads_default_detector():
    rb = synth.make_raw_batch("batch_4096_ln5kb", read_ids=range(0, 4096, 32))
    raws = [rb.signal(i) for i in range(rb.n)]
    evs, counts = compare(raws, rb.calib, 3, 2.0)
    kmers = rb.seq_off[1:] - rb.seq_off[:-1] - rb.k + 1
    assert 1.3 < counts.sum() / kmers.sum() < 2.2          # over-segmentation as the thesis describes


@pytest.mark.parametrize("window", [2, 4, 5, 6, 7, 8])
def test_windows(window):
    rb = synth.make_raw_batch("plain_64x1kb", n_reads=12)
    compare([rb.signal(i) for i in range(rb.n)], rb.calib, window, 4.0)


def test_edge_cases():
    rng = np.random.default_rng(8)
    steps = np.repeat(rng.integers(100, 900, 30), rng.integers(4, 20, 30)).astype(np.int16)
    raws = [np.zeros(0, np.int16),                                  # empty
            np.array([7], np.int16), np.array([5, 9, 7, 1, 3], np.int16),   # shorter than two windows
            np.full(200, 321, np.int16),                            # constant: no start
            steps,                                                  # noiseless steps
            np.tile(np.array([100, 300], np.int16), 150),           # alternating
            rng.integers(-32768, 32767, 5000).astype(np.int16)]     # full-range noise
    calib = np.array([[1.5, 0.2]] * len(raws), np.float32)
    for tau2 in (0.0, 2.0, 100.0):
        compare(raws, calib, 3, tau2)


def test_capacity_shorter_than_needed():
    rb = synth.make_raw_batch("plain_64x1kb", n_reads=4)
    raws = [rb.signal(i) for i in range(rb.n)]
    full = [len(eo.detect(x, 3, 2.0, rb.calib[i])[0]) for i, x in enumerate(raws)]
    caps = [f // 2 for f in full]
    evs, counts = compare(raws, rb.calib, 3, 2.0, caps)
    assert list(counts) == full
