"""GPU event detection (abea_detect_events) against the oracle: event counts,
starts and lengths identical, means and standard deviations bit-identical
(the same FP32 operations on the same exact integer sums)."""
import numpy as np
import pytest

from oracle import event_oracle as eo
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def run(raws, calib, window, tau2, caps=None, lead=0):
    """lead: samples (not part of any read) before the first read in the device array."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    raw = np.concatenate([np.full(lead, 999, np.int16)] + list(raws)).astype(np.int16)
    raw_off = np.full(len(raws) + 1, lead, np.int64)
    np.cumsum([len(r) for r in raws], out=raw_off[1:])
    raw_off[1:] += lead
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


def compare(raws, calib, window, tau2, caps=None, lead=0):
    evs, ev_off, counts = run(raws, calib, window, tau2, caps, lead)
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


TILE = 4096         # positions per tile of the device kernels


def test_starts_at_tile_edges():
    """Level changes on both sides of every tile edge (and exactly on it), reads one sample short of,
    exactly at and one past whole tiles; the windows and the local-maximum rule straddle the edges."""
    rng = np.random.default_rng(21)
    raws = []
    for n_tiles, delta in ((1, -1), (1, 0), (1, 1), (2, 0), (3, 5), (4, -3)):
        n = n_tiles * TILE + delta
        cuts = {0, n}
        for e in range(1, n_tiles + 1):
            for d in (-9, -4, 0, 3, 8):
                if 0 < e * TILE + d < n:
                    cuts.add(e * TILE + d)
        cuts |= set(int(c) for c in rng.integers(1, n, 40))
        cuts = sorted(cuts)
        x = np.zeros(n, np.int16)
        level = 500
        for u, v in zip(cuts[:-1], cuts[1:]):
            level += int(rng.choice([-1, 1])) * int(rng.integers(20, 200))
            x[u:v] = level
        x += rng.normal(0, 3, n).astype(np.int16)
        raws.append(x)
    calib = np.array([[0.5, 0.25]] * len(raws), np.float32)
    for w in (2, 3, 8):
        for tau2 in (0.0, 3.0):
            evs, counts = compare(raws, calib, w, tau2)
            assert counts.min() > 10


def test_offset_batch_and_long_read():
    """The batch starts at sample 7 of the device array; one read spans 30 tiles."""
    rb = synth.make_raw_batch("batch_4096_ln5kb", read_ids=range(0, 4096, 512))
    raws = [rb.signal(i) for i in range(rb.n)]
    rng = np.random.default_rng(4)
    long = np.repeat(rng.integers(100, 900, 9000), rng.integers(5, 22, 9000)).astype(np.int16)[:30 * TILE - 11]
    raws.append(long + rng.normal(0, 6, len(long)).astype(np.int16))
    calib = np.concatenate([rb.calib, [[1.0, 0.5]]]).astype(np.float32)
    compare(raws, calib, 3, 2.0, lead=7)


def test_integer_to_float_rounding():
    """The event kernels' own int64 -> float rounding against IEEE round-to-nearest-even (numpy's
    conversion on the host) and the platform's conversion on the device: every magnitude, the exact
    halfway cases with even and odd kept significands, and one above and below each."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(13)
    v = [np.arange(-70000, 70000, dtype=np.int64)]
    for e in range(24, 63):
        base = rng.integers(1 << 23, 1 << 24, 2000, dtype=np.int64) << (e - 23)
        half = np.int64(1) << (e - 24)
        v += [base, base + half, base - half, base + half + 1, base + half - 1, base + 1, base - 1,
              rng.integers(1 << e, (1 << e) * 2 - 1, 4000, dtype=np.int64)]
    v = np.concatenate(v)
    v = np.concatenate([v, -v[v > 0]])
    d_in = torch.from_numpy(v).to(dev)
    d_out = torch.empty(len(v), dtype=torch.float32, device=dev)
    binding.f32_from_i64(d_in, d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), v.astype(np.float32).view(np.uint32))
    assert np.array_equal(got.view(np.uint32), d_in.to(torch.float32).cpu().numpy().view(np.uint32))


def test_invalid_arguments_are_rejected():
    """Windows outside [2, 8], a negative or non-finite threshold, a non-finite calibration and
    offsets that go backwards are ABEA_ERR_ARG; nothing is launched."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    raw = torch.zeros(64, dtype=torch.int16, device=dev)
    d_ev = torch.zeros(64 * 16, dtype=torch.uint8, device=dev)
    d_n = torch.zeros(2, dtype=torch.int32, device=dev)
    ro = np.array([0, 30, 64], np.int64)
    eo = np.array([0, 20, 40], np.int64)
    cal = np.array([[0.0, 1.0], [0.0, 1.0]], np.float32)
    bad_cal = cal.copy()
    bad_cal[1, 1] = np.nan
    cases = [(ro, cal, 1, 2.0), (ro, cal, 9, 2.0), (ro, cal, 3, -1.0), (ro, cal, 3, float("inf")),
             (ro, bad_cal, 3, 2.0), (np.array([0, 40, 30], np.int64), cal, 3, 2.0)]
    with binding.Context(0) as ctx:
        for r_off, c, w, tau2 in cases:
            with pytest.raises(binding.AbeaError) as ei:
                ctx.detect_events(2, raw, r_off, c, w, tau2, d_ev, eo, d_n)
            assert ei.value.code == binding.ABEA_ERR_ARG, (w, tau2)
