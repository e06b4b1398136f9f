"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bar: per-read status, end event, in-matrix cell count and the pair list are
identical to the FP32 oracle's; the FP32 score is bit-identical to the FP32
oracle's (both take every decision on the same FP32 values) and within 1e-4
relative of the FP64 oracle's.
"""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def ctx():
    c = binding.Context(0)
    yield c
    c.close()


# block mode for every read a block can take (one per block, longest first)
ALL_BLOCK = 1e-9


def run_gpu(ctx, batch, W=None, theta=1.0, **kw):
    ctx.set_model(batch.k, batch.model_mean, batch.model_stdv)
    ctx.set_block_mode(theta)
    try:
        return ctx.align_packed(batch, W=W, **kw)
    finally:
        ctx.set_block_mode(1.0)


def gpu_pairs(pairs, pair_off, res, i):
    return pairs[pair_off[i]:pair_off[i] + res["n_pairs"][i]]


def compare(batch, res, pairs, pair_off, W=None, check_f64=True, ids=None):
    """Compare GPU results of `batch` with the oracle (all reads, or `ids`)."""
    W = batch.W if W is None else W
    sub = batch if ids is None else batch.subset(ids)
    idx = np.arange(batch.n) if ids is None else np.asarray(ids)
    o32 = oracle.abea_batch(sub, "f32", n_threads=THREADS, W=W)
    o64 = oracle.abea_batch(sub, "f64", n_threads=THREADS, W=W) if check_f64 else None
    bad = []
    for t, i in enumerate(idx):
        st = int(res["status"][i])
        if st != int(o32["status"][t]):
            bad.append((i, "status", st, int(o32["status"][t])))
            continue
        if st != oracle.ST_OK:
            continue
        if np.float32(o32["score"][t]) != res["score"][i]:
            bad.append((i, "score", float(res["score"][i]), o32["score"][t]))
        if int(res["e_end"][i]) != int(o32["e_end"][t]) or int(res["cells"][i]) != int(o32["cells"][t]):
            bad.append((i, "e_end/cells", int(res["e_end"][i]), int(o32["e_end"][t]), int(res["cells"][i]),
                        int(o32["cells"][t])))
        a = gpu_pairs(pairs, pair_off, res, i)
        b = o32["pairs"][o32["pair_off"][t]:o32["pair_off"][t] + o32["n_pairs"][t]]
        if not np.array_equal(a, b):
            bad.append((i, "pairs", len(a), len(b)))
        if o64 is not None and o64["status"][t] == oracle.ST_OK:
            rel = abs(float(res["score"][i]) - o64["score"][t]) / abs(o64["score"][t])
            if rel > 1e-4:
                bad.append((i, "f64", rel))
    assert not bad, bad[:10]
    return o32, o64


def test_plain_64x1kb(ctx):
    b = synth.make_batch("plain_64x1kb")
    res, pairs, po = run_gpu(ctx, b)
    assert np.all(res["status"] == 0)
    compare(b, res, pairs, po)


def _lengths_batch(lengths, k=6, W=100, seed=5, dwell_mean=1.8):
    w = synth.Workload("ragged", len(lengths), k, W, seed, ("fixed", 1), dwell_mean=dwell_mean)
    mm, ms = synth.make_model(k, seed)
    reads = [synth.make_read(w, r, max(L, 1), mm, ms) for r, L in enumerate(lengths)]
    seqs = [r[0][:L].tobytes() for r, L in zip(reads, lengths)]
    return synth.custom_batch([r[1] for r in reads], seqs, [r[2] for r in reads], mm, ms, k, W)


def test_ragged_lengths(ctx):
    lengths = [6, 7, 8, 10, 20, 49, 50, 51, 52, 99, 100, 101, 102, 103, 150, 151, 300, 999, 1000, 2500, 3001]
    b = _lengths_batch(lengths)
    res, pairs, po = run_gpu(ctx, b)
    compare(b, res, pairs, po)


# 30, 60, 120: two lanes above the band (L = 30); 31, 61, 62, 93, 121, 124: one lane above it (L = 31)
@pytest.mark.parametrize("W", [2, 3, 4, 5, 7, 16, 30, 31, 32, 33, 50, 60, 61, 62, 63, 64, 65, 93, 100, 101, 120, 121,
                               124, 127, 128, 129, 160, 200, 201, 255, 256])
def test_band_widths(ctx, W):
    lengths = [6, 9, 30, 80, 150, 260, 420, 700]
    b = _lengths_batch(lengths, W=W, seed=W)
    res, pairs, po = run_gpu(ctx, b, W=W)
    compare(b, res, pairs, po, W=W)


# one width per (lanes, offsets per lane) combination that block mode has
@pytest.mark.parametrize("W", [32, 36, 64, 72, 96, 100, 128, 144, 160, 192, 200, 224, 248])
def test_block_mode_band_widths(ctx, W):
    """Block mode (the four warps of a block share a read) on every read,
    and per-warp mode only, both against the oracle."""
    lengths = [6, 9, 30, 80, 150, 260, 420, 700, 1500]
    b = _lengths_batch(lengths, W=W, seed=300 + W)
    res, pairs, po = run_gpu(ctx, b, W=W, theta=ALL_BLOCK)
    compare(b, res, pairs, po, W=W, check_f64=False)
    res0, pairs0, po0 = run_gpu(ctx, b, W=W, theta=0.0)
    assert np.array_equal(res, res0)
    assert np.array_equal(pairs, pairs0)


def test_block_mode_long_reads(ctx):
    """Long reads in block mode (renormalisation, walks across many trace
    chunks) next to short ones in the same launch."""
    w = synth.WORKLOADS["batch_4096_ln5kb"]
    L = synth.read_lengths(w)
    ids = sorted(set(np.argsort(-L)[:2].tolist()) | {0, 1, 2, 3})     # two 50 kb reads and four others
    b = synth.make_batch(w, read_ids=ids)
    for theta in (ALL_BLOCK, 1.0, 0.0):
        res, pairs, po = run_gpu(ctx, b, theta=theta)
        assert np.all(res["status"] == 0)
        compare(b, res, pairs, po, check_f64=False)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 7, 9])
def test_kmer_sizes(ctx, k):
    lengths = [k, k + 1, 40, 300, 900]
    b = _lengths_batch(lengths, k=k, seed=10 + k)
    res, pairs, po = run_gpu(ctx, b)
    compare(b, res, pairs, po)


@pytest.mark.parametrize("theta", [1.0, ALL_BLOCK])
def test_bad_inputs_and_neighbours(ctx, theta):
    good = _lengths_batch([300, 500, 700], seed=3)
    ev, sq, sc = [], [], []
    for i in range(good.n):
        e, s, c = good.read(i)
        ev.append(e)
        sq.append(s)
        sc.append(c)
    e0, s0, c0 = ev[0], sq[0], sc[0]
    bad_seq = s0[:50] + b"N" + s0[51:]
    nan_ev = e0.copy()
    nan_ev[7] = np.nan
    inf_ev = e0.copy()
    inf_ev[-1] = np.inf
    cases = [(e0, bad_seq, c0), (nan_ev, s0, c0), (inf_ev, s0, c0), (e0, s0, (1.0, 0.0, 0.0)),
             (e0[:0], s0, c0), (e0, s0[:5], c0), (e0, s0, (np.nan, 0.0, 1.0))]
    all_ev = [ev[1]] + [c[0] for c in cases] + [ev[2]]
    all_sq = [sq[1]] + [c[1] for c in cases] + [sq[2]]
    all_sc = [sc[1]] + [c[2] for c in cases] + [sc[2]]
    b = synth.custom_batch(all_ev, all_sq, all_sc, good.model_mean, good.model_stdv, good.k, good.W)
    res, pairs, po = run_gpu(ctx, b, theta=theta)
    assert res["status"][0] == 0 and res["status"][-1] == 0
    assert np.all(res["status"][1:-1] == binding.READ_BAD_INPUT), res["status"]
    assert np.all(np.isneginf(res["score"][1:-1]))
    compare(b, res, pairs, po, ids=[0, b.n - 1])


@pytest.mark.parametrize("theta", [1.0, ALL_BLOCK])
def test_capacity(ctx, theta):
    b = _lengths_batch([200, 400, 600], seed=8)
    o = oracle.abea_batch(b, "f32", n_threads=THREADS)
    need = o["n_pairs"]
    caps = need.astype(np.int64).copy()
    caps[1] = need[1] - 1                        # one pair short
    po = np.zeros(b.n + 1, np.int64)
    np.cumsum(caps, out=po[1:])
    res, pairs, po = run_gpu(ctx, b, pair_off=po, theta=theta)
    assert res["status"][1] == binding.READ_CAPACITY and res["n_pairs"][1] == need[1]
    assert res["status"][0] == 0 and res["status"][2] == 0
    for i in (0, 2):
        assert np.array_equal(gpu_pairs(pairs, po, res, i), o["pairs"][o["pair_off"][i]:o["pair_off"][i] + need[i]])
    # the single-read call reports the shortfall as ABEA_ERR_CAPACITY
    ctx.set_model(b.k, b.model_mean, b.model_stdv)
    e, s, c = b.read(1)
    import ctypes
    ev = np.ascontiguousarray(e, np.float32)
    sq = np.frombuffer(s, np.uint8).copy()
    rd = binding.Read(binding._p(ev).value, len(ev), binding._p(sq).value, len(sq), binding.Scalings(*c))
    out = binding.Result()
    buf = np.zeros((need[1], 2), np.int32)
    rc = ctx.lib.abea_align(ctx.h, ctypes.byref(rd), b.W, ctypes.byref(out), binding._p(buf), int(need[1]) - 1)
    assert rc == binding.ABEA_ERR_CAPACITY and out.n_pairs == need[1]


def test_extreme_events(ctx):
    # events far outside the model: the FP32 emission overflows to -inf
    # (z^2 > 3.4e38), leaving only trim/skip paths for those cells; every
    # finite event, up to the largest float, is aligned (no BAD_INPUT)
    rng = np.random.default_rng(4)
    base = _lengths_batch([40, 60, 90, 200, 400], seed=44)
    evs, sqs, scs = [], [], []
    for i in range(base.n):
        e, s, c = base.read(i)
        e = e.copy()
        pos = rng.choice(len(e), max(1, len(e) // 10), replace=False)
        e[pos] = rng.choice(np.array([1e20, -1e20, 3e4, -3e4], np.float32), len(pos))
        # finite events just below the largest float are aligned like any other event
        e[rng.choice(len(e), 1)] = np.float32(3.2e38) if i % 2 else np.float32(-np.finfo(np.float32).max)
        evs.append(e)
        sqs.append(s)
        scs.append(c)
    b = synth.custom_batch(evs, sqs, scs, base.model_mean, base.model_stdv, base.k, base.W)
    for W, theta in ((3, 1.0), (100, 1.0), (100, ALL_BLOCK)):
        res, pairs, po = run_gpu(ctx, b, W=W, theta=theta)
        compare(b, res, pairs, po, W=W, check_f64=False)


def test_single_read_call_matches_batch(ctx):
    b = synth.make_batch("plain_64x1kb", n_reads=3)
    res, pairs, po = run_gpu(ctx, b)
    for i in range(b.n):
        e, s, c = b.read(i)
        r1, p1 = ctx.align(e, s, c, b.W)
        assert r1["status"] == 0 and np.float32(r1["score"]) == res["score"][i]
        assert np.array_equal(p1, gpu_pairs(pairs, po, res, i))


def test_align_batch_records(ctx):
    b = synth.make_batch("plain_64x1kb", n_reads=5)
    res, pairs, po = run_gpu(ctx, b)
    evs, sqs, scs = zip(*[b.read(i) for i in range(b.n)])
    r2, p2, po2 = ctx.align_batch(list(evs), list(sqs), list(scs), b.W)
    assert np.array_equal(res, r2)
    for i in range(b.n):
        assert np.array_equal(gpu_pairs(pairs, po, res, i), gpu_pairs(p2, po2, r2, i))


def test_device_api_matches_host_api(ctx):
    torch = pytest.importorskip("torch")
    b = synth.make_batch("plain_64x1kb", n_reads=20)
    res, pairs, po = run_gpu(ctx, b)
    dev = torch.device("cuda", 0)
    d_seq = torch.from_numpy(b.seq).to(dev)
    d_ev = torch.from_numpy(b.events).to(dev)
    d_out = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
    d_pairs = torch.zeros(int(po[-1]) * 2, dtype=torch.int32, device=dev)
    torch.cuda.synchronize(dev)
    s = torch.cuda.Stream(dev)            # a real stream: NULL would select the context's own stream
    ctx.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_out, d_pairs, po,
                           stream=s.cuda_stream)
    s.synchronize()
    r2 = binding.results_from_bytes(d_out.cpu().numpy())
    p2 = d_pairs.cpu().numpy().reshape(-1, 2)
    assert np.array_equal(res, r2)
    for i in range(b.n):
        assert np.array_equal(gpu_pairs(pairs, po, res, i), gpu_pairs(p2, po, r2, i))


def test_memory_budget_waves():
    b = synth.make_batch("plain_64x1kb", n_reads=24)
    with binding.Context(0) as big:
        r1, p1, po1 = run_gpu(big, b)
    # a budget of roughly three reads' working set (~130 KB each) forces many waves
    with binding.Context(0, mem_budget_bytes=400_000) as small:
        r2, p2, po2 = run_gpu(small, b)
        launches, _ = small.last_launch_stats()
    assert launches >= 2 * 6            # a pre-kernel and a core kernel per wave
    assert np.array_equal(r1, r2)
    assert np.array_equal(p1, p2)


def test_batch_4096_ln5kb_full(ctx):
    """The one-launch batch workload at full size: every read against the FP32
    oracle (FP64 on a sample)."""
    b = synth.make_batch("batch_4096_ln5kb")
    res, pairs, po = run_gpu(ctx, b)
    assert np.all(res["status"] == 0)
    compare(b, res, pairs, po, check_f64=False)
    rng = np.random.default_rng(0)
    sample = sorted(set(rng.choice(b.n, 48, replace=False).tolist()) | {int(np.argmax(b.n_events()))})
    compare(b, res, pairs, po, ids=sample)


def test_batch_4096_ln5kb_against_fp64(ctx):
    """The whole one-launch batch against the FP64 oracle (the accuracy
    reference; the FP32 oracle above shares the kernel's canonical form).
    Near-tie reads are those whose FP64 run took a decision (a traced cell's
    three-way maximum, a band move or the end cell) by less than 1e-3.  On
    every other read the GPU path equals the FP64 path element by element.
    On every read the score is within 1e-4 relative of FP64, and the GPU
    path, scored in FP64, is within 1e-3 of the FP64 optimum: where a
    near-tie lets the paths differ, the GPU's is optimal up to the tie."""
    from oracle import rescore
    b = synth.make_batch("batch_4096_ln5kb")
    res, pairs, po = run_gpu(ctx, b)
    assert np.all(res["status"] == 0)
    o64 = oracle.abea_batch(b, "f64", n_threads=THREADS)
    acc = rescore.accuracy_against_fp64(b, res, pairs, po, o64)
    print("accuracy against FP64:", acc)
    assert acc["reads"] == b.n
    assert acc["path_mismatch_non_tie"] == 0, acc
    assert acc["max_rel_err_fp64"] <= 1e-4, acc
    assert acc["max_fp64_gap_of_path"] <= 1e-3, acc
    assert 0.0 < acc["near_tie_frac"] < 0.9, acc


def test_wide_k9_w200_sample(ctx):
    w = synth.WORKLOADS["wide_10k_ln10kb_k9_w200"]
    b = synth.make_batch(w, read_ids=range(0, w.n_reads, w.n_reads // 40))
    res, pairs, po = run_gpu(ctx, b)
    assert np.all(res["status"] == 0)
    compare(b, res, pairs, po)


def test_large_workload_sample_with_ultra_long_reads(ctx):
    """Reads of the 50,000-read workload, the three longest (about 200 kb, half a
    million bands) among them, in one launch and then in memory-budget waves;
    every read against the FP32 oracle."""
    w = synth.WORKLOADS["large_50k_ln8kb"]
    L = synth.read_lengths(w)
    ids = sorted(set(np.argsort(-L)[:3].tolist()) | set(range(0, w.n_reads, w.n_reads // 12)))
    b = synth.make_batch(w, read_ids=ids)
    res, pairs, po = run_gpu(ctx, b)
    assert np.all(res["status"] == 0)
    compare(b, res, pairs, po, check_f64=False)
    # the same reads under a budget that forces several waves (the longest read alone needs ~40 MB)
    with binding.Context(0, mem_budget_bytes=64 << 20) as small:
        r2, p2, po2 = run_gpu(small, b)
        launches, _ = small.last_launch_stats()
    assert launches >= 4
    assert np.array_equal(res, r2) and np.array_equal(pairs, p2)


def test_prep_double_to_float_rounding():
    """The pre-kernel rounds its FP64 k-mer operands to float with integer operations
    (abea_f32_from_f64): identical to numpy's cast and to the device's own conversion on every
    binade of the float range, on halfway cases with even and odd kept significands (and one unit
    above and below), on carries into the exponent and past the largest float, on the
    subnormal, zero, infinite and NaN inputs that take the conversion instruction, and on the
    pre-kernel's own operand ranges."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(17)
    u = []
    for e in range(1023 - 130, 1023 + 131):
        m = rng.integers(0, 1 << 23, 400, dtype=np.uint64)
        for rest in (0x10000000, 0x0FFFFFFF, 0x10000001, 0, 0x1FFFFFFF):
            u.append((np.uint64(e) << np.uint64(52)) | (m << np.uint64(29)) | np.uint64(rest))
        u.append((np.uint64(e) << np.uint64(52)) | rng.integers(0, 1 << 52, 2000, dtype=np.uint64))
        u.append((np.uint64(e) << np.uint64(52)) | (np.uint64(0x7FFFFF) << np.uint64(29)) | np.uint64(0x10000000))
    u = np.concatenate([np.atleast_1d(x) for x in u])
    v = u.view(np.float64)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, 1e-310, 3.4028234663852886e38,
                        3.4028235677973366e38, 1.1754943508222875e-38, 1.1754942e-38], np.float64)
    # the pre-kernel's operands: a = sqrt(1/2)/sigma', b = -mu'*a, c = ln(1/sqrt(2 pi)) - ln sigma' + lp_step
    ops = np.concatenate([0.7071067811865476 / rng.uniform(1, 4.5, 20000),
                          -rng.uniform(50, 150, 20000) * (0.7071067811865476 / rng.uniform(1, 4.5, 20000)),
                          -0.9189385332046727 - np.log(rng.uniform(1, 4.5, 20000)) + rng.uniform(-2, -0.05, 20000)])
    v = np.concatenate([v, -v, special, ops])
    d_in = torch.from_numpy(v).to(dev)
    d_out = torch.empty(len(v), dtype=torch.float32, device=dev)
    binding.f32_from_f64(d_in, d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint32)
    with np.errstate(over="ignore"):
        want = v.astype(np.float32)
    nan = np.isnan(want)
    assert np.array_equal(got[~nan], want[~nan].view(np.uint32))
    assert np.all(np.isnan(got[nan].view(np.float32)))
    dev_cast = d_in.to(torch.float32).cpu().numpy()
    assert np.array_equal(got[~nan], dev_cast[~nan].view(np.uint32))


def test_paired_walks_with_rejected_and_short_slots(ctx):
    """8,000 short reads (far more than the launch's warps), so that most reads are walked two at
    a time: every 97th read is rejected (a non-ACGT base), every 89th has one pair slot too few,
    and the lengths vary so that a walk's partner is shorter or longer.  Statuses, scores,
    end events, cell counts and pairs equal the FP32 oracle's (rejected and short-slot reads by
    status and pair count)."""
    rng = np.random.default_rng(21)
    lengths = rng.integers(150, 700, 8000).tolist()
    b = _lengths_batch(lengths, seed=13)
    ev, sq, sc = [], [], []
    for i in range(b.n):
        e, s, c = b.read(i)
        if i % 97 == 5:
            s = s[:40] + b"N" + s[41:]
        ev.append(e)
        sq.append(s)
        sc.append(c)
    b = synth.custom_batch(ev, sq, sc, b.model_mean, b.model_stdv, b.k, b.W)
    o = oracle.abea_batch(b, "f32", n_threads=THREADS)
    short = np.arange(b.n) % 89 == 3
    short &= o["status"] == oracle.ST_OK
    caps = np.maximum(b.n_events() + np.maximum(b.n_kmers(), 1) - 1, 1).astype(np.int64)
    caps[short] = o["n_pairs"][short] - 1
    po = np.zeros(b.n + 1, np.int64)
    np.cumsum(caps, out=po[1:])
    res, pairs, po = run_gpu(ctx, b, pair_off=po, theta=0.0)
    rejected = np.arange(b.n) % 97 == 5
    assert np.all(res["status"][rejected] == binding.READ_BAD_INPUT)
    assert np.all(res["status"][short] == binding.READ_CAPACITY)
    assert np.array_equal(res["n_pairs"][short], o["n_pairs"][short])
    ok = ~rejected & ~short
    assert np.all(res["status"][ok] == o["status"][ok])
    bad = []
    for i in np.nonzero(ok & (o["status"] == oracle.ST_OK))[0]:
        if np.float32(o["score"][i]) != res["score"][i] or res["e_end"][i] != o["e_end"][i] or \
                res["cells"][i] != o["cells"][i]:
            bad.append((int(i), "result"))
        elif not np.array_equal(gpu_pairs(pairs, po, res, i),
                                o["pairs"][o["pair_off"][i]:o["pair_off"][i] + o["n_pairs"][i]]):
            bad.append((int(i), "pairs"))
    assert not bad, bad[:10]


def test_block_mode_then_paired_walks(ctx):
    """A launch that starts with block-mode reads (the four longest, one per block) and then walks
    the remaining 5,000 short reads mostly two at a time (warp 0 of those blocks reuses the region
    its block-mode walk used): every read equals the FP32 oracle."""
    rng = np.random.default_rng(23)
    lengths = [9000, 8500, 8000, 7500] + rng.integers(120, 400, 5000).tolist()
    b = _lengths_batch(lengths, seed=19)
    res, pairs, po = run_gpu(ctx, b, theta=ALL_BLOCK)
    assert np.all(res["status"] == 0)
    compare(b, res, pairs, po, check_f64=False)


# (events, bases) of reads whose band leaves the matrix early on one side, and tiny near-square ones
DEGENERATE_SHAPES = [(1, 6), (1, 7), (1, 60), (1, 400), (2, 6), (2, 105), (3, 300), (3, 1000), (40, 6),
                     (500, 6), (2000, 7), (150, 8), (5, 5000), (7, 7), (8, 13), (120, 110)]


def _degenerate_batch(k=6, W=100, seed=41):
    mm, ms = synth.make_model(k, 31)
    rng = np.random.default_rng(seed)
    events, seqs, sc = [], [], []
    for n_e, L in DEGENERATE_SHAPES:
        seqs.append(rng.choice(np.frombuffer(b"ACGT", np.uint8), L).tobytes())
        events.append(rng.uniform(60.0, 130.0, n_e).astype(np.float32))
        sc.append((1.0, 0.0, 1.0))
    return synth.custom_batch(events, seqs, sc, mm, ms, k, W)


@pytest.mark.parametrize("theta", [1.0, ALL_BLOCK])
def test_degenerate_shapes(ctx, theta):
    """One to three events against up to 5,000 bases, one or two k-mers against up to 2,000 events,
    and tiny near-square reads, per warp and in block mode: status, end event, cells, pairs and
    score equal the FP32 oracle's on every read."""
    b = _degenerate_batch()
    res, pairs, po = run_gpu(ctx, b, theta=theta)
    compare(b, res, pairs, po)


@pytest.mark.parametrize("theta", [1.0, ALL_BLOCK])
def test_page_locked_host_buffers(ctx, theta):
    """abea_align_packed with page-locked host arrays takes the direct path (copies straight to and
    from the caller's arrays, no staging on the host).  Results and every aligned read's pairs equal
    the pageable call's and the FP32 oracle's, with spare capacity in the slots and a read one pair
    short of its alignment (status CAPACITY with the required count), per warp and in block mode."""
    torch = pytest.importorskip("torch")
    b = _lengths_batch([200, 400, 600, 5000, 30, 12000, 80, 2500], seed=12)
    o = oracle.abea_batch(b, "f32", n_threads=THREADS)
    need = o["n_pairs"].astype(np.int64)
    caps = need + 7
    caps[1] = need[1] - 1                          # one pair short
    po = np.zeros(b.n + 1, np.int64)
    np.cumsum(caps, out=po[1:])
    ref_res, ref_pairs, _ = run_gpu(ctx, b, pair_off=po, theta=theta)
    assert ref_res["status"][1] == binding.READ_CAPACITY and ref_res["n_pairs"][1] == need[1]

    def pin(a):
        return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()

    seq, ev = pin(b.seq), pin(b.events)
    out = pin(np.zeros(b.n * 24, np.uint8))
    pairs = pin(np.full(int(po[-1]) * 2, -7, np.int32))
    sc = np.ascontiguousarray(b.scalings, np.float32)
    ctx.set_model(b.k, b.model_mean, b.model_stdv)
    ctx.set_block_mode(theta)
    try:
        rc = ctx.lib.abea_align_packed(ctx.h, b.n, b.W, binding._p(seq), binding._p(b.seq_off), binding._p(ev),
                                       binding._p(b.ev_off), binding._p(sc), binding._p(out), binding._p(pairs),
                                       binding._p(po), None)
    finally:
        ctx.set_block_mode(1.0)
    assert rc == 0
    res = binding.results_from_bytes(out)
    assert np.array_equal(res, ref_res)
    pairs = pairs.reshape(-1, 2)
    for i in range(b.n):
        if res["status"][i] != binding.READ_OK:
            continue
        lo, m = int(po[i]), int(res["n_pairs"][i])
        assert np.array_equal(pairs[lo:lo + m], ref_pairs[lo:lo + m])
        assert np.array_equal(pairs[lo:lo + m], o["pairs"][o["pair_off"][i]:o["pair_off"][i] + m])
