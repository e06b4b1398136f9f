"""GPU: the launch-geometry autotuner (abea_autotune).  It reports one
choice per length bucket the sample populates, with measured rates of both
modes where block mode exists, and batches aligned after tuning are
identical to the FP32 oracle (the mode changes where a read runs, never its
result)."""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 4


def sample_of_every_bucket():
    w = synth.WORKLOADS["large_50k_ln8kb"]
    L = synth.read_lengths(w)
    order = np.argsort(-L)
    # the two longest (ultra-long, >= 65,536 bands), reads of 5-20 kb, and short ones
    ids = list(order[:2]) + list(order[np.searchsorted(-L[order], -20_000):][:6])
    ids += list(np.nonzero((L > 1500) & (L < 4000))[0][:24]) + list(np.nonzero(L < 1200)[0][:40])
    return synth.make_batch(w, read_ids=sorted(set(int(i) for i in ids)))


def test_autotune_reports_every_bucket_and_keeps_results():
    b = sample_of_every_bucket()
    bands = b.n_events() + b.n_kmers() + 1
    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        ch = ctx.autotune(b)
        res, pairs, po = ctx.align_packed(b)
    lo = np.array([0, 4096, 16384, 65536])
    want = sorted(set(int(lo[np.searchsorted(lo, x, side="right") - 1]) for x in bands))
    assert sorted(ch["min_bands"].tolist()) == want
    for c in ch:
        inb = (bands >= c["min_bands"]) & ((bands < c["max_bands"]) if c["max_bands"] > 0 else True)
        assert c["sample_reads"] == int(inb.sum()) and c["W"] == b.W
        assert c["reads_per_cta"] in (1, 4) and c["gcups_per_warp"] > 0 and c["gcups_block"] > 0
        assert c["threads_per_band"] == (25 if c["reads_per_cta"] == 4 else 100) and c["record_words"] == 8
    # block mode, once chosen, stays chosen for every longer bucket
    blk = ch["reads_per_cta"][np.argsort(ch["min_bands"])] == 1
    assert not np.any(blk[:-1] & ~blk[1:])
    o = oracle.abea_batch(b, "f32", n_threads=THREADS)
    assert np.all(res["status"] == 0)
    for i in range(b.n):
        assert np.float32(o["score"][i]) == res["score"][i], i
        assert np.array_equal(pairs[po[i]:po[i] + res["n_pairs"][i]],
                              o["pairs"][o["pair_off"][i]:o["pair_off"][i] + o["n_pairs"][i]]), i


def test_autotune_without_block_mode_and_bad_arguments():
    b = synth.make_batch("plain_64x1kb", n_reads=16)
    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        ch = ctx.autotune(b, W=30)              # W < 32: no block mode
        assert len(ch) == 1 and ch[0]["reads_per_cta"] == 4 and ch[0]["gcups_block"] == 0
        with pytest.raises(binding.AbeaError):
            ctx.autotune(b, W=1)
