"""Wide model (k = 9, W = 200) and the band-width sweep W in {50, 100, 200}.

At each W the GPU's FP32 score is within 1e-4 relative of the FP64 oracle at
the same W.  Across W the scores are not ordered (the band follows the
scores, so a narrower band may end elsewhere); the test prints, per W, how
often the path equals the path at W = 200 and how the FP64 score moves, which
is what the band width trades for work.
"""
import os

import numpy as np
import pytest

from oracle import oracle
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu

THREADS = os.cpu_count() or 4


def test_wide_model_band_width_sweep():
    w = synth.WORKLOADS["wide_10k_ln10kb_k9_w200"]
    b = synth.make_batch(w, read_ids=range(0, w.n_reads, w.n_reads // 48))
    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        gpu = {W: ctx.align_packed(b, W=W) for W in (50, 100, 200)}
    o64 = {W: oracle.abea_batch(b, "f64", n_threads=THREADS, W=W) for W in (50, 100, 200)}
    lines = []
    for W in (50, 100, 200):
        res, pairs, po = gpu[W]
        o = o64[W]
        ok = (res["status"] == 0) & (o["status"] == oracle.ST_OK)
        rel = np.abs(res["score"][ok].astype(np.float64) - o["score"][ok]) / np.abs(o["score"][ok])
        assert np.all(res["status"] == o["status"])
        assert rel.max() <= 1e-4, (W, rel.max())
        r2, p2, po2 = gpu[200]
        same = [np.array_equal(pairs[po[i]:po[i] + res["n_pairs"][i]], p2[po2[i]:po2[i] + r2["n_pairs"][i]])
                for i in range(b.n)]
        d = (o["score"] - o64[200]["score"]) / np.abs(o64[200]["score"])
        lines.append(f"W={W}: reads={b.n} cells={int(res['cells'].sum())} fp32_vs_fp64_rel_max={rel.max():.2e} "
                     f"mean={rel.mean():.2e} path_equal_to_W200={np.mean(same):.3f} "
                     f"fp64_score_vs_W200_rel_mean={d.mean():+.2e} min={d.min():+.2e} max={d.max():+.2e}")
    print("\n" + "\n".join(lines))
