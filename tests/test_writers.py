"""The host text writers of the C ABI (abea_eventalign_tsv, abea_summary_tsv)
against the formats their declarations give, on rows and summaries the CPU
oracles compute (no GPU: the writers make no CUDA call)."""
import numpy as np

from oracle import eventalign_oracle as ea
from oracle import oracle
from paper_2101_05012_gb300 import binding, synth


def kmer(rank: int, k: int) -> str:
    if rank < 0:
        return "N" * k
    return "".join("ACGT"[(rank >> (2 * (k - 1 - t))) & 3] for t in range(k))


def oracle_rows_and_summaries():
    b = synth.make_batch("plain_64x1kb", n_reads=5)
    o = oracle.abea_batch(b, "f32", n_threads=2)
    rows, summ = [], []
    for i in range(b.n):
        e, sq, sc = b.read(i)
        p = o["pairs"][o["pair_off"][i]:o["pair_off"][i] + o["n_pairs"][i]]
        ref, pos = synth.make_ref_alignment(sq, 9, i)
        rows.append(ea.rows(i, b.model_mean, b.model_stdv, b.k, sq, e, sc, p, ref, pos))
        summ.append(ea.read_summary(i, len(e), len(sq) - b.k + 1, int(o["status"][i]), o["score"][i], p))
    return b, np.concatenate(rows), np.concatenate(summ)


def test_eventalign_tsv():
    b, rows, _ = oracle_rows_and_summaries()
    text = binding.eventalign_tsv(rows, b.k)
    lines = text.splitlines()
    assert lines[0].split("\t") == ["read", "event", "kmer", "ref_pos", "ref_kmer", "model_kmer", "level",
                                    "model_mean", "model_stdv", "z"]
    want = ["\t".join([str(r["read"]), str(r["event"]), str(r["kmer"]), str(r["ref_pos"]), kmer(r["ref_rank"], b.k),
                       kmer(r["model_rank"], b.k), "%.2f" % r["level"], "%.2f" % r["model_mean"],
                       "%.2f" % r["model_stdv"], "%.3f" % r["z"]]) for r in rows]
    assert lines[1:] == want
    assert binding.eventalign_tsv(rows[:3], b.k, header=False).count("\n") == 3


def test_summary_tsv():
    _, _, summ = oracle_rows_and_summaries()
    lines = binding.summary_tsv(summ).splitlines()
    assert lines[0].split("\t")[:3] == ["read", "status", "n_events"] and len(lines) == len(summ) + 1
    for line, s in zip(lines[1:], summ):
        f = line.split("\t")
        assert [int(v) for v in f[:10]] == [int(s[n]) for n in binding.SUMMARY_DTYPE.names[:10]]
        assert f[10] == "%.3f" % s["score"] and f[11] == "%.3f" % s["score_per_event"] and int(f[12]) == s["flags"]


def test_writer_capacity_is_reported():
    import ctypes
    b, rows, _ = oracle_rows_and_summaries()
    lib = binding.load()
    r = np.ascontiguousarray(rows[:10], binding.EVENTALIGN_DTYPE)
    need = ctypes.c_size_t()
    buf = ctypes.create_string_buffer(16)
    rc = lib.abea_eventalign_tsv(binding._p(r), 10, b.k, 1, buf, 16, ctypes.byref(need))
    assert rc == binding.ABEA_ERR_CAPACITY and need.value > 16 and len(buf.value) == 15
    assert lib.abea_eventalign_tsv(binding._p(r), 10, 0, 1, None, 0, ctypes.byref(need)) == binding.ABEA_ERR_ARG
