"""GPU eventalign rows (abea_eventalign) against the oracle, from ABEA's own
device outputs: every field identical, in both level modes; reads that did
not align produce no rows."""
import numpy as np
import pytest

from oracle import eventalign_oracle as ea
from paper_2101_05012_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def test_rows_match_the_oracle():
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    b0 = synth.make_batch("plain_64x1kb", n_reads=24)
    # one read with a bad base: ABEA rejects it, eventalign writes nothing for it
    evs, sqs, scs = zip(*[b0.read(i) for i in range(b0.n)])
    sqs = list(sqs)
    sqs[5] = sqs[5][:100] + b"N" + sqs[5][101:]
    evs = list(evs)
    evs[7] = np.full_like(evs[7], 400.0)        # every event far off the model: trimmed, low score
    b = synth.custom_batch(list(evs), sqs, list(scs), b0.model_mean, b0.model_stdv, b0.k, b0.W)
    # one reference holding every read's reference, with per-base positions into it
    refs, pos = [], np.zeros(len(b.seq), np.int32)
    base = 0
    for i in range(b.n):
        r, p = synth.make_ref_alignment(b.seq[b.seq_off[i]:b.seq_off[i + 1]].tobytes(), 9, i)
        pos[b.seq_off[i]:b.seq_off[i + 1]] = np.where(p >= 0, p + base, -1)
        refs.append(r)
        base += len(r)
    ref = np.concatenate(refs)
    ref[::97] = ord("N")                    # reference k-mers over a non-ACGT base get no rank
    po = binding.pair_offsets(b.n_events(), np.maximum(b.n_kmers(), 1))
    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        d_seq = torch.from_numpy(b.seq).to(dev)
        d_ev = torch.from_numpy(b.events).to(dev)
        d_res = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
        d_pairs = torch.zeros(int(po[-1]) * 2, dtype=torch.int32, device=dev)
        d_pos = torch.from_numpy(pos).to(dev)
        d_ref = torch.from_numpy(ref).to(dev)
        s = torch.cuda.Stream(dev)
        ctx.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_res, d_pairs, po,
                               stream=s.cuda_stream)
        out = {}
        for mode in (False, True):
            d_rows = torch.zeros(int(po[-1]) * 40, dtype=torch.uint8, device=dev)
            ctx.eventalign(b.n, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_res, d_pairs, po, d_pos, d_ref,
                           len(ref), mode, d_rows, stream=s.cuda_stream)
            s.synchronize()
            out[mode] = np.frombuffer(d_rows.cpu().numpy().tobytes(), binding.EVENTALIGN_DTYPE)
        d_sum = torch.zeros(b.n * binding.SUMMARY_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        ctx.summarise(b.n, b.seq_off, b.ev_off, d_res, d_pairs, po, d_sum, stream=s.cuda_stream)
        s.synchronize()
        summ = np.frombuffer(d_sum.cpu().numpy().tobytes(), binding.SUMMARY_DTYPE)
        res = binding.results_from_bytes(d_res.cpu().numpy())
        pairs = d_pairs.cpu().numpy().reshape(-1, 2)
    assert res["status"][5] == binding.READ_BAD_INPUT and np.sum(res["status"] == 0) == b.n - 1
    # per-read summaries against the oracle's, from the same alignments
    for i in range(b.n):
        want = ea.read_summary(i, int(b.n_events()[i]), int(b.n_kmers()[i]), int(res["status"][i]),
                               res["score"][i], pairs[po[i]:po[i] + res["n_pairs"][i]])
        for f in binding.SUMMARY_DTYPE.names:
            assert np.array_equal(summ[f][i], want[f][0]), (i, f, summ[f][i], want[f][0])
    assert summ["flags"][5] == binding.QC_NOT_ALIGNED
    assert summ["flags"][7] & (binding.QC_TRIMMED | binding.QC_LOW_SCORE)
    assert np.all(summ["flags"][[i for i in range(b.n) if i not in (5, 7)]] == 0)
    for mode in (False, True):
        rows = out[mode]
        for i in range(b.n):
            got = rows[po[i]:po[i + 1]]
            if res["status"][i] != 0:
                assert np.all(got["read"] == 0) and np.all(got["z"] == 0)    # untouched
                continue
            n = int(res["n_pairs"][i])
            e, sq, sc = b.read(i)
            want = ea.rows(i, b.model_mean, b.model_stdv, b.k, sq, e, sc, pairs[po[i]:po[i] + n], ref,
                           pos[b.seq_off[i]:b.seq_off[i + 1]], scale_events=mode)
            g = got[:n]
            for f in binding.EVENTALIGN_DTYPE.names:
                assert np.array_equal(g[f], want[f]), (mode, i, f)
    # the reference positions of the k-mers are shifted by the read's indels, and some bases are insertions
    assert np.any(out[False]["ref_pos"] < 0)
    assert np.any((out[False]["ref_pos"] >= 0) & (out[False]["ref_rank"] < 0))


@pytest.mark.parametrize("workload,rows_offset", [("wide_10k_ln10kb_k9_w200", 0), ("plain_64x1kb", 4)])
def test_global_model_and_unaligned_rows(workload, rows_offset):
    """k = 9 (the model table stays in global memory) and a row buffer that starts 4 bytes past an
    8-byte boundary (rows written as 4-byte words): every field identical to the oracle."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    b = synth.make_batch(workload, n_reads=16)
    refs, pos = [], np.zeros(len(b.seq), np.int32)
    base = 0
    for i in range(b.n):
        r, p = synth.make_ref_alignment(b.seq[b.seq_off[i]:b.seq_off[i + 1]].tobytes(), 5, i)
        pos[b.seq_off[i]:b.seq_off[i + 1]] = np.where(p >= 0, p + base, -1)
        refs.append(r)
        base += len(r)
    ref = np.concatenate(refs)
    po = binding.pair_offsets(b.n_events(), np.maximum(b.n_kmers(), 1))
    with binding.Context(0) as ctx:
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        d_seq = torch.from_numpy(b.seq).to(dev)
        d_ev = torch.from_numpy(b.events).to(dev)
        d_res = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
        d_pairs = torch.zeros(int(po[-1]) * 2, dtype=torch.int32, device=dev)
        d_pos = torch.from_numpy(pos).to(dev)
        d_ref = torch.from_numpy(ref).to(dev)
        s = torch.cuda.Stream(dev)
        ctx.align_batch_device(b.n, b.W, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_res, d_pairs, po,
                               stream=s.cuda_stream)
        store = torch.zeros(int(po[-1]) * 40 + 8, dtype=torch.uint8, device=dev)
        d_rows = store[rows_offset:rows_offset + int(po[-1]) * 40]
        assert d_rows.data_ptr() % 8 == rows_offset
        ctx.eventalign(b.n, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_res, d_pairs, po, d_pos, d_ref,
                       len(ref), True, d_rows, stream=s.cuda_stream)
        s.synchronize()
        rows = np.frombuffer(d_rows.cpu().numpy().tobytes(), binding.EVENTALIGN_DTYPE)
        res = binding.results_from_bytes(d_res.cpu().numpy())
        pairs = d_pairs.cpu().numpy().reshape(-1, 2)
    assert np.all(res["status"] == 0)
    for i in range(b.n):
        n = int(res["n_pairs"][i])
        e, sq, sc = b.read(i)
        want = ea.rows(i, b.model_mean, b.model_stdv, b.k, sq, e, sc, pairs[po[i]:po[i] + n], ref,
                       pos[b.seq_off[i]:b.seq_off[i + 1]], scale_events=True)
        got = rows[po[i]:po[i] + n]
        for f in binding.EVENTALIGN_DTYPE.names:
            assert np.array_equal(got[f], want[f]), (workload, i, f)


def test_invalid_arguments_and_missing_model():
    """A negative reference length or a zero scale is ABEA_ERR_ARG; a context without a model
    answers ABEA_ERR_NO_MODEL (eventalign and the scaling estimate)."""
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    b = synth.make_batch("plain_64x1kb", n_reads=2)
    po = binding.pair_offsets(b.n_events(), np.maximum(b.n_kmers(), 1))
    d_seq = torch.from_numpy(b.seq).to(dev)
    d_ev = torch.from_numpy(b.events).to(dev)
    d_res = torch.zeros(b.n * 24, dtype=torch.uint8, device=dev)
    d_pairs = torch.zeros(int(po[-1]) * 2, dtype=torch.int32, device=dev)
    d_pos = torch.zeros(len(b.seq), dtype=torch.int32, device=dev)
    d_ref = torch.zeros(16, dtype=torch.uint8, device=dev)
    d_rows = torch.zeros(int(po[-1]) * 40, dtype=torch.uint8, device=dev)
    d_sc = torch.zeros(b.n * 3, dtype=torch.float32, device=dev)
    d_st = torch.zeros(b.n, dtype=torch.int32, device=dev)
    with binding.Context(0) as ctx:
        with pytest.raises(binding.AbeaError) as ei:
            ctx.eventalign(b.n, d_seq, b.seq_off, d_ev, b.ev_off, b.scalings, d_res, d_pairs, po, d_pos, d_ref,
                           16, False, d_rows)
        assert ei.value.code == binding.ABEA_ERR_NO_MODEL
        with pytest.raises(binding.AbeaError) as ei:
            ctx.estimate_scalings(b.n, d_seq, b.seq_off, d_ev, b.ev_off, d_sc, d_st)
        assert ei.value.code == binding.ABEA_ERR_NO_MODEL
        ctx.set_model(b.k, b.model_mean, b.model_stdv)
        zero = np.array(b.scalings, np.float32)
        zero[1, 0] = 0.0
        for sc, ref_len in ((b.scalings, -1), (zero, 16)):
            with pytest.raises(binding.AbeaError) as ei:
                ctx.eventalign(b.n, d_seq, b.seq_off, d_ev, b.ev_off, sc, d_res, d_pairs, po, d_pos, d_ref,
                               ref_len, False, d_rows)
            assert ei.value.code == binding.ABEA_ERR_ARG
