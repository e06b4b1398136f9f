"""Pins of the eventalign oracle: a hand-worked example, the reference mapping
through an alignment with indels, the equality of z with and without
scale_events, and planted mistakes."""
import numpy as np
import pytest

from oracle import eventalign_oracle as ea

MEAN = np.array([60.0, 80.0, 100.0, 120.0], np.float32)      # k = 1: A C G T
STDV = np.array([1.0, 2.0, 4.0, 8.0], np.float32)


def test_hand_example():
    pairs = [(0, 0), (1, 1), (2, 1), (3, 2), (4, 3)]
    ev = np.array([61.0, 79.0, 82.0, 104.0, 116.0], np.float32)
    ref = np.frombuffer(b"TACGT", np.uint8)
    ref_pos = np.array([1, 2, 3, 4], np.int32)                 # read ACGT at ref 1..4
    r = ea.rows(7, MEAN, STDV, 1, b"ACGT", ev, (1.0, 0.0, 1.0), pairs, ref, ref_pos)
    assert list(r["z"]) == [1.0, -0.5, 1.0, 1.0, -0.5]
    assert list(r["ref_pos"]) == [1, 2, 2, 3, 4] and list(r["ref_rank"]) == [0, 1, 1, 2, 3]
    assert list(r["model_rank"]) == [0, 1, 1, 2, 3] and list(r["read"]) == [7] * 5
    # scalings: mean = mu * 2 + 10, stdv = sigma * 1.5
    r = ea.rows(0, MEAN, STDV, 1, b"ACGT", ev, (2.0, 10.0, 1.5), pairs[:1], ref, ref_pos)
    assert r["model_mean"][0] == 130.0 and r["model_stdv"][0] == 1.5
    assert r["z"][0] == np.float32(np.float32(61.0 - 130.0) / np.float32(1.5))


def test_reference_positions_through_indels():
    # read GATTACA (k = 3); the reference lacks the read's second T and has an extra C after A
    seq = b"GATTACA"
    ref = np.frombuffer(b"GATACCA", np.uint8)
    ref_pos = np.array([0, 1, 2, -1, 3, 5, 6], np.int32)        # T (read 3) inserted; ref C at 4 extra
    mean = np.arange(64, dtype=np.float32) + 60
    stdv = np.ones(64, np.float32)
    pairs = [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4)]
    ev = mean[:5]
    r = ea.rows(0, mean, stdv, 3, seq, ev, (1.0, 0.0, 1.0), pairs, ref, ref_pos)
    rank = lambda s: int("".join(str("ACGT".index(c)) for c in s), 4)
    assert list(r["ref_pos"]) == [0, 1, 2, -1, 3]
    assert list(r["ref_rank"]) == [rank("GAT"), rank("ATA"), rank("TAC"), -1, rank("ACC")]
    assert list(r["model_rank"]) == [rank("GAT"), rank("ATT"), rank("TTA"), rank("TAC"), rank("ACA")]
    # a k-mer running past the reference end has no reference rank
    r = ea.rows(0, mean, stdv, 3, seq, ev, (1.0, 0.0, 1.0), [(0, 4)], ref[:5], ref_pos)
    assert r["ref_rank"][0] == -1


def test_scale_events_gives_the_same_z():
    rng = np.random.default_rng(3)
    mean = rng.uniform(60, 130, 4 ** 4).astype(np.float32)
    stdv = rng.uniform(1, 3, 4 ** 4).astype(np.float32)
    seq = np.array(rng.choice(list(b"ACGT"), 300), np.uint8).tobytes()
    pairs = np.stack([np.arange(250), np.arange(250) // 2 + 10], 1)
    ev = rng.normal(100, 15, 250).astype(np.float32)
    sc = (1.07, -3.5, 1.2)
    ref_pos = np.arange(300, dtype=np.int32)
    a = ea.rows(0, mean, stdv, 4, seq, ev, sc, pairs, np.frombuffer(seq, np.uint8), ref_pos)
    b = ea.rows(0, mean, stdv, 4, seq, ev, sc, pairs, np.frombuffer(seq, np.uint8), ref_pos, scale_events=True)
    assert np.allclose(a["z"], b["z"], rtol=1e-5, atol=1e-5)
    assert np.array_equal(a["ref_rank"], a["model_rank"])                  # the reference is the read


def _hand_rows():
    pairs = [(0, 0), (1, 1), (2, 1), (3, 2), (4, 3)]
    ev = np.array([61.0, 79.0, 82.0, 104.0, 116.0], np.float32)
    ref = np.frombuffer(b"TACGT", np.uint8)
    ref_pos = np.array([1, 2, 3, 4], np.int32)
    return ea.rows(7, MEAN, STDV, 1, b"ACGT", ev, (1.0, 0.0, 2.0), pairs, ref, ref_pos)


def _indel_rows():
    mean = np.arange(64, dtype=np.float32) + 60
    return ea.rows(0, mean, np.ones(64, np.float32), 3, b"GATTACA", mean[:5], (1.0, 0.0, 1.0),
                   [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4)], np.frombuffer(b"GATACCA", np.uint8),
                   np.array([0, 1, 2, -1, 3, 5, 6], np.int32))


# Planted mistakes (applied to the oracle's output where the mistake would act): each must
# disagree with the pinned values above.
@pytest.mark.parametrize("mistake", ["sign", "stdv_without_var", "ref_of_last_base"])
def test_planted_mistakes_fail(mistake):
    good_z = [0.5, -0.25, 0.5, 0.5, -0.25]                      # var = 2 doubles the model stdv
    good_ref = [0, 1, 2, -1, 3]
    r, q = _hand_rows(), _indel_rows()
    assert list(r["z"]) == good_z and list(q["ref_pos"]) == good_ref
    if mistake == "sign":
        assert list(-r["z"]) != good_z
    elif mistake == "stdv_without_var":
        assert list((r["level"] - r["model_mean"]) / STDV[r["model_rank"]]) != good_z
    else:
        ref_pos = np.array([0, 1, 2, -1, 3, 5, 6], np.int32)
        assert [int(ref_pos[j + 2]) for j in q["kmer"]] != good_ref


def test_read_summary_hand_worked():
    """Read summary of a hand-walked path (reading of eventalign's per-read summary): 8 events,
    5 k-mers, pairs (1,0) (2,0) (3,1) (3,2) (3,3) (4,4): one stay (2,0), two skips (3,2) (3,3), so
    4 events aligned; events 0, 5, 6 and 7 trimmed (4 of 8, not more than half); 2 skips, above a
    fifth of 5 k-mers; score -12 over 8 events = -1.5 per event."""
    pairs = np.array([(1, 0), (2, 0), (3, 1), (3, 2), (3, 3), (4, 4)], np.int32)
    s = ea.read_summary(3, 8, 5, 0, -12.0, pairs)[0]
    assert (s["read"], s["status"], s["n_events"], s["n_kmers"], s["n_pairs"]) == (3, 0, 8, 5, 6)
    assert (s["first_event"], s["last_event"], s["events_aligned"], s["stays"], s["skips"]) == (1, 4, 4, 1, 2)
    assert s["score"] == np.float32(-12.0) and s["score_per_event"] == np.float32(-1.5)
    assert s["flags"] == ea.QC_SKIPS
    # more than half of the events trimmed and a low score per event; no skip
    s = ea.read_summary(0, 10, 3, 0, -120.0, np.array([(6, 0), (7, 1), (8, 2)], np.int32))[0]
    assert (s["stays"], s["skips"], s["events_aligned"]) == (0, 0, 3)
    assert s["flags"] == ea.QC_TRIMMED | ea.QC_LOW_SCORE
    # no alignment: flagged, no pairs counted
    s = ea.read_summary(1, 10, 3, 1, -np.inf, np.zeros((0, 2), np.int32))[0]
    assert s["flags"] == ea.QC_NOT_ALIGNED and s["n_pairs"] == 0 and s["first_event"] == -1
