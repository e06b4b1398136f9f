"""Mutation check of the oracle's pins (no GPU).

Each mutant is a plausible mistake planted in a copy of oracle/abea_oracle.c
(a dropped term, a wrong sign, index or operand, a wrong reading).  The copy
is compiled on the CPU and every pin of test_oracle_pins.py is run against it
in a child process; at least one pin must fail (or the child must crash).
A mutant that survives means the pins do not cover that part of the oracle.

One reading has nothing outside the oracle to pin it and is left out here:
the order D > U > L among exactly equal candidates (exact floating-point
ties).  The parity of the band-move alternation while both band ends are -inf
is pinned by band positions worked by hand from the author comment in
Alg. adaptivebandedcpu (tests/golden/band_positions.json).
"""
import os
import subprocess
import sys
import textwrap

import pytest

from oracle import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("stay_uses_step", "real score_u = up + p->lp_stay + lp_emission;", "real score_u = up + p->lp_step + lp_emission;"),
    ("stay_drops_emission", "real score_u = up + p->lp_stay + lp_emission;", "real score_u = up + p->lp_stay;"),
    ("skip_adds_emission", "real score_l = left + p->lp_skip;", "real score_l = left + p->lp_skip + lp_emission;"),
    ("emission_sign", "- 0.5 * z * z;", "+ 0.5 * z * z;"),
    ("emission_no_log_sigma", "return LOG_INV_SQRT_2PI - log(p->sigma[k]) - 0.5 * z * z;",
     "return LOG_INV_SQRT_2PI - 0.5 * z * z;"),
    ("scaling_drops_scale", "p->mu[i] = (double)model_mean[ranks[i]] * (double)scale + (double)shift;",
     "p->mu[i] = (double)model_mean[ranks[i]] + (double)shift;"),
    ("scaling_drops_var", "p->sigma[i] = (double)model_stdv[ranks[i]] * (double)var;",
     "p->sigma[i] = (double)model_stdv[ranks[i]];"),
    ("epk_inverted", "(double)n_events / (double)n_kmers", "(double)n_kmers / (double)n_events"),
    ("step_drops_epsilon", "log(1.0 - exp(lp_skip) - exp(lp_stay))", "log(1.0 - exp(lp_stay))"),
    ("trim_prob", "log(1.0 / 100.0)", "log(1.0 / 10.0)"),
    ("up_offset", "int32_t j_up = ll_e[b - 1] - (e - 1);", "int32_t j_up = ll_e[b - 1] - e;"),
    ("left_offset", "int32_t j_left = (kk - 1) - ll_k[b - 1];", "int32_t j_left = kk - ll_k[b - 1];"),
    ("diag_from_previous_band", "? SCORE(b - 2, j_diag)", "? SCORE(b - 1, j_diag)"),
    ("sk_rule_reversed", "advance_kmer = lower_left < upper_right;", "advance_kmer = lower_left > upper_right;"),
    ("sk_parity_flipped", "advance_kmer = (int)(b & 1);", "advance_kmer = (int)((b & 1) ^ 1);"),
    ("trim_count", "SCORE(b, jt) = (real)(e + 1) * p.lp_trim;", "SCORE(b, jt) = (real)(e) * p.lp_trim;"),
    ("end_trim_count", "band_frame[b] + (double)(SCORE(b, j) + (real)(n_e - 1 - e) * p.lp_trim);",
     "band_frame[b] + (double)(SCORE(b, j) + (real)(n_e - e) * p.lp_trim);"),
    ("f32_frame_not_added_back", "double cand = band_frame[b] + (double)(SCORE(b, j)",
     "double cand = 0.0 + (double)(SCORE(b, j)"),
    ("f32_renorm_shifts_one_band", "                    SCORE(b - 1, j) -= R;\n", ""),
    ("origin_offset", "ll_e[0] = half - 1;", "ll_e[0] = half;"),
    ("backtrack_up_moves_kmer", "else if (t == TR_U) { e--; }\n            else { kk--; }\n        }\n        if (overflow == 2)",
     "else if (t == TR_U) { kk--; }\n            else { kk--; }\n        }\n        if (overflow == 2)"),
    ("f32_emission_sign", "return fmaf(-z, z, p->c[k]);", "return fmaf(z, z, p->c[k]);"),
    ("f32_max_drops_emission", "real s = m + lp_emission;", "real s = m;"),
    ("f32_b_sign", "p->b[i] = (float)(-(mu_p * a));", "p->b[i] = (float)(mu_p * a);"),
]

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
    from oracle import oracle
    import test_oracle_pins as P
    lib = oracle.load({lib!r})
    pins = [("constants", lambda: P.pin_constants(lib)),
            ("emission_f64", lambda: P.pin_emission(lib, "f64")),
            ("emission_f32", lambda: P.pin_emission(lib, "f32")),
            ("hand_f64", lambda: P.pin_hand_examples(lib, "f64")),
            ("hand_f32", lambda: P.pin_hand_examples(lib, "f32")),
            ("brute_force", lambda: P.pin_brute_force(lib, n_cases=40)),
            ("wide_band", lambda: P.pin_wide_band_is_full_dp(lib, n_reads=3)),
            ("invariants", lambda: P.pin_invariants(lib, n_reads=2)),
            ("band_positions", lambda: P.pin_band_positions(lib)),
            ("fp32_long_read", lambda: P.pin_fp32_long_read(lib))]
    failed = []
    for name, fn in pins:
        try:
            fn()
        except Exception as e:
            failed.append(name)
    print("FAILED:", ",".join(failed))
    sys.exit(0 if failed else 1)
""")


def test_mutant_list_applies():
    src = open(oracle.SRC).read()
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, (name, src.count(old))


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(oracle.SRC).read()
    assert src.count(old) == 1
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = str(tmp_path / "libmutant.so")
    oracle.build(str(mpath), lib)
    code = CHILD.format(root=ROOT, tests=os.path.join(ROOT, "tests"), lib=lib)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert p.returncode != 1, f"mutant {name} survived every pin:\n{p.stdout}\n{p.stderr[-2000:]}"
