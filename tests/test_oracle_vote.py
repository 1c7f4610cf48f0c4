"""Pins for the oracle's voter (Sec. IV.D: compare redundant results and
determine the presumable correct result; the DMR case of the paper is R = 2).

* brute force: every assignment of a small alphabet of values to R <= 5
  replicas, checked against a formulation by groups of equal values (written
  here without support counts);
* textbook TMR: for R = 3 integer replicas with at least two equal, the word
  vote equals the bit-wise majority function (a&b)|(a&c)|(b&c);
* hand-worked non-transitive cases (tests/golden/vote_nontransitive.txt);
* invariants on generated workloads: identical replicas, a single faulty
  replica per element, permutation of replicas, and the digest of the voted
  buffer against the digest of the clean source.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1405_2912_b300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _group_vote(labels, group_of):
    """Expected (winner, majority, mismatching set) from groups of equal values:
    the largest group wins; among equally large groups the one holding the
    lowest replica index; the winner is that group's lowest index."""
    R = len(labels)
    groups = {}
    for r, lab in enumerate(labels):
        groups.setdefault(group_of[lab], []).append(r)
    best = max(groups.values(), key=lambda g: (len(g), -g[0]))
    return best[0], 2 * len(best) > R, [r for r in range(R) if r not in best]


def _brute(R, dtype, alphabet, group_of, abs_tol, rel_tol):
    names = list(alphabet)
    pats = list(itertools.product(names, repeat=R))
    t = oracle.NP_OF[dtype]
    reps = [np.array([alphabet[p[r]] for p in pats], dtype=t) for r in range(R)]
    res = oracle.vote(reps, dtype, abs_tol, rel_tol)
    exp_mism = np.zeros(R, dtype=np.int64)
    exp_first = np.full(R, -1, dtype=np.int64)
    exp_nomaj, exp_fnomaj = 0, -1
    for i, p in enumerate(pats):
        w, maj, bad = _group_vote(p, group_of)
        assert res["out"][i].tobytes() == reps[w][i].tobytes(), (p, w)
        for r in bad:
            exp_mism[r] += 1
            if exp_first[r] < 0:
                exp_first[r] = i
        if not maj:
            exp_nomaj += 1
            if exp_fnomaj < 0:
                exp_fnomaj = i
    assert list(res["mismatch"]) == list(exp_mism)
    assert list(res["first_mismatch"]) == list(exp_first)
    assert res["no_majority"] == exp_nomaj
    assert res["first_no_majority"] == exp_fnomaj


@pytest.mark.parametrize("R", [2, 3, 4, 5])
def test_brute_force_float_clusters(R):
    # C and Cp lie within rel 1e-5 of each other; F1, F2 are far from all.
    alphabet = {"C": 1.0, "Cp": float(np.float32(1.0) + np.float32(2 ** -22)),
                "F1": -3.5, "F2": 1e20}
    group_of = {"C": "c", "Cp": "c", "F1": "f1", "F2": "f2"}
    _brute(R, "f32", alphabet, group_of, 1e-6, 1e-5)
    alphabet64 = {"C": 1.0, "Cp": 1.0 + 2 ** -50, "F1": 1.0 + 1e-9, "F2": float("inf")}
    _brute(R, "f64", alphabet64, group_of, 0.0, 1e-12)


@pytest.mark.parametrize("R", [2, 3, 5, 6])
@pytest.mark.parametrize("dtype", ["i32", "u8", "u64"])
def test_brute_force_integers(R, dtype):
    alphabet = {"a": 5, "b": 6, "c": 7, "d": 200}
    group_of = {k: k for k in alphabet}
    _brute(R, dtype, alphabet, group_of, 0.0, 0.0)


def test_brute_force_r8_sampled():
    rng = np.random.default_rng(8)
    alphabet = [0, 1, 2]
    pats = [tuple(rng.integers(0, 3, size=8)) for _ in range(2000)]
    reps = [np.array([p[r] for p in pats], dtype=np.int32) for r in range(8)]
    res = oracle.vote(reps, "i32")
    for i, p in enumerate(pats):
        w, maj, bad = _group_vote(p, {a: a for a in alphabet})
        assert res["out"][i] == p[w]


def test_textbook_tmr_bitwise_majority():
    rng = np.random.default_rng(11)
    n = 50000
    a = rng.integers(0, 2 ** 32, size=n, dtype=np.uint32)
    b = a.copy()
    c = a.copy()
    who = rng.integers(0, 3, size=n)              # which replica (if any) is hit
    hit = rng.random(n) < 0.3
    noise = rng.integers(1, 2 ** 32, size=n, dtype=np.uint32)
    for r, arr in enumerate((a, b, c)):
        m = hit & (who == r)
        arr[m] ^= noise[m]
    res = oracle.vote([a, b, c], "u32")
    maj = (a & b) | (a & c) | (b & c)
    assert np.array_equal(res["out"], maj)
    assert res["no_majority"] == 0


def test_dmr_detection_only():
    # R = 2, the paper's DMR: agreement passes, disagreement is detected
    # (no majority) and the value of replica 0 is kept.
    a = np.arange(100, dtype=np.int32)
    b = a.copy()
    b[[3, 50, 99]] += 1
    res = oracle.vote([a, b], "i32")
    assert np.array_equal(res["out"], a)
    assert list(res["mismatch"]) == [0, 3]
    assert list(res["first_mismatch"]) == [-1, 3]
    assert res["no_majority"] == 3 and res["first_no_majority"] == 3


def _nontransitive_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "vote_nontransitive.txt")) as f:
        for line in f:
            body = line.split("#", 1)[0].strip()
            if not body:
                continue
            vals, w, maj, bad = [x.strip() for x in body.split("|")]
            rows.append((vals.split(), int(w), bool(int(maj)),
                         [] if bad == "-" else [int(x) for x in bad.split(",")]))
    return rows


@pytest.mark.parametrize("row", _nontransitive_rows(), ids=lambda r: " ".join(r[0]))
def test_nontransitive_hand_cases(row):
    names, w, maj, bad = row
    val = {"A": 1024.0, "B": 1025.0, "C": 1026.0, "D": 4096.0}
    reps = [np.array([val[x]], dtype=np.float32) for x in names]
    res = oracle.vote(reps, "f32", 0.0, 2.0 ** -10)
    assert res["out"][0] == val[names[w]]
    assert (res["no_majority"] == 0) == maj
    assert [r for r in range(len(names)) if res["mismatch"][r]] == bad


# ---------------------------------------------------------------- invariants

def test_identical_replicas():
    p = synth.cfg2(n=50_000)
    a = p.replicas[0]
    res = oracle.vote([a, a.copy(), a.copy()], "f32", p.abs_tol, p.rel_tol)
    assert res["out"].tobytes() == a.tobytes()
    assert list(res["mismatch"]) == [0, 0, 0]
    assert list(res["first_mismatch"]) == [-1, -1, -1]
    assert res["no_majority"] == 0 and res["first_no_majority"] == -1
    assert np.array_equal(res["block_crc"], oracle.block_crc32c(a))


@pytest.mark.parametrize("dtype", ["f32", "f64", "i32"])
def test_single_faulty_replica_recovered(dtype):
    rng = np.random.default_rng(5)
    n, R = 40_000, 5
    if dtype == "i32":
        clean = synth.uniform_int(rng, n, "i32")
        tol = (0.0, 0.0)
    else:
        clean = synth.lognormal(rng, n, dtype)
        tol = synth.TOL[dtype]
    reps = [clean.copy() for _ in range(R)]
    who = rng.integers(0, R, size=n)
    idx = np.flatnonzero(rng.random(n) < 0.05)
    bits = rng.integers(0, 8 * clean.dtype.itemsize, size=idx.size)
    expected = [[] for _ in range(R)]
    within = np.zeros(n, dtype=bool)
    for i, bt in zip(idx, bits):
        r = who[i]
        synth.bit_flip(reps[r], np.array([i]), np.array([bt]))
        # a flip that stays within tolerance is not a fault under the stated rule
        if not oracle.eq(dtype, reps[r][i:i + 1], clean[i:i + 1], *tol):
            expected[r].append(int(i))
        else:
            within[i] = True
    res = oracle.vote(reps, dtype, *tol)
    out = res["out"]
    # real faults are voted away bit-exactly; where the flipped value is still
    # equal under the tolerance it may win (it is then equal to the clean value)
    assert out[~within].tobytes() == clean[~within].tobytes()
    for i in np.flatnonzero(within):
        assert oracle.eq(dtype, out[i:i + 1], clean[i:i + 1], *tol)
    if dtype == "i32":
        assert not within.any()
    assert res["no_majority"] == 0
    for r in range(R):
        assert res["mismatch"][r] == len(expected[r])
        assert res["first_mismatch"][r] == (expected[r][0] if expected[r] else -1)
    assert np.array_equal(res["block_crc"], oracle.block_crc32c(out))
    if out.tobytes() == clean.tobytes():
        assert np.array_equal(res["block_crc"], oracle.block_crc32c(clean))


def test_cfg1_faults_are_the_filtered_flips():
    p = synth.cfg1(n=1 << 16, flips=300)
    res = oracle.vote(p.replicas, "f32", p.abs_tol, p.rel_tol)
    clean, c = p.truth["clean"], p.replicas[2]
    exp = [int(i) for i in p.truth["flip_idx"]
           if not oracle.eq("f32", c[i:i + 1], clean[i:i + 1], p.abs_tol, p.rel_tol)]
    assert res["mismatch"][2] == len(exp) > 0
    assert res["first_mismatch"][2] == exp[0]
    # +-1..2 ULP on values in [-1, 1] is inside rel 1e-5 / abs 1e-6: not a fault
    assert res["mismatch"][1] == 0 and res["mismatch"][0] == 0


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_permutation_equivariance(seed):
    f64, i32 = synth.cfg3(n=1 << 14, block=1 << 10, ties=64)
    for p in (f64, i32):
        base = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol, with_ties=True)
        keep = (base["tie"] & 1) == 0
        reps = [np.where(keep, r, p.replicas[0]) for r in p.replicas]
        base = oracle.vote(reps, p.dtype, p.abs_tol, p.rel_tol)
        perm = np.random.default_rng(seed).permutation(p.R)
        res = oracle.vote([reps[k] for k in perm], p.dtype, p.abs_tol, p.rel_tol)
        assert list(res["mismatch"]) == [base["mismatch"][k] for k in perm]
        assert list(res["first_mismatch"]) == [base["first_mismatch"][k] for k in perm]
        assert res["no_majority"] == base["no_majority"]


def test_tie_sites_follow_lowest_index_rule():
    f64, i32 = synth.cfg3(n=1 << 14, block=1 << 10, ties=64)
    for p in (f64, i32):
        res = oracle.vote(p.replicas, p.dtype, p.abs_tol, p.rel_tol, with_ties=True)
        t = p.truth["tie_idx"]
        # {0,3} and {1,2} tie with support 2 each: replica 0 wins, no majority
        assert res["out"][t].tobytes() == p.replicas[0][t].tobytes()
        assert np.all(res["tie"][t] != 0)
        assert res["no_majority"] >= t.size
