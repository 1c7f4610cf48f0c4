"""The oracle's pins catch plausible mistakes in the oracle.

Each case copies oracle/ref_vote.c, plants one mistake in the copy (a flipped
tie rule, a dropped tolerance term, a wrong CRC parameter, ...), builds it, and
runs a compact set of the pins used in test_oracle_*.py against it: the
published CRC32C vectors, the SSE4.2 instruction on a partial block, the
hand-derived table of float comparisons, brute force against the group
formulation, the paper's R = 2 case.  Every mutant must fail at least one pin,
and the unmodified source must pass them all.  The oracle under oracle/ is not
touched."""
import ctypes
import itertools
import os
import re
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = open(os.path.join(ROOT, "oracle", "ref_vote.c")).read()
DT = {"i32": 0, "f32": 5, "f64": 6}
NP = {"i32": np.int32, "f32": np.float32, "f64": np.float64}

MUTANTS = {
    "tie_highest_index": (r"if \(s\[r\] > s\[w\]\)", "if (s[r] >= s[w])"),
    "majority_ge": (r"if \(!\(2 \* s\[w\] > R\)\)", "if (!(2 * s[w] >= R))"),
    "abs_term_dropped": (r"return d <= abs_t \|\| d <= t;", "return d <= t;"),
    "min_instead_of_max": (r"float m = fabsf\(a\) > fabsf\(b\) \? fabsf\(a\) : fabsf\(b\);",
                           "float m = fabsf(a) < fabsf(b) ? fabsf(a) : fabsf(b);"),
    "relative_to_a_only": (r"float t = rel_t \* m;", "float t = rel_t * fabsf(a);"),
    "inf_rule_dropped": (r"if \(isinf\(a\) \|\| isinf\(b\)\)\n        return 0;                               /\* \(iii\) \*/\n    float",
                         "float"),
    "exclusive_boundary_f64": (r"return d <= abs_t \|\| d <= t;\n}\n\n/\* eq of two",
                               "return d < abs_t || d < t;\n}\n\n/* eq of two"),
    "first_index_overwritten": (r"if \(first_mismatch\[r\] < 0\)\n                    first_mismatch\[r\]",
                                "first_mismatch[r]"),
    "mismatch_vs_replica0": (r"if \(!e\[r\]\[w\]\) \{", "if (!e[r][0]) {"),
    "crc_no_final_xor": (r"c = crc_table\[\(c \^ p\[i\]\) & 0xFFu\] \^ \(c >> 8\);\n    return c \^ 0xFFFFFFFFu;",
                         "c = crc_table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);\n    return c;"),
    "crc_init_zero": (r"uint32_t ref_crc32c\(const uint8_t \*p, uint64_t n\)\n\{\n    uint32_t c = 0xFFFFFFFFu;",
                      "uint32_t ref_crc32c(const uint8_t *p, uint64_t n)\n{\n    uint32_t c = 0;"),
    "crc32_polynomial": (r"c = \(c & 1u\) \? \(c >> 1\) \^ 0x82F63B78u : \(c >> 1\);\n        crc_table",
                         "c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : (c >> 1);\n        crc_table"),
    "tail_block_full_length": (r"uint64_t len = nbytes - off < block_bytes \? nbytes - off : block_bytes;",
                               "uint64_t len = block_bytes;"),
    "fast_math": None,
}


def _build(src, tmp, name, extra=()):
    c = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(c, "w") as f:
        f.write(src)
    flags = ["-O2", "-std=c11", "-fPIC", "-shared"] + list(extra)
    if not extra:
        flags += ["-ffp-contract=off", "-fno-fast-math"]
    subprocess.check_call(["gcc"] + flags + ["-o", so, c, "-lm"])
    L = ctypes.CDLL(so)
    L.ref_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.ref_crc32c.restype = ctypes.c_uint32
    L.ref_block_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p]
    L.ref_eq.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
    L.ref_vote.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                           ctypes.c_double] + [ctypes.c_void_p] * 7
    return L


class _Lib:
    def __init__(self, L):
        self.L = L

    def crc(self, b):
        b = np.ascontiguousarray(np.frombuffer(bytes(b), dtype=np.uint8))
        return int(self.L.ref_crc32c(b.ctypes.data if b.size else None, b.size))

    def block_crc(self, b, block):
        nb = (b.size + block - 1) // block
        out = np.zeros(nb, dtype=np.uint32)
        self.L.ref_block_crc32c(b.ctypes.data, b.size, block, out.ctypes.data)
        return out

    def eq(self, dt, a, b, at, rt):
        x = np.array([a], dtype=np.uint32 if dt == "f32" else np.uint64)
        y = np.array([b], dtype=x.dtype)
        return bool(self.L.ref_eq(DT[dt], x.ctypes.data, y.ctypes.data, at, rt))

    def vote(self, reps, dt, at=0.0, rt=0.0):
        reps = [np.ascontiguousarray(r) for r in reps]
        R, n = len(reps), reps[0].size
        ptrs = (ctypes.c_void_p * R)(*[r.ctypes.data for r in reps])
        out = np.empty(n, dtype=reps[0].dtype)
        mism = np.zeros(R, dtype=np.uint64)
        first = np.zeros(R, dtype=np.int64)
        nm = np.zeros(1, dtype=np.uint64)
        fnm = np.zeros(1, dtype=np.int64)
        self.L.ref_vote(ctypes.cast(ptrs, ctypes.c_void_p), R, n, DT[dt], at, rt, out.ctypes.data, None,
                        mism.ctypes.data, first.ctypes.data, nm.ctypes.data, fnm.ctypes.data, None)
        return out, list(mism), list(first), int(nm[0]), int(fnm[0])


def _pins(lib, hw):
    """Returns the names of the pins that fail."""
    failed = []
    # published CRC32C values
    if lib.crc(b"123456789") != 0xE3069283 or lib.crc(bytes(32)) != 0x8A9136AA or \
            lib.crc(bytes(range(32))) != 0x46DD794E:
        failed.append("crc_vectors")
    # partial last block against the hardware instruction
    rng = np.random.default_rng(0)
    b = rng.integers(0, 256, size=3 * 4096 + 1000, dtype=np.uint8)
    got = lib.block_crc(b, 4096)
    if [int(x) for x in got] != [hw(b[i:i + 4096]) for i in range(0, b.size, 4096)]:
        failed.append("block_partition")
    # hand-derived comparisons
    with open(os.path.join(HERE, "golden", "eq_special.txt")) as f:
        for line in f:
            body = line.split("#", 1)[0].strip()
            if not body:
                continue
            dt, a, bb, at, rt, exp = body.split()
            if lib.eq(dt, int(a, 16), int(bb, 16), float(at), float(rt)) != bool(int(exp)) or \
                    lib.eq(dt, int(bb, 16), int(a, 16), float(at), float(rt)) != bool(int(exp)):
                failed.append("eq_table")
                break
    # brute force against groups of equal values
    for R, dt, alphabet, group in ((3, "f32", {"C": 1.0, "Cp": float(np.float32(1.0) + np.float32(2 ** -22)),
                                              "F1": -3.5, "F2": 1e20}, {"C": "c", "Cp": "c", "F1": 1, "F2": 2}),
                                   (4, "i32", {"a": 5, "b": 6, "c": 7, "d": 200}, None)):
        group = group or {k: k for k in alphabet}
        pats = list(itertools.product(list(alphabet), repeat=R))
        reps = [np.array([alphabet[p[r]] for p in pats], dtype=NP[dt]) for r in range(R)]
        out, mism, first, nm, fnm = lib.vote(reps, dt, 1e-6, 1e-5)
        exp_m, exp_f, exp_nm = [0] * R, [-1] * R, 0
        ok = True
        for i, p in enumerate(pats):
            groups = {}
            for r, lab in enumerate(p):
                groups.setdefault(group[lab], []).append(r)
            best = max(groups.values(), key=lambda g: (len(g), -g[0]))
            ok &= out[i].tobytes() == reps[best[0]][i].tobytes()
            for r in range(R):
                if r not in best:
                    exp_m[r] += 1
                    exp_f[r] = i if exp_f[r] < 0 else exp_f[r]
            exp_nm += 0 if 2 * len(best) > R else 1
        if not ok or [int(x) for x in mism] != exp_m or [int(x) for x in first] != exp_f or nm != exp_nm:
            failed.append(f"brute_force_R{R}")
    # the paper's R = 2 case
    a = np.arange(50, dtype=np.int32)
    b2 = a.copy()
    b2[[3, 40]] += 1
    out, mism, first, nm, fnm = lib.vote([a, b2], "i32")
    if [int(x) for x in mism] != [0, 2] or [int(x) for x in first] != [-1, 3] or nm != 2:
        failed.append("dmr")
    return failed


@pytest.fixture(scope="module")
def hw(tmp_path_factory):
    with open("/proc/cpuinfo") as f:
        if "sse4_2" not in f.read():
            pytest.skip("host CPU has no SSE4.2")
    so = str(tmp_path_factory.mktemp("hw") / "libhw.so")
    subprocess.check_call(["gcc", "-O2", "-msse4.2", "-fPIC", "-shared", "-o", so,
                           os.path.join(HERE, "pins", "crc32c_sse42.c")])
    L = ctypes.CDLL(so)
    L.hw_crc32c.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
    L.hw_crc32c.restype = ctypes.c_uint32
    return lambda b: int(L.hw_crc32c(np.ascontiguousarray(b).ctypes.data, b.size))


def test_unmodified_oracle_passes(tmp_path, hw):
    assert _pins(_Lib(_build(SRC, str(tmp_path), "orig")), hw) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, hw, name):
    m = MUTANTS[name]
    if m is None:
        # flush-to-zero and contraction: the subnormal rows of the table catch it
        lib = _Lib(_build(SRC, str(tmp_path), name, extra=["-ffast-math"]))
    else:
        pat, rep = m
        src, k = re.subn(pat, lambda _: rep, SRC, count=1)
        assert k == 1, f"mutation {name} did not apply"
        lib = _Lib(_build(src, str(tmp_path), name))
    assert _pins(lib, hw), f"no pin caught the mutant {name}"
