"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a wrong operand, a wrong
index) in a copy of the oracle's C source, builds it, and runs the pin
tests (closed forms, invariants, brute force, and the big-integer
restatement of the query) against it in a subprocess: at least one pin must
fail.  The real
oracle is untouched."""
from __future__ import annotations

import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ptrhash_oracle.c")

MUTATIONS = {
    "part uses lo instead of hi": ("*part = orc_hi(L->P, h);", "*part = orc_lo(L->P, h);"),
    "gamma3 drops the x/256 term": ("return half_sum - (half_sum >> 8) + (x >> 8);",
                                    "return half_sum - (half_sum >> 8);"),
    "gamma3 cube from the wrong operand": ("uint64_t x3 = orc_hi(x2, x);", "uint64_t x3 = orc_hi(x2, x2);"),
    "slot drops the part offset": ("return part * m->L.S + orc_reduce(m->L.reduce, m->C, x, m->L.S);",
                                   "return orc_reduce(m->L.reduce, m->C, x, m->L.S);"),
    "reduce uses lo instead of hi": ("if (reduce == ORC_REDUCE_POW2) return orc_hi(C, x) % S;",
                                     "if (reduce == ORC_REDUCE_POW2) return orc_lo(C, x) % S;"),
    "pilot hash adds instead of xor": ("return C * (pilot ^ seed); }", "return C * (pilot + seed); }"),
    "clef lookup drops -i": ("return 256 * (offset + sel - i) + line[20 + i];",
                             "return 256 * (offset + sel) + line[20 + i];"),
    "clef encode drops the index bit": ("uint64_t bit = i + ((v[i] >> 8) - offset);",
                                        "uint64_t bit = (v[i] >> 8) - offset;"),
    "remap without predecessor fill": ("        else F[j] = prev;\n", "\n"),
    "buckets per part ignore alpha": ("uint64_t B = (uint64_t)ceil(alpha * (double)S / lambda);",
                                      "uint64_t B = (uint64_t)ceil((double)S / lambda);"),
    "string mixer with a wrong shift": ("    z ^= z >> 27;\n", "    z ^= z >> 28;\n"),
    "string hash drops the seed from the finish": ("return str_mix(acc ^ (len * K2) ^ seed);",
                                                   "return str_mix(acc ^ (len * K2));"),
    "string fold drops the high half": ("return (uint64_t)(p >> 64) ^ (uint64_t)p;", "return (uint64_t)p;"),
    "string words combined with xor": ("acc += str_fold(w ^ (seed + j * K1), K3);", "acc ^= str_fold(w ^ (seed + j * K1), K3);"),
    "string word tweak off by one word": ("acc += str_fold(w ^ (seed + j * K1), K3);",
                                          "acc += str_fold(w ^ (seed + (j + 1) * K1), K3);"),
    "string words read big-endian": ("w |= byte << (8 * b);", "w |= byte << (56 - 8 * b);"),
    "string hash drops the length": ("return str_mix(acc ^ (len * K2) ^ seed);", "return str_mix(acc ^ seed);"),
    "x mod S layout keeps an even S": ("            if (S % 2 == 0) S += 1;\n",
                                      "            if (is_pow2(S)) S += 1;\n"),
    "128-bit query buckets by the low half": ("orc_part_bucket(&m->L, m->gamma, hb, &part, &b);",
                                              "orc_part_bucket(&m->L, m->gamma, hs, &part, &b);"),
    "128-bit build parts by the low half": ("for (uint64_t i = 0; i < n; i++) part_start[orc_hi(L.P, hb[i]) + 1]++;",
                                            "for (uint64_t i = 0; i < n; i++) part_start[orc_hi(L.P, h[i]) + 1]++;"),
    # Consistent in the builder and the query, so every structure stays a
    # bijection: only the independent restatement of Eq. hp / Eq. slot sees them.
    "pilot hash drops the factor C": ("return C * (pilot ^ seed); }", "return (pilot ^ seed); }"),
    "slot adds hp instead of xor (builder and query)": [
        ("uint64_t x = hs ^ orc_hp(m->C, m->seed, pilot);", "uint64_t x = hs + orc_hp(m->C, m->seed, pilot);"),
        ("orc_reduce(m->L.reduce, m->C, ps->h[j] ^ hp, m->L.S);", "orc_reduce(m->L.reduce, m->C, ps->h[j] + hp, m->L.S);"),
    ],
}
PIN_FILES = ["test_oracle_pins.py", "test_oracle_bigint.py"]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, tmp_path):
    edits = MUTATIONS[name]
    src = open(SRC).read()
    for old, new in ([edits] if isinstance(edits, tuple) else edits):
        assert src.count(old) == 1, f"mutation anchor not found: {name}"
        src = src.replace(old, new)
    mutant = tmp_path / "ptrhash_oracle.c"
    mutant.write_text(src)
    (tmp_path / "ptrhash_oracle.h").write_text(open(os.path.join(ROOT, "oracle", "ptrhash_oracle.h")).read())
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", str(lib),
                           str(mutant), "-lm"])
    env = dict(os.environ, PTRHASH_ORACLE_LIB=str(lib))
    res = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                          *[os.path.join(ROOT, "tests", f) for f in PIN_FILES]],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"no pin caught: {name}\n{res.stdout[-2000:]}"
