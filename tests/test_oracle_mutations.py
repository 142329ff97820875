"""The oracle's pins catch plausible mistakes: each test plants one mistake
in a copy of the oracle's C source (a wrong constant, index, sign, dropped
term or transposed operand), builds it, and runs the pin tests against it
(through QPADL_ORACLE_LIB); at least one pin must fail.  The unmodified
source, built the same way, must pass them all."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "qpadl_oracle.c")

# (name, text in the source, replacement): every text must occur exactly once, and
# every mutant reads only inside its arrays (transposed indices stay in range)
MUTATIONS = [
    ("splitmix gamma", "(i + 1u) * 0x9E3779B97F4A7C15ull", "(i + 1u) * 0x9E3779B97F4A7C17ull"),
    ("splitmix counter off by one", "seed + (i + 1u) *", "seed + i *"),
    ("splitmix finaliser shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;",
     "z = (z ^ (z >> 28)) * 0x94D049BB133111EBull;"),
    ("gen_a low half", "(uint32_t)(oracle_splitmix64_at(seed, j * n + k) >> 32)",
     "(uint32_t)(oracle_splitmix64_at(seed, j * n + k))"),
    ("gen_a column-major counter", "oracle_splitmix64_at(seed, j * n + k)", "oracle_splitmix64_at(seed, k * C + j)"),
    ("hint signed digits", "acc += (uint32_t)D[(uint64_t)i * C + j] * A[j * n + k];",
     "acc += (uint32_t)(int8_t)D[(uint64_t)i * C + j] * A[j * n + k];"),
    ("hint transposed A", "acc += (uint32_t)D[(uint64_t)i * C + j] * A[j * n + k];",
     "acc += (uint32_t)D[(uint64_t)i * C + j] * A[k * C + j];"),
    ("hint last column dropped", "for (uint64_t j = 0; j < C; ++j)\n                acc += (uint32_t)D[(uint64_t)i * C + j] * A",
     "for (uint64_t j = 0; j + 1 < C; ++j)\n                acc += (uint32_t)D[(uint64_t)i * C + j] * A"),
    ("query noise dropped", "        acc += (uint32_t)e[j];\n", "\n"),
    ("query noise sign", "        acc += (uint32_t)e[j];\n", "        acc -= (uint32_t)e[j];\n"),
    ("query Delta at the wrong column", "if (j == col)", "if (j == col + 1)"),
    ("query secret index", "acc += A[j * n + k] * s[k];", "acc += A[j * n + k] * s[n - 1 - k];"),
    ("answer signed digits", "acc += (uint32_t)D[(uint64_t)i * C + j] * qu[j];",
     "acc += (uint32_t)(int8_t)D[(uint64_t)i * C + j] * qu[j];"),
    ("answer transposed D", "acc += (uint32_t)D[(uint64_t)i * C + j] * qu[j];",
     "acc += (uint32_t)D[j * R + (uint64_t)i] * qu[j];"),
    ("answer_batch query order", "oracle_answer(D, R, C, Q + b * C, ans + b * R, nthreads);",
     "oracle_answer(D, R, C, Q + (B - 1 - b) * C, ans + b * R, nthreads);"),
    ("recover floor instead of round", "out[i] = (uint8_t)((uint32_t)(x + half) >> shift);",
     "out[i] = (uint8_t)((uint32_t)(x) >> shift);"),
    ("recover mask added", "uint32_t x = ans[i] - mask;", "uint32_t x = ans[i] + mask;"),
    ("recover shift off by one", "uint32_t shift = 32u - log2_p;", "uint32_t shift = 31u - log2_p;"),
    ("recover transposed H", "mask += H[i * n + k] * s[k];", "mask += H[k * R + i] * s[k];"),
    ("chor OR instead of XOR", "rho[c] ^= db[i * w + c];", "rho[c] |= db[i * w + c];"),
    ("chor query bit order", "if ((qb[i / 32] >> (i % 32)) & 1u) {", "if ((qb[i / 32] >> (31 - i % 32)) & 1u) {"),
    ("chor last row skipped", "for (uint64_t i = 0; i < r; ++i) {\n            if ((qb",
     "for (uint64_t i = 0; i + 1 < r; ++i) {\n            if ((qb"),
    ("chor unit bit misplaced", "acc ^= 1u << (theta % 32);", "acc ^= 1u << ((theta + 1) % 32);"),
    ("chor reconstruct drops a response", "for (uint64_t j = 0; j < ell; ++j)\n            acc ^= responses",
     "for (uint64_t j = 1; j < ell; ++j)\n            acc ^= responses"),
    ("goldberg wrong modulus", "acc = (acc + (uint64_t)qb[j] * D[(uint64_t)i * C + j]) % p;",
     "acc = (acc + (uint64_t)qb[j] * D[(uint64_t)i * C + j]) % (p + 1);"),
    ("goldberg transposed D", "acc = (acc + (uint64_t)qb[j] * D[(uint64_t)i * C + j]) % p;",
     "acc = (acc + (uint64_t)qb[j] * D[j * R + (uint64_t)i]) % p;"),
    ("goldberg secret at the wrong record", "(j == theta ? 1u : 0u)", "(j == theta + 1 ? 1u : 0u)"),
    ("goldberg reversed coefficients", "v = (v * alpha[k] + coef[j * t + (u - 1)]) % p;",
     "v = (v * alpha[k] + coef[j * t + (t - u)]) % p;"),
    ("goldberg Lagrange denominator sign", "den = den * ((alpha[m] + p - alpha[s]) % p) % p;",
     "den = den * ((alpha[s] + p - alpha[m]) % p) % p;"),
    ("goldberg Lagrange numerator point", "num = num * alpha[m] % p;", "num = num * alpha[s] % p;"),
    ("delta first entry big-endian", "db[b * C + j] = (uint8_t)(first >> (8 * b));",
     "db[b * C + j] = (uint8_t)(first >> (8 * (3 - b)));"),
    ("delta width one byte short", "while (w < 4 && dmax >= (1u << (8 * w)))", "while (w < 4 && dmax > (1u << (8 * w)))"),
    ("delta difference two back", "- oracle_entry(x, n, j * E + i - 1);\n            for (uint32_t b = 0; b < w; ++b)",
     "- oracle_entry(x, n, j * E + (i >= 2 ? i - 2 : 0));\n            for (uint32_t b = 0; b < w; ++b)"),
    ("delta decode byte order", "d |= (uint32_t)digits[4 + (i - 1) * w + b] << (8 * b);",
     "d |= (uint32_t)digits[4 + (i - 1) * w + b] << (8 * (w - 1 - b));"),
    ("delta padding with zeros", "return k < n ? x[k] : x[n - 1];", "return k < n ? x[k] : 0u;"),
]


def _build(src_text: str, out_dir) -> str:
    c = os.path.join(str(out_dir), "oracle.c")
    so = os.path.join(str(out_dir), "liboracle.so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", c, "-o", so], check=True)
    return so


def _run_pins(so: str) -> int:
    env = dict(os.environ, QPADL_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                        "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT, env=env, capture_output=True,
                       timeout=600)
    return r.returncode


def test_unmodified_source_passes_the_pins(tmp_path):
    assert _run_pins(_build(open(SRC).read(), tmp_path)) == 0


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site of '{name}' not unique"
    # pytest exits 1 when a test fails (a crash would give another code)
    assert _run_pins(_build(src.replace(old, new), tmp_path)) == 1, f"no pin caught: {name}"
