"""Planted mistakes in the oracle are caught by its pins.

Each mutant is one plausible slip in oracle/mpgemm_oracle.c: a wrong sign,
a dropped term, a wrong index or operand, a wrong rounding rule, an
off-by-one limit.  For each one the test compiles a mutated copy of the
oracle (CPU only), points the oracle package at it through
MPGEMM_ORACLE_LIB, runs the oracle's pin tests (all but the slow
million-pair ones) in a child process and
requires them to fail (a failed assertion, or a loud abort of the oracle's
own range checks).  The unmutated source, compiled the same way, must pass,
so that a failure is the mutant's doing and not the harness's.  A mutant
that survives means a pin is missing.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpgemm_oracle.c")
PINS = ["tests/test_oracle_scalar.py", "tests/test_oracle_gemm.py", "tests/test_oracle_ozaki.py",
        "tests/test_oracle_via_mp.py"]

# name: (text in the source, its replacement, which occurrence (0-based), how many occurrences)
MUTANTS = {
    # error-free transformations
    "two_sum error sign": ("*e = ar + br;", "*e = ar - br;", 0, 1),
    "two_sum drops b's remainder": ("*e = ar + br;", "*e = ar;", 0, 1),
    "fast_two_sum error sign": ("*e = b - z;", "*e = z - b;", 0, 1),
    "two_prod error sign": ("*e = fma(a, b, -x);", "*e = -fma(a, b, -x);", 0, 1),
    # DD (double-word algorithms)
    "dd_add drops the low-word error": ("w = tl + vl;", "w = vl;", 0, 1),
    "dd_add adds lo to the other hi": ("two_sum(x.lo, y.lo, &th, &tl);", "two_sum(x.lo, y.hi, &th, &tl);", 0, 1),
    "dd_mul drops lo(x) hi(y)": ("cl2 = fma(x.lo, y.hi, tl1);", "cl2 = tl1;", 0, 1),
    "dd_mul uses hi(y) for lo(y)": ("tl1 = fma(x.hi, y.lo, tl0);", "tl1 = fma(x.hi, y.hi, tl0);", 0, 1),
    # QD (exact result rounded to four terms)
    "qd_add drops the fourth terms": ("for (int i = 0; i < 4; i++) { wfx_add_double(&W, a.x[i]); wfx_add_double(&W, b.x[i]); }",
                                      "for (int i = 0; i < 3; i++) { wfx_add_double(&W, a.x[i]); wfx_add_double(&W, b.x[i]); }", 0, 1),
    "qd_mul truncated to i + j < 4": ("for (int j = 0; j < 4; j++) wfx_add_prod(&W, a.x[i], b.x[j]);",
                                      "for (int j = 0; i + j < 4; j++) wfx_add_prod(&W, a.x[i], b.x[j]);", 0, 1),
    "exact rounding ties away from zero": ("if (rbit && (sticky || (mant & 1))) mant += 1;", "if (rbit) mant += 1;", 0, 1),
    "exact rounding ignores the sticky bits": ("sticky = wfx_any_below(&a, top - 53);", "sticky = 0;", 0, 1),
    "greedy terms add instead of subtract": ("wfx_add_double(a, -x[t]);", "wfx_add_double(a, x[t]);", 0, 1),
    "exact accumulator drops a borrow": ("borrow = (cur == 0);", "borrow = 0;", 0, 1),
    # multi-limb (RNE multiply and add)
    "multi-limb rounding ties away": ("if (rbit && (sticky || (M[0] & 1))) {", "if (rbit) {", 0, 1),
    "multi-limb rounding loses the sticky bits": ("int sticky = bi_any_below(S, sn, sh - 1);", "int sticky = 0;", 0, 1),
    "multi-limb round-up carry keeps the exponent": ("            *k += 1;\n", "            *k += 0;\n", 0, 1),
    "multi-limb product sign": ("r.s = x->s ^ y->s;", "r.s = x->s;", 0, 1),
    "multi-limb product exponent off by one": ("r.e = x->e + y->e - 32 * w + k;", "r.e = x->e + y->e - 32 * w + k + 1;", 0, 1),
    "multi-limb difference takes x's sign": ("else { bi_sub(S, Y, X, n); sign = y->s; }",
                                             "else { bi_sub(S, Y, X, n); sign = x->s; }", 0, 1),
    "multi-limb sum exponent from x": ("r.e = y->e + k;", "r.e = x->e + k;", 0, 1),
    "multi-limb far operand dropped too early": ("if (d >= p + 2) return *x;", "if (d >= p) return *x;", 0, 1),
    # conversions between expansions and multi-limb numbers
    "double to multi-limb exponent off by one": ("    r.e = ex;", "    r.e = ex + 1;", 0, 1),
    "multi-limb to double loses the lower limbs": (
        "int sticky = (top & 0x3FFu) != 0 || bi_any_below(v->m, w, (int64_t)p - 64);",
        "int sticky = (top & 0x3FFu) != 0;", 0, 1),
    "expansion to multi-limb reads term 0 only": ("mp_t x = mp_of_double(X[t * count + i], w);",
                                                  "mp_t x = mp_of_double(X[i], w);", 0, 1),
    "greedy expansion adds the term back": ("mp_t x = mp_of_double(-d, w);", "mp_t x = mp_of_double(d, w);", 0, 1),
    # Eq 1 / Eq 2 / Eq 3
    "simple: B transposed": ("for (int64_t k = 0; k < l; k++) el_mac(f, c, at(f, A, i, k), at(f, B, k, j));",
                             "for (int64_t k = 0; k < l; k++) el_mac(f, c, at(f, A, i, k), at(f, B, j, k));", 0, 1),
    "simple: k descending": ("for (int64_t k = 0; k < l; k++) el_mac(f, c, at(f, A, i, k), at(f, B, k, j));",
                             "for (int64_t k = l - 1; k >= 0; k--) el_mac(f, c, at(f, A, i, k), at(f, B, k, j));", 0, 1),
    "block: K panel one short": ("int64_t k1 = k0 + n_min < l ? k0 + n_min : l;",
                                 "int64_t k1 = k0 + n_min < l ? k0 + n_min - 1 : l;", 0, 1),
    "block: C zeroed per K panel": ("for (int64_t k = k0; k < k1; k++) el_mac(",
                                    "if (k0) el_zero(f, c); for (int64_t k = k0; k < k1; k++) el_mac(", 0, 1),
    "Strassen: P4 = A22 (B11 - B21)": ("mat_addsub(f, l2, n2, T, B21, B11, 1);", "mat_addsub(f, l2, n2, T, B11, B21, 1);", 0, 1),
    "Strassen: P7 with A12 + A22": ("mat_addsub(f, m2, l2, S, A12, A22, 1);", "mat_addsub(f, m2, l2, S, A12, A22, 0);", 0, 1),
    "Strassen: C22 adds P2": ("mat_addsub(f, m2, n2, C22, C22, P[2], 1);", "mat_addsub(f, m2, n2, C22, C22, P[2], 0);", 0, 1),
    "Strassen: C12 = P3 + P4": ("mat_addsub(f, m2, n2, C12, P[3], P[5], 0);", "mat_addsub(f, m2, n2, C12, P[3], P[4], 0);", 0, 1),
    "Strassen: zero extension copied back one column off": ("memcpy(at(&f, c, i, 0), at(&f, cp, i, 0), (size_t)n * f.esz);",
                                                            "memcpy(at(&f, c, i, 0), at(&f, cp, i, 1), (size_t)n * f.esz);", 0, 1),
    # exact checker
    "checker adds the tested value": ("wfx_add_double(&W, -Ct[q * NC + (size_t)(i * n + j)]);",
                                      "wfx_add_double(&W, Ct[q * NC + (size_t)(i * n + j)]);", 0, 1),
    "checker |A||B| ignores A's sign": ("wfx_add_prod(&Wa, sa * a[p], sb * b[q]);", "wfx_add_prod(&Wa, a[p], sb * b[q]);", 0, 1),
    "exact entries: wrong plane of B": ("wfx_add_prod(&W, A[p * NA + (size_t)(i * l + k)], B[q * NB + (size_t)(k * n + j)]);",
                                        "wfx_add_prod(&W, A[p * NA + (size_t)(i * l + k)], B[p * NB + (size_t)(k * n + j)]);", 0, 1),
    # split precision
    "row exponent one too large": ("e[i] = mx == INT32_MIN ? 0 : mx;", "e[i] = mx == INT32_MIN ? 0 : mx + 1;", 0, 1),
    "column exponent of the first row only": ("for (int64_t k = 0; k < rows; k++) {\n            int t = frexp_expo(hi[k * cols + j]);",
                                              "for (int64_t k = 0; k < 1; k++) {\n            int t = frexp_expo(hi[k * cols + j]);", 0, 1),
    "truncation ignores lo at an integer hi": ("if (hi > 0 && lo < 0) t = hi - 1.0;", "if (hi > 0 && lo < 0) t = hi;", 0, 1),
    "int8 digits scale lo by 2^6": ("double yh = ldexp(xh, 7), yl = ldexp(xl, 7);", "double yh = ldexp(xh, 7), yl = ldexp(xl, 6);", 0, 1),
    "levels drop the pairs of level S + 1": ("for (int t = 1; s + t <= S + 1; t++) {", "for (int t = 1; s + t <= S; t++) {", 0, 1),
    "int8 recombination: e - f": ("ldexp((double)v, e[i] + f[j] - 7 * g)", "ldexp((double)v, e[i] - f[j] - 7 * g)", 0, 1),
    "base-32 digits: lo without the headroom bit": ("double xh = ldexp(hi, -(e + 1)), xl = ldexp(lo, -(e + 1));",
                                                    "double xh = ldexp(hi, -(e + 1)), xl = ldexp(lo, -e);", 0, 1),
    "base-32 balancing keeps 16": ("        if (mag[s] >= 16) {", "        if (mag[s] > 16) {", 0, 2),
    "base-32 balancing drops the carry": ("            mag[s - 1] += 1;\n", "            mag[s - 1] += 0;\n", 0, 2),
    "base-32 recombination: one headroom bit": ("e[i] + f[j] + 2 * head - bits * g", "e[i] + f[j] + head - bits * g", 0, 2),
    "expansion digits read one digit high": ("mag[s] = (int)wfx_bits(&W, top - 5 * (s + 1), 5);",
                                             "mag[s] = (int)wfx_bits(&W, top - 5 * s, 5);", 0, 1),
    "expansion digits: balancing keeps 16": ("        if (mag[s] >= 16) {", "        if (mag[s] > 16) {", 1, 2),
    "expansion recombination: one headroom bit": ("e[i] + f[j] + 2 * head - bits * g", "e[i] + f[j] + head - bits * g", 1, 2),
    # second batch: rarer paths (zeros, carries, partial limbs, negative edges)
    "dd_mul drops the product's error": ("cl3 = cl1 + cl2;", "cl3 = cl2;", 0, 1),
    "schoolbook product drops the carry": ("uint64_t t = (uint64_t)x->m[i] * y->m[j] + P[i + j] + c;",
                                           "uint64_t t = (uint64_t)x->m[i] * y->m[j] + P[i + j];", 0, 1),
    "exact cancellation keeps x's sign": ("if (c == 0) return mp_zero(0);", "if (c == 0) return mp_zero(x->s);", 0, 1),
    "zero plus zero ORs the signs": ("return mp_zero(x->s & y->s);", "return mp_zero(x->s | y->s);", 0, 1),
    "multi-limb accumulator starts at -0": ("if (f->kind == F_MP) ((uint32_t *)c)[1] = 2u;",
                                            "if (f->kind == F_MP) ((uint32_t *)c)[1] = 3u;", 0, 1),
    "short multi-limb sum: exponent sign": ("*k = L - p;", "*k = p - L;", 0, 1),
    "exact rounding: sticky misses the partial limb": (
        "if (r && q < WFX_LIMBS && (a->w[q] & ((1u << r) - 1u))) return 1;", ";", 0, 1),
    "multi-limb rounding: sticky misses the partial limb": ("if (r && q < n && (a[q] & ((1u << r) - 1u))) return 1;", ";", 0, 1),
    "truncation ignores lo at a negative integer hi": ("else if (hi < 0 && lo > 0) t = hi + 1.0;",
                                                       "else if (hi < 0 && lo > 0) t = hi;", 0, 1),
    "int8 digits drop lo after the first": ("two_sum(yh - t, yl, &xh, &xl);", "two_sum(yh - t, 0.0, &xh, &xl);", 0, 2),
    "base-32 digits drop lo after the first": ("two_sum(yh - t, yl, &xh, &xl);", "two_sum(yh - t, 0.0, &xh, &xl);", 1, 2),
    "expansion to multi-limb starts at -0": ("mp_t c = mp_zero(0);", "mp_t c = mp_zero(1);", 0, 1),
    "greedy expansion never subtracts": ("r = mp_add(&r, &x, w);", "(void)x;", 0, 1),
    "checker |A||B| ignores B's sign": ("sb = b[0] < 0 ? -1.0 : 1.0;", "sb = 1.0;", 0, 1),
    "Strassen: P1 with B11 - B22": ("mat_addsub(f, l2, n2, T, B11, B22, 0);", "mat_addsub(f, l2, n2, T, B11, B22, 1);", 0, 1),
    "Strassen: P6 with A11 - A21": ("mat_addsub(f, m2, l2, S, A21, A11, 1);", "mat_addsub(f, m2, l2, S, A11, A21, 1);", 0, 1),
    "Strassen: P2 with B22": ("gemm_strassen(f, m2, l2, n2, S, B11, P[2], n_min, depth - 1);",
                              "gemm_strassen(f, m2, l2, n2, S, B22, P[2], n_min, depth - 1);", 0, 1),
    "levels start at slice 2": ("for (int s = 1; s <= S; s++)\n        for (int t = 1;", "for (int s = 2; s <= S; s++)\n        for (int t = 1;", 0, 1),
    "int8 recombination: 7 (g - 1)": ("e[i] + f[j] - 7 * g)", "e[i] + f[j] - 7 * (g - 1))", 0, 1),
    "zero has exponent 0 in the row maximum": ("if (x == 0.0) return INT32_MIN;", "if (x == 0.0) return 0;", 0, 1),
    # third batch: element operations of Eq 3, the final rounding, conversions, the checker
    "QD difference adds": ("sub ? qd_neg(Y) : Y", "Y", 0, 1),
    "multi-limb difference adds": ("if (sub) Y = mp_neg(Y);", "(void)sub;", 0, 1),
    "greedy rounding one term short": ("for (int t = 0; t < nterms; t++) {", "for (int t = 0; t + 1 < nterms; t++) {", 0, 1),
    "exact rounding: exponent off by one": ("r = ldexp((double)mant, top - 52 - WFX_FRAC);",
                                           "r = ldexp((double)mant, top - 53 - WFX_FRAC);", 0, 1),
    "double to multi-limb drops the low word": ("r.m[w - 2] = (uint32_t)top;", "r.m[w - 2] = 0;", 0, 1),
    "checker reads A's leading term only": ("            for (int p = 0; p < terms; p++)\n                for (int q = 0; q < terms; q++) {",
                                            "            for (int p = 0; p < 1; p++)\n                for (int q = 0; q < terms; q++) {", 0, 1),
}


def _mutate(text, old, new, which, count):
    assert text.count(old) == count, f"{old!r} occurs {text.count(old)} times, expected {count}"
    at = -1
    for _ in range(which + 1):
        at = text.index(old, at + 1)
    return text[:at] + new + text[at + len(old):]


def _run(name, src_text, workdir):
    sys.path.insert(0, ROOT)
    import oracle
    tag = "%02d" % (list(MUTANTS).index(name) if name in MUTANTS else 99)
    src = os.path.join(workdir, f"mutant_{tag}.c")
    lib = os.path.join(workdir, f"mutant_{tag}.so")
    with open(src, "w") as fh:
        fh.write(src_text)
    oracle.compile_source(src, lib)
    env = dict(os.environ, MPGEMM_ORACLE_LIB=lib, OMP_NUM_THREADS="1")
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m",
                        "not gpu and not slow", *PINS], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    tail = (p.stdout + p.stderr).strip().splitlines()[-3:]
    return p.returncode, tail


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    workdir = str(tmp_path_factory.mktemp("mutants"))
    with open(SRC) as fh:
        text = fh.read()
    jobs = {"(unmutated)": text}
    for name, (old, new, which, count) in MUTANTS.items():
        jobs[name] = _mutate(text, old, new, which, count)
    with ThreadPoolExecutor(max_workers=max(2, min(16, os.cpu_count() or 2))) as ex:
        futs = {name: ex.submit(_run, name, t, workdir) for name, t in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_unmutated_oracle_passes_its_pins(outcomes):
    rc, tail = outcomes["(unmutated)"]
    assert rc == 0, tail


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_is_caught(outcomes, name):
    rc, tail = outcomes[name]
    # 1: a pin failed; negative / 134: the oracle aborted on one of its range checks
    assert rc not in (0, 5), f"mutant survived the pins: {name}"
