"""Planted mistakes in the oracle must fail its pins.

Each case below is a plausible slip in ``oracle/messi_oracle.c`` -- a wrong
divisor, a flipped comparison, a dropped term, a swapped operand, an
off-by-one window, a reversed tie-break.  The test compiles a copy of the
source with that one change (the committed source is never touched), runs
``tests/test_oracle_pins.py`` against the mutated library in a subprocess,
and requires at least one pin to fail.  The Python side of the oracle (leaf
grouping, streamed k-NN) gets the same treatment through a copy of the
package with one line changed."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "messi_oracle.c")
HDR = os.path.join(ROOT, "oracle", "messi_oracle.h")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

MUTANTS = [
    ("PAA divides by m + 1",
     "paa[s] = sum / (double)m;", "paa[s] = sum / (double)(m + 1);"),
    ("a PAA on a breakpoint takes the lower symbol",
     "if (beta[j - 1] <= paa[s]) ++count;", "if (beta[j - 1] < paa[s]) ++count;"),
    ("breakpoints at j / (c + 1)",
     "std_normal_quantile((double)j / (double)card)", "std_normal_quantile((double)j / (double)(card + 1))"),
    ("CDF series loses its alternating sign",
     "dd_mul(power, (dd_t){-half_x2.hi, -half_x2.lo})", "dd_mul(power, half_x2)"),
    ("quantile rounded to the farther of its two neighbours",
     "return cdf_minus_dd(m, p).hi < 0.0 ? hi : lo;", "return cdf_minus_dd(m, p).hi < 0.0 ? lo : hi;"),
    ("CDF series term divided by 2n - 1",
     "dd_t term = dd_div_d(power, (double)(2 * n + 1));", "dd_t term = dd_div_d(power, (double)(2 * n - 1));"),
    ("iSAX key takes the symbol bits LSB first",
     "uint32_t bit = (sym[s] >> (b - 1 - j)) & 1u;", "uint32_t bit = (sym[s] >> j) & 1u;"),
    ("ED adds instead of subtracting",
     "double d = (double)q[t] - (double)x[t];", "double d = (double)q[t] + (double)x[t];"),
    ("ED mindist drops the segment length",
     "        s += d * d;\n    }\n    return (double)m * s;\n}\n\n/* ----------------------------------------------------------------"
     " Sec. 3.4 */",
     "        s += d * d;\n    }\n    return s;\n}\n\n/* ----------------------------------------------------------------"
     " Sec. 3.4 */"),
    ("DTW mindist tests the lower envelope against the region floor",
     "if (paaU[k] < lo) d = lo - paaU[k];", "if (paaL[k] < lo) d = lo - paaL[k];"),
    ("envelope window one point short on the right",
     "        int b = i + r > n - 1 ? n - 1 : i + r;\n        double hi = (double)q[a], lo = (double)q[a];",
     "        int b = i + r - 1 > n - 1 ? n - 1 : i + r - 1;\n        double hi = (double)q[a], lo = (double)q[a];"),
    ("LB_Keogh with the envelope's sides swapped",
     "        if (c > U[i]) d = c - U[i];\n        else if (c < L[i]) d = c - L[i];",
     "        if (c > L[i]) d = c - L[i];\n        else if (c < U[i]) d = c - U[i];"),
    ("LB_Improved drops its second term",
     "return first + second;", "return first;"),
    ("LB_Improved does not clamp the candidate",
     "h[i] = c > U[i] ? U[i] : (c < L[i] ? L[i] : c);", "h[i] = c;"),
    ("DTW without the diagonal step",
     "                if (i > 0 && j > 0 && D[(size_t)(i - 1) * n + j - 1] < best)\n"
     "                    best = D[(size_t)(i - 1) * n + j - 1];\n",
     ""),
    ("DTW window one cell narrow",
     "        int jhi = i + r > n - 1 ? n - 1 : i + r;",
     "        int jhi = i + r - 1 > n - 1 ? n - 1 : i + r - 1;\n        if (jhi < jlo) jhi = jlo;"),
    ("ties go to the larger id",
     "return da < db || (da == db && ia < ib);", "return da < db || (da == db && ia > ib);"),
    ("window z-normalisation with the sample variance",
     "const double var = ss / (double)n;", "const double var = ss / (double)(n - 1);"),
    ("window mean over n + 1 points",
     "const double mean = sum / (double)n;", "const double mean = sum / (double)(n + 1);"),
    ("region upper edge one breakpoint too high",
     "static double region_hi(int v, int card, const double *beta) { return v == card - 1 ? INFINITY : beta[v]; }",
     "static double region_hi(int v, int card, const double *beta) { return v >= card - 2 ? INFINITY : beta[v + 1]; }"),
    ("envelope keeps min and max the wrong way round",
     "            if ((double)q[j] > hi) hi = (double)q[j];\n            if ((double)q[j] < lo) lo = (double)q[j];",
     "            if ((double)q[j] < hi) hi = (double)q[j];\n            if ((double)q[j] > lo) lo = (double)q[j];"),
    ("summaries read every row from the first",
     "        orc_paa(data + i * (int64_t)n, n, w, paa);", "        orc_paa(data, n, w, paa);"),
    ("k-NN ignores the id base of a block",
     "topk_insert(bd + base, bi + base, &bc[(size_t)t * nq + qi], k, d, id_base + row);",
     "topk_insert(bd + base, bi + base, &bc[(size_t)t * nq + qi], k, d, row);"),
    ("k-NN drops a full array's last slot on a tie",
     "    if (*cnt == k && !before(d, id, kd[k - 1], ki[k - 1])) return;",
     "    if (*cnt == k && !before(d, id, kd[k - 1], ki[k - 1])) return;\n    if (*cnt == k - 1 && k > 1) return;"),
    ("windows ignore the stride",
     "        const float *x = series + i * stride;\n        float *o = out + i * (int64_t)n;",
     "        const float *x = series + i;\n        float *o = out + i * (int64_t)n;"),
    ("DTW mindist BELOW case against the region floor",
     "else if (paaL[k] > hi) d = paaL[k] - hi;", "else if (paaL[k] > lo) d = paaL[k] - lo;"),
    ("iSAX key interleaves segment-major",
     "            int p = j * w + s;                          /* position from the MSB */",
     "            int p = s * b + j;                          /* position from the MSB */"),
]


@pytest.fixture(scope="module")
def source():
    return open(SRC).read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(tmp_path, source, name, old, new):
    assert source.count(old) == 1, f"mutation site not found exactly once: {name}"
    (tmp_path / "messi_oracle.c").write_text(source.replace(old, new))
    shutil.copy(HDR, tmp_path / "messi_oracle.h")
    lib = tmp_path / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(lib), str(tmp_path / "messi_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, MESSI_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"planted mistake survived every pin: {name}\n{r.stdout[-2000:]}"


def test_control_unmutated_copy_passes(tmp_path, source):
    # the same harness on the unchanged source: every pin passes, so a failure
    # above comes from the planted mistake and not from the harness
    (tmp_path / "messi_oracle.c").write_text(source)
    shutil.copy(HDR, tmp_path / "messi_oracle.h")
    lib = tmp_path / "liboracle.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                    "-o", str(lib), str(tmp_path / "messi_oracle.c"), "-lm"], check=True)
    env = dict(os.environ, MESSI_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "passed" in r.stdout


PY_MUTANTS = [
    ("leaf split on the bit after the next one",
     "        while mid < hi and bit(sk[mid], d) == 0:", "        while mid < hi and bit(sk[mid], d + 1) == 0:"),
    ("a node splits only above twice its capacity",
     "        if hi - lo <= cap or d >= total:", "        if hi - lo <= 2 * cap or d >= total:"),
    ("root children by the first w - 1 bits",
     "        if i == N or prefix(sk[i], w) != prefix(sk[start], w):",
     "        if i == N or prefix(sk[i], w - 1) != prefix(sk[start], w - 1):"),
    ("streamed k-NN keeps the first block's answer",
     "        best = part if best is None else merge_topk([best, part], k)",
     "        best = part if best is None else best"),
]


def run_pins_on_package_copy(tmp_path, init_text):
    """Pins of a copy of the repository's oracle package whose __init__.py is
    `init_text` (the copy compiles its own library); returns the pytest run."""
    root = tmp_path / "root"
    (root / "oracle").mkdir(parents=True)
    (root / "tests").mkdir()
    (root / "oracle" / "__init__.py").write_text(init_text)
    for f in ("messi_oracle.c", "messi_oracle.h"):
        shutil.copy(os.path.join(ROOT, "oracle", f), root / "oracle" / f)
    for f in ("conftest.py", "test_oracle_pins.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), root / "tests" / f)
    os.symlink(os.path.join(ROOT, "tests", "golden"), root / "tests" / "golden")
    os.symlink(os.path.join(ROOT, "synth"), root / "synth")
    env = dict(os.environ, OMP_NUM_THREADS="4")
    env.pop("MESSI_ORACLE_LIB", None)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           str(root / "tests" / "test_oracle_pins.py")],
                          cwd=str(root), env=env, capture_output=True, text=True, timeout=600)


@pytest.mark.parametrize("name,old,new", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_pins_catch_planted_python_mistake(tmp_path, name, old, new):
    init = open(os.path.join(ROOT, "oracle", "__init__.py")).read()
    assert init.count(old) == 1, f"mutation site not found exactly once: {name}"
    r = run_pins_on_package_copy(tmp_path, init.replace(old, new))
    assert r.returncode != 0, f"planted mistake survived every pin: {name}\n{r.stdout[-2000:]}"


def test_control_unmutated_package_copy_passes(tmp_path):
    r = run_pins_on_package_copy(tmp_path, open(os.path.join(ROOT, "oracle", "__init__.py")).read())
    assert r.returncode == 0, r.stdout[-3000:]
    assert "passed" in r.stdout
