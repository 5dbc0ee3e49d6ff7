"""Planted mistakes in the oracle: every one must fail a pin.

The oracle is trusted because its pins tie it to things other than itself
(library routines, closed forms, brute force, invariants, the paper's counts).
That trust holds only if a plausible mistake anywhere in it fails at least one
pin.  Each mutant below is one such mistake (a dropped term, a wrong sign, a
swapped index or operand, an off-by-one, a missing clamp or buffer swap),
written as a textual replacement in a copy of the oracle package.  The copy is
compiled on its own, and the CPU pin suite is run against it in a child
process (``FIC_ORACLE_DIR`` points the ``orc`` fixture at the copy).  The
unmodified copy must pass; every mutant must make at least one pin fail.

Runs on the CPU only; nothing here touches the GPU or the product library.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = ["tests/test_oracle_pins.py", "tests/test_oracle_quadtree.py", "tests/test_oracle_refine.py"]

C = "fic_oracle.c"
PY = "__init__.py"

# (name, file, original text, planted text); the original must occur exactly once
MUTANTS = [
    # the eight symmetries (Section V)
    ("rot90 turns counter-clockwise", C,
     "case 1: *sy = n - 1 - x; *sx = y;         break;",
     "case 1: *sy = x;         *sx = n - 1 - y; break;"),
    ("mirror L-R flips top-bottom", C,
     "case 4: *sy = y;         *sx = n - 1 - x; break;",
     "case 4: *sy = n - 1 - y; *sx = x;         break;"),
    ("anti-transpose read as rot180", C,
     "default: *sy = n - 1 - x; *sx = n - 1 - y; break;",
     "default: *sy = n - 1 - y; *sx = n - 1 - x; break;"),
    # the contraction tau (2x2 mean)
    ("tau drops a pixel of the 2x2 mean", C,
     "a[y * n + x] = 0.25 * (p0[0] + p0[1] + p1[0] + p1[1]);",
     "a[y * n + x] = 0.25 * (p0[0] + p0[1] + p1[0] + p1[0]);"),
    ("tau sums instead of averaging", C,
     "a[y * n + x] = 0.25 * (p0[0]",
     "a[y * n + x] = 1.0 * (p0[0]"),
    ("tau samples at stride 1", C,
     "img + (size_t)(dy + 2 * y) * w + (dx + 2 * x);",
     "img + (size_t)(dy + y) * w + (dx + x);"),
    # block geometry
    ("search domain origin transposed", C,
     "for (int d = 0; d < U * V; ++d) {\n            contract(img, w, (d / U) * p->t, (d % U) * p->t, n, a0);",
     "for (int d = 0; d < U * V; ++d) {\n            contract(img, w, (d % U) * p->t, (d / U) * p->t, n, a0);"),
    ("range grid transposed", C,
     "const int nx = w / n;\n    const int ry = (r / nx) * n, rx = (r % nx) * n;",
     "const int nx = w / n;\n    const int ry = (r % nx) * n, rx = (r / nx) * n;"),
    ("last domain column dropped", C,
     "{ return (w - 2 * p->n) / p->t + 1; }",
     "{ return (w - 2 * p->n) / p->t; }"),
    # least squares (eq 9-12)
    ("variance term with a plus sign", C,
     "const double den = md * Saa - Sa * Sa;",
     "const double den = md * Saa + Sa * Sa;"),
    ("slope numerator uses Sa for Sb", C,
     "(md * Sab - Sa * Sb) / den",
     "(md * Sab - Sa * Sa) / den"),
    ("slope numerator drops the mean term", C,
     "(md * Sab - Sa * Sb) / den",
     "(md * Sab) / den"),
    ("flat domain gives slope 1", C,
     "(den == 0.0) ? 0.0 :",
     "(den == 0.0) ? 1.0 :"),
    ("offset from the unquantised slope", C,
     "const double o = (Sb - f->s_hat * Sa) / md;",
     "const double o = (Sb - f->s_ls * Sa) / md;"),
    ("offset not divided by the pixel count", C,
     "const double o = (Sb - f->s_hat * Sa) / md;",
     "const double o = (Sb - f->s_hat * Sa);"),
    # quantisation
    ("slope code truncated", C,
     "f->c = (int32_t)round(sc * Ls);",
     "f->c = (int32_t)(sc * Ls);"),
    ("slope not clamped to [-1, 1]", C,
     "const double sc = clampd(s, -1.0, 1.0);",
     "const double sc = s;"),
    ("offset level on the inverted scale", C,
     "f->o_hat = (double)f->e * P / Lo;",
     "f->o_hat = (double)f->e * Lo / P;"),
    ("offset not clamped to [-P, P]", C,
     "const double oc = clampd(o, -P, P);",
     "const double oc = o;"),
    ("slope levels one short", C,
     "const double Ls = (double)((1 << (p->s_bits - 1)) - 1);",
     "const double Ls = (double)((1 << (p->s_bits - 1)) - 2);"),
    # residual (eq 8) and the argmin
    ("residual drops the offset", C,
     "const double r = f->s_hat * a[i] + f->o_hat - b[i];",
     "const double r = f->s_hat * a[i] - b[i];"),
    ("residual of the unquantised fit", C,
     "const double r = f->s_hat * a[i] + f->o_hat - b[i];",
     "const double r = f->s_ls * a[i] + f->o_raw - b[i];"),
    ("residual not squared", C,
     "R += r * r;",
     "R += fabs(r);"),
    ("last of equal minima kept", C,
     "if (f.err < best.err) {",
     "if (f.err <= best.err) {"),
    ("symmetries 7 not searched", C,
     "for (int k = 0; k < 8; ++k) {",
     "for (int k = 0; k < 7; ++k) {"),
    # decoding
    ("decode subtracts the offset", C,
     "= s_hat[r] * a + o_hat[r];",
     "= s_hat[r] * a - o_hat[r];"),
    ("decode ignores the symmetry", C,
     "sym_src(sym[r], n, y, x, &sy, &sx);",
     "sym_src(0, n, y, x, &sy, &sx);"),
    ("decode never swaps its buffers", C,
     "        double *tmp = x0;\n        x0 = x1;\n        x1 = tmp;\n",
     "        (void)x1;\n"),
    ("decode does not clamp the result", C,
     "out[i] = clamp ? clampd(x0[i], 0.0, P) : x0[i];",
     "out[i] = x0[i];"),
    ("decode starts from zero", C,
     "for (size_t i = 0; i < npx; ++i) x0[i] = init;",
     "for (size_t i = 0; i < npx; ++i) x0[i] = 0.0;"),
    # refinement gradient (adjoint of the unrolled decode)
    ("loss gradient without the factor 2", C,
     "g[i] = 2.0 * dlt / (double)npx;",
     "g[i] = dlt / (double)npx;"),
    ("offset gradient overwritten", C,
     "grad_o[r] += gp;",
     "grad_o[r] = gp;"),
    ("adjoint drops the slope", C,
     "const double back = 0.25 * s[r] * gp;",
     "const double back = 0.25 * gp;"),
    ("adjoint reads the next iterate", C,
     "const double *xt = x + npx * t;",
     "const double *xt = x + npx * (t + 1);"),
    ("adjoint scatters twice to one pixel", C,
     "g2[q + w + 1] += back;",
     "g2[q + w] += back;"),
    # PSNR
    ("PSNR with P for P^2", C,
     "10.0 * log10(P * P / mse)",
     "10.0 * log10(P / mse)"),
    ("PSNR of the summed error", C,
     "const double mse = se / (double)npx;",
     "const double mse = se;"),
    # quadtree rule and counts (Python side of the oracle)
    ("quadtree RMS over n, not n^2 pixels", PY,
     'rms = np.sqrt(fits["err"] / float(n * n))',
     'rms = np.sqrt(fits["err"] / float(n))'),
    ("quadtree domains at stride 2n", PY,
     "fits = encode(im, n=n, t=n,",
     "fits = encode(im, n=n, t=2 * n,"),
    ("quadtree never reaches the minimum size", PY,
     "split = (rms > thr) & (n > n_min)",
     "split = (rms > thr) & (n > 2 * n_min)"),
    ("quadtree children on the parent's row width", PY,
     "children.append((2 * ry + dy) * (2 * nx) + 2 * rx + dx)",
     "children.append((2 * ry + dy) * nx + 2 * rx + dx)"),
    ("domain count off by one", PY,
     "((h - 2 * n) // t + 1) * ((w - 2 * n) // t + 1)",
     "((h - 2 * n) // t) * ((w - 2 * n) // t + 1)"),
]


def _copy(dst, mutant=None):
    """Copy the oracle package (sources only) to dst/oracle, planting mutant."""
    pkg = os.path.join(dst, "oracle")
    shutil.copytree(ORACLE, pkg, ignore=shutil.ignore_patterns("_lib", "__pycache__", "*.so", "*.tmp"))
    if mutant is not None:
        _, fname, old, new = mutant
        path = os.path.join(pkg, fname)
        with open(path) as fh:
            src = fh.read()
        assert src.count(old) == 1, f"{mutant[0]}: original text found {src.count(old)} times"
        with open(path, "w") as fh:
            fh.write(src.replace(old, new))
    return dst


def _run_pins(alt):
    env = dict(os.environ, FIC_ORACLE_DIR=alt, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"] + PINS
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def _first_failure(out):
    for line in out.splitlines():
        if line.startswith("FAILED "):
            return line.split()[1]
    return None


def test_unmodified_copy_passes_the_pins(tmp_path):
    r = _run_pins(_copy(str(tmp_path)))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    def one(i):
        m = MUTANTS[i]
        d = _copy(str(tmp_path / f"m{i:02d}"), m)
        r = _run_pins(d)
        return m[0], r.returncode, _first_failure(r.stdout), r.stdout[-1500:] + r.stderr[-1500:]

    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, range(len(MUTANTS))))
    survived = [name for name, rc, _, _ in results if rc == 0]
    crashed = [(name, rc, tail) for name, rc, _, tail in results if rc not in (0, 1)]
    assert not crashed, crashed
    assert not survived, f"mutants that pass every pin: {survived}"
    for name, rc, first, _ in results:
        assert first is not None, f"{name}: no failing pin reported"


@pytest.mark.parametrize("m", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_text_is_current(m):
    """The original text of each mutant still occurs exactly once in the oracle."""
    with open(os.path.join(ORACLE, m[1])) as fh:
        assert fh.read().count(m[2]) == 1
