"""Planted mistakes: every plausible slip in the oracles (a dropped term, a
wrong sign, factor, exponent or index, a transposed operand) must fail at
least one pin.  Each mutant is a scratch copy of the oracle, under the
git-ignored tests/_scratch folder, with one edit; the oracle itself is never
modified.  This checks the pins, not the oracle: an unmutated copy passes."""

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what, text in oracle/prost_oracle.c, replacement)
C_MUTANTS = [
    ("eta sign", "eta[e] = -prm->p * w[e % P]", "eta[e] = prm->p * w[e % P]"),
    ("eta exponent", "pow(r[e] * r[e] + prm->mu, 0.5 * prm->p - 1.0);\n}",
     "pow(r[e] * r[e] + prm->mu, 0.5 * prm->p - 0.5);\n}"),
    ("cost exponent", "return pow(r * r + mu, 0.5 * p);", "return pow(r * r + mu, p);"),
    ("line step sign", "double alpha = den > 0.0 ? num / den : 0.0;", "double alpha = den > 0.0 ? -num / den : 0.0;"),
    ("Fletcher-Reeves for Polak-Ribiere", "num_b += gn[j] * (gn[j] - g[j]);", "num_b += gn[j] * gn[j];"),
    ("beta not clamped at 0", "if (beta < 0.0) beta = 0.0;", ""),
    ("weights dropped from the line step", "double c = w[e % P] * pow(", "double c = 1.0 * pow("),
    ("geodesic sine sign", "double coef = cm1 * uv - sn * s_e;", "double coef = cm1 * uv + sn * s_e;"),
    ("geodesic cosine term dropped", "double coef = cm1 * uv - sn * s_e;", "double coef = - sn * s_e;"),
    ("sigma without |y|", "double sigma = pin * yn;", "double sigma = pin;"),
    ("projection skipped", "out[e] = h[e] - s;", "out[e] = h[e];"),
    ("threshold doubled", "(uint8_t)(mx >= prm->delta)", "(uint8_t)(mx > 2*prm->delta)"),
    ("labels from the first channel only", "if (a > mx) mx = a;", "if (c == 0 && a > mx) mx = a;"),
    ("weights inverted", "(labels && labels[q]) ? prm->omega : 1.0", "(labels && labels[q]) ? 1.0 : prm->omega"),
    ("step-size decay sign", "double t = exp(-tau * (double)i) * prm->t_init;",
     "double t = exp(tau * (double)i) * prm->t_init;"),
    ("input offset sign", "x[e] = prm->in_scale * v - prm->in_offset;", "x[e] = prm->in_scale * v + prm->in_offset;"),
    ("Cholesky transposed", "s -= R[l * k + a] * R[l * k + b];", "s -= R[a * k + l] * R[b * k + l];"),
    ("y <- R y dropped", "for (int a = 0; a < k; ++a) y[a] = ry[a];", ""),
    ("mu heuristic without the square", "return delta * delta * (1.0 - p);", "return delta * (1.0 - p);"),
    ("frame counter off by one", "orc_step_size(prm, i)", "orc_step_size(prm, i + 1)"),
    ("mask always from the updated U", "const double *Ul = Uold ? Uold : U;", "const double *Ul = U;"),
    ("pixel index of the weight", "f += w[e % P] * orc_h", "f += w[e / prm->channels % P] * orc_h"),
]

# (file under oracle/, what, text, replacement)
PY_MUTANTS = [
    ("window.py", "weights inverted", "w = np.where(lab, omega, 1.0)", "w = np.where(lab, 1.0, omega)"),
    ("window.py", "channels interleaved", "np.tile(w, (1, channels))", "np.repeat(w, channels, axis=1)"),
    ("window.py", "residual sign", "R = X.T - U @ Y ", "R = U @ Y - X.T "),
    ("window.py", "mu squared", "Z = R * R + mu", "Z = R * R + mu * mu"),
    ("window.py", "cost exponent", "F = float(np.sum(W.T * Z ** (0.5 * p)))", "F = float(np.sum(W.T * Z ** p))"),
    ("window.py", "weights dropped from eta", "H = -p * W.T * R * Z ** (0.5 * p - 1.0)",
     "H = -p * R * Z ** (0.5 * p - 1.0)"),
    ("window.py", "eta sign", "H = -p * W.T * R * Z ** (0.5 * p - 1.0)", "H = p * W.T * R * Z ** (0.5 * p - 1.0)"),
    ("window.py", "eta factor", "H = -p * W.T * R * Z ** (0.5 * p - 1.0)",
     "H = -0.5 * p * W.T * R * Z ** (0.5 * p - 1.0)"),
    ("window.py", "dF/dU scaled", "dU = H @ Y.T", "dU = H @ Y.T * 1.0001"),
    ("window.py", "dF/dY scaled", "dY = U.T @ H", "dY = U.T @ H * 1.0001"),
    ("window.py", "weights dropped from dF/dmu", "dmu = float(np.sum(W.T * (0.5 * p) * Z ** (0.5 * p - 1.0)))",
     "dmu = float(np.sum((0.5 * p) * Z ** (0.5 * p - 1.0)))"),
    ("window.py", "dF/dmu factor", "dmu = float(np.sum(W.T * (0.5 * p) * Z ** (0.5 * p - 1.0)))",
     "dmu = float(np.sum(W.T * p * Z ** (0.5 * p - 1.0)))"),
    ("window.py", "projection skipped", "G = dU - U @ (U.T @ dU)", "G = dU"),
    ("window.py", "projection transposed", "G = dU - U @ (U.T @ dU)", "G = dU - U @ (dU.T @ U)"),
    ("window.py", "ascent step", "V = U - t * G", "V = U + t * G"),
    ("window.py", "retraction solve transposed", "return np.linalg.solve(R.T, V.T).T", "return np.linalg.solve(R, V.T).T"),
    ("window.py", "Cholesky factor transposed", "R = np.linalg.cholesky(V.T @ V).T", "R = np.linalg.cholesky(V.T @ V)"),
    ("prepost.py", "resampling scale inverted", "    s = n_in / n_out\n    A", "    s = n_out / n_in\n    A"),
    ("prepost.py", "footprint one pixel wide", "lo, hi = i * s, (i + 1) * s", "lo, hi = i * s, i * s + 1"),
    ("prepost.py", "footprint weights not normalised", "A[i, q] = ov / s", "A[i, q] = ov"),
    ("prepost.py", "footprint end rounded down", "for q in range(int(np.floor(lo)), min(n_in, int(np.ceil(hi)))):",
     "for q in range(int(np.floor(lo)), min(n_in, int(np.floor(hi)))):"),
    ("prepost.py", "partial pixels counted whole", "ov = min(hi, q + 1) - max(lo, q)", "ov = 1.0"),
    ("prepost.py", "columns resampled with the transpose", "return np.stack([Ay @ f[c] @ Ax.T for c in range(C)])",
     "return np.stack([Ay @ f[c] @ Ax for c in range(C)]) if W == H else "
     "np.stack([Ay @ f[c] @ Ax.T for c in range(C)])"),
    ("prepost.py", "deviation divides by n", "var = (self.s2 - self.s1 * self.s1 / self.cnt) / (self.cnt - 1)",
     "var = (self.s2 - self.s1 * self.s1 / self.cnt) / self.cnt"),
    ("prepost.py", "phase one frame too long", "if self.n < self.i_init:", "if self.n <= self.i_init:"),
    ("prepost.py", "running mean off by one", "self.mean += (v - self.mean) / self.n",
     "self.mean += (v - self.mean) / (self.n + 1)"),
    ("prepost.py", "sum of magnitudes", "self.s1 += float(v.sum())", "self.s1 += float(np.abs(v).sum())"),
    ("prepost.py", "frames counted for entries", "self.cnt += v.size", "self.cnt += 1"),
    ("prepost.py", "divided by the variance", "return (v - self.mean) / self.std()", "return (v - self.mean) / self.std() ** 2"),
    ("prepost.py", "mean not subtracted", "return (v - self.mean) / self.std()", "return v / self.std()"),
    ("prepost.py", "border zero-padded", 'p = np.pad(m, 1, mode="edge")', 'p = np.pad(m, 1, mode="constant")'),
    ("prepost.py", "median threshold 4 of 9", "return (count >= 5).astype(np.uint8)", "return (count >= 4).astype(np.uint8)"),
    ("prepost.py", "neighbourhood index", "count += p[dy:dy + H, dx:dx + W]", "count += p[dy:dy + H, dy:dy + W]"),
]

C_PINS = ["test_oracle_pins.py"]
PY_PINS = ["test_window_pins.py", "test_prepost_pins.py"]


def _tree(dst, pins):
    """A minimal tree under dst: the oracle (sources only), the input
    generators, conftest, the golden fixtures and the given pin files."""
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("__init__.py", "prost_oracle.c", "window.py", "prepost.py"):
        shutil.copy(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    shutil.copytree(os.path.join(ROOT, "synth"), os.path.join(dst, "synth"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ["conftest.py"] + pins:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    # its own root, so that pytest neither climbs into this tree's conftest
    # nor imports the real oracle
    with open(os.path.join(dst, "pytest.ini"), "w") as f:
        f.write("[pytest]\n")


def _plant(dst, rel, old, new):
    path = os.path.join(dst, "oracle", rel)
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, f"{rel}: the text to replace must occur once: {old!r}"
    with open(path, "w") as f:
        f.write(src.replace(old, new))


def _pins_pass(dst, pins):
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "-c", os.path.join(dst, "pytest.ini"), "--rootdir", dst, "--confcutdir", dst]
                       + [os.path.join("tests", p) for p in pins],
                       cwd=dst, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode in (0, 1), r.stdout[-2000:] + r.stderr[-2000:]
    return r.returncode == 0


def _missed(scratch, mutants, pins):
    jobs = [(None, "unmutated", None, None)] + mutants
    dirs = []
    for i, (rel, what, old, new) in enumerate(jobs):
        d = os.path.join(str(scratch), f"m{i:02d}")
        _tree(d, pins)
        if rel is not None:
            _plant(d, rel, old, new)
        dirs.append(d)
    try:
        with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
            passed = list(ex.map(lambda d: _pins_pass(d, pins), dirs))
    finally:
        shutil.rmtree(str(scratch), ignore_errors=True)
    assert passed[0], "the pins fail on an unmutated copy of the oracle"
    return [jobs[i][1] for i in range(1, len(jobs)) if passed[i]]


@pytest.mark.slow
def test_every_planted_mistake_in_the_frame_oracle_fails_a_pin(scratch):
    mutants = [("prost_oracle.c", what, old, new) for what, old, new in C_MUTANTS]
    assert _missed(scratch, mutants, C_PINS) == []


@pytest.mark.slow
def test_every_planted_mistake_in_the_window_and_prepost_oracles_fails_a_pin(scratch):
    assert _missed(scratch, PY_MUTANTS, PY_PINS) == []
