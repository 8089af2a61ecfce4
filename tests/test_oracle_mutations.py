"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a temporary copy of ``oracle/kite_oracle.c`` (on the
CPU, never in the tree), rebuilds it, and re-runs the pin suite against the mutant:
at least one pin has to fail.  This is what makes the pins evidence rather than
restatements of the oracle.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
import tempfile
from pathlib import Path

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("velocity bond sign", "dx[1] = -0.5;", "dx[1] = 0.5;"),
    ("wrong neighbour cell",
     "nb[1] = 2 * (orc_wrap(y - 1, Ly) * Lx + orc_wrap(x + 1, Lx)) + 1;",
     "nb[1] = 2 * (orc_wrap(y - 1, Ly) * Lx + orc_wrap(x - 1, Lx)) + 1;"),
    ("inverted DOS weight (printed Eq. e8 prefactor)",
     "sum += 2.0 * (g ? g[n] : 1.0) * mu[n] * t;", "sum += 0.5 * (g ? g[n] : 1.0) * mu[n] * t;"),
    ("recursion sign", "nxt[k] = 2.0 * nxt[k] - prev[k];", "nxt[k] = 2.0 * nxt[k] + prev[k];"),
    ("conjugation dropped in <a|b>",
     "si += a[2 * o] * b[2 * o + 1] - a[2 * o + 1] * b[2 * o];",
     "si += a[2 * o] * b[2 * o + 1] + a[2 * o + 1] * b[2 * o];"),
    ("disorder not centred", "v = sys->W * (u - 0.5);", "v = sys->W * u;"),
    ("Gaussian variance halved", "sqrt(-2.0 * log(u1))", "sqrt(-log(u1))"),
    ("Gaussian angle from the radius word", "(double)x[3] * 0x1p-32", "(double)x[0] * 0x1p-32"),
    ("Gaussian bound too tight", "#define ORC_GAUSS_ZMAX 8.58", "#define ORC_GAUSS_ZMAX 5.0"),
    ("Peierls phase without the bond midpoint", "k * (yo - 0.5 * h->dy[4 * o + b])", "k * (yo)"),
    ("Peierls flux doubled", "* sys->flux / cell_area;", "* 2.0 * sys->flux / cell_area;"),
    ("Peierls honeycomb cell area", "sys->lattice == 0 ? 0.5 * sqrt(3.0) : 1.0;", "1.0;"),
    ("Peierls phase conjugated on one component", "xi = sn * xr + c * xi;", "xi = -sn * xr + c * xi;"),
    ("velocity loses its sign", "double w = off[4 * o + k] * h->tt;",
     "double w = fabs(off[4 * o + k]) * h->tt;"),
    ("y bond offset sign", "dy[1] = 0.5 * acc;", "dy[1] = -0.5 * acc;"),
    ("velocity direction ignored", "const double* off = dir ? h->dy : h->dx;", "const double* off = h->dx;"),
    ("Jackson kernel off by one",
     "g[n] = ((double)(M - n + 1) * cos(q * n) + sin(q * n) * cot) / (double)(M + 1);",
     "g[n] = ((double)(M - n) * cos(q * n) + sin(q * n) * cot) / (double)(M + 1);"),
    ("CPGF branch flipped", "double complex num = cexp(-s * I * (double)n * theta);",
     "double complex num = cexp(s * I * (double)n * theta);"),
    ("on-site term dropped", "double re = h->Vt[o] * x[2 * o], im = h->Vt[o] * x[2 * o + 1];",
     "double re = 0.0 * x[2 * o], im = 0.0 * x[2 * o + 1];"),
    ("normalised by N instead of N_eff", "if (!h->vac[o]) h->n_eff++;", "h->n_eff++;"),
    ("vacancy draw ignored", "vac[o] = ((uint64_t)x[2] < thr) ? 1 : 0;", "vac[o] = 0;"),
    ("velocity without the Peierls phases", "if (h->ph) { /* [r, H~]_oj", "if (0) { /* [r, H~]_oj"),
    ("open x drops the wrong honeycomb bond", "if ((ox && x + 1 == Lx) || (oy && y == 0)) nb[1] = -1;",
     "if ((ox && x + 1 == Lx) || (oy && y == 0)) nb[2] = -1;"),
    ("open y ignored on the square lattice", "nb[2] = (sys->open_y && y == 0) ? -1 :", "nb[2] = (0 && y == 0) ? -1 :"),
    ("flux check ignores an open y boundary", "if (sys->flux == 0.0 || sys->open_y) return 0;",
     "if (sys->flux == 0.0) return 0;"),
    ("Bastin derivative without the band-edge term", "+ (z / (s1 * s1))[None, :]))",
     "+ 0.0 * (z / (s1 * s1))[None, :]))", "__init__.py"),
    ("Bastin advanced term on the retarded branch", "for sg in (+1, -1):", "for sg in (+1, +1):",
     "__init__.py"),
    ("Kubo-Greenwood delta functions without the (2 - d_n0) weight",
     "w = np.where(np.arange(M) == 0, 1.0, 2.0) * g", "w = np.where(np.arange(M) == 0, 1.0, 1.0) * g", "__init__.py"),
    ("optical conductivity with the sign of Gamma flipped", "G = -mu * w0[:, None] * w0[None, :]",
     "G = mu * w0[:, None] * w0[None, :]", "__init__.py"),
    ("honeycomb unit-cell factor halved", "return 2.0 * 2.0 / np.sqrt(3.0) if lattice == HONEYCOMB else 1.0",
     "return 2.0 / np.sqrt(3.0) if lattice == HONEYCOMB else 1.0", "__init__.py"),
    ("Bastin Fermi sea from the top of the band", "theta = thF + (np.pi - thF) * 0.5 * (x + 1.0)\n        wq = w *",
     "theta = thF * 0.5 * (x + 1.0)\n        wq = w *", "__init__.py"),
    ("Philox Weyl constant off by one", "k1 += 0xBB67AE85u;", "k1 += 0xBB67AE86u;"),
    ("AdamW bias correction on the first moment only", "vh = v / (1 - beta2 ** t)", "vh = v", "mlp.py"),
    ("AdamW second moment decayed at the first moment's rate", "v = beta2 * v + (1 - beta2) * g * g",
     "v = beta1 * v + (1 - beta1) * g * g", "mlp.py"),
    ("cosine schedule one step late", "np.pi * (t - 1) / max(1, total)", "np.pi * t / max(1, total)", "mlp.py"),
]


def run_pins_on_copy(tmp_path, old, new, threads=None, target="kite_oracle.c"):
    src_dir = os.path.join(ROOT, "oracle")
    dst = tmp_path / "oracle"
    dst.mkdir()
    for f in os.listdir(src_dir):  # every module of the oracle package, not the build
        if f.endswith((".py", ".h", ".c")):
            shutil.copy(os.path.join(src_dir, f), dst / f)
    with open(os.path.join(src_dir, target)) as f:
        src = f.read()
    assert old in src, f"mutation anchor missing: {old}"
    (dst / target).write_text(src.replace(old, new, 1))
    shutil.copy(os.path.join(ROOT, "tests", "test_oracle_pins.py"), tmp_path / "test_oracle_pins.py")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "golden")
    env = dict(os.environ, PYTHONPATH=str(tmp_path))
    if threads:
        env["OMP_NUM_THREADS"] = str(threads)
    return subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                           "-p", "no:randomly", str(tmp_path / "test_oracle_pins.py")],
                          cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)


def test_unmutated_copy_passes(tmp_path):
    """The control: the copied oracle and pins pass as they are, so a failure below is
    the planted mistake's doing."""
    r = run_pins_on_copy(tmp_path, "", "")
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.fixture(scope="module")
def mutant_runs():
    """Every mutant's pin run, side by side (each in its own copy and process, a few
    OpenMP threads each), so the module takes about as long as one run."""
    cores = os.cpu_count() or 1
    workers = max(1, min(len(MUTATIONS), cores // 2))
    base = Path(tempfile.mkdtemp(prefix="oracle_mutants_"))

    def one(i):
        d = base / f"m{i}"
        d.mkdir()
        return run_pins_on_copy(d, *MUTATIONS[i][1:3], threads=2, target=(MUTATIONS[i] + ("kite_oracle.c",))[3])

    try:
        with cf.ThreadPoolExecutor(max_workers=workers) as ex:
            results = list(ex.map(one, range(len(MUTATIONS))))
    finally:
        shutil.rmtree(base, ignore_errors=True)
    return {MUTATIONS[i][0]: r for i, r in enumerate(results)}


@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_pins_catch_planted_mistake(mutant_runs, name):
    r = mutant_runs[name]
    assert r.returncode != 0, f"no pin caught mutation '{name}':\n{r.stdout[-2000:]}"
    assert "failed" in r.stdout, r.stdout[-2000:]
