"""The mixed path's double-float arithmetic (psq_df.cuh), built for the CPU, against
high-precision references: e^-x, quotients, square roots, the radial factors of chi, lap chi
and the aux potential V^P (eq 16 through the Laplace expansion, integer incomplete gamma
functions) and the unnormalised real harmonics.  The contraction keeps 39 bits of each
128-point window's largest value, so every value must carry clearly more: the bar is 2^-44
relative (V^P and the harmonics are compared with their largest term's scale where they
cancel), plus 2^-140 absolute: below about 1e-31 the lo word of a
pair is subnormal, which limits the relative precision of values that small (irrelevant at
the 1e-9 absolute target)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")
mpmath.mp.dps = 40

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2510_15204_gb300", "csrc")
TOL = 2.0 ** -44
FLOOR = 2.0 ** -140


def dfx(x):
    """The value the driver works with: x split into a float32 pair (hi, lo)."""
    h = np.float32(x)
    return float(h) + float(np.float32(x - float(h)))


@pytest.fixture(scope="module")
def run(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("df") / "df_host_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
                    os.path.join(HERE, "df_host_check.cpp"), "-o", exe], check=True)

    def call(lines):
        r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, check=True)
        out = []
        for ln in r.stdout.strip().split("\n"):
            # each printed value round-trips to its float32 (9 significant digits)
            v = [float(np.float32(t)) for t in ln.split()]
            out.append([v[i] + v[i + 1] for i in range(0, len(v), 2)])
        return out
    return call


def test_exp_neg(run):
    xs = [0.0, 1e-6, 0.3, 0.7, 1.0, 2.5, 7.3, 13.0, 31.7, 60.1, 86.0]
    xs += list(np.random.default_rng(0).uniform(0, 80, 200))
    got = run(["exp %.17g" % x for x in xs])
    for x, g in zip(xs, got):
        ref = mpmath.exp(-mpmath.mpf(dfx(x)))
        assert abs(g[0] - float(ref)) <= TOL * float(ref) + FLOOR, (x, g[0], float(ref))


def test_div_sqrt(run):
    rng = np.random.default_rng(1)
    a = rng.uniform(-50, 50, 100)
    b = rng.uniform(0.01, 30, 100)
    got = run(["div %.17g %.17g" % (x, y) for x, y in zip(a, b)])
    for x, y, g in zip(a, b, got):
        ref = mpmath.mpf(dfx(x)) / mpmath.mpf(dfx(y))
        assert abs(g[0] - float(ref)) <= TOL * abs(float(ref)), (x, y)
    got = run(["sqrt %.17g" % y for y in b])
    for y, g in zip(b, got):
        ref = mpmath.sqrt(mpmath.mpf(dfx(y)))
        assert abs(g[0] - float(ref)) <= TOL * float(ref), y


def _radial_ref(kind, n, l, x):
    x = mpmath.mpf(dfx(x))
    if kind == 0:
        return x ** (n - 1) * mpmath.exp(-x), None
    if kind == 1:
        f = (n * (n - 1) - l * (l + 1)) / x ** 2 - 2 * n / x + 1
        g = x ** (n - 1) * mpmath.exp(-x)
        # the bracket cancels near its zeros: compare with its largest term
        scale = (abs(n * (n - 1) - l * (l + 1)) / x ** 2 + 2 * n / x + 1) * g
        return f * g, scale
    k1, k2 = n + l + 2, n - l + 1
    inner = mpmath.gammainc(k1, 0, x) / x ** (l + 1)
    outer = mpmath.gammainc(k2, x, mpmath.inf) * x ** l
    return inner + outer, None


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_radial_factors(run, kind):
    cases = []
    for (n, l) in [(1, 0), (2, 0), (2, 1), (3, 2), (4, 3), (5, 4), (6, 5), (3, 0), (7, 6)]:
        for x in (1e-3, 0.05, 0.4, 1.0, 2.9, 3.0, 3.1, n + l + 1.5, n + l + 2.0, n + l + 2.5, 9.0, 17.0, 40.0, 60.0):
            cases.append((n, l, x))
    # far points of refined grids around distant pairs: x up to ~1e5 (sums must not overflow)
    cases += [(n, l, x) for (n, l) in [(1, 0), (5, 4), (7, 6), (12, 6)] for x in (90.0, 500.0, 5e4, 3e6)]
    got = run(["radial %d %d %d %.17g" % (kind, n, l, x) for (n, l, x) in cases])
    for (n, l, x), g in zip(cases, got):
        assert all(math.isfinite(v) for v in g), (kind, n, l, x, g)
        ref, scale = _radial_ref(kind, n, l, x)
        if x >= 87 and kind != 2:
            # e^-x flushed to 0 past x = 87: the exact value is below 1e-20 of the function's
            # largest, x^(n-1) e^-x at x = n - 1
            top = max(1.0, float((n - 1) ** (n - 1) * mpmath.exp(-(n - 1))))
            assert g[0] == 0.0 and abs(float(ref)) < 1e-20 * top, (kind, n, l, x, g[0], float(ref))
            continue
        scale = abs(float(ref)) if scale is None else float(scale)
        assert abs(g[0] - float(ref)) <= TOL * scale + FLOOR, (kind, n, l, x, g[0], float(ref))


def test_real_harmonics(run):
    """Unnormalised real harmonics Q_l^|m|(u_z) {cos, sin}(|m| phi) sin^|m| theta against their
    definition through mpmath's associated Legendre functions (no Condon-Shortley phase)."""
    rng = np.random.default_rng(2)
    L = 6
    for _ in range(12):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        got = run(["ylm %d %.17g %.17g %.17g" % (L, u[0], u[1], u[2])])[0]
        ux, uy, uz = (mpmath.mpf(dfx(c)) for c in u)
        th = mpmath.acos(uz / mpmath.sqrt(ux * ux + uy * uy + uz * uz))
        ph = mpmath.atan2(uy, ux)
        for l in range(L + 1):
            for m in range(-l, l + 1):
                am = abs(m)
                # Q_l^m(z) sin^m(theta) = (-1)^m P_l^m(cos theta) in mpmath's (Condon-Shortley) convention
                q = (-1) ** am * mpmath.legenp(l, am, mpmath.cos(th))
                ref = q * (mpmath.cos(am * ph) if m >= 0 else mpmath.sin(am * ph))
                scale = float(mpmath.fac(l + am) / mpmath.fac(l - am)) ** 0.5 * math.factorial(2 * l) / (2 ** l * math.factorial(l))
                assert abs(got[l * l + l + m] - float(ref)) <= TOL * scale, (l, m, got[l * l + l + m], float(ref))
