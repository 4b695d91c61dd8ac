"""Host checks of the tables behind the kernels' exponential and logarithm
(Tang, ACM TOMS 15(2), 1989 and 16(4), 1990): the committed header is the
generator's output, every entry is the correctly rounded value of its
definition (60-digit decimal arithmetic), and the logarithm's method with
this table -- emulated on the host with exactly rounded fma -- stays within
the bound the GPU test applies to the kernel (3 ulp or 2.5e-16 absolute).
The exponential's method (256-entry table, degree-4 polynomial) with its
table stays within 2 ulp of the exact value, and the kernels' Newton reciprocal, emulated the same way from a
correctly rounded FP32 estimate, within 1 ulp of the IEEE quotient."""

import importlib.util
import io
import math
import re
from contextlib import redirect_stdout
from decimal import Decimal, localcontext
from fractions import Fraction
from pathlib import Path

import numpy as np

CSRC = Path(__file__).resolve().parents[1] / "paper_1712_00953_gb300" / "csrc"


def _generator_output():
    spec = importlib.util.spec_from_file_location("gen_exp_table", CSRC / "gen_exp_table.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    buf = io.StringIO()
    with redirect_stdout(buf):
        mod.main()
    return buf.getvalue()


def _header():
    text = (CSRC / "exp2_table.h").read_text()
    exp_vals = [float.fromhex(v) for v in re.findall(r"^\s+(0x[0-9a-fp.+-]+)", text, re.M)]
    inv_c = [float.fromhex(v) for v in re.search(r"#define RK_LOG_INV_C_VALUES (.*)", text).group(1).split(", ")]
    ln_c = [float.fromhex(v) for v in re.search(r"#define RK_LOG_LN_C_VALUES (.*)", text).group(1).split(", ")]
    consts = {k: float.fromhex(v) for k, v in re.findall(r"constexpr double (\w+) = (\S+);", text)}
    return text, exp_vals, inv_c, ln_c, consts


def _is_correctly_rounded(f, exact):
    """f is the binary64 number nearest to the Decimal `exact`."""
    lo, hi = np.nextafter(f, -np.inf), np.nextafter(f, np.inf)
    d = abs(Decimal(f) - exact)
    return d <= abs(Decimal(float(lo)) - exact) and d <= abs(Decimal(float(hi)) - exact)


def test_header_is_the_generator_output():
    text, *_ = _header()
    assert text.strip() == _generator_output().strip()


def test_table_entries_are_correctly_rounded():
    with localcontext() as ctx:
        ctx.prec = 60
        _check_entries()


def _check_entries():
    _, exp_vals, inv_c, ln_c, c = _header()
    ln2 = Decimal(2).ln()
    assert len(exp_vals) == 256 and len(inv_c) == len(ln_c) == 128
    for j in range(256):
        assert _is_correctly_rounded(exp_vals[j], (ln2 * j / 256).exp())
    for j in range(128):
        assert _is_correctly_rounded(inv_c[j], 1 / (1 + (Decimal(j) + Decimal("0.5")) / 128))
        assert _is_correctly_rounded(ln_c[j], -Decimal(inv_c[j]).ln())
    # ln 2 split: the head has 32 trailing zero bits (e * head exact for |e| < 2^20)
    assert Fraction(c["RK_LN2_HI"]).denominator <= 2 ** 21
    assert abs(Decimal(c["RK_LN2_HI"]) + Decimal(c["RK_LN2_LO"]) - ln2) < Decimal(2) ** -75
    assert Fraction(c["RK_LN2_OVER_N_HI"]).denominator <= 2 ** 29
    assert abs(Decimal(c["RK_LN2_OVER_N_HI"]) + Decimal(c["RK_LN2_OVER_N_LO"]) - ln2 / 256) < Decimal(2) ** -83
    assert _is_correctly_rounded(c["RK_INV_LN10"], 1 / Decimal(10).ln())


def _fma(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _log_method(x, inv_c, ln_c, c):
    """Tang's table-driven ln with the kernel's steps, each rounded once."""
    m, e2 = math.frexp(x)  # x = m 2^e2, m in [0.5, 1)
    m, e = 2.0 * m, e2 - 1  # m in [1, 2)
    j = int((m - 1.0) * 128)
    r = _fma(m, inv_c[j], -1.0)
    q = _fma(r, 1.0 / 7.0, -1.0 / 6.0)
    for coef in (0.2, -0.25, 1.0 / 3.0, -0.5):
        q = _fma(q, r, coef)
    p = _fma(r * r, q, r)
    return _fma(float(e), c["RK_LN2_HI"], ln_c[j]) + _fma(float(e), c["RK_LN2_LO"], p)


def test_log_method_meets_the_kernel_bound():
    with localcontext() as ctx:
        ctx.prec = 40
        _check_log_method()


def _check_log_method():
    _, _, inv_c, ln_c, c = _header()
    rng = np.random.default_rng(5)
    xs = np.concatenate([10.0 ** rng.uniform(-300, 300, 600), rng.uniform(200.0, 6000.0, 300),
                         1.0 + rng.uniform(-1e-2, 1e-2, 300), rng.uniform(0.5, 2.0, 300),
                         [1.0, 0.5, 2.0, 1.0 - 2.0 ** -53, np.finfo(float).tiny, np.finfo(float).max]])
    for j in range(128):  # every interval, at both ends and the centre
        xs = np.append(xs, [1 + j / 128, 1 + (j + 0.5) / 128, np.nextafter(1 + (j + 1) / 128, 0.0)])
    for x in xs:
        y = _log_method(float(x), inv_c, ln_c, c)
        exact = Decimal(float(x)).ln()
        err = abs(Decimal(y) - exact)
        bound = max(Decimal(3) * Decimal(float(np.spacing(abs(float(exact))))), Decimal("2.5e-16"))
        assert err <= bound, (x, y, float(exact))
    assert _log_method(1.0, inv_c, ln_c, c) == 0.0 or abs(_log_method(1.0, inv_c, ln_c, c)) < 1e-18


def _rcp_method(x):
    """Two Newton steps r <- r + r (1 - x r) from the correctly rounded FP32
    reciprocal, each operation rounded once, as in the kernels."""
    r = float(np.float32(1.0) / np.float32(x))
    e = _fma(-x, r, 1.0)
    r = _fma(r, e, r)
    e = _fma(-x, r, 1.0)
    return _fma(r, e, r)


def test_newton_reciprocal_method_within_one_ulp():
    rng = np.random.default_rng(6)
    xs = np.concatenate([2.0 ** rng.uniform(-124.9, 124.9, 2000), 1.0 + rng.uniform(0.0, 1.0, 500),
                         [1.0, 3.0, 0.1, 2.0 ** -125, np.nextafter(2.0 ** 125, 0.0), 1.0 - 2.0 ** -53]])
    xs = np.concatenate([xs, -xs])
    for x in xs:
        y, ref = _rcp_method(float(x)), 1.0 / float(x)
        assert abs(np.array(y).view(np.int64) - np.array(ref).view(np.int64)) <= 1, (x, y, ref)


def _exp_method(x, tab, c):
    """Tang's table-driven exp with the kernel's steps, each rounded once:
    k = round(x 256 / ln2) by the 1.5 2^52 shifter, r = x - k ln2/256 in two
    parts, e^r - 1 = r + r^2 (1/2 + r/6 + r^2/24), 2^(k/256) from the table and
    2^(k >> 8) by exponent scaling."""
    shifter = 6755399441055744.0
    kt = _fma(x, c["RK_N_OVER_LN2"], shifter)
    k = int(kt - shifter)
    kd = kt - shifter
    r = _fma(-kd, c["RK_LN2_OVER_N_HI"], x)
    r = _fma(-kd, c["RK_LN2_OVER_N_LO"], r)
    q = _fma(r, 1.0 / 24.0, 1.0 / 6.0)
    q = _fma(q, r, 0.5)
    p = _fma(r * r, q, r)
    t = tab[k & 255]
    return math.ldexp(_fma(t, p, t), k >> 8)


def test_exp_method_within_two_ulp():
    _, exp_vals, _, _, c = _header()
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.uniform(-700.0, 700.0, 1500), rng.uniform(-3.0, 3.0, 500),
                         [0.0, 1.0, -1.0, 1e-300, np.log(2.0), 700.0, -700.0]])
    with localcontext() as ctx:
        ctx.prec = 40
        for x in xs:
            y = _exp_method(float(x), exp_vals, c)
            exact = Decimal(float(x)).exp()
            err_ulp = abs(Decimal(y) - exact) / Decimal(float(np.spacing(float(exact))))
            assert err_ulp <= 2, (x, y, float(exact), float(err_ulp))
