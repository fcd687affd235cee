"""Pins for the oracle's rounding and arithmetic (Section 2 and Table 1).

Each check compares the oracle with something other than itself: the values
printed in Table 1, numpy's binary16/binary32 conversions and arithmetic, and
torch's bfloat16 conversion and arithmetic.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_formats.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, eb, fb, u, big, small_n, small_s = line.split()
            rows[name] = dict(eb=int(eb), fb=int(fb), u=float(u), big=float(big),
                              small_n=float(small_n), small_s=float(small_s))
    return rows


def _sig5(x):
    return float(f"{x:.4e}")


@pytest.mark.parametrize("name,fmt", [("fp32", O.FP32), ("fp16", O.FP16)])
def test_table1_constants(oracle_lib, name, fmt):
    """Largest, smallest normal, smallest subnormal and unit roundoff of the
    oracle's formats match Table 1 as printed."""
    row = _table1()[name]
    # largest finite value: itself, and the next value up overflows
    big = row["big"]
    big_exact = float(np.finfo(np.float32 if name == "fp32" else np.float16).max)
    assert _sig5(big_exact) == big
    assert O.round_to([big_exact], fmt)[0] == big_exact
    ulp_top = 2.0 ** (np.log2(big_exact).__floor__() - (row["fb"] - 1))
    assert np.isinf(O.round_to([big_exact + ulp_top / 2], fmt)[0])
    assert O.round_to([big_exact + ulp_top / 2 * 0.999], fmt)[0] == big_exact
    # smallest normal 2^emin and smallest subnormal 2^(emin - p + 1)
    emin = -(2 ** (row["eb"] - 1) - 2)
    assert _sig5(2.0 ** emin) == row["small_n"]
    sub = 2.0 ** (emin - row["fb"] + 1)
    assert _sig5(sub) == row["small_s"]
    assert O.round_to([sub], fmt)[0] == sub
    assert O.round_to([sub * 0.5], fmt)[0] == 0.0          # tie -> even (zero)
    assert O.round_to([sub * 0.5000001], fmt)[0] == sub
    assert O.round_to([sub * 1.5], fmt)[0] == 2 * sub       # tie -> even (2 sub)
    # unit roundoff u = 2^-p: 1 + u is a tie that rounds to 1, just above rounds up
    u = 2.0 ** (-row["fb"])
    assert _sig5(u) == row["u"]
    assert O.round_to([1.0 + u], fmt)[0] == 1.0
    assert O.round_to([1.0 + u * 1.0001], fmt)[0] == 1.0 + 2 * u
    assert O.round_to([1.0 + 3 * u], fmt)[0] == 1.0 + 4 * u  # tie -> even


def test_table1_fp64_identity(oracle_lib):
    row = _table1()["fp64"]
    assert _sig5(np.finfo(np.float64).eps / 2) == row["u"]
    x = np.random.default_rng(0).standard_normal(1000)
    assert np.array_equal(O.round_to(x, O.FP64), x)


def _random_doubles(rng, n, lo_exp, hi_exp):
    mant = rng.uniform(1.0, 2.0, n)
    ex = rng.integers(lo_exp, hi_exp, n)
    sign = rng.choice([-1.0, 1.0], n)
    return sign * np.ldexp(mant, ex)


def test_round_fp16_matches_numpy(oracle_lib):
    rng = np.random.default_rng(1)
    x = _random_doubles(rng, 2_000_000, -30, 18)
    # exact ties and near-ties between adjacent halves (normal and subnormal)
    h = rng.integers(0, 0x7BFF, 200_000, dtype=np.uint16).view(np.float16).astype(np.float64)
    ulp = np.spacing(h.astype(np.float16)).astype(np.float64)
    ties = np.concatenate([h + ulp / 2, h - ulp / 4, h + ulp / 2 * (1 + 2 ** -40),
                           -(h + ulp / 2)])
    x = np.concatenate([x, ties, [0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e9, -1e9]])
    ref = x.astype(np.float16).astype(np.float64)
    got = O.round_to(x, O.FP16)
    assert np.array_equal(got, ref)
    assert np.array_equal(np.signbit(got), np.signbit(ref))


def test_round_fp32_matches_numpy(oracle_lib):
    rng = np.random.default_rng(2)
    x = _random_doubles(rng, 2_000_000, -160, 130)
    f = rng.standard_normal(100_000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(f.astype(np.float32)).astype(np.float64)
    x = np.concatenate([x, f + ulp / 2, f - ulp / 2, f + ulp / 3])
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    assert np.array_equal(O.round_to(x, O.FP32), ref)


def test_round_bf16_matches_torch(oracle_lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2 ** 32, 3_000_000, dtype=np.uint64).astype(np.uint32)
    f = bits.view(np.float32)
    f = f[np.isfinite(f)]
    # add exact bf16 ties: bf16 value + half a bf16 ulp is a float32 value
    hb = (rng.integers(0, 0x7F7F, 100_000, dtype=np.uint32) << 16).view(np.float32)
    tie = (hb.view(np.uint32) | np.uint32(0x8000)).view(np.float32)
    f = np.concatenate([f, hb, tie, -tie])
    ref = torch.from_numpy(f.copy()).to(torch.bfloat16).to(torch.float64).numpy()
    got = O.round_to(f.astype(np.float64), O.BF16)
    assert np.array_equal(got, ref)


def _all_finite_halves():
    b = np.arange(0, 0x10000, dtype=np.uint32).astype(np.uint16)
    h = b.view(np.float16)
    return h[np.isfinite(h)]


@pytest.mark.parametrize("name,npop", [("add", np.add), ("sub", np.subtract),
                                       ("mul", np.multiply)])
def test_fp16_arithmetic_matches_numpy(oracle_lib, name, npop):
    """Every finite half against a random sample of 600 halves: the oracle's
    correctly rounded op equals numpy's float16 ufunc."""
    a = _all_finite_halves()
    rng = np.random.default_rng(4)
    bsel = rng.choice(a, 600, replace=False)
    A = np.repeat(a, bsel.size)
    B = np.tile(bsel, a.size)
    with np.errstate(over="ignore", invalid="ignore"):
        ref = npop(A, B).astype(np.float64)
    got = O.op(name, A.astype(np.float64), B.astype(np.float64), O.FP16)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.signbit(got[fin]), np.signbit(ref[fin]))
    assert np.array_equal(np.isinf(got[~fin]), np.isinf(ref[~fin]))


@pytest.mark.parametrize("name,npop", [("add", np.add), ("sub", np.subtract),
                                       ("mul", np.multiply)])
def test_fp32_arithmetic_matches_numpy(oracle_lib, name, npop):
    rng = np.random.default_rng(5)
    A = (rng.standard_normal(1_000_000) * np.exp(rng.uniform(-20, 20, 1_000_000))).astype(np.float32)
    B = (rng.standard_normal(1_000_000) * np.exp(rng.uniform(-20, 20, 1_000_000))).astype(np.float32)
    ref = npop(A, B).astype(np.float64)
    got = O.op(name, A.astype(np.float64), B.astype(np.float64), O.FP32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("name", ["add", "sub", "mul"])
def test_bf16_arithmetic_matches_torch(oracle_lib, name):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(6)
    n = 1_000_000
    A = torch.from_numpy(rng.standard_normal(n) * np.exp(rng.uniform(-30, 30, n))).to(torch.bfloat16)
    B = torch.from_numpy(rng.standard_normal(n) * np.exp(rng.uniform(-30, 30, n))).to(torch.bfloat16)
    ref = {"add": A + B, "sub": A - B, "mul": A * B}[name].to(torch.float64).numpy()
    got = O.op(name, A.to(torch.float64).numpy(), B.to(torch.float64).numpy(), O.BF16)
    assert np.array_equal(got, ref)


def test_stencil_c2_fp16_value(oracle_lib):
    """1/24 rounded to binary16 is 0x2955 = 0.041656494140625."""
    assert O.stencil_c2(O.FP16) == 0.041656494140625
    assert np.float16(O.stencil_c2(O.FP16)).view(np.uint16) == 0x2955
    assert O.stencil_c2(O.FP16) == float(np.float16(1.0 / 24.0))
    assert O.stencil_c2(O.FP32) == float(np.float32(1.0 / 24.0))
    assert O.stencil_c2(O.FP64) == 1.0 / 24.0


def test_rounding_exhaustive_all_binary32(oracle_lib, tmp_path):
    """Every finite binary32 bit pattern (2^32 - 2^24) rounds to binary16 and
    to bfloat16 exactly as the independent references in
    tests/exhaustive/rounding_all_binary32.c (the compiler's _Float16
    conversion; the round-to-nearest-even bit formula) do, sign included.
    About a minute on 8 cores."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = os.path.join(os.path.dirname(__file__), "exhaustive", "rounding_all_binary32.c")
    exe = str(tmp_path / "rounding_all_binary32")
    subprocess.check_call([gcc, "-O2", "-fopenmp", src, "-o", exe, "-ldl", "-lm"])
    out = subprocess.run([exe, O.build()], capture_output=True, text=True, timeout=900, check=True).stdout
    words = out.split()
    got = dict(zip(words[0::2], map(int, words[1::2])))
    assert got == {"checked": 2 ** 32 - 2 ** 24, "fp16_mismatches": 0, "bf16_mismatches": 0}, out


@pytest.fixture(scope="module")
def ops_all_pairs_exe(tmp_path_factory):
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    src = os.path.join(os.path.dirname(__file__), "exhaustive", "ops_all_pairs.c")
    exe = str(tmp_path_factory.mktemp("exhaustive") / "ops_all_pairs")
    subprocess.check_call([gcc, "-O2", "-fopenmp", src, "-o", exe, "-ldl", "-lm"])
    return exe


@pytest.mark.parametrize("fmt,op", [(O.FP16, 0), (O.FP16, 2), (O.BF16, 0), (O.BF16, 2)])
def test_arithmetic_exhaustive_all_pairs(oracle_lib, ops_all_pairs_exe, fmt, op):
    """Every pair of finite binary16 (bfloat16) operands: the oracle's a + b and
    a * b equal the references of tests/exhaustive/ops_all_pairs.c, computed in
    binary32 and rounded by the compiler's _Float16 conversion (by the
    round-to-nearest-even bit formula), value and sign; a - b is a + (-b).
    10 to 30 s each on 8 cores."""
    import subprocess
    out = subprocess.run([ops_all_pairs_exe, O.build(), str(fmt), str(op)], capture_output=True, text=True,
                         timeout=900, check=True).stdout
    words = out.split()
    got = dict(zip(words[0::2], map(int, words[1::2])))
    nfin = 63488 if fmt == O.FP16 else 65280
    assert got == {"pairs": nfin * nfin, "mismatches": 0}, out
