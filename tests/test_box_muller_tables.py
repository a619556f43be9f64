"""The constant tables of the Gaussian draw's table-driven logarithm and sine/cosine (csrc/box_muller_tables.cuh)
against the functions they tabulate, evaluated here with Python's libm: 1/F_j, ln F_j = hi + lo with hi a
multiple of 2^-40, cos and sin of 2 pi k / 256, ln 2 = hi + lo and 2 pi 2^-53."""
import math
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1406_5802_gb300", "csrc", "box_muller_tables.cuh")


def _tables():
    text = open(HDR).read()

    def rows(name):
        body = text[text.index(name):]
        body = body[body.index("{") + 1:body.index("};")]
        return [[float.fromhex(v) for v in re.findall(r"[-0-9a-fx.p+]+", r)] for r in re.findall(r"\{([^{}]*)\}", body)]

    consts = {m.group(1): float.fromhex(m.group(2))
              for m in re.finditer(r"constexpr double (\w+) = ([-0-9a-fx.p+]+);", text)}
    return rows("kLogTable"), rows("kSinCosTable"), consts


def ulp(x):
    return math.ulp(abs(x)) if x != 0 else math.ulp(0.0)


def test_log_table():
    lt, _, c = _tables()
    assert len(lt) == 256
    for j, (inv, hi, lo) in enumerate(lt):
        F = 1 + j / 256
        assert abs(inv - 1 / F) <= ulp(1 / F)
        assert hi * 2**40 == round(hi * 2**40)  # a multiple of 2^-40
        assert abs(lo) <= 2.0**-41
        assert abs((hi - math.log(F)) + lo) <= 2 * ulp(math.log(F)) + 1e-30
    assert c["kLn2Hi"] * 2**40 == round(c["kLn2Hi"] * 2**40)
    assert abs((c["kLn2Hi"] - math.log(2)) + c["kLn2Lo"]) <= ulp(math.log(2))
    assert c["kTwoPi53"] == (2 * math.pi) * 2.0**-53


def _cos_sin_turn(k):
    """cos, sin of 2 pi k / 256 from the first octant by exact symmetries (the angle is rounded only there,
    where it is below pi / 4)."""
    k %= 256
    q, r = divmod(k, 64)  # quadrant, position in it (0 .. 63 of pi/128 steps)
    if r <= 32:
        a = math.pi * r / 128
        c, s = math.cos(a), math.sin(a)
    else:
        a = math.pi * (64 - r) / 128
        c, s = math.sin(a), math.cos(a)
    for _ in range(q):  # rotate by a quarter turn
        c, s = -s, c
    return c, s


def test_sincos_table():
    _, sc, _ = _tables()
    assert len(sc) == 256
    for k, (cv, sv) in enumerate(sc):
        c, s = _cos_sin_turn(k)
        assert abs(cv - c) <= 2 * ulp(1.0) and abs(sv - s) <= 2 * ulp(1.0), k
    assert sc[0] == [1.0, 0.0] and sc[64] == [0.0, 1.0] and sc[128] == [-1.0, 0.0] and sc[192] == [0.0, -1.0]
