"""Writes box_muller_tables.cuh: the constant tables of the table-driven logarithm and sine/cosine that
gaussian_kernel (gen.cu) uses for the Box-Muller transform, evaluated with mpmath at 50 digits and rounded
to FP64.

Logarithm (Tang, "Table-driven implementation of the logarithm function in IEEE floating-point
arithmetic", ACM TOMS 16(4), 1990): for F_j = 1 + j/256, j = 0..255, 1/F_j and ln F_j split as
hi + lo with hi a multiple of 2^-40, so that e ln2_hi + hi is exact for the exponents Box-Muller meets.
Sine/cosine: cos and sin of 2 pi k / 256, k = 0..255, for the reduction theta = 2 pi k / 256 + phi.

Run: python gen_box_muller_tables.py > box_muller_tables.cuh
"""
import mpmath as mp

mp.mp.dps = 50


def rn(x):
    """x rounded to the nearest FP64 value (mpmath rounds to nearest, ties to even, at 53 bits)."""
    return float(mp.mpf(x))


def hex_double(x):
    return float(x).hex()


def split40(x):
    """(hi, lo): hi = x rounded to a multiple of 2^-40, lo = x - hi rounded to FP64."""
    hi = mp.nint(x * mp.mpf(2) ** 40) / mp.mpf(2) ** 40
    return float(hi), rn(x - hi)


def main():
    ln2 = mp.log(2)
    ln2_hi, ln2_lo = split40(ln2)
    assert mp.mpf(ln2_hi) * 2**40 == int(mp.mpf(ln2_hi) * 2**40)
    out = []
    out.append("// box_muller_tables.cuh -- written by gen_box_muller_tables.py (mpmath, 50 digits, rounded to FP64).")
    out.append("// Tables of the table-driven logarithm (Tang 1990) and of cos, sin at 2 pi k / 256 used by")
    out.append("// gaussian_kernel's Box-Muller transform.")
    out.append("#pragma once")
    out.append("")
    out.append("namespace rmge {")
    out.append("namespace bm {")
    out.append(f"constexpr double kLn2Hi = {hex_double(ln2_hi)};  // ln 2 to a multiple of 2^-40")
    out.append(f"constexpr double kLn2Lo = {hex_double(ln2_lo)};")
    out.append(f"constexpr double kTwoPi53 = {hex_double(rn(2 * mp.pi) * 2.0**-53)};  // RN(2 pi) 2^-53")
    out.append("")
    out.append("// {1 / F_j, hi(ln F_j), lo(ln F_j)}, F_j = 1 + j / 256")
    out.append("__device__ const double kLogTable[256][3] = {")
    for j in range(256):
        F = 1 + mp.mpf(j) / 256
        hi, lo = split40(mp.log(F))
        out.append(f"    {{{hex_double(rn(1 / F))}, {hex_double(hi)}, {hex_double(lo)}}},")
    out.append("};")
    out.append("")
    out.append("// {cos, sin} of 2 pi k / 256")
    out.append("__device__ const double kSinCosTable[256][2] = {")
    for k in range(256):
        a = mp.mpf(k) / 128  # the angle in units of pi: cospi and sinpi are exact at multiples of 1/2
        out.append(f"    {{{hex_double(rn(mp.cospi(a)))}, {hex_double(rn(mp.sinpi(a)))}}},")
    out.append("};")
    out.append("}  // namespace bm")
    out.append("}  // namespace rmge")
    print("\n".join(out))


if __name__ == "__main__":
    main()
