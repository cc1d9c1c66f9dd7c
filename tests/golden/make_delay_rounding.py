"""Write delay_rounding.txt: dispersion delays whose exact value pins the
rounding mode of the delay table.

The delay of channel c at trial DM d is the cold-plasma sweep, described in
words in the paper's Section 2.2 and taken here with the constant
4.148808e3 s MHz^2 / (pc cm^-3):

    delay[d][c] = round( 4.148808e3 * DM_d * (f_c^-2 - f_max^-2) / t_samp )

with f in MHz, t_samp = 64 us, channel centres f_c = 1581.8 - (c + 1/2) * df
(highest first, f_max = f_0) and round = nearest, halves away from zero.

This script evaluates the expression inside round() EXACTLY, in rational
arithmetic (fractions.Fraction) from the decimal inputs, so it depends on no
floating-point code and on nothing in the repository.  It keeps entries whose
exact fractional part lies in [0.55, 0.95] (round != floor, truncation) and
in [0.05, 0.45] (round != ceil), away from every boundary by far more than
double rounding can move them, over the 1024-channel and 64-channel bands and
their DM grids.  Run: python tests/golden/make_delay_rounding.py
"""
from fractions import Fraction
import math
import os

KDM = Fraction("4.148808e3")
TSAMP = Fraction("64e-6")
F_TOP = Fraction("1581.8")
BW = Fraction(400)


def centres(nchan):
    df = BW / nchan
    return [F_TOP - (c + Fraction(1, 2)) * df for c in range(nchan)]


def piecewise_dms():
    out = []
    for lo, hi, step in ((0, 100, Fraction(1, 4)), (100, 300, Fraction(1, 2)), (300, 1000, Fraction(1))):
        n = int((hi - lo) / step)
        out += [lo + step * i for i in range(n)]
    return out


def linear_dms(ndm, end):
    return [Fraction(end) * i / ndm for i in range(ndm)]


def exact_delay(dm, f, fmax):
    return KDM * dm * (1 / (f * f) - 1 / (fmax * fmax)) / TSAMP


def pick(nchan, dms, dm_rule, want_hi, want_lo):
    f = centres(nchan)
    hi, lo = [], []
    # at most one entry per trial, trials spread over the whole grid, channels
    # walked from a different start for each trial
    ntr = want_hi + want_lo
    for k in range(ntr):
        d = 1 + (len(dms) - 2) * k // max(1, ntr - 1)
        need_hi = len(hi) < want_hi and (k % 3 != 2 or len(lo) >= want_lo)
        for j in range(nchan - 1):
            c = 1 + (j * 7 + k * 131) % (nchan - 1)
            v = exact_delay(dms[d], f[c], f[0])
            frac = v - math.floor(v)
            if need_hi and Fraction(55, 100) <= frac <= Fraction(95, 100):
                hi.append((nchan, dm_rule, d, c, v))
                break
            if not need_hi and Fraction(5, 100) <= frac <= Fraction(45, 100):
                lo.append((nchan, dm_rule, d, c, v))
                break
    return hi + lo


def main():
    rows = pick(1024, piecewise_dms(), "piecewise1000", 8, 3) + pick(64, linear_dms(64, 100), "linear64x100", 4, 2)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "delay_rounding.txt")
    with open(path, "w") as fh:
        fh.write("# Dispersion delays (samples) evaluated exactly in rational arithmetic by\n"
                 "# make_delay_rounding.py; paper Section 2.2 (dispersive delay, in words),\n"
                 "# constant 4.148808e3 s MHz^2 cm^3/pc, t_samp 64 us, channel centres\n"
                 "# 1581.8 - (c+1/2)*400/nchan MHz, f_max = channel 0, round half away from zero.\n"
                 "# columns: nchan dm_grid trial channel exact_value(15 decimals) rounded floor ceil\n")
        for nchan, rule, d, c, v in rows:
            fl = math.floor(v)
            rounded = fl + 1 if v - fl >= Fraction(1, 2) else fl
            fh.write(f"{nchan} {rule} {d} {c} {float(v):.15f} {rounded} {fl} {math.ceil(v)}\n")
    print(f"wrote {len(rows)} entries to {path}")


if __name__ == "__main__":
    main()
