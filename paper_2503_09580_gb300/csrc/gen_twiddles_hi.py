"""Write twiddles_hi.h: W_n^m = exp(-2 pi i m / n) for n = 64 and 48 as
unevaluated sums of two doubles (hi + lo, hi the correctly rounded double,
lo the correctly rounded remainder), from 60-digit decimal arithmetic.  The
library's FFT twiddles of every precision (double, float, and the two-fold
forms) are derived from this table on the host.

It also writes the scaled form of W_32^m used by the register transforms
(fft_reg.cuh): W = sc (1 + i q) where |cos| >= |sin|, else W = sc (q + i),
so that |q| <= 1 and a butterfly with a twiddle takes six fused
multiply-adds (the scaled-twiddle radix-2 butterfly of Linzer and Feig);
sc and q are the correctly rounded doubles of the exact values.

    python gen_twiddles_hi.py > twiddles_hi.h
"""
from decimal import Decimal, getcontext

getcontext().prec = 60


def pi():
    # Machin: pi = 16 atan(1/5) - 4 atan(1/239)
    def atan_inv(x):
        x = Decimal(x)
        term, s, k, x2 = 1 / x, Decimal(0), 0, x * x
        while True:
            t = term / (2 * k + 1)
            if t < Decimal(10) ** -58:
                break
            s += -t if k % 2 else t
            term /= x2
            k += 1
        return s
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def cos_sin(a):
    c, s, term, k = Decimal(0), Decimal(0), Decimal(1), 0
    while abs(term) > Decimal(10) ** -58 or k < 4:
        if k % 4 == 0:
            c += term
        elif k % 4 == 1:
            s += term
        elif k % 4 == 2:
            c -= term
        else:
            s -= term
        k += 1
        term = term * a / k
    return c, s


def split(x):
    # round off the series' last digits, so that exact values (0, +-1/2, +-1)
    # come out exact
    x = x.quantize(Decimal(10) ** -50)
    hi = float(x)
    lo = float(x - Decimal(hi))
    return hi, lo


def table(n):
    P = pi()
    rows = []
    for m in range(n):
        c, s = cos_sin(-2 * P * m / n)
        rows.append(split(c) + split(s))
    return rows


def scaled(n):
    P = pi()
    rows = []
    for m in range(n // 2):
        c, s = cos_sin(-2 * P * m / n)
        c, s = c.quantize(Decimal(10) ** -50), s.quantize(Decimal(10) ** -50)
        if abs(c) >= abs(s):
            rows.append((0, float(c), float(s / c)))
        else:
            rows.append((1, float(s), float(c / s)))
    return rows


def emit_scaled(name, n, rows):
    print("// W_%d^m, m < %d: kind 0: sc (1 + i q); kind 1: sc (q + i)" % (n, n // 2))
    print("struct ScaledTw {")
    print("  int kind;")
    print("  double sc, q;")
    print("};")
    print("LBO_HD constexpr ScaledTw %s(int m) {" % name)
    print("  switch (m) {")
    for m, (k, sc, q) in enumerate(rows):
        print("    case %d: return {%d, %s, %s};" % (m, k, sc.hex(), q.hex()))
    print("    default: return {0, 0.0, 0.0};")
    print("  }")
    print("}")


def emit_cos(name, n):
    P = pi()
    print("// cos(2 pi m / %d), m < %d, correctly rounded" % (n, n))
    print("LBO_HD constexpr double %s(int m) {" % name)
    print("  switch (m) {")
    for m in range(n):
        c, _ = cos_sin(2 * P * m / n)
        print("    case %d: return %s;" % (m, float(c.quantize(Decimal(10) ** -50)).hex()))
    print("    default: return 0.0;")
    print("  }")
    print("}")


def emit(name, rows):
    print("static const double %s[%d][4] = {" % (name, len(rows)))
    for r in rows:
        print("    {%s, %s, %s, %s}," % tuple(x.hex() for x in r))
    print("};")


if __name__ == "__main__":
    print("// Generated by gen_twiddles_hi.py: W_n^m = exp(-2 pi i m/n) as double pairs")
    print("// {cos_hi, cos_lo, sin_hi, sin_lo}, hi + lo accurate to ~2^-106.")
    print("#pragma once")
    emit("kTw64Hi", table(64))
    emit("kTw48Hi", table(48))
    print("#ifndef LBO_HD")
    print("#ifdef __CUDACC__")
    print("#define LBO_HD __host__ __device__")
    print("#else")
    print("#define LBO_HD")
    print("#endif")
    print("#endif")
    emit_scaled("scaled_tw32", 32, scaled(32))
    emit_cos("cos32", 32)
