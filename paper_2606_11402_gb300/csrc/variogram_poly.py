#!/usr/bin/env python3
"""Writes variogram_poly.cuh: FP32 polynomials for the small-argument part of
the variogram gamma(r) = kappa(0) - kappa(r) (common.cuh, gamma_d2).

Each polynomial interpolates, at Chebyshev nodes of its interval, a smooth
positive function whose product with a^2 (or u) and e^-a gives gamma / s2
without cancellation:
  Matern-3/2:  phi(a) = (e^a - 1 - a) / a^2              on [0, 1]
  Matern-5/2:  phi(a) = (e^a - 1 - a - a^2/3) / a^2      on [0, 2]
  SE, Matern-1/2:  psi(u) = (1 - e^-u) / u               on [0, 1/2]
The interpolants are computed in 40-digit arithmetic (mpmath), converted to
monomial coefficients, rounded to FP32, and the largest relative error of
the FP32 Horner evaluation over a fine grid is printed beside them.

Run: python variogram_poly.py > variogram_poly.cuh
"""
import mpmath as mp
import numpy as np

mp.mp.dps = 40


def cheb_interp(f, lo, hi, deg):
    n = deg + 1
    nodes = [mp.mpf(lo + hi) / 2 + mp.mpf(hi - lo) / 2 * mp.cos(mp.pi * (2 * j + 1) / (2 * n))
             for j in range(n)]
    vals = [f(x) for x in nodes]
    # monomial coefficients by solving the Vandermonde system exactly enough
    A = mp.matrix([[x ** p for p in range(n)] for x in nodes])
    c = mp.lu_solve(A, mp.matrix(vals))
    return [c[p] for p in range(n)]


def horner32(cs, x):
    h = np.float32(cs[-1])
    for c in reversed(cs[:-1]):
        h = np.float32(np.float32(h * np.float32(x)) + np.float32(c))
    return h


def check(f, cs, lo, hi):
    worst = 0.0
    for x in np.linspace(lo, hi, 2001):
        x32 = float(np.float32(x))
        ref = f(mp.mpf(x32))
        got = horner32([float(np.float32(float(c))) for c in cs], x32)
        worst = max(worst, abs(float(got) / float(ref) - 1))
    return worst


def phi32(a):
    return (mp.e ** a - 1 - a) / a ** 2 if a != 0 else mp.mpf(1) / 2


def phi52(a):
    return (mp.e ** a - 1 - a - a * a / 3) / a ** 2 if a != 0 else mp.mpf(1) / 6


def psi(u):
    return (1 - mp.e ** (-u)) / u if u != 0 else mp.mpf(1)


def emit(name, f, lo, hi, deg, doc):
    cs = cheb_interp(f, lo, hi, deg)
    err = check(f, cs, lo, hi)
    body = ", ".join("%.9ef" % float(np.float32(float(c))) for c in cs)
    print(f"// {doc}: degree {deg} on [{lo}, {hi}], max relative error {err:.1e} in FP32")
    print(f"__device__ __forceinline__ float {name}(float x) {{")
    print(f"  constexpr float c[{deg + 1}] = {{{body}}};")
    print(f"  float h = c[{deg}];")
    print("#pragma unroll")
    print(f"  for (int i = {deg - 1}; i >= 0; i--) h = fmaf(h, x, c[i]);")
    print("  return h;")
    print("}")
    print()


if __name__ == "__main__":
    print("// Generated by variogram_poly.py (Chebyshev interpolation of the functions")
    print("// named below); do not edit.")
    print("#pragma once")
    print()
    print("namespace ggp {")
    print()
    emit("poly_m32", phi32, 0.0, 1.0, 6, "(e^a - 1 - a) / a^2")
    emit("poly_m52", phi52, 0.0, 2.0, 8, "(e^a - 1 - a - a^2/3) / a^2")
    emit("poly_exp1", psi, 0.0, 0.5, 5, "(1 - e^-u) / u")
    print("}  // namespace ggp")
