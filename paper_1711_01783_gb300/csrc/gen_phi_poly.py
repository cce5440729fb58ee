"""Generate phi_poly.h: polynomial pieces of the float phi(x) = -ln tanh(x/2).

Two unit systems are fitted.  Natural units (LLRs in nats, used by the
weighted-BP kernels) and base-2 units (LLRs in bits, y = x log2 e, used by the
decoding kernels), where the map is psi(y) = log2(e) phi(y ln 2):

  y <  Y0 :  psi(y) = C0 - lg2(y) - u * Qs(u),   u = y^2,  C0 = 1 - log2(ln 2)
  y >= Y0 :  psi(y) = e * Ql(e^2),               e = 2^-y
with Y0 = X0 log2 e.  In bits the hardware ex2 takes -y directly, which saves
the multiplication by log2 e that the natural-unit large piece needs.  The
device evaluates both base-2 pieces and takes their maximum: with a positive
top coefficient of Qs the small piece drops below the large one past Y0, and
the large piece stays below the small one under Y0 (check_max_of_pieces).

Build-time script for the CUDA decoder (run by hand when the split point or
degrees change; its output is committed).  The device evaluates phi on
[phi(25), 25] as

  x <  X0 :  phi(x) = ln 2 - ln(x) - t * Ps(t),      t = x^2
             where t * Ps(t) approximates h(x) = ln(tanh(x/2) / (x/2)),
             an even function analytic for |x| < pi;
  x >= X0 :  phi(x) = 2 atanh(e) = e * Pl(e^2),      e = exp(-x)
             where Pl(z) approximates 2 atanh(sqrt z) / sqrt z.

ln(x) and exp(-x) come from the hardware base-2 approximations (MUFU lg2 /
ex2).  The coefficients are least-squares fits on Chebyshev nodes of the
interval (a near-minimax fit), computed in float64 from the closed forms
above with numpy.
"""
import os

import numpy as np

X0 = 1.25
# Natural units: one fit (weighted BP).  Base-2 units: "accurate" (used with
# float message storage; 1.5e-7 relative, about one float ulp) and "half"
# (used with half storage: two coefficients per piece, 2.0e-4 relative,
# below the 2^-11 = 4.9e-4 rounding of a stored message).
FITS = {"": (5, 4)}                # natural units: prefix -> (coefficients of Ps, of Pl)
FITS2 = {"2": (4, 4), "2H": (2, 2)}  # base-2 units: accurate and half


def _cheb(lo, hi, k=6000):
    return lo + (hi - lo) * (np.cos(np.linspace(0, np.pi, k)) + 1) / 2


def fit(deg_small, deg_large):
    t = _cheb(1e-10, X0 * X0)
    x = np.sqrt(t)
    h = np.log(np.tanh(x / 2) / (x / 2))
    cs = np.polynomial.polynomial.polyfit(t, h / t, deg_small - 1)
    err_s = np.max(np.abs(np.polynomial.polynomial.polyval(t, cs) * t - h))
    z = _cheb(1e-14, np.exp(-2 * X0))
    e = np.sqrt(z)
    pl = 2.0 * np.arctanh(e) / e
    cl = np.polynomial.polynomial.polyfit(z, pl, deg_large - 1)
    err_l = np.max(np.abs(np.polynomial.polynomial.polyval(z, cl) / pl - 1))
    return cs, cl, err_s, err_l


def fit2(deg_small, deg_large):
    """Base-2 pieces: Qs(u) = log2e h(sqrt(u) ln2) / u and Ql(z) = log2e 2 atanh(sqrt z)/sqrt z."""
    ln2, log2e = np.log(2.0), 1.0 / np.log(2.0)
    y0 = X0 * log2e
    u = _cheb(1e-10, y0 * y0)
    x = np.sqrt(u) * ln2
    hs = log2e * np.log(np.tanh(x / 2) / (x / 2))
    cs = np.polynomial.polynomial.polyfit(u, hs / u, deg_small - 1)
    err_s = np.max(np.abs(np.polynomial.polynomial.polyval(u, cs) * u - hs))
    z = _cheb(1e-14, np.exp(-2 * X0))
    e = np.sqrt(z)
    pl = log2e * 2.0 * np.arctanh(e) / e
    cl = np.polynomial.polynomial.polyfit(z, pl, deg_large - 1)
    err_l = np.max(np.abs(np.polynomial.polynomial.polyval(z, cl) / pl - 1))
    return cs, cl, err_s, err_l


def check_max_of_pieces(cs, cl, lmax_nats=25.0):
    """The device takes psi(y) = max(small piece, large piece).  Check, with
    the coefficients rounded to float, that the maximum picks the accurate
    piece everywhere on [psi(lmax), lmax]: past the split the small piece
    must fall below the large one, which needs a positive top coefficient of
    Qs.  Returns the maximum's largest relative error against psi."""
    ln2 = np.log(2.0)
    assert cs[-1] > 0, "top coefficient of Qs must be positive for the max() form"
    ymax = lmax_nats / ln2
    ymin = np.log1p(2.0 / np.expm1(lmax_nats)) / ln2
    y = np.geomspace(ymin, ymax, 400001)
    c32s = cs.astype(np.float32).astype(np.float64)
    c32l = cl.astype(np.float32).astype(np.float64)
    u = y * y
    small = (1.0 - np.log2(ln2)) - u * np.polynomial.polynomial.polyval(u, c32s) - np.log2(y)
    e = 2.0 ** -y
    large = e * np.polynomial.polynomial.polyval(e * e, c32l)
    ref = np.log1p(2.0 / np.expm1(y * ln2)) / ln2
    got = np.maximum(small, large)
    piece = np.where(y < X0 / ln2, small, large)
    err_piece = np.max(np.abs(piece / ref - 1))
    err = np.max(np.abs(got / ref - 1))
    assert err <= 1.01 * err_piece + 1e-7, (err, err_piece)
    return err


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "phi_poly.h")
    lines = [
        "// Generated by gen_phi_poly.py -- polynomial pieces of phi(x) = -ln tanh(x/2).",
        f"// small branch x < {X0}: phi = ln2 - ln x - t*Ps(t), t = x^2",
        "// large branch: phi = e*Pl(e^2), e = exp(-x)",
        "#pragma once",
        f"#define MLD_PHI_X0 {X0:.9g}f",
    ]
    for pre, (ds, dl) in FITS.items():
        cs, cl, err_s, err_l = fit(ds, dl)
        lines.append(f"// fit '{pre or 'accurate'}': max |small fit error| {err_s:.2e}, "
                     f"max relative large fit error {err_l:.2e}")
        for i, c in enumerate(cs):
            lines.append(f"#define MLD_PHI{pre}_S{i} ({c:.9e}f)")
        for i, c in enumerate(cl):
            lines.append(f"#define MLD_PHI{pre}_L{i} ({c:.9e}f)")
        print(pre, err_s, err_l)
    ln2, log2e = np.log(2.0), 1.0 / np.log(2.0)
    lines.append(f"#define MLD_PHI2_Y0 {X0 * log2e:.9g}f")
    lines.append(f"#define MLD_PHI2_C0 {1.0 - np.log2(ln2):.9g}f")
    for pre, (ds, dl) in FITS2.items():
        cs, cl, err_s, err_l = fit2(ds, dl)
        err_max = check_max_of_pieces(cs, cl)
        lines.append(f"// base-2 fit '{pre}': max |small fit error| {err_s:.2e} (bits), "
                     f"max relative large fit error {err_l:.2e}; max(small, large) "
                     f"relative error {err_max:.2e} on [psi(lmax), lmax]")
        for i, c in enumerate(cs):
            lines.append(f"#define MLD_PHI{pre}_S{i} ({c:.9e}f)")
        for i, c in enumerate(cl):
            lines.append(f"#define MLD_PHI{pre}_L{i} ({c:.9e}f)")
        print(pre, err_s, err_l)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
