"""Writes csrc/swkb_fc_tables.h: the FC-Gram continuation operator the
library's patch-wise path uses (Sec. 2.2; FC-Gram of Bruno & Lyon 2010 and
Albin & Bruno 2011).

Run once when the parameters change (needs mpmath):
    python -m paper_2301_03814_gb300.fc_tables

The operator maps the d samples ending a patch (ordered towards the end) to
the C values that continue them and blend to zero.  Construction, in 100-digit
arithmetic:
  * Gram polynomials q_0 .. q_{d-1}: classical Gram-Schmidt (applied twice) of
    1, x, .., x^{d-1} in the inner product sum_{x=0}^{d-1} f(x) g(x); column j
    of G holds q_j's values at x = 0 .. d-1 and its monomial coefficients are
    kept alongside;
  * each q_j is blended to zero by the trigonometric polynomial of period
    2 (d + C) with H harmonics fitted in the least-squares sense to q_j on
    [0, d - 1] and to 0 on [d + C, 2 d + C - 1], both sampled o times per
    unit, solved through its normal equations, and evaluated at d .. d + C - 1;
  * operator = B G^T (B: C x d blends), independent of the signs of the q_j.
d = 5, C = 25, H = 12, o = 20.
"""
from __future__ import annotations

import os

D, C, HARMONICS, OVERSAMPLE, DIGITS = 5, 25, 12, 20, 100


def continuation_operator():
    import mpmath as mp

    with mp.workdps(DIGITS):
        xs = [mp.mpf(x) for x in range(D)]
        # Gram-Schmidt on monomials: polys[j] = monomial coefficients of q_j
        polys = []
        for j in range(D):
            coef = [mp.mpf(0)] * D
            coef[j] = mp.mpf(1)
            for _ in range(2):
                for q in polys:
                    dot = mp.fsum(mp.polyval(coef[::-1], x) * mp.polyval(q[::-1], x) for x in xs)
                    coef = [a - dot * b for a, b in zip(coef, q)]
            nrm = mp.sqrt(mp.fsum(mp.polyval(coef[::-1], x) ** 2 for x in xs))
            polys.append([a / nrm for a in coef])
        period = 2 * (D + C)

        def trig_row(x):
            row = [mp.mpf(1)]
            for m in range(1, HARMONICS + 1):
                a = 2 * mp.pi * m * x / period
                row.append(mp.cos(a))
                row.append(mp.sin(a))
            return row

        fit_match = [mp.mpf(i) / OVERSAMPLE for i in range((D - 1) * OVERSAMPLE + 1)]
        fit_zero = [D + C + mp.mpf(i) / OVERSAMPLE for i in range((D - 1) * OVERSAMPLE + 1)]
        rows = [trig_row(x) for x in fit_match + fit_zero]
        ncol = len(rows[0])
        normal = mp.matrix(ncol, ncol)
        for a in range(ncol):
            for b in range(a, ncol):
                v = mp.fsum(r[a] * r[b] for r in rows)
                normal[a, b] = v
                normal[b, a] = v
        blends = []
        for q in polys:
            rhs = mp.matrix(ncol, 1)
            target = [mp.polyval(q[::-1], x) for x in fit_match] + [mp.mpf(0)] * len(fit_zero)
            for a in range(ncol):
                rhs[a] = mp.fsum(r[a] * t for r, t in zip(rows, target))
            sol = mp.lu_solve(normal, rhs)
            blends.append([mp.fsum(c * s for c, s in zip(trig_row(mp.mpf(D + i)), sol))
                           for i in range(C)])
        gram = [[mp.polyval(q[::-1], x) for q in polys] for x in xs]    # G[x][j]
        return [[float(mp.fsum(blends[j][i] * gram[x][j] for j in range(D))) for x in range(D)]
                for i in range(C)]


def write_header(path: str | None = None) -> str:
    op = continuation_operator()
    path = path or os.path.join(os.path.dirname(__file__), "csrc", "swkb_fc_tables.h")
    lines = [
        "// Generated by paper_2301_03814_gb300/fc_tables.py -- do not edit.",
        "// FC-Gram continuation operator (d = 5 matching points, C = 25",
        "// continuation points, 12-harmonic blend-to-zero fits): row i gives the",
        "// i-th value past a patch end as a combination of the d samples ending",
        "// the patch, ordered towards the end.",
        "#pragma once",
        "",
        "namespace swkb {",
        f"constexpr int FC_D = {D};",
        f"constexpr int FC_C = {C};",
        "static const double kFcContinuation[FC_C][FC_D] = {",
    ]
    for row in op:
        lines.append("    {" + ", ".join(f"{v:.17e}" for v in row) + "},")
    lines += ["};", "}  // namespace swkb", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))
    return path


if __name__ == "__main__":
    print(write_header())
