"""Iteration ratios n(alpha) / n(1) of the red-black CGNE solve (Sec. 3, Table 1).

For one parameter row (mass, Ls, Mobius b, c or the Zolotarev coefficients)
every (field, point source, alpha) combination is solved to the FP64 true
Schur residual `tol` in one batched dwf_cgne_solve call per field (the alphas
are per right-hand side, so one handle serves the whole scan).  The 4D
propagator does not depend on alpha (Eq. tosolve1); only the conditioning of
D_bb, and hence the iteration count n, does.  Reported per alpha: the mean and
standard deviation over fields and sources of n(alpha)/n(1), the best alpha
and the speed-up 1 - n(best)/n(1) in percent.

Iteration counts are exact to 2 (the solver polls its residual every 2
iterations here).

Usage:
    python -m paper_1501_04950_gb300.alpha_scan --row 2 --lattice 16,16,16,32
The rows are those of Table 1; fields are synthetic (seeded) SU(3) links, so
the numbers are a trend, not a reproduction of the MILC ensembles.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

# (mass, Ls, b, c); b = c = None selects the Zolotarev coefficients on [0.05, 6]
TABLE1_ROWS = [
    (0.06, 4, 1.0, 1.0),
    (0.06, 6, 1.0, 1.0),
    (0.06, 8, 1.0, 1.0),
    (0.06, 10, 1.0, 1.0),
    (0.06, 12, 1.0, 1.0),
    (0.01, 8, 1.0, 1.0),
    (0.06, 8, 1.7, 0.7),
    (0.06, 10, None, None),
]


ORDERS = ("concave", "ascending", "descending", "random")


def order_coefficients(a, order):
    """Place the Zolotarev coefficients a_i along the 5th dimension (Sec. 3): concave
    (smallest at s = 1 and Ls, largest in the centre), ascending, descending, or a
    seeded random permutation."""
    from synthetic import concave_order
    a = np.sort(np.asarray(a, dtype=np.float64))
    if order == "concave":
        return concave_order(a)
    if order == "ascending":
        return a
    if order == "descending":
        return a[::-1].copy()
    if order == "random":
        return np.random.default_rng(7).permutation(a)
    raise ValueError("order must be one of %s" % (ORDERS,))


def row_coefficients(row, order="concave"):
    from synthetic import zolotarev_sign_coefficients
    mass, Ls, b, c = row
    if b is None:
        a, _ = zolotarev_sign_coefficients(Ls, 0.05, 6.0)
        a = order_coefficients(a, order)
        return mass, Ls, 0.5 * (a + 1.0), 0.5 * (a - 1.0)
    return mass, Ls, np.full(Ls, float(b)), np.full(Ls, float(c))


def scan(row, lattice=(16, 16, 16, 32), alphas=None, fields=1, eps=0.5, M5=-1.8, tol=1e-8,
         precision=None, sources=12, device="cuda", form=0, order="concave", solver=None):
    """Run the scan for one row; returns a dict of per-alpha ratio statistics and
    the iteration counts [field][source][alpha].

    form selects the red-black operator of Sec. 3 (dwf.SCHUR_*: 0 Eq. redblack,
    1 Eq. redblack1, 2 Eq. redblack1 with scaled rows); order places the
    Zolotarev coefficients of a Zolotarev row (ORDERS); solver is a
    dwf.SOLVER_* (default: inner precision with FP64 reliable updates)."""
    import torch
    from synthetic import gauge_field, point_source4d
    from . import dwf

    mass, Ls, b, c = row_coefficients(row, order)
    if alphas is None:
        alphas = [round(0.3 + 0.05 * k, 2) for k in range(19)]  # 0.3 .. 1.2
    alphas = list(alphas)
    if 1.0 not in alphas:
        alphas.append(1.0)
    precision = dwf.FP32 if precision is None else precision
    pts = [(sp, col) for sp in range(4) for col in range(3)][:sources]
    n = np.zeros((fields, len(pts), len(alphas)))
    t0 = time.perf_counter()
    for f in range(fields):
        U = torch.from_numpy(gauge_field(lattice, eps, seed=f)).to(device)
        srcs = np.stack([point_source4d(lattice, sp, col) for sp, col in pts])
        src = torch.from_numpy(np.concatenate([srcs] * len(alphas))).to(device)
        al = [a for a in alphas for _ in pts]
        # poll every 2 iterations: the counts are exact to 2 instead of 16
        extra = {} if solver is None else {"solver": solver}
        op = dwf.DWF(lattice, Ls, M5, mass, 1.0, b, c, rel_tol=tol, precision_inner=precision,
                     check_every=2, schur_form=form, **extra)
        op.load_gauge(U)
        prop = torch.empty_like(src)
        st = op.cgne_solve(src, prop, nrhs=len(al), alphas=al)
        op.close()
        its = np.array([x["iterations"] for x in st], dtype=float).reshape(len(alphas), len(pts))
        n[f] = its.T
    one = alphas.index(1.0)
    ratio = n / n[:, :, one:one + 1]
    mean = ratio.mean(axis=(0, 1))
    std = ratio.std(axis=(0, 1))
    best = int(np.argmin(mean))
    return {
        "row": {"mass": mass, "Ls": Ls, "b": "zolotarev" if row[2] is None else row[2],
                "c": "zolotarev" if row[3] is None else row[3]},
        "form": form, "order": order if row[2] is None else None, "lattice": list(lattice), "fields": fields, "sources": len(pts), "tol": tol,
        "alphas": alphas, "ratio_mean": mean.tolist(), "ratio_std": std.tolist(),
        "iterations_alpha1_mean": float(n[:, :, one].mean()),
        "best_alpha": alphas[best], "speedup_percent": 100.0 * (1.0 - mean[best]),
        "iterations": n.astype(int).tolist(),
        "seconds": time.perf_counter() - t0,
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--row", type=int, action="append",
                    help="Table 1 row index 0..7 (repeatable; default: all)")
    ap.add_argument("--lattice", default="16,16,16,32")
    ap.add_argument("--fields", type=int, default=1)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--alphas", default=None, help="comma-separated alpha values")
    ap.add_argument("--form", type=int, default=0,
                    help="red-black operator: 0 Eq. redblack, 1 Eq. redblack1, 2 row-scaled")
    ap.add_argument("--order", default="concave", choices=ORDERS,
                    help="placement of the Zolotarev coefficients along the 5th dimension")
    args = ap.parse_args(argv)
    lattice = tuple(int(v) for v in args.lattice.split(","))
    alphas = [float(a) for a in args.alphas.split(",")] if args.alphas else None
    rows = args.row if args.row else list(range(len(TABLE1_ROWS)))
    out = []
    for r in rows:
        res = scan(TABLE1_ROWS[r], lattice=lattice, alphas=alphas, fields=args.fields,
                   tol=args.tol, form=args.form, order=args.order)
        print(json.dumps(res), flush=True)
        out.append(res)
    return out


if __name__ == "__main__":
    main()
