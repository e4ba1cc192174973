"""Run the constrained minimax fits for a range of orders and write the table.

Usage:  python -m paper_2504_07637_gb300.fit.run_fits --bits 53 --n 0-37 [--jobs 8]

Orders N default to Table I of the paper (Sec. 3): for 53-bit targets
N = 10 (n = 0-1), 11 (2-6), 12 (7-10), 13 (11-17), 14 (18 and up); for 24-bit
targets N = 4 (0-1), 5 (2-9), 6 (10 and up).  The blank N cells of the
printed table are read as repeating the row above.

The JSON written holds every fitted quantity as a decimal string with 40
significant digits, so the code generator can round it to any precision.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mproc
import os
import time

import mpmath as mp

from . import boys_fit as bf

HERE = os.path.dirname(os.path.abspath(__file__))
COEFF_DIR = os.path.join(os.path.dirname(HERE), "coeffs")


def table_order(n: int, bits: int) -> int:
    if bits > 24:
        return 10 if n <= 1 else 11 if n <= 6 else 12 if n <= 10 else 13 if n <= 17 else 14
    return 4 if n <= 1 else 5 if n <= 9 else 6


def _s(v) -> str:
    return mp.nstr(v, 40, strip_zeros=False)


def _factors(f):
    quad, lin, poly = f
    return {"quad": [[_s(y), _s(a)] for y, a in quad], "lin": [_s(y) for y in lin], "poly": [_s(c) for c in poly]}


def job(args):
    n, N, bits, warm = args
    t0 = time.time()
    r, errors = None, []
    dps = 50 if bits > 24 else 40
    if warm is not None:
        # Remez started from a neighbouring order's alternation points
        try:
            mp.mp.dps = dps
            r = bf.fit(n, N, bits, dps=dps, verbose=False, warm=[mp.mpf(v) for v in warm])
        except Exception as exc:
            errors.append(repr(exc))
    # a singular solve or a spurious pole depends on the grid; retry on others
    for grid, iters in ((600, 30), (800, 40), (450, 25)) if r is None else ():
        try:
            r = bf.fit(n, N, bits, dps=dps, grid=grid, verbose=False, lawson_iters=iters)
            break
        except Exception as exc:
            errors.append(repr(exc))
    if r is None:  # a failed order is reported, not fatal
        return {"n": n, "N": N, "bits": bits, "error": "; ".join(errors)}
    k = r["k"]
    return {
        "n": n,
        "N": N,
        "bits": bits,
        "z": _s(r["z"]),
        "X_fit": _s(r["X"]),
        "c": _s(k["c"]),
        "alpha": _s(k["alpha"]),
        "beta": _s(k["beta"]),
        "q0": _s(k["q0"]),
        "q1": _s(k["q1"]),
        "q2": _s(k["q2"]),
        "u": _factors(r["fu"]),
        "v": _factors(r["fv"]),
        "E": _s(r["E"]),
        "ref_x": [_s(v) for v in r["ref_x"]],
        "eps_bits": float(-mp.log(r["E"], 2)),
        "seconds": round(time.time() - t0, 1),
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--bits", type=int, default=53)
    ap.add_argument("--n", default="0-37")
    ap.add_argument("--N", type=int, default=0, help="override the order (0 = Table I)")
    ap.add_argument("--N-offset", type=int, default=0, help="order = Table I's N plus this offset")
    ap.add_argument("--jobs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--out", default="")
    ap.add_argument("--seed", type=int, default=-1,
                    help="start Remez from the alternation points of this fitted order "
                         "(1000 = nearest order with the same N; -1 = Lawson start)")
    ap.add_argument("--keep-better", action="store_true", help="keep an existing fit with more bits")
    args = ap.parse_args()
    lo, _, hi = args.n.partition("-")
    ns = list(range(int(lo), int(hi or lo) + 1))
    out = args.out or os.path.join(COEFF_DIR, f"boys_fit_b{args.bits}.json")
    existing = {}
    if os.path.exists(out):
        with open(out) as fh:
            for rec in json.load(fh)["fits"]:
                existing[rec["n"]] = rec

    def seed_for(n: int, N: int):
        """Alternation points of the nearest fitted order with the same N,
        rescaled by the ratio of the cut-offs."""
        if args.seed < 0:
            return None
        src = existing.get(args.seed) if args.seed != 1000 else None
        if src is None:
            cands = [k for k in existing if existing[k]["N"] == N and k != n and existing[k].get("ref_x")]
            if not cands:
                return None
            src = existing[min(cands, key=lambda k: abs(k - n))]
        mp.mp.dps = 50
        scale = bf.cutoff(n, args.bits) / mp.mpf(src["z"])
        return [mp.nstr(mp.mpf(v) * scale, 40) for v in src["ref_x"]]

    todo = [(n, args.N or table_order(n, args.bits) + args.N_offset, args.bits) for n in ns]
    todo = [(n, N, b, seed_for(n, N)) for n, N, b in todo]
    ctx = mproc.get_context("spawn")
    with ctx.Pool(args.jobs) as pool:
        for rec in pool.imap_unordered(job, todo):
            tag = rec.get("error") or f"eps = {rec['eps_bits']:.3f} bits ({rec['seconds']} s)"
            print(f"n={rec['n']:2d} N={rec['N']:2d} b={rec['bits']}: {tag}", flush=True)
            if "error" not in rec:
                old = existing.get(rec["n"])
                if args.keep_better and old and old["N"] == rec["N"] and old["eps_bits"] > rec["eps_bits"] + 1e-6:
                    continue
                existing[rec["n"]] = rec
                with open(out, "w") as fh:
                    json.dump({"bits": args.bits, "fits": [existing[k] for k in sorted(existing)]}, fh, indent=1)


if __name__ == "__main__":
    main()
