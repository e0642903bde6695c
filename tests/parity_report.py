"""Markdown table of the parity record that the GPU tests write.

    FACERT_PARITY_LOG=<log.jsonl> python -m pytest tests -m gpu
    python -m tests.parity_report <log.jsonl>

One row per checked result: its kind, size, maximum and 99.99th-percentile
error against the FP64 oracle (relative per pixel for images; per component
relative to max(|o|, 1e-3 * group max) for gradients), and for gradients the
components that passed only through a named exception (tests/parity.py).
"""
from __future__ import annotations

import json
import sys


def rows(path):
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


GROUPS = ["alpha", "beta", "delta", "cspec", "pose", "lights"]


def table(rs):
    """Images and values one row each; a gradient result one row with the
    strict maximum error of each parameter group."""
    out = ["| result | kind | n | max error | 99.99th pct | tolerance | notes |", "|---|---|---|---|---|---|---|"]
    grads = {}
    order = []
    for r in rs:
        k = r["kind"]
        if k == "grad":
            if r["what"] not in grads:
                grads[r["what"]] = []
                order.append(("grad", r["what"]))
            grads[r["what"]].append(r)
        elif k in ("image", "value", "vertex"):
            order.append((k, r))
    for k, r in order:
        if k == "image":
            out.append(f"| {r['what']} | image | {r['n']} | {r['max']:.1e} | {r['p9999']:.1e} | "
                       f"1e-4 per pixel | {r['flipped']} flipped pixels ({r['allowed']} allowed) |")
        elif k == "value":
            out.append(f"| {r['what']} | value | {r['n']} | {r['max']:.1e} | {r['p9999']:.1e} | {r['tol']:.1e} | |")
        elif k == "vertex":
            out.append(f"| {r['what']} | per-vertex dX | {r['n']} | {r['max']:.1e} | {r['p9999']:.1e} | "
                       f"1e-3, 1 % floor | {r['n_mass_only']} entries by 1e-4 x mass |")
        else:
            rows = grads[r]
            n = sum(g["n"] for g in rows)
            per = ", ".join(f"{g['group']} {g['max']:.1e}" if not g.get("zero") else f"{g['group']} 0"
                            for g in rows)
            worst = max(g["max"] for g in rows if not g.get("zero")) if any(not g.get("zero") for g in rows) else 0
            p = max(g["p9999"] for g in rows if not g.get("zero")) if any(not g.get("zero") for g in rows) else 0
            named = sum(g.get("n_named", 0) for g in rows)
            only = sum(len(g["mass_only"]) for g in rows)
            kap = [g["kappa"] for g in rows if g.get("kappa")]
            tol = "1e-3 strict" + (f"; named {kap[0]:g} x mass" if kap else "")
            note = per + (f"; {named} named, {only} passed only by name" if named else "")
            out.append(f"| {r} | gradient | {n} | {worst:.1e} | {p:.1e} | {tol} | {note} |")
    return "\n".join(out)


if __name__ == "__main__":
    print(table([r for r in rows(sys.argv[1]) if r["kind"] != "same-library"]))
