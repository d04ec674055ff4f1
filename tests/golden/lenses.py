"""Loader for the printed lens configurations in paper_lenses.txt."""
from pathlib import Path

KEYS = ("x0", "y0", "q", "phi", "theta_e", "gamma", "g1", "g2")


def paper_lenses() -> dict:
    out = {}
    for line in (Path(__file__).parent / "paper_lenses.txt").read_text().splitlines():
        if not line.strip() or line.startswith("#"):
            continue
        name, *vals = line.split()
        out[name] = dict(zip(KEYS, map(float, vals)))
    return out
