"""Test helper: make sure libpwave.so is built before the binding loads."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2405_12631_gb300")
LIB = os.path.join(PKG, "libpwave.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    csrc = os.path.join(PKG, "csrc")
    newest = max(os.path.getmtime(os.path.join(csrc, f)) for f in os.listdir(csrc))
    return newest > t


def ensure_built():
    if _stale():
        sys.path.insert(0, PKG)
        try:
            import _build
            _build.build()
        finally:
            sys.path.pop(0)
    return LIB


GOLDEN = os.path.join(ROOT, "tests", "golden")


def golden(name: str):
    """A fixture of tests/golden: '#' lines are the citation; every other
    line is a key followed by integers. Returns {key: [list of int lists]}."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out.setdefault(key, []).append([int(v) for v in vals])
    return out
