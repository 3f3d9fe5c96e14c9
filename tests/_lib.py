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
