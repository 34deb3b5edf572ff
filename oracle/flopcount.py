"""Algorithmic flop count of the method as the oracle writes it out (test
infrastructure, like the rest of oracle/).

Builds oracle/flopcount.cpp, which compiles the oracle's C source with
`double` replaced by a counting scalar, and runs one RK4 step of a periodic
8^3 block: additions/subtractions and multiplications per interior cell and
stage, divisions, square roots and powers tallied separately.

    python oracle/flopcount.py        # prints one JSON line per order
"""
from __future__ import annotations

import json
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_EXE = os.path.join(_BUILD, "flopcount")


def build() -> str:
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, "flopcount.cpp"), os.path.join(_HERE, "z4c_oracle.c")]
    if not os.path.exists(_EXE) or os.path.getmtime(_EXE) < max(os.path.getmtime(s) for s in srcs):
        subprocess.check_call(["g++", "-std=c++17", "-O1", "-ffp-contract=off", "-fpermissive", "-w", "-o", _EXE,
                               srcs[0]])
    return _EXE


def count(order: int) -> dict:
    out = subprocess.check_output([build(), str(order)], text=True)
    return json.loads(out)


if __name__ == "__main__":
    for o in (2, 4, 6):
        print(json.dumps(count(o)))
