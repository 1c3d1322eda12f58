"""Reader for tests/golden/closed_forms.txt (hand-derived qdot cases)."""
from __future__ import annotations

import os
from dataclasses import dataclass
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "closed_forms.txt")
_CLS = {"P": 0, "H": 1, "S": 2, "D": 3, "Z": 4}


@dataclass
class Case:
    name: str
    x: np.ndarray
    y: np.ndarray
    eps: float
    block: int
    split: int
    mant: int
    classes: np.ndarray
    z: float


def _eval(expr: str):
    env = {"F": Fraction, "X": Fraction(1) + Fraction(1, 2**20) + Fraction(1, 2**40)}
    env.update(_CLS)
    return eval(expr, {"__builtins__": {}}, env)  # noqa: S307 - trusted fixture file in this repo


def _to_float(v) -> float:
    # float(Fraction) rounds the exact rational once, to nearest-even
    return float(Fraction(v))


def load_cases() -> list[Case]:
    cases = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            f = [p.strip() for p in line.split("|")]
            name, xs, ys, eps, block, split, mant, classes, z = f
            x = np.array([_to_float(v) for v in _eval(xs)], dtype=np.float64)
            y = np.array([_to_float(v) for v in _eval(ys)], dtype=np.float64)
            cases.append(Case(name, x, y, _to_float(_eval(eps)), int(block), int(split), int(mant),
                              np.array(_eval(classes), dtype=np.uint8), _to_float(_eval(z))))
    return cases
