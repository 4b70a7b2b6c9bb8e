"""Readers for the worked examples in this folder.  Each fixture is a text
file of values derived by hand from the paper's equations (the citation and
the derivation are in the file); none comes from the oracle or the CUDA
path."""
from __future__ import annotations

import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def _lines(name: str) -> list[str]:
    out = []
    for raw in open(os.path.join(HERE, name)):
        line = raw.split("#", 1)[0].strip()
        if line:
            out.append(line)
    return out


def tanimoto_cases() -> list[tuple[np.ndarray, np.ndarray, float]]:
    """(x, y, Tan(x, y)) of tanimoto_worked.txt."""
    cases = []
    for line in _lines("tanimoto_worked.txt"):
        x, y, t = (part.strip() for part in line.split(";"))
        cases.append((np.array(x.split(), float), np.array(y.split(), float), float(t)))
    return cases


def _matrices(lines: list[str]) -> list[tuple[str, object]]:
    """Sections 'NAME' followed by rows of numbers, or 'NAME value' on one line."""
    items, i = [], 0
    while i < len(lines):
        head = lines[i].split()
        i += 1
        if len(head) == 2:
            items.append((head[0], float(head[1])))
            continue
        rows = []
        while i < len(lines) and _numeric(lines[i]):
            rows.append([float(v) for v in lines[i].split()])
            i += 1
        items.append((head[0], np.array(rows)))
    return items


def _numeric(line: str) -> bool:
    try:
        [float(v) for v in line.split()]
        return True
    except ValueError:
        return False


def step_2x3() -> dict:
    """The worked iteration: inputs W, P, C and, per alpha, the expected
    W', h and (alpha = 1 only) P', C'."""
    items = _matrices(_lines("step_2x3_identity_priors.txt"))
    out: dict = {"cases": []}
    cur = None
    for name, val in items:
        if name in ("W", "P", "C") and cur is None:
            out[name] = val
        elif name == "alpha":
            cur = {"alpha": val}
            out["cases"].append(cur)
        else:
            cur[name.rstrip("'")] = val
    return out


def pearson_3x3() -> tuple[np.ndarray, np.ndarray]:
    d = dict(_matrices(_lines("pearson_3x3.txt")))
    return d["X"], d["R"]
