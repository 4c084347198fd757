"""Readers of the fixtures under tests/golden/ (no arithmetic of the method)."""
import math
import os

import numpy as np

import synth

HERE = os.path.join(os.path.dirname(__file__), "golden")
_NS = {"__builtins__": {}, "pi": math.pi, "exp": math.exp, "cos": math.cos, "sqrt": math.sqrt}


def _num(expr):
    return float(eval(expr, _NS))  # fixture expressions: numbers, pi, exp, cos, sqrt


def closed_form_cases():
    """The cases of aev_closed_forms.txt as dicts: name, cite, spec, species,
    coords, expect [(centre, index, value)], zero [(centre, first, last)]."""
    cases, cur = [], None
    for raw in open(os.path.join(HERE, "aev_closed_forms.txt")):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        key, *rest = line.split()
        if key == "case":
            cur = {"name": rest[0], "params": {}, "atoms": [], "expect": [], "zero": []}
        elif key == "cite":
            cur["cite"] = " ".join(rest)
        elif key == "param":
            cur["params"][rest[0]] = [_num(v) for v in rest[1:]]
        elif key == "atom":
            cur["atoms"].append((int(rest[0]), [_num(v) for v in rest[1:4]]))
        elif key == "expect":
            cur["expect"].append((int(rest[0]), int(rest[1]), _num(rest[2])))
        elif key == "zero":
            cur["zero"].append((int(rest[0]), int(rest[1]), int(rest[2])))
        elif key == "end":
            q = cur["params"]
            p = synth.AevParams(2, q["rc_r"][0], q["eta_r"][0], tuple(q["shf_r"]), q["rc_a"][0],
                                q["eta_a"][0], q["zeta"][0], tuple(q["shf_a"]), tuple(q["shf_z"]))
            D = synth.aev_dim(p)
            cur["spec"] = synth.ModelSpec(p, (D, 32, 32, 32, 1), 1, 0.1, (1, 8))
            cur["species"] = np.array([a[0] for a in cur["atoms"]], dtype=np.uint8)
            cur["coords"] = np.array([a[1] for a in cur["atoms"]], dtype=np.float64)
            cases.append(cur)
            cur = None
        else:
            raise ValueError(f"unknown fixture line: {raw!r}")
    return cases


def paper_constants():
    """paper_constants.txt as {key: [value tuples]}."""
    out = {}
    for raw in open(os.path.join(HERE, "paper_constants.txt")):
        line = raw.split("#", 1)[0].split("|", 1)[0].strip()
        if not line:
            continue
        key, *vals = line.split()
        out.setdefault(key, []).append(tuple(float(v) for v in vals))
    return out
