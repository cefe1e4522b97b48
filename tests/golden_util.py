"""Loads the hand-derived worked examples of tests/golden/worked_examples.json
into float32 structure-of-arrays inputs and float64 expected values."""

import json
import math
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
_ENV = {"exp": math.exp, "cos": math.cos, "sin": math.sin, "sqrt": math.sqrt,
        "pi": math.pi, "__builtins__": {}}


def _ev(a):
    return np.array([[float(eval(str(e), _ENV)) for e in row] for row in a], dtype=np.float64)


def _f32(a):
    return np.ascontiguousarray(_ev(a).astype(np.float32))


def _param(v):
    return math.inf if str(v) == "inf" else float(v)


def load_examples():
    with open(os.path.join(HERE, "worked_examples.json")) as f:
        doc = json.load(f)
    out = {}
    for ex in doc["examples"]:
        fld, q = ex["field"], ex["query"]
        out[ex["name"]] = {
            "mean": _f32(fld["mean"]), "quat": _f32(fld["quat"]),
            "logscale": np.log(_ev(fld["scale"])).astype(np.float32),
            "spectrum": _f32(fld["spectrum"]),
            "x": _f32(q["x"]), "n": _f32(q["n"]), "wo": _f32(q["wo"]),
            "albedo": _f32(q["albedo"]) if "albedo" in q else None,
            "mode": 0 if ex["params"]["mode"] == "SUM" else 1,
            "r_max": _param(ex["params"]["r_max"]),
            "cutoff_sigma": _param(ex["params"]["cutoff_sigma"]),
            "expected": _ev(ex["expected"]),
            "cite": ex["cite"],
        }
    grads = {}
    for g in doc["gradients"]:
        grads[g["name"]] = {"example": g["example"], "grad_out": _ev(g["grad_out"]),
                            "expected": {k: _ev(v) for k, v in g["expected"].items()}}
    return out, grads


def load_constants():
    with open(os.path.join(HERE, "paper_constants.json")) as f:
        doc = json.load(f)
    return {k: v["value"] for k, v in doc.items() if not k.startswith("_")}
