"""Readers for the paper-transcribed fixtures under tests/golden/."""
import os
import re
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if ln and not ln.startswith("#"):
                yield ln


def generators():
    """{'s1': 3x3, ...}, printed orders, corrected orders, group order."""
    gens, printed, corrected, order = {}, {}, {}, None
    for ln in _lines("generators_s4.txt"):
        key, val = [p.strip() for p in ln.split(":", 1)]
        if key in ("s1", "s2", "s3"):
            gens[key] = np.array([[int(v) for v in row.split()] for row in val.split(";")])
        elif key.startswith("printed_order"):
            printed[key.split()[1]] = int(val)
        elif key.startswith("corrected_order"):
            corrected[key.split()[1]] = int(val)
        elif key == "group_order":
            order = int(val)
    return gens, printed, corrected, order


def _linear_form(expr):
    """'l+m+n' or '-m-n' -> coefficients over (n, m, l)."""
    coef = {"n": 0, "m": 0, "l": 0}
    for sign, var in re.findall(r"([+-]?)\s*([nml])", expr.replace(" ", "")):
        coef[var] += -1 if sign == "-" else 1
    return np.array([coef["n"], coef["m"], coef["l"]])


def power_form():
    """(24, 3, 3) array E with exponent vector = E[t] @ (n, m, l)."""
    out = []
    for ln in _lines("power_form_a3.txt"):
        out.append(np.stack([_linear_form(p) for p in ln.split(";")]))
    return np.stack(out)


def polynomials():
    """{'x': (scale, [(coef, (a,b,c)), ...]), ...} from parametrization.txt."""
    polys, cur = {}, None
    for ln in _lines("parametrization.txt"):
        if ":" in ln:
            name, scale = [p.strip() for p in ln.split(":")]
            cur = polys.setdefault(name, (float(Fraction(scale)), []))
        else:
            c, a, b, d = ln.split()
            cur[1].append((float(c), (int(a), int(b), int(d))))
    return polys


def eval_poly(poly, theta):
    """Evaluate scale * sum coef * exp(2 pi i e . theta); theta (..., 3)."""
    scale, terms = poly
    theta = np.asarray(theta, dtype=np.float64)
    acc = 0j
    for c, e in terms:
        acc = acc + c * np.exp(2j * np.pi * (theta @ np.array(e, dtype=np.float64)))
    return scale * acc


def lemma1():
    d = {}
    for ln in _lines("lemma1_zeros.txt"):
        k, v = [p.strip() for p in ln.split(":", 1)]
        d[k] = v
    return d
