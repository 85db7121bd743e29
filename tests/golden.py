"""Parsers for the hand-transcribed paper tables under tests/golden/."""
import math
import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _lines(name):
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                yield line


def _eval(expr, env):
    return float(eval(expr, {"__builtins__": {}}, dict(env, sqrt=math.sqrt)))


def table1(E, g0, g1, g2, c1=0.3, c2=0.2):
    """{row: [c_2, c_1, c_0, c_-1, c_-2]} for the rows that are real at these couplings."""
    env = dict(E=E, g0=g0, g1=g1, g2=g2, c1=c1, c2=c2)
    out = {}
    for line in _lines("table1_thomas_fermi.txt"):
        parts = [p.strip() for p in line.split("|")]
        try:
            out[int(parts[0])] = [_eval(p, env) for p in parts[1:6]]
        except (ValueError, ZeroDivisionError):
            pass                     # a coefficient is not real here
    return out


def table2(E, g0, g1, g2, c1=0.3, c2=0.2):
    """{row: ((F_par, F_perp, A00), flags)}."""
    env = dict(E=E, g0=g0, g1=g1, g2=g2, c1=c1, c2=c2)
    out = {}
    for line in _lines("table2_characteristics.txt"):
        parts = [p.strip() for p in line.split("|")]
        try:
            vals = tuple(_eval(p, env) for p in parts[1:4])
        except (ValueError, ZeroDivisionError):
            continue
        out[int(parts[0])] = (vals, parts[4] if len(parts) > 4 else "")
    return out


def table3(E, g0, g1, g2):
    """{mf: [(a1, b1, a2) for both roots]} from the transcribed Table III."""
    rows, defs = [], {}
    for line in _lines("pade_table3.txt"):
        if "=" in line and "|" not in line:
            k, v = line.split("=", 1)
            defs[k.strip()] = v.strip()
        else:
            rows.append([p.strip() for p in line.split("|")])
    env = dict(E=E, g0=g0, g1=g1, g2=g2)
    for k, v in defs.items():
        env[k] = _eval(v, env)
    out = {}
    for mf, a1e, b1e, a2e in rows:
        roots = []
        for sgn in ("+", "-"):
            e = dict(env)
            e["a1"] = _eval(a1e.replace("pm", sgn), e)
            e["b1"] = _eval(b1e, e)
            e["a2"] = _eval(a2e, e)
            roots.append((e["a1"], e["b1"], e["a2"]))
        out[int(mf)] = roots
    return out
