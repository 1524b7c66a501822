"""Readers for the text fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _val(v):
    if "," in v:
        return [int(x) for x in v.split(",")]
    try:
        return int(v)
    except ValueError:
        return v


def paper_examples():
    out = {}
    with open(os.path.join(GOLDEN, "paper_examples.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, *kvs = line.split()
            out[name] = {k: _val(v) for k, v in (kv.split("=", 1) for kv in kvs)}
    return out


def comprange():
    dims, comp = [], []
    with open(os.path.join(GOLDEN, "tab_comprange.txt")) as f:
        for line in f:
            s = line.strip()
            if s.startswith("#e"):
                _, qb, e = s.split()
                comp.append((int(qb), int(e)))
            elif s and not s.startswith("#"):
                qb, d = s.split()
                dims.append((int(qb), int(d)))
    return dims, comp
