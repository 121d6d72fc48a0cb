"""Small text fixtures of values the paper prints, each with its citation."""
import os

_HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden(name):
    """Parse ``key = value  # citation`` lines into a dict of floats."""
    out = {}
    with open(os.path.join(_HERE, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = float(v)
    return out
