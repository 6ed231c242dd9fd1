"""Reader of tests/golden/paper_values.txt: the values the paper prints (each
line cites the section and test it comes from)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")


def paper_values():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, value = line.split()[:2]
            out[key] = float(value)
    return out


PAPER = paper_values()
