"""Reader for the values printed in the paper (tests/golden/paper_values.txt)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_values.txt")


def load() -> dict:
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = float(v)
    return out
