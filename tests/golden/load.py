"""Reader for the small text fixtures in tests/golden/ (key value... lines,
'#' comments)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def read(name):
    rows = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            rows.setdefault(key, []).append(vals)
    return rows
