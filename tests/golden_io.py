"""Reader for the text fixtures under tests/golden.

Each fixture line is ``key  v1 [v2 ...]  # citation``; blank lines and lines starting
with ``#`` are ignored.
"""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            body = line.split("#", 1)[0].strip()
            if not body:
                continue
            parts = body.split()
            out[parts[0]] = [float(v) for v in parts[1:]]
    return out


def load_all():
    return {fn.rsplit(".", 1)[0]: load(fn) for fn in sorted(os.listdir(GOLDEN))
            if fn.endswith(".txt")}
