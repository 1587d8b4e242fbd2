"""Reader for the small text fixtures under tests/golden/."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_blocks(name):
    """Parse '[tag d0 d1 ...]' headers followed by whitespace-separated rows."""
    blocks = {}
    tag, shape, rows = None, None, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s.startswith("["):
                if tag is not None:
                    blocks[tag] = np.array(rows, dtype=np.float64).reshape(shape)
                parts = s.strip("[]").split()
                tag, shape, rows = parts[0], tuple(int(x) for x in parts[1:]), []
                continue
            rows.append([float(x) for x in s.split()])
    if tag is not None:
        blocks[tag] = np.array(rows, dtype=np.float64).reshape(shape + (-1,) if len(shape) == 1 else shape)
    return blocks
