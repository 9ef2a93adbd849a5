"""Reader for the text fixtures under tests/golden/ (values printed in the paper)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name):
    """Parse '[section]' blocks of whitespace-separated numbers; '#' starts a comment."""
    out, cur, rows = {}, None, []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                if cur is not None:
                    out[cur] = np.array(rows, dtype=np.float64)
                cur, rows = line[1:-1], []
            else:
                rows.append([float(x) for x in line.split()])
    if cur is not None:
        out[cur] = np.array(rows, dtype=np.float64)
    return out
