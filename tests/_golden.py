"""Reader for the small text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_sections(name):
    """Parse `[section]` blocks of whitespace-separated numbers; '#' starts a comment."""
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("[") and line.endswith("]"):
                cur = line[1:-1]
                out[cur] = []
                continue
            out[cur].append(line.split())
    return out


def worked_example():
    s = read_sections("cfar_worked_example.txt")
    win = {row[0]: [float(v) for v in row[1:]] for row in s["window"]}
    P = np.array([[float(v) for v in r] for r in s["map"]])
    sref = np.array([[float(v) for v in r] for r in s["sref"]])
    det = np.array([[int(v) for v in r] for r in s["det"]], dtype=np.uint8)
    tr_r, tr_c = (int(v) for v in win["train"])
    gd_r, gd_c = (int(v) for v in win["guard"])
    return P, (tr_r, tr_c, gd_r, gd_c, win["pfa"][0]), sref, det
