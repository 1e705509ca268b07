"""Reader for the small text fixtures under tests/golden/."""
from fractions import Fraction
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


class Fixture:
    pass


def load(name):
    f = Fixture()
    f.edges, f.attrs, f.ps_rows, f.pa_rows, f.kv = [], [], {}, {}, {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] in ("n_u", "n_v", "n_a"):
                setattr(f, tok[0], int(tok[1]))
            elif tok[0] == "edge":
                f.edges.append((int(tok[1]), int(tok[2]), float(tok[3])))
            elif tok[0] == "attr":
                f.attrs.append((int(tok[1]), int(tok[2]), float(tok[3])))
            elif tok[0] in ("ps_row", "pa_row"):
                row = [Fraction(t) for t in tok[2:]]
                getattr(f, tok[0] + "s")[int(tok[1])] = row
            else:                       # any other key: its values as fractions
                f.kv[tok[0]] = [Fraction(t) for t in tok[1:]]
    e = np.array(f.edges) if f.edges else np.zeros((0, 3))
    a = np.array(f.attrs) if f.attrs else np.zeros((0, 3))
    f.e_u, f.e_v, f.e_w = e[:, 0].astype(np.uint32), e[:, 1].astype(np.uint32), e[:, 2]
    f.ea_u, f.ea_a, f.ea_w = a[:, 0].astype(np.uint32), a[:, 1].astype(np.uint32), a[:, 2]
    return f
