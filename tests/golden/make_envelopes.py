"""Write tests/golden/envelopes.json: the oracle's log M (Eq. 45, Nelder-Mead
from the Dirichlet kernel plus extra starts) for the parameter points that the
GPU tests and bench.py replay.  Calls only oracle/.

    python tests/golden/make_envelopes.py
"""
import json
import os
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402


def points():
    out = []
    # K = 16, beta' = 20, C3/C2 = 75 (acceptance ~1e-2), both proposals
    for prop in (O.UNIFORM, O.PAPER):
        out.append((16, 1.0, 20.0, 75.0, prop))
    # K = 32, beta' = geomspace(20, 60, 8), beta' C3/C2 = 9000
    for b in np.geomspace(20.0, 60.0, 8):
        for prop in (O.UNIFORM, O.PAPER):
            out.append((32, 1.0, float(b), 9000.0 / float(b), prop))
    return out


def key(K, E0, bp, r, prop):
    return "K%d_E%.17g_b%.17g_r%.17g_p%d" % (K, E0, bp, r, prop)


def main():
    def one(args):
        K, E0, bp, r, prop = args
        pt = O.make_point(K, E0, bp, r, prop)
        return key(*args), {"K": K, "E0": E0, "beta_p": bp, "r": r, "proposal": prop,
                            "logM": O.log_M(pt, 4), "alpha": pt.alpha}

    with ThreadPoolExecutor(max_workers=2) as ex:
        res = dict(ex.map(one, points()))
    with open(os.path.join(HERE, "envelopes.json"), "w") as f:
        json.dump({"_source": "oracle.log_M (Nelder-Mead, Eq. 45), written by make_envelopes.py",
                   "points": res}, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
