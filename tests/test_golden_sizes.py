"""The paper's printed problem sizes (Sec. 4, Test Problems 2 and 3) are reproduced by the
geometry descriptors the oracle and the GPU path both consume."""
import json
import os

import numpy as np

import synth
from oracle import proj as P

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_problem_sizes.json")


def test_paper_problem_sizes():
    spec = json.load(open(GOLDEN))
    for key in ("test_problem_2", "test_problem_3"):
        t = spec[key]
        nd = t["m"] // t["views"]
        if t["kind"] == "parallel2d":
            g = synth.parallel2d(t["N"], t["views"], nd)
        else:
            g = synth.fanflat2d(t["N"], t["views"], nd, 2.0 * t["N"], 3.0 * t["N"])
        assert g.m == t["m"] and g.n == t["n"]
    g = synth.parallel2d(128, 50, 128)
    y = P.forward(g, np.ones(g.n))
    assert y.size == 6400
