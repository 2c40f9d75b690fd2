"""Writes tests/golden/oracle_small.json: small oracle solutions kept as a
regression fixture (it guards the oracle against later changes and against
platform differences).  Calls only the oracle and the seeded generators."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402


def cases():
    out = {}
    bands, B = synth.random_tri_case(N=8, M=3, seed=0)
    out["random_tri_N8_M3_seed0"] = (bands, B)
    bands, B = synth.random_penta_case(N=6, M=2, seed=0)
    out["random_penta_N6_M2_seed0"] = (bands, B)
    rng = np.random.default_rng(0)
    out["clamped_penta_N8_M2"] = (synth.clamped_hyperdiffusion_bands(8, 0.1), rng.standard_normal((8, 2)))
    out["spline_N5_M2"] = (synth.spline_bands(5), rng.uniform(-1, 1, (5, 2)))
    return out


def main():
    doc = {}
    for name, (bands, B) in cases().items():
        X = oracle.solve(bands, B)
        doc[name] = {"bands": bands.tolist(), "B": B.tolist(), "X": X.tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small.json")
    with open(path, "w") as f:
        json.dump(doc, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
