"""Writes the oracle-computed fixtures in this folder.

Run from the repository root: python tests/golden/make_golden.py
It calls only the FP64 oracle (oracle/) and the seeded scene generators, so
every stored value here comes from the oracle, never from the CUDA path.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2101_12408_gb300 import scenes  # noqa: E402

# one backward-Euler step of a moving droplet under gravity (section
# "Discretization"), solved far below any comparison tolerance
DROPLET = dict(n=16, r_cells=4.0, seed=71, v0=[0.2, -0.1, 0.05], spin=0.7, lambda_l=50.0, gravity=[0.0, -9.8, 0.0])
TIGHT = dict(newton_tol=1e-11, cg_rtol=1e-11, max_cg=5000)


def droplet_scene():
    kw = dict(DROPLET)
    kw["v0"] = tuple(kw["v0"])
    kw["gravity"] = tuple(kw["gravity"])
    sc = scenes.droplet(**kw)
    for k, v in TIGHT.items():
        setattr(sc.params, k, v)
    return sc


def droplet_step():
    sc = droplet_scene()
    sim = oracle.OracleSim(sc)
    sim.step()
    rng = np.random.default_rng(0)
    act = np.flatnonzero(sim.grid["m"] > 0)
    nodes = np.sort(rng.choice(act, 24, replace=False))
    parts = np.sort(rng.choice(sc.n_particles, 24, replace=False))
    s = sim.sc
    return {
        "what": "one oracle step of scenes.droplet(**scene) with the solver settings in 'tight'",
        "scene": DROPLET,
        "tight": TIGHT,
        "nodes": nodes.tolist(),
        "vhat": sim.vhat[nodes].tolist(),
        "vhat_absmax": float(np.abs(sim.vhat).max()),
        "particles": parts.tolist(),
        "v": s.v[parts].tolist(),
        "x": s.x[parts].tolist(),
        "v_absmax": float(np.abs(s.v).max()),
        "momentum": np.sum(s.m[:, None] * s.v, 0).tolist(),
        "newton_iters": int(sim.stats["newton"]),
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_droplet_step.json"), "w") as f:
        json.dump(droplet_step(), f, indent=1)
        f.write("\n")
