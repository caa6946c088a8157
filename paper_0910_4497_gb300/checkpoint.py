"""Checkpoint of an MD trajectory: positions, velocities, forces, the box, the
step count and the seed of the run in one .npz file, so that a run can stop
and resume.  Plain NumPy I/O on host arrays; TBSystem.checkpoint / restore
move the device state in and out.

The resumed run repeats the continuous one to the mu-search tolerance: the
first step after a restart starts its chemical-potential search without the
previous step's mu as a guess, so mu (and through it the forces) can differ
by the search's stopping tolerance |N(mu) - N_e| <= mu_tol N_e.
"""
import json

import numpy as np

FORMAT = 1


def save(path, pos, vel, F, L, step, seed, params=None, prec=""):
    """Write the state; arrays are copied as float64 (n x 3)."""
    pos, vel, F = (np.ascontiguousarray(np.asarray(x, dtype=np.float64)) for x in (pos, vel, F))
    if not (pos.shape == vel.shape == F.shape and pos.ndim == 2 and pos.shape[1] == 3):
        raise ValueError("pos, vel and F must be n x 3 arrays of the same n")
    np.savez(path, format=np.int64(FORMAT), pos=pos, vel=vel, F=F, L=np.float64(L),
             step=np.int64(step), seed=np.int64(seed),
             params=np.array(json.dumps(params or {}, sort_keys=True)), prec=np.array(prec))


def load(path):
    """Read a state written by save(); returns a dict with the arrays and the
    scalars as Python numbers (params as a dict)."""
    with np.load(path, allow_pickle=False) as d:
        if int(d["format"]) != FORMAT:
            raise ValueError(f"checkpoint format {int(d['format'])}, expected {FORMAT}")
        return {"pos": d["pos"].copy(), "vel": d["vel"].copy(), "F": d["F"].copy(),
                "L": float(d["L"]), "step": int(d["step"]), "seed": int(d["seed"]),
                "params": json.loads(str(d["params"])), "prec": str(d["prec"])}
