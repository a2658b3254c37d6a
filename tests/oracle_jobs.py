"""Oracle runs for the stated-size parity tests, executed in spawned CPU
processes (test infrastructure only; no GPU call is made here).

Each job builds its inputs from the seeded generators of `workloads` and steps
the FP64 oracle; the GPU side of the test builds the same inputs itself.  The
jobs are top-level functions so that a `spawn` pool can pickle them.
"""
import numpy as np

from paper_2111_04577_gb300 import workloads as wl
from oracle import step as ostep

VISCO_IDX2 = [(0, 0), (0, 1), (1, 1)]
VISCO_IDX3 = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _fields(ref, dim):
    out = {"phi": ref.phi, "u": ref.vel[0], "v": ref.vel[1], "w": ref.vel[2], "p": ref.p}
    if ref.d.visco:
        idx = VISCO_IDX2 if dim == 2 else VISCO_IDX3
        out["theta"] = np.stack([ref.theta[..., a, b] for a, b in idx])
    return out


def run_oracle(spec):
    """spec: dict(workload=Workload, steps=int, vel_seed=int or None, vel_amp=float).
    Returns the oracle's fields after `steps` steps from the seeded state."""
    w = spec["workload"]
    g = w.grid
    phi0 = wl.initial_phi(w)
    vel = None
    if spec.get("vel_seed") is not None:
        vel = wl.random_velocity(g, spec["vel_seed"], spec.get("vel_amp", 0.1))
    ref = ostep.State(g, w.params.as_dict(), phi0, vel0=vel)
    for _ in range(spec["steps"]):
        ref.step()
    return _fields(ref, g.dim)
