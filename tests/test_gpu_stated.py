"""Parity on the configurations' full sizes and stated step counts.

Against the FP64 oracle, element by element (1e-10 relative per field for the
FP64 GPU path; 2e-4 max-abs on phi and 1e-3 relative on velocity and on every
Theta component for the mixed paths):
 - the 2D viscoelastic droplet at its full size (coarse 256x128 / fine
   512x256: 512-point fine and 256-point coarse x lines) for 20 steps from a
   seeded velocity, and for its stated 2000 steps from rest;
 - 3D cases whose x and y lines are the full-size ones (fine 512 and 256,
   coarse 256 and 128: the all-radix-8 and the radix-4-first register
   transforms) with a shallow z, so that the oracle can follow;
 - three problems of the 64-problem batch (coarse 64, 160 and 224: radix-2,
   radix-5 and radix-7 lines) after the stated 500 steps of the batched sweep.
Where the oracle cannot follow (the 3D droplets, 8.4 M and 67 M fine cells, for
their stated 1000 and 500 steps), the mixed paths are compared with the FP64
GPU path, which the cases above pin to the oracle on the same code paths.

The oracle runs in spawned CPU processes, started when this module begins, so
that it proceeds while the GPU works.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

from paper_2111_04577_gb300 import autotune, binding, build, workloads as wl
import oracle_jobs as oj

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-10
PHI_ABS, REL = 2e-4, 1e-3
C5_SAMPLE = (9, 24, 21)   # coarse 64, 160 and 224 in the seeded 64-problem list


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def shallow3d(nx, nz, physics):
    """Coarse nx x nx x nz on the 5 x 5 box of the 3D configurations."""
    w = wl.scaled(wl.config(physics), nx, nz)
    return w


def jobs():
    c2 = wl.config("c2")
    out = {
        "c2_20": dict(workload=c2, steps=20, vel_seed=5, vel_amp=0.1),
        "c2_stated": dict(workload=wl.config("c2"), steps=c2.steps),
        "lines_512": dict(workload=shallow3d(256, 4, "c4"), steps=2, vel_seed=6, vel_amp=0.1),
        "lines_256": dict(workload=shallow3d(128, 4, "c3"), steps=2, vel_seed=7, vel_amp=0.1),
    }
    ws = wl.batch_problems(64, seed=0)
    for b in C5_SAMPLE:
        out[f"c5_{b}"] = dict(workload=ws[b], steps=ws[b].steps)
    return out


@pytest.fixture(scope="module")
def oracle():
    specs = jobs()
    ex = cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn"))
    # the longest first
    order = ["c2_stated", "c5_21", "c5_24", "lines_512", "lines_256", "c2_20", "c5_9"]
    futs = {k: ex.submit(oj.run_oracle, specs[k]) for k in order}
    yield futs
    # a failed test (-x) must not leave the run waiting for oracle work
    procs = list(getattr(ex, "_processes", {}).values())
    ex.shutdown(wait=False, cancel_futures=True)
    for p in procs:
        if p.is_alive():
            p.terminate()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    binding.load()


def gpu_fields(w, prec, steps, vel_seed=None, vel_amp=0.1, tune=False):
    g = w.grid
    s = binding.Solver(g, w.params, prec)
    if tune:
        autotune.apply(s, autotune.tuned(g, w.params, prec, phi0=wl.initial_phi(w).astype(s.dtype)))
    vel = wl.random_velocity(g, vel_seed, vel_amp) if vel_seed is not None else None
    s.load_state(wl.initial_phi(w), vel)
    s.step(steps)
    out = {"phi": s.fine("phi"), "u": s.coarse("u"), "w": s.coarse("w"), "p": s.coarse("p")}
    if g.dim == 3:
        out["v"] = s.coarse("v")
    if w.params.wi > 0 and w.params.beta < 1:
        out["theta"] = s.coarse("theta")
    s.close()
    return out


def check_fp64(gpu, ref, dim):
    names = ["phi", "u", "w", "p"] + (["v"] if dim == 3 else []) + (["theta"] if "theta" in ref else [])
    for n in names:
        if n == "theta":
            for q in range(ref["theta"].shape[0]):
                assert rel(gpu["theta"][q], ref["theta"][q]) < FP64_TOL, (n, q)
        else:
            assert rel(gpu[n], ref[n]) < FP64_TOL, n


def check_mixed(gpu, ref, dim):
    assert np.max(np.abs(gpu["phi"] - ref["phi"])) < PHI_ABS
    for n in ["u", "w"] + (["v"] if dim == 3 else []):
        assert rel(gpu[n], ref[n]) < REL, n
    if "theta" in ref:
        scale = max(np.max(np.abs(ref["theta"])), 1e-300)
        for q in range(ref["theta"].shape[0]):
            assert np.max(np.abs(gpu["theta"][q] - ref["theta"][q])) < REL * scale, q


def test_c2_fullsize_fp64_vs_oracle(oracle):
    """512-point fine and 256-point coarse x lines, 128-row coarse and 256-row
    fine z solves, density ratio 1000 and Oldroyd-B, from a seeded velocity."""
    spec = jobs()["c2_20"]
    gpu = gpu_fields(spec["workload"], binding.PF_FP64, spec["steps"], spec["vel_seed"], spec["vel_amp"])
    check_fp64(gpu, oracle["c2_20"].result(), 2)


@pytest.mark.parametrize("key", ["lines_512", "lines_256"])
def test_3d_fullsize_lines_fp64_vs_oracle(oracle, key):
    """x and y lines of the 3D configurations (fine 512 / coarse 256, and fine
    256 / coarse 128) in FP64 against the oracle, with a shallow z."""
    spec = jobs()[key]
    gpu = gpu_fields(spec["workload"], binding.PF_FP64, spec["steps"], spec["vel_seed"], spec["vel_amp"])
    check_fp64(gpu, oracle[key].result(), 3)


@pytest.mark.slow
def test_c2_stated_steps_vs_oracle(oracle):
    """The 2D viscoelastic droplet as stated: full size, from rest, 2000 steps;
    FP64 at 1e-10, both mixed paths at the mixed tolerances."""
    w = wl.config("c2")
    res = {p: gpu_fields(w, p, w.steps) for p in (binding.PF_FP64, binding.PF_MIXED, binding.PF_MIXED_Z64,
                                                   binding.PF_MIXED_Z2F)}
    ref = oracle["c2_stated"].result()
    check_fp64(res[binding.PF_FP64], ref, 2)
    check_mixed(res[binding.PF_MIXED], ref, 2)
    check_mixed(res[binding.PF_MIXED_Z64], ref, 2)
    check_mixed(res[binding.PF_MIXED_Z2F], ref, 2)


@pytest.mark.slow
@pytest.mark.parametrize("cfg", ["c3", "c4"])
def test_3d_stated_steps_mixed_vs_fp64(cfg):
    """The 3D droplets as stated (full size, from rest; 1000 steps of the
    Newtonian droplet, 500 of the Oldroyd-B one), the mixed paths in the
    bench's launch configuration against the FP64 GPU path."""
    w = wl.config(cfg)
    d = gpu_fields(w, binding.PF_FP64, w.steps)
    for prec in (binding.PF_MIXED, binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F):
        m = gpu_fields(w, prec, w.steps, tune=prec == binding.PF_MIXED)
        check_mixed(m, d, 3)
        if prec == binding.PF_MIXED:
            assert np.max(np.abs(d["phi"])) < 1.5  # the run stayed a droplet


@pytest.mark.slow
def test_c5_batch_stated_steps(oracle):
    """The 64 uneven problems of the batched sweep, stated sizes (coarse 64 to
    256) and steps (500): FP64 batch against the oracle on three sampled
    problems at 1e-10, and every problem of the mixed batch against the FP64
    batch at the mixed tolerances."""
    ws = wl.batch_problems(64, seed=0)
    res = {}
    for prec in (binding.PF_FP64, binding.PF_MIXED):
        bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], prec)
        for b, w in enumerate(ws):
            bt.set(b, "phi", wl.initial_phi(w))
        bt.step(ws[0].steps)
        res[prec] = []
        for b, w in enumerate(ws):
            f = {n: bt.get(b, n).astype(np.float64) for n in ("phi", "u", "w", "p")}
            if w.params.wi > 0:
                f["theta"] = bt.get(b, "theta").astype(np.float64)
            res[prec].append(f)
        bt.close()
    for b in C5_SAMPLE:
        ref = oracle[f"c5_{b}"].result()
        gpu = dict(res[binding.PF_FP64][b])
        g = ws[b].grid
        gpu["phi"] = gpu["phi"].reshape(g.fine_shape)
        for n in ("u", "p"):
            gpu[n] = gpu[n].reshape(g.coarse_shape)
        gpu["w"] = gpu["w"].reshape((g.nz + 1, g.ny, g.nx))
        if "theta" in gpu:
            gpu["theta"] = gpu["theta"].reshape((3,) + g.coarse_shape)
        check_fp64(gpu, ref, 2)
    for b, w in enumerate(ws):
        m, d = res[binding.PF_MIXED][b], res[binding.PF_FP64][b]
        assert np.max(np.abs(m["phi"] - d["phi"])) < PHI_ABS, b
        for n in ("u", "w"):
            assert rel(m[n], d[n]) < REL, (b, n)
        if "theta" in d:
            scale = max(np.max(np.abs(d["theta"])), 1e-300)
            assert np.max(np.abs(m["theta"] - d["theta"])) < REL * scale, b
