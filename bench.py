"""Benchmark of the dual-resolution phase-field step on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (one GPU): the 3D viscoelastic droplet -- coarse 256x256x128 flow mesh,
fine 512x512x256 phase-field mesh, Oldroyd-B droplet (Wi = 2, beta = 0.3),
density ratio 1000, viscosity ratio 20, 90 deg contact angle, mixed precision,
seeded synthetic initial state.  Metric: fine-mesh cell-steps/s of the whole
time step (CH + restriction + NS + polymer), inputs resident in HBM; every
field is larger than L2, so no flush is needed.

Also reported: the same GPU's FP64 path and single-resolution paths (CSR: phi
on the coarse mesh; RSR: every field on the fine mesh), the mixed path's phi
error against the FP64 path, the dominant kernel against the measured HBM
copy bandwidth, the CPU oracle on a bounded sample, an end-to-end figure
through the C ABI with host buffers, and SM clocks sampled during the run.

With torchrun (N > 1) every rank advances its own independent replica
(weak scaling); the timed region is bracketed by barriers and the max over
ranks is taken.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fine-mesh cell-steps/s (dual-res 3D) vs FP64 GPU path at stated error; HBM roof %"
UNIT = "fine cell-steps/s"


def rank_env(env=os.environ):
    """(world, rank, local_rank) as torchrun exports them; 1 process by default."""
    return int(env.get("WORLD_SIZE", "1")), int(env.get("RANK", "0")), int(env.get("LOCAL_RANK", "0"))


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over all ranks (the slowest replica sets the job's time)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(cells, steps, world, elapsed):
    """Whole-job throughput of `world` independent replicas, each advancing `cells`
    fine cells by `steps` steps, over the max-over-ranks elapsed time."""
    return cells * steps * world / elapsed


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of each kernel in
# one step, in bytes per fine cell, from one ncu capture of the 512x512x64 fine
# case of this workload's physics; every pass moves data in proportion to the
# cells, so a full launch scales by its fine cells.  Each entry keeps the
# sha256 of the source files that define the kernel when the counters were
# taken: once a kernel changes its traffic reads null until it is measured again.
TRAFFIC = {
    "ch_rhs": (23.110, ["paper_2111_04577_gb300/csrc/ch_march.cuh", "paper_2111_04577_gb300/csrc/ch.cuh"], "53d3dddcf51ae53d"),
    "ns_rhs": (17.577, ["paper_2111_04577_gb300/csrc/ns_march.cuh", "paper_2111_04577_gb300/csrc/ns_rhs.cuh", "paper_2111_04577_gb300/csrc/ns.cuh"], "e0327193f48bff5a"),
    "polymer_stage2": (13.902, ["paper_2111_04577_gb300/csrc/polymer.cuh"], "9cad53f3b20ccdc3"),
    "polymer_stage1": (7.259, ["paper_2111_04577_gb300/csrc/polymer.cuh"], "9cad53f3b20ccdc3"),
    "fft_y_fine": (10.578, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
    "fft_y_coarse": (4.041, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
    "ch_G_restrict": (6.739, ["paper_2111_04577_gb300/csrc/ch_march.cuh", "paper_2111_04577_gb300/csrc/ch.cuh"], "53d3dddcf51ae53d"),
    "ch_ifftx_finish": (25.825, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
    "zsolve_pair": (4.675, ["paper_2111_04577_gb300/csrc/zsolve_seg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh"], "e81cbcc2b80e6a28"),
    "zsolve": (2.062, ["paper_2111_04577_gb300/csrc/zsolve_seg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh"], "e81cbcc2b80e6a28"),
    "irfft_x_coarse": (4.987, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
    "rfft_x_fine": (5.013, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
    "rfft_x_coarse": (1.486, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
    "correct": (2.485, ["paper_2111_04577_gb300/csrc/ns.cuh"], "733228b8845497aa"),
    "div_rfft_x_coarse": (1.486, ["paper_2111_04577_gb300/csrc/fft_reg.cuh", "paper_2111_04577_gb300/csrc/spectral.cuh", "paper_2111_04577_gb300/csrc/fft.cuh"], "d0c7ac2200da19dd"),
}


def _sha(paths):
    import hashlib
    h = hashlib.sha256()
    for q in paths:
        with open(os.path.join(ROOT, q), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel, fine_cells):
    ent = TRAFFIC.get(kernel)
    if not ent:
        return None
    per_cell, srcs, sha = ent
    try:
        if _sha(srcs) != sha:
            return None
    except OSError:
        return None
    return per_cell * fine_cells


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def alg_bytes(grid, esize, visco=True, compensated=None):
    """Algorithmic bytes per step of each kernel (all its launches in one step).

    Minimal traffic of the operation: each input read once, each output
    written once (no halos, no re-reads).  FP32 contexts keep phi as a
    compensated pair (value and rounding remainder): the CH right side reads
    both remainders, the finishing transform reads both and writes one."""
    if compensated is None:
        compensated = esize == 4
    nzf, nyf, nxf = grid.fine_shape
    nf = nzf * nyf * nxf
    nz, ny, nx = grid.coarse_shape
    nc = nz * ny * nx
    ncw = (nz + 1) * ny * nx
    d3 = grid.dim == 3
    E = esize
    sf = (nxf // 2 + 1) * nyf * nzf          # fine spectral complex elements
    sc = (nx // 2 + 1) * ny * nz             # coarse spectral complex elements (per component)
    nvel = 3 if d3 else 2
    ncomp = 6 if d3 else 3
    nsolve = nvel + 1                        # velocity components + pressure
    b = {
        "ch_rhs": 3 * E * nf + 2 * nvel * E * nc + (2 * E * nf if compensated else 0),
        "rfft_x_fine": E * nf + 2 * E * sf,
        "fft_y_fine": 2 * 2 * (2 * E * sf) if d3 else 0,
        "zsolve_pair": 2 * 2 * E * sf,
        "ch_ifftx_finish": 2 * E * sf + 3 * E * nf + (3 * E * nf if compensated else 0),
        "ch_G_restrict": E * nf + (11 if d3 else 7) * E * nc,
        "ns_rhs": (2 * (nvel + 1) + (2 * ncomp if visco else 0) + (11 if d3 else 7) + nvel) * E * nc,
        "rfft_x_coarse": nvel * (E * nc + 2 * E * sc),
        "div_rfft_x_coarse": nvel * E * nc + 2 * E * sc,  # reads u~, v~, w~: the Poisson right side formed in place
        "fft_y_coarse": (2 * nsolve * 2 * (2 * E * sc)) if d3 else 0,
        "zsolve": nsolve * 2 * (2 * E * sc),
        "zero_mode": 0,
        # the velocity solves' epilogue adds u* = 2 u^n - u^{n-1} back to the increment
        "irfft_x_coarse": nsolve * (2 * E * sc + E * nc) + nvel * 2 * E * nc,
        "correct": (2 * nvel + 3) * E * nc,
        "polymer_stage1": (2 * ncomp + nvel) * E * nc,
        "polymer_stage2": (4 * ncomp + nvel + 1) * E * nc,
    }
    return b


def clocks_start():
    f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
    try:
        p = subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "50"], stdout=f, stderr=subprocess.DEVNULL)
    except Exception:
        return None, f.name
    return p, f.name


def clocks_stop(p, path, gpu_index=0):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except Exception:
        p.kill()
    sm, mx, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
    finally:
        try:
            os.unlink(path)
        except OSError:
            pass
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def workload(name="c4"):
    from paper_2111_04577_gb300 import workloads as wl
    return wl.config(name)


def cpu_sample(w, steps, nx=64):
    """Time the FP64 oracle on the workload's physics at a reduced resolution."""
    from paper_2111_04577_gb300 import workloads as wl
    from oracle import step as ostep
    ws = wl.scaled(w, nx, nx // 2)
    phi0 = wl.initial_phi(ws)
    st = ostep.State(ws.grid, ws.params.as_dict(), phi0)
    st.step()  # warm caches / FFT plans
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(steps):
        st.step()
    dt, cpu = time.perf_counter() - t0, time.process_time() - c0
    cells = ws.grid.fine_cells()
    # cores actually used: the process's CPU time over the wall time of the sample
    return {"value": cells * steps / dt, "unit": UNIT, "cores": round(cpu / dt, 1), "kind": "oracle",
            "sample": f"FP64 NumPy/SciPy oracle, same physics at coarse {nx}x{nx}x{nx // 2} / fine "
                      f"{2 * nx}x{2 * nx}x{nx}, {steps} steps, {dt:.1f} s wall, {cpu:.1f} s CPU "
                      f"({os.cpu_count()} host cores)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.config)
    steps, warm = args.steps, args.warmup
    from paper_2111_04577_gb300 import workloads as wl
    from oracle import step as ostep
    nx = 48
    ws = wl.scaled(w, nx, nx // 2)
    st = ostep.State(ws.grid, ws.params.as_dict(), wl.initial_phi(ws))
    for _ in range(warm):
        st.step()
    t0, c0 = time.perf_counter(), time.process_time()
    for _ in range(steps):
        st.step()
    dt, cpu = time.perf_counter() - t0, time.process_time() - c0
    val = ws.grid.fine_cells() * steps / dt
    sample = (f"FP64 NumPy/SciPy oracle, workload physics at coarse {nx}x{nx}x{nx // 2} / fine "
              f"{2 * nx}x{2 * nx}x{nx}, one oracle time step per step")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": dt / steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name + f" (sampled at {nx}x{nx}x{nx // 2})", "precision": "fp64"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": round(cpu / dt, 1), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(solver, stream, steps):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    solver.step(steps)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1e3


def side_path(w, grid, precision, steps, warm, stream):
    """Cell-steps/s of another configuration of the same physics."""
    import gc
    import torch
    from paper_2111_04577_gb300 import binding, workloads as wl
    s = binding.Solver(grid, w.params, precision, stream=stream.cuda_stream)
    ww = wl.Workload(w.name, grid, w.params, w.steps, w.R0, w.seed, w.amp)
    s.load_state(wl.initial_phi(ww).astype(s.dtype))
    s.step(warm)
    t = time_steps(s, stream, steps)
    s.close()
    del s
    gc.collect()
    torch.cuda.synchronize()
    return grid.fine_cells() * steps / t, t / steps * 1e3


def gradients_leg(w, stream, nx=128, steps=10):
    """Cost of the two gradient paths on the workload's physics at coarse
    nx x nx x nx/2: pf_tangent (dJ/dWi through the whole coupled step, FP64
    values and derivatives) and pf_adjoint (reverse sweep of the CH step,
    velocity fixed, mixed), against the plain FP64 and mixed steps.  Wall
    clock around each call (synchronising): the tangent's time includes the
    copy of the state into its derivative-carrying buffers."""
    import gc
    import time
    import torch
    from paper_2111_04577_gb300 import binding, workloads as wl
    ww = wl.scaled(w, nx, nx // 2)
    g = ww.grid
    out = {"grid": f"coarse {g.nx}x{g.ny}x{g.nz} / fine {2 * g.nx}x{2 * g.ny}x{2 * g.nz}", "steps": steps}
    s = binding.Solver(g, ww.params, binding.PF_FP64, stream=stream.cuda_stream)
    s.load_state(wl.initial_phi(ww))
    s.step(2)
    s.tangent(2, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, dJ = s.tangent(steps, binding.PF_PARAM_WI, binding.PF_OBJ_WETTED)
    t_tan = time.perf_counter() - t0
    t64 = time_steps(s, stream, steps)
    out["tangent_wi"] = {"ms_per_step": t_tan / steps * 1e3, "fp64_ms_per_step": t64 / steps * 1e3,
                         "ratio": t_tan / t64, "J": J, "dJ_dWi": dJ}
    s.close()
    del s
    s = binding.Solver(g, ww.params, binding.PF_MIXED, stream=stream.cuda_stream)
    s.load_state(wl.initial_phi(ww).astype(s.dtype))
    s.adjoint(steps, 5, binding.PF_OBJ_WETTED, want_phi=True)  # warm-up (allocates the checkpoints)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.adjoint(steps, 5, binding.PF_OBJ_WETTED, want_phi=True)
    t_adj = time.perf_counter() - t0
    s.load_state(wl.initial_phi(ww).astype(s.dtype))
    t0 = time.perf_counter()
    s.adjoint(steps, 5, binding.PF_OBJ_WETTED, want_phi=False)
    t_adj_nophi = time.perf_counter() - t0
    s.load_state(wl.initial_phi(ww).astype(s.dtype))
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    s.step(2, binding.PF_STEP_CH_ONLY)
    a.record(stream)
    s.step(steps, binding.PF_STEP_CH_ONLY)
    b.record(stream)
    b.synchronize()
    t_ch = a.elapsed_time(b) / 1e3
    out["coupled_adjoint"] = coupled_adjoint_leg(stream)
    out["ch_adjoint"] = {"ms_per_step": t_adj / steps * 1e3, "ch_step_ms": t_ch / steps * 1e3,
                         "ratio": t_adj / t_ch, "ckpt_every": 5,
                         "ms_per_step_without_dphi0_to_host": t_adj_nophi / steps * 1e3,
                         "ratio_without_dphi0_to_host": t_adj_nophi / t_ch}
    s.close()
    del s
    gc.collect()
    torch.cuda.synchronize()
    return out


def coupled_adjoint_leg(stream, problem=8, steps=500, ckpt=50):
    """The reverse sweep through the whole coupled 2D step (pf_adjoint_ex) on
    one problem of the 64-problem sweep (coarse 128 x 64, its contact angle and
    Wi), mixed precision, over the stated 500 steps with checkpoints every 50:
    dJ/dphi0, dJ/dtheta, dJ/dM and dJ/dWi of the final wetted length in one
    sweep, against the forward steps alone."""
    import time
    import torch
    from paper_2111_04577_gb300 import binding, workloads as wl
    w = wl.batch_problems(64, seed=0)[problem]
    s = binding.Solver(w.grid, w.params, binding.PF_MIXED, stream=stream.cuda_stream)
    phi0 = wl.initial_phi(w)
    s.load_state(phi0)
    s.adjoint_coupled(10, 5, binding.PF_OBJ_WETTED)  # warm-up (allocations, graphs)
    s.load_state(phi0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, dth, dm, dwi, dphi = s.adjoint_coupled(steps, ckpt, binding.PF_OBJ_WETTED)
    t_adj = time.perf_counter() - t0
    s.load_state(phi0)
    t_fwd = time_steps(s, stream, steps)
    s.close()
    return {"grid": f"coarse {w.grid.nx}x{w.grid.nz} / fine {2 * w.grid.nx}x{2 * w.grid.nz} (2D)",
            "theta_deg": w.params.theta_bot_deg, "wi": w.params.wi, "steps": steps, "ckpt_every": ckpt,
            "precision": "mixed", "ms_per_step": t_adj / steps * 1e3, "forward_ms_per_step": t_fwd / steps * 1e3,
            "ratio": t_adj / t_fwd, "J": J, "dJ_dtheta_per_deg": dth, "dJ_dM": dm, "dJ_dWi": dwi,
            "dJ_dphi0_norm": float(np.sqrt(np.sum(np.asarray(dphi, dtype=np.float64) ** 2)))}


def accuracy_leg(stream, steps=200):
    """Section 4.1's comparison on the 3D Newtonian droplet (coarse 128^2 x 64,
    mixed): dual resolution (DR), single resolution with phi on the coarse
    mesh (CSR) and with every field on the fine mesh (RSR), from the same
    droplet, after `steps` steps of the same dt.  RSR is the reference: DR's phi
    is compared on the fine mesh, CSR's against RSR's phi averaged over each
    coarse cell; velocities on the coarse faces against RSR's face velocities
    averaged over the fine faces that tile each coarse face."""
    import gc
    import torch
    from paper_2111_04577_gb300 import binding, workloads as wl
    w = wl.config("c3")
    g = w.grid
    grids = {"dr": g, "csr": wl.Grid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, 0),
             "rsr": wl.Grid(2 * g.nx, 2 * g.ny, 2 * g.nz, g.lx, g.ly, g.lz, 0)}
    out = {}
    for name, gg in grids.items():
        ww = wl.Workload(w.name, gg, w.params, w.steps, w.R0, w.seed, 0.0)  # no seeded noise: one droplet
        s = binding.Solver(gg, w.params, binding.PF_MIXED, stream=stream.cuda_stream)
        s.load_state(wl.initial_phi(ww).astype(s.dtype))
        s.step(steps)
        out[name] = {"phi": s.fine("phi"), "u": s.coarse("u"), "v": s.coarse("v"), "w": s.coarse("w")}
        s.close()
        del s
        gc.collect()
        torch.cuda.synchronize()
    r = out["rsr"]
    nz, ny, nx = g.coarse_shape
    phi_c = r["phi"].reshape(nz, 2, ny, 2, nx, 2).mean(axis=(1, 3, 5))
    u_c = r["u"][:, :, 0::2].reshape(nz, 2, ny, 2, nx).mean(axis=(1, 3))
    v_c = r["v"][:, 0::2, :].reshape(nz, 2, ny, nx, 2).mean(axis=(1, 4))
    w_c = r["w"][0::2].reshape(nz + 1, ny, 2, nx, 2).mean(axis=(2, 4))

    def rel(a, b):
        return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))

    res = {"steps": steps, "time": steps * w.params.dt, "grid": f"coarse {g.nx}x{g.ny}x{g.nz} / fine 2x",
           "reference": "RSR (every field on the fine mesh)"}
    for name in ("dr", "csr"):
        o = out[name]
        dphi = o["phi"] - (r["phi"] if name == "dr" else phi_c)
        res[name] = {"phi_maxabs": float(np.max(np.abs(dphi))),
                     "phi_rms": float(np.sqrt(np.mean(dphi ** 2))),
                     "u_rel": rel(o["u"], u_c), "v_rel": rel(o["v"], v_c), "w_rel": rel(o["w"], w_c)}
    return res


def paper_case_leg(stream, steps=5, warm=2):
    """Section 4.5's performance case at its size: two coalescing drops on a
    180 deg wall in a 6^3 box, dual resolution 384^3 (phase field 768^3)
    against single resolution 768^3, Newtonian and Oldroyd-B (Wi = 10,
    beta = 0.1), mixed precision, built-in launch shapes.  Time per step of
    each, and the ratio the paper reports (about 2 Newtonian, above 2
    viscoelastic, on 256-2304 CPU cores)."""
    import gc
    import torch
    from paper_2111_04577_gb300 import binding, workloads as wl
    res = {"box": "6 x 6 x 6, periodic x, y; walls z (180 / 90 deg)", "steps": steps}
    phi = None
    for visco in (False, True):
        key = "viscoelastic" if visco else "newtonian"
        res[key] = {}
        for dual, n in ((1, 384), (0, 768)):
            w = wl.config("e9", dual=dual, visco=visco, n=n)
            if phi is None:
                phi = wl.drops_phi(w, np.float32)  # the same 768^3 field for both meshes
            try:
                s = binding.Solver(w.grid, w.params, binding.PF_MIXED, stream=stream.cuda_stream)
            except binding.PFError as e:
                res[key]["dr" if dual else "sr"] = {"unavailable": str(e)}
                continue
            s.load_state(phi)
            s.step(warm)
            t = time_steps(s, stream, steps)
            s.close()
            del s
            gc.collect()
            torch.cuda.synchronize()
            res[key]["dr" if dual else "sr"] = {"grid": f"{n}^3" + (" (phase field 768^3)" if dual else ""),
                                                "ms_per_step": t / steps * 1e3,
                                                "fine_cell_steps_per_s": 768 ** 3 * steps / t}
        if "ms_per_step" in res[key].get("dr", {}) and "ms_per_step" in res[key].get("sr", {}):
            res[key]["sr_over_dr"] = res[key]["sr"]["ms_per_step"] / res[key]["dr"]["ms_per_step"]
    res["paper_sr_over_dr"] = {"newtonian": "about 2", "viscoelastic": "above 2 (above 3 on few cores)",
                               "hardware": "CPU cluster, 256-2304 cores"}
    return res


def batch_leg(stream, nprob=64, steps=20):
    """64 uneven 2D droplets (coarse 64x32 .. 256x128, fine 2x, theta ~ U(30,150),
    Wi ~ U(0,2), beta = 0.5, mixed precision): one persistent launch per step
    versus stepping each problem through its own graph."""
    import gc
    import torch
    from paper_2111_04577_gb300 import binding, workloads as wl
    ws = wl.batch_problems(nprob, seed=0)
    cells = sum(w.grid.fine_cells() for w in ws)
    bt = binding.Batch([w.grid for w in ws], [w.params for w in ws], binding.PF_MIXED, stream=stream.cuda_stream)
    for b, w in enumerate(ws):
        bt.set(b, "phi", wl.initial_phi(w))
    bt.step(3)
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    bt.step(steps)
    e.record(stream)
    e.synchronize()
    t_b = a.elapsed_time(e) / 1e3
    bt.close()
    del bt
    solvers = []
    for w in ws:
        s = binding.Solver(w.grid, w.params, binding.PF_MIXED, stream=stream.cuda_stream)
        s.load_state(wl.initial_phi(w))
        s.step(3)
        solvers.append(s)
    torch.cuda.synchronize()
    a.record(stream)
    for s in solvers:
        s.step(steps)
    e.record(stream)
    e.synchronize()
    t_s = a.elapsed_time(e) / 1e3
    for s in solvers:
        s.close()
    del solvers
    gc.collect()
    return {"problems": nprob, "fine_cells": cells, "steps": steps,
            "cell_steps_per_s": cells * steps / t_b, "ms_per_step": t_b / steps * 1e3,
            "unbatched_cell_steps_per_s": cells * steps / t_s, "unbatched_ms_per_step": t_s / steps * 1e3,
            "speedup": t_s / t_b, "launches_per_step": 1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c4")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 / single-resolution legs")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--nx", type=int, default=0,
                    help="run the workload's physics at another coarse nx (ny = nx, nz = nx/2); profiling only")
    ap.add_argument("--nz", type=int, default=0, help="with --nx: coarse nz (default nx/2); profiling only")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    world, rank, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    from paper_2111_04577_gb300 import binding, build, workloads as wl
    build.build()
    w = workload(args.config)
    if args.nx:
        w = wl.scaled(w, args.nx, args.nz or args.nx // 2)
    g = w.grid
    stream = torch.cuda.Stream()
    prec = binding.PF_MIXED
    solver = binding.Solver(g, w.params, prec, stream=stream.cuda_stream)
    phi0 = wl.initial_phi(w)
    phi0_f = phi0.astype(np.float32)
    tuning = {}
    if not args.no_tune:
        from paper_2111_04577_gb300 import autotune
        tuning = autotune.tuned(g, w.params, prec, phi0=phi0_f)
        autotune.apply(solver, tuning)
    solver.load_state(phi0_f)
    # clocks are sampled from the warm-up on; more untimed warm-up steps run
    # until the sampler has reported (at most 5 s), so samples are under load
    clk, clk_path = clocks_start() if rank == 0 else (None, None)
    solver.step(args.warmup)
    torch.cuda.synchronize()
    t_wait = time.perf_counter()
    while clk is not None and time.perf_counter() - t_wait < 5.0:
        try:
            if os.path.getsize(clk_path) > 0:
                break
        except OSError:
            break
        solver.step(max(1, args.warmup))
        torch.cuda.synchronize()

    # ---------------- timed region (device-resident inputs) ----------------
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    elapsed = time_steps(solver, stream, args.steps)
    torch.cuda.synchronize()
    elapsed = max_over_ranks(elapsed, dist, "cuda")
    if dist:
        dist.barrier()
    clocks = clocks_stop(clk, clk_path) if rank == 0 else None
    ms_per_step = elapsed / args.steps * 1e3
    value = replica_value(g.fine_cells(), args.steps, world, elapsed)

    # ---------------- per-kernel profile and roofline ----------------
    prof, per_step = solver.profile(3)
    esize = 4
    ab = alg_bytes(g, esize, visco=True)
    peak, peak_kind = peaks()
    rows = []
    for name, ms, cnt in prof:
        byt = ab.get(name, 0)
        trk = traffic_for(name, g.fine_cells())
        rows.append({"kernel": name, "launches": cnt, "ms": ms, "alg_bytes": byt,
                     "gbs": byt / (ms * 1e-3) / 1e9 if ms > 0 else 0.0,
                     "dram_bytes": trk})
    dom = max(rows, key=lambda r: r["ms"])
    total_ms = sum(r["ms"] for r in rows)
    tr = traffic_for(dom["kernel"], g.fine_cells())
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["gbs"], "peak": peak, "unit": "GB/s",
                "frac": dom["gbs"] / peak,
                "traffic": None if tr is None else tr / max(1, dom["launches"]), "peak_kind": peak_kind,
                "alg_bytes_per_launch": dom["alg_bytes"] / max(1, dom["launches"]),
                "launch_ms": dom["ms"] / max(1, dom["launches"])}
    step_bytes = sum(ab.values())

    # ---------------- end to end through the C ABI with host buffers ----------------
    pin_in = torch.from_numpy(phi0_f).pin_memory()
    pin_out = torch.empty(phi0_f.size, dtype=torch.float32).pin_memory()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solver.set("phi", pin_in)
    solver.step(args.steps)
    solver.get("phi", out=pin_out)
    diag = solver.diagnostics()
    t_e2e = time.perf_counter() - t0
    t_e2e = max_over_ranks(t_e2e, dist, "cuda")
    h2d = 2 * phi0_f.nbytes  # phi^n and its start-up twin phi^{n-1}
    d2h = phi0_f.nbytes + 6 * 8
    e2e = {"value": replica_value(g.fine_cells(), args.steps, world, t_e2e), "unit": UNIT,
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "note": "pf_set_fields(phi from pinned host) + pf_step(K) + pf_get_fields(phi) + pf_diagnostics"}
    launches = per_step * args.steps + (args.steps // 50 + 1)

    extra = {}
    if rank == 0 and not args.no_compare:
        # accuracy of the mixed paths against the FP64 GPU path on the same input,
        # per field, after the workload's stated number of steps
        nst = w.steps if not args.nx else 20
        fields = ("phi", "u", "v", "w", "p", "theta", "tau")

        def run_fields(prec, x0):
            sv = binding.Solver(g, w.params, prec, stream=stream.cuda_stream)
            sv.load_state(x0)
            sv.step(nst)
            out = {f: sv.get(f).astype(np.float64) for f in fields}
            return sv, out

        def field_err(a, b):
            e = {"phi_maxabs": float(np.max(np.abs(a["phi"] - b["phi"])))}
            for f in fields[1:]:
                e[f + "_rel"] = float(np.max(np.abs(a[f] - b[f])) / max(np.max(np.abs(b[f])), 1e-300))
            return e

        sm, fm = run_fields(binding.PF_MIXED, phi0_f)
        sm.close()
        del sm
        sz, fz = run_fields(binding.PF_MIXED_Z64, phi0_f)
        sz.step(2)
        tz = time_steps(sz, stream, 5)
        sz.close()
        del sz
        sf, ff = run_fields(binding.PF_MIXED_Z2F, phi0_f)
        sf.step(2)
        tf = time_steps(sf, stream, 5)
        sf.close()
        del sf
        sd, fd = run_fields(binding.PF_FP64, phi0)
        sd.step(2)
        t64 = time_steps(sd, stream, 5)
        sd.close()
        del sd
        torch.cuda.empty_cache()
        extra["fp64_path"] = {"value": g.fine_cells() * 5 / t64, "ms_per_step": t64 / 5 * 1e3,
                              "speedup_mixed_over_fp64": (value / world) / (g.fine_cells() * 5 / t64),
                              "mixed_err_vs_fp64_after_steps": field_err(fm, fd),
                              "steps_compared": nst}
        extra["mixed_z64_path"] = {"what": "mixed with FP64 wall-normal eliminations",
                                   "value": g.fine_cells() * 5 / tz, "ms_per_step": tz / 5 * 1e3,
                                   "err_vs_fp64_after_steps": field_err(fz, fd)}
        extra["mixed_z2f_path"] = {"what": "mixed with double-float (48-bit significand) wall-normal eliminations",
                                   "value": g.fine_cells() * 5 / tf, "ms_per_step": tf / 5 * 1e3,
                                   "err_vs_fp64_after_steps": field_err(ff, fd),
                                   "err_vs_z64_after_steps": field_err(ff, fz)}
        # single resolution: CSR (phi on the coarse mesh) and RSR (all fields on the fine mesh)
        csr = wl.Grid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, 0)
        rsr = wl.Grid(2 * g.nx, 2 * g.ny, 2 * g.nz, g.lx, g.ly, g.lz, 0)
        v_csr, ms_csr = side_path(w, csr, binding.PF_MIXED, 10, 2, stream)
        v_rsr, ms_rsr = side_path(w, rsr, binding.PF_MIXED, 5, 2, stream)
        extra["single_res"] = {
            "csr": {"grid": f"{csr.nx}x{csr.ny}x{csr.nz} (phi coarse)", "cell_steps_per_s": v_csr,
                    "ms_per_step": ms_csr},
            "rsr": {"grid": f"{rsr.nx}x{rsr.ny}x{rsr.nz} (all fine)", "cell_steps_per_s": v_rsr,
                    "ms_per_step": ms_rsr,
                    "dual_speedup_at_same_phi_resolution": ms_rsr / ms_per_step},
        }
    if rank == 0 and not args.no_compare:
        extra["accuracy_dr_csr_vs_rsr"] = accuracy_leg(stream)
        extra["paper_case_coalescing_drops"] = paper_case_leg(stream)
        extra["batch_sweep"] = batch_leg(stream)
        if w.params.wi > 0:
            extra["gradients"] = gradients_leg(w, stream)
    cpu = cpu_sample(workload(args.config), 12, 64) if (rank == 0 and not args.no_cpu) else None

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (FP64 contact-line flux, zero mode, reductions)",
            "data": "synthetic",
            "config": {"workload": w.name + f" (coarse {g.nx}x{g.ny}x{g.nz} / fine "
                                   f"{g.fine_shape[2]}x{g.fine_shape[1]}x{g.fine_shape[0]}, mixed)",
                       "fine_cells": g.fine_cells(), "l2": "inputs larger than L2 (no flush)",
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks,
            "kernels": rows, "alg_bytes_per_fine_cell_step": step_bytes / g.fine_cells(),
            "step_roof_frac": (step_bytes / (ms_per_step * 1e-3) / 1e9) / peak,
            "profile_sum_ms": total_ms, "diagnostics": diag, "tuning": tuning,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    solver.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
