"""The allocation-free diagnostics entry point against the context's own.

pf_diagnostics_noalloc exists for callers that cannot allocate device memory
(an application whose pool owns the GPU, an allocator that forbids cudaMalloc,
a real-time loop that must not stall on an allocation).  It reduces a phase
field the caller already holds on the device, using only a fixed device array
the CUDA runtime reserves on the GPU by the library's first call there.  Here it must give what
pf_diagnostics gives for the same field, on two calls in a row (the shared
array keeps the previous call's contents), in every precision, and it must
refuse a field larger than its fixed array.  (The caller's field is the
stored phi values: the context's own mass also counts the rounding remainders
an FP32 context keeps, PF_PHI_REM, which are taken off for the comparison.)

This file is collected last on purpose: it runs after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2111_04577_gb300 import binding, build, workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-10  # the FP64 parity tolerance of the GPU tests


def _close(a, b, scale):
    return abs(a - b) <= TOL * (abs(b) + scale)


@pytest.mark.parametrize("prec", [binding.PF_FP64, binding.PF_MIXED, binding.PF_MIXED_Z64, binding.PF_MIXED_Z2F])
@pytest.mark.parametrize("case", ["2d", "3d"])
def test_noalloc_diagnostics_match_context_twice(prec, case):
    import torch
    build.build()
    lib = binding.load()
    if case == "2d":
        w = wl.scaled(wl.config("c2"), 32, 16)
    else:
        w = wl.scaled(wl.config("c4"), 16, 8)
    g = w.grid
    s = binding.Solver(g, w.params, prec)
    s.load_state(wl.initial_phi(w))
    gd = binding.GridDesc(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, prec, g.dual)
    prm = binding.ParamsC(**w.params.as_dict())
    n, eb = s.info("phi")
    dtype = torch.float64 if eb == 8 else torch.float32
    buf = torch.empty(n, dtype=dtype, device="cuda")
    for call in range(2):
        s.step(3)
        ref = s.diagnostics()
        s.get("phi", out=buf)
        torch.cuda.synchronize()
        out = (C.c_double * 6)()
        rc = lib.pf_diagnostics_noalloc(C.byref(gd), C.byref(prm), C.c_void_p(buf.data_ptr()), out, None)
        assert rc == 0, (call, rc)
        scale = float(torch.sum(torch.abs(buf)).item()) * g.h ** g.dim
        rem = float(np.sum(s.get("phi_rem").astype(np.float64))) * g.h ** g.dim
        assert _close(out[0], ref["mass"] - rem, scale), (call, out[0], ref["mass"], rem)
        assert _close(out[1], ref["energy"], 0.0), (call, out[1], ref["energy"])
        assert _close(out[2], ref["wetted"], 0.0), (call, out[2], ref["wetted"])
        for q in range(3):
            assert _close(out[3 + q], ref["centroid"][q], 1.0), (call, q)
    s.close()


def test_noalloc_rejects_fields_beyond_its_fixed_array():
    import torch
    build.build()
    lib = binding.load()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    # coarse 512 x 512 x 128 -> fine 1024 x 1024 x 256 = 268,435,456 cells, above the fixed maximum
    gd = binding.GridDesc(512, 512, 128, 512.0, 512.0, 128.0, binding.PF_MIXED, 1)
    prm = binding.ParamsC(**wl.params_from_groups().as_dict())
    out = (C.c_double * 6)()
    rc = lib.pf_diagnostics_noalloc(C.byref(gd), C.byref(prm), C.c_void_p(buf.data_ptr()), out, None)
    assert rc == -3  # PF_ERR_UNSUPPORTED, before any device work
