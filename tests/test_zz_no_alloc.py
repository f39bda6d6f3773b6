"""GPU check of sldqmc_weight_noalloc, the allocation-free form of the exact
weight for callers that cannot call cudaMalloc or cudaFree (for example code
running under a host framework that owns the whole device heap, or a
latency-critical path that must not take cudaFree's implicit device
synchronisation).  It must give the same result as the context-based
sldqmc_weight_batch_dev, on two calls in a row (the second call reuses the
static workspace the first one left behind).  This file is collected last."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LD_RTOL = 1e-9  # the FP64-mode tolerance of the weight parity tests


def test_noalloc_weight_matches_context_path_on_two_calls():
    import torch
    from paper_1612_03804_gb300 import build, sldqmc
    from paper_1612_03804_gb300.inputs import batch_uniform

    build.build()
    torch.cuda.set_device(0)
    lib = sldqmc.load()
    B = 3
    with sldqmc.Context(8, 8, mu=-0.5, xi=1.0, beta=4.0, dtau=0.05, n_wrap=10, max_batch=B) as ctx:
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call, (seed, eta) in enumerate(((11, -1), (12, 1))):
            fields = batch_uniform(seed, B, ctx.M, ctx.N)
            d_s = torch.from_numpy(fields).cuda()
            ref_ld = torch.zeros(B, dtype=torch.float64, device="cuda")
            ref_sg = torch.zeros(B, dtype=torch.int32, device="cuda")
            ctx.weight_batch_dev(d_s, eta, ref_ld, ref_sg)
            ctx.sync()
            ld = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
            sg = torch.zeros(B, dtype=torch.int32, device="cuda")
            rc = lib.sldqmc_weight_noalloc(ctypes.byref(ctx.params), stream, ctypes.c_void_p(d_s.data_ptr()), B,
                                           eta, ctypes.c_void_p(ld.data_ptr()), ctypes.c_void_p(sg.data_ptr()))
            assert rc == 0, f"call {call}: status {rc}"
            a, r = ld.cpu().numpy(), ref_ld.cpu().numpy()
            assert np.all(np.isfinite(a))
            np.testing.assert_array_equal(sg.cpu().numpy(), ref_sg.cpu().numpy())
            assert np.all(np.abs(a - r) <= LD_RTOL * np.abs(r)), (call, a, r)


def test_noalloc_rejects_problems_beyond_its_workspace():
    from paper_1612_03804_gb300 import build, sldqmc
    build.build()
    lib = sldqmc.load()
    p = sldqmc.Params(32, 32, 1.0, -0.5, 1.0, 10.0, 0.05, 10, 1.0, 2.774, 0, 1)
    # 32x32 needs about 80 MB of workspace: rejected before any device work
    assert lib.sldqmc_weight_noalloc(ctypes.byref(p), None, ctypes.c_void_p(1), 1, -1, ctypes.c_void_p(1),
                                     None) == -6


# Runs in a fresh interpreter: the allocation-free call is the first use of
# the library there (no context was created before it), at a lattice size
# whose LU panels need more than the default 48 KiB of shared memory.
_FRESH = r"""
import ctypes, json, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_1612_03804_gb300 import sldqmc
from paper_1612_03804_gb300.inputs import batch_uniform
torch.cuda.set_device(0)
lib = sldqmc.load()
p = sldqmc.Params(16, 16, 1.0, -0.5, 1.0, 1.0, 0.05, 10, 1.0, 2.774, 0, 2)
B, M, N = 2, 20, 256
out = []
for seed in (21, 22):
    d_s = torch.from_numpy(batch_uniform(seed, B, M, N)).cuda()
    ld = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
    sg = torch.zeros(B, dtype=torch.int32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.sldqmc_weight_noalloc(ctypes.byref(p), st, ctypes.c_void_p(d_s.data_ptr()), B, -1,
                                   ctypes.c_void_p(ld.data_ptr()), ctypes.c_void_p(sg.data_ptr()))
    out.append({"rc": rc, "ld": ld.cpu().tolist(), "sg": sg.cpu().tolist()})
print(json.dumps(out))
"""


def test_noalloc_first_call_in_fresh_process_16x16_matches_oracle():
    from oracle import oracle as O
    from paper_1612_03804_gb300 import build
    from paper_1612_03804_gb300.inputs import batch_uniform

    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    calls = json.loads(r.stdout.strip().splitlines()[-1])
    m = O.Model(16, 16, t=1.0, mu=-0.5, xi=1.0, beta=1.0, dtau=0.05, n_wrap=10)
    for call, seed in zip(calls, (21, 22)):
        assert call["rc"] == 0, call
        fields = batch_uniform(seed, 2, m.M, m.N)
        for b in range(2):
            ld, sg = O.weight(m, fields[b], -1)
            assert call["sg"][b] == sg
            assert abs(call["ld"][b] - ld) <= LD_RTOL * abs(ld), (call, ld)
