"""rpca_solve_host keeps its device buffers, stream and context between calls; a device reset
between two calls (which ends the process's own CUDA context and every object in it) must not
leave it using the dead objects.  Run in a child process that uses no other CUDA client, with
host (numpy) buffers only: solve, cudaDeviceReset, solve again; both solves must agree."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import synth
import paper_1711_05519_gb300.rpca as R
L = R.lib()
cudart = ctypes.CDLL("libcudart.so.13")
inst = synth.planted_instance(600, 560, 3, 0.1, 1.0, 81)
p = inst.params()
D = np.ascontiguousarray(inst.D.astype(np.float32))
m, n, r = 600, 560, 3
cap = m * n
ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
res = []
for call in range(2):
    U = np.zeros((m, r)); s = np.zeros(r); V = np.zeros((n, r))
    idx = np.zeros(cap, dtype=np.int64); val = np.zeros(cap)
    nnz, iters, err = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_double(0)
    code = L.rpca_solve_host(ptr(D), m, n, r, p["beta"], p["gamma"], 1e-5, ptr(U), ptr(s), ptr(V), ptr(idx), ptr(val),
                             cap, ctypes.byref(nnz), ctypes.byref(iters), ctypes.byref(err))
    res.append({"code": code, "nnz": nnz.value, "iters": iters.value, "err": err.value,
                "L": float(np.linalg.norm((U * s) @ V.T)), "idx": idx[: nnz.value].tolist()[:50]})
    if call == 0:
        assert cudart.cudaDeviceReset() == 0
print(json.dumps(res))
"""


def test_solve_host_survives_a_device_reset():
    import json

    out = subprocess.run([sys.executable, "-c", CHILD, ROOT], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-3000:]
    a, b = json.loads(out.stdout.strip().splitlines()[-1])
    assert a["code"] == b["code"] == 0
    assert a["iters"] == b["iters"] and a["nnz"] == b["nnz"] and a["idx"] == b["idx"]
    assert abs(a["L"] - b["L"]) <= 1e-12 * a["L"]
    assert a["err"] == b["err"]
