"""Shared helpers for the GPU parity tests (oracle <-> CUDA path)."""
import numpy as np

import oracle
import synth

F64_TOL = 1e-12   # FP64 path: max |gpu - oracle| / max |oracle|


def desc_for(fc, w, dtype, nforests=1, lmax=None):
    order, lim = {"none": (2, 0), "lw": (2, 0), "mc": (2, 1), "first": (1, 0)}[w.limiter]
    domain = {"walls": fc.WALLS, "periodic": fc.PERIODIC, "sphere": fc.SPHERE,
              "brick": fc.BRICK}[w.domain]
    return fc.make_desc(domain=domain, mx=w.mx,
                        lmin=w.lmin, lmax=w.lmax if lmax is None else lmax, dtype=dtype,
                        velocity=w.velocity, order=order, limiter=lim,
                        transverse=w.transverse, nforests=nforests,
                        indicator={"gradient": 0, "maxmin": 1}[w.indicator],
                        smooth=int(w.smooth), reflux=int(w.reflux), brick=w.brick)


def pair(fc, workloads, dtype):
    """An oracle forest and a GPU forest with the same initial layout and data."""
    ws = workloads if isinstance(workloads, (list, tuple)) else [workloads]
    ref = oracle.initial_forest(ws)
    lmax = max(w.lmax for w in ws)
    gpu = fc.Forest(desc_for(fc, ws[0], dtype, nforests=len(ws), lmax=lmax), ref.leaves())
    q0 = ref.get_q()
    if dtype == fc.F32:
        q0 = q0.astype(np.float32).astype(np.float64)
        ref.set_q(q0)
    gpu.set_q(q0)
    return ref, gpu


def relerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
