"""Several lattices on one device, created and stepped from several host
threads at once.  The launchers keep what they look up about a device (its
SM count, the fused kernel's shared-memory attribute, which belongs to the
device context) per device, so each thread's run must equal the same run
made alone.  The threads run in a fresh spawned process, so that the first
launch on the device, which sets that per-device state, is the concurrent
one."""
import multiprocessing as mp
import os
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (24, 20, 40)
CASES = [dict(storage="f32", tau=(0.8, 1.0), G12=-1.3),
         dict(storage="bf16_dev", rho0_dev=0.5, tau=(0.7, 0.7), G12=-1.2, collision="regularized"),
         dict(storage="f32", tau=(0.9, 0.9), G12=-1.2, collision="regularized3", periodic=(1, 1, 0)),
         dict(storage="f64", tau=(1.0, 0.8), G12=-1.1)]
STEPS = 60


def _run(kw):
    from paper_1601_01237_gb300 import Lattice, workloads as wl
    r1, r2, u = wl.random_state(SHAPE, seed=13, u_max=0.02)
    lat = Lattice(SHAPE, torch_stream=False, **kw)   # each lattice on its own library stream
    lat.init_fields(r1, r2, u)
    lat.step(STEPS)
    f = lat.get_populations()
    lat.close()
    return f


def _child(conn):
    """Fresh process: every case on its own thread, started together, then
    every case again alone; returns whether each pair is bitwise equal."""
    import torch
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    import sys
    sys.path.insert(0, root)
    torch.cuda.set_device(0)
    out = [None] * len(CASES)
    errors = []
    gate = threading.Barrier(len(CASES))

    def work(k):
        try:
            gate.wait()
            out[k] = _run(CASES[k])
        except Exception as e:   # reported to the parent
            errors.append(repr(e))

    th = [threading.Thread(target=work, args=(k,)) for k in range(len(CASES))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errors:
        conn.send(("error", errors))
        return
    same = [bool(np.array_equal(out[k], _run(CASES[k]))) for k in range(len(CASES))]
    conn.send(("ok", same))


def test_lattices_on_concurrent_threads(gpu_lib):
    ctx = mp.get_context("spawn")
    parent, child = ctx.Pipe()
    p = ctx.Process(target=_child, args=(child,))
    p.start()
    assert parent.poll(300), "child process did not answer"
    status, res = parent.recv()
    p.join(60)
    assert status == "ok", res
    assert all(res), res
