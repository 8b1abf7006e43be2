"""Failure detection on the GPU without a fault: every wait in the sweep
kernels is bounded and reports a status word instead of hanging.  The probe
runs that bounded wait on an mbarrier nothing arrives at; the wait must give
up within a few seconds, report NQS_ERR_DEVICE_TIMEOUT, and leave the
context usable (a fidelity call afterwards still matches the oracle)."""

import time

import pytest

import workloads as W

from _gpu_util import REL_TOL, oracle_result

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_reports():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    t0 = time.perf_counter()
    status = nqs.nqs_selftest_bounded_wait()
    dt = time.perf_counter() - t0
    assert status == nqs.NQS_ERR_DEVICE_TIMEOUT
    assert dt < 30.0
    assert nqs.nqs_strerror(status)
    # the context is still usable
    w = W.c1_line6()
    ref = oracle_result(w, 1)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    r = circ.fidelity(nqs.basis(w.psi["bits"]), nqs.basis(w.v["bits"]), 1)
    circ.close()
    assert r["status"] == 0
    assert abs(r["F"] - ref["F"].real) <= REL_TOL * abs(ref["F"].real)
