"""The launch list of a schedule (nqs_schedule_launches) against what the
library itself measures: the algorithmic bytes of its sweep passes over one
call equal the profiled total, and its operation counts match the plan."""

import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_launch_list_matches_profiled_bytes_and_plan():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    nqs.use_torch_allocator()
    w = W.random_circuit(61, 14, 80, 6, rate_lo=1e-3, rate_hi=2e-2)
    circ = nqs.NoisyCircuit(W.to_ir_text(w))
    psi, v = nqs.basis(w.psi["bits"]), nqs.basis(w.v["bits"])
    circ.fidelity(psi, v, 2)   # builds the schedule
    L = nqs.nqs_schedule_launches(circ.h)
    passes = [x for x in L if x["kind"] == "pass"]
    assert passes and all(x["states"] in (1, 2, 3) for x in passes)
    assert all(x["reg_qubits"] in (3, 4) and x["phases"] >= 1 for x in passes)   # n >= 12: register kernel
    nqs.nqs_set_profiling(circ.h, 1)
    circ.fidelity(psi, v, 2)
    stats = nqs.nqs_get_kernel_stats(circ.h, 0)
    nqs.nqs_set_profiling(circ.h, 0)
    assert stats["launches"] == len(passes)
    total = sum(x["algorithmic_bytes"] for x in passes)
    assert abs(stats["algorithmic_bytes"] - total) <= 1e-9 * total
    # the backward sweep saves phi once per site; the forward sweep spawns three states per site
    assert sum(x["saves"] for x in passes) == w.n_noise
    assert sum(x["spawned"] for x in passes) >= 3 * (w.n_noise - 1)
    circ.close()
