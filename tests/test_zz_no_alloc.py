"""The allocation-free reduced-matrix entry point.

nqs_reduced_matrix_noalloc serves callers that cannot allocate device memory
(their device heap belongs to another runtime's pool, or cudaMalloc's
device-wide synchronisation is not acceptable where they call it): its
scratch is a fixed device array inside the library.  Here it is called
through the C ABI twice in a row, on different inputs, and each result is
compared with the allocating entry point nqs_reduced_matrix on the same
inputs, at the tolerance of the other GPU parity tests.  The file sorts last
so that a run stopping at the first failure has already run every other
test; it sets up everything it needs, so it also passes alone.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _reference(nqs, torch, phi, chi, n, q):
    nb = nqs.nqs_reduced_matrix_scratch_bytes(n)
    scratch = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    nqs.nqs_reduced_matrix(phi, chi, n, q, out, scratch, nb)
    return out.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_two_calls():
    import torch
    from paper_2211_17028_gb300 import nqs
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    g = torch.Generator(device="cpu").manual_seed(2211)
    cases = [(20, 7), (13, 0), (1, 0), (24, 23)]
    for n, q in cases:
        results = []
        for call in range(2):   # two calls in a row share the library's scratch array
            a = torch.randn(1 << n, 2, generator=g, dtype=torch.float32)
            b = torch.randn(1 << n, 2, generator=g, dtype=torch.float32)
            phi = torch.view_as_complex(a).contiguous().cuda()
            chi = torch.view_as_complex(b).contiguous().cuda()
            out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
            nqs.nqs_reduced_matrix_noalloc(phi, chi, n, q, out)
            got = out.cpu().numpy()
            want = _reference(nqs, torch, phi, chi, n, q)
            scale = np.abs(want).max()
            assert np.all(np.isfinite(got))
            assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * scale), (n, q, call, got, want)
            results.append(got)
        assert not np.allclose(results[0], results[1])   # the second call saw new data


def test_noalloc_rejects_sizes_beyond_its_capacity():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_reduced_matrix_noalloc(x, x, nqs.NQS_NOALLOC_MAX_QUBITS + 1, 0, out)
    assert e.value.code == nqs.NQS_ERR_TOO_LARGE
    with pytest.raises(nqs.NqsError) as e:
        nqs.nqs_reduced_matrix_noalloc(x, x, 2, 2, out)
    assert e.value.code == nqs.NQS_ERR_ARG
