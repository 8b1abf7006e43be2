"""The allocation-free reduced-matrix entry point.

nqs_reduced_matrix_noalloc serves callers that cannot allocate device memory
(their device heap belongs to another runtime's pool, or cudaMalloc's
device-wide synchronisation is not acceptable where they call it): its
scratch is a fixed device array inside the library.  Here it is called
through the C ABI twice in a row, on different inputs, and each result is
compared with the allocating entry point nqs_reduced_matrix on the same
inputs and with the reduced matrix written out in FP64 numpy,
R[a][b] = sum_rest conj(phi[rest, a]) chi[rest, b], at the tolerance of the
other GPU parity tests.  The file sorts last
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


def _numpy_reduced(phi, chi, n, q):
    """R[a][b] = sum over the other qubits of conj(phi[.., a, ..]) chi[.., b, ..]
    on qubit q, in FP64, as (re, im) of R00, R01, R10, R11."""
    p = phi.cpu().numpy().astype(np.complex128).reshape(-1, 2, 1 << q)
    c = chi.cpu().numpy().astype(np.complex128).reshape(-1, 2, 1 << q)
    R = np.einsum("iak,ibk->ab", p.conj(), c)
    return np.array([[z.real, z.imag] for z in R.reshape(-1)]).reshape(-1)


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
            exact = _numpy_reduced(phi, chi, n, q)
            scale = np.abs(exact).max()
            assert np.all(np.isfinite(got))
            assert np.allclose(got, want, rtol=1e-5, atol=1e-5 * scale), (n, q, call, got, want)
            assert np.allclose(got, exact, rtol=1e-5, atol=1e-5 * scale), (n, q, call, got, exact)
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


def test_noalloc_rejects_memory_the_device_cannot_use():
    import torch
    from paper_2211_17028_gb300 import nqs
    torch.cuda.set_device(0)
    n = 6
    dev = torch.zeros(1 << n, dtype=torch.complex64, device="cuda")
    host = torch.zeros(1 << n, dtype=torch.complex64)                 # pageable host memory
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    out_host = torch.zeros(8, dtype=torch.float64)
    for args in ((host, dev, out), (dev, host, out), (dev, dev, out_host)):
        with pytest.raises(nqs.NqsError) as e:
            nqs.nqs_reduced_matrix_noalloc(args[0], args[1], n, 0, args[2])
        assert e.value.code == nqs.NQS_ERR_ARG
    # pinned host memory is a valid destination for the result
    out_pinned = torch.zeros(8, dtype=torch.float64).pin_memory()
    dev.fill_(1.0)
    nqs.nqs_reduced_matrix_noalloc(dev, dev, n, 0, out_pinned)
    torch.cuda.synchronize()
    assert out_pinned[0].item() == pytest.approx(float(1 << (n - 1)))
