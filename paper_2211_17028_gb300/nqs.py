"""Python binding of libnqs (include/nqs.h): argument marshalling only.

Every function keeps the C name and forwards to the shared library; all
computation happens in the library's CUDA kernels.  PyTorch provides device
memory (the library's allocator hook is pointed at torch's caching
allocator) and streams.  Importing this module fails loudly when the
compiled library is missing: there is no fallback.
"""

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnqs.so")

NQS_OK = 0
NQS_ERR_ARG = 1
NQS_ERR_PARSE = 2
NQS_ERR_NOT_CPTP = 3
NQS_ERR_NOT_DOMINANT = 4
NQS_ERR_NOMEM = 5
NQS_ERR_CUDA = 6
NQS_ERR_ORDER = 7
NQS_ERR_DEVICE_TIMEOUT = 8
NQS_ERR_UNSUPPORTED = 9
NQS_ERR_TOO_LARGE = 10
NQS_ERR_COMPILE = 11
NQS_NOALLOC_MAX_QUBITS = 34

NQS_STATE_BASIS = 0
NQS_STATE_DENSE = 1
NQS_STATE_IDEAL = 2
NQS_PREP_PRUNE_ZERO_RANK = 1
NQS_MAX_LEVEL = 16
NQS_OPT_CKPT_SPACING = 1
NQS_OPT_SWEEP_RB = 2
NQS_OPT_MAX_OPS = 3
NQS_OPT_MAX_SITES = 4
NQS_OPT_JIT = 5
NQS_OPT_SHARD_RANK = 6
NQS_OPT_SHARD_COUNT = 7


class NqsError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (code %d)" % (where, _lib().nqs_strerror(code).decode(), code))


class nqs_state(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("bits", ctypes.c_uint64), ("dev", ctypes.c_void_p)]


class nqs_noise(ctypes.Structure):
    _fields_ = [("after_gate", ctypes.c_int32), ("qubit", ctypes.c_uint32), ("n_kraus", ctypes.c_uint32),
                ("kraus", ctypes.POINTER(ctypes.c_double))]


class nqs_result(ctypes.Structure):
    _fields_ = [("F", ctypes.c_double), ("T", ctypes.c_double * (NQS_MAX_LEVEL + 1)),
                ("imag_residual", ctypes.c_double), ("n_terms", ctypes.c_uint64), ("bound", ctypes.c_double),
                ("level", ctypes.c_int32), ("status", ctypes.c_int32)]

    def to_dict(self):
        return {"F": self.F, "T": [self.T[u] for u in range(self.level + 1)],
                "imag_residual": self.imag_residual, "n_terms": int(self.n_terms), "bound": self.bound,
                "level": self.level, "status": self.status}


class nqs_is_result(ctypes.Structure):
    _fields_ = [("estimate", ctypes.c_double), ("stderr_", ctypes.c_double), ("ess", ctypes.c_double),
                ("samples", ctypes.c_uint64), ("distinct", ctypes.c_uint64), ("n_sets", ctypes.c_uint64),
                ("alpha", ctypes.c_double), ("level", ctypes.c_int32), ("status", ctypes.c_int32)]

    def to_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class nqs_info(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("n_gates", ctypes.c_int32), ("n_sites", ctypes.c_int32),
                ("n_ops", ctypes.c_int32), ("n_passes", ctypes.c_int32), ("tile_qubits", ctypes.c_int32),
                ("workspace_bytes", ctypes.c_uint64), ("upload_bytes", ctypes.c_uint64),
                ("launches_per_call", ctypes.c_uint64), ("ckpt_spacing", ctypes.c_int32),
                ("n_states", ctypes.c_int32), ("jit_launches", ctypes.c_int32), ("jit_state", ctypes.c_int32)]


class nqs_launch_info(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("states", ctypes.c_int32), ("reg_qubits", ctypes.c_int32),
                ("phases", ctypes.c_int32), ("grid", ctypes.c_int32), ("ops", ctypes.c_int32 * 8),
                ("jit", ctypes.c_int32), ("algorithmic_bytes", ctypes.c_double)]


class nqs_kernel_stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("algorithmic_bytes", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_L = None

# name -> (restype, argtypes)
_SIGS = {
    "nqs_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, ctypes.c_void_p]),
    "nqs_load_circuit": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    "nqs_prepare_noise": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_noise), ctypes.c_size_t,
                                         ctypes.c_uint32]),
    "nqs_fidelity": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_state), ctypes.POINTER(nqs_state),
                                    ctypes.c_int, ctypes.POINTER(nqs_result), ctypes.c_void_p]),
    "nqs_batch_fidelity": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t,
                                          ctypes.POINTER(nqs_state), ctypes.POINTER(nqs_state),
                                          ctypes.POINTER(ctypes.c_int), ctypes.POINTER(nqs_result),
                                          ctypes.c_void_p]),
    "nqs_enumerate_terms": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                           ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "nqs_noise_factors": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
    "nqs_term_values": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t)]),
    "nqs_truncation_bound": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "nqs_plan_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "nqs_jit_compile_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "nqs_shard_mask": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "nqs_general_factors": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nqs_offdiagonal": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_state), ctypes.POINTER(nqs_state),
                                       ctypes.POINTER(nqs_state), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(nqs_result), ctypes.c_void_p]),
    "nqs_fidelity_adaptive": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_state), ctypes.POINTER(nqs_state),
                                             ctypes.c_double, ctypes.c_int, ctypes.c_uint32,
                                             ctypes.POINTER(nqs_result), ctypes.c_void_p]),
    "nqs_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_info)]),
    "nqs_set_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]),
    "nqs_selftest_bounded_wait": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_void_p]),
    "nqs_schedule_launches": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                             ctypes.POINTER(ctypes.c_size_t)]),
    "nqs_get_option": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "nqs_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_state), ctypes.POINTER(nqs_state), ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(nqs_result), ctypes.c_void_p]),
    "nqs_set_profiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "nqs_get_kernel_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(nqs_kernel_stats)]),
    "nqs_reduced_matrix": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]),
    "nqs_reduced_matrix_scratch_bytes": (ctypes.c_size_t, [ctypes.c_int]),
    "nqs_reduced_matrix_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_void_p, ctypes.c_void_p]),
    "nqs_prepare_sets": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(nqs_state), ctypes.POINTER(nqs_state),
                                        ctypes.c_void_p]),
    "nqs_eval_sets": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "nqs_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "nqs_mlp_param_count": (ctypes.c_size_t, [ctypes.c_void_p]),
    "nqs_mlp_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "nqs_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "nqs_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                       ctypes.c_void_p]),
    "nqs_mlp_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_size_t,
                                         ctypes.c_void_p]),
    "nqs_mlp_train": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_void_p]),
    "nqs_mlp_destroy": (None, [ctypes.c_void_p]),
    "nqs_site_features": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "nqs_pair_training_data": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "nqs_is_estimate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(nqs_is_result), ctypes.c_void_p]),
    "nqs_is_proposal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                                       ctypes.POINTER(ctypes.c_size_t), ctypes.c_void_p]),
    "nqs_destroy": (None, [ctypes.c_void_p]),
    "nqs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "nqs_version": (ctypes.c_char_p, []),
}


def _lib():
    global _L
    if _L is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libnqs.so is not built (run __graft_entry__.build()): " + LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _L = L
    return _L


def library():
    return _lib()


def _check(rc, where):
    if rc != NQS_OK:
        raise NqsError(rc, where)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# --------------------------------------------------------------- allocator
_alloc_refs = None


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_refs
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _check(_lib().nqs_set_allocator(a, f, None), "nqs_set_allocator")
    _alloc_refs = (a, f)


def use_cuda_allocator():
    global _alloc_refs
    _check(_lib().nqs_set_allocator(ALLOC_FN(), FREE_FN(), None), "nqs_set_allocator")
    _alloc_refs = None


def nqs_set_allocator(alloc, release, ctx=None):
    _check(_lib().nqs_set_allocator(alloc, release, ctx), "nqs_set_allocator")


# --------------------------------------------------------------- states
def basis(bits):
    return nqs_state(NQS_STATE_BASIS, int(bits), None)


def dense(tensor):
    """A complex64 CUDA tensor (or its data pointer)."""
    ptr = tensor if isinstance(tensor, int) else tensor.data_ptr()
    return nqs_state(NQS_STATE_DENSE, 0, ctypes.c_void_p(ptr))


def ideal():
    return nqs_state(NQS_STATE_IDEAL, 0, None)


def _as_state(s):
    if isinstance(s, nqs_state):
        return s
    if isinstance(s, dict):
        if s["kind"] == "basis":
            return basis(s["bits"])
        if s["kind"] == "ideal":
            return ideal()
        if s["kind"] == "dense":
            return dense(s["tensor"])
    raise TypeError("unsupported state descriptor")


# --------------------------------------------------------------- entry points
def nqs_load_circuit(ir_text):
    h = ctypes.c_void_p()
    _check(_lib().nqs_load_circuit(ir_text.encode() if isinstance(ir_text, str) else ir_text, ctypes.byref(h)),
           "nqs_load_circuit")
    return h


def _noise_array(sites):
    import numpy as np
    arr = (nqs_noise * len(sites))()
    keep = []
    for i, (after_gate, qubit, kraus) in enumerate(sites):
        buf = np.ascontiguousarray(np.array([np.asarray(k, dtype=np.complex128).reshape(4) for k in kraus])
                                   .view(np.float64).reshape(-1))
        keep.append(buf)
        arr[i] = nqs_noise(int(after_gate), int(qubit), len(kraus),
                           buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return arr, keep


def nqs_prepare_noise(h, sites=None, flags=0):
    """sites: None (use the circuit text's noise records) or a list of
    (after_gate, qubit, [2x2 Kraus matrices])."""
    if sites is None:
        _check(_lib().nqs_prepare_noise(h, None, 0, flags), "nqs_prepare_noise")
    else:
        arr, keep = _noise_array(sites)
        _check(_lib().nqs_prepare_noise(h, arr, len(sites), flags), "nqs_prepare_noise")


def nqs_fidelity(h, psi, v, level, stream=None, out=None):
    """Returns the nqs_result (host copy; the call synchronises through the
    pageable result copy unless `out` is a device/pinned nqs_result)."""
    res = out if out is not None else nqs_result()
    ps, vs = _as_state(psi), _as_state(v)
    _check(_lib().nqs_fidelity(h, ctypes.byref(ps), ctypes.byref(vs), int(level), ctypes.byref(res),
                               _stream_ptr(stream)), "nqs_fidelity")
    return res


def nqs_batch_fidelity(hs, psis, vs, levels, stream=None):
    n = len(hs)
    harr = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in hs])
    parr = (nqs_state * n)(*[_as_state(p) for p in psis])
    varr = (nqs_state * n)(*[_as_state(v) for v in vs])
    larr = (ctypes.c_int * n)(*[int(x) for x in levels])
    outs = (nqs_result * n)()
    _check(_lib().nqs_batch_fidelity(harr, n, parr, varr, larr, outs, _stream_ptr(stream)),
           "nqs_batch_fidelity")
    return list(outs)


def nqs_enumerate_terms(h, level):
    cnt = ctypes.c_size_t()
    _check(_lib().nqs_enumerate_terms(h, level, None, 0, ctypes.byref(cnt)), "nqs_enumerate_terms")
    buf = (ctypes.c_uint64 * max(1, cnt.value))()
    _check(_lib().nqs_enumerate_terms(h, level, buf, cnt.value, ctypes.byref(cnt)), "nqs_enumerate_terms")
    return [int(buf[i]) for i in range(cnt.value)]


def nqs_noise_factors(h, site):
    import numpy as np
    d = (ctypes.c_double * 4)()
    k = (ctypes.c_double * 32)()
    _check(_lib().nqs_noise_factors(h, site, d, k), "nqs_noise_factors")
    kk = np.array(list(k)).view(np.complex128).reshape(4, 2, 2)
    return np.array(list(d)), kk


def nqs_term_values(h):
    import numpy as np
    cnt = ctypes.c_size_t()
    _check(_lib().nqs_term_values(h, None, 0, ctypes.byref(cnt)), "nqs_term_values")
    out = np.zeros(max(1, cnt.value), dtype=np.float64)
    _check(_lib().nqs_term_values(h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cnt.value,
                                  ctypes.byref(cnt)), "nqs_term_values")
    return out[:cnt.value]


def nqs_plan_check(h):
    """Largest entry difference between the plan's operator product and the
    circuit's (host only, n <= 10)."""
    out = ctypes.c_double()
    _check(_lib().nqs_plan_check(h, ctypes.byref(out)), "nqs_plan_check")
    return out.value


def nqs_jit_compile_check(h, states, max_passes):
    """Number of pass-specialised kernels generated and compiled (no device)."""
    out = ctypes.c_int()
    _check(_lib().nqs_jit_compile_check(h, states, max_passes, ctypes.byref(out)), "nqs_jit_compile_check")
    return out.value


def nqs_truncation_bound(h, level):
    out = ctypes.c_double()
    _check(_lib().nqs_truncation_bound(h, level, ctypes.byref(out)), "nqs_truncation_bound")
    return out.value


NQS_ADAPT_BOUND = 1
NQS_ADAPT_OBSERVED = 2


def nqs_fidelity_adaptive(h, psi, v, tol, max_level=NQS_MAX_LEVEL, criteria=NQS_ADAPT_BOUND | NQS_ADAPT_OBSERVED,
                          stream=None):
    """Raise the level until the truncation bound or the last level's sum is
    within tol (synchronises the stream); the result of the level reached."""
    ps, vs = _as_state(psi), _as_state(v)
    out = nqs_result()
    _check(_lib().nqs_fidelity_adaptive(h, ctypes.byref(ps), ctypes.byref(vs), float(tol), int(max_level),
                                        int(criteria), ctypes.byref(out), _stream_ptr(stream)),
           "nqs_fidelity_adaptive")
    return out.to_dict()


def nqs_offdiagonal(h, psi, x, y, level, stream=None):
    """<x|rho_l|y> by the polarization identity (four level-l calls); returns
    (complex value, [four result dicts])."""
    ps, xs, ys = _as_state(psi), _as_state(x), _as_state(y)
    out = (ctypes.c_double * 2)()
    parts = (nqs_result * 4)()
    _check(_lib().nqs_offdiagonal(h, ctypes.byref(ps), ctypes.byref(xs), ctypes.byref(ys), int(level), out, parts,
                                  _stream_ptr(stream)), "nqs_offdiagonal")
    return complex(out[0], out[1]), [parts[k].to_dict() for k in range(4)]


def nqs_shard_mask(h, level, rank, count):
    """Boolean mask over the canonical kept terms: the ones shard `rank` of
    `count` evaluates (NQS_OPT_SHARD_RANK / NQS_OPT_SHARD_COUNT)."""
    import numpy as np
    n = ctypes.c_size_t()
    _check(_lib().nqs_shard_mask(h, level, rank, count, None, 0, ctypes.byref(n)), "nqs_shard_mask")
    mask = np.zeros(n.value, np.uint8)
    _check(_lib().nqs_shard_mask(h, level, rank, count, mask.ctypes.data_as(ctypes.c_void_p), n.value,
                                 ctypes.byref(n)), "nqs_shard_mask")
    return mask.astype(bool)


def merge_level_sums(parts):
    """Merge the per-level sums T_u of several shards of one call, in the
    order given (Neumaier compensation across the shards): the whole call's
    T_u and F."""
    L = max(len(p) for p in parts)
    T = []
    for u in range(L):
        s, c = 0.0, 0.0
        for p in parts:
            x = p[u] if u < len(p) else 0.0
            t = s + x
            c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
            s = t
        T.append(s + c)
    s, c = 0.0, 0.0
    for x in T:
        t = s + x
        c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
        s = t
    return T, s + c


def merge_level_sums_distributed(T, group=None):
    """All shards of a torch.distributed group exchange their T_u (a few
    doubles) and merge them in rank order; every rank gets the whole call's
    (T_u, F)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, list(T), group=group)
    return merge_level_sums(parts)


def nqs_general_factors(h, site):
    """(singular values, KA, KB, same) of a general-noise site as numpy arrays
    (KA, KB: m x d x d complex128)."""
    import numpy as np
    m, d, same = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(_lib().nqs_general_factors(h, site, ctypes.byref(m), ctypes.byref(d), ctypes.byref(same), None, None, None),
           "nqs_general_factors")
    sv = np.zeros(m.value)
    ka = np.zeros((m.value, d.value, d.value), np.complex128)
    kb = np.zeros_like(ka)
    _check(_lib().nqs_general_factors(h, site, ctypes.byref(m), ctypes.byref(d), ctypes.byref(same),
                                      sv.ctypes.data_as(ctypes.c_void_p), ka.ctypes.data_as(ctypes.c_void_p),
                                      kb.ctypes.data_as(ctypes.c_void_p)), "nqs_general_factors")
    return sv, ka, kb, bool(same.value)


def nqs_get_info(h):
    info = nqs_info()
    _check(_lib().nqs_get_info(h, ctypes.byref(info)), "nqs_get_info")
    return {f: getattr(info, f) for f, _ in nqs_info._fields_}


LAUNCH_KINDS = ("pass", "finish", "fill", "copy", "reduce2", "sum", "normalize")
OP_COUNT_NAMES = ("g1", "g2", "d1", "d2", "sites", "reductions", "spawned", "saves")


def nqs_schedule_launches(h):
    """Launch list of the current schedule as a list of dicts."""
    cnt = ctypes.c_size_t()
    _check(_lib().nqs_schedule_launches(h, None, 0, ctypes.byref(cnt)), "nqs_schedule_launches")
    buf = (nqs_launch_info * max(1, cnt.value))()
    _check(_lib().nqs_schedule_launches(h, buf, cnt.value, ctypes.byref(cnt)), "nqs_schedule_launches")
    out = []
    for i in range(cnt.value):
        r = buf[i]
        d = {"kind": LAUNCH_KINDS[r.kind], "states": r.states, "reg_qubits": r.reg_qubits, "phases": r.phases,
             "grid": r.grid, "jit": r.jit, "algorithmic_bytes": r.algorithmic_bytes}
        d.update({k: r.ops[j] for j, k in enumerate(OP_COUNT_NAMES)})
        out.append(d)
    return out


def nqs_set_option(h, option, value):
    _check(_lib().nqs_set_option(h, option, int(value)), "nqs_set_option")


def nqs_get_option(h, option):
    v = ctypes.c_int64()
    _check(_lib().nqs_get_option(h, option, ctypes.byref(v)), "nqs_get_option")
    return v.value


def nqs_autotune(h, psi, v, level, trials=2, stream=None):
    ps, vs = _as_state(psi), _as_state(v)
    out = nqs_result()
    _check(_lib().nqs_autotune(h, ctypes.byref(ps), ctypes.byref(vs), level, trials, ctypes.byref(out),
                               _stream_ptr(stream)), "nqs_autotune")
    return out.to_dict()


def nqs_set_profiling(h, on):
    _check(_lib().nqs_set_profiling(h, int(bool(on))), "nqs_set_profiling")


def nqs_get_kernel_stats(h, kind):
    s = nqs_kernel_stats()
    _check(_lib().nqs_get_kernel_stats(h, kind, ctypes.byref(s)), "nqs_get_kernel_stats")
    return {"launches": int(s.launches), "total_ms": s.total_ms, "algorithmic_bytes": s.algorithmic_bytes}


def nqs_reduced_matrix(phi, chi, n, qubit, r_out, scratch, scratch_bytes, stream=None):
    """phi, chi, r_out, scratch: device pointers (ints) or tensors."""
    def ptr(x):
        return x if isinstance(x, int) else x.data_ptr()
    _check(_lib().nqs_reduced_matrix(ctypes.c_void_p(ptr(phi)), ctypes.c_void_p(ptr(chi)), n, qubit,
                                     ctypes.c_void_p(ptr(r_out)), ctypes.c_void_p(ptr(scratch)),
                                     scratch_bytes, _stream_ptr(stream)), "nqs_reduced_matrix")


def nqs_reduced_matrix_noalloc(phi, chi, n, qubit, r_out, stream=None):
    """Allocation-free reduced matrix: phi, chi, r_out are device pointers
    (ints) or tensors; r_out must be device-accessible (8 doubles)."""
    def ptr(x):
        return x if isinstance(x, int) else x.data_ptr()
    _check(_lib().nqs_reduced_matrix_noalloc(ctypes.c_void_p(ptr(phi)), ctypes.c_void_p(ptr(chi)), n, qubit,
                                             ctypes.c_void_p(ptr(r_out)), _stream_ptr(stream)),
           "nqs_reduced_matrix_noalloc")


def nqs_reduced_matrix_scratch_bytes(n):
    return int(_lib().nqs_reduced_matrix_scratch_bytes(n))


def nqs_prepare_sets(h, psi, v, stream=None):
    ps, vs = _as_state(psi), _as_state(v)
    _check(_lib().nqs_prepare_sets(h, ctypes.byref(ps), ctypes.byref(vs), _stream_ptr(stream)), "nqs_prepare_sets")


def nqs_eval_sets(h, sets, stream=None):
    """sets: integer array [m x k] of ascending site indices; returns W [m]."""
    import numpy as np
    s = np.ascontiguousarray(sets, dtype=np.int32)
    if s.ndim == 1:
        s = s[:, None]
    W = np.zeros(s.shape[0], dtype=np.float64)
    _check(_lib().nqs_eval_sets(h, s.shape[1], s.ctypes.data, s.shape[0], W.ctypes.data, _stream_ptr(stream)),
           "nqs_eval_sets")
    return W


def _ptr(x):
    return ctypes.c_void_p(x if isinstance(x, int) else x.data_ptr())


def nqs_mlp_create(n_in, hidden=256, hidden_layers=3, seed=0):
    m = ctypes.c_void_p()
    _check(_lib().nqs_mlp_create(n_in, hidden, hidden_layers, seed, ctypes.byref(m)), "nqs_mlp_create")
    return m


def nqs_mlp_param_count(m):
    return int(_lib().nqs_mlp_param_count(m))


def nqs_mlp_get_params(m):
    import numpy as np
    out = np.zeros(nqs_mlp_param_count(m), dtype=np.float32)
    _check(_lib().nqs_mlp_get_params(m, out.ctypes.data, out.size), "nqs_mlp_get_params")
    return out


def nqs_mlp_set_params(m, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(_lib().nqs_mlp_set_params(m, p.ctypes.data, p.size), "nqs_mlp_set_params")


def nqs_mlp_forward(m, X, y, stream=None):
    """X: [batch x n_in] fp32 CUDA tensor; y: [batch] fp32 CUDA tensor (output)."""
    _check(_lib().nqs_mlp_forward(m, _ptr(X), X.shape[0], _ptr(y), _stream_ptr(stream)), "nqs_mlp_forward")


def nqs_mlp_loss_grad(m, X, y, stream=None):
    import numpy as np
    g = np.zeros(nqs_mlp_param_count(m), dtype=np.float32)
    loss = ctypes.c_double()
    _check(_lib().nqs_mlp_loss_grad(m, _ptr(X), _ptr(y), X.shape[0], ctypes.byref(loss), g.ctypes.data, g.size,
                                    _stream_ptr(stream)), "nqs_mlp_loss_grad")
    return loss.value, g


def nqs_mlp_train(m, X, y, batch, steps, lr, seed=0, stream=None):
    loss = ctypes.c_double()
    _check(_lib().nqs_mlp_train(m, _ptr(X), _ptr(y), X.shape[0], batch, steps, lr, seed, ctypes.byref(loss),
                                _stream_ptr(stream)), "nqs_mlp_train")
    return loss.value


def nqs_mlp_destroy(m):
    _lib().nqs_mlp_destroy(m)


def nqs_site_features(h, W1):
    import numpy as np
    w = np.ascontiguousarray(W1, dtype=np.float64)
    out = np.zeros((w.size, 4), dtype=np.float32)
    _check(_lib().nqs_site_features(h, w.ctypes.data, out.ctypes.data), "nqs_site_features")
    return out


def nqs_pair_training_data(h, feats, W2):
    import numpy as np
    f = np.ascontiguousarray(feats, dtype=np.float32)
    w2 = np.ascontiguousarray(W2, dtype=np.float64)
    cnt = ctypes.c_size_t()
    _check(_lib().nqs_pair_training_data(h, f.ctypes.data, w2.ctypes.data, None, None, 0, ctypes.byref(cnt)),
           "nqs_pair_training_data")
    X = np.zeros((cnt.value, 8), dtype=np.float32)
    y = np.zeros(cnt.value, dtype=np.float32)
    _check(_lib().nqs_pair_training_data(h, f.ctypes.data, w2.ctypes.data, X.ctypes.data, y.ctypes.data, cnt.value,
                                         ctypes.byref(cnt)), "nqs_pair_training_data")
    return X, y


def nqs_is_estimate(h, mlp, level, samples, alpha, seed, feats, W1, stream=None):
    import numpy as np
    f = None if feats is None else np.ascontiguousarray(feats, dtype=np.float32)
    w1 = np.ascontiguousarray(W1, dtype=np.float64)
    out = nqs_is_result()
    _check(_lib().nqs_is_estimate(h, mlp, level, samples, alpha, seed, None if f is None else f.ctypes.data,
                                  w1.ctypes.data, ctypes.byref(out), _stream_ptr(stream)), "nqs_is_estimate")
    return out.to_dict()


def nqs_is_proposal(h, mlp, level, alpha, feats, W1, stream=None):
    """Proposal probabilities over every site set of the level (canonical order)."""
    import numpy as np
    f = None if feats is None else np.ascontiguousarray(feats, dtype=np.float32)
    w1 = np.ascontiguousarray(W1, dtype=np.float64)
    cnt = ctypes.c_size_t()
    args = (h, mlp, level, alpha, None if f is None else f.ctypes.data, w1.ctypes.data)
    _check(_lib().nqs_is_proposal(*args, None, 0, ctypes.byref(cnt), _stream_ptr(stream)), "nqs_is_proposal")
    q = np.zeros(cnt.value, dtype=np.float64)
    _check(_lib().nqs_is_proposal(*args, q.ctypes.data, q.size, ctypes.byref(cnt), _stream_ptr(stream)),
           "nqs_is_proposal")
    return q


def nqs_selftest_bounded_wait(stream=None):
    """Status word written by the bounded-wait probe (NQS_ERR_DEVICE_TIMEOUT expected)."""
    st = ctypes.c_int(-1)
    _check(_lib().nqs_selftest_bounded_wait(ctypes.byref(st), _stream_ptr(stream)), "nqs_selftest_bounded_wait")
    return st.value


def nqs_destroy(h):
    _lib().nqs_destroy(h)


def nqs_strerror(code):
    return _lib().nqs_strerror(code).decode()


def nqs_version():
    return _lib().nqs_version().decode()


class NoisyCircuit:
    """Owns one handle: circuit text in, noise prepared, fidelity calls."""

    def __init__(self, ir_text, sites=None, flags=0):
        self.h = nqs_load_circuit(ir_text)
        try:
            nqs_prepare_noise(self.h, sites, flags)
        except Exception:
            nqs_destroy(self.h)
            raise

    def fidelity(self, psi, v, level, stream=None):
        return nqs_fidelity(self.h, psi, v, level, stream).to_dict()

    def term_values(self):
        return nqs_term_values(self.h)

    def info(self):
        return nqs_get_info(self.h)

    def close(self):
        if self.h is not None:
            nqs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
