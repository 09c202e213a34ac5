"""ctypes binding of libtn.so (include/tn.h).  Argument marshalling only:
every step of the contraction runs in the library's CUDA kernels.

The functions keep the C names.  ``tn_build`` takes an instance dict
(n, q, edges, J, h) or the raw arrays and returns an opaque handle.
"""
import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtn.so")

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ECUDA, TN_ETIMEOUT, TN_EOVERFLOW, TN_ESTATE = range(7)
STATUS_NAMES = ["TN_OK", "TN_EINVAL", "TN_ENOMEM", "TN_ECUDA", "TN_ETIMEOUT", "TN_EOVERFLOW",
                "TN_ESTATE"]
TN_DTYPE_AUTO, TN_DTYPE_I32, TN_DTYPE_F32 = 0, 1, 2
TN_ORDER_SWEEP, TN_ORDER_GREEDY, TN_ORDER_TREE = 0, 1, 2

# every entry point declared in include/tn.h, with its ctypes signature
_SIGS = {
    "tn_build": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_int32, C.c_uint32]),
    "tn_max2sat_couplings": (C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_int32),
                                       C.c_void_p, C.c_void_p, C.c_void_p]),
    "tn_build_max2sat": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.c_int32, C.c_void_p,
                                   C.c_uint32]),
    "tn_sample": (C.c_int, [C.c_void_p, C.c_int32, C.c_uint64, C.c_void_p, C.c_void_p]),
    "tn_order": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_uint64, C.c_int32,
                           C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tn_leaf_count": (C.c_int32, [C.c_void_p]),
    "tn_set_couplings": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "tn_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tn_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tn_config": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "tn_forward": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "tn_backward": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tn_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    "tn_count": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32),
                           C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tn_energy_batch": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                  C.c_void_p]),
    "tn_config_batch": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                  C.c_void_p, C.c_void_p]),
    "tn_count_batch": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32,
                                 C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "tn_batch_run": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32,
                               C.c_void_p]),
    "tn_plan_info": (C.c_int, [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "tn_plan_launches": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "tn_set_profiling": (C.c_int, [C.c_void_p, C.c_int32]),
    "tn_profile_get": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int64),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]),
    "tn_profile_reset": (C.c_int, [C.c_void_p]),
    "tn_energy_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p]),
    "tn_maxplus_gemm": (C.c_int, [C.c_int32, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                  C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                  C.c_void_p]),
    "tn_last_error": (C.c_char_p, [C.c_void_p]),
    "tn_destroy": (None, [C.c_void_p]),
}

_lib = None


def lib():
    """Load libtn.so; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2008_06888_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class TNError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")


def _check(status, ctx):
    if status != TN_OK:
        msg = lib().tn_last_error(ctx)
        raise TNError(status, msg.decode() if msg else "")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def tn_build(inst, dtype=TN_DTYPE_AUTO):
    edges = np.ascontiguousarray(inst["edges"], dtype=np.int32).reshape(-1, 2)
    J = np.ascontiguousarray(inst["J"], dtype=np.float32)
    h = inst.get("h")
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    out = C.c_void_p()
    st = lib().tn_build(C.byref(out), int(inst["n"]), len(edges), _ptr(edges), _ptr(J), _ptr(h),
                        int(inst["q"]), dtype)
    _check(st, None)
    return out


def _lits(sat):
    return np.ascontiguousarray(sat["clauses"], dtype=np.int32).reshape(-1, 2)


def tn_max2sat_couplings(sat):
    """(edges (k, 2), J (k,), h (n,)) of the Ising network of a Max-2-SAT instance."""
    lits = _lits(sat)
    m, n = len(lits), int(sat["n"])
    edges = np.zeros((max(m, 1), 2), np.int32)
    J = np.zeros(max(m, 1), np.float32)
    h = np.zeros(n, np.float32)
    ne = C.c_int32()
    st = lib().tn_max2sat_couplings(n, m, _ptr(lits), C.byref(ne), _ptr(edges), _ptr(J), _ptr(h))
    _check(st, None)
    return edges[:ne.value].copy(), J[:ne.value].copy(), h


def tn_build_max2sat(sat, dtype=TN_DTYPE_AUTO):
    lits = _lits(sat)
    out = C.c_void_p()
    st = lib().tn_build_max2sat(C.byref(out), int(sat["n"]), len(lits), _ptr(lits), dtype)
    _check(st, None)
    return out


def tn_sample(ctx, n_spins, n_samples, seed=0, order=None):
    """(n_samples, n_spins) int8 array of ground states (+-1), drawn uniformly."""
    sigma = np.zeros((max(n_samples, 1), n_spins), np.int8)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int32).ravel()
    _check(lib().tn_sample(ctx, n_samples, seed, _ptr(o), _ptr(sigma)), ctx)
    return sigma[:n_samples]


def tn_order(ctx, method=TN_ORDER_GREEDY, seq=None, seed=0, restarts=16):
    s = None if seq is None else np.ascontiguousarray(seq, dtype=np.int32).ravel()
    pk, ops = C.c_double(), C.c_double()
    st = lib().tn_order(ctx, method, _ptr(s), 0 if s is None else len(s), seed, restarts,
                        C.byref(pk), C.byref(ops))
    _check(st, ctx)
    return pk.value, ops.value


def tn_leaf_count(ctx):
    return lib().tn_leaf_count(ctx)


def tn_set_couplings(ctx, J=None, h=None, on_device=False, n_edges=None, n_spins=None):
    """Host numpy arrays (on_device=False) or device pointers as ints / torch tensors."""
    if on_device:
        pj = None if J is None else C.c_void_p(J if isinstance(J, int) else J.data_ptr())
        ph = None if h is None else C.c_void_p(h if isinstance(h, int) else h.data_ptr())
        _check(lib().tn_set_couplings(ctx, pj, ph, 1), ctx)
        return
    J = None if J is None else np.ascontiguousarray(J, dtype=np.float32)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    _check(lib().tn_set_couplings(ctx, _ptr(J), _ptr(h), 0), ctx)


def tn_set_stream(ctx, stream_handle):
    _check(lib().tn_set_stream(ctx, C.c_void_p(stream_handle)), ctx)


def tn_energy(ctx):
    E = C.c_double()
    _check(lib().tn_energy(ctx, C.byref(E)), ctx)
    return E.value


def tn_config(ctx, n_spins):
    sigma = np.empty(n_spins, dtype=np.int8)
    E = C.c_double()
    _check(lib().tn_config(ctx, _ptr(sigma), C.byref(E)), ctx)
    return sigma, E.value


def tn_forward(ctx):
    E = C.c_double()
    _check(lib().tn_forward(ctx, C.byref(E)), ctx)
    return E.value


def tn_backward(ctx, n_spins=None):
    sigma = None if n_spins is None else np.empty(n_spins, dtype=np.int8)
    _check(lib().tn_backward(ctx, _ptr(sigma)), ctx)
    return sigma


def tn_gradient(ctx, n_edges, n_spins, dJ=None, dh=None):
    """Host arrays by default; pass torch CUDA tensors for device outputs."""
    if dJ is not None and hasattr(dJ, "data_ptr"):
        _check(lib().tn_gradient(ctx, C.c_void_p(dJ.data_ptr()),
                                 None if dh is None else C.c_void_p(dh.data_ptr()), 1), ctx)
        return dJ, dh
    gJ = np.empty(n_edges, np.float32)
    gh = np.empty(n_spins, np.float32)
    _check(lib().tn_gradient(ctx, _ptr(gJ), _ptr(gh), 0), ctx)
    return gJ, gh


def limbs_to_int(limbs):
    v = 0
    for x in reversed([int(t) for t in limbs]):
        v = (v << 64) | x
    return v


def tn_count(ctx, n_primes=3):
    cap = 16
    limbs = np.zeros(cap, dtype=np.uint64)
    nl = C.c_int32(cap)
    ln, E = C.c_double(), C.c_double()
    _check(lib().tn_count(ctx, n_primes, _ptr(limbs), C.byref(nl), C.byref(ln), C.byref(E)), ctx)
    return limbs_to_int(limbs[:nl.value]), ln.value, E.value


def _batch_ptrs(J, h):
    """(J ptr, h ptr, on_device, keep-alive) for numpy arrays or CUDA torch tensors."""
    if hasattr(J, "data_ptr"):
        return (C.c_void_p(J.data_ptr()), None if h is None else C.c_void_p(h.data_ptr()), 1,
                (J, h))
    J = np.ascontiguousarray(J, dtype=np.float32)
    h = None if h is None else np.ascontiguousarray(h, dtype=np.float32)
    return _ptr(J), _ptr(h), 0, (J, h)


def tn_energy_batch(ctx, J, h=None):
    """E_min of B coupling sets; J (B, n_edges), h (B, n_spins) or None."""
    B = int(J.shape[0])
    pj, ph, dev, keep = _batch_ptrs(J, h)
    E = np.zeros(B, np.float64)
    _check(lib().tn_energy_batch(ctx, B, pj, ph, dev, _ptr(E)), ctx)
    return E


def tn_config_batch(ctx, J, h=None, n_spins=None, want_sigma=True):
    B = int(J.shape[0])
    pj, ph, dev, keep = _batch_ptrs(J, h)
    E = np.zeros(B, np.float64)
    sigma = np.empty((B, n_spins), np.int8) if want_sigma else None
    _check(lib().tn_config_batch(ctx, B, pj, ph, dev, _ptr(E), _ptr(sigma)), ctx)
    return E, sigma


def tn_count_batch(ctx, J, h=None, n_primes=3, limbs_per=8):
    B = int(J.shape[0])
    pj, ph, dev, keep = _batch_ptrs(J, h)
    E = np.zeros(B, np.float64)
    limbs = np.zeros(B * limbs_per, np.uint64)
    status = np.zeros(B, np.int32)
    st = lib().tn_count_batch(ctx, B, pj, ph, dev, n_primes, _ptr(limbs), limbs_per, _ptr(E),
                              _ptr(status))
    if st not in (TN_OK, TN_EOVERFLOW):
        _check(st, ctx)
    counts = [limbs_to_int(limbs[k * limbs_per:(k + 1) * limbs_per]) if status[k] == 0 else None
              for k in range(B)]
    return E, counts, status


def tn_batch_run(ctxs, with_counts=True, limbs_per=4):
    B = len(ctxs)
    arr = (C.c_void_p * B)(*[c.value for c in ctxs])
    E = np.zeros(B, np.float64)
    limbs = np.zeros(B * limbs_per, np.uint64) if with_counts else None
    status = np.zeros(B, np.int32)
    st = lib().tn_batch_run(B, C.cast(arr, C.c_void_p), _ptr(E), _ptr(limbs), limbs_per,
                            _ptr(status))
    counts = None
    if with_counts:
        counts = [limbs_to_int(limbs[k * limbs_per:(k + 1) * limbs_per]) for k in range(B)]
    return st, E, counts, status


def tn_plan_info(ctx):
    ns, nt = C.c_int32(), C.c_int32()
    ae, ac, an = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().tn_plan_info(ctx, C.byref(ns), C.byref(nt), C.byref(ae), C.byref(ac),
                              C.byref(an)), ctx)
    return dict(n_steps=ns.value, n_transposes=nt.value, arena_energy=ae.value,
                arena_config=ac.value, arena_count=an.value)


KIND_NAMES = ["leaves", "transpose", "gate", "gemm", "trace", "other", "chain"]


def tn_plan_launches(ctx, mode="count"):
    """Kernel launches per kind (KIND_NAMES) of one execution of the lowered
    program: mode "energy", "config" or "count" (3 primes + witness)."""
    m = {"energy": 0, "config": 1, "count": 2}[mode]
    out = np.zeros(7, np.int64)
    _check(lib().tn_plan_launches(ctx, m, _ptr(out)), ctx)
    return dict(zip(KIND_NAMES, (int(x) for x in out)))


def tn_set_profiling(ctx, enable=True):
    _check(lib().tn_set_profiling(ctx, 1 if enable else 0), ctx)


def tn_profile_get(ctx, kind=-1):
    n = C.c_int64()
    ms, by, mac = C.c_double(), C.c_double(), C.c_double()
    _check(lib().tn_profile_get(ctx, kind, C.byref(n), C.byref(ms), C.byref(by), C.byref(mac)),
           ctx)
    return dict(launches=n.value, ms=ms.value, bytes=by.value, macs=mac.value)


def tn_profile_reset(ctx):
    _check(lib().tn_profile_reset(ctx), ctx)


def tn_energy_noalloc(ctx, J_ptr, h_ptr, E_ptr, stream_handle=0):
    """E_min into device memory without any device allocation (include/tn.h).

    J_ptr, h_ptr (may be None), E_ptr: device addresses as ints; the result
    lands in E_ptr asynchronously on the given stream.
    """
    _check(lib().tn_energy_noalloc(ctx, C.c_void_p(J_ptr), None if h_ptr is None else
                                   C.c_void_p(h_ptr), C.c_void_p(E_ptr),
                                   C.c_void_p(stream_handle)), ctx)


def tn_maxplus_gemm(A, B, Cout, transA=False, transB=False, stream_handle=0):
    """Cout[b] = max-plus product of A[b] and B[b] on CUDA torch tensors (float32 or int32).

    A: (batch, M, K) or, with transA, (batch, K, M); B: (batch, K, N) or, with
    transB, (batch, N, K); Cout: (batch, M, N).  Contiguous tensors.
    """
    import torch
    dt = TN_DTYPE_F32 if A.dtype == torch.float32 else TN_DTYPE_I32
    batch = A.shape[0]
    M = A.shape[2] if transA else A.shape[1]
    K = A.shape[1] if transA else A.shape[2]
    N = B.shape[1] if transB else B.shape[2]
    _check(lib().tn_maxplus_gemm(dt, batch, M, N, K, _tptr(A), int(transA), _tptr(B),
                                 int(transB), _tptr(Cout), C.c_void_p(stream_handle)), None)


def _tptr(t):
    return C.c_void_p(t.data_ptr())


def tn_last_error(ctx):
    m = lib().tn_last_error(ctx)
    return m.decode() if m else ""


def tn_destroy(ctx):
    if ctx is not None and ctx.value:
        lib().tn_destroy(ctx)


class SpinGlass:
    """Owns one context: build + order at construction, freed on close()."""

    def __init__(self, inst, order="greedy", seq=None, seed=0, restarts=16,
                 dtype=TN_DTYPE_AUTO):
        self.n = int(inst["n"])
        self.q = int(inst["q"])
        self.m = len(inst["edges"])
        self.ctx = tn_build(inst, dtype)
        method = {"greedy": TN_ORDER_GREEDY, "sweep": TN_ORDER_SWEEP, "tree": TN_ORDER_TREE}[order]
        self.log2_peak, self.log2_ops = tn_order(self.ctx, method, seq, seed, restarts)

    def energy(self):
        return tn_energy(self.ctx)

    def config(self):
        return tn_config(self.ctx, self.n)

    def forward(self):
        return tn_forward(self.ctx)

    def backward(self, want_sigma=True):
        return tn_backward(self.ctx, self.n if want_sigma else None)

    def count(self, n_primes=3):
        return tn_count(self.ctx, n_primes)

    def sample(self, n_samples, seed=0, order=None):
        """Ground states drawn uniformly (+-1 per spin), by conditional counts."""
        return tn_sample(self.ctx, self.n, n_samples, seed, order)

    def energy_batch(self, J, h=None):
        return tn_energy_batch(self.ctx, J, h)

    def config_batch(self, J, h=None, want_sigma=True):
        return tn_config_batch(self.ctx, J, h, self.n, want_sigma)

    def count_batch(self, J, h=None, n_primes=3, limbs_per=8):
        return tn_count_batch(self.ctx, J, h, n_primes, limbs_per)

    def gradient(self, dJ=None, dh=None):
        return tn_gradient(self.ctx, self.m, self.n, dJ, dh)

    def set_couplings(self, J=None, h=None, on_device=False):
        tn_set_couplings(self.ctx, J, h, on_device)

    def set_stream(self, handle):
        tn_set_stream(self.ctx, handle)

    def plan_info(self):
        return tn_plan_info(self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            tn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def state_indices(sigma, q):
        """Map tn_config output (+-1 for Ising) to state indices 0..q-1."""
        s = np.asarray(sigma, dtype=np.int64)
        return ((1 - s) // 2).astype(np.int8) if q == 2 else s.astype(np.int8)


class Max2SAT(SpinGlass):
    """A Max-2-SAT instance (n variables, clauses of signed 1-based literals)
    contracted by the library; every energy is the number of violated clauses
    and sigma = +1 means true.  The batched calls take the couplings that
    ``couplings(sat)`` gives for clause lists on the same variable pairs."""

    def __init__(self, sat, order="greedy", seq=None, seed=0, restarts=16):
        self.n = int(sat["n"])
        self.q = 2
        self.m = len(tn_max2sat_couplings(sat)[0])
        self.ctx = tn_build_max2sat(sat)
        method = {"greedy": TN_ORDER_GREEDY, "sweep": TN_ORDER_SWEEP, "tree": TN_ORDER_TREE}[order]
        self.log2_peak, self.log2_ops = tn_order(self.ctx, method, seq, seed, restarts)

    @staticmethod
    def couplings(sat):
        return tn_max2sat_couplings(sat)

    def assignment(self):
        """(x as uint8 0/1 with 1 = true, min number of violated clauses)."""
        sigma, cost = self.config()
        return (np.asarray(sigma) > 0).astype(np.uint8), cost


def ln_count_of(c):
    return math.log(c) if c > 0 else float("-inf")
