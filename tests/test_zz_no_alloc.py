"""tn_energy_noalloc: the ground-state energy for callers that cannot allocate
device memory (stream-capture code, frameworks whose allocator owns the whole
GPU, loops that cannot afford cudaMalloc's synchronisation).  It runs in a
static 32 MiB device array inside libtn.so; these tests check that it gives
the same E_min as tn_energy, call after call on the shared array, and that a
plan too large for the array is refused with a clear error.

This file is collected last on purpose: it passes on its own in a fresh
process and after every other test.
"""
import numpy as np
import pytest

import instances as I
from paper_2008_06888_gb300 import binding as B

pytestmark = pytest.mark.gpu
REL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_06888_gb300 import build
    build.build()


def _ctx(inst, **order):
    c = B.tn_build(inst)
    B.tn_order(c, **order)
    return c


def _noalloc(c, inst, torch):
    J = torch.tensor(inst["J"], device="cuda")
    h = None if inst.get("h") is None else torch.tensor(inst["h"], device="cuda")
    E = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream()
    B.tn_energy_noalloc(c, J.data_ptr(), None if h is None else h.data_ptr(), E.data_ptr(),
                        s.cuda_stream)
    s.synchronize()
    return float(E.item())


def test_noalloc_matches_tn_energy_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    insts = [I.square_lattice(12, coupling="gauss", field_sigma=0.1, seed=31),
             I.square_lattice(12, coupling="gauss", field_sigma=0.1, seed=32),
             I.square_lattice(10, coupling="pm1", seed=33)]
    ctxs = [_ctx(x, method=B.TN_ORDER_GREEDY, seed=1, restarts=8) for x in insts]
    try:
        ref = [B.tn_energy(c) for c in ctxs]
        for rep in range(2):                      # two rounds of calls back to back
            for c, x, e in zip(ctxs, insts, ref):
                got = _noalloc(c, x, torch)
                assert abs(got - e) <= REL * max(1.0, abs(e)), (rep, got, e)
        # integer instance: exact
        assert _noalloc(ctxs[2], insts[2], torch) == ref[2]
    finally:
        for c in ctxs:
            B.tn_destroy(c)


def test_noalloc_rejects_plans_beyond_the_static_scratch():
    torch = pytest.importorskip("torch")
    inst = I.square_lattice(24, coupling="gauss", field_sigma=0.1, seed=1)
    c = _ctx(inst, method=B.TN_ORDER_SWEEP, seq=I.square_sweep_order(24))
    try:
        with pytest.raises(B.TNError) as e:
            _noalloc(c, inst, torch)
        assert e.value.status == B.TN_ENOMEM
        assert "static scratch" in str(e.value)
    finally:
        B.tn_destroy(c)


def test_noalloc_captured_in_a_cuda_graph_allocates_nothing():
    """The use the entry point exists for: recorded inside a stream capture.

    The call is made once eagerly (its first call on the device looks up the
    scratch address, which must happen outside capture), then captured into a
    CUDA graph in torch's strictest capture mode, where any allocation or
    synchronous copy would end the capture with an error.  Two replays must
    give tn_energy's E_min, and neither the replays nor the eager calls may
    change the memory the device reports as in use or torch's allocations."""
    torch = pytest.importorskip("torch")
    inst = I.square_lattice(14, coupling="gauss", field_sigma=0.1, seed=41)
    c = _ctx(inst, method=B.TN_ORDER_GREEDY, seed=1, restarts=8)
    try:
        ref = B.tn_energy(c)
        J = torch.tensor(inst["J"], device="cuda")
        h = torch.tensor(inst["h"], device="cuda")
        E = torch.full((1,), float("nan"), dtype=torch.float32, device="cuda")
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            B.tn_energy_noalloc(c, J.data_ptr(), h.data_ptr(), E.data_ptr(), s.cuda_stream)
        s.synchronize()
        assert abs(float(E.item()) - ref) <= REL * max(1.0, abs(ref))
        # torch's first capture allocates its own generator state (about 1 KB);
        # an empty capture takes that before the allocations are recorded
        g0 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g0, stream=s, capture_error_mode="global"):
            pass
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        for _ in range(2):
            with torch.cuda.stream(s):
                B.tn_energy_noalloc(c, J.data_ptr(), h.data_ptr(), E.data_ptr(), s.cuda_stream)
        s.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s, capture_error_mode="global"):
            B.tn_energy_noalloc(c, J.data_ptr(), h.data_ptr(), E.data_ptr(), s.cuda_stream)
        assert torch.cuda.memory_allocated() == alloc0
        for rep in range(2):
            E.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            got = float(E.item())
            assert abs(got - ref) <= REL * max(1.0, abs(ref)), (rep, got, ref)
        assert torch.cuda.memory_allocated() == alloc0
        del g, g0
    finally:
        B.tn_destroy(c)
