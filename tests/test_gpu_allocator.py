"""External device allocator (clbm_set_allocator): lattices created under
PyTorch's caching allocator take their buffers from it and give them back on
destroy, step exactly as lattices on cudaMalloc, and the library refuses a
misaligned pointer (after handing it back) and reports a failed allocation."""
import numpy as np
import pytest

from paper_1908_05396_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def clbm():
    from paper_1908_05396_gb300 import build
    build.build()
    from paper_1908_05396_gb300 import clbm as c
    c.lib()
    yield c
    c.set_allocator()


def _counting_torch(torch, log, offset=0):
    held = {}

    def alloc(nbytes, device, stream):
        p = torch.cuda.caching_allocator_alloc(nbytes + offset, device, stream)
        held[p + offset] = p
        log.append(("alloc", p + offset, nbytes, stream))
        return p + offset

    def free(ptr, nbytes, device, stream):
        log.append(("free", ptr, nbytes, stream))
        torch.cuda.caching_allocator_delete(held.pop(ptr))
    return alloc, free, held


@pytest.mark.parametrize("dtype", ["f32", "f16r"])
def test_lattice_on_torch_allocator(clbm, dtype):
    import torch
    prob = wl.cavity(40, 200.0, 0.7, dims=(40, 36, 20))
    log = []
    alloc, free, held = _counting_torch(torch, log)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    clbm.set_allocator(alloc, free)
    try:
        lat = clbm.Lattice(**prob.kwargs(), dtype=dtype)
    finally:
        clbm.set_allocator()
    with clbm.Lattice(**prob.kwargs(), dtype=dtype) as ref:     # on cudaMalloc
        lat.step(200)
        ref.step(200)
        assert np.array_equal(lat.get_state(), ref.get_state())
        R, R_ref = lat.residual()[0], ref.residual()[0]
        assert abs(R - R_ref) <= 1e-12 * R_ref      # FP64 sums in atomic (unordered) adds
    n_alloc = sum(1 for e in log if e[0] == "alloc")
    # populations (two buffers), F16R references (two), check velocities, sums
    assert n_alloc == (6 if dtype == "f16r" else 4)
    assert all(p % 256 == 0 for _, p, _, _ in log)
    assert len({e[3] for e in log}) == 1 and log[0][3] != 0      # the lattice's own stream
    held_bytes = torch.cuda.memory_allocated() - base
    assert held_bytes >= sum(e[2] for e in log)
    lat.close()
    frees = [e for e in log if e[0] == "free"]
    assert sorted((p, n) for _, p, n, _ in frees) == \
        sorted((p, n) for k, p, n, _ in log if k == "alloc")
    assert not held
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base


def test_allocator_errors(clbm):
    import torch
    prob = wl.cavity(16, 100.0, 1.0)
    log = []
    alloc, free, held = _counting_torch(torch, log, offset=16)     # misaligned by 16 B
    clbm.set_allocator(alloc, free)
    try:
        with pytest.raises(clbm.CLBMError) as ei:
            clbm.Lattice(**prob.kwargs(), dtype="f32")
        assert ei.value.code == clbm.ERR_ARG
        assert not held                              # handed back
        clbm.set_allocator(lambda n, d, s: 0, lambda p, n, d, s: None)
        with pytest.raises(clbm.CLBMError) as ei:
            clbm.Lattice(**prob.kwargs(), dtype="f32")
        assert ei.value.code == clbm.ERR_OOM
    finally:
        clbm.set_allocator()
    with clbm.Lattice(**prob.kwargs(), dtype="f32") as lat:   # cudaMalloc again
        lat.step(10)
    with pytest.raises(ValueError):
        clbm.set_allocator(alloc, None)
