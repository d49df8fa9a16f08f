"""``clbm_step_noalloc``: the step for callers that cannot allocate.

Some callers cannot call cudaMalloc while they step (a fixed device-memory
pool reserved at start-up, a framework that already holds the whole device,
code that must not stall on the allocator).  They pass their own population,
velocity and result buffers, and the library keeps its reduction scratch in a
fixed array of its own.  This file checks that entry point against the
handle-based clbm_step() at its check steps, on two calls in a row, within
the tolerances of the other parity tests: FP64 1e-14 and FP32 1e-6 per
population, so the mass may differ by at most 19 N times that; F16S one
FP16 ulp of the stored deviation; the residual to 1e-12 (FP64), 1e-4 (FP32,
the FP32 velocity tolerance) and 1e-3 (F16S) relative.  It also checks that
a NaN planted from the host raises the divergence entry, on a stream of the
caller's.  It is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

from paper_1908_05396_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-14, "f32": 1e-6}
RTOL = {"f64": 1e-12, "f32": 1e-4, "f16s": 1e-3}
W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


@pytest.fixture(scope="module")
def clbm():
    from paper_1908_05396_gb300 import build
    build.build()
    from paper_1908_05396_gb300 import clbm as c
    c.lib()
    return c


def _stored(torch, dev, dtype):
    """Deviations f - w rho0 as the storage form holds them (F16S: x1024,
    rounded to FP32 and then to FP16, both to nearest even)."""
    if dtype == "f16s":
        h = (dev.astype(np.float32) * np.float32(1024.0)).astype(np.float16)
        return torch.tensor(h.reshape(-1), device="cuda")
    tdt = torch.float64 if dtype == "f64" else torch.float32
    return torch.tensor(dev.reshape(-1), dtype=tdt, device="cuda")


def _decoded(buf, dtype, shape):
    d = buf.double().cpu().numpy().reshape((19,) + shape)
    return d / 1024.0 if dtype == "f16s" else d


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s"])
def test_noalloc_matches_check_steps(clbm, dtype):
    torch = pytest.importorskip("torch")
    tdt = torch.float64 if dtype == "f64" else torch.float32
    prob = wl.Problem("mixed", 37, 21, 11, (wl.WALL, wl.WALL, wl.WALL, wl.LID, wl.PERIODIC, wl.PERIODIC),
                      K=0.01, n=0.7, U_lid=(0.04, 0.0, 0.02), body_force=(1e-5, 0.0, -2e-6))
    shape = (prob.nz, prob.ny, prob.nx)
    N = prob.N
    r = wl.noise((19,) + shape, seed=21, amp=0.03)

    # Existing entry point: a handle whose every step is a check step.
    lat = clbm.Lattice(**prob.kwargs(), dtype=dtype, check_interval=1)
    rest = lat.get_state()
    f0 = rest * (1 + r)
    lat.set_state(f0)

    # Caller-owned buffers for the new entry point (dense layout).
    a = _stored(torch, f0 - rest, dtype)
    b = torch.zeros_like(a)
    u_prev = torch.zeros(3 * N, dtype=tdt, device="cuda")
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    kw = dict(nx=prob.nx, ny=prob.ny, nz=prob.nz, face=prob.face, K=prob.K, n=prob.n,
              U_lid=prob.U_lid, body_force=prob.body_force, dtype=dtype)

    for call, (src, dst) in enumerate([(a, b), (b, a)]):
        rc = clbm.step_noalloc(**kw, src=src.data_ptr(), dst=dst.data_ptr(),
                               u_prev=u_prev.data_ptr(), stats=stats.data_ptr())
        assert rc == clbm.OK, clbm.last_error()
        torch.cuda.synchronize()
        lat.step(1)
        f_ref = lat.get_state()
        f_new = _decoded(dst, dtype, shape) + rest
        if dtype == "f16s":
            dev = np.abs(f_ref - W[:, None, None, None])
            assert np.all(np.abs(f_new - f_ref) <= dev * 2.0 ** -10 + 1e-7)
        else:
            assert np.abs(f_new - f_ref).max() <= TOL[dtype]
        s = stats.cpu().numpy()
        assert s[3] == 0.0
        assert abs(N * 1.0 + s[2] - lat.mass()) <= 19 * N * TOL.get(dtype, 1e-6)
        R_ref, rc_ref = lat.residual()
        assert rc_ref == clbm.OK
        if call == 0:
            assert math.isinf(R_ref)
        else:
            R = math.sqrt(s[0]) / math.sqrt(s[1])     # check interval 1
            assert abs(R - R_ref) <= RTOL[dtype] * R_ref
    lat.close()


def test_noalloc_rejects_lattice_beyond_scratch(clbm):
    torch = pytest.importorskip("torch")
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = buf.data_ptr()
    prob = wl.cavity(256, 100.0, 1.0)
    rc = clbm.step_noalloc(nx=256, ny=256, nz=256, face=prob.face, K=prob.K, n=1.0,
                           U_lid=prob.U_lid, body_force=None, dtype="f32",
                           src=p, dst=p + 64, u_prev=p + 128, stats=p + 192)
    assert rc == clbm.ERR_ARG
    assert "65536" in clbm.last_error()


def test_noalloc_reports_divergence_on_caller_stream(clbm):
    # A NaN population planted from the host: the step reports it in the
    # divergence entry of stats, on a stream the caller owns.
    torch = pytest.importorskip("torch")
    prob = wl.cavity(20, 100.0, 0.8, dims=(20, 18, 10))
    shape = (prob.nz, prob.ny, prob.nx)
    N = prob.N
    dev = np.zeros((19,) + shape)
    dev[3, 4, 5, 6] = np.nan
    a = _stored(torch, dev, "f32")
    b = torch.zeros_like(a)
    u_prev = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    stats = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    kw = dict(nx=prob.nx, ny=prob.ny, nz=prob.nz, face=prob.face, K=prob.K, n=prob.n,
              U_lid=prob.U_lid, body_force=None, dtype="f32")
    torch.cuda.synchronize()
    rc = clbm.step_noalloc(**kw, src=a.data_ptr(), dst=b.data_ptr(), u_prev=u_prev.data_ptr(),
                           stats=stats.data_ptr(), stream=st.cuda_stream)
    assert rc == clbm.OK, clbm.last_error()
    st.synchronize()
    assert stats.cpu().numpy()[3] == 1.0
    # the next call on a clean state clears it again (the scratch keeps the
    # last call's partial sums, which each call overwrites)
    a.zero_()
    torch.cuda.synchronize()
    rc = clbm.step_noalloc(**kw, src=a.data_ptr(), dst=b.data_ptr(), u_prev=u_prev.data_ptr(),
                           stats=stats.data_ptr(), stream=st.cuda_stream)
    assert rc == clbm.OK, clbm.last_error()
    st.synchronize()
    s = stats.cpu().numpy()
    assert s[3] == 0.0 and abs(s[2]) <= 1e-9
