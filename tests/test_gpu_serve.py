"""Continuous-batching server: results are the same alone and in the mix,
admission respects the memory budget, and unfinished work is cancelled on
shutdown.  Tolerances are the per-form ones of the parity tests (FP64
exact, FP32 1e-6 per population-derived field, F16S and F16R one FP16 ulp)."""
import time

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
    return c


def _requests():
    # small cavities and channels that settle within a few thousand steps
    reqs = []
    for L, Re, n in [(12, 20.0, 0.8), (16, 30.0, 1.2), (10, 15.0, 1.0), (14, 25.0, 0.6)]:
        p = wl.cavity(L, Re, n, dims=(L, L + 2, L - 2))
        reqs.append(p)
    reqs.append(wl.channel(20, 0.7, u_max=0.01, Re=2.0, nx=4, nz=3))
    return reqs


def _submit(srv, p, tol):
    return srv.submit(**p.kwargs(), tol=tol, max_steps=6000, keep_fields=True)


def _server(clbm, form, **kw):
    """A server of storage form `form`; "f16s_sr": F16S lattices with
    stochastically rounded stores."""
    srv = clbm.Server("f16s" if form == "f16s_sr" else form, **kw)
    if form == "f16s_sr":
        srv.set_rounding("stochastic")
    return srv


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s", "f16s_sr", "f16r"])
def test_same_result_alone_and_in_the_mix(clbm, dtype):
    probs = _requests()
    tol = {"f16s": 1e-4, "f16s_sr": 1e-4, "f16r": 1e-5}.get(dtype, 1e-6)
    mixed = {}
    with _server(clbm, dtype, hbm_budget_bytes=4e9, max_active=3, check_interval=50) as srv:
        ids = []
        for k, p in enumerate(probs):
            ids.append(_submit(srv, p, tol))
            time.sleep(0.01 * k)                  # staggered arrivals
        for k, rid in enumerate(ids):
            res = srv.wait(rid, timeout=120)
            mixed[k] = (res, srv.fields(rid))
    for k, p in enumerate(probs):
        with _server(clbm, dtype, hbm_budget_bytes=4e9, max_active=1, check_interval=50) as srv:
            rid = _submit(srv, p, tol)
            res = srv.wait(rid, timeout=120)
            rho, u, gd = srv.fields(rid)
        res_m, (rho_m, u_m, gd_m) = mixed[k]
        assert res["status"] == res_m["status"] and res["steps"] == res_m["steps"], (res, res_m)
        assert res["status"] in (0, 1)
        if dtype == "f64":
            assert np.array_equal(u, u_m) and np.array_equal(rho, rho_m)
        else:
            scale = np.abs(u).max()
            utol = 1e-6 if dtype == "f32" else 1e-3
            assert np.abs(u - u_m).max() <= utol * scale


def test_admission_respects_budget(clbm):
    probs = [wl.cavity(24, 50.0, 1.0) for _ in range(6)]
    one = 2 * 19 * (32 * 24 * 24) * 4 + 3 * 32 * 24 * 24 * 4 + 4096   # FP32 bytes of one
    budget = 2.5 * one
    with clbm.Server("f32", hbm_budget_bytes=budget, max_active=8, check_interval=50) as srv:
        ids = [srv.submit(**p.kwargs(), tol=0.0, max_steps=400) for p in probs]
        peak = 0
        while True:
            st = srv.info()
            peak = max(peak, st["active"])
            assert st["used_bytes"] <= budget
            if st["done"] == len(ids):
                break
            time.sleep(0.002)
        res = [srv.wait(i, timeout=60) for i in ids]
    assert peak <= 2
    assert all(r["status"] == 1 and r["steps"] == 400 for r in res)   # MAX_STEPS
    # a request larger than the whole budget is rejected, not queued forever
    with clbm.Server("f32", hbm_budget_bytes=1e6, max_active=2) as srv:
        rid = srv.submit(**wl.cavity(40, 50.0, 1.0).kwargs(), tol=1e-6, max_steps=100)
        assert srv.wait(rid, timeout=30)["status"] == 4


def test_destroy_cancels_unfinished(clbm):
    srv = clbm.Server("f32", hbm_budget_bytes=4e9, max_active=1, check_interval=50)
    ids = [srv.submit(**wl.cavity(20, 100.0, 1.0).kwargs(), tol=0.0, max_steps=10 ** 9)
           for _ in range(3)]
    time.sleep(0.2)
    info = srv.info()
    assert info["active"] == 1 and info["queued"] == 2
    srv.close()


def test_served_results_vs_oracle(clbm, oracle):
    # FP64 requests served together (two slots for three requests, so one
    # joins while the others run), each stopped by its step cap, against the
    # oracle run for the same number of steps: max|du| <= 1e-10 of the
    # request's velocity scale.
    probs = _requests()[:2] + [_requests()[4]]
    caps = [700, 900, 500]
    with clbm.Server("f64", hbm_budget_bytes=4e9, max_active=2, check_interval=50) as srv:
        ids = [srv.submit(**p.kwargs(), tol=0.0, max_steps=c, keep_fields=True)
               for p, c in zip(probs, caps)]
        res = [srv.wait(rid, timeout=120) for rid in ids]
        fields = [srv.fields(rid) for rid in ids]
    for p, c, r, (rho, u, _) in zip(probs, caps, res, fields):
        assert r["status"] == 1 and r["steps"] == c          # the step cap
        op = oracle.Params(nx=p.nx, ny=p.ny, nz=p.nz, face=p.face, K=p.K, n=p.n, U=p.U_lid,
                           F=p.body_force)
        f_ref = oracle.run(op, oracle.rest_state(op), c)
        rho_ref, u_ref, _ = oracle.fields(op, f_ref)
        scale = np.abs(u_ref).max()
        assert scale > 1e-6
        assert np.abs(u - u_ref).max() <= 1e-10 * scale
        assert np.abs(rho - rho_ref).max() <= 1e-12
