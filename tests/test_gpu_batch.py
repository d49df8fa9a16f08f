"""Batched stepping: many uneven lattices in one persistent launch must give
the same result as each lattice stepped alone (same storage form), including
lattices that join and leave while others run, and the per-lattice residuals
of the batch's check steps must match the lone lattices'.  The same holds for
the batch's second mode, one launch per lattice on several streams.

FP64 results are bitwise identical.  The FP32-math forms agree to FP32
rounding (nvcc may fuse a different set of multiply-adds in the batch
kernel's force path): 1e-6 per population for FP32 storage, one FP16 ulp of
the stored deviation for F16S and F16R (whose stored remainder is smaller
than the deviation)."""
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


def _mix(seed=0):
    rng = np.random.default_rng(seed)
    probs = []
    for _ in range(4):
        L = int(rng.integers(12, 40))
        probs.append(wl.cavity(L, float(rng.uniform(50, 500)), float(rng.uniform(0.5, 1.5)),
                               dims=(L, int(rng.integers(10, 40)), int(rng.integers(6, 30)))))
    probs.append(wl.channel(int(rng.integers(16, 48)), 0.7, u_max=0.02, Re=20.0, nx=5, nz=3))
    probs.append(wl.Problem("box", 17, 9, 11, (wl.PERIODIC,) * 6, K=0.02, n=1.3,
                            body_force=(1e-5, -2e-6, 3e-6)))
    return probs


W = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)


def _lat(clbm, p, form, **kw):
    """A lattice of storage form `form`; "f16s_sr": F16S with stochastically
    rounded stores."""
    lat = clbm.Lattice(**p.kwargs(), dtype="f16s" if form == "f16s_sr" else form, **kw)
    if form == "f16s_sr":
        lat.set_rounding("stochastic")
    return lat


def _same(f, f_ref, dtype):
    if dtype == "f64":
        assert np.array_equal(f, f_ref), np.abs(f - f_ref).max()
    elif dtype == "f32":
        assert np.abs(f - f_ref).max() <= 1e-6
    elif dtype == "f16s_sr":
        # the same random bits alone and batched; where the two kernels' FP32
        # roundings differ, a stochastic rounding may fall the other way, and
        # the one-ulp difference then spreads to its neighbours' roundings
        dev = np.abs(f_ref - W[:, None, None, None])
        assert np.all(np.abs(f - f_ref) <= dev * 2.0 ** -7 + 1e-6)
        assert np.mean(np.abs(f - f_ref) > dev * 2.0 ** -10 + 1e-7) <= 1e-2
    else:
        dev = np.abs(f_ref - W[:, None, None, None])
        assert np.all(np.abs(f - f_ref) <= dev * 2.0 ** -10 + 1e-7)


def _set_mode(b, mode):
    if mode == "per_lattice":
        b.set_lattice_launch(32, 2, 5, 3)
    else:
        b.set_launch(32, 4, 1, 4)       # uncapped: the arithmetic of the lone default kernel


@pytest.mark.parametrize("mode", ["persistent", "per_lattice"])
@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s", "f16s_sr", "f16r"])
def test_batch_equals_alone(clbm, dtype, mode):
    if mode == "per_lattice" and dtype in ("f16r", "f16s_sr"):
        pytest.skip("stochastically rounding lattices take the persistent kernel")
    probs = _mix()
    steps = 257                      # graph chunks + single steps + odd count
    alone = []
    for p in probs:
        with _lat(clbm, p, dtype, check_interval=50) as lat:
            if mode == "per_lattice":
                lat.set_launch(32, 2, 5)       # the kernel the batch launches: bitwise FP64
            lat.step(steps)
            R, _ = lat.residual()
            alone.append((lat.get_state(), R, lat.mass()))
    lats = [_lat(clbm, p, dtype, check_interval=50) for p in probs]
    with clbm.Batch("f16s" if dtype == "f16s_sr" else dtype, capacity=8, check_interval=50) as b:
        _set_mode(b, mode)
        slots = [b.add(lt) for lt in lats]
        b.step(steps)
        al = b.stats_all()
        assert np.isnan(al["residual"][len(lats):]).all() and not al["diverged"].any()
        assert (al["steps"][len(lats):] == -1).all()
        for s, lt, (f_ref, R_ref, m_ref) in zip(slots, lats, alone):
            st = b.stats(s)
            assert st["residual"] == al["residual"][s] and st["mass"] == al["mass"][s]
            assert st["steps"] == al["steps"][s]
            assert st["steps"] == steps and not st["diverged"]
            f = lt.get_state()
            _same(f, f_ref, dtype)
            rtol = 1e-12 if dtype == "f64" else 1e-3 if dtype == "f16s_sr" else 1e-4
            assert abs(st["residual"] - R_ref) <= rtol * R_ref
            assert abs(st["mass"] - m_ref) <= 1e-9 * m_ref
    for lt in lats:
        lt.close()


@pytest.mark.parametrize("mode", ["persistent", "per_lattice"])
def test_batch_join_and_leave(clbm, mode):
    probs = _mix(1)
    counts = {}
    lats = [clbm.Lattice(**p.kwargs(), dtype="f32", check_interval=50) for p in probs]
    with clbm.Batch("f32", capacity=4, check_interval=50) as b:
        _set_mode(b, mode)
        s0 = b.add(lats[0])
        s1 = b.add(lats[1])
        b.step(120)
        b.add(lats[2])               # joins mid-interval
        b.step(75)
        b.remove(s0)                 # leaves; runs on alone for a while
        lats[0].step(33)
        b.add(lats[3])
        b.step(101)
        b.remove(s1)
        b.add(lats[0])               # re-joins
        b.step(40)
        for lt in lats[:4]:
            counts[id(lt)] = lt.steps_done()
    for p, lt in zip(probs[:4], lats[:4]):
        n = counts[id(lt)]
        with clbm.Lattice(**p.kwargs(), dtype="f32", check_interval=50) as ref:
            ref.step(n)
            _same(lt.get_state(), ref.get_state(), "f32")
        lt.close()
    assert counts[id(lats[0])] == 120 + 75 + 33 + 40
    assert counts[id(lats[3])] == 101 + 40


def test_batch_autotune_restores_state(clbm):
    probs = _mix(2)[:3]
    lats = [clbm.Lattice(**p.kwargs(), dtype="f32") for p in probs]
    with clbm.Batch("f32", capacity=4) as b:
        for lt in lats:
            b.add(lt)
        b.step(30)
        before = [lt.get_state() for lt in lats]
        info = b.autotune(3)
        assert info["us_per_step"] > 0
        assert info["mode"] == "per_lattice" or info["zc"] >= 1
        after = [lt.get_state() for lt in lats]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        assert all(lt.steps_done() == 30 for lt in lats)
        # the kept launch steps on correctly, whichever mode won
        b.step(70)
        b.apply_launch(info)
        b.step(1)
    for lt, p in zip(lats, probs):
        with clbm.Lattice(**p.kwargs(), dtype="f32") as ref:
            ref.step(101)
            _same(lt.get_state(), ref.get_state(), "f32")
        lt.close()


@pytest.mark.parametrize("dtype", ["f64", "f32", "f16s", "f16r"])
def test_default_launch_within_form_tolerance(clbm, dtype):
    # The batch's untuned default launch (register-capped for the FP32-math
    # forms) against the lattices alone: the velocity bar of each form.
    probs = _mix(3)
    lats = [clbm.Lattice(**p.kwargs(), dtype=dtype, check_interval=50) for p in probs]
    with clbm.Batch(dtype, capacity=8, check_interval=50) as b:
        for lt in lats:
            b.add(lt)
        b.step(300)
        got = [lt.fields()[1] for lt in lats]
    tol = {"f64": 1e-12, "f32": 1e-4, "f16s": 2e-3, "f16r": 2e-3}[dtype]
    for lt, p, u in zip(lats, probs, got):
        with clbm.Lattice(**p.kwargs(), dtype=dtype, check_interval=50) as ref:
            ref.step(300)
            u_ref = ref.fields()[1]
        assert np.linalg.norm(u - u_ref) <= tol * np.linalg.norm(u_ref)
        lt.close()


def test_lattice_launch_limits(clbm):
    lat = clbm.Lattice(**wl.cavity(10, 100.0, 1.0).kwargs(), dtype="f16r")
    with clbm.Batch("f16r", capacity=2) as b:
        with pytest.raises(clbm.CLBMError):
            b.set_lattice_launch(32, 2, 5, 2)
        b.add(lat)
        assert b.autotune(2)["mode"] == "persistent"
    with clbm.Batch("f32", capacity=2) as b:
        for bad in ((24, 2, 5, 2), (32, 2, 2, 2), (32, 2, 5, 0), (32, 2, 5, 17), (512, 1, 1, 2)):
            with pytest.raises(clbm.CLBMError):
                b.set_lattice_launch(*bad)
    lat.close()


def test_step_refused_while_batched(clbm):
    lat = clbm.Lattice(**wl.cavity(10, 100.0, 1.0).kwargs(), dtype="f32")
    with clbm.Batch("f32", capacity=2) as b:
        b.add(lat)
        with pytest.raises(clbm.CLBMError):
            lat.step(1)
    lat.step(1)                      # the batch is gone: stepping alone works again
    lat.close()


def _oracle_params(oracle, prob):
    return oracle.Params(nx=prob.nx, ny=prob.ny, nz=prob.nz, face=prob.face, K=prob.K, n=prob.n,
                         U=prob.U_lid, F=prob.body_force)


@pytest.mark.parametrize("mode", ["persistent", "per_lattice"])
def test_batch_members_vs_oracle(clbm, oracle, mode):
    # Every member of an FP64 batch (cavities, a forced channel and a forced
    # periodic box) against the oracle directly, not only through the lone
    # lattice: the FP64 bar, max|du| <= 1e-10 of the member's velocity scale
    # and the populations to 1e-12.
    probs = _mix(4)
    steps = 300
    lats = [clbm.Lattice(**p.kwargs(), dtype="f64", check_interval=50) for p in probs]
    with clbm.Batch("f64", capacity=8, check_interval=50) as b:
        _set_mode(b, mode)
        for lt in lats:
            b.add(lt)
        b.step(steps)
        got = [(lt.get_state(), lt.fields()[1]) for lt in lats]
    for lt, p, (f, u) in zip(lats, probs, got):
        op = _oracle_params(oracle, p)
        f_ref = oracle.run(op, oracle.rest_state(op), steps)
        _, u_ref, _ = oracle.fields(op, f_ref)
        scale = np.abs(u_ref).max()
        assert scale > 1e-6
        assert np.abs(u - u_ref).max() <= 1e-10 * scale
        assert np.abs(f - f_ref).max() <= 1e-12
        lt.close()
