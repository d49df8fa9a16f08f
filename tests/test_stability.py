"""Stability-limit sweep (Sec. 5, second study): the bisection logic on the
CPU with a runner whose thresholds are known, and on the GPU the FP64 batch
runner against a runner built on the oracle, on a small cavity where both
take the same stable / unstable decisions."""
import numpy as np
import pytest

from paper_1908_05396_gb300 import stability as st


def _fake_runner(thresholds, calls):
    def run(cases, U):
        calls.append(len(cases))
        return [u < thresholds[c] for c, u in zip(cases, U)]
    return run


def test_bisection_brackets_each_threshold():
    cases = [st.Case(1.0, 0.505), st.Case(0.8, 0.51), st.Case(1.5, 0.52, label="x"),
             st.Case(1.0, 0.55, rates=(1.0,) * 10, label="y")]
    thr = {cases[0]: 0.0731, cases[1]: 0.2, cases[2]: 0.9, cases[3]: 0.001}
    calls = []
    res = st.max_lid_velocity(cases, _fake_runner(thr, calls), u_hi=0.5, rounds=8)
    step = 0.5 / 2 ** 8
    for c, (lo, hi) in zip(cases, res):
        if thr[c] >= 0.5:
            assert (lo, hi) == (0.5, None)
        else:
            assert lo < thr[c] <= hi and abs((hi - lo) - step) < 1e-15
    # the first call tests u_hi for every case, later ones only the open cases
    assert calls == [4] + [3] * 8


def test_case_consistency_from_tau():
    # mu_p = c_s^2 (tau_p - 1/2), c_s^2 = 1/3 (Sec. 5)
    assert st.Case(1.0, 0.53).K == pytest.approx(0.01)
    assert st.Case(0.8, 0.5).K == 0.0


def _oracle_runner(oracle, L, steps, check):
    def run(cases, U):
        out = []
        for c, u in zip(cases, U):
            p = oracle.Params(nx=L, ny=L, nz=L, face=st.CAVITY_FACES, K=c.K, n=c.n,
                              U=(float(u), 0.0, 0.0), F=(0.0, 0.0, 0.0))
            if c.rates is not None:
                p.omega_high = {j: c.rates[j - 9] for j in range(9, 19)}
            f, ok = oracle.rest_state(p), True
            for _ in range(steps // check):
                f = oracle.run(p, f, check)
                rho, _, _ = oracle.fields(p, f)
                if not (np.all(np.isfinite(f)) and rho.min() >= 0.5 and rho.max() <= 2.0):
                    ok = False
                    break
            out.append(ok)
        return out
    return run


@pytest.mark.gpu
def test_stability_limit_f64_matches_oracle(oracle):
    from paper_1908_05396_gb300 import build
    build.build()
    over = (1.0,) + (1.5,) * 9
    cases = [st.Case(1.0, 0.505), st.Case(0.8, 0.505), st.Case(1.0, 0.505, rates=over, label="1.5")]
    L, steps, check, rounds, u_hi = 16, 3000, 500, 5, 0.25
    gpu = st.max_lid_velocity(cases, st.batch_runner(L, steps, "f64", check, check, autotune=False),
                              u_hi=u_hi, rounds=rounds)
    ref = st.max_lid_velocity(cases, _oracle_runner(oracle, L, steps, check), u_hi=u_hi,
                              rounds=rounds)
    step = u_hi / 2 ** rounds
    for g, r in zip(gpu, ref):
        assert r[1] is not None and r[1] - r[0] == pytest.approx(step)
        # the same decisions, up to a run whose blow-up falls within rounding
        # of a check: then the brackets are neighbours
        assert abs(g[0] - r[0]) <= step * (1 + 1e-9), (gpu, ref)
    # over-relaxed third and fourth orders lower the limit
    assert ref[2][1] <= ref[0][0]


def test_bisection_edge_cases():
    calls = []
    assert st.max_lid_velocity([], _fake_runner({}, calls), rounds=4) == []
    c = st.Case(1.0, 0.6)
    calls = []
    # stable at the upper end: no bisection runs
    assert st.max_lid_velocity([c], _fake_runner({c: 1.0}, calls), u_hi=0.25, rounds=6) == \
        [(0.25, None)]
    assert calls == [1]
    # unstable even near rest: the bracket closes on 0
    calls = []
    lo, hi = st.max_lid_velocity([c], _fake_runner({c: 0.0}, calls), u_hi=0.25, rounds=3)[0]
    assert lo == 0.0 and hi == 0.25 / 8 and calls == [1, 1, 1, 1]
