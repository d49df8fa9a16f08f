"""Host-side logic of bench.py that needs no GPU: the serving statistics,
the reference arm's slab size and the profile-note lookup."""
import types

import bench


def test_latency_stats():
    clbm = types.SimpleNamespace(SOLVE_STATUS={0: "converged", 1: "max_steps", 3: "diverged"})
    res = [{"t_submit": 0.0, "t_done": 1.0, "status": 0, "steps": 100},
           {"t_submit": 0.5, "t_done": 2.5, "status": 1, "steps": 300},
           {"t_submit": 1.0, "t_done": 5.0, "status": 3, "steps": 200}]
    out = bench._latency_stats(clbm, res)
    assert out["makespan_s"] == 5.0
    assert abs(out["solves_per_s"] - 3 / 5.0) < 1e-15
    assert out["p50_latency_s"] == 2.0 and out["p99_latency_s"] == 4.0
    assert out["status"] == {"converged": 1, "max_steps": 1, "diverged": 1}
    assert out["mean_steps"] == 200.0


def test_reference_slab_uses_every_core():
    # the oracle's OpenMP loop runs over z-planes: one plane per core
    assert bench.ref_slab(16) == 16
    assert bench.ref_slab(72) == 72
    assert bench.ref_slab(4) == 16
    assert bench.ref_slab(1000) == bench.L_BENCH


def test_profile_notes_match_only_current_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda form="f32": "abc123")
    (tmp_path / "profiles" / "traffic.txt").write_text(
        "# comment\nstep_kernel<float> abc123 276000000\nstep_kernel<float> old999 1\n")
    (tmp_path / "profiles" / "fp64_ops.txt").write_text("step_kernel<double> abc123 1.5 2.5 3.0\n")
    assert bench._traffic_note("step_kernel<float>") == 276000000.0
    assert bench._traffic_note("step_kernel<half>") is None
    assert bench._fp64_ops_note("step_kernel<double>") == [1.5, 2.5, 3.0]


def test_form_names():
    import bench
    assert bench.form_spec("f16s_sr") == ("f16s", False, "stochastic")
    assert bench.form_spec("f32_inplace") == ("f32", True, None)
    assert bench.form_spec("f16r") == ("f16r", False, None)


def test_serving_bench_headline_and_forms(monkeypatch):
    import types
    import numpy as np
    import bench
    fake = types.SimpleNamespace(SOLVE_STATUS={0: "converged", 1: "max_steps", 3: "diverged"})
    trace = [types.SimpleNamespace(problem=None, arrival=0.1 * k) for k in range(3)]
    u = np.ones((3, 2, 2, 2))

    def serve(clbm, tr, dtype, tol, cap, plateau, check):
        res = [{"t_submit": 0.1 * k, "t_done": 1.0 + k, "status": 0, "steps": 100} for k in range(3)]
        return res, [u * (1 + 1e-4 * (dtype != "f64")) for _ in tr], {"lattice_updates": 1e6,
                                                                       "busy_seconds": 1.0}

    monkeypatch.setattr(bench, "_serve_trace", serve)
    monkeypatch.setattr(bench, "_solve_alone", lambda *a: ("converged", 100, u))
    out = bench._serving_bench(fake, trace, 1e-7, 100, 20, 10, "three requests")
    assert out["form"] == "f16r"
    assert set(out["other_forms"]) == {"f16s_sr", "f16s", "f32"}
    assert out["velocity_l2_vs_f64"]["within_bar"] == "3/3 at L2 <= 0.002"
    assert out["speedup_vs_sequential_f64"] > 0
