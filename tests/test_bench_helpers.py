"""The benchmark's host-side helpers (CPU only): throughput aggregation, the FP32 peak model, the
accuracy comparisons against the oracle (single step and per replica of the batch), and the
consistency of the workload tables."""
import numpy as np

import bench


def test_aggregate_and_units():
    # 4 ranks x 100 steps in 50 ms (slowest rank): 8,000 steps/s; 2 fs per step
    assert abs(bench.aggregate_steps_per_s(50.0, 100, 4) - 8000.0) < 1e-9
    assert abs(bench.NS_PER_DAY_PER_STEP_PER_S - 2e-6 * 86400) < 1e-12
    assert abs(bench.alu_peak_tflops(2070.0) - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9


def test_accuracy_against_the_oracle_record():
    rng = np.random.default_rng(1)
    ref = {"q": rng.normal(size=50), "F_elyt": rng.normal(size=(20, 3)), "U": np.float64(-12.5),
           "H": np.float64(-20.0)}
    q = ref["q"] + np.r_[3e-7, np.zeros(49)]
    F = ref["F_elyt"] * 1.001
    acc = bench.accuracy_against(ref, {"q": np.r_[q, [9.0]], "F_elyt": np.r_[F.reshape(-1), [5.0, 5.0, 5.0]],
                                       "energy": np.array([-12.5 * (1 + 2e-6), -20.0, 0.0, 0.0])})
    assert abs(acc["dq_max_e"] - 3e-7) < 1e-15                    # trailing padding ignored
    assert abs(acc["force_rms_rel"] - 1e-3) < 1e-12
    assert abs(acc["energy_U_rel"] - 2e-6) < 1e-12 and acc["energy_H_rel"] == 0.0


def test_workload_tables_are_consistent():
    for name in bench.WORKLOADS:
        assert name in bench.GEOMETRY_NAME and name in bench.NCU_TRAFFIC_MIXED
        assert isinstance(bench.WORKLOADS[name][1], int)
    assert set(bench.MD_WORKLOADS) <= set(bench.WORKLOADS)
    w = bench.workload(bench.WORKLOADS["paper-md"][1], "paper-md")
    assert w.n_elec == 3024 and len(w.elyt_q[0]) == 2000 and bench.GEOMETRY_NAME["paper-md"] == "finite field"
    w = bench.workload(bench.WORKLOADS["paper"][1], "paper")
    assert w.n_elec == 3024 and w.grid == (40, 36, 168) and w.order == 5


def test_batched_accuracy_per_replica():
    rng = np.random.default_rng(2)
    q_ref = rng.normal(size=(3, 5))
    q = q_ref.copy()
    q[0, 2] += 1e-6
    q[2, 4] -= 2e-5
    acc = bench.batched_accuracy(q_ref, q.reshape(-1))
    assert acc["dq_max_e_per_replica"] == [1e-6, 0.0, 2e-5]
    assert abs(acc["dq_max_e"] - 2e-5) < 1e-15 and acc["replicas_within_1e-5_e"] == 2 and acc["replicas"] == 3


def test_precision_errors_against_the_float64_path():
    rng = np.random.default_rng(3)
    f64 = {"q": rng.normal(size=40), "F_elyt": rng.normal(size=(10, 3)), "F_elec": rng.normal(size=(40, 3)),
           "energy": np.array([-30.0, -31.0, 0.5, 1.0])}
    mix = {"q": f64["q"] + 2e-7, "F_elyt": f64["F_elyt"] * (1 + 1e-6), "F_elec": f64["F_elec"] * (1 - 3e-6),
           "energy": f64["energy"] * np.array([1 + 1e-7, 1 - 2e-7, 1.0, 1.0])}
    e = bench.precision_errors(mix, f64)
    assert abs(e["dq_max_e"] - 2e-7) < 1e-15
    assert abs(e["force_rms_rel_elyt"] - 1e-6) < 1e-12 and abs(e["force_rms_rel_elec"] - 3e-6) < 1e-12
    assert abs(e["energy_U_rel"] - 1e-7) < 1e-13 and abs(e["energy_H_rel"] - 2e-7) < 1e-13


def test_sampled_oracle_time_model():
    """A full step on p workers is a + b/p from the per-worker sample time T(f) = a + b f."""
    class Fake(bench.SampledOracle):
        def __init__(self):
            self.procs, self.pool, self.seed = 4, None, 0

        def sample(self, frac):
            return 0.5 + 800.0 * frac
    a, b = Fake().fit(0.001, 0.004)
    assert abs(a - 0.5) < 1e-9 and abs(b - 800.0) < 1e-6


def test_batched_oracle_charges_are_neutral_per_replica():
    q, step_s = bench.batched_oracle_charges(n_rep=2)
    assert q.shape == (2, 672) and np.all(np.isfinite(q))
    assert np.max(np.abs(q.sum(axis=1))) <= 1e-12
    assert np.max(np.abs(q[0] - q[1])) > 1e-3          # different electrolytes and dpsi (0 and 4 V)
    base = bench.batched_cpu_baseline(step_s, 8)
    assert step_s > 0 and base["unit"] == "replica-steps/s" and base["kind"] == "oracle"
    assert abs(base["value"] - 1.0 / step_s) <= 1e-4 and base["cores"] == 8


def test_plain_cell_oracle_comparison_and_baselines(tmp_path):
    """The 672-site plain cell's oracle children: the comparison against a result, and the oracle's
    step time on all cores and on one core."""
    import pickle
    import synth
    from oracle import cpm as ocpm
    w = synth.config_plain_ff()
    wfile = str(tmp_path / "plain.pkl")
    with open(wfile, "wb") as f:
        pickle.dump(w, f)
    out = ocpm.Reference(w).step(0)
    res = {"q": out["q"] + 1e-7, "F_elyt": out["F_elyt"], "energy": np.array([out["U"], out["H"], 0.0, 0.0])}
    obj = {}
    bench.finish_plain_cell(obj, res, wfile, str(tmp_path))
    acc = obj["accuracy"]["vs_oracle"]
    assert abs(acc["dq_max_e"] - 1e-7) < 1e-12 and acc["force_rms_rel"] == 0.0 and acc["energy_U_rel"] == 0.0
    base = obj["cpu_baseline"]
    assert base["kind"] == "oracle" and base["unit"] == "ns/day" and base["seconds_per_step"] > 0
    assert base["one_core"]["cores"] == 1 and base["one_core"]["seconds_per_step"] > 0
