"""bench.py's CPU-baseline leg on CPU: the per-workload oracle timings keep
their keys and report the thread counts in force (tiny time budget)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_cpu_baseline_leg_per_workload(oracle_lib):
    import bench
    import oracle as O
    before = O.set_threads()
    d = bench.oracle_per_config(budget=0.02)
    assert O.set_threads() == before  # the thread count is restored
    assert d["kind"] == "oracle" and d["unit"] == "Mpoint-updates/s" and d["cores"] == before
    for name in ("acoustic2d_256", "acoustic3d_sample_64", "elastic2d_1024"):
        row = d[name]
        assert set(row) == {"fp64_1t", "fp16_emulation_1t", f"fp64_{before}t", f"fp16_emulation_{before}t"}
        assert all(v > 0 for v in row.values())


def test_pareto_marks_dominated_variants():
    import bench
    variants = {"a": {"value": 100.0}, "b": {"value": 90.0}, "c": {"value": 150.0}}
    acc = {"acoustic3d_recipe_256_cfl0.4_400": {
        "a": {"energy_drift_max": 1e-5, "rel_l2_vs_fp32": 1e-3},
        "b": {"energy_drift_max": 2e-5, "rel_l2_vs_fp32": 2e-3},     # worse than a in all three
        "c": {"energy_drift_max": 1e-3, "rel_l2_vs_fp32": 5e-3}}}
    rows = {r["variant"]: r for r in bench.pareto(variants, acc)}
    assert rows["a"]["pareto_optimal"] and rows["c"]["pareto_optimal"]
    assert not rows["b"]["pareto_optimal"]
