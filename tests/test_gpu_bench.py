"""The benchmark's time-to-first-satisfying-particle measurement runs end to
end through the search forms it reports (a small harvest, a short training
and one seed: the same code path as the full measurement)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_time_to_first_satisfying_measurement_runs():
    import bench
    import scenegen as sg
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as pkg
    torch.cuda.set_device(0)
    out = bench.measure_ttfs(pkg, sg, seeds=[3002], budget_iters=100, harvest_scenes=4, train_steps=20)
    assert set(out["forms"]) == {"plain_sequential_uniform", "batched_ik", "batched_learned_ik"}
    for form in out["forms"].values():
        assert form["of"] == 1 and len(form["per_seed"]) == 1
