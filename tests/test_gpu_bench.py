"""The benchmark's extra measurements run end to end on small cases through
the same code paths as the full ones: time to the first satisfying particle
(both workloads, all three forms), the learned-vs-uniform iteration count, and
the plain small-batch loop forms."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import bench
    import scenegen as sg
    from paper_2411_11833_b300.build import build_library
    build_library()
    import paper_2411_11833_b300 as pkg
    torch.cuda.set_device(0)
    net, info = bench.train_network(sg, harvest_scenes=4, train_steps=20)
    yield bench, sg, pkg, net, info
    net.close()


def test_time_to_first_satisfying_measurement_runs(env):
    bench, sg, pkg, net, info = env
    assert info["harvest_scenes"] == 4 and info["train_steps"] == 20
    out = bench.measure_ttfs(pkg, sg, net, seeds=[3002], budget_iters=100, pick_place_seeds=[20000])
    for part in ("stacking", "pick_place"):
        assert set(out[part]["forms"]) == {"plain_sequential_uniform", "batched_ik", "batched_learned_ik"}
        for form in out[part]["forms"].values():
            assert form["of"] == 1 and len(form["per_seed"]) == 1


def test_learned_vs_uniform_and_plain_loop_measurements_run(env):
    bench, sg, pkg, net, _ = env
    c4 = bench.measure_config4(pkg, sg, net, n_scenes=2, budget=50)
    assert c4["scenes"] == 2 and set(c4) >= {"uniform", "learned", "learned_over_uniform_mean_iters"}
    ps = bench.measure_plain_small(pkg, sg, reps=2, warmup=1)
    for k in ("host_loop_check_every_10", "cuda_graph_device_stop", "optimize_steps_device_stop",
              "one_fused_launch_no_stop"):
        assert ps[k] > 0
