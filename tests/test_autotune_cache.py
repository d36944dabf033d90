"""Host logic of the autotuner's persistent cache (CPU only, a scripted scene)."""
import json

from paper_2411_11833_b300 import autotune


class FakeScene:
    def __init__(self):
        self.device = 0
        self.shape = dict(n_joints=7, n_spheres=35, n_boxes=6, spheres_per_box=8, n_obs=8, n_surf=1)
        self.timed, self.installed = 0, []

    def problem_info(self, pid):
        return 126, 67, [0, 1, 2, 4, 6] * 13 + [7, 7]

    def autotune(self, pids, trial_steps):
        self.timed += 1
        return 2, 6, 1.5

    def set_tuning(self, pids, lanes, warps):
        self.installed.append((tuple(pids), lanes, warps))


def test_tune_times_once_then_installs_from_the_file(tmp_path):
    path = str(tmp_path / "at.json")
    sc = FakeScene()
    r1 = autotune.tune(sc, [0], [4096], path=path, gpu=("B300", 148))
    assert sc.timed == 1 and not r1["cached"] and (r1["lanes"], r1["warps"]) == (2, 6)
    r2 = autotune.tune(sc, [0], [4096], path=path, gpu=("B300", 148))
    assert sc.timed == 1 and r2["cached"] and sc.installed == [((0,), 2, 6)]
    # another GPU or another batch size is another key
    autotune.tune(sc, [0], [4096], path=path, gpu=("B200", 148))
    autotune.tune(sc, [0], [2048], path=path, gpu=("B300", 148))
    assert sc.timed == 3
    assert len(json.load(open(path))) == 3


def test_signature_depends_on_the_work():
    s = dict(n_joints=7, n_spheres=35)
    a = autotune.signature(s, [(126, [0, 1], 4096)])
    assert a == autotune.signature(dict(s), [(126, [0, 1], 4096)])
    assert a != autotune.signature(s, [(126, [0, 1], 4095)])
    assert a != autotune.signature(dict(s, n_spheres=100), [(126, [0, 1], 4096)])
    assert a != autotune.signature(s, [(126, [0, 2], 4096)])


def test_unreadable_cache_is_ignored(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    assert autotune.load(str(p)) == {}
    sc = FakeScene()
    autotune.tune(sc, [1], [100], path=str(p), gpu=("B300", 148))
    assert sc.timed == 1 and len(json.load(open(p))) == 1
