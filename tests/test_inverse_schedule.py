"""Host logic of the staged inverse loop (no GPU)."""
import numpy as np

from paper_1910_05200_gb300 import inverse as INV
from paper_1910_05200_gb300 import synthetic as S


def test_schedule_covers_every_iteration_in_order():
    for n in (1, 7, 100, 500):
        st = INV.schedule(n)
        assert len(st) == n
        assert np.all(np.diff(st) >= 0)
        assert np.all((st >= 0) & (st < len(INV.STAGES)))
        if n >= 2 * len(INV.STAGES):
            assert st[0] == 0 and st[-1] == len(INV.STAGES) - 1
    counts = np.bincount(INV.schedule(500), minlength=5)
    assert counts.tolist() == [100, 150, 100, 75, 75]


def test_learning_rate_vector_freezes_other_groups():
    o = S.param_offsets()
    lr = INV.lr_vector(("delta", "lights"))
    assert np.all(lr[o["delta"]:o["cspec"]] == INV.LEARNING_RATES["delta"])
    assert np.all(lr[o["lights"]:] == INV.LEARNING_RATES["lights"])
    assert np.all(lr[:o["delta"]] == 0) and np.all(lr[o["cspec"]:o["lights"]] == 0)
    # every parameter is optimised in some stage
    union = np.zeros_like(lr)
    for _, _, groups in INV.STAGES:
        union += INV.lr_vector(groups)
    assert np.all(union > 0)


def test_parameter_errors_zero_at_truth():
    th = S.make_theta(S.make_scene("tiny"), seed=3)
    e = INV.parameter_errors(th, th)
    assert all(v == 0 for v in e.values())
