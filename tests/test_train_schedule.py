"""The paper's learning-rate schedule (Sec. 4.2: Adam, lr multiplied by 0.1
every 100 epochs), as the trainer applies it step by step.  CPU only."""
import pytest

from paper_2508_16121_gb300.train import step_decay_lr


def test_step_decay_sequence():
    lrs = [step_decay_lr(1e-4, s, every=100) for s in range(1, 401)]
    assert lrs[0] == lrs[99] == 1e-4
    assert lrs[100] == lrs[199] == pytest.approx(1e-5)
    assert lrs[200] == pytest.approx(1e-6)
    assert lrs[399] == pytest.approx(1e-7)
    assert len(set(lrs)) == 4


def test_constant_without_decay_and_other_factor():
    assert all(step_decay_lr(1e-3, s, every=None) == 1e-3 for s in (1, 50, 10_000))
    assert step_decay_lr(1e-3, 7, every=3, factor=0.5) == pytest.approx(1e-3 * 0.25)
    with pytest.raises(ValueError):
        step_decay_lr(1e-3, 0, every=3)
