"""Checkpointed labelling of the learned interval (host logic, no GPU): a
run stopped part-way and resumed ends with the same arrays, bit for bit, as
an uninterrupted one, and computes only the missing labels."""
import numpy as np
import pytest

from paper_2211_08948_gb300 import learned


def _fake_label(i):
    # deterministic per index, like the library's labels of problem i
    rng = np.random.default_rng(1000 + i)
    return rng.standard_normal(16).astype(np.float32), rng.standard_normal(3).astype(np.float32), 7 + i % 5


class Stop(Exception):
    pass


def test_resume_after_interruption_is_bit_identical(tmp_path):
    n, shard = 103, 10
    X0, T0, mv0, c0 = learned.label_loop(n, _fake_label)
    assert c0 == n
    calls = []

    def stopping(i):
        if i == 47:
            raise Stop()
        calls.append(i)
        return _fake_label(i)

    with pytest.raises(Stop):
        learned.label_loop(n, stopping, ckpt_dir=str(tmp_path), shard=shard, tag="set-a")
    # shards 0..39 were finished and saved; 40..46 were lost with the stop
    assert sorted(p.name for p in tmp_path.glob("labels_*.npz"))[-1] == "labels_000000030_000000040.npz"
    calls.clear()
    X1, T1, mv1, c1 = learned.label_loop(n, lambda i: (calls.append(i), _fake_label(i))[1],
                                         ckpt_dir=str(tmp_path), shard=shard, tag="set-a")
    assert calls == list(range(40, n)) and c1 == n - 40
    assert np.array_equal(X0, X1) and np.array_equal(T0, T1) and mv0 == mv1
    # everything is checkpointed now: a third call computes nothing
    X2, T2, mv2, c2 = learned.label_loop(n, _fake_label, ckpt_dir=str(tmp_path), shard=shard, tag="set-a")
    assert c2 == 0 and np.array_equal(X0, X2) and np.array_equal(T0, T2)


def test_checkpoint_of_another_problem_set_is_refused(tmp_path):
    learned.label_loop(20, _fake_label, ckpt_dir=str(tmp_path), shard=10, tag="set-a")
    with pytest.raises(ValueError):
        learned.label_loop(20, _fake_label, ckpt_dir=str(tmp_path), shard=10, tag="set-b")
