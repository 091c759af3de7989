"""Host logic of the training loop (Sec. 3.2-3.4, Tab. 3-4): learning-rate schedule, epoch order,
batching, the fixed sample set and the checkpoint format.  No GPU needed."""
import numpy as np

from paper_2607_16906_b300 import synth
from paper_2607_16906_b300 import train_precond as tp


def test_cosine_schedule_runs_from_lr_max_to_lr_min():
    total = 1000
    lrs = [tp.cosine_lr(s, total, 1e-3, 1e-5) for s in range(total + 1)]
    assert lrs[0] == 1e-3 and abs(lrs[-1] - 1e-5) < 1e-18
    assert abs(lrs[total // 2] - 0.5 * (1e-3 + 1e-5)) < 1e-15
    assert all(a >= b for a, b in zip(lrs, lrs[1:]))
    assert tp.cosine_lr(5000, total, 1e-3, 1e-5) == lrs[-1]     # clamped after the end


def test_epoch_order_is_a_seeded_permutation():
    a = tp.epoch_order(3, 100, 42)
    assert sorted(a.tolist()) == list(range(100))
    assert (a == tp.epoch_order(3, 100, 42)).all()               # resumable: same order again
    assert not (a == tp.epoch_order(4, 100, 42)).all()           # reshuffled every epoch


def test_batches_cover_full_batches_only():
    order = np.arange(10)
    got = list(tp.batches(order, 4))
    assert [b.tolist() for b in got] == [[0, 1, 2, 3], [4, 5, 6, 7]]


def test_sample_set_is_fixed_by_its_seed():
    c1, b1, k1 = tp.make_sample_set("D0", 12, 16, 4, 7)
    c2, b2, k2 = tp.make_sample_set("D0", 12, 16, 4, 7)
    assert c1.shape == (12, 24, 24) and c1.dtype == np.float32 and b1.dtype == np.complex64
    assert (c1 == c2).all() and (b1 == b2).all() and k1 == k2
    assert set(v for _, v in k1) <= {"uniform", "skull"}          # D0's velocity menu
    c3, _, _ = tp.make_sample_set("D0", 12, 16, 4, 8)
    assert not (c1 == c3).all()


class _FakeNet:
    def __init__(self, n):
        rng = synth.rng_for(1)
        self.w, self.m, self.v, self.step = rng.standard_normal(n), rng.standard_normal(n), rng.random(n), 17

    def weights(self):
        return self.w

    def adam_state(self):
        return self.m, self.v, self.step


def test_checkpoint_round_trip(tmp_path):
    net = _FakeNet(50)
    state = {"epoch": 3, "step": 120, "best": {"mean_iters": 81.5, "converged": 4, "epoch": 2}, "history": []}
    path = str(tmp_path / "ck.npz")
    tp.save_checkpoint(path, net, state)
    w, (m, v, step), st = tp.load_checkpoint(path)
    assert (w == net.w).all() and (m == net.m).all() and (v == net.v).all() and step == 17 and st == state


def test_validation_ranking():
    a = {"converged": 4, "mean_iters": 100.0}
    assert tp.better(a, None)
    assert tp.better({"converged": 4, "mean_iters": 90.0}, a)
    assert not tp.better({"converged": 3, "mean_iters": 10.0}, a)
