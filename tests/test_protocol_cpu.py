"""Host sequencing of the paper's protocol (Sec. III-C) on the CPU, against fake lattices.

``protocol.run`` only orders calls of the C ABI; these fakes record the calls, so the test
pins the order the protocol prescribes: the initialisation's pure steps with a metric
record every `record_every` steps, the pure-LBM arm copied from the state after the
initialisation, then per round K steps, training with that round's (decreasing) epoch
count, the correction, and the pure arm's K steps, with both arms' metrics after each round.
"""
import numpy as np

from paper_2504_10539_gb300 import protocol as P
from paper_2504_10539_gb300 import workloads as wl


class FakeLattice:
    made = []

    def __init__(self, params):
        self.step_count, self.calls, self.from_state = 0, [], None
        FakeLattice.made.append(self)

    def init_droplets(self, *a):
        self.calls.append("init")

    def set_weights(self, blob):
        self.calls.append("weights")

    def step(self, n):
        self.calls.append(("step", n))
        self.step_count += n

    def correct(self):
        self.calls.append("correct")

    def metrics(self):
        self.calls.append("metrics")
        return {k: float(self.step_count) for k in P.METRICS}

    def state(self):
        return np.full((9, 2, 2), float(self.step_count)), self.step_count

    def set_state(self, f, step):
        self.calls.append(("set_state", step))
        self.step_count, self.from_state = step, f

    def status(self):
        return 0

    def close(self):
        pass


class FakeTrainer:
    def __init__(self, lattice, max_epochs, **hyper):
        self.lattice, self.max_epochs = lattice, max_epochs

    def train(self, epochs):
        assert epochs <= self.max_epochs
        self.lattice.calls.append(("train", epochs))

    def losses(self, epochs):
        return np.linspace(1.0, 0.5, epochs)[:, None] * np.ones((1, 4))

    def close(self):
        pass


def test_protocol_orders_the_calls_of_sec_iii_c(monkeypatch):
    monkeypatch.setattr(P.B, "Lattice", FakeLattice)
    monkeypatch.setattr(P.B, "Trainer", FakeTrainer)
    monkeypatch.setattr(P.B, "job_params", lambda job: job)
    FakeLattice.made = []
    job = wl.Lattice(64, 64, storage=wl.F32, droplets=[(32.0, 32.0, 11.0)], K=100)
    out = P.run(job, init_steps=500, K=100, record_every=50)
    pinn, pure = FakeLattice.made
    # initialisation: pure steps with a record every 50 steps, from step 0
    assert [s for s, _ in out["init"]] == list(range(0, 501, 50))
    assert all(m["W"] == s for s, m in out["init"])
    assert pinn.calls[:3] == ["init", "weights", "metrics"]
    # the pure arm starts from the state after the initialisation
    assert pure.calls[0] == ("set_state", 500) and np.all(pure.from_state == 500.0)
    # rounds: K steps, training with decreasing epochs, correction; pure arm K steps
    assert pinn.calls[3:23] == [("step", 50), "metrics"] * 10
    rounds = pinn.calls[23:]
    expect = []
    for e in P.DEFAULT_EPOCHS:
        expect += [("step", 100), ("train", e), "correct", "metrics"]
    assert rounds == expect
    assert list(P.DEFAULT_EPOCHS) == sorted(P.DEFAULT_EPOCHS, reverse=True) and P.DEFAULT_EPOCHS[0] == 300
    assert pure.calls[1:] == [("step", 100), "metrics"] * len(P.DEFAULT_EPOCHS)
    steps = [600 + 100 * k for k in range(len(P.DEFAULT_EPOCHS))]
    assert [(s, e) for s, e, _, _ in out["pinn"]] == list(zip(steps, P.DEFAULT_EPOCHS))
    assert [s for s, _ in out["pure"]] == steps
    assert all(m["W"] == s for s, _, m, _ in out["pinn"]) and all(m["W"] == s for s, m in out["pure"])
    assert all(l == (1.0, 0.5) for _, _, _, l in out["pinn"])
    assert out["status"] == {"pinn": 0, "pure": 0}
