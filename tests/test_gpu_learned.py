"""What the trained closure gains over the solver without it (small scale, GB300).

Coarse 16^3 runs are paired with 32^3 runs of the same linear field (30 steps,
a = 0.1 -> 1.0, dx = 1 Mpc/h on the coarse grid); the network is trained on the 120 pairs
with the library's own forward and backward kernels and then (a) scored on held-out pairs
of another seed and (b) run inside the solver for a whole held-out run. Measured when this
test was written: held-out loss 1.09 (plain solver) -> 0.60 (trained); final density error
against the restricted fine run 0.092 -> 0.063. The bars leave room for the run-to-run
spread of float atomics in the weight gradient.
"""
import pytest

from gpu_helpers import lib, need_gpu

pytestmark = pytest.mark.gpu


def test_trained_closure_beats_the_plain_solver():
    need_gpu()
    lib()
    from paper_2502_02294_gb300 import learned
    r = learned.experiment(n=16, seeds=4, run_steps=30, iters=300, batch=2, lr=2e-3,
                           eval_n=0)
    assert r["heldout_loss_untrained"] > 0.9 * r["heldout_loss_plain_solver"]
    assert r["heldout_loss_trained"] < 0.75 * r["heldout_loss_plain_solver"], r
    assert r["train_loss_last"] < 0.7 * r["train_loss_first"], r
    plain, corr = r["run_error"]["plain"], r["run_error"]["closure"]
    for f in ("rho", "m", "eps"):
        assert corr[f] < 0.9 * plain[f], (f, r["run_error"])
