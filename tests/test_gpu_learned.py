"""GPU test of what training gains: the U-Net, trained by the library's own forward,
backward and Adam kernels on (residual, error) pairs from FP64 Schwarz-PCG runs,
must leave less error on residuals of a held-out geometry than no correction at all.

The loss of a pair is ||e - c||_K^2 / ||e||_K^2 (1 = the correction c changes
nothing); the network's trained quality has no paper value to pin it to, so the
test compares against the method without the network, on held-out data.
"""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_training_reduces_the_error_left_on_held_out_residuals():
    from paper_1809_00828_gb300 import fcm, learned
    snaps = (3, 6, 12, 25, 50, 100)
    train_w = learned.training_workloads([1000, 1001, 1002], n=16, p=2, count=12)
    held_w = learned.training_workloads([1100], n=16, p=2, count=12)
    samples, solvers, gamma = learned.generate(train_w, snaps, log=None)
    held, held_solvers, _ = learned.generate(held_w, snaps, log=None)
    assert len(samples) >= 12 and len(held) >= 4 and gamma > 0
    net = fcm.UNet(in_ch=4, out_ch=3, base=8, levels=3, seed=0)
    before = learned.evaluate(net, held, gamma)
    hist = learned.train(net, samples, gamma, steps=300, batch=4, lr=2e-3, log=None)
    after = learned.evaluate(net, held, gamma)
    print(f"held-out loss: untrained {before:.4f}, trained {after:.4f}; last training losses {hist[-5:]}")
    # the trained correction removes part of the error on geometry it has not seen
    assert after < 0.95
    assert after < before
    net.close()
    for s in solvers + held_solvers:
        s.close()
