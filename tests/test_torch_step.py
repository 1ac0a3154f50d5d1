"""Pins of the plain PyTorch step (the reference for the adjoint's VJPs):
its forward equals the pinned C oracle, and autograd through it agrees
with central finite differences."""
import numpy as np
import pytest
import torch

from oracle.torch_step import TorchStep
from paper_1507_03521_gb300 import workloads as W


@pytest.mark.parametrize("walls", [False, True])
def test_forward_equals_c_oracle(orc, walls):
    p, phi, _, _ = W.small_case(14, 11, seed=21, walls=walls, gravity=2e-5, u_wall=0.02)
    ts = TorchStep(p)
    M = torch.tensor(p["M"], dtype=torch.float64)
    sg = torch.tensor(p["sigma"], dtype=torch.float64)
    f, g = ts.init(torch.from_numpy(phi), M, sg)
    for _ in range(12):
        f, g = ts.step(f, g, M, sg)
    o = orc.Oracle(p)
    o.init_phi(phi)
    o.step(12)
    of, og = o.pops()
    scale = np.abs(og).max()
    assert np.abs(g.numpy() - og).max() <= 1e-13 * scale
    assert np.abs(f.numpy() - of).max() <= 1e-13 * max(np.abs(of).max(), 1e-12)
    tf = ts.fields(f, g, M, sg)
    ref = o.fields()
    for k in ("phi", "ux", "uy", "p", "mu"):
        assert np.abs(tf[k].numpy() - ref[k]).max() <= 1e-12 * max(np.abs(ref[k]).max(), 1e-9), k


def test_autograd_matches_finite_differences():
    p, phi, _, _ = W.small_case(10, 9, seed=22, walls=True, gravity=1e-5, u_wall=0.01)
    ts = TorchStep(p)
    target = torch.from_numpy(np.roll(phi, 1, axis=1))
    M = torch.tensor(p["M"], dtype=torch.float64, requires_grad=True)
    sg = torch.tensor(p["sigma"], dtype=torch.float64, requires_grad=True)
    ph = torch.from_numpy(phi).clone().requires_grad_(True)
    L = ts.rollout_loss(ph, M, sg, 6, target)
    L.backward()
    rng = np.random.default_rng(1)
    v = torch.from_numpy(rng.standard_normal(phi.shape))
    with torch.no_grad():
        def loss(dphi=0.0, dM=0.0, ds=0.0):
            return ts.rollout_loss(torch.from_numpy(phi) + dphi, M + dM, sg + ds, 6, target).item()
        h = 1e-6
        fd_phi = (loss(dphi=h * v) - loss(dphi=-h * v)) / (2 * h)
        fd_M = (loss(dM=h * p["M"]) - loss(dM=-h * p["M"])) / (2 * h * p["M"])
        fd_s = (loss(ds=h * p["sigma"]) - loss(ds=-h * p["sigma"])) / (2 * h * p["sigma"])
    assert (ph.grad * v).sum().item() == pytest.approx(fd_phi, rel=1e-6)
    assert M.grad.item() == pytest.approx(fd_M, rel=1e-6)
    assert sg.grad.item() == pytest.approx(fd_s, rel=1e-6)
