"""Gradients of an interface-shape loss through many time steps.

``rollout_loss(phi0, M, sigma, params, steps, target)`` returns
L = sum_x (phi_T(x) - target(x))^2 after `steps` steps from the
equilibrium state of phi0 (u = 0), as a torch scalar that supports
backward() with respect to phi0, M (mobility lambda) and sigma (surface
tension).  Forward and backward run in the CUDA library: the forward keeps
a checkpoint every K steps; the backward hands each segment of K steps,
last first, to lbm_adj_segment, which recomputes the segment's states from
its checkpoint and applies the hand-written adjoint step K times in
reverse (replayed from a CUDA graph after the first segment of each
length), and finally the adjoint of the initial state (lbm_adj_init).
Memory: steps/K checkpoints plus K states.  With overlap=True (the
default) two buffers of K states alternate: while the reverse steps of one
segment run, a second stream recomputes the states of the next
(lbm_adj_reverse_overlap), at the cost of K more states.
"""
from __future__ import annotations

import torch

from . import lbm


class LBMRollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi0, M, sigma, params, steps, target, K, dtype, overlap):
        p = dict(params, M=float(M), sigma=float(sigma))
        # a stream of its own: the backward replays its segments as CUDA
        # graphs, which cannot be captured on the default stream
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            sim = lbm.Sim(p, dtype, stream=stream)
            sim.init_phi(phi0.detach())
            ckpt = []
            t = 0
            while t < steps:
                ckpt.append(sim.get_state()[0])
                n = min(K, steps - t)
                sim.step(n)
                t += n
            state_T, _ = sim.get_state()
            work = sim.adj_work()
            lam = torch.empty_like(state_T)
            loss = sim.adj_seed(state_T, target.detach(), lam, work)
        ctx.sim, ctx.ckpt, ctx.lam, ctx.work = sim, ckpt, lam, work
        ctx.steps, ctx.K, ctx.overlap = steps, K, overlap
        ctx.save_for_backward(phi0.detach())
        return torch.tensor(loss, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        sim, lam, work = ctx.sim, ctx.lam, ctx.work
        (phi0,) = ctx.saved_tensors
        steps, K = ctx.steps, ctx.K
        with torch.cuda.stream(sim.stream):
            sb = sim.state_bytes()
            stride = (sb + 255) // 256 * 256
            states = torch.empty(min(K, steps) * stride, dtype=torch.uint8, device=lam.device)
            other = torch.empty_like(lam)
            sim.adj_set_graph(True)
            nseg = len(ctx.ckpt)
            seg_len = [min(K, steps - s * K) for s in range(nseg)]
            if not ctx.overlap:
                # one call per segment, last segment first: level 0 of
                # `states` takes the checkpoint, the library recomputes the
                # rest of the segment and runs its reverse steps (graph
                # replay after the first segment of each length)
                for seg in reversed(range(nseg)):
                    states[:sb].copy_(ctx.ckpt[seg])
                    sim.adj_segment(seg_len[seg], states, stride, lam, other, work)
            else:
                # two state buffers: the reverse steps of segment seg run on
                # `cur` while segment seg-1 is recomputed into `nxt`
                cur, nxt = states, torch.empty_like(states)
                cur[:sb].copy_(ctx.ckpt[nseg - 1])
                sim.adj_recompute(seg_len[nseg - 1], cur, stride)
                for seg in reversed(range(nseg)):
                    n_next = seg_len[seg - 1] if seg > 0 else 0
                    if n_next:
                        nxt[:sb].copy_(ctx.ckpt[seg - 1])
                    sim.adj_reverse_overlap(seg_len[seg], cur, stride, lam, other, work, n_next, nxt)
                    cur, nxt = nxt, cur
            phi_bar = sim.adj_init(phi0, lam, work)
            dM, dS = sim.adj_grads(work)
        g = float(grad_out)
        sim.close()
        return (phi_bar.to(device=phi0.device, dtype=phi0.dtype) * g,
                torch.tensor(dM * g, dtype=torch.float64),
                torch.tensor(dS * g, dtype=torch.float64), None, None, None, None, None, None)


def rollout_loss(phi0, M, sigma, params, steps, target, K=200, dtype="f64", overlap=True):
    """L = sum (phi_T - target)^2; differentiable in phi0, M, sigma."""
    if not torch.is_tensor(M):
        M = torch.tensor(float(M), dtype=torch.float64)
    if not torch.is_tensor(sigma):
        sigma = torch.tensor(float(sigma), dtype=torch.float64)
    return LBMRollout.apply(phi0, M, sigma, params, int(steps), target, int(K), dtype, bool(overlap))
