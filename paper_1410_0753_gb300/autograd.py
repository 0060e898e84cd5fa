"""torch.autograd binding of the split-step run: initial free surface -> gauge eta records.

The forward is cliffs_set_initial + cliffs_step_n; the backward is the library's hand-written
adjoint (cliffs_adjoint_n), which recomputes the forward from checkpoints on the device and
transposes every sweep with the forward's branches frozen. Argument marshalling only: all
arithmetic runs in the library's CUDA kernels.
"""
import torch

from . import CliffsGrid, cliffs_adjoint_n, cliffs_read_gauges


class GaugeRun(torch.autograd.Function):
    """eta0 [ny][nx] (float32, CUDA) -> gauge eta records [n // gout + 1][G] of the next n steps."""

    @staticmethod
    def forward(ctx, eta0, grid: CliffsGrid, n: int, checkpoint_every: int = 100):
        eta0 = eta0.detach().contiguous().float()
        grid.set_initial(eta0)
        grid.step(n)
        nrec = cliffs_read_gauges(grid.h, 0)
        rec = torch.empty((nrec, grid.n_gauges, 3), dtype=torch.float32, device=eta0.device)
        cliffs_read_gauges(grid.h, 0, rec)
        ctx.grid, ctx.n, ctx.k = grid, int(n), int(checkpoint_every)
        ctx.save_for_backward(eta0)
        return rec[:, :, 0].contiguous()

    @staticmethod
    def backward(ctx, grad):
        (eta0,) = ctx.saved_tensors
        grid = ctx.grid
        grid.set_initial(eta0)                  # the adjoint starts from the run's X_0
        out = torch.empty_like(eta0)
        cliffs_adjoint_n(grid.h, ctx.n, ctx.k, grad.detach().contiguous().float(), out)
        return out, None, None, None


def gauge_run(eta0, grid, n, checkpoint_every=100):
    return GaugeRun.apply(eta0, grid, n, checkpoint_every)
