"""torch.autograd binding of the split-step run: initial free surface -> gauge records
(eta only, or eta, u and v).

The forward is cliffs_set_initial + cliffs_step_n with the run recorded for the adjoint
(cliffs_adjoint_record: a checkpoint every K steps); the backward is the library's
hand-written adjoint of that recorded run (cliffs_adjoint_recorded_records), which
recomputes each segment from its checkpoint and transposes every sweep with the forward's
branches frozen. If the grid has run something else in between, the backward starts over
from eta0 (cliffs_adjoint_records, with its own checkpoint pass). Argument marshalling only:
all arithmetic runs in the library's CUDA kernels.
"""
import torch

from . import CliffsGrid, cliffs_adjoint_recorded_records, cliffs_adjoint_records, cliffs_read_gauges


class GaugeRun(torch.autograd.Function):
    """eta0 [ny][nx] (float32, CUDA) -> gauge eta records [n // gout + 1][G] of the next n steps,
    or with records=True the whole records [n // gout + 1][G][3] of (eta, u, v)."""

    @staticmethod
    def forward(ctx, eta0, grid: CliffsGrid, n: int, checkpoint_every: int = 100, records: bool = False):
        eta0 = eta0.detach().contiguous().float()
        grid.set_initial(eta0)
        grid.adjoint_record(checkpoint_every)
        grid.step(n)
        nrec = cliffs_read_gauges(grid.h, 0)
        rec = torch.empty((nrec, grid.n_gauges, 3), dtype=torch.float32, device=eta0.device)
        cliffs_read_gauges(grid.h, 0, rec)
        ctx.grid, ctx.n, ctx.k, ctx.run_id, ctx.records = grid, int(n), int(checkpoint_every), grid.run_id, records
        ctx.save_for_backward(eta0)
        return rec if records else rec[:, :, 0].contiguous()

    @staticmethod
    def backward(ctx, grad):
        (eta0,) = ctx.saved_tensors
        grid = ctx.grid
        out = torch.empty_like(eta0)
        seed = grad.detach().contiguous().float()
        if not ctx.records:                     # dL/d eta only: the u and v parts are zero
            seed = torch.stack([seed, torch.zeros_like(seed), torch.zeros_like(seed)], dim=2).contiguous()
        if grid.run_id == ctx.run_id:
            cliffs_adjoint_recorded_records(grid.h, seed, out)
        else:
            grid.adjoint_record(0)
            grid.set_initial(eta0)              # the adjoint starts from the run's X_0
            cliffs_adjoint_records(grid.h, 0, ctx.n, ctx.k, seed, out)
        return out, None, None, None, None


def gauge_run(eta0, grid, n, checkpoint_every=None, records=False):
    """Run n steps from eta0 and return the gauge records (see GaugeRun). With
    checkpoint_every None the run keeps every state when they fit in half the free device
    memory (the backward then recomputes nothing), else a checkpoint every 100 steps."""
    if checkpoint_every is None:
        free, _ = torch.cuda.mem_get_info()
        pitch = (grid.nx + 31) // 32 * 32
        need = 12 * pitch * grid.ny * (int(n) + 1)
        checkpoint_every = 1 if need < free // 2 else 100
    return GaugeRun.apply(eta0, grid, n, checkpoint_every, records)
