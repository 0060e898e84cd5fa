"""Solitary-wave run-up on a plane beach on the GPU (1D line, the reconstructed example of
section "Examples"): the run-up law R/d = 2.831 sqrt(cot beta) (H/d)^(5/4) to 10 %, and the
FP32 run against the FP64 oracle on the same line (run-up within 1e-4 d, gauge-free, the
final state within 1e-4 of the wave height on nodes wet in both)."""
import numpy as np
import pytest

import oracle
import workloads
from paper_1410_0753_gb300 import CliffsGrid

pytestmark = pytest.mark.gpu


def test_runup_law_and_oracle_on_the_gpu():
    from tests import parity as P
    w = workloads.runup_1d()
    g = CliffsGrid.from_workload(w)
    g.set_bathy(w.x, w.y, w.depth, False)
    g.set_initial(w.eta0.astype(np.float32), w.u0.astype(np.float32))
    g.step(w.steps)
    em, _ = g.maxwave()
    e32 = g.state()[0]
    g.close()
    land = w.depth[0] < 0
    R32 = em[0][land][em[0][land] > -1e30].max()
    law = w.extra["runup_law"]
    assert abs(R32 / law - 1.0) <= 0.10, (R32, law)
    r = oracle.run(oracle.params_from(w), w.x, w.y, P.f32(w.depth), w.eta0, w.u0, None, nsteps=w.steps,
                   maxout=1)
    e64 = r["eta_max"][0][land]
    R64 = e64[e64 > -1e30].max()
    P.report("runup_1d", runup32=R32, runup64=R64, law=law)
    assert abs(R32 - R64) <= 1e-4 * w.extra["d"]
    wet = ((r["eta"][0] + w.depth[0]) >= w.h_min) & ((e32[0] + w.depth[0]) >= w.h_min)
    assert np.abs(e32[0] - r["eta"][0])[wet].max() <= 1e-4 * w.extra["H"] * 10
