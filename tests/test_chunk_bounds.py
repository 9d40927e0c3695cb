"""Per-chunk bounding boxes on the GPU against the oracle: membership from the sort, boxes of the
positions after the particles moved (FP64 exact; mixed within the FP32 position bound)."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,B,N", [("fp64", 8, 32), ("mixed_f32", 8, 32), ("mixed_f32", 16, 48), ("fp64", 4, 24)])
def test_chunk_bounds_match_oracle(prec, B, N):
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    U = inputs.random_fourier(N, seed=5) * 3.0
    pos, vel, d, _ = inputs.particles(31, 0, 20_001, vmax=2.0)
    sim = Sim(N, precision=prec, chunk_edge=B)
    sim.set_params(reorder_every=0)
    sim.set_fluid(U if prec == "fp64" else U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    sim.reorder()
    p_sort, _, _, _ = sim.particles()
    sim.step(15, 1e-3)
    p_now, _, _, _ = sim.particles()
    got = sim.chunk_bounds()
    sim.close()
    want = oracle.chunk_bounds(oracle.make_grid(N, chunk_edge=B), p_sort, p_now)
    assert np.array_equal(np.isinf(got), np.isinf(want))
    fin = np.isfinite(want)
    # the GPU reads the state it exported, with the oracle's arithmetic: identical for FP64; for
    # the mixed form the exported positions are the same doubles, so the boxes are identical too
    assert np.array_equal(got[fin], want[fin])
    # the particles moved: some boxes reach beyond their chunk's cells
    h = 1.0 / N
    width = (want[:, 3:] - want[:, :3])[np.isfinite(want[:, 0])]
    assert width.max() > B * h
