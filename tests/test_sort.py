"""The stable counting sort by chunk-major key, against the oracle's stable sort."""
import numpy as np
import pytest

import oracle
from paper_2603_26691_gb300 import inputs
from tests.helpers import chunk_keys_from_cells, face_distance

pytestmark = pytest.mark.gpu

BAND = 1e-9


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _oracle_keys(G, pos):
    return oracle.keys_of_positions(G, pos)


def _cells_near(pos, N):
    """Cells within one cell (per axis, periodic) of the given positions' cells, as a mask."""
    mask = np.zeros(N ** 3, dtype=bool)
    c = [np.clip(np.floor(pos[q] * N).astype(np.int64), 0, N - 1) for q in range(3)]
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                mask[(c[0] + dx) % N + N * (((c[1] + dy) % N) + N * ((c[2] + dz) % N))] = True
    return mask


def _compare_order(got_ids, want_order, ambiguous):
    """Same sequence of ids once particles that sit within the band of a face are removed."""
    amb = set(np.flatnonzero(ambiguous).tolist())
    g = [i for i in got_ids.tolist() if i not in amb]
    w = [i for i in want_order.tolist() if i not in amb]
    assert g == w


@pytest.mark.parametrize("prec", ["fp64", "mixed_f32", "mixed_bf16"])
@pytest.mark.parametrize("N,B", [(16, 4), (24, 8), (32, 32)])
def test_reorder_matches_oracle_stable_sort(Sim, prec, N, B):
    n = 30_011
    pos, vel, d, _ = inputs.particles(31, 0, n)
    G = oracle.make_grid(N, chunk_edge=B)
    sim = Sim(N, precision=prec, chunk_edge=B)
    sim.set_params(reorder_every=0)
    sim.set_fluid(inputs.random_fourier(N, seed=2))
    sim.add_particles(pos, d, vel)
    sim.reorder()
    ids1 = sim.particles()[3].astype(np.int64)
    k0 = _oracle_keys(G, pos)
    amb0 = face_distance(pos, (N, N, N)) <= BAND
    want1 = oracle.sort_perm(k0)
    _compare_order(ids1, want1, amb0)
    counts = sim.cell_counts()
    # every cell is compared except those next to a particle within the band of a face (which may
    # belong to either side)
    keep = ~_cells_near(pos[:, amb0], N)
    assert keep.mean() > 0.99
    assert np.array_equal(counts[keep], oracle.cell_counts(G, pos)[keep])
    assert counts.sum() == n
    # move, then sort again: the new order is the stable sort of the previous one
    steps, dt = 7, 1e-3
    sim.step(steps, dt)
    sim.reorder()
    ids2 = sim.particles()[3].astype(np.int64)
    opos, _, _, _ = oracle.run(G, inputs.random_fourier(N, seed=2) if prec == "fp64"
                               else inputs.random_fourier(N, seed=2).astype(np.float32).astype(np.float64),
                               pos, vel, d, steps, dt)
    k1 = _oracle_keys(G, opos)
    band = {"fp64": BAND, "mixed_f32": 1e-4, "mixed_bf16": 3e-2}[prec]
    amb1 = face_distance(opos, (N, N, N)) <= band
    prev = ids1
    want2 = prev[np.argsort(k1[prev], kind="stable")]
    _compare_order(ids2, want2, amb1 | amb0)
    sim.close()


def test_sort_is_a_stable_sort_of_the_previous_order_at_scale(Sim):
    """Property at 2e7 particles: sorted keys non-decreasing and ties in previous storage order."""
    N, B, n = 128, 8, 20_000_000
    sim = Sim(N, precision="mixed_f32", chunk_edge=B)
    sim.set_params(reorder_every=0)
    q = inputs.lognormal_qtable()
    pos, vel, d, ids = sim.gen_particles(3, 0, n, q)
    sim.add_particles(pos, d, vel)
    del pos, vel, d, ids
    before_cells = sim.cells()
    before_ids = sim.particles()[3].astype(np.int64)
    keys = chunk_keys_from_cells(before_cells, (N, N, N), B)
    sim.reorder()
    after_ids = sim.particles()[3].astype(np.int64)
    want = before_ids[np.argsort(keys, kind="stable")]
    assert np.array_equal(after_ids, want)
    after_keys = chunk_keys_from_cells(sim.cells(), (N, N, N), B)
    assert np.all(np.diff(after_keys.astype(np.int64)) >= 0)
    counts = sim.cell_counts()
    assert np.array_equal(counts, np.bincount(before_cells, minlength=N ** 3))
    sim.close()
