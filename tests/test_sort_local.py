"""The neighbourhood sort (particles sorted before and moved at most into the units of 8^3 cells
around their sort-time unit) gives the stable sort by key, and so does the general sort it falls
back to when a particle moved farther.

The expected order is the previous storage order stably sorted by the chunk-major keys of the
cells the library reports before the sort; reading the cells turns the pre-sort records back into
arrays, so these cases sort from the arrays, and a second run without reads (sorting from the
records) must give bit-identical states."""
import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs
from tests.helpers import chunk_keys_from_cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Sim():
    import torch

    assert torch.cuda.is_available()
    from paper_2603_26691_gb300.sim import Sim

    return Sim


def _setup(Sim, prec, grid, B, n, seed, vmax=0.0, reorder_every=0):
    # a field moving particles ~0.1 cell per step of 5e-4 s, as the 256^3 bench workload does
    scale = 256.0 / max(grid)
    U = (inputs.random_fourier(max(grid), seed=4) * scale)
    if tuple(grid) != (max(grid),) * 3:
        U = inputs.taylor_green(grid) * scale + 0.1 * scale
    pos, vel, d, _ = inputs.particles(seed, 0, n, vmax=vmax)
    sim = Sim(grid, precision=prec, chunk_edge=B)
    sim.set_params(reorder_every=reorder_every)
    sim.set_fluid(U.astype(np.float32))
    sim.add_particles(pos, d, vel)
    return sim


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
@pytest.mark.parametrize("grid,B", [((8, 8, 8), 8), ((16, 16, 16), 8), ((24, 24, 24), 8), ((40, 48, 56), 8),
                                    ((32, 32, 32), 16), ((64, 64, 64), 32)])
def test_neighbourhood_sort_is_the_stable_sort(Sim, prec, grid, B):
    n = 100_003
    sim = _setup(Sim, prec, grid, B, n, seed=41)
    sim.reorder()  # first sort: the general one (nothing was sorted before)
    for _ in range(3):
        sim.step(6, 5e-4)
        cells = sim.cells()
        before = sim.particles()[3].astype(np.int64)
        keys = chunk_keys_from_cells(cells, grid, B)
        sim.reorder()
        after = sim.particles()[3].astype(np.int64)
        assert np.array_equal(after, before[np.argsort(keys, kind="stable")])
        assert np.array_equal(sim.cells(), cells[np.argsort(keys, kind="stable")])
        assert np.array_equal(sim.cell_counts(), np.bincount(cells, minlength=int(np.prod(grid))))
    sim.close()


@pytest.mark.parametrize("frac_fast", [1e-5, 0.5])
def test_particles_beyond_the_neighbouring_units_take_the_general_sort(Sim, frac_fast):
    """A few (or many) particles launched fast enough to cross several units between sorts: the
    neighbourhood sort gives way to the general sort, which gives the same stable order."""
    grid, B, n = (32, 32, 32), 8, 200_003
    sim = _setup(Sim, "mixed_f32", grid, B, n, seed=43)
    sim.reorder()
    fast = int(max(1, frac_fast * n))
    pos, vel, d, _ = inputs.particles(44, n, fast, vmax=400.0)
    sim.add_particles(pos, d, vel)
    sim.reorder()  # particles were added: the general sort
    sim.step(3, 5e-4)  # the fast ones move ~20 cells
    cells = sim.cells()
    before = sim.particles()[3].astype(np.int64)
    keys = chunk_keys_from_cells(cells, grid, B)
    sim.reorder()
    after = sim.particles()[3].astype(np.int64)
    assert np.array_equal(after, before[np.argsort(keys, kind="stable")])
    assert np.array_equal(sim.cell_counts(), np.bincount(cells, minlength=int(np.prod(grid))))
    # and the next sort, with every particle near its unit again, is a neighbourhood sort
    sim.step(1, 1e-6)
    cells = sim.cells()
    before = sim.particles()[3].astype(np.int64)
    keys = chunk_keys_from_cells(cells, grid, B)
    sim.reorder()
    after = sim.particles()[3].astype(np.int64)
    assert np.array_equal(after, before[np.argsort(keys, kind="stable")])
    sim.close()


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_sorting_from_records_equals_sorting_from_arrays(Sim, prec):
    """With a sort every 5 steps the step before each sort writes 32-byte records and the
    neighbourhood sort gathers from them; reading the state in between turns them back into arrays
    and the sort gathers from the arrays: the states must agree bit for bit."""
    grid, B, n = (32, 32, 32), 8, 150_001
    out = []
    for read_between in (False, True):
        sim = _setup(Sim, prec, grid, B, n, seed=45, reorder_every=5)
        for _ in range(4):
            sim.step(5, 5e-4)
            if read_between:
                sim.cells()
        sim.step(1, 5e-4)
        g = dict(src=sim.sources(host=True), cells=sim.cells(), counts=sim.cell_counts())
        g["pos"], g["vel"], g["d"], g["ids"] = sim.particles()
        sim.close()
        out.append(g)
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_deferred_gather_paths_agree(Sim, prec):
    """A sort after a record-writing step leaves its payload gather to the next sorted step.  Sorting
    again first, changing the physics (a kernel that cannot gather) or reading the state in between all
    run the gather at once; every path gives the same bits as gathering right away."""
    grid, B, n = (32, 32, 32), 8, 60_001

    def run(read_between):
        sim = _setup(Sim, prec, grid, B, n, seed=47, reorder_every=5)
        out = []
        rd = (lambda: sim.invariants()) if read_between else (lambda: None)
        sim.step(5, 5e-4)          # sort, 4 plain steps, the record-writing step
        rd()
        sim.reorder()              # deferred gather
        rd()
        sim.reorder()              # the pending gather first, then a sort from the arrays
        rd()
        sim.step(5, 5e-4)
        rd()
        sim.reorder()              # after a record-writing step again: deferred
        rd()
        sim.set_physics(deposit="cic")
        sim.step(2, 5e-4)          # the physics instance cannot gather: the gather runs first
        sim.set_physics()
        rd()
        sim.step(6, 5e-4)          # through a deferred sort and its gathering step
        out.append(sim.sources(host=True))
        out.append(sim.cells())
        out.extend(sim.particles())
        sim.close()
        return out

    a, b = run(False), run(True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_bf16"])
def test_deferred_gather_with_the_general_sort(Sim, prec):
    """Fast particles make the neighbourhood sort give way to the general sort while a sort's payload
    gather is left to the next step: the ids then move in a kernel of their own.  Reading the state
    after every step turns each step's records back into arrays, so that no gather is deferred; both
    runs give the same bits."""
    grid, B, n = (32, 32, 32), 8, 80_001

    def run(read_between):
        sim = _setup(Sim, prec, grid, B, n, seed=49, reorder_every=5)
        pos, vel, d, _ = inputs.particles(50, n, 50, vmax=400.0)
        sim.add_particles(pos, d, vel)
        for _ in range(16):
            sim.step(1, 5e-4)
            if read_between:
                sim.cells()
        out = [sim.sources(host=True), sim.cells(), sim.cell_counts()]
        out.extend(sim.particles())
        sim.close()
        return out

    a, b = run(False), run(True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
