"""The accumulated source as exact fixed-point integers (st_get_sources_fixed), the form the sum over
several GPUs uses: the words carry exactly the value st_get_sources reports, and two handles' words
summed as integers after shifting to the finer scale equal the sum of the two runs to FP64 rounding."""
import numpy as np
import pytest

from paper_2603_26691_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(prec, seed, n, d_scale=1.0):
    import torch  # noqa: F401

    from paper_2603_26691_gb300.sim import Sim

    N = 16
    sim = Sim(N, precision=prec)
    sim.set_fluid(inputs.random_fourier(N, seed=5).astype(np.float32))
    pos, vel, d, _ = inputs.particles(seed, 0, n, vmax=0.3)
    sim.add_particles(pos, d * d_scale, vel)
    sim.step(7, 5e-4)
    w, E = sim.sources_fixed()
    src = sim.sources(host=True)
    sim.close()
    return w, E, src


@pytest.mark.parametrize("prec", ["fp64", "mixed_f32"])
def test_fixed_point_words_hold_the_sources(prec):
    from paper_2603_26691_gb300.dist import _limbs, _to_f64

    w, E, src = _run(prec, 3, 20_000)
    val = _to_f64(_limbs(w.cpu(), 0, 6), E).numpy()
    assert np.all(np.abs(val - src) <= np.spacing(np.abs(src)))
    # normalised: digits in [0, 2^32) below the top word
    lo = w[..., :3].cpu()
    assert int(lo.min()) >= 0 and int(lo.max()) < 2 ** 32


def test_two_handles_sum_exactly():
    from paper_2603_26691_gb300.dist import _limbs, _to_f64

    wa, Ea, sa = _run("mixed_f32", 3, 20_000)
    wb, Eb, sb = _run("mixed_f32", 4, 20_000, d_scale=3.0)  # heavier particles: a coarser exponent
    assert Ea != Eb
    e = max(Ea, Eb)
    tot = _to_f64(_limbs(wa.cpu(), e - Ea, 8) + _limbs(wb.cpu(), e - Eb, 8), e).numpy()
    assert np.abs(tot - (sa + sb)).max() <= 4 * np.spacing(np.abs(sa + sb).max())
