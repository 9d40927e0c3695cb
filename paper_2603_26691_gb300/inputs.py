"""Seeded synthetic inputs for the Lagrangian step: particles and fluid fields.

This module generates inputs only; it contains none of the method's
arithmetic (no interpolation, drag, integration, relocation or deposit).
Both the CUDA path and the FP64 CPU oracle take their inputs from here.  The
particle generator is counter-based, so any particle can be generated on its
own from (seed, index); the library's device-side generator
(``st_gen_particles``) implements the same definition and is checked
bit-for-bit against this one.

Particle definition (index p, seed s):
  * 64-bit words come from SplitMix64 (Steele, Lea and Flood 2014; output
    function as published by Vigna): the generator is seeded with
    key = mix64(s XOR 0x5DEECE66D) and word c is its (c+1)-th output,
    mix64(key + (c+1) * 0x9E3779B97F4A7C15), with c = 8 p + stream;
  * position component q (streams 0-2): L_q * (word >> 11) * 2^-53;
  * diameter (stream 3): lognormal by inverse-transform sampling with a
    piecewise-linear quantile function through K+1 = 65537 exact lognormal
    quantiles (median d50, geometric std sg, tails clipped at probabilities
    1/(4K) and 1 - 1/(4K)): segment = word >> 48, fraction = bits 11..47 of
    the word times 2^-37, d = q[seg] + frac * (q[seg+1] - q[seg]), each
    operation rounded separately;
  * velocity component q (streams 4-6, optional): vmax * (2 u - 1) with
    u = (word >> 11) * 2^-53, otherwise zero;
  * id = p.

Fluid fields (cell centres at (i + 1/2) h, array layout [k][j][i][3]):
  * steady Taylor-Green vortex u = U0 sin(2 pi x) cos(2 pi y) cos(2 pi z),
    v = -U0 cos(2 pi x) sin(2 pi y) cos(2 pi z), w = 0 (in units of L);
  * divergence-free random Fourier field: integer wave vectors with
    1 <= |k| <= kmax, complex Gaussian coefficients (numpy PCG64, seeded)
    with amplitude sqrt(E(|k|) / (4 pi |k|^2)), E ~ |k|^(-5/3), projected
    orthogonal to k, Hermitian-symmetric, inverse FFT in FP64, one global
    factor so that the component rms averaged over components is `rms`.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SEED_SALT = 0x5DEECE66D
NSTREAM = 8
QTABLE_K = 65536
_S30, _S27, _S31 = np.uint64(30), np.uint64(27), np.uint64(31)


def mix64(z):
    """SplitMix64 output function on uint64 numpy arrays (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _S30)) * _M1
        z = (z ^ (z >> _S27)) * _M2
    return z ^ (z >> _S31)


def seed_key(seed: int) -> np.uint64:
    return mix64(np.uint64((int(seed) ^ SEED_SALT) & 0xFFFFFFFFFFFFFFFF))[()]


def words(seed: int, index, stream: int) -> np.ndarray:
    """Word `stream` of particles `index` (uint64 array)."""
    idx = np.asarray(index, dtype=np.uint64)
    c = idx * np.uint64(NSTREAM) + np.uint64(stream) + np.uint64(1)
    with np.errstate(over="ignore"):
        z = seed_key(seed) + c * GOLDEN
    return mix64(z)


def uniform53(w: np.ndarray) -> np.ndarray:
    return (w >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def lognormal_qtable(d50: float = 20e-6, sg: float = 1.5, K: int = QTABLE_K) -> np.ndarray:
    """K+1 exact lognormal quantiles; the end points sit at p = 1/(4K), 1 - 1/(4K)."""
    from scipy.special import ndtri

    p = np.arange(K + 1, dtype=np.float64) / K
    p[0] = 0.25 / K
    p[K] = 1.0 - 0.25 / K
    return np.exp(math.log(d50) + math.log(sg) * ndtri(p))


def diameters_from_words(w: np.ndarray, qtable: np.ndarray) -> np.ndarray:
    seg = (w >> np.uint64(48)).astype(np.int64)
    frac = ((w >> np.uint64(11)) & np.uint64((1 << 37) - 1)).astype(np.float64) * (2.0 ** -37)
    q0 = qtable[seg]
    dq = qtable[seg + 1] - q0
    t = frac * dq
    return q0 + t


def particles(seed: int, first: int, count: int, L=(1.0, 1.0, 1.0), qtable=None, vmax: float = 0.0):
    """Particles first .. first+count-1: (pos [3,n], vel [3,n], d [n], ids [n] uint32)."""
    idx = np.arange(first, first + count, dtype=np.uint64)
    return particles_at(seed, idx, L=L, qtable=qtable, vmax=vmax)


def particles_at(seed: int, idx, L=(1.0, 1.0, 1.0), qtable=None, vmax: float = 0.0):
    """The particles with the given generation indices (any order, any subset)."""
    idx = np.asarray(idx, dtype=np.uint64)
    if qtable is None:
        qtable = lognormal_qtable()
    pos = np.empty((3, idx.shape[0]))
    for q in range(3):
        pos[q] = float(L[q]) * uniform53(words(seed, idx, q))
    d = diameters_from_words(words(seed, idx, 3), qtable)
    vel = np.zeros((3, idx.shape[0]))
    if vmax != 0.0:
        for q in range(3):
            vel[q] = float(vmax) * (2.0 * uniform53(words(seed, idx, 4 + q)) - 1.0)
    return pos, vel, d, idx.astype(np.uint32)


def cell_centres(n, L=(1.0, 1.0, 1.0)):
    if isinstance(n, int):
        n = (n, n, n)
    ax = [(np.arange(n[q]) + 0.5) * (float(L[q]) / n[q]) for q in range(3)]
    z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return x, y, z


def taylor_green(n, U0: float = 1.0, L=(1.0, 1.0, 1.0)) -> np.ndarray:
    x, y, z = cell_centres(n, L)
    tx, ty, tz = (2 * np.pi * x / L[0], 2 * np.pi * y / L[1], 2 * np.pi * z / L[2])
    U = np.zeros(x.shape + (3,))
    U[..., 0] = U0 * np.sin(tx) * np.cos(ty) * np.cos(tz)
    U[..., 1] = -U0 * np.cos(tx) * np.sin(ty) * np.cos(tz)
    return U


def uniform_field(n, u) -> np.ndarray:
    if isinstance(n, int):
        n = (n, n, n)
    U = np.empty((n[2], n[1], n[0], 3))
    U[...] = np.asarray(u, dtype=np.float64)
    return U


def random_fourier(n: int, kmax: int = 8, slope: float = -5.0 / 3.0, rms: float = 1.0,
                   seed: int = 1) -> np.ndarray:
    """Divergence-free random Fourier field on an n^3 periodic grid, [k][j][i][3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ks = np.arange(-kmax, kmax + 1)
    KZ, KY, KX = np.meshgrid(ks, ks, ks, indexing="ij")
    kk = np.stack([KX, KY, KZ], axis=-1).reshape(-1, 3)
    kn = np.sqrt((kk.astype(np.float64) ** 2).sum(1))
    keep = (kn >= 1.0) & (kn <= kmax)
    kk, kn = kk[keep], kn[keep]
    # one representative of each +-k pair: the first nonzero component positive
    first = np.where(kk[:, 0] != 0, kk[:, 0], np.where(kk[:, 1] != 0, kk[:, 1], kk[:, 2]))
    half = first > 0
    kk, kn = kk[half], kn[half]
    amp = np.sqrt(kn ** slope / (4.0 * np.pi * kn ** 2))
    coef = (rng.standard_normal((kk.shape[0], 3)) + 1j * rng.standard_normal((kk.shape[0], 3)))
    coef *= amp[:, None] / np.sqrt(2.0)
    kf = kk.astype(np.float64)
    coef -= kf * ((coef * kf).sum(1) / (kn ** 2))[:, None]
    spec = np.zeros((3, n, n, n), dtype=np.complex128)  # [comp][kz][ky][kx]
    iz, iy, ix = kk[:, 2] % n, kk[:, 1] % n, kk[:, 0] % n
    jz, jy, jx = (-kk[:, 2]) % n, (-kk[:, 1]) % n, (-kk[:, 0]) % n
    for q in range(3):
        spec[q, iz, iy, ix] = coef[:, q]
        spec[q, jz, jy, jx] = np.conj(coef[:, q])
    # value at cell centres x = (i + 1/2)/n: phase shift e^{i pi k / n} per axis
    sh = [np.exp(1j * np.pi * np.fft.fftfreq(n, d=1.0 / n) / n) for _ in range(3)]
    U = np.empty((n, n, n, 3))
    for q in range(3):
        s = spec[q] * sh[2][:, None, None] * sh[1][None, :, None] * sh[0][None, None, :]
        U[..., q] = np.fft.ifftn(s).real * (n ** 3)
    del spec
    cur = math.sqrt(float((U ** 2).sum()) / (3.0 * U[..., 0].size))
    U *= rms / cur
    return U


def taylor_green_plus_fourier(n: int, U0: float = 1.0, frac: float = 0.1, seed: int = 3) -> np.ndarray:
    """Taylor-Green vortex plus a random Fourier field of rms frac * (TG component rms)."""
    tg = taylor_green(n, U0)
    tg_rms = U0 / math.sqrt(8.0)
    return tg + random_fourier(n, rms=frac * tg_rms, seed=seed)


def thermo_fields(n: int, seed: int = 7, T_mean: float = 285.0, T_amp: float = 3.0, rv_mean: float = 0.0105,
                  rv_frac: float = 0.05):
    """Fluid temperature (K) and water vapour density (kg/m^3) at cell centres, [k][j][i] each: smooth seeded
    random fields (the first and second components of a random Fourier field, rms 1 per component on
    average) scaled to T_mean +- T_amp and rv_mean (1 +- rv_frac) - a stand-in for a cloud chamber's air
    between 283 and 293 K near water saturation."""
    F = random_fourier(n, seed=seed)
    return T_mean + T_amp * F[..., 0], rv_mean * (1.0 + rv_frac * F[..., 1])


@dataclass
class Workload:
    """A seeded synthetic workload shaped like the paper's (sizes, distributions)."""
    name: str
    grid: int
    field: str                 # "taylor_green" | "fourier" | "tg_fourier" | "uniform"
    field_dtype: str           # "f64" | "f32"
    precision: str             # "fp64" | "mixed_f32" | "mixed_bf16"
    n: int
    steps: int
    dt: float
    reorder_every: int = 10
    chunk_edge: int = 8
    seed: int = 12345
    field_seed: int = 1
    vmax: float = 0.0
    uniform_u: tuple = (0.3, -0.2, 0.1)
    extra: dict = field(default_factory=dict)

    def make_field(self) -> np.ndarray:
        if self.field == "taylor_green":
            U = taylor_green(self.grid)
        elif self.field == "fourier":
            U = random_fourier(self.grid, seed=self.field_seed)
        elif self.field == "tg_fourier":
            U = taylor_green_plus_fourier(self.grid, seed=self.field_seed)
        elif self.field == "uniform":
            U = uniform_field(self.grid, self.uniform_u)
        else:
            raise ValueError(self.field)
        if self.field_dtype == "f32":
            U = U.astype(np.float32).astype(np.float64)
        return U


# Synthetic stand-ins for the paper's workloads (the cloud-chamber fields and
# scaling cases are not available): uniform positions in a periodic unit box,
# zero initial velocity, lognormal diameters (median 20 um, sigma_g 1.5),
# rho_p = 1000, mu = 1.8e-5, gravity -9.81 z.
WORKLOADS = {
    "tg32_fp64_1e5": Workload("tg32_fp64_1e5", 32, "taylor_green", "f64", "fp64", 100_000, 100, 1e-3),
    "fourier128_fp64_1e8": Workload("fourier128_fp64_1e8", 128, "fourier", "f64", "fp64", 100_000_000,
                                    50, 5e-4),
    "uniform128_fp64_1e6": Workload("uniform128_fp64_1e6", 128, "uniform", "f64", "fp64", 1_000_000, 50,
                                    5e-4, vmax=1.0),
    "fourier256_mixed_1e9": Workload("fourier256_mixed_1e9", 256, "fourier", "f32", "mixed_f32",
                                     1_000_000_000, 20, 5e-4),
    "fourier256_bf16v_1e9": Workload("fourier256_bf16v_1e9", 256, "fourier", "f32", "mixed_bf16",
                                     1_000_000_000, 20, 5e-4),
    "tgf64_adjoint_1e7": Workload("tgf64_adjoint_1e7", 64, "tg_fourier", "f32", "fp64", 10_000_000, 200,
                                  1e-3, reorder_every=20, field_seed=3, extra={"checkpoint": 20}),
    "fourier256_coupled_2e9": Workload("fourier256_coupled_2e9", 256, "fourier", "f32", "mixed_f32",
                                       2_000_000_000, 50, 5e-4, chunk_edge=32,
                                       extra={"fluid_every": 5, "nu": 1e-3}),
    # droplet microphysics (vapour and heat transfer) on the mixed-precision workload's field and particles
    "fourier256_micro_1e9": Workload("fourier256_micro_1e9", 256, "fourier", "f32", "mixed_f32",
                                     1_000_000_000, 20, 5e-4, extra={"micro": True}),
    # the mixed-precision workload's field and particles held in pinned host memory as chunks of 2.5e8
    "fourier256_chunks_1e9": Workload("fourier256_chunks_1e9", 256, "fourier", "f32", "mixed_f32",
                                      1_000_000_000, 10, 5e-4, extra={"chunk": 250_000_000}),
}

PHYSICS = dict(rho_p=1000.0, mu=1.8e-5, g=(0.0, 0.0, -9.81), drag_scale=1.0, multiplicity=1.0)
