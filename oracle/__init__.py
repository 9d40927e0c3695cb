"""FP64 CPU oracle for the per-particle Lagrangian step (test infrastructure).

This package is the plain, slow reference the CUDA path is checked against.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library under ``paper_2603_26691_gb300``
never does.  The arithmetic lives in ``oracle.c`` (plain C, double precision,
no FMA contraction); this module compiles it with gcc and wraps it with
ctypes, converting numpy arrays.  It holds no arithmetic of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, no FP contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    hdr = os.path.join(_HERE, "oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("n", C.c_int32 * 3), ("chunk_edge", C.c_int32), ("L", C.c_double * 3),
                ("rho_p", C.c_double), ("mu", C.c_double), ("g", C.c_double * 3),
                ("alpha", C.c_double), ("mult", C.c_double), ("gather", C.c_int32),
                ("integrator", C.c_int32), ("drag", C.c_int32), ("deposit", C.c_int32),
                ("rho_f", C.c_double)]


class Micro(C.Structure):
    _fields_ = [("D_v", C.c_double), ("kappa_f", C.c_double), ("cp_p", C.c_double), ("L", C.c_double),
                ("Pr", C.c_double), ("d_min", C.c_double)]


def make_micro(D_v=2.5e-5, kappa_f=0.025, cp_p=4186.0, L=2.5e6, Pr=0.71, d_min=1e-7) -> Micro:
    """Droplet microphysics parameters (defaults: water droplets in air near 285 K)."""
    M = Micro()
    M.D_v, M.kappa_f, M.cp_p, M.L, M.Pr, M.d_min = (float(D_v), float(kappa_f), float(cp_p), float(L),
                                                    float(Pr), float(d_min))
    return M


GATHERS = {"trilinear": 0, "ngp": 1}
INTEGRATORS = {"exponential": 0, "semi_implicit": 1}
DRAGS = {"stokes": 0, "schiller_naumann": 1}
DEPOSITS = {"cell": 0, "cic": 1}


def make_grid(n, L=(1.0, 1.0, 1.0), chunk_edge=8, rho_p=1000.0, mu=1.8e-5,
              g=(0.0, 0.0, -9.81), alpha=1.0, mult=1.0, gather="trilinear", integrator="exponential",
              drag="stokes", deposit="cell", rho_f=1.2) -> Grid:
    if isinstance(n, int):
        n = (n, n, n)
    G = Grid()
    G.n[:] = [int(v) for v in n]
    G.chunk_edge = int(chunk_edge)
    G.L[:] = [float(v) for v in L]
    G.rho_p, G.mu = float(rho_p), float(mu)
    G.g[:] = [float(v) for v in g]
    G.alpha, G.mult = float(alpha), float(mult)
    G.gather, G.integrator = GATHERS[gather], INTEGRATORS[integrator]
    G.drag, G.deposit = DRAGS[drag], DEPOSITS[deposit]
    G.rho_f = float(rho_f)
    return G


_P = C.POINTER


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i64, i32 = C.c_double, C.c_int64, C.c_int32
            pd, pi64, pu32 = _P(d), _P(i64), _P(C.c_uint32)
            pg = _P(Grid)
            L.orc_wrap.argtypes, L.orc_wrap.restype = [d, d], d
            L.orc_cell.argtypes, L.orc_cell.restype = [pg, pd, _P(i32)], None
            L.orc_gather.argtypes, L.orc_gather.restype = [pg, pd, pd, pd], None
            L.orc_advance.argtypes, L.orc_advance.restype = [pg, d, pd, d, pd, pd], None
            L.orc_mass.argtypes, L.orc_mass.restype = [pg, d], d
            L.orc_drag_factor.argtypes, L.orc_drag_factor.restype = [pg, d], d
            L.orc_deposit.argtypes, L.orc_deposit.restype = [pg, pd, pd, pd], None
            L.orc_particle_step.argtypes = [pg, pd, d, d, pd, pd, pi64, pd]
            L.orc_particle_step.restype = None
            L.orc_run.argtypes = [pg, pd, i64, pd, pd, pd, i32, d, pd, pi64, pi64]
            L.orc_run.restype = C.c_int
            L.orc_key.argtypes, L.orc_key.restype = [pg, i32, i32, i32], C.c_uint32
            L.orc_sort_perm.argtypes, L.orc_sort_perm.restype = [i64, pu32, pi64], None
            L.orc_cell_counts.argtypes, L.orc_cell_counts.restype = [pg, i64, pd, pi64], None
            L.orc_invariants.argtypes, L.orc_invariants.restype = [pg, i64, pd, pd, pd, pd], None
            L.orc_adjoint.argtypes = [pg, pd, i64, pd, pd, pd, i32, d, pd, pd, pd, pd]
            L.orc_adjoint.restype = C.c_int
            L.orc_ecm_estimate.argtypes, L.orc_ecm_estimate.restype = [i32, i64, pd, pd, pd, pd], None
            L.orc_chunk_bounds.argtypes, L.orc_chunk_bounds.restype = [pg, i64, pd, pd, pd], i64
            L.orc_fluid_update.argtypes = [pg, pd, pd, d, d, d, i32]
            L.orc_fluid_update.restype = C.c_int
            L.orc_couple.argtypes = [pg, pd, i64, pd, pd, pd, i32, i32, d, d, d, i32, i32, pd]
            L.orc_couple.restype = C.c_int
            L.orc_rho_sat.argtypes, L.orc_rho_sat.restype = [d], d
            L.orc_rho_sat_dT.argtypes, L.orc_rho_sat_dT.restype = [d], d
            L.orc_nusselt.argtypes, L.orc_nusselt.restype = [_P(Micro), d], d
            L.orc_micro_run.argtypes = [pg, _P(Micro), pd, pd, pd, i64, pd, pd, pd, pd, i32, d, pd, pd, pd]
            L.orc_micro_run.restype = C.c_int
            _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(_P(C.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def ncell(G: Grid) -> int:
    return int(G.n[0]) * int(G.n[1]) * int(G.n[2])


def wrap(x: float, L: float) -> float:
    return lib().orc_wrap(float(x), float(L))


def cell(G: Grid, x) -> tuple:
    x = _f64(x, (3,))
    out = (C.c_int32 * 3)()
    lib().orc_cell(C.byref(G), _pd(x), out)
    return tuple(out)


def gather(G: Grid, U: np.ndarray, x) -> np.ndarray:
    U = _f64(U)
    x = _f64(x, (3,))
    out = np.zeros(3)
    lib().orc_gather(C.byref(G), _pd(U), _pd(x), _pd(out))
    return out


def advance(G: Grid, d: float, up, dt: float, x, v):
    x = _f64(x, (3,)).copy()
    v = _f64(v, (3,)).copy()
    up = _f64(up, (3,))
    lib().orc_advance(C.byref(G), float(d), _pd(up), float(dt), _pd(x), _pd(v))
    return x, v


def mass(G: Grid, d: float) -> float:
    return lib().orc_mass(C.byref(G), float(d))


def drag_factor(G: Grid, re: float) -> float:
    return lib().orc_drag_factor(C.byref(G), float(re))


def deposit(G: Grid, x, J, src=None) -> np.ndarray:
    """Add one particle's impulse J at start position x into src [3, ncell] (a copy)."""
    x = _f64(x, (3,))
    J = _f64(J, (3,))
    src = np.zeros((3, ncell(G))) if src is None else _f64(src).reshape(3, -1).copy()
    lib().orc_deposit(C.byref(G), _pd(x), _pd(J), _pd(src))
    return src


def run(G: Grid, U, pos, vel, d, nsteps: int, dt: float, src=None, trace=False, frozen=None, inplace=False):
    """Advance particles nsteps in the frozen field U.

    pos, vel: [3, n] float64 (copied); d: [n].  Returns (pos, vel, src, trace)
    with src [3, ncell] (accumulated onto the given src if any; with inplace=True
    the given src, a C-contiguous float64 [3, ncell] array, is added to directly
    instead of a copy) and trace [nsteps, n] int64 deposit cells when requested.
    """
    U = _f64(U)
    pos = _f64(pos).reshape(3, -1).copy()
    vel = _f64(vel).reshape(3, -1).copy()
    d = _f64(d).reshape(-1)
    n = d.shape[0]
    nc = ncell(G)
    if inplace:
        if not (isinstance(src, np.ndarray) and src.dtype == np.float64 and src.flags.c_contiguous
                and src.size == 3 * nc):
            raise ValueError("inplace needs a C-contiguous float64 src of 3 * ncell values")
    else:
        src = np.zeros((3, nc)) if src is None else _f64(src).reshape(3, nc).copy()
    tr = np.zeros((max(nsteps, 0), n), dtype=np.int64) if trace else None
    fr = None
    if frozen is not None:
        fr = np.ascontiguousarray(frozen, dtype=np.int64).reshape(nsteps, n)
    rc = lib().orc_run(C.byref(G), _pd(U), n, _pd(pos), _pd(vel), _pd(d), int(nsteps), float(dt),
                       _pd(src), tr.ctypes.data_as(_P(C.c_int64)) if tr is not None else None,
                       fr.ctypes.data_as(_P(C.c_int64)) if fr is not None else None)
    if rc != 0:
        raise ValueError(f"orc_run failed ({rc})")
    return pos, vel, src, tr


def key(G: Grid, i: int, j: int, k: int) -> int:
    return int(lib().orc_key(C.byref(G), int(i), int(j), int(k)))


def keys_of_positions(G: Grid, pos) -> np.ndarray:
    pos = _f64(pos).reshape(3, -1)
    out = np.empty(pos.shape[1], dtype=np.uint32)
    for p in range(pos.shape[1]):
        i, j, k = cell(G, pos[:, p])
        out[p] = key(G, i, j, k)
    return out


def sort_perm(keys) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    n = keys.shape[0]
    perm = np.zeros(n, dtype=np.int64)
    lib().orc_sort_perm(n, keys.ctypes.data_as(_P(C.c_uint32)), perm.ctypes.data_as(_P(C.c_int64)))
    return perm


def cell_counts(G: Grid, pos) -> np.ndarray:
    pos = _f64(pos).reshape(3, -1)
    out = np.zeros(ncell(G), dtype=np.int64)
    lib().orc_cell_counts(C.byref(G), pos.shape[1], _pd(pos), out.ctypes.data_as(_P(C.c_int64)))
    return out


def invariants(G: Grid, vel, d, src=None) -> np.ndarray:
    vel = _f64(vel).reshape(3, -1)
    d = _f64(d).reshape(-1)
    out = np.zeros(8)
    s = _f64(src).reshape(-1) if src is not None else None
    lib().orc_invariants(C.byref(G), d.shape[0], _pd(vel), _pd(d), _pd(s) if s is not None else None,
                         _pd(out))
    return out


def adjoint(G: Grid, U, pos0, vel0, d, nsteps: int, dt: float, lam):
    """Gradients (dL/dd [n], dL/dalpha, dL/dU [ncell, 3]) given lam = dL/dJtot [3, ncell]."""
    U = _f64(U)
    pos0 = _f64(pos0).reshape(3, -1)
    vel0 = _f64(vel0).reshape(3, -1)
    d = _f64(d).reshape(-1)
    lam = _f64(lam).reshape(3, -1)
    n = d.shape[0]
    gd = np.zeros(n)
    ga = C.c_double(0.0)
    gU = np.zeros((ncell(G), 3))
    rc = lib().orc_adjoint(C.byref(G), _pd(U), n, _pd(pos0), _pd(vel0), _pd(d), int(nsteps), float(dt),
                           _pd(lam), _pd(gd), C.byref(ga), _pd(gU))
    if rc != 0:
        raise ValueError(f"orc_adjoint failed ({rc})")
    return gd, ga.value, gU


EXTRAPOLATORS = {"zero": 0, "const": 1, "lin": 2}


def ecm_estimate(extrap: str, s1=None, s2=None, s3=None, m=None) -> np.ndarray:
    """S_est^n from S^{n-1}, S^{n-2}, S^{n-3} (None = before the first interval)."""
    arrs = [None if a is None else _f64(a).reshape(-1) for a in (s1, s2, s3)]
    if m is None:
        m = next(a.shape[0] for a in arrs if a is not None)
    out = np.zeros(m)
    lib().orc_ecm_estimate(EXTRAPOLATORS[extrap], m, *[_pd(a) if a is not None else None for a in arrs], _pd(out))
    return out


def fluid_update(G: Grid, U, S, rho_f: float, nu: float, dtc: float, sweeps: int) -> np.ndarray:
    """One coupling interval's fluid update of U [.., 3] (copied) with the impulse S [3, ncell]."""
    shape = np.shape(U)
    U = _f64(U).reshape(-1).copy()
    S = _f64(S).reshape(-1) if S is not None else None
    rc = lib().orc_fluid_update(C.byref(G), _pd(U), _pd(S) if S is not None else None, float(rho_f), float(nu),
                                float(dtc), int(sweeps))
    if rc != 0:
        raise ValueError(f"orc_fluid_update failed ({rc})")
    return U.reshape(shape)


def couple(G: Grid, U, pos, vel, d, nint: int, K: int, dt: float, rho_f: float, nu: float, sweeps: int,
           extrap: str = "zero"):
    """Asynchronous coupled run; returns (U, pos, vel, pending [3, ncell]) (inputs copied)."""
    shape = np.shape(U)
    U = _f64(U).reshape(-1).copy()
    pos = _f64(pos).reshape(3, -1).copy()
    vel = _f64(vel).reshape(3, -1).copy()
    d = _f64(d).reshape(-1)
    pending = np.zeros((3, ncell(G)))
    rc = lib().orc_couple(C.byref(G), _pd(U), d.shape[0], _pd(pos), _pd(vel), _pd(d), int(nint), int(K), float(dt),
                          float(rho_f), float(nu), int(sweeps), EXTRAPOLATORS[extrap], _pd(pending))
    if rc != 0:
        raise ValueError(f"orc_couple failed ({rc})")
    return U.reshape(shape), pos, vel, pending


def chunk_bounds(G: Grid, pos_sort, pos_now) -> np.ndarray:
    """Per-chunk boxes [nchunk, 6] = (min xyz, max xyz) of the current positions of each chunk's
    particles (membership from pos_sort), unwrapped to the image nearest the chunk centre."""
    pos_sort = _f64(pos_sort).reshape(3, -1)
    pos_now = _f64(pos_now).reshape(3, -1)
    B = int(G.chunk_edge)
    nch = int(np.prod([(int(G.n[q]) + B - 1) // B for q in range(3)]))
    out = np.zeros((nch, 6))
    r = lib().orc_chunk_bounds(C.byref(G), pos_sort.shape[1], _pd(pos_sort), _pd(pos_now), _pd(out))
    if r < 0:
        raise ValueError("orc_chunk_bounds failed")
    return out


def rho_sat(T: float) -> float:
    """Saturation vapour density over flat water (kg/m^3) at T (K)."""
    return lib().orc_rho_sat(float(T))


def rho_sat_dT(T: float) -> float:
    """d rho_sat / dT (kg/(m^3 K)) at T (K)."""
    return lib().orc_rho_sat_dT(float(T))


def nusselt(M: Micro, re: float) -> float:
    return lib().orc_nusselt(C.byref(M), float(re))


def micro_run(G: Grid, M: Micro, U, Tf, rhov, pos, vel, d, Tp, nsteps: int, dt: float):
    """Droplets with vapour mass and heat transfer: nsteps steps in the frozen fields U [.., 3], Tf and rhov
    [ncell].  Returns (pos, vel, d, Tp, src [3, ncell], msrc [ncell], esrc [ncell]) (inputs copied)."""
    U = _f64(U)
    Tf = _f64(Tf).reshape(-1)
    rhov = _f64(rhov).reshape(-1)
    pos = _f64(pos).reshape(3, -1).copy()
    vel = _f64(vel).reshape(3, -1).copy()
    d = _f64(d).reshape(-1).copy()
    Tp = _f64(Tp).reshape(-1).copy()
    n = d.shape[0]
    nc = ncell(G)
    src, msrc, esrc = np.zeros((3, nc)), np.zeros(nc), np.zeros(nc)
    rc = lib().orc_micro_run(C.byref(G), C.byref(M), _pd(U), _pd(Tf), _pd(rhov), n, _pd(pos), _pd(vel), _pd(d),
                             _pd(Tp), int(nsteps), float(dt), _pd(src), _pd(msrc), _pd(esrc))
    if rc != 0:
        raise ValueError(f"orc_micro_run failed ({rc})")
    return pos, vel, d, Tp, src, msrc, esrc


def run_blocked(G: Grid, U, particles, n: int, nsteps: int, dt: float, block: int = 1_000_000, threads: int = 0,
                src=None, keep=None):
    """orc_run over n particles on several host threads, deterministically: the particles are cut into fixed
    blocks of `block` consecutive indices; each block runs its nsteps alone (its own partial source field,
    added to in the block's step-major particle order) and the partial fields are added to `src` in block
    order.  The sums therefore depend on `block` but not on `threads` (0 = every core).  `particles(first,
    count)` returns (pos, vel, d) of those particles, so no more than `threads` blocks are held at once.
    keep(first, pos, vel) is called with each block's final state (in block order).  Returns src
    [3, ncell]."""
    import concurrent.futures as cf

    nc = ncell(G)
    src = np.zeros((3, nc)) if src is None else src
    threads = threads or (os.cpu_count() or 1)
    U = _f64(U)
    nblocks = (n + block - 1) // block

    def work(b):
        first = b * block
        cnt = min(block, n - first)
        pos, vel, d = particles(first, cnt)
        part = np.zeros((3, nc))
        pos, vel, part, _ = run(G, U, pos, vel, d, nsteps, dt, src=part, inplace=True)
        return first, pos, vel, part

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        pending = {}
        nxt = 0
        for b in range(min(nblocks, threads)):
            pending[b] = ex.submit(work, b)
        issued = len(pending)
        while nxt < nblocks:
            first, pos, vel, part = pending.pop(nxt).result()
            np.add(src, part, out=src)
            if keep is not None:
                keep(first, pos, vel)
            del part
            nxt += 1
            if issued < nblocks:
                pending[issued] = ex.submit(work, issued)
                issued += 1
    return src


def adjoint_blocked(G: Grid, U, particles, n: int, nsteps: int, dt: float, lam, block: int = 20_000,
                    threads: int = 0, keep=None):
    """orc_adjoint over n particles on several host threads, deterministically: fixed blocks of `block`
    consecutive particles, each block's adjoint run alone (its trajectory stored whole), the blocks'
    dL/dalpha and dL/dU added in block order (independent of `threads`; 0 = every core).  The loss is
    any L(Jtot) with lam = dL/dJtot held fixed (a loss linear in Jtot), so the particles' contributions
    are independent.  `particles(first, count)` returns (pos0, vel0, d); keep(first, grad_d) receives each
    block's dL/dd in block order.  Returns (dL/dalpha, dL/dU [ncell, 3])."""
    import concurrent.futures as cf

    threads = threads or (os.cpu_count() or 1)
    U = _f64(U)
    lam = _f64(lam).reshape(3, -1)
    nblocks = (n + block - 1) // block
    ga_tot = 0.0
    gU_tot = np.zeros((ncell(G), 3))

    def work(b):
        first = b * block
        cnt = min(block, n - first)
        pos, vel, d = particles(first, cnt)
        gd, ga, gU = adjoint(G, U, pos, vel, d, nsteps, dt, lam)
        return first, gd, ga, gU

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        pending = {b: ex.submit(work, b) for b in range(min(nblocks, threads))}
        issued = len(pending)
        for b in range(nblocks):
            first, gd, ga, gU = pending.pop(b).result()
            ga_tot = ga_tot + ga
            np.add(gU_tot, gU, out=gU_tot)
            if keep is not None:
                keep(first, gd)
            if issued < nblocks:
                pending[issued] = ex.submit(work, issued)
                issued += 1
    return ga_tot, gU_tot
