"""Python binding of the Lagrangian step: a thin wrapper over the C ABI.

PyTorch supplies device memory (the library allocates through torch's
caching allocator) and the CUDA stream; every step of the path runs in the
CUDA library.  Arrays go in and out as torch CUDA tensors or numpy arrays.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import StError, check


def _is_cuda(x) -> bool:
    return isinstance(x, torch.Tensor) and x.is_cuda


def _as_f64(x, shape=None, device=None):
    """Contiguous float64 tensor or numpy array, and whether it lives on the device."""
    if isinstance(x, torch.Tensor):
        t = x.to(torch.float64).contiguous()
        if shape is not None:
            t = t.reshape(shape)
        return t, t.is_cuda
    a = np.ascontiguousarray(x, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a, False


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return C.c_void_p(x.data_ptr())
    return C.c_void_p(x.ctypes.data)


class Sim:
    """One simulation: a periodic grid, a frozen fluid field and particles.

    Parameters follow st_create_grid: grid (nx, ny, nz), box lengths, chunk edge
    B, precision "fp64" | "mixed_f32" | "mixed_bf16".
    """

    def __init__(self, grid, box=(1.0, 1.0, 1.0), chunk_edge: int = 8, precision: str = "fp64",
                 device="cuda", stream: torch.cuda.Stream | None = None, torch_allocator: bool = True):
        self.lib = _lib.load()
        if isinstance(grid, int):
            grid = (grid, grid, grid)
        self.grid = tuple(int(g) for g in grid)
        self.box = tuple(float(b) for b in box)
        self.ncell = self.grid[0] * self.grid[1] * self.grid[2]
        self.precision = precision
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._alloc = None
        if torch_allocator:
            dev, strm = self.device.index, self.stream

            def _a(size, user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(size), dev, strm)
                except Exception:
                    return None

            def _f(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_fns = (_lib.ALLOC_FN(_a), _lib.FREE_FN(_f))
            self._alloc = _lib.Allocator(self._alloc_fns[0], self._alloc_fns[1], None)
        h = C.c_void_p()
        self.chunk_edge = int(chunk_edge)
        st = self.lib.st_create_grid(*self.grid, *self.box, int(chunk_edge), _lib.PRECISIONS[precision],
                                     C.byref(self._alloc) if self._alloc is not None else None,
                                     C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if st != _lib.ST_OK:
            raise StError(st, "st_create_grid", "")
        self.h = h
        self.params = dict(rho_p=1000.0, mu=1.8e-5, g=(0.0, 0.0, -9.81), drag_scale=1.0, multiplicity=1.0,
                           reorder_every=10)
        # bumped by every call that changes the particles, parameters, physics, fluid or the recorded
        # adjoint run, so that a differentiable forward can tell whether its run is still the one the
        # handle would differentiate
        self.generation = 0

    def _changed(self):
        self.generation += 1

    # -- lifetime ------------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.st_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _chk(self, st, where):
        check(st, self.h, where)

    # -- parameters and fields ---------------------------------------------------------------
    def set_params(self, rho_p=1000.0, mu=1.8e-5, g=(0.0, 0.0, -9.81), drag_scale=1.0, multiplicity=1.0,
                   reorder_every=10):
        self.params = dict(rho_p=rho_p, mu=mu, g=tuple(g), drag_scale=drag_scale, multiplicity=multiplicity,
                           reorder_every=reorder_every)
        garr = (C.c_double * 3)(*[float(x) for x in g])
        self._changed()
        self._chk(self.lib.st_set_params(self.h, float(rho_p), float(mu), garr, float(drag_scale),
                                         float(multiplicity), int(reorder_every)), "st_set_params")

    GATHERS = {"trilinear": 0, "ngp": 1}
    INTEGRATORS = {"exponential": 0, "semi_implicit": 1}
    DRAGS = {"stokes": 0, "schiller_naumann": 1}
    DEPOSITS = {"cell": 0, "cic": 1}

    def set_physics(self, gather="trilinear", integrator="exponential", drag="stokes", deposit="cell", rho_f=1.2):
        """Physics variants: nearest-grid-point gather, semi-implicit Euler, Schiller-Naumann drag
        (rho_f: fluid density in the particle Reynolds number), cloud-in-cell deposit."""
        self.physics = dict(gather=gather, integrator=integrator, drag=drag, deposit=deposit, rho_f=rho_f)
        self._changed()
        self._chk(self.lib.st_set_physics(self.h, self.GATHERS[gather], self.INTEGRATORS[integrator],
                                          self.DRAGS[drag], self.DEPOSITS[deposit], float(rho_f)),
                  "st_set_physics")

    def probe_fma(self):
        """(FP64, FP32) fused multiply-add rates of this GPU in GFLOP/s."""
        a, b = C.c_double(), C.c_double()
        self._chk(self.lib.st_probe_fma(self.h, C.byref(a), C.byref(b)), "st_probe_fma")
        return a.value, b.value

    TIMERS = ("step", "sort", "adjoint", "fluid")

    def timers(self, on=None, reset=False):
        """Library kernel timers: timers(True) clears and starts, timers(False) stops; timers() returns
        {kind: (ms, launches)} (synchronises)."""
        if on is not None:
            self._chk(self.lib.st_timers_enable(self.h, int(bool(on))), "st_timers_enable")
            return None
        ms = (C.c_double * 4)()
        cnt = (C.c_int64 * 4)()
        self._chk(self.lib.st_timers_read(self.h, ms, cnt, int(reset)), "st_timers_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.TIMERS)}

    def set_fluid(self, U):
        """Cell-centred velocity [nz, ny, nx, 3] (float32 or float64; numpy or torch)."""
        self._changed()
        if isinstance(U, torch.Tensor):
            t = U.contiguous()
            if t.dtype not in (torch.float32, torch.float64):
                t = t.to(torch.float64)
            dt = _lib.ST_DTYPE_F32 if t.dtype == torch.float32 else _lib.ST_DTYPE_F64
            if t.numel() != 3 * self.ncell:
                raise ValueError("fluid field has the wrong size")
            self._chk(self.lib.st_set_fluid(self.h, C.c_void_p(t.data_ptr()), dt, int(t.is_cuda)), "st_set_fluid")
        else:
            a = np.ascontiguousarray(U)
            if a.dtype not in (np.float32, np.float64):
                a = a.astype(np.float64)
            if a.size != 3 * self.ncell:
                raise ValueError("fluid field has the wrong size")
            dt = _lib.ST_DTYPE_F32 if a.dtype == np.float32 else _lib.ST_DTYPE_F64
            self._chk(self.lib.st_set_fluid(self.h, C.c_void_p(a.ctypes.data), dt, 0), "st_set_fluid")

    # -- particles -----------------------------------------------------------------------
    def reserve(self, n: int):
        self._chk(self.lib.st_reserve(self.h, int(n)), "st_reserve")

    def add_particles(self, pos, d, vel=None, ids=None):
        """Append particles: pos [3, n], d [n], vel [3, n] or None, ids [n] uint32 or None."""
        self._changed()
        dd, dev = _as_f64(d, (-1,))
        n = int(dd.shape[0])
        pp, pdev = _as_f64(pos, (3, n))
        vv = None
        if vel is not None:
            vv, vdev = _as_f64(vel, (3, n))
            if vdev != dev:
                raise ValueError("all particle arrays must be on the same side (host or device)")
        if pdev != dev:
            raise ValueError("all particle arrays must be on the same side (host or device)")
        ii = None
        if ids is not None:
            if isinstance(ids, torch.Tensor):
                ii = ids.to(torch.int32).contiguous() if ids.dtype != torch.int32 else ids.contiguous()
                if ii.is_cuda != dev:
                    raise ValueError("ids must be on the same side as the other arrays")
            else:
                ii = np.ascontiguousarray(ids, dtype=np.uint32)
        if dev and pp.device != self.device:
            raise ValueError("device arrays must be on the simulation's device")
        self._chk(self.lib.st_add_particles(self.h, n, _ptr(pp), _ptr(vv), _ptr(dd), _ptr(ii), int(dev)),
                  "st_add_particles")

    @property
    def n(self) -> int:
        v = C.c_int64()
        self._chk(self.lib.st_num_particles(self.h, C.byref(v)), "st_num_particles")
        return int(v.value)

    @property
    def kernel_launches(self) -> int:
        v = C.c_int64()
        self._chk(self.lib.st_kernel_launches(self.h, C.byref(v)), "st_kernel_launches")
        return int(v.value)

    def clear_particles(self):
        self._changed()
        self._chk(self.lib.st_clear_particles(self.h), "st_clear_particles")

    def adjoint_forward(self, nsteps: int, dt: float, checkpoint_every: int):
        self._changed()
        self._chk(self.lib.st_adjoint_forward(self.h, int(nsteps), float(dt), int(checkpoint_every)),
                  "st_adjoint_forward")

    def adjoint_backward(self, lam):
        """Gradients of L(Jtot) given lam = dL/dJtot [3, ncell]: (dL/dd [n], dL/dalpha, dL/dU [ncell, 3])."""
        n = self.n
        if isinstance(lam, torch.Tensor) and lam.is_cuda:
            lt = lam.to(torch.float64).contiguous()
            gd = torch.empty(n, dtype=torch.float64, device=self.device)
            gU = torch.empty((self.ncell, 3), dtype=torch.float64, device=self.device)
            ga = C.c_double()
            self._chk(self.lib.st_adjoint_backward(self.h, _ptr(lt), 1, _ptr(gd), C.byref(ga), _ptr(gU), 1),
                      "st_adjoint_backward")
            return gd, ga.value, gU
        la = np.ascontiguousarray(lam, dtype=np.float64)
        gd = np.empty(n)
        gU = np.empty((self.ncell, 3))
        ga = C.c_double()
        self._chk(self.lib.st_adjoint_backward(self.h, _ptr(la), 0, _ptr(gd), C.byref(ga), _ptr(gU), 0),
                  "st_adjoint_backward")
        return gd, ga.value, gU

    def step(self, nsteps: int, dt: float):
        self._changed()
        self._chk(self.lib.st_step(self.h, int(nsteps), float(dt)), "st_step")

    def reorder(self):
        self._changed()
        self._chk(self.lib.st_reorder(self.h), "st_reorder")

    # -- asynchronous two-way coupling -------------------------------------------------------
    EXTRAPOLATORS = {"zero": 0, "const": 1, "lin": 2}

    def couple_params(self, rho_f: float = 1.2, nu: float = 1e-3, sweeps: int = 10, steps_per_interval: int = 5,
                      extrapolator: str = "zero"):
        self._changed()
        self._chk(self.lib.st_couple_params(self.h, float(rho_f), float(nu), int(sweeps), int(steps_per_interval),
                                            self.EXTRAPOLATORS[extrapolator]), "st_couple_params")

    def couple_run(self, nintervals: int, dt: float):
        self._changed()
        self._chk(self.lib.st_couple_run(self.h, int(nintervals), float(dt)), "st_couple_run")

    def fluid(self, host: bool = True):
        """Current fluid field [nz, ny, nx, 3] float64 (numpy if host, else a device tensor)."""
        shape = (self.grid[2], self.grid[1], self.grid[0], 3)
        if host:
            a = np.empty(shape)
            self._chk(self.lib.st_get_fluid(self.h, C.c_void_p(a.ctypes.data), 0), "st_get_fluid")
            return a
        out = torch.empty(shape, dtype=torch.float64, device=self.device)
        self._chk(self.lib.st_get_fluid(self.h, C.c_void_p(out.data_ptr()), 1), "st_get_fluid")
        return out

    def pending_sources(self, host: bool = True):
        """Sources not yet received by the fluid [3, ncell] float64."""
        if host:
            a = np.empty((3, self.ncell))
            self._chk(self.lib.st_get_pending_sources(self.h, C.c_void_p(a.ctypes.data), 0), "st_get_pending_sources")
            return a
        out = torch.empty((3, self.ncell), dtype=torch.float64, device=self.device)
        self._chk(self.lib.st_get_pending_sources(self.h, C.c_void_p(out.data_ptr()), 1), "st_get_pending_sources")
        return out

    def synchronize(self):
        """Wait for the handle's queued work and asynchronous transfers; report pending errors."""
        self._chk(self.lib.st_synchronize(self.h), "st_synchronize")

    def set_fluid_async(self, U: torch.Tensor):
        """Queue the upload of a host field [nz, ny, nx, 3] (float32 or float64 CPU tensor, pinned for the
        copy to overlap) for the work queued next; U must stay unchanged until the next call on the Sim
        other than sources_async (see st_set_fluid_async)."""
        self._changed()
        if U.is_cuda or U.dtype not in (torch.float32, torch.float64) or not U.is_contiguous():
            raise ValueError("a contiguous float32 or float64 host tensor is required")
        if U.numel() != 3 * self.ncell:
            raise ValueError("fluid field has the wrong size")
        dt = _lib.ST_DTYPE_F32 if U.dtype == torch.float32 else _lib.ST_DTYPE_F64
        self._chk(self.lib.st_set_fluid_async(self.h, C.c_void_p(U.data_ptr()), dt), "st_set_fluid_async")

    def sources_async(self, out: torch.Tensor, reset: bool = False):
        """Queue the copy of the accumulated sources into the float64 host tensor out [3, ncell] (pinned for
        the copy to overlap); out holds them after synchronize() (see st_get_sources_async)."""
        if out.is_cuda or out.dtype != torch.float64 or not out.is_contiguous() or out.numel() != 3 * self.ncell:
            raise ValueError("a contiguous float64 host tensor of 3 x ncell values is required")
        self._chk(self.lib.st_get_sources_async(self.h, C.c_void_p(out.data_ptr()), int(bool(reset))),
                  "st_get_sources_async")

    # -- outputs ---------------------------------------------------------------------------
    def sources(self, reset: bool = False, out: torch.Tensor | None = None, host: bool = False):
        """Accumulated per-cell impulse [3, ncell] float64 (device tensor, or numpy if host)."""
        if host:
            a = np.empty((3, self.ncell))
            self._chk(self.lib.st_get_sources(self.h, C.c_void_p(a.ctypes.data), int(reset), 0), "st_get_sources")
            return a
        if out is None:
            out = torch.empty((3, self.ncell), dtype=torch.float64, device=self.device)
        self._chk(self.lib.st_get_sources(self.h, C.c_void_p(out.data_ptr()), int(reset), 1), "st_get_sources")
        return out

    def sources_fixed(self):
        """The accumulated source as exact fixed-point integers: (words [3, ncell, 4] int64 device tensor
        with 32-bit digits below a signed top word, E) with value = sum_k words[..., k] 2^(32 k - E)."""
        w = torch.empty((3, self.ncell, 4), dtype=torch.int64, device=self.device)
        E = C.c_int()
        self._chk(self.lib.st_get_sources_fixed(self.h, _ptr(w), C.byref(E), 1), "st_get_sources_fixed")
        return w, int(E.value)

    def source_density(self, elapsed: float, reset: bool = False, host: bool = False):
        """The momentum source of Sec. 2.1, Eq. 11, as a rate density: the accumulated impulse per cell
        divided by the cell volume and by the time it was accumulated over (`elapsed`, in s) [3, ncell]."""
        if not elapsed > 0:
            raise ValueError("elapsed must be > 0")
        vol = 1.0
        for b, g in zip(self.box, self.grid):
            vol *= b / g
        return self.sources(reset=reset, host=host) / (vol * elapsed)

    def particles(self, first: int = 0, count: int | None = None, host: bool = True):
        """(pos [3, count], vel [3, count], d [count], ids [count]) in storage order."""
        if count is None:
            count = self.n - first
        if host:
            pos, vel = np.empty((3, count)), np.empty((3, count))
            d, ids = np.empty(count), np.empty(count, dtype=np.uint32)
        else:
            kw = dict(device=self.device)
            pos = torch.empty((3, count), dtype=torch.float64, **kw)
            vel = torch.empty((3, count), dtype=torch.float64, **kw)
            d = torch.empty(count, dtype=torch.float64, **kw)
            ids = torch.empty(count, dtype=torch.int32, **kw)
        self._chk(self.lib.st_get_particles(self.h, int(first), int(count), _ptr(pos), _ptr(vel), _ptr(d), _ptr(ids),
                                            int(not host)), "st_get_particles")
        return pos, vel, d, ids

    def cells(self, first: int = 0, count: int | None = None) -> np.ndarray:
        if count is None:
            count = self.n - first
        out = np.empty(count, dtype=np.int32)
        self._chk(self.lib.st_get_cells(self.h, int(first), int(count), C.c_void_p(out.ctypes.data), 0), "st_get_cells")
        return out

    def cell_counts(self) -> np.ndarray:
        out = np.empty(self.ncell, dtype=np.int64)
        self._chk(self.lib.st_get_cell_counts(self.h, C.c_void_p(out.ctypes.data), 0), "st_get_cell_counts")
        return out

    def chunk_bounds(self) -> np.ndarray:
        """Per-chunk boxes [nchunk, 6] (min xyz, max xyz) of the chunks' current positions."""
        B = self.chunk_edge
        nch = int(np.prod([(g + B - 1) // B for g in self.grid]))
        a = np.empty((nch, 6))
        self._chk(self.lib.st_chunk_bounds(self.h, C.c_void_p(a.ctypes.data), 0), "st_chunk_bounds")
        return a

    def invariants(self) -> np.ndarray:
        out = (C.c_double * 8)()
        self._chk(self.lib.st_invariants(self.h, out), "st_invariants")
        return np.array(out[:])

    # -- chunked particle sets (larger than device memory) -------------------------------------------
    def chunks_create(self, chunk_particles: int):
        """Keep the particles as chunks of chunk_particles in pinned host memory (see st_chunks_create)."""
        self._changed()
        self._chk(self.lib.st_chunks_create(self.h, int(chunk_particles)), "st_chunks_create")

    def chunks_add(self, pos, d, vel=None):
        """Append particles (pos [3, n], d [n], vel [3, n] or None) as new chunks."""
        self._changed()
        dd, dev = _as_f64(d, (-1,))
        n = int(dd.shape[0])
        pp, _ = _as_f64(pos, (3, n))
        vv = None if vel is None else _as_f64(vel, (3, n))[0]
        self._chk(self.lib.st_chunks_add(self.h, n, _ptr(pp), _ptr(vv), _ptr(dd), int(dev)), "st_chunks_add")

    def chunks_step(self, nsteps: int, dt: float):
        """Advance every chunk; returns {wall, compute, h2d, d2h} in ms (CUDA events)."""
        self._changed()
        ms = (C.c_double * 4)()
        self._chk(self.lib.st_chunks_step(self.h, int(nsteps), float(dt), ms), "st_chunks_step")
        return dict(zip(("wall_ms", "compute_ms", "h2d_ms", "d2h_ms"), ms[:]))

    def chunks_count(self):
        a, b = C.c_int64(), C.c_int64()
        self._chk(self.lib.st_chunks_count(self.h, C.byref(a), C.byref(b)), "st_chunks_count")
        return int(a.value), int(b.value)

    def chunks_particles(self, first: int = 0, count: int | None = None):
        """(pos [3, count], vel [3, count], d [count], ids [count]) of the chunks, host arrays."""
        if count is None:
            count = self.chunks_count()[0] - first
        pos, vel = np.empty((3, count)), np.empty((3, count))
        d, ids = np.empty(count), np.empty(count, dtype=np.uint32)
        self._chk(self.lib.st_chunks_get(self.h, int(first), int(count), _ptr(pos), _ptr(vel), _ptr(d), _ptr(ids)),
                  "st_chunks_get")
        return pos, vel, d, ids

    # -- droplet microphysics (vapour mass and heat transfer) ------------------------------------
    def set_microphysics(self, enable: bool = True, D_v: float = 2.5e-5, kappa_f: float = 0.025, cp_p: float = 4186.0,
                         latent_heat: float = 2.5e6, prandtl: float = 0.71, d_min: float = 1e-7,
                         T_init: float = 293.15):
        """Vapour mass and heat transfer of the droplets (off by default; see st_set_microphysics)."""
        self._changed()
        self._chk(self.lib.st_set_microphysics(self.h, int(bool(enable)), float(D_v), float(kappa_f), float(cp_p),
                                               float(latent_heat), float(prandtl), float(d_min), float(T_init)),
                  "st_set_microphysics")

    def set_thermo(self, T, rho_v):
        """Fluid temperature (K) and vapour density (kg/m^3) at cell centres, [nz, ny, nx] each."""
        self._changed()
        if isinstance(T, torch.Tensor) and T.is_cuda:
            t = T.to(torch.float64).contiguous().reshape(-1)
            r = torch.as_tensor(rho_v, dtype=torch.float64, device=t.device).contiguous().reshape(-1)
            if t.numel() != self.ncell or r.numel() != self.ncell:
                raise ValueError("thermo fields have the wrong size")
            self._chk(self.lib.st_set_thermo(self.h, _ptr(t), _ptr(r), _lib.ST_DTYPE_F64, 1), "st_set_thermo")
            return
        t = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
        r = np.ascontiguousarray(rho_v, dtype=np.float64).reshape(-1)
        if t.size != self.ncell or r.size != self.ncell:
            raise ValueError("thermo fields have the wrong size")
        self._chk(self.lib.st_set_thermo(self.h, _ptr(t), _ptr(r), _lib.ST_DTYPE_F64, 0), "st_set_thermo")

    def set_temperatures(self, T, first: int = 0):
        """Particle temperatures (K) of particles [first, first + len(T)) in storage order."""
        self._changed()
        t, dev = _as_f64(T, (-1,))
        self._chk(self.lib.st_set_temperatures(self.h, int(first), int(t.shape[0]), _ptr(t), int(dev)),
                  "st_set_temperatures")

    def temperatures(self, first: int = 0, count: int | None = None) -> np.ndarray:
        """Particle temperatures (K) in storage order."""
        if count is None:
            count = self.n - first
        out = np.empty(count)
        self._chk(self.lib.st_get_temperatures(self.h, int(first), int(count), _ptr(out), 0), "st_get_temperatures")
        return out

    def micro_sources(self, reset: bool = False, host: bool = True):
        """Vapour mass (kg) and energy (J) the fluid gained per cell, [2, ncell] float64."""
        if host:
            a = np.empty((2, self.ncell))
            self._chk(self.lib.st_get_micro_sources(self.h, _ptr(a), int(reset), 0), "st_get_micro_sources")
            return a
        out = torch.empty((2, self.ncell), dtype=torch.float64, device=self.device)
        self._chk(self.lib.st_get_micro_sources(self.h, _ptr(out), int(reset), 1), "st_get_micro_sources")
        return out

    def micro_invariants(self) -> np.ndarray:
        """(sum of particle masses, sum of C_p m T) in FP64."""
        out = (C.c_double * 2)()
        self._chk(self.lib.st_micro_invariants(self.h, out), "st_micro_invariants")
        return np.array(out[:])

    # -- seeded input generator (device twin of inputs.particles) --------------------------
    def gen_particles(self, seed: int, first: int, count: int, qtable, vmax: float = 0.0, L=None):
        """Device FP64 arrays (pos [3,count], vel [3,count], d [count], ids [count] int32)."""
        L = self.box if L is None else L
        q = torch.as_tensor(np.asarray(qtable, dtype=np.float64), device=self.device)
        kw = dict(device=self.device)
        pos = torch.empty((3, count), dtype=torch.float64, **kw)
        vel = torch.empty((3, count), dtype=torch.float64, **kw)
        d = torch.empty(count, dtype=torch.float64, **kw)
        ids = torch.empty(count, dtype=torch.int32, **kw)
        Larr = (C.c_double * 3)(*[float(x) for x in L])
        self._chk(self.lib.st_gen_particles(self.h, int(seed) & 0xFFFFFFFFFFFFFFFF, int(first), int(count), Larr,
                                            float(vmax), C.c_void_p(q.data_ptr()), int(q.numel() - 1), _ptr(pos),
                                            _ptr(vel), _ptr(d), _ptr(ids)), "st_gen_particles")
        return pos, vel, d, ids
