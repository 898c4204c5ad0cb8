"""ctypes binding of the C ABI in ``include/lbib.h`` (argument marshalling only).

Every step of the LB-IB path runs in the CUDA library ``_build/liblbib.so``;
if it has not been built this module raises instead of computing anything
on the host.  Names follow the C calls: ``Sim`` wraps ``lbib_create`` /
``lbib_add_particle`` / ``lbib_set_receptors`` / ``lbib_step`` /
``lbib_read_state``, ``Batch`` wraps ``lbib_batch_*``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# LBIB_DEBUG=1 in the environment loads the bounds-checked debug build
LIB_PATH = os.path.join(HERE, "_build", "liblbib_debug.so" if os.environ.get("LBIB_DEBUG") == "1"
                        else "liblbib.so")
LATTICE_VARIANTS = 6        # LBIB_LATTICE_VARIANTS of include/lbib.h

WALL = {"zou_he": 0, "bounce_back": 1, "periodic": 2}
STORAGE = {"f32": 0, "f64": 1, "f16": 2, "bf16": 3}
STATUS = {0: "OK", 1: "E_ARG", 2: "E_OOM", 3: "E_CUDA", 4: "E_STATE", 5: "E_UNSTABLE",
          6: "E_TIMEOUT", 7: "E_UNSUPPORTED", 8: "E_BOUNDS"}

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class LbibError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("wall_bottom", C.c_int32), ("wall_top", C.c_int32),
        ("tau", C.c_double), ("u_bottom", C.c_double), ("u_top", C.c_double),
        ("gx", C.c_double), ("gy", C.c_double),
        ("k_f", C.c_double), ("k_r0", C.c_double), ("kBT", C.c_double),
        ("sigma_star_ratio", C.c_double), ("y_cr", C.c_double), ("y_eq_ratio", C.c_double),
        ("hamaker", C.c_double), ("eps_min", C.c_double),
        ("receptor_bottom", C.c_double), ("receptor_top", C.c_double),
        ("seed", C.c_uint64), ("sim_id", C.c_uint64),
        ("storage", C.c_int32), ("rounding", C.c_int32),
        ("f16_scale", C.c_double),
        ("cuda_stream", C.c_void_p),
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("ib_iterations", C.c_int32), ("ib_spread", C.c_int32),
        ("stream_mode", C.c_int32), ("reserved2", C.c_int32),
    ]


class Particle(C.Structure):
    _fields_ = [
        ("n_vertices", C.c_int32), ("fixed", C.c_int32),
        ("vx", C.POINTER(C.c_double)), ("vy", C.POINTER(C.c_double)),
        ("shape", C.c_int32), ("reserved0", C.c_int32),
        ("a", C.c_double), ("b", C.c_double),
        ("xc", C.c_double), ("yc", C.c_double), ("theta", C.c_double),
        ("rho_p", C.c_double), ("ligand_density", C.c_double), ("sigma", C.c_double),
    ]


class ParticleState(C.Structure):
    _fields_ = [
        ("xc", C.c_double), ("yc", C.c_double), ("theta", C.c_double),
        ("u", C.c_double), ("v", C.c_double), ("omega", C.c_double),
        ("Fh", C.c_double * 2), ("Mh", C.c_double),
        ("Fb", C.c_double * 2), ("Mb", C.c_double),
        ("Fw", C.c_double * 2),
        ("area", C.c_double), ("mass", C.c_double), ("inertia", C.c_double),
        ("r_eq", C.c_double),
        ("nl", C.c_int32), ("n_ligands", C.c_int32), ("n_probing", C.c_int32),
        ("n_bonded", C.c_int32), ("p_adhesion", C.c_double),
        ("gap_bottom", C.c_double), ("gap_top", C.c_double),
    ]


class ParticleRecord(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("xc", "yc", "theta", "u", "v", "omega",
                                          "xc1", "yc1", "theta1", "u1", "v1", "omega1")] + [
        ("step", C.c_int64)]


class State(C.Structure):
    _fields_ = [("step", C.c_int64), ("n_particles", C.c_int32), ("storage", C.c_int32),
                ("nx", C.c_int32), ("ny", C.c_int32)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load the CUDA library; raises if it was not built (no host fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_1808_01448_gb300.build.build()")
            L = C.CDLL(LIB_PATH)
            vp, i32, i64, d = C.c_void_p, C.c_int32, C.c_int64, C.c_double
            pd = C.POINTER(C.c_double)
            sig = {
                "lbib_create": [C.POINTER(Config), C.POINTER(vp)],
                "lbib_destroy": [vp],
                "lbib_add_particle": [vp, C.POINTER(Particle), C.POINTER(i32)],
                "lbib_set_receptors": [vp, i32, d],
                "lbib_set_populations": [vp, pd],
                "lbib_step": [vp, i64],
                "lbib_batch_create": [C.POINTER(vp), i32, C.POINTER(vp)],
                "lbib_batch_step": [vp, i64],
                "lbib_batch_destroy": [vp],
                "lbib_batch_set_timing": [vp, i32],
                "lbib_batch_kernel_times": [vp, pd, C.POINTER(i64)],
                "lbib_batch_pass_nodes": [vp, C.POINTER(i64)],
                "lbib_batch_step_flushed": [vp, i64, vp, C.c_size_t, i32, pd],
                "lbib_batch_set_particle_threads": [vp, i32],
                "lbib_batch_read_particles_async": [vp],
                "lbib_batch_synchronize": [vp],
                "lbib_batch_read_particles": [vp, C.POINTER(ParticleState), i32, C.POINTER(i32),
                                              C.POINTER(C.c_size_t)],
                "lbib_batch_autotune": [vp, i32, C.POINTER(i32), pd],
                "lbib_batch_set_variant": [vp, i32],
                "lbib_synchronize": [vp],
                "lbib_read_state": [vp, C.POINTER(State), C.POINTER(ParticleState), i32,
                                    pd, pd, pd, C.c_size_t],
                "lbib_read_populations": [vp, pd],
                "lbib_read_bonds": [vp, i32, C.POINTER(C.c_uint8), pd, i32],
                "lbib_read_ib_force": [vp, pd, pd],
                "lbib_ib_force_noalloc": [C.POINTER(Config), vp, C.POINTER(Particle), d, d, d,
                                          vp, vp],
                "lbib_get_particle_record": [vp, i32, C.POINTER(ParticleRecord)],
                "lbib_set_particle_record": [vp, i32, C.POINTER(ParticleRecord)],
                "lbib_checkpoint_size": [vp, C.POINTER(C.c_size_t)],
                "lbib_checkpoint_save": [vp, vp, C.c_size_t],
                "lbib_checkpoint_load": [vp, vp, C.c_size_t],
                "lbib_device_bytes": [vp, C.POINTER(C.c_size_t)],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.lbib_last_error.restype = C.c_char_p
            L.lbib_last_error.argtypes = []
            L.lbib_version.restype = C.c_char_p
            L.lbib_version.argtypes = []
            _lib = L
    return _lib


def _check(code):
    if code != 0:
        raise LbibError(code, lib().lbib_last_error().decode())


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(storage="f32", stream=None, allocator=None, **kw) -> Config:
    c = Config()
    defaults = dict(nx=32, ny=16, wall_bottom="bounce_back", wall_top="bounce_back",
                    tau=0.8, u_bottom=0.0, u_top=0.0, gx=0.0, gy=0.0, k_f=0.85,
                    k_r0=1e-4, kBT=0.1, sigma_star_ratio=0.5, y_cr=1.36,
                    y_eq_ratio=0.5, hamaker=0.0, eps_min=1e-3, receptor_bottom=1.0,
                    receptor_top=0.0, seed=1, sim_id=0, f16_scale=0.0, rounding="stochastic",
                    ib_iterations=1, ib_spread=0, stream_mode="ab")
    defaults.update(kw)
    for k, v in defaults.items():
        if k in ("wall_bottom", "wall_top") and isinstance(v, str):
            v = WALL[v]
        if k == "rounding" and isinstance(v, str):
            v = {"stochastic": 0, "nearest": 1}[v]
        if k == "stream_mode" and isinstance(v, str):
            v = {"ab": 0, "aa": 1}[v]
        setattr(c, k, v)
    c.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    c.cuda_stream = stream
    if allocator is not None:
        c.alloc, c.free = allocator
    return c


def torch_allocator():
    """(alloc, free) callbacks that take device memory from PyTorch's caching
    allocator; keep the returned tuple alive as long as the simulations."""
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      stream or 0)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass

    return ALLOC_FN(_alloc), FREE_FN(_free)


class Sim:
    """One channel simulation resident on the GPU."""

    def __init__(self, storage="f32", stream=None, allocator=None, **cfg):
        self.cfg = make_config(storage=storage, stream=stream, allocator=allocator, **cfg)
        self._alloc_ref = allocator
        self.nx, self.ny = self.cfg.nx, self.cfg.ny
        h = C.c_void_p()
        _check(lib().lbib_create(C.byref(self.cfg), C.byref(h)))
        self._h = h
        self.n_particles = 0
        self._nl = []

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().lbib_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def add_particle(self, vx=None, vy=None, xc=0.0, yc=0.0, theta=0.0, rho_p=1.0,
                     ligand_density=0.5, sigma=1.0, fixed=False, shape=0, a=0.0, b=0.0,
                     n_vertices=0) -> int:
        p = Particle()
        keep = []
        if vx is not None:
            vx = np.ascontiguousarray(vx, dtype=np.float64)
            vy = np.ascontiguousarray(vy, dtype=np.float64)
            keep = [vx, vy]
            p.vx, p.vy, p.n_vertices = _dp(vx), _dp(vy), len(vx)
        else:
            p.n_vertices = n_vertices
        p.fixed, p.shape, p.a, p.b = int(fixed), shape, a, b
        p.xc, p.yc, p.theta, p.rho_p = xc, yc, theta, rho_p
        p.ligand_density, p.sigma = ligand_density, sigma
        pid = C.c_int32()
        _check(lib().lbib_add_particle(self._h, C.byref(p), C.byref(pid)))
        del keep
        self.n_particles += 1
        st = self.particles()[pid.value]
        self._nl.append(st["nl"])
        return pid.value

    def set_receptors(self, wall, density):
        _check(lib().lbib_set_receptors(self._h, int(wall), float(density)))

    def set_populations(self, f_post):
        f = np.ascontiguousarray(f_post, dtype=np.float64).reshape(9, self.ny, self.nx)
        _check(lib().lbib_set_populations(self._h, _dp(f)))

    def step(self, n=1):
        _check(lib().lbib_step(self._h, int(n)))

    def synchronize(self):
        _check(lib().lbib_synchronize(self._h))

    def state(self) -> dict:
        st = State()
        _check(lib().lbib_read_state(self._h, C.byref(st), None, 0, None, None, None, 0))
        return {k: getattr(st, k) for k, _ in State._fields_}

    @property
    def step_count(self):
        return self.state()["step"]

    def fields(self):
        r = np.empty((self.ny, self.nx)); u = np.empty_like(r); v = np.empty_like(r)
        _check(lib().lbib_read_state(self._h, None, None, 0, _dp(r), _dp(u), _dp(v),
                                     self.nx * self.ny))
        return r, u, v

    def particles(self) -> list:
        n = max(self.n_particles, 1)
        arr = (ParticleState * n)()
        _check(lib().lbib_read_state(self._h, None, arr, n, None, None, None, 0))
        out = []
        for k in range(self.n_particles):
            d = {name: getattr(arr[k], name) for name, _ in ParticleState._fields_}
            for key in ("Fh", "Fb", "Fw"):
                d[key] = tuple(d[key])
            out.append(d)
        return out

    def particle(self, pid=0) -> dict:
        return self.particles()[pid]

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        _check(lib().lbib_read_populations(self._h, _dp(f)))
        return f

    def bonds(self, pid=0):
        n = self._nl[pid]
        b = np.zeros(n, dtype=np.uint8); ax = np.zeros(n)
        _check(lib().lbib_read_bonds(self._h, pid, b.ctypes.data_as(C.POINTER(C.c_uint8)),
                                     _dp(ax), n))
        return b, ax

    def ib_force(self):
        fx = np.empty((self.ny, self.nx)); fy = np.empty_like(fx)
        _check(lib().lbib_read_ib_force(self._h, _dp(fx), _dp(fy)))
        return fx, fy

    def record(self, pid=0) -> dict:
        """Pose, velocities, their values one step earlier and the step
        count of a particle (``lbib_get_particle_record``)."""
        r = ParticleRecord()
        _check(lib().lbib_get_particle_record(self._h, pid, C.byref(r)))
        return {k: getattr(r, k) for k, _ in ParticleRecord._fields_}

    def set_record(self, pid=0, **fields):
        """Overwrite a particle's record (``lbib_set_particle_record``);
        fields not given keep their current values."""
        cur = self.record(pid)
        cur.update(fields)
        r = ParticleRecord(**cur)
        _check(lib().lbib_set_particle_record(self._h, pid, C.byref(r)))

    def checkpoint(self) -> bytes:
        """The simulation's state as a host blob (``lbib_checkpoint_save``)."""
        n = C.c_size_t()
        _check(lib().lbib_checkpoint_size(self._h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib().lbib_checkpoint_save(self._h, buf, n.value))
        return buf.raw

    def restore(self, blob: bytes):
        """Load a blob from ``checkpoint`` (``lbib_checkpoint_load``)."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        _check(lib().lbib_checkpoint_load(self._h, buf, len(blob)))

    def device_bytes(self) -> int:
        n = C.c_size_t()
        _check(lib().lbib_device_bytes(self._h, C.byref(n)))
        return n.value


class Batch:
    """Simulations stepped together: one lattice and one particle kernel per
    step over all members (``lbib_batch_*``)."""

    def __init__(self, sims):
        self.sims = list(sims)
        # keep the members' allocator callbacks alive as long as the batch
        self._allocs = [s._alloc_ref for s in self.sims]
        arr = (C.c_void_p * len(self.sims))(*[s.handle for s in self.sims])
        h = C.c_void_p()
        _check(lib().lbib_batch_create(arr, len(self.sims), C.byref(h)))
        self._h = h

    def step(self, n=1):
        _check(lib().lbib_batch_step(self._h, int(n)))

    def particles(self):
        """Particle states of all members in member order, one readback for
        the batch (``lbib_batch_read_particles``; collects a readback started
        by ``read_particles_async``); a list per member.  The bytes the
        readback copied are left in ``last_d2h_bytes``."""
        total = sum(s.n_particles for s in self.sims)
        arr = (ParticleState * max(total, 1))()
        cnt = C.c_int32()
        nb = C.c_size_t()
        _check(lib().lbib_batch_read_particles(self._h, arr, total, C.byref(cnt), C.byref(nb)))
        self.last_d2h_bytes = nb.value
        out, k = [], 0
        for s in self.sims:
            row = []
            for _ in range(s.n_particles):
                d = {name: getattr(arr[k], name) for name, _ in ParticleState._fields_}
                for key in ("Fh", "Fb", "Fw"):
                    d[key] = tuple(d[key])
                row.append(d)
                k += 1
            out.append(row)
        return out

    def read_particles_async(self):
        """Enqueue the readback of every member's particle states (after the
        work enqueued so far); the next ``particles()`` collects it."""
        _check(lib().lbib_batch_read_particles_async(self._h))

    def step_flushed(self, n, flush_ptr, flush_bytes, clean=True):
        """Step n times with the L2 flushed (device buffer at ``flush_ptr``
        overwritten, and read back when ``clean``) before every step; returns
        the summed device ms of the steps, their bulk lattice passes and the
        flushes, and of the near-box plus particle passes
        (``lbib_batch_step_flushed``)."""
        ms = (C.c_double * 4)()
        _check(lib().lbib_batch_step_flushed(self._h, int(n), C.c_void_p(int(flush_ptr)),
                                             int(flush_bytes), 1 if clean else 0, ms))
        return {"step_ms": ms[0], "bulk_ms": ms[1], "flush_ms": ms[2], "chain_ms": ms[3]}

    def set_timing(self, nsamples):
        _check(lib().lbib_batch_set_timing(self._h, int(nsamples)))

    def synchronize(self):
        """Wait for the batch's work; raises on a member's device error (one
        copy of the members' error words, ``lbib_batch_synchronize``)."""
        _check(lib().lbib_batch_synchronize(self._h))

    def kernel_times(self):
        ms = (C.c_double * 3)(); cnt = (C.c_int64 * 3)()
        _check(lib().lbib_batch_kernel_times(self._h, ms, cnt))
        return {"lattice_ms": ms[0], "lattice_n": cnt[0], "particle_ms": ms[1],
                "particle_n": cnt[1], "near_ms": ms[2], "near_n": cnt[2]}

    def autotune(self, reps=20):
        """Time the lattice-pass kernel variants on this batch (without
        changing its state) and keep the fastest; returns (variant, ms per
        variant)."""
        v = C.c_int32()
        ms = (C.c_double * LATTICE_VARIANTS)()
        _check(lib().lbib_batch_autotune(self._h, int(reps), C.byref(v), ms))
        return v.value, list(ms)

    def set_variant(self, variant):
        _check(lib().lbib_batch_set_variant(self._h, int(variant)))

    def set_particle_threads(self, threads):
        """256 or 512 threads per particle CTA (``lbib_batch_set_particle_threads``)."""
        _check(lib().lbib_batch_set_particle_threads(self._h, int(threads)))

    def pass_nodes(self):
        """Nodes updated per step by the bulk and near-box lattice passes at
        the current particle positions, and all nodes of the members."""
        n = (C.c_int64 * 3)()
        _check(lib().lbib_batch_pass_nodes(self._h, n))
        return {"bulk": n[0], "near": n[1], "total": n[2]}

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            lib().lbib_batch_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ib_force_noalloc(cfg: dict, f_dev_ptr: int, vx, vy, xc, yc, theta=0.0, u=0.0, v=0.0,
                     omega=0.0, fx_dev_ptr: int = 0, fy_dev_ptr: int = 0, stream=None,
                     rho_p=1.0, ligand_density=0.0, sigma=0.0):
    """lbib_ib_force_noalloc: IB force density of one particle written into
    caller-owned device arrays, without any allocation by the library.
    f_dev_ptr points to [9][ny][nx] FP32 deviations f - w on the device;
    fx/fy_dev_ptr to [ny][nx] doubles on the device."""
    c = make_config(storage="f32", stream=stream, **cfg)
    vx = np.ascontiguousarray(vx, dtype=np.float64)
    vy = np.ascontiguousarray(vy, dtype=np.float64)
    p = Particle()
    p.vx, p.vy, p.n_vertices = _dp(vx), _dp(vy), len(vx)
    p.xc, p.yc, p.theta, p.rho_p = xc, yc, theta, rho_p
    p.ligand_density, p.sigma = ligand_density, sigma
    _check(lib().lbib_ib_force_noalloc(C.byref(c), f_dev_ptr, C.byref(p), u, v, omega,
                                       fx_dev_ptr, fy_dev_ptr))


def version() -> str:
    return lib().lbib_version().decode()
