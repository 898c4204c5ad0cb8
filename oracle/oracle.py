"""ctypes front end of the FP64 CPU oracle (``lbib_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path never loads it.

``build()`` compiles the C oracle with gcc (``-ffp-contract=off`` so that the
same IEEE double operations run on x86-64 and aarch64 hosts), with OpenMP for
its per-node loops where the compiler supports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "liblbib_oracle.so")
SRC = os.path.join(HERE, "lbib_oracle.c")
HDR = os.path.join(HERE, "lbib_oracle.h")

WALL = {"zou_he": 0, "bounce_back": 1, "periodic": 2}

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library in-tree; returns its path."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    stale = not os.path.exists(LIB_PATH) or max(
        os.path.getmtime(SRC), os.path.getmtime(HDR)) > os.path.getmtime(LIB_PATH)
    if force or stale:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-fast-math",
                "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        # the node loops in parallel where OpenMP is available (same results
        # for any thread count; OMP_NUM_THREADS=1 runs them on one thread)
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.check_call(base)
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class OrConfig(C.Structure):
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
        ("ib_iterations", C.c_int32), ("ib_spread", C.c_int32),
    ]


class OrParticleIn(C.Structure):
    _fields_ = [
        ("n_vertices", C.c_int32), ("fixed", C.c_int32),
        ("vx", C.POINTER(C.c_double)), ("vy", C.POINTER(C.c_double)),
        ("xc", C.c_double), ("yc", C.c_double), ("theta", C.c_double),
        ("rho_p", C.c_double), ("ligand_density", C.c_double), ("sigma", C.c_double),
    ]


class OrParticleState(C.Structure):
    _fields_ = [
        ("xc", C.c_double), ("yc", C.c_double), ("theta", C.c_double),
        ("u", C.c_double), ("v", C.c_double), ("omega", C.c_double),
        ("Fh", C.c_double * 2), ("Mh", C.c_double),
        ("Fb", C.c_double * 2), ("Mb", C.c_double),
        ("Fw", C.c_double * 2),
        ("area", C.c_double), ("mass", C.c_double), ("inertia", C.c_double),
        ("r_eq", C.c_double),
        ("nl", C.c_int32), ("n_ligands", C.c_int32), ("n_probing", C.c_int32),
        ("n_bonded", C.c_int32),
        ("margin_p", C.c_double), ("margin_gap", C.c_double),
        ("gap_bottom", C.c_double), ("gap_top", C.c_double),
    ]


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
            pd, pi32, pu64 = C.POINTER(d), C.POINTER(i32), C.POINTER(u64)
            sig = {
                "or_create": (C.c_void_p, [C.POINTER(OrConfig)]),
                "or_destroy": (None, [C.c_void_p]),
                "or_add_particle": (C.c_int, [C.c_void_p, C.POINTER(OrParticleIn)]),
                "or_set_populations": (C.c_int, [C.c_void_p, pd]),
                "or_get_populations": (C.c_int, [C.c_void_p, pd]),
                "or_step": (C.c_int, [C.c_void_p, i64]),
                "or_step_count": (i64, [C.c_void_p]),
                "or_fields": (C.c_int, [C.c_void_p, pd, pd, pd]),
                "or_ib_force": (C.c_int, [C.c_void_p, pd, pd]),
                "or_particle_get": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(OrParticleState)]),
                "or_bonds_get": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint8), pd,
                                           C.POINTER(C.c_int8)]),
                "or_bonds_set": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_uint8), pd,
                                           C.POINTER(C.c_int8)]),
                "or_lattice": (None, [pi32, pi32, pd, pi32]),
                "or_equilibrium": (None, [d, d, d, pd]),
                "or_guo_source": (None, [d, d, d, d, d, pd]),
                "or_collide_node": (None, [pd, d, d, d, pd]),
                "or_weight": (d, [d]),
                "or_mls_shape": (C.c_int, [C.POINTER(OrConfig), d, d, pi32, pi32, pd]),
                "or_mls_fit": (C.c_int, [C.POINTER(OrConfig), pd, d, d, pd, pd, pd]),
                "or_spread": (None, [C.POINTER(OrConfig), C.c_int, pd, pd, pd, pd, pd, pd, pd]),
                "or_interp": (None, [C.POINTER(OrConfig), pd, C.c_int, pd, pd, pd]),
                "or_vb_eps": (C.c_int, [C.POINTER(OrConfig), C.c_int, pd, pd, pd]),
                "or_loads": (None, [C.POINTER(OrConfig), pd, pd, pd, C.c_int, pd, pd,
                                    d, d, d, pd]),
                "or_elements": (None, [C.c_int, pd, pd, d, d, d, pd, pd, pd, pd, pd]),
                "or_philox4x64": (None, [pu64, pu64, pu64]),
                "or_uniform": (d, [u64, u64, i64, i32, i32]),
                "or_prob_forward": (d, [d, d]),
                "or_prob_reverse": (d, [d, d, d, d, d, d]),
                "or_bdf2_velocity": (d, [d, d, d]),
                "or_bdf2_position": (d, [d, d, d]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def make_config(**kw) -> OrConfig:
    """Config struct from keyword arguments (the same keys the GPU binding
    takes); wall kinds are given by name."""
    c = OrConfig()
    defaults = dict(nx=32, ny=16, wall_bottom="bounce_back", wall_top="bounce_back",
                    tau=0.8, u_bottom=0.0, u_top=0.0, gx=0.0, gy=0.0, k_f=0.85,
                    k_r0=1e-4, kBT=0.1, sigma_star_ratio=0.5, y_cr=1.36,
                    y_eq_ratio=0.5, hamaker=0.0, eps_min=1e-3, receptor_bottom=1.0,
                    receptor_top=0.0, seed=1, sim_id=0, ib_iterations=1, ib_spread=0)
    defaults.update(kw)
    for k, v in defaults.items():
        if k in ("wall_bottom", "wall_top") and isinstance(v, str):
            v = WALL[v]
        setattr(c, k, v)
    return c


class OracleSim:
    """One oracle simulation (host memory, single thread)."""

    def __init__(self, **cfg):
        self.cfg = make_config(**cfg)
        self.nx, self.ny = self.cfg.nx, self.cfg.ny
        self._h = lib().or_create(C.byref(self.cfg))
        if not self._h:
            raise ValueError("oracle rejected the configuration")
        self.n_particles = 0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_destroy(h)
            self._h = None

    def add_particle(self, vx, vy, xc, yc, theta=0.0, rho_p=1.0, ligand_density=0.5,
                     sigma=1.0, fixed=False) -> int:
        vx = np.ascontiguousarray(vx, dtype=np.float64)
        vy = np.ascontiguousarray(vy, dtype=np.float64)
        p = OrParticleIn(len(vx), int(fixed), _dp(vx), _dp(vy), xc, yc, theta, rho_p,
                         ligand_density, sigma)
        pid = lib().or_add_particle(self._h, C.byref(p))
        if pid < 0:
            raise ValueError("oracle rejected the particle")
        self.n_particles += 1
        return pid

    def set_populations(self, f_post):
        f = np.ascontiguousarray(f_post, dtype=np.float64).reshape(9, self.ny, self.nx)
        if lib().or_set_populations(self._h, _dp(f)) != 0:
            raise RuntimeError("populations can only be set before the first step")

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        lib().or_get_populations(self._h, _dp(f))
        return f

    def step(self, n=1):
        if lib().or_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle step failed")

    @property
    def step_count(self):
        return lib().or_step_count(self._h)

    def fields(self):
        r = np.empty((self.ny, self.nx)); u = np.empty_like(r); v = np.empty_like(r)
        lib().or_fields(self._h, _dp(r), _dp(u), _dp(v))
        return r, u, v

    def ib_force(self):
        fx = np.empty((self.ny, self.nx)); fy = np.empty_like(fx)
        lib().or_ib_force(self._h, _dp(fx), _dp(fy))
        return fx, fy

    def particle(self, pid=0) -> dict:
        st = OrParticleState()
        if lib().or_particle_get(self._h, pid, C.byref(st)) != 0:
            raise IndexError(pid)
        out = {k: getattr(st, k) for k, _ in OrParticleState._fields_}
        for k in ("Fh", "Fb", "Fw"):
            out[k] = tuple(out[k])
        return out

    def bonds(self, pid=0, walls=False):
        """Bond flags and anchor x of every element (and, with walls=True,
        the anchor wall: 0 bottom, 1 top)."""
        n = self.particle(pid)["nl"]
        b = np.zeros(n, dtype=np.uint8); ax = np.zeros(n); aw = np.zeros(n, dtype=np.int8)
        lib().or_bonds_get(self._h, pid, b.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(ax),
                           aw.ctypes.data_as(C.POINTER(C.c_int8)))
        return (b, ax, aw) if walls else (b, ax)

    def set_bonds(self, pid, bond, anchor_x, anchor_wall):
        n = self.particle(pid)["nl"]
        b = np.ascontiguousarray(bond, dtype=np.uint8)
        ax = np.ascontiguousarray(anchor_x, dtype=np.float64)
        aw = np.ascontiguousarray(anchor_wall, dtype=np.int8)
        if not (len(b) == len(ax) == len(aw) == n):
            raise ValueError(f"particle {pid} has {n} elements")
        if lib().or_bonds_set(self._h, pid, b.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(ax),
                              aw.ctypes.data_as(C.POINTER(C.c_int8))) != 0:
            raise RuntimeError("or_bonds_set failed")


# ---- building blocks -------------------------------------------------------

def lattice():
    ex = (C.c_int32 * 9)(); ey = (C.c_int32 * 9)(); w = (C.c_double * 9)(); op = (C.c_int32 * 9)()
    lib().or_lattice(ex, ey, w, op)
    return np.array(ex), np.array(ey), np.array(w), np.array(op)


def equilibrium(rho, ux, uy):
    out = np.empty(9)
    lib().or_equilibrium(rho, ux, uy, _dp(out))
    return out


def guo_source(tau, ux, uy, Fx, Fy):
    out = np.empty(9)
    lib().or_guo_source(tau, ux, uy, Fx, Fy, _dp(out))
    return out


def collide_node(f, tau, Fx, Fy):
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.empty(9)
    lib().or_collide_node(_dp(f), tau, Fx, Fy, _dp(out))
    return out


def weight(r):
    return lib().or_weight(float(r))


def mls_shape(cfg: OrConfig, X, Y):
    ix = np.zeros(16, dtype=np.int32); iy = np.zeros(16, dtype=np.int32); phi = np.zeros(16)
    n = lib().or_mls_shape(C.byref(cfg), X, Y, ix.ctypes.data_as(C.POINTER(C.c_int32)),
                           iy.ctypes.data_as(C.POINTER(C.c_int32)), _dp(phi))
    return ix[:n], iy[:n], phi[:n]


def mls_fit(cfg: OrConfig, field, X, Y):
    field = np.ascontiguousarray(field, dtype=np.float64)
    v = C.c_double(); a = C.c_double(); b = C.c_double()
    n = lib().or_mls_fit(C.byref(cfg), _dp(field), X, Y, C.byref(v), C.byref(a), C.byref(b))
    return n, v.value, a.value, b.value


def spread(cfg: OrConfig, X, Y, Fx, Fy, eps):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (X, Y, Fx, Fy, eps)]
    fx = np.zeros((cfg.ny, cfg.nx)); fy = np.zeros_like(fx)
    lib().or_spread(C.byref(cfg), len(arrs[0]), *[_dp(a) for a in arrs], _dp(fx), _dp(fy))
    return fx, fy


def interp(cfg: OrConfig, field, X, Y):
    field = np.ascontiguousarray(field, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64); Y = np.ascontiguousarray(Y, dtype=np.float64)
    out = np.zeros(len(X))
    lib().or_interp(C.byref(cfg), _dp(field), len(X), _dp(X), _dp(Y), _dp(out))
    return out


def vb_eps(cfg: OrConfig, X, Y):
    """Solved spreading scales of markers at (X, Y) (or_vb_eps)."""
    X = np.ascontiguousarray(X, dtype=np.float64); Y = np.ascontiguousarray(Y, dtype=np.float64)
    out = np.zeros(len(X))
    if lib().or_vb_eps(C.byref(cfg), len(X), _dp(X), _dp(Y), _dp(out)) != 0:
        raise RuntimeError("singular spreading-scale system")
    return out


def loads(cfg: OrConfig, rho, ux, uy, vx, vy, xc, yc, theta):
    a = [np.ascontiguousarray(v, dtype=np.float64) for v in (rho, ux, uy, vx, vy)]
    out = np.zeros(3)
    lib().or_loads(C.byref(cfg), _dp(a[0]), _dp(a[1]), _dp(a[2]), len(a[3]), _dp(a[3]),
                   _dp(a[4]), xc, yc, theta, _dp(out))
    return out


def elements(vx, vy, xc, yc, theta):
    vx = np.ascontiguousarray(vx, dtype=np.float64); vy = np.ascontiguousarray(vy, dtype=np.float64)
    n = len(vx)
    out = [np.zeros(n) for _ in range(5)]
    lib().or_elements(n, _dp(vx), _dp(vy), xc, yc, theta, *[_dp(o) for o in out])
    return out


def philox4x64(ctr, key):
    c = (C.c_uint64 * 4)(*[int(x) for x in ctr]); k = (C.c_uint64 * 2)(*[int(x) for x in key])
    o = (C.c_uint64 * 4)()
    lib().or_philox4x64(c, k, o)
    return [int(x) for x in o]


def uniform(seed, sim_id, step, pid, l):
    return lib().or_uniform(seed, sim_id, step, pid, l)


def prob_forward(k_f, Nl):
    return lib().or_prob_forward(k_f, Nl)


def prob_reverse(k_r0, sigma, sigma_star, y, y_eq, kBT):
    return lib().or_prob_reverse(k_r0, sigma, sigma_star, y, y_eq, kBT)


def bdf2_velocity(u1, u2, acc):
    return lib().or_bdf2_velocity(u1, u2, acc)


def bdf2_position(x1, x2, u_new):
    return lib().or_bdf2_position(x1, x2, u_new)
