"""ctypes wrapper of the FP64 CPU oracle in hlbm_oracle.c.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it to check and time against; the product
path never imports it.  It imports nothing from the CUDA package.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "hlbm_oracle.c")
HDR = os.path.join(HERE, "hlbm_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")
# the same source built with -fopenmp (loops shared among the host cores;
# identical results), for timing only
LIB_OMP = os.path.join(HERE, "liboracle_omp.so")

SPHERE, ELLIPSOID, CUBOID, CAPSULE, GRID = 0, 1, 2, 3, 4
WALL_X, WALL_Y, WALL_Z = 1, 2, 4

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def _compile(out, extra, force):
    newest = max(os.path.getmtime(SRC), os.path.getmtime(HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=HERE)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", *extra, SRC, "-o", tmp, "-lm"]
    try:
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    finally:
        if os.path.exists(tmp):
            os.remove(tmp)
    return out


def build(force=False, omp=False):
    """Compile the oracle with gcc (C99, -O2, no contraction, no fast-math);
    omp: the -fopenmp build."""
    return _compile(LIB_OMP, ["-fopenmp"], force) if omp else _compile(LIB, [], force)


_libs = {}


def lib(omp=False):
    if omp not in _libs:
        L = ctypes.CDLL(build(omp=omp))
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double, ctypes.c_double,
                                                         ctypes.c_int, _dp, _dp]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_add_particles.argtypes = [ctypes.c_void_p, ctypes.c_int, _ip, _dp, _dp, _dp,
                                           _dp, _dp, _dp]
        L.oracle_set_particle_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.oracle_particle_state.argtypes = [ctypes.c_void_p] + [_dp] * 6
        L.oracle_get_populations.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_set_populations.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.oracle_steps_done.restype = ctypes.c_long
        L.oracle_steps_done.argtypes = [ctypes.c_void_p]
        L.oracle_num_particles.argtypes = [ctypes.c_void_p]
        L.oracle_mea.restype = ctypes.c_long
        L.oracle_mea.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp]
        L.oracle_mea_printed_cell.argtypes = [ctypes.c_void_p, _ip, _dp, _dp]
        L.oracle_indicator_field.argtypes = [ctypes.c_void_p, _dp, _ip]
        L.oracle_collide_only.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_stream_only.argtypes = [ctypes.c_void_p, _dp]
        L.oracle_integrate_only.argtypes = [ctypes.c_void_p, _dp, _dp]
        L.oracle_velocity_set.argtypes = [_ip, _dp, _ip]
        L.oracle_equilibrium.argtypes = [ctypes.c_double, _dp, _dp]
        L.oracle_indicator.restype = ctypes.c_double
        L.oracle_indicator.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_sdf_body.restype = ctypes.c_double
        L.oracle_sdf_body.argtypes = [ctypes.c_int, _dp, _dp]
        L.oracle_rotation.argtypes = [_dp, _dp]
        L.oracle_inside_fp32.argtypes = [ctypes.c_int, _dp, _dp, _dp, _ip, _ip, ctypes.c_int]
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_set_contact.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double]
        L.oracle_add_grid.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_float)]
        L.oracle_grid_sdf.restype = ctypes.c_double
        L.oracle_grid_sdf.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        L.oracle_grid_properties.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp]
        L.oracle_inside_grid_fp32.argtypes = [ctypes.c_void_p, ctypes.c_int, _dp, _dp, _ip]
        L.oracle_contact_forces.argtypes = [ctypes.c_void_p, _dp, _dp]
        _libs[omp] = L
    return _libs[omp]


def threads(omp=False):
    """Threads the oracle's loops use (1 for the plain build)."""
    return lib(omp).oracle_threads()


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


def velocity_set():
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    opp = np.zeros(19, np.int32)
    lib().oracle_velocity_set(c.ctypes.data_as(_ip), w.ctypes.data_as(_dp), opp.ctypes.data_as(_ip))
    return c, w, opp


def equilibrium(rho, u):
    u, up = _d(u)
    out = np.zeros(19)
    lib().oracle_equilibrium(float(rho), up, out.ctypes.data_as(_dp))
    return out


def indicator(d, eps):
    return lib().oracle_indicator(float(d), float(eps))


def sdf_body(shape, a, r_body):
    a, ap = _d(np.broadcast_to(np.asarray(a, float), (3,)) if np.ndim(a) == 0 else a)
    r, rp = _d(r_body)
    return lib().oracle_sdf_body(int(shape), ap, rp)


def rotation(q):
    q, qp = _d(q)
    R = np.zeros(9)
    lib().oracle_rotation(qp, R.ctypes.data_as(_dp))
    return R.reshape(3, 3)


def inside_fp32(shape, a, q, X, cell, n, bc):
    a, ap = _d(np.broadcast_to(np.asarray(a, float), (3,)) if np.ndim(a) == 0 else a)
    q, qp = _d(q)
    X, Xp = _d(X)
    cell, cp = _i(cell)
    n, npp = _i(n)
    return bool(lib().oracle_inside_fp32(int(shape), ap, qp, Xp, cp, npp, int(bc)))


class Oracle:
    """One FP64 HLBM lattice with its particles (two-lattice push streaming)."""

    def __init__(self, n, tau, eps=0.5, bc=0, gravity=(0, 0, 0), fluid_force=(0, 0, 0), omp=False):
        self._L = lib(omp)
        self.n = tuple(int(v) for v in n)
        g, gp = _d(gravity)
        ff, ffp = _d(fluid_force)
        self._keep = (g, ff)
        self.h = self._L.oracle_create(self.n[0], self.n[1], self.n[2], float(tau), float(eps),
                                     int(bc), gp, ffp)
        if not self.h:
            raise ValueError("oracle_create rejected the lattice arguments")
        self.ncell = self.n[0] * self.n[1] * self.n[2]

    def close(self):
        if self.h:
            self._L.oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_particles(self):
        return self._L.oracle_num_particles(self.h)

    def add_particles(self, shape, a, X, U=None, omega=None, quat=None, rho_p=None):
        shape, sp = _i(shape)
        n = shape.shape[0]
        a, ap = _d(np.asarray(a, float).reshape(n, -1) if n else np.zeros((0, 3)))
        if a.shape[1] == 1:
            a, ap = _d(np.repeat(a, 3, axis=1))
        X, Xp = _d(np.asarray(X, float).reshape(n, 3))
        U, Up = _d(np.zeros((n, 3)) if U is None else np.asarray(U, float).reshape(n, 3))
        W, Wp = _d(np.zeros((n, 3)) if omega is None else np.asarray(omega, float).reshape(n, 3))
        if quat is None:
            quat = np.tile([1.0, 0, 0, 0], (n, 1))
        qv, qp = _d(np.asarray(quat, float).reshape(n, 4))
        rho, rp = _d(np.asarray(rho_p, float).reshape(n))
        rc = self._L.oracle_add_particles(self.h, n, sp, ap, Xp, Up, Wp, qp, rp)
        if rc != 0:
            raise ValueError(f"oracle_add_particles failed ({rc})")

    def set_particle_state(self, X=None, U=None, omega=None, quat=None):
        n = self.num_particles
        args = []
        keep = []
        for v, k in ((X, 3), (U, 3), (omega, 3), (quat, 4)):
            if v is None:
                args.append(None)
            else:
                arr, p = _d(np.asarray(v, float).reshape(n, k))
                keep.append(arr)
                args.append(p)
        if self._L.oracle_set_particle_state(self.h, *args) != 0:
            raise ValueError("oracle_set_particle_state failed")

    def particle_state(self):
        n = self.num_particles
        out = {k: np.zeros((n, 4 if k == "quat" else 3)) for k in ("X", "U", "omega", "quat", "F", "T")}
        self._L.oracle_particle_state(self.h, *[out[k].ctypes.data_as(_dp) for k in
                                              ("X", "U", "omega", "quat", "F", "T")])
        return out

    def populations(self):
        f = np.zeros((19, self.n[2], self.n[1], self.n[0]))
        self._L.oracle_get_populations(self.h, f.ctypes.data_as(_dp))
        return f

    def set_populations(self, f):
        f, fp = _d(np.asarray(f, float).reshape(19, self.n[2], self.n[1], self.n[0]))
        self._L.oracle_set_populations(self.h, fp)

    def step(self, nsteps=1):
        self._L.oracle_step(self.h, int(nsteps))

    @property
    def steps_done(self):
        return self._L.oracle_steps_done(self.h)

    def mea(self, p):
        F = np.zeros(3)
        T = np.zeros(3)
        cnt = self._L.oracle_mea(self.h, int(p), F.ctypes.data_as(_dp), T.ctypes.data_as(_dp))
        return F, T, cnt

    def mea_printed_cell(self, x, up):
        x, xp = _i(x)
        up, upp = _d(up)
        Fh = np.zeros(3)
        self._L.oracle_mea_printed_cell(self.h, xp, upp, Fh.ctypes.data_as(_dp))
        return Fh

    def indicator_field(self):
        B = np.zeros((self.n[2], self.n[1], self.n[0]))
        pid = np.zeros((self.n[2], self.n[1], self.n[0]), np.int32)
        self._L.oracle_indicator_field(self.h, B.ctypes.data_as(_dp), pid.ctypes.data_as(_ip))
        return B, pid

    def collide_only(self):
        post = np.zeros((19, self.n[2], self.n[1], self.n[0]))
        self._L.oracle_collide_only(self.h, post.ctypes.data_as(_dp))
        return post

    def stream_only(self, post):
        post, pp = _d(post)
        self._L.oracle_stream_only(self.h, pp)

    def add_grid(self, values, h):
        """Register a signed-distance grid (values[z, y, x], spacing h, body
        frame centred at the origin); returns its id."""
        v = np.ascontiguousarray(values, dtype=np.float32)
        nz, ny, nx = v.shape
        gid = self._L.oracle_add_grid(self.h, nx, ny, nz, float(h),
                                      v.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if gid < 0:
            raise ValueError(f"oracle_add_grid refused the grid ({gid})")
        return gid

    def grid_sdf(self, grid, r_body):
        r, rp = _d(r_body)
        return self._L.oracle_grid_sdf(self.h, int(grid), rp)

    def grid_properties(self, grid):
        out = np.zeros(6)
        self._L.oracle_grid_properties(self.h, int(grid), out.ctypes.data_as(_dp))
        return {"V": out[0], "I1": out[1:4].copy(), "rc": out[4], "rinf": out[5]}

    def inside_grid_fp32(self, grid, q, X, cell):
        q, qp = _d(q)
        X, Xp = _d(X)
        cell, cp = _i(cell)
        return bool(self._L.oracle_inside_grid_fp32(self.h, int(grid), qp, Xp, cp))

    def set_contact(self, k, zeta=1.0):
        """Contact stiffness k (0: off) and range zeta of the repulsion
        between the particles' enclosing capsules and with the walls."""
        if self._L.oracle_set_contact(self.h, float(k), float(zeta)) != 0:
            raise ValueError("oracle_set_contact: k must be >= 0 and zeta > 0")

    def contact_forces(self):
        n = self.num_particles
        F, T = np.zeros((n, 3)), np.zeros((n, 3))
        self._L.oracle_contact_forces(self.h, F.ctypes.data_as(_dp), T.ctypes.data_as(_dp))
        return F, T

    def integrate_only(self, F, T):
        n = self.num_particles
        F, Fp = _d(np.asarray(F, float).reshape(n, 3))
        T, Tp = _d(np.asarray(T, float).reshape(n, 3))
        self._L.oracle_integrate_only(self.h, Fp, Tp)


def from_workload(w, omp=False):
    """Build an oracle lattice from a workload description (see the workloads
    module); omp: on the -fopenmp build."""
    o = Oracle(w["n"], w["tau"], w["eps"], w["bc"], w["gravity"], w.get("fluid_force", (0, 0, 0)), omp=omp)
    for values, h in w.get("grids", ()):
        o.add_grid(values, h)
    P = w["particles"]
    if len(P["shape"]):
        o.add_particles(P["shape"], P["a"], P["X"], P["U"], P["omega"], P["quat"], P["rho_p"])
    return o
