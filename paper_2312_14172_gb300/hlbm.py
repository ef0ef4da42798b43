"""Python binding of libhlbm.so (the C-ABI in include/hlbm.h).

Argument marshalling only: every step of the HLBM time step runs in the CUDA
kernels behind the C-ABI.  PyTorch supplies device memory (one uint8 buffer
per handle) and the CUDA stream.  There is no CPU fallback: loading fails
loudly when the library is missing or no GPU is present.

The functions carry the C names; ``Lattice`` wraps a handle for convenience.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhlbm.so")

HLBM_OK, HLBM_ERR_ARG, HLBM_ERR_CUDA, HLBM_ERR_UNSTABLE, HLBM_ERR_CAPACITY, HLBM_ERR_STATE = 0, -1, -2, -3, -4, -5
HLBM_FP32, HLBM_FP16 = 0, 1
HLBM_SPHERE, HLBM_ELLIPSOID, HLBM_CUBOID, HLBM_CAPSULE, HLBM_GRID = 0, 1, 2, 3, 4
HLBM_WALL_X, HLBM_WALL_Y, HLBM_WALL_Z, HLBM_CUT_Z = 1, 2, 4, 8
HLBM_MEA_KERNEL, HLBM_MEA_MOMENTS = 0, 1

ERRORS = {HLBM_ERR_ARG: "HLBM_ERR_ARG", HLBM_ERR_CUDA: "HLBM_ERR_CUDA",
          HLBM_ERR_UNSTABLE: "HLBM_ERR_UNSTABLE", HLBM_ERR_CAPACITY: "HLBM_ERR_CAPACITY",
          HLBM_ERR_STATE: "HLBM_ERR_STATE"}

# every symbol include/hlbm.h declares
EXPORTS = ["hlbm_default_params", "hlbm_required_bytes", "hlbm_init_lattice", "hlbm_init_batch",
           "hlbm_add_particles", "hlbm_set_particle_state", "hlbm_step", "hlbm_sync",
           "hlbm_particle_state", "hlbm_get_populations", "hlbm_set_populations",
           "hlbm_num_particles", "hlbm_steps_done", "hlbm_set_launch", "hlbm_get_launch",
           "hlbm_set_fluid_force", "hlbm_set_contact", "hlbm_fluid_momentum", "hlbm_add_grid",
           "hlbm_set_owned_planes", "hlbm_plane_slots", "hlbm_step_forces", "hlbm_step_with_forces",
           "hlbm_set_mea_mode", "hlbm_get_mea_mode",
           "hlbm_autotune", "hlbm_kernel_times", "hlbm_interior_cells",
           "hlbm_checkpoint_bytes", "hlbm_save", "hlbm_load", "hlbm_last_error", "hlbm_destroy",
           "hlbm_mea_noalloc"]
HLBM_NOALLOC_MAX_PARTICLES = 1024


class hlbm_box(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("bc_flags", ctypes.c_int)]


class hlbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("eps", ctypes.c_double),
                ("gravity", ctypes.c_double * 3), ("fluid_force", ctypes.c_double * 3),
                ("precision", ctypes.c_int), ("fp16_scale_log2", ctypes.c_int),
                ("max_particles", ctypes.c_int), ("bin_capacity", ctypes.c_int),
                ("grid_floats", ctypes.c_longlong)]


class HLBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_fp = ctypes.POINTER(ctypes.c_float)
_vp = ctypes.c_void_p
_h = ctypes.c_void_p
_lib = None


def load(path=LIB_PATH):
    """Load libhlbm.so and declare its signatures (no CUDA call is made)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it first (paper_2312_14172_gb300.build)")
    L = ctypes.CDLL(path)
    L.hlbm_default_params.argtypes = [ctypes.POINTER(hlbm_params)]
    L.hlbm_default_params.restype = None
    L.hlbm_required_bytes.argtypes = [ctypes.c_int, ctypes.POINTER(hlbm_box), ctypes.POINTER(hlbm_params)]
    L.hlbm_required_bytes.restype = ctypes.c_size_t
    L.hlbm_init_lattice.argtypes = [ctypes.POINTER(_h), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.POINTER(hlbm_params), _vp, _vp, ctypes.c_size_t]
    L.hlbm_init_batch.argtypes = [ctypes.POINTER(_h), ctypes.c_int, ctypes.POINTER(hlbm_box),
                                  ctypes.POINTER(hlbm_params), _vp, _vp, ctypes.c_size_t]
    L.hlbm_add_particles.argtypes = [_h, ctypes.c_int, _ip, _ip, _dp, _dp, _dp, _dp, _dp, _dp]
    L.hlbm_set_particle_state.argtypes = [_h, _dp, _dp, _dp, _dp]
    L.hlbm_step.argtypes = [_h, ctypes.c_int]
    L.hlbm_sync.argtypes = [_h]
    L.hlbm_particle_state.argtypes = [_h, _dp, _dp, _dp, _dp, _dp, _dp]
    L.hlbm_get_populations.argtypes = [_h, ctypes.c_int, _dp]
    L.hlbm_set_populations.argtypes = [_h, ctypes.c_int, _dp]
    L.hlbm_num_particles.argtypes = [_h]
    L.hlbm_steps_done.argtypes = [_h]
    L.hlbm_steps_done.restype = ctypes.c_longlong
    L.hlbm_set_launch.argtypes = [_h, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hlbm_get_launch.argtypes = [_h, _ip, _ip, _ip]
    L.hlbm_set_mea_mode.argtypes = [_h, ctypes.c_int]
    L.hlbm_set_fluid_force.argtypes = [_h, _dp]
    L.hlbm_set_contact.argtypes = [_h, ctypes.c_double, ctypes.c_double]
    L.hlbm_fluid_momentum.argtypes = [_h, ctypes.c_int, _dp]
    L.hlbm_add_grid.argtypes = [_h, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _fp, _ip]
    L.hlbm_set_owned_planes.argtypes = [_h, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.hlbm_plane_slots.argtypes = [_h, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_int]
    L.hlbm_step_forces.argtypes = [_h, _dp, _dp]
    L.hlbm_step_with_forces.argtypes = [_h, _dp, _dp]
    L.hlbm_get_mea_mode.argtypes = [_h]
    L.hlbm_autotune.argtypes = [_h, ctypes.c_int, _ip, _ip, _ip, _fp]
    L.hlbm_kernel_times.argtypes = [_h, ctypes.c_int, _fp]
    L.hlbm_interior_cells.argtypes = [_h, ctypes.POINTER(ctypes.c_longlong)]
    L.hlbm_checkpoint_bytes.argtypes = [_h, ctypes.POINTER(ctypes.c_size_t)]
    L.hlbm_save.argtypes = [_h, _vp, ctypes.c_size_t]
    L.hlbm_load.argtypes = [_h, _vp, ctypes.c_size_t]
    L.hlbm_last_error.argtypes = [_h]
    L.hlbm_last_error.restype = ctypes.c_char_p
    L.hlbm_destroy.argtypes = [_h]
    L.hlbm_destroy.restype = None
    L.hlbm_mea_noalloc.argtypes = [_vp, ctypes.c_longlong] + [ctypes.c_int] * 8 + [_vp] * 9
    L.hlbm_mea_noalloc.restype = ctypes.c_int
    _lib = L
    return L


def _arr(a, dtype, shape):
    if a is None:
        return None, None
    a = np.ascontiguousarray(np.asarray(a, dtype=dtype).reshape(shape))
    ptr = a.ctypes.data_as(_dp if dtype == np.float64 else _ip)
    return a, ptr


def hlbm_default_params():
    p = hlbm_params()
    load().hlbm_default_params(ctypes.byref(p))
    return p


def make_params(tau=0.6, eps=0.5, gravity=(0, 0, 0), fluid_force=(0, 0, 0), precision="fp32",
                fp16_scale_log2=14, max_particles=0, bin_capacity=0, grid_floats=0):
    p = hlbm_default_params()
    p.tau, p.eps = float(tau), float(eps)
    for j in range(3):
        p.gravity[j] = float(gravity[j])
        p.fluid_force[j] = float(fluid_force[j])
    p.precision = {"fp32": HLBM_FP32, "fp16": HLBM_FP16}[precision] if isinstance(precision, str) else int(precision)
    p.fp16_scale_log2 = int(fp16_scale_log2)
    p.max_particles = int(max_particles)
    p.bin_capacity = int(bin_capacity)
    p.grid_floats = int(grid_floats)
    return p


def hlbm_required_bytes(boxes, params):
    arr = (hlbm_box * len(boxes))(*[hlbm_box(*[int(v) for v in b]) for b in boxes])
    return int(load().hlbm_required_bytes(len(boxes), arr, ctypes.byref(params)))


def _check(h, rc):
    if rc != HLBM_OK:
        msg = load().hlbm_last_error(h)
        raise HLBMError(rc, msg.decode() if msg else "")
    return rc


class Lattice:
    """One handle: a single box or a batch of boxes, with torch-owned device memory.

    boxes: list of (nx, ny, nz, bc_flags).  The buffer is a torch uint8 tensor
    on the current CUDA device; the stream is torch's current stream unless one
    is given.
    """

    def __init__(self, boxes, params, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libhlbm needs a CUDA GPU; there is no CPU fallback")
        L = load()
        self.boxes = [tuple(int(v) for v in b) for b in boxes]
        self.params = params
        self.nbytes = hlbm_required_bytes(self.boxes, params)
        if self.nbytes == 0:
            raise HLBMError(HLBM_ERR_ARG, "invalid lattice arguments")
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.buffer = torch.empty(self.nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        h = _h()
        arr = (hlbm_box * len(self.boxes))(*[hlbm_box(*b) for b in self.boxes])
        rc = L.hlbm_init_batch(ctypes.byref(h), len(self.boxes), arr, ctypes.byref(params),
                               _vp(self.stream.cuda_stream), _vp(self.buffer.data_ptr()),
                               ctypes.c_size_t(self.nbytes))
        _check(None, rc)
        self.h = h

    # --- lifetime
    def close(self):
        if getattr(self, "h", None):
            load().hlbm_destroy(self.h)
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

    # --- calls
    def add_particles(self, shape, shape_params, X, U=None, omega=None, quat=None, rho_p=None,
                      box_id=None):
        shape, sp = _arr(shape, np.int32, (-1,))
        n = shape.shape[0]
        a = np.asarray(shape_params, float).reshape(n, -1)
        if a.shape[1] == 1:
            a = np.repeat(a, 3, axis=1)
        a, ap = _arr(a, np.float64, (n, 3))
        X, Xp = _arr(X, np.float64, (n, 3))
        U, Up = _arr(U, np.float64, (n, 3))
        W, Wp = _arr(omega, np.float64, (n, 3))
        q, qp = _arr(quat, np.float64, (n, 4))
        r, rp = _arr(rho_p, np.float64, (n,))
        b, bp = _arr(box_id, np.int32, (n,))
        _check(self.h, load().hlbm_add_particles(self.h, n, bp, sp, ap, Xp, Up, Wp, qp, rp))

    def add_workload_particles(self, P, box_id=None):
        if len(P["shape"]):
            self.add_particles(P["shape"], P["a"], P["X"], P["U"], P["omega"], P["quat"], P["rho_p"],
                               box_id)

    def set_particle_state(self, X=None, U=None, omega=None, quat=None):
        n = self.num_particles
        X, Xp = _arr(X, np.float64, (n, 3))
        U, Up = _arr(U, np.float64, (n, 3))
        W, Wp = _arr(omega, np.float64, (n, 3))
        q, qp = _arr(quat, np.float64, (n, 4))
        _check(self.h, load().hlbm_set_particle_state(self.h, Xp, Up, Wp, qp))

    def step(self, nsteps=1):
        _check(self.h, load().hlbm_step(self.h, int(nsteps)))

    def sync(self):
        _check(self.h, load().hlbm_sync(self.h))

    def particle_state(self, out=None, check=True):
        n = self.num_particles
        if out is None:
            out = {k: np.zeros((n, 4 if k == "quat" else 3)) for k in ("X", "U", "omega", "quat", "F", "T")}
        ptrs = [out[k].ctypes.data_as(_dp) for k in ("X", "U", "omega", "quat", "F", "T")]
        rc = load().hlbm_particle_state(self.h, *ptrs)
        if check:
            _check(self.h, rc)
        return out

    def populations(self, box=0):
        nx, ny, nz = self.boxes[box][:3]
        f = np.zeros((19, nz, ny, nx))
        _check(self.h, load().hlbm_get_populations(self.h, int(box), f.ctypes.data_as(_dp)))
        return f

    def set_populations(self, f, box=0):
        nx, ny, nz = self.boxes[box][:3]
        f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(19, nz, ny, nx))
        _check(self.h, load().hlbm_set_populations(self.h, int(box), f.ctypes.data_as(_dp)))

    @property
    def num_particles(self):
        return load().hlbm_num_particles(self.h)

    @property
    def steps_done(self):
        return load().hlbm_steps_done(self.h)

    def set_launch(self, tile_y, tile_z, cells_x=None):
        """Collision launch shape: bricks of 32 x tile_y x tile_z cells and
        cells_x (1 or 2) x-adjacent cells per thread (None keeps the current)."""
        if cells_x is None:
            cells_x = self.get_launch()[2]
        _check(self.h, load().hlbm_set_launch(self.h, int(tile_y), int(tile_z), int(cells_x)))

    def get_launch(self):
        ty, tz, cx = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(self.h, load().hlbm_get_launch(self.h, ctypes.byref(ty), ctypes.byref(tz), ctypes.byref(cx)))
        return ty.value, tz.value, cx.value

    def set_fluid_force(self, f):
        """Uniform body-force density on the fluid from the next step on."""
        f = np.ascontiguousarray(np.asarray(f, np.float64).reshape(3))
        _check(self.h, load().hlbm_set_fluid_force(self.h, f.ctypes.data_as(_dp)))

    def set_contact(self, k, zeta=1.0):
        """Contact stiffness k (0: off) and range zeta (cells) between the
        particles' enclosing capsules and with the walls."""
        _check(self.h, load().hlbm_set_contact(self.h, float(k), float(zeta)))

    def add_grid(self, values, h):
        """Register a signed-distance grid (FP32 samples values[z, y, x],
        spacing h, body frame centred at the origin); returns its id."""
        v = np.ascontiguousarray(values, dtype=np.float32)
        nz, ny, nx = v.shape
        gid = ctypes.c_int(-1)
        _check(self.h, load().hlbm_add_grid(self.h, nx, ny, nz, float(h), v.ctypes.data_as(_fp),
                                            ctypes.byref(gid)))
        return gid.value

    def set_owned_planes(self, z_lo, z_hi, box=0):
        _check(self.h, load().hlbm_set_owned_planes(self.h, int(box), int(z_lo), int(z_hi)))

    def plane_slots(self, z, direction, box=0):
        """The five stored slots with c_z = direction of plane z, raw
        storage values [5, ny, nx] (float32 or float16)."""
        nx, ny, _ = self.boxes[box][:3]
        out = np.empty((5, ny, nx), np.float32 if self.params.precision == HLBM_FP32 else np.float16)
        _check(self.h, load().hlbm_plane_slots(self.h, int(box), int(z), int(direction), out.ctypes.data, 0))
        return out

    def set_plane_slots(self, z, direction, values, box=0):
        nx, ny, _ = self.boxes[box][:3]
        dt = np.float32 if self.params.precision == HLBM_FP32 else np.float16
        v = np.ascontiguousarray(values, dtype=dt).reshape(5, ny, nx)
        _check(self.h, load().hlbm_plane_slots(self.h, int(box), int(z), int(direction), v.ctypes.data, 1))

    def step_forces(self):
        """Open a split step: the partial momentum exchange over this
        handle's owned cells, (F, T) of shape [n, 3]."""
        n = self.num_particles
        F, T = np.zeros((n, 3)), np.zeros((n, 3))
        _check(self.h, load().hlbm_step_forces(self.h, F.ctypes.data_as(_dp), T.ctypes.data_as(_dp)))
        return F, T

    def step_with_forces(self, F, T):
        """Close a split step with the total hydrodynamic force and torque."""
        F = np.ascontiguousarray(F, np.float64)
        T = np.ascontiguousarray(T, np.float64)
        _check(self.h, load().hlbm_step_with_forces(self.h, F.ctypes.data_as(_dp), T.ctypes.data_as(_dp)))

    def fluid_momentum(self, box=0):
        """(sum of rho - 1, total momentum [3]) of one box, summed on the GPU."""
        out = np.zeros(4)
        _check(self.h, load().hlbm_fluid_momentum(self.h, int(box), out.ctypes.data_as(_dp)))
        return out[0], out[1:].copy()

    def set_mea_mode(self, mode):
        m = {"kernel": HLBM_MEA_KERNEL, "moments": HLBM_MEA_MOMENTS}.get(mode, mode)
        _check(self.h, load().hlbm_set_mea_mode(self.h, int(m)))

    def get_mea_mode(self):
        return {HLBM_MEA_KERNEL: "kernel", HLBM_MEA_MOMENTS: "moments"}[load().hlbm_get_mea_mode(self.h)]

    def autotune(self, nsteps=10):
        """Times every launch shape and momentum-exchange mode, keeps the
        fastest; returns (tile_y, tile_z, cells_x, ms per step)."""
        ty, tz, cx, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_float()
        _check(self.h, load().hlbm_autotune(self.h, int(nsteps), ctypes.byref(ty), ctypes.byref(tz),
                                            ctypes.byref(cx), ctypes.byref(ms)))
        return ty.value, tz.value, cx.value, ms.value

    def kernel_times(self, nsteps=5):
        ms = (ctypes.c_float * 3)()
        _check(self.h, load().hlbm_kernel_times(self.h, int(nsteps), ms))
        return {"mea": ms[0], "update": ms[1], "collide_stream": ms[2]}

    def interior_cells(self):
        """(cell, particle) pairs with the cell centre inside the particle at
        the current state (moments mode, after a step)."""
        n = ctypes.c_longlong(0)
        _check(self.h, load().hlbm_interior_cells(self.h, ctypes.byref(n)))
        return n.value

    def save(self):
        """Snapshot of the whole state the next step reads (bytes)."""
        L = load()
        n = ctypes.c_size_t(0)
        _check(self.h, L.hlbm_checkpoint_bytes(self.h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.h, L.hlbm_save(self.h, buf, n.value))
        return buf.raw

    def load_snapshot(self, data):
        """Restore a snapshot (from save()) into this new handle."""
        data = bytes(data)
        _check(self.h, load().hlbm_load(self.h, data, len(data)))


def hlbm_mea_noalloc(f, plane, nx, ny, nz, bc_flags, precision, fp16_scale_log2, parity, n, shape,
                     shape_params, X, U, omega, quat, F, T, stream):
    """The allocation-free momentum exchange; every array argument is a
    device address (int) or None, as in include/hlbm.h.  Returns the C code."""
    vp = lambda v: _vp(v) if v else None
    return load().hlbm_mea_noalloc(vp(f), ctypes.c_longlong(plane), nx, ny, nz, bc_flags, precision,
                                   fp16_scale_log2, parity, n, vp(shape), vp(shape_params), vp(X), vp(U),
                                   vp(omega), vp(quat), vp(F), vp(T), vp(stream))


def from_workload(w, precision=None, stream=None, **kw):
    """Lattice of one workload description (see the workloads module)."""
    prec = precision or w.get("precision", "fp32")
    P = w["particles"]
    grids = w.get("grids", ())
    kw.setdefault("grid_floats", sum(int(np.asarray(v).size) for v, _ in grids))
    params = make_params(tau=w["tau"], eps=w["eps"], gravity=w["gravity"],
                         fluid_force=w.get("fluid_force", (0, 0, 0)), precision=prec,
                         max_particles=max(1, len(P["shape"])), **kw)
    lat = Lattice([tuple(w["n"]) + (w["bc"],)], params, stream=stream)
    for values, h in grids:
        lat.add_grid(values, h)
    lat.add_workload_particles(P)
    return lat
