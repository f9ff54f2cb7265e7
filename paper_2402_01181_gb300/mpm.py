"""Python binding of the C ABI in include/mpm.h (ctypes; argument marshalling
only -- every step of the simulation runs in the CUDA library).

The functions mpm_* mirror the C entry points one to one.  `Sim` is a small
convenience wrapper that passes PyTorch's current CUDA stream and caching
allocator to the library and accepts numpy arrays (host) or CUDA tensors
(device).  Importing this module loads libgbmpm.so and raises if it has not
been built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

from . import build as _build

MPM_OK = 0
MPM_ERR_ARG = -1
MPM_ERR_ALLOC = -2
MPM_ERR_CUDA = -3
MPM_ERR_NUMERIC = -4
MPM_ERR_DOMAIN = -5
MPM_ERR_TIMEOUT = -6
MPM_ERR_STATE = -7
MPM_ERR_CAPACITY = -8
MPM_ERR_CFL = -9
MPM_MAX_TOOLS = 8
MPM_PIPELINE_FUSED = 0
MPM_PIPELINE_SPLIT = 1
MPM_TOOL_NONE = -1
MPM_TOOL_CAPSULE = 0
MPM_TOOL_BOX = 1
MPM_TOOL_SAMPLED = 2
MPM_MAX_FIELDS = 16
MPM_KERNEL_CONFIGS = 5
KERNEL_CONFIG_NAMES = {0: "256 threads, 2 passes per flush", 1: "256 threads, 1 pass per flush",
                       2: "128 threads, 2 passes per flush", 3: "128 threads, 1 pass per flush",
                       4: "256 threads, 2 passes per flush, 2 CTAs per SM"}
MPM_MAX_FIELD_RES = 1024

STATUS_NAMES = {0: "MPM_OK", -1: "MPM_ERR_ARG", -2: "MPM_ERR_ALLOC", -3: "MPM_ERR_CUDA", -4: "MPM_ERR_NUMERIC",
                -5: "MPM_ERR_DOMAIN", -6: "MPM_ERR_TIMEOUT", -7: "MPM_ERR_STATE", -8: "MPM_ERR_CAPACITY",
                -9: "MPM_ERR_CFL"}


class mpm_config(ct.Structure):
    _fields_ = [("n_grid", ct.c_int32), ("bound", ct.c_int32), ("dt", ct.c_float),
                ("gravity", ct.c_float * 3), ("E", ct.c_float), ("nu", ct.c_float), ("rho", ct.c_float),
                ("theta", ct.c_float), ("friction_mu", ct.c_float), ("pipeline", ct.c_int32),
                ("n_envs", ct.c_int32), ("max_particles", ct.c_int64)]


mpm_alloc_fn = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p, ct.c_void_p)
mpm_free_fn = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p, ct.c_void_p)

_FP = ct.POINTER(ct.c_float)
_DP = ct.POINTER(ct.c_double)
_U32P = ct.POINTER(ct.c_uint32)

# (name, restype, argtypes) of every exported entry point declared in mpm.h
SIGNATURES = [
    ("mpm_create", ct.c_int, [ct.POINTER(mpm_config), ct.c_void_p, mpm_alloc_fn, mpm_free_fn, ct.c_void_p,
                              ct.POINTER(ct.c_void_p)]),
    ("mpm_destroy", ct.c_int, [ct.c_void_p]),
    ("mpm_load_particles", ct.c_int, [ct.c_void_p, ct.c_int64, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                      ct.c_float, ct.c_int]),
    ("mpm_set_tool_pose", ct.c_int, [ct.c_void_p, ct.c_int32, _DP, _FP]),
    ("mpm_load_batch", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64), ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                  ct.c_void_p, _FP, ct.c_int]),
    ("mpm_set_env_material", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_float, ct.c_float, ct.c_float]),
    ("mpm_set_env_tool_pose", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_int32, _DP, _FP]),
    ("mpm_step", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("mpm_read_particles", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int]),
    ("mpm_last_error", ct.c_char_p, []),
    ("mpm_num_particles", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64)]),
    ("mpm_substeps_taken", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int64)]),
    ("mpm_synchronize", ct.c_int, [ct.c_void_p]),
    ("mpm_clear_error", ct.c_int, [ct.c_void_p]),
    ("mpm_set_stream", ct.c_int, [ct.c_void_p, ct.c_void_p]),
    ("mpm_read_grid", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    ("mpm_grid_velocity", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_int]),
    ("mpm_read_order", ct.c_int, [ct.c_void_p, _U32P, _U32P]),
    ("mpm_block_sort_noalloc", ct.c_int, [ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_void_p, ct.c_void_p,
                                          ct.c_void_p]),
    ("mpm_add_sampled_field", ct.c_int, [ct.c_void_p, ct.c_int32, _DP, ct.c_double, ct.c_void_p, ct.c_int,
                                         ct.POINTER(ct.c_int32)]),
    ("mpm_tape_record", ct.c_int, [ct.c_void_p, ct.c_int32, _DP, ct.c_int32]),
    ("mpm_set_kernel_config", ct.c_int, [ct.c_void_p, ct.c_int32]),
    ("mpm_read_particles_async", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    ("mpm_wait_read", ct.c_int, [ct.c_void_p]),
    ("mpm_extract_surface", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_float, ct.c_void_p, ct.c_int64,
                                       ct.POINTER(ct.c_int64), ct.c_int]),
    ("mpm_get_kernel_config", ct.c_int, [ct.c_void_p, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32),
                                         ct.POINTER(ct.c_int32)]),
    ("mpm_autotune", ct.c_int, [ct.c_void_p, ct.c_int32, _FP, ct.POINTER(ct.c_int32)]),
    ("mpm_tape_backward", ct.c_int, [ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_int,
                                     _DP, _DP, ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p]),
    ("mpm_tape_read_substep", ct.c_int, [ct.c_void_p, ct.c_int32, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                         ct.c_void_p, ct.c_void_p, ct.c_int]),
]


def _load():
    path = _build.library_path()
    if not os.path.exists(path):
        raise RuntimeError("libgbmpm.so is not built (%s); run __graft_entry__.build() first" % path)
    lib = ct.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()

# thin pass-throughs with the C names
mpm_create = lib.mpm_create
mpm_destroy = lib.mpm_destroy
mpm_load_particles = lib.mpm_load_particles
mpm_set_tool_pose = lib.mpm_set_tool_pose
mpm_load_batch = lib.mpm_load_batch
mpm_set_env_material = lib.mpm_set_env_material
mpm_set_env_tool_pose = lib.mpm_set_env_tool_pose
mpm_step = lib.mpm_step
mpm_read_particles = lib.mpm_read_particles
mpm_num_particles = lib.mpm_num_particles
mpm_substeps_taken = lib.mpm_substeps_taken
mpm_synchronize = lib.mpm_synchronize
mpm_clear_error = lib.mpm_clear_error
mpm_set_stream = lib.mpm_set_stream
mpm_read_grid = lib.mpm_read_grid
mpm_grid_velocity = lib.mpm_grid_velocity
mpm_read_order = lib.mpm_read_order
mpm_block_sort_noalloc = lib.mpm_block_sort_noalloc
mpm_add_sampled_field = lib.mpm_add_sampled_field
mpm_tape_record = lib.mpm_tape_record
mpm_set_kernel_config = lib.mpm_set_kernel_config
mpm_read_particles_async = lib.mpm_read_particles_async
mpm_wait_read = lib.mpm_wait_read
mpm_extract_surface = lib.mpm_extract_surface
mpm_get_kernel_config = lib.mpm_get_kernel_config
mpm_autotune = lib.mpm_autotune
mpm_tape_backward = lib.mpm_tape_backward
mpm_tape_read_substep = lib.mpm_tape_read_substep


def mpm_last_error() -> str:
    return (lib.mpm_last_error() or b"").decode()


class MPMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


def check(status: int) -> int:
    if status != MPM_OK:
        raise MPMError(status, mpm_last_error())
    return status


def make_config(n_grid, dt, E, nu, rho, gravity=(0.0, -9.8, 0.0), bound=3, theta=0.0, friction=0.0,
                pipeline=MPM_PIPELINE_FUSED, max_particles=1, n_envs=1) -> mpm_config:
    c = mpm_config()
    c.n_grid = int(n_grid)
    c.bound = int(bound)
    c.dt = float(dt)
    for i in range(3):
        c.gravity[i] = float(gravity[i])
    c.E, c.nu, c.rho = float(E), float(nu), float(rho)
    c.theta, c.friction_mu = float(theta), float(friction)
    c.pipeline = int(pipeline)
    c.n_envs = int(n_envs)
    c.max_particles = int(max_particles)
    return c


def _host_f32(a, cols):
    if a is None:
        return None
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).reshape(-1, cols)
    return a


class Sim:
    """One simulated scene on the current CUDA device.

    Uses PyTorch's caching allocator for device memory and the current
    stream at construction for all work.
    """

    def __init__(self, cfg: mpm_config, use_torch_allocator: bool = True, stream=None):
        import torch
        self._torch = torch
        self.cfg = cfg
        dev = torch.cuda.current_device()
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._keep = []
        self._fields = {}
        self.tape_shape = (0,)
        if use_torch_allocator:
            def _alloc(nbytes, stream, ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, self.stream)
                except Exception:
                    return None

            def _free(ptr, stream, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            a, f = mpm_alloc_fn(_alloc), mpm_free_fn(_free)
            self._keep += [a, f]
        else:
            a, f = mpm_alloc_fn(), mpm_free_fn()
        h = ct.c_void_p()
        check(mpm_create(ct.byref(cfg), ct.c_void_p(self.stream.cuda_stream), a, f, None, ct.byref(h)))
        self.h = h
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            check(mpm_destroy(self.h))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- state
    def load(self, x, particle_volume, v=None, F=None, C=None):
        t = self._torch
        if isinstance(x, t.Tensor) and x.is_cuda:
            arrs = [None if a is None else a.contiguous().float() for a in (x, v, F, C)]
            self._keep_load = arrs
            ptrs = [None if a is None else ct.c_void_p(a.data_ptr()) for a in arrs]
            n = arrs[0].shape[0]
            check(mpm_load_particles(self.h, n, *ptrs, ct.c_float(particle_volume), 1))
        else:
            arrs = [_host_f32(x, 3), _host_f32(v, 3), _host_f32(F, 9), _host_f32(C, 9)]
            ptrs = [None if a is None else a.ctypes.data_as(ct.c_void_p) for a in arrs]
            n = arrs[0].shape[0]
            check(mpm_load_particles(self.h, n, *ptrs, ct.c_float(particle_volume), 0))
        self.n = n

    def load_batch(self, xs, volumes, vs=None, Fs=None, Cs=None):
        """Host arrays per environment (lists); every output concatenates the
        environments in this order."""
        counts = (ct.c_int64 * len(xs))(*[int(np.asarray(x).shape[0]) for x in xs])
        vol = np.ascontiguousarray(np.asarray(volumes, dtype=np.float32))
        cat = lambda arrs, c: None if arrs is None else np.ascontiguousarray(
            np.concatenate([np.asarray(a, np.float32).reshape(-1, c) for a in arrs]))
        arrs = [cat(xs, 3), cat(vs, 3), cat(Fs, 9), cat(Cs, 9)]
        ptrs = [None if a is None else a.ctypes.data_as(ct.c_void_p) for a in arrs]
        check(mpm_load_batch(self.h, counts, *ptrs, vol.ctypes.data_as(_FP), 0))
        self.n = int(sum(counts))
        self.counts = [int(c) for c in counts]

    def set_env_material(self, env, E, nu, rho):
        check(mpm_set_env_material(self.h, int(env), float(E), float(nu), float(rho)))

    def add_field(self, samples, origin, spacing) -> int:
        """Register a sampled distance field (res^3 samples, x fastest) and
        return its id for tools of kind MPM_TOOL_SAMPLED."""
        o = np.ascontiguousarray(np.asarray(origin, dtype=np.float64).reshape(3))
        fid = ct.c_int32()
        if hasattr(samples, "is_cuda") and samples.is_cuda:
            t = samples.contiguous().float()
            res = int(round(t.numel() ** (1.0 / 3.0)))
            assert res ** 3 == t.numel(), "samples must hold res^3 values"
            check(mpm_add_sampled_field(self.h, res, o.ctypes.data_as(_DP), float(spacing),
                                        ct.c_void_p(t.data_ptr()), 1, ct.byref(fid)))
        else:
            a = np.ascontiguousarray(np.asarray(samples, dtype=np.float32))
            res = int(round(a.size ** (1.0 / 3.0)))
            assert res ** 3 == a.size, "samples must hold res^3 values"
            check(mpm_add_sampled_field(self.h, res, o.ctypes.data_as(_DP), float(spacing),
                                        a.ctypes.data_as(ct.c_void_p), 0, ct.byref(fid)))
        return int(fid.value)

    def _shape_for(self, shape, field):
        s = np.array(np.asarray(shape, dtype=np.float32).reshape(8))
        if field is not None and int(s[0]) == MPM_TOOL_SAMPLED:
            key = id(field)
            if key not in self._fields:
                self._fields[key] = (self.add_field(field.samples, field.origin, field.h), field)
            s[1] = self._fields[key][0]
        return s

    def set_env_tool(self, env, tool_id, pose, shape, field=None):
        """Tool pose and shape; a sampled shape (kind MPM_TOOL_SAMPLED) takes
        its distances from `field` (a scenes.SampledField, registered once)."""
        p = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(6))
        s = self._shape_for(shape, field)
        check(mpm_set_env_tool_pose(self.h, int(env), int(tool_id), p.ctypes.data_as(_DP), s.ctypes.data_as(_FP)))

    def set_tool(self, tool_id, pose, shape, field=None):
        p = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(6))
        s = self._shape_for(shape, field)
        check(mpm_set_tool_pose(self.h, int(tool_id), p.ctypes.data_as(_DP), s.ctypes.data_as(_FP)))

    def extract_surface(self, iso=0.5, env=0, device=False):
        """Triangles (T, 3, 3) of the iso-surface of the grid density
        (mpm_extract_surface): a numpy array, or a CUDA tensor if device."""
        n_tri = ct.c_int64()
        check(mpm_extract_surface(self.h, int(env), float(iso), None, 0, ct.byref(n_tri), 0))
        T = n_tri.value
        if device:
            torch = self._torch
            out = torch.empty((max(T, 1), 3, 3), dtype=torch.float32, device="cuda")
            check(mpm_extract_surface(self.h, int(env), float(iso), ct.c_void_p(out.data_ptr()), T, ct.byref(n_tri), 1))
            return out[:T]
        out = np.zeros((max(T, 1), 3, 3), dtype=np.float32)
        check(mpm_extract_surface(self.h, int(env), float(iso), out.ctypes.data_as(ct.c_void_p), T, ct.byref(n_tri), 0))
        return out[:T]

    def set_kernel_config(self, config):
        check(mpm_set_kernel_config(self.h, int(config)))

    def kernel_config(self):
        c, t, g = ct.c_int32(), ct.c_int32(), ct.c_int32()
        check(mpm_get_kernel_config(self.h, ct.byref(c), ct.byref(t), ct.byref(g)))
        return {"config": c.value, "threads": t.value, "ctas": g.value}

    def autotune(self, n_substeps=25):
        """Time every fused-kernel configuration on this state, keep the
        fastest; returns (best, times in ms per configuration)."""
        times = (ct.c_float * MPM_KERNEL_CONFIGS)()
        best = ct.c_int32()
        check(mpm_autotune(self.h, int(n_substeps), times, ct.byref(best)))
        return best.value, [float(t) for t in times]

    def tape_record(self, poses, checkpoint_every=50):
        """Record a rollout of len(poses) sub-steps, poses (K, n_tools, 6):
        the pose of every tool at the end of each sub-step."""
        p = np.ascontiguousarray(np.asarray(poses, dtype=np.float64))
        K = p.shape[0] if p.ndim > 0 else 0
        check(mpm_tape_record(self.h, int(K), p.ctypes.data_as(_DP), int(checkpoint_every)))
        self.tape_shape = p.shape

    def tape_backward(self, x_bar=None, v_bar=None, F_bar=None, C_bar=None, want_state=False):
        """Reverse mode of the recorded rollout from dL/d(final state) (torch
        CUDA tensors or None).  Returns dict(E, nu, poses[, x, v, F, C])."""
        torch = self._torch
        dev = torch.device("cuda", torch.cuda.current_device())

        def arg(t, cols):
            if t is None:
                return None, ct.c_void_p()
            t = t.detach().to(device=dev, dtype=torch.float32).contiguous().reshape(self.n, cols)
            return t, ct.c_void_p(t.data_ptr())

        keep = [arg(x_bar, 3), arg(v_bar, 3), arg(F_bar, 9), arg(C_bar, 9)]
        gm = np.zeros(2)
        gp = np.zeros(self.tape_shape if len(self.tape_shape) == 3 else (0,))
        outs = {}
        ptrs = []
        for name, cols in (("x", 3), ("v", 3), ("F", 9), ("C", 9)):
            if want_state:
                outs[name] = torch.empty((self.n, cols), dtype=torch.float32, device=dev)
                ptrs.append(ct.c_void_p(outs[name].data_ptr()))
            else:
                ptrs.append(ct.c_void_p())
        check(mpm_tape_backward(self.h, keep[0][1], keep[1][1], keep[2][1], keep[3][1], 1, gm.ctypes.data_as(_DP),
                                gp.ctypes.data_as(_DP) if gp.size else None, *ptrs))
        res = {"E": float(gm[0]), "nu": float(gm[1]), "poses": gp}
        res.update(outs)
        return res

    def tape_read_substep(self, j):
        """The recorded state (x, v, F, C) and grid of sub-step j of the last
        segment of a fused-pipeline record (host numpy arrays)."""
        n, ng = self.n, self.cfg.n_grid
        out = {k: np.empty((n, c), np.float32) for k, c in (("x", 3), ("v", 3), ("F", 9), ("C", 9))}
        out["grid"] = np.empty((ng, ng, ng, 4), np.float32)
        ptrs = [out[k].ctypes.data_as(ct.c_void_p) for k in ("x", "v", "F", "C", "grid")]
        check(mpm_tape_read_substep(self.h, int(j), *ptrs, 0))
        return out

    def step(self, n_substeps=1):
        check(mpm_step(self.h, int(n_substeps)))

    def synchronize(self):
        check(mpm_synchronize(self.h))

    def read(self, x=True, v=True, F=True, C=True):
        """Host (numpy) copies of the requested state arrays, in load order."""
        n = self.n
        out = {k: (np.empty((n, c), np.float32) if want else None)
               for k, c, want in (("x", 3, x), ("v", 3, v), ("F", 9, F), ("C", 9, C))}
        ptrs = [None if out[k] is None else out[k].ctypes.data_as(ct.c_void_p) for k in ("x", "v", "F", "C")]
        check(mpm_read_particles(self.h, *ptrs, 0))
        return out

    def read_device(self, x=None, v=None, F=None, C=None):
        """Fill the given CUDA tensors (any may be None)."""
        ptrs = [None if a is None else ct.c_void_p(a.data_ptr()) for a in (x, v, F, C)]
        check(mpm_read_particles(self.h, *ptrs, 1))

    def read_grid(self):
        n, ne = self.cfg.n_grid, max(1, self.cfg.n_envs)
        g = np.empty((ne, n, n, n, 4), np.float32)
        check(mpm_read_grid(self.h, g.ctypes.data_as(ct.c_void_p), 0))
        return g[0] if ne == 1 else g

    def grid_velocity(self):
        n, ne = self.cfg.n_grid, max(1, self.cfg.n_envs)
        g = np.empty((ne, n, n, n, 3), np.float32)
        check(mpm_grid_velocity(self.h, g.ctypes.data_as(ct.c_void_p), 0))
        return g[0] if ne == 1 else g

    def read_order(self):
        ids = np.empty(self.n, np.uint32)
        keys = np.empty(self.n, np.uint32)
        check(mpm_read_order(self.h, ids.ctypes.data_as(_U32P), keys.ctypes.data_as(_U32P)))
        return ids, keys

    def status(self) -> int:
        return mpm_synchronize(self.h)

    def clear_error(self):
        check(mpm_clear_error(self.h))


def sim_from_scene(sc, pipeline=MPM_PIPELINE_FUSED, max_particles=None, load=True, **kw) -> Sim:
    cfg = make_config(sc.n_grid, sc.dt, sc.E, sc.nu, sc.rho, gravity=sc.gravity, bound=sc.bound, theta=sc.theta,
                      friction=sc.friction, pipeline=pipeline, max_particles=max_particles or max(sc.n, 1))
    s = Sim(cfg, **kw)
    if load:
        s.load(sc.x, sc.particle_volume, sc.v, sc.F, sc.C)
        for t, tool in enumerate(sc.tools):
            s.set_tool(t, tool.pose(-1), tool.shape, tool.field)
    return s
