"""ctypes binding of libvrps.so: same names as the C ABI, argument marshalling only.

Every computation happens in the CUDA library; this module checks tensor dtypes, devices,
sizes and contiguity, passes raw pointers and the current CUDA stream, and turns status
codes into exceptions.  There is no CPU fallback: if the library is missing the import
fails with an error that says how to build it.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import _build

_LIB_PATH = _build.LIB

ALGOS = {"ISTA": 0, "FISTA": 1, "SVRG": 2, "SAGA": 3, "PROXSKIP": 4, "VR_PROXSKIP": 5}
ESTIMATORS = {"SVRG": 0, "SAGA": 1, "LSVRG": 2, "SGD": 3}
STORAGE = {"FP32": 0, "BF16": 1, "FP16": 2}
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OUT_OF_MEMORY", -3: "CUDA", -4: "TIMEOUT",
          -5: "DIVERGED", -6: "UNSUPPORTED", -7: "INTERNAL"}


class VrpsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"vrps error {code} ({STATUS.get(code, '?')}): {msg}")
        self.code = code


class SolveOpts(ctypes.Structure):
    _fields_ = [
        ("estimator", ctypes.c_int), ("fgp_iters", ctypes.c_int), ("max_iters", ctypes.c_int),
        ("nonneg", ctypes.c_int), ("power_iters", ctypes.c_int), ("eval_every", ctypes.c_int),
        ("f_star", ctypes.c_double), ("target_gap", ctypes.c_double),
        ("x0", ctypes.c_void_p), ("history", ctypes.c_void_p), ("history_cap", ctypes.c_int),
        ("host_io", ctypes.c_int), ("n_subsets", ctypes.c_int), ("job", ctypes.c_uint32),
        ("storage", ctypes.c_int), ("correction_epochs", ctypes.c_int),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int), ("prox_calls", ctypes.c_int), ("snapshots", ctypes.c_int),
        ("evaluations", ctypes.c_int), ("passes", ctypes.c_double), ("gamma", ctypes.c_double),
        ("lipschitz", ctypes.c_double), ("objective", ctypes.c_double), ("seconds", ctypes.c_double),
        ("reached", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class JobDesc(ctypes.Structure):
    _fields_ = [
        ("geom", ctypes.c_void_p), ("b", ctypes.c_void_p), ("x_out", ctypes.c_void_p),
        ("alpha", ctypes.c_double), ("p", ctypes.c_double), ("gamma", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("job", ctypes.c_uint32), ("estimator", ctypes.c_int),
        ("fgp_iters", ctypes.c_int), ("max_iters", ctypes.c_int), ("n_subsets", ctypes.c_int),
        ("nonneg", ctypes.c_int), ("storage", ctypes.c_int), ("correction_epochs", ctypes.c_int),
    ]


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i, d, i64, u32, u64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                               ctypes.c_uint32, ctypes.c_uint64)
    P = ctypes.POINTER
    sig = {
        "vrps_last_error": (ctypes.c_char_p, []),
        "vrps_version": (i, []),
        "vrps_geom_par2d": (i, [i, i, d, i, P(d), i, d, i, P(vp)]),
        "vrps_geom_cone3d": (i, [i, i, i, d, i, P(d), i, i, d, d, d, d, i, P(vp)]),
        "vrps_geom_free": (i, [vp]),
        "vrps_geom_sizes": (i, [vp, i, P(i64), P(i64), P(i), P(i), P(i)]),
        "vrps_geom_samples": (i, [vp, i, P(i64)]),
        "vrps_autotune": (i, [vp, i, P(d), vp]),
        "vrps_set_launch_shape": (i, [vp, i, i, i, i, i, i]),
        "vrps_launch_shape": (i, [vp, P(i)]),
        "vrps_proj_fwd": (i, [vp, i, vp, vp, vp]),
        "vrps_proj_adj": (i, [vp, i, vp, vp, vp]),
        "vrps_prox_tv": (i, [vp, vp, vp, ctypes.c_float, i, i, vp, vp]),
        "vrps_prox_tv2d_noalloc": (i, [i, i, vp, vp, ctypes.c_float, i, i, vp, vp]),
        "vrps_power_iteration": (i, [vp, i, u64, P(d), vp]),
        "vrps_objective": (i, [vp, vp, vp, d, P(d), vp]),
        "vrps_check_error": (i, [vp, vp]),
        "vrps_selftest_bounded_wait": (i, [u32, vp]),
        "vrps_philox_schedule": (i, [u64, u32, i64, i, i, d, vp, vp]),
        "vrps_launch_shape_full": (i, [vp, P(i)]),
        "vrps_solve_opts_default": (None, [P(SolveOpts)]),
        "vrps_solve": (i, [vp, vp, d, i, d, d, u64, P(SolveOpts), vp, P(Report), vp]),
        "vrps_kernel_launches": (u64, []),
        "vrps_profile_enable": (i, [i]),
        "vrps_profile_read": (i, [P(KernelStat), i, P(i)]),
        "vrps_pdhg": (i, [vp, vp, d, i, i, i, P(d), i, vp, P(Report), vp]),
        "vrps_batch_create": (i, [P(vp)]),
        "vrps_batch_free": (i, [vp]),
        "vrps_batch_set_graphs": (i, [vp, i]),
        "vrps_batch_set_stream_priority": (i, [vp, i]),
        "vrps_batch_set_grid_share": (i, [vp, d]),
        "vrps_batch_submit": (i, [vp, P(JobDesc), P(i)]),
        "vrps_batch_step": (i, [vp, i, P(i)]),
        "vrps_batch_poll": (i, [vp, i, P(i), P(Report)]),
        "vrps_batch_wait": (i, [vp, i, P(Report)]),
        "vrps_batch_sync": (i, [vp]),
        "vrps_batch_ticks": (i, [vp, P(ctypes.c_longlong), P(i)]),
        "vrps_job_footprint": (i, [vp, P(JobDesc), P(ctypes.c_size_t)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(code: int):
    if code != 0:
        raise VrpsError(code, lib.vrps_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _dev_ptr(t: torch.Tensor, name: str, numel: int | None = None, dtype=torch.float32):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(t: torch.Tensor, name: str, numel: int, dtype=torch.float32):
    if t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be a contiguous CPU {dtype} tensor of {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Sizes:
    n: int
    m: int
    rows: int
    row_len: int
    dims: int


class Geometry:
    """Owning wrapper of a vrps_geom handle (vrps_geom_par2d / vrps_geom_cone3d)."""

    def __init__(self, handle, shape, desc):
        self._h = handle
        self.shape = shape          # image / volume shape (ny, nx) or (nz, ny, nx)
        self.desc = desc
        s = self.sizes(-1)
        self.n, self.m, self.row_len, self.dims = s.n, s.m, s.row_len, s.dims

    @classmethod
    def par2d(cls, nx, ny, pixel, angles, n_bins, bin_spacing, n_subsets):
        arr = (ctypes.c_double * len(angles))(*[float(a) for a in angles])
        h = ctypes.c_void_p()
        _check(lib.vrps_geom_par2d(int(nx), int(ny), float(pixel), len(angles), arr, int(n_bins),
                                   float(bin_spacing), int(n_subsets), ctypes.byref(h)))
        return cls(h, (int(ny), int(nx)), dict(kind="par2d", n_angles=len(angles), n_bins=int(n_bins),
                                                n_subsets=int(n_subsets)))

    @classmethod
    def cone3d(cls, nx, ny, nz, voxel, betas, nu, nv, du, dv, sod, sdd, n_subsets):
        arr = (ctypes.c_double * len(betas))(*[float(a) for a in betas])
        h = ctypes.c_void_p()
        _check(lib.vrps_geom_cone3d(int(nx), int(ny), int(nz), float(voxel), len(betas), arr, int(nu),
                                    int(nv), float(du), float(dv), float(sod), float(sdd), int(n_subsets),
                                    ctypes.byref(h)))
        return cls(h, (int(nz), int(ny), int(nx)), dict(kind="cone3d", n_angles=len(betas), nu=int(nu),
                                                         nv=int(nv), n_subsets=int(n_subsets)))

    @classmethod
    def from_spec(cls, spec):
        """Build from a synthetic.Par2DSpec / Cone3DSpec (plain parameter records)."""
        if hasattr(spec, "n_bins"):
            return cls.par2d(spec.nx, spec.ny, spec.pixel, spec.angles, spec.n_bins, spec.bin_spacing,
                             spec.n_subsets)
        return cls.cone3d(spec.nx, spec.ny, spec.nz, spec.voxel, spec.betas, spec.nu, spec.nv, spec.du,
                          spec.dv, spec.sod, spec.sdd, spec.n_subsets)

    @property
    def handle(self):
        if self._h is None:
            raise ValueError("geometry already freed")
        return self._h

    def sizes(self, subset=-1) -> Sizes:
        n, m = ctypes.c_int64(), ctypes.c_int64()
        rows, rl, dims = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.vrps_geom_sizes(self.handle, int(subset), ctypes.byref(n), ctypes.byref(m),
                                   ctypes.byref(rows), ctypes.byref(rl), ctypes.byref(dims)))
        return Sizes(n.value, m.value, rows.value, rl.value, dims.value)

    def samples(self, subset=-1) -> int:
        """Joseph samples (ray-voxels) of a subset (vrps_geom_samples)."""
        out = ctypes.c_int64()
        _check(lib.vrps_geom_samples(self.handle, int(subset), ctypes.byref(out)))
        return out.value

    def close(self):
        if self._h is not None:
            lib.vrps_geom_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def vrps_geom_par2d(*a, **k):
    return Geometry.par2d(*a, **k)


def vrps_geom_cone3d(*a, **k):
    return Geometry.cone3d(*a, **k)


def autotune(g: Geometry, reps: int = 5, stream=None) -> dict:
    """vrps_autotune: 2D forward band and adjoint pixels per thread, or the 3D FGP chunk and
    adjoint voxels per thread, by timing."""
    out = (ctypes.c_double * 4)()
    _check(lib.vrps_autotune(g.handle, int(reps), out, _stream(stream)))
    if g.dims == 3:
        return {"fgp3d_chunk_planes": int(out[0]), "fgp3_iterations_us": float(out[2]),
                "adj3d_voxels_per_thread": int(out[1]), "adj3d_subset_us": float(out[3])}
    shape = launch_shape(g)
    full = launch_shape_full(g)
    return {"fwd_band_bytes": int(out[0]), "fwd_bands_per_cta": int(out[3]), "adj_pixels_per_thread": int(out[1]),
            "adj_angle_shares": max(1, shape[5]), "fgp_tile": ["32x32|27", "32x16", "16x16", "32x32", "32x27"][shape[4]],
            "fwd_adj_us": float(out[2]),
            "all_angles": {"fwd_band_bytes": full[0], "fwd_bands_per_cta": full[1], "adj_angle_shares": full[2]}}


def set_launch_shape(g: Geometry, fwd_band_bytes: int = 0, fwd_group: int = 0, adj_pixels_per_thread: int = 0,
                     fgp3_chunk: int = 0, fgp_tile: int = 0, adj_split: int = 0):
    """vrps_set_launch_shape (0 = built-in default for each).  adj_pixels_per_thread: 1 or 2
    for 2D geometries, voxels per thread along z (16 or 32) for 3D ones."""
    _check(lib.vrps_set_launch_shape(g.handle, int(fwd_band_bytes), int(fwd_group), int(adj_pixels_per_thread),
                                     int(fgp3_chunk), int(fgp_tile), int(adj_split)))


def launch_shape(g: Geometry) -> list:
    """vrps_launch_shape: [fwd band bytes, bands per CTA, adjoint pixels per thread (3D: voxels
    per thread along z), 3D FGP chunk, 2D FGP tile, adjoint angle shares]."""
    out = (ctypes.c_int * 6)()
    _check(lib.vrps_launch_shape(g.handle, out))
    return list(out)


def launch_shape_full(g: Geometry) -> list:
    """vrps_launch_shape_full: [fwd band bytes, bands per CTA, adjoint angle shares] of the 2D
    all-angle passes (0 = as for subsets)."""
    out = (ctypes.c_int * 3)()
    _check(lib.vrps_launch_shape_full(g.handle, out))
    return list(out)


def proj_fwd(g: Geometry, subset: int, x: torch.Tensor, y: torch.Tensor | None = None, stream=None):
    rows = g.sizes(subset).rows
    if y is None:
        y = torch.empty(rows * g.row_len, device=x.device, dtype=torch.float32)
    _check(lib.vrps_proj_fwd(g.handle, int(subset), _dev_ptr(x, "x", g.n), _dev_ptr(y, "y", rows * g.row_len),
                             _stream(stream)))
    return y


def proj_adj(g: Geometry, subset: int, r: torch.Tensor, x: torch.Tensor | None = None, stream=None):
    rows = g.sizes(subset).rows
    if x is None:
        x = torch.empty(g.n, device=r.device, dtype=torch.float32)
    _check(lib.vrps_proj_adj(g.handle, int(subset), _dev_ptr(r, "r", rows * g.row_len), _dev_ptr(x, "x", g.n),
                             _stream(stream)))
    return x


def prox_tv(g: Geometry, v: torch.Tensor, tau: float, iters: int, nonneg: bool = True,
            dual: torch.Tensor | None = None, x: torch.Tensor | None = None, stream=None):
    if x is None:
        x = torch.empty(g.n, device=v.device, dtype=torch.float32)
    dp = _dev_ptr(dual, "dual", g.dims * g.n) if dual is not None else None
    _check(lib.vrps_prox_tv(g.handle, _dev_ptr(v, "v", g.n), _dev_ptr(x, "x", g.n), float(tau), int(iters),
                            1 if nonneg else 0, dp, _stream(stream)))
    return x


def prox_tv2d_noalloc(nx: int, ny: int, v: torch.Tensor, tau: float, iters: int, nonneg: bool = True,
                      dual: torch.Tensor | None = None, x: torch.Tensor | None = None, stream=None):
    """vrps_prox_tv2d_noalloc: the 2D prox without a geometry handle and without allocation
    (fixed device scratch; see include/vrps.h for its limits)."""
    n = int(nx) * int(ny)
    if x is None:
        x = torch.empty(n, device=v.device, dtype=torch.float32)
    dp = _dev_ptr(dual, "dual", 2 * n) if dual is not None else None
    _check(lib.vrps_prox_tv2d_noalloc(int(nx), int(ny), _dev_ptr(v, "v", n), _dev_ptr(x, "x", n), float(tau),
                                      int(iters), 1 if nonneg else 0, dp, _stream(stream)))
    return x


def power_iteration(g: Geometry, iters: int = 100, seed: int = 0, stream=None) -> float:
    out = ctypes.c_double()
    _check(lib.vrps_power_iteration(g.handle, int(iters), int(seed), ctypes.byref(out), _stream(stream)))
    return out.value


def objective(g: Geometry, x: torch.Tensor, b: torch.Tensor, alpha: float, stream=None):
    out = (ctypes.c_double * 3)()
    _check(lib.vrps_objective(g.handle, _dev_ptr(x, "x", g.n), _dev_ptr(b, "b", g.m), float(alpha), out,
                              _stream(stream)))
    return out[0], out[1], out[2]


def selftest_bounded_wait(polls: int = 1000, stream=None):
    """vrps_selftest_bounded_wait: a device-side wait that can only end by its poll limit gives
    up, reports it in the error word, and leaves the device usable (raises VrpsError if not)."""
    _check(lib.vrps_selftest_bounded_wait(int(polls), _stream(stream)))


def check_error(g: Geometry, stream=None):
    """vrps_check_error: synchronises the stream; raises VrpsError (TIMEOUT) when a bounded
    device-side wait of an earlier call on this geometry had expired."""
    _check(lib.vrps_check_error(g.handle, _stream(stream)))


def philox_schedule(seed: int, job: int, k0: int, count: int, n_subsets: int, p: float, stream=None):
    out = torch.empty(count * 3, device="cuda", dtype=torch.int32)
    _check(lib.vrps_philox_schedule(int(seed), int(job), int(k0), int(count), int(n_subsets), float(p),
                                    _dev_ptr(out, "out", count * 3, torch.int32), _stream(stream)))
    return out.view(count, 3)


def solve(b: torch.Tensor, g: Geometry, alpha: float, algo: str = "VR_PROXSKIP", p: float = 1.0,
          gamma: float = 0.0, seed: int = 0, *, estimator: str = "SVRG", fgp_iters: int = 50,
          max_iters: int = 100, nonneg: bool = True, power_iters: int = 100, eval_every: int = 0,
          f_star: float = 0.0, target_gap: float = 0.0, x0: torch.Tensor | None = None,
          history_cap: int = 0, n_subsets: int = 0, job: int = 0, x_out: torch.Tensor | None = None,
          storage: str = "FP32", correction_epochs: int = 0, stream=None):
    """vrps_solve.  b and x_out on the GPU, or both on the host (then the copies happen
    inside the call).  Returns (x_out, report dict, history array [evaluations, 4])."""
    host_io = not b.is_cuda
    o = SolveOpts()
    lib.vrps_solve_opts_default(ctypes.byref(o))
    o.estimator = ESTIMATORS[estimator.upper()]
    o.fgp_iters, o.max_iters, o.nonneg = int(fgp_iters), int(max_iters), 1 if nonneg else 0
    o.power_iters, o.eval_every = int(power_iters), int(eval_every)
    o.f_star, o.target_gap = float(f_star), float(target_gap)
    o.host_io, o.n_subsets, o.job = 1 if host_io else 0, int(n_subsets), int(job)
    o.storage = STORAGE[storage.upper()]
    o.correction_epochs = int(correction_epochs)
    if host_io:
        bp = _host_ptr(b, "b", g.m)
        if x_out is None:
            x_out = torch.empty(g.n, dtype=torch.float32, pin_memory=True)
        xp = _host_ptr(x_out, "x_out", g.n)
        if x0 is not None:
            o.x0 = _host_ptr(x0, "x0", g.n).value
    else:
        bp = _dev_ptr(b, "b", g.m)
        if x_out is None:
            x_out = torch.empty(g.n, device=b.device, dtype=torch.float32)
        xp = _dev_ptr(x_out, "x_out", g.n)
        if x0 is not None:
            o.x0 = _dev_ptr(x0, "x0", g.n).value
    hist = None
    if history_cap > 0:
        hist = (ctypes.c_double * (4 * history_cap))()
        o.history = ctypes.cast(hist, ctypes.c_void_p).value
        o.history_cap = int(history_cap)
    rep = Report()
    code = lib.vrps_solve(bp, g.handle, float(alpha), ALGOS[algo.upper()], float(p), float(gamma), int(seed),
                          ctypes.byref(o), xp, ctypes.byref(rep), _stream(stream))
    _check(code)
    rd = rep.as_dict()
    h = []
    if hist is not None:
        for e in range(min(rep.evaluations, history_cap)):
            h.append([hist[4 * e + q] for q in range(4)])
    return x_out, rd, h


def pdhg(b: torch.Tensor, g: Geometry, alpha: float, iters: int, *, nonneg: bool = True, eval_every: int = 0,
         history_cap: int = 0, x_out: torch.Tensor | None = None, stream=None):
    """vrps_pdhg: preconditioned PDHG reference run.  Returns (x, report dict, history)."""
    if x_out is None:
        x_out = torch.empty(g.n, device=b.device, dtype=torch.float32)
    hist = (ctypes.c_double * (2 * history_cap))() if history_cap > 0 else None
    rep = Report()
    _check(lib.vrps_pdhg(_dev_ptr(b, "b", g.m), g.handle, float(alpha), int(iters), 1 if nonneg else 0,
                         int(eval_every), hist, int(history_cap), _dev_ptr(x_out, "x_out", g.n), ctypes.byref(rep),
                         _stream(stream)))
    h = [(hist[2 * e], hist[2 * e + 1]) for e in range(min(rep.evaluations, history_cap))] if hist else []
    return x_out, rep.as_dict(), h


def kernel_launches() -> int:
    """Cumulative number of CUDA kernels launched by the library in this process."""
    return int(lib.vrps_kernel_launches())


def profile_enable(on: bool = True):
    _check(lib.vrps_profile_enable(1 if on else 0))


def profile_read() -> dict:
    """{kernel name: (launches, total ms, algorithmic bytes)} of the launches recorded while
    profiling was on."""
    cap = 64
    arr = (KernelStat * cap)()
    cnt = ctypes.c_int()
    _check(lib.vrps_profile_read(arr, cap, ctypes.byref(cnt)))
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms), float(arr[k].bytes))
            for k in range(min(cnt.value, cap))}


def _job_desc(g: Geometry, b: torch.Tensor, x_out: torch.Tensor, alpha: float, p: float, gamma: float, seed: int,
              job: int, estimator: str, fgp_iters: int, max_iters: int, n_subsets: int, nonneg: bool,
              storage: str, correction_epochs: int) -> JobDesc:
    d = JobDesc()
    d.geom = g.handle.value if isinstance(g.handle, ctypes.c_void_p) else g.handle
    d.b = _dev_ptr(b, "b", g.m).value
    d.x_out = _dev_ptr(x_out, "x_out", g.n).value
    d.alpha, d.p, d.gamma = float(alpha), float(p), float(gamma)
    d.seed, d.job = int(seed), int(job)
    d.estimator = ESTIMATORS[estimator.upper()]
    d.fgp_iters, d.max_iters, d.n_subsets = int(fgp_iters), int(max_iters), int(n_subsets)
    d.nonneg = 1 if nonneg else 0
    d.storage = STORAGE[storage.upper()]
    d.correction_epochs = int(correction_epochs)
    return d


class Batch:
    """vrps_batch_*: many VR-ProxSkip jobs (all 2D or all 3D) advancing together, one
    iteration per job per tick, each tick's phases one persistent launch over all jobs
    (continuous batching)."""

    def __init__(self, graphs: bool = True, priority: int | None = None, grid_share: float = 1.0):
        h = ctypes.c_void_p()
        _check(lib.vrps_batch_create(ctypes.byref(h)))
        self.handle = h
        self._keep = {}
        if not graphs:
            _check(lib.vrps_batch_set_graphs(self.handle, 0))
        if priority is not None:
            _check(lib.vrps_batch_set_stream_priority(self.handle, int(priority)))
        if grid_share != 1.0:
            _check(lib.vrps_batch_set_grid_share(self.handle, float(grid_share)))

    def submit(self, g: Geometry, b: torch.Tensor, *, alpha: float, p: float, gamma: float, seed: int = 0,
               job: int = 0, estimator: str = "SVRG", fgp_iters: int = 50, max_iters: int = 100,
               n_subsets: int = 0, nonneg: bool = True, storage: str = "FP32", correction_epochs: int = 0,
               x_out: torch.Tensor | None = None) -> int:
        if x_out is None:
            x_out = torch.empty(g.n, device=b.device, dtype=torch.float32)
        d = _job_desc(g, b, x_out, alpha, p, gamma, seed, job, estimator, fgp_iters, max_iters, n_subsets, nonneg,
                      storage, correction_epochs)
        torch.cuda.current_stream().synchronize()   # b must be ready: the batch runs on its own stream
        jid = ctypes.c_int()
        _check(lib.vrps_batch_submit(self.handle, ctypes.byref(d), ctypes.byref(jid)))
        self._keep[jid.value] = (g, b, x_out)
        return jid.value

    def step(self, ticks: int = 1) -> int:
        act = ctypes.c_int()
        _check(lib.vrps_batch_step(self.handle, int(ticks), ctypes.byref(act)))
        return act.value

    def poll(self, jid: int):
        done, rep = ctypes.c_int(), Report()
        _check(lib.vrps_batch_poll(self.handle, int(jid), ctypes.byref(done), ctypes.byref(rep)))
        return bool(done.value), (rep.as_dict() if done.value else None)

    def wait(self, jid: int) -> dict:
        rep = Report()
        _check(lib.vrps_batch_wait(self.handle, int(jid), ctypes.byref(rep)))
        return rep.as_dict()

    def result(self, jid: int) -> torch.Tensor:
        return self._keep[jid][2]

    def release(self, jid: int):
        self._keep.pop(jid, None)

    def sync(self):
        _check(lib.vrps_batch_sync(self.handle))

    def ticks(self):
        t, a = ctypes.c_longlong(), ctypes.c_int()
        _check(lib.vrps_batch_ticks(self.handle, ctypes.byref(t), ctypes.byref(a)))
        return t.value, a.value

    def close(self):
        if self.handle:
            _check(lib.vrps_batch_free(self.handle))
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def job_footprint(g: Geometry, *, max_iters: int, storage: str = "FP32") -> int:
    """vrps_job_footprint: device bytes of one job's state (admission by HBM footprint)."""
    d = JobDesc()
    d.geom = g.handle.value if isinstance(g.handle, ctypes.c_void_p) else g.handle
    d.max_iters = int(max_iters)
    d.storage = STORAGE[storage.upper()]
    out = ctypes.c_size_t()
    _check(lib.vrps_job_footprint(g.handle, ctypes.byref(d), ctypes.byref(out)))
    return out.value
