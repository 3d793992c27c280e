"""ctypes binding of the C ABI in ``include/ps_poisson.h`` (argument marshalling only).

Every solve step runs in the CUDA library ``libps_poisson.so``; this module only
passes pointers, sizes and the current CUDA stream. Importing it raises if the
library has not been built (there is no fallback of any kind). Build it with
``python -m paper_1802_10323_gb300.build`` or ``__graft_entry__.build()``.

The functions ``ps_*`` mirror the C calls one to one; ``Plan`` wraps a plan
with torch-tensor conveniences (device pointers from ``data_ptr()``, the
workspace as a uint8 tensor, the stream from ``torch.cuda.current_stream()``).
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libps_poisson.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                      "(python -m paper_1802_10323_gb300.build)")
_lib = ctypes.CDLL(LIB_PATH)

PS_OK, PS_INVALID_ARG, PS_UNSUPPORTED_SIZE, PS_CUDA_ERROR = 0, 1, 2, 3
PS_OUT_OF_MEMORY, PS_NOT_CONVERGED, PS_TIMEOUT = 4, 5, 6
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED_SIZE", 3: "CUDA_ERROR",
                4: "OUT_OF_MEMORY", 5: "NOT_CONVERGED", 6: "TIMEOUT"}
BC = {"P": 0, "NN": 1, "DD": 2, "ND": 3, "DN": 4, "FD": 5}  # FD: face unknowns (x, y: n <= 4096)
PRECISION = {"fp64": 0, "fp32": 1, "fp32_refine": 2}


class PsInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("r_norm", ctypes.c_double),
                ("f_norm", ctypes.c_double)]


class PsGridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("zf", ctypes.POINTER(ctypes.c_double)), ("dz", ctypes.c_double),
                ("bcx", ctypes.c_int), ("bcy", ctypes.c_int), ("bcz", ctypes.c_int)]


class PsKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_int),
                ("active_launches", ctypes.c_int), ("total_ms", ctypes.c_double),
                ("active_ms", ctypes.c_double)]


_vp, _i, _d, _st = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int
_SIGS = {
    "ps_plan_create": [ctypes.POINTER(_vp), _i, _i, _i, _d, _d, _vp, _d, _i, _i, _i, _i, _d, _i],
    "ps_plan_create_helmholtz": [ctypes.POINTER(_vp), _i, _i, _i, _d, _d, _vp, _d, _i, _i, _i, _i, _d, _i, _d],
    "ps_ns_substep": [_vp, _i, _d, _d, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "ps_workspace_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "ps_solve": [_vp, _vp, _vp, _vp, _vp, _vp],
    "ps_solve_f32": [_vp, _vp, _vp, _vp, _vp, _vp],
    "ps_solve_transpose": [_vp, _vp, _vp, _vp, _vp, _vp],
    "ps_solve_transpose_f32": [_vp, _vp, _vp, _vp, _vp, _vp],
    "ps_solve_host": [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "ps_solve_host_seq": [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                          ctypes.POINTER(_vp), _vp, _vp, ctypes.POINTER(PsInfo)],
    "ps_plan_destroy": [_vp],
    "ps_solve_static": [_vp, _vp, _vp, _vp, _vp],
    "ps_div": [_vp, _vp, _vp, _vp],
    "ps_grad_correct": [_vp, _vp, _vp, _vp, _vp],
    "ps_grad_adjoint": [_vp, _vp, _vp, _vp],
    "ps_div_adjoint_correct": [_vp, _vp, _vp, _vp, _vp],
    "ps_profile_enable": [_vp, _i],
    "ps_profile_read": [_vp, ctypes.POINTER(PsKernelStat), _i, ctypes.POINTER(_i)],
    "ps_batch_create": [ctypes.POINTER(_vp), _i, ctypes.POINTER(PsGridDesc), _i, _d, _i],
    "ps_batch_create_helmholtz": [ctypes.POINTER(_vp), _i, ctypes.POINTER(PsGridDesc), _i, _d, _i,
                                  ctypes.POINTER(ctypes.c_double)],
    "ps_batch_workspace_bytes": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "ps_batch_solve": [_vp, _vp, _vp, _vp, _vp, _vp],
    "ps_batch_destroy": [_vp],
    "ps_batch_autotune": [_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_double)],
    "ps_batch_configure": [_vp, _d, _i],
    "ps_probe_fp64": [_i, ctypes.POINTER(_d), ctypes.POINTER(_d), _vp],
    "ps_inject_alloc_failures": [_i],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _st
_lib.ps_last_error.argtypes = [_vp]
_lib.ps_last_error.restype = ctypes.c_char_p
_lib.ps_batch_last_error.argtypes = [_vp]
_lib.ps_batch_last_error.restype = ctypes.c_char_p
_lib.ps_batch_tile_scale.argtypes = [_vp]
_lib.ps_batch_tile_scale.restype = ctypes.c_int

_OTHER = ["ps_last_error", "ps_batch_last_error", "ps_batch_tile_scale"]
EXPORTS = sorted(list(_SIGS) + _OTHER)


def __getattr__(name):
    if name in _SIGS or name in _OTHER:
        return getattr(_lib, name)
    raise AttributeError(name)


class PoissonError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(status, handle=None):
    if status != PS_OK:
        msg = _lib.ps_last_error(handle)
        raise PoissonError(status, msg.decode() if msg else "")


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def inject_alloc_failures(count):
    """Test hook: the next `count` plan/batch device allocations fail on the host."""
    _check(_lib.ps_inject_alloc_failures(int(count)))


def probe_fp64(iters=20000, stream=None):
    """Measured FP64 FMA throughput of the current device: (TFLOP/s, ms of the timed launch)."""
    tf, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.ps_probe_fp64(int(iters), ctypes.byref(tf), ctypes.byref(ms), _stream_ptr(stream)))
    return tf.value, ms.value


def info_tensor(device="cuda"):
    """A device buffer for one ps_info (32 bytes)."""
    import torch
    return torch.zeros(4, dtype=torch.float64, device=device)


def read_info(t):
    """Decode a ps_info device buffer (after the stream is synchronised)."""
    raw = t.detach().cpu().numpy().tobytes()
    return PsInfo.from_buffer_copy(raw[: ctypes.sizeof(PsInfo)])


class Plan:
    """A solver plan for one grid (see ps_plan_create); alpha > 0 makes it a
    Helmholtz plan, (A − α·I)·p = f (see ps_plan_create_helmholtz)."""

    def __init__(self, nx, ny, nz, dx, dy, zf=None, dz=None, bcs=("P", "P", "NN"),
                 precision="fp64", rtol=1e-10, max_iter=5, alpha=0.0):
        self.shape = (nz, ny, nx)
        self.precision = precision
        self.bcs = tuple(bcs)
        self.alpha = float(alpha)
        self._zf = None if zf is None else np.ascontiguousarray(zf, dtype=np.float64)
        h = _vp()
        zp = None if self._zf is None else self._zf.ctypes.data_as(_vp)
        args = (ctypes.byref(h), nx, ny, nz, float(dx), float(dy), zp, float(dz or 0.0),
                BC[bcs[0]], BC[bcs[1]], BC[bcs[2]], PRECISION[precision], float(rtol), int(max_iter))
        if self.alpha != 0.0:
            _check(_lib.ps_plan_create_helmholtz(*args, self.alpha))
        else:
            _check(_lib.ps_plan_create(*args))
        self.handle = h
        n = ctypes.c_size_t()
        _check(_lib.ps_workspace_bytes(h, ctypes.byref(n)), h)
        self.workspace_bytes = n.value
        self._ws = None

    def workspace(self, device="cuda"):
        import torch
        if self._ws is None or self._ws.device != torch.device(device):
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)
        return self._ws

    def _call(self, fn, f, out, info, stream):
        import torch
        if out is None:
            out = torch.empty_like(f)
        ws = self.workspace(f.device)
        ip = _vp(info.data_ptr()) if info is not None else None
        _check(fn(self.handle, _vp(f.data_ptr()), _vp(out.data_ptr()), _vp(ws.data_ptr()),
                  _stream_ptr(stream), ip), self.handle)
        return out

    def solve(self, f, out=None, info=None, stream=None):
        """Φ with A·Φ = f; f a contiguous CUDA tensor [nz, ny, nx] (float64, or float32 for fp32)."""
        assert f.is_cuda and f.is_contiguous() and tuple(f.shape) == self.shape
        fn = _lib.ps_solve_f32 if self.precision == "fp32" else _lib.ps_solve
        return self._call(fn, f, out, info, stream)

    def solve_transpose(self, g, out=None, info=None, stream=None):
        assert g.is_cuda and g.is_contiguous() and tuple(g.shape) == self.shape
        fn = _lib.ps_solve_transpose_f32 if self.precision == "fp32" else _lib.ps_solve_transpose
        return self._call(fn, g, out, info, stream)

    def ns_substep(self, k, dt, nu, u, ustar, ad, p, phi, rhs, info=None, stream=None):
        """One RK3 substep k ∈ {1, 2, 3} around the solve (see ps_ns_substep): u, ustar, ad
        are stacked (3, nz, ny, nx) face fields, p, phi, rhs cell fields, all contiguous CUDA
        tensors of the plan's dtype; u, ad, p, phi are updated in place."""
        for t, shp in ((u, (3,) + self.shape), (ustar, (3,) + self.shape), (ad, (3,) + self.shape),
                       (p, self.shape), (phi, self.shape), (rhs, self.shape)):
            assert t.is_cuda and t.is_contiguous() and tuple(t.shape) == shp
        ws = self.workspace(u.device)
        ip = _vp(info.data_ptr()) if info is not None else None
        _check(_lib.ps_ns_substep(self.handle, int(k), float(dt), float(nu), _vp(u.data_ptr()),
                                  _vp(ustar.data_ptr()), _vp(ad.data_ptr()), _vp(p.data_ptr()),
                                  _vp(phi.data_ptr()), _vp(rhs.data_ptr()), _vp(ws.data_ptr()),
                                  _stream_ptr(stream), ip), self.handle)

    def solve_host(self, f_host, p_host, f_dev, p_dev, stream=None):
        """End-to-end solve from host memory (copies inside the call); returns PsInfo."""
        ws = self.workspace(f_dev.device)
        info = PsInfo()
        _check(_lib.ps_solve_host(self.handle, _vp(f_host.data_ptr()), _vp(p_host.data_ptr()),
                                  _vp(f_dev.data_ptr()), _vp(p_dev.data_ptr()), _vp(ws.data_ptr()),
                                  _stream_ptr(stream), ctypes.cast(ctypes.byref(info), _vp)), self.handle)
        return info

    def solve_host_seq(self, f_hosts, p_hosts, f_devs, p_devs, stream=None):
        """A sequence of solves from host memory, copies pipelined across problems
        (ps_solve_host_seq): f_hosts, p_hosts lists of host tensors (pinned for
        overlap), f_devs, p_devs the two device slots. Returns a list of PsInfo."""
        n = len(f_hosts)
        if len(p_hosts) != n or len(f_devs) != 2 or len(p_devs) != 2:
            raise ValueError("f_hosts and p_hosts of one length; two device slots each")
        ws = self.workspace(f_devs[0].device)
        arr = lambda ts: (_vp * max(len(ts), 1))(*[t.data_ptr() for t in ts])
        infos = (PsInfo * max(n, 1))()
        _check(_lib.ps_solve_host_seq(self.handle, n, arr(f_hosts), arr(p_hosts), arr(f_devs), arr(p_devs),
                                      _vp(ws.data_ptr()), _stream_ptr(stream), infos), self.handle)
        return [infos[i] for i in range(n)]

    def profile(self, enable=True):
        _check(_lib.ps_profile_enable(self.handle, 1 if enable else 0), self.handle)

    def profile_read(self):
        """Per-kernel-kind timing since the last read: {name: (launches, active, total_ms, active_ms)}."""
        arr = (PsKernelStat * 32)()
        n = ctypes.c_int()
        _check(_lib.ps_profile_read(self.handle, arr, 32, ctypes.byref(n)), self.handle)
        return {arr[i].name.decode(): (arr[i].launches, arr[i].active_launches, arr[i].total_ms,
                                       arr[i].active_ms) for i in range(n.value)}

    def close(self):
        if getattr(self, "handle", None):
            _lib.ps_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent grids solved by one persistent launch (see ps_batch_create).

    grids: list of dicts with nx, ny, nz, dx, dy, zf (array or None), dz, bcs, and an
    optional Helmholtz shift alpha (see ps_batch_create_helmholtz).
    """

    def __init__(self, grids, rtol=1e-10, max_iter=3):
        self.count = len(grids)
        self._zf = []
        descs = (PsGridDesc * self.count)()
        for g, d in enumerate(grids):
            zf = d.get("zf")
            zp = None
            if zf is not None:
                arr = np.ascontiguousarray(zf, dtype=np.float64)
                self._zf.append(arr)
                zp = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            bcs = d.get("bcs", ("P", "P", "NN"))
            descs[g] = PsGridDesc(d["nx"], d["ny"], d["nz"], float(d["dx"]), float(d["dy"]), zp,
                                  float(d.get("dz") or 0.0), BC[bcs[0]], BC[bcs[1]], BC[bcs[2]])
        h = _vp()
        alphas = [float(d.get("alpha", 0.0)) for d in grids]
        if any(alphas):
            arr = (ctypes.c_double * self.count)(*alphas)
            st = _lib.ps_batch_create_helmholtz(ctypes.byref(h), self.count, descs, PRECISION["fp32_refine"],
                                                float(rtol), int(max_iter), arr)
        else:
            st = _lib.ps_batch_create(ctypes.byref(h), self.count, descs, PRECISION["fp32_refine"],
                                      float(rtol), int(max_iter))
        if st != PS_OK:
            raise PoissonError(st, _lib.ps_batch_last_error(None).decode())
        self.handle = h
        n = ctypes.c_size_t()
        self._chk(_lib.ps_batch_workspace_bytes(h, ctypes.byref(n)))
        self.workspace_bytes = n.value
        self._ws = None
        self._ptrs = None

    def _chk(self, st):
        if st != PS_OK:
            raise PoissonError(st, _lib.ps_batch_last_error(self.handle).decode())

    def workspace(self, device="cuda"):
        import torch
        if self._ws is None:
            self._ws = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8, device=device)
        return self._ws

    def pointers(self, fs, ps):
        """Device arrays of the fields' device pointers (kept alive by the batch)."""
        import torch
        dev = fs[0].device
        fptr = torch.tensor([t.data_ptr() for t in fs], dtype=torch.int64, device=dev)
        pptr = torch.tensor([t.data_ptr() for t in ps], dtype=torch.int64, device=dev)
        self._ptrs = (fptr, pptr, list(fs), list(ps))
        return fptr, pptr

    def solve(self, fptr, pptr, infos=None, stream=None):
        ws = self.workspace(fptr.device)
        ip = _vp(infos.data_ptr()) if infos is not None else None
        self._chk(_lib.ps_batch_solve(self.handle, _vp(fptr.data_ptr()), _vp(pptr.data_ptr()),
                                      _vp(ws.data_ptr()), _stream_ptr(stream), ip))

    def autotune(self, fptr, pptr, stream=None):
        ws = self.workspace(fptr.device)
        best = ctypes.c_double()
        self._chk(_lib.ps_batch_autotune(self.handle, _vp(fptr.data_ptr()), _vp(pptr.data_ptr()),
                                         _vp(ws.data_ptr()), _stream_ptr(stream), ctypes.byref(best)))
        return _lib.ps_batch_tile_scale(self.handle), best.value

    def configure(self, wait_limit_seconds=2.0, inject_unsatisfiable_wait=False):
        self._chk(_lib.ps_batch_configure(self.handle, float(wait_limit_seconds),
                                          1 if inject_unsatisfiable_wait else 0))

    def close(self):
        if getattr(self, "handle", None):
            _lib.ps_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def infos_tensor(count, device="cuda"):
    """Device buffer for `count` ps_info records."""
    import torch
    return torch.zeros(count * 4, dtype=torch.float64, device=device)


def read_infos(t, count):
    raw = t.detach().cpu().numpy().tobytes()
    sz = ctypes.sizeof(PsInfo)
    return [PsInfo.from_buffer_copy(raw[i * sz:(i + 1) * sz]) for i in range(count)]
