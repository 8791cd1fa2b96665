"""ctypes binding of libdds (include/dds.h): argument marshalling only.

Every step of set-up and solve runs inside libdds.so (CUDA kernels for sm_103a); this module
only converts Python arguments to the C ABI.  Fields are complex128 arrays of shape
(nrhs, *G[::-1]) on the global extended grid, either torch CUDA tensors (passed by device
pointer, on torch's current stream) or numpy arrays (host buffers, staged by the library).
There is no fallback: if libdds.so is missing, :func:`load` raises.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdds.so")

STATUS = {0: "DDS_OK", 1: "DDS_EINVAL", 2: "DDS_ENOMEM", 3: "DDS_ECUDA", 4: "DDS_ENOCONV",
          5: "DDS_ETIMEOUT", 6: "DDS_EBUSY"}
PRECISION = {"fp64": 0, "mixed": 1, "mixed_bf16": 2, "mixed_fp32": 3}
PLAN = {"auto": 0, "direct": 1, "trace": 2}

EXPORTS = ["dds_setup", "dds_sweep", "dds_sweep_strip", "dds_solve", "dds_apply", "dds_local_solve",
           "dds_set_stream", "dds_get_info", "dds_kernel_launches", "dds_last_error",
           "dds_destroy", "dds_profile", "dds_profile_read", "dds_local_solve_noalloc",
           "dds_server_create", "dds_server_submit", "dds_server_step", "dds_server_poll",
           "dds_server_destroy", "dds_work_per_ddm", "dds_autotune", "dds_set_zero_skip",
           "dds_local_solve_counts", "dds_set_memory_budget", "dds_set_wait_limit",
           "dds_server_slots", "dds_set_launch_shape",
           "dds_tensor_rate"]
KERNEL_KINDS = {"assemble": 0, "subst": 1, "extract": 2, "trace_step": 3, "krylov": 4,
                "other": 5}


class DDSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double),
                ("omega", ctypes.c_double), ("c", ctypes.POINTER(ctypes.c_double)),
                ("parts", ctypes.c_int * 3), ("pml_cells", ctypes.c_int),
                ("pml_strength", ctypes.c_double), ("pml_power", ctypes.c_int),
                ("halo", ctypes.c_int), ("precision", ctypes.c_int), ("plan", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("G", ctypes.c_int * 3), ("M", ctypes.c_int * 3), ("n_sub", ctypes.c_int),
                ("n_factors", ctypes.c_int), ("trace_len", ctypes.c_int), ("plan", ctypes.c_int),
                ("factor_bytes", ctypes.c_longlong), ("setup_seconds", ctypes.c_double),
                ("device_bytes", ctypes.c_longlong), ("trace_kernel", ctypes.c_int),
                ("subst_kernel", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libdds.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libdds.so not found at {path}; run paper_2003_02585_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.dds_setup.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(vp)]
    lib.dds_sweep.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int]
    lib.dds_sweep_strip.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int]
    lib.dds_solve.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_double, ctypes.c_int,
                              ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_double)]
    lib.dds_apply.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.dds_local_solve.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp]
    lib.dds_local_solve_noalloc.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp]
    lib.dds_set_stream.argtypes = [vp, vp]
    lib.dds_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
    lib.dds_kernel_launches.argtypes = [vp]
    lib.dds_kernel_launches.restype = ctypes.c_longlong
    lib.dds_last_error.argtypes = [vp]
    lib.dds_last_error.restype = ctypes.c_char_p
    lib.dds_destroy.argtypes = [vp]
    lib.dds_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                 ctypes.POINTER(ctypes.c_int)]
    lib.dds_work_per_ddm.argtypes = [vp, ctypes.c_int, ctypes.c_int,
                                     ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    lib.dds_destroy.restype = None
    lib.dds_server_create.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_int, ctypes.POINTER(vp)]
    lib.dds_server_submit.argtypes = [vp, vp, ctypes.c_longlong]
    lib.dds_server_step.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.dds_server_poll.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong), vp,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    lib.dds_server_destroy.argtypes = [vp]
    lib.dds_server_slots.argtypes = [vp]
    lib.dds_server_slots.restype = ctypes.c_int
    lib.dds_server_destroy.restype = None
    lib.dds_profile.argtypes = [vp, ctypes.c_int]
    lib.dds_set_zero_skip.argtypes = [vp, ctypes.c_int]
    lib.dds_set_memory_budget.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]
    lib.dds_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
    lib.dds_set_launch_shape.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.dds_set_launch_shape.restype = ctypes.c_int
    lib.dds_tensor_rate.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    lib.dds_tensor_rate.restype = ctypes.c_int
    lib.dds_local_solve_counts.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]
    lib.dds_profile_read.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                     ctypes.POINTER(ctypes.c_double)]
    for name in ["dds_setup", "dds_sweep", "dds_sweep_strip", "dds_solve", "dds_apply", "dds_local_solve",
                 "dds_set_stream", "dds_get_info", "dds_profile", "dds_profile_read",
                 "dds_local_solve_noalloc", "dds_server_create", "dds_server_submit",
                 "dds_server_step", "dds_server_poll", "dds_set_zero_skip",
                 "dds_local_solve_counts", "dds_set_memory_budget", "dds_set_wait_limit"]:
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def local_field_count(b, M, dim):
    """Number of right-hand sides in a local field array of shape M[::-1] or (nrhs,) + M[::-1]
    (complex128, contiguous); raises TypeError / ValueError otherwise."""
    if _is_torch(b):
        import torch
        if b.dtype != torch.complex128:
            raise TypeError(f"local fields must be complex128, got {b.dtype}")
        if not b.is_contiguous():
            raise ValueError("local fields must be contiguous")
    else:
        if np.asarray(b).dtype != np.complex128:
            raise TypeError(f"local fields must be complex128, got {np.asarray(b).dtype}")
    shape = tuple(b.shape)
    loc = tuple(M[::-1])
    if shape == loc:
        return 1
    if len(shape) == dim + 1 and shape[1:] == loc and shape[0] >= 1:
        return int(shape[0])
    raise ValueError(f"local field shape must be {loc} or (nrhs,) + {loc}, got {shape}")


def check_noalloc_pair(b, out, M, dim, device_index):
    """Checks of dds_local_solve_noalloc's arguments made before any pointer is handed over:
    the library reads and writes nrhs * prod(M) * 16 bytes at both addresses, so b and out must
    be complex128 CUDA tensors on the context's device, contiguous, of one local-field shape.
    Returns nrhs."""
    if not (_is_torch(b) and _is_torch(out)):
        raise TypeError("b and out must be torch CUDA tensors (device memory)")
    if not (b.is_cuda and out.is_cuda):
        raise TypeError("b and out must be CUDA tensors")
    for name, t in (("b", b), ("out", out)):
        if device_index is not None and t.device.index != device_index:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the context on "
                             f"cuda:{device_index}")
    nrhs = local_field_count(b, M, dim)
    local_field_count(out, M, dim)
    if tuple(out.shape) != tuple(b.shape):
        raise ValueError(f"out has shape {tuple(out.shape)}, b {tuple(b.shape)}")
    return nrhs


def tensor_rate(kind="tf32"):
    """Measured dense tensor-core rate (TFLOP/s of pieces) of the current device for the TF32 or
    BF16 split-product pieces (dds_tensor_rate)."""
    lib = load()
    v = ctypes.c_double(0.0)
    st = lib.dds_tensor_rate({"tf32": 0, "bf16": 1}[kind], ctypes.byref(v))
    if st != 0:
        raise DDSError(f"dds_tensor_rate failed with status {st}")
    return v.value


class Context:
    """One set-up problem (dds_setup); owns the device factors and buffers."""

    def __init__(self, n, h, omega, c, parts, pml_cells, pml_strength=30.0, pml_power=2,
                 halo=0, precision="fp64", plan="auto"):
        self._lib = load()
        n = tuple(int(v) for v in n)
        parts = tuple(int(v) for v in parts)
        dim = len(n)
        c = np.ascontiguousarray(np.asarray(c, dtype=np.float64))
        if c.shape != n[::-1]:
            raise ValueError(f"c must have shape {n[::-1]}")
        self._c = c
        p = _Problem()
        p.dim = dim
        for a in range(3):
            p.n[a] = n[a] if a < dim else 1
            p.parts[a] = parts[a] if a < dim else 1
        p.h = float(h)
        p.omega = float(omega)
        p.c = c.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.pml_cells = int(pml_cells)
        p.pml_strength = float(pml_strength)
        p.pml_power = int(pml_power)
        p.halo = int(halo)
        p.precision = PRECISION[precision]
        p.plan = PLAN[plan]
        handle = ctypes.c_void_p()
        st = self._lib.dds_setup(ctypes.byref(p), ctypes.byref(handle))
        if st != 0:
            raise DDSError(st, "dds_setup failed (see stderr)")
        self._h = handle
        self.n, self.parts, self.dim = n, parts, dim
        self.precision = precision
        info = self.info()
        self.G = tuple(info["G"][:dim])
        self.M = tuple(info["M"][:dim])
        self.device_index = None
        try:
            import torch
            if torch.cuda.is_available():
                self.device_index = torch.cuda.current_device()
        except ImportError:  # pragma: no cover
            pass

    # -- helpers -----------------------------------------------------------------------------
    def _check(self, st):
        if st != 0:
            raise DDSError(st, self._lib.dds_last_error(self._h).decode())

    def _bind_stream(self, *arrays):
        if any(_is_torch(a) and a.is_cuda for a in arrays):
            import torch
            self._check(self._lib.dds_set_stream(self._h, torch.cuda.current_stream().cuda_stream))

    @staticmethod
    def _ptr(a):
        if _is_torch(a):
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return ctypes.c_void_p(a.data_ptr())
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)

    def _like(self, a, shape):
        if _is_torch(a):
            import torch
            return torch.empty(shape, dtype=torch.complex128, device=a.device)
        return np.empty(shape, dtype=np.complex128)

    def _fields(self, f):
        if _is_torch(f):
            import torch
            if f.dtype != torch.complex128:
                raise TypeError("fields must be complex128")
        else:
            f = np.ascontiguousarray(f, dtype=np.complex128)
        if tuple(f.shape[-self.dim:]) != self.G[::-1]:
            raise ValueError(f"field shape must end with {self.G[::-1]}")
        nrhs = 1 if f.ndim == self.dim else int(f.shape[0])
        return f, nrhs

    # -- API -----------------------------------------------------------------------------------
    def sweep(self, f, rounds=1):
        """u_DDM of Algorithm 2.1 / 4.1 for sources f (dds_sweep)."""
        f, nrhs = self._fields(f)
        u = self._like(f, tuple(f.shape))
        self._bind_stream(f, u)
        self._check(self._lib.dds_sweep(self._h, self._ptr(f), nrhs, self._ptr(u), int(rounds)))
        return u

    def sweep_strip(self, f, nsweeps=3):
        """One-dimensional sweeping DDM of Section 3.2 on a strip partition with nsweeps
        alternating sweeps (dds_sweep_strip)."""
        f, nrhs = self._fields(f)
        u = self._like(f, tuple(f.shape))
        self._bind_stream(f, u)
        self._check(self._lib.dds_sweep_strip(self._h, self._ptr(f), nrhs, self._ptr(u),
                                              int(nsweeps)))
        return u

    def solve(self, f, tol=1e-6, maxit=50, rounds=1):
        """FGMRES with the DDM preconditioner (dds_solve).  Returns (u, iters, relres)."""
        f, nrhs = self._fields(f)
        u = self._like(f, tuple(f.shape))
        self._bind_stream(f, u)
        it = ctypes.c_int(0)
        rel = (ctypes.c_double * nrhs)()
        st = self._lib.dds_solve(self._h, self._ptr(f), nrhs, self._ptr(u), float(tol),
                                 int(maxit), int(rounds), ctypes.byref(it), rel)
        if st not in (0, 4):
            self._check(st)
        return u, int(it.value), np.array(rel[:])

    def apply(self, u):
        """L u = J^{-1} A u (dds_apply)."""
        u, nrhs = self._fields(u)
        out = self._like(u, tuple(u.shape))
        self._bind_stream(u, out)
        self._check(self._lib.dds_apply(self._h, self._ptr(u), nrhs, self._ptr(out)))
        return out

    def local_solve(self, sub, b):
        """Block-tridiagonal local solve on subdomain `sub` (dds_local_solve)."""
        if not _is_torch(b):
            b = np.ascontiguousarray(b, dtype=np.complex128)
        nrhs = local_field_count(b, self.M, self.dim)
        x = self._like(b, tuple(b.shape))
        self._bind_stream(b, x)
        self._check(self._lib.dds_local_solve(self._h, int(sub), self._ptr(b), nrhs, self._ptr(x)))
        return x

    def local_solve_noalloc(self, sub, b, out):
        """Local solve whose scratch is the library's fixed device array (no allocation in
        the call): b and out must be preallocated complex128 CUDA tensors of one shape,
        M[::-1] or (nrhs,) + M[::-1], on the context's device."""
        nrhs = check_noalloc_pair(b, out, self.M, self.dim, self.device_index)
        self._bind_stream(b, out)
        self._check(self._lib.dds_local_solve_noalloc(self._h, int(sub), self._ptr(b), nrhs,
                                                      self._ptr(out)))
        return out

    def info(self):
        inf = _Info()
        self._check(self._lib.dds_get_info(self._h, ctypes.byref(inf)))
        return {"G": list(inf.G), "M": list(inf.M), "n_sub": inf.n_sub,
                "n_factors": inf.n_factors, "trace_len": inf.trace_len, "plan": inf.plan,
                "factor_bytes": inf.factor_bytes, "setup_seconds": inf.setup_seconds,
                "trace_kernel": inf.trace_kernel, "subst_kernel": inf.subst_kernel,
                "device_bytes": inf.device_bytes}

    def launches(self):
        return int(self._lib.dds_kernel_launches(self._h))

    def autotune(self, nrhs, rounds=1):
        """Time the tunable launch shapes (dds_autotune) and keep the fastest; returns
        {"panel_width", "trace_ctas_per_sm", "panels_per_cta",
         "table": [(width, panels per CTA, trace CTAs per SM, ms per DDM application)]};
        trace_ctas_per_sm = 0 is the tensor-core trace kernel."""
        n = ctypes.c_int(0)
        cap = 32
        table = (ctypes.c_double * (4 * cap))()
        best = (ctypes.c_int * 3)()
        self._check(self._lib.dds_autotune(self._h, int(nrhs), int(rounds), cap, ctypes.byref(n),
                                           table, best))
        rows = [(int(table[4 * i]), int(table[4 * i + 1]), int(table[4 * i + 2]),
                 float(table[4 * i + 3])) for i in range(min(n.value, cap))]
        return {"panel_width": int(best[0]), "trace_ctas_per_sm": int(best[1]),
                "panels_per_cta": int(best[2]), "table": rows}

    def work_per_ddm(self, nrhs, rounds=1):
        """(substitution flops, trace-map flops) of one DDM application (dds_work_per_ddm)."""
        a = ctypes.c_double(0.0)
        b = ctypes.c_double(0.0)
        self._check(self._lib.dds_work_per_ddm(self._h, int(nrhs), int(rounds), ctypes.byref(a),
                                               ctypes.byref(b)))
        return a.value, b.value

    def profile(self, enable=True):
        """Enable/disable per-launch CUDA-event timing (dds_profile)."""
        self._check(self._lib.dds_profile(self._h, 1 if enable else 0))

    def kernel_stats(self):
        """{kind: (launches, device ms)} accumulated since profiling was enabled."""
        out = {}
        for name, k in KERNEL_KINDS.items():
            n = ctypes.c_longlong(0)
            ms = ctypes.c_double(0.0)
            self._check(self._lib.dds_profile_read(self._h, k, ctypes.byref(n), ctypes.byref(ms)))
            out[name] = (int(n.value), float(ms.value))
        return out

    def set_memory_budget(self, nbytes):
        """Cap the device memory of this context (dds_set_memory_budget); returns bytes held."""
        used = ctypes.c_longlong(0)
        self._check(self._lib.dds_set_memory_budget(self._h, int(nbytes), ctypes.byref(used)))
        return int(used.value)

    def set_launch_shape(self, panel_width=0, panels_per_cta=1, trace_kernel=2):
        """Pin the launch shapes dds_autotune would choose (dds_set_launch_shape)."""
        self._check(self._lib.dds_set_launch_shape(self._h, int(panel_width), int(panels_per_cta),
                                                   int(trace_kernel)))

    def set_wait_limit(self, polls=0):
        """Polls of a level-completion wait before it gives up (dds_set_wait_limit; 0 = default)."""
        self._check(self._lib.dds_set_wait_limit(self._h, int(polls)))

    def set_zero_skip(self, enable=True):
        """Zero-work skipping of local problems with a zero right-hand side (dds_set_zero_skip)."""
        self._check(self._lib.dds_set_zero_skip(self._h, 1 if enable else 0))

    def local_solve_counts(self, reset=False):
        """(local problems solved, local problems assembled) in compacted substitution launches
        since set-up or the last reset (dds_local_solve_counts)."""
        a = ctypes.c_longlong(0)
        b = ctypes.c_longlong(0)
        self._check(self._lib.dds_local_solve_counts(self._h, ctypes.byref(a), ctypes.byref(b),
                                                     1 if reset else 0))
        return int(a.value), int(b.value)

    def set_stream(self, stream_handle):
        self._check(self._lib.dds_set_stream(self._h, ctypes.c_void_p(stream_handle)))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dds_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- layout helpers (no arithmetic) ----------------------------------------------------------
    def extend(self, f_interior):
        """Place interior-node fields on the global extended grid (zeros in halo/PML)."""
        E = (self.G[0] - self.n[0]) // 2
        lead = f_interior.shape[:-self.dim]
        out = np.zeros(lead + self.G[::-1], dtype=np.complex128)
        sl = tuple(slice(E, E + na) for na in self.n[::-1])
        out[(Ellipsis,) + sl] = f_interior
        return out

    def interior(self, u_ext):
        E = (self.G[0] - self.n[0]) // 2
        sl = tuple(slice(E, E + na) for na in self.n[::-1])
        return u_ext[(Ellipsis,) + sl]


class Server:
    """Continuous-batching server over one Context (dds_server_*): every step admits queued
    right-hand sides into free slots and advances all active ones by one FGMRES iteration with a
    single batched DDM application."""

    def __init__(self, ctx: Context, max_slots: int, tol: float = 1e-6, maxit: int = 30,
                 rounds: int = 1):
        self.ctx = ctx
        self._lib = ctx._lib
        h = ctypes.c_void_p()
        st = self._lib.dds_server_create(ctx._h, int(max_slots), float(tol), int(maxit),
                                         int(rounds), ctypes.byref(h))
        if st != 0:
            raise DDSError(st, self._lib.dds_last_error(ctx._h).decode())
        self._h = h
        self.G = ctx.G
        self.slots = int(self._lib.dds_server_slots(h))   # admitted by device memory

    def submit(self, f, tag: int):
        f, _ = self.ctx._fields(f)
        self.ctx._bind_stream(f)
        self.ctx._check(self._lib.dds_server_submit(self._h, self.ctx._ptr(f), int(tag)))

    def step(self):
        a = ctypes.c_int(0)
        q = ctypes.c_int(0)
        self.ctx._check(self._lib.dds_server_step(self._h, ctypes.byref(a), ctypes.byref(q)))
        return int(a.value), int(q.value)

    def poll(self, out=None):
        """(tag, u, iterations, relres) of one finished request, or None."""
        if out is None:
            out = np.empty(self.G[::-1], dtype=np.complex128)
        tag = ctypes.c_longlong(0)
        it = ctypes.c_int(0)
        rel = ctypes.c_double(0.0)
        self.ctx._bind_stream(out)
        st = self._lib.dds_server_poll(self._h, ctypes.byref(tag), self.ctx._ptr(out),
                                       ctypes.byref(it), ctypes.byref(rel))
        if st == 6:
            return None
        self.ctx._check(st)
        return int(tag.value), out, int(it.value), float(rel.value)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.dds_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
