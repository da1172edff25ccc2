"""Python binding of libpsq (prolate-spheroidal quadrature of STO integrals on GB300).

Argument marshalling only: every step of the computation runs in the CUDA kernels behind the
C ABI of ``include/psq.h``.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if ``libpsq.so`` is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpsq.so")

S, T, V, J2, J3 = 1, 2, 4, 8, 16
ALL = 31
CLASSES = ("S", "T", "V", "J2", "J3")
FP64, MIXED = 0, 1

STATUS = {0: "PSQ_OK", 1: "PSQ_ERR_ARG", 2: "PSQ_ERR_OOM", 3: "PSQ_ERR_CUDA", 4: "PSQ_ERR_TIMEOUT",
          5: "PSQ_ERR_GEOMETRY", 6: "PSQ_ERR_UNSUPPORTED"}


class PsqError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


class psq_atom(ctypes.Structure):
    _fields_ = [("Z", ctypes.c_int), ("xyz", ctypes.c_double * 3)]


class psq_shell(ctypes.Structure):
    _fields_ = [("atom", ctypes.c_int), ("n", ctypes.c_int), ("l", ctypes.c_int), ("zeta", ctypes.c_double)]


class psq_grid_spec(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int) for k in ("n_mu", "n_nu", "n_phi", "q_mu", "q_nu", "q_phi", "n_sp")]


_lib = None

# (name, restype, argtypes) of every exported entry point
_VP, _I, _U, _SZ, _D = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t, ctypes.c_double
_PD = ctypes.POINTER(ctypes.c_double)
SIGNATURES = [
    ("psq_context_create", _I, [_I, ctypes.POINTER(_VP)]),
    ("psq_context_destroy", _I, [_VP]),
    ("psq_job_create", _I, [_VP, ctypes.POINTER(psq_atom), _I, ctypes.POINTER(psq_shell), _I,
                            ctypes.POINTER(psq_shell), _I, ctypes.POINTER(psq_grid_spec), _I, _I,
                            ctypes.POINTER(_VP)]),
    ("psq_job_destroy", _I, [_VP]),
    ("psq_job_sizes", _I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    ("psq_job_workspace", _I, [_VP, _U, ctypes.POINTER(_SZ)]),
    ("psq_job_stats", _I, [_VP, _U, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_int64),
                           ctypes.POINTER(_D), ctypes.POINTER(_I)]),
    ("psq_job_issued_flops", _I, [_VP, _U, ctypes.POINTER(ctypes.c_double)]),
    ("psq_job_autotune", _I, [_VP, _U, _VP, _SZ, ctypes.POINTER(_VP), _VP, ctypes.POINTER(_I),
                              ctypes.POINTER(ctypes.c_float)]),
    ("psq_compute", _I, [_VP, _U, _VP, _SZ, ctypes.POINTER(_VP), _VP]),
    ("psq_compute_host", _I, [_VP, _U, _VP, _SZ, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]),
    ("psq_compute_graph", _I, [_VP, _U, _VP, _SZ, ctypes.POINTER(_VP), _VP]),
    ("psq_job_grid_info", _I, [_VP, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                               ctypes.POINTER(ctypes.c_int64)]),
    ("psq_job_grid_points", _I, [_VP, _I, _VP, _SZ, _VP, _VP]),
    ("psq_job_grid_functions", _I, [_VP, _I, _I, _VP, _SZ, _VP, ctypes.POINTER(_I), _VP]),
    ("psq_job_io_bytes", _I, [_VP, _U, ctypes.POINTER(_SZ), ctypes.POINTER(_SZ)]),
    ("psq_profile_enable", _I, [_VP, _I]),
    ("psq_profile_read", _I, [_VP, _PD, ctypes.POINTER(_I)]),
    ("psq_check", _I, [_VP, _U, _VP, _VP]),
    ("psq_job_set_wait_limit", _I, [_VP, ctypes.c_uint64]),
    ("psq_job_set_wave_budget", _I, [_VP, _SZ]),
    ("psq_job_test_stall", _I, [_VP, _I]),
    ("psq_compute_noalloc", _I, [_VP, _U, ctypes.POINTER(_VP), _VP]),
    ("psq_server_create", _I, [_VP, _VP, _SZ, _I, ctypes.POINTER(_VP)]),
    ("psq_server_submit", _I, [_VP, _VP, _U, ctypes.POINTER(_VP), ctypes.POINTER(ctypes.c_uint64)]),
    ("psq_server_poll", _I, [_VP, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
    ("psq_server_wait", _I, [_VP, ctypes.c_uint64, _D]),
    ("psq_server_destroy", _I, [_VP]),
    ("psq_last_error", ctypes.c_char_p, []),
    ("psq_ri_factor", _I, [_I, _VP, _VP, _VP, _VP]),
    ("psq_ri_solve", _I, [_I, ctypes.c_int64, _VP, _VP, _VP]),
    ("psq_ri_eri", _I, [_I, ctypes.c_int64, _VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                        _VP, _VP]),
    ("psq_ri_eri_mixed_workspace", _I, [_I, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(_SZ)]),
    ("psq_ri_eri_mixed", _I, [_I, ctypes.c_int64, _VP, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                              _VP, _VP, _SZ, _VP]),
    ("psq_measure_peaks", _I, [_VP, _PD, _PD, _PD]),
]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpsq.so is not built: run paper_2510_15204_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise PsqError(status, lib().psq_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dev_f64(t, name):
    if not (t.is_cuda and t.dtype.is_floating_point and t.element_size() == 8 and t.is_contiguous()):
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def measure_peaks(stream=None):
    """Measured FP64 / FP32 FMA rates (TFLOP/s) and SFU rate (G ops/s) of the current device
    (psq_measure_peaks); synchronises the stream."""
    f64, f32, sfu = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().psq_measure_peaks(_stream_ptr(stream), ctypes.byref(f64), ctypes.byref(f32), ctypes.byref(sfu)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value, "sfu_gops": sfu.value}


def ri_factor(J2, L=None, stream=None):
    """Cholesky factor of the RI metric (P|Q) (eq 14's (PQ)^-1 is L^-T L^-1): returns (L, info),
    info a 1-element int32 CUDA tensor, 0 or k + 1 for a non-positive k-th pivot.  Asynchronous."""
    import torch
    n = J2.shape[0]
    if J2.shape != (n, n):
        raise ValueError("J2 must be square")
    L = torch.empty_like(J2) if L is None else L
    info = torch.empty(1, dtype=torch.int32, device=J2.device)
    _check(lib().psq_ri_factor(n, _dev_f64(J2, "J2"), _dev_f64(L, "L"), ctypes.c_void_p(info.data_ptr()),
                               _stream_ptr(stream)))
    return L, info


def ri_solve(L, B, stream=None):
    """B <- L^-1 B in place (B: n_aux rows; (P|ij) reshaped to n_aux x n_bf^2).  Asynchronous."""
    n = L.shape[0]
    m = B.numel() // n if n else 0
    if B.shape[0] != n:
        raise ValueError("B must have n rows")
    _check(lib().psq_ri_solve(n, m, _dev_f64(L, "L"), _dev_f64(B, "B"), _stream_ptr(stream)))
    return B


def ri_eri(B, c0, nc, d0, nd, out=None, stream=None):
    """Block of RI 4-index integrals (eq 14): out[c][d] = (ij|kl) for ij = c0 + c, kl = d0 + d
    (pair index i * n_bf + j), B from ri_solve.  Asynchronous."""
    import torch
    n = B.shape[0]
    m = B.numel() // n if n else 0
    out = torch.empty((nc, nd), dtype=torch.float64, device=B.device) if out is None else out
    _check(lib().psq_ri_eri(n, m, _dev_f64(B, "B"), c0, nc, d0, nd, _dev_f64(out, "out"), _stream_ptr(stream)))
    return out


def ri_eri_mixed(B, c0, nc, d0, nd, out=None, ws=None, stream=None):
    """ri_eri on the tensor cores (five 8-bit digits per value, within ~2^-38 of the
    window-maximum bound);
    ws: a uint8 CUDA tensor of at least ri_eri_mixed_workspace bytes (allocated if None).
    Asynchronous."""
    import torch
    n = B.shape[0]
    m = B.numel() // n if n else 0
    need = ctypes.c_size_t()
    _check(lib().psq_ri_eri_mixed_workspace(n, nc, nd, ctypes.byref(need)))
    if ws is None:
        ws = torch.empty(max(256, need.value), dtype=torch.uint8, device=B.device)
    out = torch.empty((nc, nd), dtype=torch.float64, device=B.device) if out is None else out
    _check(lib().psq_ri_eri_mixed(n, m, _dev_f64(B, "B"), c0, nc, d0, nd, _dev_f64(out, "out"),
                                  ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream_ptr(stream)))
    return out


class Context:
    """A CUDA device bound to the library."""

    def __init__(self, device: int = 0):
        self.device = device
        h = ctypes.c_void_p()
        _check(lib().psq_context_create(device, ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().psq_context_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Job:
    """An integral job: atoms (Z, (x, y, z)) in bohr, shells (atom, n, l, zeta), one grid spec
    or one per atom pair (n_mu, n_nu, n_phi, q_mu, q_nu, q_phi, n_sp)."""

    def __init__(self, ctx: Context, atoms, basis, aux, specs, precision: int = FP64):
        self.ctx = ctx
        A = (psq_atom * len(atoms))()
        for i, (Z, xyz) in enumerate(atoms):
            A[i].Z = int(Z)
            for c in range(3):
                A[i].xyz[c] = float(xyz[c])
        Bs = (psq_shell * max(1, len(basis)))()
        for i, (a, n, l, z) in enumerate(basis):
            Bs[i].atom, Bs[i].n, Bs[i].l, Bs[i].zeta = int(a), int(n), int(l), float(z)
        As = (psq_shell * max(1, len(aux)))()
        for i, (a, n, l, z) in enumerate(aux):
            As[i].atom, As[i].n, As[i].l, As[i].zeta = int(a), int(n), int(l), float(z)
        Sp = (psq_grid_spec * len(specs))()
        for i, s in enumerate(specs):
            for k, v in zip(("n_mu", "n_nu", "n_phi", "q_mu", "q_nu", "q_phi", "n_sp"), s):
                setattr(Sp[i], k, int(v))
        h = ctypes.c_void_p()
        _check(lib().psq_job_create(ctx.handle, A, len(atoms), Bs, len(basis), As, len(aux), Sp, len(specs),
                                    int(precision), ctypes.byref(h)))
        self.handle = h
        nb, na = ctypes.c_int(), ctypes.c_int()
        _check(lib().psq_job_sizes(h, ctypes.byref(nb), ctypes.byref(na)))
        self.n_bf, self.n_aux = nb.value, na.value

    @classmethod
    def from_synth(cls, ctx, job, precision=FP64):
        return cls(ctx, job.atoms, job.basis, job.aux, job.specs, precision)

    def close(self):
        if getattr(self, "handle", None):
            lib().psq_job_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, mask=ALL) -> int:
        n = ctypes.c_size_t()
        _check(lib().psq_job_workspace(self.handle, mask, ctypes.byref(n)))
        return n.value

    def stats(self, mask=ALL) -> dict:
        g, p, c, n = ctypes.c_int(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int()
        _check(lib().psq_job_stats(self.handle, mask, ctypes.byref(g), ctypes.byref(p), ctypes.byref(c),
                                   ctypes.byref(n)))
        f = ctypes.c_double()
        _check(lib().psq_job_issued_flops(self.handle, mask, ctypes.byref(f)))
        return {"grids": g.value, "points": p.value, "contractions": c.value, "launches": n.value,
                "issued_flops": f.value}

    def out_shapes(self, mask=ALL):
        nb, na = self.n_bf, self.n_aux
        shapes = {"S": (nb, nb), "T": (nb, nb), "V": (nb, nb), "J2": (na, na), "J3": (na, nb, nb)}
        return {k: shapes[k] for i, k in enumerate(CLASSES) if (mask >> i) & 1}

    def alloc(self, mask=ALL, device=None, headroom=0.0):
        """Device workspace and output tensors for mask (torch allocations); headroom is the
        extra fraction of workspace, room for the candidates of autotune()."""
        import torch
        dev = torch.device("cuda", self.ctx.device if device is None else device)
        need = self.workspace_bytes(mask)
        ws = torch.empty(max(256, int(need * (1.0 + headroom))), dtype=torch.uint8, device=dev)
        out = {k: torch.empty(s, dtype=torch.float64, device=dev) for k, s in self.out_shapes(mask).items()}
        return ws, out

    def compute(self, mask=ALL, ws=None, out=None, stream=None):
        """Launches the computation on stream (default: torch's current stream); returns the
        dict of output tensors.  Asynchronous: synchronise before reading."""
        if ws is None or out is None:
            ws2, out2 = self.alloc(mask)
            ws = ws if ws is not None else ws2
            out = out if out is not None else out2
        ptrs = (ctypes.c_void_p * 5)()
        for i, k in enumerate(CLASSES):
            ptrs[i] = out[k].data_ptr() if k in out else None
        _check(lib().psq_compute(self.handle, mask, ctypes.c_void_p(ws.data_ptr()), ws.numel(), ptrs,
                                 _stream_ptr(stream)))
        return out

    def autotune(self, mask, ws, out, stream=None):
        """Times the candidate work splits on ws/out and keeps the fastest plan for mask;
        returns (chosen split, mean ms of one compute).  Synchronises the stream."""
        ptrs = (ctypes.c_void_p * 5)()
        for i, k in enumerate(CLASSES):
            ptrs[i] = out[k].data_ptr() if k in out else None
        split, ms = ctypes.c_int(), ctypes.c_float()
        _check(lib().psq_job_autotune(self.handle, mask, ctypes.c_void_p(ws.data_ptr()), ws.numel(), ptrs,
                                      _stream_ptr(stream), ctypes.byref(split), ctypes.byref(ms)))
        return split.value, ms.value

    def compute_graph(self, mask, ws, out, stream):
        """compute() through the job's captured CUDA graph (stream must not be the default)."""
        ptrs = (ctypes.c_void_p * 5)()
        for i, k in enumerate(CLASSES):
            ptrs[i] = out[k].data_ptr() if k in out else None
        _check(lib().psq_compute_graph(self.handle, mask, ctypes.c_void_p(ws.data_ptr()), ws.numel(), ptrs,
                                       _stream_ptr(stream)))
        return out

    def compute_noalloc(self, mask, out, stream=None):
        """psq_compute_noalloc: the library's fixed device scratch instead of a workspace;
        mask must have been planned (workspace_bytes(mask)) first."""
        ptrs = (ctypes.c_void_p * 5)()
        for i, k in enumerate(CLASSES):
            ptrs[i] = out[k].data_ptr() if k in out else None
        _check(lib().psq_compute_noalloc(self.handle, mask, ptrs, _stream_ptr(stream)))
        return out

    def compute_host(self, mask, ws, out, host_out, stream=None):
        """compute() plus device-to-host copies into host_out (pinned CPU tensors) and a sync."""
        d = (ctypes.c_void_p * 5)()
        h = (ctypes.c_void_p * 5)()
        for i, k in enumerate(CLASSES):
            d[i] = out[k].data_ptr() if k in out else None
            h[i] = host_out[k].data_ptr() if k in host_out else None
        _check(lib().psq_compute_host(self.handle, mask, ctypes.c_void_p(ws.data_ptr()), ws.numel(), d, h,
                                      _stream_ptr(stream)))
        return host_out

    def check(self, mask, ws, stream=None):
        """Waits for the stream; raises PsqError(PSQ_ERR_TIMEOUT) if a kernel gave up a wait.
        ws None: the allocation-free entry point's scratch on the current device."""
        ptr = None if ws is None else ctypes.c_void_p(ws.data_ptr())
        _check(lib().psq_check(self.handle, mask, ptr, _stream_ptr(stream)))

    def set_wave_budget(self, nbytes: int):
        """psq_job_set_wave_budget: the mixed path's operand + packed bytes per wave (0: default)."""
        _check(lib().psq_job_set_wave_budget(self.handle, int(nbytes)))

    def test_stall(self, on: bool):
        """psq_job_test_stall: raise a flag that nothing clears, so the contraction's wait runs out."""
        _check(lib().psq_job_test_stall(self.handle, 1 if on else 0))

    def set_wait_limit(self, ns: int):
        """psq_job_set_wait_limit: the bound of the contraction's device waits, nanoseconds."""
        _check(lib().psq_job_set_wait_limit(self.handle, int(ns)))

    def io_bytes(self, mask=ALL):
        h, d = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib().psq_job_io_bytes(self.handle, mask, ctypes.byref(h), ctypes.byref(d)))
        return h.value, d.value

    PROFILE_KINDS = ("upload", "eval", "contract", "reduce", "assemble", "pack", "k6", "k7")

    def profile(self, on: bool):
        _check(lib().psq_profile_enable(self.handle, 1 if on else 0))

    def profile_read(self):
        """{kind: (total_ms, count)} of the launches recorded since the last read."""
        ms = (ctypes.c_double * 8)()
        cnt = (ctypes.c_int * 8)()
        _check(lib().psq_profile_read(self.handle, ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.PROFILE_KINDS) if cnt[i]}

    # ------------------------------------------------------------- diagnostics
    def grid_info(self, g):
        A, B, C, K = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().psq_job_grid_info(self.handle, g, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C),
                                       ctypes.byref(K)))
        return A.value, B.value, (None if C.value < 0 else C.value), K.value

    def n_grids(self):
        return self.stats(ALL)["grids"]

    def grid_points(self, g, stream=None):
        import torch
        K = self.grid_info(g)[3]
        dev = torch.device("cuda", self.ctx.device)
        ws = torch.empty(max(256, self.workspace_bytes(ALL)), dtype=torch.uint8, device=dev)
        out = torch.empty((8, K), dtype=torch.float64, device=dev)
        _check(lib().psq_job_grid_points(self.handle, g, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def grid_functions(self, g, kind, stream=None):
        import torch
        K = self.grid_info(g)[3]
        dev = torch.device("cuda", self.ctx.device)
        ws = torch.empty(max(256, self.workspace_bytes(ALL)) + (1 << 20) + 64 * (K // 128 + 1),
                         dtype=torch.uint8, device=dev)
        nrows = self.n_bf + self.n_aux  # upper bound
        out = torch.empty((nrows, K), dtype=torch.float64, device=dev)
        rows = ctypes.c_int()
        _check(lib().psq_job_grid_functions(self.handle, g, kind, ctypes.c_void_p(ws.data_ptr()), ws.numel(),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.byref(rows),
                                            _stream_ptr(stream)))
        return out[: rows.value]


class Server:
    """Continuous-batching request loop over one device arena (psq_server_*)."""

    def __init__(self, ctx: Context, arena_bytes: int, max_inflight: int = 4):
        import torch
        self.ctx = ctx
        self.arena = torch.empty(arena_bytes, dtype=torch.uint8, device=torch.device("cuda", ctx.device))
        h = ctypes.c_void_p()
        _check(lib().psq_server_create(ctx.handle, ctypes.c_void_p(self.arena.data_ptr()), arena_bytes,
                                       max_inflight, ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, job: Job, mask, host_out) -> int:
        """host_out: dict class -> pinned CPU float64 tensor of the output shape."""
        ptrs = (ctypes.c_void_p * 5)()
        for i, k in enumerate(CLASSES):
            ptrs[i] = host_out[k].data_ptr() if k in host_out else None
        t = ctypes.c_uint64()
        _check(lib().psq_server_submit(self.handle, job.handle, mask, ptrs, ctypes.byref(t)))
        self._keep[t.value] = (job, host_out)
        return t.value

    def poll(self, ticket):
        d, lat = ctypes.c_int(), ctypes.c_double()
        _check(lib().psq_server_poll(self.handle, ticket, ctypes.byref(d), ctypes.byref(lat)))
        return bool(d.value), lat.value

    def wait(self, ticket, timeout_s=600.0):
        """Latency of a finished ticket (s, submission to results in host memory); the server no
        longer needs the job or its host buffers afterwards."""
        _check(lib().psq_server_wait(self.handle, ticket, timeout_s))
        lat = self.poll(ticket)[1]
        self._keep.pop(ticket, None)
        return lat

    def close(self):
        if getattr(self, "handle", None):
            lib().psq_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
