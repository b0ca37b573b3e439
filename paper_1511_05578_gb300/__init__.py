"""GB300-native spherical curvelet transform (arXiv:1511.05578): Python binding.

Thin ctypes marshalling over libcrv.so, whose C ABI is include/crv.h. Every step of
the transform runs in the library's CUDA kernels; this module only converts
arguments (torch CUDA tensors or raw device pointers, streams) and raises on error
codes. There is no CPU fallback: if libcrv.so is missing or no GPU is visible the
calls raise.

The functions carry the C names (crv_plan_create, crv_analysis, ...). `Plan` is a
small convenience owner of a plan handle with tensor allocation helpers.
"""
import ctypes
import os

__all__ = [
    "CRV_OK", "CRV_EINVAL", "CRV_ENOMEM", "CRV_ECUDA", "CRV_ETIMEOUT", "CRV_EUNSUPPORTED", "CRV_EGUARD", "CRV_F_GUARD",
    "crv_plan_check_guards", "crv_plan_guard_count", "crv_debug_poke_guard", "crv_debug_check_tc_ranges",
    "CRV_NRULE_CURVELET", "CRV_F_REAL", "CRV_F_MIXED", "CRV_F_W_FP32", "CRV_F_UNROTATED", "CRV_F_TUNE", "CRV_F_FP64_TC", "CrvError",
    "lib_path", "load", "crv_plan_create", "crv_plan_destroy", "crv_plan_clone", "crv_plan_bytes", "crv_plan_tuning", "crv_plan_info", "crv_plan_check", "crv_plan_check_stream", "crv_debug_bounded_wait", "crv_plan_kernel",
    "crv_plan_scaling", "crv_plan_delta", "crv_sht_fwd", "crv_sht_inv", "crv_analysis",
    "crv_synthesis", "crv_analysis_lm", "crv_synthesis_lm", "crv_rotate_wigner", "crv_rotate_wigner_adjoint", "crv_delta_table_noalloc", "CRV_NOALLOC_MAX_L", "crv_last_error", "crv_status_string",
    "crv_launch_count", "crv_profile_enable", "crv_profile_kinds", "crv_profile_read", "crv_profile_reset",
    "Plan",
]

CRV_OK, CRV_EINVAL, CRV_ENOMEM, CRV_ECUDA, CRV_ETIMEOUT, CRV_EUNSUPPORTED, CRV_EGUARD = range(7)
CRV_NRULE_CURVELET = 0
CRV_F_REAL, CRV_F_MIXED, CRV_F_W_FP32, CRV_F_UNROTATED, CRV_F_TUNE, CRV_F_FP64_TC, CRV_F_GUARD = 1, 2, 4, 8, 16, 32, 64

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class CrvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def lib_path():
    return os.path.join(_HERE, "libcrv.so")


def load():
    """Load libcrv.so (built by paper_1511_05578_gb300.build.build()); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = lib_path()
    if not os.path.exists(p):
        raise CrvError(CRV_EUNSUPPORTED, f"CUDA extension {p} is not built; run paper_1511_05578_gb300.build.build()")
    h = ctypes.CDLL(p)
    vp, i, u, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_double, ctypes.c_size_t
    sig = {
        "crv_plan_create": (i, [ctypes.POINTER(vp), i, d, i, i, i, u, i, vp]),
        "crv_plan_destroy": (i, [vp]),
        "crv_plan_clone": (i, [ctypes.POINTER(vp), vp, vp]),
        "crv_plan_bytes": (i, [vp, ctypes.POINTER(sz), ctypes.POINTER(sz)]),
        "crv_plan_tuning": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(sz), ctypes.POINTER(i)]),
        "crv_plan_info": (i, [vp, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(sz), ctypes.POINTER(i),
                              ctypes.POINTER(sz)]),
        "crv_plan_check": (i, [vp]),
        "crv_plan_check_stream": (i, [vp, vp]),
        "crv_debug_bounded_wait": (i, [vp, ctypes.c_long, vp]),
        "crv_plan_check_guards": (i, [vp, ctypes.POINTER(i)]),
        "crv_plan_guard_count": (i, [vp, ctypes.POINTER(i)]),
        "crv_debug_poke_guard": (i, [vp, i]),
        "crv_debug_check_tc_ranges": (i, [i, i, i, i, i, i, ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_longlong)]),
        "crv_plan_kernel": (i, [vp, i, ctypes.POINTER(d)]),
        "crv_plan_scaling": (i, [vp, ctypes.POINTER(d)]),
        "crv_plan_delta": (i, [vp, i, ctypes.POINTER(d)]),
        "crv_sht_fwd": (i, [vp, vp, vp, i, vp]),
        "crv_sht_inv": (i, [vp, vp, vp, i, vp]),
        "crv_analysis": (i, [vp, vp, ctypes.POINTER(vp), vp, i, vp]),
        "crv_synthesis": (i, [vp, ctypes.POINTER(vp), vp, vp, i, vp]),
        "crv_analysis_lm": (i, [vp, vp, ctypes.POINTER(vp), vp, i, vp]),
        "crv_synthesis_lm": (i, [vp, ctypes.POINTER(vp), vp, vp, i, vp]),
        "crv_rotate_wigner": (i, [vp, i, vp, vp, i, vp]),
        "crv_rotate_wigner_adjoint": (i, [vp, i, vp, vp, i, vp]),
        "crv_last_error": (ctypes.c_char_p, []),
        "crv_status_string": (ctypes.c_char_p, [i]),
        "crv_launch_count": (ctypes.c_ulonglong, []),
        "crv_delta_table_noalloc": (i, [i, vp, vp]),
        "crv_profile_enable": (i, [u]),
        "crv_profile_num_kinds": (i, []),
        "crv_profile_kind_name": (ctypes.c_char_p, [i]),
        "crv_profile_read": (i, [i, ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(d)]),
        "crv_profile_reset": (i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(h, name)
        f.restype, f.argtypes = res, args
    _lib = h
    return h


def _check(status):
    if status != CRV_OK:
        h = load()
        raise CrvError(status, f"{h.crv_status_string(status).decode()}: {h.crv_last_error().decode()}")


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("libcrv takes device memory: pass CUDA tensors")
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take a device pointer from {type(x)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _ptr_array(xs, n):
    arr = (ctypes.c_void_p * n)()
    for j, x in enumerate(xs):
        arr[j] = _ptr(x)
    return arr


def crv_last_error():
    return load().crv_last_error().decode()


def crv_status_string(s):
    return load().crv_status_string(int(s)).decode()


def crv_launch_count():
    return int(load().crv_launch_count())


def crv_profile_enable(kind_mask):
    _check(load().crv_profile_enable(int(kind_mask)))


def crv_profile_kinds():
    h = load()
    return [h.crv_profile_kind_name(k).decode() for k in range(h.crv_profile_num_kinds())]


def crv_profile_read(k):
    n = ctypes.c_ulonglong()
    t = ctypes.c_double()
    _check(load().crv_profile_read(int(k), ctypes.byref(n), ctypes.byref(t)))
    return int(n.value), float(t.value)


def crv_profile_reset():
    _check(load().crv_profile_reset())


def crv_plan_create(L, lam, J0, spin=0, nrule=CRV_NRULE_CURVELET, flags=0, max_batch=1, stream=None):
    h = load()
    out = ctypes.c_void_p()
    _check(h.crv_plan_create(ctypes.byref(out), int(L), float(lam), int(J0), int(spin), int(nrule), int(flags),
                             int(max_batch), _stream(stream)))
    return out


def crv_plan_destroy(plan):
    _check(load().crv_plan_destroy(plan))


def crv_plan_clone(plan, stream=None):
    """A second instance sharing `plan`'s read-only tables, with its own workspace."""
    h = load()
    out = ctypes.c_void_p()
    _check(h.crv_plan_clone(ctypes.byref(out), plan, _stream(stream)))
    return out


def crv_plan_bytes(plan):
    """(table_bytes, workspace_bytes) of a plan: its shared tables and its own workspace."""
    t, w = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().crv_plan_bytes(plan, ctypes.byref(t), ctypes.byref(w)))
    return t.value, w.value


def crv_plan_tuning(plan):
    """{'workers', 'ring_bytes', 'tuned'}: the plan's launch settings."""
    w, t = ctypes.c_int(), ctypes.c_int()
    r = ctypes.c_size_t()
    _check(load().crv_plan_tuning(plan, ctypes.byref(w), ctypes.byref(r), ctypes.byref(t)))
    return {"workers": w.value, "ring_bytes": r.value, "tuned": bool(t.value)}


def crv_plan_info(plan):
    h = load()
    J = ctypes.c_int()
    _check(h.crv_plan_info(plan, ctypes.byref(J), None, None, None, None))
    n = J.value + 1
    Lj = (ctypes.c_int * n)()
    we = (ctypes.c_size_t * n)()
    Lp = ctypes.c_int()
    ws = ctypes.c_size_t()
    _check(h.crv_plan_info(plan, ctypes.byref(J), Lj, we, ctypes.byref(Lp), ctypes.byref(ws)))
    return {"J": J.value, "Lj": list(Lj), "w_elems": list(we), "L_phi": Lp.value, "workspace_bytes": ws.value}


def crv_plan_check(plan):
    """Synchronise and raise CrvError(CRV_ETIMEOUT) if a bounded device wait gave up."""
    _check(load().crv_plan_check(plan))


def crv_plan_check_stream(plan, stream=None):
    """Wait for the work queued on `stream` only, then raise CrvError(CRV_ETIMEOUT) if a
    bounded device wait of this plan gave up (no device-wide synchronisation)."""
    _check(load().crv_plan_check_stream(plan, _stream(stream)))


def crv_debug_bounded_wait(plan, polls, stream=None):
    """Launch the self-test of the bounded-wait error path (see include/crv.h)."""
    _check(load().crv_debug_bounded_wait(plan, int(polls), _stream(stream)))


def crv_plan_check_guards(plan):
    """Compare every guard region of a CRV_F_GUARD plan with its pattern: returns the status
    (CRV_OK or CRV_EGUARD) and the number of changed regions."""
    n = ctypes.c_int()
    st = load().crv_plan_check_guards(plan, ctypes.byref(n))
    if st not in (CRV_OK, CRV_EGUARD):
        _check(st)
    return st, n.value


def crv_plan_guard_count(plan):
    n = ctypes.c_int()
    _check(load().crv_plan_guard_count(plan, ctypes.byref(n)))
    return n.value


def crv_debug_poke_guard(plan, which):
    """Change one byte inside guard region `which` (tests the check itself)."""
    _check(load().crv_debug_poke_guard(plan, int(which)))


def crv_debug_check_tc_ranges(Lb, lmin_b, lmin_a, real, spin=0, unrot=False):
    """(tiles that break the tensor-core engines' run rules, tiles checked) for one scale; host only."""
    tiles, bad = ctypes.c_longlong(), ctypes.c_longlong()
    _check(load().crv_debug_check_tc_ranges(int(Lb), int(lmin_b), int(lmin_a), int(bool(real)), int(spin),
                                            int(bool(unrot)), ctypes.byref(tiles), ctypes.byref(bad)))
    return bad.value, tiles.value


def crv_plan_kernel(plan, j, out):
    """out: float64 numpy array of L_j * (2L_j - 1) entries (host)."""
    _check(load().crv_plan_kernel(plan, int(j), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def crv_plan_scaling(plan, out):
    _check(load().crv_plan_scaling(plan, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def crv_plan_delta(plan, l, out):
    _check(load().crv_plan_delta(plan, int(l), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


CRV_NOALLOC_MAX_L = 512


def crv_delta_table_noalloc(L, Q, stream=None):
    """Delta quarter table [L][L][L] (float64 device tensor Q) built without any device
    allocation by the library: for callers that must not allocate (see include/crv.h)."""
    _check(load().crv_delta_table_noalloc(int(L), _ptr(Q), _stream(stream)))


def crv_sht_fwd(plan, fmap, flm, B, stream=None):
    _check(load().crv_sht_fwd(plan, _ptr(fmap), _ptr(flm), int(B), _stream(stream)))


def crv_sht_inv(plan, flm, fmap, B, stream=None):
    _check(load().crv_sht_inv(plan, _ptr(flm), _ptr(fmap), int(B), _stream(stream)))


def crv_analysis(plan, fmap, W, Wphi, B, stream=None):
    _check(load().crv_analysis(plan, _ptr(fmap), _ptr_array(W, len(W)), _ptr(Wphi), int(B), _stream(stream)))


def crv_synthesis(plan, W, Wphi, fmap, B, stream=None):
    _check(load().crv_synthesis(plan, _ptr_array(W, len(W)), _ptr(Wphi), _ptr(fmap), int(B), _stream(stream)))


def crv_analysis_lm(plan, flm, W, Wphi, B, stream=None):
    _check(load().crv_analysis_lm(plan, _ptr(flm), _ptr_array(W, len(W)), _ptr(Wphi), int(B), _stream(stream)))


def crv_synthesis_lm(plan, W, Wphi, flm, B, stream=None):
    _check(load().crv_synthesis_lm(plan, _ptr_array(W, len(W)), _ptr(Wphi), _ptr(flm), int(B), _stream(stream)))


def crv_rotate_wigner(plan, j, wt, w, B, stream=None):
    """Wigner coefficients of the rotated curvelet coefficients of scale j from those of the
    unrotated ones (see include/crv.h): wt [B][2][L_j][2L_j-1], w [B][L_j][2L_j-1][2L_j-1],
    complex128 device tensors."""
    _check(load().crv_rotate_wigner(plan, int(j), _ptr(wt), _ptr(w), int(B), _stream(stream)))


def crv_rotate_wigner_adjoint(plan, j, w, wt, B, stream=None):
    _check(load().crv_rotate_wigner_adjoint(plan, int(j), _ptr(w), _ptr(wt), int(B), _stream(stream)))


class Plan:
    """Owns a plan handle; allocates correctly shaped torch tensors for its data."""

    def __init__(self, L, lam=2.0, J0=2, spin=0, flags=0, max_batch=1, stream=None, share=None):
        """share: an existing Plan of the same parameters whose read-only tables this one
        shares (crv_plan_clone); only a workspace is allocated."""
        self.L, self.lam, self.J0, self.spin, self.flags, self.max_batch = L, lam, J0, spin, flags, max_batch
        if share is not None:
            self.handle = crv_plan_clone(share.handle, stream)
        else:
            self.handle = crv_plan_create(L, lam, J0, spin, CRV_NRULE_CURVELET, flags, max_batch, stream)
        info = crv_plan_info(self.handle)
        self.J, self.Lj, self.L_phi, self.bytes = info["J"], info["Lj"], info["L_phi"], info["workspace_bytes"]
        self.real = bool(flags & CRV_F_REAL)
        self.w_dtype_name = "float32" if flags & CRV_F_W_FP32 else "float64"

    def clone(self, stream=None):
        """A Plan sharing this one's tables, for concurrent use on another stream."""
        return Plan(self.L, self.lam, self.J0, self.spin, self.flags, self.max_batch, stream, share=self)

    def table_bytes(self):
        return crv_plan_bytes(self.handle)[0]

    def own_bytes(self):
        return crv_plan_bytes(self.handle)[1]

    def close(self):
        if self.handle is not None:
            crv_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- allocation helpers (torch) --
    def _t(self):
        import torch
        return torch

    def map_tensor(self, B=1, L=None):
        torch = self._t()
        L = self.L if L is None else L
        shape = (B, L, 2 * L - 1) + (() if self.real else (2,))
        return torch.zeros(shape, dtype=torch.float64, device="cuda")

    def flm_tensor(self, B=1):
        torch = self._t()
        return torch.zeros((B, self.L * self.L), dtype=torch.complex128, device="cuda")

    def W_tensors(self, B=1):
        torch = self._t()
        dt = torch.float32 if self.w_dtype_name == "float32" else torch.float64
        out = []
        for j in range(self.J + 1):
            if j < self.J0:
                out.append(None)
                continue
            Lb = self.Lj[j]
            N = 2 * Lb - 1
            shape = (B, Lb, N, N) + (() if self.real else (2,))
            out.append(torch.zeros(shape, dtype=dt, device="cuda"))
        return out

    def wigner_tensor(self, j, B=1):
        """Dense Wigner coefficients of scale j: complex128 [B][L_j][2L_j-1][2L_j-1]."""
        torch = self._t()
        Lb = self.Lj[j]
        return torch.zeros((B, Lb, 2 * Lb - 1, 2 * Lb - 1), dtype=torch.complex128, device="cuda")

    def wigner_edge_tensor(self, j, B=1):
        """Unrotated (|n| = l) Wigner coefficients of scale j: complex128 [B][2][L_j][2L_j-1]."""
        torch = self._t()
        Lb = self.Lj[j]
        return torch.zeros((B, 2, Lb, 2 * Lb - 1), dtype=torch.complex128, device="cuda")

    def Wphi_tensor(self, B=1):
        return self.map_tensor(B, self.L_phi)

    def kernel(self, j):
        import numpy as np
        Lb = self.Lj[j]
        out = np.zeros(Lb * (2 * Lb - 1))
        return crv_plan_kernel(self.handle, j, out).reshape(Lb, 2 * Lb - 1)

    def scaling(self):
        import numpy as np
        return crv_plan_scaling(self.handle, np.zeros(self.L))

    def delta(self, l):
        import numpy as np
        return crv_plan_delta(self.handle, l, np.zeros((l + 1) * (l + 1))).reshape(l + 1, l + 1)
