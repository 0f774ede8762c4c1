"""Python binding of libgint (ctypes): argument marshalling only.

Every function here forwards to the C ABI declared in include/gint.h with the same name;
tensors are passed as raw device pointers, the stream is torch's current CUDA stream.  No
step of the grid integration runs in Python or PyTorch: if the CUDA library cannot be built
or loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

GINT_OK, GINT_EINVAL, GINT_ENOMEM, GINT_ECUDA, GINT_ETIMEOUT, GINT_ESTATE = range(6)
PREC = {"fp64": 0, "fp32": 1, "tf32x3": 2, "bf16x3": 3, "bf16x6": 4, "fp16x3": 5}
PREC_NAME = {v: k for k, v in PREC.items()}

EXPORTS = ["gint_setup", "gint_destroy", "gint_block_layout", "gint_get_info", "gint_update_positions",
           "gint_vlocal", "gint_rho", "gint_force", "gint_rho_force", "gint_strain_derivative", "gint_fold",
           "gint_unfold", "gint_density_matrix",
           "gint_vlocal_backward", "gint_charge",
           "gint_block_dot",
           "gint_block_dot_noalloc", "gint_run_host", "gint_batch_create", "gint_batch_launch", "gint_batch_destroy",
           "gint_autotune", "gint_batched", "gint_get_status", "gint_last_error"]


class GintError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libgint error {code}: {msg}")
        self.code = code


class _Species(C.Structure):
    _fields_ = [("nrad", C.c_int), ("l", C.POINTER(C.c_int)), ("rcut", C.c_double), ("dr", C.c_double),
                ("ntab", C.c_int), ("ftab", C.POINTER(C.c_double)), ("dfdr0", C.POINTER(C.c_double))]


class _Options(C.Structure):
    _fields_ = [("batch", C.c_int * 3), ("batch_rho", C.c_int * 3), ("wait_budget", C.c_int), ("reserved", C.c_int)]


class _Info(C.Structure):
    _fields_ = [("npts", C.c_int64), ("nblocks", C.c_int64), ("nvalues", C.c_int64), ("nbatches", C.c_int64),
                ("nslots", C.c_int64), ("max_orbitals", C.c_int), ("max_slots", C.c_int), ("dV", C.c_double),
                ("flops_useful", C.c_double), ("flops_dense", C.c_double), ("nbatches_rho", C.c_int64),
                ("max_orbitals_rho", C.c_int), ("nbasis", C.c_int), ("flops_dense_rho", C.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgint.so (building it in-tree if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build_library()
        if not os.path.exists(path):
            raise GintError(GINT_ECUDA, f"libgint.so not built at {path}")
        lib = C.CDLL(path)
        P, vp = C.POINTER, C.c_void_p
        i32, i64, d = C.c_int, C.c_int64, C.c_double
        lib.gint_setup.argtypes = [P(vp), P(d), i32, P(i32), P(d), i32, P(_Species), P(i32), P(_Options)]
        lib.gint_destroy.argtypes = [vp]
        lib.gint_block_layout.argtypes = [vp, P(i64), P(i64), P(P(C.c_int32)), P(P(i64))]
        lib.gint_get_info.argtypes = [vp, P(_Info)]
        lib.gint_update_positions.argtypes = [vp, P(d)]
        lib.gint_vlocal.argtypes = [vp, vp, vp, i32, vp]
        lib.gint_rho.argtypes = [vp, vp, vp, i32, vp]
        lib.gint_force.argtypes = [vp, vp, vp, vp, i32, vp]
        lib.gint_rho_force.argtypes = [vp, vp, vp, vp, vp, i32, vp]
        lib.gint_strain_derivative.argtypes = [vp, vp, vp, vp, i32, vp]
        lib.gint_fold.argtypes = [vp, vp, i32, P(d), vp, vp]
        lib.gint_unfold.argtypes = [vp, vp, i32, P(d), P(d), vp, vp]
        lib.gint_density_matrix.argtypes = [vp, i32, P(d), P(d), i32, vp, vp, vp, i32, vp]
        lib.gint_vlocal_backward.argtypes = [vp, vp, vp, vp, vp, i32, vp]
        lib.gint_charge.argtypes = [vp, vp, vp, vp]
        lib.gint_block_dot.argtypes = [vp, vp, vp, vp, vp]
        lib.gint_block_dot_noalloc.argtypes = [vp, vp, vp, vp, vp]
        lib.gint_run_host.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp]
        lib.gint_batched.argtypes = [i32, P(vp), P(vp), P(vp), P(vp), P(vp), i32, vp]
        lib.gint_batch_create.argtypes = [P(vp), i32, P(vp), P(vp), P(vp), P(vp), P(vp), i32]
        lib.gint_batch_launch.argtypes = [vp, vp]
        lib.gint_batch_destroy.argtypes = [vp]
        lib.gint_autotune.argtypes = [P(d), i32, P(i32), P(d), i32, P(_Species), P(i32), i32, P(_Options), P(d), P(d)]
        lib.gint_get_status.argtypes = [vp]
        lib.gint_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "gint_last_error":
                getattr(lib, name).restype = C.c_int
        _lib = lib
        return lib


def _check(rc):
    if rc != GINT_OK:
        msg = load().gint_last_error().decode(errors="replace")
        raise GintError(rc, msg)


def _ptr(t) -> int:
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _cptr(t) -> int:
    """Device pointer of a contiguous complex128 (or float64) CUDA tensor."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype not in (torch.complex128, torch.float64) \
            or not t.is_contiguous():
        raise TypeError("expected a contiguous complex128 CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return int(stream)
    import torch
    return torch.cuda.current_stream().cuda_stream


def _prec(p):
    if isinstance(p, str):
        return PREC[p]
    return int(p)


class Handle:
    """A set-up structure (geometry, species, grid) owned by libgint."""

    def __init__(self, ptr, natoms):
        self._ptr = C.c_void_p(ptr)
        self.natoms = natoms
        self._info = None
        self._layout = None
        self.nvalues = self.info["nvalues"]   # the block list, hence nvalues, is fixed for the handle

    @property
    def info(self):
        """gint_get_info as a dict (read again after a position update)."""
        if self._info is None:
            info = _Info()
            _check(load().gint_get_info(self._ptr, C.byref(info)))
            self._info = {k: getattr(info, k) for k, _ in _Info._fields_}
        return self._info

    @property
    def ptr(self):
        return self._ptr

    def layout(self):
        """(keys [nblocks, 5] int32, offsets [nblocks+1] int64) as numpy copies."""
        if self._layout is None:
            nb, nv = C.c_int64(), C.c_int64()
            kp, op = C.POINTER(C.c_int32)(), C.POINTER(C.c_int64)()
            _check(load().gint_block_layout(self._ptr, C.byref(nb), C.byref(nv), C.byref(kp), C.byref(op)))
            keys = np.ctypeslib.as_array(kp, shape=(nb.value * 5,)).reshape(-1, 5).copy() if nb.value else np.zeros((0, 5), np.int32)
            offs = np.ctypeslib.as_array(op, shape=(nb.value + 1,)).copy()
            self._layout = (keys, offs)
        return self._layout

    def close(self):
        if self._ptr:
            load().gint_destroy(self._ptr)
            self._ptr = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gint_setup(cell, species, tau, tables, grid, batch=(4, 4, 4), batch_rho=(4, 4, 8), wait_budget=0) -> Handle:
    """cell [3,3] rows (bohr), species [natoms] ints, tau [natoms,3] (bohr), tables: list of
    objects with .l, .rcut, .dr, .ftab [nrad, ntab], .dfdr0 (see synth.SpeciesTables)."""
    lib = load()
    cell = np.ascontiguousarray(cell, np.float64).reshape(9)
    species = np.ascontiguousarray(species, np.int32)
    tau = np.ascontiguousarray(tau, np.float64).reshape(-1)
    grid_a = (C.c_int * 3)(*[int(g) for g in grid])
    keep = []
    sp = (_Species * len(tables))()
    for i, t in enumerate(tables):
        l = np.ascontiguousarray(t.l, np.int32)
        f = np.ascontiguousarray(t.ftab, np.float64)
        d0 = np.ascontiguousarray(t.dfdr0, np.float64)
        keep += [l, f, d0]
        sp[i].nrad = len(l)
        sp[i].l = l.ctypes.data_as(C.POINTER(C.c_int))
        sp[i].rcut = float(t.rcut)
        sp[i].dr = float(t.dr)
        sp[i].ntab = int(f.shape[-1])
        sp[i].ftab = f.ctypes.data_as(C.POINTER(C.c_double))
        sp[i].dfdr0 = d0.ctypes.data_as(C.POINTER(C.c_double))
    opt = _Options()
    for i in range(3):
        opt.batch[i] = int(batch[i])
        opt.batch_rho[i] = int(batch_rho[i])
    opt.wait_budget = int(wait_budget)
    out = C.c_void_p()
    _check(lib.gint_setup(C.byref(out), cell.ctypes.data_as(C.POINTER(C.c_double)), len(species),
                          species.ctypes.data_as(C.POINTER(C.c_int)), tau.ctypes.data_as(C.POINTER(C.c_double)),
                          len(tables), sp, grid_a, C.byref(opt)))
    return Handle(out.value, len(species))


def gint_destroy(h: Handle):
    h.close()


def gint_block_layout(h: Handle):
    return h.layout()


def gint_get_info(h: Handle):
    return dict(h.info)


def gint_update_positions(h: Handle, tau):
    tau = np.ascontiguousarray(tau, np.float64).reshape(-1)
    _check(load().gint_update_positions(h.ptr, tau.ctypes.data_as(C.POINTER(C.c_double))))
    h._layout = None
    h._info = None


def gint_vlocal(h: Handle, V, H, prec="fp64", stream=None):
    _check(load().gint_vlocal(h.ptr, _ptr(V), _ptr(H), _prec(prec), _stream(stream)))


def gint_rho(h: Handle, DM, rho, prec="fp64", stream=None):
    _check(load().gint_rho(h.ptr, _ptr(DM), _ptr(rho), _prec(prec), _stream(stream)))


def gint_force(h: Handle, V, DM, F, prec="fp64", stream=None):
    _check(load().gint_force(h.ptr, _ptr(V), _ptr(DM), _ptr(F), _prec(prec), _stream(stream)))


def gint_rho_force(h: Handle, V, DM, rho, F, prec="fp64", stream=None):
    _check(load().gint_rho_force(h.ptr, _ptr(V), _ptr(DM), _ptr(rho), _ptr(F), _prec(prec), _stream(stream)))


def gint_strain_derivative(h: Handle, V, DM, dLde, prec="fp64", stream=None):
    """dLde (device, 9 doubles, row-major) <- dL/deps for L = <DM, V_mu,nu>; the grid part of
    the stress sigma = -dL/deps / Omega."""
    _check(load().gint_strain_derivative(h.ptr, _ptr(V), _ptr(DM), _ptr(dLde), _prec(prec), _stream(stream)))


def _kpoints(kfrac):
    import numpy as np
    k = np.ascontiguousarray(np.atleast_2d(np.asarray(kfrac, np.float64)))
    if k.ndim != 2 or k.shape[1] != 3:
        raise ValueError("k points: shape (nk, 3)")
    return k


def gint_fold(h: Handle, X, kfrac, Xk, stream=None):
    """Xk (device, complex128 [nk, nbasis, nbasis] or float64 view) <- Sum_R X(R) exp(i k.R)."""
    import ctypes as _c
    k = _kpoints(kfrac)
    _check(load().gint_fold(h.ptr, _ptr(X), len(k), k.ctypes.data_as(_c.POINTER(_c.c_double)), _cptr(Xk),
                            _stream(stream)))


def gint_unfold(h: Handle, Xk, kfrac, w, X, stream=None):
    """X (device, block store) <- Re Sum_k w_k Xk exp(-i k.R)."""
    import ctypes as _c
    import numpy as np
    k = _kpoints(kfrac)
    w = np.ascontiguousarray(np.asarray(w, np.float64).reshape(-1))
    if len(w) != len(k):
        raise ValueError("one weight per k point")
    _check(load().gint_unfold(h.ptr, _cptr(Xk), len(k), k.ctypes.data_as(_c.POINTER(_c.c_double)),
                              w.ctypes.data_as(_c.POINTER(_c.c_double)), _ptr(X), _stream(stream)))


def gint_density_matrix(h: Handle, kfrac, w, C, f, DM, prec="fp64", stream=None):
    """DM (device, block store) <- Re Sum_k w_k Sum_n f_nk c_n,mu c*_n,nu exp(-i k.R)
    (Eq. density_matrix).  C: complex128 CUDA tensor [nk, nbasis, nbands]; f: float64 [nk, nbands]."""
    import ctypes as _c
    import numpy as np
    k = _kpoints(kfrac)
    w = np.ascontiguousarray(np.asarray(w, np.float64).reshape(-1))
    if len(w) != len(k) or C.dim() != 3 or C.shape[0] != len(k) or tuple(f.shape) != (len(k), C.shape[2]):
        raise ValueError("C [nk, nbasis, nbands], f [nk, nbands] and one weight per k point")
    _check(load().gint_density_matrix(h.ptr, len(k), k.ctypes.data_as(_c.POINTER(_c.c_double)),
                                      w.ctypes.data_as(_c.POINTER(_c.c_double)), int(C.shape[2]), _cptr(C), _ptr(f),
                                      _ptr(DM), _prec(prec), _stream(stream)))


def gint_vlocal_backward(h: Handle, V, gH, gV, gtau, prec="fp64", stream=None):
    _check(load().gint_vlocal_backward(h.ptr, _ptr(V), _ptr(gH), _ptr(gV), _ptr(gtau), _prec(prec), _stream(stream)))


def gint_charge(h: Handle, rho, out, stream=None):
    _check(load().gint_charge(h.ptr, _ptr(rho), _ptr(out), _stream(stream)))


def gint_block_dot(h: Handle, A, B, out, stream=None):
    _check(load().gint_block_dot(h.ptr, _ptr(A), _ptr(B), _ptr(out), _stream(stream)))


def gint_block_dot_noalloc(h: Handle, A, B, out, stream=None):
    """<A, B> over the block store without allocating (static device scratch)."""
    _check(load().gint_block_dot_noalloc(h.ptr, _ptr(A), _ptr(B), _ptr(out), _stream(stream)))


def _host_ptr(a, writable=False):
    if a is None:
        return None
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous():
            raise TypeError("expected a contiguous float64 CPU tensor")
        return a.data_ptr()
    if a.dtype != np.float64 or not a.flags.c_contiguous or (writable and not a.flags.writeable):
        raise TypeError("expected a contiguous float64 numpy array")
    return a.ctypes.data


def gint_run_host(h: Handle, V, DM, H=None, rho=None, F=None, prec="fp64", stream=None):
    """Host buffers in, host buffers out (copies inside, synchronous)."""
    _check(load().gint_run_host(h.ptr, _host_ptr(V), _host_ptr(DM), _host_ptr(H, True), _host_ptr(rho, True),
                                _host_ptr(F, True), _prec(prec), _stream(stream)))


def gint_batched(handles, V, H, DM=None, rho=None, prec="fp64", stream=None):
    n = len(handles)
    arr = lambda xs: (C.c_void_p * n)(*[_ptr(x) for x in xs])
    hs = (C.c_void_p * n)(*[h.ptr.value for h in handles])
    _check(load().gint_batched(n, hs, arr(V), arr(H), arr(DM) if DM is not None else None,
                               arr(rho) if rho is not None else None, _prec(prec), _stream(stream)))


class Batch:
    """A multi-structure job: one persistent launch per kernel over all structures, replayed
    from a CUDA graph.  Keeps references to the handles and tensors it is bound to."""

    def __init__(self, handles, V, H, DM=None, rho=None, prec="tf32x3"):
        n = len(handles)
        arr = lambda xs: (C.c_void_p * n)(*[_ptr(x) for x in xs])
        hs = (C.c_void_p * n)(*[h.ptr.value for h in handles])
        out = C.c_void_p()
        _check(load().gint_batch_create(C.byref(out), n, hs, arr(V), arr(H), arr(DM) if DM is not None else None,
                                        arr(rho) if rho is not None else None, _prec(prec)))
        self._ptr = out
        self._keep = (list(handles), list(V), list(H), list(DM or []), list(rho or []))

    def launch(self, stream=None):
        _check(load().gint_batch_launch(self._ptr, _stream(stream)))

    def close(self):
        if self._ptr:
            load().gint_batch_destroy(self._ptr)
            self._ptr = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spin_channels(h: Handle, V, H, DM=None, rho=None, prec="tf32x3") -> Batch:
    """Spin channels on one geometry as one multi-structure job (one persistent launch per
    kernel for all channels): collinear spin passes [V_up, V_down] (and [DM_up, DM_down]);
    non-collinear spin passes the four real components [V_uu, V_dd, Re V_ud, Im V_ud] and the
    matching density-matrix components.  H[c] <- vlocal(V[c]); rho[c] <- rho(DM[c])."""
    return Batch([h] * len(V), V, H, DM, rho, prec)


def gint_batch_create(handles, V, H, DM=None, rho=None, prec="tf32x3") -> Batch:
    return Batch(handles, V, H, DM, rho, prec)


def gint_batch_launch(b: Batch, stream=None):
    b.launch(stream)


def gint_batch_destroy(b: Batch):
    b.close()


def gint_autotune(st, prec="tf32x3"):
    """Fastest (batch, batch_rho) shapes for a synth.Structure on the current device, with
    their vlocal and rho times in ms."""
    lib = load()
    cell = np.ascontiguousarray(st.cell, np.float64).reshape(9)
    species = np.ascontiguousarray(st.species, np.int32)
    tau = np.ascontiguousarray(st.tau, np.float64).reshape(-1)
    keep = []
    sp = (_Species * len(st.tables))()
    for i, t in enumerate(st.tables):
        l = np.ascontiguousarray(t.l, np.int32)
        f = np.ascontiguousarray(t.ftab, np.float64)
        d0 = np.ascontiguousarray(t.dfdr0, np.float64)
        keep += [l, f, d0]
        sp[i].nrad, sp[i].l, sp[i].rcut, sp[i].dr = len(l), l.ctypes.data_as(C.POINTER(C.c_int)), float(t.rcut), float(t.dr)
        sp[i].ntab, sp[i].ftab = int(f.shape[-1]), f.ctypes.data_as(C.POINTER(C.c_double))
        sp[i].dfdr0 = d0.ctypes.data_as(C.POINTER(C.c_double))
    grid = (C.c_int * 3)(*[int(g) for g in st.grid])
    best = _Options()
    tv, tr = C.c_double(), C.c_double()
    _check(lib.gint_autotune(cell.ctypes.data_as(C.POINTER(C.c_double)), len(species),
                             species.ctypes.data_as(C.POINTER(C.c_int)), tau.ctypes.data_as(C.POINTER(C.c_double)),
                             len(st.tables), sp, grid, _prec(prec), C.byref(best), C.byref(tv), C.byref(tr)))
    return tuple(best.batch), tuple(best.batch_rho), tv.value, tr.value


def gint_get_status(h: Handle):
    return load().gint_get_status(h.ptr)


def setup_structure(st, batch=(4, 4, 4), batch_rho=(4, 4, 8), tau=None, wait_budget=0) -> Handle:
    """Convenience: gint_setup from a synth.Structure."""
    return gint_setup(st.cell, st.species, st.tau if tau is None else tau, st.tables, st.grid, batch, batch_rho,
                      wait_budget)
