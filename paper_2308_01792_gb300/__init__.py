"""Python binding of the GB300 matrix-free P1/P2 library (``include/hytet.h``).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``lib/libhytet.so``.  Device vectors are torch CUDA tensors (used
for memory and streams); they are passed to the C ABI as raw pointers.  The
library is loaded on first use and every call fails loudly (RuntimeError) if
it has not been built or a call returns an error code.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libhytet.so")

HG_F32, HG_F64 = 0, 1
HG_SPACE_P1, HG_SPACE_P2 = 1, 2
HG_REPLACE, HG_ADD = 0, 1
HG_MASK_INNER, HG_MASK_ALL = 0, 1
HG_OP_P1_LAPLACE, HG_OP_P1_MASS, HG_OP_P1_DIVKGRAD = 0, 1, 2
HG_OP_P1_DIVKGRAD_STORED = 6
HG_OP_N1_CURLCURL = 7
HG_OP_P1_DIVKGRAD_SURROGATE = 8
HG_OP_P2_LAPLACE, HG_OP_P2_MASS, HG_OP_P2_DIVKGRAD = 3, 4, 5

_P = ctypes.c_void_p
_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double
_PL = ctypes.POINTER(ctypes.c_int64)
_PD = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); every function declared in include/hytet.h
SIGNATURES = {
    "hg_last_error": (ctypes.c_char_p, []),
    "hg_mesh_create": (_I, [_P, _L, _P, _L, ctypes.POINTER(_P)]),
    "hg_mesh_destroy": (None, [_P]),
    "hg_mesh_counts": (_I, [_P, _PL]),
    "hg_hier_create": (_I, [_P, _I, _I, ctypes.POINTER(_P)]),
    "hg_hier_destroy": (None, [_P]),
    "hg_function_size": (_I, [_P, _I, _I, _PL, _PL, _PL, _PL]),
    "hg_canonical_info": (_I, [_P, _I, _I, _P, _P, _P]),
    "hg_to_canonical": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "hg_from_canonical": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "hg_function_create": (_I, [_P, _I, _I, ctypes.POINTER(_P)]),
    "hg_function_destroy": (None, [_P]),
    "hg_function_bind": (_I, [_P, _I, _P, _L]),
    "hg_function_data": (_I, [_P, _I, ctypes.POINTER(_P)]),
    "hg_function_copy_canonical": (_I, [_P, _I, _P, _I, _L, _I, _P]),
    "hg_apply_function": (_I, [_P, _I, _P, _P, _I, _I, _P]),
    "hg_solve_function": (_I, [_P, _I, _P, _P, _D, _I, ctypes.POINTER(ctypes.c_int), _PD, _P]),
    "hg_index_tw": (_I, [_L, _L, _L, _L, _PL]),
    "hg_index_enumerate": (_I, [_L, _P, _P]),
    "hg_interface_dump": (_I, [_P, _I, _I, _P, _PL, _PL, _P]),
    "hg_op_create": (_I, [_P, _I, _P, ctypes.POINTER(_P)]),
    "hg_op_destroy": (None, [_P]),
    "hg_op_create_surrogate": (_I, [_P, _P, _I, ctypes.POINTER(_P)]),
    "hg_partition_cells": (_I, [_P, _I, _P]),
    "hg_exchange_plan": (_I, [_P, _I, _P, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P]),
    "hg_apply": (_I, [_P, _I, _I, _P, _P, _I, _I, _P]),
    "hg_residual": (_I, [_P, _I, _I, _P, _P, _P, _P]),
    "hg_jacobi": (_I, [_P, _I, _I, _D, _P, _P, _P, _P]),
    "hg_restrict": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "hg_prolong_add": (_I, [_P, _I, _I, _I, _P, _P, _P]),
    "hg_dot": (_I, [_P, _I, _I, _I, _P, _P, _I, _PD, _P]),
    "hg_device_status": (_I, [_P, _P]),
    "hg_dot_noalloc": (_I, [_P, _I, _I, _I, _P, _P, _I, _P, _P]),
    "hg_gmg_default_params": (None, [_P]),
    "hg_gmg_create": (_I, [_P, _P, ctypes.POINTER(_P)]),
    "hg_gmg_destroy": (None, [_P]),
    "hg_vcycle": (_I, [_P, _I, _I, _P, _P, _P]),
    "hg_solve": (_I, [_P, _I, _P, _P, _D, _I, ctypes.POINTER(ctypes.c_int), _PD, _P]),
    "hg_gmg_history": (_I, [_P, _PD, _I, ctypes.POINTER(ctypes.c_int)]),
    "hg_mlp_create": (_I, [ctypes.POINTER(_P)]),
    "hg_mlp_destroy": (None, [_P]),
    "hg_mlp_set_params": (_I, [_P, _P]),
    "hg_mlp_get_params": (_I, [_P, _P]),
    "hg_mlp_forward": (_I, [_P, _P, _L, _P, _P]),
    "hg_mlp_grad": (_I, [_P, _P, _P, _L, _P, _PD, _P]),
    "hg_mlp_train": (_I, [_P, _P, _P, _L, _I, _L, _D, _PD, _P]),
    "hg_learn_samples": (_I, [_P, _I, _P, _P, _P, _D, _I, _I, _P, _P, _PL, _P]),
    "hg_gmg_set_learned": (_I, [_P, _P]),
    "hg_learned_step": (_I, [_P, _P, _I, _P, _P, _D, _P, _P]),
    "hg_gmg_learned_fallbacks": (_I, [_P, ctypes.POINTER(ctypes.c_int)]),
    "hg_gmg_clone": (_I, [_P, ctypes.POINTER(_P)]),
    "hg_quadrature_rule": (_I, [_P, _P, ctypes.POINTER(ctypes.c_int)]),
    "hg_gauss_seidel": (_I, [_P, _I, _I, _I, _P, _P, _P, _P]),
    "hg_gs_colours": (_I, [_P, _I, _P]),
    "hg_batch_create": (_I, [_P, _I, _P, _P, _I, ctypes.POINTER(_P)]),
    "hg_batch_destroy": (None, [_P]),
    "hg_batch_solve": (_I, [_P, _D, _I, _P, _P, _P]),
    "hg_batch_tuning": (_I, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _PD]),
    "hg_gmg_lambda": (_I, [_P, _I, _PD]),
    "hg_gmg_set_lambda": (_I, [_P, _I, _D]),
    "hg_gmg_potential_lambda": (_I, [_P, _I, _PD]),
    "hg_gmg_set_potential_lambda": (_I, [_P, _I, _D]),
    "hg_gmg_power_lambda": (_I, [_P, _I, _P, _I, _PD, _P]),
    "hg_fmg": (_I, [_P, _I, _I, _P, _P, _I, _P]),
    "hg_n1_prolong_table": (_I, [_P, _P, _P, _P, _P]),
    "hg_plane_tiles": (_I, [_I, _P, ctypes.POINTER(ctypes.c_int)]),
    "hg_stream_plan": (_I, [_I, _I, _I, _I, _P, _P, _P, _P, _P]),
    "hg_set_p1_kernel": (_I, [_I]),
    "hg_march_items": (_I, [_I, _P, ctypes.POINTER(ctypes.c_int)]),
    "hg_stream_layout": (_I, [_I, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_int)]),
    "hg_p2_anchors": (_I, [_I, _P, _P, ctypes.POINTER(ctypes.c_int)]),
    "hg_n1_restrict_table": (_I, [_P, _P, _P, _P]),
    "hg_n1_prolong_add": (_I, [_P, _I, _I, _P, _P, _P]),
    "hg_n1_restrict": (_I, [_P, _I, _I, _P, _P, _P]),
    "hg_n1_gradient": (_I, [_P, _I, _I, _P, _P, _P]),
    "hg_n1_gradient_t": (_I, [_P, _I, _I, _P, _P, _P]),
}

HG_BATCH_GRAPH, HG_BATCH_AUTOTUNE = 1, 2
HG_COPY_TO_HOST, HG_COPY_FROM_HOST = 0, 1

HG_PREC_F64, HG_PREC_MIXED = 0, 1
HG_SMOOTH_JACOBI, HG_SMOOTH_GS, HG_SMOOTH_CHEB = 0, 1, 2


class GmgParams(ctypes.Structure):
    _fields_ = [("nu1", ctypes.c_int), ("nu2", ctypes.c_int), ("omega", ctypes.c_double),
                ("lmin", ctypes.c_int), ("inner_cycles", ctypes.c_int), ("smoother", ctypes.c_int),
                ("cheb_order", ctypes.c_int), ("cheb_iters", ctypes.c_int),
                ("cheb_lo", ctypes.c_double), ("cheb_hi", ctypes.c_double)]

_lib = None


class HGError(RuntimeError):
    def __init__(self, name, code, msg):
        super().__init__(f"{name} failed with code {code}: {msg}")
        self.code = code


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2308_01792_gb300.build.build() (nvcc, sm_103a)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _call(name, *args):
    r = getattr(lib(), name)(*args)
    if r != 0:
        raise HGError(name, r, lib().hg_last_error().decode())
    return r


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float32:
        return HG_F32
    if t.dtype == torch.float64:
        return HG_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _ptr(t, n=None):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} elements, need {n}")
    return ctypes.c_void_p(t.data_ptr())


class Mesh:
    """Macro mesh (Sec. 2): vertices (nv,3) float64, cells (nc,4) int64."""

    def __init__(self, xyz, cells):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        h = _P()
        _call("hg_mesh_create", xyz.ctypes.data_as(_P), len(xyz), cells.ctypes.data_as(_P),
              len(cells), ctypes.byref(h))
        self._h = h
        self.n_cells = len(cells)

    def counts(self):
        c = (ctypes.c_int64 * 6)()
        _call("hg_mesh_counts", self._h, c)
        return dict(zip(["vertices", "edges", "faces", "cells", "boundary_faces",
                         "interior_faces"], list(c)))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_mesh_destroy(self._h)
            self._h = None


def partition_cells(mesh: "Mesh", nparts):
    """Part (0..nparts-1) of every macro cell (hg_partition_cells; host only)."""
    part = np.empty(mesh.n_cells, dtype=np.int32)
    _call("hg_partition_cells", mesh._h, int(nparts), part.ctypes.data_as(_P))
    return part


def exchange_plan(mesh: "Mesh", level, part, rank):
    """hg_exchange_plan of `rank` on `level` (host only) as NumPy arrays."""
    part = np.ascontiguousarray(part, dtype=np.int32)
    nparts = int(part.max()) + 1 if part.size else 1
    sz = np.zeros(6, dtype=np.int64)
    args = (mesh._h, int(level), part.ctypes.data_as(_P), nparts, int(rank))
    _call("hg_exchange_plan", *args, sz.ctypes.data_as(_P), *([None] * 7))
    ns, nr, npt, nt, ntg, stride = (int(v) for v in sz)
    out = {"send_count": np.zeros(nparts, np.int64), "send_idx": np.zeros(ns, np.int64),
           "recv_count": np.zeros(nparts, np.int64), "point_start": np.zeros(npt + 1, np.int64),
           "term_src": np.zeros(nt, np.int64), "target_start": np.zeros(npt + 1, np.int64),
           "target_idx": np.zeros(ntg, np.int64)}
    _call("hg_exchange_plan", *args, sz.ctypes.data_as(_P),
          *[out[k].ctypes.data_as(_P) for k in ("send_count", "send_idx", "recv_count",
                                                 "point_start", "term_src", "target_start",
                                                 "target_idx")])
    out["stride"] = stride
    return out


class Hierarchy:
    """Levels lmin..lmax of the refined macro mesh (Sec. 3.1, Sec. 5.1)."""

    def __init__(self, mesh: Mesh, lmin: int, lmax: int):
        h = _P()
        _call("hg_hier_create", mesh._h, lmin, lmax, ctypes.byref(h))
        self._h = h
        self.mesh = mesh
        self.lmin, self.lmax = lmin, lmax
        self._n_stored = {}

    def _vec(self, level, space, dtype, *ts):
        """Check that each tensor is a contiguous CUDA tensor of `dtype` with
        at least the stored length of `level` in `space`: the kernels index
        that many elements of every vector they are given."""
        key = (level, space)
        n = self._n_stored.get(key)
        if n is None:
            n = self._n_stored[key] = self.size(level, space)[0]
        for t in ts:
            if t.dtype != dtype:
                raise TypeError(f"vector of dtype {t.dtype} where {dtype} is expected")
            _ptr(t, n)

    def size(self, level, space=HG_SPACE_P1):
        v = [ctypes.c_int64() for _ in range(4)]
        _call("hg_function_size", self._h, space, level, *[ctypes.byref(x) for x in v])
        return tuple(x.value for x in v)   # n_stored, n_unique, n_inner, cell_stride

    def canonical_info(self, level, space=HG_SPACE_P1):
        ns, nu, _, _ = self.size(level, space)
        s2c = np.empty(ns, dtype=np.int64)
        xyz = np.empty((nu, 3), dtype=np.float64)
        dirich = np.empty(nu, dtype=np.uint8)
        _call("hg_canonical_info", self._h, space, level, s2c.ctypes.data_as(_P),
              xyz.ctypes.data_as(_P), dirich.ctypes.data_as(_P))
        return s2c, xyz, dirich.astype(bool)

    def zeros(self, level, dtype, space=HG_SPACE_P1):
        import torch
        return torch.zeros(self.size(level, space)[0], dtype=dtype, device="cuda")

    def to_canonical(self, level, x, space=HG_SPACE_P1, stream=None, out=None):
        import torch
        ns, nu, _, _ = self.size(level, space)
        if out is None:
            out = torch.empty(nu, dtype=x.dtype, device=x.device)
        _call("hg_to_canonical", self._h, space, level, _dtype_code(x), _ptr(x, ns),
              _ptr(out, nu), _stream(stream))
        return out

    def from_canonical(self, level, c, out=None, space=HG_SPACE_P1, stream=None):
        import torch
        ns, nu, _, _ = self.size(level, space)
        if out is None:
            out = torch.zeros(ns, dtype=c.dtype, device=c.device)
        _call("hg_from_canonical", self._h, space, level, _dtype_code(c), _ptr(c, nu),
              _ptr(out, ns), _stream(stream))
        return out

    def interface_dump(self, level, space=HG_SPACE_P1, stream=None):
        import torch
        nr, mc = ctypes.c_int64(), ctypes.c_int64()
        _call("hg_interface_dump", self._h, space, level, None, ctypes.byref(nr),
              ctypes.byref(mc), _stream(stream))
        out = torch.full((max(nr.value, 1), 2 * mc.value + 1), -1, dtype=torch.int64,
                         device="cuda")
        _call("hg_interface_dump", self._h, space, level, _ptr(out), ctypes.byref(nr),
              ctypes.byref(mc), _stream(stream))
        return out[:nr.value]

    def restrict(self, fine_level, r_fine, r_coarse, space=HG_SPACE_P1, stream=None):
        self._vec(fine_level, space, r_fine.dtype, r_fine)
        self._vec(fine_level - 1, space, r_fine.dtype, r_coarse)
        _call("hg_restrict", self._h, space, fine_level, _dtype_code(r_fine), _ptr(r_fine),
              _ptr(r_coarse), _stream(stream))

    def prolong_add(self, fine_level, e_coarse, x_fine, space=HG_SPACE_P1, stream=None):
        self._vec(fine_level - 1, space, e_coarse.dtype, e_coarse)
        self._vec(fine_level, space, e_coarse.dtype, x_fine)
        _call("hg_prolong_add", self._h, space, fine_level, _dtype_code(e_coarse),
              _ptr(e_coarse), _ptr(x_fine), _stream(stream))

    def dot(self, level, x, y, mask=HG_MASK_INNER, space=HG_SPACE_P1, stream=None):
        r = ctypes.c_double()
        self._vec(level, space, x.dtype, x, y)
        _call("hg_dot", self._h, space, level, _dtype_code(x), _ptr(x), _ptr(y), mask,
              ctypes.byref(r), _stream(stream))
        return r.value

    def dot_noalloc(self, level, x, y, out, mask=HG_MASK_INNER, space=HG_SPACE_P1, stream=None):
        """hg_dot_noalloc: writes the dot into out[0] (CUDA float64 tensor), no sync."""
        import torch
        self._vec(level, space, x.dtype, x, y)
        if out.dtype != torch.float64:
            raise TypeError("out must be a float64 tensor")
        _ptr(out, 1)
        _call("hg_dot_noalloc", self._h, space, level, _dtype_code(x), _ptr(x), _ptr(y), mask,
              _ptr(out), _stream(stream))

    def gs_colours(self, level):
        """Gauss-Seidel colour (0..3) of every unique DoF, canonical order (host)."""
        nu = self.size(level)[1]
        out = np.zeros(nu, dtype=np.uint8)
        _call("hg_gs_colours", self._h, level, out.ctypes.data_as(_P))
        return out

    def device_status(self, stream=None):
        _call("hg_device_status", self._h, _stream(stream))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_hier_destroy(self._h)
            self._h = None


def _host_ptr(a, n):
    """Data pointer and element code of a contiguous host array (NumPy or a CPU
    torch tensor, float32/float64) of exactly n values."""
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous or a.dtype not in (np.float32, np.float64) or a.size != n:
            raise ValueError(f"expected a contiguous float32/float64 array of {n} values")
        return ctypes.c_void_p(a.ctypes.data), (HG_F64 if a.dtype == np.float64 else HG_F32)
    if a.is_cuda or not a.is_contiguous() or a.numel() != n:
        raise ValueError(f"expected a contiguous host tensor of {n} values")
    return ctypes.c_void_p(a.data_ptr()), _dtype_code(a)


class Function:
    """A finite-element function on the levels of a hierarchy (Sec. 5.1): one
    stored vector per level, bound through the C ABI (the tensors are kept
    alive here), with copies from and to host memory in canonical order."""

    def __init__(self, hier: Hierarchy, dtype, space=HG_SPACE_P1, levels=None):
        import torch
        if dtype not in (torch.float32, torch.float64):
            raise TypeError(f"a function holds float32 or float64 vectors, not {dtype}")
        h = _P()
        self.dtype = dtype
        code = HG_F64 if dtype == torch.float64 else HG_F32
        _call("hg_function_create", hier._h, space, code, ctypes.byref(h))
        self._h = h
        self.hier, self.space = hier, space
        self._t = {}
        top = hier.lmax - (1 if space == HG_SPACE_P2 else 0)
        for level in (levels if levels is not None else range(hier.lmin, top + 1)):
            self.bind(level, hier.zeros(level, dtype, space))

    def bind(self, level, t):
        ns = self.hier.size(level, self.space)[0]
        if t.dtype != self.dtype:
            raise TypeError(f"vector of dtype {t.dtype} where {self.dtype} is expected")
        _call("hg_function_bind", self._h, level, _ptr(t, ns), t.element_size() * t.numel())
        self._t[level] = t

    def __getitem__(self, level):
        return self._t[level]

    def copy_from_host(self, level, host, stream=None):
        """Host values in canonical order -> every stored copy on `level`."""
        nu = self.hier.size(level, self.space)[1]
        p, code = _host_ptr(host, nu)
        _call("hg_function_copy_canonical", self._h, level, p, code, nu, HG_COPY_FROM_HOST,
              _stream(stream))

    def copy_to_host(self, level, host, stream=None):
        """One value per unique DoF of `level` into `host` (canonical order);
        valid once `stream` has been synchronised."""
        nu = self.hier.size(level, self.space)[1]
        p, code = _host_ptr(host, nu)
        _call("hg_function_copy_canonical", self._h, level, p, code, nu, HG_COPY_TO_HOST,
              _stream(stream))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_function_destroy(self._h)
            self._h = None


class Operator:
    """A matrix-free operator (Sec. 5.2) on every level of a hierarchy."""

    def __init__(self, hier: Hierarchy, kind=HG_OP_P1_LAPLACE, coeff=None, degree=None):
        h = _P()
        carr = None
        if coeff is not None:
            carr = np.ascontiguousarray(coeff, dtype=np.float64).ravel()
            if kind in (HG_OP_P1_DIVKGRAD, HG_OP_P1_DIVKGRAD_STORED, HG_OP_P1_DIVKGRAD_SURROGATE):
                need = hier.size(hier.lmax)[1]     # k at the unique vertices of level lmax
            elif kind in (HG_OP_P2_DIVKGRAD, HG_OP_N1_CURLCURL):
                need = 2                           # {a, b} / {alpha, beta}
            else:
                need = carr.size
            if carr.size != need:
                raise ValueError(f"operator kind {kind} takes {need} coefficient values, "
                                 f"got {carr.size}")
        if kind == HG_OP_P1_DIVKGRAD_SURROGATE:
            if degree is None or carr is None:
                raise ValueError("the surrogate operator takes the coefficient k and a degree")
            _call("hg_op_create_surrogate", hier._h, carr.ctypes.data_as(_P), int(degree),
                  ctypes.byref(h))
        else:
            _call("hg_op_create", hier._h, kind,
                  carr.ctypes.data_as(_P) if carr is not None else None, ctypes.byref(h))
        self._h = h
        self.hier = hier
        self.kind = kind
        # P2 and N1 vectors live in the P2 space; their finest level is lmax - 1
        self.space = HG_SPACE_P2 if kind in (HG_OP_P2_LAPLACE, HG_OP_P2_MASS, HG_OP_P2_DIVKGRAD,
                                             HG_OP_N1_CURLCURL) else HG_SPACE_P1
        self.lmax = hier.lmax - (1 if self.space == HG_SPACE_P2 else 0)

    def apply(self, level, x, y, mode=HG_REPLACE, mask=HG_MASK_INNER, stream=None):
        self.hier._vec(level, self.space, x.dtype, x, y)
        _call("hg_apply", self._h, level, _dtype_code(x), _ptr(x), _ptr(y), mode, mask,
              _stream(stream))

    def apply_function(self, level, x: Function, y: Function, mode=HG_REPLACE,
                       mask=HG_MASK_INNER, stream=None):
        _call("hg_apply_function", self._h, level, x._h, y._h, mode, mask, _stream(stream))

    def residual(self, level, x, b, r, stream=None):
        self.hier._vec(level, self.space, x.dtype, x, b, r)
        _call("hg_residual", self._h, level, _dtype_code(x), _ptr(x), _ptr(b), _ptr(r),
              _stream(stream))

    def gauss_seidel(self, level, x, b, x_out, colour, stream=None):
        """One colour sub-sweep (out of place) of 4-colour Gauss-Seidel."""
        self.hier._vec(level, self.space, x.dtype, x, b, x_out)
        _call("hg_gauss_seidel", self._h, level, _dtype_code(x), int(colour), _ptr(x), _ptr(b),
              _ptr(x_out), _stream(stream))

    def n1_prolong_add(self, fine_level, ec, xf, stream=None):
        self.hier._vec(fine_level - 1, HG_SPACE_P2, ec.dtype, ec)
        self.hier._vec(fine_level, HG_SPACE_P2, ec.dtype, xf)
        _call("hg_n1_prolong_add", self._h, fine_level, _dtype_code(ec), _ptr(ec), _ptr(xf),
              _stream(stream))

    def n1_restrict(self, fine_level, rf, rc, stream=None):
        self.hier._vec(fine_level, HG_SPACE_P2, rf.dtype, rf)
        self.hier._vec(fine_level - 1, HG_SPACE_P2, rf.dtype, rc)
        _call("hg_n1_restrict", self._h, fine_level, _dtype_code(rf), _ptr(rf), _ptr(rc),
              _stream(stream))

    def n1_gradient(self, level, phi, u, stream=None):
        self.hier._vec(level, HG_SPACE_P1, phi.dtype, phi)
        self.hier._vec(level, HG_SPACE_P2, phi.dtype, u)
        _call("hg_n1_gradient", self._h, level, _dtype_code(phi), _ptr(phi), _ptr(u),
              _stream(stream))

    def n1_gradient_t(self, level, r, rp, stream=None):
        self.hier._vec(level, HG_SPACE_P2, r.dtype, r)
        self.hier._vec(level, HG_SPACE_P1, r.dtype, rp)
        _call("hg_n1_gradient_t", self._h, level, _dtype_code(r), _ptr(r), _ptr(rp),
              _stream(stream))

    def jacobi(self, level, x, b, x_out, omega=2.0 / 3.0, stream=None):
        self.hier._vec(level, self.space, x.dtype, x, b, x_out)
        _call("hg_jacobi", self._h, level, _dtype_code(x), float(omega), _ptr(x), _ptr(b),
              _ptr(x_out), _stream(stream))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_op_destroy(self._h)
            self._h = None


class GMG:
    """Geometric multigrid (V-cycles) for an operator on its hierarchy."""

    def __init__(self, op: Operator, nu1=3, nu2=3, omega=2.0 / 3.0, lmin=-1, inner_cycles=1,
                 smoother=HG_SMOOTH_JACOBI, cheb_order=2, cheb_iters=20, cheb_interval=(0.1, 1.1)):
        p = GmgParams()
        lib().hg_gmg_default_params(ctypes.byref(p))
        p.nu1, p.nu2, p.omega, p.lmin, p.inner_cycles = nu1, nu2, omega, lmin, inner_cycles
        p.smoother = smoother
        p.cheb_order, p.cheb_iters = cheb_order, cheb_iters
        p.cheb_lo, p.cheb_hi = cheb_interval
        h = _P()
        _call("hg_gmg_create", op._h, ctypes.byref(p), ctypes.byref(h))
        self._h = h
        self.op = op

    def vcycle(self, level, x, b, stream=None):
        self.op.hier._vec(level, self.op.space, x.dtype, x, b)
        _call("hg_vcycle", self._h, level, _dtype_code(x), _ptr(x), _ptr(b), _stream(stream))

    def fmg(self, level, x, b, cycles=5, stream=None):
        """Full multigrid to `level`: x <- FMG(b) with `cycles` V-cycles per level."""
        self.op.hier._vec(level, self.op.space, x.dtype, x, b)
        _call("hg_fmg", self._h, level, _dtype_code(x), _ptr(x), _ptr(b), cycles, _stream(stream))

    def lam(self, level):
        """lambda_max(D^-1 A) the Chebyshev smoother uses on `level`."""
        v = ctypes.c_double()
        _call("hg_gmg_lambda", self._h, level, ctypes.byref(v))
        return v.value

    def set_lam(self, level, lam):
        _call("hg_gmg_set_lambda", self._h, level, float(lam))

    def lam_potential(self, level):
        """Nedelec multigrid: lambda_max(D^-1 K) of the potential space on `level`."""
        v = ctypes.c_double()
        _call("hg_gmg_potential_lambda", self._h, level, ctypes.byref(v))
        return v.value

    def set_lam_potential(self, level, lam):
        _call("hg_gmg_set_potential_lambda", self._h, level, float(lam))

    def power_lambda(self, level, v0, iters=20, stream=None):
        """Power-iteration estimate of lambda_max(D^-1 A) from the FP64 stored vector v0."""
        import torch
        v = ctypes.c_double()
        self.op.hier._vec(level, self.op.space, torch.float64, v0)
        _call("hg_gmg_power_lambda", self._h, level, _ptr(v0), iters, ctypes.byref(v),
              _stream(stream))
        return v.value

    def solve(self, x, b, tol=1e-8, max_iter=100, precision=HG_PREC_F64, stream=None,
              check=True):
        import torch
        it = ctypes.c_int()
        rel = ctypes.c_double()
        self.op.hier._vec(self.op.lmax, self.op.space, torch.float64, x, b)
        r = lib().hg_solve(self._h, precision, _ptr(x), _ptr(b), tol, max_iter, ctypes.byref(it),
                           ctypes.byref(rel), _stream(stream))
        if r != 0 and (check or r != -5):
            raise HGError("hg_solve", r, lib().hg_last_error().decode())
        return it.value, rel.value

    def solve_function(self, x: Function, b: Function, tol=1e-8, max_iter=100,
                       precision=HG_PREC_F64, stream=None):
        it = ctypes.c_int()
        rel = ctypes.c_double()
        _call("hg_solve_function", self._h, precision, x._h, b._h, tol, max_iter,
              ctypes.byref(it), ctypes.byref(rel), _stream(stream))
        return it.value, rel.value

    def set_learned(self, mlp=None):
        _call("hg_gmg_set_learned", self._h, mlp._h if mlp is not None else None)
        self.mlp = mlp

    def learned_fallbacks(self):
        n = ctypes.c_int()
        _call("hg_gmg_learned_fallbacks", self._h, ctypes.byref(n))
        return n.value

    def history(self):
        n = ctypes.c_int()
        _call("hg_gmg_history", self._h, None, 0, ctypes.byref(n))
        out = (ctypes.c_double * max(n.value, 1))()
        _call("hg_gmg_history", self._h, out, n.value, ctypes.byref(n))
        return list(out)[:n.value]

    def clone(self):
        """A GMG for the same operator/parameters with its own work vectors."""
        h = _P()
        _call("hg_gmg_clone", self._h, ctypes.byref(h))
        g = GMG.__new__(GMG)
        g._h = h
        g.op = self.op
        return g

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_gmg_destroy(self._h)
            self._h = None


class Batch:
    """Many independent GMG problems solved together by persistent stage
    launches (optionally replayed as CUDA graphs, with autotuned variants).
    ``problems``: distinct GMG objects; ``x``/``b``: FP64 finest-level stored
    vectors, one per problem, kept alive by the batch."""

    def __init__(self, problems, x, b, graph=True, autotune=True):
        import torch
        n = len(problems)
        if not (n == len(x) == len(b)) or n == 0:
            raise ValueError("problems, x and b need the same nonzero length")
        for v in list(x) + list(b):
            if v.dtype != torch.float64 or not v.is_cuda or not v.is_contiguous():
                raise ValueError("x and b must be contiguous FP64 CUDA tensors")
        hs = (_P * n)(*[g._h.value for g in problems])
        xs = (_P * n)(*[v.data_ptr() for v in x])
        bs = (_P * n)(*[v.data_ptr() for v in b])
        flags = (HG_BATCH_GRAPH if graph else 0) | (HG_BATCH_AUTOTUNE if autotune else 0)
        h = _P()
        _call("hg_batch_create", hs, n, xs, bs, flags, ctypes.byref(h))
        self._h = h
        self._keep = (list(problems), list(x), list(b))
        self.count = n

    def solve(self, tol=1e-8, max_iter=100, stream=None, check=True):
        """Returns (iters, rel_res) as numpy arrays (per problem)."""
        it = np.zeros(self.count, dtype=np.int32)
        rel = np.zeros(self.count, dtype=np.float64)
        r = lib().hg_batch_solve(self._h, tol, max_iter, it.ctypes.data_as(_P),
                                 rel.ctypes.data_as(_P), _stream(stream))
        if r != 0 and (check or r != -5):
            raise HGError("hg_batch_solve", r, lib().hg_last_error().decode())
        return it, rel

    def tuning(self):
        rows, gf, us = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        _call("hg_batch_tuning", self._h, ctypes.byref(rows), ctypes.byref(gf), ctypes.byref(us))
        return rows.value, gf.value, us.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_batch_destroy(self._h)
            self._h = None


N_MLP_PARAMS = 512 + 1024 + 32


def _samples(X, dtype, t=None):
    """n rows of 16 features of `dtype` (contiguous CUDA) and, if given, n FP32
    targets: the network kernels read 16 n features and n targets."""
    import torch
    if X.dtype != dtype or X.dim() != 2 or X.shape[1] != 16:
        raise ValueError(f"samples must be [n, 16] of {dtype}, got {tuple(X.shape)} {X.dtype}")
    _ptr(X)
    if t is not None:
        if t.dtype != torch.float32:
            raise TypeError("targets must be float32")
        _ptr(t, X.shape[0])


class MLP:
    """The learned local smoother network (BF16 tensor-core kernels)."""

    def __init__(self, params=None):
        h = _P()
        _call("hg_mlp_create", ctypes.byref(h))
        self._h = h
        if params is not None:
            self.set_params(params)

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if p.size != N_MLP_PARAMS:
            raise ValueError(f"need {N_MLP_PARAMS} parameters")
        _call("hg_mlp_set_params", self._h, p.ctypes.data_as(_P))

    def params(self):
        p = np.empty(N_MLP_PARAMS, dtype=np.float32)
        _call("hg_mlp_get_params", self._h, p.ctypes.data_as(_P))
        return p

    def forward(self, X, out=None, stream=None):
        import torch
        _samples(X, torch.float32)
        if out is None:
            out = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        if out.dtype != torch.float32:
            raise TypeError("out must be float32")
        _ptr(out, X.shape[0])
        _call("hg_mlp_forward", self._h, _ptr(X), X.shape[0], _ptr(out), _stream(stream))
        return out

    def grad(self, X, t, stream=None):
        import torch
        _samples(X, torch.bfloat16, t)
        g = np.empty(N_MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _call("hg_mlp_grad", self._h, _ptr(X), _ptr(t), X.shape[0], g.ctypes.data_as(_P),
              ctypes.byref(loss), _stream(stream))
        return loss.value, g

    def train(self, X, t, steps, batch, lr, stream=None):
        import torch
        _samples(X, torch.bfloat16, t)
        loss = ctypes.c_double()
        _call("hg_mlp_train", self._h, _ptr(X), _ptr(t), X.shape[0], steps, batch, lr,
              ctypes.byref(loss), _stream(stream))
        return loss.value

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.hg_mlp_destroy(self._h)
            self._h = None


def learned_step(op, mlp, level, x, r, x_out, omega, stream=None):
    """One learned smoothing step x_out = x + omega s + N(s) (hg_learned_step)."""
    import torch
    op.hier._vec(level, op.space, torch.float32, x, r, x_out)
    _call("hg_learned_step", op._h, mlp._h, level, _ptr(x), _ptr(r), omega, _ptr(x_out),
          _stream(stream))


def learn_samples(op, level, r, xstar, x, omega, stride, offset, stream=None):
    """Training pairs (X bf16 [count,16], t float32 [count]) from one state."""
    import torch
    op.hier._vec(level, op.space, torch.float32, r, xstar, x)
    cnt = ctypes.c_int64()
    _call("hg_learn_samples", op._h, level, None, None, None, omega, stride, offset, None, None,
          ctypes.byref(cnt), _stream(stream))
    X = torch.empty((cnt.value, 16), dtype=torch.bfloat16, device="cuda")
    t = torch.empty(cnt.value, dtype=torch.float32, device="cuda")
    _call("hg_learn_samples", op._h, level, _ptr(r), _ptr(xstar), _ptr(x), omega, stride, offset,
          _ptr(X), _ptr(t), ctypes.byref(cnt), _stream(stream))
    return X, t


def n1_prolong_table():
    """The library's Nedelec prolongation class table (host): dict of numpy
    arrays n (64,), off, dir, w (64, 6), fine_dir (64,)."""
    n = np.zeros(64, dtype=np.int32)
    off = np.zeros((64, 6), dtype=np.int32)
    dr = np.zeros((64, 6), dtype=np.int32)
    w = np.zeros((64, 6), dtype=np.float64)
    fd = np.zeros(64, dtype=np.int32)
    _call("hg_n1_prolong_table", n.ctypes.data_as(_P), off.ctypes.data_as(_P),
          dr.ctypes.data_as(_P), w.ctypes.data_as(_P), fd.ctypes.data_as(_P))
    return {"n": n, "off": off, "dir": dr, "w": w, "fine_dir": fd}


def plane_tiles(level):
    """The apply kernels' plane-window tiles of one cell lattice (host): (n, 4) int32."""
    n = ctypes.c_int()
    _call("hg_plane_tiles", level, None, ctypes.byref(n))
    out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    _call("hg_plane_tiles", level, out.ctypes.data_as(_P), ctypes.byref(n))
    return out[:n.value]


def march_items(level):
    """The column-march kernel's items of one cell lattice (host): (n, 2) int32."""
    n = ctypes.c_int()
    _call("hg_march_items", level, None, ctypes.byref(n))
    out = np.zeros((max(n.value, 1), 2), dtype=np.int32)
    _call("hg_march_items", level, out.ctypes.data_as(_P), ctypes.byref(n))
    return out[:n.value]


HG_P1_KERNEL_AUTO, HG_P1_KERNEL_WINDOWS, HG_P1_KERNEL_STREAM, HG_P1_KERNEL_MARCH = 0, 1, 2, 3


def set_p1_kernel(mode):
    """Kernel of the P1 constant-stencil operators for later calls (HG_P1_KERNEL_*)."""
    _call("hg_set_p1_kernel", mode)


def stream_plan(level, ncells, nctas, dtype_code):
    """Plan of the streaming apply kernel (host): dict of copies (n, 4), items
    (m, 12), cta_copies and cta_items (nctas + 1,), band_rows."""
    cnt = np.zeros(3, dtype=np.int32)
    _call("hg_stream_plan", level, ncells, nctas, dtype_code, None, None, None, None,
          cnt.ctypes.data_as(_P))
    copies = np.zeros((max(cnt[0], 1), 4), dtype=np.int32)
    items = np.zeros((max(cnt[1], 1), 12), dtype=np.int32)
    cc = np.zeros(nctas + 1, dtype=np.int32)
    ci = np.zeros(nctas + 1, dtype=np.int32)
    _call("hg_stream_plan", level, ncells, nctas, dtype_code, copies.ctypes.data_as(_P),
          items.ctypes.data_as(_P), cc.ctypes.data_as(_P), ci.ctypes.data_as(_P),
          cnt.ctypes.data_as(_P))
    return {"copies": copies[:cnt[0]], "items": items[:cnt[1]], "cta_copies": cc,
            "cta_items": ci, "band_rows": int(cnt[2])}


def stream_layout(level, dtype_code):
    """Shared-memory layout of the streaming kernel (host): (ring slots, slot elements, guard)."""
    r, s, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _call("hg_stream_layout", level, dtype_code, ctypes.byref(r), ctypes.byref(s), ctypes.byref(g))
    return r.value, s.value, g.value


def p2_anchors(level):
    """Anchors of the P2/N1 colour phases (host): (anchors (n, 3) int, colour offsets (9,))."""
    n = ctypes.c_int()
    off = np.zeros(9, dtype=np.int32)
    _call("hg_p2_anchors", level, None, off.ctypes.data_as(_P), ctypes.byref(n))
    a = np.zeros(max(n.value, 1), dtype=np.uint32)
    _call("hg_p2_anchors", level, a.ctypes.data_as(_P), off.ctypes.data_as(_P), ctypes.byref(n))
    a = a[:n.value].astype(np.int64)
    return np.stack([a & 1023, (a >> 10) & 1023, a >> 20], axis=1), off


def n1_restrict_table():
    """The transposed (restriction) lists of the Nedelec prolongation table
    (host): dict with start (9,), d, w, fine_dir (start[8],)."""
    start = np.zeros(9, dtype=np.int32)
    _call("hg_n1_restrict_table", start.ctypes.data_as(_P), None, None, None)
    m = int(start[8])
    d = np.zeros(max(m, 1), dtype=np.int32)
    w = np.zeros(max(m, 1), dtype=np.float64)
    fd = np.zeros(max(m, 1), dtype=np.int32)
    _call("hg_n1_restrict_table", start.ctypes.data_as(_P), d.ctypes.data_as(_P),
          w.ctypes.data_as(_P), fd.ctypes.data_as(_P))
    return {"start": start, "d": d[:m], "w": w[:m], "fine_dir": fd[:m]}


def quadrature_rule():
    """(bary (14,4), weights (14,)) of the library's P2 quadrature rule (host)."""
    b = np.zeros((14, 4))
    w = np.zeros(14)
    n = ctypes.c_int()
    _call("hg_quadrature_rule", b.ctypes.data_as(_P), w.ctypes.data_as(_P), ctypes.byref(n))
    return b[:n.value], w[:n.value]


def index_tw(w, i, j, k):
    out = ctypes.c_int64()
    _call("hg_index_tw", w, i, j, k, ctypes.byref(out))
    return out.value


def index_enumerate(w, out, stream=None):
    _call("hg_index_enumerate", w, _ptr(out), _stream(stream))
