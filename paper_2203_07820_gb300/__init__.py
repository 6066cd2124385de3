"""Python binding of libdftfe_gb300 (argument marshalling only).

Every function has the name of the C entry point it calls (include/dftfe_gb300.h);
all computation runs in the library's CUDA kernels.  Device arrays are torch
tensors (FP64, CUDA, row-major with unit column stride; a column slice of a wider
block is fine and its row stride is passed as the leading dimension).  Host arrays
are numpy.  A non-zero status raises DftfeError with the library's message.

The library must have been built (``__graft_entry__.build()`` or
``python -m paper_2203_07820_gb300._build``); importing without it raises.

One pass at the Gamma point (FP64 or a split precision)::

    mesh = dftfe_mesh_create(L, ncell, degree)
    ham = dftfe_ham_create(mesh)
    dftfe_ham_set_potential(ham, v_quad)                # CUDA float64, ncells x quad_per_cell
    dftfe_ham_set_nonlocal(ham, h, rowptr, node, chi)   # optional projectors (host CSR)
    X = torch.empty((M, N), dtype=torch.float64, device="cuda"); dftfe_random_uniform(X, seed)
    b = dftfe_spectrum_bounds(ham, 20, seed, N)
    dftfe_chfsi_pass(ham, X, block, degree, b, evals, resid, DFTFE_MIXED_TF32X3)

At a Bloch k-point the block is complex128 and the calls end in ``_z``::

    dftfe_ham_set_kpoint(ham, k, disp)                  # disp: projector displacements
    Z = torch.empty((M, N), dtype=torch.complex128, device="cuda")
    dftfe_chfsi_pass_z(ham, Z, block, degree, dftfe_spectrum_bounds_z(ham, 20, seed, N), evals, resid)

Many systems (each its own ham, Gamma or k-point items) in one batched pass::

    batch = dftfe_batch_create(hams)
    dftfe_batch_chfsi_pass(batch, blocks_X, blocks, degrees, bounds, evals, resids)
"""
import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdftfe_gb300.so")

DFTFE_FP64 = 0
DFTFE_MIXED_BF16X3 = 1
DFTFE_MIXED_TF32X3 = 2
DFTFE_FP64_FLOAT_PAIRS = 3
DFTFE_FP64_SLICES = 4

DFTFE_OK, DFTFE_ERR_ARG, DFTFE_ERR_OOM, DFTFE_ERR_CUDA = 0, 1, 2, 3
DFTFE_ERR_NOT_SPD, DFTFE_ERR_NOCONV, DFTFE_ERR_TIMEOUT, DFTFE_ERR_STATE = 4, 5, 6, 7

STATUS = {0: "DFTFE_OK", 1: "DFTFE_ERR_ARG", 2: "DFTFE_ERR_OOM", 3: "DFTFE_ERR_CUDA",
          4: "DFTFE_ERR_NOT_SPD", 5: "DFTFE_ERR_NOCONV", 6: "DFTFE_ERR_TIMEOUT",
          7: "DFTFE_ERR_STATE"}


class DftfeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("ncell", C.c_int * 3), ("degree", C.c_int),
                ("periodic", C.c_int * 3), ("vquad", C.c_int), ("nq1d", C.c_int)]


class Bounds(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("a0", C.c_double)]

    def __repr__(self):
        return f"Bounds(a={self.a!r}, b={self.b!r}, a0={self.a0!r})"


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                      "(there is no CPU fallback)")
_lib = C.CDLL(LIB_PATH)

_vp, _i64, _int, _dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
_SIGS = {
    "dftfe_mesh_create": [C.POINTER(MeshDesc), C.POINTER(_vp)],
    "dftfe_mesh_info": [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_int), C.POINTER(_int)],
    "dftfe_mesh_coords": [_vp, _vp, _vp],
    "dftfe_mesh_destroy": [_vp],
    "dftfe_ham_create": [_vp, _vp, C.POINTER(_vp)],
    "dftfe_ham_create_shared": [_vp, C.POINTER(_vp)],
    "dftfe_ham_set_potential": [_vp, _vp],
    "dftfe_ham_set_nonlocal": [_vp, _int, _vp, _vp, _vp, _vp],
    "dftfe_ham_destroy": [_vp],
    "dftfe_ham_export": [_vp, _vp, _vp, _i64, _i64, _vp],
    "dftfe_ham_apply": [_vp, _vp, _i64, _vp, _i64, _int, _int],
    "dftfe_random_uniform": [_vp, _i64, C.c_uint64, _i64, _vp],
    "dftfe_lanczos": [_vp, _int, _vp, C.c_uint64, _vp],
    "dftfe_spectrum_bounds": [_vp, _int, C.c_uint64, _int, C.POINTER(Bounds)],
    "dftfe_chebyshev_filter": [_vp, _vp, _i64, _int, _int, C.POINTER(Bounds), _int],
    "dftfe_cholgs": [_vp, _vp, _i64, _int, _int],
    "dftfe_rayleigh_ritz": [_vp, _vp, _i64, _int, _vp, _vp, _i64, _int],
    "dftfe_residuals": [_vp, _vp, _vp, _i64, _int, _vp, _vp, _int],
    "dftfe_chfsi_pass": [_vp, _vp, _i64, _int, _int, _int, C.POINTER(Bounds), _vp, _vp, _int],
    "dftfe_cholgs_noalloc": [_vp, _i64, _i64, _int, _vp],
    "dftfe_rayleigh_ritz_split": [_vp, _vp, _i64, _int, _int, _vp, _vp, _i64, _int],
    "dftfe_fermi_level": [_vp, _int, _int, _dbl, _dbl, _vp, C.POINTER(_dbl), _vp],
    "dftfe_density": [_vp, _vp, _i64, _int, _vp, _i64, _int, _vp, _vp],
    "dftfe_batch_create": [C.POINTER(_vp), _int, C.POINTER(_vp)],
    "dftfe_batch_chfsi_pass": [_vp, _vp, _int],
    "dftfe_batch_destroy": [_vp],
    "dftfe_batch_use_graphs": [_vp, _int],
    "dftfe_batch_graph_query": [_vp, C.POINTER(_i64), C.POINTER(_i64)],
    "dftfe_mlp_forward": [_vp, _int, _int, _int, _vp, _i64, _vp, _vp],
    "dftfe_mlp_loss_grad": [_vp, _int, _int, _int, _vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "dftfe_mlp_adam": [_vp, _vp, _vp, _vp, _i64, _int, C.c_float, C.c_float, C.c_float, C.c_float, _vp],
    "dftfe_ham_use_graphs": [_vp, _int],
    "dftfe_graph_query": [_vp, C.POINTER(_i64), C.POINTER(_i64)],
    "dftfe_ham_autotune": [_vp, _int],
    "dftfe_autotune_query": [_vp, _int, C.POINTER(_int), C.POINTER(_dbl), C.POINTER(_dbl)],
    "dftfe_autotune_query_mixed": [_vp, C.POINTER(_int), C.POINTER(_int), C.POINTER(_int), C.POINTER(_dbl),
                                   C.POINTER(_dbl)],
    "dftfe_batch_autotune": [_vp, _int],
    "dftfe_batch_autotune_query": [_vp, _int, C.POINTER(_int), C.POINTER(_int), C.POINTER(_int), C.POINTER(_int),
                                   C.POINTER(_int), C.POINTER(_int), C.POINTER(_dbl), C.POINTER(_dbl)],
    "dftfe_ham_set_kpoint": [_vp, _vp, _vp],
    "dftfe_mesh_kpoint_stencil": [_vp, _vp, _vp],
    "dftfe_ham_apply_z": [_vp, _vp, _i64, _vp, _i64, _int, _int],
    "dftfe_lanczos_z": [_vp, _int, _vp, C.c_uint64, _vp],
    "dftfe_spectrum_bounds_z": [_vp, _int, C.c_uint64, _int, C.POINTER(Bounds)],
    "dftfe_chebyshev_filter_z": [_vp, _vp, _i64, _int, _int, C.POINTER(Bounds), _int],
    "dftfe_cholgs_z": [_vp, _vp, _i64, _int, _int],
    "dftfe_rayleigh_ritz_z": [_vp, _vp, _i64, _int, _vp, _vp, _i64, _int],
    "dftfe_residuals_z": [_vp, _vp, _vp, _i64, _int, _vp, _vp, _int],
    "dftfe_chfsi_pass_z": [_vp, _vp, _i64, _int, _int, _int, C.POINTER(Bounds), _vp, _vp, _int],
    "dftfe_ham_set_wait_test": [_vp, _i64, _int],
    "dftfe_profile_enable": [_vp, _int],
    "dftfe_profile_query": [_vp, C.c_char_p, C.POINTER(_dbl), C.POINTER(_i64)],
}
for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.dftfe_mlp_param_count.argtypes = [_int, _int, _int]
_lib.dftfe_mlp_param_count.restype = C.c_int64
_lib.dftfe_launch_count.argtypes = []
_lib.dftfe_launch_count.restype = C.c_int64
_lib.dftfe_last_error.argtypes = []
_lib.dftfe_last_error.restype = C.c_char_p


def _check(rc):
    if rc != 0:
        raise DftfeError(rc, _lib.dftfe_last_error().decode())


def _dev(t, name="array"):
    """Pointer and leading dimension of a CUDA FP64 tensor with unit column stride."""
    if t is None:
        return None, 0
    if not t.is_cuda or t.dtype.itemsize != 8 or not t.dtype.is_floating_point:
        raise TypeError(f"{name} must be a CUDA float64 tensor")
    if t.dim() == 1:
        return _vp(t.data_ptr()), 1
    if t.dim() != 2 or (t.stride(1) != 1 and t.shape[1] > 1):
        raise ValueError(f"{name} must be 2-D with unit column stride")
    return _vp(t.data_ptr()), t.stride(0)


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(_vp)


def _stream(stream):
    if stream is None:
        import torch
        return _vp(torch.cuda.current_stream().cuda_stream)
    return _vp(int(stream))


def lib():
    """The loaded ctypes library (for tests that call the ABI directly)."""
    return _lib


# ------------------------------------------------------------------ mesh
def dftfe_mesh_create(L, ncell, degree, vquad=0, nq1d=0):
    L = np.broadcast_to(np.asarray(L, np.float64), (3,))
    n = np.broadcast_to(np.asarray(ncell, np.int64), (3,))
    d = MeshDesc((C.c_double * 3)(*L), (C.c_int * 3)(*[int(x) for x in n]), int(degree),
                 (C.c_int * 3)(1, 1, 1), int(vquad), int(nq1d))
    out = _vp()
    _check(_lib.dftfe_mesh_create(C.byref(d), C.byref(out)))
    return out


def dftfe_mesh_info(mesh):
    nd, ncl, npc, nqp = _i64(), _i64(), _int(), _int()
    _check(_lib.dftfe_mesh_info(mesh, C.byref(nd), C.byref(ncl), C.byref(npc), C.byref(nqp)))
    return nd.value, ncl.value, npc.value, nqp.value


def dftfe_mesh_coords(mesh, nodes=True, quad=True):
    nd, ncl, npc, nqp = dftfe_mesh_info(mesh)
    node_xyz = np.empty((nd, 3)) if nodes else None
    quad_xyz = np.empty((ncl, nqp, 3)) if quad else None
    _check(_lib.dftfe_mesh_coords(mesh, None if node_xyz is None else node_xyz.ctypes.data_as(_vp),
                                  None if quad_xyz is None else quad_xyz.ctypes.data_as(_vp)))
    return node_xyz, quad_xyz


def dftfe_mesh_destroy(mesh):
    _check(_lib.dftfe_mesh_destroy(mesh))


# ------------------------------------------------------------ Hamiltonian
def dftfe_ham_create(mesh, stream=None):
    out = _vp()
    _check(_lib.dftfe_ham_create(mesh, _stream(stream), C.byref(out)))
    return out


def dftfe_ham_create_shared(src):
    out = _vp()
    _check(_lib.dftfe_ham_create_shared(src, C.byref(out)))
    return out


def dftfe_ham_set_potential(ham, v_quad):
    p, _ = _dev(v_quad.reshape(-1), "v_quad")
    _check(_lib.dftfe_ham_set_potential(ham, p))


def dftfe_ham_set_nonlocal(ham, h, rowptr, node, chi):
    h, ph = _host(h, np.float64)
    rowptr, pr = _host(rowptr, np.int64)
    node, pn = _host(node, np.int64)
    chi, pc = _host(chi, np.float64)
    _check(_lib.dftfe_ham_set_nonlocal(ham, int(h.size), ph, pr, pn, pc))


def dftfe_ham_destroy(ham):
    _check(_lib.dftfe_ham_destroy(ham))


def dftfe_ham_export(ham, mass=None, cell_map=None, c0=0, cell_mats=None):
    pm = None if mass is None else _vp(mass.data_ptr())
    pc = None if cell_map is None else _vp(cell_map.data_ptr())
    count = 0 if cell_mats is None else cell_mats.shape[0]
    pmat = None if cell_mats is None else _vp(cell_mats.data_ptr())
    _check(_lib.dftfe_ham_export(ham, pm, pc, int(c0), int(count), pmat))


def dftfe_ham_apply(ham, X, Y, prec=DFTFE_FP64):
    px, ldx = _dev(X, "X")
    py, ldy = _dev(Y, "Y")
    ncol = 1 if X.dim() == 1 else X.shape[1]
    _check(_lib.dftfe_ham_apply(ham, px, ldx, py, ldy, ncol, prec))


def dftfe_ham_use_graphs(ham, enable=True):
    _check(_lib.dftfe_ham_use_graphs(ham, 1 if enable else 0))


def dftfe_graph_query(ham):
    """(graph launches, instantiations) since graphs were switched on."""
    r, n = _i64(), _i64()
    _check(_lib.dftfe_graph_query(ham, C.byref(r), C.byref(n)))
    return r.value, n.value


def dftfe_ham_autotune(ham, enable=True):
    _check(_lib.dftfe_ham_autotune(ham, 1 if enable else 0))


def dftfe_autotune_query(ham, ncol):
    """(rows_per_cta, best_ms, heuristic_ms) for ncol real columns; rows_per_cta -1 = not tuned."""
    r, b, hm = _int(), _dbl(), _dbl()
    _check(_lib.dftfe_autotune_query(ham, int(ncol), C.byref(r), C.byref(b), C.byref(hm)))
    return r.value, b.value, hm.value


def dftfe_autotune_query_mixed(ham):
    """(atmem, deep, deal, best_ms, default_ms) of the tuned TF32x3 cell-kernel shape; -1 = not tuned."""
    a, dp, d, b, dm = _int(), _int(), _int(), _dbl(), _dbl()
    _check(_lib.dftfe_autotune_query_mixed(ham, C.byref(a), C.byref(dp), C.byref(d), C.byref(b), C.byref(dm)))
    return a.value, dp.value, d.value, b.value, dm.value


# ------------------------------------------------------------ ChFSI steps
def dftfe_random_uniform(out, seed, offset=0, stream=None):
    _check(_lib.dftfe_random_uniform(_vp(out.data_ptr()), out.numel(), C.c_uint64(seed), int(offset),
                                     _stream(stream)))


def dftfe_lanczos(ham, k, v0=None, seed=0):
    out = (C.c_double * 3)()
    pv = None if v0 is None else _vp(v0.data_ptr())
    _check(_lib.dftfe_lanczos(ham, int(k), pv, C.c_uint64(seed), C.cast(out, _vp)))
    return out[0], out[1], out[2]


def dftfe_spectrum_bounds(ham, k, seed, nstates):
    b = Bounds()
    _check(_lib.dftfe_spectrum_bounds(ham, int(k), C.c_uint64(seed), int(nstates), C.byref(b)))
    return b


def make_bounds(a, b, a0=math.nan):
    return Bounds(float(a), float(b), float(a0))


def dftfe_chebyshev_filter(ham, X, degree, bounds, prec=DFTFE_FP64):
    px, ld = _dev(X, "X")
    _check(_lib.dftfe_chebyshev_filter(ham, px, ld, X.shape[1], int(degree), C.byref(bounds), prec))


def dftfe_cholgs(ham, X, prec=DFTFE_FP64):
    px, ld = _dev(X, "X")
    _check(_lib.dftfe_cholgs(ham, px, ld, X.shape[1], prec))


def dftfe_rayleigh_ritz(ham, X, evals, HX=None, prec=DFTFE_FP64):
    px, ld = _dev(X, "X")
    ph, ldh = _dev(HX, "HX")
    _check(_lib.dftfe_rayleigh_ritz(ham, px, ld, X.shape[1], _vp(evals.data_ptr()), ph, ldh, prec))


def dftfe_residuals(ham, X, HX, evals, resid, kind=0):
    px, ld = _dev(X, "X")
    ph, ldh = _dev(HX, "HX")
    if ldh != ld:
        raise ValueError("X and HX must share the leading dimension")
    _check(_lib.dftfe_residuals(ham, px, ph, ld, X.shape[1], _vp(evals.data_ptr()),
                                _vp(resid.data_ptr()), int(kind)))


def dftfe_chfsi_pass(ham, X, block, degree, bounds, evals, resid, prec=DFTFE_FP64):
    px, ld = _dev(X, "X")
    _check(_lib.dftfe_chfsi_pass(ham, px, ld, X.shape[1], int(block), int(degree), C.byref(bounds),
                                 _vp(evals.data_ptr()), _vp(resid.data_ptr()), prec))
    return bounds


def dftfe_rayleigh_ritz_split(ham, X, nfr, evals, Xfr, prec=DFTFE_FP64):
    px, ld = _dev(X, "X")
    pf, ldf = _dev(Xfr, "Xfr")
    _check(_lib.dftfe_rayleigh_ritz_split(ham, px, ld, X.shape[1], int(nfr), _vp(evals.data_ptr()), pf, ldf, prec))


# ------------------------------------------------------------ Bloch k-points
def _zdev(t, name="array"):
    """Pointer and leading dimension (complex elements) of a CUDA complex128 tensor with unit
    column stride."""
    if t is None:
        return None, 0
    import torch
    if not t.is_cuda or t.dtype != torch.complex128:
        raise TypeError(f"{name} must be a CUDA complex128 tensor")
    if t.dim() == 1:
        return _vp(t.data_ptr()), 1
    if t.dim() != 2 or (t.stride(1) != 1 and t.shape[1] > 1):
        raise ValueError(f"{name} must be 2-D with unit column stride")
    return _vp(t.data_ptr()), t.stride(0)


def dftfe_ham_set_kpoint(ham, k, disp=None):
    """k: 3 floats (bohr^-1); disp: host nnz x 3 displacements of the projector CSR entries."""
    kk, pk = _host(np.asarray(k, np.float64).reshape(3), np.float64)
    if disp is None:
        _check(_lib.dftfe_ham_set_kpoint(ham, pk, None))
    else:
        dd, pd = _host(np.asarray(disp, np.float64).reshape(-1, 3), np.float64)
        _check(_lib.dftfe_ham_set_kpoint(ham, pk, pd))


def dftfe_mesh_kpoint_stencil(mesh, k, degree):
    """Host table of the k.grad stencil, shape (3, p, 2p + 1)."""
    kk, pk = _host(np.asarray(k, np.float64).reshape(3), np.float64)
    out = np.zeros((3, degree, 2 * degree + 1))
    _check(_lib.dftfe_mesh_kpoint_stencil(mesh, pk, out.ctypes.data_as(_vp)))
    return out


def dftfe_ham_apply_z(ham, X, Y, prec=DFTFE_FP64):
    px, ldx = _zdev(X, "X")
    py, ldy = _zdev(Y, "Y")
    ncol = 1 if X.dim() == 1 else X.shape[1]
    _check(_lib.dftfe_ham_apply_z(ham, px, ldx, py, ldy, ncol, prec))


def dftfe_lanczos_z(ham, k, v0=None, seed=0):
    out = (C.c_double * 3)()
    pv = None if v0 is None else _vp(v0.data_ptr())
    _check(_lib.dftfe_lanczos_z(ham, int(k), pv, C.c_uint64(seed), C.cast(out, _vp)))
    return out[0], out[1], out[2]


def dftfe_spectrum_bounds_z(ham, k, seed, nstates):
    b = Bounds()
    _check(_lib.dftfe_spectrum_bounds_z(ham, int(k), C.c_uint64(seed), int(nstates), C.byref(b)))
    return b


def dftfe_chebyshev_filter_z(ham, X, degree, bounds, prec=DFTFE_FP64):
    px, ld = _zdev(X, "X")
    _check(_lib.dftfe_chebyshev_filter_z(ham, px, ld, X.shape[1], int(degree), C.byref(bounds), prec))


def dftfe_cholgs_z(ham, X, prec=DFTFE_FP64):
    px, ld = _zdev(X, "X")
    _check(_lib.dftfe_cholgs_z(ham, px, ld, X.shape[1], prec))


def dftfe_rayleigh_ritz_z(ham, X, evals, HX=None, prec=DFTFE_FP64):
    px, ld = _zdev(X, "X")
    ph, ldh = _zdev(HX, "HX")
    _check(_lib.dftfe_rayleigh_ritz_z(ham, px, ld, X.shape[1], _vp(evals.data_ptr()), ph, ldh, prec))


def dftfe_residuals_z(ham, X, HX, evals, resid, kind=0):
    px, ld = _zdev(X, "X")
    ph, ldh = _zdev(HX, "HX")
    if ldh != ld:
        raise ValueError("X and HX must share the leading dimension")
    _check(_lib.dftfe_residuals_z(ham, px, ph, ld, X.shape[1], _vp(evals.data_ptr()), _vp(resid.data_ptr()),
                                  int(kind)))


def dftfe_chfsi_pass_z(ham, X, block, degree, bounds, evals, resid, prec=DFTFE_FP64):
    px, ld = _zdev(X, "X")
    _check(_lib.dftfe_chfsi_pass_z(ham, px, ld, X.shape[1], int(block), int(degree), C.byref(bounds),
                                   _vp(evals.data_ptr()), _vp(resid.data_ptr()), prec))
    return bounds


class BatchItem(C.Structure):
    _fields_ = [("X", _vp), ("ld", _i64), ("ncol", _int), ("block", _int), ("degree", _int),
                ("bounds", Bounds), ("evals", _vp), ("resid", _vp), ("kpoint", _int)]


def dftfe_batch_create(hams):
    arr = (_vp * len(hams))(*hams)
    out = _vp()
    _check(_lib.dftfe_batch_create(arr, len(hams), C.byref(out)))
    return out


def dftfe_batch_destroy(batch):
    _check(_lib.dftfe_batch_destroy(batch))


def dftfe_batch_use_graphs(batch, enable=True):
    _check(_lib.dftfe_batch_use_graphs(batch, 1 if enable else 0))


def dftfe_batch_graph_query(batch):
    r, n = _i64(), _i64()
    _check(_lib.dftfe_batch_graph_query(batch, C.byref(r), C.byref(n)))
    return r.value, n.value


def dftfe_batch_autotune(batch, enable=True):
    _check(_lib.dftfe_batch_autotune(batch, 1 if enable else 0))


def dftfe_batch_autotune_query(batch):
    """Every tuned launch of the batch: a list of dicts (nodes_per_cell, work_items, atmem,
    deep, deal, order, best_ms, default_ms)."""
    out = []
    while True:
        v = [_int() for _ in range(6)]
        b, dm = _dbl(), _dbl()
        _check(_lib.dftfe_batch_autotune_query(batch, len(out), *[C.byref(x) for x in v], C.byref(b), C.byref(dm)))
        if v[0].value < 0:
            return out
        out.append(dict(nodes_per_cell=v[0].value, work_items=v[1].value, atmem=v[2].value, deep=v[3].value,
                        deal=v[4].value, order=v[5].value, best_ms=b.value, default_ms=dm.value))


def dftfe_batch_chfsi_pass(batch, Xs, blocks, degrees, bounds, evals, resids, prec=DFTFE_FP64):
    """One pass for every system of the batch; `bounds` (list of Bounds) are updated in place.
    A complex128 block is filtered at its ham's k-point (dftfe_ham_set_kpoint)."""
    n = len(Xs)
    items = (BatchItem * n)()
    for i in range(n):
        cplx = Xs[i].is_complex()
        px, ld = _zdev(Xs[i], "X") if cplx else _dev(Xs[i], "X")
        items[i] = BatchItem(px, ld, Xs[i].shape[1], int(blocks[i]), int(degrees[i]), bounds[i],
                             _vp(evals[i].data_ptr()), _vp(resids[i].data_ptr()), 1 if cplx else 0)
    _check(_lib.dftfe_batch_chfsi_pass(batch, C.cast(items, _vp), prec))
    for i in range(n):
        bounds[i].a, bounds[i].b, bounds[i].a0 = items[i].bounds.a, items[i].bounds.b, items[i].bounds.a0
    return bounds


def _f32(t, name):
    if t is None:
        return None
    if not t.is_cuda or t.dtype.itemsize != 4 or not t.dtype.is_floating_point or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor")
    return _vp(t.data_ptr())


def dftfe_mlp_param_count(n_in, n_hidden, n_out):
    return int(_lib.dftfe_mlp_param_count(int(n_in), int(n_hidden), int(n_out)))


def dftfe_mlp_forward(params, shape, X, Y, stream=None):
    n_in, n_h, n_out = shape
    _check(_lib.dftfe_mlp_forward(_f32(params, "params"), n_in, n_h, n_out, _f32(X, "X"), X.shape[0],
                                  _f32(Y, "Y"), _stream(stream)))


def dftfe_mlp_loss_grad(params, shape, X, T, w, loss, grad, stream=None):
    n_in, n_h, n_out = shape
    _check(_lib.dftfe_mlp_loss_grad(_f32(params, "params"), n_in, n_h, n_out, _f32(X, "X"), _f32(T, "T"),
                                    _f32(w, "w"), X.shape[0], _f32(loss, "loss"), _f32(grad, "grad"),
                                    _stream(stream)))


def dftfe_mlp_adam(params, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(_lib.dftfe_mlp_adam(_f32(params, "params"), _f32(grad, "grad"), _f32(m, "m"), _f32(v, "v"),
                               params.numel(), int(t), float(lr), float(beta1), float(beta2), float(eps),
                               _stream(stream)))


def dftfe_fermi_level(evals_fr, n_oc, n_elec, kT, f_fr, stream=None):
    mu = _dbl()
    _check(_lib.dftfe_fermi_level(_vp(evals_fr.data_ptr()), evals_fr.numel(), int(n_oc), float(n_elec), float(kT),
                                  _vp(f_fr.data_ptr()), C.byref(mu), _stream(stream)))
    return mu.value


def dftfe_density(ham, Xo, Xfr, f_fr, rho):
    po, ldo = _dev(Xo, "Xo")
    if Xfr is None:
        pf, ldf, nfr, pff = None, 0, 0, None
    else:
        pf, ldf = _dev(Xfr, "Xfr")
        nfr, pff = Xfr.shape[1], _vp(f_fr.data_ptr())
    _check(_lib.dftfe_density(ham, po, ldo, Xo.shape[1], pf, ldf, nfr, pff, _vp(rho.data_ptr())))


def dftfe_cholgs_noalloc(X, stream=None):
    """Allocation-free CholGS of X (M x ncol, ncol <= 512) on `stream` (no handle needed)."""
    px, ld = _dev(X, "X")
    _check(_lib.dftfe_cholgs_noalloc(px, ld, X.shape[0], X.shape[1], _stream(stream)))


# -------------------------------------------------------- instrumentation
def dftfe_ham_set_wait_test(ham, spin_limit=0, withhold_arrival=False):
    """Test hook: spin limit of the eigensolver's bounded grid-barrier waits (0 = default)
    and one arrival withheld so that the next wait runs out (False = normal operation)."""
    _check(_lib.dftfe_ham_set_wait_test(ham, int(spin_limit), 1 if withhold_arrival else 0))


def dftfe_profile_enable(ham, enable=True):
    _check(_lib.dftfe_profile_enable(ham, 1 if enable else 0))


def dftfe_profile_query(ham, kernel):
    ms, n = _dbl(), _i64()
    _check(_lib.dftfe_profile_query(ham, kernel.encode(), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def dftfe_launch_count():
    return _lib.dftfe_launch_count()


def dftfe_last_error():
    return _lib.dftfe_last_error().decode()
