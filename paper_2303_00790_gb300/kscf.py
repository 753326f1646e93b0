"""Thin ctypes binding of libkscf (include/kscf.h).

Argument marshalling only: every computation runs in the CUDA library.  Device
arrays are torch tensors (PyTorch provides device memory and streams); their raw
pointers and the current stream are passed through the C ABI.  There is no CPU
fallback: if libkscf.so cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkscf.so")

KSCF_OK = 0
KSCF_ERR_INVALID = -1
KSCF_ERR_CUDA = -2
KSCF_ERR_WORKSPACE = -3
KSCF_ERR_NOT_SPD = -4
KSCF_ERR_NONFINITE = -5
KSCF_ERR_NO_CONVERGE = -6
KSCF_ERR_UNSUPPORTED = -7
KSCF_ERR_HOST_ALLOC = -8
KSCF_ERR_TIMEOUT = -9
KSCF_F64, KSCF_F32 = 0, 1
KSCF_GEMM_NATIVE, KSCF_GEMM_TENSOR = 0, 1
KSCF_OP_APPLY, KSCF_OP_FILTER, KSCF_OP_ORTHO, KSCF_OP_RR = 0, 1, 2, 3
KSCF_ORTHO_ALLOW_SHIFT = 0x100
KSCF_NOALLOC_SCRATCH_BYTES = 4 << 20     # size of the fixed array of kscf_hamiltonian_apply_noalloc


class KscfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"kscf error {code}: {msg}")
        self.code = code


class kscf_atom(C.Structure):
    _fields_ = [("x", C.c_double), ("y", C.c_double), ("z", C.c_double),
                ("z_number", C.c_int32), ("reserved", C.c_int32)]


class kscf_species(C.Structure):
    _fields_ = [("z_number", C.c_int32), ("n_proj", C.c_int32),
                ("z_valence", C.c_double), ("r_c", C.c_double), ("a_gauss", C.c_double),
                ("r_gauss", C.c_double), ("e_s", C.c_double), ("e_p", C.c_double),
                ("r_p", C.c_double), ("r_cut", C.c_double)]


class kscf_grid_info(C.Structure):
    _fields_ = [("n_points", C.c_int64), ("n_slots", C.c_int64), ("n_bricks", C.c_int64),
                ("brick", C.c_int32), ("lo", C.c_int32 * 3), ("extent", C.c_int32 * 3),
                ("reserved", C.c_int32), ("h", C.c_double), ("center", C.c_double * 3)]


class kscf_scf_params(C.Structure):
    _fields_ = [("k", C.c_int32), ("degree", C.c_int32), ("dtype", C.c_int32), ("gemm_mode", C.c_int32),
                ("block", C.c_int32), ("first_iters", C.c_int32), ("history", C.c_int32),
                ("poisson_maxiter", C.c_int32), ("mix_alpha", C.c_double), ("sre_tol_ry", C.c_double),
                ("poisson_rtol", C.c_double), ("kT", C.c_double), ("kerker_q0", C.c_double),
                ("degree_max", C.c_int32), ("degree_min", C.c_int32), ("degree_group", C.c_int32),
                ("upper_bound", C.c_int32), ("adapt_reduction", C.c_double), ("adapt_tol_floor", C.c_double)]


class kscf_scf_report(C.Structure):
    _fields_ = [("step", C.c_int32), ("converged", C.c_int32), ("poisson_iters", C.c_int32),
                ("chefsi_iters", C.c_int32), ("sre_ry", C.c_double), ("e_band", C.c_double),
                ("e_total", C.c_double), ("homo", C.c_double), ("lumo", C.c_double), ("electrons", C.c_double),
                ("mu", C.c_double), ("minus_ts", C.c_double), ("occ_last", C.c_double),
                ("kerker_iters", C.c_int32), ("reserved", C.c_int32), ("filter_work", C.c_double),
                ("upper_bound", C.c_double)]


KSCF_FIELD_RHO, KSCF_FIELD_V_IN, KSCF_FIELD_V_H, KSCF_FIELD_V_XC = 0, 1, 2, 3
KSCF_FIELD_V_ION, KSCF_FIELD_V_START, KSCF_FIELD_EPS_XC = 4, 5, 6


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libkscf.so not built ({LIB_PATH}); run __graft_entry__.build()")
    return C.CDLL(LIB_PATH)


lib = _load()
_vp, _i32, _i64, _d, _sz = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_size_t
_sigs = {
    "kscf_last_error": ([], C.c_char_p),
    "kscf_launch_counter": ([], C.c_uint64),
    "kscf_build_grid": ([C.POINTER(_d), _d, _d, _i32, C.POINTER(_vp)], _i32),
    "kscf_build_grid_box": ([_i32, _i32, _i32, _d, _i32, C.POINTER(_vp)], _i32),
    "kscf_grid_get_info": ([_vp, C.POINTER(kscf_grid_info)], _i32),
    "kscf_grid_slots": ([_vp, _vp, _vp], _i32),
    "kscf_grid_free": ([_vp], _i32),
    "kscf_build_hamiltonian": ([_vp, C.POINTER(kscf_atom), _i32, C.POINTER(kscf_species), _i32,
                                C.POINTER(_vp)], _i32),
    "kscf_ham_free": ([_vp], _i32),
    "kscf_ham_grid_info": ([_vp, C.POINTER(kscf_grid_info)], _i32),
    "kscf_set_potential": ([_vp, _vp, _vp], _i32),
    "kscf_get_potential": ([_vp, _vp, _vp], _i32),
    "kscf_spectral_bounds": ([_vp, C.POINTER(_d), C.POINTER(_d)], _i32),
    "kscf_workspace_size": ([_vp, _i32, _i32, _i32, _i32, _i32, C.POINTER(_sz)], _i32),
    "kscf_hamiltonian_apply": ([_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp, _sz, _vp], _i32),
    "kscf_hamiltonian_apply_noalloc": ([_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp], _i32),
    "kscf_chebyshev_filter": ([_vp, _vp, _i64, _i32, _i32, _d, _d, _d, _i32, _i32, _vp, _sz, _vp], _i32),
    "kscf_orthonormalize": ([_vp, _vp, _i64, _i32, _i32, _i32, _vp, _sz, _vp], _i32),
    "kscf_rayleigh_ritz": ([_vp, _vp, _i64, _i32, _i32, _i32, C.POINTER(_d), _vp, _sz, _vp], _i32),
    "kscf_density": ([_vp, _vp, _i64, _i32, _i32, _vp, _vp, _vp], _i32),
    "kscf_random_subspace": ([_vp, _vp, _i64, _i32, _i32, C.c_uint64, _vp], _i32),
    "kscf_points_to_slots": ([_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp], _i32),
    "kscf_slots_to_points": ([_vp, _vp, _i64, _vp, _i64, _i32, _i32, _vp], _i32),
    "kscf_hilbert_index3": ([C.c_uint32, C.c_uint32, C.c_uint32, _i32], C.c_uint64),
    "kscf_gram": ([_vp, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _d, _vp, _i64, _vp, _sz, _vp], _i32),
    "kscf_rotate": ([_vp, _i64, _vp, _i64, _i64, _i32, _i32, _i32, _i32, _i32, _vp, _i64, _vp, _sz, _vp], _i32),
    "kscf_gemm_workspace_size": ([_i32, _i64, _i32, _i32, _i32, _i32, C.POINTER(_sz)], _i32),
    "kscf_sym_eig_work_bytes": ([_i32, C.POINTER(_sz)], _i32),
    "kscf_sym_eig": ([_vp, _i64, _i32, _vp, _vp, _sz, _vp], _i32),
    "kscf_check_status": ([], _i32),
    "kscf_selftest_barrier_timeout": ([_vp], _i32),
    "kscf_selftest_eig_barrier_timeout": ([_vp], _i32),
    "kscf_scf_create": ([_vp, C.POINTER(kscf_atom), _i32, C.POINTER(kscf_species), _i32, C.POINTER(_d),
                         C.POINTER(kscf_scf_params), _vp, _i64, _vp, C.POINTER(_vp)], _i32),
    "kscf_scf_start": ([_vp, _vp, _i32, C.c_uint64, C.POINTER(_d)], _i32),
    "kscf_scf_step": ([_vp, C.POINTER(kscf_scf_report), C.POINTER(_d)], _i32),
    "kscf_scf_get": ([_vp, _i32, _vp], _i32),
    "kscf_scf_evaluate": ([_vp, C.POINTER(kscf_scf_report), C.POINTER(_d), C.POINTER(_d)], _i32),
    "kscf_scf_refine": ([_vp, _i32, _d, C.POINTER(kscf_scf_report), C.POINTER(_d), C.POINTER(_d),
                         C.POINTER(_i32)], _i32),
    "kscf_scf_hartree": ([_vp, _vp, _vp, C.POINTER(_i32)], _i32),
    "kscf_scf_free": ([_vp], _i32),
    "kscf_lda_xc": ([_vp, _vp, _vp, _vp, _vp], _i32),
    "kscf_descriptors": ([_vp, C.POINTER(kscf_atom), _i32, _vp, _vp], _i32),
    "kscf_mlp_forward": ([_vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp], _i32),
    "kscf_mlp_work_size": ([_i64, C.POINTER(_sz)], _i32),
    "kscf_mlp_loss_grad": ([_vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _sz, _vp], _i32),
    "kscf_lanczos_bounds": ([_vp, _i32, C.c_uint64, C.POINTER(_d), C.POINTER(_d), C.POINTER(_d), _vp, _vp, _vp],
                            _i32),
    "kscf_dos": ([_vp, _i32, _i32, _d, _d, _i32, _vp, C.POINTER(_d)], _i32),
    "kscf_mlp_adam": ([_vp, _vp, _vp, _vp, _i32, C.c_float, C.c_float, C.c_float, C.c_float, _vp], _i32),
    "kscf_mlp_training_data": ([_vp, _vp, _vp, _vp], _i32),
    "kscf_mlp_standardize": ([_vp, _vp, _i64, _vp, _vp, _vp, C.POINTER(_d), _vp], _i32),
    "kscf_mlp_correction": ([_vp, _vp, _vp, _d, _d, _vp, _i64, _i32, _vp, _vp, _vp], _i32),
}
for _name, (_args, _res) in _sigs.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_sigs)


def _check(code: int):
    if code != KSCF_OK:
        raise KscfError(code, lib.kscf_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _stream(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float64:
        return KSCF_F64
    if t.dtype == torch.float32:
        return KSCF_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def _rows(t, k: int):
    if not t.is_cuda or t.dim() != 2 or t.stride(1) != 1 or t.shape[1] < k:
        raise ValueError("X must be a 2-D CUDA tensor with unit column stride")
    return t.stride(0)


def _work(ham, op, k, dtype, mode=0, block=0, work=None):
    need = kscf_workspace_size(ham, op, k, dtype, mode, block)
    if work is None:
        torch = _torch()
        work = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    return work, need


# ------------------------------------------------------------------ grid
def kscf_build_grid(center, radius: float, h: float, brick: int = 8):
    c = (C.c_double * 3)(*[float(x) for x in center])
    out = C.c_void_p()
    _check(lib.kscf_build_grid(c, float(radius), float(h), int(brick), C.byref(out)))
    return Grid(out)


def kscf_build_grid_box(nx: int, ny: int, nz: int, h: float, brick: int = 8):
    out = C.c_void_p()
    _check(lib.kscf_build_grid_box(nx, ny, nz, float(h), int(brick), C.byref(out)))
    return Grid(out)


def _info_dict(info: kscf_grid_info) -> dict:
    return {"n_points": info.n_points, "n_slots": info.n_slots, "n_bricks": info.n_bricks,
            "brick": info.brick, "lo": tuple(info.lo), "extent": tuple(info.extent), "h": info.h,
            "center": tuple(info.center)}


class Grid:
    def __init__(self, handle):
        self.handle = handle
        info = kscf_grid_info()
        _check(lib.kscf_grid_get_info(handle, C.byref(info)))
        self.info = _info_dict(info)

    def slots(self):
        """(lex_of_slot int64 (n_slots,), ijk_of_slot int32 (n_slots, 3))"""
        n = self.info["n_slots"]
        lex = np.empty(n, dtype=np.int64)
        ijk = np.empty((n, 3), dtype=np.int32)
        _check(lib.kscf_grid_slots(self.handle, lex.ctypes.data_as(C.c_void_p), ijk.ctypes.data_as(C.c_void_p)))
        return lex, ijk

    def free(self):
        if self.handle:
            lib.kscf_grid_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------------ Hamiltonian
def species_array(species):
    arr = (kscf_species * len(species))()
    for i, s in enumerate(species):
        arr[i] = kscf_species(int(s["z_number"]), int(s["n_proj"]), float(s["z_valence"]), float(s["r_c"]),
                              float(s["a_gauss"]), float(s["r_gauss"]), float(s["e_s"]), float(s["e_p"]),
                              float(s["r_p"]), float(s["r_cut"]))
    return arr


def atom_array(pos, z):
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    arr = (kscf_atom * max(len(pos), 1))()
    for i in range(len(pos)):
        arr[i] = kscf_atom(float(pos[i, 0]), float(pos[i, 1]), float(pos[i, 2]), int(z[i]), 0)
    return arr, len(pos)


def kscf_build_hamiltonian(grid: Grid, atom_pos, atom_z, species):
    atoms, n = atom_array(atom_pos, atom_z)
    sp = species_array(species)
    out = C.c_void_p()
    _check(lib.kscf_build_hamiltonian(grid.handle, atoms, n, sp, len(species), C.byref(out)))
    return Hamiltonian(out)


class Hamiltonian:
    def __init__(self, handle):
        self.handle = handle
        info = kscf_grid_info()
        _check(lib.kscf_ham_grid_info(handle, C.byref(info)))
        self.info = _info_dict(info)
        self.n_slots = self.info["n_slots"]
        self.h3 = self.info["h"] ** 3

    def free(self):
        if self.handle:
            lib.kscf_ham_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def kscf_spectral_bounds(ham: Hamiltonian):
    lo, hi = C.c_double(), C.c_double()
    _check(lib.kscf_spectral_bounds(ham.handle, C.byref(lo), C.byref(hi)))
    return lo.value, hi.value


def kscf_lanczos_bounds(ham: Hamiltonian, steps: int = 12, seed: int = 7, stream=None):
    """(upper, theta_max, theta_min, alpha, beta) of a K-step Lanczos run."""
    up, tmax, tmin = C.c_double(), C.c_double(), C.c_double()
    a = np.zeros(steps)
    b = np.zeros(steps)
    _check(lib.kscf_lanczos_bounds(ham.handle, steps, int(seed), C.byref(up), C.byref(tmax), C.byref(tmin),
                                   a.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p), _stream(stream)))
    return up.value, tmax.value, tmin.value, a, b


def kscf_set_potential(ham: Hamiltonian, v_slots, stream=None):
    torch = _torch()
    assert v_slots.is_cuda and v_slots.dtype == torch.float64 and v_slots.numel() >= ham.n_slots
    _check(lib.kscf_set_potential(ham.handle, C.c_void_p(v_slots.data_ptr()), _stream(stream)))


def kscf_get_potential(ham: Hamiltonian, stream=None):
    torch = _torch()
    v = torch.empty(ham.n_slots, dtype=torch.float64, device="cuda")
    _check(lib.kscf_get_potential(ham.handle, C.c_void_p(v.data_ptr()), _stream(stream)))
    return v


def kscf_workspace_size(ham: Hamiltonian, op: int, k: int, dtype: int, mode: int = 0, block: int = 0) -> int:
    n = C.c_size_t()
    _check(lib.kscf_workspace_size(ham.handle, op, k, dtype, mode, block, C.byref(n)))
    return n.value


# ------------------------------------------------------------------ hot path
def kscf_hamiltonian_apply(ham: Hamiltonian, Y, HY, k: int | None = None, work=None, stream=None):
    k = Y.shape[1] if k is None else k
    dt = _dtype_code(Y)
    work, need = _work(ham, KSCF_OP_APPLY, k, dt, work=work)
    _check(lib.kscf_hamiltonian_apply(ham.handle, C.c_void_p(Y.data_ptr()), _rows(Y, k), C.c_void_p(HY.data_ptr()),
                                      _rows(HY, k), k, dt, C.c_void_p(work.data_ptr()), work.numel(),
                                      _stream(stream)))
    return HY


def kscf_hamiltonian_apply_noalloc(ham: Hamiltonian, Y, HY, k: int | None = None, stream=None):
    """H Y without a work buffer (fixed library-owned scratch; see include/kscf.h)."""
    k = Y.shape[1] if k is None else k
    _check(lib.kscf_hamiltonian_apply_noalloc(ham.handle, C.c_void_p(Y.data_ptr()), _rows(Y, k),
                                              C.c_void_p(HY.data_ptr()), _rows(HY, k), k, _dtype_code(Y),
                                              _stream(stream)))
    return HY


def kscf_chebyshev_filter(ham: Hamiltonian, X, degree: int, a: float, b: float, a0: float, k: int | None = None,
                          block: int = 0, work=None, stream=None):
    k = X.shape[1] if k is None else k
    dt = _dtype_code(X)
    work, need = _work(ham, KSCF_OP_FILTER, k, dt, block=block, work=work)
    _check(lib.kscf_chebyshev_filter(ham.handle, C.c_void_p(X.data_ptr()), _rows(X, k), k, degree, a, b, a0, dt,
                                     block, C.c_void_p(work.data_ptr()), work.numel(), _stream(stream)))
    return X


def kscf_orthonormalize(ham: Hamiltonian, X, mode: int = KSCF_GEMM_NATIVE, k: int | None = None, work=None,
                        stream=None, allow_shift: bool = False):
    k = X.shape[1] if k is None else k
    dt = _dtype_code(X)
    work, need = _work(ham, KSCF_OP_ORTHO, k, dt, mode=mode, work=work)
    _check(lib.kscf_orthonormalize(ham.handle, C.c_void_p(X.data_ptr()), _rows(X, k), k, dt,
                                   mode | (KSCF_ORTHO_ALLOW_SHIFT if allow_shift else 0),
                                   C.c_void_p(work.data_ptr()), work.numel(), _stream(stream)))
    return X


def kscf_rayleigh_ritz(ham: Hamiltonian, X, mode: int = KSCF_GEMM_NATIVE, k: int | None = None, work=None,
                       stream=None):
    k = X.shape[1] if k is None else k
    dt = _dtype_code(X)
    work, need = _work(ham, KSCF_OP_RR, k, dt, mode=mode, work=work)
    lam = np.empty(k, dtype=np.float64)
    _check(lib.kscf_rayleigh_ritz(ham.handle, C.c_void_p(X.data_ptr()), _rows(X, k), k, dt, mode,
                                  lam.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(work.data_ptr()),
                                  work.numel(), _stream(stream)))
    return lam


def kscf_density(ham: Hamiltonian, X, n_occ: int, occ=None, rho=None, stream=None):
    torch = _torch()
    if rho is None:
        rho = torch.empty(ham.n_slots, dtype=torch.float64, device="cuda")
    occ_ptr = C.c_void_p(occ.data_ptr()) if occ is not None else C.c_void_p(0)
    _check(lib.kscf_density(ham.handle, C.c_void_p(X.data_ptr()), _rows(X, n_occ), n_occ, _dtype_code(X), occ_ptr,
                            C.c_void_p(rho.data_ptr()), _stream(stream)))
    return rho


def kscf_random_subspace(ham: Hamiltonian, X, seed: int, k: int | None = None, stream=None):
    k = X.shape[1] if k is None else k
    _check(lib.kscf_random_subspace(ham.handle, C.c_void_p(X.data_ptr()), _rows(X, k), k, _dtype_code(X),
                                    int(seed), _stream(stream)))
    return X


def kscf_points_to_slots(ham: Hamiltonian, P, X, k: int | None = None, stream=None):
    """X (slot layout, n_slots rows) <- P (n_points rows in lexicographic point order)."""
    k = P.shape[1] if k is None else k
    _check(lib.kscf_points_to_slots(ham.handle, C.c_void_p(P.data_ptr()), _rows(P, k), C.c_void_p(X.data_ptr()),
                                    _rows(X, k), k, _dtype_code(X), _stream(stream)))
    return X


def kscf_slots_to_points(ham: Hamiltonian, X, P, k: int | None = None, stream=None):
    """P (n_points rows in lexicographic point order) <- X (slot layout)."""
    k = X.shape[1] if k is None else k
    _check(lib.kscf_slots_to_points(ham.handle, C.c_void_p(X.data_ptr()), _rows(X, k), C.c_void_p(P.data_ptr()),
                                    _rows(P, k), k, _dtype_code(X), _stream(stream)))
    return P


def kscf_gemm_workspace_size(op: int, rows: int, m: int, n: int, dtype: int, mode: int) -> int:
    b = C.c_size_t()
    _check(lib.kscf_gemm_workspace_size(op, rows, m, n, dtype, mode, C.byref(b)))
    return b.value


def kscf_gram(A, B, scale: float = 1.0, mode: int = KSCF_GEMM_NATIVE, C_out=None, m: int | None = None,
              n: int | None = None, rows: int | None = None, work=None, stream=None):
    """C = scale * A^T B (FP64, column-major, returned as a (n, m) row-major view's transpose)."""
    torch = _torch()
    m = A.shape[1] if m is None else m
    n = B.shape[1] if n is None else n
    rows = A.shape[0] if rows is None else rows
    dt = _dtype_code(A)
    if C_out is None:
        C_out = torch.empty((n, m), dtype=torch.float64, device="cuda")   # column-major m x n
    if work is None:
        work = torch.empty(max(256, kscf_gemm_workspace_size(0, rows, m, n, dt, mode)), dtype=torch.uint8,
                           device="cuda")
    _check(lib.kscf_gram(C.c_void_p(A.data_ptr()), _rows(A, m), C.c_void_p(B.data_ptr()), _rows(B, n), rows, m, n,
                         dt, mode, scale, C.c_void_p(C_out.data_ptr()), m, C.c_void_p(work.data_ptr()), work.numel(),
                         _stream(stream)))
    return C_out.t()


def kscf_rotate(A, Q, mode: int = KSCF_GEMM_NATIVE, minus_identity: bool = False, out=None, work=None, stream=None):
    """out = A Q (Q FP64 (kin, kout) row-major torch tensor; passed column-major)."""
    torch = _torch()
    rows, kin = A.shape[0], Q.shape[0]
    kout = Q.shape[1]
    Qc = Q.t().contiguous()       # column-major storage of Q
    dt = _dtype_code(A)
    if out is None:
        out = torch.empty((rows, kout), dtype=A.dtype, device="cuda")
    if work is None:
        work = torch.empty(max(256, kscf_gemm_workspace_size(1, rows, kin, kout, dt, mode)), dtype=torch.uint8,
                           device="cuda")
    _check(lib.kscf_rotate(C.c_void_p(A.data_ptr()), _rows(A, kin), C.c_void_p(Qc.data_ptr()), kin, rows, kin, kout,
                           dt, mode, 1 if minus_identity else 0, C.c_void_p(out.data_ptr()), _rows(out, kout),
                           C.c_void_p(work.data_ptr()), work.numel(), _stream(stream)))
    return out


def kscf_sym_eig(A, w=None, work=None, stream=None):
    """In place: A (n x n FP64 device tensor, symmetric) <- eigenvectors; returns w
    (device, ascending).  A row-major torch tensor is the transpose of the column-major
    matrix the library sees; for a symmetric A both are the same, and the eigenvector of
    w[j] is row j of the result (column j of its column-major reading)."""
    torch = _torch()
    n = A.shape[0]
    if w is None:
        w = torch.empty(n, dtype=torch.float64, device=A.device)
    if work is None:
        b = C.c_size_t()
        _check(lib.kscf_sym_eig_work_bytes(n, C.byref(b)))
        work = torch.empty(b.value, dtype=torch.uint8, device=A.device)
    _check(lib.kscf_sym_eig(C.c_void_p(A.data_ptr()), A.stride(0), n, C.c_void_p(w.data_ptr()),
                            C.c_void_p(work.data_ptr()), work.numel(), _stream(stream)))
    return w


def kscf_check_status():
    _check(lib.kscf_check_status())


def kscf_selftest_barrier_timeout(stream=None):
    """Raises KscfError(KSCF_ERR_TIMEOUT) when the bounded grid barrier works (see kscf.h)."""
    _check(lib.kscf_selftest_barrier_timeout(_stream(stream)))


def kscf_selftest_eig_barrier_timeout(stream=None):
    """Raises KscfError(KSCF_ERR_TIMEOUT) when the eigensolver's bounded grid barrier works."""
    _check(lib.kscf_selftest_eig_barrier_timeout(_stream(stream)))


def kscf_launch_counter() -> int:
    return int(lib.kscf_launch_counter())


def kscf_hilbert_index3(x: int, y: int, z: int, bits: int) -> int:
    return int(lib.kscf_hilbert_index3(x, y, z, bits))


# ------------------------------------------------------------------ SCF
def kscf_lda_xc(ham: Hamiltonian, rho, eps=None, vxc=None, stream=None):
    """(eps_xc, V_xc) of a slot-ordered FP64 density (device)."""
    torch = _torch()
    if eps is None:
        eps = torch.empty(ham.n_slots, dtype=torch.float64, device="cuda")
    if vxc is None:
        vxc = torch.empty(ham.n_slots, dtype=torch.float64, device="cuda")
    _check(lib.kscf_lda_xc(ham.handle, C.c_void_p(rho.data_ptr()), C.c_void_p(eps.data_ptr()),
                           C.c_void_p(vxc.data_ptr()), _stream(stream)))
    return eps, vxc


def scf_params(k: int, degree: int, dtype: int = KSCF_F64, gemm_mode: int = KSCF_GEMM_NATIVE, block: int = 0,
               first_iters: int = 4, history: int = 8, mix_alpha: float = 0.3, sre_tol_ry: float = 1e-4,
               poisson_rtol: float = 1e-12, poisson_maxiter: int = 20000, kT: float = 0.0,
               kerker_q0: float = 0.0, degree_max: int = 0, degree_min: int = 0, degree_group: int = 64,
               upper_bound: int = 0, adapt_reduction: float = 0.1, adapt_tol_floor: float = 1e-6) -> kscf_scf_params:
    return kscf_scf_params(k, degree, dtype, gemm_mode, block, first_iters, history, poisson_maxiter, mix_alpha,
                           sre_tol_ry, poisson_rtol, kT, kerker_q0, degree_max, degree_min, degree_group, upper_bound,
                           adapt_reduction, adapt_tol_floor)


class Scf:
    """SCF state (kscf_scf handle) over a Hamiltonian and a caller-owned subspace X."""

    def __init__(self, ham: Hamiltonian, atom_pos, atom_z, species, params: kscf_scf_params, X=None, stream=None):
        torch = _torch()
        self.ham = ham
        self.params = params
        self.k = params.k
        if X is None:
            ld = (params.k + 31) // 32 * 32
            X = torch.zeros((ham.n_slots, ld), dtype=torch.float64 if params.dtype == KSCF_F64 else torch.float32,
                            device="cuda")
        if _dtype_code(X) != params.dtype:
            raise TypeError("X dtype does not match params.dtype")
        self.X = X
        self.stream = stream
        atoms, n = atom_array(atom_pos, atom_z)
        sp = species_array(species)
        radius = (C.c_double * len(species))(*[float(s["r_start"]) for s in species])
        out = C.c_void_p()
        _check(lib.kscf_scf_create(ham.handle, atoms, n, sp, len(species), radius, C.byref(params),
                                   C.c_void_p(X.data_ptr()), _rows(X, params.k), _stream(stream), C.byref(out)))
        self.handle = out

    def start(self, seed: int = 1, init_x: bool = True, dv_start=None):
        lam = np.empty(self.k, dtype=np.float64)
        dv = C.c_void_p(dv_start.data_ptr()) if dv_start is not None else C.c_void_p(0)
        _check(lib.kscf_scf_start(self.handle, dv, 1 if init_x else 0, int(seed),
                                  lam.ctypes.data_as(C.POINTER(C.c_double))))
        return lam

    def step(self):
        rep = kscf_scf_report()
        lam = np.empty(self.k, dtype=np.float64)
        _check(lib.kscf_scf_step(self.handle, C.byref(rep), lam.ctypes.data_as(C.POINTER(C.c_double))))
        d = {f: getattr(rep, f) for f, _ in kscf_scf_report._fields_}
        d["lam"] = lam
        return d

    def evaluate(self):
        """FP64 Rayleigh quotients, residual norms and energies of the last step's vectors."""
        rep = kscf_scf_report()
        lam = np.empty(self.k, dtype=np.float64)
        res = np.empty(self.k, dtype=np.float64)
        _check(lib.kscf_scf_evaluate(self.handle, C.byref(rep), lam.ctypes.data_as(C.POINTER(C.c_double)),
                                     res.ctypes.data_as(C.POINTER(C.c_double))))
        d = {f: getattr(rep, f) for f, _ in kscf_scf_report._fields_}
        d["lam"] = lam
        d["resid"] = res
        return d

    def refine(self, max_iters: int = 40, resid_tol: float = 1e-7):
        """Converged mode at the current V_in (see kscf_scf_refine)."""
        rep = kscf_scf_report()
        lam = np.empty(self.k, dtype=np.float64)
        res = np.empty(self.k, dtype=np.float64)
        it = C.c_int()
        _check(lib.kscf_scf_refine(self.handle, int(max_iters), float(resid_tol), C.byref(rep),
                                   lam.ctypes.data_as(C.POINTER(C.c_double)), res.ctypes.data_as(C.POINTER(C.c_double)),
                                   C.byref(it)))
        d = {f: getattr(rep, f) for f, _ in kscf_scf_report._fields_}
        d["lam"] = lam
        d["resid"] = res
        d["iters"] = it.value
        return d

    def run(self, max_steps: int = 40):
        reports = []
        for _ in range(max_steps):
            r = self.step()
            reports.append(r)
            if r["converged"]:
                break
        return reports

    def get(self, field: int, out=None):
        torch = _torch()
        if out is None:
            out = torch.empty(self.ham.n_slots, dtype=torch.float64, device="cuda")
        _check(lib.kscf_scf_get(self.handle, field, C.c_void_p(out.data_ptr())))
        return out

    def hartree(self, rho, vh=None):
        torch = _torch()
        if vh is None:
            vh = torch.zeros(self.ham.n_slots, dtype=torch.float64, device="cuda")
        it = C.c_int()
        _check(lib.kscf_scf_hartree(self.handle, C.c_void_p(rho.data_ptr()), C.c_void_p(vh.data_ptr()), C.byref(it)))
        return vh, it.value

    def free(self):
        if getattr(self, "handle", None):
            lib.kscf_scf_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------------------ DOS
def kscf_dos(eigvals, n_occ: int, bin_ev: float = 0.1, e_lo_ev: float = -15.0, n_bins: int = 200):
    """(hist (n_bins,), bin left edges in eV, gap in eV) of the Ritz values (host arrays)."""
    ev = np.ascontiguousarray(eigvals, dtype=np.float64)
    hist = np.empty(n_bins, dtype=np.float64)
    gap = C.c_double()
    _check(lib.kscf_dos(ev.ctypes.data_as(C.c_void_p), len(ev), n_occ, bin_ev, e_lo_ev, n_bins,
                        hist.ctypes.data_as(C.c_void_p), C.byref(gap)))
    return hist, e_lo_ev + bin_ev * np.arange(n_bins), gap.value


# ------------------------------------------------------------------ learned start
KSCF_MLP_N_IN, KSCF_MLP_N_HID = 32, 128
KSCF_MLP_N_PARAMS = 32 * 128 + 128 + 128 * 128 + 128 + 128 + 1
KSCF_MLP_FP32, KSCF_MLP_BF16 = 0, 1


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def kscf_descriptors(ham: Hamiltonian, atom_pos, atom_z, D=None, stream=None):
    """(n_slots, 32) float32 device tensor of radial descriptors."""
    torch = _torch()
    if D is None:
        D = torch.empty((ham.n_slots, KSCF_MLP_N_IN), dtype=torch.float32, device="cuda")
    atoms, n = atom_array(atom_pos, atom_z)
    _check(lib.kscf_descriptors(ham.handle, atoms, n, _p(D), _stream(stream)))
    return D


def kscf_mlp_forward(params, mu, inv_sd, D, precision: int = KSCF_MLP_FP32, y=None, stream=None):
    torch = _torch()
    n = D.shape[0]
    if y is None:
        y = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib.kscf_mlp_forward(_p(params), _p(mu), _p(inv_sd), _p(D), n, precision, _p(y), _stream(stream)))
    return y


def kscf_mlp_training_data(scf, D_slots, n_points: int):
    """(D, t): descriptors and dV = V_in - V_start of the domain points (lexicographic
    rows, float32 device tensors) of a self-consistent SCF handle."""
    torch = _torch()
    D = torch.empty((n_points, KSCF_MLP_N_IN), dtype=torch.float32, device="cuda")
    t = torch.empty(n_points, dtype=torch.float32, device="cuda")
    _check(lib.kscf_mlp_training_data(scf.handle, _p(D_slots), _p(D), _p(t)))
    return D, t


def kscf_mlp_standardize(D, t, stream=None):
    """(mu, inv_sd, t_norm, t_shift, t_scale) of a training set (synchronous)."""
    torch = _torch()
    n = D.shape[0]
    mu = torch.empty(KSCF_MLP_N_IN, dtype=torch.float32, device="cuda")
    inv_sd = torch.empty_like(mu)
    t_norm = torch.empty(n, dtype=torch.float32, device="cuda")
    ss = (C.c_double * 2)()
    _check(lib.kscf_mlp_standardize(_p(D), _p(t), n, _p(mu), _p(inv_sd), _p(t_norm), ss, _stream(stream)))
    return mu, inv_sd, t_norm, ss[0], ss[1]


def kscf_mlp_correction(params, mu, inv_sd, t_shift: float, t_scale: float, D, precision: int = KSCF_MLP_FP32,
                        dv=None, stream=None):
    """dV per row of D (float64 device tensor): the network output de-standardised."""
    torch = _torch()
    n = D.shape[0]
    if dv is None:
        dv = torch.empty(n, dtype=torch.float64, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    _check(lib.kscf_mlp_correction(_p(params), _p(mu), _p(inv_sd), float(t_shift), float(t_scale), _p(D), n,
                                   precision, _p(y), _p(dv), _stream(stream)))
    return dv


def kscf_mlp_work_size(n: int) -> int:
    b = C.c_size_t()
    _check(lib.kscf_mlp_work_size(n, C.byref(b)))
    return b.value


def kscf_mlp_loss_grad(params, mu, inv_sd, D, t, grad=None, loss=None, work=None, stream=None):
    torch = _torch()
    n = D.shape[0]
    if grad is None:
        grad = torch.empty(KSCF_MLP_N_PARAMS, dtype=torch.float32, device="cuda")
    if work is None:
        work = torch.empty(kscf_mlp_work_size(n), dtype=torch.uint8, device="cuda")
    _check(lib.kscf_mlp_loss_grad(_p(params), _p(mu), _p(inv_sd), _p(D), _p(t), n, _p(grad), _p(loss), _p(work),
                                  work.numel(), _stream(stream)))
    return grad


def kscf_mlp_adam(params, grad, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
                  eps: float = 1e-8, stream=None):
    _check(lib.kscf_mlp_adam(_p(params), _p(grad), _p(m), _p(v), step, lr, beta1, beta2, eps, _stream(stream)))


# ------------------------------------------------------------------ convenience
def build_cluster(atom_pos, atom_z, species, radius: float, h: float, brick: int = 8, center=None):
    """Grid (centred on atom 0 unless `center`) and Hamiltonian for a cluster."""
    c = np.asarray(atom_pos, dtype=np.float64)[0] if center is None else center
    g = kscf_build_grid(c, radius, h, brick)
    H = kscf_build_hamiltonian(g, atom_pos, atom_z, species)
    return g, H
