"""Thin Python binding of the qmlr C ABI (ctypes).

Argument marshalling only: torch tensors supply device memory and the current
CUDA stream; every step runs in the library's CUDA kernels. If the library is
missing or a call fails, a QMLRError is raised; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np
import torch

from .params import FCHL19Params  # noqa: F401  (re-exported)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqmlr.so")

OK, EINVAL, ENOMEM, ECUDA, EBUSY, ETIMEOUT, ENOTCONV, EDEVICE = range(8)
SORF_PER_ATOM, SORF_PER_MOL, SORF_ENERGY, SORF_SIN_T = 0, 1, 2, 4


class QMLRError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qmlr error {code}: {msg}")
        self.code = code


class _Params(C.Structure):
    _fields_ = [("n_el", C.c_int32), ("n2", C.c_int32), ("n3", C.c_int32), ("nfourier", C.c_int32),
                ("eta2", C.c_double), ("eta3", C.c_double), ("N2", C.c_double), ("N3", C.c_double),
                ("c3", C.c_double), ("zeta", C.c_double), ("rcut", C.c_double)]


class ServeConfig(C.Structure):
    _fields_ = [("n_lanes", C.c_int32), ("max_batch_atoms", C.c_int32), ("max_batch_mols", C.c_int32),
                ("max_slots", C.c_int32), ("max_inflight_atoms", C.c_int64), ("mem_budget_bytes", C.c_int64),
                ("use_graphs", C.c_int32)]


class ServeStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("rejected", C.c_int64), ("batches", C.c_int64),
                ("p50_us", C.c_double), ("p99_us", C.c_double), ("mean_us", C.c_double), ("max_us", C.c_double),
                ("throughput_rps", C.c_double), ("us_per_atom", C.c_double), ("mean_batch_atoms", C.c_double)]


class GramOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("promote", C.c_int32), ("tile_n", C.c_int32)]


class SolveOpts(C.Structure):
    _fields_ = [("method", C.c_int32), ("max_iter", C.c_int32), ("tol", C.c_double),
                ("shift", C.c_double), ("iters_done", C.c_int32), ("rel_resid", C.c_double),
                ("shift_used", C.c_double), ("factor_ms", C.c_float), ("refine_ms", C.c_float),
                ("factor", C.c_int32)]


_lib = None
P, I32, I64, D, VP = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_void_p
GRAM_FP32, GRAM_BF16X3, GRAM_BF16X6, GRAM_BF16X1, GRAM_FP8X1 = 0, 1, 2, 3, 4
GRAM_SPLITS = {GRAM_BF16X1: 1, GRAM_BF16X3: 2, GRAM_BF16X6: 3}
SOLVE_PCG, SOLVE_REFINE = 0, 1
FACTOR_FP64, FACTOR_MIXED = 0, 1

# name -> (restype, argtypes)
_SIGS = {
    "qmlr_version": (C.c_char_p, []),
    "qmlr_last_error": (C.c_char_p, []),
    "qmlr_launch_count": (C.c_int64, []),
    "qmlr_device_status": (C.c_int, [VP, C.POINTER(C.c_int32)]),
    "qmlr_fchl19_rep_dim": (C.c_int, [C.POINTER(_Params), C.POINTER(C.c_int32)]),
    "qmlr_fchl19": (C.c_int, [P, P, P, I32, I32, I32, C.POINTER(_Params), P, I32, VP]),
    "qmlr_fchl19_vjp": (C.c_int, [P, P, P, I32, I32, I32, C.POINTER(_Params), P, I32, P, I32, VP]),
    "qmlr_jac_offsets": (C.c_int, [P, I32, P, C.POINTER(C.c_int64), VP]),
    "qmlr_fchl19_vjp_atoms": (C.c_int, [P, P, P, I32, I32, I32, C.POINTER(_Params), P, I32, P, P, C.c_float,
                                        P, I32, VP]),
    "qmlr_fchl19_jac": (C.c_int, [P, P, P, I32, I32, I32, C.POINTER(_Params), P, P, I32, P, VP]),
    "qmlr_force_rows": (C.c_int, [P, I32, P, P, I32, P, P, I32, I32, D, P, I64, I64, VP]),
    "qmlr_group_workspace_bytes": (C.c_int64, [I32]),
    "qmlr_group_by_element": (C.c_int, [P, I32, I32, P, P, P, I64, VP]),
    "qmlr_group_by_element_noalloc": (C.c_int, [P, I32, I32, P, P, VP]),
    "qmlr_project_workspace_bytes": (C.c_int64, [I32, I32, I32]),
    "qmlr_project": (C.c_int, [P, I32, I32, P, P, I32, I32, P, I32, P, P, I64, VP]),
    "qmlr_project_t": (C.c_int, [P, I32, P, P, I32, I32, P, I32, I32, P, I32, P, I64, VP]),
    "qmlr_sorf": (C.c_int, [P, I32, P, I32, I32, P, I32, P, I32, D, P, I32, P, VP]),
    "qmlr_model_file_write": (C.c_int, [C.c_char_p, C.POINTER(_Params), I32, I32, I32, I32, D, D,
                                        P, P, P, P]),
    "qmlr_model_file_info": (C.c_int, [C.c_char_p, C.POINTER(_Params), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "qmlr_model_file_read": (C.c_int, [C.c_char_p, P, P, P, P]),
    "qmlr_periodic_environment_count": (C.c_int, [P, I32, P, D, P]),
    "qmlr_periodic_environment": (C.c_int, [P, I32, P, D, P, P, P]),
    "qmlr_periodic_reverse": (C.c_int, [P, P, I32, P, P]),
    "qmlr_fchl19_periodic": (C.c_int, [P, P, I32, P, P, P, P, I32, C.POINTER(_Params), P, I32, VP]),
    "qmlr_fchl19_periodic_vjp": (C.c_int, [P, P, I32, P, P, P, P, I32, C.POINTER(_Params), P, I32, P, P, P,
                                           C.c_float, P, I32, VP]),
    "qmlr_rff": (C.c_int, [P, I32, P, I32, I32, P, P, I32, D, I32, P, VP]),
    "qmlr_rff_tc_workspace_bytes": (C.c_int64, [I32, I32, I32, I32]),
    "qmlr_rff_tc": (C.c_int, [P, I32, P, I32, I32, P, P, I32, D, I32, P, P, I64, VP]),
    "qmlr_sorf_parts": (C.c_int32, [I32, I32]),
    "qmlr_sorf_grad": (C.c_int, [P, I32, P, I32, I32, P, I32, P, I32, D, P, P, P, P, VP]),
    "qmlr_gram_operand": (C.c_int, [P, I64, I32, I64, I32, P, I64, VP]),
    "qmlr_gram": (C.c_int, [I32, P, I64, I32, I64, P, I64, P, VP]),
    "qmlr_gram_operand_fp8": (C.c_int, [P, I64, I32, I64, P, I64, P, VP]),
    "qmlr_gram_tc": (C.c_int, [C.POINTER(GramOpts), P, I64, I32, P, P, VP]),
    "qmlr_zty_workspace_bytes": (C.c_int64, [I64, I32]),
    "qmlr_zty": (C.c_int, [P, I64, I32, I64, P, P, P, I64, VP]),
    "qmlr_cholesky": (C.c_int, [P, I64, I32, C.POINTER(C.c_int32), VP]),
    "qmlr_cholesky_mixed_workspace_bytes": (C.c_int64, [I32]),
    "qmlr_cholesky_mixed": (C.c_int, [P, I64, I32, P, I64, C.POINTER(C.c_int32), VP]),
    "qmlr_cholesky_solve": (C.c_int, [P, I64, I32, P, VP]),
    "qmlr_normal_apply_workspace_bytes": (C.c_int64, [I64, I32]),
    "qmlr_normal_apply": (C.c_int, [P, I64, I32, I64, D, P, P, P, I64, VP]),
    "qmlr_solve_workspace_bytes": (C.c_int64, [I64, I32]),
    "qmlr_gram_solve": (C.c_int, [P, P, I64, I32, I64, P, D, C.POINTER(SolveOpts), P, P, I64, VP]),
    "qmlr_pca_workspace_bytes": (C.c_int64, [I32, I32]),
    "qmlr_pca_fit": (C.c_int, [P, I32, I32, P, P, I32, I32, I32, P, P, I64, VP]),
    "qmlr_model_create": (C.c_int, [C.POINTER(_Params), I32, P, I32, P, I32, P, I32, D, P,
                                    C.POINTER(C.c_void_p)]),
    "qmlr_model_destroy": (C.c_int, [VP]),
    "qmlr_model_set_alpha": (C.c_int, [VP, P]),
    "qmlr_model_set_alpha_device": (C.c_int, [VP, P, VP]),
    "qmlr_model_reserve": (C.c_int, [VP, I32]),
    "qmlr_model_set_timing": (C.c_int, [VP, I32]),
    "qmlr_model_timings": (C.c_int, [VP, P, I32]),
    "qmlr_model_set_sorf_tc": (C.c_int, [VP, I32]),
    "qmlr_model_sorf_tc": (I32, [VP]),
    "qmlr_sorf_tc_table_bytes": (I64, [I32]),
    "qmlr_sorf_tc_workspace_bytes": (I64, [I32, I32]),
    "qmlr_sorf_tc_tables": (C.c_int, [P, I32, I32, I32, P, VP]),
    "qmlr_sorf_grad_tc": (C.c_int, [P, I32, P, I32, I32, P, I32, P, I32, D, P, P, P, P, P, I64, VP]),
    "qmlr_sorf_tc_segment_workspace_bytes": (I64, [I32, I32]),
    "qmlr_sorf_segment_sum_tc": (C.c_int, [P, I32, P, I32, I32, P, I32, P, I32, D, P, I64, P, I64, VP]),
    "qmlr_predict_ef": (C.c_int, [VP, P, P, P, I32, I32, P, P, VP]),
    "qmlr_energy_vjp": (C.c_int, [P, P, I32, I32, P, P, VP]),
    "qmlr_unit_rates": (C.c_int, [P, I32, VP]),
    "qmlr_predict_features": (C.c_int, [VP, P, P, P, I32, I32, VP]),
    "qmlr_predict_ef_from_features": (C.c_int, [VP, P, P, P, I32, I32, P, P, VP]),
    "qmlr_serve_create": (C.c_int, [VP, C.POINTER(ServeConfig), C.POINTER(C.c_void_p)]),
    "qmlr_serve_submit": (C.c_int, [VP, P, P, I32, C.POINTER(C.c_uint64)]),
    "qmlr_serve_poll": (C.c_int, [VP, C.c_uint64, P, P, I64]),
    "qmlr_serve_stats": (C.c_int, [VP, C.POINTER(ServeStats)]),
    "qmlr_serve_reset_stats": (C.c_int, [VP]),
    "qmlr_serve_latencies": (C.c_int, [VP, P, P, I64, C.POINTER(C.c_int64)]),
    "qmlr_serve_destroy": (C.c_int, [VP]),
    "qmlr_serve_replay": (C.c_int, [VP, P, P, P, I32, P, P, I32, C.POINTER(C.c_int64), C.POINTER(ServeStats)]),
}


def lib():
    """Load the library (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        from . import build as _build
        if not _build.up_to_date():
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise QMLRError(ECUDA, f"CUDA library not found at {LIB_PATH}")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def declared_symbols():
    return list(_SIGS)


def _check(rc: int):
    if rc != OK:
        raise QMLRError(rc, lib().qmlr_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype):
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.ascontiguousarray(t))
    t = t.to(device="cuda", dtype=dtype)
    return t.contiguous()


def c_params(p: FCHL19Params) -> _Params:
    return _Params(p.n_el, p.n2, p.n3, p.nfourier, p.eta2, p.eta3, p.N2, p.N3, p.c3, p.zeta, p.rcut)


def version() -> str:
    return lib().qmlr_version().decode()


def device_status() -> int:
    code = C.c_int32(0)
    rc = lib().qmlr_device_status(_stream(), C.byref(code))
    if rc not in (OK, EDEVICE):
        _check(rc)
    return code.value


# ----------------------------------------------------------------------------
# FCHL19


def rep_ld_of(rep_dim: int) -> int:
    return (rep_dim + 3) // 4 * 4


def fchl19(coords, elem, mol_ptr, max_atoms: int, p: FCHL19Params, rep_ld: int | None = None,
           out=None):
    coords = _dev(coords, torch.float32)
    elem = _dev(elem, torch.int32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
    rep_ld = rep_ld or rep_ld_of(p.rep_dim)
    if out is None:
        out = torch.empty((n_atoms, rep_ld), device="cuda", dtype=torch.float32)
    cp = c_params(p)
    _check(lib().qmlr_fchl19(_ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol, n_atoms, max_atoms,
                             C.byref(cp), _ptr(out), rep_ld, _stream()))
    return out


def fchl19_vjp(coords, elem, mol_ptr, max_atoms: int, p: FCHL19Params, grad_rep, out=None,
               accumulate: bool = False):
    coords = _dev(coords, torch.float32)
    elem = _dev(elem, torch.int32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    grad_rep = _dev(grad_rep, torch.float32)
    n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
    if out is None:
        out = torch.zeros((n_atoms, 3), device="cuda", dtype=torch.float32)
    cp = c_params(p)
    _check(lib().qmlr_fchl19_vjp(_ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol, n_atoms, max_atoms,
                                 C.byref(cp), _ptr(grad_rep), grad_rep.shape[1], _ptr(out),
                                 int(accumulate), _stream()))
    return out


def fchl19_vjp_atoms(coords, elem, mol_ptr, max_atoms: int, p: FCHL19Params, grad_rep, scale: float = 1.0):
    """The VJP with one warp per centre (scratch sized from the molecule sizes)."""
    coords = _dev(coords, torch.float32)
    elem = _dev(elem, torch.int32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    grad_rep = _dev(grad_rep, torch.float32)
    n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
    pair_ptr = torch.empty(n_mol + 1, device="cuda", dtype=torch.int64)
    total = C.c_int64(0)
    _check(lib().qmlr_jac_offsets(_ptr(mol_ptr), n_mol, _ptr(pair_ptr), C.byref(total), _stream()))
    contrib = torch.empty(max(total.value, 1), device="cuda", dtype=torch.float32)
    out = torch.empty((n_atoms, 3), device="cuda", dtype=torch.float32)
    cp = c_params(p)
    _check(lib().qmlr_fchl19_vjp_atoms(_ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol, n_atoms, max_atoms,
                                       C.byref(cp), _ptr(grad_rep), grad_rep.shape[1], _ptr(pair_ptr),
                                       _ptr(contrib), scale, _ptr(out), 0, _stream()))
    return out


# ----------------------------------------------------------------------------
# projection


def group_by_element(elem, n_el: int):
    elem = _dev(elem, torch.int32)
    n = elem.shape[0]
    perm = torch.empty(n, device="cuda", dtype=torch.int32)
    offs = torch.empty(n_el + 1, device="cuda", dtype=torch.int32)
    wb = lib().qmlr_group_workspace_bytes(n)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_group_by_element(_ptr(elem), n, n_el, _ptr(perm), _ptr(offs), _ptr(work), wb,
                                       _stream()))
    return perm, offs


def project(rep, rep_dim: int, perm, offs, n_el: int, U, out=None):
    rep = _dev(rep, torch.float32)
    U = _dev(U, torch.float32)
    d = U.shape[-1]
    n = rep.shape[0]
    if out is None:
        out = torch.empty((n, d), device="cuda", dtype=torch.float32)
    wb = lib().qmlr_project_workspace_bytes(n_el, rep_dim, d)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_project(_ptr(rep), rep.shape[1], rep_dim, _ptr(perm), _ptr(offs), n, n_el,
                              _ptr(U), d, _ptr(out), _ptr(work), wb, _stream()))
    return out


def project_t(gx, perm, offs, n_el: int, U, rep_dim: int, rep_ld: int | None = None, out=None):
    gx = _dev(gx, torch.float32)
    U = _dev(U, torch.float32)
    if gx.dim() == 2:
        gx = gx.unsqueeze(0)
    n_part, n, d = gx.shape
    rep_ld = rep_ld or rep_ld_of(rep_dim)
    if out is None:
        out = torch.empty((n, rep_ld), device="cuda", dtype=torch.float32)
    wb = lib().qmlr_project_workspace_bytes(n_el, rep_dim, d)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_project_t(_ptr(gx), n_part, _ptr(perm), _ptr(offs), n, n_el, _ptr(U), d,
                                rep_dim, _ptr(out), rep_ld, _ptr(work), wb, _stream()))
    return out


# ----------------------------------------------------------------------------
# SORF


def pack_signs_host(signs) -> np.ndarray:
    """Rademacher signs [n_stack, T, d] (+1/-1) -> uint32 bit words [n_stack, T, ceil(d/32)] (bit set = -1)."""
    s = np.asarray(signs)
    n_stack, T, d = s.shape
    W = (d + 31) // 32
    neg = np.zeros((n_stack, T, W * 32), dtype=np.uint64)
    neg[:, :, :d] = (s < 0)
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    return (neg.reshape(n_stack, T, W, 32) * weights).sum(axis=-1).astype(np.uint32)


def unpack_signs_host(words: np.ndarray, d: int) -> np.ndarray:
    """Inverse of pack_signs_host: bit words [n_stack, T, W] -> int8 signs [n_stack, T, d]."""
    w = np.asarray(words, dtype=np.uint32)
    bits = (w[..., None] >> np.arange(32, dtype=np.uint32)) & 1
    bits = bits.reshape(w.shape[0], w.shape[1], -1)[:, :, :d]
    return np.where(bits == 1, -1, 1).astype(np.int8)


def pack_signs(signs) -> torch.Tensor:
    """Rademacher signs [n_stack, T, d] (+1/-1) -> bit words [n_stack, T, ceil(d/32)] (bit set = -1), on the device."""
    return torch.as_tensor(pack_signs_host(signs).view(np.int32)).cuda()


def periodic_environment(coords, cell, rcut: float):
    """Lattice-image environments of a periodic system (host): (env_ptr int64 [N+1],
    env_atom int32 [E], env_shift int32 [E, 3]) with entries sorted by (j, n) per atom."""
    x = np.ascontiguousarray(np.asarray(coords, dtype=np.float64))
    A = np.ascontiguousarray(np.asarray(cell, dtype=np.float64))
    n = x.shape[0]
    ptr = np.zeros(n + 1, np.int64)
    _check(lib().qmlr_periodic_environment_count(x.ctypes.data, n, A.ctypes.data, float(rcut), ptr.ctypes.data))
    atom = np.zeros(max(int(ptr[-1]), 1), np.int32)
    shift = np.zeros((max(int(ptr[-1]), 1), 3), np.int32)
    _check(lib().qmlr_periodic_environment(x.ctypes.data, n, A.ctypes.data, float(rcut), ptr.ctypes.data,
                                           atom.ctypes.data, shift.ctypes.data))
    return ptr, atom[:ptr[-1]], shift[:ptr[-1]]


class PeriodicSystem:
    """A periodic system on the device: coordinates, elements, the cell and its
    lattice-image environments (host cell list, uploaded once) with the entries
    grouped by atom for the adjoint."""

    def __init__(self, coords, elem, cell, rcut: float):
        x = np.ascontiguousarray(np.asarray(coords, dtype=np.float32))
        self.cell = np.ascontiguousarray(np.asarray(cell, dtype=np.float64))
        self.n_atoms = x.shape[0]
        env_ptr, env_atom, env_shift = periodic_environment(x.astype(np.float64), self.cell, rcut)
        rev_ptr = np.zeros(self.n_atoms + 1, np.int64)
        rev_entry = np.zeros(max(int(env_ptr[-1]), 1), np.int64)
        ea = np.ascontiguousarray(env_atom.astype(np.int32))
        _check(lib().qmlr_periodic_reverse(env_ptr.ctypes.data, ea.ctypes.data, self.n_atoms, rev_ptr.ctypes.data,
                                           rev_entry.ctypes.data))
        self.max_env = int(np.max(np.diff(env_ptr))) if self.n_atoms else 0
        self.n_entries = int(env_ptr[-1])
        self.coords = torch.as_tensor(x).cuda()
        self.elem = _dev(elem, torch.int32)
        self.env_ptr = torch.as_tensor(env_ptr).cuda()
        self.env_atom = torch.as_tensor(np.ascontiguousarray(ea if len(ea) else np.zeros(1, np.int32))).cuda()
        sh = env_shift.astype(np.int32) if len(env_shift) else np.zeros((1, 3), np.int32)
        self.env_shift = torch.as_tensor(np.ascontiguousarray(sh)).cuda()
        self.rev_ptr = torch.as_tensor(rev_ptr).cuda()
        self.rev_entry = torch.as_tensor(rev_entry).cuda()


def fchl19_periodic(system: "PeriodicSystem", p: FCHL19Params, rep_ld: int | None = None, coords=None):
    """Rows [n_atoms, rep_ld] of a periodic system (coords: optional replacement positions)."""
    rep_ld = rep_ld or rep_ld_of(p.rep_dim)
    x = system.coords if coords is None else _dev(coords, torch.float32)
    out = torch.empty((system.n_atoms, rep_ld), device="cuda", dtype=torch.float32)
    cp = c_params(p)
    _check(lib().qmlr_fchl19_periodic(_ptr(x), _ptr(system.elem), system.n_atoms, system.cell.ctypes.data,
                                      _ptr(system.env_ptr), _ptr(system.env_atom), _ptr(system.env_shift),
                                      system.max_env, C.byref(cp), _ptr(out), rep_ld, _stream()))
    return out


def fchl19_periodic_vjp(system: "PeriodicSystem", p: FCHL19Params, grad_rep, scale: float = 1.0, coords=None):
    """scale * sum_i (d rho_i / d R)^T grad_rep[i] for a periodic system, [n_atoms, 3]."""
    x = system.coords if coords is None else _dev(coords, torch.float32)
    grad_rep = _dev(grad_rep, torch.float32)
    contrib = torch.empty((system.n_entries + system.n_atoms, 3), device="cuda", dtype=torch.float32)
    out = torch.empty((system.n_atoms, 3), device="cuda", dtype=torch.float32)
    cp = c_params(p)
    _check(lib().qmlr_fchl19_periodic_vjp(_ptr(x), _ptr(system.elem), system.n_atoms, system.cell.ctypes.data,
                                          _ptr(system.env_ptr), _ptr(system.env_atom), _ptr(system.env_shift),
                                          system.max_env, C.byref(cp), _ptr(grad_rep), grad_rep.shape[1],
                                          _ptr(system.rev_ptr), _ptr(system.rev_entry), _ptr(contrib), scale,
                                          _ptr(out), 0, _stream()))
    return out


def save_model(path: str, p: FCHL19Params, U, signs, T: int, b, sigma: float, lam: float, alpha) -> None:
    """Write a trained model to a checksummed model file (host only)."""
    def host(a, dt):
        a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else np.asarray(a)
        return np.ascontiguousarray(a, dtype=dt)
    U = host(U, np.float32)
    bits = np.ascontiguousarray(pack_signs_host(signs))
    b = host(b, np.float32)
    alpha = host(alpha, np.float64)
    n_el, rep_dim, d = U.shape
    assert bits.shape[1] == T and b.shape[0] == alpha.shape[0] == bits.shape[0] * d
    cp = c_params(p)
    _check(lib().qmlr_model_file_write(str(path).encode(), C.byref(cp), rep_dim, d, T, b.shape[0],
                                       float(sigma), float(lam), U.ctypes.data, bits.ctypes.data,
                                       b.ctypes.data, alpha.ctypes.data))


def load_model(path: str) -> dict:
    """Read a model file: dict with params (FCHL19Params), U, signs (int8 +1/-1), T, b, sigma, lam, alpha."""
    cp = _Params()
    rep_dim, d, T, nf = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    sigma, lam = C.c_double(), C.c_double()
    path_b = str(path).encode()
    _check(lib().qmlr_model_file_info(path_b, C.byref(cp), C.byref(rep_dim), C.byref(d), C.byref(T),
                                      C.byref(nf), C.byref(sigma), C.byref(lam)))
    U = np.empty((cp.n_el, rep_dim.value, d.value), np.float32)
    bits = np.empty((nf.value // d.value, T.value, (d.value + 31) // 32), np.uint32)
    b = np.empty(nf.value, np.float32)
    alpha = np.empty(nf.value, np.float64)
    _check(lib().qmlr_model_file_read(path_b, U.ctypes.data, bits.ctypes.data, b.ctypes.data,
                                      alpha.ctypes.data))
    params = FCHL19Params(n_el=cp.n_el, n2=cp.n2, n3=cp.n3, nfourier=cp.nfourier, eta2=cp.eta2, eta3=cp.eta3,
                          N2=cp.N2, N3=cp.N3, c3=cp.c3, zeta=cp.zeta, rcut=cp.rcut)
    return {"params": params, "U": U, "signs": unpack_signs_host(bits, d.value), "T": T.value, "b": b,
            "sigma": sigma.value, "lam": lam.value, "alpha": alpha}


def sorf(x, mol_ptr, sign_bits, T: int, b, sigma: float, mode: int, alpha=None, n_features=None):
    x = _dev(x, torch.float32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    b = _dev(b, torch.float32)
    n_atoms, d = x.shape
    n_mol = mol_ptr.shape[0] - 1
    nf = n_features or b.shape[0]
    if mode in (SORF_PER_ATOM, SORF_SIN_T):
        out = torch.empty((n_atoms, nf), device="cuda", dtype=torch.float32)
    elif mode == SORF_PER_MOL:
        out = torch.empty((n_mol, nf), device="cuda", dtype=torch.float32)
    else:
        out = torch.empty((n_mol,), device="cuda", dtype=torch.float64)
    al = None if alpha is None else _dev(alpha, torch.float32)
    _check(lib().qmlr_sorf(_ptr(x), d, _ptr(mol_ptr), n_mol, n_atoms, _ptr(sign_bits), T, _ptr(b),
                           nf, float(sigma), _ptr(al), mode, _ptr(out), _stream()))
    return out


def rff(x, mol_ptr, G, b, sigma: float, mode: int):
    """Dense RFF features z = sqrt(2/N_F) cos(G x / sigma + b), per atom or summed per molecule."""
    x = _dev(x, torch.float32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    G = _dev(G, torch.float32)
    b = _dev(b, torch.float32)
    n_atoms, d = x.shape
    n_mol = mol_ptr.shape[0] - 1
    nf = b.shape[0]
    rows = n_atoms if mode == SORF_PER_ATOM else n_mol
    out = torch.empty((rows, nf), device="cuda", dtype=torch.float32)
    _check(lib().qmlr_rff(_ptr(x), d, _ptr(mol_ptr), n_mol, n_atoms, _ptr(G), _ptr(b), nf, float(sigma),
                          mode, _ptr(out), _stream()))
    return out


def rff_tc(x, mol_ptr, G, b, sigma: float, mode: int):
    """Dense RFF features on the tensor cores (same result form as rff)."""
    x = _dev(x, torch.float32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    G = _dev(G, torch.float32)
    b = _dev(b, torch.float32)
    n_atoms, d = x.shape
    n_mol = mol_ptr.shape[0] - 1
    nf = b.shape[0]
    rows = n_atoms if mode == SORF_PER_ATOM else n_mol
    out = torch.empty((rows, nf), device="cuda", dtype=torch.float32)
    wb = lib().qmlr_rff_tc_workspace_bytes(n_atoms, d, nf, mode)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_rff_tc(_ptr(x), d, _ptr(mol_ptr), n_mol, n_atoms, _ptr(G), _ptr(b), nf, float(sigma), mode,
                             _ptr(out), _ptr(work), wb, _stream()))
    return out


def sorf_parts(n_features: int, d: int) -> int:
    return lib().qmlr_sorf_parts(n_features, d)


def sorf_grad(x, mol_ptr, sign_bits, T: int, b, sigma: float, alpha):
    x = _dev(x, torch.float32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    b = _dev(b, torch.float32)
    alpha = _dev(alpha, torch.float32)
    n_atoms, d = x.shape
    n_mol = mol_ptr.shape[0] - 1
    nf = b.shape[0]
    n_part = sorf_parts(nf, d)
    E = torch.empty((n_mol,), device="cuda", dtype=torch.float64)
    gx = torch.empty((n_part, n_atoms, d), device="cuda", dtype=torch.float32)
    atom_e = torch.empty((n_part, max(n_atoms, 1)), device="cuda", dtype=torch.float64)
    _check(lib().qmlr_sorf_grad(_ptr(x), d, _ptr(mol_ptr), n_mol, n_atoms, _ptr(sign_bits), T,
                                _ptr(b), nf, float(sigma), _ptr(alpha), _ptr(atom_e), _ptr(E), _ptr(gx),
                                _stream()))
    return E, gx


def sorf_tc_tables(sign_bits, T: int, n_features: int, d: int = 128):
    """FP16 chain tables of the tensor-core SORF ([2, N_F, 128] as int16 bits)."""
    nbytes = lib().qmlr_sorf_tc_table_bytes(n_features)
    tables = torch.empty((nbytes // 2,), device="cuda", dtype=torch.int16)
    _check(lib().qmlr_sorf_tc_tables(_ptr(sign_bits), d, T, n_features, _ptr(tables), _stream()))
    return tables


def sorf_grad_tc(x, mol_ptr, tables, T: int, b, sigma: float, alpha):
    """Energies [n_mol] and gradients [1, n_atoms, d] from the tensor-core chains."""
    x = _dev(x, torch.float32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    b = _dev(b, torch.float32)
    alpha = _dev(alpha, torch.float32)
    n_atoms, d = x.shape
    n_mol = mol_ptr.shape[0] - 1
    nf = b.shape[0]
    E = torch.empty((n_mol,), device="cuda", dtype=torch.float64)
    gx = torch.empty((1, n_atoms, d), device="cuda", dtype=torch.float32)
    atom_e = torch.empty((max(n_atoms, 1),), device="cuda", dtype=torch.float64)
    wb = lib().qmlr_sorf_tc_workspace_bytes(n_atoms, nf)
    work = torch.empty((wb + 256,), device="cuda", dtype=torch.uint8)
    off = (-work.data_ptr()) % 256
    _check(lib().qmlr_sorf_grad_tc(_ptr(x), d, _ptr(mol_ptr), n_mol, n_atoms, _ptr(tables), T, _ptr(b), nf,
                                   float(sigma), _ptr(alpha), _ptr(atom_e), _ptr(E), _ptr(gx),
                                   work.data_ptr() + off, wb, _stream()))
    return E, gx


def sorf_segment_sum_tc(x, mol_ptr, tables, T: int, b, sigma: float, out=None):
    """Energy rows Z [n_mol, N_F] (float32) from the tensor-core chains; out may be
    a row block of a larger float32 matrix (row stride >= N_F, unit column stride)."""
    x = _dev(x, torch.float32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    b = _dev(b, torch.float32)
    n_atoms, d = x.shape
    n_mol = mol_ptr.shape[0] - 1
    nf = b.shape[0]
    if out is None:
        out = torch.empty((n_mol, nf), device="cuda", dtype=torch.float32)
    assert out.dtype == torch.float32 and out.stride(1) == 1 and out.shape == (n_mol, nf)
    wb = lib().qmlr_sorf_tc_segment_workspace_bytes(n_atoms, nf)
    work = torch.empty((wb + 256,), device="cuda", dtype=torch.uint8)
    off = (-work.data_ptr()) % 256
    _check(lib().qmlr_sorf_segment_sum_tc(_ptr(x), d, _ptr(mol_ptr), n_mol, n_atoms, _ptr(tables), T, _ptr(b),
                                          nf, float(sigma), _ptr(out), out.stride(0), work.data_ptr() + off, wb,
                                          _stream()))
    return out


# ----------------------------------------------------------------------------
# normal equations


def k_pad_of(n_rows: int) -> int:
    return max(64, (n_rows + 63) // 64 * 64)


def gram_operand(Z, n_split: int = 2):
    """Transposed split-BF16 operand [n_split, N_F, k_pad] (int16 holding bf16 bits)."""
    Z = _dev(Z, torch.float32)
    n_rows, nf = Z.shape
    kp = k_pad_of(n_rows)
    zt = torch.empty((n_split, nf, kp), device="cuda", dtype=torch.int16)
    _check(lib().qmlr_gram_operand(_ptr(Z), n_rows, nf, Z.stride(0), n_split, _ptr(zt), kp, _stream()))
    return zt


def gram_operand_fp8(Z):
    """e4m3 operand [N_F, k_pad] (uint8) and per-feature inverse scales [N_F] (float32)."""
    Z = _dev(Z, torch.float32)
    n_rows, nf = Z.shape
    kp = max(128, (n_rows + 127) // 128 * 128)
    zt = torch.empty((nf, kp), device="cuda", dtype=torch.uint8)
    inv = torch.empty(nf, device="cuda", dtype=torch.float32)
    _check(lib().qmlr_gram_operand_fp8(_ptr(Z), n_rows, nf, Z.stride(0), _ptr(zt), kp, _ptr(inv), _stream()))
    return zt, inv


def gram(Z, precision: int = GRAM_BF16X6, operand=None):
    """G = Z^T Z (float32, full symmetric)."""
    Z = _dev(Z, torch.float32)
    n_rows, nf = Z.shape
    G = torch.empty((nf, nf), device="cuda", dtype=torch.float32)
    if precision == GRAM_FP8X1:
        return gram_tc(Z, precision, operand=operand)
    if precision in GRAM_SPLITS:
        zt = operand if operand is not None else gram_operand(Z, GRAM_SPLITS[precision])
        _check(lib().qmlr_gram(precision, _ptr(Z), n_rows, nf, Z.stride(0), _ptr(zt), zt.shape[2],
                               _ptr(G), _stream()))
    else:
        _check(lib().qmlr_gram(precision, _ptr(Z), n_rows, nf, Z.stride(0), None, 0, _ptr(G), _stream()))
    return G


def gram_tc(Z, precision: int, promote: int = 0, tile_n: int = 0, operand=None):
    """G = Z^T Z on the tensor cores with explicit accumulation (promote) and tile
    width (tile_n); operand: the split operand, or (zt, inv_scale) for FP8X1."""
    Z = _dev(Z, torch.float32)
    n_rows, nf = Z.shape
    G = torch.empty((nf, nf), device="cuda", dtype=torch.float32)
    inv = None
    if precision == GRAM_FP8X1:
        zt, inv = operand if operand is not None else gram_operand_fp8(Z)
        kp = zt.shape[1]
    else:
        zt = operand if operand is not None else gram_operand(Z, GRAM_SPLITS[precision])
        kp = zt.shape[2]
    o = GramOpts(precision, promote, tile_n)
    _check(lib().qmlr_gram_tc(C.byref(o), _ptr(zt), kp, nf, _ptr(inv), _ptr(G), _stream()))
    return G


def zty(Z, y):
    Z = _dev(Z, torch.float32)
    y = _dev(y, torch.float64)
    n_rows, nf = Z.shape
    c = torch.empty(nf, device="cuda", dtype=torch.float64)
    wb = lib().qmlr_zty_workspace_bytes(n_rows, nf)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_zty(_ptr(Z), n_rows, nf, Z.stride(0), _ptr(y), _ptr(c), _ptr(work), wb, _stream()))
    return c


def cholesky(A):
    """Lower Cholesky factor of a symmetric positive definite matrix (float64)."""
    L = _dev(A, torch.float64).clone()
    n = L.shape[0]
    info = C.c_int32(0)
    _check(lib().qmlr_cholesky(_ptr(L), n, n, C.byref(info), _stream()))
    return L, info.value


def cholesky_mixed(A):
    """Mixed-precision lower factor (FP64 panels, tensor-core trailing updates)."""
    L = _dev(A, torch.float64).clone()
    n = L.shape[0]
    wb = lib().qmlr_cholesky_mixed_workspace_bytes(n)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    info = C.c_int32(0)
    _check(lib().qmlr_cholesky_mixed(_ptr(L), n, n, _ptr(work), wb, C.byref(info), _stream()))
    return L, info.value


def cholesky_solve(L, v):
    v = _dev(v, torch.float64).clone()
    n = L.shape[0]
    _check(lib().qmlr_cholesky_solve(_ptr(L), L.stride(0), n, _ptr(v), _stream()))
    return v


def normal_apply(Z, p, lam: float):
    """q = Z^T (Z p) + lam p (float64), the solve's exact operator."""
    Z = _dev(Z, torch.float32)
    p = _dev(p, torch.float64)
    n_rows, nf = Z.shape
    q = torch.empty(nf, device="cuda", dtype=torch.float64)
    wb = lib().qmlr_normal_apply_workspace_bytes(n_rows, nf)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_normal_apply(_ptr(Z), n_rows, nf, Z.stride(0), float(lam), _ptr(p), _ptr(q),
                                   _ptr(work), wb, _stream()))
    return q


def gram_solve(G, Z, y, lam: float, method: int = SOLVE_PCG, max_iter: int = 50, tol: float = 1e-10,
               shift: float = -2.0 ** -16, raise_on_notconv: bool = False, factor: int = FACTOR_MIXED):
    """alpha for (Z^T Z + lam I) alpha = Z^T y with a factor of G + (lam + shift) I
    (shift < 0: relative to max diag G; factor FACTOR_FP64 or FACTOR_MIXED).
    Returns (alpha, iterations, relative residual)."""
    G = _dev(G, torch.float32)
    Z = _dev(Z, torch.float32)
    y = _dev(y, torch.float64)
    n_rows, nf = Z.shape
    alpha = torch.empty(nf, device="cuda", dtype=torch.float64)
    wb = lib().qmlr_solve_workspace_bytes(n_rows, nf)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    opts = SolveOpts(method, max_iter, tol, shift, 0, 0.0, 0.0, 0.0, 0.0, factor)
    rc = lib().qmlr_gram_solve(_ptr(G), _ptr(Z), n_rows, nf, Z.stride(0), _ptr(y), float(lam),
                               C.byref(opts), _ptr(alpha), _ptr(work), wb, _stream())
    global last_solve
    last_solve = opts
    if rc == ENOTCONV and not raise_on_notconv:
        return alpha, opts.iters_done, opts.rel_resid
    _check(rc)
    return alpha, opts.iters_done, opts.rel_resid


last_solve = None


UNIT_RATES = ("dfma", "ffma", "fadd", "fadd_x2", "expf", "sinf", "shfl")


def unit_rates() -> dict:
    """Measured per-unit throughput of the current GPU (operations per second)."""
    out = (C.c_double * len(UNIT_RATES))()
    _check(lib().qmlr_unit_rates(out, len(UNIT_RATES), _stream()))
    return dict(zip(UNIT_RATES, list(out)))


def launch_count() -> int:
    return lib().qmlr_launch_count()


# ----------------------------------------------------------------------------
# PCA fit and the model handle


def pca_fit(rep, rep_dim: int, perm, offs, n_el: int, d: int, max_per_element: int = 4096):
    rep = _dev(rep, torch.float32)
    U = torch.empty((n_el, rep_dim, d), device="cuda", dtype=torch.float32)
    wb = lib().qmlr_pca_workspace_bytes(rep.shape[1], d)
    work = torch.empty(wb, device="cuda", dtype=torch.uint8)
    _check(lib().qmlr_pca_fit(_ptr(rep), rep.shape[1], rep_dim, _ptr(perm), _ptr(offs), n_el,
                              max_per_element, d, _ptr(U), _ptr(work), wb, _stream()))
    return U


class Model:
    """Device-resident trained model (owns a qmlr_model handle)."""

    def __init__(self, p: FCHL19Params, max_mol_atoms: int, U, signs, T: int, b, sigma: float,
                 alpha):
        U = np.ascontiguousarray(np.asarray(U.cpu() if isinstance(U, torch.Tensor) else U,
                                            dtype=np.float32))
        bits = pack_signs(signs).cpu().numpy().view(np.uint32) if not isinstance(signs, torch.Tensor) \
            else signs.cpu().numpy().view(np.uint32)
        bits = np.ascontiguousarray(bits)
        b = np.ascontiguousarray(np.asarray(b, dtype=np.float32))
        al = np.ascontiguousarray(np.asarray(alpha.cpu() if isinstance(alpha, torch.Tensor) else alpha,
                                             dtype=np.float32))
        self.p, self.d, self.T, self.n_features = p, U.shape[2], T, b.shape[0]
        self.max_mol_atoms = max_mol_atoms
        cp = c_params(p)
        h = C.c_void_p()
        _check(lib().qmlr_model_create(C.byref(cp), max_mol_atoms, U.ctypes.data, self.d,
                                       bits.ctypes.data, T, b.ctypes.data, self.n_features,
                                       float(sigma), al.ctypes.data, C.byref(h)))
        self.handle = h
        self.capacity = 0

    @classmethod
    def from_file(cls, path: str, max_mol_atoms: int) -> "Model":
        """A device model from a model file written by save_model."""
        m = load_model(path)
        return cls(m["params"], max_mol_atoms, m["U"], m["signs"], m["T"], m["b"], m["sigma"], m["alpha"])

    def set_alpha(self, alpha):
        al = np.ascontiguousarray(np.asarray(alpha.cpu() if isinstance(alpha, torch.Tensor) else alpha,
                                             dtype=np.float32))
        _check(lib().qmlr_model_set_alpha(self.handle, al.ctypes.data))

    def set_alpha_device(self, alpha64: torch.Tensor):
        _check(lib().qmlr_model_set_alpha_device(self.handle, _ptr(alpha64), _stream()))

    TIMINGS = ("fchl19", "group_project", "sorf_energy_grad", "project_t", "fchl19_vjp")

    def set_sorf_tc(self, enable: bool = True):
        """SORF energies + gradients of E+F predictions on the tensor cores (else the FWHT kernel)."""
        _check(lib().qmlr_model_set_sorf_tc(self.handle, int(enable)))

    @property
    def sorf_tc(self) -> bool:
        return bool(lib().qmlr_model_sorf_tc(self.handle))

    def set_timing(self, enable: bool = True):
        """Record CUDA events around the prediction's kernels (diagnostics)."""
        _check(lib().qmlr_model_set_timing(self.handle, int(enable)))

    def timings(self) -> dict:
        """ms of the last prediction's kernels (waits for them)."""
        out = (C.c_float * 5)()
        _check(lib().qmlr_model_timings(self.handle, out, 5))
        return dict(zip(self.TIMINGS, list(out)))

    def reserve(self, n_atoms: int):
        if n_atoms > self.capacity:
            _check(lib().qmlr_model_reserve(self.handle, n_atoms))
            self.capacity = n_atoms

    def predict(self, coords, elem, mol_ptr, forces: bool = True, out=None):
        """Energies [n_mol] (float64) and forces [n_atoms, 3] (float32) on the device."""
        coords = _dev(coords, torch.float32)
        elem = _dev(elem, torch.int32)
        mol_ptr = _dev(mol_ptr, torch.int32)
        n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
        self.reserve(n_atoms)
        if out is None:
            E = torch.empty(n_mol, device="cuda", dtype=torch.float64)
            F = torch.empty((n_atoms, 3), device="cuda", dtype=torch.float32) if forces else None
        else:
            E, F = out
        _check(lib().qmlr_predict_ef(self.handle, _ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol, n_atoms,
                                     _ptr(E), _ptr(F), _stream()))
        return E, F

    def predict_features(self, coords, elem, mol_ptr):
        """First half of predict (representations, grouping, projection) on the
        current stream; independent of the weights."""
        coords = _dev(coords, torch.float32)
        elem = _dev(elem, torch.int32)
        mol_ptr = _dev(mol_ptr, torch.int32)
        n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
        self.reserve(n_atoms)
        _check(lib().qmlr_predict_features(self.handle, _ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol, n_atoms,
                                           _stream()))

    def predict_from_features(self, coords, elem, mol_ptr, forces: bool = True):
        """Second half of predict for the batch given to predict_features."""
        coords = _dev(coords, torch.float32)
        elem = _dev(elem, torch.int32)
        mol_ptr = _dev(mol_ptr, torch.int32)
        n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
        E = torch.empty(n_mol, device="cuda", dtype=torch.float64)
        F = torch.empty((n_atoms, 3), device="cuda", dtype=torch.float32) if forces else None
        _check(lib().qmlr_predict_ef_from_features(self.handle, _ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol,
                                                   n_atoms, _ptr(E), _ptr(F), _stream()))
        return E, F

    def close(self):
        if getattr(self, "handle", None):
            lib().qmlr_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------
# autograd: energies with forces from the hand-written adjoint


class FCHL19SORFEnergy(torch.autograd.Function):
    """Molecule energies E [n_mol] (float64) of a device-resident Model as a
    differentiable function of the coordinates [n_atoms, 3] (float32).

    Forward runs the model's path (FCHL19 -> per-element projection -> SORF
    with the weight dot product, atomic energies summed per molecule); when the
    coordinates require a gradient it also runs the hand-written adjoint in the
    same call (SORF backward -> transposed projection -> FCHL19 vector-Jacobian
    product) and keeps F = -dE/dr. Backward maps an upstream gradient g [n_mol]
    to dL/dr_k = -g[mol(k)] F_k (qmlr_energy_vjp): every atom belongs to one
    molecule, so that is the whole chain rule. Double backward is not supported.

        E = FCHL19SORFEnergy.apply(coords, model, elem, mol_ptr)
    """

    @staticmethod
    def forward(ctx, coords, model, elem, mol_ptr):
        elem = _dev(elem, torch.int32)
        mol_ptr = _dev(mol_ptr, torch.int32)
        need = ctx.needs_input_grad[0]
        E, F = model.predict(coords.detach(), elem, mol_ptr, forces=need)
        if need:
            ctx.save_for_backward(F, mol_ptr)
            ctx.coords_dtype = coords.dtype
        return E

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, grad_E):
        F, mol_ptr = ctx.saved_tensors
        g = _dev(grad_E, torch.float64)
        out = torch.empty_like(F)
        _check(lib().qmlr_energy_vjp(_ptr(F), _ptr(mol_ptr), mol_ptr.shape[0] - 1, F.shape[0], _ptr(g),
                                     _ptr(out), _stream()))
        return out.to(ctx.coords_dtype), None, None, None


def energy(coords, model: "Model", elem, mol_ptr):
    """E [n_mol] through FCHL19SORFEnergy (differentiable in coords)."""
    return FCHL19SORFEnergy.apply(coords, model, elem, mol_ptr)


# ----------------------------------------------------------------------------
# force rows for energy + force training


def fchl19_jacobian(coords, elem, mol_ptr, max_atoms: int, p: FCHL19Params, rep_ld: int | None = None):
    """(jac_ptr, jac [n_rows, rep_ld], row_elem) of FCHL19 Jacobian rows."""
    coords = _dev(coords, torch.float32)
    elem = _dev(elem, torch.int32)
    mol_ptr = _dev(mol_ptr, torch.int32)
    n_atoms, n_mol = coords.shape[0], mol_ptr.shape[0] - 1
    rep_ld = rep_ld or rep_ld_of(p.rep_dim)
    jac_ptr = torch.empty(n_mol + 1, device="cuda", dtype=torch.int64)
    total = C.c_int64(0)
    _check(lib().qmlr_jac_offsets(_ptr(mol_ptr), n_mol, _ptr(jac_ptr), C.byref(total), _stream()))
    jac = torch.empty((max(total.value, 1), rep_ld), device="cuda", dtype=torch.float32)
    row_elem = torch.empty(max(total.value, 1), device="cuda", dtype=torch.int32)
    cp = c_params(p)
    _check(lib().qmlr_fchl19_jac(_ptr(coords), _ptr(elem), _ptr(mol_ptr), n_mol, n_atoms, max_atoms,
                                 C.byref(cp), _ptr(jac_ptr), _ptr(jac), rep_ld, _ptr(row_elem), _stream()))
    return jac_ptr, jac[:total.value], row_elem[:total.value]


def force_rows(tangents, jac_ptr, mol_ptr, sin_t, sign_bits, T: int, n_features: int, sigma: float,
               out=None, row0: int = 0):
    """Force rows [3 n_atoms, N_F] (or written into `out` from row `row0`)."""
    mol_ptr = _dev(mol_ptr, torch.int32)
    n_mol = mol_ptr.shape[0] - 1
    n_atoms = sin_t.shape[0]
    d = tangents.shape[1]
    if out is None:
        out = torch.empty((3 * n_atoms, n_features), device="cuda", dtype=torch.float32)
    _check(lib().qmlr_force_rows(_ptr(tangents), d, _ptr(jac_ptr), _ptr(mol_ptr), n_mol, _ptr(sin_t),
                                 _ptr(sign_bits), T, n_features, float(sigma), _ptr(out), out.stride(0),
                                 row0, _stream()))
    return out


# ----------------------------------------------------------------------------
# serving


class Server:
    """Continuous-batching prediction server around a Model (host arrays in and out)."""

    def __init__(self, model: "Model", n_lanes: int = 2, max_batch_atoms: int = 16384,
                 max_batch_mols: int = 1024, max_slots: int = 100000, max_inflight_atoms: int = 10_000_000,
                 mem_budget_bytes: int = 0, use_graphs: bool = True):
        self.model = model
        cfg = ServeConfig(n_lanes, max_batch_atoms, max_batch_mols, max_slots, max_inflight_atoms,
                          mem_budget_bytes, int(use_graphs))
        h = C.c_void_p()
        _check(lib().qmlr_serve_create(model.handle, C.byref(cfg), C.byref(h)))
        self.handle = h

    def submit(self, coords, elem) -> int:
        """Ticket, or raises QMLRError (code EBUSY when not admitted)."""
        c = np.ascontiguousarray(coords, dtype=np.float32)
        e = np.ascontiguousarray(elem, dtype=np.int32)
        t = C.c_uint64(0)
        _check(lib().qmlr_serve_submit(self.handle, c.ctypes.data, e.ctypes.data, len(e), C.byref(t)))
        return t.value

    def try_submit(self, coords, elem):
        c = np.ascontiguousarray(coords, dtype=np.float32)
        e = np.ascontiguousarray(elem, dtype=np.int32)
        t = C.c_uint64(0)
        rc = lib().qmlr_serve_submit(self.handle, c.ctypes.data, e.ctypes.data, len(e), C.byref(t))
        return rc, t.value

    def poll(self, ticket: int, n_atoms: int, timeout_us: int = 10_000_000):
        """(rc, E, F[n_atoms, 3])."""
        E = C.c_double(0.0)
        F = np.empty((n_atoms, 3), dtype=np.float32)
        rc = lib().qmlr_serve_poll(self.handle, ticket, C.byref(E), F.ctypes.data, timeout_us)
        return rc, E.value, F

    def stats(self) -> dict:
        st = ServeStats()
        _check(lib().qmlr_serve_stats(self.handle, C.byref(st)))
        return {k: getattr(st, k) for k, _ in ServeStats._fields_}

    def reset_stats(self):
        _check(lib().qmlr_serve_reset_stats(self.handle))

    def latencies(self):
        """(latency_us float32 [n], atoms int32 [n]) of the requests since the last reset."""
        n = C.c_int64(0)
        _check(lib().qmlr_serve_latencies(self.handle, None, None, 0, C.byref(n)))
        lat = np.zeros(max(n.value, 1), np.float32)
        at = np.zeros(max(n.value, 1), np.int32)
        _check(lib().qmlr_serve_latencies(self.handle, lat.ctypes.data, at.ctypes.data, n.value, C.byref(n)))
        return lat[:n.value], at[:n.value]

    def replay(self, coords, elem, mol_ptr, arrival_s, pick) -> dict:
        """Replay a request trace from native threads; returns the run's statistics."""
        c = np.ascontiguousarray(coords, dtype=np.float32)
        e = np.ascontiguousarray(elem, dtype=np.int32)
        mp = np.ascontiguousarray(mol_ptr, dtype=np.int32)
        at = np.ascontiguousarray(np.asarray(arrival_s, dtype=np.float64) * 1e6)
        pk = np.ascontiguousarray(pick, dtype=np.int32)
        rej = C.c_int64(0)
        st = ServeStats()
        _check(lib().qmlr_serve_replay(self.handle, c.ctypes.data, e.ctypes.data, mp.ctypes.data, len(mp) - 1,
                                       at.ctypes.data, pk.ctypes.data, len(pk), C.byref(rej), C.byref(st)))
        out = {k: getattr(st, k) for k, _ in ServeStats._fields_}
        out["rejected"] = rej.value
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().qmlr_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
