"""Thin Python binding of libed (argument marshalling only).

Every computation runs in libed's CUDA kernels; this module converts numpy /
torch arguments to the C structs of include/ed.h and back.  It never falls
back to a CPU implementation: if libed.so is missing it raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libed.so")

ED_F64, ED_F32, ED_C64, ED_C128 = 0, 1, 2, 3
STATUS = ["ED_OK", "ED_ERR_ARG", "ED_ERR_NOT_GROUP", "ED_ERR_NOT_SYMMETRIC", "ED_ERR_NOT_SUBLATTICE_STABLE",
          "ED_ERR_CHAR_NOT_HOMOMORPHISM", "ED_ERR_SPINFLIP_SZ", "ED_ERR_EMPTY_SECTOR", "ED_ERR_NOMEM",
          "ED_ERR_INDEX_NOT_FOUND", "ED_ERR_TIMEOUT", "ED_ERR_NOT_CONVERGED", "ED_ERR_CUDA", "ED_ERR_TABLE_TOO_LARGE"]

P = ctypes.POINTER
c_i32, c_i64, c_u8, c_u16, c_u32, c_u64, c_dbl, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint8,
                                                         ctypes.c_uint16, ctypes.c_uint32, ctypes.c_uint64,
                                                         ctypes.c_double, ctypes.c_void_p)


class EdError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        self.name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{self.name}: {msg}")


class ed_sector(ctypes.Structure):
    _fields_ = [("n_sites", c_i32), ("n_up", c_i32), ("n_sym", c_i32), ("perm", P(c_i32)), ("spinflip", P(c_u8)),
                ("chi", P(c_dbl)), ("n_sublat", c_i32)]


class ed_sector_sun(ctypes.Structure):
    _fields_ = [("n_sites", c_i32), ("n_colors", c_i32), ("counts", P(c_i32)), ("n_sym", c_i32),
                ("perm", P(c_i32)), ("chi", P(c_dbl)), ("n_sublat", c_i32)]


class ed_terms(ctypes.Structure):
    _fields_ = [("n_bonds", c_i32), ("bond", P(c_i32)), ("J", P(c_dbl)), ("n_tri", c_i32), ("tri", P(c_i32)),
                ("Jchi", P(c_dbl))]


ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, ctypes.c_size_t, c_vp, c_vp)


class ed_allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_vp)]


class ed_lanczos_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("n_eig", c_i32), ("tol", c_dbl), ("max_iter", c_i32), ("reorth", c_i32),
                ("seed", c_u64), ("refine", c_i32), ("check_every", c_i32), ("host_vectors", c_i32)]


class ed_block_lanczos_opts(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("block", c_i32), ("n_eig", c_i32), ("tol", c_dbl), ("max_iter", c_i32),
                ("seed", c_u64), ("use_graph", c_i32), ("check_every", c_i32), ("reorth", c_i32)]


class ed_block_lanczos_report(ctypes.Structure):
    _fields_ = [("iters", c_i32), ("converged_sectors", c_i32), ("krylov_dim", c_i32), ("used_graph", c_i32),
                ("seconds", c_dbl), ("step_seconds", c_dbl)]


class ed_lanczos_report(ctypes.Structure):
    _fields_ = [("iters", c_i32), ("converged", c_i32), ("n_apply", c_i32), ("ritz", c_dbl * 8),
                ("resid_bound", c_dbl * 8), ("refined", c_dbl * 8), ("refined_resid", c_dbl * 8),
                ("seconds", c_dbl)]


_lib = None


def lib():
    """Load libed.so (built in-tree by paper_2210_03511_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libed.so not built ({LIB_PATH}); run paper_2210_03511_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.ed_basis_build.argtypes = [P(ed_sector), P(ed_allocator), c_vp, P(c_vp)]
        L.ed_basis_dim.argtypes = [c_vp, P(c_i64)]
        L.ed_basis_build_sun.argtypes = [P(ed_sector_sun), P(ed_allocator), c_vp, P(c_vp)]
        L.ed_hamiltonian_create_sun.argtypes = [c_vp, P(ed_terms), ctypes.c_size_t, c_vp, P(c_vp)]
        L.ed_basis_export.argtypes = [c_vp, P(c_u64), P(c_u16)]
        L.ed_sector_tables.argtypes = [P(ed_sector), P(c_u16), P(c_u32), P(c_u16), P(c_i64), P(c_u16), P(c_u8)]
        L.ed_representatives.argtypes = [P(ed_sector), P(c_u64), c_i64, P(c_u64), P(c_i32), P(c_i32), P(c_u8)]
        L.ed_representatives.restype = ctypes.c_int
        L.ed_basis_free.argtypes = [c_vp]
        L.ed_basis_free.restype = None
        L.ed_hamiltonian_create.argtypes = [c_vp, P(ed_terms), P(c_vp)]
        L.ed_hamiltonian_is_real.argtypes = [c_vp, P(c_i32)]
        L.ed_hamiltonian_free.argtypes = [c_vp]
        L.ed_hamiltonian_free.restype = None
        L.ed_apply.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_i32, c_vp]
        L.ed_apply_counters.argtypes = [c_vp, c_vp, P(c_i64), P(c_i64)]
        L.ed_hamiltonian_store.argtypes = [c_vp, ctypes.c_int, c_i32, ctypes.c_size_t, c_vp, P(ctypes.c_size_t)]
        L.ed_hamiltonian_store_info.argtypes = [c_vp, P(c_i64), P(c_i32), P(c_i32), P(ctypes.c_size_t)]
        L.ed_hamiltonian_store_autotune.argtypes = [c_vp, ctypes.c_int, ctypes.c_size_t, c_vp, P(c_i32),
                                                    P(ctypes.c_size_t)]
        L.ed_hamiltonian_store_free.argtypes = [c_vp]
        L.ed_hamiltonian_store_set_lanes.argtypes = [c_vp, c_i32]
        L.ed_hamiltonian_store_schedule.argtypes = [c_vp, P(c_i32), P(c_i32)]
        L.ed_hamiltonian_store_free.restype = None
        L.ed_lanczos.argtypes = [c_vp, P(ed_lanczos_opts), P(c_dbl), c_vp, P(ed_lanczos_report), c_vp]
        L.ed_batch_create.argtypes = [P(c_vp), c_i32, P(c_vp)]
        L.ed_batch_rows.argtypes = [c_vp, P(c_i64)]
        L.ed_apply_batch.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_i32, c_vp]
        L.ed_batch_autotune.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_i32, c_vp, P(c_i32)]
        L.ed_apply_autotune.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_i32, c_vp, P(c_i32)]
        L.ed_apply_set_blocks.argtypes = [c_vp, ctypes.c_int, c_i32, c_i32]
        L.ed_tridiag_eigs.argtypes = [P(c_dbl), P(c_dbl), c_i32, c_i32, c_dbl, c_i32, P(c_dbl), P(c_i32)]
        L.ed_band_eigs.argtypes = [P(c_dbl), c_i32, c_i32, c_i32, P(c_dbl), P(c_dbl), P(c_i32)]
        L.ed_expectation.argtypes = [c_vp, ctypes.c_int, c_vp, c_i32, c_vp, P(c_dbl)]
        L.ed_time_evolve.argtypes = [c_vp, ctypes.c_int, c_vp, c_dbl, c_i32, c_vp, P(c_dbl), P(c_i32)]
        L.ed_restrict.argtypes = [c_vp, c_vp, ctypes.c_int, c_vp, c_vp, c_i32, c_vp]
        L.ed_apply_sz.argtypes = [c_vp, c_vp, P(c_dbl), ctypes.c_int, c_vp, c_vp, c_i32, c_vp]
        L.ed_lanczos_tridiag.argtypes = [c_vp, ctypes.c_int, c_vp, c_i32, c_i32, c_vp, P(c_dbl), P(c_dbl), P(c_dbl),
                                         P(c_i32)]
        L.ed_batch_free.argtypes = [c_vp]
        L.ed_batch_free.restype = None
        L.ed_lanczos_batch.argtypes = [c_vp, P(ed_block_lanczos_opts), P(c_dbl), P(ed_block_lanczos_report), c_vp]
        for f in ("ed_batch_create", "ed_batch_rows", "ed_apply_batch", "ed_batch_autotune", "ed_lanczos_batch"):
            getattr(L, f).restype = ctypes.c_int
        L.ed_last_error.restype = ctypes.c_char_p
        L.ed_version.restype = ctypes.c_char_p
        for f in ("ed_basis_build", "ed_basis_dim", "ed_basis_export", "ed_sector_tables", "ed_hamiltonian_create",
                  "ed_hamiltonian_is_real", "ed_apply", "ed_apply_counters", "ed_apply_autotune",
                  "ed_apply_set_blocks", "ed_lanczos", "ed_tridiag_eigs", "ed_expectation",
                  "ed_time_evolve", "ed_restrict", "ed_apply_sz", "ed_lanczos_tridiag", "ed_hamiltonian_store",
                  "ed_hamiltonian_store_info", "ed_hamiltonian_store_autotune", "ed_basis_build_sun",
                  "ed_hamiltonian_create_sun"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def check(status: int):
    if status != 0:
        raise EdError(status, lib().ed_last_error().decode())


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(P(ct))


def _stream_handle(stream) -> int | None:
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream))


def _sector_struct(sector):
    perm = np.ascontiguousarray(sector.perm, dtype=np.int32)
    flip = np.ascontiguousarray(sector.spinflip, dtype=np.uint8)
    chi = np.asarray(sector.chi, dtype=complex)
    chi2 = np.ascontiguousarray(np.stack([chi.real, chi.imag], axis=1), dtype=np.float64)
    s = ed_sector(int(sector.n_sites), int(sector.n_up), int(len(perm)), _ptr(perm, c_i32), _ptr(flip, c_u8),
                  _ptr(chi2, c_dbl), int(sector.n_sublat))
    return s, [perm, flip, chi2]


def tridiag_eigs(alpha, beta, k, eps_vectors=2.0 ** -53, filter=True):
    """ed_tridiag_eigs: lowest k eigenvalues of the T-matrix (host only)."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    if len(b) < max(0, len(a) - 1):
        raise ValueError("beta needs n-1 entries")
    out = np.zeros(k, np.float64)
    nf = c_i32()
    check(lib().ed_tridiag_eigs(_ptr(a, c_dbl), _ptr(b, c_dbl), len(a), k, eps_vectors, int(filter),
                                _ptr(out, c_dbl), ctypes.byref(nf)))
    return out[:nf.value]


def band_eigs(band, k, vectors=True):
    """ed_band_eigs: lowest k eigenpairs of a Hermitian band matrix given by its lower
    band (complex array [n][bw+1], entry (i, q) = T[i][i-q]); host only.  Returns
    (eigenvalues, eigenvectors as rows or None)."""
    L = np.asarray(band, dtype=np.complex128)
    n, w = L.shape
    buf = np.ascontiguousarray(np.stack([L.real, L.imag], axis=-1), dtype=np.float64)
    ev = np.zeros(k, np.float64)
    vec = np.zeros((k, n, 2), np.float64) if vectors else None
    nf = c_i32()
    check(lib().ed_band_eigs(_ptr(buf, c_dbl), n, w - 1, k, _ptr(ev, c_dbl),
                             _ptr(vec, c_dbl) if vectors else None, ctypes.byref(nf)))
    m = nf.value
    return ev[:m], (vec[:m, :, 0] + 1j * vec[:m, :, 1]) if vectors else None


def sector_tables(sector) -> dict:
    """ed_sector_tables: host-side validation and sublattice-coding tables (no GPU needed)."""
    s, keep = _sector_struct(sector)
    N, n_sub, G = int(sector.n_sites), int(sector.n_sublat), int(len(keep[0]))
    m = N // n_sub if n_sub else 0
    n = c_i64()
    check(lib().ed_sector_tables(ctypes.byref(s), None, None, None, ctypes.byref(n), None, None))
    S = 1 << m
    rep = np.zeros(n_sub * S, np.uint16)
    off = np.zeros(n_sub * (S + 1), np.uint32)
    ids = np.zeros(max(n.value, 1), np.uint16)
    sa = np.zeros(G * n_sub * S, np.uint16)
    dest = np.zeros(G * n_sub, np.uint8)
    check(lib().ed_sector_tables(ctypes.byref(s), _ptr(rep, c_u16), _ptr(off, c_u32), _ptr(ids, c_u16),
                                 ctypes.byref(n), _ptr(sa, c_u16), _ptr(dest, c_u8)))
    return dict(m=m, rep=rep.reshape(n_sub, S), sym_off=off.reshape(n_sub, S + 1), sym_ids=ids[:n.value],
                sa=sa.reshape(G, n_sub, S), dest=dest.reshape(G, n_sub))


def representatives(sector, states):
    """ed_representatives: (rep, g, |Stab rep|, compatible) of each state, computed on the device."""
    sec, keep = _sector_struct(sector)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    n = len(st)
    rep = np.zeros(n, np.uint64)
    g = np.zeros(n, np.int32)
    ns = np.zeros(n, np.int32)
    cp = np.zeros(n, np.uint8)
    check(lib().ed_representatives(ctypes.byref(sec), _ptr(st, c_u64), n, _ptr(rep, c_u64), _ptr(g, c_i32),
                                   _ptr(ns, c_i32), _ptr(cp, c_u8)))
    return rep, g, ns, cp.astype(bool)


class Basis:
    """ed_basis_build / ed_basis_dim / ed_basis_export / ed_basis_free."""

    def __init__(self, sector, stream=None):
        self._sec, self._keep = _sector_struct(sector)
        self.n_sites = int(sector.n_sites)
        self.handle = c_vp()
        check(lib().ed_basis_build(ctypes.byref(self._sec), None, _stream_handle(stream), ctypes.byref(self.handle)))
        d = c_i64()
        check(lib().ed_basis_dim(self.handle, ctypes.byref(d)))
        self.dim = int(d.value)

    def export(self):
        reps = np.zeros(self.dim, dtype=np.uint64)
        stab = np.zeros(self.dim, dtype=np.uint16)
        check(lib().ed_basis_export(self.handle, _ptr(reps, c_u64), _ptr(stab, c_u16)))
        return reps, stab

    def restrict_to(self, sub: "Basis", x, y=None, stream=None):
        """ed_restrict: the vectors x (torch CUDA tensor [D] or [nvec, D] in this
        basis) written in the basis `sub` of a subgroup's sector whose characters
        are this sector's restricted to the subgroup.  Returns y (allocated when
        not given: same dtype, last dimension sub.dim)."""
        import torch
        dt = {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64, torch.complex128: ED_C128}[x.dtype]
        if not x.is_cuda or not x.is_contiguous() or x.shape[-1] != self.dim:
            raise ValueError("x must be a contiguous CUDA tensor with last dimension = basis dimension")
        shape = tuple(x.shape[:-1]) + (sub.dim,)
        if y is None:
            y = torch.empty(shape, dtype=x.dtype, device=x.device)
        elif y.dtype != x.dtype or tuple(y.shape) != shape or not y.is_cuda or not y.is_contiguous():
            raise ValueError("y must be a contiguous CUDA tensor of x's dtype with last dimension = sub.dim")
        nvec = 1 if x.dim() == 1 else x.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        check(lib().ed_restrict(self.handle, sub.handle, dt, x.data_ptr(), y.data_ptr(), nvec, _stream_handle(stream)))
        return y

    def apply_sz(self, to: "Basis", c, x, y=None, stream=None):
        """ed_apply_sz: y = (sum_i c_i S^z_i) x from this sector into the sector of
        `to` (same group; characters multiplied by the operator's phases).  c:
        complex [n_sites]; x: torch CUDA tensor [D] or [nvec, D].  Returns y."""
        import torch
        dt = {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64, torch.complex128: ED_C128}[x.dtype]
        if not x.is_cuda or not x.is_contiguous() or x.shape[-1] != self.dim:
            raise ValueError("x must be a contiguous CUDA tensor with last dimension = basis dimension")
        cc = np.asarray(c, dtype=complex)
        if cc.shape != (self.n_sites,):
            raise ValueError("c must have one coefficient per site")
        c2 = np.ascontiguousarray(np.stack([cc.real, cc.imag], axis=1), dtype=np.float64)
        shape = tuple(x.shape[:-1]) + (to.dim,)
        if y is None:
            y = torch.empty(shape, dtype=x.dtype, device=x.device)
        elif y.dtype != x.dtype or tuple(y.shape) != shape or not y.is_cuda or not y.is_contiguous():
            raise ValueError("y must be a contiguous CUDA tensor of x's dtype with last dimension = to.dim")
        nvec = 1 if x.dim() == 1 else x.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        check(lib().ed_apply_sz(self.handle, to.handle, _ptr(c2, c_dbl), dt, x.data_ptr(), y.data_ptr(), nvec,
                                _stream_handle(stream)))
        return y

    def close(self):
        if self.handle:
            lib().ed_basis_free(self.handle)
            self.handle = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BasisSUN(Basis):
    """ed_basis_build_sun: the basis of an SU(N) sector (colours packed in
    ceil(log2 n_colors) bits per site; export() returns the packed words)."""

    def __init__(self, sector, stream=None):
        perm = np.ascontiguousarray(sector.perm, dtype=np.int32)
        counts = np.ascontiguousarray(sector.counts, dtype=np.int32)
        chi = np.asarray(sector.chi, dtype=complex)
        chi2 = np.ascontiguousarray(np.stack([chi.real, chi.imag], axis=1), dtype=np.float64)
        self._sec = ed_sector_sun(int(sector.n_sites), int(sector.n_colors), _ptr(counts, c_i32), int(len(perm)),
                                  _ptr(perm, c_i32), _ptr(chi2, c_dbl), int(sector.n_sublat))
        self._keep = [perm, counts, chi2]
        self.n_sites = int(sector.n_sites)
        self.n_colors = int(sector.n_colors)
        self.handle = c_vp()
        check(lib().ed_basis_build_sun(ctypes.byref(self._sec), None, _stream_handle(stream),
                                       ctypes.byref(self.handle)))
        d = c_i64()
        check(lib().ed_basis_dim(self.handle, ctypes.byref(d)))
        self.dim = int(d.value)


class Hamiltonian:
    """ed_hamiltonian_create / ed_apply / ed_lanczos (ed_hamiltonian_create_sun for an SU(N) basis)."""

    def __init__(self, basis: Basis, terms, max_bytes: int | None = None, stream=None):
        self.basis = basis
        bonds = np.ascontiguousarray(np.asarray(terms.bonds, dtype=np.int32).reshape(-1, 2))
        J = np.ascontiguousarray(terms.J, dtype=np.float64)
        tris = np.ascontiguousarray(np.asarray(terms.tris, dtype=np.int32).reshape(-1, 3))
        Jc = np.ascontiguousarray(terms.Jchi, dtype=np.float64)
        self._keep = [bonds, J, tris, Jc]
        t = ed_terms(len(bonds), _ptr(bonds, c_i32), _ptr(J, c_dbl), len(tris), _ptr(tris, c_i32), _ptr(Jc, c_dbl))
        self.handle = c_vp()
        if isinstance(basis, BasisSUN):
            lim = (1 << 63) if max_bytes is None else int(max_bytes)
            check(lib().ed_hamiltonian_create_sun(basis.handle, ctypes.byref(t), lim, _stream_handle(stream),
                                                  ctypes.byref(self.handle)))
        else:
            check(lib().ed_hamiltonian_create(basis.handle, ctypes.byref(t), ctypes.byref(self.handle)))
        r = c_i32()
        check(lib().ed_hamiltonian_is_real(self.handle, ctypes.byref(r)))
        self.is_real = bool(r.value)

    @property
    def dim(self) -> int:
        return self.basis.dim

    def apply_ptr(self, dtype: int, x_ptr: int, y_ptr: int, nvec: int = 1, stream=None):
        check(lib().ed_apply(self.handle, dtype, x_ptr, y_ptr, nvec, _stream_handle(stream)))

    def apply(self, x, y, stream=None):
        """y = H x for torch CUDA tensors of shape [D] or [nvec, D] (contiguous)."""
        import torch
        dt = {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64, torch.complex128: ED_C128}[x.dtype]
        if x.dtype != y.dtype or x.shape != y.shape or not x.is_cuda or not y.is_cuda:
            raise ValueError("x and y must be CUDA tensors of the same dtype and shape")
        if not (x.is_contiguous() and y.is_contiguous()) or x.shape[-1] != self.dim:
            raise ValueError("x and y must be contiguous with last dimension = basis dimension")
        nvec = 1 if x.dim() == 1 else x.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        self.apply_ptr(dt, x.data_ptr(), y.data_ptr(), nvec, stream)
        return y

    def evolve(self, psi, dt, m=30, stream=None):
        """ed_time_evolve: psi <- exp(-i H dt) psi in place (complex torch CUDA tensor [D]);
        returns (error estimate, Krylov dimension used)."""
        import torch
        dt_ = {torch.complex64: ED_C64, torch.complex128: ED_C128}[psi.dtype]
        if not psi.is_cuda or not psi.is_contiguous() or psi.numel() != self.dim:
            raise ValueError("psi must be a contiguous CUDA tensor of the basis dimension")
        if stream is None:
            stream = torch.cuda.current_stream(psi.device)
        err = c_dbl()
        mu = c_i32()
        check(lib().ed_time_evolve(self.handle, dt_, psi.data_ptr(), float(dt), int(m), _stream_handle(stream),
                                   ctypes.byref(err), ctypes.byref(mu)))
        return float(err.value), int(mu.value)

    def expectation(self, x, stream=None, raw=False):
        """ed_expectation: <x|H|x> / <x|x> for a torch CUDA tensor of shape [D] or [nvec, D]
        (complex numpy array, one entry per vector); raw=True returns the pair
        (<x|H|x>, <x|x>) of arrays instead."""
        import torch
        dt = {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64, torch.complex128: ED_C128}[x.dtype]
        if not x.is_cuda or not x.is_contiguous() or x.shape[-1] != self.dim:
            raise ValueError("x must be a contiguous CUDA tensor with last dimension = basis dimension")
        nvec = 1 if x.dim() == 1 else x.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        out = np.zeros((nvec, 3), np.float64)
        check(lib().ed_expectation(self.handle, dt, x.data_ptr(), nvec, _stream_handle(stream), _ptr(out, c_dbl)))
        if raw:
            return out[:, 0] + 1j * out[:, 1], out[:, 2].copy()
        return (out[:, 0] + 1j * out[:, 1]) / out[:, 2]

    def lanczos_tridiag(self, x, m, reorth=False, stream=None):
        """ed_lanczos_tridiag: (alpha, beta, <x|x>) of the Lanczos recursion started
        from the torch CUDA tensor x [D]; len(alpha) = len(beta) = steps taken."""
        import torch
        dt = {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64, torch.complex128: ED_C128}[x.dtype]
        if not x.is_cuda or not x.is_contiguous() or x.numel() != self.dim:
            raise ValueError("x must be a contiguous CUDA tensor of the basis dimension")
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        a = np.zeros(int(m), np.float64)
        b = np.zeros(int(m), np.float64)
        n2 = c_dbl()
        mu = c_i32()
        check(lib().ed_lanczos_tridiag(self.handle, dt, x.data_ptr(), int(m), 1 if reorth else 0,
                                       _stream_handle(stream), _ptr(a, c_dbl), _ptr(b, c_dbl), ctypes.byref(n2),
                                       ctypes.byref(mu)))
        k = int(mu.value)
        return a[:k].copy(), b[:k].copy(), float(n2.value)

    def autotune(self, x, y, stream=None):
        """ed_apply_autotune on torch CUDA tensors shaped as for apply(); returns blocks per SM."""
        import torch
        dt = {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64, torch.complex128: ED_C128}[x.dtype]
        nvec = 1 if x.dim() == 1 else x.shape[0]
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        b = c_i32()
        check(lib().ed_apply_autotune(self.handle, dt, x.data_ptr(), y.data_ptr(), nvec, _stream_handle(stream),
                                      ctypes.byref(b)))
        return int(b.value)

    def set_blocks(self, dtype: int, nvec: int, blocks: int):
        """ed_apply_set_blocks: resident blocks per SM for (dtype, nvec class); 0 = default."""
        check(lib().ed_apply_set_blocks(self.handle, dtype, nvec, blocks))

    def store(self, dtype=None, seg_log2: int = 0, max_bytes: int | None = None, stream=None) -> int:
        """ed_hamiltonian_store: keep H's structure on the device for later applies
        (segments sized for `dtype`, default the Hamiltonian's FP64 kind); returns
        its size in bytes.  max_bytes defaults to no limit."""
        if dtype is None:
            dtype = ED_F64 if self.is_real else ED_C128
        nb = ctypes.c_size_t()
        lim = (1 << 63) if max_bytes is None else int(max_bytes)
        check(lib().ed_hamiltonian_store(self.handle, int(dtype), int(seg_log2), lim, _stream_handle(stream),
                                         ctypes.byref(nb)))
        return int(nb.value)

    def store_autotune(self, dtype=None, max_bytes: int | None = None, stream=None) -> tuple[int, int]:
        """ed_hamiltonian_store_autotune: (chosen log2 segment size, bytes)."""
        if dtype is None:
            dtype = ED_F64 if self.is_real else ED_C128
        sl = c_i32()
        nb = ctypes.c_size_t()
        lim = (1 << 63) if max_bytes is None else int(max_bytes)
        check(lib().ed_hamiltonian_store_autotune(self.handle, int(dtype), lim, _stream_handle(stream),
                                                  ctypes.byref(sl), ctypes.byref(nb)))
        return int(sl.value), int(nb.value)

    def store_info(self) -> dict:
        e, s, c, b = c_i64(), c_i32(), c_i32(), ctypes.c_size_t()
        check(lib().ed_hamiltonian_store_info(self.handle, ctypes.byref(e), ctypes.byref(s), ctypes.byref(c),
                                              ctypes.byref(b)))
        return dict(entries=int(e.value), segments=int(s.value), codes=int(c.value), bytes=int(b.value))

    def store_set_lanes(self, lanes_per_row: int):
        """ed_hamiltonian_store_set_lanes: lanes per row of the one-vector stored pass (1, 2, 4, 8)."""
        check(lib().ed_hamiltonian_store_set_lanes(self.handle, int(lanes_per_row)))

    def store_schedule(self) -> dict:
        """ed_hamiltonian_store_schedule: log2 segment size and lanes per row (0, 0 without a structure)."""
        sl, ln = c_i32(), c_i32()
        check(lib().ed_hamiltonian_store_schedule(self.handle, ctypes.byref(sl), ctypes.byref(ln)))
        return dict(seg_log2=int(sl.value), lanes_per_row=int(ln.value))

    def store_free(self):
        lib().ed_hamiltonian_store_free(self.handle)

    def counters(self, stream=None):
        g = c_i64()
        s = c_i64()
        check(lib().ed_apply_counters(self.handle, _stream_handle(stream), ctypes.byref(g), ctypes.byref(s)))
        return int(g.value), int(s.value)

    def lanczos(self, n_eig=1, tol=1e-10, max_iter=300, dtype=None, reorth=True, seed=1, refine=False,
                check_every=1, evecs=None, stream=None, raise_on_nonconv=True, host_vectors=False):
        if dtype is None:
            dtype = ED_F64 if self.is_real else ED_C128
        refine = 40 if refine is True else int(refine)
        o = ed_lanczos_opts(dtype, n_eig, tol, max_iter, int(reorth), seed, refine, check_every, int(host_vectors))
        ev = (c_dbl * 8)()
        rep = ed_lanczos_report()
        ptr = None
        if evecs is not None:
            import torch
            want = {ED_F64: torch.float64, ED_F32: torch.float32, ED_C128: torch.complex128, ED_C64: torch.complex64}[dtype]
            if evecs.dtype != want or not evecs.is_contiguous() or evecs.numel() < n_eig * self.dim:
                raise ValueError(f"evecs must be a contiguous {want} tensor of n_eig x dim elements")
            ptr = evecs.data_ptr()
        st = lib().ed_lanczos(self.handle, ctypes.byref(o), ev, ptr, ctypes.byref(rep), _stream_handle(stream))
        if st != 0 and not (st == 11 and not raise_on_nonconv):
            check(st)
        return np.array(ev[:n_eig]), rep

    def close(self):
        if self.handle:
            lib().ed_hamiltonian_free(self.handle)
            self.handle = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def report_dict(rep: ed_lanczos_report, n: int) -> dict:
    return dict(iters=rep.iters, converged=bool(rep.converged), n_apply=rep.n_apply, ritz=list(rep.ritz[:n]),
                resid_bound=list(rep.resid_bound[:n]), refined=list(rep.refined[:n]),
                refined_resid=list(rep.refined_resid[:n]), seconds=rep.seconds)


class Batch:
    """ed_batch_create / ed_apply_batch / ed_batch_autotune / ed_lanczos_batch."""

    def __init__(self, hamiltonians):
        self.hs = list(hamiltonians)
        arr = (c_vp * len(self.hs))(*[h.handle for h in self.hs])
        self.handle = c_vp()
        check(lib().ed_batch_create(arr, len(self.hs), ctypes.byref(self.handle)))
        ro = np.zeros(len(self.hs) + 1, np.int64)
        check(lib().ed_batch_rows(self.handle, _ptr(ro, c_i64)))
        self.row_off = ro
        self.n = len(self.hs)
        self.total = int(ro[-1])
        self.is_real = all(h.is_real for h in self.hs)

    @staticmethod
    def _dt(x):
        import torch
        return {torch.float64: ED_F64, torch.float32: ED_F32, torch.complex64: ED_C64,
                torch.complex128: ED_C128}[x.dtype]

    def apply(self, x, y, nvec=1, stream=None):
        """y = H x for concatenated vectors (nvec per sector, column-major within a sector)."""
        import torch
        if x.numel() != nvec * self.total or y.numel() != x.numel() or x.dtype != y.dtype:
            raise ValueError("x, y must hold nvec * total rows of one dtype")
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        check(lib().ed_apply_batch(self.handle, self._dt(x), x.data_ptr(), y.data_ptr(), nvec, _stream_handle(stream)))
        return y

    def autotune(self, x, y, nvec=1, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(x.device)
        w = c_i32()
        check(lib().ed_batch_autotune(self.handle, self._dt(x), x.data_ptr(), y.data_ptr(), nvec,
                                      _stream_handle(stream), ctypes.byref(w)))
        return int(w.value)

    def lanczos(self, block=8, n_eig=3, tol=1e-10, max_iter=60, seed=1, use_graph=True, check_every=1,
                dtype=None, raise_on_nonconv=True, reorth=True):
        if dtype is None:
            dtype = ED_F64 if self.is_real else ED_C128
        o = ed_block_lanczos_opts(dtype, block, n_eig, tol, max_iter, seed, int(use_graph), check_every, int(reorth))
        ev = np.zeros(self.n * n_eig, np.float64)
        rep = ed_block_lanczos_report()
        st = lib().ed_lanczos_batch(self.handle, ctypes.byref(o), _ptr(ev, c_dbl), ctypes.byref(rep), None)
        if st != 0 and not (st == 11 and not raise_on_nonconv):
            check(st)
        return ev.reshape(self.n, n_eig), rep

    def close(self):
        if self.handle:
            lib().ed_batch_free(self.handle)
            self.handle = c_vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
