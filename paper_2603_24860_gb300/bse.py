"""Thin ctypes binding of the C ABI declared in include/bse.h.

Argument marshalling only: every step of the computation runs in the CUDA
library ``libbse_gb300.so``.  There is no fallback; if the library is
missing or a call fails, an exception is raised.

Device buffers are torch tensors (torch provides device memory and streams).
Matrices written by the library are column-major; the helpers below return
torch views indexed as [row, column].
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbse_gb300.so")

BSE_OK, BSE_EINVAL, BSE_ENOMEM, BSE_ECUDA, BSE_ESYMM, BSE_ETIMEOUT, BSE_EUNSUPPORTED, BSE_ESOLVER = (
    0, -1, -2, -3, -4, -5, -6, -7)
BSE_FP64, BSE_BF16_SPLIT, BSE_FP16_SPLIT, BSE_FP32 = 0, 1, 2, 3
BSE_TERM_DIAG, BSE_TERM_EXCHANGE, BSE_TERM_DIRECT, BSE_TERM_ALL = 1, 2, 4, 7
BSE_BANDS_CC, BSE_BANDS_VV, BSE_BANDS_CV = 0, 1, 2
BSE_SOLVER_AUTO, BSE_SOLVER_DENSE, BSE_SOLVER_TRIDIAG, BSE_SOLVER_TRIDIAG_BLOCKED = 0, 1, 2, 3
BSE_SOLVER_TRIDIAG_BLOCKED_DF = 4
BSE_SOLVER_TRIDIAG_TWOSTAGE = 5
BSE_IRREP_ALL = -1

_P32 = C.POINTER(C.c_int32)
_P64 = C.POINTER(C.c_int64)
_PD = C.POINTER(C.c_double)


class BseSystem(C.Structure):
    _fields_ = [
        ("lattice", C.c_double * 9), ("n_ops", C.c_int32), ("rot", _P32), ("tau", _PD),
        ("mesh", C.c_int32 * 3), ("nv", C.c_int32), ("nc", C.c_int32), ("npw_max", C.c_int32),
        ("npw", _P32), ("gk", _P32), ("coef", C.c_void_p), ("eps", C.c_void_p),
        ("ng_max", C.c_int32), ("ng", _P32), ("gq", _P32), ("w", C.c_void_p),
        ("eps_inf", C.c_double * 9), ("w_div", C.c_double), ("qhat", C.c_double * 3),
        ("scissor", C.c_double), ("spin_factor", C.c_int32), ("device_inputs", C.c_int32),
    ]


class BseTablesView(C.Structure):
    _fields_ = [
        ("n_ops", C.c_int32), ("nk", C.c_int32), ("n_stars", C.c_int32), ("n_irreps", C.c_int32),
        ("n_orbits", C.c_int32), ("n_product", C.c_int64),
        ("rotk", _P32), ("star_of_k", _P32), ("star_rep", _P32), ("s_k", _P32),
        ("class_of_op", _P32), ("chi", _P32), ("irrep_dim", _P32), ("bright", _P32),
        ("block_dim", _P64), ("orbit_of", _P32), ("w_div", C.c_double), ("partner_dim", _P64),
        ("fold", _P32), ("npw_max", C.c_int32), ("ng_max", C.c_int32), ("npw", _P32), ("gk", _P32),
        ("ng", _P32), ("gq", _P32),
    ]


class BseWork(C.Structure):
    _fields_ = [("rho", C.c_double), ("contract", C.c_double), ("project", C.c_double),
                ("exchange", C.c_double), ("k_pairs", C.c_int64), ("overlap", C.c_int64), ("tiles", C.c_int64),
                ("seeds", C.c_int64), ("rotated", C.c_int64), ("rotate", C.c_double)]


class BseStats(C.Structure):
    _fields_ = [("launches", C.c_int64), ("direct_launches", C.c_int64), ("ms_direct", C.c_float),
                ("ms_project", C.c_float), ("ms_exchange", C.c_float), ("ms_eig", C.c_float),
                ("ms_spectrum", C.c_float), ("ms_create", C.c_float), ("ms_create_tables", C.c_float),
                ("ms_create_upload", C.c_float), ("ms_create_gamma", C.c_float), ("ms_create_wdiv", C.c_float),
                ("ms_basis", C.c_float), ("solver", C.c_int32), ("ms_reduce", C.c_float),
                ("ms_rotate", C.c_float), ("reduce_kind", C.c_int32),
                ("tc_pairs_per_cta", C.c_int32), ("pad_", C.c_int32)]


EXPORTS = {
    "bse_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(BseSystem), C.c_void_p]),
    "bse_destroy": (C.c_int, [C.c_void_p]),
    "bse_last_error": (C.c_char_p, []),
    "bse_tables": (C.c_int, [C.c_void_p, C.POINTER(BseTablesView)]),
    "bse_pairdens": (C.c_int, [C.c_void_p, _P32, _P32, C.c_int64, C.c_int32, C.c_int32, C.c_void_p]),
    "bse_build_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_uint32, C.c_void_p, C.c_int64]),
    "bse_build_full": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p, C.c_int64]),
    "bse_block_basis": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64]),
    "bse_dipoles": (C.c_int, [C.c_void_p, C.c_void_p]),
    "bse_block_spectrum": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                     C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bse_sync": (C.c_int, [C.c_void_p]),
    "bse_build_work": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.POINTER(BseWork)]),
    "bse_build_partner_block": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_uint32, C.c_void_p, C.c_int64]),
    "bse_partner_spectrum": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                       C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    "bse_set_timing": (C.c_int, [C.c_void_p, C.c_int32]),
    "bse_get_stats": (C.c_int, [C.c_void_p, C.POINTER(BseStats)]),
    "bse_head_correction_noalloc": (C.c_int, [_PD, _P32, _PD, C.c_void_p, C.c_void_p]),
    "bse_block_star_columns": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, _P64]),
    "bse_set_solver": (C.c_int, [C.c_void_p, C.c_int32]),
    "bse_set_seeds": (C.c_int, [C.c_void_p, C.c_int32]),
    "bse_set_wait_limit": (C.c_int, [C.c_void_p, C.c_int64]),
    "bse_loss_spectrum": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_double,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "bse_block_dim": (C.c_int, [C.c_void_p, C.c_int32, _P64]),
    "bse_block_spectrum_lanczos": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int64, C.c_int32,
                                             C.c_void_p, C.c_int64, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p,
                                             _P32]),
    "bse_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int32, _P32, _P32, C.c_int32,
                                   C.c_uint32, C.POINTER(C.c_void_p), _P64]),
    "bse_batch_run": (C.c_int, [C.c_void_p]),
    "bse_batch_kernels": (C.c_int, [C.c_void_p, _P64]),
    "bse_batch_tuning": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64]),
    "bse_batch_destroy": (C.c_int, [C.c_void_p]),
    "bse_build_blocks_batched": (C.c_int, [C.POINTER(C.c_void_p), C.c_int32, _P32, _P32, C.c_int32, C.c_uint32,
                                           C.POINTER(C.c_void_p), _P64]),
    "bse_build_blocks_work": (C.c_int, [C.c_void_p, C.c_int32, _P32, _P32, C.POINTER(BseWork)]),
    "bse_build_blocks": (C.c_int, [C.c_void_p, C.c_int32, _P32, _P32, C.c_int32, C.c_uint32,
                                   C.POINTER(C.c_void_p), _P64]),
}

_lib = None


def lib():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbse_gb300.so is not built; run __graft_entry__.build() first")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class BseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("bse error %d: %s" % (code, msg))
        self.code = code


def _check(code):
    if code != BSE_OK:
        raise BseError(code, lib().bse_last_error().decode())


def _ptr(t):
    """Device (torch) or host (numpy) buffer address."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return C.c_void_p(t.ctypes.data)


def _stream_handle(stream):
    if stream is None:
        return None
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


class Context:
    """An opened bse_ctx; keeps the host arrays of the system alive."""

    def __init__(self, handle, keep):
        self.handle = handle
        self._keep = keep

    def __del__(self):
        try:
            bse_destroy(self)
        except Exception:
            pass


def bse_create(inputs: dict, stream=None, device=None, w_div: float | None = None) -> Context:
    """Open a context from an input dictionary (see synth.generate).

    device: optional dict with torch CUDA tensors for 'coef', 'eps' and 'w'
    (already resident); otherwise the host arrays of ``inputs`` are copied.
    """
    keep = {}

    def arr(name, dtype):
        a = np.ascontiguousarray(inputs[name], dtype=dtype)
        keep[name] = a
        return a

    rot = arr("rot", np.int32)
    tau = arr("tau", np.float64)
    npw = arr("nk_count", np.int32)
    gk = arr("gk", np.int32)
    ng = arr("ng_count", np.int32)
    gq = arr("gq", np.int32)
    s = BseSystem()
    s.lattice[:] = [float(x) for x in np.asarray(inputs["lattice"], dtype=np.float64).ravel()]
    s.n_ops = len(rot)
    s.rot = rot.ctypes.data_as(_P32)
    s.tau = tau.ctypes.data_as(_PD)
    s.mesh[:] = [int(x) for x in inputs["mesh"]]
    s.nv, s.nc = int(inputs["nv"]), int(inputs["nc"])
    s.npw_max = gk.shape[1]
    s.npw = npw.ctypes.data_as(_P32)
    s.gk = gk.ctypes.data_as(_P32)
    s.ng_max = gq.shape[1]
    s.ng = ng.ctypes.data_as(_P32)
    s.gq = gq.ctypes.data_as(_P32)
    if device is not None:
        keep["device"] = device
        s.coef = device["coef"].data_ptr()
        s.eps = device["eps"].data_ptr()
        s.w = device["w"].data_ptr()
        s.device_inputs = 1
    else:
        coef = arr("coef", np.complex128)
        eps = arr("eps", np.float64)
        w = arr("w", np.complex128)
        s.coef = coef.ctypes.data
        s.eps = eps.ctypes.data
        s.w = w.ctypes.data
        s.device_inputs = 0
    s.eps_inf[:] = [float(x) for x in np.asarray(inputs["eps_inf"], dtype=np.float64).ravel()]
    s.w_div = math.nan if w_div is None else float(w_div)
    s.qhat[:] = [float(x) for x in inputs["qhat"]]
    s.scissor = float(inputs["scissor"])
    s.spin_factor = int(inputs["spin_factor"])
    h = C.c_void_p()
    _check(lib().bse_create(C.byref(h), C.byref(s), _stream_handle(stream)))
    return Context(h, keep)


def bse_destroy(ctx: Context):
    if ctx.handle is not None and ctx.handle.value:
        _check(lib().bse_destroy(ctx.handle))
    ctx.handle = None


def bse_tables(ctx: Context) -> dict:
    """Copies of the integer tables (and W^div)."""
    v = BseTablesView()
    _check(lib().bse_tables(ctx.handle, C.byref(v)))
    def get(p, n, shape=None):
        a = np.ctypeslib.as_array(p, shape=(n,)).copy()
        return a.reshape(shape) if shape else a
    ni, no, nk = v.n_irreps, v.n_ops, v.nk
    return dict(
        n_ops=no, nk=nk, n_stars=v.n_stars, n_irreps=ni, n_orbits=v.n_orbits, n_product=v.n_product,
        rotk=get(v.rotk, no * nk, (no, nk)), star_of_k=get(v.star_of_k, nk), star_rep=get(v.star_rep, v.n_stars),
        s_k=get(v.s_k, nk), class_of_op=get(v.class_of_op, no), chi=get(v.chi, ni * no, (ni, no)),
        irrep_dim=get(v.irrep_dim, ni), bright=get(v.bright, ni), block_dim=get(v.block_dim, ni),
        orbit_of=get(v.orbit_of, v.n_product), w_div=v.w_div, partner_dim=get(v.partner_dim, ni),
        fold=get(v.fold, no * nk * 3, (no, nk, 3)), npw=get(v.npw, nk), gk=get(v.gk, nk * v.npw_max * 3,
                                                                               (nk, v.npw_max, 3)),
        ng=get(v.ng, nk), gq=get(v.gq, nk * v.ng_max * 3, (nk, v.ng_max, 3)))


def bse_pairdens(ctx: Context, k, kp, bands: int, out, prec: int = BSE_FP64):
    """rho for pairs (k[i], kp[i]) into the CUDA tensor out [npairs, n, n',
    ng_max]: complex128 for BSE_FP64, complex64 for the mixed precisions."""
    k = np.ascontiguousarray(k, dtype=np.int32)
    kp = np.ascontiguousarray(kp, dtype=np.int32)
    assert len(k) == len(kp)
    _check(lib().bse_pairdens(ctx.handle, k.ctypes.data_as(_P32), kp.ctypes.data_as(_P32), len(k), bands, prec,
                              _ptr(out)))
    return out


def bse_build_block(ctx: Context, irrep: int, prec: int, terms: int, out, ld: int):
    """H_mu into ``out`` (complex128 CUDA tensor of >= ld*dim elements,
    column-major with leading dimension ld)."""
    _check(lib().bse_build_block(ctx.handle, irrep, prec, terms, _ptr(out), ld))
    return out


def bse_build_partner_block(ctx: Context, irrep: int, prec: int, terms: int, out, ld: int):
    """H_mu^(1) (partner block) into ``out``, column-major with leading dimension ld."""
    _check(lib().bse_build_partner_block(ctx.handle, irrep, prec, terms, _ptr(out), ld))
    return out


def bse_build_blocks(ctx: Context, irreps, partners, prec: int, terms: int, outs, lds):
    """Several blocks in one build (one direct pass shared by all targets);
    ``outs`` are device buffers (or None for an empty block)."""
    n = len(irreps)
    ir = np.ascontiguousarray(irreps, dtype=np.int32)
    pa = None if partners is None else np.ascontiguousarray(partners, dtype=np.int32)
    ptrs = (C.c_void_p * max(n, 1))(*[_ptr(o) if o is not None else None for o in outs])
    ld = np.ascontiguousarray(lds, dtype=np.int64)
    _check(lib().bse_build_blocks(ctx.handle, n, ir.ctypes.data_as(_P32),
                                  None if pa is None else pa.ctypes.data_as(_P32), prec, terms, ptrs,
                                  ld.ctypes.data_as(_P64)))
    return outs


class Batch:
    """A planned batched build (bse_batch_create); keeps its contexts and
    outputs referenced."""

    def __init__(self, handle, ctxs, outs):
        self.handle, self.ctxs, self.outs = handle, ctxs, outs


def _batch_args(ctxs, irreps, partners, outs, lds):
    n = len(ctxs)
    hs = (C.c_void_p * n)(*[c.handle for c in ctxs])
    ir = np.ascontiguousarray(irreps, dtype=np.int32)
    pa = None if partners is None else np.ascontiguousarray(partners, dtype=np.int32)
    ptrs = (C.c_void_p * n)(*[_ptr(o) if o is not None else None for o in outs])
    ld = np.ascontiguousarray(lds, dtype=np.int64)
    return n, hs, ir, pa, ptrs, ld


def bse_batch_create(ctxs, irreps, partners, prec: int, terms: int, outs, lds) -> Batch:
    n, hs, ir, pa, ptrs, ld = _batch_args(ctxs, irreps, partners, outs, lds)
    h = C.c_void_p()
    _check(lib().bse_batch_create(C.byref(h), hs, n, ir.ctypes.data_as(_P32),
                                  None if pa is None else pa.ctypes.data_as(_P32), prec, terms, ptrs,
                                  ld.ctypes.data_as(_P64)))
    return Batch(h, list(ctxs), list(outs))


def bse_batch_run(batch: Batch):
    _check(lib().bse_batch_run(batch.handle))


def bse_batch_kernels(batch: Batch) -> int:
    v = C.c_int64()
    _check(lib().bse_batch_kernels(batch.handle, C.byref(v)))
    return v.value


def bse_batch_tuning(batch: Batch) -> dict:
    """The autotuner's choices for the batch (JSON from the library)."""
    import json as _json
    buf = C.create_string_buffer(8192)
    _check(lib().bse_batch_tuning(batch.handle, buf, len(buf)))
    return _json.loads(buf.value.decode())


def bse_batch_destroy(batch: Batch):
    if batch.handle:
        _check(lib().bse_batch_destroy(batch.handle))
        batch.handle = None


def bse_build_blocks_batched(ctxs, irreps, partners, prec: int, terms: int, outs, lds):
    n, hs, ir, pa, ptrs, ld = _batch_args(ctxs, irreps, partners, outs, lds)
    _check(lib().bse_build_blocks_batched(hs, n, ir.ctypes.data_as(_P32),
                                          None if pa is None else pa.ctypes.data_as(_P32), prec, terms, ptrs,
                                          ld.ctypes.data_as(_P64)))
    return outs


def bse_partner_spectrum(ctx: Context, irrep: int, h, ld: int, omega, eta: float, omega_out, osc, im_eps):
    _check(lib().bse_partner_spectrum(ctx.handle, irrep, _ptr(h), ld, _ptr(omega), omega.numel(), eta,
                                      _ptr(omega_out), _ptr(osc), _ptr(im_eps)))


def bse_block_spectrum_lanczos(ctx: Context, irrep: int, partner: bool, h, ld: int, steps: int, omega, eta: float,
                               ritz, weights, im_eps) -> int:
    """Returns the number of Lanczos steps performed."""
    done = np.zeros(1, dtype=np.int32)
    _check(lib().bse_block_spectrum_lanczos(ctx.handle, irrep, 1 if partner else 0, _ptr(h), ld, steps, _ptr(omega),
                                            omega.numel(), eta, _ptr(ritz), _ptr(weights), _ptr(im_eps),
                                            done.ctypes.data_as(_P32)))
    return int(done[0])


def bse_block_star_columns(ctx: Context, irrep: int, partner: bool = False):
    """Column range [out[a], out[a+1]) of each k star in the (partner) block."""
    n = int(bse_tables(ctx)["n_stars"])
    out = np.zeros(n + 1, dtype=np.int64)
    _check(lib().bse_block_star_columns(ctx.handle, irrep, 1 if partner else 0, out.ctypes.data_as(_P64)))
    return out


def bse_build_full(ctx: Context, terms: int, out, ld: int):
    _check(lib().bse_build_full(ctx.handle, terms, _ptr(out), ld))
    return out


def bse_block_basis(ctx: Context, irrep: int, out, ld: int):
    _check(lib().bse_block_basis(ctx.handle, irrep, _ptr(out), ld))
    return out


def bse_dipoles(ctx: Context, out):
    _check(lib().bse_dipoles(ctx.handle, _ptr(out)))
    return out


def bse_block_spectrum(ctx: Context, irrep: int, h, ld: int, omega, eta: float, omega_out, osc, im_eps):
    _check(lib().bse_block_spectrum(ctx.handle, irrep, _ptr(h), ld, _ptr(omega), omega.numel(), eta,
                                    _ptr(omega_out), _ptr(osc), _ptr(im_eps)))


def bse_sync(ctx: Context):
    _check(lib().bse_sync(ctx.handle))


def bse_build_work(ctx: Context, irrep: int, partner: bool = False) -> dict:
    w = BseWork()
    _check(lib().bse_build_work(ctx.handle, irrep, 1 if partner else 0, C.byref(w)))
    return {f: getattr(w, f) for f, _ in BseWork._fields_}


def bse_build_blocks_work(ctx: Context, irreps, partners=None) -> dict:
    ir = np.ascontiguousarray(irreps, dtype=np.int32)
    pa = None if partners is None else np.ascontiguousarray(partners, dtype=np.int32)
    w = BseWork()
    _check(lib().bse_build_blocks_work(ctx.handle, len(ir), ir.ctypes.data_as(_P32),
                                       None if pa is None else pa.ctypes.data_as(_P32), C.byref(w)))
    return {f: getattr(w, f) for f, _ in BseWork._fields_}


def bse_block_dim(ctx: Context, irrep: int) -> int:
    v = C.c_int64()
    _check(lib().bse_block_dim(ctx.handle, irrep, C.byref(v)))
    return v.value


def bse_loss_spectrum(ctx: Context, omega_levels, osc, omega, eta: float, omega_long, osc_long, loss):
    _check(lib().bse_loss_spectrum(ctx.handle, omega_levels.numel(), _ptr(omega_levels), _ptr(osc), _ptr(omega),
                                   omega.numel(), eta, _ptr(omega_long), _ptr(osc_long), _ptr(loss)))


def loss_spectrum(ctx: Context, omega_levels, osc, omega, eta: float):
    """(longitudinal levels, their strengths, -Im eps_M^-1(omega)) from the
    output of spectrum / partner_spectrum."""
    import torch
    n = omega_levels.numel()
    ol = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    ow = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    ls = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
    bse_loss_spectrum(ctx, omega_levels.contiguous(), osc.contiguous(), omega, eta, ol, ow, ls)
    return ol[:n], ow[:n], ls


def bse_set_seeds(ctx: Context, on: bool):
    _check(lib().bse_set_seeds(ctx.handle, 1 if on else 0))


def bse_set_wait_limit(ctx: Context, polls: int):
    _check(lib().bse_set_wait_limit(ctx.handle, polls))


def bse_set_solver(ctx: Context, solver: int):
    _check(lib().bse_set_solver(ctx.handle, solver))


def bse_set_timing(ctx: Context, on: bool):
    _check(lib().bse_set_timing(ctx.handle, 1 if on else 0))


def bse_get_stats(ctx: Context) -> dict:
    s = BseStats()
    _check(lib().bse_get_stats(ctx.handle, C.byref(s)))
    return {f: getattr(s, f) for f, _ in BseStats._fields_}


def bse_head_correction_noalloc(lattice, mesh, eps_inf, out, stream=None):
    """W^div into the one-element float64 CUDA tensor ``out`` using the
    library's fixed scratch (no device memory is allocated)."""
    lat = np.ascontiguousarray(lattice, dtype=np.float64).ravel()
    msh = np.ascontiguousarray(mesh, dtype=np.int32).ravel()
    ein = np.ascontiguousarray(eps_inf, dtype=np.float64).ravel()
    _check(lib().bse_head_correction_noalloc(lat.ctypes.data_as(_PD), msh.ctypes.data_as(_P32),
                                             ein.ctypes.data_as(_PD), _ptr(out), _stream_handle(stream)))
    return out


# ---------------------------------------------------------------------------
# conveniences (still marshalling only)
# ---------------------------------------------------------------------------

def colmajor(buf, rows: int, cols: int, ld: int):
    """View of a column-major (rows x cols, leading dim ld) matrix stored in a
    flat tensor, indexed [row, column]."""
    return buf[: ld * cols].view(cols, ld)[:, :rows].transpose(0, 1)


def block(ctx: Context, irrep: int, prec: int = BSE_FP64, terms: int = BSE_TERM_ALL):
    """Build H_mu and return it as a [dim, dim] complex128 CUDA view."""
    import torch
    dim = int(bse_tables(ctx)["block_dim"][irrep])
    buf = torch.empty(max(dim * dim, 1), dtype=torch.complex128, device="cuda")
    bse_build_block(ctx, irrep, prec, terms, buf, max(dim, 1))
    return colmajor(buf, dim, dim, max(dim, 1))


def partner_block(ctx: Context, irrep: int, prec: int = BSE_FP64, terms: int = BSE_TERM_ALL):
    """Build the partner block and return it as a [n, n] complex128 CUDA view."""
    import torch
    n = int(bse_tables(ctx)["partner_dim"][irrep])
    buf = torch.empty(max(n * n, 1), dtype=torch.complex128, device="cuda")
    bse_build_partner_block(ctx, irrep, prec, terms, buf, max(n, 1))
    return colmajor(buf, n, n, max(n, 1))


def blocks(ctx: Context, irreps=None, partner: bool = False, prec: int = BSE_FP64, terms: int = BSE_TERM_ALL):
    """Build the blocks of several irreps (default: all) in one pass; returns
    a list of [dim, dim] complex128 CUDA views in the order of ``irreps``."""
    import torch
    t = bse_tables(ctx)
    if irreps is None:
        irreps = list(range(int(t["n_irreps"])))
    dims = [int(t["partner_dim" if partner else "block_dim"][mu]) for mu in irreps]
    bufs = [torch.empty(max(n * n, 1), dtype=torch.complex128, device="cuda") for n in dims]
    bse_build_blocks(ctx, irreps, [int(partner)] * len(irreps), prec, terms, bufs, [max(n, 1) for n in dims])
    return [colmajor(b, n, n, max(n, 1)) for b, n in zip(bufs, dims)]


def partner_spectrum(ctx: Context, irrep: int, h, omega, eta: float):
    """(levels, oscillator strengths summed over partners, Im eps_M)."""
    import torch
    n = h.shape[0]
    ld = h.stride(1) if n else 1
    om = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    osc = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
    im = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
    bse_partner_spectrum(ctx, irrep, h, ld, omega, eta, om, osc, im)
    return om[:n], osc[:n], im


def lanczos_spectrum(ctx: Context, irrep: int, h, omega, eta: float, steps: int, partner: bool = False,
                     ritz: bool = True):
    """(Ritz values, Gauss weights, Im eps_M) of the Lanczos-Haydock spectrum
    of a block (or partner block) after at most `steps` steps; with
    ritz=False only Im eps_M (the first two are None)."""
    import torch
    n = h.shape[0]
    ld = h.stride(1) if n else 1
    rz = torch.empty(max(steps, 1), dtype=torch.float64, device="cuda") if ritz else None
    wt = torch.empty(max(steps, 1), dtype=torch.float64, device="cuda") if ritz else None
    im = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
    k = bse_block_spectrum_lanczos(ctx, irrep, partner, h, ld, steps, omega, eta, rz, wt, im)
    return (rz[:k], wt[:k], im) if ritz else (None, None, im)


def full(ctx: Context, terms: int = BSE_TERM_ALL):
    import torch
    n = int(bse_tables(ctx)["n_product"])
    buf = torch.empty(n * n, dtype=torch.complex128, device="cuda")
    bse_build_full(ctx, terms, buf, n)
    return colmajor(buf, n, n, n)


def basis(ctx: Context, irrep: int):
    import torch
    t = bse_tables(ctx)
    n, dim = int(t["n_product"]), int(t["block_dim"][irrep])
    buf = torch.empty(max(n * dim, 1), dtype=torch.complex128, device="cuda")
    bse_block_basis(ctx, irrep, buf, n)
    return colmajor(buf, n, dim, n)


def spectrum(ctx: Context, irrep: int, h, omega, eta: float):
    """(Omega, |B_lambda|^2, Im eps_M) of a block built by ``block``."""
    import torch
    dim = h.shape[0]
    ld = h.stride(1) if dim else 1
    om = torch.empty(max(dim, 1), dtype=torch.float64, device="cuda")
    osc = torch.empty(max(dim, 1), dtype=torch.float64, device="cuda")
    im = torch.empty(omega.numel(), dtype=torch.float64, device="cuda")
    hh = h.transpose(0, 1)   # underlying column-major storage
    bse_block_spectrum(ctx, irrep, hh, ld, omega, eta, om, osc, im)
    return om[:dim], osc[:dim], im
