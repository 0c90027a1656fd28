"""Python binding of liblaph (include/laph.h): argument marshalling only.

Every function has the name of its C entry point and forwards to it through
ctypes.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; complex128
arrays are passed as interleaved doubles.  The work runs in the CUDA library:
if liblaph.so is missing this module raises on import, there is no fallback.
"""
import ctypes
import os

import numpy as np

from .build import LIB

if not os.path.exists(LIB):
    raise ImportError(f"{LIB} is not built; run paper_1104_3870_gb300.build.build() (needs nvcc)")

_lib = ctypes.CDLL(LIB)

LAPH_OK, LAPH_ERR_ARG, LAPH_ERR_CUDA, LAPH_ERR_NOT_CONVERGED, LAPH_ERR_TIMEOUT, LAPH_ERR_NOMEM = range(6)
PLAIN_FP64, MIXED_FP32, MIXED_BF16, LEARNED = range(4)
CH_PION, CH_RHO, CH_SCALAR, CH_PIPI_I2 = range(4)
DIL_NONE, DIL_FULL, DIL_BLOCK, DIL_INTERLACE = range(4)
HOP_CLOVINV, HOP_CLOVINV_XPAY, HOP_APPLY = range(3)
PREC_FP64, PREC_FP32, PREC_BF16 = range(3)


class LaphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"liblaph error {code}: {msg}")
        self.code = code


class Lattice(ctypes.Structure):
    _fields_ = [("ns", ctypes.c_int), ("nt", ctypes.c_int), ("xi", ctypes.c_double)]


class DiracParams(ctypes.Structure):
    _fields_ = [("m0", ctypes.c_double), ("csw", ctypes.c_double)]


class SolverParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxiter", ctypes.c_int), ("mode", ctypes.c_int),
                ("rhs_block", ctypes.c_int), ("inner_tol", ctypes.c_double), ("fallback", ctypes.c_int),
                ("weights", ctypes.c_void_p), ("gcr_restart", ctypes.c_int), ("check_every", ctypes.c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("status", ctypes.c_int),
                ("fallback_used", ctypes.c_int), ("true_resid", ctypes.c_double)]


class EigParams(ctypes.Structure):
    _fields_ = [("lambda_L", ctypes.c_double), ("lambda_C", ctypes.c_double), ("cheb_order", ctypes.c_int),
                ("krylov_dim", ctypes.c_int), ("max_restarts", ctypes.c_int), ("tol", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class EigReport(ctypes.Structure):
    _fields_ = [("restarts", ctypes.c_int), ("matvecs", ctypes.c_int), ("nconv", ctypes.c_int),
                ("max_resid", ctypes.c_double), ("lambda_C", ctypes.c_double)]


class Dil1(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("J", ctypes.c_int)]


class Dilution(ctypes.Structure):
    _fields_ = [("T", Dil1), ("S", Dil1), ("L", Dil1)]


class CorrSpec(ctypes.Structure):
    _fields_ = [("channel", ctypes.c_int), ("t0", ctypes.c_int), ("nv", ctypes.c_int), ("dil", Dilution),
                ("nb", ctypes.c_int), ("b_list", ctypes.POINTER(ctypes.c_int))]


class PipiSpec(ctypes.Structure):
    _fields_ = [("iso", ctypes.c_int), ("iso3", ctypes.c_int), ("t0", ctypes.c_int), ("nv", ctypes.c_int),
                ("dil_fwd", Dilution), ("nb_fwd", ctypes.c_int), ("b_fwd", ctypes.POINTER(ctypes.c_int)),
                ("dil_smt", Dilution), ("nb_smt", ctypes.c_int), ("b_smt", ctypes.POINTER(ctypes.c_int))]


class BaryonSpec(ctypes.Structure):
    _fields_ = [("t0", ctypes.c_int), ("nv", ctypes.c_int), ("dil", Dilution), ("nb", ctypes.c_int),
                ("b_list", ctypes.POINTER(ctypes.c_int)), ("c_snk", ctypes.POINTER(ctypes.c_double)),
                ("c_src", ctypes.POINTER(ctypes.c_double)), ("flav_snk", ctypes.c_int * 3),
                ("flav_src", ctypes.c_int * 3)]


_vp = ctypes.c_void_p
_sig = {
    "laph_ctx_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_vp)]),
    "laph_ctx_destroy": (None, [_vp]),
    "laph_last_error": (ctypes.c_char_p, []),
    "laph_version": (ctypes.c_char_p, []),
    "laph_stout_smear": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_int, _vp]),
    "laph_eigvecs": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.c_int, ctypes.POINTER(EigParams),
                                    _vp, _vp, ctypes.POINTER(EigReport), _vp]),
    "laph_make_sources": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.c_int, ctypes.c_uint16,
                                         ctypes.c_uint16, ctypes.POINTER(Dilution), _vp, ctypes.c_int, _vp, _vp,
                                         _vp]),
    "dirac_solve_batch": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), _vp, _vp,
                                         ctypes.c_int, ctypes.POINTER(SolverParams), _vp, _vp]),
    "laph_dirac_apply": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), _vp, _vp,
                                        ctypes.c_int, _vp]),
    "laph_tuned_block": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "laph_dslash_eo": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, ctypes.c_int, _vp]),
    "laph_sinks": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.c_int, _vp, ctypes.c_int, _vp, _vp]),
    "correlate": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.POINTER(CorrSpec), _vp, _vp, _vp, _vp]),
    "correlate_noalloc": (ctypes.c_int, [ctypes.POINTER(Lattice), ctypes.POINTER(CorrSpec), _vp, _vp, _vp, _vp]),
    "laph_mom_overlaps": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.c_int, ctypes.c_int, _vp, _vp,
                                         _vp]),
    "correlate_mom": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.POINTER(CorrSpec), _vp, _vp, _vp, _vp,
                                     _vp]),
    "laph_meson_loops": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.POINTER(CorrSpec), _vp, _vp, _vp,
                                        ctypes.c_int, _vp, _vp]),
    "correlate_disconnected": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.c_int, ctypes.c_int, _vp, _vp,
                                              ctypes.c_double, ctypes.c_double, _vp, _vp]),
    "laph_displaced_overlaps": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, _vp, ctypes.c_int, _vp, ctypes.c_int,
                                               _vp, ctypes.c_int, _vp, _vp, _vp]),
    "correlate_pipi": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.POINTER(PipiSpec), _vp, _vp, _vp, _vp, _vp,
                                      _vp, _vp, _vp]),
    "laph_baryon_tensor": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.c_int, _vp, _vp, _vp]),
    "correlate_baryon": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), ctypes.POINTER(BaryonSpec), _vp, _vp, _vp, _vp,
                                        _vp]),
    "laph_precond_size": (ctypes.c_int, []),
    "laph_precond_init": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_double, _vp]),
    "laph_precond_train": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), _vp, _vp,
                                          ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _vp,
                                          _vp, ctypes.POINTER(ctypes.c_double), _vp]),
    "laph_precond_grad": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), _vp, _vp, _vp,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp, _vp]),
    "laph_precond_apply": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), _vp, _vp, _vp,
                                          ctypes.c_int, _vp]),
    "laph_precond_apply_tc": (ctypes.c_int, [_vp, ctypes.POINTER(Lattice), _vp, ctypes.POINTER(DiracParams), _vp, _vp, _vp,
                                          ctypes.c_int, _vp]),
    "laph_launch_count": (ctypes.c_long, []),
    "laph_profile_enable": (None, [ctypes.c_int]),
    "laph_profile_families": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_int]),
    "laph_profile_reset": (None, []),
    "laph_profile_read": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_long), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
}
_missing = [n for n in _sig if not hasattr(_lib, n)]
if _missing:
    raise ImportError(f"{LIB} lacks {', '.join(_missing)}: rebuild with paper_1104_3870_gb300.build")
for _name, (_res, _args) in _sig.items():
    f = getattr(_lib, _name)
    f.restype = _res
    f.argtypes = _args


def exported_symbols():
    return [n for n in _sig if hasattr(_lib, n)]


def _check(rc, allow=()):
    if rc != LAPH_OK and rc not in allow:
        raise LaphError(rc, _lib.laph_last_error().decode())
    return rc


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays passed to liblaph must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors passed to liblaph must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _stream(stream=None):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def lattice(ns, nt, xi):
    return Lattice(int(ns), int(nt), float(xi))


def dilution(T, S, L):
    return Dilution(Dil1(*T), Dil1(*S), Dil1(*L))


class Context:
    """Owns a laph_ctx (device workspace, autotune cache)."""

    def __init__(self, device=0):
        self.ptr = _vp()
        _check(_lib.laph_ctx_create(int(device), ctypes.byref(self.ptr)))

    def close(self):
        if self.ptr:
            _lib.laph_ctx_destroy(self.ptr)
            self.ptr = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def version():
    return _lib.laph_version().decode()


def laph_launch_count():
    return int(_lib.laph_launch_count())


def laph_profile_enable(level=1):
    """0: off; 1: time the Dirac stencil launches; 2: time every instrumented kernel family."""
    _lib.laph_profile_enable(int(level))


def laph_profile_families():
    buf = ctypes.create_string_buffer(4096)
    _lib.laph_profile_families(buf, 4096)
    return [f for f in buf.value.decode().split(",") if f]


def laph_profile_reset():
    _lib.laph_profile_reset()


def laph_profile_read(family):
    """(launches, total ms, algorithmic bytes, flops) of a kernel family timed with CUDA events."""
    n = ctypes.c_long()
    ms, b, f = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.laph_profile_read(family.encode(), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(b), ctypes.byref(f)))
    return n.value, ms.value, b.value, f.value


def laph_stout_smear(ctx, lat, links, rho, nsteps, spatial_only, stream=None):
    _check(_lib.laph_stout_smear(ctx.ptr, ctypes.byref(lat), _ptr(links), float(rho), int(nsteps),
                                 int(spatial_only), _stream(stream)))


def laph_eigvecs(ctx, lat, links3d, nv, evals, evecs, params=None, stream=None, allow_not_converged=False):
    rep = EigReport()
    rc = _lib.laph_eigvecs(ctx.ptr, ctypes.byref(lat), _ptr(links3d), int(nv),
                           ctypes.byref(params) if params is not None else None, _ptr(evals), _ptr(evecs),
                           ctypes.byref(rep), _stream(stream))
    _check(rc, allow=(LAPH_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return rep


def laph_make_sources(ctx, lat, evecs, nv, noise_id, config_id, dil, b_list, rhs, noise=None, stream=None):
    if hasattr(b_list, "data_ptr"):   # an int32 tensor, host or device, passed as it is
        if str(b_list.dtype) != "torch.int32":
            raise ValueError("b_list tensors must be int32")
        bptr, nb = _ptr(b_list), int(b_list.numel())
    else:
        b = np.ascontiguousarray(np.asarray(b_list, dtype=np.int32))
        bptr, nb = b.ctypes.data, len(b)
    _check(_lib.laph_make_sources(ctx.ptr, ctypes.byref(lat), _ptr(evecs), int(nv), int(noise_id), int(config_id),
                                  ctypes.byref(dil), bptr, nb, _ptr(rhs), _ptr(noise), _stream(stream)))


def solver_params(tol=1e-10, maxiter=100000, mode=MIXED_FP32, rhs_block=0, inner_tol=0.0, fallback=1,
                  weights=None, gcr_restart=16, check_every=0):
    return SolverParams(tol, maxiter, mode, rhs_block, inner_tol, fallback, _ptr(weights), gcr_restart, check_every)


def dirac_solve_batch(ctx, lat, links, m0, csw, rhs, sol, nrhs, params=None, stream=None, allow_not_converged=False):
    reps = (SolveReport * max(nrhs, 1))()
    prm = params if params is not None else solver_params()
    rc = _lib.dirac_solve_batch(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                                _ptr(rhs), _ptr(sol), int(nrhs), ctypes.byref(prm), reps, _stream(stream))
    _check(rc, allow=(LAPH_ERR_NOT_CONVERGED,) if allow_not_converged else ())
    return [reps[i] for i in range(nrhs)]


def laph_dirac_apply(ctx, lat, links, m0, csw, inp, out, nrhs, stream=None):
    _check(_lib.laph_dirac_apply(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                                 _ptr(inp), _ptr(out), int(nrhs), _stream(stream)))


def laph_tuned_block(ctx, vh, nmax):
    return int(_lib.laph_tuned_block(ctx.ptr, int(vh), int(nmax)))


def laph_dslash_eo(ctx, lat, links, m0, csw, parity, mode, precision, inp, z, out, nrhs, stream=None):
    _check(_lib.laph_dslash_eo(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                               int(parity), int(mode), int(precision), _ptr(inp), _ptr(z), _ptr(out), int(nrhs),
                               _stream(stream)))


def laph_sinks(ctx, lat, evecs, nv, sol, nrhs, coef, stream=None):
    _check(_lib.laph_sinks(ctx.ptr, ctypes.byref(lat), _ptr(evecs), int(nv), _ptr(sol), int(nrhs), _ptr(coef),
                           _stream(stream)))


def correlate(ctx, lat, channel, t0, nv, dil, b_list, coefs, noises, corr, stream=None):
    b = np.ascontiguousarray(np.asarray(b_list, dtype=np.int32))
    spec = CorrSpec(int(channel), int(t0), int(nv), dil, len(b), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    cp = (_vp * len(coefs))(*[_ptr(c) for c in coefs])
    npt = (_vp * len(noises))(*[_ptr(n) for n in noises])
    _check(_lib.correlate(ctx.ptr, ctypes.byref(lat), ctypes.byref(spec), cp, npt, _ptr(corr), _stream(stream)))


def laph_precond_size():
    return int(_lib.laph_precond_size())


def laph_precond_init(seed, diag, weights):
    _check(_lib.laph_precond_init(int(seed), float(diag), _ptr(weights)))


def laph_precond_train(ctx, lat, links, m0, csw, rho, phi, npairs, epochs, batch, lr, step0, weights, adam,
                       stream=None):
    loss = ctypes.c_double()
    _check(_lib.laph_precond_train(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                                   _ptr(rho), _ptr(phi), int(npairs), int(epochs), int(batch), float(lr), int(step0),
                                   _ptr(weights), _ptr(adam), ctypes.byref(loss), _stream(stream)))
    return loss.value


def laph_precond_grad(ctx, lat, links, m0, csw, weights, rho, phi, npairs, grad, stream=None):
    loss = ctypes.c_double()
    _check(_lib.laph_precond_grad(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                                  _ptr(weights), _ptr(rho), _ptr(phi), int(npairs), ctypes.byref(loss), _ptr(grad),
                                  _stream(stream)))
    return loss.value


def laph_precond_apply(ctx, lat, links, m0, csw, weights, inp, out, nrhs, stream=None):
    _check(_lib.laph_precond_apply(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                                   _ptr(weights), _ptr(inp), _ptr(out), int(nrhs), _stream(stream)))


def laph_precond_apply_tc(ctx, lat, links, m0, csw, weights, inp, out, nrhs, stream=None):
    _check(_lib.laph_precond_apply_tc(ctx.ptr, ctypes.byref(lat), _ptr(links), ctypes.byref(DiracParams(m0, csw)),
                                   _ptr(weights), _ptr(inp), _ptr(out), int(nrhs), _stream(stream)))


def correlate_noalloc(lat, channel, t0, nv, dil, b_list, coefs, noises, corr, stream=None):
    """correlate() without any GPU allocation: device arrays only, scratch in the
    library's fixed device array (see include/laph.h)."""
    b = np.ascontiguousarray(np.asarray(b_list, dtype=np.int32))
    spec = CorrSpec(int(channel), int(t0), int(nv), dil, len(b), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    cp = (_vp * len(coefs))(*[_ptr(c) for c in coefs])
    npt = (_vp * len(noises))(*[_ptr(n) for n in noises])
    _check(_lib.correlate_noalloc(ctypes.byref(lat), ctypes.byref(spec), cp, npt, _ptr(corr), _stream(stream)))


def _spec(channel, t0, nv, dil, b_list):
    b = np.ascontiguousarray(np.asarray(b_list, dtype=np.int32))
    return CorrSpec(int(channel), int(t0), int(nv), dil, len(b), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), b


def laph_mom_overlaps(ctx, lat, evecs, nv, moms, phi, stream=None):
    """phi[nmom][nt][nv][nv] = V^dag e^{-ip.x} V for the integer momenta in moms."""
    m = np.ascontiguousarray(np.asarray(moms, dtype=np.int32).reshape(-1, 3))
    _check(_lib.laph_mom_overlaps(ctx.ptr, ctypes.byref(lat), _ptr(evecs), int(nv), int(m.shape[0]), _ptr(m),
                                  _ptr(phi), _stream(stream)))


def correlate_mom(ctx, lat, channel, t0, nv, dil, b_list, coefs, noises, phi, corr, stream=None):
    spec, _b = _spec(channel, t0, nv, dil, b_list)
    cp = (_vp * 2)(*[_ptr(c) for c in coefs])
    npt = (_vp * 2)(*[_ptr(n) for n in noises])
    _check(_lib.correlate_mom(ctx.ptr, ctypes.byref(lat), ctypes.byref(spec), cp, npt, _ptr(phi), _ptr(corr),
                              _stream(stream)))


def laph_meson_loops(ctx, lat, channel, nv, dil, b_list, coef, noise, phi, reverse, loops, stream=None):
    spec, _b = _spec(channel, 0, nv, dil, b_list)
    _check(_lib.laph_meson_loops(ctx.ptr, ctypes.byref(lat), ctypes.byref(spec), _ptr(coef), _ptr(noise), _ptr(phi),
                                 int(reverse), _ptr(loops), _stream(stream)))


def correlate_disconnected(ctx, lat, t0, nc, loops1, loops2, vev, corr, stream=None):
    _check(_lib.correlate_disconnected(ctx.ptr, ctypes.byref(lat), int(t0), int(nc), _ptr(loops1), _ptr(loops2),
                                       float(np.real(vev)), float(np.imag(vev)), _ptr(corr), _stream(stream)))


def laph_displaced_overlaps(ctx, lat, links3d, evecs, nv, mom, path_bar, path, phi, stream=None):
    """phi[nt][nv][nv] = Phi_{p,jk}: qbar displaced along path_bar, q along path (signed steps)."""
    m = np.ascontiguousarray(np.asarray(mom, dtype=np.int32).reshape(3))
    pb = np.ascontiguousarray(np.asarray(path_bar, dtype=np.int32).reshape(-1))
    pk = np.ascontiguousarray(np.asarray(path, dtype=np.int32).reshape(-1))
    _check(_lib.laph_displaced_overlaps(ctx.ptr, ctypes.byref(lat), _ptr(links3d), _ptr(evecs), int(nv), _ptr(m),
                                        int(pb.size), _ptr(pb) if pb.size else None, int(pk.size),
                                        _ptr(pk) if pk.size else None, _ptr(phi), _stream(stream)))


def laph_baryon_tensor(ctx, lat, evecs, nv, mom, T, stream=None):
    """T[nt][nv][nv][nv] = sum_x e^{-ip.x} eps_abc V_n1(x)_a V_n2(x)_b V_n3(x)_c for the integer momentum mom."""
    m = np.ascontiguousarray(np.asarray(mom, dtype=np.int32).reshape(3))
    _check(_lib.laph_baryon_tensor(ctx.ptr, ctypes.byref(lat), _ptr(evecs), int(nv), _ptr(m), _ptr(T),
                                   _stream(stream)))


def correlate_baryon(ctx, lat, t0, nv, dil, b_list, c_snk, c_src, flav_snk, flav_src, coefs, noises, T, corr,
                     stream=None):
    """Eq. (baryoncorr) for three lines; c_snk, c_src are [4][4][4] complex spin tensors, flav_* three labels."""
    b = np.ascontiguousarray(np.asarray(b_list, dtype=np.int32))
    cs = np.ascontiguousarray(np.asarray(c_snk, dtype=np.complex128).reshape(64)).view(np.float64)
    cr = np.ascontiguousarray(np.asarray(c_src, dtype=np.complex128).reshape(64)).view(np.float64)
    dptr = ctypes.POINTER(ctypes.c_double)
    spec = BaryonSpec(int(t0), int(nv), dil, len(b), b.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                      cs.ctypes.data_as(dptr), cr.ctypes.data_as(dptr), (ctypes.c_int * 3)(*map(int, flav_snk)),
                      (ctypes.c_int * 3)(*map(int, flav_src)))
    cp = (_vp * 3)(*[_ptr(c) for c in coefs])
    npt = (_vp * 3)(*[_ptr(n) for n in noises])
    _check(_lib.correlate_baryon(ctx.ptr, ctypes.byref(lat), ctypes.byref(spec), cp, npt, _ptr(T), _ptr(corr),
                                 _stream(stream)))


def correlate_pipi(ctx, lat, iso, iso3, t0, nv, dil_fwd, b_fwd, coef_fwd, noise_fwd, dil_smt=None, b_smt=(),
                   coef_smt=(), noise_smt=(), phi_p=None, phi_mp=None, corr=None, stream=None):
    """Two-pion correlator |I, I3> (pions of momenta p, -p) from four forward and two same-time lines."""
    bf = np.ascontiguousarray(np.asarray(b_fwd, dtype=np.int32))
    bs = np.ascontiguousarray(np.asarray(b_smt, dtype=np.int32).reshape(-1))
    ip = ctypes.POINTER(ctypes.c_int)
    spec = PipiSpec(int(iso), int(iso3), int(t0), int(nv), dil_fwd, len(bf), bf.ctypes.data_as(ip),
                    dil_smt if dil_smt is not None else Dilution(), len(bs), bs.ctypes.data_as(ip) if bs.size else None)
    cf = (_vp * 4)(*[_ptr(c) for c in coef_fwd])
    nf = (_vp * 4)(*[_ptr(n) for n in noise_fwd])
    cs = (_vp * 2)(*[_ptr(c) for c in coef_smt]) if len(coef_smt) else None
    ns = (_vp * 2)(*[_ptr(n) for n in noise_smt]) if len(noise_smt) else None
    _check(_lib.correlate_pipi(ctx.ptr, ctypes.byref(lat), ctypes.byref(spec), cf, nf, cs, ns, _ptr(phi_p),
                               _ptr(phi_mp), _ptr(corr), _stream(stream)))
