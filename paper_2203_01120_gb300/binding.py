"""Thin ctypes binding of include/tdlz.h (argument marshalling only).

The functions keep the C names (``tdlz_create``, ``tdlz_load_ground_state``,
``tdlz_apply_liouvillian``, ``tdlz_lanczos_run``, ``tdlz_spectrum``, ...).  Every
step of the hot path runs inside the CUDA library; there is no Python or CPU
fallback: if the library is missing or no GPU is usable, calls raise.

PyTorch is used only to hold device memory and to hand over stream handles.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_ext

TDLZ_OK, TDLZ_ERR_ARG, TDLZ_ERR_STATE, TDLZ_ERR_CUDA, TDLZ_ERR_OOM = 0, 1, 2, 3, 4
TDLZ_ERR_BREAKDOWN, TDLZ_ERR_NUMERIC, TDLZ_ERR_TIMEOUT = 5, 6, 7
TDLZ_FP64, TDLZ_MIXED = 0, 1
TDLZ_NONHERMITIAN, TDLZ_PSEUDOHERMITIAN, TDLZ_PSEUDOHERMITIAN_POSDEF = 0, 1, 2
FLAVORS = {"nh": 0, "ph": 1, "phm": 2}
STATUS_NAMES = {0: "ok", 1: "arg", 2: "state", 3: "cuda", 4: "oom", 5: "breakdown",
                6: "numeric", 7: "timeout"}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class TdlzGroundState(C.Structure):
    _fields_ = [
        ("lattice", C.c_double * 9), ("fft", C.c_int * 3), ("ecutwfc", C.c_double),
        ("nk", C.c_int), ("nocc", C.c_int), ("npwx", C.c_int), ("nproj", C.c_int),
        ("kpts", _dp), ("q", C.c_double * 3), ("wk", _dp),
        ("npw_k", _ip), ("npw_kq", _ip), ("miller_k", _ip), ("miller_kq", _ip),
        ("evals", _dp), ("coeff_k", _dp), ("coeff_kq", _dp),
        ("vloc", _dp), ("bfield", _dp), ("n0", _dp), ("m0", _dp),
        ("beta_kq", _dp), ("dnl", _dp), ("kernel_mask", C.c_int),
    ]


class TdlzLanczosParams(C.Structure):
    _fields_ = [("nchain", C.c_int), ("qslot", _ip), ("mu", _ip), ("nsteps", C.c_int),
                ("flavor", C.c_int), ("precision", C.c_int), ("ncomp", C.c_int)]


class TdlzLanczosResult(C.Structure):
    _fields_ = [("alpha", _dp), ("beta", _dp), ("gamma", _dp), ("z", _dp), ("n0", _dp),
                ("wk", _dp), ("steps_done", _ip), ("status", _ip)]


class TdlzCoeffs(C.Structure):
    _fields_ = [("nchain", C.c_int), ("nsteps", C.c_int), ("steps", _ip), ("alpha", _dp),
                ("beta", _dp), ("gamma", _dp), ("z", _dp), ("n0", _dp), ("wk", _dp),
                ("ncomp", C.c_int)]


class TdlzSpectrumParams(C.Structure):
    _fields_ = [("start", C.c_double), ("end", C.c_double), ("step", C.c_double),
                ("eta", C.c_double), ("units", C.c_int), ("itermax0", C.c_int),
                ("itermax", C.c_int), ("extrapolation", C.c_int)]


def parse_autotune_report(text):
    """{"stage/shape": (choice, ms)} from tdlz_autotune_report's "stage/shape=choice (ms)"
    lines (the shape itself holds "=" signs; the choice follows the last one)."""
    out = {}
    for line in text.splitlines():
        key, _, rest = line.rpartition("=")
        val, _, ms = rest.partition(" (")
        out[key] = (int(val), float(ms.rstrip(" ms)")))
    return out


EXTRAPOLATION = {"no": 0, "constant": 1, "osc": 2}


EXPORTS = {
    "tdlz_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p]),
    "tdlz_destroy": (None, [C.c_void_p]),
    "tdlz_last_error": (C.c_char_p, [C.c_void_p]),
    "tdlz_synchronize": (C.c_int, [C.c_void_p]),
    "tdlz_load_ground_state": (C.c_int, [C.c_void_p, C.POINTER(TdlzGroundState), _ip]),
    "tdlz_vec_layout": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64), _ip]),
    "tdlz_apply_liouvillian": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                         C.c_int]),
    "tdlz_chain_create": (C.c_int, [C.c_void_p, C.POINTER(TdlzLanczosParams),
                                    C.POINTER(C.c_void_p)]),
    "tdlz_chain_advance": (C.c_int, [C.c_void_p, C.c_int]),
    "tdlz_chain_read": (C.c_int, [C.c_void_p, C.POINTER(TdlzLanczosResult)]),
    "tdlz_chain_destroy": (None, [C.c_void_p]),
    "tdlz_chain_state_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64)]),
    "tdlz_chain_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "tdlz_chain_restore": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "tdlz_lanczos_run": (C.c_int, [C.c_void_p, C.POINTER(TdlzLanczosParams),
                                   C.POINTER(TdlzLanczosResult)]),
    "tdlz_spectrum": (C.c_int, [C.c_void_p, C.POINTER(TdlzCoeffs),
                                C.POINTER(TdlzSpectrumParams), _dp, _ip]),
    "tdlz_spectrum_noalloc": (C.c_int, [C.c_void_p, C.POINTER(TdlzCoeffs),
                                        C.POINTER(TdlzSpectrumParams), C.c_void_p, C.c_int]),
    "tdlz_structure_factor": (C.c_int, [C.c_void_p, _dp, C.c_int, _dp, _dp]),
    "tdlz_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "tdlz_profile_read": (C.c_int, [C.c_void_p, _dp, C.POINTER(C.c_int64), _dp, _dp]),
    "tdlz_stage_name": (C.c_char_p, [C.c_int]),
    "tdlz_autotune_report": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int64,
                                       C.POINTER(C.c_int64)]),
    "tdlz_launch_count": (C.c_int64, []),
}
NSTAGE = 11

_LIB = None


def library_path() -> str:
    return build_ext.LIB


def load_library(build_if_missing: bool = False):
    """dlopen the in-tree libtdlz.so (raises if absent; never falls back)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"tdlz CUDA library not built ({path}); run build_ext.build()")
        build_ext.build()
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


class TdlzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tdlz status {status} ({STATUS_NAMES.get(status, '?')}): {msg}")
        self.status = status


def _dptr(a):
    return a.ctypes.data_as(_dp) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(_ip) if a is not None else None


class Context:
    """Owns a tdlz context on one CUDA device; methods mirror the C entry points."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        self.h = C.c_void_p()
        st = self.lib.tdlz_create(C.byref(self.h), int(device),
                                  C.c_void_p(stream) if stream else None)
        if st != TDLZ_OK:
            raise TdlzError(st, "tdlz_create failed (no usable CUDA device?)")
        self._keep = []

    def close(self):
        if self.h:
            self.lib.tdlz_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != TDLZ_OK:
            msg = self.lib.tdlz_last_error(self.h)
            raise TdlzError(st, msg.decode() if msg else "")

    def synchronize(self):
        self._check(self.lib.tdlz_synchronize(self.h))

    # ---------------------------------------------------------------- load
    def load_ground_state(self, gs) -> int:
        """gs: synth.GroundState-like object with the bundle arrays (host, FP64)."""
        keep = {}

        def arr(name, dtype):
            a = np.ascontiguousarray(getattr(gs, name), dtype=dtype)
            keep[name] = a
            return a

        s = TdlzGroundState()
        s.lattice[:] = list(np.asarray(gs.lattice, dtype=np.float64).ravel())
        s.fft[:] = [int(v) for v in gs.fft]
        s.ecutwfc = float(gs.ecutwfc)
        s.nk, s.nocc, s.npwx, s.nproj = int(gs.nk), int(gs.nocc), int(gs.npwx), int(gs.nproj)
        s.kpts = _dptr(arr("kpts", np.float64))
        s.q[:] = [float(v) for v in gs.q]
        s.wk = _dptr(arr("wk", np.float64))
        s.npw_k = _iptr(arr("npw_k", np.int32))
        s.npw_kq = _iptr(arr("npw_kq", np.int32))
        s.miller_k = _iptr(arr("miller_k", np.int32))
        s.miller_kq = _iptr(arr("miller_kq", np.int32))
        s.evals = _dptr(arr("evals", np.float64))
        s.coeff_k = _dptr(arr("coeff_k", np.complex128).view(np.float64))
        s.coeff_kq = _dptr(arr("coeff_kq", np.complex128).view(np.float64))
        s.vloc = _dptr(arr("vloc", np.float64))
        s.bfield = _dptr(arr("bfield", np.float64))
        s.n0 = _dptr(arr("n0", np.float64))
        s.m0 = _dptr(arr("m0", np.float64))
        s.beta_kq = _dptr(arr("beta_kq", np.complex128).view(np.float64)) if gs.nproj else None
        s.dnl = _dptr(arr("dnl", np.complex128).view(np.float64)) if gs.nproj else None
        s.kernel_mask = int(gs.kernel_mask)
        q = C.c_int(-1)
        self._check(self.lib.tdlz_load_ground_state(self.h, C.byref(s), C.byref(q)))
        return q.value

    def profile(self, enable=True):
        self._check(self.lib.tdlz_profile(self.h, int(bool(enable))))

    def profile_read(self):
        """{stage: {"ms", "launches", "bytes", "flops"}} accumulated since profile(True)."""
        ms = np.zeros(NSTAGE)
        ln = np.zeros(NSTAGE, np.int64)
        by = np.zeros(NSTAGE)
        fl = np.zeros(NSTAGE)
        self._check(self.lib.tdlz_profile_read(self.h, _dptr(ms),
                                               ln.ctypes.data_as(C.POINTER(C.c_int64)),
                                               _dptr(by), _dptr(fl)))
        return {self.lib.tdlz_stage_name(i).decode(): {"ms": float(ms[i]), "launches": int(ln[i]),
                                                       "bytes": float(by[i]),
                                                       "flops": float(fl[i])}
                for i in range(NSTAGE)}

    def launch_count(self):
        return int(self.lib.tdlz_launch_count())

    def autotune_report(self):
        """{"stage/shape": (choice, ms)} of the autotuner's decisions so far."""
        need = C.c_int64()
        self._check(self.lib.tdlz_autotune_report(self.h, None, 0, C.byref(need)))
        buf = C.create_string_buffer(need.value + 1)
        self._check(self.lib.tdlz_autotune_report(self.h, buf, need.value + 1, C.byref(need)))
        return parse_autotune_report(buf.value.decode())

    def vec_layout(self, qslot):
        n = C.c_int64()
        npwx = C.c_int()
        self._check(self.lib.tdlz_vec_layout(self.h, int(qslot), C.byref(n), C.byref(npwx)))
        return n.value, npwx.value

    # ---------------------------------------------------------------- apply
    def apply_liouvillian(self, qslot, x, y, adjoint=False, precision=TDLZ_FP64):
        """x, y: torch CUDA tensors (complex128 for FP64, complex64 for MIXED)."""
        self._check(self.lib.tdlz_apply_liouvillian(self.h, int(qslot), C.c_void_p(x.data_ptr()),
                                                    C.c_void_p(y.data_ptr()), int(bool(adjoint)),
                                                    int(precision)))

    # -------------------------------------------------------------- Lanczos
    def chain_create(self, qslots, mus, nsteps, flavor="ph", precision=TDLZ_FP64, ncomp=3):
        """mus: 0, 1, 2 = spin x, y, z perturbations, 3 = the charge; ncomp = 3 records
        z for the spin components, 4 also for the charge (the 4x4 susceptibility)."""
        return Chain(self, qslots, mus, nsteps, flavor, precision, ncomp)

    def lanczos_run(self, qslots, mus, nsteps, flavor="ph", precision=TDLZ_FP64, ncomp=3):
        ch = self.chain_create(qslots, mus, nsteps, flavor, precision, ncomp)
        try:
            ch.advance(nsteps)
            return ch.read()
        finally:
            ch.close()

    def spectrum(self, coeffs, start, end, step, eta, units=1, itermax0=0, itermax=0,
                 extrapolation="no"):
        """chi[nchain][ncomp][nomega] from a coefficient dict as returned by Chain.read()
        (ncomp = the dict's z rows: 3, or 4 with the charge last)."""
        nc, cap = coeffs["beta"].shape
        nl = int(coeffs["z"].shape[1])
        steps = np.ascontiguousarray(coeffs["steps_done"], dtype=np.int32)
        al = np.ascontiguousarray(coeffs["alpha"], dtype=np.complex128)
        be = np.ascontiguousarray(coeffs["beta"], dtype=np.float64)
        ga = np.ascontiguousarray(coeffs["gamma"], dtype=np.complex128)
        z = np.ascontiguousarray(coeffs["z"], dtype=np.complex128)
        n0 = np.ascontiguousarray(coeffs["n0"], dtype=np.float64)
        wk = np.ascontiguousarray(coeffs["wk"], dtype=np.float64)
        c = TdlzCoeffs(nc, cap, _iptr(steps), _dptr(al.view(np.float64)), _dptr(be),
                       _dptr(ga.view(np.float64)), _dptr(z.view(np.float64)), _dptr(n0), _dptr(wk),
                       nl)
        sp = TdlzSpectrumParams(float(start), float(end), float(step), float(eta), int(units),
                                int(itermax0), int(itermax), EXTRAPOLATION[extrapolation])
        nw = C.c_int()
        self._check(self.lib.tdlz_spectrum(self.h, C.byref(c), C.byref(sp), None, C.byref(nw)))
        chi = np.zeros((nc, nl, nw.value), dtype=np.complex128)
        self._check(self.lib.tdlz_spectrum(self.h, C.byref(c), C.byref(sp),
                                           _dptr(chi.view(np.float64)), C.byref(nw)))
        return chi


    def spectrum_noalloc(self, dev, start, end, step, eta, units, chi_dev):
        """tdlz_spectrum_noalloc: every array in ``dev`` and ``chi_dev`` is a CUDA tensor
        the caller allocated (steps int32, alpha/gamma/z complex128, beta/n0/wk float64);
        chi_dev is complex128 [nchain][ncomp][nomega] (ncomp = z's rows).  Enqueued on the
        context stream."""
        nc, cap = dev["beta"].shape
        vp = lambda t: C.cast(C.c_void_p(t.data_ptr()), _dp)  # noqa: E731
        c = TdlzCoeffs(nc, cap, C.cast(C.c_void_p(dev["steps_done"].data_ptr()), _ip),
                       vp(dev["alpha"]), vp(dev["beta"]), vp(dev["gamma"]), vp(dev["z"]),
                       vp(dev["n0"]), vp(dev["wk"]), int(dev["z"].shape[1]))
        sp = TdlzSpectrumParams(float(start), float(end), float(step), float(eta), int(units))
        self._check(self.lib.tdlz_spectrum_noalloc(self.h, C.byref(c), C.byref(sp),
                                                   C.c_void_p(chi_dev.data_ptr()),
                                                   int(chi_dev.shape[-1])))

    def structure_factor(self, chi3, q):
        """S(q, omega) = -Im Tr[P_perp(q) chi] from chi3[mu][lambda][nomega] (complex)."""
        chi3 = np.ascontiguousarray(chi3, dtype=np.complex128)
        if chi3.ndim != 3 or chi3.shape[:2] != (3, 3):
            raise ValueError("chi3 must be [3][3][nomega]")
        nw = chi3.shape[2]
        qq = np.ascontiguousarray(q, dtype=np.float64)
        out = np.zeros(nw, dtype=np.float64)
        self._check(self.lib.tdlz_structure_factor(self.h, _dptr(chi3.view(np.float64)), int(nw),
                                                   _dptr(qq), _dptr(out)))
        return out

    def spectrum_nomega(self, start, end, step, units=1):
        """Frequency-grid length (tdlz_spectrum with chi = NULL; allocates nothing)."""
        one = np.zeros(1)
        onei = np.zeros(1, np.int32)
        c = TdlzCoeffs(1, 1, _iptr(onei), _dptr(one), _dptr(one), _dptr(one), _dptr(one),
                       _dptr(one), _dptr(one))
        sp = TdlzSpectrumParams(float(start), float(end), float(step), 1.0, int(units))
        nw = C.c_int()
        self._check(self.lib.tdlz_spectrum(self.h, C.byref(c), C.byref(sp), None, C.byref(nw)))
        return nw.value


class Chain:
    """Lanczos chains advancing on the device (tdlz_chain_*)."""

    def __init__(self, ctx: Context, qslots, mus, nsteps, flavor="ph", precision=TDLZ_FP64,
                 ncomp=3):
        self.ctx = ctx
        self.nchain = len(qslots)
        self.cap = int(nsteps)
        self.ncomp = int(ncomp)
        self._q = np.ascontiguousarray(qslots, dtype=np.int32)
        self._m = np.ascontiguousarray(mus, dtype=np.int32)
        fl = FLAVORS[flavor] if isinstance(flavor, str) else int(flavor)
        p = TdlzLanczosParams(self.nchain, _iptr(self._q), _iptr(self._m), self.cap, fl,
                              int(precision), self.ncomp)
        self.h = C.c_void_p()
        ctx._check(ctx.lib.tdlz_chain_create(ctx.h, C.byref(p), C.byref(self.h)))

    def advance(self, nsteps):
        self.ctx._check(self.ctx.lib.tdlz_chain_advance(self.h, int(nsteps)))

    def read(self):
        nc, m = self.nchain, self.cap
        out = {
            "alpha": np.zeros((nc, m), np.complex128), "beta": np.zeros((nc, m)),
            "gamma": np.zeros((nc, m), np.complex128),
            "z": np.zeros((nc, self.ncomp, m), np.complex128),
            "n0": np.zeros(nc), "wk": np.zeros(nc), "steps_done": np.zeros(nc, np.int32),
            "status": np.zeros(nc, np.int32),
        }
        r = TdlzLanczosResult(_dptr(out["alpha"].view(np.float64)), _dptr(out["beta"]),
                              _dptr(out["gamma"].view(np.float64)), _dptr(out["z"].view(np.float64)),
                              _dptr(out["n0"]), _dptr(out["wk"]), _iptr(out["steps_done"]),
                              _iptr(out["status"]))
        self.ctx._check(self.ctx.lib.tdlz_chain_read(self.h, C.byref(r)))
        return out

    def save(self) -> bytes:
        """Restart image of the chains (host bytes)."""
        n = C.c_int64()
        self.ctx._check(self.ctx.lib.tdlz_chain_state_size(self.h, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self.ctx._check(self.ctx.lib.tdlz_chain_save(self.h, buf, n.value))
        return buf.raw

    def restore(self, image: bytes):
        buf = C.create_string_buffer(image, len(image))
        self.ctx._check(self.ctx.lib.tdlz_chain_restore(self.h, buf, len(image)))

    def close(self):
        if self.h:
            self.ctx.lib.tdlz_chain_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
