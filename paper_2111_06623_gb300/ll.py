"""Python binding of libll.so (ctypes): argument marshalling only.

Every step of the Liouvillian application, the Lanczos recursions and the spectrum runs in
the library's CUDA kernels; this module converts NumPy arrays to the C ABI of
include/ll.h and back.  Importing it without the built library raises ImportError: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# LL_LIBRARY in the environment selects another build of the same library (the bounds-checked
# libll_check.so of build_library(check=True)); default: the in-tree libll.so
LIB_PATH = os.environ.get("LL_LIBRARY") or os.path.join(_HERE, "libll.so")

LL_OK, LL_EINVAL, LL_ENOMEM, LL_EBREAKDOWN, LL_ENOTPD, LL_ETIMEOUT, LL_ECUDA = 0, 1, 2, 3, 4, 5, 6
LL_PENDING, LL_ENOTFOUND, LL_EUNSUPPORTED, LL_ECANCELED = 7, 8, 9, 10
LL_EXTRAP_NO, LL_EXTRAP_CONSTANT, LL_EXTRAP_OSC = 0, 1, 2
APPROX = {"ipa": 0, "rpa": 1, "tddft": 2}
FLAVOUR = {"ph": 0, "nh": 1}
PRECISION = {"fp64": 0, "fp32": 1}

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


class LLError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class SystemDesc(C.Structure):
    _fields_ = [
        ("lattice", (C.c_double * 3) * 3), ("nfft", C.c_int), ("nks", C.c_int), ("nbnd", C.c_int),
        ("nproj", C.c_int), ("q_cart", C.c_double * 3), ("kcart", _dp), ("npw_k", _ip), ("miller_k", _ip),
        ("npw_kq", _ip), ("miller_kq", _ip), ("u_k", _dp), ("u_kq", _dp), ("eps_k", _dp), ("vloc_r", _dp),
        ("rho_r", _dp), ("beta_kq", _dp), ("dij", _dp), ("approx", C.c_int), ("flavour", C.c_int),
        ("precision", C.c_int), ("max_steps", C.c_int), ("where", C.c_int),
        ("kweight", _dp), ("nsym", C.c_int), ("sym", _ip),
        ("occ_k", _dp), ("occ_kq", _dp), ("eps_kq", _dp),
    ]


LL_WHERE_HOST, LL_WHERE_DEVICE = 0, 1


def _on_device(a) -> bool:
    """True for a CUDA tensor (torch), whose data_ptr() is a device address."""
    return bool(getattr(a, "is_cuda", False))


def _dev_ptr(t, what: str):
    """The device address of a contiguous float64 / complex128 CUDA tensor (packed layout)."""
    import torch
    if t.dtype not in (torch.float64, torch.complex128) or not t.is_contiguous():
        raise ValueError(f"{what}: a contiguous float64 or complex128 CUDA tensor is required")
    return C.cast(C.c_void_p(t.data_ptr()), _dp)


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"the library is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    sig = {
        "ll_create": (C.c_int, [C.POINTER(SystemDesc), vp, C.POINTER(vp)]),
        "ll_create_sharing": (C.c_int, [C.POINTER(SystemDesc), vp, vp, C.POINTER(vp)]),
        "ll_destroy": (C.c_int, [vp]),
        "ll_lanczos": (C.c_int, [vp, C.c_int, _dp, _dp, _dp, _dp, _ip]),
        "ll_lanczos_spectrum": (C.c_int, [vp, C.c_int, _dp, C.c_int, C.c_double, _dp, _dp, _dp]),
        "ll_spectrum": (C.c_int, [_dp, _dp, _dp, C.c_int, C.c_double, _dp, _dp, C.c_int, C.c_double, _dp, _dp, _dp, vp]),
        "ll_spectrum_static": (C.c_int, [_dp, _dp, _dp, C.c_int, C.c_double, _dp, _dp, C.c_int, C.c_double, _dp,
                                         _dp, _dp, vp]),
        "ll_lanczos_spectrum_x": (C.c_int, [vp, C.c_int, C.c_int, C.c_int, _dp, C.c_int, C.c_double, _dp, _dp, _dp]),
        "ll_spectrum_x": (C.c_int, [_dp, _dp, _dp, C.c_int, C.c_int, C.c_int, C.c_double, _dp, _dp, C.c_int,
                                    C.c_double, _dp, _dp, _dp, vp]),
        "ll_apply": (C.c_int, [vp, C.c_int, _dp, _dp]),
        "ll_get_map": (C.c_int, [vp, _ip]),
        "ll_get_start": (C.c_int, [vp, _dp]),
        "ll_footprint": (C.c_int, [C.POINTER(SystemDesc), C.POINTER(C.c_size_t)]),
        "ll_bytes": (C.c_int, [vp, C.POINTER(C.c_size_t)]),
        "ll_fsum": (C.c_int, [_dp, _dp, C.c_int, C.c_double, C.c_double, _dp, _dp, vp]),
        "ll_profile": (C.c_int, [vp, C.c_int]),
        "ll_profile_read": (C.c_int, [vp, _dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
        "ll_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(vp)]),
        "ll_server_set_chunk": (C.c_int, [vp, C.c_int]),
        "ll_submit": (C.c_int, [vp, vp, C.POINTER(C.c_uint64)]),
        "ll_poll": (C.c_int, [vp, C.c_uint64, C.POINTER(C.c_int), vp]),
        "ll_cancel": (C.c_int, [vp, C.c_uint64]),
        "ll_release": (C.c_int, [vp, C.c_uint64]),
        "ll_server_stats": (C.c_int, [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(C.c_int),
                                      C.POINTER(C.c_int)]),
        "ll_server_last_error": (C.c_char_p, []),
        "ll_server_destroy": (C.c_int, [vp]),
        "ll_last_error": (C.c_char_p, []),
        "ll_version": (C.c_char_p, []),
        "ll_fma_peak": (C.c_int, [C.c_int, _dp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    return lib


_lib = _load()
EXPORTS = ("ll_create", "ll_create_sharing", "ll_destroy", "ll_lanczos", "ll_lanczos_spectrum", "ll_spectrum", "ll_spectrum_static",
           "ll_lanczos_spectrum_x", "ll_spectrum_x",
           "ll_apply", "ll_get_map", "ll_get_start", "ll_footprint", "ll_bytes", "ll_fsum", "ll_profile", "ll_profile_read", "ll_last_error",
           "ll_version", "ll_fma_peak", "ll_server_create",
           "ll_server_set_chunk", "ll_submit", "ll_poll", "ll_cancel", "ll_release", "ll_server_stats", "ll_server_last_error",
           "ll_server_destroy")
PROF_CLASSES = ("zinv", "xy1", "hxc", "xy2", "zfwd", "update")


def version() -> str:
    return _lib.ll_version().decode()


def fma_peak(precision: str = "fp32", stream=None) -> float:
    """Measured FMA throughput of the device, TFLOP/s (ll_fma_peak)."""
    out = C.c_double(0.0)
    _check(_lib.ll_fma_peak(PRECISION[precision], C.byref(out), C.c_void_p(stream) if stream else None))
    return float(out.value)


def _check(rc: int):
    if rc != LL_OK:
        raise LLError(rc, _lib.ll_last_error().decode())


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _is_packed(a) -> bool:
    """A host array already in the descriptor's packed layout (1-D complex128, contiguous)."""
    return isinstance(a, np.ndarray) and a.ndim == 1 and a.dtype == np.complex128 and a.flags.c_contiguous


def _cat_complex(blocks) -> np.ndarray:
    if _is_packed(blocks):
        return blocks                      # used in place (no copy)
    return np.ascontiguousarray(np.concatenate([np.ascontiguousarray(b, dtype=np.complex128).ravel() for b in blocks]))


def _make_desc(*, lattice, nfft, kcart, miller_k, miller_kq, u_k, u_kq, eps_k, vloc_r, rho_r, beta_kq=None,
               dij=None, q_cart, approx="tddft", flavour="ph", precision="fp64", max_steps=1000, kweight=None,
               sym=None, occ_k=None, occ_kq=None, eps_kq=None):
    """An ll_system_desc and the arrays it points into (keep them alive while it is used).

    u_k, u_kq, beta_kq, vloc_r and rho_r are host arrays (u_k, u_kq, beta_kq as lists of
    per-k (rows, npw) arrays, or each one 1-D complex128 array already in the packed layout of
    ll_system_desc, used in place: pinned host memory then copies at full link speed), or all
    of them CUDA tensors (torch) in the packed layout: the descriptor then points at device
    memory (where = LL_WHERE_DEVICE).
    occ_k, occ_kq, eps_kq ((nks, nbnd) host arrays): the occupations and k+Q levels of a metal."""
    nks = len(miller_k)
    dev = _on_device(u_k)
    if dev:
        nbnd = int(np.shape(eps_k)[1])
        nproj = int(len(dij)) if dij is not None and beta_kq is not None else 0
    elif _is_packed(u_k):
        nbnd = int(np.shape(eps_k)[1])
        nproj = int(len(dij)) if dij is not None and beta_kq is not None else 0
    else:
        nbnd = int(u_k[0].shape[0])
        nproj = int(beta_kq[0].shape[0]) if beta_kq is not None and len(beta_kq) and beta_kq[0].shape[0] else 0
    if dev:
        arrs = {"u_k": u_k, "u_kq": u_kq, "vloc_r": vloc_r, "rho_r": rho_r}
        if nproj:
            arrs["beta_kq"] = beta_kq
        for name, t in arrs.items():
            if not _on_device(t):
                raise ValueError(f"{name}: with u_k on the device every large array must be a CUDA tensor")
        d, k = _make_desc_device(lattice=lattice, nfft=nfft, kcart=kcart, miller_k=miller_k, miller_kq=miller_kq,
                                 arrs=arrs, eps_k=eps_k, dij=dij, nbnd=nbnd, nproj=nproj, q_cart=q_cart,
                                 approx=approx, flavour=flavour, precision=precision, max_steps=max_steps)
        _set_symmetry(d, k, kweight, sym)
        _set_occupations(d, k, occ_k, occ_kq, eps_kq)
        return d, k
    k = dict(
        kcart=np.ascontiguousarray(kcart, dtype=np.float64),
        npw_k=np.array([len(m) for m in miller_k], dtype=np.int32),
        miller_k=np.ascontiguousarray(np.concatenate(miller_k), dtype=np.int32),
        npw_kq=np.array([len(m) for m in miller_kq], dtype=np.int32),
        miller_kq=np.ascontiguousarray(np.concatenate(miller_kq), dtype=np.int32),
        u_k=_cat_complex(u_k), u_kq=_cat_complex(u_kq),
        eps_k=np.ascontiguousarray(eps_k, dtype=np.float64),
        vloc_r=np.ascontiguousarray(vloc_r, dtype=np.float64),
        rho_r=np.ascontiguousarray(rho_r, dtype=np.float64),
        beta_kq=_cat_complex(beta_kq) if nproj else np.zeros(2),
        dij=np.ascontiguousarray(dij if nproj else np.zeros(1), dtype=np.float64),
    )
    sk, sq = int(k["npw_k"].sum()), int(k["npw_kq"].sum())
    for name, rows, n in (("u_k", nbnd, sk), ("u_kq", nbnd, sq), ("beta_kq", nproj, sq)):
        if (name != "beta_kq" or nproj) and k[name].size != rows * n:
            raise ValueError(f"{name}: {k[name].size} coefficients, the spheres and rows need {rows * n}")
    d = SystemDesc()
    for i in range(3):
        for j in range(3):
            d.lattice[i][j] = float(lattice[i][j])
        d.q_cart[i] = float(q_cart[i])
    d.nfft, d.nks, d.nbnd, d.nproj = int(nfft), nks, nbnd, nproj
    d.kcart, d.npw_k, d.miller_k = _d(k["kcart"]), _i(k["npw_k"]), _i(k["miller_k"])
    d.npw_kq, d.miller_kq = _i(k["npw_kq"]), _i(k["miller_kq"])
    d.u_k, d.u_kq, d.eps_k = _d(k["u_k"].view(np.float64)), _d(k["u_kq"].view(np.float64)), _d(k["eps_k"])
    d.vloc_r, d.rho_r = _d(k["vloc_r"]), _d(k["rho_r"])
    d.beta_kq = _d(k["beta_kq"].view(np.float64)) if nproj else None
    d.dij = _d(k["dij"])
    d.approx, d.flavour, d.precision = APPROX[approx], FLAVOUR[flavour], PRECISION[precision]
    d.max_steps = int(max_steps)
    d.where = LL_WHERE_HOST
    _set_symmetry(d, k, kweight, sym)
    _set_occupations(d, k, occ_k, occ_kq, eps_kq)
    return d, k


def _set_symmetry(d, keep, kweight, sym):
    """k-point weights (star sizes of the small group of Q) and the group's integer matrices on
    the FFT grid (Sec. 2.6); None: the plain full-mesh sums."""
    if kweight is not None:
        keep["kweight"] = np.ascontiguousarray(kweight, dtype=np.float64)
        d.kweight = _d(keep["kweight"])
    if sym is not None and len(sym) > 1:
        keep["sym"] = np.ascontiguousarray(sym, dtype=np.int32).reshape(-1)
        d.nsym, d.sym = len(sym), _i(keep["sym"])


def _set_occupations(d, keep, occ_k, occ_kq, eps_kq):
    """A metal's occupations at k and k+Q and the levels at k+Q (Sec. 2.6); None: an insulator."""
    if occ_k is None:
        return
    for name, a in (("occ_k", occ_k), ("occ_kq", occ_kq), ("eps_kq", eps_kq)):
        keep[name] = np.ascontiguousarray(a, dtype=np.float64)
        setattr(d, name, _d(keep[name]))


def _make_desc_device(*, lattice, nfft, kcart, miller_k, miller_kq, arrs, eps_k, dij, nbnd, nproj, q_cart, approx,
                      flavour, precision, max_steps):
    k = dict(
        kcart=np.ascontiguousarray(kcart, dtype=np.float64),
        npw_k=np.array([len(m) for m in miller_k], dtype=np.int32),
        miller_k=np.ascontiguousarray(np.concatenate(miller_k), dtype=np.int32),
        npw_kq=np.array([len(m) for m in miller_kq], dtype=np.int32),
        miller_kq=np.ascontiguousarray(np.concatenate(miller_kq), dtype=np.int32),
        eps_k=np.ascontiguousarray(eps_k, dtype=np.float64),
        dij=np.ascontiguousarray(dij if nproj else np.zeros(1), dtype=np.float64),
        device=arrs,
    )
    d = SystemDesc()
    for i in range(3):
        for j in range(3):
            d.lattice[i][j] = float(lattice[i][j])
        d.q_cart[i] = float(q_cart[i])
    d.nfft, d.nks, d.nbnd, d.nproj = int(nfft), len(miller_k), nbnd, nproj
    d.kcart, d.npw_k, d.miller_k = _d(k["kcart"]), _i(k["npw_k"]), _i(k["miller_k"])
    d.npw_kq, d.miller_kq = _i(k["npw_kq"]), _i(k["miller_kq"])
    d.u_k, d.u_kq = _dev_ptr(arrs["u_k"], "u_k"), _dev_ptr(arrs["u_kq"], "u_kq")
    d.vloc_r, d.rho_r = _dev_ptr(arrs["vloc_r"], "vloc_r"), _dev_ptr(arrs["rho_r"], "rho_r")
    d.beta_kq = _dev_ptr(arrs["beta_kq"], "beta_kq") if nproj else None
    d.eps_k, d.dij = _d(k["eps_k"]), _d(k["dij"])
    d.approx, d.flavour, d.precision = APPROX[approx], FLAVOUR[flavour], PRECISION[precision]
    d.max_steps = int(max_steps)
    d.where = LL_WHERE_DEVICE
    return d, k


class Chain:
    """One Lanczos chain resident on the device (ll_create ... ll_destroy)."""

    def __init__(self, *, stream=None, share=None, **system):
        """share: a Chain of the same ground state whose u(r) grids this one uses
        (ll_create_sharing: another momentum transfer Q on one ground state)."""
        d, k = _make_desc(**system)
        self._keep = k
        self.desc = d
        self.nks, self.nbnd, self.max_steps = d.nks, d.nbnd, d.max_steps
        self.npw_kq = k["npw_kq"].copy()
        self.lattice = np.asarray(system["lattice"], dtype=np.float64)
        self.q_cart = np.asarray(system["q_cart"], dtype=np.float64)
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        if share is not None:
            _check(_lib.ll_create_sharing(C.byref(d), share._h, st, C.byref(h)))
        else:
            _check(_lib.ll_create(C.byref(d), st, C.byref(h)))
        self._h = h
        self.steps = 0

    def close(self):
        if getattr(self, "_h", None):
            _lib.ll_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def lanczos(self, n_steps: int):
        """Runs n_steps more steps; returns (beta, gamma, z) of every step so far (the
        vanishing diagonal alpha of every step so far is kept in self.alpha)."""
        cap = self.max_steps
        alpha = np.full(cap, np.nan)
        beta = np.zeros(cap)
        gamma = np.zeros(cap, dtype=np.complex128)
        z = np.zeros(cap, dtype=np.complex128)
        done = C.c_int(0)
        rc = _lib.ll_lanczos(self._h, int(n_steps), _d(alpha), _d(beta), _d(gamma.view(np.float64)),
                             _d(z.view(np.float64)), C.byref(done))
        self.steps = done.value
        self.alpha = alpha[: done.value].copy()
        if rc != LL_OK:
            err = LLError(rc, _lib.ll_last_error().decode())
            err.partial = (beta[: done.value], gamma[: done.value], z[: done.value])
            raise err
        return beta[: done.value].copy(), gamma[: done.value].copy(), z[: done.value].copy()

    def spectrum(self, omega_ev, eta_ev: float, m: int = 0, extrapolation: str = "no", m_total: int = 0):
        """chi, eps^-1, eps from the chain's first m coefficients (0: all), optionally
        extrapolated ('constant' or 'osc') to m_total (ll_lanczos_spectrum[_x])."""
        w = np.ascontiguousarray(omega_ev, dtype=np.float64)
        out = [np.zeros(len(w), dtype=np.complex128) for _ in range(3)]
        if extrapolation == "no":
            _check(_lib.ll_lanczos_spectrum(self._h, int(m), _d(w), len(w), float(eta_ev),
                                            *[_d(o.view(np.float64)) for o in out]))
        else:
            _check(_lib.ll_lanczos_spectrum_x(self._h, int(m), EXTRAP[extrapolation], int(m_total), _d(w), len(w),
                                              float(eta_ev), *[_d(o.view(np.float64)) for o in out]))
        return tuple(out)

    def _split(self, flat):
        out, pos = [], 0
        for n in self.npw_kq:
            out.append(flat[pos:pos + self.nbnd * n].reshape(self.nbnd, n))
            pos += self.nbnd * n
        return out

    def apply(self, x, upper: bool):
        xin = _cat_complex(x)
        out = np.zeros_like(xin)
        _check(_lib.ll_apply(self._h, int(bool(upper)), _d(xin.view(np.float64)), _d(out.view(np.float64))))
        return self._split(out)

    def index_map(self):
        m = np.zeros(int(self.npw_kq.sum()), dtype=np.int32)
        _check(_lib.ll_get_map(self._h, _i(m)))
        out, pos = [], 0
        for n in self.npw_kq:
            out.append(m[pos:pos + n].copy())
            pos += n
        return out

    def start_vector(self):
        y = np.zeros(self.nbnd * int(self.npw_kq.sum()), dtype=np.complex128)
        _check(_lib.ll_get_start(self._h, _d(y.view(np.float64))))
        return self._split(y)

    def profile(self, enable: bool):
        _check(_lib.ll_profile(self._h, int(bool(enable))))

    def profile_read(self):
        """({class: device ms}, {class: launches}, total launches) since profile(True)."""
        ms = np.zeros(len(PROF_CLASSES))
        n = (C.c_longlong * len(PROF_CLASSES))()
        tot = C.c_longlong(0)
        _check(_lib.ll_profile_read(self._h, _d(ms), n, C.byref(tot)))
        return dict(zip(PROF_CLASSES, ms.tolist())), dict(zip(PROF_CLASSES, list(n))), int(tot.value)

    def footprint(self) -> int:
        b = C.c_size_t(0)
        _check(_lib.ll_footprint(C.byref(self.desc), C.byref(b)))
        return int(b.value)

    def bytes(self) -> int:
        """ll_bytes: device bytes the chain holds now."""
        b = C.c_size_t(0)
        _check(_lib.ll_bytes(self._h, C.byref(b)))
        return int(b.value)


def fsum(omega_ev, eps_inv, nelec: float, omega_cell: float, stream=None):
    """ll_fsum: (trapezoid first moment of -Im eps^-1 over the grid, (pi/2) omega_p^2), Ha^2."""
    w = np.ascontiguousarray(omega_ev, dtype=np.float64)
    e = np.ascontiguousarray(eps_inv, dtype=np.complex128)
    if e.shape != w.shape:
        raise ValueError("omega_ev and eps_inv differ in length")
    m, x = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.ll_fsum(_d(w), _d(e.view(np.float64)), len(w), float(nelec), float(omega_cell), C.byref(m),
                        C.byref(x), C.c_void_p(stream) if stream else None))
    return m.value, x.value


def spectrum_bytes(n_omega: int) -> int:
    """LL_SPECTRUM_BYTES: device bytes of a chain's spectrum staging for n_omega frequencies."""
    return int(n_omega) * 56 + 256


def footprint(**system) -> int:
    """ll_footprint: an upper bound of the device bytes one chain of this system would hold
    (what the request loop admits by), computed on the host without creating the chain."""
    d, _keep = _make_desc(**system)
    b = C.c_size_t(0)
    _check(_lib.ll_footprint(C.byref(d), C.byref(b)))
    return int(b.value)


EXTRAP = {"no": LL_EXTRAP_NO, "constant": LL_EXTRAP_CONSTANT, "osc": LL_EXTRAP_OSC}


def spectrum(beta, gamma, z, omega_cell, q_cart, omega_ev, eta_ev, stream=None, extrapolation: str = "no",
             m_total: int = 0):
    """chi, eps^-1, eps from caller-held coefficients (ll_spectrum), optionally extrapolated
    ('constant' or 'osc') to m_total coefficients (ll_spectrum_x)."""
    b = np.ascontiguousarray(beta, dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.complex128)
    zz = np.ascontiguousarray(z, dtype=np.complex128)
    q = np.ascontiguousarray(q_cart, dtype=np.float64)
    w = np.ascontiguousarray(omega_ev, dtype=np.float64)
    out = [np.zeros(len(w), dtype=np.complex128) for _ in range(3)]
    st = C.c_void_p(stream) if stream else None
    if extrapolation == "no":
        _check(_lib.ll_spectrum(_d(b), _d(g.view(np.float64)), _d(zz.view(np.float64)), len(b), float(omega_cell),
                                _d(q), _d(w), len(w), float(eta_ev), *[_d(o.view(np.float64)) for o in out], st))
    else:
        _check(_lib.ll_spectrum_x(_d(b), _d(g.view(np.float64)), _d(zz.view(np.float64)), len(b),
                                  EXTRAP[extrapolation], int(m_total), float(omega_cell), _d(q), _d(w), len(w),
                                  float(eta_ev), *[_d(o.view(np.float64)) for o in out], st))
    return tuple(out)


SPECTRUM_STATIC_MAX_COEF = 16384
SPECTRUM_STATIC_MAX_OMEGA = 16384


def spectrum_static(beta, gamma, z, omega_cell, q_cart, omega_ev, eta_ev, stream=None):
    """ll_spectrum_static: the same results as spectrum() without any device allocation,
    staged through the library's static device array (limits SPECTRUM_STATIC_MAX_*)."""
    b = np.ascontiguousarray(beta, dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.complex128)
    zz = np.ascontiguousarray(z, dtype=np.complex128)
    q = np.ascontiguousarray(q_cart, dtype=np.float64)
    w = np.ascontiguousarray(omega_ev, dtype=np.float64)
    out = [np.zeros(len(w), dtype=np.complex128) for _ in range(3)]
    _check(_lib.ll_spectrum_static(_d(b), _d(g.view(np.float64)), _d(zz.view(np.float64)), len(b),
                                   float(omega_cell), _d(q), _d(w), len(w), float(eta_ev),
                                   *[_d(o.view(np.float64)) for o in out], C.c_void_p(stream) if stream else None))
    return tuple(out)


class JobDesc(C.Structure):
    _fields_ = [("sys", SystemDesc), ("n_steps", C.c_int), ("omega_ev", _dp), ("n_omega", C.c_int),
                ("eta_ev", C.c_double)]


class JobResult(C.Structure):
    _fields_ = [("status", C.c_int), ("steps_done", C.c_int), ("queue_s", C.c_double), ("run_s", C.c_double),
                ("beta", _dp), ("gamma", _dp), ("z", _dp), ("chi", _dp), ("eps_inv", _dp), ("eps", _dp)]


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


def _srv_check(rc: int):
    if rc != LL_OK:
        raise LLError(rc, _lib.ll_server_last_error().decode())


class Server:
    """The request loop (ll_server_*): continuous batching of chains under an HBM budget."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, chunk: int | None = None):
        h = C.c_void_p()
        _srv_check(_lib.ll_server_create(C.c_size_t(int(hbm_budget_bytes)), int(max_slots), C.byref(h)))
        self._h = h
        self._jobs = {}
        if chunk:
            _srv_check(_lib.ll_server_set_chunk(self._h, int(chunk)))

    def submit(self, n_steps: int, omega_ev, eta_ev: float, **system) -> int:
        d, keep = _make_desc(**system)
        w = np.ascontiguousarray(omega_ev if omega_ev is not None else np.zeros(0), dtype=np.float64)
        jd = JobDesc()
        jd.sys = d
        jd.n_steps = int(n_steps)
        jd.omega_ev = _d(w) if len(w) else None
        jd.n_omega = len(w)
        jd.eta_ev = float(eta_ev)
        jid = C.c_uint64(0)
        _srv_check(_lib.ll_submit(self._h, C.byref(jd), C.byref(jid)))
        self._jobs[jid.value] = (int(n_steps), len(w))
        return jid.value

    def poll(self, job_id: int):
        """(state, result dict): status, steps_done, queue_s, run_s, and once the job has ended
        its coefficients and spectrum."""
        n, nw = self._jobs.get(job_id, (0, 0))
        out = dict(beta=np.zeros(n), gamma=np.zeros(n, dtype=np.complex128), z=np.zeros(n, dtype=np.complex128),
                   chi=np.zeros(nw, dtype=np.complex128), eps_inv=np.zeros(nw, dtype=np.complex128),
                   eps=np.zeros(nw, dtype=np.complex128))
        r = JobResult()
        for key in ("beta", "gamma", "z", "chi", "eps_inv", "eps"):
            setattr(r, key, _d(out[key].view(np.float64)) if out[key].size else None)
        st = C.c_int(0)
        _srv_check(_lib.ll_poll(self._h, C.c_uint64(job_id), C.byref(st), C.byref(r)))
        res = dict(status=r.status, steps_done=r.steps_done, queue_s=r.queue_s, run_s=r.run_s)
        if st.value in (JOB_DONE, JOB_FAILED):
            m = r.steps_done
            res.update(beta=out["beta"][:m], gamma=out["gamma"][:m], z=out["z"][:m], chi=out["chi"],
                       eps_inv=out["eps_inv"], eps=out["eps"])
            if st.value == JOB_FAILED:
                res["error"] = _lib.ll_server_last_error().decode()
        return st.value, res

    def cancel(self, job_id: int):
        """ll_cancel: a queued job ends at once, a running one after the current round; either
        ends FAILED with status LL_ECANCELED and keeps the coefficients of its finished steps."""
        _srv_check(_lib.ll_cancel(self._h, C.c_uint64(job_id)))

    def release(self, job_id: int):
        """ll_release: frees the record of an ended job (LL_PENDING while it runs)."""
        _srv_check(_lib.ll_release(self._h, C.c_uint64(job_id)))
        self._jobs.pop(job_id, None)

    def stats(self):
        used, peak = C.c_size_t(0), C.c_size_t(0)
        run, q = C.c_int(0), C.c_int(0)
        _srv_check(_lib.ll_server_stats(self._h, C.byref(used), C.byref(peak), C.byref(run), C.byref(q)))
        return dict(used=used.value, peak=peak.value, running=run.value, queued=q.value)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ll_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
