"""Python binding of the C ABI in include/lno_ot.h (ctypes; marshalling only).

Every step of the computation runs in the library's CUDA kernels; PyTorch is
used here only to hold device memory and to name the stream.  The library is
loaded from the package's ``_lib`` folder; if it is missing or fails to load,
``load_library`` raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes as C
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblno_ot.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lno_ot.h")

OK, EINVAL, EDEVICE, ENOMEM, ECUDA, ETIMEOUT, EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
FP64, BF16X3, TF32, BF16X6, BF16X10, BF16X15 = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": FP64, "bf16x3": BF16X3, "tf32": TF32, "bf16x6": BF16X6,
              "bf16x10": BF16X10, "bf16x15": BF16X15}
CASES = ("aaa", "aab", "abb", "bbb")


class Options(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("stream", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("tune_cache", C.c_char_p),
                ("keep_operands", C.c_int)]


class Domain(C.Structure):
    _fields_ = [("nbas", C.c_int), ("naux", C.c_int), ("nocc", C.c_int * 2),
                ("B", C.c_void_p * 2), ("eps", C.c_void_p * 2), ("t1", C.c_void_p * 2),
                ("t2aa", C.c_void_p), ("t2bb", C.c_void_p), ("t2ab", C.c_void_p),
                ("fov", C.c_void_p * 2), ("e_trip", C.c_void_p * 4),
                ("trip_sel", C.c_void_p * 4), ("n_sel", C.c_int64 * 4),
                ("e_orb", C.c_void_p * 2)]


class Result(C.Structure):
    _fields_ = [("e", C.c_double * 5), ("status", C.c_int)]


class Grad(C.Structure):
    _fields_ = [("dB", C.c_void_p * 2), ("deps", C.c_void_p * 2), ("dt1", C.c_void_p * 2),
                ("dt2aa", C.c_void_p), ("dt2bb", C.c_void_p), ("dt2ab", C.c_void_p),
                ("dfov", C.c_void_p * 2)]


class Central(C.Structure):
    _fields_ = [("nq", C.c_int), ("s", C.c_void_p), ("w", C.c_void_p), ("spin", C.c_int),
                ("nlmo", C.c_int), ("U", C.c_void_p), ("dE", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("ms_total", C.c_double), ("ms_stage", C.c_double),
                ("ms_contract", C.c_double), ("ms_energy", C.c_double),
                ("flops_algorithmic", C.c_double), ("flops_executed", C.c_double),
                ("tensor_flops", C.c_double), ("contract_launches", C.c_int64),
                ("energy_launches", C.c_int64), ("other_launches", C.c_int64),
                ("triplets", C.c_int64), ("elements", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def exported_names():
    """Function names the public header declares (LNO_OT_API)."""
    txt = open(HEADER).read()
    return re.findall(r"LNO_OT_API\s+[\w\s\*]+?\b(lno_ot_\w+)\s*\(", txt)


def load_library(build_if_missing=False):
    """Load (optionally build) the in-tree library; raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _b
        _b.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"lno_ot library not built: {LIB_PATH} (run __graft_entry__.build())")
    lib = C.CDLL(LIB_PATH)
    lib.lno_ot_init.argtypes = [C.POINTER(C.c_void_p), C.POINTER(Options)]
    lib.lno_ot_init.restype = C.c_int
    lib.lno_ot_destroy.argtypes = [C.c_void_p]
    lib.lno_ot_destroy.restype = None
    lib.lno_ot_energy.argtypes = [C.c_void_p, C.POINTER(Domain), C.POINTER(Result)]
    lib.lno_ot_energy.restype = C.c_int
    lib.lno_ot_energy_batched.argtypes = [C.c_void_p, C.c_int, C.POINTER(Domain),
                                          C.POINTER(Result)]
    lib.lno_ot_energy_batched.restype = C.c_int
    lib.lno_ot_backward.argtypes = [C.c_void_p, C.POINTER(Domain), C.c_double, C.POINTER(Grad)]
    lib.lno_ot_backward.restype = C.c_int
    lib.lno_ot_last_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    lib.lno_ot_last_stats.restype = C.c_int
    lib.lno_ot_strerror.argtypes = [C.c_int]
    lib.lno_ot_strerror.restype = C.c_char_p
    lib.lno_ot_version.argtypes = []
    lib.lno_ot_version.restype = C.c_char_p
    lib.lno_ot_last_error.argtypes = []
    lib.lno_ot_last_error.restype = C.c_char_p
    lib.lno_ot_energy_central.argtypes = [C.c_void_p, C.POINTER(Domain), C.POINTER(Central)]
    lib.lno_ot_energy_central.restype = C.c_int
    lib.lno_ot_release.argtypes = [C.c_void_p]
    lib.lno_ot_release.restype = C.c_int
    lib.lno_ot_naf.argtypes = [C.c_void_p, C.POINTER(Domain), C.c_double, C.c_void_p * 2,
                               C.POINTER(C.c_int), C.c_void_p]
    lib.lno_ot_naf.restype = C.c_int
    lib.lno_ot_laplace_quadrature.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int,
                                              C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]
    lib.lno_ot_laplace_quadrature.restype = C.c_int
    lib.lno_ot_selftest_gemm.argtypes = [C.c_int] * 5 + [C.c_void_p] * 4
    lib.lno_ot_selftest_gemm.restype = C.c_int
    lib.lno_ot_selftest_timeout.argtypes = [C.c_int, C.c_longlong, C.POINTER(C.c_int),
                                            C.c_void_p]
    lib.lno_ot_selftest_timeout.restype = C.c_int
    lib.lno_ot_selftest_energy_timeout.argtypes = [C.c_int, C.c_longlong, C.POINTER(C.c_int),
                                                   C.c_void_p]
    lib.lno_ot_selftest_energy_timeout.restype = C.c_int
    _lib = lib
    return lib


class LnoError(RuntimeError):
    def __init__(self, code, where=""):
        lib = load_library()
        msg = lib.lno_ot_strerror(code).decode()
        last = lib.lno_ot_last_error().decode()
        super().__init__(f"{where}: {msg} ({code}) {last}".strip())
        self.code = code


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _check_tensor(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 torch tensor")


def make_domain_struct(dom, e_trip=None, trip_sel=None, e_orb=None):
    """lno_ot_domain from a dict of device tensors (layouts as in the header).

    ``dom["fov"]`` (optional): list of 2 device tensors (or None) with the
    occupied-virtual Fock blocks; ``e_trip``: optional list of 4 device
    float64 tensors (or None); ``trip_sel``: optional list of 4 host int64
    numpy arrays (or None); ``e_orb``: optional list of 2 device float64
    tensors [nocc[s]] for the orbital contributions.
    Returns (struct, keepalive) -- keep ``keepalive`` until the call returns.
    """
    d = Domain()
    d.nbas, d.naux = int(dom["nbas"]), int(dom["naux"])
    d.nocc[0], d.nocc[1] = int(dom["nocc"][0]), int(dom["nocc"][1])
    for s in (0, 1):
        for key in ("B", "eps", "t1"):
            _check_tensor(dom[key][s], f"{key}[{s}]")
        d.B[s] = dom["B"][s].data_ptr()
        d.eps[s] = dom["eps"][s].data_ptr()
        d.t1[s] = dom["t1"][s].data_ptr()
    for key in ("t2aa", "t2bb", "t2ab"):
        _check_tensor(dom[key], key)
    d.t2aa, d.t2bb, d.t2ab = (dom["t2aa"].data_ptr(), dom["t2bb"].data_ptr(),
                              dom["t2ab"].data_ptr())
    keep = []
    fov = dom.get("fov")
    for s in (0, 1):
        if fov is not None and fov[s] is not None:
            _check_tensor(fov[s], f"fov[{s}]")
            d.fov[s] = fov[s].data_ptr()
        if e_orb is not None and e_orb[s] is not None:
            d.e_orb[s] = e_orb[s].data_ptr()
    for c in range(4):
        if e_trip is not None and e_trip[c] is not None:
            d.e_trip[c] = e_trip[c].data_ptr()
        if trip_sel is not None and trip_sel[c] is not None:
            import numpy as np
            a = np.ascontiguousarray(trip_sel[c], dtype=np.int64)
            n = a.size
            if n == 0:   # an empty selection still needs a non-NULL pointer
                a = np.zeros(1, dtype=np.int64)
            keep.append(a)
            d.trip_sel[c] = a.ctypes.data
            d.n_sel[c] = n
    return d, keep


class Context:
    """An lno_ot context (device, precision, stream)."""

    def __init__(self, device=0, precision="fp64", stream=None, workspace_bytes=0,
                 tune_cache=None, keep_operands=False):
        self.lib = load_library()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        if stream is None:  # order the library's work after torch's pending work
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream(device).cuda_stream or None
        self._tune = None if tune_cache is None else str(tune_cache).encode()
        opt = Options(device, prec, None if stream is None else C.c_void_p(stream), workspace_bytes,
                      self._tune, 1 if keep_operands else 0)
        h = C.c_void_p()
        rc = self.lib.lno_ot_init(C.byref(h), C.byref(opt))
        if rc != OK:
            raise LnoError(rc, "lno_ot_init")
        self.h = h
        self.precision = prec

    def close(self):
        if getattr(self, "h", None):
            self.lib.lno_ot_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def energy(self, dom, e_trip=None, trip_sel=None, raise_on_error=True, e_orb=None):
        """E(T) of one domain: dict aaa, aab, abb, bbb, total (floats)."""
        d, keep = make_domain_struct(dom, e_trip, trip_sel, e_orb)
        r = Result()
        rc = self.lib.lno_ot_energy(self.h, C.byref(d), C.byref(r))
        del keep
        if rc != OK and raise_on_error:
            raise LnoError(rc, "lno_ot_energy")
        out = dict(zip(CASES + ("total",), list(r.e)))
        out["status"] = rc
        return out

    def release(self):
        """Free the operands kept by keep_operands (lno_ot_release)."""
        rc = self.lib.lno_ot_release(self.h)
        if rc != OK:
            raise LnoError(rc, "lno_ot_release")

    def energy_raw(self, d):
        """Call lno_ot_energy on a prepared Domain struct; returns (rc, Result)."""
        r = Result()
        rc = self.lib.lno_ot_energy(self.h, C.byref(d), C.byref(r))
        return rc, r

    def energy_batched(self, doms):
        structs, keep = [], []
        for dm in doms:
            s, k = make_domain_struct(dm)
            structs.append(s)
            keep.append(k)
        arr = (Domain * len(structs))(*structs)
        res = (Result * len(structs))()
        rc = self.lib.lno_ot_energy_batched(self.h, len(structs), arr, res)
        out = [dict(zip(CASES + ("total",), list(r.e)), status=r.status) for r in res]
        return rc, out

    def backward(self, dom, gE, grads, trip_sel=None):
        """grads: dict with optional device tensors dB, deps (lists), dt1 (list),
        dt2aa, dt2bb, dt2ab; overwritten with gE * dE/d(input)."""
        d, keep = make_domain_struct(dom, trip_sel=trip_sel)
        g = Grad()
        for s in (0, 1):
            for key in ("dB", "deps", "dt1", "dfov"):
                if grads.get(key) is not None and grads[key][s] is not None:
                    getattr(g, key)[s] = grads[key][s].data_ptr()
        for key in ("dt2aa", "dt2bb", "dt2ab"):
            if grads.get(key) is not None:
                setattr(g, key, grads[key].data_ptr())
        rc = self.lib.lno_ot_backward(self.h, C.byref(d), C.c_double(gE), C.byref(g))
        if rc != OK:
            raise LnoError(rc, "lno_ot_backward")

    def energy_central(self, dom, spin, U, s, w):
        """dE of eq local_pt for each row of U (device float64 [nlmo][nocc[spin]],
        central orbitals of spin ``spin``) with the quadrature (s, w)."""
        import numpy as np
        _check_tensor(U, "U")
        d, keep = make_domain_struct(dom)
        sa = np.ascontiguousarray(s, dtype=np.float64)
        wa = np.ascontiguousarray(w, dtype=np.float64)
        out = np.zeros(max(int(U.shape[0]), 1))
        c = Central(int(sa.size), sa.ctypes.data, wa.ctypes.data, int(spin), int(U.shape[0]),
                    U.data_ptr(), out.ctypes.data)
        rc = self.lib.lno_ot_energy_central(self.h, C.byref(d), C.byref(c))
        del keep
        if rc != OK:
            raise LnoError(rc, "lno_ot_energy_central")
        return out[:int(U.shape[0])]

    def naf(self, dom, eps_naf=1e-2):
        """NAF compression of dom's B factors (Sec. 3.6): returns (dict like dom
        with B replaced by the compressed device tensors and naux by the number
        of NAFs, eigenvalues of W descending as a numpy array)."""
        import numpy as np
        import torch
        d, keep = make_domain_struct(dom)
        naux, nbas = int(dom["naux"]), int(dom["nbas"])
        outs = [torch.empty((naux, nbas, nbas), dtype=torch.float64, device=dom["B"][s].device)
                for s in (0, 1)]
        ptrs = (C.c_void_p * 2)(outs[0].data_ptr(), outs[1].data_ptr())
        nk = C.c_int(0)
        lam = np.zeros(naux)
        rc = self.lib.lno_ot_naf(self.h, C.byref(d), float(eps_naf), ptrs, C.byref(nk),
                                 lam.ctypes.data)
        del keep
        if rc != OK:
            raise LnoError(rc, "lno_ot_naf")
        k = nk.value
        out = dict(dom)
        out["B"] = [outs[0][:k].contiguous(), outs[1][:k].contiguous()]
        out["naux"] = k
        return out, lam

    def stats(self):
        st = Stats()
        rc = self.lib.lno_ot_last_stats(self.h, C.byref(st))
        if rc != OK:
            raise LnoError(rc, "lno_ot_last_stats")
        return st.as_dict()


def laplace_quadrature(xmin, xmax, tol=1e-2, nmax=16):
    """(s, w) numpy arrays from lno_ot_laplace_quadrature (host only)."""
    import numpy as np
    lib = load_library()
    s = np.zeros(32)
    w = np.zeros(32)
    n = C.c_int(0)
    rc = lib.lno_ot_laplace_quadrature(float(xmin), float(xmax), float(tol), int(nmax),
                                       s.ctypes.data, w.ctypes.data, C.byref(n))
    if rc != OK:
        raise LnoError(rc, "lno_ot_laplace_quadrature")
    return s[:n.value].copy(), w[:n.value].copy()


def to_device(dom, device="cuda"):
    """Domain dict of numpy arrays -> dict of contiguous float64 device tensors."""
    import torch

    def t(x):
        return torch.as_tensor(x, dtype=torch.float64).contiguous().to(device)
    out = dict(nbas=int(dom["nbas"]), naux=int(dom["naux"]),
               nocc=(int(dom["nocc"][0]), int(dom["nocc"][1])),
               B=[t(dom["B"][0]), t(dom["B"][1])], eps=[t(dom["eps"][0]), t(dom["eps"][1])],
               t1=[t(dom["t1"][0]), t(dom["t1"][1])], t2aa=t(dom["t2aa"]),
               t2bb=t(dom["t2bb"]), t2ab=t(dom["t2ab"]))
    if dom.get("fov") is not None:
        out["fov"] = [None if f is None else t(f) for f in dom["fov"]]
    return out


def _triples_autograd():
    import torch

    class LnoTriples(torch.autograd.Function):
        """E(T) of one domain as a differentiable scalar.

        Forward calls lno_ot_energy (the context's precision); backward calls
        lno_ot_backward (float64 adjoint, W recomputed per triplet).  Inputs
        are the device tensors of the domain (the two f_ov blocks may be
        None); gradients of B and of the same-spin T2 blocks are projected
        onto their symmetry.
        """

        @staticmethod
        def _dom(meta, Ba, Bb, ea, eb, t1a, t1b, t2aa, t2bb, t2ab, fa, fb):
            _, nocc, naux, _ = meta
            dom = dict(nbas=Ba.shape[1], naux=naux, nocc=nocc, B=[Ba, Bb], eps=[ea, eb],
                       t1=[t1a, t1b], t2aa=t2aa, t2bb=t2bb, t2ab=t2ab)
            if fa is not None or fb is not None:
                dom["fov"] = [fa, fb]
            return dom

        @staticmethod
        def forward(fctx, Ba, Bb, ea, eb, t1a, t1b, t2aa, t2bb, t2ab, fa, fb, meta):
            handle, trip_sel = meta[0], meta[3]
            dom = LnoTriples._dom(meta, Ba, Bb, ea, eb, t1a, t1b, t2aa, t2bb, t2ab, fa, fb)
            out = handle.energy(dom, trip_sel=trip_sel)
            fctx.save_for_backward(Ba, Bb, ea, eb, t1a, t1b, t2aa, t2bb, t2ab, fa, fb)
            fctx.meta = meta
            return torch.tensor(out["total"], dtype=torch.float64, device=Ba.device)

        @staticmethod
        def backward(fctx, gE):
            Ba, Bb, ea, eb, t1a, t1b, t2aa, t2bb, t2ab, fa, fb = fctx.saved_tensors
            handle, trip_sel = fctx.meta[0], fctx.meta[3]
            dom = LnoTriples._dom(fctx.meta, Ba, Bb, ea, eb, t1a, t1b, t2aa, t2bb, t2ab, fa, fb)
            need = fctx.needs_input_grad
            z = lambda x, k: torch.empty_like(x) if need[k] and x is not None else None
            g = dict(dB=[z(Ba, 0), z(Bb, 1)], deps=[z(ea, 2), z(eb, 3)], dt1=[z(t1a, 4), z(t1b, 5)],
                     dt2aa=z(t2aa, 6), dt2bb=z(t2bb, 7), dt2ab=z(t2ab, 8),
                     dfov=[z(fa, 9), z(fb, 10)])
            handle.backward(dom, float(gE), g, trip_sel=trip_sel)
            return (g["dB"][0], g["dB"][1], g["deps"][0], g["deps"][1], g["dt1"][0], g["dt1"][1],
                    g["dt2aa"], g["dt2bb"], g["dt2ab"], g["dfov"][0], g["dfov"][1], None)

    return LnoTriples


_LNO_FN = None


def triples_energy(ctx, dom, trip_sel=None):
    """Differentiable E(T) (torch scalar) of a domain dict of device tensors."""
    global _LNO_FN
    if _LNO_FN is None:
        _LNO_FN = _triples_autograd()
    fov = dom.get("fov") or [None, None]
    return _LNO_FN.apply(dom["B"][0], dom["B"][1], dom["eps"][0], dom["eps"][1], dom["t1"][0],
                         dom["t1"][1], dom["t2aa"], dom["t2bb"], dom["t2ab"], fov[0], fov[1],
                         (ctx, tuple(dom["nocc"]), int(dom["naux"]), trip_sel))
