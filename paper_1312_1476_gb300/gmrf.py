"""Python binding of the C ABI in include/gmrf.h (argument marshalling only).

Every computation runs in ``libgmrf.so``'s CUDA kernels.  Arrays may be
``torch`` tensors (CUDA or CPU) or ``numpy`` arrays; they are passed to the
library as raw pointers, which accepts host or device memory.  There is no
fallback: if the library is missing or fails to load, importing the module
raises.

Names follow the paper's notation: Q (precision), z (noise), x = Q^{-1/2} z
(Section 4, Algorithm 1), M (preconditioner, Proposition 1), log det Q
(Section 6).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgmrf.so")

OK = 0
ERR_INVALID = -1
ERR_OOM = -2
ERR_NOT_CONVERGED = -3
ERR_NOT_SPD = -4
ERR_NUMERIC = -5
ERR_CUDA = -6
ERR_TIMEOUT = -7
ERR_UNSUPPORTED = -8

BC = {"periodic": 0, "neumann": 1, "dirichlet": 2}
OP = {"shifted_laplacian": 0, "spde_squared": 1, "spde_plus_diag": 2}
PREC = {"none": 0, "circulant": 1, "mirror": 2}
PRECISION = {"fp32": 0, "fp64": 1}


class GmrfDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("bc", ctypes.c_int32), ("op", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("kappa2", ctypes.c_void_p), ("kappa2_const", ctypes.c_double),
                ("tau", ctypes.c_double), ("kappa2_precond", ctypes.c_double),
                ("precision", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GmrfSparseDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("rowptr", ctypes.c_void_p), ("colind", ctypes.c_void_p),
                ("val", ctypes.c_void_p), ("f_rowptr", ctypes.c_void_p), ("f_colind", ctypes.c_void_p),
                ("f_val", ctypes.c_void_p), ("tau", ctypes.c_double), ("precision", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GmrfSampleOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("m_max", ctypes.c_int32), ("nsamples", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("z_in", ctypes.c_void_p), ("check_every", ctypes.c_int32),
                ("v_storage", ctypes.c_int32)]


class GmrfResultInfo(ctypes.Structure):
    _fields_ = [("m_used", ctypes.c_int32), ("status", ctypes.c_int32), ("err_est", ctypes.c_double)]


class GmrfLogdetOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("m_max", ctypes.c_int32), ("nprobes", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("probes_in", ctypes.c_void_p), ("check_every", ctypes.c_int32),
                ("colour_dist", ctypes.c_int32)]


class GmrfSolveOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("m_max", ctypes.c_int32), ("nrhs", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GmrfServerOpts(ctypes.Structure):
    _fields_ = [("nslots", ctypes.c_int32), ("m_max", ctypes.c_int32), ("tol", ctypes.c_double),
                ("check_every", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GmrfTuning(ctypes.Structure):
    _fields_ = [("block_width", ctypes.c_int32), ("zchunk", ctypes.c_int32), ("vec_steps_per_s", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("host_loop", ctypes.c_int32)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgmrf.so is not built; run paper_1312_1476_gb300._build.build() "
                          "(or __graft_entry__.build()) first")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.c_void_p
    sig = {
        "gmrf_create": (ctypes.c_int, [ctypes.POINTER(GmrfDesc), P, ctypes.POINTER(P)]),
        "gmrf_size": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_sample": (ctypes.c_int, [P, ctypes.POINTER(GmrfSampleOpts), P, ctypes.POINTER(GmrfResultInfo)]),
        "gmrf_logdet": (ctypes.c_int, [P, ctypes.POINTER(GmrfLogdetOpts), ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(GmrfResultInfo)]),
        "gmrf_solve": (ctypes.c_int, [P, ctypes.POINTER(GmrfSolveOpts), P, P, ctypes.POINTER(GmrfResultInfo)]),
        "gmrf_sample_logdet": (ctypes.c_int, [P, ctypes.POINTER(GmrfSampleOpts), ctypes.POINTER(GmrfLogdetOpts), P,
                                              ctypes.POINTER(GmrfResultInfo), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(GmrfResultInfo)]),
        "gmrf_submit_sample": (ctypes.c_int, [P, ctypes.POINTER(GmrfSampleOpts), P, ctypes.POINTER(GmrfResultInfo),
                                              ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_submit_logdet": (ctypes.c_int, [P, ctypes.POINTER(GmrfLogdetOpts), ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), P, ctypes.POINTER(GmrfResultInfo),
                                              ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_submit_solve": (ctypes.c_int, [P, ctypes.POINTER(GmrfSolveOpts), P, P, ctypes.POINTER(GmrfResultInfo),
                                             ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_poll": (ctypes.c_int, [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]),
        "gmrf_wait": (ctypes.c_int, [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32)]),
        "gmrf_apply": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int64, P, P]),
        "gmrf_rng": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, ctypes.c_int64,
                                    ctypes.c_uint64, P, P]),
        "gmrf_trace": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_apply_inv_sqrt_noalloc": (ctypes.c_int, [P, ctypes.c_int64, P, P]),
        "gmrf_autotune": (ctypes.c_int, [P, ctypes.c_int32, ctypes.POINTER(GmrfTuning)]),
        "gmrf_set_tuning": (ctypes.c_int, [P, ctypes.POINTER(GmrfTuning)]),
        "gmrf_create_sparse": (ctypes.c_int, [ctypes.POINTER(GmrfSparseDesc), P, ctypes.POINTER(P)]),
        "gmrf_ichol": (ctypes.c_int, [ctypes.c_int64, P, P, P, ctypes.c_double, ctypes.c_double, ctypes.c_int64,
                                      P, P, P, ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_server_create": (ctypes.c_int, [P, ctypes.POINTER(GmrfServerOpts), ctypes.POINTER(P)]),
        "gmrf_server_submit": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double, P,
                                              ctypes.POINTER(ctypes.c_int64)]),
        "gmrf_server_step": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32)]),
        "gmrf_server_poll": (ctypes.c_int, [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                            ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(GmrfResultInfo),
                                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
        "gmrf_server_destroy": (None, [P]),
        "gmrf_destroy": (None, [P]),
        "gmrf_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


class GmrfError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s: %s (%d)" % (what, _lib.gmrf_strerror(code).decode(), code))


def strerror(code: int) -> str:
    return _lib.gmrf_strerror(code).decode()


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError("expected a torch tensor or numpy array, got %r" % type(a))


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


@dataclass
class SampleInfo:
    m_used: int
    status: int
    err_est: float


class Problem:
    """A lattice GMRF precision Q (gmrf_create) with its sampler and log det."""

    def __init__(self, shape, bc="periodic", op="shifted_laplacian", kappa2=None, kappa2_const=0.0, tau=1.0,
                 precond="none", kappa2_precond=0.0, precision="fp32", stream=None):
        shape = tuple(int(s) for s in shape)
        if len(shape) not in (2, 3):
            raise ValueError("shape must be (ny, nx) or (nz, ny, nx)")
        d = GmrfDesc()
        d.dim = len(shape)
        d.bc = BC[bc]
        d.op = OP[op]
        d.precond = PREC[precond]
        d.nx = shape[-1]
        d.ny = shape[-2]
        d.nz = shape[0] if len(shape) == 3 else 1
        self._kappa2 = None
        if kappa2 is not None:
            if hasattr(kappa2, "dtype") and str(kappa2.dtype) not in ("float32", "torch.float32"):
                raise TypeError("kappa2 must be float32")
            self._kappa2 = kappa2
            d.kappa2 = _ptr(kappa2)
        else:
            d.kappa2 = None
        d.kappa2_const = float(kappa2_const)
        d.tau = float(tau)
        d.kappa2_precond = float(kappa2_precond)
        d.precision = PRECISION[precision]
        d.reserved = 0
        self.shape = shape
        self.precision = precision
        self.n = int(np.prod(shape))
        self._h = ctypes.c_void_p()
        rc = _lib.gmrf_create(ctypes.byref(d), _stream(stream), ctypes.byref(self._h))
        if rc != OK:
            raise GmrfError(rc, "gmrf_create")
        self._stream = stream
        self._tickets = []  # submitted calls: their buffers live until close()

    @property
    def dtype(self):
        return np.float64 if self.precision == "fp64" else np.float32

    def close(self):
        for sv in list(getattr(self, "_servers", [])):
            sv.close()                  # a server is destroyed before its problem
        if self._h:
            _lib.gmrf_destroy(self._h)  # runs what was submitted first
            self._h = ctypes.c_void_p()
        self._tickets = []              # their buffers may go now

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def sample(self, out, nsamples=1, tol=1e-6, m_max=300, seed=2, z=None, check_every=16, raise_on_error=True,
               v_storage="native"):
        """x ~= Q^{-1/2} z into ``out`` ([nsamples][n], host or device); returns
        (return code, list of SampleInfo).  v_storage "bf16" keeps the basis
        for the assembly in bfloat16 (FP32 problems; see include/gmrf.h)."""
        o = GmrfSampleOpts(float(tol), int(m_max), int(nsamples), int(seed) & (2 ** 64 - 1),
                           _ptr(z) if z is not None else None, int(check_every), VSTORE[v_storage])
        info = (GmrfResultInfo * int(nsamples))()
        rc = _lib.gmrf_sample(self._h, ctypes.byref(o), _ptr(out), info)
        infos = [SampleInfo(i.m_used, i.status, i.err_est) for i in info]
        if raise_on_error and rc not in (OK, ERR_NOT_CONVERGED):
            raise GmrfError(rc, "gmrf_sample")
        return rc, infos

    def logdet(self, nprobes=16, tol=1e-6, m_max=300, seed=3, probes=None, check_every=16, raise_on_error=True,
               colour_dist=0):
        """Hutchinson / Lanczos-quadrature log det Q; returns
        (logdet, std_err, q array, list of SampleInfo, return code).  With
        colour_dist p > 0 the coloured estimator runs (p + 1)^dim quadratures
        per draw; q and the infos then have nprobes * (p + 1)^dim entries."""
        o = GmrfLogdetOpts(float(tol), int(m_max), int(nprobes), int(seed) & (2 ** 64 - 1),
                           _ptr(probes) if probes is not None else None, int(check_every), int(colour_dist))
        ld = ctypes.c_double()
        se = ctypes.c_double()
        nq = int(nprobes) * (int(colour_dist) + 1) ** len(self.shape)
        q = np.zeros(nq, dtype=np.float64)
        info = (GmrfResultInfo * nq)()
        rc = _lib.gmrf_logdet(self._h, ctypes.byref(o), ctypes.byref(ld), ctypes.byref(se),
                              ctypes.c_void_p(q.ctypes.data), info)
        infos = [SampleInfo(i.m_used, i.status, i.err_est) for i in info]
        if raise_on_error and rc not in (OK, ERR_NOT_CONVERGED):
            raise GmrfError(rc, "gmrf_logdet")
        return ld.value, se.value, q, infos, rc

    def sample_logdet(self, out, nsamples=1, nprobes=16, tol=1e-6, m_max=300, seed=2, probe_seed=3, z=None,
                      probes=None, check_every=16, colour_dist=0, raise_on_error=True):
        """Samples and log-det probes in one Lanczos batch (bitwise the results
        of ``sample`` and ``logdet`` with the same arguments); returns
        (return code, sample infos, logdet, std_err, q array, probe infos)."""
        so = GmrfSampleOpts(float(tol), int(m_max), int(nsamples), int(seed) & (2 ** 64 - 1),
                            _ptr(z) if z is not None else None, int(check_every), VSTORE["native"])
        lo = GmrfLogdetOpts(float(tol), int(m_max), int(nprobes), int(probe_seed) & (2 ** 64 - 1),
                            _ptr(probes) if probes is not None else None, int(check_every), int(colour_dist))
        nq = int(nprobes) * (int(colour_dist) + 1) ** len(self.shape)
        sinfo = (GmrfResultInfo * int(nsamples))()
        linfo = (GmrfResultInfo * nq)()
        ld = ctypes.c_double()
        se = ctypes.c_double()
        q = np.zeros(nq, dtype=np.float64)
        rc = _lib.gmrf_sample_logdet(self._h, ctypes.byref(so), ctypes.byref(lo), _ptr(out), sinfo,
                                     ctypes.byref(ld), ctypes.byref(se), ctypes.c_void_p(q.ctypes.data), linfo)
        sinfos = [SampleInfo(i.m_used, i.status, i.err_est) for i in sinfo]
        linfos = [SampleInfo(i.m_used, i.status, i.err_est) for i in linfo]
        if raise_on_error and rc not in (OK, ERR_NOT_CONVERGED):
            raise GmrfError(rc, "gmrf_sample_logdet")
        return rc, sinfos, ld.value, se.value, q, linfos

    # ---- asynchronous calls: return a Ticket at once (see include/gmrf.h)
    def _track(self, t):
        self._tickets = [x for x in self._tickets if x.rc is None] + [t]
        return t

    def submit_sample(self, out, nsamples=1, tol=1e-6, m_max=300, seed=2, z=None, check_every=16,
                      v_storage="native"):
        o = GmrfSampleOpts(float(tol), int(m_max), int(nsamples), int(seed) & (2 ** 64 - 1),
                           _ptr(z) if z is not None else None, int(check_every), VSTORE[v_storage])
        info = (GmrfResultInfo * int(nsamples))()
        t = ctypes.c_int64()
        rc = _lib.gmrf_submit_sample(self._h, ctypes.byref(o), _ptr(out), info, ctypes.byref(t))
        if rc != OK:
            raise GmrfError(rc, "gmrf_submit_sample")
        return self._track(Ticket(self, t.value, "sample", info, keep=(out, z)))

    def submit_logdet(self, nprobes=16, tol=1e-6, m_max=300, seed=3, probes=None, check_every=16, colour_dist=0):
        o = GmrfLogdetOpts(float(tol), int(m_max), int(nprobes), int(seed) & (2 ** 64 - 1),
                           _ptr(probes) if probes is not None else None, int(check_every), int(colour_dist))
        nq = int(nprobes) * (int(colour_dist) + 1) ** len(self.shape)
        info = (GmrfResultInfo * nq)()
        q = np.zeros(nq, dtype=np.float64)
        ld, se = ctypes.c_double(), ctypes.c_double()
        t = ctypes.c_int64()
        rc = _lib.gmrf_submit_logdet(self._h, ctypes.byref(o), ctypes.byref(ld), ctypes.byref(se),
                                     ctypes.c_void_p(q.ctypes.data), info, ctypes.byref(t))
        if rc != OK:
            raise GmrfError(rc, "gmrf_submit_logdet")
        return self._track(Ticket(self, t.value, "logdet", info, keep=(probes, q, ld, se), logdet=(ld, se, q)))

    def submit_solve(self, b, out, nrhs=1, tol=1e-6, m_max=300, check_every=16):
        o = GmrfSolveOpts(float(tol), int(m_max), int(nrhs), int(check_every), 0)
        info = (GmrfResultInfo * int(nrhs))()
        t = ctypes.c_int64()
        rc = _lib.gmrf_submit_solve(self._h, ctypes.byref(o), _ptr(b), _ptr(out), info, ctypes.byref(t))
        if rc != OK:
            raise GmrfError(rc, "gmrf_submit_solve")
        return self._track(Ticket(self, t.value, "solve", info, keep=(b, out)))

    def solve(self, b, out, nrhs=1, tol=1e-6, m_max=300, check_every=16, raise_on_error=True):
        """x = Q^{-1} b into ``out`` ([nrhs][n], host or device) by the Lanczos
        form of (preconditioned) conjugate gradients; returns (return code,
        list of SampleInfo with err_est = the relative residual)."""
        o = GmrfSolveOpts(float(tol), int(m_max), int(nrhs), int(check_every), 0)
        info = (GmrfResultInfo * int(nrhs))()
        rc = _lib.gmrf_solve(self._h, ctypes.byref(o), _ptr(b), _ptr(out), info)
        infos = [SampleInfo(i.m_used, i.status, i.err_est) for i in info]
        if raise_on_error and rc not in (OK, ERR_NOT_CONVERGED):
            raise GmrfError(rc, "gmrf_solve")
        return rc, infos

    def apply_inv_sqrt_noalloc(self, v, y, nvec=1):
        """y = M^{-1/2} v without any device allocation (device pointers only;
        scratch in a fixed library-wide device array, see include/gmrf.h)."""
        rc = _lib.gmrf_apply_inv_sqrt_noalloc(self._h, int(nvec), _ptr(v), _ptr(y))
        if rc != OK:
            raise GmrfError(rc, "gmrf_apply_inv_sqrt_noalloc")

    def autotune(self, nvec_max):
        """Times candidate block widths (and 3-D z chunks) and keeps the best
        for later calls; returns the choice as a dict."""
        t = GmrfTuning()
        rc = _lib.gmrf_autotune(self._h, int(nvec_max), ctypes.byref(t))
        if rc != OK:
            raise GmrfError(rc, "gmrf_autotune")
        return {"block_width": t.block_width, "zchunk": t.zchunk, "vec_steps_per_s": t.vec_steps_per_s,
                "candidates": t.candidates, "host_loop": bool(t.host_loop)}

    def set_tuning(self, block_width=0, zchunk=0, host_loop=False):
        """Explicit tuning (0 = library default for either field); host_loop
        True: host-replayed step graphs instead of the device-side loop."""
        t = GmrfTuning(int(block_width), int(zchunk), 0.0, 0, 1 if host_loop else 0)
        rc = _lib.gmrf_set_tuning(self._h, ctypes.byref(t))
        if rc != OK:
            raise GmrfError(rc, "gmrf_set_tuning")

    def apply(self, which, v, y, nvec=1):
        """which 0: y = Q v; 1: y = A v (preconditioned operator); 2: y = M^{-1/2} v."""
        rc = _lib.gmrf_apply(self._h, int(which), int(nvec), _ptr(v), _ptr(y))
        if rc != OK:
            raise GmrfError(rc, "gmrf_apply")


class Server:
    """Continuous batching over one problem (gmrf_server_*): a table of
    ``nslots`` resident vector slots that the requests' samples and probes
    share; see include/gmrf.h.  While it exists the problem serves it alone."""

    def __init__(self, prob, nslots, m_max=300, tol=1e-6, check_every=16):
        self.prob = prob
        self._h = ctypes.c_void_p()
        o = GmrfServerOpts(int(nslots), int(m_max), float(tol), int(check_every), 0)
        rc = _lib.gmrf_server_create(prob._h, ctypes.byref(o), ctypes.byref(self._h))
        if rc != OK:
            raise GmrfError(rc, "gmrf_server_create")
        self._keep = {}  # request id -> output buffer (kept alive until polled)
        if not hasattr(prob, "_servers"):
            prob._servers = []
        prob._servers.append(self)

    def submit_sample(self, out, count, seed, tau=1.0):
        """count samples (the streams of Problem.sample(seed=seed)) into the
        device buffer ``out`` [count][n]; returns the request id."""
        r = ctypes.c_int64()
        rc = _lib.gmrf_server_submit(self._h, 0, int(count), int(seed) & (2 ** 64 - 1), float(tau), _ptr(out),
                                     ctypes.byref(r))
        if rc != OK:
            raise GmrfError(rc, "gmrf_server_submit")
        self._keep[r.value] = (out, int(count))
        return r.value

    def submit_logdet(self, nprobes, seed, tau=1.0):
        """A log det with nprobes Rademacher probes (Problem.logdet's streams)."""
        r = ctypes.c_int64()
        rc = _lib.gmrf_server_submit(self._h, 1, int(nprobes), int(seed) & (2 ** 64 - 1), float(tau), None,
                                     ctypes.byref(r))
        if rc != OK:
            raise GmrfError(rc, "gmrf_server_submit")
        self._keep[r.value] = (None, int(nprobes))
        return r.value

    def step(self):
        """One round: admit, run check_every steps, finish; returns the number
        of vectors running or waiting."""
        a = ctypes.c_int32()
        rc = _lib.gmrf_server_step(self._h, ctypes.byref(a))
        if rc != OK:
            raise GmrfError(rc, "gmrf_server_step")
        return a.value

    def poll(self, req):
        """None while request req runs; then (result code, list of SampleInfo,
        logdet, std_err) and the request is forgotten."""
        done, res = ctypes.c_int32(), ctypes.c_int32()
        count = self._keep[req][1]
        info = (GmrfResultInfo * count)()
        ld, se = ctypes.c_double(), ctypes.c_double()
        rc = _lib.gmrf_server_poll(self._h, int(req), ctypes.byref(done), ctypes.byref(res), info, ctypes.byref(ld),
                                   ctypes.byref(se))
        if rc != OK:
            raise GmrfError(rc, "gmrf_server_poll")
        if not done.value:
            return None
        del self._keep[req]
        return res.value, [SampleInfo(i.m_used, i.status, i.err_est) for i in info], ld.value, se.value

    def close(self):
        if self._h:
            _lib.gmrf_server_destroy(self._h)
            self._h = ctypes.c_void_p()
        self._keep = {}
        if self in getattr(self.prob, "_servers", []):
            self.prob._servers.remove(self)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ticket:
    """An asynchronous call in flight: holds its buffers until it completes."""

    def __init__(self, prob, ticket, kind, info, keep=(), logdet=None):
        self.prob, self.ticket, self.kind, self._info, self._keep, self._ld = prob, ticket, kind, info, keep, logdet
        self.rc = None

    def poll(self):
        """True once the call has completed (its return code is then in .rc)."""
        if self.rc is not None:
            return True
        d, r = ctypes.c_int32(), ctypes.c_int32()
        rc = _lib.gmrf_poll(self.prob._h, self.ticket, ctypes.byref(d), ctypes.byref(r))
        if rc != OK:
            raise GmrfError(rc, "gmrf_poll")
        if d.value:
            self.rc = r.value
        return bool(d.value)

    def wait(self):
        """Blocks until completion; returns (return code, infos) or, for a log
        det, (logdet, std_err, q, infos, return code) as the synchronous calls."""
        if self.rc is None:
            r = ctypes.c_int32()
            rc = _lib.gmrf_wait(self.prob._h, self.ticket, ctypes.byref(r))
            if rc != OK:
                raise GmrfError(rc, "gmrf_wait")
            self.rc = r.value
        infos = [SampleInfo(i.m_used, i.status, i.err_est) for i in self._info]
        if self.kind == "logdet":
            ld, se, q = self._ld
            return ld.value, se.value, q, infos, self.rc
        return self.rc, infos


def rng(kind, nvec, n, seed, out, precision="fp32", stream=None):
    """Device Philox streams: kind 0 Gaussian, 1 Rademacher, 2 raw words."""
    rc = _lib.gmrf_rng(int(kind), PRECISION[precision], int(nvec), int(n), int(seed) & (2 ** 64 - 1),
                       _ptr(out), _stream(stream))
    if rc != OK:
        raise GmrfError(rc, "gmrf_rng")


VSTORE = {"native": 0, "bf16": 1, "none": 2}
KERNEL_CLASSES = {"stencil_step": 0, "pre_row_fwd": 1, "pre_col": 2, "pre_row_mid": 3, "pre_row_last": 4,
                  "init": 5, "rng": 6, "tm": 7, "assemble": 8, "pre_apply": 9, "other": 10, "sparse_step": 11}


def trace_reset():
    _lib.gmrf_trace(0, -1, None, None, None)


def trace_timing(enable: bool):
    _lib.gmrf_trace(1 if enable else 2, -1, None, None, None)


def trace_query(kclass="all"):
    """(total kernel ms, launches, timed launches) of a kernel class or all."""
    k = -1 if kclass == "all" else KERNEL_CLASSES[kclass]
    ms = ctypes.c_double()
    la = ctypes.c_int64()
    ti = ctypes.c_int64()
    rc = _lib.gmrf_trace(3, k, ctypes.byref(ms), ctypes.byref(la), ctypes.byref(ti))
    if rc != OK:
        raise GmrfError(rc, "gmrf_trace")
    return ms.value, la.value, ti.value


# ---------------------------------------------------------------- sparse Q
def _csr_parts(Q):
    """(n, rowptr int64, colind int32, val float64) from a scipy sparse matrix
    or a (rowptr, colind, val) triple (argument marshalling only)."""
    if isinstance(Q, tuple):
        rowptr, colind, val = Q
    else:
        Q = Q.tocsr()
        rowptr, colind, val = Q.indptr, Q.indices, Q.data
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return len(rowptr) - 1, rowptr, colind, val


def ichol(Q, droptol=-1.0, shift=0.0):
    """Threshold incomplete Cholesky factor F of Q + shift diag(Q) (gmrf_ichol;
    droptol < 0: IC(0)).  Returns (f_rowptr, f_colind, f_val) CSR arrays."""
    n, rp, ci, va = _csr_parts(Q)
    nnz = ctypes.c_int64()
    f_rowptr = np.zeros(n + 1, dtype=np.int64)
    rc = _lib.gmrf_ichol(n, _ptr(rp), _ptr(ci), _ptr(va), float(droptol), float(shift), 0, _ptr(f_rowptr), None,
                         None, ctypes.byref(nnz))
    if rc != OK:
        raise GmrfError(rc, "gmrf_ichol (column %d)" % nnz.value if rc == ERR_NOT_SPD else "gmrf_ichol")
    f_col = np.zeros(nnz.value, dtype=np.int32)
    f_val = np.zeros(nnz.value, dtype=np.float64)
    rc = _lib.gmrf_ichol(n, _ptr(rp), _ptr(ci), _ptr(va), float(droptol), float(shift), nnz.value, _ptr(f_rowptr),
                         _ptr(f_col), _ptr(f_val), ctypes.byref(nnz))
    if rc != OK:
        raise GmrfError(rc, "gmrf_ichol")
    return f_rowptr, f_col, f_val


class SparseProblem(Problem):
    """A general sparse precision tau Q in CSR (gmrf_create_sparse), optionally
    preconditioned by an incomplete-Cholesky factor F (M = F F^T, Section 5.2).
    Q and F: scipy sparse matrices or (rowptr, colind, val) triples."""

    def __init__(self, Q, F=None, tau=1.0, precision="fp32", stream=None):
        n, rp, ci, va = _csr_parts(Q)
        d = GmrfSparseDesc()
        d.n = n
        d.rowptr, d.colind, d.val = _ptr(rp), _ptr(ci), _ptr(va)
        keep = [rp, ci, va]
        if F is not None:
            fn, frp, fci, fva = _csr_parts(F)
            if fn != n:
                raise ValueError("F must be n x n")
            d.f_rowptr, d.f_colind, d.f_val = _ptr(frp), _ptr(fci), _ptr(fva)
            keep += [frp, fci, fva]
        else:
            d.f_rowptr = d.f_colind = d.f_val = None
        d.tau = float(tau)
        d.precision = PRECISION[precision]
        d.reserved = 0
        self.shape = (n,)
        self.precision = precision
        self.n = n
        self._kappa2 = None
        self._h = ctypes.c_void_p()
        rc = _lib.gmrf_create_sparse(ctypes.byref(d), _stream(stream), ctypes.byref(self._h))
        del keep
        if rc != OK:
            raise GmrfError(rc, "gmrf_create_sparse")
        self._stream = stream
        self._tickets = []
