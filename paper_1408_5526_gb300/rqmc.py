"""Thin ctypes binding of librqmc.so (include/rqmc.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current CUDA stream.
The library must have been built (``__graft_entry__.build()`` or
``python paper_1408_5526_gb300/_build.py``); there is no CPU fallback and a
missing library raises ``RuntimeError``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librqmc.so")

HALTON_RS, RASRAP, SOBOL_DS, PHILOX, SOBOL_LMS = 0, 1, 2, 3, 4
FP64, FP32 = 0, 1
UNIFORM, NORMAL, RAW = 0, 1, 2
_SEQ = {"halton_rs": HALTON_RS, "rasrap": RASRAP, "sobol_ds": SOBOL_DS, "philox": PHILOX, "sobol_lms": SOBOL_LMS}
_PREC = {"fp64": FP64, "fp32": FP32}
_TR = {"uniform": UNIFORM, "normal": NORMAL, "raw": RAW}
STATUS = {0: "RQMC_OK", 1: "RQMC_EINVAL", 2: "RQMC_ENOMEM", 3: "RQMC_ECUDA", 4: "RQMC_ETIMEOUT",
          5: "RQMC_EUNSUPPORTED", 6: "RQMC_ENOTABLE"}

# every symbol include/rqmc.h declares
EXPORTS = ["rqmc_set_sobol_table", "rqmc_points", "rqmc_integrate_product", "price_caplets", "price_mbs",
           "price_adjoint", "price_batch", "rqmc_plan_product", "rqmc_plan_caplets", "rqmc_plan_mbs",
           "rqmc_plan_adjoint", "rqmc_plan_batch", "rqmc_plan_output_size", "rqmc_plan_launches",
           "rqmc_plan_set_launch", "rqmc_plan_execute", "rqmc_plan_check", "rqmc_plan_destroy",
           "rqmc_status_string", "rqmc_last_error", "rqmc_abi_version", "rqmc_price_caplets_noalloc",
           "rqmc_plan_points", "rqmc_probe_pipes", "rqmc_plan_batch_stats", "rqmc_plan_get_launch"]


class RqmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LmmParams(C.Structure):
    _fields_ = [("n_fwd", C.c_int), ("n_factors", C.c_int), ("scheme", C.c_int), ("init", C.c_int),
                ("delta", C.c_double), ("L0", C.POINTER(C.c_double)), ("vol", C.POINTER(C.c_double)),
                ("loadings", C.POINTER(C.c_double))]


class MbsParams(C.Structure):
    _fields_ = [("months", C.c_int), ("reserved", C.c_int), ("i0", C.c_double), ("K1", C.c_double),
                ("K2", C.c_double), ("K3", C.c_double), ("K4", C.c_double), ("sigma", C.c_double),
                ("c", C.c_double)]


class Instrument(C.Structure):
    _fields_ = [("kind", C.c_int), ("size", C.c_int), ("N", C.c_int64), ("rate", C.c_double),
                ("vol", C.c_double), ("strike", C.c_double), ("mbs", MbsParams)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load librqmc.so and hand it the Joe-Kuo Sobol' table; raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"librqmc.so not built ({path}); run __graft_entry__.build() -- no CPU fallback")
        L = C.CDLL(path)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
        st = C.c_int
        L.rqmc_set_sobol_table.argtypes = [C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int, C.c_int]
        L.rqmc_points.argtypes = [C.c_int, i64, C.c_int, C.c_int, C.c_uint64, i64, C.c_int, C.c_int, vp, vp]
        L.rqmc_integrate_product.argtypes = [C.c_int, i64, C.c_int, C.c_int, C.c_uint64, dp, C.c_int, dp, dp, dp, vp]
        L.price_caplets.argtypes = [C.POINTER(LmmParams), dp, C.c_int, i64, C.c_int, C.c_int, C.c_uint64, C.c_int,
                                    dp, dp, dp, vp]
        L.price_mbs.argtypes = [C.POINTER(MbsParams), i64, C.c_int, C.c_int, C.c_uint64, C.c_int, dp, dp, dp, vp]
        L.price_adjoint.argtypes = [C.POINTER(LmmParams), dp, C.c_int, dp, i64, C.c_int, C.c_int, C.c_uint64,
                                    C.c_int, C.c_int, dp, dp, dp, vp]
        L.rqmc_price_caplets_noalloc.argtypes = [C.POINTER(LmmParams), dp, C.c_int, i64, C.c_int, C.c_int,
                                                 C.c_uint64, C.c_int, dp, vp]
        L.price_batch.argtypes = [C.POINTER(Instrument), C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, dp, vp]
        pp = C.POINTER(vp)
        L.rqmc_plan_product.argtypes = [C.c_int, i64, i64, C.c_int, C.c_int, C.c_uint64, dp, C.c_int, pp]
        L.rqmc_plan_caplets.argtypes = [C.POINTER(LmmParams), dp, C.c_int, i64, i64, C.c_int, C.c_int, C.c_uint64,
                                        C.c_int, pp]
        L.rqmc_plan_mbs.argtypes = [C.POINTER(MbsParams), i64, i64, C.c_int, C.c_int, C.c_uint64, C.c_int, pp]
        L.rqmc_plan_adjoint.argtypes = [C.POINTER(LmmParams), dp, C.c_int, dp, i64, i64, C.c_int, C.c_int,
                                        C.c_uint64, C.c_int, C.c_int, pp]
        L.rqmc_plan_batch.argtypes = [C.POINTER(Instrument), C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_int, pp]
        L.rqmc_plan_points.argtypes = [C.c_int, i64, i64, C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_int, pp]
        L.rqmc_probe_pipes.argtypes = [dp, C.c_int]
        L.rqmc_plan_batch_stats.argtypes = [vp, dp, C.c_int]
        L.rqmc_plan_output_size.argtypes = [vp]
        L.rqmc_plan_output_size.restype = i64
        L.rqmc_plan_launches.argtypes = [vp]
        L.rqmc_plan_set_launch.argtypes = [vp, C.c_int, C.c_int]
        L.rqmc_plan_get_launch.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.rqmc_plan_execute.argtypes = [vp, dp, vp]
        L.rqmc_plan_check.argtypes = [vp, vp]
        L.rqmc_plan_destroy.argtypes = [vp]
        L.rqmc_status_string.argtypes = [st]
        L.rqmc_status_string.restype = C.c_char_p
        L.rqmc_last_error.restype = C.c_char_p
        for name in EXPORTS:
            getattr(L, name)
        poly, vinit = inputs.joe_kuo_table()
        n = min(len(poly), 4096)
        _check(L, L.rqmc_set_sobol_table(poly.ctypes.data_as(C.POINTER(C.c_int64)),
                                         vinit.ctypes.data_as(C.POINTER(C.c_int64)), n, vinit.shape[1]))
        _lib = L
        return L


def _check(L, status):
    if status != 0:
        raise RqmcError(status, L.rqmc_last_error().decode())


def _check_out(t, n: int, dtype, what: str):
    """A caller's output tensor must hold n elements of dtype, contiguous, on a CUDA device:
    the library writes through the raw pointer and cannot check it."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{what}: a torch tensor is required")
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() < n:
        raise ValueError(f"{what}: need a contiguous CUDA {dtype} tensor of at least {n} elements, got "
                         f"{t.dtype} {tuple(t.shape)} on {t.device}")


def _enum(v, table):
    return table[v] if isinstance(v, str) else int(v)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


def _lmm_struct(lmm: dict, keep: list) -> LmmParams:
    """The model dict as rqmc_lmm_params: the initial curve is "B0" (bond prices B_0..B_nf+1,
    converted by the library with eq. BL) when present, else "L0" (forwards L_0..L_nf)."""
    bonds = lmm.get("B0") is not None
    L0 = np.ascontiguousarray(lmm["B0"] if bonds else lmm["L0"], dtype=np.float64)
    vol = np.ascontiguousarray(lmm["vol"], dtype=np.float64)
    keep += [L0, vol]
    st = LmmParams(int(lmm["n_fwd"]), int(lmm.get("d", 1)), int(lmm.get("scheme", 0)), 1 if bonds else 0,
                   float(lmm["delta"]), _dp(L0), _dp(vol), None)
    if lmm.get("loadings") is not None:
        ld = np.ascontiguousarray(lmm["loadings"], dtype=np.float64)
        keep.append(ld)
        st.loadings = _dp(ld)
    return st


def _mbs_struct(mbs: dict) -> MbsParams:
    return MbsParams(int(mbs["months"]), 0, float(mbs["i0"]), float(mbs["K1"]), float(mbs["K2"]),
                     float(mbs["K3"]), float(mbs["K4"]), float(mbs["sigma"]), float(mbs.get("c", 1.0)))


# ------------------------------------------------------------------ diagnostics
def probe_pipes() -> dict:
    """Measured issue rates (operations per SM per clock, at the SM clock the probes ran at)
    of ex2, rcp, lg2, the forward update's ex2 + rcp pair, FP32 FMA, FP64 FMA and the FP64
    update pair on the current GPU, and that clock in MHz."""
    L = load()
    r = np.zeros(8)
    _check(L, L.rqmc_probe_pipes(_dp(r), 8))
    return dict(zip(("ex2", "rcp", "lg2", "ex2_rcp_pair", "ffma", "dfma", "fp64_pair", "sm_mhz"), map(float, r)))


# ------------------------------------------------------------------ point stream
def rqmc_points(s, N, M, seq, seed, offset=0, prec="fp32", transform="uniform", out=None, stream=None):
    """Coordinates [M, s, N] on the current CUDA device (torch tensor)."""
    import torch
    L = load()
    tr = _enum(transform, _TR)
    pr = _enum(prec, _PREC)
    dt = torch.int64 if tr == RAW else (torch.float32 if pr == FP32 else torch.float64)
    if out is None:
        out = torch.empty((M, s, N), dtype=dt, device="cuda")
    _check_out(out, M * s * N, dt, "rqmc_points out")
    _check(L, L.rqmc_points(s, N, M, _enum(seq, _SEQ), seed, offset, pr, tr, C.c_void_p(out.data_ptr()),
                            _stream(stream)))
    return out


# ------------------------------------------------------------------ one-shot estimators
def _stats_out(M, nout):
    return np.zeros((M, nout)), np.zeros(nout), np.zeros(nout)


def rqmc_integrate_product(s, N, M, seq, seed, a, prec="fp64", stream=None):
    L = load()
    a = np.ascontiguousarray(a, dtype=np.float64)
    th, rq, sd = _stats_out(M, 1)
    _check(L, L.rqmc_integrate_product(s, N, M, _enum(seq, _SEQ), seed, _dp(a), _enum(prec, _PREC), _dp(th),
                                       _dp(rq), _dp(sd), _stream(stream)))
    return th[:, 0], rq[0], sd[0]


def price_caplets(lmm: dict, strikes, N, M, seq, seed, prec="fp32", stream=None):
    """theta [M, n_fwd*n_strikes], RQ and sd over m per caplet/strike."""
    L = load()
    keep: list = []
    p = _lmm_struct(lmm, keep)
    K = np.ascontiguousarray(strikes, dtype=np.float64)
    nout = p.n_fwd * len(K)
    th, rq, sd = _stats_out(M, nout)
    _check(L, L.price_caplets(C.byref(p), _dp(K), len(K), N, M, _enum(seq, _SEQ), seed, _enum(prec, _PREC),
                              _dp(th), _dp(rq), _dp(sd), _stream(stream)))
    return th, rq, sd


def price_mbs(mbs: dict, N, M, seq, seed, prec="fp32", stream=None):
    L = load()
    p = _mbs_struct(mbs)
    th, rq, sd = _stats_out(M, 1)
    _check(L, L.price_mbs(C.byref(p), N, M, _enum(seq, _SEQ), seed, _enum(prec, _PREC), _dp(th), _dp(rq), _dp(sd),
                          _stream(stream)))
    return th[:, 0], rq[0], sd[0]


def price_adjoint(lmm: dict, strikes, weights, N, M, seq, seed, prec="fp32", stream=None):
    """Per replication: value of V = sum w_{n,k} caplet_{n,k}, dV/dL_n(0) and dV/dvol_n."""
    L = load()
    keep: list = []
    p = _lmm_struct(lmm, keep)
    K = np.ascontiguousarray(strikes, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    nf = p.n_fwd
    value, delta, vega = np.zeros(M), np.zeros((M, nf)), np.zeros((M, nf))
    _check(L, L.price_adjoint(C.byref(p), _dp(K), len(K), _dp(w), N, M, _enum(seq, _SEQ), seed, _enum(prec, _PREC), 0,
                              _dp(value), _dp(delta), _dp(vega), _stream(stream)))
    return value, delta, vega


def _instruments(insts) -> "C.Array":
    """Batch descriptors from dicts: {"kind": "lmm", "n_fwd", "N", "rate", "vol", "strike"} or
    {"kind": "mbs", "months", "N", mbs constants (defaults: the paper's)}."""
    arr = (Instrument * len(insts))()
    for a, d in zip(arr, insts):
        if d["kind"] == "lmm":
            a.kind, a.size = 0, int(d["n_fwd"])
            a.rate, a.vol = float(d.get("rate", 0.05)), float(d.get("vol", 0.15))
            a.strike = float(d.get("strike", a.rate))
        else:
            a.kind, a.size = 1, int(d["months"])
            mb = dict(inputs.mbs_paper(int(d["months"])), **{k: v for k, v in d.items() if k in
                                                              ("i0", "K1", "K2", "K3", "K4", "sigma", "c")})
            a.mbs = _mbs_struct(mb)
        a.N = int(d["N"])
    return arr


def _split_batch(theta, insts, M):
    out, off = [], 0
    for d in insts:
        nout = int(d["n_fwd"]) if d["kind"] == "lmm" else 1
        out.append(np.asarray(theta[off:off + M * nout]).reshape(M, nout))
        off += M * nout
    return out


def price_batch(insts, M, seq, seed, prec="fp32", stream=None):
    """Per instrument a theta array [M, n_out] (n_out = n_fwd caplets or 1 MBS value)."""
    L = load()
    arr = _instruments(insts)
    n_total = sum(M * (int(d["n_fwd"]) if d["kind"] == "lmm" else 1) for d in insts)
    th = np.zeros(n_total)
    _check(L, L.price_batch(arr, len(insts), M, _enum(seq, _SEQ), seed, _enum(prec, _PREC), _dp(th), _stream(stream)))
    return _split_batch(th, insts, M)


def price_caplets_noalloc(lmm: dict, strikes, N, M, seq, seed, theta, prec="fp32", stream=None):
    """Caplet values into the device tensor `theta` [M, n_fwd*n_strikes] (float64) with no
    allocation by the library (scratch is a fixed 16 MiB array inside it); asynchronous."""
    import torch
    L = load()
    keep: list = []
    p = _lmm_struct(lmm, keep)
    K = np.ascontiguousarray(strikes, dtype=np.float64)
    _check_out(theta, M * p.n_fwd * len(K), torch.float64, "price_caplets_noalloc theta")
    _check(L, L.rqmc_price_caplets_noalloc(C.byref(p), _dp(K), len(K), N, M, _enum(seq, _SEQ), seed,
                                           _enum(prec, _PREC),
                                           C.cast(C.c_void_p(theta.data_ptr()), C.POINTER(C.c_double)),
                                           _stream(stream)))
    return theta


# ------------------------------------------------------------------ plans
class Plan:
    """Device-resident plan: tables built once, `execute` launches kernels only."""

    def __init__(self, handle, M, nout):
        self._h = handle
        self.M = M
        self.nout = nout

    @classmethod
    def points(cls, s, N, M, seq, seed, prec="fp32", transform="uniform", offset=0):
        """Point stream: execute(out) fills out [M, s, N] (float32 / float64, int64 for raw)."""
        L = load()
        h = C.c_void_p()
        tr = _enum(transform, _TR)
        pr = _enum(prec, _PREC)
        _check(L, L.rqmc_plan_points(s, N, offset, M, _enum(seq, _SEQ), seed, pr, tr, C.byref(h)))
        pl = cls(h, M, 0)
        pl.points_shape = (M, s, N)
        pl.points_dtype = "int64" if tr == RAW else ("float32" if pr == FP32 else "float64")
        return pl

    @classmethod
    def product(cls, s, N, M, seq, seed, a, prec="fp64", offset=0):
        L = load()
        a = np.ascontiguousarray(a, dtype=np.float64)
        h = C.c_void_p()
        _check(L, L.rqmc_plan_product(s, N, offset, M, _enum(seq, _SEQ), seed, _dp(a), _enum(prec, _PREC),
                                      C.byref(h)))
        return cls(h, M, 1)

    @classmethod
    def caplets(cls, lmm, strikes, N, M, seq, seed, prec="fp32", offset=0):
        L = load()
        keep: list = []
        p = _lmm_struct(lmm, keep)
        K = np.ascontiguousarray(strikes, dtype=np.float64)
        h = C.c_void_p()
        _check(L, L.rqmc_plan_caplets(C.byref(p), _dp(K), len(K), N, offset, M, _enum(seq, _SEQ), seed,
                                      _enum(prec, _PREC), C.byref(h)))
        return cls(h, M, p.n_fwd * len(K))

    @classmethod
    def mbs(cls, mbs, N, M, seq, seed, prec="fp32", offset=0):
        L = load()
        p = _mbs_struct(mbs)
        h = C.c_void_p()
        _check(L, L.rqmc_plan_mbs(C.byref(p), N, offset, M, _enum(seq, _SEQ), seed, _enum(prec, _PREC),
                                  C.byref(h)))
        return cls(h, M, 1)

    @classmethod
    def adjoint(cls, lmm, strikes, weights, N, M, seq, seed, prec="fp32", offset=0):
        """Outputs per replication: [value, dV/dL_n(0) (nf), dV/dvol_n (nf), caplet prices (nf*nK)]."""
        L = load()
        keep: list = []
        p = _lmm_struct(lmm, keep)
        K = np.ascontiguousarray(strikes, dtype=np.float64)
        w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
        h = C.c_void_p()
        _check(L, L.rqmc_plan_adjoint(C.byref(p), _dp(K), len(K), _dp(w), N, offset, M, _enum(seq, _SEQ), seed,
                                      _enum(prec, _PREC), 0, C.byref(h)))
        return cls(h, M, 1 + 2 * p.n_fwd + p.n_fwd * len(K))

    @classmethod
    def batch(cls, insts, M, seq, seed, prec="fp32"):
        """One persistent graph-captured launch over all instruments; execute() returns the
        concatenated [M, n_out_i] blocks (use split_batch to separate them)."""
        L = load()
        arr = _instruments(insts)
        h = C.c_void_p()
        _check(L, L.rqmc_plan_batch(arr, len(insts), M, _enum(seq, _SEQ), seed, _enum(prec, _PREC), C.byref(h)))
        pl = cls(h, M, 0)
        pl.insts = list(insts)
        return pl

    def batch_stats(self) -> dict:
        """Timing of the last execute of a batch plan: busiest SM / mean SM, span of all CTAs and
        of each work class (ms)."""
        L = load()
        r = np.zeros(5)
        _check(L, L.rqmc_plan_batch_stats(self._h, _dp(r), 5))
        return {"imbalance": float(r[0]), "span_ms": float(r[1]), "class_160_ms": float(r[2]),
                "class_mbs_ms": float(r[3]), "class_small_ms": float(r[4])}

    def batch_imbalance(self) -> float:
        return self.batch_stats()["imbalance"]

    def split_batch(self, theta):
        return _split_batch(theta.cpu().numpy() if hasattr(theta, "cpu") else theta, self.insts, self.M)

    def output_size(self):
        return int(load().rqmc_plan_output_size(self._h))

    def launches(self):
        return int(load().rqmc_plan_launches(self._h))

    def launch_shape(self):
        """(threads per block, paths per thread) the plan launches with (a batch plan: the
        autotuner's tile)."""
        L = load()
        t, p = C.c_int(), C.c_int()
        _check(L, L.rqmc_plan_get_launch(self._h, C.byref(t), C.byref(p)))
        return t.value, p.value

    def set_launch(self, threads=0, paths_per_thread=0):
        _check(load(), load().rqmc_plan_set_launch(self._h, threads, paths_per_thread))

    def execute(self, theta=None, stream=None):
        import torch
        if theta is None:
            if hasattr(self, "points_shape"):
                theta = torch.empty(self.points_shape, dtype=getattr(torch, self.points_dtype), device="cuda")
            else:
                theta = torch.empty(self.output_size(), dtype=torch.float64, device="cuda")
        L = load()
        if hasattr(self, "points_shape"):
            _check_out(theta, self.output_size(), getattr(torch, self.points_dtype), "Plan.execute out")
        else:
            _check_out(theta, self.output_size(), torch.float64, "Plan.execute theta")
        _check(L, L.rqmc_plan_execute(self._h, C.cast(C.c_void_p(theta.data_ptr()), C.POINTER(C.c_double)),
                                      _stream(stream)))
        return theta

    def check(self, stream=None):
        _check(load(), load().rqmc_plan_check(self._h, _stream(stream)))

    def close(self):
        if self._h:
            load().rqmc_plan_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ autograd
def _caplet_strip_function():
    import torch

    class CapletStrip(torch.autograd.Function):
        """Caplet prices RQ_{M,N} [n_fwd * n_strikes] as a function of the initial forwards
        L_n(0) (n = 1..nf) and the vols; the backward pass is the library's pathwise adjoint
        with grad_output as the caplet weights."""

        @staticmethod
        def forward(ctx, L0, vol, lmm, strikes, N, M, seq, seed):
            lm = dict(lmm)
            full = np.array(lmm["L0"], dtype=np.float64).copy()
            full[1:] = L0.detach().cpu().numpy()
            lm["L0"] = full
            lm["vol"] = vol.detach().cpu().numpy().astype(np.float64)
            K = np.asarray(strikes, dtype=np.float64)
            nf = int(lm["n_fwd"])
            zero = np.zeros(nf * len(K))
            plan = Plan.adjoint(lm, K, zero, N, M, seq, seed)
            out = plan.execute().cpu().numpy().reshape(M, -1)
            plan.close()
            prices = out[:, 1 + 2 * nf:].mean(axis=0)
            ctx.args = (lm, K, N, M, seq, seed)
            return torch.as_tensor(prices, dtype=L0.dtype, device=L0.device)

        @staticmethod
        def backward(ctx, grad):
            lm, K, N, M, seq, seed = ctx.args
            w = grad.detach().cpu().numpy().astype(np.float64)
            _, delta, vega = price_adjoint(lm, K, w, N, M, seq, seed)
            dL = torch.as_tensor(delta.mean(axis=0), dtype=grad.dtype, device=grad.device)
            dv = torch.as_tensor(vega.mean(axis=0), dtype=grad.dtype, device=grad.device)
            return dL, dv, None, None, None, None, None, None

    return CapletStrip


def caplet_strip(L0, vol, lmm: dict, strikes, N, M, seq, seed):
    """Differentiable caplet prices: see CapletStrip."""
    return _caplet_strip_function().apply(L0, vol, lmm, strikes, N, M, seq, seed)
