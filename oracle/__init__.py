"""FP64 CPU oracle for the RQMC method of Xu & Okten (arXiv:1408.5526).

TEST INFRASTRUCTURE ONLY.  This package may be imported by ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` -- nothing in the product package imports or calls it.
It wraps ``oracle.c`` (plain C, FP64, compiled with gcc -O2, no fast-math)
through ctypes.  The C source shares no code with the CUDA library.

Every wrapper takes plain numpy arrays; seeded inputs (parameter sets, the
Joe-Kuo direction-number table) come from ``paper_1408_5526_gb300.inputs``,
which holds no arithmetic of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

HALTON_RS, RASRAP, SOBOL_DS, PHILOX, SOBOL_LMS = 0, 1, 2, 3, 4
UNIFORM, NORMAL, RAW = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


class _Lmm(C.Structure):
    _fields_ = [("n_fwd", C.c_int), ("d", C.c_int), ("scheme", C.c_int), ("substeps", C.c_int),
                ("delta", C.c_double), ("L0", C.POINTER(C.c_double)),
                ("vol", C.POINTER(C.c_double)), ("load", C.POINTER(C.c_double))]


class _Mbs(C.Structure):
    _fields_ = [("months", C.c_int), ("i0", C.c_double), ("K1", C.c_double), ("K2", C.c_double),
                ("K3", C.c_double), ("K4", C.c_double), ("sigma", C.c_double), ("c", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        u32p, u64p, i64p, dp = (C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                C.POINTER(C.c_int64), C.POINTER(C.c_double))
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_first_primes.argtypes = [C.c_int, u32p]
        L.orc_halton_K.argtypes = [C.c_uint32]
        L.orc_halton_K.restype = C.c_int
        L.orc_ipow.argtypes = [C.c_uint32, C.c_int]
        L.orc_ipow.restype = C.c_uint64
        L.orc_halton_start.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_uint32, C.c_int]
        L.orc_halton_start.restype = C.c_uint64
        L.orc_halton_perm.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_uint32, C.c_int,
                                      C.POINTER(C.c_uint16)]
        L.orc_permuted_vdc_numerator.argtypes = [C.c_uint32, C.c_int, C.POINTER(C.c_uint16), C.c_uint64]
        L.orc_permuted_vdc_numerator.restype = C.c_uint64
        L.orc_sobol_directions.argtypes = [C.c_int, i64p, i64p, C.c_int, u32p]
        L.orc_sobol_directions.restype = C.c_int
        L.orc_sobol_binary.argtypes = [u32p, C.c_uint64]
        L.orc_sobol_binary.restype = C.c_uint32
        L.orc_sobol_shift.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int]
        L.orc_sobol_lms_rows.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int, u32p]
        L.orc_sobol_lms_rows.restype = None
        L.orc_sobol_lms_apply.argtypes = [u32p, C.c_uint32]
        L.orc_sobol_lms_apply.restype = C.c_uint32
        L.orc_stream_raw.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint64, C.c_uint64, u64p]
        L.orc_stream_raw.restype = C.c_int
        L.orc_stream_rows.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64, C.c_int, u64p]
        L.orc_stream_rows.restype = C.c_int
        L.orc_sobol_shift.restype = C.c_uint32
        L.orc_philox_path_word.argtypes = [C.c_uint64, C.c_uint32, C.c_int, C.c_int, C.c_uint64]
        L.orc_philox_path_word.restype = C.c_uint32
        L.orc_seq_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_uint32, i64p, i64p, C.c_int]
        L.orc_seq_create.restype = C.c_void_p
        L.orc_seq_destroy.argtypes = [C.c_void_p]
        L.orc_coord_raw.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_uint64, u64p]
        L.orc_coord_raw.restype = C.c_uint64
        L.orc_ndtri_lower.argtypes = [C.c_double]
        L.orc_ndtri_lower.restype = C.c_double
        L.orc_points.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int, C.c_void_p, C.c_int]
        L.orc_product_theta.argtypes = [C.c_void_p, C.c_int64, C.c_int64, dp, C.c_int, C.c_int, dp, C.c_int]
        L.orc_lmm_caplets.argtypes = [C.c_void_p, C.POINTER(_Lmm), dp, C.c_int, C.c_int64, C.c_int64,
                                      C.c_int, C.c_int, dp, C.c_int]
        L.orc_lmm_caplets.restype = C.c_int
        L.orc_lmm_adjoint.argtypes = [C.c_void_p, C.POINTER(_Lmm), dp, C.c_int, dp, C.c_int64, C.c_int64,
                                      C.c_int, C.c_int, dp, dp, dp, C.c_int]
        L.orc_lmm_adjoint.restype = C.c_int
        L.orc_mbs_theta.argtypes = [C.c_void_p, C.POINTER(_Mbs), C.c_int64, C.c_int64, C.c_int, C.c_int,
                                    dp, C.c_int]
        L.orc_mbs_theta.restype = C.c_int
        L.orc_rq_stats.argtypes = [dp, C.c_int, C.c_int, dp, dp]
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# ---------------------------------------------------------------- generators
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def first_primes(s: int) -> np.ndarray:
    out = np.zeros(s, dtype=np.uint32)
    lib().orc_first_primes(s, _p(out, C.c_uint32))
    return out


def halton_K(p: int) -> int:
    return int(lib().orc_halton_K(p))


def ipow(p: int, e: int) -> int:
    return int(lib().orc_ipow(p, e))


def halton_start(seed: int, inst: int, m: int, j: int, p: int, K: int) -> int:
    return int(lib().orc_halton_start(seed, inst, m, j, p, K))


def halton_perm(seed: int, inst: int, m: int, j: int, p: int, identity: bool = False) -> np.ndarray:
    out = np.zeros(p, dtype=np.uint16)
    lib().orc_halton_perm(seed, inst, m, j, p, int(identity), _p(out, C.c_uint16))
    return out


def permuted_vdc_numerator(p: int, K: int, sigma, n: int) -> int:
    sg = np.ascontiguousarray(sigma, dtype=np.uint16)
    return int(lib().orc_permuted_vdc_numerator(p, K, _p(sg, C.c_uint16), n))


def sobol_directions(s: int, poly, vinit) -> np.ndarray:
    poly = np.ascontiguousarray(poly, dtype=np.int64)
    vinit = np.ascontiguousarray(vinit, dtype=np.int64)
    V = np.zeros((s, 32), dtype=np.uint32)
    rc = lib().orc_sobol_directions(s, _p(poly, C.c_int64), _p(vinit, C.c_int64), vinit.shape[1],
                                    _p(V, C.c_uint32))
    if rc != 0:
        raise ValueError(f"orc_sobol_directions failed ({rc})")
    return V


def sobol_binary(Vj, n: int) -> int:
    v = np.ascontiguousarray(Vj, dtype=np.uint32)
    return int(lib().orc_sobol_binary(_p(v, C.c_uint32), n))


def sobol_shift(seed: int, inst: int, m: int, j: int) -> int:
    return int(lib().orc_sobol_shift(seed, inst, m, j))


def ndtri_lower(q: float) -> float:
    return float(lib().orc_ndtri_lower(q))


def ndtri(u: float) -> float:
    """Phi^-1(u) through the lower-half solver and symmetry."""
    return ndtri_lower(u) if u <= 0.5 else -ndtri_lower(1.0 - u)


# ---------------------------------------------------------------- sequences
class Sequence:
    """All randomizations (starts, permutations, shifts) of one call."""

    def __init__(self, seq: int, s: int, M: int, seed: int, inst: int = 0, joe_kuo=None):
        self.seq, self.s, self.M, self.seed, self.inst = seq, s, M, seed, inst
        if seq in (SOBOL_DS, SOBOL_LMS):
            if joe_kuo is None:
                raise ValueError("Sobol' needs the Joe-Kuo table (poly, vinit)")
            poly = np.ascontiguousarray(joe_kuo[0][:s], dtype=np.int64)
            vinit = np.ascontiguousarray(joe_kuo[1][:s], dtype=np.int64)
            self._keep = (poly, vinit)
            h = lib().orc_seq_create(seq, s, M, seed, inst, _p(poly, C.c_int64), _p(vinit, C.c_int64),
                                     vinit.shape[1])
        else:
            h = lib().orc_seq_create(seq, s, M, seed, inst, None, None, 0)
        if not h:
            raise ValueError("orc_seq_create failed")
        self.h = C.c_void_p(h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_seq_destroy(self.h)
            self.h = None

    def stream(self, n_start: int, count: int, threads: int = 0) -> np.ndarray:
        """Raw states [M, s, count] from the recursive CPU generators of Table 1 (Algorithm 2
        for Halton/Rasrap, Gray-code order for Sobol'; Philox is counter-based)."""
        out = np.zeros((self.M, self.s, count), dtype=np.uint64)
        rc = lib().orc_stream_rows(self.h, n_start, count, threads or max_threads(), _p(out, C.c_uint64))
        if rc != 0:
            raise ValueError("point range outside the representable digits")
        return out

    def raw(self, m: int, j: int, n: int):
        D = C.c_uint64(0)
        r = lib().orc_coord_raw(self.h, m, j, n, C.byref(D))
        return int(r), int(D.value)

    def points(self, N: int, offset: int = 0, transform: int = UNIFORM, threads: int = 0) -> np.ndarray:
        dt = np.uint64 if transform == RAW else np.float64
        out = np.zeros((self.M, self.s, N), dtype=dt)
        lib().orc_points(self.h, N, offset, transform, out.ctypes.data_as(C.c_void_p), threads or max_threads())
        return out


def _stats(theta):
    M, nout = theta.shape
    rq = np.zeros(nout)
    sd = np.zeros(nout)
    t = np.ascontiguousarray(theta, dtype=np.float64)
    lib().orc_rq_stats(_p(t, C.c_double), M, nout, _p(rq, C.c_double), _p(sd, C.c_double))
    return rq, sd


def product_theta(seq: Sequence, N: int, a, offset: int = 0, m_range=None, threads: int = 0):
    """theta_N^m of the product integrand for every replication m."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    lo, hi = m_range or (0, seq.M)
    theta = np.zeros(seq.M)
    lib().orc_product_theta(seq.h, N, offset, _p(a, C.c_double), lo, hi, _p(theta, C.c_double),
                            threads or max_threads())
    return theta[lo:hi]


def _lmm_struct(lmm: dict, keep: list):
    L0 = np.ascontiguousarray(lmm["L0"], dtype=np.float64)
    vol = np.ascontiguousarray(lmm["vol"], dtype=np.float64)
    keep += [L0, vol]
    st = _Lmm(int(lmm["n_fwd"]), int(lmm.get("d", 1)), int(lmm.get("scheme", 0)),
              int(lmm.get("substeps", 1)), float(lmm["delta"]), _p(L0, C.c_double), _p(vol, C.c_double),
              None)
    if lmm.get("loadings") is not None:
        ld = np.ascontiguousarray(lmm["loadings"], dtype=np.float64)
        keep.append(ld)
        st.load = _p(ld, C.c_double)
    return st


def lmm_caplets(seq: Sequence, lmm: dict, strikes, N: int, offset: int = 0, m_range=None, threads: int = 0):
    """theta[m, (n-1)*nK + k] for caplet n = 1..n_fwd and strike k."""
    keep: list = []
    st = _lmm_struct(lmm, keep)
    K = np.ascontiguousarray(strikes, dtype=np.float64)
    nout = st.n_fwd * len(K)
    lo, hi = m_range or (0, seq.M)
    theta = np.zeros((seq.M, nout))
    rc = lib().orc_lmm_caplets(seq.h, C.byref(st), _p(K, C.c_double), len(K), N, offset, lo, hi,
                               _p(theta, C.c_double), threads or max_threads())
    if rc != 0:
        raise ValueError(f"orc_lmm_caplets failed ({rc})")
    return theta[lo:hi]


def lmm_adjoint(seq: Sequence, lmm: dict, strikes, weights, N: int, offset: int = 0, m_range=None,
                threads: int = 0):
    """Per-replication value, dV/dL_n(0) and dV/dvol_n of V = sum w_{n,k} caplet_{n,k}."""
    keep: list = []
    st = _lmm_struct(lmm, keep)
    K = np.ascontiguousarray(strikes, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64).reshape(-1)
    nf = st.n_fwd
    lo, hi = m_range or (0, seq.M)
    value = np.zeros(seq.M)
    delta = np.zeros((seq.M, nf))
    vega = np.zeros((seq.M, nf))
    rc = lib().orc_lmm_adjoint(seq.h, C.byref(st), _p(K, C.c_double), len(K), _p(w, C.c_double), N, offset,
                               lo, hi, _p(value, C.c_double), _p(delta, C.c_double), _p(vega, C.c_double),
                               threads or max_threads())
    if rc != 0:
        raise ValueError(f"orc_lmm_adjoint failed ({rc})")
    return value[lo:hi], delta[lo:hi], vega[lo:hi]


def mbs_theta(seq: Sequence, mbs: dict, N: int, offset: int = 0, m_range=None, threads: int = 0):
    st = _Mbs(int(mbs["months"]), float(mbs["i0"]), float(mbs["K1"]), float(mbs["K2"]), float(mbs["K3"]),
              float(mbs["K4"]), float(mbs["sigma"]), float(mbs.get("c", 1.0)))
    lo, hi = m_range or (0, seq.M)
    theta = np.zeros(seq.M)
    rc = lib().orc_mbs_theta(seq.h, C.byref(st), N, offset, lo, hi, _p(theta, C.c_double),
                             threads or max_threads())
    if rc != 0:
        raise ValueError(f"orc_mbs_theta failed ({rc})")
    return theta[lo:hi]


def rq_stats(theta):
    """RQ_{M,N} (mean over m) and the sample standard deviation over m."""
    theta = np.asarray(theta, dtype=np.float64)
    if theta.ndim == 1:
        theta = theta[:, None]
    return _stats(theta)
