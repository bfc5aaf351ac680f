"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds no arithmetic of the RQMC method: it only assembles
parameter sets (model tuples, initial curves, volatility loadings, batch
descriptors) and loads the Joe-Kuo Sobol' table.  Randomness that the
method itself draws (random starts, digit permutations, digital shifts,
pseudorandom path uniforms) is NOT drawn here -- both the library and the
oracle derive it from the seed with their own Philox4x32-10.

Workloads (Xu & Okten, arXiv:1408.5526):
  * product test integrand, s = 8, N = 4096, M = 32            (Sec. 1 estimator)
  * LMM caplets: 40 quarterly forwards, flat 5 %, vol 15 %,
    strikes 4.5/5/5.5 %, N = 65536, M = 64                       (Sec. 5)
  * MBS with the paper's constants, 360 months, N = 65536, M = 64 (Sec. 6)
  * two-factor 80-forward caplet strip for pathwise Greeks       (extension)
  * 512-instrument batch (384 LMM, 128 MBS)                      (extension)
"""
from __future__ import annotations

import os

import numpy as np

HALTON_RS, RASRAP, SOBOL_DS, PHILOX = 0, 1, 2, 3
SEQ_NAMES = {HALTON_RS: "halton_rs", RASRAP: "rasrap", SOBOL_DS: "sobol_ds", PHILOX: "philox"}

_JOE_KUO_CACHE = None


def joe_kuo_table():
    """(poly, vinit) of the Joe-Kuo primitive polynomials and initial direction
    numbers (Sec. 3.2 uses Joe & Kuo's table).  Read from the copy that scipy
    installs; poly[j] encodes the whole polynomial (degree = bit length - 1),
    vinit[j, :degree] are m_1..m_degree.  Row 0 is the van der Corput row."""
    global _JOE_KUO_CACHE
    if _JOE_KUO_CACHE is None:
        import scipy.stats
        path = os.path.join(os.path.dirname(scipy.stats.__file__), "_sobol_direction_numbers.npz")
        with np.load(path) as z:
            _JOE_KUO_CACHE = (np.ascontiguousarray(z["poly"], dtype=np.int64),
                              np.ascontiguousarray(z["vinit"], dtype=np.int64))
    return _JOE_KUO_CACHE


# ---------------------------------------------------------------- product integrand
def product_weights(s: int = 8) -> np.ndarray:
    """a_i = i for i = 1..s: f(x) = prod_i (|4 x_i - 2| + a_i)/(1 + a_i), integral 1."""
    return np.arange(1, s + 1, dtype=np.float64)


# ---------------------------------------------------------------- LIBOR market model
def lmm_flat(n_fwd: int = 40, delta: float = 0.25, rate: float = 0.05, vol: float = 0.15,
             d: int = 1, scheme: int = 0) -> dict:
    """Flat initial curve: L_n(0) = rate for n = 0..n_fwd, flat scalar vol.
    Equivalent bond prices B_n(0) = prod_{j<n} (1 + delta rate)^-1 (eq. BL)."""
    return {
        "n_fwd": n_fwd, "d": d, "delta": delta, "scheme": scheme, "substeps": 1,
        "L0": np.full(n_fwd + 1, rate, dtype=np.float64),
        "vol": np.full(n_fwd, vol, dtype=np.float64),
        "loadings": None if d == 1 else np.tile(np.eye(d)[0], (n_fwd, 1)),
    }


def lmm_from_bonds(B: np.ndarray, delta: float, vol) -> dict:
    """Initial forwards from bond prices B_0(0)=1, B_1(0), ..., B_{nf+1}(0):
    L_n(0) = (B_n - B_{n+1}) / (delta B_{n+1}) (eq. BL), n = 0..nf."""
    B = np.asarray(B, dtype=np.float64)
    L0 = (B[:-1] - B[1:]) / (delta * B[1:])
    nf = len(L0) - 1
    return {"n_fwd": nf, "d": 1, "delta": delta, "scheme": 0, "substeps": 1, "L0": L0,
            "vol": np.broadcast_to(np.asarray(vol, dtype=np.float64), (nf,)).copy(), "loadings": None}


def pca_loadings(n_fwd: int, d: int, beta: float = 0.1) -> np.ndarray:
    """Unit loadings b_n (rows) of the top-d principal components of the
    correlation rho_ij = exp(-beta |i - j|), rows renormalized to length 1."""
    idx = np.arange(n_fwd)
    rho = np.exp(-beta * np.abs(idx[:, None] - idx[None, :]))
    w, v = np.linalg.eigh(rho)
    order = np.argsort(w)[::-1][:d]
    B = v[:, order] * np.sqrt(w[order])[None, :]
    B /= np.linalg.norm(B, axis=1, keepdims=True)
    return np.ascontiguousarray(B)


def lmm_two_factor(n_fwd: int = 80, seed: int = 1, delta: float = 0.25, rate: float = 0.05) -> dict:
    """Two-factor strip: correlation exp(-0.1|i-j|) reduced to 2 factors,
    vols uniform in [10 %, 25 %] drawn per seed (numpy's PCG64)."""
    rng = np.random.default_rng(seed)
    return {"n_fwd": n_fwd, "d": 2, "delta": delta, "scheme": 0, "substeps": 1,
            "L0": np.full(n_fwd + 1, rate, dtype=np.float64),
            "vol": rng.uniform(0.10, 0.25, size=n_fwd),
            "loadings": pca_loadings(n_fwd, 2)}


LMM_STRIKES = np.array([0.045, 0.05, 0.055])

# ---------------------------------------------------------------- MBS
def mbs_paper(months: int = 360) -> dict:
    """(i0, K1, K2, K3, K4, sigma^2) = (0.007, 0.01, -0.005, 10, 0.5, 0.0004)
    (Sec. 6); sigma is the standard deviation of xi_k, c = 1."""
    return {"months": months, "i0": 0.007, "K1": 0.01, "K2": -0.005, "K3": 10.0, "K4": 0.5,
            "sigma": 0.02, "c": 1.0}


# ---------------------------------------------------------------- Treasury curve
TREASURY_2012_02_24 = {   # Table 3: maturity in years -> yield in percent
    1 / 12: 0.08, 0.25: 0.10, 0.5: 0.14, 1: 0.18, 2: 0.31, 3: 0.43, 5: 0.89, 7: 1.41, 10: 1.98, 20: 2.75,
    30: 3.10}


def treasury_bonds(n: int, delta: float = 0.5, table: dict = TREASURY_2012_02_24) -> np.ndarray:
    """Bond prices B_0(0) = 1, B_1(0), ..., B_n(0) at T_k = k delta from the Treasury yields of
    Table 3: a natural cubic spline through (maturity, yield), evaluated every delta years,
    read as bond-equivalent (semiannual) yields, B(T) = (1 + y(T)/2)^(-2T)."""
    from scipy.interpolate import CubicSpline
    mats = np.array(sorted(table), dtype=np.float64)
    ys = np.array([table[m] for m in sorted(table)], dtype=np.float64) / 100.0
    spline = CubicSpline(mats, ys, bc_type="natural")
    t = delta * np.arange(1, n + 1)
    B = (1.0 + spline(t) / 2.0) ** (-2.0 * t)
    return np.concatenate([[1.0], B])


def lmm_treasury(T: float = 5.0, delta: float = 0.5, vol: float = 0.04) -> dict:
    """The Treasury-curve LMM study of Sec. 5: forwards L_0..L_nf (nf = T / delta) from the
    24 Feb 2012 curve (eq. BL), flat vol; the caplet of the study is the one on L_nf, fixed
    at T and paid at T + delta, with strike 1 %."""
    nf = int(round(T / delta))
    return lmm_from_bonds(treasury_bonds(nf + 1, delta), delta, vol)


TREASURY_STUDY = {"T": 5.0, "delta": 0.5, "K": 0.01, "vol": 0.04, "M": 100}


# ---------------------------------------------------------------- batch
def batch_instruments(seed: int = 1, n_lmm: int = 384, n_mbs: int = 128) -> list:
    """512 heterogeneous instruments: LMM caplet strips with 8..160 quarterly
    forwards (1 factor, flat 5 %, vol 15 %, ATM strike) and MBS with
    120..360 months (paper constants); N = 2^e with e uniform in 12..18.
    Sizes are drawn with numpy's PCG64 from the seed."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_lmm):
        out.append({"kind": "lmm", "n_fwd": int(rng.integers(8, 161)),
                    "N": 1 << int(rng.integers(12, 19))})
    for _ in range(n_mbs):
        out.append({"kind": "mbs", "months": int(rng.integers(120, 361)),
                    "N": 1 << int(rng.integers(12, 19))})
    return out


# ---------------------------------------------------------------- named workloads
CONFIGS = {
    "product_s8": {"s": 8, "N": 4096, "M": 32, "seq": HALTON_RS, "seed": 1},
    "lmm_caplets_40": {"n_fwd": 40, "N": 65536, "M": 64, "seed": 1},
    "mbs_360": {"months": 360, "N": 65536, "M": 64, "seed": 1},
    "adjoint_2f_80": {"n_fwd": 80, "N": 1 << 18, "M": 32, "seed": 1},
    "batch_512": {"M": 32, "seed": 1},
}
