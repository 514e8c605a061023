"""FP64 CPU oracle of the localized Gaussian-windowed EVD clutter filter.

TEST INFRASTRUCTURE ONLY: a plain, slow, obviously correct implementation
that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it; the library never does.

The arithmetic lives in ``lcf_oracle.c`` (double precision, one step per
equation of the paper: Eq. 11-12 windowed Gram, Eq. 2 Jacobi EVD, the
thresholding methods, Eq. 4 reconstruction, power Doppler, Eq. 13 blend);
this module only marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

T_FIXED, T_CURVATURE, T_SLOPE, T_MEDIAN, T_SIGMOID, T_ADAPTIVE_SOFT, T_NONE = range(7)
T_NCC = 8   # method 4 (Eq. 8); method 5 takes its k with thresh_mode T_SIGMOID, k_src T_NCC
FLAG_NOCONV, FLAG_DEGENERATE = 1, 2


class _Cfg(C.Structure):
    _fields_ = [("nz", C.c_int), ("nx", C.c_int), ("nt", C.c_int),
                ("wz", C.c_int), ("wx", C.c_int),
                ("sigma_scale", C.c_double), ("support_sigmas", C.c_double),
                ("all_ones_window", C.c_int),
                ("thresh_mode", C.c_int), ("beta", C.c_double), ("k_fixed", C.c_int),
                ("k_src", C.c_int), ("beta_src", C.c_double),
                ("pd_mode", C.c_int), ("alpha_mode", C.c_int), ("curv_norm", C.c_int),
                ("max_sweeps", C.c_int)]


@dataclass
class OracleConfig:
    nz: int
    nx: int
    nt: int
    wz: int = 1
    wx: int = 1
    sigma_scale: float = 1.0
    support_sigmas: float = 3.0
    all_ones_window: int = 0
    thresh_mode: int = T_FIXED
    beta: float = 1.0
    k_fixed: int = 0
    k_src: int = T_FIXED
    beta_src: float = 1.0
    pd_mode: int = 0
    alpha_mode: int = 0
    curv_norm: int = 0
    max_sweeps: int = 60

    def c(self) -> _Cfg:
        return _Cfg(self.nz, self.nx, self.nt, self.wz, self.wx, self.sigma_scale,
                    self.support_sigmas, self.all_ones_window, self.thresh_mode, self.beta,
                    self.k_fixed, self.k_src, self.beta_src, self.pd_mode, self.alpha_mode,
                    self.curv_norm, self.max_sweeps)

    @property
    def nd(self) -> int:
        return self.wz * self.wx


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        dp, ip, fp = P(C.c_double), P(C.c_int), P(C.c_float)
        L.ora_filter.argtypes = [fp, P(_Cfg), dp, dp, dp, ip, dp, ip, ip, dp, dp, dp, C.c_int,
                                 dp, C.c_int]
        L.ora_filter.restype = C.c_int
        L.ora_filter_k.argtypes = [fp, P(_Cfg), dp, dp, dp, ip, dp, ip, ip, dp, dp, dp, C.c_int,
                                   dp, C.c_int, ip]
        L.ora_filter_k.restype = C.c_int
        L.ora_rule_scores.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_int, dp]
        L.ora_rule_scores.restype = C.c_int
        L.ora_eigh.argtypes = [C.c_int, dp, dp, dp, C.c_int]
        L.ora_eigh.restype = C.c_int
        L.ora_weights.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_int, C.c_int, C.c_double,
                                  C.c_int, dp]
        L.ora_weights.restype = C.c_int
        L.ora_gram.argtypes = [fp, P(_Cfg), C.c_int, dp]
        L.ora_gram.restype = None
        L.ora_window_box.argtypes = [P(_Cfg), C.c_int, ip, dp]
        L.ora_window_box.restype = C.c_int
        L.ora_window_weights.argtypes = [P(_Cfg), C.c_int, dp]
        L.ora_window_weights.restype = None
        L.ora_ncc_curve.argtypes = [fp, P(_Cfg), C.c_int, dp]
        L.ora_ncc_curve.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _iq_f32(iq: np.ndarray) -> np.ndarray:
    """complex64 packet [nt][nz][nx] -> contiguous interleaved float32 view."""
    a = np.ascontiguousarray(iq, dtype=np.complex64)
    return a.view(np.float32)


@dataclass
class OracleResult:
    pd: np.ndarray                      # [nz, nx] float64
    lam: np.ndarray                     # [nd, nt] descending eigenvalues
    wt: np.ndarray                      # [nd, nt]
    k: np.ndarray                       # [nd] cutoff (hard rules / sigmoid centre), -1 soft
    alpha: np.ndarray                   # [nd]
    flags: np.ndarray                   # [nd]
    sweeps: np.ndarray                  # [nd]
    R: np.ndarray | None = None         # [nd, nt, nt] complex128
    V: np.ndarray | None = None         # [nd, nt, nt] complex128
    pdk: np.ndarray | None = None       # [nd, nz, nx]
    filt: np.ndarray | None = None      # [nt, nz, nx] complex128, subset dbg_subset
    extra: dict = field(default_factory=dict)


def filter(iq: np.ndarray, cfg: OracleConfig, want_R=False, want_V=False, want_pdk=False,
           dbg_subset: int = -1, nthreads: int = 0, k_override=None) -> OracleResult:
    """Run the whole localized filter on one packet iq[nt][nz][nx] (complex64).

    k_override: optional int array [nd]; entries >= 0 replace the rule's
    cutoff of that window (to evaluate an equally valid cutoff at a near-tie).
    """
    assert iq.shape == (cfg.nt, cfg.nz, cfg.nx), (iq.shape, cfg)
    nd, nt, npx = cfg.nd, cfg.nt, cfg.nz * cfg.nx
    buf = _iq_f32(iq)
    pd = np.zeros(npx, np.float64)
    lam = np.zeros((nd, nt)); wt = np.zeros((nd, nt))
    kk = np.zeros(nd, np.int32); al = np.zeros(nd); fl = np.zeros(nd, np.int32)
    sw = np.zeros(nd, np.int32)
    R = np.zeros((nd, nt, nt), np.complex128) if want_R else None
    V = np.zeros((nd, nt, nt), np.complex128) if want_V else None
    pdk = np.zeros((nd, cfg.nz, cfg.nx)) if want_pdk else None
    filt = np.zeros((nt, cfg.nz, cfg.nx), np.complex128) if dbg_subset >= 0 else None
    cc = cfg.c()
    ko = None if k_override is None else np.ascontiguousarray(k_override, dtype=np.int32)
    rc = lib().ora_filter_k(_ptr(buf, C.c_float), C.byref(cc), _ptr(pd, C.c_double),
                            _ptr(lam, C.c_double), _ptr(wt, C.c_double), _ptr(kk, C.c_int),
                            _ptr(al, C.c_double), _ptr(fl, C.c_int), _ptr(sw, C.c_int),
                            None if R is None else R.ctypes.data_as(C.POINTER(C.c_double)),
                            None if V is None else V.ctypes.data_as(C.POINTER(C.c_double)),
                            _ptr(pdk, C.c_double), int(dbg_subset),
                            None if filt is None else filt.ctypes.data_as(C.POINTER(C.c_double)),
                            int(nthreads), _ptr(ko, C.c_int))
    if rc != 0:
        raise RuntimeError(f"ora_filter failed: {rc}")
    return OracleResult(pd.reshape(cfg.nz, cfg.nx), lam, wt, kk, al, fl, sw, R, V, pdk, filt)


def rule_scores(mode: int, lam: np.ndarray, beta: float = 1.0, curv_norm: int = 0) -> np.ndarray:
    """Per-index quantity a hard rule decides on (curvature, descent, lambda/T)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    sc = np.zeros_like(lam)
    lib().ora_rule_scores(int(mode), lam.size, _ptr(lam, C.c_double), float(beta), int(curv_norm),
                          _ptr(sc, C.c_double))
    return sc


def eigh(A: np.ndarray, max_sweeps: int = 60):
    """Hermitian EVD by the oracle's cyclic Jacobi: (lam descending, V, sweeps)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    V = np.zeros((n, n), np.complex128)
    lam = np.zeros(n)
    sw = lib().ora_eigh(n, A.ctypes.data_as(C.POINTER(C.c_double)),
                        V.ctypes.data_as(C.POINTER(C.c_double)), _ptr(lam, C.c_double),
                        int(max_sweeps))
    return lam, V, sw


def weights(mode: int, lam: np.ndarray, beta: float = 1.0, k_fixed: int = 0,
            k_src: int = T_FIXED, beta_src: float = 1.0, curv_norm: int = 0):
    """Eigen-weights of one subset from its descending eigenvalues: (wt, k)."""
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    wt = np.zeros_like(lam)
    k = lib().ora_weights(int(mode), lam.size, _ptr(lam, C.c_double), float(beta), int(k_fixed),
                          int(k_src), float(beta_src), int(curv_norm), _ptr(wt, C.c_double))
    return wt, k


def gram(iq: np.ndarray, cfg: OracleConfig, k: int) -> np.ndarray:
    """Windowed Gram R_k (Eq. 12) of window k, complex128 [nt, nt]."""
    buf = _iq_f32(iq)
    R = np.zeros((cfg.nt, cfg.nt), np.complex128)
    cc = cfg.c()
    lib().ora_gram(_ptr(buf, C.c_float), C.byref(cc), int(k), R.ctypes.data_as(C.POINTER(C.c_double)))
    return R


def ncc_curve(iq: np.ndarray, cfg: OracleConfig, k: int):
    """Method 4 (Eq. 8) of window k from the oracle's own Gram and EVD: (k, curve), where
    curve[j] = NCC at cutoff j + 1 (NaN where the fn-neighbourhoods do not exist)."""
    buf = _iq_f32(iq)
    curve = np.zeros(cfg.nt)
    cc = cfg.c()
    kk = lib().ora_ncc_curve(_ptr(buf, C.c_float), C.byref(cc), int(k), _ptr(curve, C.c_double))
    return int(kk), curve


def window_box(cfg: OracleConfig, k: int):
    """(z0, z1, x0, x1) support box and (cz, cx, sz, sx) of window k."""
    box = np.zeros(4, np.int32); geom = np.zeros(4)
    cc = cfg.c()
    lib().ora_window_box(C.byref(cc), int(k), _ptr(box, C.c_int), _ptr(geom, C.c_double))
    return tuple(int(v) for v in box), tuple(float(v) for v in geom)


def window_weights(cfg: OracleConfig, k: int) -> np.ndarray:
    """Full-grid Gaussian weights g_k [nz, nx] (0 outside the support)."""
    g = np.zeros(cfg.nz * cfg.nx)
    cc = cfg.c()
    lib().ora_window_weights(C.byref(cc), int(k), _ptr(g, C.c_double))
    return g.reshape(cfg.nz, cfg.nx)
