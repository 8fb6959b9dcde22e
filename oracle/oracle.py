"""ctypes wrapper of the FP64 CPU oracle (gaps_oracle.cpp).

Test infrastructure: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module. The product path never does.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gaps_oracle.cpp")
LIB = os.path.join(HERE, "liboracle_%s.so" % platform.machine())

CFLAGS = ["-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread"]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (plain g++)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", *CFLAGS, "-o", tmp, SRC])
        os.replace(tmp, LIB)
    return LIB


class OracleConfig(ctypes.Structure):
    _fields_ = [
        ("process", ctypes.c_int), ("nf", ctypes.c_int), ("nmax", ctypes.c_int),
        ("fixed_alpha", ctypes.c_int), ("channel_mask", ctypes.c_uint32),
        ("pair_fixed", ctypes.c_int),
        ("sqrt_s", ctypes.c_double), ("alpha_s_mz", ctypes.c_double),
        ("t_cut", ctypes.c_double), ("p_s", ctypes.c_double),
        ("t_start", ctypes.c_double), ("y_fixed", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("pdf", ctypes.c_void_p),
        ("mll_lo", ctypes.c_double), ("mll_hi", ctypes.c_double),
    ]


class OracleOut(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in (
        "p", "flav", "col", "acol", "initial", "npart", "status", "n_emit",
        "weight", "eta", "t_first", "obs", "counters")]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i, u32, vp = ctypes.c_double, ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p
        P = ctypes.POINTER
        _lib.oracle_run.argtypes = [P(OracleConfig), ctypes.c_uint64, ctypes.c_uint64, P(OracleOut)]
        _lib.oracle_hard.argtypes = _lib.oracle_run.argtypes
        _lib.oracle_run_threads.argtypes = [P(OracleConfig), ctypes.c_uint64, ctypes.c_uint64,
                                            P(OracleOut), i]
        _lib.oracle_run_mix.argtypes = [vp, vp, i, ctypes.c_uint64, ctypes.c_uint64, P(OracleOut), vp, i]
        _lib.oracle_mix_rows.argtypes = [ctypes.c_uint64, vp, i, ctypes.c_uint64, ctypes.c_uint64, vp]
        _lib.oracle_philox.argtypes = [vp, vp, vp]
        _lib.oracle_uniform.argtypes = [u32, u32]
        _lib.oracle_uniform.restype = d
        _lib.oracle_pdf_xf.argtypes = [vp, i, d, d]
        _lib.oracle_pdf_xf.restype = d
        _lib.oracle_pdf_xf_batch.argtypes = [vp, i, i, vp, vp, vp]
        _lib.oracle_pdf_bound.argtypes = [vp, i, i, d]
        _lib.oracle_pdf_bound.restype = d
        _lib.oracle_alpha_s.argtypes = [P(OracleConfig), d]
        _lib.oracle_alpha_s.restype = d
        _lib.oracle_li2.argtypes = [d]
        _lib.oracle_li2.restype = d
        _lib.oracle_exp.argtypes = [d]
        _lib.oracle_exp.restype = d
        _lib.oracle_log.argtypes = [d]
        _lib.oracle_log.restype = d
        _lib.oracle_sincos2pi.argtypes = [d, vp]
        _lib.oracle_collinear.argtypes = [d, d, i, d]
        _lib.oracle_collinear.restype = d
        _lib.oracle_born_me2.argtypes = [i]
        _lib.oracle_born_me2.restype = d
        _lib.oracle_born_density.argtypes = [P(OracleConfig), i, d, d]
        _lib.oracle_born_density.restype = d
        _lib.oracle_ee_dsigma.argtypes = [d, i, d]
        _lib.oracle_ee_dsigma.restype = d
        _lib.oracle_ll_dsigma.argtypes = [d, i, d]
        _lib.oracle_ll_dsigma.restype = d
        _lib.oracle_z_limits.argtypes = [i, d, d, d, vp]
        _lib.oracle_shape_sample.argtypes = [i, d, d, d, vp]
        _lib.oracle_shape_integral.argtypes = [i, d, d]
        _lib.oracle_shape_integral.restype = d
        _lib.oracle_basis.argtypes = [vp, vp, vp, vp]
        _lib.oracle_ee_shapes.argtypes = [vp, i, vp]
        _lib.oracle_antikt.argtypes = [vp, i, d, vp]
        _lib.oracle_antikt.restype = i
        _lib.oracle_first_emission.argtypes = [P(OracleConfig), i, i, d, d, ctypes.c_uint64, vp]
        _lib.oracle_first_emission_record.argtypes = [P(OracleConfig), i, i, d, d, ctypes.c_uint64, vp, vp,
                                                      vp]
        _lib.oracle_if_map.argtypes = [d, d, d, vp]
        _lib.oracle_mlp_forward.argtypes = [vp, vp, ctypes.c_uint64, vp]
        _lib.oracle_mlp_loss_grad.argtypes = [vp, vp, vp, ctypes.c_uint64, d, vp]
        _lib.oracle_mlp_loss_grad.restype = d
        _lib.oracle_ii_map.argtypes = [d, d, d, vp]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Settings:
    process: int = 0
    sqrt_s: float = 91.2
    t_cut: float = 1.0
    alpha_s_mz: float = 0.118
    nf: int = 5
    nmax: int = 64
    seed: int = 1
    p_s: float = 0.5
    fixed_alpha: bool = False
    channel_mask: int = 0
    pair_fixed: int = -1
    t_start: float = 0.0
    y_fixed: float = math.nan
    mll_lo: float = 66.0   # process 3: dilepton mass window (GeV)
    mll_hi: float = 116.0

    def to_c(self, pdf: np.ndarray | None) -> OracleConfig:
        return OracleConfig(self.process, self.nf, self.nmax, int(self.fixed_alpha),
                            self.channel_mask, self.pair_fixed, self.sqrt_s, self.alpha_s_mz,
                            self.t_cut, self.p_s, self.t_start, self.y_fixed,
                            self.seed, None if pdf is None else pdf.ctypes.data,
                            self.mll_lo, self.mll_hi)


COUNTER_NAMES = ("steps", "trials", "isr_trials", "vetoes", "accepts", "violations")


def run(settings: Settings, first: int, n: int, pdf: np.ndarray | None = None,
        threads: int = 1, hard_only: bool = False) -> dict:
    """Generate, shower and measure events [first, first + n). Returns numpy arrays."""
    if pdf is not None:
        pdf = np.ascontiguousarray(pdf, dtype=np.float32)
    nm = settings.nmax
    out = {
        "p": np.zeros((n, nm, 4)), "flav": np.zeros((n, nm), np.int32),
        "col": np.zeros((n, nm), np.int32), "acol": np.zeros((n, nm), np.int32),
        "initial": np.zeros((n, nm), np.int32), "npart": np.zeros(n, np.int32),
        "status": np.zeros(n, np.int32), "n_emit": np.zeros(n, np.int32),
        "weight": np.zeros(n), "eta": np.zeros((n, 2)), "t_first": np.zeros(n),
        "obs": np.zeros((n, 8)), "counters": np.zeros((n, 6), np.uint64),
    }
    o = OracleOut(**{k: _ptr(v) for k, v in out.items()})
    c = settings.to_c(pdf)
    L = lib()
    if hard_only:
        rc = L.oracle_hard(ctypes.byref(c), first, n, ctypes.byref(o))
    elif threads > 1:
        rc = L.oracle_run_threads(ctypes.byref(c), first, n, ctypes.byref(o), threads)
    else:
        rc = L.oracle_run(ctypes.byref(c), first, n, ctypes.byref(o))
    if rc != 0:
        raise RuntimeError("oracle_run failed (%d)" % rc)
    return out


def run_mix(rows: list, fractions, first: int, n: int, pdf: np.ndarray | None = None,
            threads: int = 1) -> dict:
    """Mixed batch: rows are Settings (equal seed and nmax), fractions their
    shares; event first + i takes the row of its Philox draw 2^62. Returns the
    arrays of run() plus "row" [n]."""
    if pdf is not None:
        pdf = np.ascontiguousarray(pdf, dtype=np.float32)
    nm = rows[0].nmax
    out = {
        "p": np.zeros((n, nm, 4)), "flav": np.zeros((n, nm), np.int32),
        "col": np.zeros((n, nm), np.int32), "acol": np.zeros((n, nm), np.int32),
        "initial": np.zeros((n, nm), np.int32), "npart": np.zeros(n, np.int32),
        "status": np.zeros(n, np.int32), "n_emit": np.zeros(n, np.int32),
        "weight": np.zeros(n), "eta": np.zeros((n, 2)), "t_first": np.zeros(n),
        "obs": np.zeros((n, 8)), "counters": np.zeros((n, 6), np.uint64),
    }
    o = OracleOut(**{k: _ptr(v) for k, v in out.items()})
    cfgs = (OracleConfig * len(rows))(*[r.to_c(pdf if r.process else None) for r in rows])
    fr = np.ascontiguousarray(fractions, dtype=np.float64)
    row = np.zeros(n, np.int32)
    rc = lib().oracle_run_mix(ctypes.cast(cfgs, ctypes.c_void_p), _ptr(fr), len(rows), first, n,
                              ctypes.byref(o), _ptr(row), threads)
    if rc != 0:
        raise RuntimeError("oracle_run_mix failed (%d)" % rc)
    out["row"] = row
    return out


def mix_rows(seed: int, fractions, first: int, n: int) -> np.ndarray:
    """Row of each event first .. first + n - 1 of a mixed batch."""
    fr = np.ascontiguousarray(fractions, dtype=np.float64)
    out = np.zeros(n, np.int32)
    if lib().oracle_mix_rows(seed, _ptr(fr), len(fr), first, n, _ptr(out)) != 0:
        raise RuntimeError("oracle_mix_rows failed")
    return out


def philox(ctr, key) -> list[int]:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox(_ptr(c), _ptr(k), _ptr(o))
    return [int(v) for v in o]


def uniform(lo: int, hi: int) -> float:
    return lib().oracle_uniform(lo, hi)


def pdf_xf(pdf: np.ndarray, f: int, x: float, q2: float) -> float:
    return lib().oracle_pdf_xf(_ptr(pdf), f, x, q2)


def pdf_xf_batch(pdf: np.ndarray, f: int, x, q2) -> np.ndarray:
    x = np.ascontiguousarray(np.broadcast_to(x, np.broadcast(x, q2).shape), dtype=np.float64)
    q2 = np.ascontiguousarray(np.broadcast_to(q2, x.shape), dtype=np.float64)
    out = np.zeros(x.shape)
    lib().oracle_pdf_xf_batch(_ptr(pdf), f, x.size, _ptr(x), _ptr(q2), _ptr(out))
    return out


def pdf_bound(pdf: np.ndarray, num: int, den: int, eta: float) -> float:
    return lib().oracle_pdf_bound(_ptr(pdf), num, den, eta)


def alpha_s(settings: Settings, t: float) -> float:
    c = settings.to_c(None)
    return lib().oracle_alpha_s(ctypes.byref(c), t)


def li2(x: float) -> float:
    return lib().oracle_li2(x)


def exp(x: float) -> float:
    return lib().oracle_exp(x)


def log(x: float) -> float:
    return lib().oracle_log(x)


def sincos2pi(R: float):
    o = np.zeros(2)
    lib().oracle_sincos2pi(R, _ptr(o))
    return float(o[0]), float(o[1])


def collinear(as_: float, L: float, which: str, x: float = 0.0) -> float:
    idx = {"A": 0, "B": 1, "g": 2, "hqq": 3, "hqg": 4}[which]
    return lib().oracle_collinear(as_, L, idx, x)


def born_me2(f: int) -> float:
    return lib().oracle_born_me2(f)


def born_density(settings: Settings, pdf: np.ndarray, k: int, ea: float, eb: float) -> float:
    c = settings.to_c(pdf)
    return lib().oracle_born_density(ctypes.byref(c), k, ea, eb)


def ee_dsigma(s: float, f: int, cth: float) -> float:
    return lib().oracle_ee_dsigma(s, f, cth)


def ll_dsigma(s: float, f: int, cth: float) -> float:
    """q qbar -> gamma*/Z -> e- e+: dsigma/dcos(theta*) in GeV^-2 (theta* between quark and electron)."""
    return lib().oracle_ll_dsigma(s, f, cth)


def z_limits(dtype: int, t: float, s: float, eta: float):
    o = np.zeros(2)
    ok = lib().oracle_z_limits(dtype, t, s, eta, _ptr(o))
    return (bool(ok), float(o[0]), float(o[1]))


def shape_sample(shape: int, zm: float, delta: float, R: float):
    o = np.zeros(2)
    lib().oracle_shape_sample(shape, zm, delta, R, _ptr(o))
    return float(o[0]), float(o[1])


def shape_integral(shape: int, zm: float, delta: float) -> float:
    return lib().oracle_shape_integral(shape, zm, delta)


def basis(P, K):
    P = np.ascontiguousarray(P, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float64)
    e1 = np.zeros(4)
    e2 = np.zeros(4)
    lib().oracle_basis(_ptr(P), _ptr(K), _ptr(e1), _ptr(e2))
    return e1, e2


def ee_shapes(p: np.ndarray):
    p = np.ascontiguousarray(p, dtype=np.float64)
    o = np.zeros(3)
    lib().oracle_ee_shapes(_ptr(p), p.shape[0], _ptr(o))
    return o


def antikt(p: np.ndarray, R: float = 0.4) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64)
    out = np.zeros((max(1, p.shape[0]), 4))
    nj = lib().oracle_antikt(_ptr(p), p.shape[0], R, _ptr(out))
    return out[:nj]


DIPOLE_FF, DIPOLE_FI_IF, DIPOLE_II = 0, 1, 2


def first_emission(settings: Settings, pdf: np.ndarray | None, dipole: int, flq: int,
                   s: float, eta: float, n: int) -> np.ndarray:
    """Scale of the first emission of an isolated dipole (0 = none), n trials.

    dipole: DIPOLE_FF (final q + final qbar), DIPOLE_FI_IF (final q + incoming q
    at eta), DIPOLE_II (incoming q at eta from beam 1 + incoming qbar from beam 2).
    """
    if pdf is not None:
        pdf = np.ascontiguousarray(pdf, dtype=np.float32)
    out = np.zeros(n)
    c = settings.to_c(pdf)
    rc = lib().oracle_first_emission(ctypes.byref(c), dipole, flq, s, eta, n, _ptr(out))
    if rc != 0:
        raise RuntimeError("oracle_first_emission failed")
    return out


def first_emission_record(settings: Settings, pdf: np.ndarray | None, dipole: int, flq: int,
                          s: float, eta: float, n: int) -> dict:
    """As first_emission, with the record after the first emission:
    "p" [n][3][4], "flav", "col", "acol", "initial" [n][3] (slots 0..2; the
    third is empty when nothing was emitted) and "eta" [n][2]."""
    if pdf is not None:
        pdf = np.ascontiguousarray(pdf, dtype=np.float32)
    t = np.zeros(n)
    rec = np.zeros((n, 3, 8))
    eta_out = np.zeros((n, 2))
    c = settings.to_c(pdf)
    rc = lib().oracle_first_emission_record(ctypes.byref(c), dipole, flq, s, eta, n, _ptr(t), _ptr(rec),
                                            _ptr(eta_out))
    if rc != 0:
        raise RuntimeError("oracle_first_emission_record failed")
    return {"t": t, "p": rec[:, :, :4], "flav": rec[:, :, 4].astype(int), "col": rec[:, :, 5].astype(int),
            "acol": rec[:, :, 6].astype(int), "initial": rec[:, :, 7].astype(bool), "eta": eta_out}


def if_map(r: float, z: float, omz: float):
    o = np.zeros(4)
    ok = lib().oracle_if_map(r, z, omz, _ptr(o))
    return bool(ok), o


def ii_map(r: float, z: float, omz: float):
    o = np.zeros(3)
    ok = lib().oracle_ii_map(r, z, omz, _ptr(o))
    return bool(ok), o


MLP_PARAMS = 64 * 4 + 64 + 64 * 64 + 64 + 64 + 1


def mlp_forward(params, X) -> np.ndarray:
    """FP64 reference forward of the 4-64-64-1 ReLU network."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0])
    lib().oracle_mlp_forward(_ptr(P), _ptr(X), X.shape[0], _ptr(out))
    return out


def mlp_loss_grad(params, X, T, tau: float):
    """FP64 reference expectile loss and its gradient by backpropagation."""
    P = np.ascontiguousarray(params, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    g = np.zeros(MLP_PARAMS)
    loss = lib().oracle_mlp_loss_grad(_ptr(P), _ptr(X), _ptr(T), X.shape[0], tau, _ptr(g))
    return loss, g
