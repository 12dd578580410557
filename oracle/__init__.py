"""FP64 CPU oracle for the A-DOT scheme (test infrastructure only).

Only the tests, the smoke check and the CPU-baseline leg of ``bench.py`` import
this package. The CUDA library does not depend on it and shares no code with
it. ``build()`` compiles ``adot_oracle.c`` with gcc (``-O2
-ffp-contract=off -fopenmp``) into ``liboracle.so`` beside this file.

Every routine follows the paper (arXiv 1912.04791) as cited in the C source:
Eq. W&A_definition (flux matrix), Eq. charPol / lambda / parameters /
parameters_bis (analytic eigenvalues), Eq. RR / RR-1 / circPerm (eigenvectors),
Eq. asbA / ExAbsA (|A|), Eq. path / DOTjumpN (fluctuations), Eq. PRICEjump /
AiPRICE / Apsi / Im (the PRICE-C comparison scheme), Eq. scheme
(update, with the Strickler friction source of Sec. 2 when K_s > 0), the
sediment feed through an end of the Soni case (Sec. 5.1), and a second-order
MUSCL-Hancock variant of the scheme (path-conservative reconstruction of
states) built on the same DOT edge. ``exact.py`` holds closed-form and exact solutions used as pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adot_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status codes (mirror the C enum)
OK, E_INVALID, E_DEPTH, E_NONFINITE, E_NONHYPERBOLIC, E_NOCONVERGE = range(6)
LAW_GRASS, LAW_MPM, LAW_GRASS_THR, LAW_POWER = 0, 1, 2, 3
ABS_ANALYTIC, ABS_NUMERIC, ABS_SYLVESTER, ABS_NEWTON = 0, 1, 2, 3
SCHEME_DOT, SCHEME_PRICE_C = 0, 1
BC_TRANSMISSIVE, BC_PERIODIC, BC_INFLOW_Q, BC_OUTFLOW_H, BC_INFLOW_QZ, BC_INFLOW_QS, \
    BC_OUTFLOW_HS = range(7)


class OracleError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"oracle {where} failed with status {status}")
        self.status = status


class Law(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("g", ctypes.c_double),
        ("xi", ctypes.c_double),
        ("Ag", ctypes.c_double),
        ("s_rel", ctypes.c_double),
        ("d50", ctypes.c_double),
        ("manning_n", ctypes.c_double),
        ("u_cr", ctypes.c_double),
        ("beta", ctypes.c_double),
    ]


class Cfg(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("x_min", ctypes.c_double),
        ("x_max", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("law", Law),
        ("abs_method", ctypes.c_int),
        ("bc_left", ctypes.c_int),
        ("bc_right", ctypes.c_int),
        ("bcl", ctypes.c_double * 3),
        ("bcr", ctypes.c_double * 3),
        ("ks", ctypes.c_double),
        ("order", ctypes.c_int),
        ("limiter", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("price_eps", ctypes.c_double),
    ]


def grass(Ag: float, xi: float = 1.0, g: float = 9.81) -> Law:
    """Grass law q_s = A_g u^3 (Eq. Grass)."""
    return Law(LAW_GRASS, g, xi, Ag, 0.0, 0.0, 0.0)


def grass_thr(Ag: float, u_cr: float, xi: float = 1.0, g: float = 9.81) -> Law:
    """Grass law with a threshold velocity (Eq. GrassThr), read as
    q_s = A_g sign(u) max(|u| - u_cr, 0)^3."""
    return Law(LAW_GRASS_THR, g, xi, Ag, 0.0, 0.0, 0.0, u_cr)


def power(alpha: float, beta: float, u_cr: float = 0.0, xi: float = 1.0, g: float = 9.81) -> Law:
    """Power law of the velocity, q_s = alpha sign(u) max(|u| - u_cr, 0)^beta
    (Eq. Soni_qs with u_cr = 0; Eq. GrassThr at beta = 3)."""
    return Law(LAW_POWER, g, xi, alpha, 0.0, 0.0, 0.0, u_cr, beta)


def mpm(s_rel: float, d50: float, manning_n: float, xi: float = 1.0, g: float = 9.81) -> Law:
    """Meyer-Peter & Mueller law with a Manning friction slope (Eq. MPM, Eq. Shields)."""
    return Law(LAW_MPM, g, xi, 0.0, s_rel, d50, manning_n)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc; returns the library path."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
            return _LIB_PATH
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(Law)
        L.orc_sediment.argtypes = [lp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_flux_matrix.argtypes = [lp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_eigvals_analytic.argtypes = [lp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_eigvecs_analytic.argtypes = [lp, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        L.orc_qr_eigenvalues.argtypes = [dp, dp]
        L.orc_eig_numeric.argtypes = [dp, dp, dp, dp]
        L.orc_inverse3.argtypes = [dp, dp]
        L.orc_abs_matrix.argtypes = [lp, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_fluct_edge.argtypes = [lp, ctypes.c_int, dp, dp, dp, dp]
        L.orc_fluct.argtypes = [lp, ctypes.c_int, ctypes.c_int64, dp, dp, dp, dp]
        L.orc_spectral_radius.argtypes = [lp, ctypes.c_double, ctypes.c_double, dp]
        L.orc_run.argtypes = [ctypes.POINTER(Cfg), dp, dp, dp, ctypes.c_int64, ctypes.c_double,
                              dp, ctypes.POINTER(ctypes.c_int64), dp, dp]
        L.orc_abs_psi_batch.argtypes = [lp, ctypes.c_int, ctypes.c_int64, dp, dp, dp]
        L.orc_a_psi.argtypes = [lp, dp, dp, dp]
        L.orc_price_fluct.argtypes = [lp, ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double,
                                      dp, dp]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(st: int, where: str):
    if st != OK:
        raise OracleError(st, where)


def sediment(law: Law, h: float, q: float):
    """(q_s, dq_s/dh, dq_s/dq) at one state."""
    out = np.zeros(3)
    o = [ctypes.c_double() for _ in range(3)]
    _check(lib().orc_sediment(ctypes.byref(law), h, q, *[ctypes.byref(x) for x in o]), "sediment")
    out[:] = [x.value for x in o]
    return out


def flux_matrix(law: Law, h: float, q: float) -> np.ndarray:
    A = np.zeros(9)
    _check(lib().orc_flux_matrix(ctypes.byref(law), h, q, _p(A)), "flux_matrix")
    return A.reshape(3, 3)


def eigvals_analytic(law: Law, h: float, q: float, with_arg: bool = False):
    lam = np.zeros(3)
    arg = ctypes.c_double()
    _check(lib().orc_eigvals_analytic(ctypes.byref(law), h, q, _p(lam), ctypes.byref(arg)),
           "eigvals_analytic")
    return (lam, arg.value) if with_arg else lam


def eigvecs_analytic(law: Law, h: float, q: float, lam: np.ndarray):
    R = np.zeros(9)
    Ri = np.zeros(9)
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    _check(lib().orc_eigvecs_analytic(ctypes.byref(law), h, q, _p(lam), _p(R), _p(Ri)),
           "eigvecs_analytic")
    return R.reshape(3, 3), Ri.reshape(3, 3)


def qr_eigenvalues(A: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    lam = np.zeros(3)
    _check(lib().orc_qr_eigenvalues(_p(A), _p(lam)), "qr_eigenvalues")
    return lam


def eig_numeric(A: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64).reshape(9)
    lam, R, Ri = np.zeros(3), np.zeros(9), np.zeros(9)
    _check(lib().orc_eig_numeric(_p(A), _p(lam), _p(R), _p(Ri)), "eig_numeric")
    return lam, R.reshape(3, 3), Ri.reshape(3, 3)


def inverse3(M: np.ndarray) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64).reshape(9)
    out = np.zeros(9)
    _check(lib().orc_inverse3(_p(M), _p(out)), "inverse3")
    return out.reshape(3, 3)


def abs_matrix(law: Law, h: float, q: float, method: int = ABS_ANALYTIC) -> np.ndarray:
    out = np.zeros(9)
    lam = np.zeros(3)
    _check(lib().orc_abs_matrix(ctypes.byref(law), method, h, q, _p(out), _p(lam)), "abs_matrix")
    return out.reshape(3, 3)


def spectral_radius(law: Law, h: float, q: float) -> float:
    r = ctypes.c_double()
    _check(lib().orc_spectral_radius(ctypes.byref(law), h, q, ctypes.byref(r)), "spectral_radius")
    return r.value


def fluct_edge(law: Law, WL, WR, method: int = ABS_ANALYTIC):
    wl = np.ascontiguousarray(WL, dtype=np.float64)
    wr = np.ascontiguousarray(WR, dtype=np.float64)
    dm, dp = np.zeros(3), np.zeros(3)
    _check(lib().orc_fluct_edge(ctypes.byref(law), method, _p(wl), _p(wr), _p(dm), _p(dp)),
           "fluct_edge")
    return dm, dp


def fluct(law: Law, WL: np.ndarray, WR: np.ndarray, method: int = ABS_ANALYTIC):
    """Batch fluctuations. WL, WR: [3, n] (rows h, q, z). Returns (Dm, Dp) as [3, n]."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    n = WL.shape[1]
    Dm = np.zeros((3, n))
    Dp = np.zeros((3, n))
    _check(lib().orc_fluct(ctypes.byref(law), method, n, _p(WL), _p(WR), _p(Dm), _p(Dp)), "fluct")
    return Dm, Dp


def abs_psi(law: Law, WL: np.ndarray, WR: np.ndarray, method: int = ABS_ANALYTIC) -> np.ndarray:
    """|A|_Psi = sum_k w_k |A(Psi(s_k))| of each edge (WL, WR: [3, n]); returns [n, 9]."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    n = WL.shape[1]
    out = np.zeros((n, 9))
    _check(lib().orc_abs_psi_batch(ctypes.byref(law), method, n, _p(WL), _p(WR), _p(out)), "abs_psi")
    return out


def a_psi(law: Law, WL, WR) -> np.ndarray:
    """A^Psi of one edge (Eq. Apsi, 3-point Gauss-Legendre rule), 3 x 3."""
    wl = np.ascontiguousarray(WL, dtype=np.float64)
    wr = np.ascontiguousarray(WR, dtype=np.float64)
    out = np.zeros(9)
    _check(lib().orc_a_psi(ctypes.byref(law), _p(wl), _p(wr), _p(out)), "a_psi")
    return out.reshape(3, 3)


def price_fluct(law: Law, WL: np.ndarray, WR: np.ndarray, nu: float, eps: float):
    """PRICE-C fluctuations (Eq. PRICEjump, Eq. AiPRICE) of a batch of edges,
    WL, WR [3, n], with nu = dt/dx and the small parameter eps; (Dm, Dp) [3, n]."""
    WL = np.ascontiguousarray(WL, dtype=np.float64)
    WR = np.ascontiguousarray(WR, dtype=np.float64)
    n = WL.shape[1]
    Dm = np.zeros((3, n))
    Dp = np.zeros((3, n))
    _check(lib().orc_price_fluct(ctypes.byref(law), n, _p(WL), _p(WR), nu, eps, _p(Dm), _p(Dp)),
           "price_fluct")
    return Dm, Dp


def make_cfg(n: int, x_min: float, x_max: float, cfl: float, law: Law,
             bc_left: int = BC_TRANSMISSIVE, bc_right: int = BC_TRANSMISSIVE,
             bcl=(0.0, 0.0, 0.0), bcr=(0.0, 0.0, 0.0), method: int = ABS_ANALYTIC,
             ks: float = 0.0, order: int = 1, limiter: int = 0, scheme: int = SCHEME_DOT,
             price_eps: float = 1.0) -> Cfg:
    """Run configuration; ks > 0 adds the Strickler friction source (Sec. 2);
    order = 2 selects the second-order MUSCL-Hancock variant (limiter 0 = minmod,
    1 = zero slopes); scheme = SCHEME_PRICE_C replaces the DOT jump function by
    PRICE-C's (Sec. 3.2) with the small parameter price_eps of Eq. Im."""
    c = Cfg()
    c.n = n
    c.x_min = x_min
    c.x_max = x_max
    c.cfl = cfl
    c.law = law
    c.abs_method = method
    c.bc_left = bc_left
    c.bc_right = bc_right
    for i in range(3):
        c.bcl[i] = bcl[i]
        c.bcr[i] = bcr[i]
    c.ks = ks
    c.order = order
    c.limiter = limiter
    c.scheme = scheme
    c.price_eps = price_eps
    return c


def run(cfg: Cfg, h, q, z, max_steps: int = 2**62, t_end: float = float("inf"), t0: float = 0.0):
    """Advances copies of (h, q, z); returns (h, q, z, t, steps, dt_last)."""
    h = np.array(h, dtype=np.float64, copy=True)
    q = np.array(q, dtype=np.float64, copy=True)
    z = np.array(z, dtype=np.float64, copy=True)
    assert h.shape == q.shape == z.shape == (cfg.n,)
    work = np.zeros(6 * (cfg.n + 1))
    t = ctypes.c_double(t0)
    steps = ctypes.c_int64(0)
    dtl = ctypes.c_double(0.0)
    st = lib().orc_run(ctypes.byref(cfg), _p(h), _p(q), _p(z), max_steps, t_end, ctypes.byref(t),
                       ctypes.byref(steps), ctypes.byref(dtl), _p(work))
    _check(st, "run")
    return h, q, z, t.value, steps.value, dtl.value


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(n)
