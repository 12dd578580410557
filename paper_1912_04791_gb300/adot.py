"""Thin ctypes binding of libadot.so (the C ABI of include/adot.h).

Functions carry the C names and only marshal arguments: numpy arrays are
passed as host pointers (on_device=0), torch CUDA tensors as device pointers
(on_device=1); every step of the computation runs in the library's CUDA
kernels. Loading fails loudly when the library has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libadot.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "adot.h")

OK, E_INVALID_ARG, E_NONPOSITIVE_DEPTH, E_NONFINITE, E_NONHYPERBOLIC, E_CUDA, E_TIMEOUT, \
    E_UNSUPPORTED = range(8)
LAW_GRASS, LAW_MPM, LAW_GRASS_THR, LAW_POWER = 0, 1, 2, 3
FP64, FP32 = 0, 1
SCHEME_DOT, SCHEME_PRICE_C = 0, 1
BC_TRANSMISSIVE, BC_PERIODIC, BC_INFLOW_Q, BC_OUTFLOW_H, BC_INFLOW_QZ, BC_INFLOW_QS, \
    BC_OUTFLOW_HS = range(7)


class AdotError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = status_string(status) if _lib is not None else str(status)
        super().__init__(f"{where}: {msg} (status {status})")


class Law(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("g", ctypes.c_double), ("xi", ctypes.c_double),
                ("Ag", ctypes.c_double), ("s_rel", ctypes.c_double), ("d50", ctypes.c_double),
                ("manning_n", ctypes.c_double), ("u_cr", ctypes.c_double),
                ("beta", ctypes.c_double)]


class Config(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int64), ("x_min", ctypes.c_double),
                ("x_max", ctypes.c_double), ("cfl", ctypes.c_double), ("law", Law),
                ("precision", ctypes.c_int32), ("bc_left", ctypes.c_int32),
                ("bc_right", ctypes.c_int32), ("bc_left_value", ctypes.c_double * 3),
                ("bc_right_value", ctypes.c_double * 3), ("block_threads", ctypes.c_int32),
                ("steps_per_graph", ctypes.c_int32), ("device", ctypes.c_int32),
                ("reg_cap", ctypes.c_int32), ("step_kernel", ctypes.c_int32),
                ("ks", ctypes.c_double), ("order", ctypes.c_int32),
                ("scheme", ctypes.c_int32), ("price_eps", ctypes.c_double)]


class EnsembleConfig(ctypes.Structure):
    _fields_ = [("n_channels", ctypes.c_int32), ("n_cells", ctypes.POINTER(ctypes.c_int64)),
                ("length", ctypes.POINTER(ctypes.c_double)), ("Ag", ctypes.POINTER(ctypes.c_double)),
                ("g", ctypes.c_double), ("xi", ctypes.c_double), ("cfl", ctypes.c_double),
                ("precision", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("steps_per_graph", ctypes.c_int32), ("device", ctypes.c_int32),
                ("step_kernel", ctypes.c_int32)]


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib() -> ctypes.CDLL:
    """Loads libadot.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: call paper_1912_04791_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        i32, i64, dbl = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        sig = {
            "adot_create": ([ctypes.POINTER(Config), _P, ctypes.POINTER(_P)], i32),
            "adot_destroy": ([_P], None),
            "adot_set_state": ([_P, _P, _P, _P, i32, dbl], i32),
            "adot_get_state": ([_P, _P, _P, _P, i32], i32),
            "adot_checkpoint_size": ([_P, ctypes.POINTER(i64)], i32),
            "adot_checkpoint_save": ([_P, _P, i64, i32], i32),
            "adot_checkpoint_load": ([_P, _P, i64, i32], i32),
            "adot_step": ([_P, i64, _D, _D], i32),
            "adot_enqueue_steps": ([_P, i64], i32),
            "adot_run_to": ([_P, dbl, ctypes.POINTER(i64)], i32),
            "adot_query": ([_P, _D, ctypes.POINTER(i64), _D], i32),
            "adot_fluctuations": ([_P, _P, _P, i64, _P, _P, _D, i32], i32),
            "adot_price_fluctuations": ([_P, _P, _P, i64, dbl, _P, _P, i32], i32),
            "adot_conserved_sums": ([_P, _D], i32),
            "adot_precision_stats": ([_P, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
            "adot_autotune": ([_P, i64, ctypes.POINTER(i32), ctypes.POINTER(i32),
                               ctypes.POINTER(i32)], i32),
            "adot_step_noalloc": ([ctypes.POINTER(Config), _P, _P, _P, i64, _D, _P], i32),
            "adot_mlp_create": ([i64, _P, ctypes.POINTER(_P)], i32),
            "adot_mlp_destroy": ([_P], None),
            "adot_mlp_set_params": ([_P, _P], i32),
            "adot_mlp_get_params": ([_P, _P], i32),
            "adot_mlp_set_engine": ([_P, i32], i32),
            "adot_mlp_set_train_engine": ([_P, i32], i32),
            "adot_mlp_inject_fault": ([_P, i32], i32),
            "adot_mlp_set_data": ([_P, _P, _P, i64, i32], i32),
            "adot_mlp_get_stats": ([_P, _P, _P], i32),
            "adot_mlp_forward": ([_P, _P, i64, _P, i32], i32),
            "adot_mlp_gradient": ([_P, _P, _P, i64, ctypes.POINTER(ctypes.c_float), _P], i32),
            "adot_mlp_train": ([_P, i64, i64, dbl, ctypes.c_uint64, _P], i32),
            "adot_mlp_apply_gradient": ([_P, _P, dbl, i64], i32),
            "adot_set_surrogate": ([_P, _P, dbl, dbl], i32),
            "adot_surrogate_stats": ([_P, ctypes.POINTER(i64), ctypes.POINTER(i64)], i32),
            "adot_surrogate_eval": ([_P, _P, i32, ctypes.POINTER(i64)], i32),
            "adot_harvest": ([_P, i64, ctypes.c_uint64, _P, _P, i32], i32),
            "adot_ensemble_create": ([ctypes.POINTER(EnsembleConfig), _P, ctypes.POINTER(_P)], i32),
            "adot_ensemble_destroy": ([_P], None),
            "adot_ensemble_set_state": ([_P, _P, _P, _P, i32], i32),
            "adot_ensemble_get_state": ([_P, _P, _P, _P, i32], i32),
            "adot_ensemble_run_to": ([_P, dbl, ctypes.POINTER(i64)], i32),
            "adot_ensemble_step": ([_P, i64], i32),
            "adot_ensemble_query": ([_P, _P, _P, ctypes.POINTER(i64)], i32),
            "adot_ensemble_info": ([_P, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                    ctypes.POINTER(i32), ctypes.POINTER(i32)], i32),
            "adot_ensemble_plan": ([_P, i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                    ctypes.POINTER(i32), ctypes.POINTER(i32), _D], i32),
            "adot_ensemble_inject_fault": ([_P, i32], i32),
            "adot_measure_pipe": ([i32, i32, _D, _D], i32),
            "adot_math_probe": ([i32, _P, _P, i64, _P], i32),
            "adot_status_string": ([i32], ctypes.c_char_p),
            "adot_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def header_functions() -> list[str]:
    """Names of the functions include/adot.h declares."""
    with open(HEADER) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adot_\w+)\s*\(", text)))


def status_string(st: int) -> str:
    return lib().adot_status_string(st).decode()


def version() -> str:
    return lib().adot_version().decode()


def _check(st: int, where: str):
    if st != OK:
        raise AdotError(st, where)


def _ptr(a, n=None):
    """(address, on_device) of a float64 contiguous numpy array or torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy arrays must be contiguous float64")
        if n is not None and a.size != n:
            raise ValueError(f"expected {n} values, got {a.size}")
        return a.ctypes.data, 0
    import torch  # only for device memory
    if not isinstance(a, torch.Tensor):
        raise TypeError("expected a numpy array or a torch tensor")
    if a.dtype != torch.float64 or not a.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    if n is not None and a.numel() != n:
        raise ValueError(f"expected {n} values, got {a.numel()}")
    return a.data_ptr(), (1 if a.is_cuda else 0)


def make_config(n_cells, x_min, x_max, cfl, Ag, xi, precision=FP32, bc_left=BC_TRANSMISSIVE,
                bc_right=BC_TRANSMISSIVE, bcl=(0.0, 0.0, 0.0), bcr=(0.0, 0.0, 0.0), g=9.81,
                law=LAW_GRASS, s_rel=0.0, d50=0.0, manning_n=0.0, block_threads=0,
                steps_per_graph=0, device=-1, reg_cap=0, step_kernel=0, u_cr=0.0, beta=0.0,
                ks=0.0, order=0, scheme=SCHEME_DOT, price_eps=1e-4) -> Config:
    c = Config()
    c.n_cells = int(n_cells)
    c.x_min, c.x_max, c.cfl = float(x_min), float(x_max), float(cfl)
    c.law = Law(law, g, xi, Ag, s_rel, d50, manning_n, u_cr, beta)
    c.precision = precision
    c.bc_left, c.bc_right = bc_left, bc_right
    for i in range(3):
        c.bc_left_value[i] = float(bcl[i])
        c.bc_right_value[i] = float(bcr[i])
    c.block_threads = block_threads
    c.steps_per_graph = steps_per_graph
    c.device = device
    c.reg_cap = reg_cap
    c.step_kernel = step_kernel
    c.ks = float(ks)
    c.order = int(order)
    c.scheme = int(scheme)
    c.price_eps = float(price_eps)
    return c


def config_for(problem, precision=FP32, **kw) -> Config:
    """Config of a workloads.Problem."""
    return make_config(problem.n, problem.x_min, problem.x_max, problem.cfl, problem.Ag,
                       problem.xi, precision, problem.bc_left, problem.bc_right, problem.bcl,
                       problem.bcr, problem.g, **kw)


def adot_create(cfg: Config, stream=None) -> int:
    s = stream
    if s is not None and not isinstance(s, int):
        s = s.cuda_stream  # torch.cuda.Stream
    out = _P()
    _check(lib().adot_create(ctypes.byref(cfg), s, ctypes.byref(out)), "adot_create")
    return out.value


def adot_destroy(ctx: int) -> None:
    lib().adot_destroy(ctx)


def adot_set_state(ctx: int, h, q, z, t0: float = 0.0, n=None) -> None:
    (ph, dh), (pq, dq), (pz, dz) = _ptr(h, n), _ptr(q, n), _ptr(z, n)
    if not dh == dq == dz:
        raise ValueError("h, q, z must all be on the host or all on the device")
    _check(lib().adot_set_state(ctx, ph, pq, pz, dh, t0), "adot_set_state")


def adot_get_state(ctx: int, h, q, z) -> None:
    (ph, dh), (pq, dq), (pz, dz) = _ptr(h), _ptr(q), _ptr(z)
    if not dh == dq == dz:
        raise ValueError("h, q, z must all be on the host or all on the device")
    _check(lib().adot_get_state(ctx, ph, pq, pz, dh), "adot_get_state")


def adot_checkpoint_size(ctx: int) -> int:
    out = ctypes.c_int64()
    _check(lib().adot_checkpoint_size(ctx, ctypes.byref(out)), "adot_checkpoint_size")
    return out.value


def _blob_ptr(buf):
    """(address, bytes, on_device) of a contiguous uint8 numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if buf.dtype != np.uint8 or not buf.flags["C_CONTIGUOUS"]:
            raise ValueError("checkpoint arrays must be contiguous uint8")
        return buf.ctypes.data, buf.size, 0
    import torch  # only for device memory
    if buf.dtype != torch.uint8 or not buf.is_contiguous():
        raise ValueError("checkpoint tensors must be contiguous uint8")
    return buf.data_ptr(), buf.numel(), (1 if buf.is_cuda else 0)


def adot_checkpoint_save(ctx: int, buf=None):
    """Writes the checkpoint blob into `buf` (uint8 numpy array or CUDA tensor),
    or into a new host array, and returns it."""
    if buf is None:
        buf = np.empty(adot_checkpoint_size(ctx), dtype=np.uint8)
    p, nb, dev = _blob_ptr(buf)
    _check(lib().adot_checkpoint_save(ctx, p, nb, dev), "adot_checkpoint_save")
    return buf


def adot_checkpoint_load(ctx: int, buf) -> None:
    p, nb, dev = _blob_ptr(buf)
    _check(lib().adot_checkpoint_load(ctx, p, nb, dev), "adot_checkpoint_load")


def adot_step(ctx: int, n_steps: int):
    t, dt = ctypes.c_double(), ctypes.c_double()
    _check(lib().adot_step(ctx, n_steps, ctypes.byref(t), ctypes.byref(dt)), "adot_step")
    return t.value, dt.value


def adot_enqueue_steps(ctx: int, n_steps: int) -> None:
    _check(lib().adot_enqueue_steps(ctx, n_steps), "adot_enqueue_steps")


def adot_run_to(ctx: int, t_end: float) -> int:
    s = ctypes.c_int64()
    _check(lib().adot_run_to(ctx, t_end, ctypes.byref(s)), "adot_run_to")
    return s.value


def adot_query(ctx: int):
    t, dt, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().adot_query(ctx, ctypes.byref(t), ctypes.byref(s), ctypes.byref(dt)), "adot_query")
    return t.value, s.value, dt.value


def adot_fluctuations(ctx: int, WL, WR, Dm=None, Dp=None):
    """D-/+ of the edges WL -> WR ([3, n] float64, numpy or CUDA tensors).
    Returns (Dm, Dp, rho_max)."""
    n = WL.shape[1]
    if Dm is None:
        Dm = np.empty((3, n)) if isinstance(WL, np.ndarray) else WL.new_empty((3, n))
    if Dp is None:
        Dp = np.empty((3, n)) if isinstance(WL, np.ndarray) else WL.new_empty((3, n))
    (pl, d1), (pr, d2), (pm, d3), (pp, d4) = _ptr(WL), _ptr(WR), _ptr(Dm), _ptr(Dp)
    if not d1 == d2 == d3 == d4:
        raise ValueError("all arrays must be on the host or all on the device")
    rho = ctypes.c_double()
    _check(lib().adot_fluctuations(ctx, pl, pr, n, pm, pp, ctypes.byref(rho), d1),
           "adot_fluctuations")
    return Dm, Dp, rho.value


def adot_price_fluctuations(ctx: int, WL, WR, dt_over_dx: float, Dm=None, Dp=None):
    """PRICE-C D-/+ of the edges WL -> WR ([3, n] float64, numpy or CUDA tensors)
    with nu = dt/dx. Returns (Dm, Dp)."""
    n = WL.shape[1]
    if Dm is None:
        Dm = np.empty((3, n)) if isinstance(WL, np.ndarray) else WL.new_empty((3, n))
    if Dp is None:
        Dp = np.empty((3, n)) if isinstance(WL, np.ndarray) else WL.new_empty((3, n))
    (pl, d1), (pr, d2), (pm, d3), (pp, d4) = _ptr(WL), _ptr(WR), _ptr(Dm), _ptr(Dp)
    if not d1 == d2 == d3 == d4:
        raise ValueError("all arrays must be on the host or all on the device")
    _check(lib().adot_price_fluctuations(ctx, pl, pr, n, float(dt_over_dx), pm, pp, d1),
           "adot_price_fluctuations")
    return Dm, Dp


def adot_autotune(ctx: int, trial_steps: int = 8):
    """Times the allowed step-kernel variants; returns (block_threads, reg_cap, step_kernel)."""
    b, r, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().adot_autotune(ctx, trial_steps, ctypes.byref(b), ctypes.byref(r), ctypes.byref(k)),
           "adot_autotune")
    return b.value, r.value, k.value


def adot_step_noalloc(cfg: Config, h, q, z, n_steps: int, t0: float = 0.0, stream=None) -> float:
    """Allocation-free stepping of caller-owned float64 CUDA tensors h, q, z
    (in place); returns the time after the steps."""
    (ph, dh), (pq, dq), (pz, dz) = _ptr(h, cfg.n_cells), _ptr(q, cfg.n_cells), _ptr(z, cfg.n_cells)
    if not (dh == dq == dz == 1):
        raise ValueError("adot_step_noalloc takes device arrays")
    s = stream
    if s is not None and not isinstance(s, int):
        s = s.cuda_stream
    t = ctypes.c_double(t0)
    _check(lib().adot_step_noalloc(ctypes.byref(cfg), ph, pq, pz, n_steps, ctypes.byref(t), s),
           "adot_step_noalloc")
    return t.value


class Ensemble:
    """Owning wrapper around an adot_ensemble (batched independent channels).

    step_kernel: 0 chosen per state (default), 3 persistent channel loops,
    5 persistent with cluster teams for the long channels, 1 per-step block
    kernel, 2 per-step warp tiles, 4 per-step, the faster of 1 and 2."""

    def __init__(self, n_cells, length, Ag, xi, cfl=0.9, g=9.81, precision=FP32, block_threads=0,
                 steps_per_graph=0, device=-1, stream=None, step_kernel=0):
        self._n = np.ascontiguousarray(n_cells, dtype=np.int64)
        self._len = np.ascontiguousarray(length, dtype=np.float64)
        self._ag = np.ascontiguousarray(Ag, dtype=np.float64)
        c = EnsembleConfig()
        c.n_channels = len(self._n)
        c.n_cells = self._n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        c.length = self._len.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.Ag = self._ag.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.g, c.xi, c.cfl = g, xi, cfl
        c.precision, c.block_threads, c.steps_per_graph, c.device = precision, block_threads, \
            steps_per_graph, device
        c.step_kernel = step_kernel
        s = stream
        if s is not None and not isinstance(s, int):
            s = s.cuda_stream
        out = _P()
        _check(lib().adot_ensemble_create(ctypes.byref(c), s, ctypes.byref(out)),
               "adot_ensemble_create")
        self.ptr = out.value
        self.C = len(self._n)
        self.total = int(self._n.sum())

    @classmethod
    def from_workload(cls, E, precision=FP32, **kw):
        return cls(E.n_cells, E.length, E.Ag, E.xi, E.cfl, E.g, precision, **kw)

    def set_state(self, h, q, z):
        (ph, dh), (pq, dq), (pz, dz) = _ptr(h, self.total), _ptr(q, self.total), _ptr(z, self.total)
        if not dh == dq == dz:
            raise ValueError("h, q, z must all be on the host or all on the device")
        _check(lib().adot_ensemble_set_state(self.ptr, ph, pq, pz, dh), "adot_ensemble_set_state")

    def get_state(self):
        h, q, z = np.empty(self.total), np.empty(self.total), np.empty(self.total)
        _check(lib().adot_ensemble_get_state(self.ptr, h.ctypes.data, q.ctypes.data, z.ctypes.data, 0),
               "adot_ensemble_get_state")
        return h, q, z

    def run_to(self, t_end: float) -> int:
        n = ctypes.c_int64()
        _check(lib().adot_ensemble_run_to(self.ptr, t_end, ctypes.byref(n)), "adot_ensemble_run_to")
        return n.value

    def step(self, n: int) -> None:
        _check(lib().adot_ensemble_step(self.ptr, n), "adot_ensemble_step")

    def query(self):
        t = np.empty(self.C)
        s = np.empty(self.C, dtype=np.int64)
        cu = ctypes.c_int64()
        _check(lib().adot_ensemble_query(self.ptr, t.ctypes.data, s.ctypes.data, ctypes.byref(cu)),
               "adot_ensemble_query")
        return t, s, cu.value

    def info(self):
        """(threads per block, tiles, resident grid, step kernel: 1 block, 2 warp tiles,
        3 persistent channel loops)."""
        b, g, k = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        nt = ctypes.c_int64()
        _check(lib().adot_ensemble_info(self.ptr, ctypes.byref(b), ctypes.byref(nt), ctypes.byref(g),
                                        ctypes.byref(k)), "adot_ensemble_info")
        return b.value, nt.value, g.value, k.value

    def inject_fault(self, kind: int = 1):
        """Test hook: kind 1 withholds one team member's first arrival in the next
        team launch (bounded waits run out, ADOT_E_TIMEOUT)."""
        _check(lib().adot_ensemble_inject_fault(self.ptr, kind), "adot_ensemble_inject_fault")

    def plan(self, which: int = 0) -> dict:
        """The plan of run_to (which = 0) or step (1): form (3 persistent, 1/2
        per-step), threads per block, cluster (1 or the team size), grid,
        channels run by teams, estimated imbalance."""
        v = [ctypes.c_int32() for _ in range(5)]
        imb = ctypes.c_double()
        _check(lib().adot_ensemble_plan(self.ptr, which, *(ctypes.byref(x) for x in v), ctypes.byref(imb)),
               "adot_ensemble_plan")
        return dict(zip(("form", "block", "cluster", "grid", "teamed"), (x.value for x in v)),
                    imbalance=imb.value)

    def close(self):
        if getattr(self, "ptr", 0):
            lib().adot_ensemble_destroy(self.ptr)
            self.ptr = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_PARAMS = 51721


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


class Mlp:
    """Owning wrapper around an adot_mlp (the |A|_Psi surrogate network)."""

    def __init__(self, max_batch: int, stream=None):
        s = stream
        if s is not None and not isinstance(s, int):
            s = s.cuda_stream
        out = _P()
        _check(lib().adot_mlp_create(max_batch, s, ctypes.byref(out)), "adot_mlp_create")
        self.ptr = out.value
        self.max_batch = max_batch

    def set_params(self, theta):
        t = _f32(theta, (MLP_PARAMS,))
        _check(lib().adot_mlp_set_params(self.ptr, t.ctypes.data), "adot_mlp_set_params")

    def get_params(self) -> np.ndarray:
        t = np.empty(MLP_PARAMS, dtype=np.float32)
        _check(lib().adot_mlp_get_params(self.ptr, t.ctypes.data), "adot_mlp_get_params")
        return t

    def set_data(self, X, T):
        """Training set from host arrays or float32 CUDA tensors X [n, 7], T [n, 9]."""
        if not isinstance(X, np.ndarray):
            n = X.shape[0]
            assert X.shape == (n, 7) and T.shape == (n, 9) and X.is_cuda and T.is_cuda
            _check(lib().adot_mlp_set_data(self.ptr, X.data_ptr(), T.data_ptr(), n, 1),
                   "adot_mlp_set_data")
            return
        X = _f32(X)
        T = _f32(T)
        n = X.shape[0]
        assert X.shape == (n, 7) and T.shape == (n, 9)
        _check(lib().adot_mlp_set_data(self.ptr, X.ctypes.data, T.ctypes.data, n, 0), "adot_mlp_set_data")

    def stats(self):
        st = np.empty(32, dtype=np.float32)
        box = np.empty(14, dtype=np.float32)
        _check(lib().adot_mlp_get_stats(self.ptr, st.ctypes.data, box.ctypes.data), "adot_mlp_get_stats")
        return st, box

    def set_engine(self, engine: int) -> None:
        """Fused inference engine of the surrogate step: 0 = tcgen05 pipeline,
        1 = mma.sync, 2 = tcgen05 with two independent tile groups."""
        _check(lib().adot_mlp_set_engine(self.ptr, int(engine)), "adot_mlp_set_engine")

    def set_train_engine(self, engine: int) -> None:
        """Training kernels: 0 = tcgen05 (default), 1 = mma.sync."""
        _check(lib().adot_mlp_set_train_engine(self.ptr, int(engine)), "adot_mlp_set_train_engine")

    def inject_fault(self, kind: int = 1) -> None:
        """Test hook: the next forward(fused=3) withholds one hand-off so that a
        bounded device-side wait runs out (ADOT_E_TIMEOUT)."""
        _check(lib().adot_mlp_inject_fault(self.ptr, int(kind)), "adot_mlp_inject_fault")

    def forward(self, Xs, fused=False) -> np.ndarray:
        """fused: 0/False per-layer kernels, 1/True mma.sync fused, 2 tcgen05 two
        groups, 3 tcgen05 pipeline."""
        Xs = _f32(Xs)
        n = Xs.shape[0]
        Y = np.empty((n, 9), dtype=np.float32)
        _check(lib().adot_mlp_forward(self.ptr, Xs.ctypes.data, n, Y.ctypes.data, int(fused)),
               "adot_mlp_forward")
        return Y

    def gradient(self, Xs, Ts):
        Xs, Ts = _f32(Xs), _f32(Ts)
        n = Xs.shape[0]
        g = np.empty(MLP_PARAMS, dtype=np.float32)
        loss = ctypes.c_float()
        _check(lib().adot_mlp_gradient(self.ptr, Xs.ctypes.data, Ts.ctypes.data, n, ctypes.byref(loss),
                                       g.ctypes.data), "adot_mlp_gradient")
        return loss.value, g

    def apply_gradient(self, grad, lr: float, total_steps: int = 0) -> None:
        """One Adam step on a given packed gradient (the training update kernel)."""
        g = _f32(grad, (MLP_PARAMS,))
        _check(lib().adot_mlp_apply_gradient(self.ptr, g.ctypes.data, float(lr), int(total_steps)),
               "adot_mlp_apply_gradient")

    def train(self, steps: int, batch: int, lr: float = 1e-3, seed: int = 1) -> np.ndarray:
        h = np.empty(max(steps, 1), dtype=np.float32)
        _check(lib().adot_mlp_train(self.ptr, steps, batch, lr, seed, h.ctypes.data), "adot_mlp_train")
        return h[:steps]

    def close(self):
        if getattr(self, "ptr", 0):
            lib().adot_mlp_destroy(self.ptr)
            self.ptr = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def adot_set_surrogate(ctx: int, mlp, fr_lo: float = 0.8, fr_hi: float = 1.2) -> None:
    _check(lib().adot_set_surrogate(ctx, mlp.ptr if mlp is not None else None, fr_lo, fr_hi),
           "adot_set_surrogate")


def adot_surrogate_stats(ctx: int):
    e, f = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().adot_surrogate_stats(ctx, ctypes.byref(e), ctypes.byref(f)), "adot_surrogate_stats")
    return e.value, f.value


def adot_surrogate_eval(ctx: int, n_edges: int, out=None):
    """The attached network's |A|_Psi on every edge of the current state:
    (absA [9, n_edges] float32 or None, fallback count). `out`: None (new host
    array), False (evaluate only) or a float32 CUDA tensor of shape (9, n_edges)."""
    fb = ctypes.c_int64()
    if out is None:
        out = np.empty((9, n_edges), dtype=np.float32)
        _check(lib().adot_surrogate_eval(ctx, out.ctypes.data, 0, ctypes.byref(fb)), "adot_surrogate_eval")
        return out, fb.value
    if out is False:
        _check(lib().adot_surrogate_eval(ctx, None, 0, ctypes.byref(fb)), "adot_surrogate_eval")
        return None, fb.value
    if tuple(out.shape) != (9, n_edges) or not out.is_cuda:
        raise ValueError("out must be a CUDA tensor of shape (9, n_edges)")
    _check(lib().adot_surrogate_eval(ctx, out.data_ptr(), 1, ctypes.byref(fb)), "adot_surrogate_eval")
    return out, fb.value


def adot_harvest(ctx: int, n: int, seed: int = 1, X=None, T=None):
    """n edge samples of the context's state: (X [n, 7] raw inputs, T [n, 9]
    labels), into new host arrays or the given float32 CUDA tensors."""
    if X is None:
        X = np.empty((n, 7), dtype=np.float32)
        T = np.empty((n, 9), dtype=np.float32)
        _check(lib().adot_harvest(ctx, n, seed, X.ctypes.data, T.ctypes.data, 0), "adot_harvest")
        return X, T
    if X.shape != (n, 7) or T.shape != (n, 9) or not (X.is_cuda and T.is_cuda):
        raise ValueError("X, T must be CUDA tensors of shapes (n, 7) and (n, 9)")
    _check(lib().adot_harvest(ctx, n, seed, X.data_ptr(), T.data_ptr(), 1), "adot_harvest")
    return X, T


def adot_precision_stats(ctx: int):
    """(quadrature nodes of one step, nodes the float32 kernels redo in float64)
    at the current state."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().adot_precision_stats(ctx, ctypes.byref(a), ctypes.byref(b)), "adot_precision_stats")
    return a.value, b.value


PIPE_FFMA, PIPE_FFMA2, PIPE_RSQ, PIPE_SIN, PIPE_DFMA, PIPE_TANH, PIPE_TANH_BF16X2 = range(7)


def adot_math_probe(kind: int, x):
    """The library's float32 device math on a float32 CUDA tensor x: kind 0 the
    step kernels' arccos(x)/3, kind 1 CUDA's acosf(x)/3; returns a new tensor."""
    import torch
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise ValueError("adot_math_probe takes a contiguous float32 CUDA tensor")
    y = torch.empty_like(x)
    _check(lib().adot_math_probe(kind, x.data_ptr(), y.data_ptr(), x.numel(),
                                 torch.cuda.current_stream(x.device).cuda_stream), "adot_math_probe")
    return y


def adot_measure_pipe(kind: int, device: int = -1):
    """(rate, seconds) of one pipe-throughput probe: flops/s for FFMA, FFMA2
    and DFMA, ops/s for the multi-function-unit kinds."""
    r, sec = ctypes.c_double(), ctypes.c_double()
    _check(lib().adot_measure_pipe(int(kind), int(device), ctypes.byref(r), ctypes.byref(sec)),
           "adot_measure_pipe")
    return r.value, sec.value


def adot_conserved_sums(ctx: int) -> np.ndarray:
    out = (ctypes.c_double * 3)()
    _check(lib().adot_conserved_sums(ctx, out), "adot_conserved_sums")
    return np.array(out[:])


class Solver:
    """Owning wrapper around one context."""

    def __init__(self, cfg: Config, stream=None):
        self.cfg = cfg
        self.n = cfg.n_cells
        self.ctx = adot_create(cfg, stream)

    def set_state(self, h, q, z, t0=0.0):
        adot_set_state(self.ctx, h, q, z, t0, self.n)

    def get_state(self):
        h, q, z = np.empty(self.n), np.empty(self.n), np.empty(self.n)
        adot_get_state(self.ctx, h, q, z)
        return h, q, z

    def checkpoint(self, buf=None):
        return adot_checkpoint_save(self.ctx, buf)

    def restore(self, buf):
        adot_checkpoint_load(self.ctx, buf)

    def step(self, n):
        return adot_step(self.ctx, n)

    def run_to(self, t_end):
        return adot_run_to(self.ctx, t_end)

    def query(self):
        return adot_query(self.ctx)

    def fluctuations(self, WL, WR):
        return adot_fluctuations(self.ctx, WL, WR)

    def conserved_sums(self):
        return adot_conserved_sums(self.ctx)

    def close(self):
        if self.ctx:
            adot_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
