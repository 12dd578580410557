"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/adot.h declares, the ctypes structures
match the C layout, and argument validation rejects bad configurations before
any CUDA call."""
import ctypes
import os
import subprocess

import pytest

from paper_1912_04791_gb300 import adot, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return adot.lib()


def test_exports_every_declared_function(L):
    names = adot.header_functions()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "adot.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(adot_config), sizeof(adot_law),
         offsetof(adot_config, law), offsetof(adot_config, precision),
         offsetof(adot_config, bc_left_value), offsetof(adot_config, bc_right_value),
         offsetof(adot_config, block_threads), offsetof(adot_config, device),
         offsetof(adot_config, step_kernel), offsetof(adot_law, manning_n));
  printf("%zu %zu %zu %zu %zu %zu\n", offsetof(adot_config, ks), offsetof(adot_law, u_cr),
         offsetof(adot_law, beta), offsetof(adot_config, order), offsetof(adot_config, scheme),
         offsetof(adot_config, price_eps));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(adot_ensemble_config), offsetof(adot_ensemble_config, g),
         offsetof(adot_ensemble_config, precision), offsetof(adot_ensemble_config, block_threads),
         offsetof(adot_ensemble_config, device), offsetof(adot_ensemble_config, step_kernel));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    C, W, E = adot.Config, adot.Law, adot.EnsembleConfig
    want = [ctypes.sizeof(C), ctypes.sizeof(W), C.law.offset, C.precision.offset,
            C.bc_left_value.offset, C.bc_right_value.offset, C.block_threads.offset,
            C.device.offset, C.step_kernel.offset, W.manning_n.offset,
            C.ks.offset, W.u_cr.offset, W.beta.offset, C.order.offset, C.scheme.offset,
            C.price_eps.offset,
            ctypes.sizeof(E), E.g.offset, E.precision.offset, E.block_threads.offset, E.device.offset,
            E.step_kernel.offset]
    assert got == want


def test_status_strings_and_version(L):
    assert adot.status_string(adot.OK) == "ok"
    assert "depth" in adot.status_string(adot.E_NONPOSITIVE_DEPTH)
    assert adot.status_string(99) == "unknown status"
    assert "sm_103a" in adot.version()


@pytest.mark.parametrize("field,value", [
    ("n_cells", 0), ("cfl", 0.0), ("cfl", 1.5), ("x_max", -1.0), ("precision", 7),
    ("bc_left", 9), ("block_threads", 100), ("steps_per_graph", -6), ("device", -3),
    ("reg_cap", 48), ("step_kernel", 3), ("scheme", 2), ("scheme", -1), ("bc_left", 7), ("bc_right", -1), ("ks", -1.0),
    ("ks", float("nan")), ("ks", float("inf")), ("order", 3), ("order", -1)])
def test_invalid_config_rejected_without_cuda(L, field, value):
    cfg = adot.make_config(64, 0.0, 1.0, 0.8, 0.005, 5 / 3)
    setattr(cfg, field, value)
    out = ctypes.c_void_p()
    st = L.adot_create(ctypes.byref(cfg), None, ctypes.byref(out))
    assert st == adot.E_INVALID_ARG and not out.value


@pytest.mark.parametrize("beta,ucr", [(0.5, 0.0), (float("nan"), 0.0), (3.0, -0.1), (float("inf"), 0.0)])
def test_invalid_power_law_rejected(L, beta, ucr):
    cfg = adot.make_config(64, 0.0, 1.0, 0.8, 0.005, 5 / 3, law=adot.LAW_POWER, beta=beta, u_cr=ucr)
    out = ctypes.c_void_p()
    assert L.adot_create(ctypes.byref(cfg), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    assert not out.value


@pytest.mark.parametrize("kw", [{"step_kernel": 1}, {"reg_cap": -1}, {"ks": 30.0},
                                {"bc_left": adot.BC_INFLOW_QS, "bcl": (0.2, 1e-4, 0.0)}])
def test_second_order_combinations_unsupported(L, kw):
    """Order 2 runs the warp-tile kernel only, without friction or a feed."""
    cfg = adot.make_config(64, 0.0, 1.0, 0.8, 0.005, 5 / 3, order=2, **kw)
    out = ctypes.c_void_p()
    assert L.adot_create(ctypes.byref(cfg), None, ctypes.byref(out)) == adot.E_UNSUPPORTED
    assert not out.value


@pytest.mark.parametrize("kw,status", [
    ({"price_eps": -1e-4}, adot.E_INVALID_ARG), ({"price_eps": float("nan")}, adot.E_INVALID_ARG),
    ({"order": 2}, adot.E_UNSUPPORTED), ({"step_kernel": 1}, adot.E_UNSUPPORTED),
    ({"block_threads": 128}, adot.E_UNSUPPORTED), ({"reg_cap": 80}, adot.E_UNSUPPORTED),
    ({"reg_cap": -1}, adot.E_UNSUPPORTED)])
def test_price_c_combinations_rejected(L, kw, status):
    """PRICE-C runs the first-order warp-tile kernel of 256 threads (caps 64, 40, 32)."""
    cfg = adot.make_config(64, 0.0, 1.0, 0.8, 0.005, 5 / 3, scheme=adot.SCHEME_PRICE_C, **kw)
    out = ctypes.c_void_p()
    assert L.adot_create(ctypes.byref(cfg), None, ctypes.byref(out)) == status
    assert not out.value


@pytest.mark.parametrize("cap", [32, 40])
def test_price_c_caps_unsupported_for_dot(L, cap):
    cfg = adot.make_config(64, 0.0, 1.0, 0.8, 0.005, 5 / 3, reg_cap=cap)
    out = ctypes.c_void_p()
    assert L.adot_create(ctypes.byref(cfg), None, ctypes.byref(out)) == adot.E_UNSUPPORTED


def test_periodic_must_be_on_both_ends(L):
    cfg = adot.make_config(64, 0.0, 1.0, 0.8, 0.005, 5 / 3, bc_left=adot.BC_PERIODIC)
    out = ctypes.c_void_p()
    assert L.adot_create(ctypes.byref(cfg), None, ctypes.byref(out)) == adot.E_INVALID_ARG


def test_null_arguments_rejected(L):
    out = ctypes.c_void_p()
    assert L.adot_create(None, None, ctypes.byref(out)) == adot.E_INVALID_ARG
    assert L.adot_step(None, 1, None, None) == adot.E_INVALID_ARG
    assert L.adot_query(None, None, None, None) == adot.E_INVALID_ARG
    assert L.adot_fluctuations(None, None, None, 0, None, None, None, 0) == adot.E_INVALID_ARG
    assert L.adot_price_fluctuations(None, None, None, 0, 0.5, None, None, 0) == adot.E_INVALID_ARG
    assert L.adot_precision_stats(None, None, None) == adot.E_INVALID_ARG
    assert L.adot_mlp_apply_gradient(None, None, 1e-3, 0) == adot.E_INVALID_ARG
    assert L.adot_autotune(None, 8, None, None, None) == adot.E_INVALID_ARG
    assert L.adot_ensemble_plan(None, 0, None, None, None, None, None, None) == adot.E_INVALID_ARG
    assert L.adot_ensemble_inject_fault(None, 1) == adot.E_INVALID_ARG
    assert L.adot_checkpoint_size(None, None) == adot.E_INVALID_ARG
    assert L.adot_checkpoint_save(None, None, 0, 0) == adot.E_INVALID_ARG
    assert L.adot_checkpoint_load(None, None, 0, 0) == adot.E_INVALID_ARG
    assert L.adot_mlp_set_engine(None, 0) == adot.E_INVALID_ARG
    assert L.adot_mlp_set_train_engine(None, 0) == adot.E_INVALID_ARG
    assert L.adot_mlp_inject_fault(None, 1) == adot.E_INVALID_ARG
    assert L.adot_surrogate_eval(None, None, 0, None) == adot.E_INVALID_ARG
    L.adot_destroy(None)


def test_math_probe_rejects_bad_arguments(L):
    assert L.adot_math_probe(2, None, None, 0, None) == adot.E_INVALID_ARG
    assert L.adot_math_probe(0, None, None, 5, None) == adot.E_INVALID_ARG
    assert L.adot_math_probe(0, None, None, -1, None) == adot.E_INVALID_ARG
    assert L.adot_math_probe(0, None, None, 0, None) == adot.OK


def test_measure_pipe_rejects_bad_kind(L):
    r = ctypes.c_double()
    assert L.adot_measure_pipe(7, -1, ctypes.byref(r), None) == adot.E_INVALID_ARG
    assert L.adot_measure_pipe(-1, -1, ctypes.byref(r), None) == adot.E_INVALID_ARG
    assert L.adot_measure_pipe(0, -1, None, None) == adot.E_INVALID_ARG


def test_invalid_ensemble_config_rejected(L):
    import numpy as np
    n = np.array([10, 0], dtype=np.int64)
    ln = np.array([1.0, 1.0])
    ag = np.array([0.01, 0.01])
    c = adot.EnsembleConfig()
    c.n_channels = 2
    c.n_cells = n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    c.length = ln.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c.Ag = ag.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c.g, c.xi, c.cfl, c.precision, c.block_threads, c.device = 9.81, 1.0, 0.9, 1, 0, -1
    out = ctypes.c_void_p()
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    n[1] = 5
    c.cfl = 2.0
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    c.cfl = 0.9
    c.block_threads = 100
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    c.block_threads = 0
    c.step_kernel = 6
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    c.step_kernel, c.block_threads = 5, 384  # cluster teams run 768-thread CTAs only
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    c.block_threads = 0
    c.step_kernel, c.block_threads = 4, 384  # 384-thread blocks: persistent channel loops only
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    c.step_kernel, c.block_threads = 3, 128
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
    c.step_kernel, c.block_threads = 2, 128  # warp tiles run 256-thread blocks only
    assert L.adot_ensemble_create(ctypes.byref(c), None, ctypes.byref(out)) == adot.E_INVALID_ARG
