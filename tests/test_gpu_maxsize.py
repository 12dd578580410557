"""The largest state: N = 2^31 + 4097 cells of the smooth periodic workload,
past every 32-bit cell index, generated on the GPU in float64 (about 205 GB of
device memory with the float32 path's buffers). 50 steps of the FP32 path and
one of the FP64 path, checked on sampled cells against the oracle: both ends
of the periodic domain, the cells around index 2^31, random cells and the
cells around the largest spectral radius. Each sampled cell is recomputed by
the oracle's update (Eq. scheme, its fluctuations, the GPU's dt of each step)
on the window of cells it depends on; the GPU's CFL maximum is checked against the oracle's spectral
radius, not below it at any sampled cell and not above the supremum of the
continuous profile. Tolerances as elsewhere: FP64 1e-12 of each variable's
scale per cell; FP32 the sampled increments within 1e-5 in L1 relative (and
1e-4 of the largest per cell) plus the float-float state's resolution,
(K + 1) 2^-48 |W| per cell, which at this N is the larger term for the bed:
its increments per step are ~8e-14 on z ~ 0.1."""
import numpy as np
import pytest

import oracle as O
from paper_1912_04791_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = (1 << 31) + 4097
AG, CFL = 0.005, 0.8


def _profile(x):
    h = 1.0 + 0.1 * np.sin(2 * np.pi * x)
    u = 0.3 + 0.05 * np.cos(2 * np.pi * x)
    return h, h * u


def _device_state(torch, n):
    """h, q, z of the smooth periodic workload (as workloads.smooth_periodic)
    filled in chunks on the device."""
    h, q, z = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    chunk = 1 << 27
    dx = 1.0 / n
    for a in range(0, n, chunk):
        b = min(a + chunk, n)
        x = (torch.arange(a, b, dtype=torch.float64, device="cuda") + 0.5) * dx
        s, c = torch.sin(2 * np.pi * x), torch.cos(2 * np.pi * x)
        hh = 1.0 + 0.1 * s
        h[a:b] = hh
        q[a:b] = hh * (0.3 + 0.05 * c)
        z[a:b] = 0.1 * s
        del x, s, c, hh
    return h, q, z


def _samples(law, n, rng):
    # the largest spectral radius of the continuous profile, and the cells near it
    xs = np.linspace(0.0, 1.0, 20001)
    hs, qs = _profile(xs)
    rho = np.array([O.spectral_radius(law, a, b) for a, b in zip(hs, qs)])
    k = int(np.argmax(rho))
    lo, hi = xs[max(k - 1, 0)], xs[min(k + 1, len(xs) - 1)]
    fine = np.linspace(lo, hi, 2001)
    hf, qf = _profile(fine)
    rf = np.array([O.spectral_radius(law, a, b) for a, b in zip(hf, qf)])
    x_star = fine[int(np.argmax(rf))]
    sup = rf.max() * (1.0 + 1e-8)  # grid spacing 1e-7 around the maximum
    i_star = int(x_star * n)
    cells = np.concatenate([
        np.arange(0, 4), np.arange(n - 4, n), np.arange((1 << 31) - 4, (1 << 31) + 4),
        np.arange(i_star - 8, i_star + 9), rng.integers(0, n, 400)])
    return np.unique(cells % n), sup


def _local_reference(law, win, dts, n):
    """The oracle's update (Eq. scheme with its fluctuations, the given dt of
    each step) on windows of 2K + 1 cells around the sampled cells, [3, m, 2K+1]:
    after K steps the centre cell is exact (its domain of dependence)."""
    w = win.copy()
    for dt in dts:
        m, L = w.shape[1], w.shape[2]
        wl = np.ascontiguousarray(w[:, :, :-1].reshape(3, -1))
        wr = np.ascontiguousarray(w[:, :, 1:].reshape(3, -1))
        dm, dp = O.fluct(law, wl, wr)
        dm, dp = dm.reshape(3, m, L - 1), dp.reshape(3, m, L - 1)
        w[:, :, 1:-1] -= (dt * n) * (dp[:, :, :-1] + dm[:, :, 1:])  # dx = 1 / n
    return w[:, :, w.shape[2] // 2]


@pytest.mark.parametrize("prec,K", [("FP32", 50), ("FP64", 1)])
def test_max_size_steps_match_oracle_on_samples(gpu, prec, K):
    """K steps (float32: 50, so that the sampled increments, ~2e-11 per step at
    this N, stand well above the 2e-16 resolution of the float64 values the
    test compares; float64: 1)."""
    torch = pytest.importorskip("torch")
    free, _ = torch.cuda.mem_get_info()
    if free < 230e9:
        pytest.skip(f"needs ~210 GB of free device memory, {free / 1e9:.0f} GB free")
    law = O.grass(AG, xi=W.XI_P04)
    cells, sup = _samples(law, N, np.random.default_rng(2311))
    offs = np.arange(-K, K + 1)
    wcells = (cells[:, None] + offs[None, :]) % N  # [m, 2K+1]
    nb = np.unique(wcells)
    h, q, z = _device_state(torch, N)
    idx = torch.from_numpy(nb).cuda()
    w0 = np.stack([v.index_select(0, idx).cpu().numpy() for v in (h, q, z)])  # [3, len(nb)]
    # the benchmark's kernel shape, pinned (no trial launches at this size)
    cfg = gpu.make_config(N, 0.0, 1.0, CFL, AG, W.XI_P04, precision=getattr(gpu, prec),
                          bc_left=gpu.BC_PERIODIC, bc_right=gpu.BC_PERIODIC, block_threads=256,
                          reg_cap=80, step_kernel=2)
    dts = []
    with gpu.Solver(cfg, stream=torch.cuda.current_stream()) as s:
        s.set_state(h, q, z)
        for _ in range(K):
            s.step(1)
            dts.append(s.query()[2])
        t, steps, _ = s.query()
        gpu.adot_get_state(s.ctx, h, q, z)
        torch.cuda.synchronize()
    cidx = torch.from_numpy(cells).cuda()
    got = np.stack([v.index_select(0, cidx).cpu().numpy() for v in (h, q, z)])  # [3, m]
    del h, q, z, idx, cidx
    torch.cuda.empty_cache()
    assert steps == K and t == pytest.approx(sum(dts), rel=1e-14)

    pos = np.searchsorted(nb, wcells)
    win = w0[:, pos]  # [3, m, 2K+1]
    ref = _local_reference(law, win, dts, N)
    base = win[:, :, K]

    # the first step's CFL maximum: dt = cfl dx / rho
    rho_gpu = CFL / (N * dts[0])
    rho_s = max(O.spectral_radius(law, a, b) for a, b in zip(base[0], base[1]))
    if prec == "FP64":
        assert rho_gpu >= rho_s * (1 - 1e-13) and rho_gpu <= sup * (1 + 1e-12), (rho_gpu, rho_s, sup)
        for r in range(3):
            sc = np.abs(w0[r]).max()
            assert np.abs(got[r] - ref[r]).max() <= 1e-12 * sc, (r, np.abs(got[r] - ref[r]).max() / sc)
    else:
        assert rho_gpu >= rho_s * (1 - 1e-6) and rho_gpu <= sup * (1 + 1e-6), (rho_gpu, rho_s, sup)
        for r in range(3):
            inc, rinc = got[r] - base[r], ref[r] - base[r]
            err = np.abs(inc - rinc)
            # the float-float state holds a value to 2^-48 of itself: the input's
            # rounding and each step's add leave up to (K + 1) 2^-48 |W| per cell,
            # which for the bed (a step moves z ~ 0.1 by ~8e-14 at this N) is
            # ~5e-3 of a step's increment
            floor = (K + 1) * 2.0 ** -48 * np.abs(base[r])
            assert err.sum() <= 1e-5 * np.abs(rinc).sum() + floor.sum(), \
                (r, err.sum() / np.abs(rinc).sum(), floor.sum() / np.abs(rinc).sum())
            assert (err <= 1e-4 * np.abs(rinc).max() + floor).all(), (r, err.max() / np.abs(rinc).max())
